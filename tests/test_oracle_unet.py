"""Pins for oracle/unet.py: the 3x3 convolution against scipy's 2-D cross-correlation,
pooling / upsampling as adjoint pairs, the grid stencil against the assembled P1
stiffness matrix (oracle/fem.py), the residual loss against its closed forms (zero at
the exact solve), the whole network (forward and gradients) against the same
architecture assembled from torch.nn.functional in FP64 with autograd and a dense
stencil matrix, and the backward pass against central finite differences."""
import numpy as np
import scipy.sparse.linalg as spla
from scipy import signal

from oracle import unet
from oracle.fem import Mesh


def _real_stencil(N, H, W, seed):
    """Grid channels of K(m) for a random m on an N x N mesh, and the free-node mask."""
    mesh = Mesh(2, N)
    m = np.random.default_rng(seed).standard_normal(mesh.n) * 0.5
    K = mesh.stiffness(mesh.elem_mean(np.exp(m)))
    free = np.zeros((H, W))
    free[:N + 1, :N + 1] = (~mesh.dirichlet_mask).reshape(N + 1, N + 1)
    return mesh, m, K, unet.stencil_channels(K, N + 1, H, W), free


def _random_aux(rng, N, H, W):
    aux = rng.standard_normal((N, 4, H, W))
    aux[:, 1] = 4.0 + rng.uniform(size=(N, H, W))          # a diagonally dominant stencil
    return aux


def test_conv_equals_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 9, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def test_pool_up_are_adjoint_to_their_backward():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 8, 6))
    d = rng.standard_normal((1, 2, 4, 3))
    assert np.isclose((unet.pool(x) * d).sum(), (x * unet.pool_backward(d)).sum())
    u = rng.standard_normal((1, 2, 8, 6))
    assert np.isclose((unet.up(d) * u).sum(), (d * unet.up_backward(u)).sum())


def test_stencil_is_the_assembled_stiffness_on_free_nodes():
    N, H, W = 6, 8, 8
    mesh, m, K, ch, free = _real_stencil(N, H, W, 0)
    # K is exactly 5-point: rebuilding it from the channels loses nothing
    nper = N + 1
    Kd = K.toarray()
    rows, cols = np.nonzero(np.abs(Kd) > 1e-13 * np.abs(Kd).max())
    d = np.abs(rows - cols)
    assert set(d.tolist()) <= {0, 1, nper}        # the diagonal-edge couplings cancel to rounding
    v = np.random.default_rng(1).standard_normal((1, 1, H, W))
    aux = np.concatenate([np.zeros((1, 1, H, W)), ch[None]], axis=1)
    Sv = unet.stencil_apply(v, aux, free[None, None])
    fv = free[:nper, :nper].ravel()
    ref = fv * (K @ (fv * v[0, 0, :nper, :nper].ravel()))
    assert np.allclose(Sv[0, 0, :nper, :nper].ravel(), ref, atol=1e-12)
    assert not Sv[0, 0, nper:, :].any() and not Sv[0, 0, :, nper:].any()


def test_residual_loss_closed_forms():
    N, H, W = 6, 8, 8
    mesh, m, K, ch, free = _real_stencil(N, H, W, 2)
    rng = np.random.default_rng(3)
    nper = N + 1
    x = np.zeros((3, 3, H, W))
    x[:, 2] = free
    aux = np.zeros((3, 4, H, W))
    aux[:, 1:] = ch
    aux[:, 0] = rng.standard_normal((3, H, W))
    aux[2, 0] = 0.0                                        # a zero right-hand side counts 0
    # y = 0: each nonzero sample contributes 1/(2N)
    assert np.isclose(unet.residual_loss(np.zeros((3, 1, H, W)), x, aux)[0], 0.5 * 2 / 3)
    # y = the exact solve of K_ff y = b_f: zero loss
    f = ~mesh.dirichlet_mask
    y = np.zeros((3, 1, H, W))
    Kff = K[f][:, f].tocsc()
    for j in range(2):
        yy = np.zeros(mesh.n)
        yy[f] = spla.spsolve(Kff, aux[j, 0, :nper, :nper].ravel()[f])
        y[j, 0, :nper, :nper] = yy.reshape(nper, nper)
    assert unet.residual_loss(y, x, aux)[0] < 1e-24
    # invariant under a common scale of y and b
    y2 = rng.standard_normal((3, 1, H, W))
    a2 = aux.copy()
    a2[:, 0] *= 5.0
    assert np.isclose(unet.residual_loss(5.0 * y2, x, a2)[0], unet.residual_loss(y2, x, aux)[0])


def test_network_matches_torch_functional():
    torch = __import__("pytest").importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(5)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in unet.init_params(6)]
    x = rng.standard_normal((2, 3, 16, 24))
    x[:, 2] = (rng.uniform(size=(2, 16, 24)) > 0.25)
    aux = _random_aux(rng, 2, 16, 24)
    y, cache = unet.forward(params, x)
    L, dy = unet.residual_loss(y, x, aux)
    grads = unet.backward(params, cache, dy)

    tp = [(torch.tensor(w, requires_grad=True), torch.tensor(b, requires_grad=True)) for w, b in params]
    P = {name: wb for (name, *_), wb in zip(unet.LAYERS, tp)}

    def block(h, a, b):
        h = F.relu(F.conv2d(h, *P[a], padding=1))
        return F.relu(F.conv2d(h, *P[b], padding=1))

    def dec(coarse, skip, a, b):
        return block(torch.cat([F.interpolate(coarse, scale_factor=2, mode="nearest"), skip], 1), a, b)

    xt = torch.tensor(x)
    s1 = block(xt, "enc1a", "enc1b")
    s2 = block(F.avg_pool2d(s1, 2), "enc2a", "enc2b")
    s3 = block(F.avg_pool2d(s2, 2), "enc3a", "enc3b")
    bt = block(F.avg_pool2d(s3, 2), "bota", "botb")
    d1 = dec(dec(dec(bt, s3, "dec3a", "dec3b"), s2, "dec2a", "dec2b"), s1, "dec1a", "dec1b")
    yt = F.conv2d(d1, *P["out"])
    H, W = 16, 24

    def dense_S(n):                      # mask K mask as a dense (HW x HW) matrix, built entry by entry
        S = np.zeros((H * W, H * W))
        for r in range(H):
            for c in range(W):
                i = r * W + c
                S[i, i] = aux[n, 1, r, c]
                if c + 1 < W:
                    S[i, i + 1] = S[i + 1, i] = aux[n, 2, r, c]
                if r + 1 < H:
                    S[i, i + W] = S[i + W, i] = aux[n, 3, r, c]
        mk = x[n, 2].ravel()
        return torch.tensor(mk[:, None] * S * mk[None, :])

    Lt = 0.0
    for n in range(2):
        b = torch.tensor(aux[n, 0].ravel() * x[n, 2].ravel())
        r = b - dense_S(n) @ yt[n, 0].reshape(-1)
        Lt = Lt + 0.5 * (r @ r) / (b @ b) / 2
    Lt.backward()
    assert np.allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert np.isclose(L, Lt.item(), rtol=1e-12)
    for (gw, gb), (w, b) in zip(grads, tp):
        assert np.allclose(gw, w.grad.numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = unet.init_params(3)
    x = rng.standard_normal((2, 3, 16, 16))
    x[:, 2] = (rng.uniform(size=(2, 16, 16)) > 0.2)
    aux = _random_aux(rng, 2, 16, 16)
    aux[1, 0] *= 3.0

    def L(ps):
        return unet.residual_loss(unet.forward(ps, x)[0], x, aux)[0]

    y, cache = unet.forward(params, x)
    _, dy = unet.residual_loss(y, x, aux)
    grads = unet.backward(params, cache, dy)
    eps = 1e-6
    for li in [0, 3, 7, 8, 12, 14]:
        w, b = params[li]
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(3)]:
            wp = [(pw.copy(), pb) for pw, pb in params]
            wm = [(pw.copy(), pb) for pw, pb in params]
            wp[li][0][idx] += eps
            wm[li][0][idx] -= eps
            fd = (L(wp) - L(wm)) / (2 * eps)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
        j = int(rng.integers(0, b.shape[0]))
        bp = [(pw, pb.copy()) for pw, pb in params]
        bm = [(pw, pb.copy()) for pw, pb in params]
        bp[li][1][j] += eps
        bm[li][1][j] -= eps
        fd = (L(bp) - L(bm)) / (2 * eps)
        assert abs(fd - grads[li][1][j]) <= 1e-6 * max(1.0, abs(fd))
