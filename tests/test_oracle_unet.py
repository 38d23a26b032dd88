"""Pins for oracle/unet.py: the 3x3 convolution against scipy's 2-D cross-correlation,
pooling / upsampling as adjoint pairs, the loss against its closed forms, the whole
network (forward and gradients) against the same architecture assembled from
torch.nn.functional in FP64 with autograd, and the backward pass against central
finite differences of the loss."""
import numpy as np
from scipy import signal

from oracle import unet


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


def test_loss_closed_forms():
    rng = np.random.default_rng(4)
    t = rng.standard_normal((3, 1, 8, 8))
    t[2] = 0.0                                   # a zero target counts 0
    mask = (rng.uniform(size=(3, 1, 8, 8)) > 0.3).astype(float)
    # y = 0: every nonzero sample contributes exactly 1/(2N)
    assert np.isclose(unet.loss(np.zeros_like(t), t, mask)[0], 0.5 * 2 / 3)
    # y = 2t: the same (|y - t| = |t|); y = t: zero loss and gradient
    assert np.isclose(unet.loss(2 * t, t, mask)[0], 0.5 * 2 / 3)
    L0, d0 = unet.loss(t.copy(), t, mask)
    assert L0 == 0.0 and not d0.any()
    # invariant under a common scale of y and t, and blind to unmasked pixels
    y = rng.standard_normal(t.shape)
    assert np.isclose(unet.loss(7.0 * y, 7.0 * t, mask)[0], unet.loss(y, t, mask)[0])
    y2 = y + 5.0 * (1 - mask)
    assert np.isclose(unet.loss(y2, t, mask)[0], unet.loss(y, t, mask)[0])


def test_network_matches_torch_functional():
    torch = __import__("pytest").importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(5)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in unet.init_params(6)]
    x = rng.standard_normal((2, 3, 16, 24))
    t = rng.standard_normal((2, 1, 16, 24))
    mask = (rng.uniform(size=(2, 1, 16, 24)) > 0.25).astype(float)
    y, cache = unet.forward(params, x)
    L, dy = unet.loss(y, t, mask)
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
    mt, tt = torch.tensor(mask), torch.tensor(t)
    tn = ((tt * mt) ** 2).sum(dim=(1, 2, 3))
    Lt = 0.5 * ((((yt - tt) * mt) ** 2).sum(dim=(1, 2, 3)) / tn).mean()
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
    t = rng.standard_normal((2, 1, 16, 16))
    t[1] *= 3.0
    mask = (rng.uniform(size=(2, 1, 16, 16)) > 0.2).astype(float)

    def L(ps):
        return unet.loss(unet.forward(ps, x)[0], t, mask)[0]

    y, cache = unet.forward(params, x)
    _, dy = unet.loss(y, t, mask)
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
