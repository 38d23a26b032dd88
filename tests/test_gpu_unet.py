"""GPU parity of the warm-start network's kernels against the FP64 oracle
(oracle/unet.py), with the weights rounded to BF16 on both sides (the kernels keep
BF16 weights and accumulate in FP32):

  forward output                  max |y_gpu - y_oracle| <= 1e-4 max |y_oracle|
  relative-residual loss          relative 1e-5
  gradients, per layer            |g_gpu - g_oracle| <= 10 |g_oracle32 - g_oracle| + 1e-4 |g_oracle|
                                  (weights and biases), g_oracle32 = the oracle evaluated in FP32:
                                  the residual loss's dL/dy = -S(w r) is a rough field, so the
                                  weight gradients are sums of many terms of both signs and their
                                  FP32 rounding error is far above FP32 epsilon; the bound is set
                                  at ten times the error FP32 arithmetic itself makes
  one Adam step                   p1 = p0 - lr g / (|g| + eps) (first step, bias-corrected moments)

Grids 16 x 40 (a ragged last 16-wide tile), 24 x 24 and 72 x 24, batches of 2 and 3, with the 3x3
convolutions on the FP32 pipes and on the tensor cores (the default).  The tensor-core
kernels take each FP32 activation as three BF16 terms (its full significand), and the tensor
core's FP32 accumulation is not IEEE round-to-nearest: each MMA aligns its 16 products
and the accumulator and truncates the sum (Fasi, Higham, Mikaitis and Pranesh, "Numerical
behavior of NVIDIA tensor cores", PeerJ Comput. Sci. 2021), an error of up to ~2^-23 of
the accumulator per MMA, of one sign, over 27 MMAs per 16-channel slab.  That is a
relative bias of order 1e-5 per layer where FP32 FMAs make ~1e-7, so with the tensor
cores the loss bound is 1e-4 relative and the gradient bound's relative term 1e-3.
Between the two kernel families, on grids whose tiles are ragged in both directions:
forward outputs within 1e-4 of the largest output and loss within 1e-4 relative (their
gradients are compared with the oracle above: where the residual loss's gradient sums
cancel, both families are as far from the oracle as FP32 arithmetic itself, 1e-3 and more).
"""
import numpy as np
import pytest

from oracle import unet as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (b.astype(np.uint32)).view(np.float32).astype(np.float64)


def make_params(seed):
    rng = np.random.default_rng(seed)
    ps = [(w.astype(np.float32), (0.1 * rng.standard_normal(b.shape)).astype(np.float32))
          for w, b in O.init_params(seed)]
    packed = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in ps]).astype(np.float32)
    oracle_ps = [(bf16_round(w), b.astype(np.float64)) for w, b in ps]
    return packed, oracle_ps


def unpack(g):
    out, off = [], 0
    for _, ci, co, k in O.LAYERS:
        nw = co * ci * k * k
        out.append((g[off:off + nw].reshape(co, ci, k, k), g[off + nw:off + nw + co]))
        off += nw + co
    assert off == g.size
    return out


def batch(seed, N, H, W):
    """Inputs with a random free-node mask in channel 2 and loss data with a random
    diagonally dominant symmetric 5-point stencil."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, 3, H, W)).astype(np.float32)
    x[:, 2] = rng.uniform(size=(N, H, W)) > 0.2
    aux = rng.standard_normal((N, 4, H, W)).astype(np.float32)
    aux[:, 1] = 4.0 + rng.uniform(size=(N, H, W))
    return x, aux


def dev(a):
    return torch.tensor(a, device=DEV).contiguous()


@pytest.mark.parametrize("tensor_cores", [True, False], ids=["tcgen05", "fp32"])
@pytest.mark.parametrize("N,H,W", [(2, 16, 40), (3, 24, 24), (2, 72, 24)])
def test_forward_and_gradients_match_oracle(N, H, W, tensor_cores):
    from paper_1909_03948_gb300 import UNet
    packed, ops = make_params(7)
    net = UNet(H, W, batch_cap=4, tensor_cores=tensor_cores)
    assert net.tensor_cores == tensor_cores
    assert net.nparam == packed.size
    net.set_params(packed)
    assert np.array_equal(net.get_params(), packed)
    x, aux = batch(8, N, H, W)
    y = net.forward(dev(x)).cpu().numpy().astype(np.float64)
    yo, cache = O.forward(ops, x.astype(np.float64))
    print(f"forward: max error {np.abs(y - yo).max() / np.abs(yo).max():.2e} of max |y|")
    assert np.abs(y - yo).max() <= 1e-4 * np.abs(yo).max()
    L, g = net.loss_grad(dev(x), dev(aux))
    Lo, dyo = O.residual_loss(yo, x.astype(np.float64), aux.astype(np.float64))
    print(f"loss: relative error {abs(L - Lo) / abs(Lo):.2e}")
    assert abs(L - Lo) <= (1e-4 if tensor_cores else 1e-5) * abs(Lo)
    rel = 1e-3 if tensor_cores else 1e-4
    go = O.backward(ops, cache, dyo)
    # the same oracle evaluated in FP32: the scale of FP32 rounding in these gradients
    ops32 = [(w.astype(np.float32), b.astype(np.float32)) for w, b in ops]
    y32, cache32 = O.forward(ops32, x)
    _, dy32 = O.residual_loss(y32, x, aux)
    g32 = O.backward(ops32, cache32, dy32.astype(np.float32))
    nrm = np.linalg.norm
    for (gw, gb), (ow, ob), (w32, b32), (name, *_) in zip(unpack(g.astype(np.float64)), go, g32, O.LAYERS):
        ew, eb = nrm(gw - ow), nrm(gb - ob)
        bw = 10 * nrm(w32 - ow) + rel * nrm(ow)
        bb = 10 * nrm(b32 - ob) + rel * nrm(ob)
        print(f"{name}: weights {ew / nrm(ow):.2e} (fp32 oracle {nrm(w32 - ow) / nrm(ow):.2e}), "
              f"biases {eb / max(nrm(ob), 1e-30):.2e} (fp32 oracle {nrm(b32 - ob) / max(nrm(ob), 1e-30):.2e})")
        assert ew <= bw and eb <= bb, name
    net.close()


def test_one_adam_step_and_bf16_refresh():
    from paper_1909_03948_gb300 import UNet
    H = W = 16
    packed, _ = make_params(9)
    net = UNet(H, W, batch_cap=4)
    net.set_params(packed)
    x, aux = batch(10, 4, H, W)
    _, g = net.loss_grad(dev(x), dev(aux))
    lr = 1e-3
    losses = net.train(dev(x), dev(aux), epochs=1, batch=4, lr=lr, seed=0)
    assert losses.shape == (1,) and np.isfinite(losses[0])
    p1 = net.get_params().astype(np.float64)
    big = np.abs(g) > 1e-5
    expect = packed.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    assert np.abs(p1 - expect)[big].max() <= 2e-3 * lr + 1e-6
    # the kernels' BF16 weights follow the FP32 master copy
    fresh = UNet(H, W, batch_cap=4)
    fresh.set_params(net.get_params())
    assert torch.equal(net.forward(dev(x)), fresh.forward(dev(x)))
    net.close()
    fresh.close()


def test_training_reduces_the_loss():
    """Constant-coefficient 5-point Laplacian, random right-hand sides with smooth and
    rough parts: training must cut the relative residual of the guess well below the
    zero guess's (loss 1/2)."""
    from paper_1909_03948_gb300 import UNet
    from paper_1909_03948_gb300.warmstart import he_init
    H = W = 24
    rng = np.random.default_rng(11)
    N = 64
    x = np.zeros((N, 3, H, W), dtype=np.float32)
    x[:, 2, 1:-1, :] = 1.0
    aux = np.zeros((N, 4, H, W), dtype=np.float32)
    aux[:, 1], aux[:, 2], aux[:, 3] = 4.0, -1.0, -1.0
    b = rng.standard_normal((N, H, W)) * x[:, 2]
    aux[:, 0] = b
    x[:, 1] = b / 4.0 / np.sqrt((b / 4.0) ** 2).mean(axis=(1, 2), keepdims=True)
    aux[:, 0] /= np.sqrt((b / 4.0) ** 2).mean(axis=(1, 2), keepdims=True)
    net = UNet(H, W, batch_cap=8)
    net.set_params(he_init(0, out_scale=0.1))
    losses = net.train(dev(x), dev(aux), epochs=40, batch=8, lr=2e-3, seed=1)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0], losses
    net.close()


def test_invalid_network_arguments():
    from paper_1909_03948_gb300 import UNet, HPError
    with pytest.raises(HPError):
        UNet(20, 16)          # not a multiple of 8
    with pytest.raises(HPError):
        UNet(16, 16, batch_cap=0)
    net = UNet(16, 16, batch_cap=2)
    x = torch.zeros((3, 3, 16, 16), device=DEV)
    with pytest.raises(HPError):
        net.forward(x)        # more samples than batch_cap
    with pytest.raises(ValueError):
        net.set_params(np.zeros(3, dtype=np.float32))
    net.close()


@pytest.mark.parametrize("N,H,W", [(3, 40, 56), (2, 72, 24)])
def test_tensor_core_convolutions_match_the_fp32_kernels(N, H, W):
    """Both kernel families on the same network and batch: 40 x 56 and 72 x 24 leave
    partial tiles (16 rows x 16 columns, and 16 x 8 for the 192-channel input gradient)
    on every level."""
    from paper_1909_03948_gb300 import UNet
    packed, _ = make_params(21)
    x, aux = batch(22, N, H, W)
    out = {}
    for tc in (True, False):
        net = UNet(H, W, batch_cap=4, tensor_cores=tc)
        net.set_params(packed)
        y = net.forward(dev(x)).cpu().numpy().astype(np.float64)
        L, _ = net.loss_grad(dev(x), dev(aux))
        out[tc] = (y, L)
        net.close()
    (yt, Lt), (yf, Lf) = out[True], out[False]
    assert not np.array_equal(yt, yf)  # two different kernel paths ran
    print(f"forward {np.abs(yt - yf).max() / np.abs(yf).max():.2e} of max |y|, loss {abs(Lt - Lf) / abs(Lf):.2e}")
    assert np.abs(yt - yf).max() <= 1e-4 * np.abs(yf).max()
    assert abs(Lt - Lf) <= 1e-4 * abs(Lf)


def test_tensor_core_switch_arguments():
    from paper_1909_03948_gb300 import UNet, HPError, lib
    net = UNet(16, 16, batch_cap=1)
    assert net.tensor_cores
    net.tensor_cores = False
    assert not net.tensor_cores
    with pytest.raises(HPError):
        from paper_1909_03948_gb300.hp import _check
        _check(lib().hp_unet_set_tensor_cores(net._h, 2), "hp_unet_set_tensor_cores")
    net.close()
