"""U-Net warm start: FP64 reference forward and backward (oracle; test infrastructure).

The network (not part of the paper; the build's learned initial guess for the PCG
solves) maps 3 input channels on a padded nodal grid -- the log-coefficient m, the
right-hand side scaled to unit norm, and a mask of the free nodes -- to one output
channel, the initial guess (scaled back by the right-hand side's norm).  Four levels
with 16, 32, 64 and 128 channels:

    enc1: conv3x3(3->16)  relu conv3x3(16->16)  relu   -> s1          (H x W)
    enc2: avgpool2, conv(16->32) relu conv(32->32) relu -> s2         (H/2)
    enc3: avgpool2, conv(32->64) relu conv(64->64) relu -> s3         (H/4)
    bott: avgpool2, conv(64->128) relu conv(128->128) relu            (H/8)
    dec3: up2, concat[up, s3] (192), conv(192->64) relu conv(64->64) relu
    dec2: up2, concat[up, s2] (96),  conv(96->32) relu conv(32->32) relu
    dec1: up2, concat[up, s1] (48),  conv(48->16) relu conv(16->16) relu
    out : conv1x1(16->1)

3x3 convolutions are cross-correlations with zero padding and a bias; pooling is the
2x2 mean; upsampling repeats each value on a 2x2 block; concatenation puts the
upsampled channels first.

Training loss: the relative residual of the guess in the stiffness system.  Each
sample carries, on the grid (row iy, column ix), its right-hand side b and the
symmetric 5-point stencil of K (diag, cx = coupling to the right neighbour, cy =
coupling to the neighbour below) in aux = (b, diag, cx, cy); the free-node mask is
input channel 2.  With S = mask K mask,

    L = 1/(2N) sum_n |mask_n b_n - S_n y_n|^2 / |mask_n b_n|^2

(a sample with a zero right-hand side counts 0).  On the free nodes of a P1 Kuhn
triangulation K is exactly 5-point: the diagonal edge is opposite a right angle in
both of its triangles, so its coupling vanishes.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # (name, c_in, c_out, kernel)
    ("enc1a", 3, 16, 3), ("enc1b", 16, 16, 3),
    ("enc2a", 16, 32, 3), ("enc2b", 32, 32, 3),
    ("enc3a", 32, 64, 3), ("enc3b", 64, 64, 3),
    ("bota", 64, 128, 3), ("botb", 128, 128, 3),
    ("dec3a", 192, 64, 3), ("dec3b", 64, 64, 3),
    ("dec2a", 96, 32, 3), ("dec2b", 32, 32, 3),
    ("dec1a", 48, 16, 3), ("dec1b", 16, 16, 3),
    ("out", 16, 1, 1),
]


def init_params(seed: int = 0):
    """He-normal weights, zero biases: [(w (co, ci, k, k), b (co,)), ...] in LAYERS order."""
    rng = np.random.default_rng(seed)
    out = []
    for _, ci, co, k in LAYERS:
        w = rng.standard_normal((co, ci, k, k)) * np.sqrt(2.0 / (ci * k * k))
        out.append((w, np.zeros(co)))
    return out


def conv(x, w, b):
    """x (N, ci, H, W), w (co, ci, k, k) with k in {1, 3}: zero-padded cross-correlation + bias."""
    k = w.shape[2]
    if k == 1:
        return np.einsum("nchw,oc->nohw", x, w[:, :, 0, 0]) + b[None, :, None, None]
    N, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.broadcast_to(b[None, :, None, None], (N, w.shape[0], H, W)).copy()
    for dh in range(3):
        for dw in range(3):
            out += np.einsum("nchw,oc->nohw", xp[:, :, dh:dh + H, dw:dw + W], w[:, :, dh, dw])
    return out


def conv_backward(x, w, dout):
    """Gradients of conv(x, w, b) -> (dx, dw, db)."""
    k = w.shape[2]
    db = dout.sum(axis=(0, 2, 3))
    if k == 1:
        dw = np.einsum("nohw,nchw->oc", dout, x)[:, :, None, None]
        dx = np.einsum("nohw,oc->nchw", dout, w[:, :, 0, 0])
        return dx, dw, db
    N, C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for dh in range(3):
        for dwi in range(3):
            dw[:, :, dh, dwi] = np.einsum("nohw,nchw->oc", dout, xp[:, :, dh:dh + H, dwi:dwi + W])
            dxp[:, :, dh:dh + H, dwi:dwi + W] += np.einsum("nohw,oc->nchw", dout, w[:, :, dh, dwi])
    return dxp[:, :, 1:-1, 1:-1], dw, db


def pool(x):
    N, C, H, W = x.shape
    return x.reshape(N, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool_backward(d):
    return np.repeat(np.repeat(d, 2, axis=2), 2, axis=3) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up_backward(d):
    N, C, H, W = d.shape
    return d.reshape(N, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(params, x):
    """Returns (y, cache)."""
    p = dict(zip([n for n, *_ in LAYERS], params))
    cache = {}

    def cr(name, h):
        z = conv(h, *p[name])
        cache[name] = (h, z)
        return np.maximum(z, 0.0)

    s1 = cr("enc1b", cr("enc1a", x))
    s2 = cr("enc2b", cr("enc2a", pool(s1)))
    s3 = cr("enc3b", cr("enc3a", pool(s2)))
    bt = cr("botb", cr("bota", pool(s3)))
    d3 = cr("dec3b", cr("dec3a", np.concatenate([up(bt), s3], axis=1)))
    d2 = cr("dec2b", cr("dec2a", np.concatenate([up(d3), s2], axis=1)))
    d1 = cr("dec1b", cr("dec1a", np.concatenate([up(d2), s1], axis=1)))
    y = conv(d1, *p["out"])
    cache["out"] = (d1, y)
    cache["shapes"] = (bt.shape[1], d3.shape[1], d2.shape[1])
    return y, cache


def stencil_apply(v, aux, mask):
    """mask * K (mask * v) for the grid stencil aux[:, 1:4] = (diag, cx, cy)."""
    v = v * mask
    d, cx, cy = aux[:, 1:2], aux[:, 2:3], aux[:, 3:4]
    out = d * v
    out[:, :, :, :-1] += cx[:, :, :, :-1] * v[:, :, :, 1:]
    out[:, :, :, 1:] += cx[:, :, :, :-1] * v[:, :, :, :-1]
    out[:, :, :-1, :] += cy[:, :, :-1, :] * v[:, :, 1:, :]
    out[:, :, 1:, :] += cy[:, :, :-1, :] * v[:, :, :-1, :]
    return out * mask


def residual_loss(y, x, aux):
    """Returns (L, dL/dy) for network output y, input x (mask = channel 2) and aux."""
    N = y.shape[0]
    mask = x[:, 2:3]
    b = aux[:, 0:1] * mask
    r = b - stencil_apply(y, aux, mask)
    bn = (b * b).sum(axis=(1, 2, 3))
    w = np.where(bn > 0, 1.0 / (N * np.where(bn > 0, bn, 1.0)), 0.0)[:, None, None, None]
    # S is symmetric, so d/dy (1/2) w |b - S y|^2 = -S (w r)
    return float(0.5 * (w * r * r).sum()), -stencil_apply(w * r, aux, mask)


def stencil_channels(K, nper, H, W):
    """(3, H, W) grid channels (diag, cx, cy) of a 2D nodal matrix K (node ix + nper iy at
    row iy, column ix); couplings leave the grid as zero."""
    K = K.tocsr()
    out = np.zeros((3, H, W))
    for iy in range(nper):
        for ix in range(nper):
            i = ix + nper * iy
            out[0, iy, ix] = K[i, i]
            if ix + 1 < nper:
                out[1, iy, ix] = K[i, i + 1]
            if iy + 1 < nper:
                out[2, iy, ix] = K[i, i + nper]
    return out


def backward(params, cache, dy):
    """Gradients [(dw, db), ...] in LAYERS order for dL/dy = dy."""
    names = [n for n, *_ in LAYERS]
    p = dict(zip(names, params))
    g = {}

    def back(name, dh_out, relu=True):
        h, z = cache[name]
        dz = dh_out * (z > 0) if relu else dh_out
        dx, dw, db = conv_backward(h, p[name][0], dz)
        g[name] = (dw, db)
        return dx

    c_bt, c_d3, c_d2 = cache["shapes"]
    d = back("out", dy, relu=False)
    d = back("dec1a", back("dec1b", d))
    d_up2, d_s1 = d[:, :c_d2], d[:, c_d2:]
    d = back("dec2a", back("dec2b", up_backward(d_up2)))
    d_up3, d_s2 = d[:, :c_d3], d[:, c_d3:]
    d = back("dec3a", back("dec3b", up_backward(d_up3)))
    d_upb, d_s3 = d[:, :c_bt], d[:, c_bt:]
    d = back("bota", back("botb", up_backward(d_upb)))
    d = back("enc3a", back("enc3b", pool_backward(d) + d_s3))
    d = back("enc2a", back("enc2b", pool_backward(d) + d_s2))
    back("enc1a", back("enc1b", pool_backward(d) + d_s1))
    return [g[n] for n in names]
