"""FP64 numpy oracle of the learned depth prior's U-Net (test infrastructure only).

Same architecture and conventions as the CUDA path describes in
include/gevo_prior.h, written out plainly: a 3x3 zero-padded convolution is the
sum over its nine taps of a shifted input times that tap's weight matrix (numpy
matmul as the step), ReLU, 2x2 max pool (the first maximum in row-major order
receives the gradient), x2 nearest upsample, channel concatenation [upsampled,
skip], a 1x1 head to log-depth, and the masked L1 loss
L = (1/P) sum_p w_p |pred_p - target_p| (sign(0) = 0).  Backward is the exact
chain rule of each step.  Pinned by central finite differences
(tests/test_oracle_unet.py).

Weights: W[name] = (w [Cout, 9, Cin], b [Cout]), tap = 3 ky + kx; head = (w [C0], b [1]).
"""
from __future__ import annotations

import numpy as np


def bf16(x):
    """Round to bfloat16 (nearest even) through binary32, as values are stored
    between layers (activations after the ReLU, the masked gradient dZ)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32)
    b = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(x):
    return x


def _shift(x, ky, kx):
    """x[n, y + ky - 1, x + kx - 1, c] with zeros outside."""
    n, H, W, C = x.shape
    out = np.zeros_like(x)
    dy, dx = ky - 1, kx - 1
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    out[:, yd, xd, :] = x[:, ys, xs, :]
    return out


def _unshift(g, ky, kx):
    """Adjoint of _shift."""
    n, H, W, C = g.shape
    out = np.zeros_like(g)
    dy, dx = ky - 1, kx - 1
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    out[:, ys, xs, :] = g[:, yd, xd, :]
    return out


def conv3x3(x, w, b):
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for tap in range(9):
        y += _shift(x, tap // 3, tap % 3) @ w[:, tap, :].T
    return y + b


def conv3x3_bwd(x, w, dz):
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for tap in range(9):
        xs = _shift(x, tap // 3, tap % 3)
        dw[:, tap, :] = np.einsum("nhwo,nhwi->oi", dz, xs)
        dx += _unshift(dz @ w[:, tap, :], tap // 3, tap % 3)
    return dx, dw, dz.sum(axis=(0, 1, 2))


def maxpool2(x):
    n, H, W, C = x.shape
    v = np.stack([x[:, 0::2, 0::2], x[:, 0::2, 1::2], x[:, 1::2, 0::2], x[:, 1::2, 1::2]])
    arg = np.zeros(v.shape[1:], np.int64)
    best = v[0].copy()
    for k in range(1, 4):
        m = v[k] > best
        arg[m] = k
        best[m] = v[k][m]
    return best, arg


def maxpool2_bwd(arg, dy, shape):
    dx = np.zeros(shape)
    for k, (oy, ox) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        dx[:, oy::2, ox::2] += np.where(arg == k, dy, 0.0)
    return dx


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_bwd(dy):
    return dy[:, 0::2, 0::2] + dy[:, 0::2, 1::2] + dy[:, 1::2, 0::2] + dy[:, 1::2, 1::2]


def forward(params, x, chans, store_bf16=False):
    """x: [n, H, W, 8] input (RGB in channels 0..2).  Returns (pred [n*H*W], cache).
    store_bf16: round every stored activation to bfloat16 (the prior's storage
    precision) while computing each layer in double precision."""
    q = bf16 if store_bf16 else _ident
    L = len(chans)
    cache = {"x": x}
    skips = []
    h = x
    for i in range(L):
        a = q(np.maximum(conv3x3(h, *params[f"enc{i}a"]), 0.0))
        bo = q(np.maximum(conv3x3(a, *params[f"enc{i}b"]), 0.0))
        cache[f"in{i}"], cache[f"a{i}"], cache[f"b{i}"] = h, a, bo
        if i < L - 1:
            skips.append(bo)
            h, cache[f"arg{i}"] = maxpool2(bo)
    up = bo
    for i in range(L - 2, -1, -1):
        cat = np.concatenate([upsample2(up), skips[i]], axis=3)
        da = q(np.maximum(conv3x3(cat, *params[f"dec{i}a"]), 0.0))
        db = q(np.maximum(conv3x3(da, *params[f"dec{i}b"]), 0.0))
        cache[f"cat{i}"], cache[f"da{i}"], cache[f"db{i}"] = cat, da, db
        up = db
    hw, hb = params["head"]
    pred = (up @ hw + hb[0]).reshape(-1)
    cache["last"] = up
    return pred, cache


def loss_l1(pred, target, weight):
    e = pred - target
    P = pred.size
    return float((weight * np.abs(e)).sum() / P), weight * np.sign(e) / P


def backward(params, cache, dpred, chans, store_bf16=False):
    """store_bf16: round the masked gradient dZ of every layer to bfloat16 (its
    storage precision in the prior) before it enters that layer's products."""
    q = bf16 if store_bf16 else _ident
    L = len(chans)
    g = {}
    last = cache["last"]
    hw, hb = params["head"]
    dp = dpred.reshape(last.shape[:3])
    g["head"] = (np.einsum("nhw,nhwc->c", dp, last), np.array([dp.sum()]))
    dup = dp[..., None] * hw
    dskip = [None] * (L - 1)
    for i in range(L - 1):
        db_ = q(dup * (cache[f"db{i}"] > 0))
        dda, gw, gb = conv3x3_bwd(cache[f"da{i}"], params[f"dec{i}b"][0], db_)
        g[f"dec{i}b"] = (gw, gb)
        dza = q(dda * (cache[f"da{i}"] > 0))
        dcat, gw, gb = conv3x3_bwd(cache[f"cat{i}"], params[f"dec{i}a"][0], dza)
        g[f"dec{i}a"] = (gw, gb)
        cu = chans[i + 1]
        dskip[i] = dcat[..., cu:]
        dup = upsample2_bwd(dcat[..., :cu])
    dbo = dup
    for i in range(L - 1, -1, -1):
        if i < L - 1:
            dbo = dskip[i] + maxpool2_bwd(cache[f"arg{i}"], dh, cache[f"b{i}"].shape)
        dzb = q(dbo * (cache[f"b{i}"] > 0))
        da, gw, gb = conv3x3_bwd(cache[f"a{i}"], params[f"enc{i}b"][0], dzb)
        g[f"enc{i}b"] = (gw, gb)
        dza = q(da * (cache[f"a{i}"] > 0))
        dh, gw, gb = conv3x3_bwd(cache[f"in{i}"], params[f"enc{i}a"][0], dza)
        g[f"enc{i}a"] = (gw, gb)
    return g


def init_params(chans, seed=0, cin0=8):
    """Small random parameters of the same shapes as the CUDA path's."""
    rs = np.random.default_rng(seed)
    L = len(chans)
    p = {}
    def lay(name, cin, cout):
        p[name] = (rs.normal(size=(cout, 9, cin)) * np.sqrt(2.0 / (9 * cin)), rs.normal(size=cout) * 0.1)
    for i in range(L):
        lay(f"enc{i}a", cin0 if i == 0 else chans[i - 1], chans[i])
        lay(f"enc{i}b", chans[i], chans[i])
    for i in range(L - 2, -1, -1):
        lay(f"dec{i}a", chans[i + 1] + chans[i], chans[i])
        lay(f"dec{i}b", chans[i], chans[i])
    p["head"] = (rs.normal(size=chans[0]) * 0.3, np.array([0.5]))
    return p
