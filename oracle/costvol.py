"""FP64 oracle of the plain initialisation's photometric cost volume (Eq. 1,
Section III-A1), test infrastructure only.

V(u, d_k) = mean over the other keyframes i of |I_ref(u) - I_i(pi(u, d_k))|,
on images downsampled 4x (grey = mean of RGB over each 4x4 block), d_k
spaced linearly over [d0, d1], bilinear sampling with pixel i at coordinate i,
samples outside the image left out of the mean (1.0 where none remain), then
winner-take-all (lowest cost, lowest index first) and nearest x4 upsampling.
"""
from __future__ import annotations

import numpy as np


def grey4(rgb):
    nk, _, H, W = rgb.shape
    g = rgb.mean(axis=1).reshape(nk, H // 4, 4, W // 4, 4).mean(axis=(2, 4))
    return g


def _bilinear(img, u, v):
    h, w = img.shape
    ok = (u >= 0) & (v >= 0) & (u <= w - 1) & (v <= h - 1)
    x0 = np.clip(np.floor(u).astype(np.int64), 0, max(w - 2, 0))
    y0 = np.clip(np.floor(v).astype(np.int64), 0, max(h - 2, 0))
    fx, fy = u - x0, v - y0
    a = img[y0, x0]; b = img[y0, np.minimum(x0 + 1, w - 1)]
    c = img[np.minimum(y0 + 1, h - 1), x0]; d = img[np.minimum(y0 + 1, h - 1), np.minimum(x0 + 1, w - 1)]
    val = (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d)
    return np.where(ok, val, 0.0), ok


def cost_volume(rgb, cams, ref, nd=64, d0=0.25, d1=25.0):
    """rgb [nk,3,H,W]; cams [nk,16] (R, t, fx, fy, cx, cy).  Returns (V [h,w,nd],
    fragile [h,w,nd]: a sample lies within 1e-3 px of an image border)."""
    g = grey4(np.asarray(rgb, np.float64))
    nk, h, w = g.shape
    cams = np.asarray(cams, np.float64)
    cr = cams[ref]
    R0, t0 = cr[:9].reshape(3, 3), cr[9:12]
    fx, fy, cx, cy = cr[12:16] / 4.0
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    V = np.zeros((h, w, nd))
    frag = np.zeros((h, w, nd), bool)
    for k in range(nd):
        d = d0 + (d1 - d0) * k / (nd - 1)
        pc = np.stack([(xs + 0.5 - cx) / fx * d, (ys + 0.5 - cy) / fy * d, np.full_like(xs, d)], -1)
        pw = (pc - t0) @ R0
        acc = np.zeros((h, w))
        cnt = np.zeros((h, w))
        for s in range(nk):
            if s == ref:
                continue
            Rs, ts = cams[s, :9].reshape(3, 3), cams[s, 9:12]
            p = pw @ Rs.T + ts
            front = p[..., 2] > 1e-3
            z = np.where(front, p[..., 2], 1.0)
            u = cams[s, 12] / 4 * p[..., 0] / z + cams[s, 14] / 4 - 0.5
            v = cams[s, 13] / 4 * p[..., 1] / z + cams[s, 15] / 4 - 0.5
            val, ok = _bilinear(g[s], u, v)
            ok &= front
            edge = (np.abs(u) < 1e-3) | (np.abs(v) < 1e-3) | (np.abs(u - (w - 1)) < 1e-3) | \
                (np.abs(v - (h - 1)) < 1e-3) | (np.abs(p[..., 2] - 1e-3) < 1e-6)
            frag[..., k] |= edge
            acc += np.where(ok, np.abs(g[ref] - val), 0.0)
            cnt += ok
        V[..., k] = np.where(cnt > 0, acc / np.maximum(cnt, 1), 1.0)
    return V, frag


def wta_up4(V, d0=0.25, d1=25.0):
    nd = V.shape[-1]
    k = np.argmin(V, axis=-1)
    d = d0 + (d1 - d0) * k / (nd - 1)
    return d.repeat(4, axis=0).repeat(4, axis=1)


# ---------------------------------------------------------------------------
# Belief propagation (Section III-A2, with the min-sum algorithm of Felzenszwalb
# and Huttenlocher, 2006, that the paper cites): the labels are the depth
# hypotheses, the data cost of label f at pixel p is V(p, d_f), the
# discontinuity cost between neighbours is the truncated linear
# min(s |f_p - f_q|, tau), the grid is 4-connected.  Messages start at zero and
# are all updated together (synchronous iterations):
#   m_{p->q}(f_q) = min_{f_p} [ D_p(f_p) + sum_{r in N(p), r != q} m_{r->p}(f_p)
#                               + min(s |f_p - f_q|, tau) ]
# then shifted so that their minimum over f_q is 0.  After the last iteration
# the label of p minimises D_p + sum of all incoming messages (lowest label on
# ties).  The minimum over f_p is taken by brute force here.
# ---------------------------------------------------------------------------
# directions: message sent to the left, right, upper, lower neighbour
_DIRS = ((0, -1), (0, 1), (-1, 0), (1, 0))
_OPP = (1, 0, 3, 2)


def bp_message(h, s, tau):
    """min over f_p of h(f_p) + min(s |f_p - f_q|, tau), for every f_q (last axis)."""
    k = h.shape[-1]
    f = np.arange(k)
    cost = np.minimum(s * np.abs(f[:, None] - f[None, :]), tau)     # [f_p, f_q]
    m = (h[..., :, None] + cost).min(axis=-2)
    return m - m.min(axis=-1, keepdims=True)


def _incoming(msgs, d):
    """Messages arriving at each pixel from its neighbour in direction d: the
    neighbour sent them in the opposite direction (0 outside the image)."""
    dy, dx = _DIRS[d]
    src = msgs[_OPP[d]]
    out = np.zeros_like(src)
    h, w = src.shape[:2]
    ys = slice(max(dy, 0), h + min(dy, 0))
    yd = slice(max(-dy, 0), h + min(-dy, 0))
    xs = slice(max(dx, 0), w + min(dx, 0))
    xd = slice(max(-dx, 0), w + min(-dx, 0))
    out[yd, xd] = src[ys, xs]
    return out


def bp(V, s, tau, iters):
    """V [h, w, nd] data costs.  Returns (labels [h, w], beliefs [h, w, nd],
    messages [4, h, w, nd])."""
    D = np.asarray(V, np.float64)
    msgs = np.zeros((4,) + D.shape)
    for _ in range(iters):
        inc = [_incoming(msgs, d) for d in range(4)]
        tot = D + sum(inc)
        # to the neighbour in direction d: leave out what came from it
        msgs = np.stack([bp_message(tot - inc[d], s, tau) for d in range(4)])
    inc = [_incoming(msgs, d) for d in range(4)]
    B = D + sum(inc)
    return np.argmin(B, axis=-1), B, msgs


def bp_depth_up4(V, s, tau, iters, d0=0.25, d1=25.0):
    nd = V.shape[-1]
    lab, _, _ = bp(V, s, tau, iters)
    d = d0 + (d1 - d0) * lab / (nd - 1)
    return d.repeat(4, axis=0).repeat(4, axis=1)
