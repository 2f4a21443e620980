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
