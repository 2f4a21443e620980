"""Whole-view oracle runs split across host threads, for parity at the
workloads' full sizes.

The FP64 oracle's C routines hold no global state and release the GIL while
they run, so independent pieces of one computation run in parallel threads:
the projection and its derivative over chunks of Gaussians (each Gaussian is
independent; pose gradients add up), and the blend and its derivative over
bands of tile rows (a pixel's result depends only on its own tile's list; the
tiles outside a band get empty lists, so the band's call leaves them at the
background).  Every number still comes from the oracle's own routines; this
module only cuts the work into pieces and puts them back together.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle

THREADS = max(1, min(32, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                     else os.cpu_count() or 1))


def _chunks(n, k):
    k = max(1, min(k, n)) if n else 1
    edges = np.linspace(0, n, k + 1).astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a] or [(0, 0)]


def _sub(g, a, b):
    out = {k: (v[a:b] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    return out


def project(g, cam, pool):
    n = g["means"].shape[0]
    parts = list(pool.map(lambda ab: oracle.project(_sub(g, *ab), cam), _chunks(n, THREADS)))
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def _bands(W, H):
    ty = (H + 15) // 16
    return _chunks(ty, THREADS)


def _band_ranges(ranges_view, W, r0, r1):
    tx = (W + 15) // 16
    rv = np.zeros_like(ranges_view)
    rv[r0 * tx:r1 * tx] = ranges_view[r0 * tx:r1 * tx]
    return rv


def _rec(p):
    return dict(xy=p["xy"], conic=p["conic"], opacity=p["opacity"], rgb=p["rgb"], depth=p["depth"])


def render_fwd(W, H, rec, vals, ranges_view, bg, pool):
    def one(band):
        r0, r1 = band
        return band, oracle.render_fwd(W, H, rec, vals, _band_ranges(ranges_view, W, r0, r1), bg)
    res = list(pool.map(one, _bands(W, H)))
    out = {k: v.copy() for k, v in res[0][1].items()}
    for (r0, r1), o in res:
        y0, y1 = r0 * 16, min(r1 * 16, H)
        for k, v in o.items():
            if k == "rgb":
                out[k][:, y0:y1] = v[:, y0:y1]
            else:
                out[k][y0:y1] = v[y0:y1]
    return out


def render_views(g, cams, bg=(0.0, 0.0, 0.0)):
    """Same results as oracle.render_views, computed in parallel pieces."""
    with cf.ThreadPoolExecutor(THREADS) as pool:
        projs = [project(g, c, pool) for c in cams]
        sizes = [(int(c["W"]), int(c["H"])) for c in cams]
        b = oracle.bin_f32(sizes, np.stack([p["xy"].astype(np.float32) for p in projs]),
                           np.stack([p["radius"] for p in projs]),
                           np.stack([p["depth"].astype(np.float32) for p in projs]))
        outs, base = [], 0
        for v, (W, H) in enumerate(sizes):
            nt = oracle.tiles_of(W, H)
            outs.append(render_fwd(W, H, _rec(projs[v]), b["vals"], b["ranges"][base:base + nt],
                                   bg, pool))
            base += nt
    return outs, projs, b


def backward_views(g, cams, projs, b, dL_drgb, dL_ddepth=None, dL_dT=None, bg=(0.0, 0.0, 0.0)):
    """Same results as oracle.backward_views (up to the order of the sums),
    computed in parallel pieces."""
    acc = oracle.grads_like(g)
    dxis = np.zeros((len(cams), 6))
    g2ds = []
    with cf.ThreadPoolExecutor(THREADS) as pool:
        base = 0
        for v, cam in enumerate(cams):
            W, H = int(cam["W"]), int(cam["H"])
            nt = oracle.tiles_of(W, H)
            rv = b["ranges"][base:base + nt]
            base += nt
            rec = _rec(projs[v])

            def bwd(band, W=W, H=H, rv=rv, rec=rec, v=v):
                return oracle.render_bwd(W, H, rec, b["vals"], _band_ranges(rv, W, *band),
                                         dL_drgb[v], None if dL_ddepth is None else dL_ddepth[v],
                                         None if dL_dT is None else dL_dT[v], bg)
            parts = list(pool.map(bwd, _bands(W, H)))
            g2d = {k: sum(p[k] for p in parts) for k in parts[0]}
            g2ds.append(g2d)

            def pbwd(ab, cam=cam, v=v, g2d=g2d):
                a, c = ab
                sub = _sub(g, a, c)
                part = oracle.grads_like(sub)
                dxi = np.zeros(6)
                oracle.project_bwd(sub, cam, projs[v]["radius"][a:c],
                                   {k: x[a:c] for k, x in g2d.items()}, part, dxi)
                return ab, part, dxi
            for (a, c), part, dxi in pool.map(pbwd, _chunks(g["means"].shape[0], THREADS)):
                for k in acc:
                    acc[k][a:c] += part[k]
                dxis[v] += dxi
    return acc, dxis, g2ds
