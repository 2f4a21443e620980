"""Shared helpers of the GPU parity tests: upload seeded inputs, run the CUDA
path through the C ABI, run the oracle on the same inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle


def tiles_of(W, H):
    return ((W + 15) // 16) * ((H + 15) // 16)


def records_for_oracle(rec, v):
    """Binary32 synthetic records of view v, widened to float64 for the oracle."""
    return dict(xy=rec["xy"][v].astype(np.float64), conic=rec["conic"][v].astype(np.float64),
                opacity=rec["opacity"].astype(np.float64), rgb=rec["rgb"][v].astype(np.float64),
                depth=rec["depth"][v].astype(np.float64))


def upload_records(pipe, rec):
    """Write synthetic binary32 records into the pipeline's projection buffers."""
    import torch
    V, n = rec["xy"].shape[:2]
    dev = pipe.device
    co = np.zeros((V, n, 4), np.float32)
    co[..., :3] = rec["conic"]
    co[..., 3] = rec["opacity"][None, :]
    rz = np.zeros((V, n, 4), np.float32)
    rz[..., :3] = rec["rgb"]
    rz[..., 3] = rec["depth"]
    pipe.proj["xy"].copy_(torch.from_numpy(rec["xy"].reshape(V * n, 2)).to(dev))
    pipe.proj["conic_opacity"].copy_(torch.from_numpy(co.reshape(V * n, 4)).to(dev))
    pipe.proj["rgb_depth"].copy_(torch.from_numpy(rz.reshape(V * n, 4)).to(dev))
    pipe.proj["radius"].copy_(torch.from_numpy(rec["radius"].reshape(V * n)).to(dev))


def grad_close(g, ref, name, rel=1e-3, rows_skip=None):
    """Gradient tolerance: relative L2 error <= rel per tensor, and per element
    |g - ref| <= rel |ref| + rel rms(ref).  rows_skip: optional boolean mask over
    the first axis (Gaussians whose projection decision the oracle reports
    within its margin); those rows count in the relative L2 error but are left
    out of the per-element check."""
    keep = None
    if rows_skip is not None:
        g0 = np.asarray(g, np.float64)
        keep = np.repeat(~np.asarray(rows_skip, bool), int(np.prod(g0.shape[1:])))
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0.0:
        assert np.abs(g).max() <= 1e-12, name
        return
    rms = nr / np.sqrt(ref.size)
    err = np.linalg.norm(g - ref) / nr
    assert err <= rel, f"{name}: relative L2 error {err:.3e}"
    bad = np.abs(g - ref) > rel * np.abs(ref) + rel * rms
    if keep is not None:
        bad &= keep
    assert not bad.any(), (f"{name}: {bad.sum()} elements out of tolerance, worst "
                           f"{np.abs(g - ref)[bad].max():.3e} (rms {rms:.3e})")


def oracle_tile_mask(W, H, xy, radius, flags):
    """Pixels of every tile that a flagged Gaussian's rectangle covers."""
    tx, ty = (W + 15) // 16, (H + 15) // 16
    m = np.zeros((H, W), bool)
    for g in np.nonzero(flags)[0]:
        r = int(radius[g]) if radius[g] > 0 else 64
        rc = oracle.rect_f32(xy[g, 0], xy[g, 1], max(r, 1), tx, ty)
        m[rc[1] * 16:rc[3] * 16, rc[0] * 16:rc[2] * 16] = True
    return m


def excluded_pixels(pipe, n, cams, v_of, outs, projs):
    """Per view, the pixels parity tests leave out: those whose blend decisions
    the oracle reports within a margin of a threshold, and the tiles of every
    Gaussian whose projection decision is fragile and whose binary32 radius or
    tile count came out differently on the GPU.  v_of[k] is the pipeline view of
    oracle view k."""
    rad_all = pipe.proj["radius"].cpu().numpy()
    tt_all = pipe.proj["tiles_touched"].cpu().numpy()
    masks = []
    for k, (cam, out, p) in enumerate(zip(cams, outs, projs)):
        v = v_of[k]
        W, H = cam["W"], cam["H"]
        m = out["fragile"] != 0
        rad_g = rad_all[v * n:(v + 1) * n]
        tt_g = tt_all[v * n:(v + 1) * n]
        tx, ty = (W + 15) // 16, (H + 15) // 16
        differs = (p["fragile"] != 0) & ((rad_g != p["radius"]) | (tt_g != p["tiles_touched"]))
        for i in np.nonzero(differs)[0]:
            r = max(int(p["radius"][i]), int(rad_g[i]), 1)
            rc = oracle.rect_f32(p["xy"][i, 0], p["xy"][i, 1], r, tx, ty)
            m[rc[1] * 16:rc[3] * 16, rc[0] * 16:rc[2] * 16] = True
        masks.append(m)
    return masks


def check_view_images(pipe, v, out, excluded, max_err=2e-4, median_err=1e-6):
    """Images of pipeline view v against one oracle view on the pixels not
    excluded: RGB within max_err (median within median_err), n_contrib equal,
    T_final within max_err, depth within max_err relative to the depth scale."""
    ok = ~excluded
    assert ok.mean() > 0.9, ok.mean()
    rgb = pipe.view_rgb(pipe.rgb, v).cpu().numpy()
    err = np.abs(rgb - out["rgb"])[:, ok]
    assert err.max() <= max_err, err.max()
    assert np.median(err) <= median_err
    np.testing.assert_array_equal(pipe.view_plane(pipe.n_contrib, v).cpu().numpy()[ok],
                                  out["n_contrib"][ok])
    np.testing.assert_allclose(pipe.view_plane(pipe.T_final, v).cpu().numpy()[ok], out["T"][ok],
                               atol=max_err)
    dep = pipe.view_plane(pipe.depth, v).cpu().numpy()[ok]
    np.testing.assert_allclose(dep, out["depth"][ok], atol=max_err * max(1.0, np.abs(out["depth"]).max()))
