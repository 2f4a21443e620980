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


def grad_close(g, ref, name, rel=1e-3):
    """Gradient tolerance: relative L2 error <= rel per tensor, and per element
    |g - ref| <= rel |ref| + rel rms(ref)."""
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
