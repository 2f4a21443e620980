"""Small, self-contained workloads to profile one kernel at a time with ncu.

  python -m paper_2409_09295_gb300.profile_cases render   # 4 views x 640x480 of
      the 500k-Gaussian room scene: two full forward + L1 + backward steps
  python -m paper_2409_09295_gb300.profile_cases prior [B] # two depth-prior train
      steps at batch B (default 8) x 320x240; the bench line's step is B = 32

Each case holds well under 1 GB on the device while its inputs exceed the
129 MB L2, so DRAM counters stay meaningful and an ncu capture of one launch
(`-k regex:<kernel> -s 1 -c 1`) ends in seconds.
"""
from __future__ import annotations

import sys

import numpy as np
import torch


def render_case():
    from . import raster, scenes
    from .batch import BatchedReplay
    w = scenes.workload(2)
    cams = w["cams"][:4]
    g = raster.gaussians_to_device(w["scene"])
    P = sum(c["W"] * c["H"] for c in cams)
    tr = torch.full((3 * P,), 0.5, device="cuda")
    td = torch.full((P,), 3.0, device="cuda")
    t = dict(threads_per_tile=64, persistent=1, blocks_per_sm=0)
    rep = BatchedReplay(g, cams, tr, td, 1.0, autotune=False, tuning_fwd=t, tuning_bwd=t)
    for _ in range(2):
        rep.step_eager()
        torch.cuda.synchronize()
    e_fwd, e_bwd = rep.eval_counts()
    print("render case ok, duplicates", rep.n_dup, "evals fwd", e_fwd, "bwd", e_bwd)


def prior_case(nb=8):
    from .prior import DepthUNet
    net = DepthUNet(nb, 240, 320, seed=1)   # the bench line's scratch size
    rs = np.random.default_rng(0)
    rgb = torch.from_numpy(rs.uniform(size=(nb, 3, 240, 320)).astype(np.float32)).cuda()
    tar = torch.from_numpy(rs.normal(1.0, 0.3, size=nb * 240 * 320).astype(np.float32)).cuda()
    for _ in range(2):
        net.train_step(rgb, tar, torch.ones_like(tar))
    torch.cuda.synchronize()
    print("prior case ok, loss", float(net.loss.item()))


if __name__ == "__main__":
    torch.cuda.set_device(0)
    case = sys.argv[1] if len(sys.argv) > 1 else "render"
    if case == "prior":
        prior_case(int(sys.argv[2]) if len(sys.argv) > 2 else 8)
    else:
        render_case()
