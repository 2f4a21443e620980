#!/usr/bin/env python
"""Throughput of the differentiable splatting rasterizer GEVO optimises through.

Metric: forward + backward Gaussian-pixel evaluations per second (and views per
second) over 16 batched keyframe views of a 500k-Gaussian SH-3 room scene, 12
views at 640x480 and 4 at 320x240 (the rendered past keyframes of Eq. 6, at the
TUM image size of Section III-A1), against the unbatched plain path on the same
GPU.  One step = projection of all views, tile binning and sort, blending, the
L1 photometric + depth loss against stop-gradient targets, the reverse walk and
the projection backward with se(3) pose gradients.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --case render|prior [--batch B]   # small cases to profile one
                                                    # kernel with ncu; no JSON line

N > 1 runs independent replicas, one per GPU (the path has no exchange step).
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
METRIC = "fwd+bwd Gaussian-pixel evals/s & views/s at 640x480, 500k Gaussians vs plain"
WORKLOAD = "16 keyframe views (12x640x480 + 4x320x240), 500k Gaussians, SH degree 3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mapping", action="store_true")
    ap.add_argument("--case", choices=["render", "prior"], default=None,
                    help="run a small profiling case instead of the benchmark")
    ap.add_argument("--batch", type=int, default=8, help="batch of the prior case")
    ap.add_argument("--threads-fwd", type=int, default=64, help="render case: blend threads per tile")
    ap.add_argument("--threads-bwd", type=int, default=64, help="render case: walk threads per tile")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# small cases to profile one kernel at a time with ncu: each holds well under
# 1 GB on the device while its inputs exceed the 129 MB L2, so DRAM counters
# stay meaningful and a capture of one launch (-k regex:<kernel> -s 1 -c 1)
# ends in seconds
# ---------------------------------------------------------------------------
def render_case(threads_fwd=64, threads_bwd=64):
    """4 views x 640x480 of the 500k-Gaussian room scene: two full forward +
    L1 + backward steps (persistent grids with the given threads per tile)."""
    import torch

    from paper_2409_09295_gb300 import raster, scenes
    from paper_2409_09295_gb300.batch import BatchedReplay
    w = scenes.workload(2)
    cams = w["cams"][:4]
    g = raster.gaussians_to_device(w["scene"])
    P = sum(c["W"] * c["H"] for c in cams)
    tr = torch.full((3 * P,), 0.5, device="cuda")
    td = torch.full((P,), 3.0, device="cuda")
    tf = dict(threads_per_tile=threads_fwd, persistent=1, blocks_per_sm=0)
    tb = dict(threads_per_tile=threads_bwd, persistent=1, blocks_per_sm=0)
    rep = BatchedReplay(g, cams, tr, td, 1.0, autotune=False, tuning_fwd=tf, tuning_bwd=tb)
    for _ in range(2):
        rep.step_eager()
        torch.cuda.synchronize()
    e_fwd, e_bwd = rep.eval_counts()
    print("render case ok, duplicates", rep.n_dup, "evals fwd", e_fwd, "bwd", e_bwd)


def prior_case(nb=8):
    """Two depth-prior train steps at batch nb x 320x240 (the bench line's step
    is nb = 32)."""
    import numpy as np
    import torch

    from paper_2409_09295_gb300.prior import DepthUNet
    net = DepthUNet(nb, 240, 320, seed=1)
    rs = np.random.default_rng(0)
    rgb = torch.from_numpy(rs.uniform(size=(nb, 3, 240, 320)).astype(np.float32)).cuda()
    tar = torch.from_numpy(rs.normal(1.0, 0.3, size=nb * 240 * 320).astype(np.float32)).cuda()
    for _ in range(2):
        net.train_step(rgb, tar, torch.ones_like(tar))
    torch.cuda.synchronize()
    print("prior case ok, loss", float(net.loss.item()))


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(views=(12,)):
    """Forward + backward of the given views of the workload through the oracle.
    Returns (seconds, evaluations, description)."""
    import numpy as np

    import oracle
    from paper_2409_09295_gb300 import scenes
    w = scenes.workload(2)
    cams = [w["cams"][v] for v in views]
    t0 = time.perf_counter()
    outs, projs, b = oracle.render_views(w["scene"], cams)
    gC = [np.sign(o["rgb"] - 0.5) / o["rgb"].size for o in outs]
    gD = [np.sign(o["depth"] - 3.0) / o["depth"].size for o in outs]
    oracle.backward_views(w["scene"], cams, projs, b, gC, gD, None)
    dt = time.perf_counter() - t0
    E = sum(int(o["n_eval"].sum()) + int(o["n_contrib"].sum()) for o in outs)
    sizes = "+".join(f"{c['W']}x{c['H']}" for c in cams)
    return dt, E, f"views {list(views)} ({sizes}) of the 16-view 500k workload, fwd+bwd, FP64"


def run_reference(args, rank):
    if rank != 0:
        return
    total_s, total_e = 0.0, 0
    desc = ""
    for i in range(args.warmup + args.steps):
        dt, E, desc = oracle_sample()
        if i >= args.warmup:
            total_s += dt
            total_e += E
    v = total_e / total_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle, one view per step"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# Algorithmic FP32 FLOPs (FMA = 2; ex2 and rcp on the MUFU not counted).  Every
# examined list entry costs the offset and power (10) and alpha = min(0.99,
# o G) (2); a blended entry adds, in the forward, T (1 - alpha), alpha T and the
# colour + depth sums (11) and, in the reverse walk, T recovery, weight,
# dL/dalpha, suffix update, colour / depth / opacity / conic / mean terms and
# the sum of its 10 gradient values over pixels (49).
FLOP_EXAMINE, FLOP_BLEND_FWD, FLOP_BLEND_BWD = 12, 11, 49


def whole_job(ms_local: float, units_local: float, world: int, device=None):
    """Each rank times an independent replica; the job's time is the slowest
    rank's and its work the sum of the ranks': returns (max ms, total units)."""
    if world == 1:
        return ms_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local, units_local], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def main():
    args = parse()
    if args.case is not None:
        import torch
        torch.cuda.set_device(0)
        if args.case == "render":
            render_case(args.threads_fwd, args.threads_bwd)
        else:
            prior_case(args.batch)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_2409_09295_gb300 import _abi, raster, scenes
    from paper_2409_09295_gb300.batch import BatchedReplay, HostStep, PlainReplay
    _abi.load()

    dev = torch.device("cuda", local)
    w = scenes.workload(2)
    scene, cams = w["scene"], w["cams"]
    g = raster.gaussians_to_device(scene, dev)
    # stop-gradient targets: renders of the previous map (the jittered scene)
    gt = raster.gaussians_to_device(w["target_scene"], dev)
    zero_rgb = None
    tgt = BatchedReplay(gt, cams, zero_rgb, autotune=False, tuning_fwd=dict(
        threads_per_tile=256, persistent=0, blocks_per_sm=0), tuning_bwd=dict(
        threads_per_tile=256, persistent=0, blocks_per_sm=0))
    tgt.pipe.forward(gt, tgt.camt)
    target_rgb = tgt.pipe.rgb.clone()
    target_depth = tgt.pipe.depth.clone()
    del tgt
    torch.cuda.empty_cache()

    rep = BatchedReplay(g, cams, target_rgb, target_depth, lambda_depth=1.0)
    E_fwd, E_bwd, B = rep.eval_counts(blended=True)
    rep.capture()                          # the whole step: one CUDA graph
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        rep.replay()
    torch.cuda.synchronize()
    assert rep.pipe.last_error() == 0, "duplicate capacity exceeded"

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()                      # L2 flushed between timed steps
        evs[k][0].record()
        rep.replay()
        evs[k][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall1 = time.perf_counter()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    assert rep.pipe.last_error() == 0, "duplicate capacity exceeded"
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    V = len(cams)
    total_ms, evals = whole_job(sum(step_ms), (E_fwd + E_bwd) * args.steps, world, dev)
    value = evals / (total_ms / 1e3)
    views_per_s = V * args.steps * world / (total_ms / 1e3)

    # ---- per-stage times (diagnostic: the six stages as graphs of their own,
    # events between them, same L2 flush; the step above is one graph) --------
    nst = len(rep.stages())
    sevs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)]
            for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        rep.replay_stages(sevs[k])
    torch.cuda.synchronize()
    stage_ms = {name: sum(e[i].elapsed_time(e[i + 1]) for e in sevs) / args.steps
                for i, (name, _) in enumerate(rep.stages())}
    staged_ms = sum(e[0].elapsed_time(e[-1]) for e in sevs) / args.steps

    # ---- end to end with host buffers: uploads of parameters, cameras and
    # targets from pinned memory, the step, and the read-back of the loss, the
    # pose gradients and all parameter gradients, as one graph per step ------
    hs = HostStep(rep)
    h2d, d2h = hs.h2d_bytes, hs.d2h_bytes
    for _ in range(2):
        hs.step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        hs.step()
        e.record()
        e.synchronize()
        e2e_ms += s.elapsed_time(e)
    assert rep.pipe.last_error() == 0, "duplicate capacity exceeded"
    assert torch.isfinite(hs.host_out["means"]).all()
    e2e_ms, e2e_evals = whole_job(e2e_ms, (E_fwd + E_bwd) * args.steps, world, dev)
    e2e_value = e2e_evals / (e2e_ms / 1e3)

    # ---- the plain (unbatched) path on the same GPU --------------------------------------
    plain = PlainReplay(g, cams, target_rgb, target_depth, lambda_depth=1.0)
    plain.step()
    torch.cuda.synchronize()
    pms = 0.0
    for _ in range(args.plain_steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        plain.step()
        e.record()
        e.synchronize()
        pms += s.elapsed_time(e)
    pms /= args.plain_steps
    plain_line = {"evals_per_s": (E_fwd + E_bwd) / (pms / 1e3), "views_per_s": V / (pms / 1e3),
                  "ms_per_step": pms}

    active_line = active_set_section(rep, target_rgb, target_depth, flush, stage_ms)
    mapping_line = mapping_section() if not args.no_mapping else None
    micro = micro_peaks()
    prior_line = prior_section() if not args.no_mapping else None

    # ---- rooflines (algorithmic work per launch / live event time) ---------------------
    pk = peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_peak = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = sm_count * 128 * 2 * clk_peak * 1e6 / 1e12   # TFLOP/s, FMA = 2
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    N = int(g["means"].shape[0])
    VN = V * N
    vis = int((rep.pipe.proj["radius"] > 0).sum())
    D = rep.n_dup
    P = rep.pipe.P
    K = (scene["sh_degree"] + 1) ** 2
    param_b = 4 * (3 + 3 + 4 + 1 + 3 * K)
    work = {  # (bound, algorithmic amount per launch, unit)
        "project": ("hbm", param_b * N + 48 * vis + 8 * (VN - vis) + 40 * vis, "GB/s"),
        "bin_sort": ("hbm", sort_bytes(rep, VN, vis, D), "GB/s"),
        "render_fwd": ("alu", FLOP_EXAMINE * E_fwd + FLOP_BLEND_FWD * B, "TFLOP/s"),
        "loss": ("hbm", 48 * P, "GB/s"),
        "render_bwd": ("alu", FLOP_EXAMINE * E_bwd + FLOP_BLEND_BWD * B, "TFLOP/s"),
        "project_bwd": ("hbm", 2 * param_b * N + 4 * VN + 40 * vis, "GB/s"),
    }
    n_sort = _abi.gevo_bin_sort_launches(rep.pipe.layout, rep.pipe.n, rep.pipe.capacity)
    kernels = {"project": "k_project_fwd (with the 2-D gradient rows zeroed)",
               "bin_sort": ("depth-ordered path, 12 kernels (k_ord_scatter the longest)"
                            if n_sort == 12 else "k_count_off+k_scan+k_scatter_off+k_segsort"),
               "render_fwd": "k_render_fwd", "loss": "k_loss_l1",
               "render_bwd": "k_render_bwd", "project_bwd": "k_pbwd_order+k_project_bwd_col+k_project_bwd_geo"}
    roofs = {}
    for name, (bound, amount, unit) in work.items():
        sec = stage_ms[name] / 1e3
        if bound == "alu":
            ach, peak = amount / sec / 1e12, fp32_peak
        else:
            ach, peak = amount / sec / 1e9, hbm_peak
        roofs[name] = {"bound": bound, "kernel": kernels[name], "achieved": ach, "peak": peak,
                       "unit": unit, "frac": ach / peak, "ms": stage_ms[name]}
    dom = "render_bwd"   # the largest share of the step in the ncu launch list
    roof = dict(roofs[dom])
    # DRAM bytes of one reverse-walk launch: ncu (dram__bytes_read.sum + write) of the
    # current kernel (32 threads per tile) on the 4-view case
    # (`bench.py --case render --threads-bwd 32`), 51.42 MB for 245.15M walked
    # entries, scaled by entries to this launch (same scene, same resolution)
    roof.update({"traffic": 51.42e6 * E_bwd / 245.15e6,
                 "traffic_source": "ncu dram bytes of the 4-view case, scaled by walked entries",
                 "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {clk_peak:.0f} MHz"})

    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "views": V, "gaussians": int(g["means"].shape[0]),
                       "duplicates": rep.n_dup, "evals_fwd": E_fwd, "evals_bwd": E_bwd,
                       "blended": B,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "flushed (256 MB write) between timed steps",
                       "tuning_fwd": rep.tuning_fwd, "tuning_bwd": rep.tuning_bwd,
                       "graphs": "1 CUDA graph per step"},
            "views_per_s": views_per_s, "stage_ms": stage_ms,
            "stage_ms_note": ("diagnostic run of the same step as six stage graphs with "
                              f"events between them ({staged_ms:.3f} ms per step); the "
                              "rooflines use these stage times"),
            "rooflines": roofs,
            "plain": plain_line, "speedup_vs_plain": value / plain_line["evals_per_s"],
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
                    "note": "batch.HostStep, one graph per step: parameters, cameras and "
                            "targets uploaded from pinned host memory, the step, and the loss, "
                            "pose gradients and every parameter gradient read back"},
            "gpu_launches": None, "roofline": roof, "clocks": clk, "active_set": active_line,
            "mapping": mapping_line, "micro_peaks": micro, "prior": prior_line,
            "wall_s_timed": wall1 - wall0}
    line["gpu_launches"] = launches_per_step(rep) * args.steps

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, E, desc = oracle_sample(views=(0, 1, 2, 12, 13, 14))
        line["cpu_baseline"] = {"value": E / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
                                "sample": desc + f", {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def active_set_section(rep, target_rgb, target_depth, flush, stage_ms, reps=10):
    """The active-set path of the global stage (Section III-B2) on the same
    workload: the loss with the per-pixel error, the reverse walk accumulating
    E_k(g) (Eq. 5), the active set at the threshold that keeps the 15% of the
    Gaussians the views see with the highest error (Section IV-C reports active
    sets under 15% of the map; in this dense synthetic room most Gaussians are
    hidden from every view and never blended, so a share of the whole map would
    keep every visible one), and the masked reverse walk and projection backward,
    each timed alone (CUDA events, L2 flushed before each launch)."""
    import torch

    from paper_2409_09295_gb300 import _abi
    pipe = rep.pipe
    pipe.alloc_active()
    tb = rep.tuning_bwd

    def timed(fn, before=None):
        """Mean device time of fn captured in a CUDA graph (no host work inside
        the timed region)."""
        for _ in range(2):
            if before:
                before()
            fn()
        torch.cuda.synchronize()
        gph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gph):
            fn()
        ms = 0.0
        for _ in range(reps):
            if before:
                before()
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            gph.replay()
            e.record()
            e.synchronize()
            ms += s.elapsed_time(e)
        return ms / reps

    def walk(error, masked, from_state=False):
        _abi.gevo_render_bwd_active(
            pipe.layout, pipe.n, pipe.proj, pipe.vals, pipe.ranges, rep.bg, pipe.T_final,
            pipe.n_contrib, pipe.dL_drgb, pipe.dL_ddepth, None,
            pipe.pix_err if error else None, pipe.gauss_err if error else None,
            pipe.active if masked else None, pipe.grad2d, pipe.ws, tb,
            state=pipe.act_state if from_state else None)

    rep.replay()
    ms = {"loss_err": timed(lambda: pipe.loss_l1_err(target_rgb, target_depth, 1.0))}
    ms["render_bwd_full"] = timed(lambda: walk(False, False), before=pipe.grad2d_zero)
    ms["render_bwd_error"] = timed(lambda: walk(True, False),
                                   before=lambda: (pipe.grad2d_zero(), pipe.gauss_err.zero_()))
    N = pipe.n
    emax = pipe.gauss_err.view(pipe.V, N).max(dim=0).values.float().cpu()
    seen = emax[emax > 0]            # Gaussians that some keyframe blends at all
    eps = float(torch.kthvalue(seen, max(1, int(0.85 * seen.numel()))).values) if seen.numel() else 0.0
    ms["active_set"] = timed(lambda: pipe.active_set(eps))
    active = int(pipe.active_counts[0].item())
    ms["render_bwd_masked"] = timed(lambda: walk(False, True), before=pipe.grad2d_zero)
    ms["render_fwd"] = timed(lambda: pipe.render_fwd(rep.bg, tuning=rep.tuning_fwd))
    ms["render_fwd_active"] = timed(lambda: pipe.render_fwd_active(rep.bg, tuning=rep.tuning_fwd))
    ms["render_bwd_from_state"] = timed(lambda: walk(False, True, True), before=pipe.grad2d_zero)
    ms["project_bwd_masked"] = timed(lambda: pipe.project_bwd_active(rep.g, rep.camt))
    full = ms["render_bwd_full"] + stage_ms["project_bwd"]
    masked = (ms["render_fwd_active"] - ms["render_fwd"]) + ms["render_bwd_from_state"] + \
        ms["project_bwd_masked"]
    return {"active": active, "frac": active / N, "seen": int(seen.numel()), "eps": eps, "ms": ms,
            "full_ms": {"render_bwd": stage_ms["render_bwd"], "project_bwd": stage_ms["project_bwd"]},
            "backward_speedup": full / masked,
            "backward_speedup_whole_lists": full / (ms["render_bwd_masked"] + ms["project_bwd_masked"]),
            "note": "E_k from the step's own render vs the stop-gradient targets; eps = 85th "
                    "percentile of max_k E_k(g) over the Gaussians some view blends (seen)"}


def micro_peaks():
    """Measured FP32 FMA and MUFU ex2 throughput (the units the blend and its
    reverse walk use), against which the derived ALU peak can be checked."""
    import torch

    from paper_2409_09295_gb300 import _abi
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    sink = torch.empty(blocks * 256, device="cuda")

    def best_ms(fn):
        fn()
        t = []
        for _ in range(3):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            e.synchronize()
            t.append(s.elapsed_time(e))
        return min(t)
    it_f, it_e = 20000, 4000
    ms_f = best_ms(lambda: _abi.gevo_bench_fma(blocks, it_f, sink))
    ms_f2 = best_ms(lambda: _abi.gevo_bench_fma2(blocks, it_f, sink))
    ms_e = best_ms(lambda: _abi.gevo_bench_ex2(blocks, it_e, sink))
    ms_r = best_ms(lambda: _abi.gevo_bench_rcp(blocks, it_e, sink))
    return {"fp32_fma_tflops": blocks * 256 * 16 * it_f / (ms_f / 1e3) / 1e12,
            "fp32x2_fma_tflops": blocks * 256 * 32 * it_f / (ms_f2 / 1e3) / 1e12,
            "ex2_per_s": blocks * 256 * 8 * it_e / (ms_e / 1e3),
            "rcp_per_s": blocks * 256 * 8 * it_e / (ms_r / 1e3),
            "note": f"{blocks} blocks x 256 threads, 8 independent chains per thread "
                    "(fp32x2: packed pairs, 16 FMAs per step)"}


def prior_section(nb=32, H=240, W=320, steps=8):
    """Training throughput of the learned depth prior (BF16 U-Net, tcgen05) at
    batch 32 of 320x240 renders: images per second, and the convolutions'
    algorithmic FLOPs (forward 2 P 9 Cin Cout per layer, backward twice that
    but no data gradient for the first layer) per second against the measured
    BF16 tensor peak."""
    import numpy as np
    import torch

    from paper_2409_09295_gb300.prior import DepthUNet
    net = DepthUNet(nb, H, W, seed=3)
    rs = np.random.default_rng(0)
    rgb = torch.from_numpy(rs.uniform(size=(nb, 3, H, W)).astype(np.float32)).cuda()
    tar = torch.from_numpy(rs.normal(1.0, 0.3, size=nb * H * W).astype(np.float32)).cuda()
    wgt = torch.ones_like(tar)
    for _ in range(2):
        net.train_step(rgb, tar, wgt)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(steps):
        net.train_step(rgb, tar, wgt)
    e.record()
    e.synchronize()
    ms = s.elapsed_time(e) / steps
    flop = 0.0
    for name, lay in net.layers.items():
        lvl = int(name[3])
        P = nb * net.hw[lvl][0] * net.hw[lvl][1]
        cin = 3 if name == "enc0a" else lay["cin"]   # RGB input, padded to 8 channels
        f = 2.0 * P * 9 * cin * lay["cout"]
        flop += f * (2.0 if name == "enc0a" else 3.0)
    pk = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))
    ach = flop / (ms / 1e3) / 1e12
    return {"images_per_s": nb / (ms / 1e3), "ms_per_step": ms, "batch": nb, "image": f"{W}x{H}",
            "conv_tflops": ach, "bf16_peak_tflops": peak, "frac": ach / peak,
            "note": "train step (forward, L1, backward, Adam) with host launches included; "
                    "channels 16-128 keep the MMAs small, so the step is far from the tensor peak"}


def mapping_section():
    """One mapping update (local + global stage) on the same room, at 640x480:
    8 window keyframes, 4 past poses for E_pc, the 52k-Gaussian box as the
    local map; median device time per iteration and the loss trajectory."""
    import numpy as np

    from paper_2409_09295_gb300.mapping import room_update
    r = room_update(local_iters=10, global_iters=10)
    med = lambda x: float(np.median(x[1:]))
    return {"local_iter_ms": med(r["local_iter_ms"]), "global_iter_ms": med(r["global_iter_ms"]),
            "local_loss": [r["local_losses"][0], r["local_losses"][-1]],
            "global_loss": [r["global_losses"][0], r["global_losses"][-1]],
            "active": r["active"], "error_active": r["error_active"], "pruned": r["pruned"],
            "map_size": r["map_size"], "window": r["window"], "past": r["past"], "image": r["image"],
            "note": "10 + 10 iterations; the full-backward global stage (exact pose gradient)"}


def launches_per_step(rep) -> int:
    """Kernels of ours launched per step: project (1, also zeroing the 2-D
    gradient rows), bin_sort (as the library reports for these sizes: 12 on the
    depth-ordered path), render_fwd (1), loss (1), render_bwd (1), project_bwd
    (the Gaussian order, the geometry kernel, and the SH-colour kernel when
    colours are SH)."""
    from paper_2409_09295_gb300 import _abi
    p = rep.pipe
    sort = _abi.gevo_bin_sort_launches(p.layout, p.n, p.capacity)
    return 1 + sort + 1 + 1 + 1 + (2 if p.colour == "rgb" else 3)


def sort_bytes(rep, VN: int, vis: int, D: int) -> int:
    """Bytes the depth-ordered sort's passes move (model): per (view, Gaussian)
    entry the radius read and the depth-bits word written once and read twice
    (16 B); per visible entry 168 B (depth and mean read, rectangle written, the
    depth-segment scatter, the per-view depth sort's read and two writes, the
    record gather and write, the area prefix, three walks over records and
    prefixes); per duplicate the 4-byte id written; per (unit of 8192
    duplicates, tile) 16 B of counts (written, scanned in place, read); per tile
    the range and its start."""
    T = rep.pipe.T
    units = -(-D // 8192) + rep.pipe.V
    max_tiles = max(-(-w // 16) * -(-h // 16) for w, h in rep.pipe.sizes)
    return 16 * VN + 168 * vis + 4 * D + 16 * units * max_tiles + 12 * T


if __name__ == "__main__":
    main()
