"""One mapping update of GEVO: the local stage and the global stage.

Local stage (Section III-B1, Eq. 2): the local map -- the newly initialised
Gaussians -- and the window poses are optimised with E_pho + E_iso against
the sliding window's images.  The global map is rendered with it but not
changed, so that it can later render past keyframes at full fidelity.

Global stage (Section III-B2, Eq. 3): the local map is inserted into the
global map at opacity 0.2; the active set A_t = local map u E_t, E_t the
existing Gaussians whose rendering error E_k(g) (Eq. 5) exceeds eps in some
window view, is optimised with the window poses against E_pho + E_iso + E_pc,
E_pc comparing renders at four past poses with the stop-gradient renders of
the map before insertion (Eq. 6); optionally the backward runs only over the
active set (the active-set rasterizer; the pose gradient then counts only the
active Gaussians).  Afterwards active Gaussians with opacity below 0.7 are pruned (the occupancy
test of the paper is out of scope).

Every render, loss, gradient, selection, optimiser step and compaction runs in
libgevo (include/gevo.h, include/gevo_map.h); torch holds the buffers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _abi
from .raster import Pipeline, camera_tensor

# Learning rates (the 3DGS defaults; the paper does not list them), pose rates
# for the translation and rotation parts of the twist, E_iso weight.
DEFAULT_ADAM = dict(lr_means=1.6e-4, lr_log_scales=5e-3, lr_quats=1e-3, lr_logit_opacities=5e-2,
                    lr_colour_dc=2.5e-3, lr_colour_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999,
                    eps=1e-15, lambda_iso=10.0)
LR_POSE = (1e-3, 3e-3)
INSERT_OPACITY = 0.2      # Section III-B2, insertion
PRUNE_OPACITY = 0.7       # Section III-B2, pruning


def _logit(p):
    return math.log(p / (1.0 - p))


class GaussianMap:
    """A device-resident map: optimisation parameters, Adam moments, and the
    activated scales and opacities the rasterizer reads."""

    def __init__(self, scene: dict, device="cuda"):
        self.dev = torch.device(device)
        self.sh_degree = int(scene.get("sh_degree", 0)) if "sh" in scene else 0
        self.colour = "sh" if "sh" in scene else "rgb"
        col = np.asarray(scene["sh"] if self.colour == "sh" else scene["rgb"], np.float32)
        self.K = col.shape[1] if self.colour == "sh" else 1
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(self.dev)
        o = np.clip(np.asarray(scene["opacities"], np.float64), 1e-6, 1 - 1e-6)
        self.p = dict(means=f(scene["means"]), log_scales=f(np.log(scene["scales"])),
                      quats=f(scene["quats"]), logit_opacities=f(np.log(o / (1 - o))),
                      colours=f(col.reshape(-1, self.K, 3)))
        self._derived()

    @property
    def n(self) -> int:
        return int(self.p["means"].shape[0])

    def _derived(self):
        n = self.n
        self.m = {k: torch.zeros_like(t) for k, t in self.p.items()}
        self.v = {k: torch.zeros_like(t) for k, t in self.p.items()}
        self.scales = torch.empty(n, 3, device=self.dev)
        self.opacities = torch.empty(n, device=self.dev)
        self.activate()

    def activate(self):
        _abi.gevo_map_activate(self.n, self.p["log_scales"], self.p["logit_opacities"], self.scales,
                               self.opacities)

    def gaussians(self) -> dict:
        """The rasterizer's view of the map (activated scales and opacities)."""
        g = dict(means=self.p["means"], scales=self.scales, quats=self.p["quats"],
                 opacities=self.opacities)
        if self.colour == "sh":
            g["sh"] = self.p["colours"]
            g["sh_degree"] = self.sh_degree
        else:
            g["rgb"] = self.p["colours"].view(-1, 3)
        return g

    def rows(self, lo: int, hi: int) -> "GaussianMap":
        """A new map holding copies of rows [lo, hi) (fresh Adam moments)."""
        out = GaussianMap.__new__(GaussianMap)
        out.dev, out.sh_degree, out.colour, out.K = self.dev, self.sh_degree, self.colour, self.K
        out.p = {k: t[lo:hi].clone() for k, t in self.p.items()}
        out._derived()
        return out

    def append(self, other: "GaussianMap", opacity=None):
        """Inserts another map's Gaussians (their Adam moments restart); with
        `opacity` their opacity is set to that value.  Returns the index of the
        first inserted Gaussian."""
        first = self.n
        lo = other.p["logit_opacities"].clone()
        if opacity is not None:
            lo.fill_(_logit(opacity))
        parts = dict(other.p, logit_opacities=lo)
        self.p = {k: torch.cat([self.p[k], parts[k]]).contiguous() for k in self.p}
        self._derived()
        return first

    def compact(self, keep_list, counts, n_keep: int):
        """Keeps rows keep_list[0 .. n_keep) (gevo_gather_rows per array)."""
        out = {}
        for k, t in self.p.items():
            width = t[0].numel() if t.shape[0] else 1
            dst = torch.empty((n_keep,) + tuple(t.shape[1:]), device=self.dev)
            if n_keep:
                _abi.gevo_gather_rows(n_keep, keep_list, counts, width, t, dst)
            out[k] = dst
        self.p = out
        self._derived()


class MapOptimizer:
    """Runs optimisation iterations of a map and a set of poses through the
    batched rasterizer: forward, L1 loss, (masked) backward, Adam steps."""

    def __init__(self, gmap: GaussianMap, adam=None, lr_pose=LR_POSE, tuning=None):
        self.map = gmap
        self.adam = dict(DEFAULT_ADAM if adam is None else adam)
        self.lr_pose = lr_pose
        self.tuning = tuning
        self.step_no = 0
        self.pose_step_no = 0

    def _pipe(self, cams):
        sizes = [(int(c["W"]), int(c["H"])) for c in cams]
        pipe = Pipeline(self.map.n, sizes, 1 << 20, colour=self.map.colour,
                        sh_degree=self.map.sh_degree, device=self.map.dev, tuning=self.tuning)
        return pipe

    def iterate(self, cams, camt, targets, iters, fixed=None, active=None, masked=False,
                lambda_iso=None):
        """iters steps over views `cams` (pose tensor camt, updated in place for
        views not in `fixed`) against stop-gradient target images (planar,
        concatenated).  active: optional (bits, list, counts) of the rows to
        optimise (None = all).  masked=True runs the backward over the active
        rows only (the active-set rasterizer); the pose gradient is then the one
        through the active Gaussians.  masked=False runs the full backward, so
        the pose gradient counts every Gaussian, and updates the active rows.
        Returns the per-iteration losses E_pho (+ E_pc) + E_iso (host list)."""
        g = self.map.gaussians()
        pipe = self._pipe(cams)
        D = pipe.ensure_capacity(g, camt)
        if D * 1.3 > pipe.capacity:
            pipe.alloc_capacity(int(D * 1.3) + 1024)
        V = len(cams)
        fixed_t = None
        if fixed is not None:
            fixed_t = torch.tensor([1 if f else 0 for f in fixed], dtype=torch.uint8, device=self.map.dev)
        pm = torch.zeros(V, 6, device=self.map.dev)
        pv = torch.zeros(V, 6, device=self.map.dev)
        iso = torch.zeros(1, device=self.map.dev)
        cfg = dict(self.adam)
        if lambda_iso is not None:
            cfg["lambda_iso"] = lambda_iso
        losses = []
        K = self.map.K
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
        ev[0].record()
        for it in range(iters):
            pipe.project(g, camt)
            pipe.bin_sort()
            use_mask = active is not None and masked
            if use_mask:
                pipe.alloc_active()
                pipe.active.copy_(active[0])
                pipe.render_fwd_active()
            else:
                pipe.render_fwd()
            pipe.loss_l1(targets)
            if use_mask:
                pipe.render_bwd_active(pipe.dL_drgb, error=False, masked=True, from_state=True)
                pipe.active_list.copy_(active[1])
                pipe.active_counts.copy_(active[2])
                pipe.project_bwd_active(g, camt, want_dxi=True)
            else:
                pipe.render_bwd(pipe.dL_drgb)
                pipe.project_bwd(g, camt, want_dxi=True)
            rows, counts = (active[1], active[2]) if active is not None else (None, None)
            self.step_no += 1
            iso.zero_()
            _abi.gevo_map_step(self.map.n, K, self.map.p, pipe.grads, self.map.m, self.map.v, cfg,
                               self.step_no, rows, counts, self.map.scales, self.map.opacities,
                               iso)
            self.pose_step_no += 1
            _abi.gevo_pose_step(V, camt, pipe.dxi, pm, pv, self.lr_pose[0], self.lr_pose[1],
                                cfg["beta1"], cfg["beta2"], cfg["eps"], self.pose_step_no, fixed_t)
            losses.append(pipe.loss.sum() + iso[0])
            ev[it + 1].record()
        torch.cuda.synchronize()
        assert pipe.last_error() == 0
        # device time per iteration (host launch gaps included)
        self.iter_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(iters)]
        return [float(x) for x in torch.stack(losses).cpu()] if losses else []


def error_active_set(gmap: GaussianMap, cams, camt, targets, eps):
    """E_t of Section III-B2: Gaussians of `gmap` whose rendering error E_k(g)
    (Eq. 5) exceeds eps in some view.  Returns (bits, list, counts, count) on
    the device (count also on the host)."""
    g = gmap.gaussians()
    sizes = [(int(c["W"]), int(c["H"])) for c in cams]
    pipe = Pipeline(gmap.n, sizes, 1 << 20, colour=gmap.colour, sh_degree=gmap.sh_degree,
                    device=gmap.dev)
    D = pipe.ensure_capacity(g, camt)
    if D * 1.3 > pipe.capacity:
        pipe.alloc_capacity(int(D * 1.3) + 1024)
    pipe.forward(g, camt)
    pipe.loss_l1_err(targets)
    pipe.alloc_active()
    pipe.active.zero_()             # all inactive: the walk computes E_k only
    pipe.render_bwd_active(pipe.dL_drgb, error=True, masked=True)
    pipe.active_set(eps)
    torch.cuda.synchronize()
    return pipe.active.clone(), pipe.active_list.clone(), pipe.active_counts.clone(), \
        int(pipe.active_counts[0].item())


def mapping_update(global_map: GaussianMap, local: GaussianMap, window_cams, window_images,
                   past_cams, local_iters=30, global_iters=30, eps=0.0, adam=None,
                   masked_backward=False):
    """One local + global stage.  window_images: planar RGB of the window views
    (concatenated, device); past_cams: the poses whose renders of the map
    before insertion are the E_pc targets; eps: the error threshold of E_t;
    masked_backward: run the global stage's backward over the active set only
    (pose gradient through the active Gaussians).  Returns a report dict."""
    dev = global_map.dev
    rep = {}
    # ---- local stage: local map + window poses; the global map is rendered, frozen
    both = global_map.rows(0, global_map.n)
    first = both.append(local)
    n_all = both.n
    local_rows = torch.arange(first, n_all, dtype=torch.int32, device=dev)
    local_bits = _bits_of(n_all, first, n_all, dev)
    counts = torch.zeros(_abi.active_count_words(n_all), dtype=torch.int32, device=dev)
    counts[0] = n_all - first
    cam_w = camera_tensor(window_cams, dev)
    opt = MapOptimizer(both, adam)
    rep["local_losses"] = opt.iterate(window_cams, cam_w, window_images, local_iters,
                                      active=(local_bits, local_rows, counts))
    rep["local_iter_ms"] = opt.iter_ms
    local_opt = both.rows(first, n_all)
    del both

    # ---- global stage
    # E_pc targets: renders of the map before insertion at the past poses
    cam_p = camera_tensor(past_cams, dev)
    sizes_p = [(int(c["W"]), int(c["H"])) for c in past_cams]
    pp = Pipeline(global_map.n, sizes_p, 1 << 20, colour=global_map.colour,
                  sh_degree=global_map.sh_degree, device=dev)
    gm = global_map.gaussians()
    D = pp.ensure_capacity(gm, cam_p)
    if D * 1.3 > pp.capacity:
        pp.alloc_capacity(int(D * 1.3) + 1024)
    pp.forward(gm, cam_p)
    past_targets = pp.rgb.clone()
    del pp
    # E_t over the window on the map before insertion
    bits_e, _, _, n_e = error_active_set(global_map, window_cams, cam_w, window_images, eps)
    rep["error_active"] = n_e
    first = global_map.append(local_opt, opacity=INSERT_OPACITY)
    n_all = global_map.n
    bits = torch.zeros((n_all + 31) // 32, dtype=torch.int32, device=dev)
    bits[:bits_e.numel()] = bits_e
    force = _bits_of(n_all, first, n_all, dev)
    bits = torch.bitwise_or(bits, force)
    # list + count of A_t: E_t or inserted (the active-set call with no error rows)
    lst = torch.zeros(max(n_all, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(_abi.active_count_words(n_all), dtype=torch.int32, device=dev)
    none = torch.zeros(n_all, dtype=torch.float32, device=dev)
    abits = torch.zeros_like(bits)
    _abi.gevo_active_set(1, n_all, none, 1.0, bits, abits, lst, cnt)
    torch.cuda.synchronize()
    rep["active"] = int(cnt[0].item())
    cams_all = list(window_cams) + list(past_cams)
    camt_all = torch.cat([cam_w, cam_p]).contiguous()
    targets = torch.cat([window_images, past_targets]).contiguous()
    opt = MapOptimizer(global_map, adam)
    rep["global_losses"] = opt.iterate(cams_all, camt_all, targets, global_iters,
                                       fixed=[False] * len(window_cams) + [True] * len(past_cams),
                                       active=(abits, lst, cnt), masked=masked_backward)
    rep["global_iter_ms"] = opt.iter_ms
    # ---- pruning among the active set
    keep = torch.zeros_like(bits)
    klist = torch.zeros(max(n_all, 1), dtype=torch.int32, device=dev)
    kcnt = torch.zeros(_abi.active_count_words(n_all), dtype=torch.int32, device=dev)
    _abi.gevo_prune_keep(n_all, global_map.opacities, abits, PRUNE_OPACITY, keep, klist, kcnt)
    torch.cuda.synchronize()
    n_keep = int(kcnt[0].item())
    rep["pruned"] = n_all - n_keep
    global_map.compact(klist, kcnt, n_keep)
    rep["map_size"] = global_map.n
    rep["window_poses"] = camt_all[:len(window_cams)].cpu().numpy()
    return rep


def _bits_of(n, lo, hi, dev):
    """Bit mask with bits [lo, hi) set (host-built, one small copy)."""
    w = np.zeros((n + 31) // 32, np.uint64)
    idx = np.arange(lo, hi)
    np.add.at(w, idx // 32, np.uint64(1) << (idx % 32).astype(np.uint64))
    return torch.from_numpy(w.astype(np.uint32).view(np.int32)).to(dev)


def room_update(n=500_000, W=640, H=480, f=525.0, window=8, past=4, local_iters=30,
                global_iters=100, masked_backward=False, seed=5, eps=0.05):
    """One mapping update on the synthetic room: the map is the room without a
    box of it, the window (640x480 keyframes 0.15 m apart, 2.3 m from the box)
    observes the whole room, the local map is the box's Gaussians displaced by
    N(0, 3 cm) and recoloured (a noisy initialisation), the E_pc targets are
    four random past poses."""
    from . import prior_judge, scenes
    from .raster import gaussians_to_device
    w = scenes.workload(2, n=n)
    box = prior_judge.heldout_box()
    kept, n_out = prior_judge.split_scene(w["scene"], box)
    wins0, _, _ = prior_judge.window_poses(window, box, seed)
    wins = [scenes.camera(c["R"], c["t"], f, f, W / 2, H / 2, W, H) for c in wins0]
    pasts = [scenes.camera(c["R"], c["t"], f, f, W / 2, H / 2, W, H)
             for c in prior_judge.random_poses(past, seed + 1)]
    world = gaussians_to_device(w["scene"])
    pipe = Pipeline(n, [(W, H)] * window, 1 << 20, colour="sh", sh_degree=w["scene"]["sh_degree"])
    camt = camera_tensor(wins)
    D = pipe.ensure_capacity(world, camt)
    pipe.alloc_capacity(int(D * 1.3) + 1024)
    pipe.forward(world, camt)
    images = pipe.rgb.clone()
    del pipe, world
    inside = np.all((w["scene"]["means"] >= box[:, 0]) & (w["scene"]["means"] <= box[:, 1]), axis=1)
    rs = np.random.default_rng(seed)
    new = {k: (v[inside].copy() if isinstance(v, np.ndarray) else v) for k, v in w["scene"].items()}
    new["means"] = new["means"] + rs.normal(0, 0.03, size=new["means"].shape).astype(np.float32)
    new["sh"] = new["sh"] + rs.normal(0, 0.3, size=new["sh"].shape).astype(np.float32)
    new["opacities"] = np.full_like(new["opacities"], 0.9)
    gmap = GaussianMap(kept)
    local = GaussianMap(new)
    rep = mapping_update(gmap, local, wins, images, pasts, local_iters, global_iters, eps=eps,
                         masked_backward=masked_backward)
    rep.update(map_before=int(kept["means"].shape[0]), local=int(local.n), window=window, past=past,
               image=f"{W}x{H}")
    return rep


if __name__ == "__main__":
    import json
    import sys
    masked = "--masked" in sys.argv
    r = room_update(masked_backward=masked)
    r.pop("window_poses")
    med = lambda x: float(np.median(x)) if x else None
    r["local_iter_ms_median"] = med(r["local_iter_ms"][1:])
    r["global_iter_ms_median"] = med(r["global_iter_ms"][1:])
    r["masked_backward"] = masked
    print(json.dumps(r))
