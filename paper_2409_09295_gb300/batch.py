"""Batched keyframe replay: many views of uneven resolution rendered and
back-propagated together, captured into CUDA graphs, launch shapes autotuned.

GEVO replaces stored past keyframes by renders of the map (Section I; Section
III-B2): the consistency loss E_pc of Eq. 6 compares R(M'_t, T_kl) with the
stop-gradient render R(M_{t-1}, T_kl) over four past views, and the local stage
(Eq. 2) optimises over the sliding window.  `BatchedReplay` runs that forward +
L1 + backward over all views at once:
  - projection reads each Gaussian once and evaluates every view;
  - keys of all views share one global (view, tile) numbering, so one sort and
    one set of ranges serve every view;
  - blending and its reverse walk run as one persistent grid over (view, tile)
    work items, heaviest tile first;
  - the whole step is captured into one CUDA graph; replays need no host sync
    (the duplicate capacity is sized by one untimed pass plus slack, and an
    overflow is reported through the sticky error word);
  - `HostStep` wraps it for inputs and results in host memory: the uploads,
    the step and the read-back of loss, pose and parameter gradients are one
    graph too.
`PlainReplay` is the unbatched reference point: one single-view pipeline per
view, a host sync to size each sort, default launch shapes, no graph.
"""
from __future__ import annotations

import itertools

import torch

from . import _abi
from .raster import Pipeline, camera_tensor

# the autotuner's search, in two stages per direction: threads per tile x
# persistent grid; then, for a persistent best, the resident blocks per SM
# (0 = as many as the kernel's registers allow).  The staging batch stays a
# compile-time constant of each shape: as a launch parameter it cost the blend
# 16 registers and 13% of its time, and the compiled sizes measured best.
SHAPES = [dict(threads_per_tile=t, persistent=p, blocks_per_sm=0)
          for t, p in itertools.product((256, 128, 64, 32), (0, 1))]
BLOCKS_PER_SM = (2, 4, 8, 12, 16)
CANDIDATES = SHAPES   # first stage (kept under its old name)


def _time(fn, reps=3):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        s.record()
        fn()
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    return best


class BatchedReplay:
    def __init__(self, g: dict, cams, target_rgb, target_depth=None, lambda_depth=0.0,
                 bg=(0.0, 0.0, 0.0), slack=1.3, tuning_fwd=None, tuning_bwd=None,
                 want_dxi=True, autotune=True):
        self.g = g
        self.cams = cams
        self.sizes = [(int(c["W"]), int(c["H"])) for c in cams]
        self.camt = camera_tensor(cams, g["means"].device)
        self.target_rgb, self.target_depth = target_rgb, target_depth
        self.lambda_depth = float(lambda_depth)
        self.bg = bg
        self.want_dxi = want_dxi
        n = int(g["means"].shape[0])
        colour = "rgb" if "rgb" in g else "sh"
        self.pipe = Pipeline(n, self.sizes, 1 << 20, colour=colour,
                             sh_degree=g.get("sh_degree", 0), device=g["means"].device)
        D = self.pipe.ensure_capacity(g, self.camt, slack)
        if self.pipe.capacity < D * slack:
            self.pipe.alloc_capacity(int(D * slack) + 1024)
        self.n_dup = D
        self.tuning_fwd = tuning_fwd or dict(threads_per_tile=256, persistent=1, blocks_per_sm=0)
        self.tuning_bwd = tuning_bwd or dict(threads_per_tile=256, persistent=1, blocks_per_sm=0)
        self.tune_log = []
        if autotune and (tuning_fwd is None or tuning_bwd is None):
            self.autotune(fwd=tuning_fwd is None, bwd=tuning_bwd is None)
        self.graph = None
        self.stage_graphs = None
        self.bwd_graph = None

    # ---- stages with the chosen shapes ------------------------------------------------
    def _forward(self):
        self._project()
        self._bin_sort()
        self._render_fwd()
        self._loss()

    def _project(self):
        """The projection, zeroing the 2-D gradient rows the reverse walk will
        accumulate into (the visible entries') in the same pass."""
        self.pipe.project(self.g, self.camt, zero_grad2d=True)

    def _bin_sort(self):
        self.pipe.bin_sort()

    def _render_fwd(self):
        self.pipe.render_fwd(self.bg, tuning=self.tuning_fwd)

    def _loss(self):
        self.pipe.loss_l1(self.target_rgb, self.target_depth, self.lambda_depth)

    def _render_bwd(self):
        p = self.pipe
        p.render_bwd(p.dL_drgb, p.dL_ddepth if self.lambda_depth else None, None, self.bg,
                     tuning=self.tuning_bwd, zero=False)

    def _project_bwd(self):
        self.pipe.project_bwd(self.g, self.camt, self.want_dxi)

    def stages(self):
        """One step as six stages (one graph holds them all; the diagnostic
        mode captures each on its own to time it)."""
        return [("project", self._project), ("bin_sort", self._bin_sort),
                ("render_fwd", self._render_fwd), ("loss", self._loss),
                ("render_bwd", self._render_bwd), ("project_bwd", self._project_bwd)]

    def step_eager(self):
        """One step: the projection (which also zeroes the 2-D gradient rows of
        the visible entries), sort, blend, loss, reverse walk, projection
        backward."""
        for _, f in self.stages():
            f()

    # ---- autotuner ---------------------------------------------------------------------
    def _search(self, name, run, reps):
        """Staged search of one kernel's launch shape (see SHAPES and
        BLOCKS_PER_SM); returns the fastest tuning."""
        best = None

        def trial(c):
            nonlocal best
            t = _time(lambda: run(c), reps)
            self.tune_log.append((name, dict(c), t))
            if best is None or t < best[0]:
                best = (t, dict(c))
        for c in SHAPES:
            trial(c)
        if best[1]["persistent"]:
            base = dict(best[1])
            for k in BLOCKS_PER_SM:
                trial(dict(base, blocks_per_sm=k))
        return best[1]

    def autotune(self, fwd=True, bwd=True, reps=3):
        """Times candidate launch shapes of the blend and of its reverse walk on
        this workload (outputs do not depend on the shape) and keeps the fastest
        of each: threads per tile and persistent grid, then the resident blocks
        per SM of a persistent grid."""
        p = self.pipe
        self._forward()
        torch.cuda.synchronize()
        if fwd:
            self.tuning_fwd = self._search("render_fwd", lambda c: p.render_fwd(self.bg, tuning=c),
                                           reps)
            p.render_fwd(self.bg, tuning=self.tuning_fwd)
            p.loss_l1(self.target_rgb, self.target_depth, self.lambda_depth)
        if bwd:
            dd = p.dL_ddepth if self.lambda_depth else None
            self.tuning_bwd = self._search(
                "render_bwd", lambda c: p.render_bwd(p.dL_drgb, dd, None, self.bg, tuning=c,
                                                     zero=False), reps)
        torch.cuda.synchronize()

    # ---- graphs ------------------------------------------------------------------------
    def _warm(self):
        """Two eager steps on a side stream: buffers and launch attributes set up
        before any capture."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                self.step_eager()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()

    def capture(self):
        """Captures the whole step (projection, sort, blend, loss, reverse walk,
        projection backward) into one CUDA graph."""
        self._warm()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step_eager()
        torch.cuda.synchronize()

    def replay(self):
        """One step: one graph launch on the current stream, no host sync."""
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def capture_stages(self):
        """Diagnostic mode: each stage in a graph of its own, so that stages can
        be timed with events recorded between the launches."""
        self._warm()
        self.stage_graphs = []
        for name, f in self.stages():
            gph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gph):
                f()
            self.stage_graphs.append((name, gph))
        torch.cuda.synchronize()

    def replay_stages(self, events):
        """The step as its six stage graphs with events[0..6] recorded around
        them (len(stages) + 1 events) on the current stream."""
        if self.stage_graphs is None:
            self.capture_stages()
        events[0].record()
        for i, (_, gph) in enumerate(self.stage_graphs):
            gph.replay()
            events[i + 1].record()

    def replay_backward(self):
        """The backward alone, from whatever upstream gradients pipe.dL_drgb
        (and pipe.dL_ddepth) hold: record gradients zeroed, reverse walk,
        projection backward (one graph)."""
        if self.bwd_graph is None:
            # warm the three calls on a side stream (not whole steps: the loss
            # stage would overwrite the caller's upstream gradients)
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                self.pipe.grad2d_zero()
                self._render_bwd()
                self._project_bwd()
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            self.bwd_graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.bwd_graph):
                self.pipe.grad2d_zero()
                self._render_bwd()
                self._project_bwd()
            torch.cuda.synchronize()
        self.bwd_graph.replay()

    def eval_counts(self, blended=False):
        """(E_fwd, E_bwd): list entries examined by the blend (including skips and
        the stopping entry) and entries walked by the backward (sum of n_contrib);
        with blended=True also B, the entries blended."""
        p = self.pipe
        p.project(self.g, self.camt)
        p.bin_sort()
        nb = torch.zeros_like(p.n_eval)
        _abi.gevo_render_fwd_counts(p.layout, p.n, p.proj, p.vals, p.ranges, self.bg, p.rgb,
                                    p.depth, p.T_final, p.n_contrib, p.n_eval, nb, p.ws,
                                    self.tuning_fwd)
        torch.cuda.synchronize()
        out = (int(p.n_eval.sum(dtype=torch.int64)), int(p.n_contrib.sum(dtype=torch.int64)))
        return out + (int(nb.sum(dtype=torch.int64)),) if blended else out


class HostStep:
    """End-to-end step for a caller whose Gaussians, cameras and targets live in
    host memory: fill `host_in` (parameters and cameras) and `host_targets`
    (rendered target RGB and depth) -- pinned buffers owned by this object --
    call step(), synchronise, and read `host_out` (loss per view, dL/dxi per
    view, and the parameter gradients).

    One graph per step, its copies overlapped with the kernels: the cameras
    and the geometry parameters go up first, in CHUNKS pieces, each projected
    (the geometry part) as soon as it has landed; the colour parameters (the SH
    coefficients, most of the input bytes) follow and get their colour part
    beside the sort; the targets, first read by the loss, follow on another
    stream.  After the reverse walk the colour part of the projection backward
    runs piece by piece, and each piece's SH gradients go down while the next
    pieces and the geometry part run; then the loss, the pose gradients and the
    other parameter gradients.  The geometry part also zeroes the 2-D gradient
    rows of the visible entries, as in BatchedReplay.step_eager."""

    def __init__(self, rep: BatchedReplay):
        self.rep = rep
        p = rep.pipe
        keys = [k for k in ("means", "scales", "quats", "opacities", "sh", "rgb") if k in rep.g]
        self.host_in = {k: torch.empty(rep.g[k].shape, dtype=torch.float32).pin_memory()
                        for k in keys}
        self.host_in["cams"] = torch.empty(rep.camt.shape, dtype=torch.float32).pin_memory()
        self.host_targets = {"rgb": torch.empty(rep.target_rgb.shape).pin_memory()}
        if rep.target_depth is not None:
            self.host_targets["depth"] = torch.empty(rep.target_depth.shape).pin_memory()
        self.host_out = {"loss": torch.empty(p.loss.shape).pin_memory(),
                         "dxi": torch.empty(p.dxi.shape).pin_memory()}
        for k, v in p.grads.items():
            self.host_out[k] = torch.empty(v.shape).pin_memory()
        self.h2d_bytes = sum(t.numel() * 4 for t in self.host_in.values()) + \
            sum(t.numel() * 4 for t in self.host_targets.values())
        self.d2h_bytes = sum(t.numel() * 4 for t in self.host_out.values())
        for k, t in self.host_in.items():
            t.copy_(rep.camt if k == "cams" else rep.g[k])
        self.host_targets["rgb"].copy_(rep.target_rgb)
        if "depth" in self.host_targets:
            self.host_targets["depth"].copy_(rep.target_depth)
        self.graph = None

    CHUNKS = 4   # pieces of the map the uploads and the SH-gradient read-back move in

    def _chunks(self):
        """CHUNKS Gaussian ranges in whole PART_RANGE blocks (the backward's unit)."""
        n = self.rep.pipe.n
        step = -(-max(n, 1) // self.CHUNKS)
        step = -(-step // _abi.PART_RANGE) * _abi.PART_RANGE
        return [(b, min(n, b + step)) for b in range(0, n, step)]

    def _body(self):
        rep, p = self.rep, self.rep.pipe
        main = torch.cuda.current_stream()
        up, side2, down = self.side, self.side2, self.side3
        col = "sh" if "sh" in rep.g else "rgb"
        geo_keys = [k for k in self.host_in if k not in (col, "cams")]
        chunks = self._chunks()
        # the cameras and the geometry parameters go up first, in pieces; each
        # piece is projected (geometry part) as soon as it has landed
        up.wait_stream(main)
        ev_in = []
        with torch.cuda.stream(up):
            rep.camt.copy_(self.host_in["cams"], non_blocking=True)
            for b, e in chunks:
                for k in geo_keys:
                    rep.g[k][b:e].copy_(self.host_in[k][b:e], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(up)
                ev_in.append(ev)
            rep.g[col].copy_(self.host_in[col], non_blocking=True)
            ev_col_in = torch.cuda.Event()
            ev_col_in.record(up)
        for (b, e), ev in zip(chunks, ev_in):
            main.wait_event(ev)
            p.project(rep.g, rep.camt, part=_abi.PART_GEOMETRY, g_range=(b, e), zero_grad2d=True)
        ev_geo = torch.cuda.Event()
        ev_geo.record(main)
        with torch.cuda.stream(up):        # colours once they are in, beside the sort
            up.wait_event(ev_geo)
            p.project(rep.g, rep.camt, part=_abi.PART_COLOUR)
            ev_col = torch.cuda.Event()
            ev_col.record(up)
        side2.wait_event(ev_col_in)        # then the targets, first read by the loss
        with torch.cuda.stream(side2):
            rep.target_rgb.copy_(self.host_targets["rgb"], non_blocking=True)
            if "depth" in self.host_targets:
                rep.target_depth.copy_(self.host_targets["depth"], non_blocking=True)
        rep._bin_sort()
        main.wait_event(ev_col)
        rep._render_fwd()
        main.wait_stream(side2)
        rep._loss()
        rep._render_bwd()
        # the SH gradients of each piece go down as soon as its colour part has run
        for b, e in chunks:
            p.project_bwd(rep.g, rep.camt, rep.want_dxi, part=_abi.PART_COLOUR, g_range=(b, e))
            if col == "sh":
                down.wait_stream(main)
                with torch.cuda.stream(down):
                    self.host_out["sh"][b:e].copy_(p.grads["sh"][b:e], non_blocking=True)
        p.project_bwd(rep.g, rep.camt, rep.want_dxi, part=_abi.PART_GEOMETRY)
        self.host_out["loss"].copy_(p.loss, non_blocking=True)
        self.host_out["dxi"].copy_(p.dxi, non_blocking=True)
        for k, v in p.grads.items():
            if not (k == "sh" and col == "sh"):
                self.host_out[k].copy_(v, non_blocking=True)
        main.wait_stream(down)
        main.wait_stream(up)

    def capture(self):
        self.side = torch.cuda.Stream()
        self.side2 = torch.cuda.Stream()
        self.side3 = torch.cuda.Stream()
        self.rep._warm()
        for _ in range(2):
            self._body()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()
        torch.cuda.synchronize()

    def step(self):
        """Launches the step; host_out is valid after the current stream syncs."""
        if self.graph is None:
            self.capture()
        self.graph.replay()


class PlainReplay:
    """The unbatched path: one single-view pipeline per view, host-synchronised
    sizing of each sort, default launch shapes, no graph; gradients summed over
    views afterwards."""

    def __init__(self, g: dict, cams, target_rgb, target_depth=None, lambda_depth=0.0,
                 bg=(0.0, 0.0, 0.0), slack=1.3, want_dxi=True):
        self.g = g
        self.bg = bg
        self.lambda_depth = float(lambda_depth)
        self.want_dxi = want_dxi
        n = int(g["means"].shape[0])
        colour = "rgb" if "rgb" in g else "sh"
        dev = g["means"].device
        self.views = []
        base = 0
        for c in cams:
            W, H = int(c["W"]), int(c["H"])
            P = W * H
            pipe = Pipeline(n, [(W, H)], 1 << 20, colour=colour, sh_degree=g.get("sh_degree", 0),
                            device=dev)
            camt = camera_tensor([c], dev)
            D = pipe.ensure_capacity(g, camt, slack)
            tr = target_rgb[3 * base:3 * (base + P)]
            td = target_depth[base:base + P] if target_depth is not None else None
            self.views.append((pipe, camt, tr, td))
            base += P
        self.grads = {k: torch.zeros_like(v) for k, v in self.views[0][0].grads.items()}

    def step(self):
        for k in self.grads:
            self.grads[k].zero_()
        for pipe, camt, tr, td in self.views:
            pipe.project(self.g, camt)
            pipe.bin_sort()
            D = int(pipe.n_dup.item())            # host sync sizes the sort
            if D > pipe.capacity:
                pipe.last_error()
                pipe.alloc_capacity(int(D * 1.3) + 1024)
                pipe.bin_sort()
            pipe.render_fwd(self.bg)
            pipe.loss_l1(tr, td, self.lambda_depth)
            pipe.render_bwd(pipe.dL_drgb, pipe.dL_ddepth if self.lambda_depth else None, None,
                            self.bg)
            pipe.project_bwd(self.g, camt, self.want_dxi)
            for k in self.grads:
                self.grads[k].add_(pipe.grads[k])
