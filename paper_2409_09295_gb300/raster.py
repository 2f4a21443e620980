"""Buffers and call sequence of the rasterizer (stages a1-a8) on one GPU.

`Pipeline` owns the device buffers of one (Gaussian count, set of view sizes,
duplicate capacity) configuration and issues the C ABI calls in order on the
current stream; `GevoRasterize` puts the forward / backward pair behind
torch.autograd.  torch provides device memory and streams only: every stage of
the computation runs in libgevo's kernels.

Renders are the R(M, T) of GEVO's objectives (Section III-B): Eq. 2 (local
stage), Eq. 3 (global stage) and the rendered past keyframes of Eq. 6.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi as abi

DEFAULT_TUNING = {"threads_per_tile": 256, "persistent": 0, "blocks_per_sm": 0}


def camera_tensor(cams, device="cuda") -> torch.Tensor:
    """[V, 16] float32: R (row-major, world->camera), t, fx, fy, cx, cy."""
    rows = []
    for c in cams:
        r = np.zeros(16, np.float32)
        r[0:9] = np.asarray(c["R"], np.float32).reshape(9)
        r[9:12] = np.asarray(c["t"], np.float32)
        r[12:16] = [c["fx"], c["fy"], c["cx"], c["cy"]]
        rows.append(r)
    return torch.from_numpy(np.stack(rows)).to(device)


def gaussians_to_device(scene: dict, device="cuda") -> dict:
    g = {}
    for k in ("means", "scales", "quats", "opacities", "sh", "rgb"):
        if scene.get(k) is not None:
            g[k] = torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(device)
    g["sh_degree"] = int(scene.get("sh_degree", 0))
    return g


class Pipeline:
    """Device buffers + the stage calls for one configuration.

    sizes: list of (W, H) per view.  colour: "rgb" or "sh" (with sh_degree).
    dup_capacity: (Gaussian, tile) pairs the sort may hold.  keep_keys: also
    write the sorted 64-bit keys (the renderers read only the ids and ranges)."""

    def __init__(self, n: int, sizes, dup_capacity: int, colour: str = "rgb", sh_degree: int = 0,
                 device="cuda", tuning=None, keep_keys: bool = False):
        self.n = int(n)
        self.keep_keys = bool(keep_keys)
        self.sizes = [(int(w), int(h)) for w, h in sizes]
        self.V = len(self.sizes)
        self.device = torch.device(device)
        self.colour = colour
        self.sh_degree = int(sh_degree)
        self.tuning = dict(DEFAULT_TUNING if tuning is None else tuning)
        self.layout = abi.gevo_layout_init([s[0] for s in self.sizes], [s[1] for s in self.sizes])
        self.T = int(self.layout.total_tiles)
        self.P = int(self.layout.total_pixels)
        self.pix_base = [int(self.layout.pix_base[v]) for v in range(self.V + 1)]
        self.alloc_capacity(dup_capacity)
        dev, f32, i32 = self.device, torch.float32, torch.int32
        VN = max(self.V * self.n, 1)
        self.proj = dict(xy=torch.zeros(VN, 2, dtype=f32, device=dev),
                         conic_opacity=torch.zeros(VN, 4, dtype=f32, device=dev),
                         rgb_depth=torch.zeros(VN, 4, dtype=f32, device=dev),
                         radius=torch.zeros(VN, dtype=i32, device=dev),
                         tiles_touched=torch.zeros(VN, dtype=i32, device=dev))
        self.ranges = torch.zeros(self.T, 2, dtype=i32, device=dev)
        self.n_dup = torch.zeros(1, dtype=torch.int64, device=dev)
        self.rgb = torch.zeros(3 * self.P, dtype=f32, device=dev)
        self.depth = torch.zeros(self.P, dtype=f32, device=dev)
        self.T_final = torch.zeros(self.P, dtype=f32, device=dev)
        self.n_contrib = torch.zeros(self.P, dtype=i32, device=dev)
        self.n_eval = torch.zeros(self.P, dtype=i32, device=dev)
        self.grad2d = dict(xy=torch.zeros(VN, 2, dtype=f32, device=dev),
                           conic_opacity=torch.zeros(VN, 4, dtype=f32, device=dev),
                           rgb_depth=torch.zeros(VN, 4, dtype=f32, device=dev))
        self.dL_drgb = torch.zeros(3 * self.P, dtype=f32, device=dev)
        self.dL_ddepth = torch.zeros(self.P, dtype=f32, device=dev)
        self.loss = torch.zeros(self.V, dtype=f32, device=dev)
        self.dxi = torch.zeros(self.V, 6, dtype=f32, device=dev)
        K = (self.sh_degree + 1) ** 2
        n1 = max(self.n, 1)
        self.grads = dict(means=torch.zeros(n1, 3, dtype=f32, device=dev),
                          scales=torch.zeros(n1, 3, dtype=f32, device=dev),
                          quats=torch.zeros(n1, 4, dtype=f32, device=dev),
                          opacities=torch.zeros(n1, dtype=f32, device=dev))
        if colour == "rgb":
            self.grads["rgb"] = torch.zeros(n1, 3, dtype=f32, device=dev)
        else:
            self.grads["sh"] = torch.zeros(n1, K, 3, dtype=f32, device=dev)

    def alloc_capacity(self, dup_capacity: int):
        self.capacity = max(int(dup_capacity), 1)
        nbytes = abi.gevo_workspace_bytes(self.layout, self.n, self.capacity)
        self.ws = torch.zeros(nbytes, dtype=torch.uint8, device=self.device)
        self.keys = (torch.zeros(self.capacity, dtype=torch.int64, device=self.device)
                     if self.keep_keys else None)
        self.vals = torch.zeros(self.capacity, dtype=torch.int32, device=self.device)

    # ---- per-view views of the planar outputs -------------------------------------------
    def view_rgb(self, buf, v):
        W, H = self.sizes[v]
        return buf[3 * self.pix_base[v]:3 * self.pix_base[v + 1]].view(3, H, W)

    def view_plane(self, buf, v):
        W, H = self.sizes[v]
        return buf[self.pix_base[v]:self.pix_base[v + 1]].view(H, W)

    # ---- stages ----------------------------------------------------------------------
    def project(self, g, cams, part=None, g_range=None, zero_grad2d=False):
        """The projection; part = abi.PART_GEOMETRY or abi.PART_COLOUR runs one
        of its two parts (geometry first), over g_range = (begin, end) if given.
        zero_grad2d: also zero the 2-D gradient rows of the visible entries (all
        or geometry part), in place of grad2d_zero."""
        if zero_grad2d:
            b, e = g_range if g_range is not None else (0, None)
            abi.gevo_project_zero(self.layout, g, cams, self.proj, self.grad2d,
                                  abi.PART_ALL if part is None else part, self.ws, g_begin=b,
                                  g_end=e)
        elif part is None and g_range is None:
            abi.gevo_project(self.layout, g, cams, self.proj, self.ws)
        else:
            b, e = g_range if g_range is not None else (0, None)
            abi.gevo_project_part(self.layout, g, cams, self.proj,
                                  abi.PART_ALL if part is None else part, self.ws, g_begin=b, g_end=e)

    def bin_sort(self):
        abi.gevo_bin_sort(self.layout, self.n, self.proj, self.capacity, self.keys, self.vals,
                          self.ranges, self.n_dup, self.ws)

    def render_fwd(self, bg=(0.0, 0.0, 0.0), n_eval=False, tuning=None):
        abi.gevo_render_fwd(self.layout, self.n, self.proj, self.vals, self.ranges, bg, self.rgb,
                            self.depth, self.T_final, self.n_contrib,
                            self.n_eval if n_eval else None, self.ws,
                            tuning or self.tuning)

    def loss_l1(self, target_rgb, target_depth=None, lambda_depth=0.0):
        abi.gevo_loss_l1(self.layout, self.rgb, target_rgb,
                         self.depth if lambda_depth else None,
                         target_depth if lambda_depth else None, lambda_depth, self.dL_drgb,
                         self.dL_ddepth if lambda_depth else None, self.loss, self.ws)

    def grad2d_zero(self):
        abi.gevo_grad2d_zero(self.layout, self.n, self.proj, self.grad2d)

    def render_bwd(self, dL_drgb, dL_ddepth=None, dL_dT=None, bg=(0.0, 0.0, 0.0), tuning=None,
                   zero=True):
        """Record gradients; zero=False accumulates into the existing rows."""
        if zero:
            self.grad2d_zero()
        abi.gevo_render_bwd(self.layout, self.n, self.proj, self.vals, self.ranges, bg,
                            self.T_final, self.n_contrib, dL_drgb, dL_ddepth, dL_dT, self.grad2d,
                            self.ws, tuning or self.tuning)

    def project_bwd(self, g, cams, want_dxi=True, part=None, g_range=None):
        """The projection derivative; part = abi.PART_COLOUR then
        abi.PART_GEOMETRY runs it in two parts (the SH gradients final after
        the first), over g_range = (begin, end) in whole abi.PART_RANGE blocks
        if given (colour ranges in order from 0, before the geometry ones)."""
        dxi = self.dxi if want_dxi else None
        if part is None and g_range is None:
            abi.gevo_project_bwd(self.layout, g, cams, self.proj, self.grad2d, self.grads, dxi,
                                 self.ws)
        else:
            b, e = g_range if g_range is not None else (0, None)
            abi.gevo_project_bwd_part(self.layout, g, cams, self.proj, self.grad2d, self.grads,
                                      dxi, abi.PART_ALL if part is None else part, self.ws,
                                      g_begin=b, g_end=e)

    # ---- active set of the global stage (Section III-B2, Eq. 5) --------------------
    def alloc_active(self):
        """Buffers of the active-set path (allocated on first use)."""
        if getattr(self, "pix_err", None) is not None:
            return
        dev, f32, u32 = self.device, torch.float32, torch.int32
        self.pix_err = torch.zeros(self.P, dtype=f32, device=dev)
        self.gauss_err = torch.zeros(max(self.V * self.n, 1), dtype=f32, device=dev)
        nw = max((self.n + 31) // 32, 1)
        self.active = torch.zeros(nw, dtype=u32, device=dev)
        self.active_list = torch.zeros(max(self.n, 1), dtype=u32, device=dev)
        self.active_counts = torch.zeros(abi.active_count_words(self.n), dtype=u32, device=dev)
        self.act_state = dict(last=torch.zeros(self.P, dtype=u32, device=dev),
                              T=torch.ones(self.P, dtype=f32, device=dev),
                              rest=torch.zeros(self.P, 4, dtype=f32, device=dev))

    def loss_l1_err(self, target_rgb, target_depth=None, lambda_depth=0.0):
        """loss_l1 that also writes the per-pixel error e(u) into self.pix_err."""
        self.alloc_active()
        abi.gevo_loss_l1_err(self.layout, self.rgb, target_rgb,
                             self.depth if lambda_depth else None,
                             target_depth if lambda_depth else None, lambda_depth, self.dL_drgb,
                             self.dL_ddepth if lambda_depth else None, self.loss, self.pix_err,
                             self.ws)

    def render_fwd_active(self, bg=(0.0, 0.0, 0.0), tuning=None):
        """render_fwd that also records where an active-set reverse walk starts
        (self.act_state), for the mask in self.active."""
        self.alloc_active()
        abi.gevo_render_fwd_active(self.layout, self.n, self.proj, self.vals, self.ranges, bg,
                                   self.rgb, self.depth, self.T_final, self.n_contrib, self.active,
                                   self.act_state, self.ws, tuning or self.tuning)

    def render_bwd_active(self, dL_drgb, dL_ddepth=None, dL_dT=None, bg=(0.0, 0.0, 0.0),
                          error=True, masked=True, tuning=None, zero=True, from_state=False):
        """Reverse walk that accumulates E_k(g) into self.gauss_err (error=True;
        cleared first) and/or writes only the rows of active Gaussians
        (masked=True, using self.active); from_state=True starts each pixel at
        its last active entry (after render_fwd_active; needs masked, not error)."""
        self.alloc_active()
        if zero:
            self.grad2d_zero()
        if error:
            self.gauss_err.zero_()
        abi.gevo_render_bwd_active(self.layout, self.n, self.proj, self.vals, self.ranges, bg,
                                   self.T_final, self.n_contrib, dL_drgb, dL_ddepth, dL_dT,
                                   self.pix_err if error else None,
                                   self.gauss_err if error else None,
                                   self.active if masked else None, self.grad2d, self.ws,
                                   tuning or self.tuning,
                                   state=self.act_state if from_state else None)

    def active_set(self, eps, force=None):
        """Active mask, list and count from self.gauss_err (Eq. 5 threshold eps),
        or-ed with the bit mask `force` (the newly inserted Gaussians)."""
        self.alloc_active()
        abi.gevo_active_set(self.V, self.n, self.gauss_err, eps, force, self.active,
                            self.active_list, self.active_counts)

    def project_bwd_active(self, g, cams, want_dxi=True):
        abi.gevo_project_bwd_active(self.layout, g, cams, self.proj, self.grad2d,
                                    self.active_list, self.active_counts, self.grads,
                                    self.dxi if want_dxi else None, self.ws)

    # ---- composites ------------------------------------------------------------------
    def forward(self, g, cams, bg=(0.0, 0.0, 0.0), n_eval=False):
        self.project(g, cams)
        self.bin_sort()
        self.render_fwd(bg, n_eval)

    def step(self, g, cams, target_rgb, target_depth=None, lambda_depth=0.0,
             bg=(0.0, 0.0, 0.0), want_dxi=True):
        """One forward + L1 loss + backward pass over every view (no host sync)."""
        self.forward(g, cams, bg)
        self.loss_l1(target_rgb, target_depth, lambda_depth)
        self.render_bwd(self.dL_drgb, self.dL_ddepth if lambda_depth else None, None, bg)
        self.project_bwd(g, cams, want_dxi)

    def last_error(self) -> int:
        return abi.gevo_last_error(self.ws)

    # ---- what a backward pass reads from its forward --------------------------------
    def save_state(self) -> dict:
        """Copies of the buffers the reverse walk and the projection backward read
        from the forward pass: projection records, sorted values, tile ranges,
        T_final and n_contrib (alpha is not kept: the walk recomputes it).  The
        pipeline's own buffers stay where they are (captured graphs keep their
        addresses); a later forward overwrites them, not the copies."""
        return dict(proj={k: v.clone() for k, v in self.proj.items()}, vals=self.vals.clone(),
                    ranges=self.ranges.clone(), T_final=self.T_final.clone(),
                    n_contrib=self.n_contrib.clone())

    def swap_state(self, state: dict) -> dict:
        """Installs saved forward buffers and returns the ones they replace."""
        old = {k: getattr(self, k) for k in state}
        for k, v in state.items():
            setattr(self, k, v)
        return old

    def ensure_capacity(self, g, cams, slack=1.25):
        """Host-synchronising sizing pass: project + count, then grow the duplicate
        capacity if needed.  Returns the duplicate count D."""
        self.project(g, cams)
        self.bin_sort()
        D = int(self.n_dup.item())
        if D > self.capacity:
            abi.gevo_last_error(self.ws)
            self.alloc_capacity(int(D * slack) + 1024)
        return D


class GevoRasterize(torch.autograd.Function):
    """(means, scales, quats, opacities, colours, twist) -> (rgb, depth, T_final).

    colours: rgb [N,3] or SH [N,K,3] (as the pipeline was built).  twist: [V,6]
    zeros standing for a left se(3) perturbation of each view's pose; its
    gradient is dL/dxi.  Outputs are the planar view-major buffers described in
    include/gevo.h (use Pipeline.view_rgb / view_plane to slice views).

    Each call keeps its own copy of what the backward reads (projection records,
    sorted values, ranges, T_final and n_contrib; not alpha, which the backward
    recomputes), so several forwards through one pipeline may precede their
    backwards: E_pc of Eq. 6 renders the current and the past views before one
    backward.  The inputs are saved for backward, so modifying them in place
    before the backward raises torch's usual error."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, colours, twist, pipe, cams, bg):
        g = dict(means=means.detach().contiguous(), scales=scales.detach().contiguous(),
                 quats=quats.detach().contiguous(), opacities=opacities.detach().contiguous(),
                 sh_degree=pipe.sh_degree)
        g["rgb" if pipe.colour == "rgb" else "sh"] = colours.detach().contiguous()
        pipe.forward(g, cams, bg)
        ctx.save_for_backward(means, scales, quats, opacities, colours)
        ctx.pipe, ctx.g, ctx.cams, ctx.bg = pipe, g, cams.clone(), bg
        ctx.state = pipe.save_state()
        return pipe.rgb.clone(), pipe.depth.clone(), pipe.T_final.clone()

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_T):
        ctx.saved_tensors   # raises if an input was modified in place since the forward
        pipe = ctx.pipe
        z = lambda t, like: (t.contiguous() if t is not None else torch.zeros_like(like))
        keep = pipe.swap_state(ctx.state)
        try:
            pipe.render_bwd(z(g_rgb, pipe.rgb), z(g_depth, pipe.depth),
                            g_T.contiguous() if g_T is not None else None, ctx.bg)
            pipe.project_bwd(ctx.g, ctx.cams, want_dxi=True)
        finally:
            pipe.swap_state(keep)
        ctx.state = None
        gr = pipe.grads
        col = gr["rgb"] if pipe.colour == "rgb" else gr["sh"]
        return (gr["means"].clone(), gr["scales"].clone(), gr["quats"].clone(),
                gr["opacities"].clone(), col.clone(), pipe.dxi.clone(), None, None, None)


def rasterize(pipe: Pipeline, means, scales, quats, opacities, colours, cams, twist=None,
              bg=(0.0, 0.0, 0.0)):
    if twist is None:
        twist = torch.zeros(pipe.V, 6, device=means.device, requires_grad=False)
    return GevoRasterize.apply(means, scales, quats, opacities, colours, twist, pipe, cams, bg)
