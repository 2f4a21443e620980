"""ctypes binding of libgevo.so (include/gevo.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing
but turn torch tensors into device pointers and the current CUDA stream into a
handle; all arithmetic runs in the library's kernels.  If the library cannot be
loaded the import fails loudly -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MAX_VIEWS = 64
TILE = 16

STATUS = {0: "ok", 1: "invalid argument", 2: "duplicate capacity exceeded", 3: "CUDA error",
          4: "device wait timed out", 5: "non-finite value culled",
          6: "size exceeds the fixed no-allocation scratch"}


class GevoError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class Layout(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("total_tiles", ctypes.c_int32),
                ("total_pixels", ctypes.c_int64),
                ("width", ctypes.c_int32 * MAX_VIEWS), ("height", ctypes.c_int32 * MAX_VIEWS),
                ("tiles_x", ctypes.c_int32 * MAX_VIEWS), ("tiles_y", ctypes.c_int32 * MAX_VIEWS),
                ("tile_base", ctypes.c_int32 * (MAX_VIEWS + 1)),
                ("pix_base", ctypes.c_int64 * (MAX_VIEWS + 1))]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacities", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32)]


class GaussianGrads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacities", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("rgb", ctypes.c_void_p)]


class Proj(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("conic_opacity", ctypes.c_void_p),
                ("rgb_depth", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("tiles_touched", ctypes.c_void_p)]


class Grad2d(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("conic_opacity", ctypes.c_void_p),
                ("rgb_depth", ctypes.c_void_p)]


class ActiveState(ctypes.Structure):
    _fields_ = [("last", ctypes.c_void_p), ("T", ctypes.c_void_p), ("rest", ctypes.c_void_p)]


class MapParams(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("logit_opacities", ctypes.c_void_p),
                ("colours", ctypes.c_void_p)]


class MapAdam(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in (
        "lr_means", "lr_log_scales", "lr_quats", "lr_logit_opacities", "lr_colour_dc",
        "lr_colour_rest", "beta1", "beta2", "eps", "lambda_iso")]


class Tuning(ctypes.Structure):
    _fields_ = [("threads_per_tile", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32)]


# Every symbol include/gevo.h declares (checked by the CPU test-suite).
EXPORTS = ["gevo_layout_init", "gevo_workspace_bytes", "gevo_project", "gevo_bin_sort",
           "gevo_render_fwd", "gevo_render_bwd", "gevo_project_bwd", "gevo_loss_l1",
           "gevo_last_error", "gevo_status_str", "gevo_version", "gevo_bin_sort_noalloc",
           "gevo_grad2d_zero", "gevo_gemm_bf16", "gevo_loss_l1_err", "gevo_render_bwd_active",
           "gevo_active_set", "gevo_project_bwd_active", "gevo_render_fwd_active",
           "gevo_render_fwd_counts", "gevo_bin_sort_launches", "gevo_project_part",
           "gevo_project_bwd_part", "gevo_project_zero"]

# Parts of gevo_project_part / gevo_project_bwd_part and the backward's range
# unit (include/gevo.h).
PART_ALL, PART_GEOMETRY, PART_COLOUR = 0, 1, 2
PART_RANGE = 1024

# Every symbol include/gevo_prior.h declares, with its argument kinds
# (i: int32, u: uint32, I: int64, f: float, p: pointer; the last p is the stream).
PRIOR = {
    "gevo_conv3x3": "iiiipipppiiifpp",
    "gevo_conv3x3_wgrad": "iiiipipppp",
    "gevo_relu_bwd": "Iipipipppp",
    "gevo_maxpool2": "iiiipipp",
    "gevo_maxpool2_bwd": "iiiipippifp",
    "gevo_upsample2": "iiiippip",
    "gevo_upsample2_bwd": "iiiipipp",
    "gevo_flip3x3": "iippp",
    "gevo_rgb_pack": "iiippp",
    "gevo_head_fwd": "Iippppp",
    "gevo_head_bwd": "Iippppppp",
    "gevo_depth_target": "Ippppp",
    "gevo_depth_l1": "Ipppppp",
    "gevo_adam": "Ipppppffffip",
    "gevo_cost_volume": "iiiippiffpppp",
    "gevo_unproject": "iippppuuffipipppppp",
    "gevo_depth_bp": "iiipffiffppppp",
    "gevo_to_bf16": "Ippp",
}
EXPORTS = EXPORTS + list(PRIOR)

# Every symbol include/gevo_map.h declares.
MAP = ["gevo_map_activate", "gevo_map_step", "gevo_pose_step", "gevo_prune_keep",
       "gevo_gather_rows"]
EXPORTS = EXPORTS + MAP

# Every symbol include/gevo_bench.h declares (exported by libgevo_probes.so,
# the measurement-only library, not by libgevo).
BENCH = ["gevo_bench_fma", "gevo_bench_ex2", "gevo_bench_fma2", "gevo_bench_rcp"]

_lib = None
_probes = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgevo.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise OSError(f"{path} is missing: run paper_2409_09295_gb300/build.py")
        _build.build()
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, u64, f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_float)
    L.gevo_layout_init.argtypes = [P(Layout), i32, P(i32), P(i32)]
    L.gevo_layout_init.restype = ctypes.c_int
    L.gevo_workspace_bytes.argtypes = [P(Layout), i32, u64]
    L.gevo_workspace_bytes.restype = ctypes.c_size_t
    L.gevo_project.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), vp, vp]
    L.gevo_project_part.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), i32, i32, i32, vp, vp]
    L.gevo_project_zero.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), P(Grad2d), i32, i32, i32,
                                    vp, vp]
    L.gevo_bin_sort.argtypes = [P(Layout), i32, P(Proj), u64, vp, vp, vp, vp, vp, vp]
    L.gevo_bin_sort_launches.argtypes = [P(Layout), i32, u64]
    L.gevo_bin_sort_launches.restype = i32
    L.gevo_bin_sort_noalloc.argtypes = [P(Layout), i32, P(Proj), u64, vp, vp, vp, vp, vp]
    L.gevo_bin_sort_noalloc.restype = ctypes.c_int
    L.gevo_render_fwd.argtypes = [P(Layout), i32, P(Proj), vp, vp, P(f32), vp, vp, vp, vp, vp,
                                  P(Tuning), vp, vp]
    L.gevo_render_bwd.argtypes = [P(Layout), i32, P(Proj), vp, vp, P(f32), vp, vp, vp, vp, vp,
                                  P(Grad2d), P(Tuning), vp, vp]
    L.gevo_gemm_bf16.argtypes = [i32, i32, i32, vp, i32, vp, i32, vp, i32, i32, vp, i32, f32, vp, vp]
    L.gevo_gemm_bf16.restype = ctypes.c_int
    L.gevo_grad2d_zero.argtypes = [P(Layout), i32, P(Proj), P(Grad2d), vp]
    L.gevo_grad2d_zero.restype = ctypes.c_int
    L.gevo_project_bwd.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), P(Grad2d),
                                   P(GaussianGrads), vp, vp, vp]
    L.gevo_project_bwd_part.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), P(Grad2d),
                                        P(GaussianGrads), vp, i32, i32, i32, vp, vp]
    L.gevo_loss_l1.argtypes = [P(Layout), vp, vp, vp, vp, f32, vp, vp, vp, vp, vp]
    L.gevo_loss_l1_err.argtypes = [P(Layout), vp, vp, vp, vp, f32, vp, vp, vp, vp, vp, vp]
    L.gevo_render_bwd_active.argtypes = [P(Layout), i32, P(Proj), vp, vp, P(f32), vp, vp, vp, vp,
                                         vp, vp, vp, vp, P(ActiveState), P(Grad2d), P(Tuning), vp,
                                         vp]
    L.gevo_render_fwd_counts.argtypes = [P(Layout), i32, P(Proj), vp, vp, P(f32), vp, vp, vp, vp,
                                         vp, vp, P(Tuning), vp, vp]
    L.gevo_render_fwd_active.argtypes = [P(Layout), i32, P(Proj), vp, vp, P(f32), vp, vp, vp, vp,
                                         vp, P(ActiveState), P(Tuning), vp, vp]
    L.gevo_active_set.argtypes = [i32, i32, vp, f32, vp, vp, vp, vp, vp]
    L.gevo_project_bwd_active.argtypes = [P(Layout), P(Gaussians), vp, P(Proj), P(Grad2d), vp, vp,
                                          P(GaussianGrads), vp, vp, vp]
    L.gevo_last_error.argtypes = [vp, vp]
    L.gevo_map_activate.argtypes = [i32, vp, vp, vp, vp, vp]
    L.gevo_map_step.argtypes = [i32, i32, P(MapParams), P(GaussianGrads), P(MapParams),
                                P(MapParams), P(MapAdam), i32, vp, vp, vp, vp, vp, vp]
    L.gevo_pose_step.argtypes = [i32, vp, vp, vp, vp, f32, f32, f32, f32, f32, i32, vp, vp]
    L.gevo_prune_keep.argtypes = [i32, vp, vp, f32, vp, vp, vp, vp]
    L.gevo_gather_rows.argtypes = [i32, vp, vp, i32, vp, vp, vp]
    for name in MAP:
        getattr(L, name).restype = ctypes.c_int
    L.gevo_status_str.argtypes = [ctypes.c_int]
    L.gevo_status_str.restype = ctypes.c_char_p
    L.gevo_version.restype = i32
    kinds = {"i": ctypes.c_int32, "u": ctypes.c_uint32, "I": ctypes.c_int64, "f": ctypes.c_float,
             "p": vp}
    for name, sig in PRIOR.items():
        getattr(L, name).argtypes = [kinds[c] for c in sig]
        getattr(L, name).restype = ctypes.c_int
    for name in ("gevo_project", "gevo_bin_sort", "gevo_render_fwd", "gevo_render_bwd",
                 "gevo_project_bwd", "gevo_loss_l1", "gevo_last_error", "gevo_loss_l1_err",
                 "gevo_render_bwd_active", "gevo_active_set", "gevo_project_bwd_active",
                 "gevo_render_fwd_active", "gevo_render_fwd_counts"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _p(t):
    """Device pointer of a tensor (None -> NULL)."""
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(fn, code):
    if code != 0:
        raise GevoError(fn, code)


# ---------------------------------------------------------------------------
# Host-side set-up
# ---------------------------------------------------------------------------
def gevo_layout_init(widths, heights) -> Layout:
    L = Layout()
    V = len(widths)
    W = (ctypes.c_int32 * V)(*[int(w) for w in widths])
    H = (ctypes.c_int32 * V)(*[int(h) for h in heights])
    _check("gevo_layout_init", load().gevo_layout_init(ctypes.byref(L), V, W, H))
    return L


def gevo_workspace_bytes(layout: Layout, n: int, dup_capacity: int) -> int:
    return int(load().gevo_workspace_bytes(ctypes.byref(layout), int(n), int(dup_capacity)))


def gevo_bin_sort_launches(layout: Layout, n: int, dup_capacity: int) -> int:
    """Kernels gevo_bin_sort launches for these sizes (-1: invalid arguments)."""
    return int(load().gevo_bin_sort_launches(ctypes.byref(layout), int(n), int(dup_capacity)))


def gaussians_struct(g: dict) -> Gaussians:
    s = Gaussians()
    s.means, s.scales, s.quats, s.opacities = (_p(g["means"]), _p(g["scales"]), _p(g["quats"]),
                                              _p(g["opacities"]))
    s.sh = _p(g.get("sh"))
    s.rgb = _p(g.get("rgb"))
    s.n = int(g["means"].shape[0])
    s.sh_degree = int(g.get("sh_degree", 0))
    return s


def proj_struct(p: dict) -> Proj:
    s = Proj()
    s.xy, s.conic_opacity, s.rgb_depth, s.radius, s.tiles_touched = (
        _p(p["xy"]), _p(p["conic_opacity"]), _p(p["rgb_depth"]), _p(p["radius"]),
        _p(p["tiles_touched"]))
    return s


def grad2d_struct(g: dict) -> Grad2d:
    s = Grad2d()
    s.xy, s.conic_opacity, s.rgb_depth = _p(g["xy"]), _p(g["conic_opacity"]), _p(g["rgb_depth"])
    return s


def tuning_struct(t) -> Tuning | None:
    if t is None:
        return None
    s = Tuning()
    s.threads_per_tile = int(t.get("threads_per_tile", 256))
    s.persistent = int(t.get("persistent", 0))
    s.blocks_per_sm = int(t.get("blocks_per_sm", 0))
    return s


# ---------------------------------------------------------------------------
# The entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def gevo_project(layout, g: dict, cams: torch.Tensor, proj: dict, ws: torch.Tensor, stream=None):
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    _check("gevo_project", load().gevo_project(ctypes.byref(layout), ctypes.byref(G), _p(cams),
                                               ctypes.byref(P_), _p(ws), _stream(stream)))


def gevo_project_part(layout, g: dict, cams: torch.Tensor, proj: dict, part: int,
                      ws: torch.Tensor, stream=None, g_begin=0, g_end=None):
    """One part (PART_GEOMETRY or PART_COLOUR) of gevo_project, over the
    Gaussians g_begin <= g < g_end (default: all)."""
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    _check("gevo_project_part", load().gevo_project_part(
        ctypes.byref(layout), ctypes.byref(G), _p(cams), ctypes.byref(P_), int(part), int(g_begin),
        int(G.n if g_end is None else g_end), _p(ws), _stream(stream)))


def gevo_bin_sort(layout, n, proj: dict, dup_capacity, keys, vals, ranges, d_n_dup, ws,
                  stream=None):
    P_ = proj_struct(proj)
    _check("gevo_bin_sort", load().gevo_bin_sort(
        ctypes.byref(layout), int(n), ctypes.byref(P_), int(dup_capacity), _p(keys), _p(vals),
        _p(ranges), _p(d_n_dup), _p(ws), _stream(stream)))


def gevo_bin_sort_noalloc(layout, n, proj: dict, dup_capacity, keys, vals, ranges, d_n_dup,
                          stream=None):
    """gevo_bin_sort without a workspace: for callers that cannot allocate device
    memory; its scratch is a fixed static device array (see include/gevo.h)."""
    P_ = proj_struct(proj)
    _check("gevo_bin_sort_noalloc", load().gevo_bin_sort_noalloc(
        ctypes.byref(layout), int(n), ctypes.byref(P_), int(dup_capacity), _p(keys), _p(vals),
        _p(ranges), _p(d_n_dup), _stream(stream)))


def gevo_render_fwd(layout, n, proj: dict, vals, ranges, bg, rgb, depth, T_final, n_contrib,
                    n_eval, ws, tuning=None, stream=None):
    P_ = proj_struct(proj)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    tu = tuning_struct(tuning)
    _check("gevo_render_fwd", load().gevo_render_fwd(
        ctypes.byref(layout), int(n), ctypes.byref(P_), _p(vals), _p(ranges), bgv, _p(rgb),
        _p(depth), _p(T_final), _p(n_contrib), _p(n_eval),
        ctypes.byref(tu) if tu is not None else None, _p(ws), _stream(stream)))


def gevo_render_bwd(layout, n, proj: dict, vals, ranges, bg, T_final, n_contrib, dL_drgb,
                    dL_ddepth, dL_dT, grad2d: dict, ws, tuning=None, stream=None):
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    tu = tuning_struct(tuning)
    _check("gevo_render_bwd", load().gevo_render_bwd(
        ctypes.byref(layout), int(n), ctypes.byref(P_), _p(vals), _p(ranges), bgv, _p(T_final),
        _p(n_contrib), _p(dL_drgb), _p(dL_ddepth), _p(dL_dT), ctypes.byref(G2),
        ctypes.byref(tu) if tu is not None else None, _p(ws), _stream(stream)))


def active_state_struct(state):
    """dict(last, T, rest) of device tensors -> gevo_active_state (None -> None)."""
    if state is None:
        return None
    return ActiveState(_p(state["last"]), _p(state["T"]), _p(state["rest"]))


def gevo_render_fwd_counts(layout, n, proj: dict, vals, ranges, bg, rgb, depth, T_final,
                           n_contrib, n_eval, n_blend, ws, tuning=None, stream=None):
    P_ = proj_struct(proj)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    tu = tuning_struct(tuning)
    _check("gevo_render_fwd_counts", load().gevo_render_fwd_counts(
        ctypes.byref(layout), int(n), ctypes.byref(P_), _p(vals), _p(ranges), bgv, _p(rgb),
        _p(depth), _p(T_final), _p(n_contrib), _p(n_eval), _p(n_blend),
        ctypes.byref(tu) if tu is not None else None, _p(ws), _stream(stream)))


def gevo_render_fwd_active(layout, n, proj: dict, vals, ranges, bg, rgb, depth, T_final,
                           n_contrib, active, state: dict, ws, tuning=None, stream=None):
    P_ = proj_struct(proj)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    tu = tuning_struct(tuning)
    S = active_state_struct(state)
    _check("gevo_render_fwd_active", load().gevo_render_fwd_active(
        ctypes.byref(layout), int(n), ctypes.byref(P_), _p(vals), _p(ranges), bgv, _p(rgb),
        _p(depth), _p(T_final), _p(n_contrib), _p(active), ctypes.byref(S),
        ctypes.byref(tu) if tu is not None else None, _p(ws), _stream(stream)))


def gevo_render_bwd_active(layout, n, proj: dict, vals, ranges, bg, T_final, n_contrib, dL_drgb,
                           dL_ddepth, dL_dT, pix_err, gauss_err, active, grad2d: dict, ws,
                           tuning=None, stream=None, state=None):
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    tu = tuning_struct(tuning)
    S = active_state_struct(state)
    _check("gevo_render_bwd_active", load().gevo_render_bwd_active(
        ctypes.byref(layout), int(n), ctypes.byref(P_), _p(vals), _p(ranges), bgv, _p(T_final),
        _p(n_contrib), _p(dL_drgb), _p(dL_ddepth), _p(dL_dT), _p(pix_err), _p(gauss_err),
        _p(active), ctypes.byref(S) if S is not None else None, ctypes.byref(G2),
        ctypes.byref(tu) if tu is not None else None, _p(ws), _stream(stream)))


def gevo_active_set(n_views, n, gauss_err, eps, force, active, active_list, counts, stream=None):
    _check("gevo_active_set", load().gevo_active_set(
        int(n_views), int(n), _p(gauss_err), float(eps), _p(force), _p(active), _p(active_list),
        _p(counts), _stream(stream)))


def active_count_words(n: int) -> int:
    """GEVO_ACTIVE_COUNT_WORDS(n) of include/gevo.h."""
    return (int(n) + 1023) // 1024 + 1


def gevo_grad2d_zero(layout, n, proj: dict, grad2d: dict, stream=None):
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    _check("gevo_grad2d_zero", load().gevo_grad2d_zero(ctypes.byref(layout), int(n),
                                                       ctypes.byref(P_), ctypes.byref(G2),
                                                       _stream(stream)))


def gevo_project_zero(layout, g: dict, cams: torch.Tensor, proj: dict, grad2d: dict, part: int,
                      ws: torch.Tensor, stream=None, g_begin=0, g_end=None):
    """gevo_project_part (PART_ALL or PART_GEOMETRY) that also zeroes the 2-D
    gradient rows of the entries it finds visible."""
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    _check("gevo_project_zero", load().gevo_project_zero(
        ctypes.byref(layout), ctypes.byref(G), _p(cams), ctypes.byref(P_), ctypes.byref(G2),
        int(part), int(g_begin), int(G.n if g_end is None else g_end), _p(ws), _stream(stream)))


def gevo_project_bwd(layout, g: dict, cams, proj: dict, grad2d: dict, out: dict, dxi, ws,
                     stream=None):
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    O = GaussianGrads()
    O.means, O.scales, O.quats, O.opacities = (_p(out["means"]), _p(out["scales"]),
                                               _p(out["quats"]), _p(out["opacities"]))
    O.sh = _p(out.get("sh"))
    O.rgb = _p(out.get("rgb"))
    _check("gevo_project_bwd", load().gevo_project_bwd(
        ctypes.byref(layout), ctypes.byref(G), _p(cams), ctypes.byref(P_), ctypes.byref(G2),
        ctypes.byref(O), _p(dxi), _p(ws), _stream(stream)))


def gevo_project_bwd_part(layout, g: dict, cams, proj: dict, grad2d: dict, out: dict, dxi,
                          part: int, ws, stream=None, g_begin=0, g_end=None):
    """One part of gevo_project_bwd over a range of whole PART_RANGE blocks
    (default: all): PART_COLOUR first (its range at 0 first of all), then
    PART_GEOMETRY."""
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    O = GaussianGrads()
    O.means, O.scales, O.quats, O.opacities = (_p(out["means"]), _p(out["scales"]),
                                               _p(out["quats"]), _p(out["opacities"]))
    O.sh = _p(out.get("sh"))
    O.rgb = _p(out.get("rgb"))
    _check("gevo_project_bwd_part", load().gevo_project_bwd_part(
        ctypes.byref(layout), ctypes.byref(G), _p(cams), ctypes.byref(P_), ctypes.byref(G2),
        ctypes.byref(O), _p(dxi), int(part), int(g_begin), int(G.n if g_end is None else g_end),
        _p(ws), _stream(stream)))


def gevo_project_bwd_active(layout, g: dict, cams, proj: dict, grad2d: dict, active_list, counts,
                            out: dict, dxi, ws, stream=None):
    G = gaussians_struct(g)
    P_ = proj_struct(proj)
    G2 = grad2d_struct(grad2d)
    O = GaussianGrads()
    O.means, O.scales, O.quats, O.opacities = (_p(out["means"]), _p(out["scales"]),
                                               _p(out["quats"]), _p(out["opacities"]))
    O.sh = _p(out.get("sh"))
    O.rgb = _p(out.get("rgb"))
    _check("gevo_project_bwd_active", load().gevo_project_bwd_active(
        ctypes.byref(layout), ctypes.byref(G), _p(cams), ctypes.byref(P_), ctypes.byref(G2),
        _p(active_list), _p(counts), ctypes.byref(O), _p(dxi), _p(ws), _stream(stream)))


def gevo_loss_l1_err(layout, rgb, target_rgb, depth, target_depth, lambda_depth, dL_drgb,
                     dL_ddepth, loss, pix_err, ws=None, stream=None):
    _check("gevo_loss_l1_err", load().gevo_loss_l1_err(
        ctypes.byref(layout), _p(rgb), _p(target_rgb), _p(depth), _p(target_depth),
        float(lambda_depth), _p(dL_drgb), _p(dL_ddepth), _p(loss), _p(pix_err), _p(ws),
        _stream(stream)))


def gevo_loss_l1(layout, rgb, target_rgb, depth, target_depth, lambda_depth, dL_drgb, dL_ddepth,
                 loss, ws=None, stream=None):
    _check("gevo_loss_l1", load().gevo_loss_l1(
        ctypes.byref(layout), _p(rgb), _p(target_rgb), _p(depth), _p(target_depth),
        float(lambda_depth), _p(dL_drgb), _p(dL_ddepth), _p(loss), _p(ws), _stream(stream)))


def gevo_gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, out_bf16, bias, relu, beta, ws,
                   stream=None):
    _check("gevo_gemm_bf16", load().gevo_gemm_bf16(
        int(M), int(N), int(K), _p(A), int(lda), _p(B), int(ldb), _p(C), int(ldc),
        int(bool(out_bf16)), _p(bias), int(bool(relu)), float(beta), _p(ws), _stream(stream)))


def gevo_last_error(ws, stream=None) -> int:
    return int(load().gevo_last_error(_p(ws), _stream(stream)))


def gevo_status_str(code: int) -> str:
    return load().gevo_status_str(int(code)).decode()


def gevo_version() -> int:
    return int(load().gevo_version())


def prior_call(name, *args, stream=None):
    """Calls one gevo_prior.h entry point: tensors become device pointers, the
    current stream is appended."""
    conv = []
    for a in args:
        if isinstance(a, torch.Tensor):
            conv.append(_p(a))
        elif a is None:
            conv.append(None)
        else:
            conv.append(a)
    _check(name, getattr(load(), name)(*conv, _stream(stream)))


# ---- map and pose optimisation (include/gevo_map.h) ---------------------------------
def map_params_struct(d: dict) -> MapParams:
    return MapParams(_p(d["means"]), _p(d["log_scales"]), _p(d["quats"]),
                     _p(d["logit_opacities"]), _p(d["colours"]))


def map_adam_struct(cfg: dict) -> MapAdam:
    return MapAdam(*[float(cfg[k]) for k, _ in MapAdam._fields_])


def gevo_map_activate(n, log_scales, logit_opacities, scales, opacities, stream=None):
    _check("gevo_map_activate", load().gevo_map_activate(
        int(n), _p(log_scales), _p(logit_opacities), _p(scales), _p(opacities), _stream(stream)))


def gevo_map_step(n, K, params: dict, grads: dict, m: dict, v: dict, cfg: dict, step, rows,
                  counts, scales, opacities, iso_loss=None, stream=None):
    G = GaussianGrads()
    G.means, G.scales, G.quats, G.opacities = (_p(grads["means"]), _p(grads["scales"]),
                                               _p(grads["quats"]), _p(grads["opacities"]))
    G.sh = _p(grads.get("sh"))
    G.rgb = _p(grads.get("rgb"))
    Pp, Mm, Vv = map_params_struct(params), map_params_struct(m), map_params_struct(v)
    C = map_adam_struct(cfg)
    _check("gevo_map_step", load().gevo_map_step(
        int(n), int(K), ctypes.byref(Pp), ctypes.byref(G), ctypes.byref(Mm), ctypes.byref(Vv),
        ctypes.byref(C), int(step), _p(rows), _p(counts), _p(scales), _p(opacities),
        _p(iso_loss), _stream(stream)))


def gevo_pose_step(n_views, cams, dxi, m, v, lr_rho, lr_phi, beta1, beta2, eps, step, fixed=None,
                   stream=None):
    _check("gevo_pose_step", load().gevo_pose_step(
        int(n_views), _p(cams), _p(dxi), _p(m), _p(v), float(lr_rho), float(lr_phi), float(beta1),
        float(beta2), float(eps), int(step), _p(fixed), _stream(stream)))


def gevo_prune_keep(n, opacities, candidates, threshold, keep, keep_list, counts, stream=None):
    _check("gevo_prune_keep", load().gevo_prune_keep(
        int(n), _p(opacities), _p(candidates), float(threshold), _p(keep), _p(keep_list),
        _p(counts), _stream(stream)))


def gevo_gather_rows(n_max, lst, counts, width, src, dst, stream=None):
    _check("gevo_gather_rows", load().gevo_gather_rows(
        int(n_max), _p(lst), _p(counts), int(width), _p(src), _p(dst), _stream(stream)))


# ---- measurement helpers (include/gevo_bench.h, libgevo_probes.so) -------------------
def load_probes():
    """Load the measurement-only probe library (built with libgevo)."""
    global _probes
    if _probes is None:
        load()
        L = ctypes.CDLL(_build.PROBE_LIB)
        for name in BENCH:
            getattr(L, name).argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p]
            getattr(L, name).restype = ctypes.c_int
        _probes = L
    return _probes


def gevo_bench_fma(blocks, iters, sink, stream=None):
    _check("gevo_bench_fma", load_probes().gevo_bench_fma(int(blocks), int(iters), _p(sink),
                                                          _stream(stream)))


def gevo_bench_fma2(blocks, iters, sink, stream=None):
    _check("gevo_bench_fma2", load_probes().gevo_bench_fma2(int(blocks), int(iters), _p(sink),
                                                            _stream(stream)))


def gevo_bench_rcp(blocks, iters, sink, stream=None):
    _check("gevo_bench_rcp", load_probes().gevo_bench_rcp(int(blocks), int(iters), _p(sink),
                                                          _stream(stream)))


def gevo_bench_ex2(blocks, iters, sink, stream=None):
    _check("gevo_bench_ex2", load_probes().gevo_bench_ex2(int(blocks), int(iters), _p(sink), _stream(stream)))
