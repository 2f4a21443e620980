"""FP64 CPU oracle of the Gaussian-splatting rasterizer GEVO renders with.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of ``bench.py`` are the only callers.  Nothing in the CUDA library imports
this package and this package imports nothing from the library.

The arithmetic lives in ``gevo_oracle.c`` (plain C, double precision, literal
per-pixel loops); this module only marshals numpy arrays.  The rasterizer is the
"GS" renderer the paper cites in Section I and optimises through in Section III-B
(Eq. 2, Eq. 3 and the rendered past keyframes of Eq. 6).  Parity status of each
function is stated in the C file's header and pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gevo_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]

_lock = threading.Lock()
_lib = None

# Constants of the formulation (same readings as the C file; restated here only
# for the Python-side chaining of views).
TILE = 16


def build(force: bool = False) -> str:
    """Compile gevo_oracle.c into oracle/_build/liboracle.so (gcc, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _P(t):
    return ctypes.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i32, i64, u32, u64 = (ctypes.c_double, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_uint32, ctypes.c_uint64)
            L.orc_sh_basis.argtypes = [ctypes.c_int, _P(d), _P(d), _P(d)]
            L.orc_cov3d.argtypes = [_P(d), _P(d), _P(d)]
            L.orc_rect_f32.argtypes = [ctypes.c_float, ctypes.c_float, i32, i32, i32, _P(i32)]
            L.orc_project.argtypes = [i32, _P(d), _P(d), _P(d), _P(d), _P(d), i32, _P(d),
                                      _P(d), i32, i32,
                                      _P(d), _P(d), _P(d), _P(d), _P(i32), _P(d), _P(i32),
                                      _P(i32), _P(i32)]
            L.orc_bin_f32.argtypes = [i32, _P(i32), _P(i32), i32, _P(ctypes.c_float), _P(i32),
                                      _P(ctypes.c_float), i64, _P(u64), _P(u32), _P(u32), _P(i32)]
            L.orc_bin_f32.restype = i64
            L.orc_render_fwd.argtypes = [i32, i32, _P(d), _P(d), _P(d), _P(d), _P(d),
                                         _P(u32), _P(u32), _P(d),
                                         _P(d), _P(d), _P(d), _P(i32), _P(i32), _P(d), _P(i32),
                                         _P(u64), _P(d), _P(d), _P(ctypes.c_uint8), _P(i32), _P(d),
                                         _P(d), _P(i32)]
            L.orc_render_bwd.argtypes = [i32, i32, _P(d), _P(d), _P(d), _P(d), _P(d),
                                         _P(u32), _P(u32), _P(d),
                                         _P(d), _P(d), _P(d),
                                         _P(d), _P(d), _P(d), _P(d), _P(d)]
            L.orc_project_bwd.argtypes = [i32, _P(d), _P(d), _P(d), _P(d), _P(d), i32, _P(d),
                                          _P(d), i32, i32, _P(i32),
                                          _P(d), _P(d), _P(d), _P(d), _P(d),
                                          _P(d), _P(d), _P(d), _P(d), _P(d), _P(d), _P(d)]
            _lib = L
    return _lib


_CT = {np.float64: ctypes.c_double, np.int32: ctypes.c_int32, np.uint32: ctypes.c_uint32,
       np.uint64: ctypes.c_uint64, np.float32: ctypes.c_float, np.int64: ctypes.c_int64,
       np.uint8: ctypes.c_uint8}


def _ptr(a, dtype):
    if a is None:
        return None
    assert a.dtype == dtype and a.flags["C_CONTIGUOUS"], (a.dtype, dtype)
    return a.ctypes.data_as(ctypes.POINTER(_CT[np.dtype(dtype).type]))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Camera helpers.  A camera is (R[3,3] world->camera, t[3], fx, fy, cx, cy, W, H).
# ---------------------------------------------------------------------------
def cam_block(cam) -> np.ndarray:
    R, t, fx, fy, cx, cy = cam["R"], cam["t"], cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c = np.zeros(16, np.float64)
    c[0:9] = np.asarray(R, np.float64).reshape(9)
    c[9:12] = np.asarray(t, np.float64)
    c[12:16] = [fx, fy, cx, cy]
    return c


def sh_basis(deg: int, d):
    d = _f64(d).reshape(3)
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib().orc_sh_basis(deg, _ptr(d, np.float64), _ptr(Y, np.float64), _ptr(dY, np.float64))
    return Y, dY.reshape(16, 3)


def cov3d(scale, quat):
    s, q = _f64(scale).reshape(3), _f64(quat).reshape(4)
    S = np.zeros(9)
    lib().orc_cov3d(_ptr(s, np.float64), _ptr(q, np.float64), _ptr(S, np.float64))
    return S.reshape(3, 3)


def rect_f32(mx, my, r, tiles_x, tiles_y):
    out = np.zeros(4, np.int32)
    lib().orc_rect_f32(float(np.float32(mx)), float(np.float32(my)), int(r), int(tiles_x),
                       int(tiles_y), _ptr(out, np.int32))
    return out


# ---------------------------------------------------------------------------
# Step 1: projection (one view).
# ---------------------------------------------------------------------------
def project(g, cam):
    """g: dict with means[N,3], scales[N,3], quats[N,4], opacities[N], and either
    rgb[N,3] or sh[N,K,3] + sh_degree.  Returns a dict of per-Gaussian arrays."""
    n = g["means"].shape[0]
    mean, scale, quat, opac = (_f64(g["means"]), _f64(g["scales"]), _f64(g["quats"]),
                               _f64(g["opacities"]))
    rgb_in = _f64(g.get("rgb"))
    sh = _f64(g.get("sh"))
    deg = int(g.get("sh_degree", 0))
    W, H = int(cam["W"]), int(cam["H"])
    c = cam_block(cam)
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), cov2d=np.zeros((n, 3)),
               depth=np.zeros(n), radius=np.zeros(n, np.int32), rgb=np.zeros((n, 3)),
               clamped=np.zeros((n, 3), np.int32), tiles_touched=np.zeros(n, np.int32),
               fragile=np.zeros(n, np.int32))
    lib().orc_project(n, _ptr(mean, np.float64), _ptr(scale, np.float64),
                      _ptr(quat, np.float64), _ptr(opac, np.float64),
                      _ptr(sh, np.float64) if sh is not None else None, deg,
                      _ptr(rgb_in, np.float64) if rgb_in is not None else None,
                      _ptr(c, np.float64), W, H,
                      _ptr(out["xy"], np.float64), _ptr(out["conic"], np.float64),
                      _ptr(out["cov2d"], np.float64), _ptr(out["depth"], np.float64),
                      _ptr(out["radius"], np.int32), _ptr(out["rgb"], np.float64),
                      _ptr(out["clamped"], np.int32), _ptr(out["tiles_touched"], np.int32),
                      _ptr(out["fragile"], np.int32))
    out["opacity"] = opac
    return out


# ---------------------------------------------------------------------------
# Steps 2-4: keys, sort and ranges over views (binary32 binning).
# ---------------------------------------------------------------------------
def tiles_of(W, H):
    return ((W + TILE - 1) // TILE) * ((H + TILE - 1) // TILE)


def bin_f32(sizes, xy32, radius, depth32, capacity=None):
    """sizes: list of (W, H) per view; xy32 float32 [V,N,2]; radius int32 [V,N];
    depth32 float32 [V,N].  Returns dict(keys, vals, ranges[T,2], n_dup, tiles_touched)."""
    V = len(sizes)
    xy32 = np.ascontiguousarray(xy32, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    depth32 = np.ascontiguousarray(depth32, np.float32)
    n = xy32.shape[1]
    Ws = np.array([s[0] for s in sizes], np.int32)
    Hs = np.array([s[1] for s in sizes], np.int32)
    T = int(sum(tiles_of(w, h) for w, h in sizes))
    # count first (capacity 0 returns the true D)
    tt = np.zeros((V, n), np.int32)
    ranges = np.zeros((T, 2), np.uint32)
    dummy_k = np.zeros(1, np.uint64)
    dummy_v = np.zeros(1, np.uint32)
    D = lib().orc_bin_f32(V, _ptr(Ws, np.int32), _ptr(Hs, np.int32), n,
                          _ptr(xy32, np.float32), _ptr(radius, np.int32),
                          _ptr(depth32, np.float32), 0, _ptr(dummy_k, np.uint64),
                          _ptr(dummy_v, np.uint32), _ptr(ranges, np.uint32), _ptr(tt, np.int32))
    cap = D if capacity is None else int(capacity)
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    D = lib().orc_bin_f32(V, _ptr(Ws, np.int32), _ptr(Hs, np.int32), n,
                          _ptr(xy32, np.float32), _ptr(radius, np.int32),
                          _ptr(depth32, np.float32), cap, _ptr(keys, np.uint64),
                          _ptr(vals, np.uint32), _ptr(ranges, np.uint32), _ptr(tt, np.int32))
    used = D if D <= cap else 0
    return dict(keys=keys[:used], vals=vals[:used], ranges=ranges, n_dup=int(D),
                tiles_touched=tt, overflow=D > cap)


# ---------------------------------------------------------------------------
# Step 5 / 6: blending of one view and its derivative.
# ---------------------------------------------------------------------------
def render_fwd(W, H, rec, vals, ranges_view, bg=(0.0, 0.0, 0.0), pix_err=None, active=None):
    """rec: dict with xy[N,2], conic[N,3], opacity[N], rgb[N,3], depth[N] (float64).
    ranges_view: this view's [tiles,2] ranges (positions into vals).
    pix_err: optional per-pixel error e(u) [H,W]; then out["gauss_err"][g] is the
    per-Gaussian rendering error E(g) = sum_u w(g, u) e(u) of Eq. 5.
    active: optional boolean mask over Gaussians; then out["act_last"] [H,W]
    (1 + list position of the last blended active entry, 0 if none),
    out["act_T"] [H,W] (transmittance right after it) and out["act_rest"]
    [H,W,4] (colour incl. T_final bg, and depth, blended behind it)."""
    P = W * H
    xy, conic, opac, rgb, depth = (_f64(rec["xy"]), _f64(rec["conic"]), _f64(rec["opacity"]),
                                   _f64(rec["rgb"]), _f64(rec["depth"]))
    vals = np.ascontiguousarray(vals, np.uint32)
    if vals.size == 0:
        vals = np.zeros(1, np.uint32)
    rv = np.ascontiguousarray(ranges_view, np.uint32)
    bgv = _f64(np.asarray(bg, np.float64))
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), T=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int32), n_eval=np.zeros((H, W), np.int32),
               n_blend=np.zeros((H, W), np.int32),
               wsum=np.zeros((H, W)), fragile=np.zeros((H, W), np.int32),
               sig=np.zeros((H, W), np.uint64))
    n = rec["xy"].shape[0]
    pe = None
    if pix_err is not None:
        pe = _f64(np.asarray(pix_err, np.float64).reshape(H, W))
        out["gauss_err"] = np.zeros(max(n, 1))
    act = None
    if active is not None:
        act = np.ascontiguousarray(np.asarray(active, bool).astype(np.uint8))
        if act.size == 0:
            act = np.zeros(1, np.uint8)
        out["act_last"] = np.zeros((H, W), np.int32)
        out["act_T"] = np.zeros((H, W))
        out["act_rest"] = np.zeros((H, W, 4))
    lib().orc_render_fwd(W, H, _ptr(xy, np.float64), _ptr(conic, np.float64),
                         _ptr(opac, np.float64), _ptr(rgb, np.float64), _ptr(depth, np.float64),
                         _ptr(vals, np.uint32), _ptr(rv, np.uint32), _ptr(bgv, np.float64),
                         _ptr(out["rgb"], np.float64), _ptr(out["depth"], np.float64),
                         _ptr(out["T"], np.float64), _ptr(out["n_contrib"], np.int32),
                         _ptr(out["n_eval"], np.int32), _ptr(out["wsum"], np.float64),
                         _ptr(out["fragile"], np.int32), _ptr(out["sig"], np.uint64),
                         _ptr(pe, np.float64) if pe is not None else None,
                         _ptr(out["gauss_err"], np.float64) if pe is not None else None,
                         _ptr(act, np.uint8) if act is not None else None,
                         _ptr(out["act_last"], np.int32) if act is not None else None,
                         _ptr(out["act_T"], np.float64) if act is not None else None,
                         _ptr(out["act_rest"], np.float64) if act is not None else None,
                         _ptr(out["n_blend"], np.int32))
    if pe is not None:
        out["gauss_err"] = out["gauss_err"][:n]
    del P
    return out


def render_bwd(W, H, rec, vals, ranges_view, dL_drgb, dL_ddepth=None, dL_dT=None,
               bg=(0.0, 0.0, 0.0)):
    n = rec["xy"].shape[0]
    xy, conic, opac, rgb, depth = (_f64(rec["xy"]), _f64(rec["conic"]), _f64(rec["opacity"]),
                                   _f64(rec["rgb"]), _f64(rec["depth"]))
    vals = np.ascontiguousarray(vals, np.uint32)
    if vals.size == 0:
        vals = np.zeros(1, np.uint32)
    rv = np.ascontiguousarray(ranges_view, np.uint32)
    bgv = _f64(np.asarray(bg, np.float64))
    gC = _f64(dL_drgb).reshape(3, H, W)
    gD = _f64(dL_ddepth) if dL_ddepth is not None else None
    gT = _f64(dL_dT) if dL_dT is not None else None
    g = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
             rgb=np.zeros((n, 3)), depth=np.zeros(n))
    lib().orc_render_bwd(W, H, _ptr(xy, np.float64), _ptr(conic, np.float64),
                         _ptr(opac, np.float64), _ptr(rgb, np.float64), _ptr(depth, np.float64),
                         _ptr(vals, np.uint32), _ptr(rv, np.uint32), _ptr(bgv, np.float64),
                         _ptr(gC, np.float64),
                         _ptr(gD, np.float64) if gD is not None else None,
                         _ptr(gT, np.float64) if gT is not None else None,
                         _ptr(g["xy"], np.float64), _ptr(g["conic"], np.float64),
                         _ptr(g["opacity"], np.float64), _ptr(g["rgb"], np.float64),
                         _ptr(g["depth"], np.float64))
    return g


# ---------------------------------------------------------------------------
# Step 7: projection derivative (one view), accumulated into `acc`.
# ---------------------------------------------------------------------------
def grads_like(g):
    n = g["means"].shape[0]
    acc = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacities=np.zeros(n))
    if g.get("rgb") is not None:
        acc["rgb"] = np.zeros((n, 3))
    else:
        acc["sh"] = np.zeros_like(_f64(g["sh"]))
    return acc


def project_bwd(g, cam, radius, g2d, acc, dxi=None):
    n = g["means"].shape[0]
    mean, scale, quat, opac = (_f64(g["means"]), _f64(g["scales"]), _f64(g["quats"]),
                               _f64(g["opacities"]))
    rgb_in = _f64(g.get("rgb"))
    sh = _f64(g.get("sh"))
    deg = int(g.get("sh_degree", 0))
    c = cam_block(cam)
    radius = np.ascontiguousarray(radius, np.int32)
    gx, gc, go, gr, gd = (_f64(g2d["xy"]), _f64(g2d["conic"]), _f64(g2d["opacity"]),
                          _f64(g2d["rgb"]), _f64(g2d["depth"]))
    dsh = acc.get("sh")
    drgb = acc.get("rgb")
    lib().orc_project_bwd(n, _ptr(mean, np.float64), _ptr(scale, np.float64),
                          _ptr(quat, np.float64), _ptr(opac, np.float64),
                          _ptr(sh, np.float64) if sh is not None else None, deg,
                          _ptr(rgb_in, np.float64) if rgb_in is not None else None,
                          _ptr(c, np.float64), int(cam["W"]), int(cam["H"]),
                          _ptr(radius, np.int32),
                          _ptr(gx, np.float64), _ptr(gc, np.float64), _ptr(go, np.float64),
                          _ptr(gr, np.float64), _ptr(gd, np.float64),
                          _ptr(acc["means"], np.float64), _ptr(acc["scales"], np.float64),
                          _ptr(acc["quats"], np.float64), _ptr(acc["opacities"], np.float64),
                          _ptr(dsh, np.float64) if dsh is not None else None,
                          _ptr(drgb, np.float64) if drgb is not None else None,
                          _ptr(dxi, np.float64) if dxi is not None else None)
    return acc


# ---------------------------------------------------------------------------
# Step 8: L1 photometric (+ depth) loss of Eq. 2 / Eq. 6 with stop-gradient
# targets.  L = sum_v [ mean|C_v - C*_v| + lambda_d mean|D_v - D*_v| ];
# gradient sign(.)/count with sign(0) = 0.
# ---------------------------------------------------------------------------
def loss_l1(rgb, target_rgb, depth=None, target_depth=None, lambda_depth=0.0):
    """Lists over views of float arrays rgb[3,H,W], depth[H,W]."""
    L = 0.0
    g_rgb, g_depth = [], []
    for v in range(len(rgb)):
        d = np.asarray(rgb[v], np.float64) - np.asarray(target_rgb[v], np.float64)
        L += np.abs(d).sum() / d.size
        g_rgb.append(np.sign(d) / d.size)
        if depth is not None and lambda_depth != 0.0:
            e = np.asarray(depth[v], np.float64) - np.asarray(target_depth[v], np.float64)
            L += lambda_depth * np.abs(e).sum() / e.size
            g_depth.append(lambda_depth * np.sign(e) / e.size)
        else:
            g_depth.append(np.zeros(np.asarray(rgb[v]).shape[1:]))
    return L, g_rgb, g_depth


# ---------------------------------------------------------------------------
# Active set of the global stage (Section III-B2): E_t = {g : max_k E_k(g) > eps}
# with E_k(g) the per-Gaussian rendering error of Eq. 5 in keyframe k, united
# with the newly inserted Gaussians (A_t = M~_t u E_t).
# ---------------------------------------------------------------------------
def pixel_error(rgb, target_rgb):
    """Per-pixel error e(u) = |R(u) - C(u)| of Eq. 5, read as the mean over the
    three colour channels of the absolute difference (the L1 loss's per-pixel
    term).  rgb, target_rgb: [3, H, W]."""
    return np.abs(np.asarray(rgb, np.float64) - np.asarray(target_rgb, np.float64)).mean(axis=0)


def active_set(gauss_err, eps, force=None):
    """gauss_err: [K, n] E_k(g) over the window's keyframes.  Returns the boolean
    mask max_k E_k(g) > eps (strict), or-ed with `force` (the inserted
    Gaussians), and the ascending list of its indices."""
    e = np.asarray(gauss_err, np.float64)
    act = e.max(axis=0) > eps if e.shape[0] > 0 else np.zeros(e.shape[1], bool)
    if force is not None:
        act = act | np.asarray(force, bool)
    return act, np.nonzero(act)[0].astype(np.uint32)


def mask_grad2d(g2d, active):
    """The 2-D record gradients of an active-set backward: rows of inactive
    Gaussians are zero, rows of active ones are the full backward's."""
    a = np.asarray(active, bool)
    return {k: np.where(a.reshape((-1,) + (1,) * (np.ndim(v) - 1)), v, 0.0) for k, v in g2d.items()}


# ---------------------------------------------------------------------------
# Whole chain over views (steps 1-7), FP64, binning in binary32.
# ---------------------------------------------------------------------------
def render_views(g, cams, bg=(0.0, 0.0, 0.0), pix_errs=None):
    """Forward over all views.  Returns (per-view outputs, projections, binning).
    pix_errs: optional list over views of per-pixel errors e(u) [H,W]; each
    view's output then carries gauss_err (E_k(g) of Eq. 5)."""
    V = len(cams)
    projs = [project(g, cam) for cam in cams]
    sizes = [(int(c["W"]), int(c["H"])) for c in cams]
    xy32 = np.stack([p["xy"].astype(np.float32) for p in projs])
    rad = np.stack([p["radius"] for p in projs])
    d32 = np.stack([p["depth"].astype(np.float32) for p in projs])
    b = bin_f32(sizes, xy32, rad, d32)
    outs = []
    base = 0
    for v in range(V):
        W, H = sizes[v]
        nt = tiles_of(W, H)
        rec = dict(xy=projs[v]["xy"], conic=projs[v]["conic"], opacity=projs[v]["opacity"],
                   rgb=projs[v]["rgb"], depth=projs[v]["depth"])
        outs.append(render_fwd(W, H, rec, b["vals"], b["ranges"][base:base + nt], bg,
                               None if pix_errs is None else pix_errs[v]))
        base += nt
    return outs, projs, b


def backward_views(g, cams, projs, b, dL_drgb, dL_ddepth=None, dL_dT=None,
                   bg=(0.0, 0.0, 0.0), want_dxi=True):
    """Gradients of a loss with the given image gradients (lists over views)."""
    acc = grads_like(g)
    dxis = np.zeros((len(cams), 6))
    base = 0
    g2ds = []
    for v, cam in enumerate(cams):
        W, H = int(cam["W"]), int(cam["H"])
        nt = tiles_of(W, H)
        p = projs[v]
        rec = dict(xy=p["xy"], conic=p["conic"], opacity=p["opacity"], rgb=p["rgb"],
                   depth=p["depth"])
        g2d = render_bwd(W, H, rec, b["vals"], b["ranges"][base:base + nt], dL_drgb[v],
                         None if dL_ddepth is None else dL_ddepth[v],
                         None if dL_dT is None else dL_dT[v], bg)
        g2ds.append(g2d)
        project_bwd(g, cam, p["radius"], g2d, acc, dxis[v] if want_dxi else None)
        base += nt
    return acc, dxis, g2ds
