"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Every input comes from paper_2409_09295_gb300.scenes (seeded); no oracle input
and no expected value comes from the CUDA path.  Stage-isolated tests feed both
sides the same binary32 records drawn by the generator; end-to-end tests start
both sides from the same Gaussians.

Tolerances (each derived from the binary32 arithmetic of the kernels):
  - tile lists, keys, values, ranges, duplicate counts: bit-exact;
  - blended images from identical binary32 records: 1e-5 absolute;
  - end-to-end images: 1e-5 + the propagated binary32 projection error bound;
  - gradients: relative L2 <= 1e-3 per tensor and |g - ref| <= 1e-3 |ref| +
    1e-3 rms(ref) per element;
pixels or Gaussians where the oracle reports a discrete decision within a small
margin of its threshold are excluded, and their count is bounded.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from gpu_helpers import (grad_close, records_for_oracle, tiles_of,  # noqa: E402
                         upload_records)
from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import _abi, raster  # noqa: E402

TUNINGS = [dict(threads_per_tile=256, persistent=0, blocks_per_sm=0),
           dict(threads_per_tile=128, persistent=1, blocks_per_sm=0),
           dict(threads_per_tile=64, persistent=1, blocks_per_sm=2),
           dict(threads_per_tile=32, persistent=0, blocks_per_sm=0),
           dict(threads_per_tile=32, persistent=1, blocks_per_sm=12)]
TUNING_IDS = ["ppt1", "ppt2_persistent", "ppt4_persistent", "ppt8", "ppt8_persistent12"]


def _np(t):
    return t.detach().cpu().numpy()


# --------------------------------------------------------------------------
# a2-a4: keys / sort / ranges, bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["one_view", "uneven_views", "crowded_tile", "long_tiles",
                                  "equal_depths", "one_depth", "wide_depths", "huge_view",
                                  "giant_splats", "many_views", "deep_segment", "empty"])
def test_bin_sort_bit_exact(case):
    if case == "deep_segment":
        # 5500 of 6000 entries in a depth band narrower than one of the view's
        # depth segments (outliers stretch the view's depth range): the per-view
        # depth sort takes its L2 path for a segment of more than 2048 entries
        sizes, n = [(64, 48)], 6000
        rec = scenes.random_records(sizes, n, seed=39, sigma_px=(0.5, 3.0), frac_culled=0.0)
        r = np.random.default_rng(6)
        d = r.uniform(5.0, 5.001, n)
        d[:250] = r.uniform(0.5, 0.6, 250)
        d[250:500] = r.uniform(9.9, 10.0, 250)
        rec["depth"][0] = d.astype(np.float32)
    elif case == "giant_splats":
        # 90 x 90 = 8100 tiles, the depth-ordered path's largest kind of view: a
        # few splats cover every tile (8100 duplicates each, so they span several
        # 1024-duplicate warp ranges and 8192-duplicate units and start and end
        # inside them) among small ones
        sizes, n = [(1440, 1440)], 3000
        rec = scenes.random_records(sizes, n, seed=37, sigma_px=(0.5, 6.0), frac_culled=0.0)
        big = np.arange(0, n, 500)
        rec["xy"][0, big] = np.float32(720.0)
        rec["radius"][0, big] = 1100
        rec["depth"][0, big[::2]] = np.float32(0.6)   # some nearest, some among the rest
    elif case == "many_views":
        # 24 views of 12 tiles each: the unit table and the per-view scans
        sizes = [(64, 48)] * 24
        n = 400
        rec = scenes.random_records(sizes, n, seed=38, sigma_px=(0.5, 20.0))
    elif case == "huge_view":
        # 132 x 130 = 17160 tiles in one view: more than the 16384 per-view tile
        # counters the shared-memory binning holds, so the global-atomic count
        # and scatter kernels run
        sizes, n = [(2112, 2080), (64, 48)], 30000
        rec = scenes.random_records(sizes, n, seed=36)
    elif case == "one_view":
        sizes, n, rec = [(64, 48)], 3000, None
    elif case == "uneven_views":
        sizes, n, rec = [(640, 480), (320, 240), (1200, 680), (33, 17)], 4000, None
    elif case == "crowded_tile":
        sizes, n = [(64, 48)], 9000
        rec = scenes.random_records(sizes, n, seed=31, sigma_px=(0.5, 1.5))
        rec["xy"][0, :, 0] = np.random.default_rng(1).uniform(20, 27, n).astype(np.float32)
        rec["xy"][0, :, 1] = np.random.default_rng(2).uniform(20, 27, n).astype(np.float32)
        rec["radius"][0] = np.minimum(rec["radius"][0], 3)
    elif case == "long_tiles":
        # two tiles of about 3000 entries each: past the shared-memory sort, the
        # L2 ping-pong path with several blocks' worth of items
        sizes, n = [(64, 48)], 7000
        rec = scenes.random_records(sizes, n, seed=33, sigma_px=(0.5, 1.5))
        rec["xy"][0, :, 0] = np.random.default_rng(3).uniform(2, 30, n).astype(np.float32)
        rec["xy"][0, :, 1] = np.random.default_rng(4).uniform(2, 14, n).astype(np.float32)
        rec["radius"][0] = np.minimum(rec["radius"][0], 1)
    elif case == "equal_depths":
        sizes, n = [(96, 64)], 3000
        rec = scenes.random_records(sizes, n, seed=32)
        rec["depth"][0] = np.round(rec["depth"][0] * 2.0).astype(np.float32) / 2.0
    elif case == "one_depth":
        # every entry ties on depth: no radix pass, the id order decides alone
        sizes, n = [(64, 48)], 1500
        rec = scenes.random_records(sizes, n, seed=34)
        rec["depth"][0] = np.float32(3.0)
    elif case == "wide_depths":
        # depths log-uniform over 0.2 .. 1e6: the bit patterns of one tile span
        # more than 2^27, so the shared-memory sort takes all four 9-bit passes
        sizes, n = [(64, 48)], 3000
        rec = scenes.random_records(sizes, n, seed=35)
        rec["depth"][0] = np.exp(np.random.default_rng(5).uniform(np.log(0.2), np.log(1e6), n)).astype(np.float32)
    else:
        sizes, n, rec = [(64, 48)], 0, None
    if rec is None:
        rec = scenes.random_records(sizes, max(n, 1), seed=30 + len(sizes))
        if n == 0:
            rec["xy"] = np.zeros((1, 0, 2), np.float32)
            rec["conic"] = np.zeros((1, 0, 3), np.float32)
            rec["depth"] = np.zeros((1, 0), np.float32)
            rec["radius"] = np.zeros((1, 0), np.int32)
            rec["rgb"] = np.zeros((1, 0, 3), np.float32)
            rec["opacity"] = np.zeros(0, np.float32)
    ref = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    D = ref["n_dup"]
    pipe = raster.Pipeline(n, sizes, max(D, 1), keep_keys=True)
    if n > 0:
        upload_records(pipe, rec)
    pipe.bin_sort()
    torch.cuda.synchronize()
    assert pipe.last_error() == 0
    assert int(pipe.n_dup.item()) == D
    np.testing.assert_array_equal(_np(pipe.ranges).view(np.uint32), ref["ranges"])
    np.testing.assert_array_equal(_np(pipe.keys)[:D].view(np.uint64), ref["keys"])
    np.testing.assert_array_equal(_np(pipe.vals)[:D].view(np.uint32), ref["vals"])
    # without keys (what the renderers need): the same ids and ranges
    vals2, ranges2 = torch.zeros_like(pipe.vals), torch.ones_like(pipe.ranges)
    n_dup2 = torch.zeros_like(pipe.n_dup)
    _abi.gevo_bin_sort(pipe.layout, n, pipe.proj, pipe.capacity, None, vals2, ranges2, n_dup2,
                       pipe.ws)
    torch.cuda.synchronize()
    assert pipe.last_error() == 0 and int(n_dup2.item()) == D
    assert torch.equal(ranges2, pipe.ranges) and torch.equal(vals2[:D], pipe.vals[:D])
    lens = np.diff(ref["ranges"].astype(np.int64), axis=1)
    if case == "crowded_tile":
        assert lens.max() > 4096  # global-memory path
    if case == "long_tiles":
        assert ((lens > 2048) & (lens <= 4096)).sum() >= 2
    if case == "giant_splats":
        assert int(lens.min()) >= 6 and D > 6 * 8192
    if case == "wide_depths":
        k = ref["keys"] & 0xffffffff
        spans = [int(k[a:b].max()) - int(k[a:b].min()) for a, b in ref["ranges"] if 1 < b - a <= 2048]
        assert max(spans) >= 1 << 27


def test_bin_sort_overflow_sets_error_and_reports_true_count():
    sizes = [(64, 48)]
    rec = scenes.random_records(sizes, 500, seed=40)
    ref = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    D = ref["n_dup"]
    pipe = raster.Pipeline(500, sizes, D - 1)
    upload_records(pipe, rec)
    pipe.bin_sort()
    assert pipe.last_error() == 2
    assert int(pipe.n_dup.item()) == D
    assert (_np(pipe.ranges) == 0).all()
    assert pipe.last_error() == 0  # cleared by the read


# --------------------------------------------------------------------------
# a5 / a6 on identical binary32 records
# --------------------------------------------------------------------------
def _staged(sizes, n, seed, sigma_px=(0.5, 12.0), opacity=(0.02, 1.0)):
    rec = scenes.random_records(sizes, n, seed=seed, sigma_px=sigma_px, opacity=opacity)
    ref_bins = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    pipe = raster.Pipeline(n, sizes, ref_bins["n_dup"] + 16)
    upload_records(pipe, rec)
    pipe.bin_sort()
    return rec, ref_bins, pipe


@pytest.mark.parametrize("tuning", TUNINGS, ids=TUNING_IDS)
def test_render_fwd_staged_1e5(tuning):
    sizes = [(96, 80), (53, 37)]
    rec, b, pipe = _staged(sizes, 2500, seed=50)
    bg = (0.1, 0.2, 0.3)
    n_blend = torch.zeros_like(pipe.n_eval)
    from paper_2409_09295_gb300 import _abi
    _abi.gevo_render_fwd_counts(pipe.layout, pipe.n, pipe.proj, pipe.vals, pipe.ranges, bg, pipe.rgb,
                                pipe.depth, pipe.T_final, pipe.n_contrib, pipe.n_eval, n_blend, pipe.ws,
                                tuning)
    torch.cuda.synchronize()
    counted = {k: _np(getattr(pipe, k)).copy() for k in ("rgb", "n_contrib", "n_eval")}
    pipe.render_fwd(bg, n_eval=True, tuning=tuning)
    torch.cuda.synchronize()
    for k, want in counted.items():   # the counting variant renders the same image
        np.testing.assert_array_equal(_np(getattr(pipe, k)), want, err_msg=k)
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg)
        base += nt
        ok = o["fragile"] == 0
        assert ok.mean() > 0.97
        np.testing.assert_array_equal(_np(pipe.view_plane(n_blend, v))[ok], o["n_blend"][ok])
        np.testing.assert_allclose(_np(pipe.view_rgb(pipe.rgb, v))[:, ok], o["rgb"][:, ok], atol=1e-5, rtol=0)
        np.testing.assert_allclose(_np(pipe.view_plane(pipe.depth, v))[ok], o["depth"][ok], atol=1e-5 * 10, rtol=1e-5)
        np.testing.assert_allclose(_np(pipe.view_plane(pipe.T_final, v))[ok], o["T"][ok], atol=1e-5, rtol=0)
        np.testing.assert_array_equal(_np(pipe.view_plane(pipe.n_contrib, v))[ok], o["n_contrib"][ok])
        np.testing.assert_array_equal(_np(pipe.view_plane(pipe.n_eval, v))[ok], o["n_eval"][ok])


def test_render_fwd_faint_and_huge_splats():
    """Opacities down to 0.001 (below the 1/255 skip level everywhere) and
    splats up to ~800 px across: the per-warp culling box must never drop an
    entry the per-pixel test would blend.  Decisions (n_contrib, n_eval) must
    match exactly; a dropped entry would also move T by at least alpha >= 1/255
    relative, while binary32 accumulation over m blended entries moves it by
    about m * 4e-7 in T and m * 1e-6 in colour (the colour tolerance)."""
    sizes = [(160, 96)]
    rec, b, pipe = _staged(sizes, 1500, seed=53, sigma_px=(0.3, 120.0), opacity=(0.001, 1.0))
    pipe.render_fwd((0.0, 0.0, 0.0), n_eval=True)
    torch.cuda.synchronize()
    o = oracle.render_fwd(160, 96, records_for_oracle(rec, 0), b["vals"], b["ranges"], (0, 0, 0))
    ok = o["fragile"] == 0
    assert ok.mean() > 0.95
    np.testing.assert_array_equal(_np(pipe.view_plane(pipe.n_contrib, 0))[ok], o["n_contrib"][ok])
    np.testing.assert_array_equal(_np(pipe.view_plane(pipe.n_eval, 0))[ok], o["n_eval"][ok])
    T = _np(pipe.view_plane(pipe.T_final, 0))
    rel = np.abs(T / o["T"] - 1.0)[ok]
    assert rel.max() <= 2e-3, rel.max()
    tol = 1e-5 + 1e-6 * o["n_contrib"]
    err = np.abs(_np(pipe.view_rgb(pipe.rgb, 0)) - o["rgb"]).max(0)
    assert (err[ok] <= tol[ok]).all(), (err[ok] / tol[ok]).max()


def test_render_tunings_bitwise_identical():
    sizes = [(96, 80), (53, 37)]
    rec, b, pipe = _staged(sizes, 2500, seed=51)
    outs = []
    for t in TUNINGS:
        pipe.render_fwd((0.0, 0.5, 1.0), tuning=t)
        outs.append([_np(x).copy() for x in (pipe.rgb, pipe.depth, pipe.T_final, pipe.n_contrib)])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("tuning", TUNINGS, ids=TUNING_IDS)
def test_render_bwd_staged(tuning):
    sizes = [(96, 80), (53, 37)]
    rec, b, pipe = _staged(sizes, 2000, seed=52)
    bg = (0.1, 0.2, 0.3)
    pipe.render_fwd(bg, tuning=tuning)
    rs = np.random.default_rng(5)
    gC = rs.normal(size=3 * pipe.P).astype(np.float32)
    gD = rs.normal(size=pipe.P).astype(np.float32)
    gT = rs.normal(size=pipe.P).astype(np.float32)
    # pixels whose blend decisions are fragile get zero upstream gradient on both sides
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg)
        fr = o["fragile"].reshape(-1) != 0
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        for ch in range(3):
            gC[3 * p0 + ch * (p1 - p0):3 * p0 + (ch + 1) * (p1 - p0)][fr] = 0
        gD[p0:p1][fr] = 0
        gT[p0:p1][fr] = 0
        base += nt
    dev = pipe.device
    tC, tD, tT = (torch.from_numpy(x).to(dev) for x in (gC, gD, gT))
    pipe.render_bwd(tC, tD, tT, bg, tuning=tuning)
    torch.cuda.synchronize()
    n = 2000
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        g = oracle.render_bwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt],
                              gC[3 * p0:3 * p1].reshape(3, H, W), gD[p0:p1].reshape(H, W),
                              gT[p0:p1].reshape(H, W), bg)
        base += nt
        vis = rec["radius"][v] > 0
        sl = slice(v * n, (v + 1) * n)
        gxy = _np(pipe.grad2d["xy"])[sl][vis]
        gco = _np(pipe.grad2d["conic_opacity"])[sl][vis]
        grz = _np(pipe.grad2d["rgb_depth"])[sl][vis]
        grad_close(gxy, g["xy"][vis], f"v{v} dxy")
        grad_close(gco[:, :3], g["conic"][vis], f"v{v} dconic")
        grad_close(gco[:, 3], g["opacity"][vis], f"v{v} dopacity")
        grad_close(grz[:, :3], g["rgb"][vis], f"v{v} drgb")
        grad_close(grz[:, 3], g["depth"][vis], f"v{v} ddepth")


# --------------------------------------------------------------------------
# a1 projection and a7 projection backward
# --------------------------------------------------------------------------
def _scene(kind, n):
    if kind == "box_rgb":
        w = scenes.workload(0, n=n)
        return w["scene"], w["cams"]
    if kind == "room_sh3":
        w = scenes.workload(1, n=n)
        c = w["cams"][0]
        cams = [c, scenes.camera(*scenes.look_at([1.0, 0.5, -3.0], [0.0, 0.0, 0.0]), 262.5, 262.5,
                                 160, 120, 320, 240)]
        return w["scene"], cams
    if kind == "sub_sh3":
        return scenes.tracking_subscene(n)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n", [("box_rgb", 3000), ("room_sh3", 30000), ("sub_sh3", 2000)])
def test_project_parity(kind, n):
    scene, cams = _scene(kind, n)
    sizes = [(c["W"], c["H"]) for c in cams]
    colour = "rgb" if "rgb" in scene else "sh"
    pipe = raster.Pipeline(n, sizes, 1, colour=colour, sh_degree=scene["sh_degree"])
    g = raster.gaussians_to_device(scene)
    pipe.project(g, raster.camera_tensor(cams))
    torch.cuda.synchronize()
    assert pipe.last_error() == 0
    for v, cam in enumerate(cams):
        p = oracle.project(scene, cam)
        sl = slice(v * n, (v + 1) * n)
        rad = _np(pipe.proj["radius"])[sl]
        ok = p["fragile"] == 0
        assert ok.mean() > 0.99
        np.testing.assert_array_equal(rad[ok], p["radius"][ok])
        np.testing.assert_array_equal(_np(pipe.proj["tiles_touched"])[sl][ok], p["tiles_touched"][ok])
        vis = ok & (p["radius"] > 0)
        assert vis.sum() > 10
        # error bound of the binary32 projection: position ~ f |p| / z ulps,
        # conic ~ |Q| (1e-5 + 2e-6 kappa)
        mu = scene["means"].astype(np.float64)
        pc = mu @ np.asarray(cam["R"], np.float64).T + np.asarray(cam["t"], np.float64)
        z = pc[:, 2]
        f = max(cam["fx"], cam["fy"])
        tol_xy = 1e-4 + 4e-7 * f * (np.abs(pc).sum(1) + np.abs(cam["t"]).sum()) / np.abs(z)
        d_xy = np.abs(_np(pipe.proj["xy"])[sl] - p["xy"]).max(1)
        assert (d_xy[vis] <= tol_xy[vis]).all(), d_xy[vis].max()
        co = _np(pipe.proj["conic_opacity"])[sl]
        cov = p["cov2d"]
        tr = cov[:, 0] + cov[:, 2]
        det = cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
        lam_min = 0.5 * tr - np.sqrt(np.maximum(0.25 * tr * tr - det, 0))
        lam_max = 0.5 * tr + np.sqrt(np.maximum(0.25 * tr * tr - det, 0))
        kappa = lam_max / np.maximum(lam_min, 1e-30)
        qn = np.abs(p["conic"]).max(1)
        tol_c = qn * (1e-5 + 2e-6 * kappa) * (1 + 1e3 * tol_xy / f)
        d_c = np.abs(co[:, :3] - p["conic"]).max(1)
        assert (d_c[vis] <= tol_c[vis]).all(), (d_c[vis] / tol_c[vis]).max()
        np.testing.assert_allclose(co[vis, 3], scene["opacities"][vis], rtol=0, atol=0)
        rz = _np(pipe.proj["rgb_depth"])[sl]
        np.testing.assert_allclose(rz[vis, :3], p["rgb"][vis], atol=2e-6, rtol=1e-5)
        np.testing.assert_allclose(rz[vis, 3], p["depth"][vis], rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("kind,n", [("box_rgb", 3000), ("room_sh3", 20000), ("sub_sh3", 2000)])
def test_project_bwd_parity(kind, n):
    """Same synthetic record gradients into both sides' projection derivative."""
    scene, cams = _scene(kind, n)
    sizes = [(c["W"], c["H"]) for c in cams]
    colour = "rgb" if "rgb" in scene else "sh"
    pipe = raster.Pipeline(n, sizes, 1, colour=colour, sh_degree=scene["sh_degree"])
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    pipe.project(g, camt)
    rs = np.random.default_rng(9)
    V = len(cams)
    gxy = rs.normal(size=(V, n, 2)).astype(np.float32)
    gco = (rs.normal(size=(V, n, 4)) * [30.0, 30.0, 30.0, 1.0]).astype(np.float32)
    grz = rs.normal(size=(V, n, 4)).astype(np.float32)
    projs = [oracle.project(scene, cam) for cam in cams]
    for v in range(V):
        bad = projs[v]["fragile"] != 0
        gxy[v][bad] = 0
        gco[v][bad] = 0
        grz[v][bad] = 0
    dev = pipe.device
    pipe.grad2d["xy"].copy_(torch.from_numpy(gxy.reshape(V * n, 2)).to(dev))
    pipe.grad2d["conic_opacity"].copy_(torch.from_numpy(gco.reshape(V * n, 4)).to(dev))
    pipe.grad2d["rgb_depth"].copy_(torch.from_numpy(grz.reshape(V * n, 4)).to(dev))
    pipe.project_bwd(g, camt, want_dxi=True)
    torch.cuda.synchronize()
    acc = oracle.grads_like(scene)
    dxi = np.zeros((V, 6))
    for v, cam in enumerate(cams):
        g2d = dict(xy=gxy[v], conic=gco[v][:, :3], opacity=gco[v][:, 3], rgb=grz[v][:, :3],
                   depth=grz[v][:, 3])
        # the oracle's own visibility, restricted to where both sides agree
        rad = np.where(projs[v]["fragile"] != 0, 0, projs[v]["radius"])
        oracle.project_bwd(scene, cam, rad, g2d, acc, dxi[v])
    for k in acc:
        grad_close(_np(pipe.grads[k]), acc[k], k)
    grad_close(_np(pipe.dxi), dxi, "dxi")


# --------------------------------------------------------------------------
# a8 loss
# --------------------------------------------------------------------------
def test_loss_l1_parity():
    sizes = [(64, 48), (33, 17)]
    pipe = raster.Pipeline(1, sizes, 1)
    rs = np.random.default_rng(3)
    a = rs.uniform(size=3 * pipe.P).astype(np.float32)
    b = rs.uniform(size=3 * pipe.P).astype(np.float32)
    b[:50] = a[:50]  # exact ties: sign(0) = 0
    d = rs.uniform(1, 5, size=pipe.P).astype(np.float32)
    e = rs.uniform(1, 5, size=pipe.P).astype(np.float32)
    dev = pipe.device
    pipe.rgb.copy_(torch.from_numpy(a).to(dev))
    pipe.depth.copy_(torch.from_numpy(d).to(dev))
    pipe.loss_l1(torch.from_numpy(b).to(dev), torch.from_numpy(e).to(dev), 0.7)
    torch.cuda.synchronize()
    rgbs = [a[3 * pipe.pix_base[v]:3 * pipe.pix_base[v + 1]].reshape(3, h, w) for v, (w, h) in enumerate(sizes)]
    trg = [b[3 * pipe.pix_base[v]:3 * pipe.pix_base[v + 1]].reshape(3, h, w) for v, (w, h) in enumerate(sizes)]
    ds = [d[pipe.pix_base[v]:pipe.pix_base[v + 1]].reshape(h, w) for v, (w, h) in enumerate(sizes)]
    es = [e[pipe.pix_base[v]:pipe.pix_base[v + 1]].reshape(h, w) for v, (w, h) in enumerate(sizes)]
    L, gC, gD = oracle.loss_l1(rgbs, trg, ds, es, 0.7)
    assert float(_np(pipe.loss).sum()) == pytest.approx(L, rel=1e-5)
    np.testing.assert_allclose(_np(pipe.dL_drgb), np.concatenate([x.reshape(-1) for x in gC]), rtol=1e-6, atol=0)
    np.testing.assert_allclose(_np(pipe.dL_ddepth), np.concatenate([x.reshape(-1) for x in gD]), rtol=1e-6, atol=0)


# --------------------------------------------------------------------------
# a1-a7 end to end
# --------------------------------------------------------------------------
def _e2e(kind, n, tuning=None, bg=(0.0, 0.0, 0.0)):
    scene, cams = _scene(kind, n)
    sizes = [(c["W"], c["H"]) for c in cams]
    colour = "rgb" if "rgb" in scene else "sh"
    outs, projs, b = oracle.render_views(scene, cams, bg)
    pipe = raster.Pipeline(n, sizes, b["n_dup"] * 2 + 1024, colour=colour,
                           sh_degree=scene["sh_degree"], tuning=tuning)
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    pipe.forward(g, camt, bg)
    torch.cuda.synchronize()
    assert pipe.last_error() == 0
    # pixels to exclude: blend decisions near a threshold, and every pixel of a
    # tile that a Gaussian with a fragile projection decision may cover
    masks = []
    for v, (W, H) in enumerate(sizes):
        m = outs[v]["fragile"] != 0
        p = projs[v]
        rad_g = _np(pipe.proj["radius"])[v * n:(v + 1) * n]
        tt_g = _np(pipe.proj["tiles_touched"])[v * n:(v + 1) * n]
        tx, ty = (W + 15) // 16, (H + 15) // 16
        # a flagged Gaussian only matters where the two sides' discrete outcome
        # (radius, tile rectangle) actually differs
        differs = (p["fragile"] != 0) & ((rad_g != p["radius"]) | (tt_g != p["tiles_touched"]))
        for i in np.nonzero(differs)[0]:
            r = max(int(p["radius"][i]), int(rad_g[i]), 1)
            rc = oracle.rect_f32(p["xy"][i, 0], p["xy"][i, 1], r, tx, ty)
            m[rc[1] * 16:rc[3] * 16, rc[0] * 16:rc[2] * 16] = True
        masks.append(m)
    return scene, cams, sizes, outs, projs, b, pipe, g, camt, masks


@pytest.mark.parametrize("kind,n", [("box_rgb", 3000), ("room_sh3", 30000), ("sub_sh3", 2000)])
def test_end_to_end_forward(kind, n):
    scene, cams, sizes, outs, projs, b, pipe, g, camt, masks = _e2e(kind, n, bg=(0.2, 0.1, 0.0))
    for v, (W, H) in enumerate(sizes):
        ok = ~masks[v]
        assert ok.mean() > 0.9, ok.mean()
        rgb = _np(pipe.view_rgb(pipe.rgb, v))
        err = np.abs(rgb - outs[v]["rgb"])[:, ok].max()
        # 1e-5 plus the binary32 projection error carried into alpha
        assert err <= 2e-4, err
        assert np.median(np.abs(rgb - outs[v]["rgb"])[:, ok]) <= 1e-6
        np.testing.assert_array_equal(_np(pipe.view_plane(pipe.n_contrib, v))[ok], outs[v]["n_contrib"][ok])
        np.testing.assert_allclose(_np(pipe.view_plane(pipe.T_final, v))[ok], outs[v]["T"][ok], atol=2e-4)


@pytest.mark.parametrize("kind,n", [("box_rgb", 3000), ("sub_sh3", 2000), ("room_sh3", 20000)])
def test_end_to_end_gradients(kind, n):
    scene, cams, sizes, outs, projs, b, pipe, g, camt, masks = _e2e(kind, n)
    rs = np.random.default_rng(17)
    gC, gD, gT = [], [], []
    for v, (W, H) in enumerate(sizes):
        c = rs.normal(size=(3, H, W))
        d = rs.normal(size=(H, W)) * 0.1
        t = rs.normal(size=(H, W))
        c[:, masks[v]] = 0
        d[masks[v]] = 0
        t[masks[v]] = 0
        gC.append(c); gD.append(d); gT.append(t)
    acc, dxi, _ = oracle.backward_views(scene, cams, projs, b, gC, gD, gT)
    dev = pipe.device
    tC = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gC]).astype(np.float32)).to(dev)
    tD = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gD]).astype(np.float32)).to(dev)
    tT = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gT]).astype(np.float32)).to(dev)
    pipe.render_bwd(tC, tD, tT)
    pipe.project_bwd(g, camt, want_dxi=True)
    torch.cuda.synchronize()
    for k in acc:
        grad_close(_np(pipe.grads[k]), acc[k], k)
    grad_close(_np(pipe.dxi), dxi, "dxi")


def test_batched_views_equal_single_views():
    """One batched pipeline over uneven views gives bitwise the same images as
    one pipeline per view, and the same summed gradients."""
    scene, cams = _scene("room_sh3", 20000)
    cams = cams + [scenes.camera(*scenes.look_at([-2.0, 0.3, 1.0], [0.0, 0.0, 0.0]), 300, 300,
                                 100, 60, 200, 120)]
    sizes = [(c["W"], c["H"]) for c in cams]
    g = raster.gaussians_to_device(scene)
    n = 20000
    big = raster.Pipeline(n, sizes, 4_000_000, colour="sh", sh_degree=3,
                          tuning=dict(threads_per_tile=128, persistent=1, blocks_per_sm=0))
    camt = raster.camera_tensor(cams)
    big.forward(g, camt)
    rs = np.random.default_rng(2)
    gC = torch.from_numpy(rs.normal(size=3 * big.P).astype(np.float32)).to(big.device)
    big.render_bwd(gC)
    big.project_bwd(g, camt)
    tot = {k: torch.zeros_like(v) for k, v in big.grads.items()}
    for v, (W, H) in enumerate(sizes):
        one = raster.Pipeline(n, [sizes[v]], 4_000_000, colour="sh", sh_degree=3)
        c1 = camt[v:v + 1].contiguous()
        one.forward(g, c1)
        for name in ("rgb", "depth", "T_final", "n_contrib"):
            a = getattr(big, name)
            bview = big.view_rgb(a, v) if name == "rgb" else big.view_plane(a, v)
            ref = one.view_rgb(getattr(one, name), 0) if name == "rgb" else one.view_plane(getattr(one, name), 0)
            assert torch.equal(bview, ref), name
        p0, p1 = big.pix_base[v], big.pix_base[v + 1]
        one.render_bwd(gC[3 * p0:3 * p1].contiguous())
        one.project_bwd(g, c1)
        for k in tot:
            tot[k] += one.grads[k]
        grad_close(_np(one.dxi[0]), _np(big.dxi[v]), f"dxi view {v}")
    torch.cuda.synchronize()
    for k in tot:
        grad_close(_np(big.grads[k]), _np(tot[k]), k)


def test_empty_and_offscreen_scenes():
    cams = [scenes.identity_camera(40, 30, 50.0)]
    scene = scenes.camera_box_scene(100, 7, sh_degree=None, box=((5, 6), (5, 6), (-3, -1)))
    pipe = raster.Pipeline(100, [(40, 30)], 16)
    g = raster.gaussians_to_device(scene)
    pipe.forward(g, raster.camera_tensor(cams), bg=(0.25, 0.5, 0.75))
    torch.cuda.synchronize()
    assert int(pipe.n_dup.item()) == 0
    rgb = _np(pipe.view_rgb(pipe.rgb, 0))
    for ch, c in enumerate((0.25, 0.5, 0.75)):
        assert (rgb[ch] == np.float32(c)).all()
    assert (_np(pipe.T_final) == 1).all() and (_np(pipe.n_contrib) == 0).all()
    assert (_np(pipe.depth) == 0).all()


def _autograd_params(g):
    return [g[k].clone().requires_grad_(True) for k in ("means", "scales", "quats", "opacities", "sh")]


def _upstream(out, rs, H, W):
    """Seeded upstream gradient of one view's RGB, zero on pixels whose blend
    decisions the oracle reports within a margin of a threshold."""
    w = rs.normal(size=(3, H, W))
    w[:, out["fragile"] != 0] = 0.0
    return w.astype(np.float32)


def test_autograd_function_matches_oracle():
    """GevoRasterize forward + backward against the oracle on the 64x48 tracking
    sub-scene: every parameter gradient and the pose gradient, compared on every
    element (fragile pixels get zero upstream gradient on both sides; the scene
    has no Gaussian whose projection decision is fragile)."""
    scene, cams = _scene("sub_sh3", 2000)
    outs, projs, b = oracle.render_views(scene, cams)
    assert projs[0]["fragile"].sum() == 0
    w = _upstream(outs[0], np.random.default_rng(7), 48, 64)
    pipe = raster.Pipeline(2000, [(64, 48)], 1_000_000, colour="sh", sh_degree=3)
    g = raster.gaussians_to_device(scene)
    params = _autograd_params(g)
    twist = torch.zeros(1, 6, device=pipe.device, requires_grad=True)
    rgb, depth, T = raster.GevoRasterize.apply(*params, twist, pipe, raster.camera_tensor(cams),
                                               (0.0, 0.0, 0.0))
    (rgb * torch.from_numpy(w.reshape(-1)).cuda()).sum().backward()
    acc, dxi, _ = oracle.backward_views(scene, cams, projs, b, [w.astype(np.float64)], None, None)
    for p, k in zip(params, ("means", "scales", "quats", "opacities", "sh")):
        grad_close(_np(p.grad), acc[k], k)
    grad_close(_np(twist.grad), dxi, "dxi")


def test_autograd_two_forwards_then_two_backwards():
    """E_pc (Eq. 6) renders the current view and a past view through one
    pipeline before back-propagating both: the first forward's saved state must
    survive the second forward.  Gradients of the summed loss against the
    oracle's, and each view's pose gradient against its own."""
    scene, cams = _scene("sub_sh3", 2000)
    c0 = cams[0]
    R, t = scenes.look_at([-0.08, 0.02, 0.05], [0.0, 0.0, 5.0])
    c1 = scenes.camera(R, t, c0["fx"], c0["fy"], c0["cx"], c0["cy"], c0["W"], c0["H"])
    rs = np.random.default_rng(8)
    ws, refs = [], []
    for cam in (c0, c1):
        outs, projs, b = oracle.render_views(scene, [cam])
        assert projs[0]["fragile"].sum() == 0
        w = _upstream(outs[0], rs, 48, 64)
        ws.append(w)
        refs.append(oracle.backward_views(scene, [cam], projs, b, [w.astype(np.float64)], None, None))
    pipe = raster.Pipeline(2000, [(64, 48)], 1_000_000, colour="sh", sh_degree=3)
    g = raster.gaussians_to_device(scene)
    params = _autograd_params(g)
    twists = [torch.zeros(1, 6, device=pipe.device, requires_grad=True) for _ in range(2)]
    loss = 0.0
    for cam, w, tw in zip((c0, c1), ws, twists):
        rgb, _, _ = raster.GevoRasterize.apply(*params, tw, pipe, raster.camera_tensor([cam]),
                                               (0.0, 0.0, 0.0))
        loss = loss + (rgb * torch.from_numpy(w.reshape(-1)).cuda()).sum()
    loss.backward()
    for p, k in zip(params, ("means", "scales", "quats", "opacities", "sh")):
        grad_close(_np(p.grad), refs[0][0][k] + refs[1][0][k], k)
    for tw, ref in zip(twists, refs):
        grad_close(_np(tw.grad), ref[1], "dxi")


def test_maximum_view_count_batched_equals_single():
    """A layout with the maximum of 64 views (GEVO_MAX_VIEWS), of mixed small
    sizes: each view's image is bitwise the single-view one, and each view's
    pose gradient matches."""
    rs = np.random.default_rng(64)
    n = 3000
    scene = scenes.room_scene(n, 1064, sh_degree=1)
    cams = []
    for v in range(64):
        eye = rs.uniform(-3.0, 3.0, 3) * [1.0, 0.3, 1.0]
        W, H = (48, 32) if v % 3 else (37, 21)
        cams.append(scenes.camera(*scenes.look_at(eye, [0.0, 0.0, 0.0]), 40, 40, W / 2, H / 2, W, H))
    sizes = [(c["W"], c["H"]) for c in cams]
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    big = raster.Pipeline(n, sizes, 2_000_000, colour="sh", sh_degree=1,
                          tuning=dict(threads_per_tile=64, persistent=1, blocks_per_sm=0))
    big.forward(g, camt)
    gC = torch.from_numpy(rs.normal(size=3 * big.P).astype(np.float32)).to(big.device)
    big.render_bwd(gC)
    big.project_bwd(g, camt)
    torch.cuda.synchronize()
    assert big.last_error() == 0
    for v in (0, 1, 31, 62, 63):
        one = raster.Pipeline(n, [sizes[v]], 2_000_000, colour="sh", sh_degree=1)
        c1 = camt[v:v + 1].contiguous()
        one.forward(g, c1)
        assert torch.equal(big.view_rgb(big.rgb, v), one.view_rgb(one.rgb, 0))
        assert torch.equal(big.view_plane(big.n_contrib, v), one.view_plane(one.n_contrib, 0))
        p0, p1 = big.pix_base[v], big.pix_base[v + 1]
        one.render_bwd(gC[3 * p0:3 * p1].contiguous())
        one.project_bwd(g, c1)
        grad_close(_np(one.dxi[0]), _np(big.dxi[v]), f"dxi view {v}")
