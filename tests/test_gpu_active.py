"""Parity of the active-set path of the global stage (Section III-B2) with the
FP64 oracle: the per-pixel error, the per-Gaussian rendering error E_k(g) of
Eq. 5 fused into the reverse walk, the active set (bit-exact), and the masked
reverse walk and projection backward (gradient tolerance: relative L2 <= 1e-3 per tensor, |g - ref| <= 1e-3 |ref| + 1e-3 rms(ref) per
element; rows of inactive Gaussians untouched, bit for bit).

E_k(g) = sum_u w(g, u) e(u) is a weighted sum of exactly the kind the colour
gradient is (dC/dc_g = w(g, u)), so it takes the gradient tolerance.  Every
input is seeded; no oracle input comes from the CUDA path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from gpu_helpers import grad_close, records_for_oracle, tiles_of, upload_records  # noqa: E402
from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import raster  # noqa: E402

TUNINGS = [dict(threads_per_tile=256, persistent=0, blocks_per_sm=0),
           dict(threads_per_tile=64, persistent=1, blocks_per_sm=0),
           dict(threads_per_tile=32, persistent=1, blocks_per_sm=0)]


def _np(t):
    return t.detach().cpu().numpy()


def _bits(mask):
    """Boolean mask -> uint32 words, bit g % 32 of word g // 32."""
    n = mask.size
    w = np.zeros((n + 31) // 32, np.uint64)
    idx = np.nonzero(mask)[0]
    np.add.at(w, idx // 32, (np.uint64(1) << (idx % 32).astype(np.uint64)))
    return w.astype(np.uint32)


def _staged(sizes, n, seed):
    rec = scenes.random_records(sizes, n, seed=seed, sigma_px=(0.5, 12.0))
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    pipe = raster.Pipeline(n, sizes, b["n_dup"] + 16)
    upload_records(pipe, rec)
    pipe.bin_sort()
    return rec, b, pipe


def _fragile_free_inputs(rec, b, pipe, sizes, bg, seed):
    """Seeded per-pixel errors and upstream gradients, zero on pixels whose blend
    decisions the oracle flags as within a margin of a threshold."""
    rs = np.random.default_rng(seed)
    pe = rs.uniform(0.0, 1.0, size=pipe.P)
    gC = rs.normal(size=3 * pipe.P)
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg)
        fr = o["fragile"].reshape(-1) != 0
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        pe[p0:p1][fr] = 0.0
        for ch in range(3):
            gC[3 * p0 + ch * (p1 - p0):3 * p0 + (ch + 1) * (p1 - p0)][fr] = 0.0
        base += nt
    return pe.astype(np.float32), gC.astype(np.float32)


# --------------------------------------------------------------------------
# per-pixel error (fused into the L1 loss)
# --------------------------------------------------------------------------
def test_loss_l1_err_matches_loss_and_pixel_error():
    sizes = [(64, 48), (33, 17)]
    pipe = raster.Pipeline(1, sizes, 1)
    rs = np.random.default_rng(3)
    a = rs.uniform(size=3 * pipe.P).astype(np.float32)
    b = rs.uniform(size=3 * pipe.P).astype(np.float32)
    b[:50] = a[:50]
    d = rs.uniform(1, 5, size=pipe.P).astype(np.float32)
    e = rs.uniform(1, 5, size=pipe.P).astype(np.float32)
    dev = pipe.device
    pipe.rgb.copy_(torch.from_numpy(a).to(dev))
    pipe.depth.copy_(torch.from_numpy(d).to(dev))
    pipe.loss_l1_err(torch.from_numpy(b).to(dev), torch.from_numpy(e).to(dev), 0.7)
    torch.cuda.synchronize()
    rgbs = [a[3 * pipe.pix_base[v]:3 * pipe.pix_base[v + 1]].reshape(3, h, w) for v, (w, h) in enumerate(sizes)]
    trg = [b[3 * pipe.pix_base[v]:3 * pipe.pix_base[v + 1]].reshape(3, h, w) for v, (w, h) in enumerate(sizes)]
    ds = [d[pipe.pix_base[v]:pipe.pix_base[v + 1]].reshape(h, w) for v, (w, h) in enumerate(sizes)]
    es = [e[pipe.pix_base[v]:pipe.pix_base[v + 1]].reshape(h, w) for v, (w, h) in enumerate(sizes)]
    L, gC, gD = oracle.loss_l1(rgbs, trg, ds, es, 0.7)
    assert float(_np(pipe.loss).sum()) == pytest.approx(L, rel=1e-5)
    np.testing.assert_allclose(_np(pipe.dL_drgb), np.concatenate([x.reshape(-1) for x in gC]), rtol=1e-6, atol=0)
    np.testing.assert_allclose(_np(pipe.dL_ddepth), np.concatenate([x.reshape(-1) for x in gD]), rtol=1e-6, atol=0)
    want = np.concatenate([oracle.pixel_error(rgbs[v], trg[v]).reshape(-1) for v in range(len(sizes))])
    # three binary32 differences (exact: Sterbenz for values in [0, 1] within 2x,
    # else one rounding), a sum of three and a product by 1/3: a few ulps
    np.testing.assert_allclose(_np(pipe.pix_err), want, rtol=3e-7, atol=1e-8)


# --------------------------------------------------------------------------
# E_k(g) fused into the reverse walk, on identical binary32 records
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tuning", TUNINGS, ids=["ppt1", "ppt4_persistent", "ppt8_persistent"])
def test_gauss_err_staged(tuning):
    sizes = [(96, 80), (53, 37)]
    n = 2500
    bg = (0.1, 0.2, 0.3)
    rec, b, pipe = _staged(sizes, n, seed=60)
    pipe.render_fwd(bg, tuning=tuning)
    pe, gC = _fragile_free_inputs(rec, b, pipe, sizes, bg, seed=61)
    pipe.alloc_active()
    pipe.pix_err.copy_(torch.from_numpy(pe).to(pipe.device))
    pipe.render_bwd_active(torch.from_numpy(gC).to(pipe.device), bg=bg, error=True, masked=False,
                           tuning=tuning)
    torch.cuda.synchronize()
    E = _np(pipe.gauss_err).reshape(len(sizes), n)
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg,
                              pix_err=pe[p0:p1].reshape(H, W))
        base += nt
        assert (o["gauss_err"] > 0).sum() > 100
        grad_close(E[v], o["gauss_err"], f"v{v} E_k")
        # culled entries are never touched
        assert (E[v][rec["radius"][v] == 0] == 0).all()


# --------------------------------------------------------------------------
# masked reverse walk: active rows as the full walk, inactive rows untouched
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tuning", TUNINGS, ids=["ppt1", "ppt4_persistent", "ppt8_persistent"])
@pytest.mark.parametrize("frac", [0.15, 0.0, 1.0])
def test_masked_reverse_walk_staged(tuning, frac):
    sizes = [(96, 80), (53, 37)]
    n = 2000
    bg = (0.0, 0.0, 0.0)
    rec, b, pipe = _staged(sizes, n, seed=70)
    pipe.render_fwd(bg, tuning=tuning)
    pe, gC = _fragile_free_inputs(rec, b, pipe, sizes, bg, seed=71)
    act = np.random.default_rng(72).uniform(size=n) < frac
    pipe.alloc_active()
    pipe.active.copy_(torch.from_numpy(_bits(act).view(np.int32)).to(pipe.device))
    pipe.pix_err.copy_(torch.from_numpy(pe).to(pipe.device))
    pipe.render_bwd_active(torch.from_numpy(gC).to(pipe.device), bg=bg, error=True, masked=True,
                           tuning=tuning)
    torch.cuda.synchronize()
    E = _np(pipe.gauss_err).reshape(len(sizes), n)
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        r = records_for_oracle(rec, v)
        rv = b["ranges"][base:base + nt]
        base += nt
        g = oracle.mask_grad2d(oracle.render_bwd(W, H, r, b["vals"], rv, gC[3 * p0:3 * p1].reshape(3, H, W),
                                                 None, None, bg), act)
        o = oracle.render_fwd(W, H, r, b["vals"], rv, bg, pix_err=pe[p0:p1].reshape(H, W))
        # the error pass covers every Gaussian, active or not
        grad_close(E[v], o["gauss_err"], f"v{v} E_k")
        sl = slice(v * n, (v + 1) * n)
        gxy = _np(pipe.grad2d["xy"])[sl]
        gco = _np(pipe.grad2d["conic_opacity"])[sl]
        grz = _np(pipe.grad2d["rgb_depth"])[sl]
        vis = rec["radius"][v] > 0
        a = vis & act
        if a.any():
            grad_close(gxy[a], g["xy"][a], f"v{v} dxy")
            grad_close(gco[a, :3], g["conic"][a], f"v{v} dconic")
            grad_close(gco[a, 3], g["opacity"][a], f"v{v} dopacity")
            grad_close(grz[a, :3], g["rgb"][a], f"v{v} drgb")
        # zeroed by gevo_grad2d_zero, never written by the masked walk
        assert (gxy[vis & ~act] == 0).all() and (gco[vis & ~act] == 0).all() and (grz[vis & ~act] == 0).all()


# --------------------------------------------------------------------------
# the forward pass that records where an active-set walk starts, and the walk
# from there
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tuning", TUNINGS, ids=["ppt1", "ppt4_persistent", "ppt8_persistent"])
def test_render_fwd_active_state(tuning):
    sizes = [(96, 80), (53, 37)]
    n = 2500
    bg = (0.1, 0.2, 0.3)
    rec, b, pipe = _staged(sizes, n, seed=80)
    act = np.random.default_rng(81).uniform(size=n) < 0.15
    pipe.render_fwd(bg, tuning=tuning)
    plain = {k: _np(getattr(pipe, k)).copy() for k in ("rgb", "depth", "T_final", "n_contrib")}
    pipe.alloc_active()
    pipe.active.copy_(torch.from_numpy(_bits(act).view(np.int32)).to(pipe.device))
    pipe.render_fwd_active(bg, tuning=tuning)
    torch.cuda.synchronize()
    # same decisions bit for bit; the colour is summed in two parts (up to the
    # last active entry and since), so it may differ in the last bits
    for k in ("T_final", "n_contrib"):
        np.testing.assert_array_equal(_np(getattr(pipe, k)), plain[k], err_msg=k)
    np.testing.assert_allclose(_np(pipe.rgb), plain["rgb"], atol=1e-6, rtol=0)
    np.testing.assert_allclose(_np(pipe.depth), plain["depth"], atol=1e-5, rtol=1e-6)
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg,
                              active=act)
        base += nt
        ok = o["fragile"] == 0
        la = _np(pipe.view_plane(pipe.act_state["last"], v))
        np.testing.assert_array_equal(la[ok], o["act_last"][ok])
        assert (la[ok] > 0).mean() > 0.3
        Ta = _np(pipe.view_plane(pipe.act_state["T"], v))
        np.testing.assert_allclose(Ta[ok], o["act_T"][ok], atol=1e-5, rtol=0)
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        rest = _np(pipe.act_state["rest"])[p0:p1].reshape(H, W, 4)
        np.testing.assert_allclose(rest[ok], o["act_rest"][ok], atol=1e-5, rtol=0)


@pytest.mark.parametrize("tuning", TUNINGS, ids=["ppt1", "ppt4_persistent", "ppt8_persistent"])
@pytest.mark.parametrize("frac", [0.15, 0.0, 1.0])
def test_masked_walk_from_forward_state(tuning, frac):
    sizes = [(96, 80), (53, 37)]
    n = 2000
    bg = (0.2, 0.1, 0.4)
    rec, b, pipe = _staged(sizes, n, seed=90)
    act = np.random.default_rng(91).uniform(size=n) < frac
    pipe.alloc_active()
    pipe.active.copy_(torch.from_numpy(_bits(act).view(np.int32)).to(pipe.device))
    pipe.render_fwd_active(bg, tuning=tuning)
    pe, gC = _fragile_free_inputs(rec, b, pipe, sizes, bg, seed=92)
    gD = np.random.default_rng(93).normal(size=pipe.P).astype(np.float32)
    gT = np.random.default_rng(94).normal(size=pipe.P).astype(np.float32)
    base = 0
    for v, (W, H) in enumerate(sizes):         # fragile pixels carry no gradient
        nt = tiles_of(W, H)
        o = oracle.render_fwd(W, H, records_for_oracle(rec, v), b["vals"], b["ranges"][base:base + nt], bg)
        fr = o["fragile"].reshape(-1) != 0
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        gD[p0:p1][fr] = 0.0
        gT[p0:p1][fr] = 0.0
        base += nt
    dev = pipe.device
    tC, tD, tT = (torch.from_numpy(x).to(dev) for x in (gC, gD, gT))
    pipe.render_bwd_active(tC, tD, tT, bg=bg, error=False, masked=True, tuning=tuning, from_state=True)
    torch.cuda.synchronize()
    base = 0
    for v, (W, H) in enumerate(sizes):
        nt = tiles_of(W, H)
        p0, p1 = pipe.pix_base[v], pipe.pix_base[v + 1]
        g = oracle.mask_grad2d(oracle.render_bwd(W, H, records_for_oracle(rec, v), b["vals"],
                                                 b["ranges"][base:base + nt],
                                                 gC[3 * p0:3 * p1].reshape(3, H, W), gD[p0:p1].reshape(H, W),
                                                 gT[p0:p1].reshape(H, W), bg), act)
        base += nt
        sl = slice(v * n, (v + 1) * n)
        gxy = _np(pipe.grad2d["xy"])[sl]
        gco = _np(pipe.grad2d["conic_opacity"])[sl]
        grz = _np(pipe.grad2d["rgb_depth"])[sl]
        vis = rec["radius"][v] > 0
        a = vis & act
        if a.any():
            grad_close(gxy[a], g["xy"][a], f"v{v} dxy")
            grad_close(gco[a, :3], g["conic"][a], f"v{v} dconic")
            grad_close(gco[a, 3], g["opacity"][a], f"v{v} dopacity")
            grad_close(grz[a, :3], g["rgb"][a], f"v{v} drgb")
            grad_close(grz[a, 3], g["depth"][a], f"v{v} ddepth")
        assert (gxy[vis & ~act] == 0).all() and (gco[vis & ~act] == 0).all() and (grz[vis & ~act] == 0).all()


# --------------------------------------------------------------------------
# active set: bit mask, ascending list and count, bit-exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 31, 32, 1000, 1025, 70001, 2_500_000])
def test_active_set_bit_exact(n):
    V = 3
    rs = np.random.default_rng(n)
    E = rs.exponential(1.0, size=(V, n)).astype(np.float32)
    eps = np.float32(2.5)
    E[0, ::97] = eps          # exactly at the threshold: not active (strict)
    force = rs.uniform(size=n) < 0.02
    act, lst = oracle.active_set(E.astype(np.float64), float(eps), force)
    pipe = raster.Pipeline(n, [(16, 16)] * V, 1)
    pipe.alloc_active()
    dev = pipe.device
    pipe.gauss_err.copy_(torch.from_numpy(E.reshape(-1)).to(dev))
    fb = torch.from_numpy(_bits(force).view(np.int32)).to(dev)
    pipe.active.fill_(-1)
    pipe.active_list.fill_(-1)
    pipe.active_set(float(eps), fb)
    torch.cuda.synchronize()
    cnt = int(_np(pipe.active_counts)[0])
    assert cnt == lst.size
    np.testing.assert_array_equal(_np(pipe.active).view(np.uint32), _bits(act))
    np.testing.assert_array_equal(_np(pipe.active_list)[:cnt].view(np.uint32), lst)


def test_active_set_empty_and_none_active():
    pipe = raster.Pipeline(0, [(16, 16)], 1)
    pipe.alloc_active()
    pipe.active_counts.fill_(7)
    pipe.active_set(0.5)
    torch.cuda.synchronize()
    assert int(_np(pipe.active_counts)[0]) == 0
    pipe = raster.Pipeline(5000, [(16, 16)], 1)
    pipe.alloc_active()
    pipe.active_set(1e30)
    torch.cuda.synchronize()
    assert int(_np(pipe.active_counts)[0]) == 0
    assert (_np(pipe.active) == 0).all()


# --------------------------------------------------------------------------
# masked projection backward on the listed Gaussians
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n", [("box_rgb", 3000), ("room_sh3", 20000)])
def test_project_bwd_active_parity(kind, n):
    if kind == "box_rgb":
        w = scenes.workload(0, n=n)
        scene, cams = w["scene"], w["cams"]
    else:
        w = scenes.workload(1, n=n)
        c = w["cams"][0]
        cams = [c, scenes.camera(*scenes.look_at([1.0, 0.5, -3.0], [0.0, 0.0, 0.0]), 262.5, 262.5,
                                 160, 120, 320, 240)]
        scene = w["scene"]
    sizes = [(c["W"], c["H"]) for c in cams]
    colour = "rgb" if "rgb" in scene else "sh"
    pipe = raster.Pipeline(n, sizes, 1, colour=colour, sh_degree=scene["sh_degree"])
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    pipe.project(g, camt)
    rs = np.random.default_rng(19)
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
    E = rs.exponential(1.0, size=(V, n)).astype(np.float32)
    eps = float(np.quantile(E.max(axis=0), 0.85))
    act, lst = oracle.active_set(E.astype(np.float64), eps)
    dev = pipe.device
    pipe.alloc_active()
    pipe.gauss_err.copy_(torch.from_numpy(E.reshape(-1)).to(dev))
    pipe.active_set(eps)
    pipe.grad2d["xy"].copy_(torch.from_numpy(gxy.reshape(V * n, 2)).to(dev))
    pipe.grad2d["conic_opacity"].copy_(torch.from_numpy(gco.reshape(V * n, 4)).to(dev))
    pipe.grad2d["rgb_depth"].copy_(torch.from_numpy(grz.reshape(V * n, 4)).to(dev))
    for t in pipe.grads.values():
        t.fill_(7.0)
    pipe.project_bwd_active(g, camt, want_dxi=True)
    torch.cuda.synchronize()
    assert int(_np(pipe.active_counts)[0]) == lst.size
    acc = oracle.grads_like(scene)
    dxi = np.zeros((V, 6))
    for v, cam in enumerate(cams):
        g2d = oracle.mask_grad2d(dict(xy=gxy[v], conic=gco[v][:, :3], opacity=gco[v][:, 3],
                                      rgb=grz[v][:, :3], depth=grz[v][:, 3]), act)
        rad = np.where(projs[v]["fragile"] != 0, 0, projs[v]["radius"])
        oracle.project_bwd(scene, cam, rad, g2d, acc, dxi[v])
    for k in acc:
        got = _np(pipe.grads[k])
        grad_close(got[act], acc[k][act], k)
        assert (got[~act] == 7.0).all(), k
    grad_close(_np(pipe.dxi), dxi, "dxi")


# --------------------------------------------------------------------------
# end to end: render, per-pixel error, E_k, active set, masked backward
# --------------------------------------------------------------------------
def test_active_chain_end_to_end():
    n = 2000
    scene, cams = scenes.tracking_subscene(n)
    sizes = [(c["W"], c["H"]) for c in cams]
    outs, projs, b = oracle.render_views(scene, cams)
    pipe = raster.Pipeline(n, sizes, b["n_dup"] * 2 + 1024, colour="sh", sh_degree=scene["sh_degree"])
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    pipe.forward(g, camt)
    rs = np.random.default_rng(23)
    target = [rs.uniform(size=(3, H, W)) for (W, H) in sizes]
    tt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in target]).astype(np.float32)).to(pipe.device)
    pipe.loss_l1_err(tt)
    torch.cuda.synchronize()
    # pixels and tiles whose discrete decisions are fragile carry no error
    pe_ref, masks = [], []
    for v, (W, H) in enumerate(sizes):
        m = outs[v]["fragile"] != 0
        p = projs[v]
        rad_g = _np(pipe.proj["radius"])[v * n:(v + 1) * n]
        tt_g = _np(pipe.proj["tiles_touched"])[v * n:(v + 1) * n]
        differs = (p["fragile"] != 0) & ((rad_g != p["radius"]) | (tt_g != p["tiles_touched"]))
        for i in np.nonzero(differs)[0]:
            r = max(int(p["radius"][i]), int(rad_g[i]), 1)
            rc = oracle.rect_f32(p["xy"][i, 0], p["xy"][i, 1], r, (W + 15) // 16, (H + 15) // 16)
            m[rc[1] * 16:rc[3] * 16, rc[0] * 16:rc[2] * 16] = True
        masks.append(m)
        e = oracle.pixel_error(outs[v]["rgb"], target[v].astype(np.float32))
        got = _np(pipe.view_plane(pipe.pix_err, v))
        assert np.abs(got - e)[~m].max() <= 2e-4
        pe_ref.append(np.where(m, 0.0, e))
    # the walk gets the oracle's per-pixel error (an input to this stage)
    pipe.pix_err.copy_(torch.from_numpy(np.concatenate([p.reshape(-1) for p in pe_ref]).astype(np.float32)).to(pipe.device))
    gC = [np.where(masks[v][None], 0.0, rs.normal(size=(3, H, W))) for v, (W, H) in enumerate(sizes)]
    tC = torch.from_numpy(np.concatenate([x.reshape(-1) for x in gC]).astype(np.float32)).to(pipe.device)
    pipe.render_bwd_active(tC, error=True, masked=False)
    torch.cuda.synchronize()
    E = _np(pipe.gauss_err).reshape(len(sizes), n)
    o2, _, _ = oracle.render_views(scene, cams, pix_errs=pe_ref)
    Eref = np.stack([o2[v]["gauss_err"] for v in range(len(sizes))])
    grad_close(E, Eref, "E_k")
    # a threshold near the 85th percentile that no Gaussian's error lies within
    # 2% of, so both sides take the same decisions; then the masked backward
    m = np.sort(Eref.max(axis=0))
    i = int(0.85 * n)
    while m[i + 1] <= 1.02 * m[i] + 1e-6:
        i += 1
    eps = 0.5 * (m[i] + m[i + 1])
    act, lst = oracle.active_set(Eref, eps)
    pipe.active_set(eps)
    pipe.render_bwd_active(tC, error=False, masked=True)
    pipe.project_bwd_active(g, camt)
    torch.cuda.synchronize()
    full_walk = {k: _np(t).copy() for k, t in pipe.grads.items()}, _np(pipe.dxi).copy()
    # the specialised path: forward records the walk's start, the walk skips
    # everything behind each pixel's last active entry
    pipe.render_fwd_active()
    pipe.render_bwd_active(tC, error=False, masked=True, from_state=True)
    pipe.project_bwd_active(g, camt)
    torch.cuda.synchronize()
    assert int(_np(pipe.active_counts)[0]) == lst.size and 0 < lst.size < n
    np.testing.assert_array_equal(_np(pipe.active_list)[:lst.size].view(np.uint32), lst)
    acc = oracle.grads_like(scene)
    dxi = np.zeros((len(sizes), 6))
    _, _, g2ds = oracle.backward_views(scene, cams, projs, b, gC, want_dxi=False)
    for v, cam in enumerate(cams):
        oracle.project_bwd(scene, cam, projs[v]["radius"], oracle.mask_grad2d(g2ds[v], act), acc, dxi[v])
    for k in acc:
        grad_close(_np(pipe.grads[k])[act], acc[k][act], k)
        grad_close(full_walk[0][k][act], acc[k][act], k + " (whole lists)")
    grad_close(_np(pipe.dxi), dxi, "dxi")
    grad_close(full_walk[1], dxi, "dxi (whole lists)")
