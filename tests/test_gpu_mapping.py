"""The map and pose optimisation steps of the local and global stages
(include/gevo_map.h) against the FP64 oracle (oracle/optim.py), and one
mapping update (local + global stage, insertion, active set, pruning) run end
to end.  Adam steps on identical binary32 inputs agree to binary32 rounding
(relative 2e-5 on updated parameters and moments, 1e-6 absolute on the first
moment, a sum of terms of both signs); pruning and compaction are bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import optim  # noqa: E402
from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import _abi, raster  # noqa: E402
from paper_2409_09295_gb300.mapping import DEFAULT_ADAM, GaussianMap, mapping_update  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


@pytest.mark.parametrize("K,rows_mode", [(16, "all"), (16, "list"), (1, "list")])
def test_map_step_matches_oracle(K, rows_mode):
    n = 3000
    rs = np.random.default_rng(K + len(rows_mode))
    raw = dict(means=rs.normal(size=(n, 3)), log_scales=rs.normal(-3.5, 0.6, size=(n, 3)),
               quats=rs.normal(size=(n, 4)), logit_opacities=rs.normal(size=n),
               sh=rs.normal(size=(n, K, 3)) * 0.3)
    raw = {k: v.astype(np.float32).astype(np.float64) for k, v in raw.items()}
    rows = None if rows_mode == "all" else np.sort(rs.choice(n, size=700, replace=False))
    cfg = dict(DEFAULT_ADAM, lambda_iso=3.0)
    lr = dict(means=cfg["lr_means"], log_scales=cfg["lr_log_scales"], quats=cfg["lr_quats"],
              logit_opacities=cfg["lr_logit_opacities"], sh=cfg["lr_colour_dc"], sh_rest=cfg["lr_colour_rest"])
    state = {k: (np.zeros_like(v), np.zeros_like(v)) for k, v in raw.items()}
    dev = dict(means=_t(raw["means"]), log_scales=_t(raw["log_scales"]), quats=_t(raw["quats"]),
               logit_opacities=_t(raw["logit_opacities"]), colours=_t(raw["sh"]))
    m = {k: torch.zeros_like(v) for k, v in dev.items()}
    v_ = {k: torch.zeros_like(v) for k, v in dev.items()}
    scales = torch.zeros(n, 3, device="cuda")
    opac = torch.zeros(n, device="cuda")
    _abi.gevo_map_activate(n, dev["log_scales"], dev["logit_opacities"], scales, opac)
    if rows is not None:
        rl = torch.from_numpy(rows.astype(np.int32)).cuda()
        cnt = torch.zeros(_abi.active_count_words(n), dtype=torch.int32, device="cuda")
        cnt[0] = rows.size
    else:
        rl, cnt = None, None
    iso = torch.zeros(1, device="cuda")
    for step in (1, 2, 3):
        grads = dict(means=rs.normal(size=(n, 3)), scales=rs.normal(size=(n, 3)) * 5,
                     quats=rs.normal(size=(n, 4)), opacities=rs.normal(size=n),
                     sh=rs.normal(size=(n, K, 3)))
        grads = {k: v.astype(np.float32).astype(np.float64) for k, v in grads.items()}
        gd = {k: _t(v) for k, v in grads.items()}
        if K == 1:
            gd["rgb"] = gd.pop("sh").view(n, 3)
        iso.zero_()
        _abi.gevo_map_step(n, K, dev, gd, m, v_, cfg, step, rl, cnt, scales, opac, iso)
        torch.cuda.synchronize()
        raw, state, E = optim.gaussian_step(raw, grads, state, lr, step, eps=cfg["eps"],
                                            lam_iso=cfg["lambda_iso"], rows=rows)
        assert float(iso[0]) == pytest.approx(E, rel=1e-4)
    names = dict(means="means", log_scales="log_scales", quats="quats",
                 logit_opacities="logit_opacities", sh="colours")
    for k, dk in names.items():
        np.testing.assert_allclose(_np(dev[dk]).reshape(raw[k].shape), raw[k], rtol=2e-5, atol=1e-6, err_msg=k)
        # m is a sum of terms of both signs (|g| up to ~5): binary32 rounding of
        # its terms, not of m, sets the error
        np.testing.assert_allclose(_np(m[dk]).reshape(raw[k].shape), state[k][0], rtol=2e-5, atol=1e-6, err_msg=k)
        np.testing.assert_allclose(_np(v_[dk]).reshape(raw[k].shape), state[k][1], rtol=2e-5, atol=1e-12, err_msg=k)
    idx = np.arange(n) if rows is None else rows
    np.testing.assert_allclose(_np(scales)[idx], np.exp(raw["log_scales"][idx]), rtol=2e-6)
    np.testing.assert_allclose(_np(opac)[idx], optim.sigmoid(raw["logit_opacities"][idx]), rtol=2e-6)


def test_pose_step_matches_oracle():
    V = 6
    rs = np.random.default_rng(5)
    Rs = [optim.rodrigues(rs.normal(size=3)) for _ in range(V)]
    ts = [rs.normal(size=3) for _ in range(V)]
    cams = np.zeros((V, 16), np.float32)
    for k in range(V):
        cams[k, :9] = Rs[k].reshape(-1)
        cams[k, 9:12] = ts[k]
        cams[k, 12:] = [300, 300, 160, 120]
    ct = _t(cams)
    fixed = np.array([0, 1, 0, 0, 1, 0], np.uint8)
    ft = torch.from_numpy(fixed).cuda()
    m = torch.zeros(V, 6, device="cuda")
    v = torch.zeros(V, 6, device="cuda")
    ms = [np.zeros(6) for _ in range(V)]
    vs = [np.zeros(6) for _ in range(V)]
    R = [np.asarray(cams[k, :9], np.float64).reshape(3, 3) for k in range(V)]
    t = [np.asarray(cams[k, 9:12], np.float64) for k in range(V)]
    for step in (1, 2, 3):
        dxi = (rs.normal(size=(V, 6)) * [1, 1, 1, 3, 3, 3]).astype(np.float32)
        _abi.gevo_pose_step(V, ct, _t(dxi), m, v, 1e-3, 3e-3, 0.9, 0.999, 1e-15, step, ft)
        for k in range(V):
            if fixed[k]:
                continue
            R[k], t[k], ms[k], vs[k] = optim.pose_step(R[k], t[k], dxi[k].astype(np.float64), ms[k], vs[k],
                                                       1e-3, 3e-3, step)
    torch.cuda.synchronize()
    got = _np(ct)
    for k in range(V):
        np.testing.assert_allclose(got[k, :9].reshape(3, 3), R[k], atol=2e-6)
        np.testing.assert_allclose(got[k, 9:12], t[k], atol=2e-6 * (1 + np.abs(t[k]).max()))
        if fixed[k]:
            assert (got[k] == cams[k]).all()


@pytest.mark.parametrize("n", [1, 1000, 70001, 1_200_000])
def test_prune_keep_and_gather_bit_exact(n):
    rs = np.random.default_rng(n)
    o = rs.uniform(size=n).astype(np.float32)
    o[::13] = np.float32(0.7)              # exactly at the threshold: kept
    cand = rs.uniform(size=n) < 0.3
    words = np.zeros((n + 31) // 32, np.uint64)
    idx = np.nonzero(cand)[0]
    np.add.at(words, idx // 32, np.uint64(1) << (idx % 32).astype(np.uint64))
    # the decision is taken in binary32 on both sides: threshold 0.7f
    keep_ref = optim.keep_after_pruning(o.astype(np.float64), idx, float(np.float32(0.7)))
    keep = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
    lst = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(_abi.active_count_words(n), dtype=torch.int32, device="cuda")
    _abi.gevo_prune_keep(n, _t(o), torch.from_numpy(words.astype(np.uint32).view(np.int32)).cuda(), 0.7,
                         keep, lst, cnt)
    torch.cuda.synchronize()
    k = int(_np(cnt)[0])
    assert k == keep_ref.size
    np.testing.assert_array_equal(_np(lst)[:k], keep_ref)
    src = rs.normal(size=(n, 5)).astype(np.float32)
    dst = torch.zeros(n, 5, device="cuda")
    _abi.gevo_gather_rows(n, lst, cnt, 5, _t(src), dst)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(dst)[:k], src[keep_ref])


def test_mapping_update_local_and_global_stage():
    from paper_2409_09295_gb300 import prior_judge
    w = scenes.workload(2, n=120_000)
    box = prior_judge.heldout_box()
    kept, n_out = prior_judge.split_scene(w["scene"], box)
    world = raster.gaussians_to_device(w["scene"])
    wins, _, _ = prior_judge.window_poses(4, box, 11)
    rgb, _, _ = prior_judge.render_many(world, wins, batch=4)
    images = rgb.reshape(-1).contiguous()
    # the new Gaussians: the held-out ones, displaced and recoloured (a noisy
    # initialisation to be refined)
    m_in = np.all((w["scene"]["means"] >= box[:, 0]) & (w["scene"]["means"] <= box[:, 1]), axis=1)
    rs = np.random.default_rng(3)
    new = {k: (v[m_in].copy() if isinstance(v, np.ndarray) else v) for k, v in w["scene"].items()}
    new["means"] = new["means"] + rs.normal(0, 0.03, size=new["means"].shape).astype(np.float32)
    new["sh"] = new["sh"] + rs.normal(0, 0.3, size=new["sh"].shape).astype(np.float32)
    new["opacities"] = np.full_like(new["opacities"], 0.9)
    gmap = GaussianMap(kept)
    local = GaussianMap(new)
    n0 = gmap.n
    past = prior_judge.random_poses(4, 12)
    rep = mapping_update(gmap, local, wins, images, past, local_iters=12, global_iters=12, eps=0.05)
    ll, gl = rep["local_losses"], rep["global_losses"]
    assert ll[-1] < ll[0], ll
    assert gl[-1] < gl[0], gl
    assert rep["active"] >= local.n
    assert rep["map_size"] == n0 + local.n - rep["pruned"]
    assert 0 < rep["pruned"] <= rep["active"]
    # the kept Gaussians' opacities are all that pruning allows among the inserted
    assert np.isfinite(_np(gmap.opacities)).all()
