"""The plain initialisation's cost volume (Eq. 1) on the GPU against the FP64
oracle, and a reduced run of the learned-prior judge protocol."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import costvol  # noqa: E402
from paper_2409_09295_gb300 import _abi, prior_judge, raster, scenes  # noqa: E402


def _plane_keyframes(nk=8, H=240, W=320, d_star=3.37):
    """nk keyframes 0.1 m apart, slightly rotated, looking at a textured plane."""
    cams = np.zeros((nk, 16))
    rs = np.random.default_rng(4)
    for i in range(nk):
        phi = rs.normal(0, 0.02, size=3)
        th = np.linalg.norm(phi)
        K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
        R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
        cams[i, :9] = R.reshape(9)
        cams[i, 9:12] = [-0.1 * (i - nk / 2), 0.03 * np.sin(i), 0.0]
        cams[i, 12:16] = [262.5, 262.5, W / 2, H / 2]
    return scenes.plane_images(d_star, cams, H, W, seed=9), cams.astype(np.float32)


def test_cost_volume_matches_oracle():
    H, W, nk, ref = 240, 320, 8, 7
    rgb, cams = _plane_keyframes(nk, H, W)
    grey = torch.zeros(nk, H // 4, W // 4, device="cuda")
    vol = torch.zeros(H // 4 * W // 4 * 64, device="cuda")
    dep = torch.zeros(H, W, device="cuda")
    _abi.prior_call("gevo_cost_volume", nk, ref, H, W, torch.from_numpy(rgb).cuda(),
                    torch.from_numpy(cams).cuda(), 64, 0.25, 25.0, grey, vol, dep)
    torch.cuda.synchronize()
    # both sides see the same binary32 images and cameras
    V, frag = costvol.cost_volume(rgb.astype(np.float64), cams.astype(np.float64), ref)
    Vg = vol.cpu().numpy().reshape(H // 4, W // 4, 64)
    ok = ~frag
    assert ok.mean() > 0.99
    np.testing.assert_allclose(Vg[ok], V[ok], atol=2e-5, rtol=0)
    # winner-take-all where the best hypothesis is clearly ahead of the second
    srt = np.sort(V, axis=-1)
    clear = (srt[..., 1] - srt[..., 0] > 1e-4) & ~frag.any(axis=-1)
    assert clear.mean() > 0.5
    want = costvol.wta_up4(V)[::4, ::4]
    got = dep.cpu().numpy()[::4, ::4]
    np.testing.assert_allclose(got[clear], want[clear], rtol=1e-6)


def _bp_gpu(V, s, tau, iters):
    h, w, nd = V.shape
    vol = torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda()
    msgs = torch.zeros(2 * 4 * h * w * nd, device="cuda")
    depth = torch.zeros(4 * h, 4 * w, device="cuda")
    labels = torch.zeros(h, w, dtype=torch.int32, device="cuda")
    beliefs = torch.zeros(h, w, nd, device="cuda")
    _abi.prior_call("gevo_depth_bp", h, w, nd, vol, s, tau, iters, 0.25, 25.0, msgs, depth, labels,
                    beliefs)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), beliefs.cpu().numpy(), depth.cpu().numpy()


@pytest.mark.parametrize("shape,s,tau,iters", [((30, 40, 64), 0.05, 0.5, 8), ((17, 23, 37), 0.2, 1.0, 12),
                                               ((1, 50, 64), 0.1, 0.8, 60)])
def test_belief_propagation_matches_oracle(shape, s, tau, iters):
    rs = np.random.default_rng(shape[0] * 7 + iters)
    h, w, nd = shape
    # smooth depth structure plus noise: a ramp of true labels, 10% scrambled pixels
    true = (np.add.outer(np.arange(h), np.arange(w)) * nd // (h + w + 1))
    V = 0.03 * np.abs(np.arange(nd)[None, None, :] - true[..., None]) + rs.uniform(0, 0.05, size=shape)
    bad = rs.uniform(size=(h, w)) < 0.1
    V[bad] = rs.uniform(size=(bad.sum(), nd))
    V = V.astype(np.float32)
    lab, B, depth = _bp_gpu(V, s, tau, iters)
    lab_ref, B_ref, _ = costvol.bp(V.astype(np.float64), s, tau, iters)
    # beliefs: sums of up to 4 iters-deep message chains of binary32 terms
    np.testing.assert_allclose(B, B_ref, atol=2e-4 * (1 + iters * s), rtol=1e-5)
    srt = np.sort(B_ref, axis=-1)
    clear = srt[..., 1] - srt[..., 0] > 1e-3
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(lab[clear], lab_ref[clear])
    np.testing.assert_allclose(depth[::4, ::4], 0.25 + 24.75 * lab / (nd - 1), rtol=1e-6)


def test_belief_propagation_on_the_plane_cost_volume():
    H, W, nk, ref = 240, 320, 8, 7
    rgb, cams = _plane_keyframes(nk, H, W)
    V, frag = costvol.cost_volume(rgb.astype(np.float64), cams.astype(np.float64), ref)
    lab, B, _ = _bp_gpu(V, 0.01, 0.1, 10)
    lab_ref, B_ref, _ = costvol.bp(V.astype(np.float32).astype(np.float64), 0.01, 0.1, 10)
    srt = np.sort(B_ref, axis=-1)
    clear = srt[..., 1] - srt[..., 0] > 1e-3
    assert clear.mean() > 0.5
    np.testing.assert_array_equal(lab[clear], lab_ref[clear])


def test_prior_judge_depth_gain_at_equal_iterations():
    """The learned prior against the plain initialisation (Eq. 1 + belief
    propagation) on the 500k room with a 50k-Gaussian box held out, both
    optimised by the same 100 local-stage iterations (Eq. 2).  What the trained
    network gains: its depths start ~50x closer to the truth, and after the
    optimisation its new Gaussians' depth error is still below plain's, over
    all covered new-region pixels and over the pixels both cover.  Its colour
    error after the optimisation is higher than plain's (the synthetic room is a
    volume of small random splats: splats from eight keyframes at the true depth
    land on top of one another and cover fewer test pixels than plain's
    scattered ones); the test records it without asserting an order."""
    res = prior_judge.run()
    assert res["train"]["losses"][-1] < 0.15, res["train"]["losses"]   # left the plateau
    ini = res["init_depth_l1"]
    assert ini["prior"] < 0.1 * ini["plain"], ini
    for name in ("prior", "plain"):
        r = res[name]
        assert r["new_gaussians"] >= 40_000
        assert r["loss_last"] < 0.5 * r["loss_first"]
        assert np.isfinite(r["after"]["l1_rgb"])
    assert res["prior"]["after"]["l1_depth"] < res["plain"]["after"]["l1_depth"]
    c = res["common"]
    assert c["pixels"] > 100_000
    assert c["l1_depth"]["prior"] < c["l1_depth"]["plain"], c
    print("judge:", ini, {k: res[k]["after"] for k in ("prior", "plain")}, c)
