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


def test_cost_volume_matches_oracle():
    w = scenes.workload(2, n=60_000)
    box = prior_judge.heldout_box()
    cams = prior_judge.region_poses(8, box, 99)
    rgb, _, _ = prior_judge.render_many(raster.gaussians_to_device(w["scene"]), cams, batch=8)
    H, W = prior_judge.H_IMG, prior_judge.W_IMG
    ct = raster.camera_tensor(cams)
    grey = torch.zeros(8, H // 4, W // 4, device="cuda")
    vol = torch.zeros(H // 4 * W // 4 * 64, device="cuda")
    dep = torch.zeros(H, W, device="cuda")
    ref = 3
    _abi.prior_call("gevo_cost_volume", 8, ref, H, W, rgb.contiguous(), ct, 64, 0.25, 25.0, grey, vol, dep)
    torch.cuda.synchronize()
    # the oracle sees the same binary32 images and cameras, widened to double
    V, frag = costvol.cost_volume(rgb.cpu().numpy().astype(np.float64), ct.cpu().numpy().astype(np.float64), ref)
    Vg = vol.cpu().numpy().reshape(H // 4, W // 4, 64)
    ok = ~frag
    assert ok.mean() > 0.99
    np.testing.assert_allclose(Vg[ok], V[ok], atol=2e-5, rtol=0)
    # winner-take-all where the best hypothesis is clearly ahead of the second
    srt = np.sort(V, axis=-1)
    clear = (srt[..., 1] - srt[..., 0] > 1e-4) & ~frag.any(axis=-1)
    want = costvol.wta_up4(V)[::4, ::4]
    got = dep.cpu().numpy()[::4, ::4]
    np.testing.assert_allclose(got[clear], want[clear], rtol=1e-6)


def test_prior_judge_reduced_protocol_runs_and_optimises():
    res = prior_judge.run(n=120_000, n_train=128, epochs=3, iters=15, total_new=8_000)
    for name in ("prior", "plain"):
        r = res[name]
        assert r["new_gaussians"] > 4_000
        assert np.isfinite(r["after"]["l1_rgb"]) and np.isfinite(r["after"]["l1_depth"])
        assert r["loss_last"] < r["loss_first"]
    print("judge (reduced):", res["init_depth_l1"], {k: res[k]["after"] for k in ("prior", "plain")})
