"""The single-view workloads at their stated sizes against the FP64 oracle
(split across host threads): 20k Gaussians at 320x240 with RGB colours and an
L1 photometric loss; 200k SH-3 Gaussians at 640x480 with L1 photometric + L1
depth loss; 1M SH-3 Gaussians at 1200x680 (the Replica image size of
Section IV-B) with the photometric loss and the pose gradient of tracking.

Targets are the oracle's renders of the same scene with means jittered by
N(0, 0.01 m) (the stop-gradient previous map of Eq. 6).  Checks:
  - images (RGB, depth, T_final) and contributor counts on every pixel no
    fragile decision touches (2e-4 maximum, 1e-6 median; counts bit-exact);
  - the loss value of the GPU's L1 kernel against the oracle's loss, and its
    per-pixel gradient sign(C - C*)/count equal wherever |C - C*| > 1e-3;
  - the oracle's loss gradient (fragile pixels and pixels with |C - C*| <=
    1e-3 set to zero) fed to both sides' backward: record gradients, every
    parameter gradient and the se(3) pose gradient (relative L2 <= 1e-3 and
    |g - ref| <= 1e-3 |ref| + 1e-3 rms(ref); rows of Gaussians whose projection
    decision the oracle reports within its margin -- a clamp or cull that
    binary32 may take the other way -- only in the relative L2 check)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import oracle_par  # noqa: E402
from gpu_helpers import check_view_images, excluded_pixels, grad_close  # noqa: E402
from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import raster  # noqa: E402


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("index", [0, 1, 3])
def test_workload_at_stated_size(index):
    w = scenes.workload(index)
    scene, cams, lam = w["scene"], w["cams"], float(w["lambda_depth"])
    cam = cams[0]
    W, H = cam["W"], cam["H"]
    n = scene["means"].shape[0]
    tgt_outs, _, _ = oracle_par.render_views(w["target_scene"], cams)
    outs, projs, b = oracle_par.render_views(scene, cams)

    colour = "rgb" if scene.get("rgb") is not None else "sh"
    pipe = raster.Pipeline(n, [(W, H)], 1 << 20, colour=colour,
                           sh_degree=scene.get("sh_degree", 0))
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams)
    pipe.ensure_capacity(g, camt)
    pipe.forward(g, camt)
    torch.cuda.synchronize()
    assert pipe.last_error() == 0
    excl = excluded_pixels(pipe, n, cams, [0], outs, projs)[0]
    check_view_images(pipe, 0, outs[0], excl)

    # L1 loss on the GPU against the oracle's targets
    t_rgb = torch.from_numpy(tgt_outs[0]["rgb"].astype(np.float32).reshape(-1)).cuda()
    t_dep = torch.from_numpy(tgt_outs[0]["depth"].astype(np.float32).reshape(-1)).cuda()
    pipe.loss_l1(t_rgb, t_dep, lam)
    L, gC, gD = oracle.loss_l1([outs[0]["rgb"]], [tgt_outs[0]["rgb"]], [outs[0]["depth"]],
                               [tgt_outs[0]["depth"]], lambda_depth=lam)
    torch.cuda.synchronize()
    # |mean|a - t| - mean|b - t|| <= mean|a - b|: the two losses differ by at most
    # the mean image difference (plus binary32 summation error)
    bound = np.abs(_np(pipe.view_rgb(pipe.rgb, 0)) - outs[0]["rgb"]).mean()
    if lam:
        bound += lam * np.abs(_np(pipe.view_plane(pipe.depth, 0)) - outs[0]["depth"]).mean()
    assert abs(float(pipe.loss.sum()) - L) <= bound + 1e-6 * max(1.0, abs(L))
    d_rgb = np.abs(outs[0]["rgb"] - tgt_outs[0]["rgb"])
    sure = (d_rgb > 1e-3) & ~excl[None]
    np.testing.assert_allclose(_np(pipe.view_rgb(pipe.dL_drgb, 0))[sure], gC[0][sure], rtol=1e-6)
    if lam:
        d_dep = np.abs(outs[0]["depth"] - tgt_outs[0]["depth"])
        sure_d = (d_dep > 1e-3 * max(1.0, np.abs(outs[0]["depth"]).max())) & ~excl
        np.testing.assert_allclose(_np(pipe.view_plane(pipe.dL_ddepth, 0))[sure_d], gD[0][sure_d],
                                   rtol=1e-6)

    # the oracle's loss gradient, where its sign is certain, through both backwards
    c = gC[0].copy()
    c[d_rgb <= 1e-3] = 0.0
    c[:, excl] = 0.0
    c = c.astype(np.float32)
    d = None
    if lam:
        d = gD[0].copy()
        d[(d_dep <= 1e-3 * max(1.0, np.abs(outs[0]["depth"]).max())) | excl] = 0.0
        d = d.astype(np.float32)
    pipe.render_bwd(torch.from_numpy(c.reshape(-1)).cuda(),
                    None if d is None else torch.from_numpy(d.reshape(-1)).cuda())
    pipe.project_bwd(g, camt)
    torch.cuda.synchronize()
    acc, dxi, g2ds = oracle_par.backward_views(scene, cams, projs, b, [c.astype(np.float64)],
                                               None if d is None else [d.astype(np.float64)],
                                               None)
    vis = projs[0]["radius"] > 0
    grad_close(_np(pipe.grad2d["xy"])[vis], g2ds[0]["xy"][vis], "dxy")
    gco = _np(pipe.grad2d["conic_opacity"])[vis]
    grad_close(gco[:, :3], g2ds[0]["conic"][vis], "dconic")
    grad_close(gco[:, 3], g2ds[0]["opacity"][vis], "dopacity")
    grz = _np(pipe.grad2d["rgb_depth"])[vis]
    grad_close(grz[:, :3], g2ds[0]["rgb"][vis], "drgb")
    if lam:
        grad_close(grz[:, 3], g2ds[0]["depth"][vis], "ddepth")
    frag = projs[0]["fragile"] != 0
    for key in acc:
        grad_close(_np(pipe.grads[key]), acc[key], key, rows_skip=frag)
    grad_close(_np(pipe.dxi)[0], dxi[0], "dxi")
