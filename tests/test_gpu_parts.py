"""The two-part projection and projection derivative (gevo_project_part,
gevo_project_bwd_part) against the whole calls, and the end-to-end host step
(batch.HostStep), which runs the parts on overlapping streams with its copies,
against the device step on the same inputs."""
import pytest

torch = pytest.importorskip("torch")

from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import _abi, raster  # noqa: E402
from paper_2409_09295_gb300.batch import BatchedReplay, HostStep  # noqa: E402


def _cams():
    poses = scenes.circle_poses(4, 2.0, seed=72)
    return [scenes.camera(R, t, 262.5, 262.5, 160.0, 120.0, 320, 240) for R, t in poses[:3]] + \
        [scenes.camera(*poses[3], 525.0, 525.0, 320.0, 240.0, 640, 480)]


def _setup(deg, n=30_000):
    scene = scenes.room_scene(n, 71, sh_degree=deg)
    cams = _cams()
    g = raster.gaussians_to_device(scene)
    camt = raster.camera_tensor(cams, "cuda")
    sizes = [(c["W"], c["H"]) for c in cams]
    colour = "rgb" if deg is None else "sh"
    mk = lambda: raster.Pipeline(n, sizes, 1 << 20, colour=colour,  # noqa: E731
                                 sh_degree=0 if deg is None else deg)
    return g, camt, mk


def _bits(t):
    return t.contiguous().view(torch.int32)


@pytest.mark.parametrize("deg", [None, 0, 1, 2, 3])
def test_projection_parts_match_whole(deg):
    g, camt, mk = _setup(deg)
    a, b = mk(), mk()
    a.project(g, camt)
    for t in b.proj.values():
        t.fill_(7)            # the parts must write every field the whole call does
    b.project(g, camt, part=_abi.PART_GEOMETRY)
    torch.cuda.synchronize()
    vis = a.proj["radius"] > 0
    assert int(vis.sum()) > 1000
    assert torch.equal(b.proj["radius"], a.proj["radius"])
    assert torch.equal(b.proj["tiles_touched"], a.proj["tiles_touched"])
    # the geometry part: every field but the colour, colour 0
    assert torch.equal(_bits(b.proj["xy"][vis]), _bits(a.proj["xy"][vis]))
    assert torch.equal(_bits(b.proj["conic_opacity"][vis]), _bits(a.proj["conic_opacity"][vis]))
    assert torch.equal(_bits(b.proj["rgb_depth"][vis][:, 3]), _bits(a.proj["rgb_depth"][vis][:, 3]))
    assert torch.count_nonzero(b.proj["rgb_depth"][vis][:, :3]) == 0
    b.project(g, camt, part=_abi.PART_COLOUR)
    torch.cuda.synchronize()
    assert torch.equal(_bits(b.proj["rgb_depth"][vis]), _bits(a.proj["rgb_depth"][vis]))
    with pytest.raises(_abi.GevoError):
        b.project(g, camt, part=3)
    # over ranges (uneven, any split): the same records
    c = mk()
    for t in c.proj.values():
        t.fill_(7)
    n = int(g["means"].shape[0])
    for r in ((0, 777), (777, 20000), (20000, n)):
        c.project(g, camt, part=_abi.PART_GEOMETRY, g_range=r)
    for r in ((0, 15000), (15000, n)):
        c.project(g, camt, part=_abi.PART_COLOUR, g_range=r)
    torch.cuda.synchronize()
    assert torch.equal(c.proj["radius"], a.proj["radius"])
    for k in ("xy", "conic_opacity", "rgb_depth"):
        assert torch.equal(_bits(c.proj[k][vis]), _bits(a.proj[k][vis])), k
    with pytest.raises(_abi.GevoError):
        c.project(g, camt, part=_abi.PART_GEOMETRY, g_range=(10, n + 1))


def _random_grad2d(pipe, seed):
    gen = torch.Generator().manual_seed(seed)
    for k, t in pipe.grad2d.items():
        t.copy_(torch.randn(t.shape, generator=gen) * 1e-2)


@pytest.mark.parametrize("deg", [None, 1, 3])
def test_projection_backward_parts_match_whole(deg):
    g, camt, mk = _setup(deg)
    p = mk()
    p.project(g, camt)
    _random_grad2d(p, 73)
    p.project_bwd(g, camt)
    torch.cuda.synchronize()
    whole = {k: v.clone() for k, v in p.grads.items()}
    dxi = p.dxi.clone()
    for v in p.grads.values():
        v.fill_(7)
    p.dxi.fill_(7)
    p.project_bwd(g, camt, part=_abi.PART_COLOUR)
    torch.cuda.synchronize()
    if deg is not None:   # the SH gradients are final after the colour part
        assert torch.equal(_bits(p.grads["sh"]), _bits(whole["sh"]))
    p.project_bwd(g, camt, part=_abi.PART_GEOMETRY)
    torch.cuda.synchronize()
    for k, v in whole.items():
        assert torch.equal(_bits(p.grads[k]), _bits(v)), k
    # the pose twist sums with atomics, in another order
    assert torch.allclose(p.dxi, dxi, rtol=1e-5, atol=1e-6 * float(dxi.abs().max()))
    # over ranges of whole PART_RANGE blocks: colour ranges in order, then geometry
    n = int(g["means"].shape[0])
    R = _abi.PART_RANGE
    for v in p.grads.values():
        v.fill_(7)
    p.dxi.fill_(7)
    b1 = R * (n // (3 * R))
    b2 = 2 * b1
    assert 0 < b1 < b2 < n
    for r in ((0, b1), (b1, b2), (b2, n)):
        p.project_bwd(g, camt, part=_abi.PART_COLOUR, g_range=r)
    for r in ((0, b2), (b2, n)):
        p.project_bwd(g, camt, part=_abi.PART_GEOMETRY, g_range=r)
    torch.cuda.synchronize()
    for k, v in whole.items():
        assert torch.equal(_bits(p.grads[k]), _bits(v)), k
    assert torch.allclose(p.dxi, dxi, rtol=1e-5, atol=1e-6 * float(dxi.abs().max()))
    with pytest.raises(_abi.GevoError):   # not a whole range of the walk order
        p.project_bwd(g, camt, part=_abi.PART_COLOUR, g_range=(100, n))


def _rel(a, b):
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def test_host_step_matches_device_step():
    w = scenes.workload(2, n=40_000)
    cams = [w["cams"][k] for k in (0, 5, 13)]
    g = raster.gaussians_to_device(w["scene"])
    gt = raster.gaussians_to_device(w["target_scene"])
    sizes = [(c["W"], c["H"]) for c in cams]
    tp = raster.Pipeline(40_000, sizes, 1 << 21, colour="sh", sh_degree=3)
    camt = raster.camera_tensor(cams, "cuda")
    tp.ensure_capacity(gt, camt)
    tp.forward(gt, camt)
    target_rgb, target_depth = tp.rgb.clone(), tp.depth.clone()
    tune = dict(threads_per_tile=64, persistent=1, blocks_per_sm=0)
    rep = BatchedReplay(g, cams, target_rgb, target_depth, lambda_depth=1.0, autotune=False,
                        tuning_fwd=tune, tuning_bwd=dict(tune, threads_per_tile=32))
    hs = HostStep(rep)
    gen = torch.Generator().manual_seed(74)
    for it in range(2):
        # new parameters in host memory each step: the step must upload them
        hs.host_in["means"].add_(torch.randn(hs.host_in["means"].shape, generator=gen) * 1e-3)
        hs.step()
        torch.cuda.synchronize()
        assert rep.pipe.last_error() == 0
        # the device step on what was uploaded
        for k in rep.g:
            if k != "sh_degree":
                assert torch.equal(rep.g[k].cpu(), hs.host_in[k]), k
        rep.step_eager()
        torch.cuda.synchronize()
        p = rep.pipe
        assert _rel(hs.host_out["loss"], p.loss.cpu()) < 1e-6
        assert _rel(hs.host_out["dxi"], p.dxi.cpu()) < 1e-4
        for k, v in p.grads.items():
            assert float(v.norm()) > 0, k
            assert _rel(hs.host_out[k], v.cpu()) < 1e-5, (it, k)


@pytest.mark.parametrize("deg", [None, 3])
def test_projection_that_zeroes_the_gradient_rows(deg):
    g, camt, mk = _setup(deg)
    a, b = mk(), mk()
    a.project(g, camt)
    for t in b.grad2d.values():
        t.fill_(7)
    b.project(g, camt, zero_grad2d=True)
    torch.cuda.synchronize()
    vis = a.proj["radius"] > 0
    assert torch.equal(b.proj["radius"], a.proj["radius"])
    for k in ("xy", "conic_opacity", "rgb_depth"):
        assert torch.equal(_bits(b.proj[k][vis]), _bits(a.proj[k][vis])), k
    for k, t in b.grad2d.items():   # the visible entries' rows zeroed, the others untouched
        assert torch.count_nonzero(t[vis]) == 0, k
        assert bool((t[~vis] == 7).all()), k
    # the geometry part over ranges does the same for its Gaussians
    c = mk()
    for t in c.grad2d.values():
        t.fill_(7)
    n = int(g["means"].shape[0])
    for r in ((0, 9999), (9999, n)):
        c.project(g, camt, part=_abi.PART_GEOMETRY, g_range=r, zero_grad2d=True)
    c.project(g, camt, part=_abi.PART_COLOUR)
    torch.cuda.synchronize()
    assert torch.equal(_bits(c.proj["rgb_depth"][vis]), _bits(a.proj["rgb_depth"][vis]))
    for k, t in c.grad2d.items():
        assert torch.count_nonzero(t[vis]) == 0 and bool((t[~vis] == 7).all()), k
    with pytest.raises(_abi.GevoError):
        c.project(g, camt, part=_abi.PART_COLOUR, zero_grad2d=True)
