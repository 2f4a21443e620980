"""gevo_bin_sort_noalloc, the sort entry point for callers that cannot allocate
device memory (plug-ins of a host application that owns every device
allocation, real-time loops that must not call an allocator).  Its scratch is a
fixed static device array, so it must give exactly what gevo_bin_sort gives
with a caller-allocated workspace, call after call, and refuse sizes beyond
that array.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2409_09295_gb300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2409_09295_gb300 import _abi, raster  # noqa: E402


def _upload(pipe, rec):
    V, n = rec["xy"].shape[:2]
    rz = np.zeros((V, n, 4), np.float32)
    rz[..., 3] = rec["depth"]
    pipe.proj["xy"].copy_(torch.from_numpy(rec["xy"].reshape(V * n, 2)).cuda())
    pipe.proj["rgb_depth"].copy_(torch.from_numpy(rz.reshape(V * n, 4)).cuda())
    pipe.proj["radius"].copy_(torch.from_numpy(rec["radius"].reshape(V * n)).cuda())


def test_noalloc_sort_matches_workspace_sort_on_consecutive_calls():
    cases = [([(640, 480), (320, 240)], 6000, 61, (0.5, 12.0)),
             ([(96, 64)], 2500, 62, (0.5, 40.0))]   # second call: fewer tiles, fewer duplicates
    for sizes, n, seed, sig in cases:
        rec = scenes.random_records(sizes, n, seed=seed, sigma_px=sig)
        pipe = raster.Pipeline(n, sizes, 400_000, keep_keys=True)
        _upload(pipe, rec)
        pipe.bin_sort()
        D = int(pipe.n_dup.item())
        assert 0 < D <= pipe.capacity
        keys = torch.zeros_like(pipe.keys)
        vals = torch.zeros_like(pipe.vals)
        ranges = torch.zeros_like(pipe.ranges)
        n_dup = torch.zeros_like(pipe.n_dup)
        _abi.gevo_bin_sort_noalloc(pipe.layout, n, pipe.proj, pipe.capacity, keys, vals, ranges,
                                   n_dup)
        torch.cuda.synchronize()
        assert int(n_dup.item()) == D
        assert torch.equal(ranges, pipe.ranges)
        assert torch.equal(keys[:D], pipe.keys[:D])
        assert torch.equal(vals[:D], pipe.vals[:D])
        vals_only = torch.zeros_like(pipe.vals)   # keys left out: the same ids
        _abi.gevo_bin_sort_noalloc(pipe.layout, n, pipe.proj, pipe.capacity, None, vals_only,
                                   ranges, n_dup)
        torch.cuda.synchronize()
        assert torch.equal(vals_only[:D], pipe.vals[:D])
        # and, since it runs other binning kernels, bit for bit against the oracle
        ref = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
        assert ref["n_dup"] == D
        np.testing.assert_array_equal(ranges.cpu().numpy().view(np.uint32), ref["ranges"])
        np.testing.assert_array_equal(keys[:D].cpu().numpy().view(np.uint64), ref["keys"])
        np.testing.assert_array_equal(vals[:D].cpu().numpy().view(np.uint32), ref["vals"])


def test_noalloc_sort_reports_overflow_through_the_count():
    sizes = [(64, 48)]
    rec = scenes.random_records(sizes, 500, seed=63)
    pipe = raster.Pipeline(500, sizes, 100_000, keep_keys=True)
    _upload(pipe, rec)
    pipe.bin_sort()
    D = int(pipe.n_dup.item())
    keys, vals = torch.zeros_like(pipe.keys), torch.zeros_like(pipe.vals)
    ranges, n_dup = torch.ones_like(pipe.ranges), torch.zeros_like(pipe.n_dup)
    _abi.gevo_bin_sort_noalloc(pipe.layout, 500, pipe.proj, D - 1, keys, vals, ranges, n_dup)
    torch.cuda.synchronize()
    assert int(n_dup.item()) == D
    assert int(ranges.abs().sum().item()) == 0


def test_noalloc_sort_refuses_sizes_beyond_its_scratch():
    pipe = raster.Pipeline(10, [(64, 48)], 16)
    big = (1 << 21) + 1
    with pytest.raises(_abi.GevoError) as e:
        _abi.gevo_bin_sort_noalloc(pipe.layout, 10, pipe.proj, big, pipe.keys, pipe.vals,
                                   pipe.ranges, pipe.n_dup)
    assert e.value.code == 6
    wide = _abi.gevo_layout_init([4096] * 5, [4096] * 5)   # 5 x 65536 tiles > 65536
    with pytest.raises(_abi.GevoError) as e:
        _abi.gevo_bin_sort_noalloc(wide, 10, pipe.proj, 16, pipe.keys, pipe.vals, pipe.ranges,
                                   pipe.n_dup)
    assert e.value.code == 6
