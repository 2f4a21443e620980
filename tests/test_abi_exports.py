"""CPU checks of the C ABI library: it builds for sm_103a, loads without a GPU,
exports every symbol include/gevo.h declares, and its host-only set-up calls
(layout, workspace size, status strings, the sort's launch count) behave as the
header states.  Compute entry points are called here only with arguments they
refuse before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(headers=("gevo.h", "gevo_prior.h", "gevo_map.h")):
    names = set()
    for h in headers:
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gevo_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2409_09295_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_stage_calls():
    names = _declared()
    for want in ("gevo_project", "gevo_bin_sort", "gevo_render_fwd", "gevo_render_bwd",
                 "gevo_project_bwd", "gevo_loss_l1", "gevo_layout_init",
                 "gevo_workspace_bytes", "gevo_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_probe_library_exports_the_measurement_symbols_only(lib):
    from paper_2409_09295_gb300 import _abi, build
    probes = ctypes.CDLL(build.PROBE_LIB)
    bench = _declared(("gevo_bench.h",))
    assert sorted(_abi.BENCH) == bench
    assert all(hasattr(probes, n) for n in bench)
    assert not any(hasattr(lib, n) for n in bench)   # not part of the product library


def test_bad_layouts_are_rejected_before_any_launch(lib):
    """A layout that gevo_layout_init did not produce (too many views, counts or
    bases that disagree with the sizes) is refused by the entry points with
    GEVO_ERR_INVALID before they touch any pointer, so no GPU is needed."""
    from paper_2409_09295_gb300 import _abi
    L = _abi.load()
    good = _abi.gevo_layout_init([64, 32], [48, 16])
    bad = []
    for field, val in (("n_views", 65), ("n_views", 0), ("total_tiles", good.total_tiles + 1),
                       ("total_pixels", good.total_pixels - 1)):
        b = _abi.Layout.from_buffer_copy(good)
        setattr(b, field, val)
        bad.append(b)
    for arr, v, val in (("tile_base", 1, 11), ("tiles_x", 0, 5), ("pix_base", 2, 1),
                        ("width", 1, 0)):
        b = _abi.Layout.from_buffer_copy(good)
        getattr(b, arr)[v] = val
        bad.append(b)
    dummy = ctypes.c_void_p(256)       # never dereferenced: validation comes first
    proj = _abi.Proj(dummy, dummy, dummy, dummy, dummy)
    for b in bad:
        for fn in (L.gevo_bin_sort, L.gevo_bin_sort_noalloc):
            args = [ctypes.byref(b), 10, ctypes.byref(proj), 16] + [dummy] * 4
            if fn is L.gevo_bin_sort:
                args += [dummy]
            assert fn(*args, None) == 1
        assert _abi.gevo_workspace_bytes(b, 10, 16) == 0


def test_binding_lists_every_declared_symbol():
    from paper_2409_09295_gb300 import _abi
    assert sorted(_abi.EXPORTS) == sorted(n for n in _declared())


def test_layout_and_workspace_host_calls():
    from paper_2409_09295_gb300 import _abi
    L = _abi.gevo_layout_init([640] * 12 + [320] * 4, [480] * 12 + [240] * 4)
    assert L.n_views == 16
    assert L.total_tiles == 12 * 40 * 30 + 4 * 20 * 15
    assert L.total_pixels == 12 * 640 * 480 + 4 * 320 * 240
    assert [L.tile_base[v] for v in (0, 1, 12, 16)] == [0, 1200, 14400, 15600]
    L2 = _abi.gevo_layout_init([1200], [680])
    assert (L2.tiles_x[0], L2.tiles_y[0]) == (75, 43)   # partial last tile row
    ws = _abi.gevo_workspace_bytes(L, 500_000, 10_000_000)
    assert ws >= 16 * 10_000_000 and ws % 256 == 0
    with pytest.raises(_abi.GevoError):
        _abi.gevo_layout_init([], [])
    with pytest.raises(_abi.GevoError):
        _abi.gevo_layout_init([0], [10])
    assert _abi.gevo_layout_init([16] * 64, [16] * 64).n_views == 64     # the maximum
    with pytest.raises(_abi.GevoError):
        _abi.gevo_layout_init([16] * 65, [16] * 65)
    assert _abi.gevo_status_str(2) == "duplicate capacity exceeded"
    assert _abi.gevo_version() == 1


def _prior_kinds():
    src = open(os.path.join(ROOT, "include", "gevo_prior.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"gevo_status (gevo_\w+)\((.*?)\);", src, flags=re.S):
        kinds = ""
        for a in m.group(2).split(","):
            a = a.strip()
            kinds += "p" if "*" in a else {"int32_t": "i", "int64_t": "I", "float": "f", "uint32_t": "u"}[a.split()[0]]
        out[m.group(1)] = kinds
    return out


def test_prior_binding_signatures_match_header():
    from paper_2409_09295_gb300 import _abi
    assert _abi.PRIOR == _prior_kinds()


def test_sort_launch_count_follows_the_dispatch():
    """gevo_bin_sort_launches: 12 kernels on the depth-ordered path (views of at
    most 8192 tiles), 4 on the bucket-and-sort path, fewer without entries or
    without room; -1 for a bad layout.  Host logic only."""
    from paper_2409_09295_gb300 import _abi
    small = _abi.gevo_layout_init([640, 320], [480, 240])     # 1200 + 300 tiles
    edge = _abi.gevo_layout_init([1440], [1456])              # 90 x 91 = 8190 tiles
    big = _abi.gevo_layout_init([2112, 64], [2080, 48])       # 132 x 130 tiles in one view
    n, cap = 1000, 10 ** 6
    assert _abi.gevo_bin_sort_launches(small, n, cap) == 12
    assert _abi.gevo_bin_sort_launches(edge, n, cap) == 12
    assert _abi.gevo_bin_sort_launches(big, n, cap) == 4
    assert _abi.gevo_bin_sort_launches(small, 0, cap) == 5    # totals, counts, scans, scatter
    assert _abi.gevo_bin_sort_launches(small, n, 0) == 11     # no scatter
    assert _abi.gevo_bin_sort_launches(big, 0, cap) == 1
    bad = _abi.Layout.from_buffer_copy(small)
    bad.n_views = 0
    assert _abi.gevo_bin_sort_launches(bad, n, cap) == -1


def test_part_calls_refuse_bad_parts_and_ranges(lib):
    """The projection's part calls check part and range before any launch (the
    pointers below are never dereferenced), so no GPU is needed."""
    from paper_2409_09295_gb300 import _abi
    L = _abi.load()
    lay = _abi.gevo_layout_init([64], [48])
    d = ctypes.c_void_p(256)
    n = 5000
    g = _abi.Gaussians(d, d, d, d, d, None, n, 3)
    proj = _abi.Proj(d, d, d, d, d)
    g2 = _abi.Grad2d(d, d, d)
    out = _abi.GaussianGrads(d, d, d, d, d, None)
    R = _abi.PART_RANGE

    def fwd(part, b, e):
        return L.gevo_project_part(ctypes.byref(lay), ctypes.byref(g), d, ctypes.byref(proj), part,
                                   b, e, d, None)

    def zero(part, b, e, grad=g2):
        return L.gevo_project_zero(ctypes.byref(lay), ctypes.byref(g), d, ctypes.byref(proj),
                                   ctypes.byref(grad) if grad is not None else None, part, b, e,
                                   d, None)

    def bwd(part, b, e):
        return L.gevo_project_bwd_part(ctypes.byref(lay), ctypes.byref(g), d, ctypes.byref(proj),
                                       ctypes.byref(g2), ctypes.byref(out), d, part, b, e, d, None)

    for part, b, e in ((3, 0, n), (-1, 0, n), (0, 10, 5), (0, -1, n), (0, 0, n + 1)):
        assert fwd(part, b, e) == 1
        assert zero(part, b, e) == 1
    assert zero(_abi.PART_COLOUR, 0, n) == 1                  # the colour part zeroes nothing
    assert zero(_abi.PART_ALL, 0, n, grad=None) == 1
    for part, b, e in ((3, 0, n), (0, 100, n), (0, 0, R + 1), (0, R, R - 1), (0, 0, n + R)):
        assert bwd(part, b, e) == 1
    assert fwd(_abi.PART_GEOMETRY, 7, 7) == 0                 # an empty range is a no-op
