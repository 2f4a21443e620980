"""Pins of the FP64 oracle against what the mathematics fixes (no GPU needed).

Each test ties one oracle step to something other than the oracle itself: closed
forms worked out by hand (tests/golden/), textbook identities (eigenvalues of a
rotated covariance, SH orthonormality, the telescoping of blend weights),
brute-force enumeration on tiny inputs, and FP64 central finite differences of
the oracle's own forward pass for its backward pass.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2409_09295_gb300 import scenes


def _cam(d):
    return dict(R=np.array(d["R"], np.float64).reshape(3, 3), t=np.array(d["t"], np.float64),
                fx=d["fx"], fy=d["fy"], cx=d["cx"], cy=d["cy"], W=d["W"], H=d["H"])


def _one(mean, scale, quat, opac=0.5, rgb=(1.0, 0.5, 0.25)):
    return dict(means=np.array([mean], np.float64), scales=np.array([scale], np.float64),
                quats=np.array([quat], np.float64), opacities=np.array([opac], np.float64),
                rgb=np.array([rgb], np.float64), sh_degree=0)


# --------------------------------------------------------------------------
# Step 1: covariance and projection
# --------------------------------------------------------------------------
def test_cov3d_identity_quaternion_is_diag_scale_squared():
    s = np.array([0.3, 0.02, 1.7])
    S = oracle.cov3d(s, [1.0, 0.0, 0.0, 0.0])
    np.testing.assert_array_equal(S, np.diag(s * s))


def test_cov3d_unnormalised_quaternion_is_normalised():
    s = np.array([0.3, 0.02, 1.7])
    q = np.array([0.4, -0.3, 0.8, 0.1])
    np.testing.assert_allclose(oracle.cov3d(s, 7.5 * q), oracle.cov3d(s, q), rtol=1e-14,
                               atol=1e-16)


def test_cov3d_eigenvalues_are_scales_squared():
    r = np.random.default_rng(3)
    for _ in range(20):
        s = np.exp(r.normal(size=3))
        q = r.normal(size=4)
        S = oracle.cov3d(s, q)
        np.testing.assert_allclose(S, S.T, atol=1e-15)
        np.testing.assert_allclose(np.linalg.eigvalsh(S), np.sort(s * s), rtol=1e-12,
                                   atol=1e-14)


def test_cov3d_rotation_axis_is_eigenvector():
    # a rotation by theta about axis n keeps the scale along n on n
    th = 0.7
    n = np.array([0.0, 0.0, 1.0])
    q = [np.cos(th / 2), *(np.sin(th / 2) * n)]
    s = np.array([0.5, 0.1, 0.3])
    S = oracle.cov3d(s, q)
    np.testing.assert_allclose(S @ n, 0.09 * n, atol=1e-15)
    # and rotates the x axis by theta in the xy plane
    e = np.array([np.cos(th), np.sin(th), 0.0])
    np.testing.assert_allclose(S @ e, 0.25 * e, atol=1e-15)


def test_projection_golden_closed_forms(golden_dir):
    cases = json.load(open(os.path.join(golden_dir, "projection_cases.json")))["cases"]
    for c in cases:
        cam = _cam(c["camera"])
        p = oracle.project(_one(c["mean"], c["scale"], c["quat"]), cam)
        np.testing.assert_allclose(p["cov2d"][0], c["cov2d"], rtol=1e-12, atol=1e-12,
                                   err_msg=c["name"])
        np.testing.assert_allclose(p["conic"][0], c["conic"], rtol=1e-12, atol=1e-15,
                                   err_msg=c["name"])
        np.testing.assert_allclose(p["xy"][0], c["xy"], rtol=0, atol=1e-12, err_msg=c["name"])
        assert p["depth"][0] == c["depth"]
        assert p["radius"][0] == c["radius"], c["name"]
        if "tiles_touched" in c:
            assert p["tiles_touched"][0] == c["tiles_touched"]
            W, H = c["camera"]["W"], c["camera"]["H"]
            rect = oracle.rect_f32(p["xy"][0, 0], p["xy"][0, 1], p["radius"][0],
                                   (W + 15) // 16, (H + 15) // 16)
            assert list(rect) == c["rect"]


def test_projection_jacobian_matches_numeric_derivative_of_pinhole():
    """Sigma2 - 0.3 I must equal Jn W Sigma3 W^T Jn^T with Jn the numerical
    Jacobian of the pinhole map at the camera-frame mean, for a rotated and
    translated camera and an anisotropic rotated Gaussian."""
    r = np.random.default_rng(11)
    R, t = scenes.look_at([0.3, -0.4, -1.0], [0.1, 0.2, 3.0])
    cam = dict(R=R, t=t, fx=410.0, fy=395.0, cx=300.0, cy=220.0, W=640, H=480)
    for _ in range(10):
        mu = np.array([r.uniform(-0.5, 0.5), r.uniform(-0.5, 0.5), r.uniform(2.0, 4.0)])
        s = np.exp(r.normal(np.log(0.05), 0.4, 3))
        q = r.normal(size=4)
        p = oracle.project(_one(mu, s, q), cam)
        pc = R @ mu + t
        def pin(x):
            return np.array([cam["fx"] * x[0] / x[2] + cam["cx"] - 0.5,
                             cam["fy"] * x[1] / x[2] + cam["cy"] - 0.5])
        h = 1e-6
        Jn = np.stack([(pin(pc + h * e) - pin(pc - h * e)) / (2 * h) for e in np.eye(3)], 1)
        S2 = Jn @ R @ oracle.cov3d(s, q) @ R.T @ Jn.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(p["cov2d"][0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7)
        np.testing.assert_allclose(p["xy"][0], pin(pc), rtol=1e-13)
        A = np.array([[p["cov2d"][0, 0], p["cov2d"][0, 1]], [p["cov2d"][0, 1], p["cov2d"][0, 2]]])
        Q = np.linalg.inv(A)
        np.testing.assert_allclose(p["conic"][0], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-12)
        lam = np.linalg.eigvalsh(A)[-1]
        assert p["radius"][0] == int(np.ceil(3.0 * np.sqrt(lam))) or \
            abs(lam - (0.5 * np.trace(A) + np.sqrt(0.1))) < 1e-9 or \
            p["radius"][0] == int(np.ceil(3.0 * np.sqrt(0.5 * np.trace(A) + np.sqrt(0.1))))


def test_projection_guard_band_uses_clamped_jacobian():
    """Beyond 1.3x the half field of view the Jacobian is evaluated at the
    clamped direction, while the mean itself is not clamped."""
    cam = dict(R=np.eye(3), t=np.zeros(3), fx=100.0, fy=100.0, cx=50.0, cy=40.0, W=100, H=80)
    mu = np.array([2.5, 0.0, 2.0])  # x/z = 1.25 > 1.3 * 0.5 = 0.65
    s = np.array([0.05, 0.05, 0.05])
    p = oracle.project(_one(mu, s, [1, 0, 0, 0]), cam)
    z = 2.0
    tx = 0.65
    J = np.array([[100 / z, 0, -100 * tx / z], [0, 100 / z, 0]])
    S2 = 0.0025 * J @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-13)
    np.testing.assert_allclose(p["xy"][0], [100 * 1.25 + 49.5, 39.5], rtol=1e-14)
    assert p["radius"][0] == 0  # off-screen: rect empty -> culled


def test_projection_near_plane_cull():
    cam = dict(R=np.eye(3), t=np.zeros(3), fx=100.0, fy=100.0, cx=50.0, cy=40.0, W=100, H=80)
    for z, vis in [(0.2, False), (0.19, False), (0.2001, True), (-1.0, False)]:
        p = oracle.project(_one([0.0, 0.0, z], [0.001] * 3, [1, 0, 0, 0]), cam)
        assert (p["radius"][0] > 0) == vis, z


def test_sh_basis_orthonormal_on_sphere():
    """Gauss-Legendre in cos(theta) x uniform phi is exact for these degree <= 6
    products; the 16 basis functions must be orthonormal."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = np.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * np.pi * k / nphi
            d = np.array([st * np.cos(ph), st * np.sin(ph), ct])
            Y, _ = oracle.sh_basis(3, d)
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_gradient_matches_finite_difference():
    r = np.random.default_rng(5)
    for _ in range(5):
        d = r.normal(size=3)
        _, dY = oracle.sh_basis(3, d)
        h = 1e-6
        for u in range(3):
            e = np.zeros(3)
            e[u] = h
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, u], fd, atol=1e-8)


def test_sh_degree0_colour_and_clamp():
    cam = dict(R=np.eye(3), t=np.zeros(3), fx=100.0, fy=100.0, cx=50.0, cy=40.0, W=100, H=80)
    g = _one([0, 0, 2], [0.05] * 3, [1, 0, 0, 0])
    del g["rgb"]
    g["sh"] = np.array([[[0.3, -3.0, 1.0]]])
    g["sh_degree"] = 0
    p = oracle.project(g, cam)
    c0 = 0.5 / np.sqrt(np.pi)
    np.testing.assert_allclose(p["rgb"][0], [c0 * 0.3 + 0.5, 0.0, c0 + 0.5], rtol=1e-15)
    assert list(p["clamped"][0]) == [0, 1, 0]


# --------------------------------------------------------------------------
# Steps 2-4: binning, sort and ranges
# --------------------------------------------------------------------------
def test_rect_golden(golden_dir):
    for c in json.load(open(os.path.join(golden_dir, "binning_cases.json")))["cases"]:
        rect = oracle.rect_f32(c["xy"][0], c["xy"][1], c["r"], *c["tiles"])
        assert list(rect) == c["rect"], c


def test_binning_invariants_and_bruteforce_membership():
    sizes = [(64, 48), (33, 17), (16, 16)]
    rec = scenes.random_records(sizes, 200, seed=7, sigma_px=(0.5, 6.0))
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    keys, vals, ranges = b["keys"], b["vals"], b["ranges"]
    D = b["n_dup"]
    assert D == b["tiles_touched"].sum() == len(keys)
    # ascending by (key, val): an independent lexicographic check
    order = np.lexsort((vals, keys))
    np.testing.assert_array_equal(order, np.arange(D))
    # ranges partition [0, D) by tile
    lens = (ranges[:, 1].astype(np.int64) - ranges[:, 0]).sum()
    assert lens == D
    base = 0
    for v, (W, H) in enumerate(sizes):
        tx, ty = (W + 15) // 16, (H + 15) // 16
        for t in range(tx * ty):
            s, e = ranges[base + t]
            got = sorted(vals[s:e].tolist())
            # brute force: Gaussian g is in tile t iff tile t lies in its rect
            want = []
            for g in range(200):
                if rec["radius"][v, g] <= 0:
                    continue
                rc = oracle.rect_f32(rec["xy"][v, g, 0], rec["xy"][v, g, 1], rec["radius"][v, g], tx, ty)
                if rc[0] <= t % tx < rc[2] and rc[1] <= t // tx < rc[3]:
                    want.append(g)
            assert got == want
            for i in range(s, e):
                assert int(keys[i]) >> 32 == base + t
                assert int(keys[i]) & 0xFFFFFFFF == int(rec["depth"][v, vals[i]].view(np.uint32))
        base += tx * ty


def test_binning_overflow_reports_true_count():
    sizes = [(64, 48)]
    rec = scenes.random_records(sizes, 100, seed=8)
    full = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    cut = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"], capacity=full["n_dup"] - 1)
    assert cut["overflow"] and cut["n_dup"] == full["n_dup"]
    assert (cut["ranges"] == 0).all()


def test_binning_equal_depths_order_by_id():
    sizes = [(16, 16)]
    xy = np.full((1, 4, 2), 8.0, np.float32)
    radius = np.full((1, 4), 3, np.int32)
    depth = np.array([[2.0, 1.0, 2.0, 1.0]], np.float32)
    b = oracle.bin_f32(sizes, xy, radius, depth)
    assert b["vals"].tolist() == [1, 3, 0, 2]


# --------------------------------------------------------------------------
# Step 5: blending
# --------------------------------------------------------------------------
def _records(xy, conic, opac, rgb, depth):
    return dict(xy=np.array(xy, np.float64), conic=np.array(conic, np.float64),
                opacity=np.array(opac, np.float64), rgb=np.array(rgb, np.float64),
                depth=np.array(depth, np.float64))


def _render(W, H, rec, bg=(0.0, 0.0, 0.0), radius=None):
    n = rec["xy"].shape[0]
    if radius is None:
        radius = np.full(n, max(W, H), np.int32)
    b = oracle.bin_f32([(W, H)], rec["xy"][None].astype(np.float32), radius[None],
                       rec["depth"][None].astype(np.float32))
    return oracle.render_fwd(W, H, rec, b["vals"], b["ranges"], bg), b


def test_single_gaussian_closed_form():
    W, H = 32, 24
    rec = _records([[10.0, 9.0]], [[0.1, 0.02, 0.08]], [0.8], [[1.0, 0.5, 0.25]], [3.0])
    bg = (0.2, 0.3, 0.4)
    out, _ = _render(W, H, rec, bg)
    ys, xs = np.mgrid[0:H, 0:W]
    dx, dy = 10.0 - xs, 9.0 - ys
    alpha = 0.8 * np.exp(-0.5 * (0.1 * dx * dx + 0.08 * dy * dy) - 0.02 * dx * dy)
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    for ch, c in enumerate([1.0, 0.5, 0.25]):
        np.testing.assert_allclose(out["rgb"][ch], alpha * c + (1 - alpha) * bg[ch], atol=1e-15)
    np.testing.assert_allclose(out["depth"], alpha * 3.0, atol=1e-15)
    np.testing.assert_allclose(out["T"], 1 - alpha, atol=1e-15)
    np.testing.assert_array_equal(out["n_contrib"], (alpha > 0).astype(np.int32))


def test_opaque_gaussian_returns_099_of_its_colour():
    rec = _records([[8.0, 8.0]], [[0.01, 0.0, 0.01]], [1.0], [[0.9, 0.6, 0.3]], [2.0])
    out, _ = _render(16, 16, rec)
    np.testing.assert_allclose(out["rgb"][:, 8, 8], [0.99 * 0.9, 0.99 * 0.6, 0.99 * 0.3],
                               rtol=1e-15)
    assert out["T"][8, 8] == pytest.approx(0.01, rel=1e-14)


def test_stacked_opaque_gaussians_and_stop_rule():
    # alphas 0.99, 0.9 blend (T = 1e-3); a third 0.99 would push T to 1e-5 < 1e-4:
    # it stops the pixel without blending.
    o1 = 0.99 / np.exp(-0.5 * 0.01 * 0)  # centre pixel: power 0
    rec = _records([[8.0, 8.0]] * 3, [[0.01, 0.0, 0.01]] * 3, [min(o1, 1.0), 0.9, 0.99],
                   [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [1.0, 2.0, 3.0])
    out, _ = _render(16, 16, rec)
    T = out["T"][8, 8]
    assert T == pytest.approx(0.01 * 0.1, rel=1e-12)
    np.testing.assert_allclose(out["rgb"][:, 8, 8], [0.99, 0.01 * 0.9, 0.0], rtol=1e-12)
    assert out["depth"][8, 8] == pytest.approx(0.99 * 1.0 + 0.009 * 2.0, rel=1e-12)
    assert out["n_contrib"][8, 8] == 2
    assert out["n_eval"][8, 8] == 3
    assert out["n_blend"][8, 8] == 2


def test_skipped_entries_before_last_blend_are_counted():
    # front entry far away (alpha < 1/255) then a blending one: n_contrib = 2
    rec = _records([[15.0, 15.0], [4.0, 4.0]], [[0.5, 0, 0.5], [0.1, 0, 0.1]], [0.5, 0.5],
                   [[1, 1, 1], [1, 1, 1]], [1.0, 2.0])
    out, _ = _render(16, 16, rec)
    assert out["n_contrib"][4, 4] == 2
    assert out["n_eval"][4, 4] == 2
    assert out["n_blend"][4, 4] == 1   # the skipped front entry is walked, not blended


def test_partition_of_unity_and_constant_colour():
    sizes = [(48, 40)]
    rec = scenes.random_records(sizes, 300, seed=21, sigma_px=(1.0, 8.0))
    r = dict(xy=rec["xy"][0].astype(np.float64), conic=rec["conic"][0].astype(np.float64),
             opacity=rec["opacity"].astype(np.float64), rgb=np.full((300, 3), 0.7),
             depth=rec["depth"][0].astype(np.float64))
    bg = (0.1, 0.2, 0.3)
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    out = oracle.render_fwd(48, 40, r, b["vals"], b["ranges"], bg)
    np.testing.assert_allclose(out["wsum"] + out["T"], 1.0, atol=1e-14)
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], 0.7 * (1 - out["T"]) + bg[ch] * out["T"],
                                   atol=1e-14)
    assert (out["T"] >= 1e-4).all() and (out["T"] <= 1.0).all()


def test_empty_scene_gives_background():
    rec = _records(np.zeros((0, 2)), np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)), np.zeros(0))
    out, b = _render(20, 10, rec, bg=(0.5, 0.25, 1.0))
    assert b["n_dup"] == 0
    for ch, c in enumerate((0.5, 0.25, 1.0)):
        assert (out["rgb"][ch] == c).all()
    assert (out["T"] == 1).all() and (out["n_contrib"] == 0).all() and (out["depth"] == 0).all()


def test_permutation_of_ids_is_bitwise_invariant():
    w = scenes.workload(0, n=400)
    g = {k: v for k, v in w["scene"].items()}
    cams = [w["cams"][0]]
    outs, _, _ = oracle.render_views(g, cams)
    perm = np.random.default_rng(1).permutation(400)
    gp = dict(g)
    for k in ("means", "scales", "quats", "opacities", "rgb"):
        gp[k] = g[k][perm]
    outs_p, _, _ = oracle.render_views(gp, cams)
    for k in ("rgb", "depth", "T", "n_contrib"):
        np.testing.assert_array_equal(outs[0][k], outs_p[0][k])


# --------------------------------------------------------------------------
# Steps 6-7: gradients against FP64 central finite differences
# --------------------------------------------------------------------------
def _rodrigues(phi):
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th == 0:
        return np.eye(3)
    return np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K


GUARD = 1.3   # guard band of the EWA Jacobian: |x/z| clamped at 1.3 x the half field of view


def _guard_flags(g, cams):
    """Per view and Gaussian: (x/z beyond the guard band, y/z beyond it), from the
    camera-frame means.  Used to keep finite differences away from a clamp that
    flips inside [-h, h] and to count the Gaussians a case sends through the
    clamped-Jacobian branch."""
    out = []
    for c in cams:
        R = np.asarray(c["R"], np.float64)
        p = np.asarray(g["means"], np.float64) @ R.T + np.asarray(c["t"], np.float64)
        limx = GUARD * 0.5 * c["W"] / c["fx"]
        limy = GUARD * 0.5 * c["H"] / c["fy"]
        out.append(np.stack([np.abs(p[:, 0] / p[:, 2]) > limx,
                             np.abs(p[:, 1] / p[:, 2]) > limy], axis=1))
    return out


def _lin_loss(g, cams, Wts):
    outs, projs, b = oracle.render_views(g, cams)
    L = sum((o["rgb"] * w["rgb"]).sum() + (o["depth"] * w["depth"]).sum()
            + (o["T"] * w["T"]).sum() for o, w in zip(outs, Wts))
    sig = ([o["sig"] for o in outs] + [p["radius"] for p in projs]
           + [p["clamped"] for p in projs] + _guard_flags(g, cams))
    return L, outs, projs, b, sig


def _front_alpha_clamped(cams, projs, b):
    """Number of pixels whose first blended entry has o G above the 0.99 clamp.
    The first blended entry of a pixel is always blended (T = 1 before it and
    1 - 0.99 > 1e-4), so every pixel counted here sends one entry through the
    clamped-alpha branch of the backward pass."""
    n = 0
    base = 0
    for v, c in enumerate(cams):
        W, H = int(c["W"]), int(c["H"])
        tx = (W + 15) // 16
        p = projs[v]
        for py in range(H):
            for px in range(W):
                s, e = b["ranges"][base + (py // 16) * tx + px // 16]
                for i in range(s, e):
                    gi = b["vals"][i]
                    dx, dy = p["xy"][gi, 0] - px, p["xy"][gi, 1] - py
                    ca, cb, cc = p["conic"][gi]
                    power = -0.5 * (ca * dx * dx + cc * dy * dy) - cb * dx * dy
                    if power > 0:
                        continue
                    og = p["opacity"][gi] * np.exp(power)
                    if min(og, 0.99) < 1.0 / 255.0:
                        continue
                    n += og > 0.99
                    break
        base += tx * ((H + 15) // 16)
    return n


def _same(s1, s2):
    return all(np.array_equal(a, b) for a, b in zip(s1, s2))


def _fd_case(g, cams, n_per_tensor, seed, h=1e-6, n_for=None):
    """Checks sampled parameters and every pose component against central
    differences; n_for overrides the sample size per parameter tensor."""
    rs = np.random.default_rng(seed)
    g = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    Wts = [dict(rgb=rs.normal(size=(3, c["H"], c["W"])), depth=rs.normal(size=(c["H"], c["W"])),
                T=rs.normal(size=(c["H"], c["W"]))) for c in cams]
    L0, outs, projs, b, s0 = _lin_loss(g, cams, Wts)
    acc, dxi, _ = oracle.backward_views(g, cams, projs, b, [w["rgb"] for w in Wts],
                                        [w["depth"] for w in Wts], [w["T"] for w in Wts])
    checked = 0
    keys = ["means", "scales", "quats", "opacities"] + (["rgb"] if "rgb" in g else ["sh"])
    for k in keys:
        flat = g[k].reshape(-1)
        n_k = (n_for or {}).get(k, n_per_tensor)
        for i in rs.choice(flat.size, size=min(flat.size, n_k), replace=False):
            gp, gm = dict(g), dict(g)
            gp[k], gm[k] = g[k].copy(), g[k].copy()
            gp[k].reshape(-1)[i] += h
            gm[k].reshape(-1)[i] -= h
            Lp, *_, sp = _lin_loss(gp, cams, Wts)
            Lm, *_, sm = _lin_loss(gm, cams, Wts)
            if not (_same(sp, s0) and _same(sm, s0)):
                continue  # a discrete event moved inside [-h, h]: FD not valid here
            fd = (Lp - Lm) / (2 * h)
            an = acc[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-5 * abs(fd) + 1e-7 * (1 + abs(L0)), (k, i, fd, an)
            checked += 1
    for v in range(len(cams)):
        for j in range(6):
            Ls = []
            ok = True
            for sgn in (1.0, -1.0):
                xi = np.zeros(6)
                xi[j] = sgn * h
                Rx = _rodrigues(xi[3:])
                cs = [dict(c) for c in cams]
                R = np.asarray(cams[v]["R"], np.float64)
                t = np.asarray(cams[v]["t"], np.float64)
                cs[v] = dict(cams[v], R=Rx @ R, t=Rx @ t + xi[:3])
                Lx, *_, sx = _lin_loss(g, cs, Wts)
                ok &= _same(sx, s0)
                Ls.append(Lx)
            if not ok:
                continue
            fd = (Ls[0] - Ls[1]) / (2 * h)
            assert abs(fd - dxi[v, j]) <= 1e-5 * abs(fd) + 1e-7 * (1 + abs(L0)), (v, j, fd, dxi[v, j])
            checked += 1
    return checked


def test_fd_micro_scene_rgb_identity_pose():
    g = scenes.camera_box_scene(8, 5, sh_degree=None, box=((-0.3, 0.3), (-0.3, 0.3), (2, 3)))
    g["scales"] = g["scales"] * 4
    assert _fd_case(g, [scenes.identity_camera(48, 32, 60.0)], 12, 0) >= 40


def test_fd_micro_scene_sh3_two_posed_views():
    g = scenes.camera_box_scene(8, 6, sh_degree=3, box=((-0.3, 0.3), (-0.3, 0.3), (2, 3)))
    g["scales"] = g["scales"] * 4
    R1, t1 = scenes.look_at([0.1, -0.2, -0.5], [0, 0, 2.5])
    R2, t2 = scenes.look_at([-0.4, 0.1, 0.2], [0.1, 0, 2.5])
    cams = [scenes.camera(R1, t1, 60, 62, 24, 16, 48, 32), scenes.camera(R2, t2, 55, 55, 20, 20, 40, 40)]
    assert _fd_case(g, cams, 10, 1) >= 40


def test_fd_tracking_subscene_sample():
    """The 64x48 sub-scene of the 1200x680 tracking workload (2k Gaussians, SH 3):
    a random sample of parameters plus all six pose components."""
    g, cams = scenes.tracking_subscene(2000)
    assert _fd_case(g, cams, 4, 2) >= 15


def test_fd_alpha_clamp_branch():
    """Near-opaque, wide splats: pixels near their centres have o G > 0.99, so
    alpha sits at the clamp and those pixels must add nothing to the opacity,
    conic and mean gradients (finite differences see alpha not move)."""
    g = scenes.camera_box_scene(6, 7, sh_degree=None, box=((-0.6, 0.6), (-0.4, 0.4), (2, 3)))
    g["scales"] = np.tile(np.array([0.5, 0.4, 0.3]), (6, 1))
    g["opacities"] = np.linspace(0.996, 0.9995, 6)
    cams = [scenes.identity_camera(64, 48, 60.0)]
    _, projs, b = oracle.render_views(g, cams)
    assert _front_alpha_clamped(cams, projs, b) >= 5
    assert _fd_case(g, cams, 12, 3) >= 50


def test_fd_sh_clamp_branch():
    """SH-3 splats whose DC coefficient drives a channel below zero: the clamped
    channel's colour is 0 whatever its coefficients, so its SH gradients and its
    share of the view-direction (mean and pose) gradient must vanish."""
    g = scenes.camera_box_scene(8, 8, sh_degree=3, box=((-0.3, 0.3), (-0.3, 0.3), (2, 3)))
    g["scales"] = g["scales"] * 4
    sh = np.array(g["sh"], np.float64)
    sh[::2, 0, 0] = -2.2
    sh[1::3, 0, 2] = -2.0
    g["sh"] = sh
    R1, t1 = scenes.look_at([0.1, -0.2, -0.5], [0, 0, 2.5])
    cams = [scenes.camera(R1, t1, 60, 62, 24, 16, 48, 32)]
    _, projs, _ = oracle.render_views(g, cams)
    vis = projs[0]["radius"] > 0
    assert (projs[0]["clamped"][vis].sum(axis=1) > 0).sum() >= 5
    assert _fd_case(g, cams, 10, 4, n_for=dict(sh=200)) >= 150


def test_fd_guard_band_branch():
    """Wide splats whose means lie beyond 1.3 x the half field of view (in x and
    in y) but still reach the image: the EWA Jacobian uses the clamped x/z, y/z,
    and the clamped coordinate passes gradient only through 1/z."""
    g = scenes.camera_box_scene(8, 9, sh_degree=3, box=((-0.3, 0.3), (-0.3, 0.3), (2, 3)))
    m = np.array(g["means"], np.float64)
    m[:4] = [[1.5, 0.1, 2.5], [-1.6, -0.2, 2.6], [0.2, 1.1, 2.4], [-0.1, -1.2, 2.7]]
    g["means"] = m
    sc = np.array(g["scales"], np.float64)
    sc[:4] = [0.3, 0.25, 0.2]
    sc[4:] *= 4
    g["scales"] = sc
    R1, t1 = scenes.look_at([0.0, 0.0, 0.0], [0, 0, 2.5])
    R2, t2 = scenes.look_at([0.2, 0.1, 0.1], [0.1, 0, 2.5])
    cams = [scenes.camera(R1, t1, 60, 62, 24, 16, 48, 32),
            scenes.camera(R2, t2, 58, 58, 24, 16, 48, 32)]
    _, projs, _ = oracle.render_views(g, cams)
    for v, flags in enumerate(_guard_flags(g, cams)):
        seen = projs[v]["radius"] > 0
        assert (flags[:, 0] & seen).sum() >= 2 and (flags[:, 1] & seen).sum() >= 2
    assert _fd_case(g, cams, 12, 5) >= 60


def test_l1_loss_closed_form():
    a = [np.array([[[0.5, 0.2], [0.1, 0.1]]] * 3)]
    b = [np.array([[[0.25, 0.2], [0.3, 0.0]]] * 3)]
    d = [np.array([[1.0, 2.0], [3.0, 4.0]])]
    dt = [np.array([[1.5, 2.0], [2.0, 4.0]])]
    L, gC, gD = oracle.loss_l1(a, b, d, dt, lambda_depth=2.0)
    assert L == pytest.approx((0.25 + 0 + 0.2 + 0.1) / 4 + 2.0 * (0.5 + 0 + 1.0 + 0) / 4)
    np.testing.assert_array_equal(gC[0][0], np.array([[1, 0], [-1, 1]]) / 12.0)
    np.testing.assert_array_equal(gD[0], 2.0 * np.array([[-1, 0], [1, 0]]) / 4.0)
