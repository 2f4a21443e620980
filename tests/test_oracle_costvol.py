"""Pins of the cost-volume oracle (Eq. 1): the size the paper states, and depth
recovery on analytically rendered images of a textured plane (no renderer
involved)."""
import numpy as np
import pytest

from oracle import costvol


def test_cost_volume_size_matches_section_3a1():
    # 640 x 480 downsampled 4x, 64 hypotheses, binary32: "4.7 MB"
    h, w, nd = 480 // 4, 640 // 4, 64
    assert h * w * nd * 4 / 2 ** 20 == 4.6875


def _plane_images(d_star, cams, H, W):
    """Images of the plane z_world = d_star with a smooth world texture, by ray
    casting in double precision."""
    imgs = []
    for c in cams:
        R, t = c[:9].reshape(3, 3), c[9:12]
        fx, fy, cx, cy = c[12:16]
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        ray_c = np.stack([(xs + 0.5 - cx) / fx, (ys + 0.5 - cy) / fy, np.ones_like(xs)], -1)
        ray_w = ray_c @ R                      # R^T applied to row vectors
        o = -R.T @ t
        s = (d_star - o[2]) / ray_w[..., 2]
        pw = o + s[..., None] * ray_w
        tex = 0.5 + 0.25 * np.sin(3.1 * pw[..., 0]) * np.cos(2.3 * pw[..., 1]) + 0.2 * np.sin(7.0 * pw[..., 0] + 1.0)
        imgs.append(np.stack([tex, tex, tex]))
    return np.stack(imgs)


def test_wta_recovers_a_textured_plane():
    H, W = 96, 128
    cams = []
    for bx in (0.0, 0.15, -0.15, 0.3):
        c = np.zeros(16)
        c[:9] = np.eye(3).reshape(9)
        c[9:12] = [-bx, 0.0, 0.0]
        c[12:16] = [100.0, 100.0, W / 2, H / 2]
        cams.append(c)
    cams = np.stack(cams)
    d_star = 0.25 + (25.0 - 0.25) * 5 / 63        # exactly hypothesis 5
    rgb = _plane_images(d_star, cams, H, W)
    V, frag = costvol.cost_volume(rgb, cams, ref=0)
    depth = costvol.wta_up4(V)
    centre = depth[16:-16, 16:-16]
    assert np.mean(np.abs(centre - d_star) < 1e-9) > 0.9


def test_cost_volume_single_pixel_by_hand():
    rs = np.random.default_rng(0)
    H, W = 32, 40
    rgb = rs.uniform(size=(3, 3, H, W))
    cams = np.zeros((3, 16))
    for i in range(3):
        cams[i, :9] = np.eye(3).reshape(9)
        cams[i, 9:12] = [0.05 * i, -0.02 * i, 0.0]
        cams[i, 12:16] = [60.0, 60.0, 20.0, 16.0]
    V, _ = costvol.cost_volume(rgb, cams, ref=1, nd=8, d0=1.0, d1=8.0)
    g = costvol.grey4(rgb)
    y, x, k = 3, 5, 4
    d = 1.0 + 7.0 * k / 7
    pc = np.array([(x + 0.5 - 5.0) / 15.0 * d, (y + 0.5 - 4.0) / 15.0 * d, d]) - cams[1, 9:12]
    vals = []
    for s in (0, 2):
        p = pc + cams[s, 9:12]
        u = 15.0 * p[0] / p[2] + 5.0 - 0.5
        v = 15.0 * p[1] / p[2] + 4.0 - 0.5
        x0, y0 = int(np.floor(u)), int(np.floor(v))
        fx_, fy_ = u - x0, v - y0
        val = (1 - fy_) * ((1 - fx_) * g[s, y0, x0] + fx_ * g[s, y0, x0 + 1]) + \
            fy_ * ((1 - fx_) * g[s, y0 + 1, x0] + fx_ * g[s, y0 + 1, x0 + 1])
        vals.append(abs(g[1, y, x] - val))
    assert np.isclose(V[y, x, k], np.mean(vals), rtol=1e-12)


def test_bp_message_truncated_linear_by_hand():
    h = np.array([3.0, 0.0, 5.0, 5.0, 5.0])
    m = costvol.bp_message(h, 1.0, 2.5)
    # min over f_p of h(f_p) + min(|f_p - f_q|, 2.5): from label 1 (cost 0)
    np.testing.assert_allclose(m, [1.0, 0.0, 1.0, 2.0, 2.5])


def test_bp_without_smoothness_is_winner_take_all():
    rs = np.random.default_rng(0)
    V = rs.uniform(size=(6, 7, 9))
    lab, B, _ = costvol.bp(V, 0.0, 0.0, 5)
    np.testing.assert_array_equal(lab, np.argmin(V, axis=-1))


def test_bp_on_a_chain_reaches_the_exact_minimum():
    # min-sum BP is exact on a tree: on a 1 x n chain after n iterations its
    # labels minimise sum_p D_p(f_p) + sum_(p,p+1) min(s |f_p - f_p+1|, tau),
    # checked against exhaustive search.
    import itertools
    rs = np.random.default_rng(1)
    n, k, s, tau = 6, 4, 0.3, 0.7
    V = rs.uniform(size=(1, n, k))
    lab, _, _ = costvol.bp(V, s, tau, n + 1)

    def energy(f):
        e = sum(V[0, p, f[p]] for p in range(n))
        return e + sum(min(s * abs(f[p] - f[p + 1]), tau) for p in range(n - 1))
    best = min(itertools.product(range(k), repeat=n), key=energy)
    assert energy(tuple(lab[0])) == pytest.approx(energy(best), abs=1e-12)
    # and the same on a column
    labc, _, _ = costvol.bp(V.transpose(1, 0, 2), s, tau, n + 1)
    assert energy(tuple(labc[:, 0])) == pytest.approx(energy(best), abs=1e-12)


def test_bp_smooths_a_noisy_plane():
    # a constant-depth scene with 10% of the pixels' costs scrambled: BP
    # restores the true label where winner-take-all follows the noise
    rs = np.random.default_rng(2)
    h, w, k, true = 20, 24, 16, 5
    V = np.abs(np.arange(k) - true)[None, None, :] * 0.05 + rs.uniform(0, 0.02, size=(h, w, k))
    bad = rs.uniform(size=(h, w)) < 0.1
    V[bad] = rs.uniform(size=(bad.sum(), k))
    wta = np.argmin(V, axis=-1)
    lab, _, _ = costvol.bp(V, 0.2, 1.0, 20)
    assert (wta != true).sum() > 30
    assert (lab != true).sum() <= 5
