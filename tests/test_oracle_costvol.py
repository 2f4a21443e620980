"""Pins of the cost-volume oracle (Eq. 1): the size the paper states, and depth
recovery on analytically rendered images of a textured plane (no renderer
involved)."""
import numpy as np

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
