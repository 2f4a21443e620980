"""Pins of the oracle's per-Gaussian rendering error (Eq. 5) and active set
(Section III-B2): closed forms of the blending weight w(g, u) for one and for
stacked Gaussians, the telescoping identity sum_g w(g, u) = 1 - T(u), the
colour derivative dC/dc_g = w(g, u) of the (finite-difference pinned) backward,
invariance under relabelling, and hand-worked thresholds."""
import numpy as np

import oracle
from paper_2409_09295_gb300 import scenes


def _records(xy, conic, opac, rgb, depth):
    return dict(xy=np.array(xy, np.float64), conic=np.array(conic, np.float64),
                opacity=np.array(opac, np.float64), rgb=np.array(rgb, np.float64),
                depth=np.array(depth, np.float64))


def _render(W, H, rec, pix_err, radius=None):
    n = rec["xy"].shape[0]
    if radius is None:
        radius = np.full(n, max(W, H), np.int32)
    b = oracle.bin_f32([(W, H)], rec["xy"][None].astype(np.float32), radius[None],
                       rec["depth"][None].astype(np.float32))
    return oracle.render_fwd(W, H, rec, b["vals"], b["ranges"], pix_err=pix_err), b


def test_single_gaussian_error_is_alpha_weighted_sum():
    W, H = 32, 24
    rec = _records([[10.0, 9.0]], [[0.1, 0.02, 0.08]], [0.8], [[1.0, 0.5, 0.25]], [3.0])
    e = np.random.default_rng(3).uniform(size=(H, W))
    out, _ = _render(W, H, rec, e)
    ys, xs = np.mgrid[0:H, 0:W]
    dx, dy = 10.0 - xs, 9.0 - ys
    alpha = 0.8 * np.exp(-0.5 * (0.1 * dx * dx + 0.08 * dy * dy) - 0.02 * dx * dy)
    alpha = np.where(alpha < 1 / 255, 0.0, alpha)
    want = (alpha * e).sum()
    assert abs(out["gauss_err"][0] - want) <= 1e-13 * want


def test_stacked_gaussians_weights_and_stopped_entry():
    # alphas 0.99, 0.9 at the centre pixel blend with weights 0.99 and 0.01 * 0.9;
    # a third 0.99 stops the pixel without blending: weight 0.
    rec = _records([[8.0, 8.0]] * 3, [[0.01, 0.0, 0.01]] * 3, [0.99, 0.9, 0.99],
                   [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [1.0, 2.0, 3.0])
    e = np.zeros((16, 16))
    e[8, 8] = 0.5
    out, _ = _render(16, 16, rec, e)
    np.testing.assert_allclose(out["gauss_err"], [0.99 * 0.5, 0.01 * 0.9 * 0.5, 0.0], rtol=1e-13)


def test_errors_telescope_to_one_minus_transmittance():
    sizes = [(48, 40)]
    rec = scenes.random_records(sizes, 300, seed=21, sigma_px=(1.0, 8.0))
    r = dict(xy=rec["xy"][0].astype(np.float64), conic=rec["conic"][0].astype(np.float64),
             opacity=rec["opacity"].astype(np.float64), rgb=rec["rgb"][0].astype(np.float64),
             depth=rec["depth"][0].astype(np.float64))
    e = np.random.default_rng(5).uniform(size=(40, 48))
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    out = oracle.render_fwd(48, 40, r, b["vals"], b["ranges"], pix_err=e)
    total = out["gauss_err"].sum()
    want = ((1.0 - out["T"]) * e).sum()
    assert abs(total - want) <= 1e-12 * want
    assert (out["gauss_err"] >= 0).all()
    # Gaussians no pixel blends (culled, or never reached) have zero error
    culled = rec["radius"][0] == 0
    assert (out["gauss_err"][culled] == 0).all()


def test_unit_error_equals_colour_derivative_of_backward():
    # with e = 1 everywhere, E(g) = sum_u w(g, u) = dC_red / dc_red(g), which the
    # backward (pinned by finite differences) computes by a separate walk.
    sizes = [(40, 32)]
    rec = scenes.random_records(sizes, 150, seed=8, sigma_px=(1.0, 6.0))
    r = dict(xy=rec["xy"][0].astype(np.float64), conic=rec["conic"][0].astype(np.float64),
             opacity=rec["opacity"].astype(np.float64), rgb=rec["rgb"][0].astype(np.float64),
             depth=rec["depth"][0].astype(np.float64))
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    out = oracle.render_fwd(40, 32, r, b["vals"], b["ranges"], pix_err=np.ones((32, 40)))
    gC = np.zeros((3, 32, 40))
    gC[0] = 1.0
    g = oracle.render_bwd(40, 32, r, b["vals"], b["ranges"], gC)
    np.testing.assert_allclose(out["gauss_err"], g["rgb"][:, 0], rtol=1e-12, atol=1e-14)


def test_error_follows_relabelled_gaussians():
    sizes = [(32, 32)]
    rec = scenes.random_records(sizes, 120, seed=30, sigma_px=(1.0, 5.0))
    n = 120
    r = dict(xy=rec["xy"][0].astype(np.float64), conic=rec["conic"][0].astype(np.float64),
             opacity=rec["opacity"].astype(np.float64), rgb=rec["rgb"][0].astype(np.float64),
             depth=rec["depth"][0].astype(np.float64))
    e = np.random.default_rng(2).uniform(size=(32, 32))
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    base = oracle.render_fwd(32, 32, r, b["vals"], b["ranges"], pix_err=e)["gauss_err"]
    perm = np.random.default_rng(4).permutation(n)
    rp = {k: v[perm] for k, v in r.items()}
    bp = oracle.bin_f32(sizes, rec["xy"][:, perm], rec["radius"][:, perm], rec["depth"][:, perm])
    got = oracle.render_fwd(32, 32, rp, bp["vals"], bp["ranges"], pix_err=e)["gauss_err"]
    # distinct depths: the same entries blend in the same order, so E is the same
    assert len(np.unique(rec["depth"][0])) == n
    np.testing.assert_array_equal(got, base[perm])


def test_pixel_error_is_channel_mean_of_absolute_difference():
    a = np.array([[[0.5]], [[0.25]], [[1.0]]])
    b = np.array([[[0.0]], [[0.5]], [[1.0]]])
    assert oracle.pixel_error(a, b)[0, 0] == (0.5 + 0.25 + 0.0) / 3


def test_active_set_threshold_is_strict_and_unions_inserted():
    E = np.array([[0.1, 0.5, 0.2, 0.0, 0.3],
                  [0.4, 0.1, 0.2, 0.0, 0.0]])
    act, lst = oracle.active_set(E, 0.2)
    np.testing.assert_array_equal(act, [True, True, False, False, True])
    np.testing.assert_array_equal(lst, [0, 1, 4])
    act, lst = oracle.active_set(E, 0.2, force=[False, False, False, True, False])
    np.testing.assert_array_equal(lst, [0, 1, 3, 4])
    act, lst = oracle.active_set(E, 1.0)
    assert lst.size == 0


def test_mask_grad2d_zeroes_inactive_rows_only():
    g = dict(xy=np.ones((3, 2)), opacity=np.array([1.0, 2.0, 3.0]))
    m = oracle.mask_grad2d(g, [True, False, True])
    np.testing.assert_array_equal(m["xy"], [[1, 1], [0, 0], [1, 1]])
    np.testing.assert_array_equal(m["opacity"], [1.0, 0.0, 3.0])


def test_active_walk_start_state_by_hand():
    # three Gaussians of alpha 0.5 stacked on the centre pixel, the middle one
    # active: weights 0.5, 0.25, 0.125, T_final = 0.125; the walk starts after
    # entry 2 with T = 0.25 and colour behind = 0.125 c_3 + 0.125 bg.
    rec = _records([[8.0, 8.0]] * 3, [[0.01, 0.0, 0.01]] * 3, [0.5, 0.5, 0.5],
                   [[1, 0, 0], [0, 1, 0], [0, 0, 1]], [1.0, 2.0, 3.0])
    bg = (0.2, 0.4, 0.6)
    n = 3
    b = oracle.bin_f32([(16, 16)], rec["xy"][None].astype(np.float32), np.full((1, n), 16, np.int32),
                       rec["depth"][None].astype(np.float32))
    out = oracle.render_fwd(16, 16, rec, b["vals"], b["ranges"], bg, active=[False, True, False])
    assert out["act_last"][8, 8] == 2
    assert out["act_T"][8, 8] == 0.25
    np.testing.assert_allclose(out["act_rest"][8, 8], [0.125 * 0.2, 0.125 * 0.4, 0.125 + 0.125 * 0.6,
                                                       0.125 * 3.0], rtol=1e-14)
    # all active: the walk starts at n_contrib with T_final and only the background behind
    out = oracle.render_fwd(16, 16, rec, b["vals"], b["ranges"], bg, active=[True] * 3)
    np.testing.assert_array_equal(out["act_last"], out["n_contrib"])
    np.testing.assert_array_equal(out["act_T"], out["T"])
    for ch in range(3):
        np.testing.assert_allclose(out["act_rest"][..., ch], out["T"] * bg[ch], atol=1e-15)
    assert (out["act_rest"][..., 3] == 0).all()
    # none active: nothing to walk
    out = oracle.render_fwd(16, 16, rec, b["vals"], b["ranges"], bg, active=[False] * 3)
    assert (out["act_last"] == 0).all() and (out["act_T"] == 1).all() and (out["act_rest"] == 0).all()


def test_active_walk_state_where_nothing_blends_behind():
    # pixels whose last blended entry is active: the walk starts at n_contrib
    # with T_final and only the background behind; and it never starts behind
    # a pixel's last blended entry.
    sizes = [(32, 32)]
    n = 150
    rec = scenes.random_records(sizes, n, seed=12, sigma_px=(1.0, 5.0))
    r = dict(xy=rec["xy"][0].astype(np.float64), conic=rec["conic"][0].astype(np.float64),
             opacity=rec["opacity"].astype(np.float64), rgb=rec["rgb"][0].astype(np.float64),
             depth=rec["depth"][0].astype(np.float64))
    act = np.random.default_rng(13).uniform(size=n) < 0.3
    b = oracle.bin_f32(sizes, rec["xy"], rec["radius"], rec["depth"])
    bg = (0.3, 0.2, 0.1)
    out = oracle.render_fwd(32, 32, r, b["vals"], b["ranges"], bg, active=act)
    sel = (out["act_last"] == out["n_contrib"]) & (out["act_last"] > 0)
    assert sel.sum() > 10
    np.testing.assert_array_equal(out["act_T"][sel], out["T"][sel])
    for ch in range(3):
        np.testing.assert_allclose(out["act_rest"][..., ch][sel], out["T"][sel] * bg[ch], rtol=1e-12)
    assert (out["act_rest"][..., 3][sel] == 0).all()
    assert (out["act_last"] <= out["n_contrib"]).all()
    assert ((out["act_last"] > 0) | (out["act_T"] == 1)).all()
