"""Pins of the FP64 U-Net oracle (the learned depth prior's reference): its
backward against central finite differences of its own forward, guarded so a
ReLU or max-pool decision never flips inside the difference, and the
adjoint identities of its shift / pool / upsample steps."""
import numpy as np

from oracle import unet


def _events(cache, chans):
    keys = [k for k in cache if k[:1] in ("a", "b", "d") or k.startswith("arg")]
    return {k: (cache[k] > 0) if not k.startswith("arg") else cache[k] for k in keys}


def test_shift_and_unshift_are_adjoint():
    rs = np.random.default_rng(0)
    x = rs.normal(size=(2, 5, 7, 3))
    g = rs.normal(size=(2, 5, 7, 3))
    for ky in range(3):
        for kx in range(3):
            assert np.isclose((unet._shift(x, ky, kx) * g).sum(), (x * unet._unshift(g, ky, kx)).sum())


def test_conv3x3_matches_direct_sum():
    rs = np.random.default_rng(1)
    x = rs.normal(size=(1, 4, 5, 2))
    w = rs.normal(size=(3, 9, 2))
    b = rs.normal(size=3)
    y = unet.conv3x3(x, w, b)
    for yy in range(4):
        for xx in range(5):
            acc = b.copy()
            for ky in range(3):
                for kx in range(3):
                    sy, sx = yy + ky - 1, xx + kx - 1
                    if 0 <= sy < 4 and 0 <= sx < 5:
                        acc += w[:, 3 * ky + kx, :] @ x[0, sy, sx]
            np.testing.assert_allclose(y[0, yy, xx], acc, rtol=1e-13)


def test_pool_upsample_adjoints():
    rs = np.random.default_rng(2)
    x = rs.normal(size=(2, 4, 6, 3))
    m, arg = unet.maxpool2(x)
    np.testing.assert_array_equal(m, np.maximum(np.maximum(x[:, ::2, ::2], x[:, ::2, 1::2]),
                                                np.maximum(x[:, 1::2, ::2], x[:, 1::2, 1::2])))
    g = rs.normal(size=m.shape)
    dx = unet.maxpool2_bwd(arg, g, x.shape)
    assert np.isclose(dx.sum(), g.sum()) and (np.count_nonzero(dx) == g.size)
    u = rs.normal(size=(2, 3, 4, 5))
    G = rs.normal(size=(2, 6, 8, 5))
    assert np.isclose((unet.upsample2(u) * G).sum(), (u * unet.upsample2_bwd(G)).sum())


def test_unet_backward_matches_central_differences():
    chans = (8, 16)
    rs = np.random.default_rng(3)
    p = unet.init_params(chans, seed=4)
    x = rs.normal(size=(2, 8, 8, 8))
    target = rs.normal(size=2 * 64)
    weight = (rs.uniform(size=2 * 64) > 0.2).astype(float)
    pred, cache = unet.forward(p, x, chans)
    L, dpred = unet.loss_l1(pred, target, weight)
    g = unet.backward(p, cache, dpred, chans)
    ev0 = _events(cache, chans)
    h = 1e-6
    checked = 0
    for name in p:
        for which in (0, 1):
            arr = p[name][which]
            flat_idx = rs.choice(arr.size, size=min(arr.size, 6), replace=False)
            for fi in flat_idx:
                vals = []
                ok = True
                for s in (1, -1):
                    q = {k: (v[0].copy(), v[1].copy()) for k, v in p.items()}
                    q[name][which].reshape(-1)[fi] += s * h
                    pr, c2 = unet.forward(q, x, chans)
                    ev = _events(c2, chans)
                    ok &= all(np.array_equal(ev[k], ev0[k]) for k in ev0)
                    ok &= np.array_equal(np.sign(pr - target), np.sign(pred - target))
                    vals.append(unet.loss_l1(pr, target, weight)[0])
                if not ok:
                    continue
                fd = (vals[0] - vals[1]) / (2 * h)
                an = g[name][which].reshape(-1)[fi]
                assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-8, (name, which, fi, fd, an)
                checked += 1
    assert checked >= 40
