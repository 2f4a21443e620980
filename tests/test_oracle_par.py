"""The threaded whole-view oracle runner (tests/oracle_par.py) returns what the
plain oracle returns: identical forward outputs, and gradients equal up to the
order of the sums (no GPU needed)."""
import numpy as np

import oracle
import oracle_par
from paper_2409_09295_gb300 import scenes


def test_threaded_oracle_equals_plain_oracle():
    w = scenes.workload(2, n=3000)
    cams = [w["cams"][0], w["cams"][13]]
    cams = [dict(c, W=c["W"] // 4 + 3, H=c["H"] // 4 + 5, cx=c["cx"] / 4, cy=c["cy"] / 4,
                 fx=c["fx"] / 4, fy=c["fy"] / 4) for c in cams]
    scene = w["scene"]
    outs, projs, b = oracle.render_views(scene, cams)
    outs2, projs2, b2 = oracle_par.render_views(scene, cams)
    for o, o2 in zip(outs, outs2):
        for k in o:
            np.testing.assert_array_equal(o[k], o2[k], err_msg=k)
    for p, p2 in zip(projs, projs2):
        for k in p:
            np.testing.assert_array_equal(p[k], p2[k], err_msg=k)
    for k in ("keys", "vals", "ranges"):
        np.testing.assert_array_equal(b[k], b2[k])
    rs = np.random.default_rng(3)
    gC = [rs.normal(size=(3, c["H"], c["W"])) for c in cams]
    gD = [rs.normal(size=(c["H"], c["W"])) for c in cams]
    gT = [rs.normal(size=(c["H"], c["W"])) for c in cams]
    acc, dxi, g2d = oracle.backward_views(scene, cams, projs, b, gC, gD, gT)
    acc2, dxi2, g2d2 = oracle_par.backward_views(scene, cams, projs2, b2, gC, gD, gT)
    assert any(np.abs(a).max() > 0 for a in acc.values())
    for k in acc:
        np.testing.assert_allclose(acc2[k], acc[k], rtol=1e-10, atol=1e-13, err_msg=k)
    np.testing.assert_allclose(dxi2, dxi, rtol=1e-10, atol=1e-13)
    for a, a2 in zip(g2d, g2d2):
        for k in a:
            np.testing.assert_allclose(a2[k], a[k], rtol=1e-10, atol=1e-13, err_msg=k)
