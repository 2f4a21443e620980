"""Pins of the optimisation-step oracle (oracle/optim.py): the isotropic loss
against closed forms and finite differences, the activation chain rule
against finite differences, Adam against hand-worked steps, the Rodrigues
retraction against rotation identities, and pruning against a hand case."""
import numpy as np

from oracle import optim


def test_iso_loss_closed_forms_and_fd():
    E, g = optim.iso_loss([[1.0, 1.0, 1.0]], 10.0)
    assert E == 0.0 and (g == 0).all()
    E, g = optim.iso_loss([[1.0, 2.0, 3.0]], 10.0)     # |d| = 1 + 0 + 1, n = 1
    assert E == 20.0
    np.testing.assert_allclose(g, [[10 * (-1 - 0 / 3), 10 * (0 - 0 / 3), 10 * (1 - 0 / 3)]])
    rs = np.random.default_rng(0)
    s = rs.uniform(0.01, 0.1, size=(7, 3))
    E, g = optim.iso_loss(s, 3.0)
    h = 1e-7
    for i in range(7):
        for a in range(3):
            sp, sm = s.copy(), s.copy()
            sp[i, a] += h
            sm[i, a] -= h
            fd = (optim.iso_loss(sp, 3.0)[0] - optim.iso_loss(sm, 3.0)[0]) / (2 * h)
            assert abs(fd - g[i, a]) <= 1e-6, (i, a, fd, g[i, a])


def test_chain_rule_of_activations_by_fd():
    rs = np.random.default_rng(1)
    n, K = 5, 4
    raw = dict(means=rs.normal(size=(n, 3)), log_scales=rs.normal(-3, 0.5, size=(n, 3)),
               quats=rs.normal(size=(n, 4)), logit_opacities=rs.normal(size=n),
               sh=rs.normal(size=(n, K, 3)))
    # L = sum(w_s * exp(log s)) + sum(w_o * sigmoid(logit)) + linear terms
    w = dict(means=rs.normal(size=(n, 3)), scales=rs.normal(size=(n, 3)), quats=rs.normal(size=(n, 4)),
             opacities=rs.normal(size=n), sh=rs.normal(size=(n, K, 3)))

    def L(r):
        return ((w["means"] * r["means"]).sum() + (w["scales"] * np.exp(r["log_scales"])).sum()
                + (w["quats"] * r["quats"]).sum() + (w["opacities"] * optim.sigmoid(r["logit_opacities"])).sum()
                + (w["sh"] * r["sh"]).sum())
    ch, E = optim.chain_grads(raw, w, np.arange(n))
    assert E == 0.0
    h = 1e-6
    for k in optim.GROUPS:
        for i in range(raw[k].size):
            rp = {kk: v.copy() for kk, v in raw.items()}
            rm = {kk: v.copy() for kk, v in raw.items()}
            rp[k].reshape(-1)[i] += h
            rm[k].reshape(-1)[i] -= h
            fd = (L(rp) - L(rm)) / (2 * h)
            assert abs(fd - ch[k].reshape(-1)[i]) <= 1e-7 * (1 + abs(fd)), (k, i)


def test_adam_hand_worked_steps():
    p, m, v = optim.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 0.1, 0.9, 0.999, 0.0, 1)
    # first step: m_hat = g, v_hat = g^2, so the step is lr * sign(g)
    np.testing.assert_allclose(p, [0.9])
    np.testing.assert_allclose(m, [0.05])
    np.testing.assert_allclose(v, [0.00025])
    p2, m2, v2 = optim.adam(p, np.array([-1.0]), m, v, 0.1, 0.9, 0.999, 0.0, 2)
    mh = (0.9 * 0.05 - 0.1) / (1 - 0.81)
    vh = (0.999 * 0.00025 + 0.001) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p2, [0.9 - 0.1 * mh / np.sqrt(vh)])


def test_rodrigues_and_retraction():
    R = optim.rodrigues([0, 0, np.pi / 2])
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    rs = np.random.default_rng(2)
    phi = rs.normal(size=3)
    R = optim.rodrigues(phi)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    np.testing.assert_allclose(R @ phi, phi, atol=1e-14)
    # first Adam step of the twist is -lr * sign(dxi)
    R0, t0 = optim.rodrigues(rs.normal(size=3)), rs.normal(size=3)
    dxi = np.array([0.3, -0.2, 0.1, -0.4, 0.5, 0.6])
    R1, t1, m, v = optim.pose_step(R0, t0, dxi, np.zeros(6), np.zeros(6), 0.01, 0.02, 1, eps=0.0)
    xi = -np.array([0.01, 0.01, 0.01, 0.02, 0.02, 0.02]) * np.sign(dxi)
    Rx = optim.rodrigues(xi[3:])
    np.testing.assert_allclose(R1, Rx @ R0, atol=1e-14)
    np.testing.assert_allclose(t1, Rx @ t0 + xi[:3], atol=1e-14)


def test_pruning_keeps_non_candidates_and_strong_candidates():
    o = np.array([0.1, 0.9, 0.5, 0.7, 0.69, 0.2])
    keep = optim.keep_after_pruning(o, [0, 1, 3, 4], 0.7)
    np.testing.assert_array_equal(keep, [1, 2, 3, 5])
