"""FP64 numpy oracle of the map and pose optimisation steps of the local and
global stages (Section III-B1, Eq. 2; Section III-B2, Eq. 3) -- test
infrastructure only.

  - isotropic loss E_iso (the regulariser of Eq. 2, "prevents elongated or thin
    Gaussians"): lam / n * sum_g sum_a |s_ga - mean_a' s_ga'| over the scales
    of the Gaussians being optimised, with its gradient (sign(0) = 0);
  - the optimisation parameters: means, log-scales, raw quaternions,
    opacity logits and SH coefficients; the rasterizer sees exp(log-scale) and
    sigmoid(logit), so a gradient w.r.t. the activated value chains as
    dL/dlog s = dL/ds * s and dL/dlogit = dL/do * o (1 - o);
  - Adam (Kingma and Ba, 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  - the pose retraction used with the left-perturbation twist xi = (rho, phi)
    of the rasterizer's pose gradient: R <- Rod(phi) R, t <- Rod(phi) t + rho,
    Rod the Rodrigues rotation;
  - pruning after the global stage: a candidate whose opacity is below the
    threshold is removed, every other Gaussian kept, order preserved.
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "log_scales", "quats", "logit_opacities", "sh")


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def iso_loss(scales, lam):
    """E_iso and dE_iso/dscales for activated scales [n, 3]."""
    s = np.asarray(scales, np.float64)
    n = s.shape[0]
    if n == 0:
        return 0.0, np.zeros_like(s)
    d = s - s.mean(axis=1, keepdims=True)
    sg = np.sign(d)
    E = lam / n * np.abs(d).sum()
    # d|s_a - m| / ds_b = sg_a (delta_ab - 1/3)
    g = lam / n * (sg - sg.sum(axis=1, keepdims=True) / 3.0)
    return float(E), g


def adam(p, g, m, v, lr, b1, b2, eps, t):
    """One Adam step (returns new p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def gaussian_step(raw, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-15, lam_iso=0.0,
                  rows=None):
    """One optimiser step of the Gaussian parameters.

    raw: dict GROUPS -> arrays; grads: gradients w.r.t. the rasterizer inputs
    (means, scales, quats, opacities, sh); state: dict group -> (m, v); lr:
    dict group -> learning rate (0 = frozen: value and moments unchanged; the SH
    group takes lr["sh"] for the degree-0 row and lr["sh_rest"] for the others); rows: indices of the
    Gaussians being optimised (None = all); E_iso over those rows with weight
    lam_iso is added to the scale gradient.  Returns (raw', state', E_iso)."""
    idx = np.arange(raw["means"].shape[0]) if rows is None else np.asarray(rows, np.int64)
    out = {k: np.array(v, np.float64, copy=True) for k, v in raw.items()}
    st = {k: (np.array(m, np.float64, copy=True), np.array(v, np.float64, copy=True))
          for k, (m, v) in state.items()}
    chained, E = chain_grads(raw, grads, idx, lam_iso)
    for k in GROUPS:
        m, v = st[k]
        if k == "sh":
            lrs = np.full(out["sh"].shape[1:], lr["sh_rest"])
            lrs[0] = lr["sh"]
            lrs = np.broadcast_to(lrs[None], out["sh"][idx].shape)
        else:
            lrs = np.broadcast_to(np.float64(lr[k]), out[k][idx].shape)
        p2, m2, v2 = adam(out[k][idx], chained[k], m[idx], v[idx], lrs, b1, b2, eps, t)
        live = lrs != 0.0            # a zero learning rate freezes the value and its moments
        out[k][idx] = np.where(live, p2, out[k][idx])
        m[idx] = np.where(live, m2, m[idx])
        v[idx] = np.where(live, v2, v[idx])
    return out, st, E


def chain_grads(raw, grads, idx, lam_iso=0.0):
    """Gradients w.r.t. the optimisation parameters of rows idx, from those
    w.r.t. the rasterizer inputs, with E_iso over those rows added.  Returns
    (dict group -> gradient, E_iso)."""
    s = np.exp(np.asarray(raw["log_scales"], np.float64)[idx])
    o = sigmoid(np.asarray(raw["logit_opacities"], np.float64)[idx])
    E, giso = iso_loss(s, lam_iso)
    gs = np.asarray(grads["scales"], np.float64)[idx] + giso
    return {
        "means": np.asarray(grads["means"], np.float64)[idx],
        "log_scales": gs * s,
        "quats": np.asarray(grads["quats"], np.float64)[idx],
        "logit_opacities": np.asarray(grads["opacities"], np.float64)[idx] * o * (1.0 - o),
        "sh": np.asarray(grads["sh"], np.float64)[idx],
    }, E


def rodrigues(phi):
    phi = np.asarray(phi, np.float64)
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th == 0.0:
        return np.eye(3)
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / th ** 2 * K @ K


def pose_step(R, t, dxi, m, v, lr_rho, lr_phi, step, b1=0.9, b2=0.999, eps=1e-15):
    """Adam on the twist of one view, then the retraction: returns (R', t', m', v')."""
    lrs = np.array([lr_rho] * 3 + [lr_phi] * 3)
    xi, m, v = adam(np.zeros(6), np.asarray(dxi, np.float64), m, v, lrs, b1, b2, eps, step)
    Rx = rodrigues(xi[3:])
    return Rx @ np.asarray(R, np.float64), Rx @ np.asarray(t, np.float64) + xi[:3], m, v


def keep_after_pruning(opacities, candidates, threshold):
    """Indices kept (ascending): every non-candidate, and candidates whose
    opacity is not below the threshold."""
    o = np.asarray(opacities, np.float64)
    drop = np.zeros(o.size, bool)
    c = np.asarray(candidates, np.int64)
    drop[c] = o[c] < threshold
    return np.nonzero(~drop)[0]
