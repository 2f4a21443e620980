"""Judge of the learned depth prior against the paper's plain initialisation.

GEVO initialises the Gaussians of a newly observed region from a photometric
cost volume over the sliding window (Eq. 1, N = 8 keyframes, 64 hypotheses
over 0.25-25 m at 1/4 resolution) and refines them by optimisation (Section
III-A, III-B).  The protocol here, on the 500k-Gaussian room scene:

  1. a box of the room holding about 50k Gaussians is held out: the "map" is
     the scene without it, the "world" is the whole scene;
  2. the prior is trained on 2000 renders (RGB, depth) of the map only, from
     random poses, so the held-out region is never seen in training;
  3. a sliding window of 8 keyframes (0.15 m apart) looks at the region (world
     renders = observed images); pixels
     the map does not explain (depth or colour differ from the map's render)
     are the new region;
  4. new Gaussians (the same pixels for both methods) are placed at the depth
     from (a) the prior on each keyframe image, (b) the cost volume over the
     8 keyframes with belief propagation (Section III-A2);
  5. each initialisation is optimised for the same number of iterations by the
     local stage of Eq. 2 (E_pho + E_iso over the keyframes, Adam on every
     parameter of the new Gaussians, the map frozen, the keyframe poses held
     fixed); a second protocol updates only their means and colours;
  6. L1 colour and L1 depth against world renders are measured on 16 other
     views near the window, over the new-region pixels.
Every render, loss, gradient, convolution and optimiser step runs in libgevo.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _abi, scenes
from .prior import DepthUNet
from .raster import Pipeline, camera_tensor, gaussians_to_device

W_IMG, H_IMG, F_IMG = 320, 240, 262.5
INSERT_OPACITY = 0.2   # new Gaussians enter the map at opacity 0.2 (Section III-B2)
# belief propagation over the cost volume (the paper gives no parameters): the
# discontinuity cost per hypothesis step (0.39 m) and its truncation, in units
# of the mean absolute grey difference, and the iterations
BP_S, BP_TAU, BP_ITERS = 0.01, 0.1, 10


def heldout_box():
    return np.array([[1.5, 5.0], [-2.0, 2.0], [2.0, 5.0]])


def split_scene(scene, box):
    m = scene["means"]
    inside = np.all((m >= box[:, 0]) & (m <= box[:, 1]), axis=1)
    keep = {k: (v[~inside] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    return keep, int(inside.sum())


def _cam(eye, target, jitter_rs=None):
    if jitter_rs is not None:
        target = np.asarray(target) + jitter_rs.normal(0.0, 0.3, 3)
    R, t = scenes.look_at(eye, target)
    return scenes.camera(R, t, F_IMG, F_IMG, W_IMG / 2, H_IMG / 2, W_IMG, H_IMG)


def region_poses(n, box, seed):
    """Cameras outside the box, 2.5-4.5 m from its centre, looking at it."""
    rs = scenes.rng(seed)
    c = box.mean(axis=1)
    out = []
    while len(out) < n:
        d = rs.normal(size=3)
        d[1] *= 0.2
        d /= np.linalg.norm(d)
        eye = c + d * rs.uniform(2.5, 4.5)
        if np.all(eye > scenes.ROOM_LO + 0.5) and np.all(eye < scenes.ROOM_HI - 0.5) and \
                not np.all((eye >= box[:, 0]) & (eye <= box[:, 1])):
            out.append(_cam(eye, c, rs))
    return out


WINDOW_DIST = 2.3   # metres from the box centre (about 0.6 m from its face)


def window_poses(n, box, seed, step=0.15):
    """A sliding window: n consecutive keyframes WINDOW_DIST from the box centre,
    moving sideways by `step` metres per frame, all looking at the centre."""
    rs = scenes.rng(seed)
    c = box.mean(axis=1)
    while True:
        d = rs.normal(size=3)
        d[1] *= 0.2
        d /= np.linalg.norm(d)
        side = np.cross(d, np.array([0.0, 1.0, 0.0]))
        side /= np.linalg.norm(side)
        eyes = [c + WINDOW_DIST * d + (k - (n - 1) / 2) * step * side for k in range(n)]
        if all(np.all(e > scenes.ROOM_LO + 0.5) and np.all(e < scenes.ROOM_HI - 0.5) and
               not np.all((e >= box[:, 0]) & (e <= box[:, 1])) for e in eyes):
            return [_cam(e, c) for e in eyes], d, side


def near_window_poses(n, box, d, side, seed):
    """Test views near the window: +-0.6 m sideways, +-0.3 m in depth and height."""
    rs = scenes.rng(seed)
    c = box.mean(axis=1)
    out = []
    while len(out) < n:
        e = c + (WINDOW_DIST + rs.uniform(-0.3, 0.3)) * d + rs.uniform(-0.6, 0.6) * side + \
            np.array([0.0, rs.uniform(-0.3, 0.3), 0.0])
        if np.all(e > scenes.ROOM_LO + 0.3) and np.all(e < scenes.ROOM_HI - 0.3):
            out.append(_cam(e, c, rs))
    return out


def random_poses(n, seed):
    rs = scenes.rng(seed)
    out = []
    for _ in range(n):
        eye = rs.uniform(scenes.ROOM_LO + 0.5, scenes.ROOM_HI - 0.5)
        tgt = rs.uniform(scenes.ROOM_LO, scenes.ROOM_HI)
        if np.linalg.norm(tgt - eye) < 1.0:
            tgt = eye + np.array([0.0, 0.0, 1.0])
        out.append(_cam(eye, tgt))
    return out


class Renderer:
    """Forward renders of a fixed Gaussian set for batches of V equal views."""

    def __init__(self, g, V):
        self.g = g
        n = int(g["means"].shape[0])
        self.pipe = Pipeline(n, [(W_IMG, H_IMG)] * V, 1 << 22, colour="sh",
                             sh_degree=g.get("sh_degree", 3),
                             tuning=dict(threads_per_tile=64, persistent=1, blocks_per_sm=0))
        self.V = V

    def render(self, cams):
        assert len(cams) == self.V
        ct = camera_tensor(cams)
        self.pipe.project(self.g, ct)
        self.pipe.bin_sort()
        D = int(self.pipe.n_dup.item())
        if D > self.pipe.capacity:
            self.pipe.last_error()
            self.pipe.alloc_capacity(int(D * 1.3) + 1024)
            self.pipe.bin_sort()
        self.pipe.render_fwd()
        P = W_IMG * H_IMG
        return (self.pipe.rgb.view(self.V, 3, H_IMG, W_IMG).clone(),
                self.pipe.depth.view(self.V, H_IMG, W_IMG).clone(),
                self.pipe.T_final.view(self.V, H_IMG, W_IMG).clone()), P


def render_many(g, cams, batch=16):
    r = Renderer(g, batch)
    rgbs, ds, ts = [], [], []
    for i in range(0, len(cams), batch):
        cs = cams[i:i + batch]
        pad = cs + [cs[-1]] * (batch - len(cs))
        (rgb, d, t), _ = r.render(pad)
        rgbs.append(rgb[:len(cs)]); ds.append(d[:len(cs)]); ts.append(t[:len(cs)])
    return torch.cat(rgbs), torch.cat(ds), torch.cat(ts)


def train_prior(map_g, n_train=2000, epochs=30, batch=32, lr=2e-3, seed=7, log=None):
    """Trains the prior on renders of the map from random poses."""
    cams = random_poses(n_train, seed)
    rgb, D, T = render_many(map_g, cams)
    P = H_IMG * W_IMG
    target = torch.zeros(n_train * P, device="cuda")
    weight = torch.zeros_like(target)
    _abi.prior_call("gevo_depth_target", n_train * P, D.reshape(-1), T.reshape(-1), target, weight)
    net = DepthUNet(batch, H_IMG, W_IMG, seed=seed)
    steps = n_train // batch
    t0 = time.time()
    losses = []
    lr_t = lr
    for ep in range(epochs):
        lr_t = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        acc = 0.0
        for s in range(steps):
            sl = slice(s * batch, (s + 1) * batch)
            net.train_step(rgb[sl].contiguous(), target[sl.start * P:sl.stop * P],
                           weight[sl.start * P:sl.stop * P], lr=lr_t)
            acc += float(net.loss.item()) if s == steps - 1 else 0.0
        losses.append(acc)
        if log:
            log(f"epoch {ep} loss {acc:.4f}")
    torch.cuda.synchronize()
    return net, dict(train_s=time.time() - t0, losses=losses, images=n_train, epochs=epochs)


def predict_depth(net, rgb):
    """rgb [k,3,H,W] (k <= net.nb) -> depth [k,H,W] = exp(predicted log-depth)."""
    k = rgb.shape[0]
    inp = torch.zeros(net.nb, 3, H_IMG, W_IMG, device="cuda")
    inp[:k] = rgb
    pred = net.forward(inp.contiguous()).view(net.nb, H_IMG, W_IMG)[:k]
    return torch.exp(pred)


def new_region_mask(world, mapr):
    """Pixels the map does not explain: expected depth or colour differ."""
    (rw, dw, tw), (rm, dm, tm) = world, mapr
    ew = dw / torch.clamp(1 - tw, min=1e-6)
    em = dm / torch.clamp(1 - tm, min=1e-6)
    dd = torch.abs(ew - em) > 0.25 * ew
    dc = (torch.abs(rw - rm).mean(dim=1) > 0.05)
    return ((dd | dc) & ((1 - tw) > 0.5)).float()


def init_gaussians(depths, rgbs, masks, cams, total, seed=11):
    """One Gaussian per selected new-region pixel at the given depths."""
    k = len(cams)
    n_mask = float(masks.sum().item())
    keep = np.uint32(min(0xFFFFFFFF, int(0xFFFFFFFF * min(1.0, 1.05 * total / max(n_mask, 1.0)))))
    means = torch.zeros(total, 3, device="cuda")
    scales = torch.zeros(total, 3, device="cuda")
    quats = torch.zeros(total, 4, device="cuda")
    opac = torch.zeros(total, device="cuda")
    sh = torch.zeros(total, 16, 3, device="cuda")
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    camt = camera_tensor(cams)
    for i in range(k):
        _abi.prior_call("gevo_unproject", H_IMG, W_IMG, rgbs[i].contiguous(), depths[i].contiguous(),
                        masks[i].contiguous(), camt[i].contiguous(), int(keep), seed + i, 1.5,
                        INSERT_OPACITY, 3,
                        counter, total, means, scales, quats, opac, sh)
    n = min(int(counter.item()), total)
    return dict(means=means[:n].contiguous(), scales=scales[:n].contiguous(),
                quats=quats[:n].contiguous(), opacities=opac[:n].contiguous(),
                sh=sh[:n].contiguous(), sh_degree=3)


def optimise(map_g, new_g, key_cams, key_rgb, iters=100, lr_means=3e-3, lr_sh=2e-2):
    """Adam on the new Gaussians' means and SH, the map frozen."""
    nm = int(map_g["means"].shape[0])
    nn = int(new_g["means"].shape[0])
    g = {k: torch.cat([map_g[k], new_g[k]]).contiguous() for k in ("means", "scales", "quats",
                                                                    "opacities", "sh")}
    g["sh_degree"] = 3
    V = len(key_cams)
    pipe = Pipeline(nm + nn, [(W_IMG, H_IMG)] * V, 1 << 22, colour="sh", sh_degree=3,
                    tuning=dict(threads_per_tile=64, persistent=1, blocks_per_sm=0))
    camt = camera_tensor(key_cams)
    pipe.ensure_capacity(g, camt, 1.5)
    target = key_rgb.reshape(-1).contiguous()
    state = {k: (torch.zeros(nn * (3 if k == "means" else 48), device="cuda"),
                 torch.zeros(nn * (3 if k == "means" else 48), device="cuda")) for k in ("means", "sh")}
    losses = []
    for it in range(iters):
        pipe.step(g, camt, target, want_dxi=False)
        D = int(pipe.n_dup.item())
        if D > pipe.capacity:
            pipe.last_error()
            pipe.alloc_capacity(int(D * 1.3) + 1024)
            continue
        losses.append(float(pipe.loss.sum().item()))
        for k, lr in (("means", lr_means), ("sh", lr_sh)):
            w = g[k].view(-1)[nm * (3 if k == "means" else 48):]
            gr = pipe.grads[k].view(-1)[nm * (3 if k == "means" else 48):]
            m, v = state[k]
            _abi.prior_call("gevo_adam", w.numel(), w, gr, m, v, None, lr, 0.9, 0.999, 1e-8, it + 1)
    return g, losses


# Adam of the judge's local stage: the position and colour rates of the
# means-and-colour protocol, the 3DGS rates for scale, rotation and opacity,
# E_iso as in the mapping update
JUDGE_ADAM = dict(lr_means=3e-3, lr_log_scales=5e-3, lr_quats=1e-3, lr_logit_opacities=5e-2,
                  lr_colour_dc=2e-2, lr_colour_rest=2e-2, beta1=0.9, beta2=0.999, eps=1e-15,
                  lambda_iso=10.0)


def optimise_local(map_g, new_g, key_cams, key_rgb, iters=100):
    """The local stage of Eq. 2 on the new Gaussians: every parameter (mean,
    scale, rotation, opacity, SH), E_pho + E_iso against the keyframes, Adam in
    log-scale / logit space, the map frozen and the keyframe poses held fixed.
    Returns the rasterizer's view of map + optimised new Gaussians, and the
    per-iteration losses."""
    from .mapping import GaussianMap, MapOptimizer, _bits_of
    nm = int(map_g["means"].shape[0])
    nn = int(new_g["means"].shape[0])
    gm = GaussianMap.__new__(GaussianMap)
    gm.dev = map_g["means"].device
    gm.sh_degree, gm.colour, gm.K = 3, "sh", 16
    cat = lambda k: torch.cat([map_g[k], new_g[k]]).contiguous()
    o = torch.clamp(cat("opacities"), 1e-6, 1 - 1e-6)
    gm.p = dict(means=cat("means"), log_scales=torch.log(cat("scales")), quats=cat("quats"),
                logit_opacities=torch.log(o / (1 - o)), colours=cat("sh").view(-1, 16, 3).contiguous())
    gm._derived()
    n_all = nm + nn
    rows = torch.arange(nm, n_all, dtype=torch.int32, device=gm.dev)
    counts = torch.zeros(_abi.active_count_words(n_all), dtype=torch.int32, device=gm.dev)
    counts[0] = nn
    opt = MapOptimizer(gm, JUDGE_ADAM, tuning=dict(threads_per_tile=64, persistent=1, blocks_per_sm=0))
    camt = camera_tensor(key_cams)
    losses = opt.iterate(key_cams, camt, key_rgb.reshape(-1).contiguous(), iters,
                         fixed=[True] * len(key_cams), active=(_bits_of(n_all, nm, n_all, gm.dev),
                                                                rows, counts))
    return gm.gaussians(), losses


def evaluate(g, test_cams, world_test, masks, keep_maps=False):
    """L1 colour over the new-region pixels of the test views, L1 of the mean
    depth over those the render covers (1 - T > 0.5), and that coverage.
    keep_maps: also return the per-pixel errors and the covered mask, for the
    comparison over the pixels two initialisations both cover."""
    rgb, D, T = render_many(g, test_cams)
    rw, dw, tw = world_test
    m = masks > 0.5
    e_px = torch.abs(rgb - rw).mean(dim=1)
    e_rgb = e_px[m].mean().item()
    ew = dw / torch.clamp(1 - tw, min=1e-6)
    eg = D / torch.clamp(1 - T, min=1e-6)
    ok = m & ((1 - T) > 0.5)
    e_d = torch.abs(eg - ew)[ok].mean().item() if ok.any() else float("nan")
    out = dict(l1_rgb=e_rgb, l1_depth=e_d, coverage=float(ok.sum().item() / max(m.sum().item(), 1)))
    if keep_maps:
        out["maps"] = dict(e_rgb=e_px, e_depth=torch.abs(eg - ew), covered=ok)
    return out


def common_metrics(a, b):
    """L1 colour and depth of two evaluated initialisations over the pixels both
    cover (the coverage-matched comparison)."""
    both = a["maps"]["covered"] & b["maps"]["covered"]
    n = int(both.sum().item())
    if n == 0:
        return dict(pixels=0)
    return dict(pixels=n,
                l1_rgb={k: x["maps"]["e_rgb"][both].mean().item() for k, x in (("a", a), ("b", b))},
                l1_depth={k: x["maps"]["e_depth"][both].mean().item() for k, x in (("a", a), ("b", b))})


def run(n=500_000, n_train=2000, epochs=30, iters=100, total_new=50_000, log=None):
    """The whole protocol; returns a dict of results for both initialisations."""
    w = scenes.workload(2, n)
    box = heldout_box()
    world_s = w["scene"]
    map_s, n_held = split_scene(world_s, box)
    world_g = gaussians_to_device(world_s)
    map_g = gaussians_to_device(map_s)
    net, tinfo = train_prior(map_g, n_train=n_train, epochs=epochs, log=log)
    key_cams, d, side = window_poses(8, box, 2024)
    test_cams = near_window_poses(16, box, d, side, 4048)
    world_key = render_many(world_g, key_cams, batch=8)
    map_key = render_many(map_g, key_cams, batch=8)
    key_mask = new_region_mask(world_key, map_key)
    world_test = render_many(world_g, test_cams)
    test_mask = new_region_mask(world_test, render_many(map_g, test_cams))
    key_rgb = world_key[0]
    # (a) learned prior
    d_prior = predict_depth(net, key_rgb)
    # (b) plain: cost volume over the 8 keyframes, each keyframe the reference
    # once, depth by belief propagation over it (Section III-A2)
    rgb_all = key_rgb.contiguous()
    cams_t = camera_tensor(key_cams)
    h4, w4 = H_IMG // 4, W_IMG // 4
    grey = torch.zeros(8, h4, w4, device="cuda")
    vol = torch.zeros(h4 * w4 * 64, device="cuda")
    d_wta = torch.zeros(H_IMG, W_IMG, device="cuda")
    msgs = torch.zeros(2 * 4 * h4 * w4 * 64, device="cuda")
    d_plain = torch.zeros(8, H_IMG, W_IMG, device="cuda")
    for r in range(8):
        _abi.prior_call("gevo_cost_volume", 8, r, H_IMG, W_IMG, rgb_all, cams_t, 64, 0.25, 25.0,
                        grey, vol, d_wta)
        _abi.prior_call("gevo_depth_bp", h4, w4, 64, vol, BP_S, BP_TAU, BP_ITERS, 0.25, 25.0, msgs,
                        d_plain[r], None, None)
    world_depth = world_key[1] / torch.clamp(1 - world_key[2], min=1e-6)
    m = key_mask > 0.5
    res = {"held_out_gaussians": n_held, "train": tinfo,
           "train_images_per_s": tinfo["images"] * tinfo["epochs"] / tinfo["train_s"],
           "init_depth_l1": {"prior": torch.abs(d_prior - world_depth)[m].mean().item(),
                             "plain": torch.abs(d_plain - world_depth)[m].mean().item()}}
    res["new_region_pixels"] = {"keyframes": int(key_mask.sum().item()),
                                "test": int(test_mask.sum().item())}
    maps, maps_mc = {}, {}
    for name, dep in (("prior", d_prior), ("plain", d_plain)):
        new_g = init_gaussians(dep, key_rgb, key_mask, key_cams, total_new)
        if int(new_g["means"].shape[0]) == 0:
            res[name] = dict(new_gaussians=0)
            continue
        before = evaluate({k: (torch.cat([map_g[k], new_g[k]]) if k != "sh_degree" else 3)
                           for k in map_g}, test_cams, world_test, test_mask)
        g, losses = optimise_local(map_g, new_g, key_cams, key_rgb, iters=iters)
        after = evaluate(g, test_cams, world_test, test_mask, keep_maps=True)
        maps[name] = after
        # the secondary protocol: means and colours only, opacity and size as inserted
        g_mc, losses_mc = optimise(map_g, new_g, key_cams, key_rgb, iters=iters)
        after_mc = evaluate(g_mc, test_cams, world_test, test_mask, keep_maps=True)
        maps_mc[name] = after_mc
        res[name] = dict(new_gaussians=int(new_g["means"].shape[0]), before=before,
                         after={k: v for k, v in after.items() if k != "maps"},
                         loss_first=losses[0] if losses else None,
                         loss_last=losses[-1] if losses else None,
                         means_colours_only={k: v for k, v in after_mc.items() if k != "maps"})
    for key, mp in (("common", maps), ("common_means_colours_only", maps_mc)):
        if len(mp) == 2:
            c = common_metrics(mp["prior"], mp["plain"])
            res[key] = dict(pixels=c["pixels"])
            if c["pixels"]:
                res[key]["l1_rgb"] = {"prior": c["l1_rgb"]["a"], "plain": c["l1_rgb"]["b"]}
                res[key]["l1_depth"] = {"prior": c["l1_depth"]["a"], "plain": c["l1_depth"]["b"]}
    return res


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--new", type=int, default=50_000)
    a = ap.parse_args()
    out = run(n=a.n, n_train=a.train, epochs=a.epochs, iters=a.iters, total_new=a.new, log=print)
    print(json.dumps(out))
