"""Seeded synthetic inputs for the rasterizer, shaped like the workloads GEVO runs.

This module only draws random numbers and places cameras; it holds none of the
renderer's arithmetic (no projection, binning, blending or derivative).  Both the
CUDA path and the FP64 oracle take their inputs from here.

The paper's datasets (Replica and TUM RGB-D, Section IV-A) are not available, so
synthetic scenes stand in for them with the paper's image sizes: 640x480 (TUM,
Section III-A1) and 1200x680 (Replica has 2.66x the pixels, Section IV-B).  Every
generator uses numpy's Philox bit generator with a fixed seed (1000 + workload
index) so both sides see identical arrays.

A "scene" is a dict of float32 arrays:
  means [N,3], scales [N,3] (positive), quats [N,4] (w, x, y, z; unit),
  opacities [N] in (0, 1), and either rgb [N,3] or sh [N,(L+1)^2,3] + sh_degree L.
A camera is a dict: R [3,3] world->camera (x right, y down, z forward), t [3],
fx, fy, cx, cy, W, H.
"""
from __future__ import annotations

import numpy as np

ROOM_LO = np.array([-5.0, -2.0, -5.0])
ROOM_HI = np.array([5.0, 2.0, 5.0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def look_at(eye, target, down=(0.0, 1.0, 0.0)):
    """World->camera rotation and translation for a camera at `eye` looking at
    `target`, with world `down` mapped to image-down (world up = -y)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(np.asarray(down, np.float64), f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    return R, t


def camera(R, t, fx, fy, cx, cy, W, H):
    return dict(R=np.asarray(R, np.float32), t=np.asarray(t, np.float32), fx=float(fx),
                fy=float(fy), cx=float(cx), cy=float(cy), W=int(W), H=int(H))


def identity_camera(W, H, f, cx=None, cy=None):
    return camera(np.eye(3), np.zeros(3), f, f, W / 2 if cx is None else cx,
                  H / 2 if cy is None else cy, W, H)


def _attributes(r: np.random.Generator, n: int, sh_degree: int | None):
    """Scale, rotation, opacity and colour distributions shared by all workloads:
    log-scale ~ N(ln 0.03, 0.5), random unit quaternion, opacity = sigmoid(N(0,1)),
    colour uniform [0,1] (or SH: DC uniform [0,1], higher bands N(0, 0.05))."""
    scales = np.exp(r.normal(np.log(0.03), 0.5, size=(n, 3)))
    q = r.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = sigmoid(r.normal(size=n))
    out = dict(scales=scales.astype(np.float32), quats=q.astype(np.float32),
               opacities=opac.astype(np.float32))
    if sh_degree is None:
        out["rgb"] = r.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
        out["sh_degree"] = 0
    else:
        K = (sh_degree + 1) ** 2
        sh = r.normal(0.0, 0.05, size=(n, K, 3))
        sh[:, 0, :] = r.uniform(0.0, 1.0, size=(n, 3))
        out["sh"] = sh.astype(np.float32)
        out["sh_degree"] = int(sh_degree)
    return out


def camera_box_scene(n: int, seed: int, sh_degree: int | None = None,
                     box=((-2.0, 2.0), (-1.5, 1.5), (2.0, 8.0))):
    """Means uniform in a camera-frame box (identity pose)."""
    r = rng(seed)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    means = r.uniform(lo, hi, size=(n, 3)).astype(np.float32)
    s = dict(means=means)
    s.update(_attributes(r, n, sh_degree))
    return s


def room_scene(n: int, seed: int, sh_degree: int | None = 3):
    """Means uniform in the 10 x 4 x 10 m room volume."""
    r = rng(seed)
    means = r.uniform(ROOM_LO, ROOM_HI, size=(n, 3)).astype(np.float32)
    s = dict(means=means)
    s.update(_attributes(r, n, sh_degree))
    return s


def jitter_means(scene, sigma: float, seed: int):
    """Copy of `scene` with means + N(0, sigma) (the target scene of workloads 0/1)."""
    r = rng(seed)
    out = dict(scene)
    out["means"] = (scene["means"] + r.normal(0.0, sigma, size=scene["means"].shape)
                    ).astype(np.float32)
    return out


def random_room_pose(seed: int, margin: float = 0.5):
    """Uniform position at least `margin` from the walls, looking at the centre."""
    r = rng(seed)
    while True:
        eye = r.uniform(ROOM_LO + margin, ROOM_HI - margin)
        if np.linalg.norm(eye) > 0.5:
            return look_at(eye, np.zeros(3))


def circle_poses(n_views: int, radius: float, seed: int, yaw_sigma_deg: float = 10.0):
    """Poses on a circle of `radius` at y = 0, equally spaced, looking at the
    centre, with the viewing direction yawed by N(0, yaw_sigma) degrees."""
    r = rng(seed)
    poses = []
    for k in range(n_views):
        th = 2.0 * np.pi * k / n_views
        eye = np.array([radius * np.cos(th), 0.0, radius * np.sin(th)])
        yaw = np.deg2rad(r.normal(0.0, yaw_sigma_deg))
        d = -eye / np.linalg.norm(eye)
        c, s_ = np.cos(yaw), np.sin(yaw)
        d = np.array([c * d[0] + s_ * d[2], d[1], -s_ * d[0] + c * d[2]])
        poses.append(look_at(eye, eye + d))
    return poses


# ---------------------------------------------------------------------------
# The five workloads.
# ---------------------------------------------------------------------------
def workload(index: int, n: int | None = None):
    """Scene + cameras (+ target scene where the workload defines one).

    0: 20k Gaussians in a camera-frame box, RGB colours, 320x240 (f = 300).
    1: 200k Gaussians in the room, SH degree 3, one 640x480 view (f = 525).
    2: 500k Gaussians in the room, SH degree 3, 16 views on a 2 m circle:
       12 at 640x480 (f = 525) and 4 at 320x240 (f = 262.5).
    3: 1M Gaussians in the room, SH degree 3, one 1200x680 view (f = 600).
    `n` overrides the Gaussian count (smaller parity cases of the same shape)."""
    seed = 1000 + index
    if index == 0:
        n = 20_000 if n is None else n
        scene = camera_box_scene(n, seed, sh_degree=None)
        cams = [identity_camera(320, 240, 300.0, 160.0, 120.0)]
        target = jitter_means(scene, 0.01, seed + 7)
        return dict(scene=scene, cams=cams, target_scene=target, lambda_depth=0.0)
    if index == 1:
        n = 200_000 if n is None else n
        scene = room_scene(n, seed, sh_degree=3)
        R, t = random_room_pose(seed + 1)
        cams = [camera(R, t, 525.0, 525.0, 320.0, 240.0, 640, 480)]
        target = jitter_means(scene, 0.01, seed + 7)
        return dict(scene=scene, cams=cams, target_scene=target, lambda_depth=1.0)
    if index == 2:
        n = 500_000 if n is None else n
        scene = room_scene(n, seed, sh_degree=3)
        cams = []
        for k, (R, t) in enumerate(circle_poses(16, 2.0, seed + 1)):
            if k < 12:
                cams.append(camera(R, t, 525.0, 525.0, 320.0, 240.0, 640, 480))
            else:
                cams.append(camera(R, t, 262.5, 262.5, 160.0, 120.0, 320, 240))
        target = jitter_means(scene, 0.01, seed + 7)
        return dict(scene=scene, cams=cams, target_scene=target, lambda_depth=1.0)
    if index == 3:
        n = 1_000_000 if n is None else n
        scene = room_scene(n, seed, sh_degree=3)
        R, t = random_room_pose(seed + 1)
        cams = [camera(R, t, 600.0, 600.0, 600.0, 340.0, 1200, 680)]
        target = jitter_means(scene, 0.01, seed + 7)
        return dict(scene=scene, cams=cams, target_scene=target, lambda_depth=0.0)
    raise ValueError(f"no workload {index}")


def tracking_subscene(n: int = 2000, seed: int = 1003):
    """The 64x48 finite-difference sub-scene of the 1200x680 tracking workload
    (focal length scaled by 64/1200), Gaussians in a camera-frame box, SH 3."""
    scene = camera_box_scene(n, seed, sh_degree=3, box=((-2.0, 2.0), (-1.5, 1.5), (2.0, 8.0)))
    f = 600.0 * 64.0 / 1200.0
    return scene, [identity_camera(64, 48, f, 32.0, 24.0)]


# ---------------------------------------------------------------------------
# Synthetic 2-D records for stage-isolated tests (binning, blending).
# ---------------------------------------------------------------------------
def random_records(sizes, n: int, seed: int, frac_culled: float = 0.1,
                   sigma_px=(0.5, 30.0), opacity=(0.02, 1.0)):
    """Per (view, Gaussian) 2-D records drawn directly (not projected):
    xy float32 [V,N,2] (may lie off-screen), conic float32 [V,N,3] of a random
    positive-definite ellipse with axes sigma in `sigma_px`, opacity [N],
    rgb [V,N,3], depth float32 [V,N] in (0.5, 10), radius int32 [V,N] = a
    3-sigma bound on the longer axis, 0 for a random `frac_culled` share,
    opacity uniform in `opacity`."""
    r = rng(seed)
    V = len(sizes)
    xy = np.zeros((V, n, 2), np.float32)
    conic = np.zeros((V, n, 3), np.float32)
    depth = np.zeros((V, n), np.float32)
    radius = np.zeros((V, n), np.int32)
    rgb = np.zeros((V, n, 3), np.float32)
    for v, (W, H) in enumerate(sizes):
        xy[v, :, 0] = r.uniform(-20.0, W + 20.0, n)
        xy[v, :, 1] = r.uniform(-20.0, H + 20.0, n)
        s1 = np.exp(r.uniform(np.log(sigma_px[0]), np.log(sigma_px[1]), n))
        s2 = np.exp(r.uniform(np.log(sigma_px[0]), np.log(sigma_px[1]), n))
        th = r.uniform(0.0, np.pi, n)
        c, s = np.cos(th), np.sin(th)
        i1, i2 = 1.0 / s1 ** 2, 1.0 / s2 ** 2
        conic[v, :, 0] = c * c * i1 + s * s * i2
        conic[v, :, 1] = c * s * (i1 - i2)
        conic[v, :, 2] = s * s * i1 + c * c * i2
        depth[v] = r.uniform(0.5, 10.0, n)
        radius[v] = np.ceil(3.0 * np.maximum(s1, s2)).astype(np.int32) + 1
        radius[v][r.uniform(size=n) < frac_culled] = 0
        rgb[v] = r.uniform(0.0, 1.0, (n, 3))
    opac = r.uniform(opacity[0], opacity[1], n).astype(np.float32)
    return dict(xy=xy, conic=conic, depth=depth, radius=radius, rgb=rgb, opacity=opac)


def plane_images(d_star: float, cams, H: int, W: int, seed: int = 0):
    """Seeded keyframe images for the cost-volume tests: each camera (rows of
    cams [nk, 16]: R, t, fx, fy, cx, cy) sees the world plane z = d_star painted
    with a smooth random texture, ray-cast in double precision (pixel i is
    sampled at i + 0.5 - c).  Returns binary32 [nk, 3, H, W] in [0, 1]."""
    r = rng(seed)
    a = r.uniform(1.5, 4.0, size=3)
    b = r.uniform(1.5, 4.0, size=3)
    ph = r.uniform(0, 2 * np.pi, size=3)
    imgs = []
    for c in np.asarray(cams, np.float64):
        R, t = c[:9].reshape(3, 3), c[9:12]
        fx, fy, cx, cy = c[12:16]
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        ray_c = np.stack([(xs + 0.5 - cx) / fx, (ys + 0.5 - cy) / fy, np.ones_like(xs)], -1)
        ray_w = ray_c @ R
        o = -R.T @ t
        s = (d_star - o[2]) / ray_w[..., 2]
        pw = o + s[..., None] * ray_w
        chans = [0.5 + 0.2 * np.sin(a[k] * pw[..., 0] + ph[k]) * np.cos(b[k] * pw[..., 1])
                 + 0.15 * np.sin(2.7 * a[k] * pw[..., 0] + 1.3 * b[k] * pw[..., 1]) for k in range(3)]
        imgs.append(np.stack(chans))
    return np.clip(np.stack(imgs), 0.0, 1.0).astype(np.float32)
