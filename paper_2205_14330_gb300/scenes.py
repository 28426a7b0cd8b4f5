"""Seeded synthetic scenes, cameras and pixel samples.

This module holds input generation only (random draws, surface sampling and
camera placement); none of the renderer's arithmetic lives here, so both the
CUDA path and the FP64 oracle can take their inputs from it.

The paper's datasets (Blender, STNeRF, DSC; Sec. 4) are not available, so
these scenes stand in for them with the paper's shapes: point clouds of a few
hundred thousand to two million points with SH degree 0-3 (Sec. 3.3 uses
l_max = 2), viewed by pinhole cameras with known intrinsics and extrinsics
(Sec. 3.1), 16 cameras on a semicircle for the video case (Sec. 4.2).

Conventions: world->camera X = R P + t with R row-major; the camera looks
down +z with x to the right and y down in the image; fx = fy = (W/2) /
tan(fov/2), cx = W/2, cy = H/2.  Every value that enters the renderer is
rounded to float32 here, so both sides see identical inputs.
"""
from __future__ import annotations

import math

import numpy as np

SH_C0 = 0.28209  # the DC offset of the configs is +0.5 / 0.28209


def rng_for(seed: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------- cameras
def intrinsics(width: int, height: int, fov_deg: float = 50.0):
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return dict(fx=np.float32(f), fy=np.float32(f), cx=np.float32(width / 2.0),
                cy=np.float32(height / 2.0), width=int(width), height=int(height))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-6:
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    return R, t


def camera(eye, width, height, fov_deg=50.0, target=(0.0, 0.0, 0.0)):
    c = intrinsics(width, height, fov_deg)
    c["R"], c["t"] = look_at(eye, target)
    return c


def ring_cameras(n, radius, width, height, start=0.0, span=2 * math.pi, endpoint=False):
    angs = np.linspace(start, start + span, n, endpoint=endpoint)
    return [camera((radius * math.sin(a), 0.0, radius * math.cos(a)), width, height) for a in angs]


def fibonacci_hemisphere(n, radius):
    golden = math.pi * (3.0 - math.sqrt(5.0))
    eyes = []
    for i in range(n):
        y = (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - y * y))
        phi = i * golden
        eyes.append((radius * r * math.cos(phi), radius * y, radius * r * math.sin(phi)))
    return eyes


# ------------------------------------------------------------------ points
def sh_coeffs(rng, n, deg, std=0.1):
    K = (deg + 1) ** 2
    sh = rng.normal(0.0, std, size=(n, K, 3))
    sh[:, 0, :] += 0.5 / SH_C0
    return sh.astype(np.float32)


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def surface_points(rng, n, n_shapes=20, jitter=0.005):
    """Area-weighted samples of a union of random spheres and boxes."""
    shapes = []
    for s in range(n_shapes):
        centre = rng.uniform(-1.0, 1.0, 3)
        if s % 2 == 0:
            r = rng.uniform(0.1, 0.4)
            shapes.append(("sphere", centre, r, None, 4 * math.pi * r * r))
        else:
            h = rng.uniform(0.05, 0.3, 3)
            rot = _random_rotation(rng)
            area = 8.0 * (h[0] * h[1] + h[1] * h[2] + h[0] * h[2])
            shapes.append(("box", centre, h, rot, area))
    areas = np.array([s[4] for s in shapes])
    which = rng.choice(len(shapes), size=n, p=areas / areas.sum())
    pts = np.empty((n, 3))
    for k, (kind, centre, size, rot, _) in enumerate(shapes):
        idx = np.nonzero(which == k)[0]
        m = idx.size
        if m == 0:
            continue
        if kind == "sphere":
            v = rng.normal(size=(m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            pts[idx] = centre + size * v
        else:
            h = size
            fa = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]])  # faces normal to x, y, z
            axis = rng.choice(3, size=m, p=fa / fa.sum())
            sign = rng.choice([-1.0, 1.0], size=m)
            local = rng.uniform(-1.0, 1.0, size=(m, 3)) * h
            local[np.arange(m), axis] = sign * h[axis]
            pts[idx] = centre + local @ rot.T
    pts += rng.normal(0.0, jitter, size=pts.shape)
    return pts.astype(np.float32)


def log_uniform(rng, n, lo, hi):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n)).astype(np.float32)


def _scene(pos, sh, opacity, radius, deg, cams, **extra):
    d = dict(pos=pos, sh=sh, opacity=opacity, radius=radius, deg=deg, cams=cams)
    d.update(extra)
    return d


# ----------------------------------------------------------------- configs
def tiny(seed=0, n=4096, size=128):
    """4,096 points uniform in [-1,1]^3, SH degree 2 ~ N(0, 0.1) with the DC
    offset, radius 0.02, opacity 0.8; one 50-degree camera at distance 2.5
    (128 x 128).  The L2 target is rendered from positions jittered by
    N(0, 0.01)."""
    rng = rng_for(seed)
    pos = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    sh = sh_coeffs(rng, n, 2)
    opacity = np.full(n, 0.8, np.float32)
    radius = np.full(n, 0.02, np.float32)
    cams = [camera((0.0, 0.0, 2.5), size, size)]
    target_pos = (pos + rng.normal(0.0, 0.01, size=pos.shape)).astype(np.float32)
    return _scene(pos, sh, opacity, radius, 2, cams, target_pos=target_pos, loss="l2")


def static_train(seed=0, n=500_000, n_cams=4, size=800):
    """500k surface points (20 spheres/boxes, jitter 0.005), SH degree 2,
    radii log-uniform in [0.003, 0.01], opacity 0.8; four 800 x 800 cameras
    on a ring of radius 4.  The L1 target is rendered from SH coefficients
    perturbed by N(0, 0.1)."""
    rng = rng_for(seed)
    pos = surface_points(rng, n, 20)
    sh = sh_coeffs(rng, n, 2)
    radius = log_uniform(rng, n, 0.003, 0.01)
    opacity = np.full(n, 0.8, np.float32)
    cams = ring_cameras(n_cams, 4.0, size, size)
    target_sh = (sh + rng.normal(0.0, 0.1, size=sh.shape)).astype(np.float32)
    return _scene(pos, sh, opacity, radius, 2, cams, target_sh=target_sh, loss="l1")


BATCH_RESOLUTIONS = [(400, 400), (800, 800), (1280, 720), (1920, 1080)]


def batched_multiview(seed=0, n=1_000_000, n_cams=64, deg=3, resolutions=None):
    """1M surface points (40 shapes), SH degree 3, radii log-uniform in
    [0.003, 0.01]; 64 cameras on a Fibonacci upper hemisphere of radius 4 with
    resolutions drawn uniformly from {400^2, 800^2, 1280x720, 1920x1080}."""
    rng = rng_for(seed)
    pos = surface_points(rng, n, 40)
    sh = sh_coeffs(rng, n, deg)
    radius = log_uniform(rng, n, 0.003, 0.01)
    opacity = np.full(n, 0.8, np.float32)
    res = resolutions or BATCH_RESOLUTIONS
    pick = rng.integers(0, len(res), n_cams)
    cams = [camera(e, *res[k]) for e, k in zip(fibonacci_hemisphere(n_cams, 4.0), pick)]
    return _scene(pos, sh, opacity, radius, deg, cams)


def refine_cloud(seed=0, n=1_000_000, n_shapes=40, outlier_frac=0.01, deg=3):
    """Input of one coarse-to-fine update (Sec. 3.3): surface samples of
    `n_shapes` random shapes (as in batched_multiview) plus a fraction of
    uniform outliers in [-1.5, 1.5]^3, SH of degree `deg`, radii
    log-uniform in [0.003, 0.01], opacity 0.8."""
    rng = rng_for(seed)
    n_out = int(round(n * outlier_frac))
    pos = np.concatenate([surface_points(rng, n - n_out, n_shapes),
                          rng.uniform(-1.5, 1.5, (n_out, 3)).astype(np.float32)])
    pos = pos[rng.permutation(n)]
    sh = sh_coeffs(rng, n, deg)
    radius = log_uniform(rng, n, 0.003, 0.01)
    opacity = np.full(n, 0.8, np.float32)
    return dict(pos=pos, sh=sh, opacity=opacity, radius=radius, deg=deg)


def dynamic_video(seed=0, n=200_000, frames=30, n_cams=16, width=1024, height=768, deg=2):
    """Base cloud of 200k surface points deformed per frame by the sum of four
    seeded sinusoidal displacement fields (amplitude 0.05); SH degree 2;
    16 cameras on a semicircle of radius 4 at 1024 x 768.  Returns one scene
    per frame (shared SH, opacity and radii)."""
    rng = rng_for(seed)
    base = surface_points(rng, n, 20).astype(np.float64)
    sh = sh_coeffs(rng, n, deg)
    radius = log_uniform(rng, n, 0.003, 0.01)
    opacity = np.full(n, 0.8, np.float32)
    a = rng.normal(size=(4, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    w = rng.uniform(1.0, 4.0, size=(4, 3))
    ph = rng.uniform(0.0, 2 * math.pi, size=4)
    frames_pos = []
    for t in range(frames):
        disp = np.zeros_like(base)
        for k in range(4):
            disp += a[k] * np.sin(base @ w[k] + ph[k] + 2 * math.pi * t / frames)[:, None]
        frames_pos.append((base + 0.05 * disp).astype(np.float32))
    cams = ring_cameras(n_cams, 4.0, width, height, start=-math.pi / 2, span=math.pi,
                        endpoint=True)
    return dict(frames=frames_pos, sh=sh, opacity=opacity, radius=radius, deg=deg, cams=cams)


SERVE_SIZES = [100_000, 200_000, 300_000, 500_000, 750_000, 1_000_000, 1_500_000, 2_000_000]
SERVE_DEGS = [0, 1, 2, 3, 0, 1, 2, 3]


def frame_pair(seed=0, n=200_000, deg=2, jitter=0.005, frames=30):
    """Input of one frame initialisation (Sec. 3.4): the cloud of frame 0 of
    `dynamic_video` with its SH, opacity and radii as the trained previous
    frame, and frame 1's positions with N(0, jitter) noise, in a random
    order, as the new frame's initial cloud (no point correspondence)."""
    d = dynamic_video(seed=seed, n=n, frames=frames, deg=deg)
    rng = rng_for(seed + 1)
    p2 = d["frames"][1] + rng.normal(0.0, jitter, d["frames"][1].shape)
    p2 = p2[rng.permutation(n)].astype(np.float32)
    return dict(p1=d["frames"][0], sh=d["sh"], opacity=d["opacity"], radius=d["radius"],
                deg=deg, p2=p2)


def sphere_masks(cams, centres, radii):
    """Foreground masks ([H, W] uint8 per camera) of a union of spheres:
    pixel (x, y) is foreground when the ray through its centre (x + 0.5,
    y + 0.5) hits a sphere in front of the camera."""
    out = []
    for c in cams:
        W, H = int(c["width"]), int(c["height"])
        R = np.asarray(c["R"], np.float64).reshape(3, 3)
        t = np.asarray(c["t"], np.float64).reshape(3)
        eye = -R.T @ t
        xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        d = np.stack([(xs - float(c["cx"])) / float(c["fx"]), (ys - float(c["cy"])) / float(c["fy"]),
                      np.ones_like(xs)], -1) @ R  # world directions (R^T d per pixel)
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        hit = np.zeros((H, W), bool)
        for ctr, r in zip(centres, radii):
            oc = eye - ctr
            b = d @ oc
            disc = b * b - (oc @ oc - r * r)
            hit |= (disc >= 0) & (-b + np.sqrt(np.maximum(disc, 0)) > 0)
        out.append(hit.astype(np.uint8))
    return out


def hull_scene(seed=0, n_spheres=8, n_cams=16, width=256, height=256):
    """Silhouette input of the visual-hull initialisation (Sec. 3.1): a union
    of `n_spheres` spheres (centres in [-0.7, 0.7]^3, radii in [0.15, 0.4])
    seen by `n_cams` cameras on a Fibonacci hemisphere of radius 4; the
    scene box is [-1.5, 1.5]^3."""
    rng = rng_for(seed)
    centres = rng.uniform(-0.7, 0.7, (n_spheres, 3))
    radii = rng.uniform(0.15, 0.4, n_spheres)
    cams = [camera(e, width, height) for e in fibonacci_hemisphere(n_cams, 4.0)]
    return dict(cams=cams, masks=sphere_masks(cams, centres, radii), centres=centres,
                radii=radii, lo=np.full(3, -1.5, np.float32), hi=np.full(3, 1.5, np.float32))


def serving_scenes(seed=0, sizes=None, degs=None):
    """Eight resident scenes of 100k-2M points with SH degree 0-3."""
    rng = rng_for(seed)
    sizes = sizes or SERVE_SIZES
    degs = degs or SERVE_DEGS
    out = []
    for n, deg in zip(sizes, degs):
        pos = surface_points(rng, n, 20)
        out.append(dict(pos=pos, sh=sh_coeffs(rng, n, deg), deg=deg,
                        radius=log_uniform(rng, n, 0.003, 0.01),
                        opacity=np.full(n, 0.8, np.float32)))
    return out


def serving_requests(seed=0, rate=500.0, duration=10.0, n_scenes=8):
    """Poisson arrivals; each request renders a random scene from a random
    camera on a sphere of radius 3-5 at W x H uniform over multiples of 16
    (256..1920 x 256..1080)."""
    rng = rng_for(seed + 1)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        eye = d * rng.uniform(3.0, 5.0)
        W = int(rng.integers(16, 121)) * 16
        H = int(rng.integers(16, 68)) * 16
        reqs.append(dict(t=t, scene=int(rng.integers(0, n_scenes)), cam=camera(eye, W, H)))
    return reqs


# ------------------------------------------------------------ pixel samples
def sample_pixels(cams, n_random=4096, n_tiles=4, tile=16, seed=0, views=None):
    """(view, x, y) int32 triples: ``n_random`` uniform pixels per view plus
    ``n_tiles`` full tile-aligned blocks per view (one touching the bottom-
    right corner, so ragged edge tiles are covered)."""
    rng = rng_for(seed + 7)
    out = []
    for v in (range(len(cams)) if views is None else views):
        W, H = int(cams[v]["width"]), int(cams[v]["height"])
        xs = rng.integers(0, W, n_random)
        ys = rng.integers(0, H, n_random)
        out.append(np.stack([np.full(n_random, v), xs, ys], 1))
        tx, ty = -(-W // tile), -(-H // tile)
        picks = [(tx - 1, ty - 1)] + [(int(rng.integers(0, tx)), int(rng.integers(0, ty)))
                                      for _ in range(max(0, n_tiles - 1))]
        for (a, b) in picks:
            yy, xx = np.mgrid[b * tile:min(H, (b + 1) * tile), a * tile:min(W, (a + 1) * tile)]
            out.append(np.stack([np.full(xx.size, v), xx.ravel(), yy.ravel()], 1))
    return np.concatenate(out).astype(np.int32)
