"""Plain definition of the visual-hull initialisation and the consistency
check (Sec. 3.1 "Point Cloud Initialization" and the appendix's
"Additional Initialization Details").  TEST INFRASTRUCTURE ONLY: used by
the test suite to check the GPU kernels; shares no code with them.

Consistency check of a point p against N views with foreground masks M_i:
    CC(p) = 1  iff  M_i(pixel of p in view i) > 0 for every i,
where the pixel is that of the projection of Eq. 1.  Initialisation:
uniform random points in the scene volume are kept iff CC = 1 (rejection
sampling); the SH coefficients of the kept points are drawn from N(0, 1).

Readings where the paper leaves details open (each implemented below):
  H1 projection, in fp32 round-to-nearest with the same operation order as
     the renderer: X = ((R0 px + R1 py) + R2 pz) + t per row,
     u = fx (X.x / X.z) + cx, v = fy (X.y / X.z) + cy; pixel (floor u,
     floor v) (pixel (0, 0) covers [0, 1)^2).  A point with X.z <= z_near
     or a pixel outside the image counts as background.
  H2 random numbers: one counter-based generator, SplitMix64 (Steele, Lea
     and Flood, OOPSLA 2014): output i of stream `seed` is
        z = seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64),
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
        z = (z ^ (z >> 27)) * 0x94D049BB133111EB,  z ^ (z >> 31);
     a uniform in [0, 1) is (z >> 40) * 2^-24 (exact in fp32).
  H3 candidate j of the sampler: coordinates lo_a + u_a (hi_a - lo_a) in
     fp32 (product rounded, then sum rounded), with u_a = output 3 j + a.
     The result is the first n_target accepted candidates in candidate
     order.
  H4 SH of kept point q (q-th accepted, coefficient c of C = 3 K): Box-
     Muller on outputs of the stream seed ^ 0x5DEECE66D, pair index
     floor((q C + c) / 2): u1 = ((z1 >> 40) + 1) 2^-24, u2 = (z2 >> 40)
     2^-24 from outputs 2 p and 2 p + 1; r = sqrt(-2 ln u1);
     even index: r cos(2 pi u2), odd: r sin(2 pi u2).  (No decision depends
     on these values; they are compared to rounding.)

Parity status: pinned by tests/test_oracle_hull.py (projection of points on
and off the optical axis and behind the camera; the check for points deep
inside and far outside a sphere seen by several cameras; uniformity of the
candidates and normality of the SH draws by Kolmogorov-Smirnov tests; the
ordering of the kept points).
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32
U64 = np.uint64
_GOLDEN = U64(0x9E3779B97F4A7C15)
_M1 = U64(0xBF58476D1CE4E5B9)
_M2 = U64(0x94D049BB133111EB)
SH_STREAM = 0x5DEECE66D


def splitmix64(seed, idx):
    """H2: outputs idx (array of non-negative integers) of stream `seed`."""
    with np.errstate(over="ignore"):
        z = U64(seed) + (np.asarray(idx, np.uint64) + U64(1)) * _GOLDEN
        z = (z ^ (z >> U64(30))) * _M1
        z = (z ^ (z >> U64(27))) * _M2
        return z ^ (z >> U64(31))


def uniform24(z):
    return (z >> U64(40)).astype(np.float64) * 2.0 ** -24


def candidates(seed, first, count, lo, hi):
    """H3: candidates first .. first + count - 1 ([count, 3] fp32)."""
    j = np.arange(first, first + count, dtype=np.uint64)
    u = np.stack([uniform24(splitmix64(seed, U64(3) * j + U64(a))) for a in range(3)], 1)
    lo = np.asarray(lo, F32)
    ext = np.asarray(hi, F32) - lo
    return (ext * u.astype(F32)) + lo


def pixels(pos, cam, z_near=0.01):
    """H1: integer pixel (x, y) of every point, or (-1, -1) when the point is
    behind the near plane or outside the image."""
    p = np.asarray(pos, F32)
    R = np.asarray(cam["R"], F32).reshape(3, 3)
    t = np.asarray(cam["t"], F32).reshape(3)
    X = [((R[r, 0] * p[:, 0] + R[r, 1] * p[:, 1]) + R[r, 2] * p[:, 2]) + t[r] for r in range(3)]
    ok = X[2] > F32(z_near)
    z = np.where(ok, X[2], F32(1))
    u = F32(cam["fx"]) * (X[0] / z) + F32(cam["cx"])
    v = F32(cam["fy"]) * (X[1] / z) + F32(cam["cy"])
    W, H = int(cam["width"]), int(cam["height"])
    ok &= (u >= 0) & (v >= 0) & (u < W) & (v < H)
    x = np.where(ok, np.floor(np.where(ok, u, 0)), -1).astype(np.int64)
    y = np.where(ok, np.floor(np.where(ok, v, 0)), -1).astype(np.int64)
    return x, y


def consistency(pos, cams, masks, z_near=0.01):
    """CC of every point: masks[i] is view i's [H, W] array (> 0 foreground)."""
    keep = np.ones(len(pos), bool)
    for cam, m in zip(cams, masks):
        x, y = pixels(pos, cam, z_near)
        inside = x >= 0
        fg = np.zeros(len(pos), bool)
        fg[inside] = np.asarray(m)[y[inside], x[inside]] > 0
        keep &= fg
    return keep


def hull_init(lo, hi, cams, masks, n_target, seed, batch=1 << 16, max_candidates=1 << 26,
              z_near=0.01):
    """Rejection sampling (H3): the first n_target kept candidates, and the
    number of candidates drawn until then (all of the last batch's prefix up
    to the n_target-th acceptance)."""
    kept, drawn = [], 0
    need = n_target
    while need > 0 and drawn < max_candidates:
        cnt = min(batch, max_candidates - drawn)
        c = candidates(seed, drawn, cnt, lo, hi)
        ok = np.nonzero(consistency(c, cams, masks, z_near))[0]
        if len(ok) >= need:
            kept.append(c[ok[:need]])
            drawn += int(ok[need - 1]) + 1
            need = 0
            break
        kept.append(c[ok])
        need -= len(ok)
        drawn += cnt
    pos = np.concatenate(kept) if kept else np.zeros((0, 3), F32)
    return pos, drawn


def sh_normals(seed, n_points, n_coef):
    """H4: [n_points, n_coef] standard normals (fp64)."""
    k = np.arange(n_points * n_coef, dtype=np.uint64)
    pair = k // U64(2)
    s = U64(seed) ^ U64(SH_STREAM)
    u1 = ((splitmix64(s, U64(2) * pair) >> U64(40)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = uniform24(splitmix64(s, U64(2) * pair + U64(1)))
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * math.pi * u2
    out = np.where(k % U64(2) == 0, r * np.cos(ang), r * np.sin(ang))
    return out.reshape(n_points, n_coef)
