"""Plain definition of the hybrid coarse-to-fine point-cloud update
(Sec. 3.3, "Hybrid Coarse-to-Fine Updates", and Algorithm 1 of the appendix).
TEST INFRASTRUCTURE ONLY: used by the test suite to check the GPU kernels;
shares no code with them.

One pass of the update takes a point cloud S (positions, SH coefficients,
opacity, radius per point) and hyper-parameters N (voxels per axis), K
(neighbours) and eps (threshold), and runs three stages in order:
  1. voxel reduction: every non-empty voxel of an N x N x N partition is
     replaced by one point carrying the mean of its points' parameters;
  2. outlier removal: a point whose K nearest neighbours lie at distances
     with standard deviation above eps is removed;
  3. point generation: every remaining point contributes one new point whose
     parameters are the mean over its K nearest neighbours.

Readings where the paper leaves details open (each implemented below):
  R1 grid: the axis-aligned cube anchored at the per-axis minimum `lo` of
     the input positions with side = the largest per-axis extent, split into
     N^3 cubic voxels of side h = side / N.  Voxel of p: i_a = floor((p_a -
     lo_a) / h) clamped to [0, N-1], id = (i_z N + i_y) N + i_x.  These are
     integer decisions, so they are taken in fp32 round-to-nearest (the same
     operations on both sides).  h = 0 (all points equal) puts every point in
     voxel 0.
  R2 reduction: every per-point parameter is replaced by the plain mean over
     the voxel (an fp64 sum divided by the count); output in ascending voxel
     id.  The reduced cloud is a point cloud like the input, so its positions
     are stored in fp32: the fp64 mean rounded to nearest.
  R3 neighbours: the K nearest OTHER points of the same set, by fp32 squared
     distance ((dx dx + dy dy) + dz dz) with dx = x_j - x_i, ties broken by
     lower index, in ascending (distance, index) order; K_eff = min(K, n-1).
  R4 outlier test: delta = population standard deviation of the K_eff
     distances d_k = sqrt(d2_k), in fp32: mean = (sequential sum of d_k) /
     K_eff, var = (sequential sum of (d_k - mean)^2) / K_eff, delta =
     sqrt(var).  Removed iff delta > eps.  K_eff = 0 keeps the point.  Every
     point is tested against the same reduced set (a removal does not change
     another point's neighbourhood).
  R5 generation: each survivor yields one point whose parameters are the
     means over its K_eff nearest survivors (self excluded); K_eff = 0
     yields nothing.  Output = survivors (in reduced-set order) followed by
     the generated points (in the same order).

Parity status: pinned by tests/test_oracle_refine.py (voxel ids of a
hand-built lattice, voxel means in closed form, nearest neighbours against
scipy's k-d tree and lattice geometry, the standard deviation of two-valued
and hand-built distance sets in closed form, generation on a symmetric
lattice and for parameters linear in position).
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def grid(pos):
    """R1: (lo[3], side) of the voxel cube, fp32."""
    p = np.asarray(pos, F32)
    lo = p.min(axis=0)
    ext = p.max(axis=0) - lo
    return lo, F32(ext.max())


def voxel_size(pos, n_vox):
    lo, side = grid(pos)
    return lo, F32(side / F32(n_vox))


def cell_coords(pos, lo, h, n_cells):
    """Integer cell coordinates of fp32 positions in a grid with origin lo and
    cell side h, clamped to [0, n_cells - 1] (R1)."""
    p = np.asarray(pos, F32)
    if h == 0:
        return np.zeros(p.shape, np.int64)
    t = (p - lo) / F32(h)
    return np.clip(np.floor(t).astype(np.int64), 0, n_cells - 1)


def voxel_ids(pos, n_vox):
    """R1: voxel id of every point."""
    lo, h = voxel_size(pos, n_vox)
    i = cell_coords(pos, lo, h, n_vox)
    return (i[:, 2] * n_vox + i[:, 1]) * n_vox + i[:, 0]


def voxel_reduce(pos, sh, opacity, radius, n_vox):
    """Stage 1 (R1, R2).  Returns (pos, sh, opacity, radius, voxel ids) of the
    reduced set in ascending voxel id; pos fp32, the rest fp64."""
    p = np.asarray(pos, F32)
    n = p.shape[0]
    if n == 0:
        return (np.zeros((0, 3), F32), np.zeros((0,) + np.shape(sh)[1:]), np.zeros(0),
                np.zeros(0), np.zeros(0, np.int64))
    ids = voxel_ids(p, n_vox)
    order = np.argsort(ids, kind="stable")
    sid = ids[order]
    starts = np.flatnonzero(np.r_[True, sid[1:] != sid[:-1]])
    counts = np.diff(np.r_[starts, n])

    def mean64(a):
        a = np.asarray(a, np.float64)[order]
        c = counts.reshape((-1,) + (1,) * (a.ndim - 1))
        return np.add.reduceat(a, starts, axis=0) / c

    pos_out = mean64(p).astype(F32)
    return pos_out, mean64(sh), mean64(opacity), mean64(radius), sid[starts]


def sq_dist(pi, pj):
    """R3: fp32 squared distance, ((dx dx + dy dy) + dz dz), dx = x_j - x_i."""
    d = np.asarray(pj, F32) - np.asarray(pi, F32)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def knn(pos, k, ref=None, exclude_self=True, chunk=256):
    """R3: brute-force K nearest neighbours.  With ref None the query set is
    the reference set and query i skips point i.  Returns (idx [n, K_eff]
    int64, d2 [n, K_eff] fp32) in ascending (d2, index) order."""
    q = np.asarray(pos, F32)
    r = q if ref is None else np.asarray(ref, F32)
    n, m = q.shape[0], r.shape[0]
    self_set = ref is None and exclude_self
    keff = min(k, m - 1 if self_set else m)
    keff = max(keff, 0)
    idx = np.zeros((n, keff), np.int64)
    d2 = np.zeros((n, keff), F32)
    if keff == 0 or n == 0:
        return idx, d2
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        dd = sq_dist(q[a:b, None, :], r[None, :, :])
        if self_set:
            dd[np.arange(b - a), np.arange(a, b)] = np.inf
        for row in range(b - a):
            idx[a + row], d2[a + row] = _smallest(dd[row], keff)
    return idx, d2


def _smallest(dd, kk):
    """The kk entries of the row dd smallest in (value, index) order: every
    entry not above the kk-th smallest value is a candidate, sorted by
    (value, index)."""
    kth = np.partition(dd, kk - 1)[kk - 1]
    cand = np.flatnonzero(dd <= kth)
    o = cand[np.lexsort((cand, dd[cand]))][:kk]
    return o, dd[o]


def outlier_delta(pos, k):
    """R4: delta of every point (fp32), and K_eff."""
    _, d2 = knn(pos, k)
    return delta_of(d2), d2.shape[1]


def delta_of(d2):
    """R4: delta from rows of neighbour squared distances in ascending
    order ([n, K_eff] fp32)."""
    d2 = np.asarray(d2, F32)
    n, keff = d2.shape
    if keff == 0:
        return np.zeros(n, F32)
    d = np.sqrt(d2)
    s = np.zeros(n, F32)
    for j in range(keff):
        s = s + d[:, j]
    mean = s / F32(keff)
    t = np.zeros(n, F32)
    for j in range(keff):
        e = d[:, j] - mean
        t = t + e * e
    return np.sqrt(t / F32(keff))


def outlier_keep(pos, k, eps):
    """Stage 2 (R4): boolean keep flag of every point."""
    delta, keff = outlier_delta(pos, k)
    if keff == 0:
        return np.ones(len(delta), bool)
    return ~(delta > F32(eps))


def generate(pos, attrs, k):
    """Stage 3 (R5): the generated points' parameters, fp64, and the
    neighbour lists they were averaged over."""
    idx, _ = knn(pos, k)
    if idx.shape[1] == 0:
        return [np.zeros((0,) + np.shape(a)[1:]) for a in attrs], idx
    return [np.asarray(a, np.float64)[idx].mean(axis=1) for a in attrs], idx


def refine(pos, sh, opacity, radius, n_vox, k, eps, stages=7):
    """One pass of Algorithm 1.  stages: bit 0 voxel reduction, bit 1
    outlier removal, bit 2 generation.  Returns a dict with the result and
    the intermediate sets."""
    p = np.asarray(pos, F32)
    cur = [p, np.asarray(sh, np.float64), np.asarray(opacity, np.float64),
           np.asarray(radius, np.float64)]
    out = {}
    if stages & 1:
        rp, rs, ro, rr, vid = voxel_reduce(*cur, n_vox)
        cur = [rp, rs, ro, rr]
        out["voxel_ids"] = vid
    out["reduced"] = [c.copy() for c in cur]
    keep = np.ones(len(cur[0]), bool)
    if stages & 2:
        keep = outlier_keep(np.asarray(cur[0], F32), k, eps)
        cur = [c[keep] for c in cur]
    out["keep"] = keep
    out["survivors"] = [c.copy() for c in cur]
    if stages & 4:
        gen, gidx = generate(np.asarray(cur[0], F32), cur, k)
        out["gen_idx"] = gidx
        if gidx.shape[1] > 0:
            cur = [np.concatenate([np.asarray(c, np.float64), g]) for c, g in zip(cur, gen)]
    out["result"] = cur
    return out
