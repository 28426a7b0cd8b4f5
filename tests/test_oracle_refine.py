"""Pins for the coarse-to-fine update definitions (Sec. 3.3, Algorithm 1)
against closed forms, lattice geometry and scipy's k-d tree."""
import itertools
import math

import numpy as np
import pytest

from oracle import refine_ref as RR


def lattice(n, spacing=1.0):
    g = np.array(list(itertools.product(range(n), repeat=3)), np.float64)[:, ::-1]
    return (g * spacing).astype(np.float32)  # x fastest


def test_voxel_ids_of_cell_centres_and_the_far_corner():
    # cube [0, 1]^3 with N = 4: h = 0.25, centres (i + 0.5) / 4
    n = 4
    ijk = np.array(list(itertools.product(range(n), repeat=3)))
    pts = ((ijk + 0.5) / n).astype(np.float32)
    pts = np.concatenate([pts, np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0.5]], np.float32)])
    ids = RR.voxel_ids(pts, n)
    want = (ijk[:, 2] * n + ijk[:, 1]) * n + ijk[:, 0]
    assert np.array_equal(ids[:-3], want)
    # the minimum corner is voxel 0; the far corner clamps to N - 1 per axis
    assert ids[-3] == 0 and ids[-2] == n ** 3 - 1
    assert ids[-1] == (2 * n + 0) * n + (n - 1)


def test_grid_is_a_cube_over_the_largest_extent():
    pts = np.array([[0, 0, 0], [4, 1, 2]], np.float32)
    lo, side = RR.grid(pts)
    assert np.array_equal(lo, [0, 0, 0]) and side == 4
    lo, h = RR.voxel_size(pts, 8)
    assert h == 0.5
    # (4, 1, 2) -> cells (7 clamped, 2, 4)
    assert RR.voxel_ids(pts, 8)[1] == (4 * 8 + 2) * 8 + 7


def test_voxel_means_in_closed_form():
    rng = np.random.default_rng(0)
    # two clusters well inside two different voxels of a unit cube, N = 2
    a = (0.25 + 0.05 * rng.uniform(-1, 1, (5, 3))).astype(np.float32)
    b = (0.75 + 0.05 * rng.uniform(-1, 1, (3, 3))).astype(np.float32)
    corners = np.array([[0, 0, 0], [1, 1, 1]], np.float32)
    pos = np.concatenate([a, corners, b])
    sh = rng.normal(size=(len(pos), 4, 3))
    op = rng.uniform(size=len(pos))
    rad = rng.uniform(size=len(pos))
    p, s, o, r, vid = RR.voxel_reduce(pos, sh, op, rad, 2)
    assert np.array_equal(vid, [0, 7])
    ia = list(range(5)) + [5]          # cluster a and the min corner: voxel 0
    ib = [6] + list(range(7, 10))      # the max corner and cluster b: voxel 7
    for v, grp in enumerate([ia, ib]):
        assert np.allclose(p[v], pos[grp].astype(np.float64).mean(0), atol=1e-6)
        assert np.allclose(s[v], sh[grp].mean(0), atol=1e-12)
        assert np.allclose(o[v], op[grp].mean(), atol=1e-12)
        assert np.allclose(r[v], rad[grp].mean(), atol=1e-12)


def test_one_point_per_voxel_is_unchanged():
    pos = lattice(4, 0.25)
    rng = np.random.default_rng(1)
    sh = rng.normal(size=(len(pos), 1, 3))
    # extent 0.75, N = 4: voxels of side 0.1875, one lattice point in each
    # occupied voxel (0.25 / 0.1875 = 1.33, 0.5 / 0.1875 = 2.67, 0.75 -> 3)
    p, s, o, r, vid = RR.voxel_reduce(pos, sh, np.ones(len(pos)), np.ones(len(pos)), 4)
    assert len(p) == len(pos)
    order = np.argsort(RR.voxel_ids(pos, 4), kind="stable")
    assert np.array_equal(p, pos[order]) and np.array_equal(s, sh[order])


def test_crowded_voxel_mean_is_accurate():
    # 20000 points in one voxel: the reduced position is the exact mean
    # rounded once to fp32 (within half an ulp; an fp32 running sum drifts
    # by about 1e-4 relative here)
    rng = np.random.default_rng(4)
    pos = np.concatenate([rng.uniform(0.1, 0.2, (20000, 3)), [[0, 0, 0], [1, 1, 1]]]).astype(np.float32)
    p, _, _, _, _ = RR.voxel_reduce(pos, np.zeros((len(pos), 1, 3)), np.zeros(len(pos)),
                                    np.zeros(len(pos)), 2)
    # exact rational mean: the fp32 inputs are integers times 2^-30 here
    scaled = (pos[:20000].astype(np.float64) * 2.0**30).astype(np.int64)
    assert np.array_equal(scaled.astype(np.float64) / 2.0**30, pos[:20000].astype(np.float64))
    from fractions import Fraction
    for a in range(3):
        exact = Fraction(int(scaled[:, a].sum()), 2**30 * 20001)  # voxel 0 holds the min corner too
        err = abs(Fraction(float(p[0, a])) - exact)
        assert err <= Fraction(float(np.spacing(np.float32(float(exact))))) / 2


def test_knn_matches_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1, 1, (700, 3)).astype(np.float32)
    idx, d2 = RR.knn(pos, 8)
    tree = spatial.cKDTree(pos.astype(np.float64))
    dd, ii = tree.query(pos.astype(np.float64), k=9)
    assert np.array_equal(ii[:, 0], np.arange(700))  # itself first
    assert np.array_equal(idx, ii[:, 1:])
    assert np.allclose(np.sqrt(d2), dd[:, 1:], rtol=1e-6)
    # a separate reference set
    ref = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    idx2, _ = RR.knn(pos[:50], 3, ref=ref)
    _, ii2 = spatial.cKDTree(ref.astype(np.float64)).query(pos[:50].astype(np.float64), k=3)
    assert np.array_equal(idx2, ii2)


def test_knn_on_a_lattice_with_index_ties():
    pos = lattice(5)
    centre = (2 * 5 + 2) * 5 + 2
    idx, d2 = RR.knn(pos, 6)
    # the 6 axis neighbours at distance 1, ties in index order
    assert np.array_equal(d2[centre], np.ones(6, np.float32))
    want = sorted(centre + d for d in (-25, -5, -1, 1, 5, 25))
    assert list(idx[centre]) == want
    # K_eff = n - 1 when K exceeds it
    idx, d2 = RR.knn(pos[:3], 10)
    assert idx.shape == (3, 2)


def test_delta_of_two_valued_distances():
    # lattice interior: 6 neighbours at 1 and 12 at sqrt(2)
    pos = lattice(5)
    centre = (2 * 5 + 2) * 5 + 2
    d6, _ = RR.outlier_delta(pos, 6)
    assert d6[centre] == 0.0
    d18, _ = RR.outlier_delta(pos, 18)
    p = 6 / 18
    want = (math.sqrt(2) - 1) * math.sqrt(p * (1 - p))
    assert abs(d18[centre] - want) < 1e-6


def test_delta_of_hand_placed_neighbours_and_threshold():
    # a point with neighbours at distances 1, 2, 3, 4 along the axes; the
    # rest of the cloud is far away
    far = 100.0 + lattice(3)
    pts = np.concatenate([np.array([[0, 0, 0], [1, 0, 0], [0, -2, 0], [0, 0, 3],
                                    [-4, 0, 0]], np.float32), far])
    delta, keff = RR.outlier_delta(pts, 4)
    want = np.std([1.0, 2.0, 3.0, 4.0])  # population std = sqrt(1.25)
    assert keff == 4 and abs(delta[0] - want) < 1e-6
    assert not RR.outlier_keep(pts, 4, 1.1)[0]
    assert RR.outlier_keep(pts, 4, 1.2)[0]


def test_generation_on_a_symmetric_lattice_and_linear_parameters():
    pos = lattice(5)
    centre = (2 * 5 + 2) * 5 + 2
    A = np.array([[0.5, -1.0, 2.0], [1.5, 0.25, -0.75]])
    f = pos.astype(np.float64) @ A.T + np.array([0.1, -0.2])
    (gp, gf), idx = RR.generate(pos, [pos, f], 6)
    # the six axis neighbours average to the centre itself
    assert np.allclose(gp[centre], pos[centre], atol=1e-12)
    # corner (0, 0, 0): neighbours (1,0,0), (0,1,0), (0,0,1) -> (1/3, 1/3, 1/3)
    (gp3, gf3), _ = RR.generate(pos, [pos, f], 3)
    assert np.allclose(gp3[0], [1 / 3] * 3, atol=1e-12)
    # a parameter linear in position averages to its value at the mean
    assert np.allclose(gf, gp @ A.T + np.array([0.1, -0.2]), atol=1e-9)


def test_refine_composition_and_degenerate_inputs():
    rng = np.random.default_rng(3)
    pos = rng.uniform(-1, 1, (400, 3)).astype(np.float32)
    sh = rng.normal(size=(400, 4, 3))
    op, rad = rng.uniform(size=400), rng.uniform(size=400)
    out = RR.refine(pos, sh, op, rad, n_vox=6, k=5, eps=0.05)
    nred = len(out["reduced"][0])
    assert nred == len(np.unique(RR.voxel_ids(pos, 6)))
    nsurv = int(out["keep"].sum())
    assert 0 < nsurv < nred
    assert len(out["result"][0]) == 2 * nsurv
    # survivors come first, unchanged
    assert np.array_equal(out["result"][0][:nsurv], out["reduced"][0][out["keep"]])
    # all points equal: one voxel, one point, kept, nothing generated
    same = np.zeros((10, 3), np.float32)
    o2 = RR.refine(same, np.zeros((10, 1, 3)), np.ones(10), np.ones(10), 8, 4, 0.0)
    assert len(o2["result"][0]) == 1
    # empty input
    o3 = RR.refine(np.zeros((0, 3), np.float32), np.zeros((0, 1, 3)), np.zeros(0),
                   np.zeros(0), 8, 4, 0.1)
    assert len(o3["result"][0]) == 0
