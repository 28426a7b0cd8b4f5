"""Pins for the frame-initialisation definitions (Sec. 3.4): the Chamfer
distance and its gradient, the parameter transfer and the descent loop."""
import itertools

import numpy as np
import pytest

from oracle import frame_init_ref as FI

F32 = np.float32


def test_identical_clouds_have_zero_distance_and_gradient():
    rng = np.random.default_rng(0)
    p = rng.uniform(-1, 1, (200, 3)).astype(F32)
    cd, g, nn12, nn21 = FI.chamfer(p, p[::-1].copy())
    assert cd == 0.0 and np.all(g == 0)
    assert np.array_equal(nn12, np.arange(200)[::-1]) and np.array_equal(nn21, np.arange(200)[::-1])


def test_single_points_in_closed_form():
    x = np.array([[0.0, 0.0, 0.0]], F32)
    y = np.array([[0.5, -1.0, 2.0]], F32)
    cd, g, _, _ = FI.chamfer(x, y)
    d = y[0].astype(np.float64) - x[0]
    assert abs(cd - 2 * d @ d) < 1e-12
    assert np.allclose(g[0], 4 * d, atol=1e-12)


def test_small_translation_of_separated_points():
    # points 1 apart, moved by t with |t| << 0.5: every point keeps its
    # partner, CD = 2 |t|^2 and every gradient row is 4 t / n
    g0 = np.array(list(itertools.product(range(4), repeat=3)), np.float64)
    t = np.array([0.01, -0.02, 0.005])
    x = g0.astype(F32)
    y = (g0 + t).astype(F32)
    cd, g, nn12, nn21 = FI.chamfer(x, y)
    tt = (y.astype(np.float64) - x)
    n = len(g0)
    assert np.array_equal(nn12, np.arange(n)) and np.array_equal(nn21, np.arange(n))
    assert abs(cd - 2 * (tt * tt).sum() / n) < 1e-12
    assert np.allclose(g, 4 * tt / n, atol=1e-15)
    assert abs(cd - 2 * t @ t) < 1e-8


def test_distance_against_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (500, 3)).astype(F32)
    y = rng.uniform(-1, 1, (400, 3)).astype(F32)
    cd, _, _, _ = FI.chamfer(x, y)
    d12, _ = spatial.cKDTree(y.astype(np.float64)).query(x.astype(np.float64))
    d21, _ = spatial.cKDTree(x.astype(np.float64)).query(y.astype(np.float64))
    assert abs(cd - ((d12 ** 2).mean() + (d21 ** 2).mean())) < 1e-9


def test_gradient_by_central_differences():
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (60, 3)).astype(F32)
    y = rng.uniform(-1, 1, (50, 3)).astype(F32)
    _, g, _, _ = FI.chamfer(x, y)
    h = 1e-6  # CD is quadratic between assignment changes: no truncation error
    num = np.full(g.shape, np.nan)
    for j in range(len(y)):
        for a in range(3):
            yp = y.astype(np.float64).copy()
            yp[j, a] += h
            ym = y.astype(np.float64).copy()
            ym[j, a] -= h
            (cp, ap), (cm, am) = _cd64(x, yp), _cd64(x, ym)
            if all(np.array_equal(u, v) for u, v in zip(ap, am)):  # no tie crossed
                num[j, a] = (cp - cm) / (2 * h)
    ok = ~np.isnan(num)
    assert ok.mean() > 0.95
    assert np.abs(num[ok] - g[ok]).max() < 1e-8


def _cd64(x, y):
    """CD in fp64 at fp64 positions, and the two nearest-point maps."""
    x = np.asarray(x, np.float64)
    d = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return d.min(1).mean() + d.min(0).mean(), (d.argmin(1), d.argmin(0))


def test_parameter_means_on_a_lattice():
    g0 = np.array(list(itertools.product(range(5), repeat=3)), np.float64)[:, ::-1]
    p1 = g0.astype(F32)
    sh = g0 @ np.array([[1.0], [10.0], [100.0]])  # linear in position
    # a query at (2, 2, 2.3): nearest lattice point (2, 2, 2); k = 1
    (m1,), idx = FI.mean_params(np.array([[2, 2, 2.3]], F32), p1, [sh], 1)
    assert np.allclose(m1, [[2 + 20 + 200]])
    # k = 2 at (2, 2, 2.4): (2, 2, 2) and (2, 2, 3)
    (m2,), _ = FI.mean_params(np.array([[2, 2, 2.4]], F32), p1, [sh], 2)
    assert np.allclose(m2, [[(222 + 322) / 2]])


def test_descent_reduces_the_distance():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (300, 3)).astype(F32)
    y = (x + rng.normal(0, 0.02, x.shape))[rng.permutation(300)].astype(F32)
    sh = rng.normal(size=(300, 4, 3))
    y2, (sh2, op2, rad2), hist = FI.frame_init(x, [sh, np.ones(300), np.ones(300)], y,
                                               iters=40, lr=2e-3, k=1)
    assert len(hist) == 41
    assert hist[-1] < 0.5 * hist[0]
    assert y2.dtype == F32 and sh2.shape == (300, 4, 3)
