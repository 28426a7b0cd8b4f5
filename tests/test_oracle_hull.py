"""Pins for the visual-hull initialisation and consistency check (Sec. 3.1
and the appendix): the random generator against its published outputs,
the projection, the check on points inside and outside a sphere, and the
distributions of the draws."""
import math
import os

import numpy as np
import pytest

from oracle import hull_ref as H
from paper_2205_14330_gb300 import scenes

F32 = np.float32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_published_outputs():
    want = [int(l, 16) for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    got = H.splitmix64(0, np.arange(len(want)))
    assert [int(v) for v in got] == want


def test_projection_of_axis_points_and_points_behind():
    cam = scenes.camera((0.0, 0.0, 4.0), 64, 48)  # looks at the origin
    x, y = H.pixels(np.array([[0, 0, 0], [0, 0, 1], [0, 0, 5], [100, 0, 0]], F32), cam)
    # on the optical axis: the principal point (32, 24) lies on a pixel corner
    assert (x[0], y[0]) == (32, 24) and (x[1], y[1]) == (32, 24)
    # behind the camera, and far outside the field of view
    assert x[2] == -1 and y[2] == -1 and x[3] == -1


def test_check_keeps_the_object_core_and_rejects_far_points():
    d = scenes.hull_scene(seed=1, n_spheres=1, n_cams=8, width=128, height=128)
    c, r = d["centres"][0], d["radii"][0]
    rng = np.random.default_rng(0)
    # points within half the radius of the centre project well inside every
    # silhouette (their pixels' rays pass through the sphere)
    v = rng.normal(size=(500, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inner = (c + 0.5 * r * rng.uniform(0, 1, (500, 1)) * v).astype(F32)
    assert H.consistency(inner, d["cams"], d["masks"]).all()
    # points 2.5 radii from the centre in random directions: no view sees them
    # on the silhouette in all eight views
    far = (c + 2.5 * r * v).astype(F32)
    ok = H.consistency(far, d["cams"], d["masks"])
    assert not ok.any()


def test_uniform_candidates_and_normal_draws():
    stats = pytest.importorskip("scipy.stats")
    lo, hi = np.array([-1.0, 0.0, 2.0], F32), np.array([1.0, 0.5, 6.0], F32)
    c = H.candidates(3, 0, 20000, lo, hi).astype(np.float64)
    for a in range(3):
        u = (c[:, a] - lo[a]) / (hi[a] - lo[a])
        assert stats.kstest(u, "uniform").pvalue > 1e-3
        assert c[:, a].min() >= lo[a] and c[:, a].max() < hi[a]
    z = H.sh_normals(5, 1000, 27).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02


def test_sampler_keeps_the_first_accepted_candidates():
    d = scenes.hull_scene(seed=2, n_spheres=3, n_cams=6, width=96, height=96)
    pos, drawn = H.hull_init(d["lo"], d["hi"], d["cams"], d["masks"], 300, seed=11, batch=1000)
    all_c = H.candidates(11, 0, drawn, d["lo"], d["hi"])
    keep = H.consistency(all_c, d["cams"], d["masks"])
    assert keep[drawn - 1] and keep.sum() == 300
    assert np.array_equal(pos, all_c[keep])
    # a different batch size draws the same points
    pos2, drawn2 = H.hull_init(d["lo"], d["hi"], d["cams"], d["masks"], 300, seed=11, batch=777)
    assert drawn2 == drawn and np.array_equal(pos2, pos)
    # the hull holds the spheres: acceptance about their share of the box
    vol = sum(4 / 3 * math.pi * r ** 3 for r in d["radii"]) / 27.0
    assert 300 / drawn > 0.5 * vol
