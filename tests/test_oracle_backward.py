"""Pin for the oracle's hand-written adjoint (Sec. 3.3: positions and SH
coefficients are learned end to end by gradient descent through the
splatting renderer of Sec. 3.2).

The analytic gradient of L = sum_u g(u) . I(u) is compared with central
finite differences of the oracle's own forward pass on tiny scenes, with the
cutoff pushed to 8 sigma (its discontinuity is then below 1e-13) and no
transmittance stop, in the all-double screen mode.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes


def _scene(seed, n, deg, cams, o_lo=0.3, o_hi=0.9):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.35, 0.35, (n, 3))
    sh = rng.normal(0, 0.5, (n, (deg + 1) ** 2, 3))
    op = rng.uniform(o_lo, o_hi, n)
    rad = rng.uniform(0.05, 0.1, n)
    g = rng.normal(0, 1, (sum(c["width"] * c["height"] for c in cams), 3))
    return pos, sh, op, rad, g


def _loss(pos, sh, op, rad, deg, cams, g, opts):
    rgb, _, _ = O.render(pos, sh, op, rad, deg, cams, **opts)
    return float((rgb * g).sum())


def _fd(theta, f):
    out = np.zeros_like(theta)
    flat = theta.reshape(-1)
    for j in range(flat.size):
        h = 1e-6 * max(1.0, abs(flat[j]))
        keep = flat[j]
        flat[j] = keep + h
        fp = f()
        flat[j] = keep - h
        fm = f()
        flat[j] = keep
        out.reshape(-1)[j] = (fp - fm) / (2 * h)
    return out


CASES = [
    dict(name="one view, camera-frame SH, world radius", deg=2, n=6,
         cams=[((0.2, 0.1, 2.0), 24, 20)], opts=dict(bg=(0.2, 0.4, 0.1))),
    dict(name="two views, world-frame SH, ndc radius", deg=3, n=5,
         cams=[((0.0, 0.0, 2.0), 20, 20), ((1.5, 0.5, 1.2), 18, 22)],
         opts=dict(dir_frame=1, radius_mode=1)),
    dict(name="count cap", deg=1, n=6, cams=[((0.0, 0.3, 2.2), 20, 16)],
         opts=dict(max_per_pixel=2)),
    dict(name="clamped alpha", deg=0, n=6, cams=[((0.0, 0.0, 2.0), 20, 20)],
         opts=dict(), o=(1.5, 3.0)),
]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_adjoint_matches_central_differences(case):
    deg = case["deg"]
    cams = [scenes.camera(e, w, h) for e, w, h in case["cams"]]
    o_lo, o_hi = case.get("o", (0.3, 0.9))
    pos, sh, op, rad, g = _scene(13, case["n"], deg, cams, o_lo, o_hi)
    opts = dict(cutoff_k=8.0, t_eps=0.0, screen_fp32=0)
    opts.update(case["opts"])
    if opts.get("radius_mode") == 1:
        rad = rad * 0.15  # sigma = r * min(W,H) / 2 in pixels
    dpos, dsh, dop = O.backward(pos, sh, op, rad, deg, cams, g, **opts)

    def f():
        return _loss(pos, sh, op, rad, deg, cams, g, opts)

    for name, analytic, theta in (("pos", dpos, pos), ("sh", dsh, sh), ("opacity", dop, op)):
        num = _fd(theta, f)
        scale = max(1e-12, np.linalg.norm(num))
        rel = np.linalg.norm(analytic - num) / scale
        assert rel < 1e-6, (name, rel)
    assert np.linalg.norm(dpos) > 1e-3  # the case really exercises the geometry


def test_screen_adjoint_zero_for_culled_points():
    cams = [scenes.camera((0.0, 0.0, 2.0), 16, 16)]
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 5.0]])  # second is behind the camera
    sh = np.ones((2, 1, 3))
    out = O.backward(pos, sh, np.full(2, 0.5), np.full(2, 0.1), 0, cams, np.ones((256, 3)),
                     want_g2d=True)
    g2d = out[3]
    assert np.all(g2d[0, 1] == 0) and np.any(g2d[0, 0] != 0)
    assert np.all(out[0][1] == 0)
