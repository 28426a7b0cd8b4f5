"""Video frame initialisation (Sec. 3.4) on the GPU against the plain
definitions in oracle/frame_init_ref.py: nearest-point maps exactly, the
Chamfer distance to fp64 rounding, its gradient to fp32 rounding, the Adam
descent and the parameter transfer."""
import numpy as np
import pytest

from oracle import frame_init_ref as FI
from oracle import refine_ref as RR
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu

F32 = np.float32


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    r = pbr.Renderer(0)
    yield pbr, r
    r.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(n, seed=0):
    return scenes.frame_pair(seed=seed, n=n)


def test_chamfer_matches_oracle(env):
    pbr, r = env
    d = _pair(3000)
    p1, p2 = d["p1"], d["p2"][:2500]
    loss, g, nn12, nn21 = pbr.chamfer(r, _cuda(p1), _cuda(p2))
    cd, rg, r12, r21 = FI.chamfer(p1, p2)
    assert np.array_equal(nn12.cpu().numpy(), r12) and np.array_equal(nn21.cpu().numpy(), r21)
    assert abs(float(loss) - cd) <= 1e-12 * cd + 1e-18
    g = g.cpu().numpy()
    assert np.allclose(g, rg, rtol=1e-5, atol=1e-6 * np.abs(rg).max())


def test_chamfer_edge_cases(env):
    pbr, r = env
    one = np.array([[0.1, 0.2, 0.3]], F32)
    two = np.array([[1.0, 0.0, 0.0], [0.1, 0.2, 0.4]], F32)
    for a, b in ((one, two), (two, one), (one, one)):
        loss, g, _, _ = pbr.chamfer(r, _cuda(a), _cuda(b))
        cd, rg, _, _ = FI.chamfer(a, b)
        assert abs(float(loss) - cd) <= 1e-12 * max(cd, 1e-30)
        assert np.allclose(g.cpu().numpy(), rg, rtol=1e-6, atol=1e-12)
    # far-apart clouds: every query takes the coarse or exhaustive path
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, 1, (500, 3)).astype(F32)
    b = (rng.uniform(-1, 1, (400, 3)) + np.array([30.0, 0, 0])).astype(F32)
    loss, g, nn12, nn21 = pbr.chamfer(r, _cuda(a), _cuda(b))
    cd, rg, r12, r21 = FI.chamfer(a, b)
    assert np.array_equal(nn12.cpu().numpy(), r12) and np.array_equal(nn21.cpu().numpy(), r21)
    assert abs(float(loss) - cd) <= 1e-12 * cd


def test_parameter_transfer_without_descent(env):
    pbr, r = env
    d = _pair(2000)
    prev = pbr.Scene(d["p1"], d["sh"], d["opacity"], d["radius"], d["deg"])
    for k in (1, 4, 32):
        pos2 = _cuda(d["p2"][:1500].copy())
        new, hist = pbr.frame_init(r, prev, pos2, iters=0, k=k)
        assert np.array_equal(new.pos.cpu().numpy(), d["p2"][:1500])
        assert abs(hist[0] - FI.chamfer(d["p1"], d["p2"][:1500])[0]) <= 1e-12 * hist[0]
        want, _ = FI.mean_params(d["p2"][:1500], d["p1"], [d["sh"], d["opacity"], d["radius"]], k)
        for got, w in zip((new.sh, new.opacity, new.radius), want):
            assert np.allclose(got.cpu().numpy(), w, rtol=4e-7, atol=4e-7 * np.abs(w).max())


def test_descent_matches_oracle(env):
    pbr, r = env
    d = _pair(800, seed=1)
    prev = pbr.Scene(d["p1"], d["sh"], d["opacity"], d["radius"], d["deg"])
    pos2 = _cuda(d["p2"].copy())
    new, hist = pbr.frame_init(r, prev, pos2, iters=8, lr=1e-3, k=4)
    y, params, rhist = FI.frame_init(d["p1"], [d["sh"], d["opacity"], d["radius"]], d["p2"],
                                     iters=8, lr=1e-3, k=4)
    # fp32 Adam against the FP64 update rounded to fp32 every step
    assert np.allclose(new.pos.cpu().numpy(), y, rtol=0, atol=2e-6)
    assert np.allclose(hist, rhist, rtol=1e-4)
    assert hist[-1] < hist[0]
    # parameters: rows whose k closest points agree match to rounding; a
    # position difference of a few ulps may reorder a near tie elsewhere
    got = new.sh.cpu().numpy().reshape(len(y), -1)
    w = params[0].reshape(len(y), -1)
    close = np.all(np.abs(got - w) <= 4e-7 * np.abs(w).max() + 1e-12, axis=1)
    assert close.mean() >= 0.99


def test_degenerate_and_bad_arguments(env):
    pbr, r = env
    import torch
    one = pbr.Scene(np.zeros((1, 3), F32), np.ones((1, 1, 3), F32), np.ones(1, F32),
                    np.ones(1, F32), 0)
    pos2 = _cuda(np.array([[1, 0, 0], [0, 2, 0]], F32))
    new, hist = pbr.frame_init(r, one, pos2, iters=3, k=4)  # k > n1: all of S1
    assert np.allclose(new.sh.cpu().numpy(), 1.0) and len(hist) == 4
    for kw in (dict(k=0), dict(k=33), dict(iters=-1), dict(lr=-1.0), dict(beta1=1.0)):
        with pytest.raises(pbr.PBRError):
            pbr.frame_init(r, one, pos2, **kw)
    with pytest.raises(pbr.PBRError):
        pbr.chamfer(r, torch.zeros((0, 3), device="cuda"), pos2)


def test_full_size_sampled(env):
    """200k points (the dynamic-video workload's frames 0 and 1): nearest-
    point maps on sampled points by brute force, CD from the maps, descent."""
    pbr, r = env
    d = _pair(200_000)
    p1, p2 = d["p1"], d["p2"]
    loss, g, nn12, nn21 = pbr.chamfer(r, _cuda(p1), _cuda(p2))
    nn12, nn21 = nn12.cpu().numpy(), nn21.cpu().numpy()
    rng = np.random.default_rng(9)
    s1 = rng.choice(len(p1), 150, replace=False)
    s2 = rng.choice(len(p2), 150, replace=False)
    assert np.array_equal(nn12[s1], RR.knn(p1[s1], 1, ref=p2, chunk=8)[0][:, 0])
    assert np.array_equal(nn21[s2], RR.knn(p2[s2], 1, ref=p1, chunk=8)[0][:, 0])
    x64, y64 = p1.astype(np.float64), p2.astype(np.float64)
    cd = ((y64[nn12] - x64) ** 2).sum() / len(p1) + ((y64 - x64[nn21]) ** 2).sum() / len(p2)
    assert abs(float(loss) - cd) <= 1e-9 * cd
    prev = pbr.Scene(p1, d["sh"], d["opacity"], d["radius"], d["deg"])
    new, hist = pbr.frame_init(r, prev, _cuda(p2.copy()), iters=30, lr=1e-3, k=4)
    assert abs(hist[0] - float(loss)) <= 1e-9 * hist[0]
    assert hist[-1] < 0.5 * hist[0]
