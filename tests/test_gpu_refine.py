"""Coarse-to-fine update (Sec. 3.3, Algorithm 1) and the exact kNN search on
the GPU against the plain definitions in oracle/refine_ref.py.

Integer results (voxel ids and counts, neighbour indices, outlier
decisions) and every value those decisions are taken from (reduced
positions, squared distances) must match bit for bit; the other means
(SH, opacity, radius; generated points) are FP64 means in the oracle and
compensated fp32 means on the GPU, so they agree to a few 1e-7 relative."""
import numpy as np
import pytest

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


def _scene(pbr, d):
    return pbr.Scene(d["pos"], d["sh"], d["opacity"], d["radius"], d["deg"])


def _cloud(n, shapes=6, frac=0.02, deg=2, seed=0):
    return scenes.refine_cloud(seed=seed, n=n, n_shapes=shapes, outlier_frac=frac, deg=deg)


# ---------------------------------------------------------------- kNN
# grid_n = 700: 700^3 cells exceed the dense cell-table limit (2^28), so the
# fine level looks cells up by binary search
@pytest.mark.parametrize("k,grid_n", [(8, 0), (1, 0), (32, 0), (8, 1), (8, 5), (8, 200),
                                      (8, 700)])
def test_knn_self_exact(env, k, grid_n):
    pbr, r = env
    pos = _cloud(3000)["pos"]
    idx, d2 = pbr.knn(r, _cuda(pos), k, grid_n=grid_n)
    ri, rd = RR.knn(pos, k)
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.array_equal(d2.cpu().numpy(), rd)


def test_knn_queries_inside_and_outside_the_grid(env):
    pbr, r = env
    rng = np.random.default_rng(5)
    ref = _cloud(2500)["pos"]
    q = np.concatenate([rng.uniform(-1.2, 1.2, (300, 3)), rng.uniform(-6, 6, (100, 3)),
                        ref[:50]]).astype(F32)  # last rows coincide with reference points
    for grid_n in (0, 7, 64):
        idx, d2 = pbr.knn(r, _cuda(ref), 6, query=_cuda(q), grid_n=grid_n)
        ri, rd = RR.knn(q, 6, ref=ref)
        assert np.array_equal(idx.cpu().numpy(), ri)
        assert np.array_equal(d2.cpu().numpy(), rd)


def test_knn_isolated_cluster_uses_the_exhaustive_path(env):
    """A small cluster far from the rest: its neighbours lie many cells away,
    beyond the shell limit of the grid search."""
    pbr, r = env
    pos = np.concatenate([_cloud(3000)["pos"],
                          np.array([[8, 8, 8], [8.01, 8, 8], [8, 8.02, 8.01]], F32)])
    for k, grid_n in ((8, 0), (2, 0), (8, 40)):
        idx, d2 = pbr.knn(r, _cuda(pos), k, grid_n=grid_n)
        ri, rd = RR.knn(pos, k)
        assert np.array_equal(idx.cpu().numpy(), ri)
        assert np.array_equal(d2.cpu().numpy(), rd)


def test_knn_ties_duplicates_and_short_sets(env):
    pbr, r = env
    # an integer lattice: many equal distances, ties broken by index
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = g[:, ::-1].astype(F32)
    pos = np.concatenate([pos, pos[:20]])  # exact duplicates
    idx, d2 = pbr.knn(r, _cuda(pos), 18, grid_n=3)
    ri, rd = RR.knn(pos, 18)
    assert np.array_equal(idx.cpu().numpy(), ri) and np.array_equal(d2.cpu().numpy(), rd)
    # fewer points than k: rows padded with -1
    few = pos[:4]
    idx, d2 = pbr.knn(r, _cuda(few), 8)
    idx = idx.cpu().numpy()
    ri, _ = RR.knn(few, 8)
    assert np.array_equal(idx[:, :3], ri) and np.all(idx[:, 3:] == -1)
    # a single point has no neighbours
    idx, _ = pbr.knn(r, _cuda(few[:1]), 4)
    assert np.all(idx.cpu().numpy() == -1)


# ------------------------------------------------------------- refine
def _compare_refine(pbr, r, d, n_vox, k, eps, stages):
    out, counts = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=stages)
    ref = RR.refine(d["pos"], d["sh"], d["opacity"], d["radius"], n_vox, k, eps, stages)
    nred = len(ref["reduced"][0])
    nsurv = len(ref["survivors"][0])
    ntot = len(ref["result"][0])
    assert counts == (nred, nsurv, ntot)
    got = [out.pos.cpu().numpy(), out.sh.cpu().numpy(), out.opacity.cpu().numpy(),
           out.radius.cpu().numpy()]
    # survivors: positions bit-exact, other parameters within a few ulps of
    # the FP64 mean (compensated fp32 sums on the GPU)
    assert np.array_equal(got[0][:nsurv], ref["survivors"][0].astype(F32))
    for g, w in zip(got[1:], ref["survivors"][1:]):
        # a compensated sum errs by a few ulps of the sum of magnitudes
        scale = float(np.abs(w).max()) if len(w) else 0.0
        assert np.allclose(g[:nsurv], w, rtol=4e-7, atol=4e-7 * scale)
    # generated points: compensated fp32 means of fp32 parameters; the oracle
    # averages its FP64 survivor parameters, a few ulps away from the GPU's
    for g, w in zip(got, ref["result"]):
        if len(w) > nsurv:
            scale = float(np.abs(w[:nsurv]).max())
            assert np.allclose(g[nsurv:], w[nsurv:], rtol=5e-7, atol=5e-7 * scale)
    return counts


@pytest.mark.parametrize("stages", [1, 3, 5, 7, 2, 6, 4])
def test_refine_stages_match_oracle(env, stages):
    pbr, r = env
    d = _cloud(4000)
    # eps near the median delta of the reduced set: about half the decisions
    # go each way
    red = RR.voxel_reduce(d["pos"], d["sh"], d["opacity"], d["radius"], 40)[0]
    eps = float(np.median(RR.outlier_delta(red if stages & 1 else d["pos"], 8)[0]))
    counts = _compare_refine(pbr, r, d, 40, 8, eps, stages)
    if stages & 2:
        assert 0 < counts[1] < counts[0]


@pytest.mark.parametrize("n_vox,k", [(1, 4), (2, 3), (7, 1), (64, 16), (300, 32), (700, 8)])
def test_refine_grid_sizes_and_k(env, n_vox, k):
    pbr, r = env
    d = _cloud(2500, deg=1, seed=1)
    _compare_refine(pbr, r, d, n_vox, k, 0.02, 7)


def test_refine_degenerate_inputs(env):
    pbr, r = env
    deg = 0
    same = dict(pos=np.full((9, 3), 0.25, F32), sh=np.ones((9, 1, 3), F32),
                opacity=np.full(9, 0.5, F32), radius=np.full(9, 0.01, F32), deg=deg)
    assert _compare_refine(pbr, r, same, 16, 4, 0.0, 7) == (1, 1, 1)
    one = {kk: (v[:1] if isinstance(v, np.ndarray) else v) for kk, v in same.items()}
    assert _compare_refine(pbr, r, one, 16, 4, 0.0, 7) == (1, 1, 1)
    two = dict(one)
    two["pos"] = np.array([[0, 0, 0], [1, 0, 0]], F32)
    for kk in ("sh", "opacity", "radius"):
        two[kk] = np.concatenate([one[kk], one[kk] * 2])
    assert _compare_refine(pbr, r, two, 16, 4, 0.0, 7) == (2, 2, 4)
    # eps = 0 removes every point whose neighbour distances are not all equal
    d = _cloud(500, seed=2)
    _compare_refine(pbr, r, d, 12, 5, 0.0, 7)


def test_refine_rejects_bad_arguments_and_small_output(env):
    pbr, r = env
    d = _cloud(300)
    sc = _scene(pbr, d)
    for kw in (dict(n_vox=0), dict(n_vox=1025), dict(k=0), dict(k=33), dict(eps=-1.0),
               dict(stages=8)):
        with pytest.raises(pbr.PBRError):
            pbr.refine_points(r, sc, **kw)
    import ctypes as C
    import torch
    cfg = pbr.RefineCfg(16, 4, 1.0, 7)
    counts = (C.c_int64 * 3)()
    buf = [torch.empty(10, device="cuda") for _ in range(4)]
    rc = pbr.lib().pbr_refine_points(r.ctx, C.byref(sc.points()), C.byref(cfg),
                                     *[pbr._ptr(b) for b in buf], 1, counts, pbr._stream())
    assert pbr.ERRORS[rc] == "CAPACITY" and counts[2] > 1


def test_refine_full_size_sampled(env):
    """1M points with 1% outliers, N = 256, K = 8: counts and reduced positions
    exactly; outlier decisions and generated points on sampled points."""
    pbr, r = env
    d = scenes.refine_cloud(seed=0, n=1_000_000)
    n_vox, k = 256, 8
    red_pos = RR.voxel_reduce(d["pos"], d["sh"], d["opacity"], d["radius"], n_vox)[0]
    rng = np.random.default_rng(7)
    samp = rng.choice(len(red_pos), 150, replace=False)
    # delta of the sampled reduced points, by brute force over the reduced
    # set (k + 1 neighbours include the point itself, dropped by index)
    rows = []
    for row, i in zip(RR.knn(red_pos[samp], k + 1, ref=red_pos, chunk=8)[0], samp):
        nb = [j for j in row if j != i][:k]
        rows.append(RR.sq_dist(red_pos[i], red_pos[nb]))
    deltas = RR.delta_of(np.array(rows))
    eps = float(np.median(deltas))
    out, counts = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=7)
    assert counts[0] == len(red_pos)
    got = out.pos.cpu().numpy()
    nsurv = counts[1]
    surv = got[:nsurv]
    # survivors keep reduced order: a reduced point is kept iff it appears
    keyset = {tuple(p) for p in surv.view(np.uint32)}
    kept = np.array([tuple(red_pos[i].view(np.uint32)) in keyset for i in samp])
    assert np.array_equal(kept, ~(deltas > F32(eps)))
    assert counts[2] == 2 * nsurv
    # generated points of sampled survivors: means of their k nearest survivors
    gs = rng.choice(nsurv, 100, replace=False)
    gi, _ = RR.knn(surv[gs], k + 1, ref=surv, chunk=8)
    for row, q in zip(gi, gs):
        nb = [j for j in row if j != q][:k]
        want = surv[nb].astype(np.float64).mean(0)
        assert np.allclose(got[nsurv + q], want, rtol=4e-7, atol=1e-12)
