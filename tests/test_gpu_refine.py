"""Coarse-to-fine update (Sec. 3.3, Algorithm 1) and the exact kNN search on
the GPU against the plain definitions in oracle/refine_ref.py.

Neighbour indices and squared distances of the search, voxel ids and the
reduced-point count are integer (or exactly defined fp32) results and must
match bit for bit.  The voxel means are plain FP64 means in the oracle and
compensated fp32 sums on the GPU, so the reduced positions agree to
POS_ULPS ulps, and every decision taken later from them (outlier removal,
the neighbours of the generated points) agrees exactly except where the
oracle's own value lies within a stated margin of the decision's threshold:
such points are counted and printed, not asserted.
"""
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
# The oracle rounds the FP64 voxel mean once; the GPU's compensated fp32 sum
# errs by about 2u times the sum of the magnitudes of its terms, so the
# reduced positions agree to POS_ULPS ulps of max(|mean|, mean |p| over the
# voxel).
POS_ULPS = 4
# A reduced position moves by at most POS_ULPS ulps (2.4e-7 at |p| < 2), so
# a neighbour distance by twice that and the standard deviation of Alg. 1 by
# about as much: outlier decisions are exact for every point whose oracle
# delta is further than DELTA_MARGIN from eps, and a neighbour list is the
# oracle's unless its K-th and (K+1)-th distances are within TIE_MARGIN.
DELTA_MARGIN = 1e-5
TIE_MARGIN = 1e-5


def _ulps_apart(a, b, scale=0.0):
    """|a - b| in ulps of max(|a|, |b|, scale) (fp32)."""
    a = np.asarray(a, F32)
    b = np.asarray(b, F32)
    ref = np.maximum(np.maximum(np.abs(a), np.abs(b)), np.asarray(scale, F32))
    return np.abs(a.astype(np.float64) - b.astype(np.float64)) / np.spacing(ref)


def _voxel_mean_abs(pos, n_vox):
    """Mean |p| per component over each voxel (the oracle's voxels, in
    ascending voxel id): the scale of the voxel mean's rounding error."""
    ids = RR.voxel_ids(pos, n_vox)
    order = np.argsort(ids, kind="stable")
    sid = ids[order]
    starts = np.flatnonzero(np.r_[True, sid[1:] != sid[:-1]])
    counts = np.diff(np.r_[starts, len(sid)])
    return np.add.reduceat(np.abs(np.asarray(pos, np.float64))[order], starts, axis=0) / \
        counts[:, None]


def _kept_flags(red, surv):
    """Which rows of `red` the ordered subsequence `surv` keeps."""
    keep = np.zeros(len(red), bool)
    j = 0
    for i in range(len(red)):
        if j < len(surv) and np.array_equal(red[i], surv[j]):
            keep[i] = True
            j += 1
    assert j == len(surv), "survivors are not a subsequence of the reduced set"
    return keep


def _compare_refine(pbr, r, d, n_vox, k, eps, stages):
    """Runs the update on the GPU and in the oracle; returns the GPU counts.
    Prints the decisions inside the margins."""
    out, counts = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=stages)
    ref = RR.refine(d["pos"], d["sh"], d["opacity"], d["radius"], n_vox, k, eps, stages)
    nred = len(ref["reduced"][0])
    assert counts[0] == nred
    got = [out.pos.cpu().numpy(), out.sh.cpu().numpy(), out.opacity.cpu().numpy(),
           out.radius.cpu().numpy()]
    # the GPU's reduced set (stage 1 alone; the kernels are deterministic)
    if stages & 1:
        red_out, _ = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=1)
        red = [red_out.pos.cpu().numpy(), red_out.sh.cpu().numpy(),
               red_out.opacity.cpu().numpy(), red_out.radius.cpu().numpy()]
        pscale = _voxel_mean_abs(d["pos"], n_vox)
        assert _ulps_apart(red[0], ref["reduced"][0], pscale).max(initial=0) <= POS_ULPS
        for g, w in zip(red[1:], ref["reduced"][1:]):
            scale = float(np.abs(w).max()) if len(w) else 0.0
            assert np.allclose(g, w, rtol=4e-7, atol=4e-7 * scale)
    else:
        red = [np.asarray(d["pos"], F32), d["sh"], d["opacity"], d["radius"]]
        pscale = np.zeros((len(red[0]), 3))
    nsurv = counts[1]
    keep_gpu = _kept_flags(red[0], got[0][:nsurv])
    keep_ref = ref["keep"]
    band = np.zeros(nred, bool)
    if stages & 2 and stages & 1 and nred > 1:
        delta, _ = RR.outlier_delta(ref["reduced"][0], k)
        band = np.abs(delta.astype(np.float64) - eps) <= DELTA_MARGIN
    flips = keep_gpu != keep_ref
    assert not np.any(flips & ~band), "outlier decision differs outside the margin"
    if band.any() or flips.any():
        print(f"refine: {int(band.sum())} oracle deltas within {DELTA_MARGIN} of eps, "
              f"{int(flips.sum())} decided differently")
    both = keep_gpu & keep_ref
    # survivors present on both sides: parameters of their reduced points
    gi = np.cumsum(keep_gpu) - 1
    ri = np.cumsum(keep_ref) - 1
    sv = ref["survivors"]
    assert _ulps_apart(got[0][gi[both]], sv[0][ri[both]], pscale[both]).max(initial=0) <= POS_ULPS
    for g, w in zip(got[1:], sv[1:]):
        scale = float(np.abs(w).max()) if len(w) else 0.0
        assert np.allclose(g[gi[both]], w[ri[both]], rtol=4e-7, atol=4e-7 * scale)
    # generated points (when both sides kept the same survivors): means of
    # the k nearest survivors; a near-tie at the k-th neighbour may pick
    # another neighbour, which is counted
    if stages & 4 and not flips.any() and len(ref["result"][0]) > len(sv[0]):
        assert counts[2] == len(ref["result"][0])
        _, d2 = RR.knn(sv[0], k + 1)
        dd = np.sqrt(d2.astype(np.float64))
        tie = np.zeros(len(dd), bool)
        if dd.shape[1] > k:  # a (k+1)-th neighbour exists
            tie = dd[:, k] - dd[:, k - 1] <= TIE_MARGIN
        bad = np.zeros(nsurv, bool)
        for g, w in zip(got, ref["result"]):
            scale = float(np.abs(w[:nsurv]).max())
            ok = np.isclose(g[nsurv:], w[nsurv:], rtol=1e-6, atol=1e-6 * scale)
            bad |= ~ok.reshape(nsurv, -1).all(1)
        assert not np.any(bad & ~tie), "generated point differs without a neighbour tie"
        if bad.any():
            print(f"refine: {int(bad.sum())} generated points with a k-th neighbour tie")
    elif stages & 4 and not flips.any():
        assert counts[2] == len(ref["result"][0])
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
    """1M points with 1% outliers, N = 256, K = 8: reduced count and every
    reduced position against the oracle; outlier decisions and generated
    points on sampled points, from the oracle's own reduced set."""
    pbr, r = env
    d = scenes.refine_cloud(seed=0, n=1_000_000)
    n_vox, k = 256, 8
    red_pos = RR.voxel_reduce(d["pos"], d["sh"], d["opacity"], d["radius"], n_vox)[0]
    nred = len(red_pos)
    rng = np.random.default_rng(7)

    def delta_at(i):
        nb, d2 = RR.knn(red_pos[i:i + 1], k + 1, ref=red_pos)
        keep = nb[0] != i
        return RR.delta_of(d2[:, keep][:, :k])[0]

    samp = rng.choice(nred, 150, replace=False)
    deltas = np.array([delta_at(i) for i in samp])
    eps = float(np.median(deltas))
    # GPU: the reduced set alone, then the whole update
    red_out, c1 = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=1)
    out, counts = pbr.refine_points(r, _scene(pbr, d), n_vox=n_vox, k=k, eps=eps, stages=7)
    assert c1[0] == counts[0] == nred
    red_gpu = red_out.pos.cpu().numpy()
    assert _ulps_apart(red_gpu, red_pos, _voxel_mean_abs(d["pos"], n_vox)).max() <= POS_ULPS
    got = out.pos.cpu().numpy()
    nsurv = counts[1]
    assert counts[2] == 2 * nsurv
    keep_gpu = _kept_flags(red_gpu, got[:nsurv])
    band = np.abs(deltas.astype(np.float64) - eps) <= DELTA_MARGIN
    want = ~(deltas > F32(eps))
    assert np.array_equal(keep_gpu[samp][~band], want[~band])
    print(f"refine 1M: {int(band.sum())} of {len(samp)} sampled deltas within the margin")
    # generated points of sampled oracle survivors: the k nearest survivors
    # among their 4k nearest reduced points (enough when at least k of those
    # survive and the k-th survivor is nearer than the 4k-th candidate)
    gpos = np.cumsum(keep_gpu) - 1
    checked = ties = 0
    for i in rng.choice(nred, 400, replace=False):
        if checked == 60:
            break
        nb, d2 = RR.knn(red_pos[i:i + 1], 4 * k + 1, ref=red_pos)
        nb, d2 = nb[0][nb[0] != i], d2[0][nb[0] != i]
        cand_delta = np.array([delta_at(j) for j in nb])
        if abs(delta_at(i) - eps) <= DELTA_MARGIN or np.any(
                np.abs(cand_delta.astype(np.float64) - eps) <= DELTA_MARGIN):
            continue  # a decision inside the margin: not comparable
        if delta_at(i) > F32(eps):
            continue  # removed: generates nothing
        surv = ~(cand_delta > F32(eps))
        if surv.sum() <= k or d2[surv][k - 1] >= d2[-1]:
            continue  # the candidate set may not hold all k nearest survivors
        dd = np.sqrt(d2[surv].astype(np.float64))
        if dd[k] - dd[k - 1] <= TIE_MARGIN:
            ties += 1
            continue
        want_p = red_pos[nb[surv][:k]].astype(np.float64).mean(0)
        assert keep_gpu[i]
        # the survivors' positions are within 4 ulps (|p| < 2: 1e-6) of the
        # oracle's, and their compensated mean adds a few ulps
        assert np.allclose(got[nsurv + gpos[i]], want_p, rtol=1e-6, atol=2e-6)
        checked += 1
    assert checked >= 40, checked
    print(f"refine 1M: {checked} generated points checked, {ties} skipped at a neighbour tie")
