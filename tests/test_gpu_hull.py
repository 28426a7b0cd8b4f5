"""Visual-hull initialisation and consistency check (Sec. 3.1 and appendix)
on the GPU against oracle/hull_ref.py: the check's decisions, the filter's
compaction, the sampler's kept points and draw count exactly; the SH
normals to fp32 rounding."""
import numpy as np
import pytest

from oracle import hull_ref as H
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


@pytest.fixture(scope="module")
def hull():
    return scenes.hull_scene(seed=0, n_spheres=6, n_cams=10, width=160, height=120)


def test_check_matches_oracle(env, hull):
    pbr, r = env
    rng = np.random.default_rng(0)
    pts = np.concatenate([
        rng.uniform(-1.5, 1.5, (20000, 3)),
        # points near the spheres' surfaces, where decisions flip
        hull["centres"][rng.integers(0, 6, 20000)] + rng.normal(size=(20000, 3)) * 0.3,
        np.array([[0, 0, 4.0], [0, 0, 100.0], [0, 5, 0]]),  # at a camera, far, off-image
    ]).astype(F32)
    masks = pbr.pack_masks(hull["masks"])
    for z_near in (0.01, 3.0):
        keep = pbr.consistency_check(r, _cuda(pts), hull["cams"], masks, z_near).cpu().numpy()
        want = H.consistency(pts, hull["cams"], hull["masks"], z_near)
        assert np.array_equal(keep.astype(bool), want)
        assert 0 < want.sum() < len(pts) or z_near > 1


def test_filter_compacts_in_order(env, hull):
    pbr, r = env
    rng = np.random.default_rng(1)
    n = 5000
    pos = rng.uniform(-1, 1, (n, 3)).astype(F32)
    sh = rng.normal(size=(n, 4, 3)).astype(F32)
    op = rng.uniform(size=n).astype(F32)
    rad = rng.uniform(size=n).astype(F32)
    sc = pbr.Scene(pos, sh, op, rad, 1)
    out = pbr.consistency_filter(r, sc, hull["cams"], pbr.pack_masks(hull["masks"]))
    keep = H.consistency(pos, hull["cams"], hull["masks"])
    assert out.n == keep.sum()
    for got, w in zip((out.pos, out.sh, out.opacity, out.radius), (pos, sh, op, rad)):
        assert np.array_equal(got.cpu().numpy(), w[keep])


@pytest.mark.parametrize("n_target,seed", [(3000, 7), (1, 0), (0, 3)])
def test_sampler_matches_oracle(env, hull, n_target, seed):
    pbr, r = env
    masks = pbr.pack_masks(hull["masks"])
    pos, sh, drawn = pbr.visual_hull_init(r, hull["lo"], hull["hi"], hull["cams"], masks,
                                          n_target, seed=seed, sh_degree=2)
    want, wdrawn = H.hull_init(hull["lo"], hull["hi"], hull["cams"], hull["masks"], n_target,
                               seed)
    assert drawn == wdrawn
    assert np.array_equal(pos.cpu().numpy(), want)
    z = H.sh_normals(seed, n_target, 27).reshape(n_target, 9, 3)
    # fp32 logarithm and sine/cosine on the GPU against fp64: a few ulps
    assert np.allclose(sh.cpu().numpy(), z, rtol=1e-5, atol=1e-6)


def test_sampler_limits_and_empty_masks(env, hull):
    pbr, r = env
    masks = pbr.pack_masks(hull["masks"])
    # the candidate limit stops the draw early
    pos, _, drawn = pbr.visual_hull_init(r, hull["lo"], hull["hi"], hull["cams"], masks, 10**6,
                                         seed=5, max_candidates=20000)
    want, wdrawn = H.hull_init(hull["lo"], hull["hi"], hull["cams"], hull["masks"], 10**6, 5,
                               max_candidates=20000)
    assert drawn == wdrawn == 20000 and np.array_equal(pos.cpu().numpy(), want)
    # no foreground: nothing is kept
    empty = pbr.pack_masks([np.zeros_like(m) for m in hull["masks"]])
    pos, _, drawn = pbr.visual_hull_init(r, hull["lo"], hull["hi"], hull["cams"], empty, 10,
                                         max_candidates=50000)
    assert pos.shape[0] == 0 and drawn == 50000
    with pytest.raises(pbr.PBRError):
        pbr.visual_hull_init(r, hull["hi"], hull["lo"], hull["cams"], masks, 10)


def test_full_size_sampled(env):
    """16 views of 1024 x 768, 200k kept points: every kept point passes the
    oracle's check, the first kept points and the draw count agree with the
    oracle's candidate stream."""
    pbr, r = env
    h = scenes.hull_scene(seed=0, n_spheres=8, n_cams=16, width=1024, height=768)
    masks = pbr.pack_masks(h["masks"])
    pos, sh, drawn = pbr.visual_hull_init(r, h["lo"], h["hi"], h["cams"], masks, 200_000, seed=1)
    pos = pos.cpu().numpy()
    assert pos.shape == (200_000, 3)
    assert H.consistency(pos, h["cams"], h["masks"]).all()
    head = H.candidates(1, 0, 60_000, h["lo"], h["hi"])
    acc = head[H.consistency(head, h["cams"], h["masks"])]
    assert np.array_equal(pos[:len(acc)], acc)
    last = H.candidates(1, drawn - 1, 1, h["lo"], h["hi"])
    assert np.array_equal(pos[-1], last[0])
