"""Batching form: a whole batch of views (several scenes / frames, uneven
resolutions) captured as CUDA graphs, and the schedule autotuner.  Graph
replays must reproduce the eager path: the forward bit for bit, gradients
to the backward's atomic-order tolerance."""
import numpy as np
import pytest

from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    r = pbr.Renderer(0)
    yield pbr, r
    r.close()


def _batch(pbr, seed=0):
    rng = np.random.default_rng(seed)
    sc = []
    for k, (n, deg) in enumerate(((3000, 3), (2000, 1))):
        pos = scenes.surface_points(rng, n, 6)
        sc.append(pbr.Scene(pos, scenes.sh_coeffs(rng, n, deg, 0.2),
                            np.full(n, 0.8, np.float32), scenes.log_uniform(rng, n, 0.01, 0.03),
                            deg))
    cams = [scenes.camera((0.3, 0.4, 3.0), 96, 64), scenes.camera((-2.5, 0.5, 1.5), 53, 77),
            scenes.camera((1.0, 2.6, 1.2), 128, 128), scenes.camera((2.0, -1.0, 2.0), 40, 40)]
    sov = [0, 1, 0, 1]
    return sc, cams, sov


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("sched", [dict(), dict(persistent=1), dict(batch_depth=256),
                                   dict(tile=(8, 8), persistent=1)],
                         ids=["streamed", "persistent", "staged", "persistent-8x8"])
def test_graph_replay_matches_eager(env, sched):
    import torch
    pbr, R = env
    sc, cams, sov = _batch(pbr)
    opts = pbr.default_opts(**sched)
    target = torch.rand((pbr.n_pixels(cams), 3), device="cuda")
    ref, st = R.forward(sc, cams, opts, scene_of_view=sov)
    loss, g = pbr.image_loss(ref, target, "l2")
    gpos, gsh, gop = R.backward(st, g)
    G = pbr.Graph(R, sc, cams, opts, scene_of_view=sov, target=target, loss="l2")
    for _ in range(2):
        G.launch(pbr.Graph.FORWARD)
        ok, n, cap = G.check()
        assert ok and n == st.info()["n_pairs"] and cap >= n
        assert torch.equal(G.out, ref)
        G.launch(pbr.Graph.STEP)
        ok, _, _ = G.check()
        assert ok
        assert torch.equal(G.out, ref)
        assert abs(G.loss.item() - loss.item()) <= 1e-9 * max(1.0, loss.item())
        assert _rel(G.grad_pos, gpos) <= 1e-5
        assert _rel(G.grad_sh, gsh) <= 1e-5
        assert _rel(G.grad_opacity, gop) <= 1e-5
    st.close()
    G.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 32)])
def test_persistent_matches_streamed_on_a_batch(env, tile):
    """The persistent schedule (tile descriptors over several views and
    scenes of uneven sizes) against the one-block-per-tile schedule: the
    same image bit for bit, the same gradients to atomic-order rounding."""
    import torch
    pbr, R = env
    sc, cams, sov = _batch(pbr, seed=7)
    target = torch.rand((pbr.n_pixels(cams), 3), device="cuda")
    out = []
    for per in (0, 1):
        img, st = R.forward(sc, cams, pbr.default_opts(tile=tile, persistent=per),
                            scene_of_view=sov)
        _, g = pbr.image_loss(img, target, "l2")
        out.append((img, R.backward(st, g)))
        st.close()
    assert torch.equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert _rel(b, a) <= 1e-5


def test_graph_follows_in_place_updates_and_replans(env):
    import torch
    pbr, R = env
    sc, cams, sov = _batch(pbr, seed=3)
    opts = pbr.default_opts()
    G = pbr.Graph(R, sc, cams, opts, scene_of_view=sov, backward=False, headroom=0.0)
    G.launch(pbr.Graph.FORWARD)
    assert G.check()[0]
    # move the points (an optimiser step would do this in place)
    with torch.no_grad():
        sc[0].pos.mul_(0.97)
        sc[1].pos.add_(0.01)
    G.launch(pbr.Graph.FORWARD)
    ok, n, cap = G.check()
    ref, _ = R.forward(sc, cams, opts, scene_of_view=sov, keep_state=False)
    if ok:
        assert torch.equal(G.out, ref)
    # grow every splat: more pairs than planned -> reported, then re-planned
    with torch.no_grad():
        for s in sc:
            s.radius.mul_(3.0)
    G.launch(pbr.Graph.FORWARD)
    ok, n, cap = G.check()
    assert not ok and n > cap
    G.replan()
    G.launch(pbr.Graph.FORWARD)
    ok, n, cap = G.check()
    assert ok
    ref, _ = R.forward(sc, cams, opts, scene_of_view=sov, keep_state=False)
    assert torch.equal(G.out, ref)
    # new camera poses of the same sizes
    cams2 = [scenes.camera((0.2, 0.6, 2.8), c["width"], c["height"]) for c in cams]
    G.set_cameras(cams2)
    G.launch(pbr.Graph.FORWARD)
    ok, _, _ = G.check()
    ref2, _ = R.forward(sc, cams2, opts, scene_of_view=sov, keep_state=False)
    if ok:
        assert torch.equal(G.out, ref2)
    G.close()


def test_autotuner_picks_a_timed_candidate(env):
    pbr, R = env
    sc, cams, sov = _batch(pbr, seed=5)
    best, table = pbr.autotune(R, sc, cams, scene_of_view=sov, backward=True, reps=1)
    assert len(table) == pbr.N_TUNE_CANDIDATES
    key = ((best.tile_w, best.tile_h), best.batch_depth, best.persistent)
    assert key in table and table[key] == min(table.values())
    # cached: a second call returns the same choice without timing
    again, t2 = pbr.autotune(R, sc, cams, scene_of_view=sov, backward=True, report=False)
    assert (again.tile_w, again.tile_h, again.batch_depth, again.persistent) == \
        (best.tile_w, best.tile_h, best.batch_depth, best.persistent) and t2 == {}
    # every candidate renders the same image
    ref, _ = R.forward(sc, cams, pbr.default_opts(), scene_of_view=sov, keep_state=False)
    img, _ = R.forward(sc, cams, best, scene_of_view=sov, keep_state=False)
    import torch
    assert torch.equal(img, ref)
