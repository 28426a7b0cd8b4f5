"""Batching form: a whole batch of views (several scenes / frames, uneven
resolutions) captured as CUDA graphs, and the schedule autotuner.  Graph
replays must match the FP64 oracle per frame (images max abs 1e-4,
gradients and one training update rel L2 1e-3) and reproduce the eager
path of the same schedule: the forward bit for bit, gradients to the
backward's atomic-order tolerance.  Different schedules composite the same
points and agree to fp32 rounding (1e-6)."""
import json

import numpy as np
import pytest

from oracle import oracle as O
from oracle import train_ref as TR
from paper_2205_14330_gb300 import scenes

IMG_TOL = 1e-4
GRAD_TOL = 1e-3

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


def _frames(seed=0, n=1500, frames=3):
    """A small batch shaped like the dynamic-video workload: `frames` frames
    of one deforming cloud (each a scene), seen by 4 cameras of uneven size
    (the same cameras in every frame), SH degree 2."""
    d = scenes.dynamic_video(seed, n=n, frames=frames, n_cams=4, width=64, height=48)
    rng = np.random.default_rng(seed + 5)
    rad = scenes.log_uniform(rng, n, 0.02, 0.05)
    sizes = [(96, 64), (64, 64), (80, 48), (48, 72)]
    eyes = [(0.0, 0.4, 3.2), (2.6, 0.8, 1.6), (-2.4, 1.2, 1.8), (0.5, 2.8, 1.5)]
    cams = [scenes.camera(e, w, h) for e, (w, h) in zip(eyes, sizes)]
    return d["frames"], d["sh"], d["opacity"], rad, d["deg"], cams


def _rel_np(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("sched", [dict(), dict(persistent=1), dict(tile=(16, 32), persistent=1)],
                         ids=["streamed", "persistent", "persistent-16x32"])
def test_graph_frames_match_oracle(env, sched):
    """FORWARD, STEP (L2 loss + backward) and TRAIN (Eq. 8 objective and an
    SGD update) replays of a multi-frame batch (frames as scenes,
    scene_of_view) against the FP64 oracle, frame by frame."""
    import torch
    pbr, R = env
    frames, sh, op, rad, deg, cams = _frames()
    nf, nc, n, K = len(frames), len(cams), len(rad), (deg + 1) ** 2
    views = [c for _ in frames for c in cams]
    sov = [f for f in range(nf) for _ in cams]
    sc = [pbr.Scene(p, sh, op, rad, deg) for p in frames]
    rng = np.random.default_rng(9)
    sh_t = (sh + rng.normal(0, 0.1, sh.shape)).astype(np.float32)
    tgt = np.concatenate([O.render(p, sh_t, op, rad, deg, cams)[0] for p in frames])
    G = pbr.Graph(R, sc, views, pbr.default_opts(**sched), scene_of_view=sov,
                  target=torch.from_numpy(tgt.astype(np.float32)).cuda(), loss="l2")
    npx = sum(c["width"] * c["height"] for c in cams)  # pixels of one frame
    refs = [O.render(p, sh, op, rad, deg, cams)[0] for p in frames]
    G.launch(pbr.Graph.FORWARD)
    assert G.check()[0]
    out = G.out.cpu().numpy()
    err = max(float(np.abs(out[f * npx:(f + 1) * npx] - refs[f]).max()) for f in range(nf))
    # the eager forward of the same batch and schedule: tells a wrong replay
    # from a wrong reference when the comparison below fails
    eager, st = R.forward(sc, views, pbr.default_opts(**sched), scene_of_view=sov)
    st.close()
    e_eager = max(float(np.abs(eager.cpu().numpy()[f * npx:(f + 1) * npx] - refs[f]).max())
                  for f in range(nf))
    same = bool(torch.equal(G.out, eager))
    # STEP: dL/dI = 2 (I - target) per frame, adjoint per frame
    G.launch(pbr.Graph.STEP)
    assert G.check()[0]
    gp, gs, go = (G.grad_pos.cpu().numpy(), G.grad_sh.cpu().numpy(),
                  G.grad_opacity.cpu().numpy())
    e_step = []
    for f in range(nf):
        g_img = 2.0 * (refs[f] - tgt[f * npx:(f + 1) * npx])
        dpos, dsh, dop = O.backward(frames[f], sh, op, rad, deg, cams, g_img)
        e_step.append((_rel_np(gp[f * n:(f + 1) * n], dpos),
                       _rel_np(gs[f * n * K * 3:(f + 1) * n * K * 3].reshape(dsh.shape), dsh),
                       _rel_np(go[f * n:(f + 1) * n], dop)))
    # TRAIN: Eq. 8 objective (squared error + 0.01 anisotropic TV per view),
    # one SGD step moves each frame's parameters by -lr times its gradient
    lr_pos, lr_sh = 1e-3, 2e-3
    G.set_optimizer(kind="sgd", lr_pos=lr_pos, lr_sh=lr_sh, lambda_tv=0.01)
    p0 = [s.pos.clone() for s in sc]
    h0 = [s.sh.clone() for s in sc]
    G.launch(pbr.Graph.TRAIN)
    assert G.check()[0]
    _, g_all = TR.batch_loss_and_grad(np.concatenate(refs), tgt,
                                      [(c["width"], c["height"]) for c in views], 0.01, "l2")
    e_train = []
    for f in range(nf):
        dpos, dsh, _ = O.backward(frames[f], sh, op, rad, deg, cams,
                                  g_all[f * npx:(f + 1) * npx])
        e_train.append((_rel_np((sc[f].pos - p0[f]).cpu().numpy(), -lr_pos * dpos),
                        _rel_np((sc[f].sh - h0[f]).cpu().numpy().reshape(dsh.shape),
                                -lr_sh * dsh)))
    print(f"graph frames {sched}: image max abs err {err:.3e} (eager {e_eager:.3e}, replay "
          f"bitwise equal to eager: {same}); step grad rel L2 (worst frame) "
          f"{np.max(e_step, 0)}; train update rel L2 {np.max(e_train, 0)}")
    assert same
    assert err <= IMG_TOL
    assert np.max(e_step) <= GRAD_TOL
    assert np.max(e_train) <= GRAD_TOL
    G.close()


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
    scenes of uneven sizes) against the one-block-per-tile schedule: the same
    composited points at every pixel (identical list positions after the
    last one), the same image to fp32 rounding (the persistent forward blends
    a lane's two pixels with packed instructions), the same gradients to
    atomic-order rounding."""
    import torch
    pbr, R = env
    sc, cams, sov = _batch(pbr, seed=7)
    target = torch.rand((pbr.n_pixels(cams), 3), device="cuda")
    out = []
    for per in (0, 1):
        img, st = R.forward(sc, cams, pbr.default_opts(tile=tile, persistent=per),
                            scene_of_view=sov)
        _, g = pbr.image_loss(img, target, "l2")
        out.append((img, R.backward(st, g), st.read("n_contrib")))
        st.close()
    assert np.array_equal(out[0][2], out[1][2])
    assert float((out[0][0] - out[1][0]).abs().max()) <= 1e-6
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


def test_autotuner_picks_a_timed_candidate(env, tmp_path):
    pbr, R = env
    sc, cams, sov = _batch(pbr, seed=5)
    best, table = pbr.autotune(R, sc, cams, scene_of_view=sov, backward=True, reps=1)
    assert len(table) == pbr.N_TUNE_CANDIDATES
    key = ((best.tile_w, best.tile_h), best.batch_depth, best.persistent)
    assert key in table and table[key] == min(table.values())
    sched = lambda o: (o.tile_w, o.tile_h, o.batch_depth, o.persistent)  # noqa: E731
    # cached: a second call returns the same choice without timing
    info = {}
    again, t2 = pbr.autotune(R, sc, cams, scene_of_view=sov, backward=True, report=False,
                             info=info)
    assert sched(again) == sched(best) and t2 == {} and info["n_timed"] == 0
    # the cache through its file: a fresh context that loads it times nothing
    path = tmp_path / "tuning.json"
    R.save_tuning(path)
    data = json.loads(path.read_text())
    assert data["format"] == "pbr-autotune-1" and len(data["classes"]) >= 1
    R2 = pbr.Renderer(0)
    assert R2.load_tuning(path) == len(data["classes"])
    info = {}
    loaded, _ = pbr.autotune(R2, sc, cams, scene_of_view=sov, backward=True, report=False,
                             info=info)
    assert sched(loaded) == sched(best) and info["n_timed"] == 0
    # a missing file, a file of another kind and an invalid schedule are
    # refused and leave the cache as it was
    with pytest.raises(pbr.PBRError) as ei:
        R2.load_tuning(tmp_path / "absent.json")
    assert ei.value.code == pbr.PBR_ERR_NOT_FOUND
    (tmp_path / "other.json").write_text('{"classes": []}')
    bad = dict(data["classes"][0], tile_w=12, tile_h=12)
    (tmp_path / "bad.json").write_text(json.dumps({"format": "pbr-autotune-1",
                                                   "classes": [data["classes"][0], bad]}))
    for name in ("other.json", "bad.json"):
        with pytest.raises(pbr.PBRError) as ei:
            R2.load_tuning(tmp_path / name)
        assert ei.value.code == pbr.PBR_ERR_INVALID_ARG
    R2.save_tuning(tmp_path / "again.json")
    assert json.loads((tmp_path / "again.json").read_text()) == data
    R2.close()
    # every candidate renders the same image (to fp32 rounding)
    ref, _ = R.forward(sc, cams, pbr.default_opts(), scene_of_view=sov, keep_state=False)
    img, _ = R.forward(sc, cams, best, scene_of_view=sov, keep_state=False)
    assert float((img - ref).abs().max()) <= 1e-6
