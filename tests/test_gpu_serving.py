"""Serving form: resident scenes, continuous batching of mixed-size views,
admission by HBM budget.  Every request's image must match the FP64 oracle
(max abs 1e-4) and be the same whether it is rendered alone
(pbr_render_forward) or inside a mixed batch; batches admitted while others
run must overlap them on the device."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    yield pbr


def _scenes(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for n, deg in ((4000, 0), (6000, 2), (3000, 3)):
        out.append(dict(pos=scenes.surface_points(rng, n, 5), sh=scenes.sh_coeffs(rng, n, deg, 0.2),
                        opacity=np.full(n, 0.8, np.float32),
                        radius=scenes.log_uniform(rng, n, 0.01, 0.03), deg=deg))
    return out


def _requests(n, seed=1):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        W, H = int(rng.integers(2, 9)) * 16, int(rng.integers(2, 7)) * 16
        reqs.append((int(rng.integers(0, 3)), scenes.camera(d * rng.uniform(2.5, 4.0), W, H)))
    return reqs


def _alone(pbr, R, sc, cam):
    s = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    img, _ = R.forward([s], [cam], keep_state=False)
    return img


def _oracle(sc, cam):
    rgb, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], [cam])
    return rgb


def test_mixed_batch_equals_alone(env):
    pbr = env
    R = pbr.Renderer(0)
    sv = pbr.Server(R, max_batch_views=16, n_streams=2)
    data = _scenes()
    ids = [sv.upload(d) for d in data]
    reqs = _requests(24)
    subs = [sv.submit(ids[s], cam) for s, cam in reqs]
    for rid, _ in subs:
        assert sv.wait(rid) == 0
    st = sv.stats()
    assert st["completed"] == 24 and st["rejected"] == 0
    assert st["max_batch_views"] > 1  # requests really were batched together
    worst = 0.0
    for (s, cam), (_, out) in zip(reqs, subs):
        ref = _alone(pbr, R, data[s], cam)
        err = float((out - ref).abs().max())
        assert err <= IMG_TOL, err
        err_o = float(np.abs(out.cpu().numpy() - _oracle(data[s], cam)).max())
        assert err_o <= IMG_TOL, err_o
        worst = max(worst, err_o)
    print(f"served images (24 requests, batches of up to 16 views): max abs err vs FP64 "
          f"oracle {worst:.3e}")
    sv.stop()
    R.close()


def test_arrivals_while_busy_overlap_and_complete(env):
    """Requests arriving while batches run are admitted into later batches on
    the other stream slot: their device intervals (CUDA events around each
    batch) intersect those of batches still running, every request completes,
    and its image matches the oracle."""
    pbr = env
    R = pbr.Renderer(0)
    sv = pbr.Server(R, max_batch_views=8, n_streams=2)
    data = _scenes(2)
    ids = [sv.upload(d) for d in data]
    rng = np.random.default_rng(3)
    reqs = []
    for _ in range(40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        W, H = int(rng.integers(8, 41)) * 16, int(rng.integers(8, 31)) * 16
        reqs.append((int(rng.integers(0, 3)), scenes.camera(d * rng.uniform(2.5, 4.0), W, H)))
    subs = []
    for k, (s, cam) in enumerate(reqs):
        subs.append(sv.submit(ids[s], cam, arrival=pbr.now()))
        if k % 10 == 9:
            time.sleep(0.002)  # later arrivals join while earlier batches run
    for rid, _ in subs:
        assert sv.wait(rid) == 0
    st = sv.stats(reset=True)
    assert st["completed"] == 40 and st["batches"] >= 5
    assert st["p99_ms"] >= st["p50_ms"] > 0
    tr = sv.trace(reset=True)
    assert len(tr) == st["batches"]
    overlaps = [(i, j) for i in range(len(tr)) for j in range(i + 1, len(tr))
                if tr[j][0] < tr[i][1] and tr[i][0] < tr[j][1]]
    print(f"{len(tr)} batches, {len(overlaps)} pairs overlapping on the device; first "
          f"intervals (ms) {[(round(a, 3), round(b, 3), v) for a, b, v in tr[:4]]}")
    assert overlaps, "no two batches were on the device at the same time"
    for (s, cam), (_, out) in list(zip(reqs, subs))[::7]:
        got = out.cpu().numpy()
        assert float(np.abs(got - _alone(pbr, R, data[s], cam).cpu().numpy()).max()) <= IMG_TOL
        assert float(np.abs(got - _oracle(data[s], cam)).max()) <= IMG_TOL
    sv.stop()
    R.close()


def test_admission_by_hbm_budget(env):
    pbr = env
    R = pbr.Renderer(0)
    data = _scenes(4)
    # a budget that fits one request's reservation but not two: batches of
    # one, all complete
    sv = pbr.Server(R, max_batch_views=16, n_streams=2, hbm_budget=1 << 34)
    ids = [sv.upload(d) for d in data]
    reqs = [(1, scenes.camera((0.0, 0.5, 3.0), 64, 48))] * 6
    sv.set_budget(int(1.5 * sv.estimate(ids[1], reqs[0][1])))
    subs = [sv.submit(ids[s], cam) for s, cam in reqs]
    for rid, _ in subs:
        assert sv.wait(rid) == 0
    st = sv.stats()
    assert st["completed"] == 6 and st["max_batch_views"] == 1
    ref = _alone(pbr, R, data[1], reqs[0][1])
    for _, out in subs:
        assert float((out - ref).abs().max()) <= IMG_TOL
    # a budget below one request: rejected with PBR_ERR_OOM, not run
    sv.set_budget(1000)
    rid, _ = sv.submit(ids[1], reqs[0][1])
    assert sv.wait(rid) == -2
    sv.set_budget(1 << 34)
    # eviction while requests are queued is refused; unknown scenes are refused
    rid, _ = sv.submit(ids[0], reqs[0][1])
    sv.wait(rid)
    sv.evict(ids[0])
    with pytest.raises(pbr.PBRError) as e:
        sv.submit(ids[0], reqs[0][1])
    assert e.value.code == -7
    sv.stop()
    R.close()


def test_admission_estimate_covers_the_workspace(env):
    """The reservation of a request (pbr_serve_estimate) is not below what
    the forward of that view allocates (pbr_forward_workspace_size, forward
    only), on the serving scenes from near cameras at the largest size (the
    most tile pairs per point), at the smallest size, and from far."""
    pbr = env
    R = pbr.Renderer(0)
    data = scenes.serving_scenes()
    opts = pbr.default_opts()
    sv = pbr.Server(R, opts=opts, max_batch_views=4, n_streams=2)
    ratios = []
    for k, d in enumerate(data):
        sid = sv.upload(d)
        scene = pbr.Scene(d["pos"], d["sh"], d["opacity"], d["radius"], d["deg"])
        for dist, (W, H) in ((3.0, (1920, 1072)), (3.0, (256, 256)), (5.0, (1920, 1072)),
                             (0.5, (1280, 720))):  # the last camera is inside the scene
            cam = scenes.camera((0.3 * dist, 0.4 * dist, 0.866 * dist), W, H)
            exact, _ = R.workspace_size([scene], [cam], opts, keep_state=False)
            est = sv.estimate(sid, cam)
            ratios.append(est / exact)
            assert est >= exact, (k, dist, W, H, exact, est)
        # a request from inside the scene is admitted and completes
        rid, out = sv.submit(sid, scenes.camera((0.15, 0.2, 0.43), 320, 240))
        assert sv.wait(rid) == 0
        sv.evict(sid)
    print(f"admission reservation / workspace: {min(ratios):.2f} .. {max(ratios):.2f}")
    sv.stop()
    R.close()
