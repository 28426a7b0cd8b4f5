"""The two ways the backward pass gets each pixel's transmittance before each
composited point (Sec. 3.3, end-to-end gradients): recompute (divide by
1 - alpha back to front from T after the last point) and store (the forward
keeps T before the first store_depth points of every pixel), and the
forward's workspace query.  Both modes must give the FP64 oracle's
gradients (rel L2 1e-3) and agree with each other; store mode's point counts
must equal the oracle's; the workspace query must predict what a forward call
allocates."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    r = pbr.Renderer(0)
    yield pbr, r
    r.close()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _grads(pbr, R, sc, cams, g, **kw):
    scene = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    import torch
    img, st = R.forward([scene], cams, pbr.default_opts(**kw))
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g.astype(np.float32)).cuda())
    out = dict(img=img.cpu().numpy(), pos=gpos.cpu().numpy(), sh=gsh.cpu().numpy(),
               op=gop.cpu().numpy(), n_comp=st.read("n_comp"), T_store=st.read("T_store"))
    st.close()
    return out


@pytest.mark.parametrize("sched", [dict(), dict(persistent=1), dict(persistent=1, tile=(16, 32)),
                                   dict(persistent=1, store_depth=3),
                                   dict(persistent=1, tile=(16, 32), max_per_pixel=5)],
                         ids=["streamed", "persistent", "persistent-16x32", "depth-3",
                              "persistent-n5"])
def test_store_and_recompute_match_the_oracle(env, sched):
    """The tiny workload (4096 points, 128^2): both modes against the oracle's
    adjoint and against each other; store mode's per-pixel point counts equal
    the oracle's, and T before each pixel's first point is 1.  depth-3 keeps
    only the first three points of every pixel, the rest recompute."""
    pbr, R = env
    sc = scenes.tiny()
    cams = sc["cams"]
    rng = np.random.default_rng(2)
    okw = {k: v for k, v in sched.items() if k == "max_per_pixel"}
    ref, _, cnt = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams,
                           **okw)
    g = rng.normal(size=ref.shape)
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                                cams, g, **okw)
    res = {m: _grads(pbr, R, sc, cams, g, bwd_mode=m, **sched) for m in (1, 2)}
    depth = sched.get("store_depth", 32)
    st = res[2]
    assert res[1]["n_comp"].size == 0 and st["n_comp"].size == cnt.size
    assert np.array_equal(st["n_comp"], cnt.astype(np.uint32))
    T = st["T_store"].reshape(-1, depth)
    assert np.all(T[:, 0][cnt > 0] == 1.0)
    errs = {}
    for m in (1, 2):
        r = res[m]
        errs[m] = (_rel(r["pos"], dpos), _rel(r["sh"].reshape(dsh.shape), dsh), _rel(r["op"], dop))
        assert max(errs[m]) <= GRAD_TOL
    diff = max(_rel(res[2][k], res[1][k]) for k in ("pos", "sh", "op"))
    print(f"{sched}: grad rel L2 vs oracle recompute {np.round(errs[1], 9)}, store "
          f"{np.round(errs[2], 9)}; store vs recompute {diff:.2e}; pixels with more than "
          f"{depth} points: {int((cnt > depth).sum())}")
    assert diff <= 1e-4
    assert np.array_equal(res[1]["img"], res[2]["img"])


def test_auto_mode_and_staged_schedule(env):
    """Auto stores when the list takes at most an eighth of the HBM budget;
    a context with a small budget recomputes; the block-staged schedule
    always recomputes."""
    pbr, R = env
    sc = scenes.tiny()
    cams = sc["cams"]
    g = np.random.default_rng(3).normal(size=(128 * 128, 3))
    assert _grads(pbr, R, sc, cams, g)["n_comp"].size == 128 * 128       # auto: store
    small = pbr.Renderer(0, hbm_budget=8 * 128 * 128 * 100)               # list > budget / 8
    assert _grads(pbr, small, sc, cams, g)["n_comp"].size == 0
    small.close()
    assert _grads(pbr, R, sc, cams, g, bwd_mode=2, batch_depth=128)["n_comp"].size == 0


class _PoolWatch:
    """High-water mark of the device's default memory pool (the library's
    stream-ordered allocations), read through the driver API."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CUmemPool_attribute

    def __init__(self, ordinal=0):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH,
                                             ctypes.byref(zero)) == 0
        return self._get(self.USED_MEM_CURRENT)

    def high(self):
        return self._get(self.USED_MEM_HIGH)


@pytest.mark.parametrize("kw,keep", [(dict(), True), (dict(persistent=1, bwd_mode=2), True),
                                     (dict(persistent=1, tile=(8, 8)), False),
                                     (dict(bwd_mode=1, tile=(16, 32)), True)])
def test_workspace_size_predicts_the_allocations(env, kw, keep):
    """pbr_forward_workspace_size against the high-water mark of the memory
    pool the forward allocates from (allocations are rounded up by the pool,
    so the measured peak may exceed the sum by a little)."""
    import torch
    pbr, R = env
    sc = scenes.static_train(n=200_000, n_cams=3, size=320)
    cams = sc["cams"]
    scene = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    opts = pbr.default_opts(**kw)
    nbytes, store = R.workspace_size([scene], cams, opts, keep_state=keep)
    out = torch.empty((pbr.n_pixels(cams), 3), device="cuda")
    watch = _PoolWatch(torch.cuda.current_device())
    torch.cuda.synchronize()
    used0 = watch.reset()
    _, st = R.forward([scene], cams, opts, keep_state=keep, out=out)
    torch.cuda.synchronize()
    peak = watch.high() - used0
    if st is not None:
        st.close()
    print(f"{kw} keep_state={keep}: predicted {nbytes} B (store list {store} B), pool peak "
          f"{peak} B ({peak / nbytes - 1:+.3%})")
    # auto (0) and store (2) keep the list here (it is far below the budget)
    assert (store > 0) == (keep and kw.get("bwd_mode", 0) != 1)
    assert nbytes <= peak <= nbytes * 1.02 + (1 << 20)
