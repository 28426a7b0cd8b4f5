"""pbr_render_forward_noalloc: the forward render for callers that cannot
allocate device memory (plug-ins living under a host application's
allocator, real-time loops that must not call the allocator after start-up).
It keeps every intermediate buffer in a fixed 16 MiB device array inside the
library.  Checked here through the C ABI against pbr_render_forward and
against the FP64 oracle on the same inputs, on two calls in a row, with the
image tolerance of the other GPU tests; a call must leave the device's free
memory and the high-water mark of its default stream-ordered memory pool
unchanged (no cudaMalloc, no cudaMallocAsync); oversized passes must be
refused with PBR_ERR_CAPACITY.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def _scene_and_cams():
    rng = np.random.default_rng(21)
    n = 3000
    sc = dict(pos=rng.uniform(-0.8, 0.8, (n, 3)).astype(np.float32),
              sh=scenes.sh_coeffs(rng, n, 3, std=0.3),
              opacity=rng.uniform(0.2, 0.95, n).astype(np.float32),
              radius=rng.uniform(0.01, 0.05, n).astype(np.float32), deg=3)
    cams = [scenes.camera((0.3, 0.2, 2.4), 96, 80), scenes.camera((-1.7, 0.5, 1.4), 61, 47)]
    return sc, cams


class _PoolWatch:
    """High-water mark of the device's default memory pool (the pool
    cudaMallocAsync draws from), read through the driver API: reset before
    a call, read after it."""
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
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0
        return self._get(self.USED_MEM_CURRENT)

    def high(self):
        return self._get(self.USED_MEM_HIGH)


def test_noalloc_forward_matches_allocating_forward():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr

    sc, cams = _scene_and_cams()
    r = pbr.Renderer(0)
    scene = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    opts = pbr.default_opts()
    ref, _ = r.forward([scene], cams, opts, keep_state=False)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    orc, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams)
    watch = _PoolWatch(torch.cuda.current_device())
    for call in range(2):
        out = torch.full((pbr.n_pixels(cams), 3), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        used0 = watch.reset()
        pbr.render_forward_noalloc([scene], cams, opts, out=out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        high = watch.high()
        got = out.cpu().numpy()
        err = float(np.abs(got - ref).max())
        err_o = float(np.abs(got - orc).max())
        print(f"no-alloc forward, call {call}: max abs diff vs pbr_render_forward {err:.3e}, "
              f"vs FP64 oracle {err_o:.3e}; free device memory {free0} -> {free1} B, pool "
              f"high-water mark {high} B (in use before: {used0} B)")
        assert err <= IMG_TOL and err_o <= IMG_TOL
        if call == 1:  # the first call may set up the scratch array's address
            assert free1 == free0
            assert high == used0

    # a pass larger than the fixed scratch is refused before any GPU work
    big = pbr.Scene(np.zeros((400_000, 3), np.float32), np.zeros((400_000, 1, 3), np.float32),
                    np.zeros(400_000, np.float32), np.full(400_000, 0.01, np.float32), 0)
    with pytest.raises(pbr.PBRError) as exc:
        pbr.render_forward_noalloc([big], cams, opts)
    assert exc.value.code == -4 and "limit" in str(exc.value)
    r.close()
