"""pbr_render_forward_noalloc: the forward render for callers that cannot
allocate device memory (plug-ins living under a host application's
allocator, real-time loops that must not call the allocator after start-up).
It keeps every intermediate buffer in a fixed 16 MiB device array inside the
library.  Checked here through the C ABI against pbr_render_forward on the
same inputs, on two calls in a row, with the image tolerance of the other
GPU tests; oversized passes must be refused with PBR_ERR_CAPACITY.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

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
    for call in range(2):
        out = torch.full((pbr.n_pixels(cams), 3), float("nan"), device="cuda")
        pbr.render_forward_noalloc([scene], cams, opts, out=out)
        torch.cuda.synchronize()
        err = float(np.abs(out.cpu().numpy() - ref).max())
        print(f"no-alloc forward, call {call}: max abs diff vs pbr_render_forward {err:.3e}")
        assert err <= IMG_TOL

    # a pass larger than the fixed scratch is refused before any GPU work
    big = pbr.Scene(np.zeros((400_000, 3), np.float32), np.zeros((400_000, 1, 3), np.float32),
                    np.zeros(400_000, np.float32), np.full(400_000, 0.01, np.float32), 0)
    with pytest.raises(pbr.PBRError) as exc:
        pbr.render_forward_noalloc([big], cams, opts)
    assert exc.value.code == -4 and "limit" in str(exc.value)
    r.close()
