"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: tile lists, ranges, tile counts and the fp32 screen positions and
cutoff radii are compared bit for bit; images to max abs 1e-4 on colours of
order 1; gradients to relative L2 1e-3.  Every case also prints its error
against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def R():
    import __graft_entry__ as g
    g.build()
    from paper_2205_14330_gb300 import pbr
    r = pbr.Renderer(0)
    yield r
    r.close()


def _pbr():
    from paper_2205_14330_gb300 import pbr
    return pbr


def _oracle_kw(kw):
    kw = dict(kw)
    if "tile" in kw:
        kw["tile_w"], kw["tile_h"] = kw.pop("tile")
    kw.pop("batch_depth", None)
    kw.pop("persistent", None)
    return kw


def _gpu_render(R, sc, cams, **kw):
    pbr = _pbr()
    scene = pbr.Scene(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"])
    img, st = R.forward([scene], cams, pbr.default_opts(**kw))
    return img, st, scene


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _block_bits(tile):
    n = (tile[0] // 8) * (tile[1] // 8)
    return n if n > 1 else 0


def _check_lists(st, keys, vals, masks, ranges, tile):
    """The GPU's sorted pair keys (tile << B | 8 x 8 block mask), point-view
    ids and ranges against the oracle's lists, bit for bit."""
    sb = _block_bits(tile)
    gk = st.read("tile_keys")
    assert np.array_equal(gk >> np.uint32(sb), keys)
    if sb:
        assert np.array_equal(gk & np.uint32((1 << sb) - 1), masks.astype(np.uint32))
    assert np.array_equal(st.read("tile_vals"), vals)
    assert np.array_equal(st.read("ranges"), ranges)


def _small_scene(seed, n=300, deg=2, spread=0.8, r=(0.02, 0.06)):
    rng = np.random.default_rng(seed)
    return dict(pos=rng.uniform(-spread, spread, (n, 3)).astype(np.float32),
                sh=scenes.sh_coeffs(rng, n, deg, std=0.3),
                opacity=rng.uniform(0.2, 0.95, n).astype(np.float32),
                radius=rng.uniform(r[0], r[1], n).astype(np.float32), deg=deg)


# ------------------------------------------------------------------ forward
def test_tiny_config_image(R):
    sc = scenes.tiny()
    img, st, _ = _gpu_render(R, sc, sc["cams"])
    ref, T, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], sc["cams"])
    got = img.cpu().numpy()
    err = np.abs(got - ref).max()
    print(f"tiny: image max abs err vs FP64 oracle {err:.3e}")
    assert err <= IMG_TOL
    assert np.abs(st.read("T_final") - T).max() <= IMG_TOL
    full, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], sc["cams"],
                          screen_fp32=0)
    print(f"tiny: image max abs err vs all-double oracle {np.abs(got - full).max():.3e}")
    st.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 32)])
def test_bins_and_records_bit_exact(R, tile):
    sc = _small_scene(1, n=400)
    cams = [scenes.camera((0.3, 0.2, 2.2), 70, 45), scenes.camera((-1.8, 0.4, 1.5), 33, 57),
            scenes.camera((0.0, 2.0, 0.3), 16, 16)]
    img, st, _ = _gpu_render(R, sc, cams, tile=tile)
    keys, vals, masks, ranges, recs = O.bin_tiles(sc["pos"], sc["sh"], sc["radius"], sc["deg"],
                                                  cams, tile_w=tile[0], tile_h=tile[1])
    _check_lists(st, keys, vals, masks, ranges, tile)
    flat = recs.reshape(-1)
    vis = flat["visible"] == 1
    nt = st.read("ntiles")
    assert np.array_equal(nt > 0, vis)
    assert np.array_equal(nt[vis], flat["ntiles"][vis].astype(np.uint32))
    rec = st.read("records")
    assert np.array_equal(rec[vis, 0].view(np.uint32), flat["px32"][vis].view(np.uint32))
    assert np.array_equal(rec[vis, 1].view(np.uint32), flat["py32"][vis].view(np.uint32))
    assert np.array_equal(rec[vis, 2].view(np.uint32), flat["rc2_32"][vis].view(np.uint32))
    col_err = np.abs(rec[vis, 5:8] - flat["rgb"][vis]).max()
    assert col_err <= 1e-5, col_err
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams)
    err = np.abs(img.cpu().numpy() - ref).max()
    print(f"tile {tile}: {len(keys)} pairs bit-exact; image max abs err {err:.3e}")
    assert err <= IMG_TOL
    st.close()


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (16, 32)])
@pytest.mark.parametrize("schedule", [dict(), dict(persistent=1), dict(batch_depth=128)],
                         ids=["streamed", "persistent", "staged"])
def test_wide_splats_lists_and_image(R, tile, schedule):
    """Splats whose pixel box spans more than 32 tiles (listed by the
    per-row walk and emitted by whole warps), some cut by the image border,
    among small ones: lists and masks bit-exact, image and gradients against
    the oracle in every compositing schedule."""
    sc = _small_scene(4, n=250)
    sc["radius"][:6] = [0.5, 0.35, 0.7, 0.3, 0.45, 0.25]
    sc["pos"][2] = [0.9, -0.7, 0.2]
    sc["opacity"][:6] = 0.3
    cams = [scenes.camera((0.3, 0.2, 2.2), 200, 150), scenes.camera((-1.5, 0.4, 1.5), 151, 117)]
    img, st, scene = _gpu_render(R, sc, cams, tile=tile, **schedule)
    keys, vals, masks, ranges, recs = O.bin_tiles(sc["pos"], sc["sh"], sc["radius"], sc["deg"],
                                                  cams, tile_w=tile[0], tile_h=tile[1])
    wide = [(r["tx_hi"] - r["tx_lo"] + 1) * (r["ty_hi"] - r["ty_lo"] + 1)
            for r in recs.reshape(-1) if r["visible"]]
    assert max(wide) > 32
    _check_lists(st, keys, vals, masks, ranges, tile)
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams)
    err = np.abs(img.cpu().numpy() - ref).max()
    rng = np.random.default_rng(3)
    g = rng.normal(size=ref.shape)
    import torch
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g.astype(np.float32)).cuda())
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams, g)
    e = (_rel(gpos.cpu().numpy(), dpos), _rel(gsh.cpu().numpy().reshape(dsh.shape), dsh),
         _rel(gop.cpu().numpy(), dop))
    print(f"wide splats {tile} {schedule}: {len(keys)} pairs, max box {max(wide)} tiles; image "
          f"err {err:.3e}; grad rel L2 {e[0]:.2e} {e[1]:.2e} {e[2]:.2e}")
    assert err <= IMG_TOL
    assert max(e) <= GRAD_TOL
    st.close()


@pytest.mark.parametrize("hidden", [0.0, 0.6], ids=["all-visible", "mostly-hidden"])
def test_bins_exact_in_both_depth_orderings(R, hidden):
    """The depth order is built either by sorting all point-views (the
    invisible ones keyed behind every depth) or by compacting the visible
    ones first, chosen by the visible fraction (3/4).  Both must give the
    oracle's lists, including the order of equal depths (duplicated points);
    a captured graph must render the same image."""
    pbr = _pbr()
    rng = np.random.default_rng(11)
    n = 600
    pos = rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    pos[n // 2:n // 2 + 60] = pos[:60]  # equal depths in every view
    k = int(hidden * n)
    pos[n - k:] += np.float32(40.0)     # far outside every view
    sc = dict(pos=pos, sh=scenes.sh_coeffs(rng, n, 1, std=0.3),
              opacity=rng.uniform(0.2, 0.9, n).astype(np.float32),
              radius=rng.uniform(0.01, 0.04, n).astype(np.float32), deg=1)
    cams = [scenes.camera((0.2, 0.1, 2.4), 80, 60, fov_deg=60.0),
            scenes.camera((-2.0, 0.5, 1.2), 64, 64, fov_deg=60.0)]
    img, st, scene = _gpu_render(R, sc, cams)
    keys, vals, masks, ranges, recs = O.bin_tiles(sc["pos"], sc["sh"], sc["radius"], sc["deg"],
                                                  cams)
    vis_frac = float((recs.reshape(-1)["visible"] == 1).mean())
    assert (vis_frac >= 0.75) == (hidden == 0.0), vis_frac
    _check_lists(st, keys, vals, masks, ranges, (16, 16))
    G = pbr.Graph(R, [scene], cams, pbr.default_opts(), backward=False)
    G.launch(pbr.Graph.FORWARD)
    assert G.check()[0]
    import torch
    assert torch.equal(G.out, img)
    G.close()
    st.close()


def test_image_independent_of_tile_size_and_batch_depth(R):
    sc = _small_scene(2, n=500)
    cams = [scenes.camera((0.5, -0.3, 2.4), 97, 61)]
    imgs = []
    for tile, depth, per in (((16, 16), 0, 0), ((8, 8), 0, 0), ((16, 32), 0, 0), ((16, 16), 0, 1),
                             ((8, 8), 0, 1), ((16, 32), 0, 1), ((16, 16), 256, 0),
                             ((8, 8), 32, 0), ((16, 32), 512, 0), ((16, 16), 64, 0)):
        img, st, _ = _gpu_render(R, sc, cams, tile=tile, batch_depth=depth, persistent=per)
        imgs.append(img.cpu().numpy())
        st.close()
    # the same composited points everywhere; the persistent forward blends a
    # lane's two pixels with packed instructions, which agree to fp32 rounding
    for im in imgs[1:]:
        assert np.abs(im - imgs[0]).max() <= 1e-6


@pytest.mark.parametrize("per", [0, 1])
def test_pair_counting_is_optional(R, per):
    """no_pair_stats = 1 runs the compositing kernels without the pair
    counting: the same image and gradients, zero counts."""
    import torch
    sc = _small_scene(6, n=800, r=(0.01, 0.05))
    cams = [scenes.camera((0.2, -0.1, 2.3), 96, 72), scenes.camera((-1.7, 0.4, 1.4), 40, 56)]
    g = torch.from_numpy(np.random.default_rng(3).normal(size=(96 * 72 + 40 * 56, 3))
                         .astype(np.float32)).cuda()
    out = []
    for nps in (0, 1):
        img, st, _ = _gpu_render(R, sc, cams, persistent=per, no_pair_stats=nps)
        grads = R.backward(st, g)
        out.append((img, grads, st.stats()))
        st.close()
    assert torch.equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert _rel(b.cpu().numpy(), a.cpu().numpy().astype(np.float64)) <= 1e-5
    assert out[0][2]["fwd_composited"] > 0 and out[0][2]["bwd_contributing"] > 0
    assert all(v == 0 for v in out[1][2].values())


def test_forward_is_deterministic(R):
    sc = _small_scene(3, n=2000, r=(0.01, 0.05))
    cams = [scenes.camera((0.1, 0.1, 2.5), 128, 96)]
    a, sa, _ = _gpu_render(R, sc, cams)
    b, sb, _ = _gpu_render(R, sc, cams)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    sa.close()
    sb.close()


@pytest.mark.parametrize("kw", [dict(), dict(dir_frame=1), dict(radius_mode=1),
                                dict(max_per_pixel=15), dict(bg=(0.2, 0.5, 0.9)),
                                dict(t_eps=0.0, cutoff_k=4.0), dict(alpha_max=0.5),
                                dict(batch_depth=256), dict(max_per_pixel=15, batch_depth=64),
                                dict(persistent=1, max_per_pixel=15),
                                dict(persistent=1, tile=(16, 32), max_per_pixel=3),
                                dict(persistent=1, t_eps=0.0, cutoff_k=4.0),
                                dict(persistent=1, tile=(8, 8), bg=(0.2, 0.5, 0.9))],
                         ids=["default", "world-dir", "ndc-radius", "n15", "bg", "no-stop",
                              "amax", "staged", "staged-n15", "persistent-n15",
                              "persistent-16x32-n3", "persistent-no-stop", "persistent-8x8-bg"])
def test_option_variants(R, kw):
    sc = _small_scene(4, n=600)
    if kw.get("radius_mode") == 1:
        sc["radius"] = (sc["radius"] * 0.1).astype(np.float32)
    cams = [scenes.camera((1.0, 0.5, 2.0), 80, 64)]
    img, st, _ = _gpu_render(R, sc, cams, **kw)
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams,
                         **_oracle_kw(kw))
    err = np.abs(img.cpu().numpy() - ref).max()
    print(f"{kw}: image max abs err {err:.3e}")
    assert err <= IMG_TOL
    st.close()


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_sh_degrees(R, deg):
    sc = _small_scene(5 + deg, n=300, deg=deg)
    cams = [scenes.camera((0.0, -1.0, 2.0), 48, 48)]
    img, st, _ = _gpu_render(R, sc, cams)
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], deg, cams)
    assert np.abs(img.cpu().numpy() - ref).max() <= IMG_TOL
    st.close()


@pytest.mark.parametrize("sched", [dict(), dict(persistent=1, tile=(16, 32)),
                                   dict(persistent=1, tile=(8, 8), bwd_mode=2)],
                         ids=["streamed", "persistent-16x32", "persistent-8x8-store"])
def test_edge_cases(R, sched):
    import torch
    pbr = _pbr()
    cam = scenes.camera((0.0, 0.0, 2.5), 20, 12)
    # empty scene -> background everywhere, zero gradients
    empty = dict(pos=np.zeros((0, 3), np.float32), sh=np.zeros((0, 1, 3), np.float32),
                 opacity=np.zeros(0, np.float32), radius=np.zeros(0, np.float32), deg=0)
    img, st, _ = _gpu_render(R, empty, [cam], bg=(0.1, 0.2, 0.3), **sched)
    assert np.allclose(img.cpu().numpy(), [0.1, 0.2, 0.3])
    st.close()
    # every point behind the camera or at the near plane -> culled, zero gradients
    sc = _small_scene(9, n=50)
    sc["pos"][:, 2] = np.float32(2.5)  # z = 0 in the camera frame
    img, st, _ = _gpu_render(R, sc, [cam], **sched)
    assert np.all(img.cpu().numpy() == 0) and st.info()["n_pairs"] == 0
    gpos, gsh, gop = R.backward(st, torch.ones_like(img))
    assert not gpos.any() and not gsh.any() and not gop.any()
    st.close()
    # a 1x1 image and one-row and one-column images, with their gradients
    sc = _small_scene(10, n=200, spread=0.2, r=(0.05, 0.2))
    for W, H in ((1, 1), (37, 1), (1, 29)):
        c = scenes.camera((0.0, 0.0, 2.0), W, H)
        img, st, _ = _gpu_render(R, sc, [c], **sched)
        ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], [c])
        assert np.abs(img.cpu().numpy() - ref).max() <= IMG_TOL
        g = np.random.default_rng(W * 100 + H).normal(size=ref.shape)
        gpos, gsh, gop = R.backward(st, torch.from_numpy(g.astype(np.float32)).cuda())
        dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                                    [c], g)
        for a, b in ((gpos, dpos), (gop, dop)):
            a = a.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(a - b) <= GRAD_TOL * max(np.linalg.norm(b), 1e-12)
        st.close()
    # equal depths: ties broken by point index
    sc = _small_scene(11, n=40)
    sc["pos"][:, 2] = np.float32(0.25)
    img, st, _ = _gpu_render(R, sc, [cam], **sched)
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], [cam])
    assert np.abs(img.cpu().numpy() - ref).max() <= IMG_TOL
    st.close()
    # transparent points (opacity 0) are composited with alpha 0: the image
    # is the background, T stays 1, the position and SH gradients are 0 and
    # the opacity gradient is not (it carries the background term); and a
    # scene of one point
    bg = (0.2, 0.3, 0.4)
    for n, op in ((60, 0.0), (1, 0.9)):
        sc = _small_scene(12 + n, n=n, spread=0.3, r=(0.05, 0.1))
        sc["opacity"][:] = np.float32(op)
        img, st, _ = _gpu_render(R, sc, [cam], bg=bg, **sched)
        ref, T, cnt = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                               [cam], bg=bg)
        assert cnt.sum() > 0
        assert np.abs(img.cpu().numpy() - ref).max() <= IMG_TOL
        g = np.random.default_rng(n).normal(size=ref.shape)
        gpos, gsh, gop = R.backward(st, torch.from_numpy(g.astype(np.float32)).cuda())
        dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"],
                                    sc["deg"], [cam], g, bg=bg)
        if op == 0.0:
            assert np.allclose(ref, bg) and np.all(T == 1.0)
            assert not gpos.any() and not gsh.any() and np.linalg.norm(dop) > 0
        for a, b in ((gpos, dpos), (gsh, dsh), (gop, dop)):
            a = a.cpu().numpy().astype(np.float64).reshape(b.shape)
            assert np.linalg.norm(a - b) <= GRAD_TOL * max(np.linalg.norm(b), 1e-12)
        st.close()
    # invalid arguments are rejected, not run
    with pytest.raises(pbr.PBRError):
        _gpu_render(R, sc, [cam], tile=(32, 32))
    with pytest.raises(pbr.PBRError):
        _gpu_render(R, sc, [scenes.camera((0, 0, 2), 0, 10)])


def test_many_views_of_one_scene(R):
    """More views of one scene than the per-point kernels stage at a time
    (64): image and gradients of 70 small views against the oracle."""
    import torch
    sc = _small_scene(14, n=150, deg=2)
    cams = scenes.ring_cameras(70, 2.3, 12, 10)
    img, st, _ = _gpu_render(R, sc, cams)
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams)
    assert np.abs(img.cpu().numpy() - ref).max() <= IMG_TOL
    g = np.random.default_rng(2).normal(size=img.shape).astype(np.float32)
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g).cuda())
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams,
                                g.astype(np.float64))
    assert _rel(gpos.cpu().numpy(), dpos) <= GRAD_TOL
    assert _rel(gsh.cpu().numpy().reshape(dsh.shape), dsh) <= GRAD_TOL
    assert _rel(gop.cpu().numpy(), dop) <= GRAD_TOL
    st.close()


def test_multi_scene_multi_view(R):
    pbr = _pbr()
    a = _small_scene(12, n=300, deg=1)
    b = _small_scene(13, n=500, deg=3)
    cams = [scenes.camera((0.2, 0.1, 2.3), 50, 40), scenes.camera((-1.5, 0.3, 1.6), 41, 33),
            scenes.camera((0.0, 1.9, 0.6), 64, 64)]
    sov = [1, 0, 1]
    sa = pbr.Scene(a["pos"], a["sh"], a["opacity"], a["radius"], a["deg"])
    sb = pbr.Scene(b["pos"], b["sh"], b["opacity"], b["radius"], b["deg"])
    img, st = R.forward([sa, sb], cams, pbr.default_opts(), scene_of_view=sov)
    got = img.cpu().numpy()
    off = 0
    for v, c in enumerate(cams):
        sc = (a, b)[sov[v]]
        ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], [c])
        n = c["width"] * c["height"]
        assert np.abs(got[off:off + n] - ref).max() <= IMG_TOL
        off += n
    # gradients are packed per scene
    g = np.random.default_rng(0).normal(size=got.shape).astype(np.float32)
    import torch
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g).cuda())
    gpos, gsh, gop = gpos.cpu().numpy(), gsh.cpu().numpy(), gop.cpu().numpy()
    pbase, shbase = 0, 0
    for si, sc in enumerate((a, b)):
        views = [v for v in range(3) if sov[v] == si]
        pix = []
        offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
        gsel = np.concatenate([g[offs[v]:offs[v + 1]] for v in views])
        dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                                    [cams[v] for v in views], gsel)
        n, K = len(sc["pos"]), (sc["deg"] + 1) ** 2
        assert _rel(gpos[pbase:pbase + n], dpos) <= GRAD_TOL
        assert _rel(gsh[shbase:shbase + n * K * 3].reshape(n, K, 3), dsh) <= GRAD_TOL
        assert _rel(gop[pbase:pbase + n], dop) <= GRAD_TOL
        pbase += n
        shbase += n * K * 3
    st.close()


@pytest.mark.parametrize("sched", [dict(), dict(persistent=1, tile=(16, 32)),
                                   dict(batch_depth=128)],
                         ids=["streamed", "persistent-16x32", "staged"])
def test_batch_with_empty_view_and_empty_scene(R, sched):
    """A batch holding a view that sees nothing (the camera looks away from
    its scene), a scene of no points, a view of that scene between views
    that do see points, and a scene no view sees: every view's image and
    every scene's gradients against the oracle (the empty parts give the
    background and zero gradients, the unseen scene zero gradients written
    over the NaN-filled buffers, and none shifts its neighbours' offsets)."""
    import torch
    pbr = _pbr()
    a = _small_scene(21, n=300, deg=1)
    b = _small_scene(22, n=200, deg=2)
    e = dict(pos=np.zeros((0, 3), np.float32), sh=np.zeros((0, 4, 3), np.float32),
             opacity=np.zeros(0, np.float32), radius=np.zeros(0, np.float32), deg=1)
    cams = [scenes.camera((0.2, 0.1, 2.3), 48, 40),
            scenes.camera((0.0, 0.0, 2.5), 40, 24, target=(0.0, 0.0, 6.0)),  # looks away
            scenes.camera((0.3, 0.2, 2.0), 32, 32),
            scenes.camera((-1.5, 0.3, 1.6), 41, 33)]
    sov = [0, 0, 1, 2]
    u = _small_scene(24, n=70, deg=3)  # no view sees it
    groups = (a, e, b, u)
    bg = (0.1, 0.2, 0.3)
    sc = [pbr.Scene(x["pos"], x["sh"], x["opacity"], x["radius"], x["deg"]) for x in groups]
    img, st = R.forward(sc, cams, pbr.default_opts(bg=bg, **sched), scene_of_view=sov)
    got = img.cpu().numpy()
    offs = np.cumsum([0] + [c["width"] * c["height"] for c in cams])
    for v, c in enumerate(cams):
        x = groups[sov[v]]
        ref, _, cnt = O.render(x["pos"], x["sh"], x["opacity"], x["radius"], x["deg"], [c],
                               bg=bg)
        if v in (1, 2):
            assert cnt.sum() == 0 and np.allclose(ref, bg)
        err = np.abs(got[offs[v]:offs[v + 1]] - ref).max()
        assert err <= IMG_TOL, (v, err)
    g = np.random.default_rng(23).normal(size=got.shape).astype(np.float32)
    n_tot = sum(len(x["pos"]) for x in groups)
    n_sh = sum(len(x["pos"]) * (x["deg"] + 1) ** 2 * 3 for x in groups)
    out = (torch.full((n_tot, 3), float("nan"), device="cuda"),
           torch.full((n_sh,), float("nan"), device="cuda"),
           torch.full((n_tot,), float("nan"), device="cuda"))
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g).cuda(), out=out)
    gpos, gsh, gop = gpos.cpu().numpy(), gsh.cpu().numpy(), gop.cpu().numpy()
    assert np.isfinite(gpos).all() and np.isfinite(gsh).all() and np.isfinite(gop).all()
    pbase = shbase = 0
    for si, x in enumerate(groups):
        views = [v for v in range(len(cams)) if sov[v] == si]
        n, K = len(x["pos"]), (x["deg"] + 1) ** 2
        if n and not views:
            assert not gpos[pbase:pbase + n].any() and not gop[pbase:pbase + n].any()
            assert not gsh[shbase:shbase + n * K * 3].any()
        elif n:
            gsel = np.concatenate([g[offs[v]:offs[v + 1]] for v in views])
            dpos, dsh, dop = O.backward(x["pos"], x["sh"], x["opacity"], x["radius"], x["deg"],
                                        [cams[v] for v in views], gsel, bg=bg)
            assert _rel(gpos[pbase:pbase + n], dpos) <= GRAD_TOL
            assert _rel(gsh[shbase:shbase + n * K * 3].reshape(n, K, 3), dsh) <= GRAD_TOL
            assert _rel(gop[pbase:pbase + n], dop) <= GRAD_TOL
        pbase += n
        shbase += n * K * 3
    assert pbase == len(gpos) and shbase == len(gsh)
    # without the opacity gradient (a NULL buffer): the same other gradients
    gpos2, gsh2, gop2 = R.backward(st, torch.from_numpy(g).cuda(), want_opacity=False)
    assert gop2 is None
    assert _rel(gpos2.cpu().numpy(), gpos) <= 1e-5 and _rel(gsh2.cpu().numpy(), gsh) <= 1e-5
    st.close()


# ----------------------------------------------------------------- backward
def test_tiny_config_gradients(R):
    """Config: L2 loss against the image of positions jittered by N(0, 0.01).
    dL/dI comes from the oracle's images and is fed to both backward passes;
    the GPU loss kernel is checked on the GPU images."""
    import torch
    pbr = _pbr()
    sc = scenes.tiny()
    img, st, _ = _gpu_render(R, sc, sc["cams"])
    ref, _, _ = O.render(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], sc["cams"])
    tref, _, _ = O.render(sc["target_pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                          sc["cams"])
    gn = 2.0 * (ref - tref)
    gpos, gsh, gop = R.backward(st, torch.from_numpy(gn.astype(np.float32)).cuda())
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"],
                                sc["cams"], gn)
    e = (_rel(gpos.cpu().numpy(), dpos), _rel(gsh.cpu().numpy().reshape(dsh.shape), dsh),
         _rel(gop.cpu().numpy(), dop))
    print(f"tiny grads rel L2 vs FP64 oracle: pos {e[0]:.2e} sh {e[1]:.2e} opacity {e[2]:.2e}")
    assert max(e) <= GRAD_TOL
    # the loss kernel: sum of squares and its gradient
    target = torch.from_numpy(tref.astype(np.float32)).cuda()
    loss, g = pbr.image_loss(img, target, "l2")
    d = img.double() - target.double()
    assert abs(float(loss.item()) - float((d * d).sum())) <= 1e-6 * max(1.0, float((d * d).sum()))
    assert torch.allclose(g, 2 * (img - target), atol=1e-6)
    loss1, g1 = pbr.image_loss(img, target, "l1")
    assert abs(float(loss1.item()) - float(d.abs().sum())) <= 1e-6 * max(1.0, float(d.abs().sum()))
    assert torch.equal(g1, torch.sign(img - target))
    st.close()


@pytest.mark.parametrize("kw", [dict(dir_frame=1), dict(radius_mode=1), dict(max_per_pixel=15),
                                dict(bg=(0.3, 0.1, 0.7)), dict(tile=(8, 8)), dict(tile=(16, 32)),
                                dict(batch_depth=256), dict(tile=(8, 8), batch_depth=64),
                                dict(max_per_pixel=15, batch_depth=128), dict(persistent=1),
                                dict(persistent=1, tile=(16, 32), max_per_pixel=15),
                                dict(persistent=1, tile=(8, 8))],
                         ids=["world-dir", "ndc", "n15", "bg", "8x8", "16x32", "staged",
                              "staged-8x8", "staged-n15", "persistent", "persistent-16x32-n15",
                              "persistent-8x8"])
def test_gradient_variants(R, kw):
    import torch
    sc = _small_scene(20, n=400, deg=3)
    if kw.get("radius_mode") == 1:
        sc["radius"] = (sc["radius"] * 0.1).astype(np.float32)
    cams = [scenes.camera((0.4, 0.6, 2.1), 72, 56), scenes.camera((-1.2, -0.2, 1.9), 40, 48)]
    img, st, _ = _gpu_render(R, sc, cams, **kw)
    g = np.random.default_rng(1).normal(size=img.shape).astype(np.float32)
    gpos, gsh, gop = R.backward(st, torch.from_numpy(g).cuda())
    dpos, dsh, dop = O.backward(sc["pos"], sc["sh"], sc["opacity"], sc["radius"], sc["deg"], cams,
                                g.astype(np.float64), **_oracle_kw(kw))
    e = (_rel(gpos.cpu().numpy(), dpos), _rel(gsh.cpu().numpy().reshape(dsh.shape), dsh),
         _rel(gop.cpu().numpy(), dop))
    print(f"{kw}: grads rel L2 pos {e[0]:.2e} sh {e[1]:.2e} opacity {e[2]:.2e}")
    assert max(e) <= GRAD_TOL
    st.close()
