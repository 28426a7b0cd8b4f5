"""Pins for the oracle's projection, binning and blending (Sec. 3.1 Eq. 1,
Sec. 3.2 Eqs. 5-7).

Each check is fixed by something other than the oracle itself: inverse
projection, the closed-form image of one isolated splat, the transmittance
identity, full occlusion, permutation invariance, camera-centre geometry for
the world-frame direction, and brute-force enumeration for the tile lists.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2205_14330_gb300 import scenes

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def _one_point_scene(P, h_dc=None, deg=0, o=0.8, r=0.02):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0] = h_dc if h_dc is not None else (1.0 / Y00)
    return (np.asarray([P], np.float32), sh, np.asarray([o], np.float32),
            np.asarray([r], np.float32))


def test_on_axis_point_lands_on_principal_point():
    cam = scenes.camera((0.0, 0.0, 2.5), 128, 96)
    pos, sh, op, rad = _one_point_scene((0.0, 0.0, 0.0))
    recs, _ = O.preprocess(pos, sh, rad, 0, [cam])
    r = recs[0, 0]
    assert r["px"] == pytest.approx(64.0, abs=1e-12) and r["py"] == pytest.approx(48.0, abs=1e-12)
    assert r["X"][2] == pytest.approx(2.5, abs=1e-6)


def test_backprojected_pixels_project_back():
    rng = np.random.default_rng(1)
    cam = scenes.camera((1.0, 2.0, 3.0), 320, 200, fov_deg=60)
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    u = rng.uniform(0, 320, 50)
    v = rng.uniform(0, 200, 50)
    d = rng.uniform(1.0, 6.0, 50)
    Xc = np.stack([d * (u - float(cam["cx"])) / float(cam["fx"]),
                   d * (v - float(cam["cy"])) / float(cam["fy"]), d], 1)
    P = np.linalg.solve(R, (Xc - t).T).T  # R is fp32-rounded, so invert it exactly
    recs, _ = O.preprocess(P, np.zeros((50, 1, 3)), np.full(50, 0.01), 0, [cam])
    assert np.abs(recs[0]["px"] - u).max() < 1e-9
    assert np.abs(recs[0]["py"] - v).max() < 1e-9
    assert np.abs(recs[0]["X"][:, 2] - d).max() < 1e-9
    # the fp32 decision path agrees with the double one to fp32 accuracy
    assert np.abs(recs[0]["px32"] - u).max() < 1e-3


def test_isolated_splat_closed_form():
    """One point on the optical axis: I(u) = a c + (1 - a) bg inside the
    cutoff, bg outside, a = min(a_max, o exp(-d^2 / (2 s^2))), s = fx r / z."""
    W = H = 48
    cam = scenes.camera((0.0, 0.0, 2.5), W, H)
    deg = 3
    pos, _, op, rad = _one_point_scene((0.0, 0.0, 0.0), deg=deg, o=0.7, r=0.03)
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 0] = (0.9, 0.5, 0.1)  # DC
    sh[0, 2] = (0.2, 0.0, -0.1)  # Y_10 = sqrt(3/4pi) z
    sh[0, 6] = (0.0, 0.3, 0.0)  # Y_20 = sqrt(5/4pi) (3z^2-1)/2
    sh[0, 12] = (0.1, 0.1, 0.1)  # Y_30 = sqrt(7/4pi) (5z^3-3z)/2
    sh[0, 1] = (5.0, 5.0, 5.0)  # Y_1-1 ~ y vanishes on the axis
    bg = (0.25, 0.5, 0.75)
    # on the axis v = (0,0,1): Y00 = 1/(2 sqrt pi), Y10 = sqrt(3/4pi),
    # Y20 = sqrt(5/4pi), Y30 = sqrt(7/4pi)
    Yax = {0: Y00, 2: math.sqrt(3 / (4 * math.pi)), 6: math.sqrt(5 / (4 * math.pi)),
           12: math.sqrt(7 / (4 * math.pi))}
    c = sum(np.asarray(sh[0, k], np.float64) * y for k, y in Yax.items())
    rgb, T, cnt = O.render(pos, sh, op, rad, deg, [cam], bg=bg, screen_fp32=0, t_eps=0.0)
    fx = float(cam["fx"])
    r32, o32 = float(np.float32(0.03)), float(np.float32(0.7))  # inputs are fp32
    s = fx * r32 / 2.5
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx + 0.5 - W / 2) ** 2 + (yy + 0.5 - H / 2) ** 2
    a = np.minimum(0.99, o32 * np.exp(-d2 / (2 * s * s)))
    inside = d2 <= (3 * s) ** 2
    expect = np.where(inside[..., None], a[..., None] * c + (1 - a[..., None]) * np.asarray(bg),
                      np.asarray(bg)[None, None, :])
    assert np.abs(rgb.reshape(H, W, 3) - expect).max() < 1e-12
    assert np.array_equal(cnt.reshape(H, W), inside.astype(np.int32))


def test_clamped_splat_is_capped_at_alpha_max():
    cam = scenes.camera((0.0, 0.0, 2.5), 16, 16)
    pos, sh, op, rad = _one_point_scene((0.0, 0.0, 0.0), o=5.0, r=0.2)
    rgb, T, cnt = O.render(pos, sh, op, rad, 0, [cam], t_eps=0.0)
    # at the four central pixels o exp(-0.5/(2 s^2)) >> 0.99
    centre = rgb.reshape(16, 16, 3)[7:9, 7:9]
    assert np.allclose(centre, 0.99, atol=1e-12)
    assert np.allclose(T.reshape(16, 16)[7:9, 7:9], 0.01, atol=1e-12)


def _random_scene(seed, n=40, deg=2, W=40, H=32):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-0.6, 0.6, (n, 3)).astype(np.float32)
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3)).astype(np.float32)
    sh[:, 0] += 1.0
    op = rng.uniform(0.3, 0.95, n).astype(np.float32)
    rad = rng.uniform(0.03, 0.08, n).astype(np.float32)
    cam = scenes.camera((0.3, -0.2, 2.5), W, H)
    return pos, sh, op, rad, deg, [cam]


@pytest.mark.parametrize("t_eps", [0.0, 1e-3])
def test_transmittance_identity(t_eps):
    """With every colour 1 and bg = 0, I = sum_i A_i = 1 - prod(1 - a_i) = 1 - T."""
    pos, _, op, rad, _, cams = _random_scene(2, deg=0)
    sh = np.zeros((len(pos), 1, 3), np.float32)
    sh[:, 0] = 1.0 / Y00
    rgb, T, cnt = O.render(pos, sh, op, rad, 0, cams, t_eps=t_eps)
    assert cnt.max() >= 4  # the scene really overlaps
    c = float(np.float32(1.0 / Y00)) * Y00  # the fp32 coefficient times Y00 (1 up to 3e-8)
    assert np.abs(rgb - c * (1.0 - T)[:, None]).max() < 1e-12


def test_occlusion_by_an_opaque_point():
    cam = scenes.camera((0.0, 0.0, 3.0), 16, 16)
    pos = np.array([[0, 0, 0.5], [0, 0, -0.5]], np.float32)  # first is nearer the camera
    sh = np.zeros((2, 1, 3), np.float32)
    sh[0, 0] = (1.0 / Y00, 0, 0)
    sh[1, 0] = (0, 1.0 / Y00, 0)
    op = np.array([50.0, 0.6], np.float32)  # front point clamps to alpha_max
    rad = np.array([0.05, 0.05], np.float32)
    rgb, T, cnt = O.render(pos, sh, op, rad, 0, [cam], t_eps=0.0, screen_fp32=0)
    pix = 8 * 16 + 8
    # behind point contributes (1 - a_max) * a_b * c_b exactly
    fx = float(cam["fx"])
    s_b = fx * float(np.float32(0.05)) / 3.5
    d2 = 0.25 + 0.25  # pixel (8,8) centre vs principal point (8,8)
    a_b = float(np.float32(0.6)) * math.exp(-d2 / (2 * s_b * s_b))
    c = float(np.float32(1.0 / Y00)) * Y00
    assert rgb[pix, 0] == pytest.approx(0.99 * c, abs=1e-12)
    assert rgb[pix, 1] == pytest.approx(0.01 * a_b * c, abs=1e-12)
    # with t_eps above 1 - a_max the behind point is never reached
    rgb2, T2, cnt2 = O.render(pos, sh, op, rad, 0, [cam], t_eps=0.02)
    assert rgb2[pix, 1] == 0.0 and cnt2[pix] == 1


def test_permutation_invariance():
    pos, sh, op, rad, deg, cams = _random_scene(3)
    perm = np.random.default_rng(0).permutation(len(pos))
    a = O.render(pos, sh, op, rad, deg, cams)
    b = O.render(pos[perm], sh[perm], op[perm], rad[perm], deg, cams)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_max_per_pixel_keeps_the_nearest():
    pos, sh, op, rad, deg, cams = _random_scene(4)
    rgb1, T1, c1 = O.render(pos, sh, op, rad, deg, cams, max_per_pixel=1, t_eps=0.0)
    assert c1.max() == 1
    # per pixel, the single composited point is the nearest candidate
    order = np.argsort(O.preprocess(pos, sh, rad, deg, cams)[0][0]["z32"], kind="stable")
    rgb_all = np.zeros_like(rgb1)
    done = np.zeros(len(rgb1), bool)
    for i in order:  # nearest first: render each point alone, keep the first hit
        ri, Ti, ci = O.render(pos[i:i + 1], sh[i:i + 1], op[i:i + 1], rad[i:i + 1], deg, cams,
                              t_eps=0.0)
        hit = (ci == 1) & ~done
        rgb_all[hit] = ri[hit]
        done |= hit
    assert np.abs(rgb_all - rgb1).max() < 1e-12


def test_empty_scene_is_background():
    cam = scenes.camera((0.0, 0.0, 2.5), 8, 4)
    rgb, T, cnt = O.render(np.zeros((0, 3)), np.zeros((0, 1, 3)), np.zeros(0), np.zeros(0), 0,
                           [cam], bg=(0.1, 0.2, 0.3))
    assert np.allclose(rgb, [0.1, 0.2, 0.3]) and np.all(T == 1) and np.all(cnt == 0)


def test_point_behind_camera_and_near_plane_is_culled():
    cam = scenes.camera((0.0, 0.0, 2.5), 16, 16)
    pos = np.array([[0, 0, 3.0], [0, 0, 2.495], [0, 0, 2.48]], np.float32)  # z = -0.5, 0.005, 0.02
    recs, _ = O.preprocess(pos, np.zeros((3, 1, 3)), np.full(3, 0.01), 0, [cam])
    assert list(recs[0]["visible"]) == [0, 0, 1]


def test_world_frame_direction_uses_camera_centre():
    """dir_frame=1 evaluates the SH at (P - C)/|P - C|, C the camera centre."""
    rng = np.random.default_rng(6)
    pos = rng.uniform(-0.5, 0.5, (10, 3)).astype(np.float32)
    sh = rng.normal(0, 1, (10, 9, 3)).astype(np.float32)
    eye = np.array([1.5, 1.0, 2.0])
    cam = scenes.camera(eye, 32, 32)
    recs, _ = O.preprocess(pos, sh, np.full(10, 0.02), 2, [cam], dir_frame=1)
    d = pos.astype(np.float64) - eye  # camera centre is the eye
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(2, d)
    c = np.einsum("nk,nkc->nc", Y, sh.astype(np.float64))
    vis = recs[0]["visible"] == 1
    assert vis.sum() >= 5
    assert np.abs(recs[0]["rgb"][vis] - c[vis]).max() < 1e-6  # camera given in fp32
    # camera frame: the direction of an on-axis point is (0,0,1) (a radius
    # wide enough for its cutoff disc to include pixels, so it is visible)
    recs0, _ = O.preprocess(np.zeros((1, 3), np.float32), sh[:1], np.full(1, 0.1), 2,
                            [scenes.camera((0, 0, 2.0), 8, 8)])
    assert recs0[0, 0]["visible"]
    assert np.allclose(recs0[0, 0]["dir"], [0, 0, 1], atol=1e-7)


def test_ndc_radius_is_depth_independent():
    cam = scenes.camera((0.0, 0.0, 2.5), 64, 48)
    pos = np.array([[0, 0, 1.0], [0.1, 0, -1.0]], np.float32)
    recs, _ = O.preprocess(pos, np.zeros((2, 1, 3)), np.full(2, 0.05), 0, [cam], radius_mode=1)
    assert np.allclose(recs[0]["s32"], 0.05 * 48 / 2)


def test_sh_degree_zero_padding_is_inert():
    pos, sh, op, rad, _, cams = _random_scene(7, deg=2)
    sh3 = np.zeros((len(pos), 16, 3), np.float32)
    sh3[:, :9] = sh
    a = O.render(pos, sh, op, rad, 2, cams)
    b = O.render(pos, sh3, op, rad, 3, cams)
    assert np.abs(a[0] - b[0]).max() < 1e-14


# ---------------------------------------------------------------- binning
def _included_pixels(r, W, H):
    """(ys, xs) of the pixels whose centre passes the Sec. 3.2 cutoff test in
    fp32 round-to-nearest: d2 = (ux - px)^2 + (uy - py)^2 <= rc^2, tested at
    every pixel of the image (numpy fp32 arithmetic, one rounding per
    operation)."""
    f32 = np.float32
    if not (f32(r["z32"]) > f32(0.01) and f32(r["s32"]) > 0):
        return np.zeros(0, int), np.zeros(0, int)
    dx = (np.arange(W, dtype=f32) + f32(0.5)) - f32(r["px32"])
    dy = (np.arange(H, dtype=f32) + f32(0.5)) - f32(r["py32"])
    d2 = (dx * dx)[None, :] + (dy * dy)[:, None]
    return np.nonzero(d2 <= f32(r["rc2_32"]))


def _lists_from_pixels(recs, cams, tw, th):
    """The binning from its definition: (tile, pv) is listed iff some pixel
    of the tile is included, with bit (y % th // 8) * (tw // 8) + x % tw // 8
    set for each included pixel (x, y); ordered by (tile, depth bits, pv)."""
    out = []
    n = recs.shape[1]
    tile_base = 0
    for v, cam in enumerate(cams):
        W, H = cam["width"], cam["height"]
        tpr = -(-W // tw)
        for i in range(n):
            r = recs[v, i]
            ys, xs = _included_pixels(r, W, H)
            got = {}
            for x, y in zip(xs.tolist(), ys.tolist()):
                t = tile_base + (y // th) * tpr + x // tw
                got[t] = got.get(t, 0) | 1 << ((y % th) // 8 * (tw // 8) + (x % tw) // 8)
            zb = int(np.float32(r["z32"]).view(np.uint32))
            out += [(t, zb, v * n + i, m) for t, m in got.items()]
        tile_base += tpr * -(-H // th)
    out.sort()
    return (np.array([o[0] for o in out], np.uint32), np.array([o[2] for o in out], np.uint32),
            np.array([o[3] for o in out], np.uint8))


def _scene_with_big_splats(seed, W, H):
    """A random scene plus a few splats wide enough that their pixel box
    spans more than 32 tiles of 8 x 8, some cut by the image border."""
    pos, sh, op, rad, deg, cams = _random_scene(seed, n=60, W=W, H=H)
    rad = rad.copy()
    rad[:4] = [0.45, 0.3, 0.6, 0.25]
    pos = pos.copy()
    pos[2] = [0.9, -0.7, 0.2]
    return pos, sh, op, rad, deg, cams


@pytest.mark.parametrize("tw,th", [(16, 16), (8, 8), (16, 32)])
def test_bin_lists_are_the_pixel_inclusion_sets(tw, th):
    """Both directions: every included pixel's tile lists the point with the
    pixel's 8 x 8 block bit set, and every listed (tile, block) holds an
    included pixel; ordered by (tile, depth bits, point-view)."""
    pos, sh, op, rad, deg, cams = _scene_with_big_splats(8, 70, 45)
    cams = cams + [scenes.camera((-1.0, 0.5, 2.0), 33, 17)]
    keys, vals, masks, ranges, recs = O.bin_tiles(pos, sh, rad, deg, cams, tile_w=tw, tile_h=th)
    k2, v2, m2 = _lists_from_pixels(recs, cams, tw, th)
    assert np.array_equal(keys, k2) and np.array_equal(vals, v2) and np.array_equal(masks, m2)
    # boxes wider than 32 tiles really occur at 8 x 8
    if tw == 8:
        wide = [(r["tx_hi"] - r["tx_lo"] + 1) * (r["ty_hi"] - r["ty_lo"] + 1) for r in recs[0]]
        assert max(wide) > 32
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        assert np.all(keys[s:e] == t)
    assert int((ranges[:, 1] - ranges[:, 0]).sum()) == len(keys)
    # a point-view is visible iff it includes a pixel
    for v, cam in enumerate(cams):
        for i in range(len(pos)):
            has = _included_pixels(recs[v, i], cam["width"], cam["height"])[0].size > 0
            assert bool(recs[v, i]["visible"]) == has


def test_pixel_box_covers_every_included_pixel():
    """Every pixel that passes the fp32 cutoff test lies in the point's box."""
    pos, sh, op, rad, deg, cams = _random_scene(9, n=50, W=64, H=40)
    recs, _ = O.preprocess(pos, sh, rad, deg, cams)
    W, H = 64, 40
    ux = (np.arange(W, dtype=np.float32) + np.float32(0.5))
    uy = (np.arange(H, dtype=np.float32) + np.float32(0.5))
    for r in recs[0]:
        if not r["visible"]:
            continue
        dx = ux[None, :] - np.float32(r["px32"])
        dy = uy[:, None] - np.float32(r["py32"])
        d2 = (dx * dx).astype(np.float32) + (dy * dy).astype(np.float32)
        ys, xs = np.nonzero(d2 <= np.float32(r["rc2_32"]))
        if xs.size:
            assert xs.min() >= r["px_lo"] and xs.max() <= r["px_hi"]
            assert ys.min() >= r["py_lo"] and ys.max() <= r["py_hi"]
        # and the box is tight: at most two pixels wider than the disc
        assert r["px_hi"] - r["px_lo"] <= 2 * r["rc32"] + 3
