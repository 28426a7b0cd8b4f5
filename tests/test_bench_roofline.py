"""The bench's roofline arithmetic (host logic, no GPU): per-stage
algorithmic bytes, flops and ex2 counts of one training step, the binding
roof of each stage and the whole-step fraction, checked against sums
written out by hand for a small made-up step, and the captured-traffic
lookup's refusal of a changed kernel source."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


SIZES = {"n_point_views": 1000, "n_visible": 800, "n_pairs": 3000, "n_tiles": 50,
         "n_pixels": 10000}
PAIRS = {"fwd_composited": 20000, "bwd_contributing": 20000, "fwd_examined": 50000,
         "bwd_examined": 45000}


def test_stage_bytes_and_roofs():
    ms = {"preprocess_fwd": 1.0, "depth_sort": 1.0, "emit_pairs": 1.0, "tile_sort": 1.0,
          "tile_ranges": 1.0, "raster_fwd": 1.0, "raster_bwd": 1.0, "preprocess_bwd": 1.0}
    param, grad = 123456, 654321
    hbm, fp32, ex2 = 1000.0, 1.0, 10.0          # GB/s, TFLOP/s, G ex2/s
    r = bench.stage_roofline(ms, SIZES, PAIRS, param, grad, hbm, fp32, ex2, step_ms=10.0)
    st = r["stages"]
    # bytes written out from the definitions of the stages
    assert st["preprocess_fwd"]["bytes"] == param + 32 * 800 + 8 * 1000
    assert st["depth_sort"]["bytes"] == 16 * 800
    assert st["emit_pairs"]["bytes"] == 8 * 3000 + 12 * 800
    assert st["tile_sort"]["bytes"] == 16 * 3000
    assert st["tile_ranges"]["bytes"] == 4 * 3000 + 8 * 50
    assert st["raster_fwd"]["bytes"] == 32 * 800 + 4 * 3000 + 20 * 10000
    assert st["raster_bwd"]["bytes"] == 32 * 800 + 4 * 3000 + 20 * 10000 + 28 * 1000
    assert st["preprocess_bwd"]["bytes"] == 28 * 1000 + grad
    # flops and ex2 of the compositing stages
    assert st["raster_fwd"]["flops"] == 20000 * (bench.FLOP_TEST + bench.FLOP_FWD)
    assert st["raster_fwd"]["ex2"] == 20000
    assert st["raster_bwd"]["flops"] == 20000 * (bench.FLOP_TEST + bench.FLOP_BWD)
    assert st["raster_bwd"]["ex2"] == 2 * 20000
    # roofline time of a stage = the largest of its three times
    for k, v in st.items():
        t_b = v["bytes"] / (hbm * 1e9) * 1e3
        t_f = v["flops"] / (fp32 * 1e12) * 1e3
        t_x = v["ex2"] / (ex2 * 1e9) * 1e3
        assert v["roofline_ms"] == pytest.approx(max(t_b, t_f, t_x))
        assert v["bound"] == ["hbm", "fp32", "ex2"][[t_b, t_f, t_x].index(max(t_b, t_f, t_x))]
        assert v["frac"] == pytest.approx(v["roofline_ms"] / 1.0)
    total = sum(v["roofline_ms"] for v in st.values())
    assert r["roofline_ms"] == pytest.approx(total)
    assert r["step_frac"] == pytest.approx(total / 10.0)


def test_captured_traffic_needs_the_same_kernel_source(tmp_path, monkeypatch):
    key = next(iter(bench.CAPTURED_TRAFFIC))
    kernel, tile, depth, persistent = key
    sched = {"tile": tile, "batch_depth": depth, "persistent": persistent}
    rec = bench.CAPTURED_TRAFFIC[key]
    src = os.path.join(ROOT, rec["file"])
    # a copy of the tree with the kernel source changed by one byte
    root = tmp_path / "tree"
    dst = root / rec["file"]
    dst.parent.mkdir(parents=True)
    data = open(src, "rb").read()
    dst.write_bytes(data + b"\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.captured_traffic(kernel, sched) is None
    dst.write_bytes(data)
    import hashlib
    if hashlib.sha256(data).hexdigest() == rec["sha256"]:
        assert bench.captured_traffic(kernel, sched) == rec["bytes"]
    assert bench.captured_traffic(kernel, dict(sched, tile="1x1")) is None
