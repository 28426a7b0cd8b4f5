"""The C ABI library builds for sm_103a, loads without a GPU and exports
every function that include/pbr.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pbr_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2205_14330_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pbr_render_forward", "pbr_render_backward", "pbr_create", "pbr_destroy",
                     "pbr_state_free", "pbr_last_error", "pbr_forward_workspace_size",
                     "pbr_upload_scene", "pbr_evict_scene", "pbr_submit_request", "pbr_poll",
                     "pbr_serve_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\b(pbr_\w+)\b", out))
    assert set(_declared()) <= exported


def test_host_only_calls_work_without_a_gpu(libpath):
    from paper_2205_14330_gb300 import pbr
    o = pbr.default_opts()
    assert (o.tile_w, o.tile_h, o.batch_depth) == (16, 16, 0)
    assert abs(o.alpha_max - 0.99) < 1e-7 and abs(o.cutoff_k - 3.0) < 1e-7
    assert b"sm_103a" in pbr.lib().pbr_version()


STRUCTS = [("pbr_camera", "Camera"), ("pbr_render_opts", "Opts"), ("pbr_points", "Points"),
           ("pbr_state_info_t", "StateInfo"), ("pbr_optimizer_cfg", "OptimizerCfg"),
           ("pbr_serve_stats_t", "ServeStats"), ("pbr_refine_cfg", "RefineCfg"),
           ("pbr_frame_cfg", "FrameCfg")]


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the Python binding passes across the boundary has the
    header's size and field offsets (checked with the host C compiler)."""
    from paper_2205_14330_gb300 import pbr
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pbr.h"', "int main(void) {"]
    for c_name, py_name in STRUCTS:
        cls = getattr(pbr, py_name)
        lines.append(f'printf("{py_name} size %zu\\n", sizeof({c_name}));')
        for f in cls._fields_:
            lines.append(f'printf("{py_name} {f[0]} %zu\\n", offsetof({c_name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        cls_name, field, value = line.split()
        got[(cls_name, field)] = int(value)
    for _, py_name in STRUCTS:
        cls = getattr(pbr, py_name)
        assert got[(py_name, "size")] == ctypes.sizeof(cls), py_name
        for f in cls._fields_:
            assert got[(py_name, f[0])] == getattr(cls, f[0]).offset, (py_name, f[0])
