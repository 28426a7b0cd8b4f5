"""ctypes binding of libpbr.so (declared in include/pbr.h).

Argument marshalling only: every stage of the renderer runs in the library's
CUDA kernels.  PyTorch provides device memory (tensors) and the current
stream.  There is no CPU fallback: if the library cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is required for device memory
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpbr.so")

PBR_OK = 0
PBR_ERR_INVALID_ARG, PBR_ERR_NOT_FOUND = -1, -7
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "CAPACITY", -5: "TIMEOUT",
          -6: "DEVICE_STATUS", -7: "NOT_FOUND", -8: "BUSY"}


class PBRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pbr error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("width", C.c_int32), ("height", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("radius_mode", C.c_int32), ("dir_frame", C.c_int32), ("cutoff_k", C.c_float),
                ("alpha_max", C.c_float), ("t_eps", C.c_float), ("max_per_pixel", C.c_int32),
                ("bg", C.c_float * 3), ("z_near", C.c_float), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("batch_depth", C.c_int32), ("persistent", C.c_int32),
                ("no_pair_stats", C.c_int32), ("bwd_mode", C.c_int32),
                ("store_depth", C.c_int32)]


class Points(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("sh", C.c_void_p), ("opacity", C.c_void_p),
                ("radius", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32),
                ("reserved", C.c_int32)]


class StateInfo(C.Structure):
    _fields_ = [("n_point_views", C.c_int64), ("n_visible", C.c_int64), ("n_pairs", C.c_int64),
                ("n_tiles", C.c_int64), ("n_pixels", C.c_int64),
                ("tile_keys", C.c_void_p), ("tile_vals", C.c_void_p), ("ranges", C.c_void_p),
                ("records", C.c_void_p), ("ntiles", C.c_void_p), ("T_final", C.c_void_p),
                ("n_contrib", C.c_void_p)]


class OptimizerCfg(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lr_pos", C.c_float), ("lr_sh", C.c_float),
                ("lr_opacity", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("lambda_tv", C.c_float), ("loss_kind", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class RefineCfg(C.Structure):
    _fields_ = [("n_vox", C.c_int32), ("k", C.c_int32), ("eps", C.c_float),
                ("stages", C.c_int32)]


class FrameCfg(C.Structure):
    _fields_ = [("iters", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("k", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("queued", C.c_int64), ("in_flight_batches", C.c_int64), ("batches", C.c_int64),
                ("max_batch_views", C.c_int64), ("mean_batch_views", C.c_double),
                ("megapixels", C.c_double), ("span_s", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("hbm_in_use", C.c_size_t), ("hbm_budget", C.c_size_t)]


STAGES = ["preprocess_fwd", "compact", "depth_sort", "emit_pairs", "tile_sort", "tile_ranges",
          "raster_fwd", "raster_bwd", "preprocess_bwd", "other", "voxel_reduce", "knn",
          "refine_other"]

_lib = None
_lock = threading.Lock()


def lib():
    """Loads libpbr.so (raising if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpbr.so is missing ({LIB_PATH}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.pbr_create.argtypes = [C.POINTER(vp), C.c_int, C.c_size_t]
            L.pbr_destroy.argtypes = [vp]
            L.pbr_last_error.restype = C.c_char_p
            L.pbr_last_error.argtypes = [C.c_void_p]
            L.pbr_version.restype = C.c_char_p
            L.pbr_default_opts.argtypes = [C.POINTER(Opts)]
            L.pbr_default_opts.restype = None
            L.pbr_render_forward.argtypes = [vp, C.POINTER(Points), i32, vp, C.POINTER(Camera),
                                             i32, C.POINTER(Opts), vp, C.POINTER(vp), vp]
            L.pbr_render_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.pbr_forward_workspace_size.argtypes = [vp, C.POINTER(Points), i32, vp,
                                                     C.POINTER(Camera), i32, C.POINTER(Opts), i32,
                                                     C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                                     vp]
            L.pbr_state_free.argtypes = [vp, vp]
            L.pbr_state_info.argtypes = [vp, C.POINTER(StateInfo)]
            L.pbr_state_read.argtypes = [vp, i32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
            L.pbr_image_loss.argtypes = [i32, vp, vp, i64, vp, vp, vp]
            L.pbr_render_forward_noalloc.argtypes = [C.POINTER(Points), i32, vp,
                                                     C.POINTER(Camera), i32, C.POINTER(Opts),
                                                     vp, vp]
            L.pbr_graph_create.argtypes = [vp, C.POINTER(Points), i32, vp, C.POINTER(Camera), i32,
                                           C.POINTER(Opts), vp, vp, i32, vp, vp, vp, vp, vp,
                                           C.c_double, vp, C.POINTER(vp)]
            L.pbr_graph_launch.argtypes = [vp, i32, vp]
            L.pbr_graph_check.argtypes = [vp, vp, C.POINTER(i64), C.POINTER(i64)]
            L.pbr_graph_replan.argtypes = [vp, vp]
            L.pbr_graph_set_cameras.argtypes = [vp, C.POINTER(Camera), i32, vp]
            L.pbr_graph_destroy.argtypes = [vp]
            L.pbr_autotune.argtypes = [vp, C.POINTER(Points), i32, vp, C.POINTER(Camera), i32,
                                       C.POINTER(Opts), i32, i32, C.POINTER(C.c_double),
                                       C.POINTER(i32), vp]
            L.pbr_autotune_save.argtypes = [vp, C.c_char_p]
            L.pbr_autotune_load.argtypes = [vp, C.c_char_p, C.POINTER(i32)]
            L.pbr_serve_start.argtypes = [vp, C.POINTER(Opts), i32, i32]
            L.pbr_serve_stop.argtypes = [vp]
            L.pbr_serve_set_budget.argtypes = [vp, C.c_size_t]
            L.pbr_upload_scene.argtypes = [vp, C.POINTER(Points), C.POINTER(i32)]
            L.pbr_evict_scene.argtypes = [vp, i32]
            L.pbr_submit_request.argtypes = [vp, i32, C.POINTER(Camera), vp, C.c_double,
                                             C.POINTER(C.c_uint64)]
            L.pbr_poll.argtypes = [vp, C.c_uint64, C.POINTER(i32), C.POINTER(i32)]
            L.pbr_wait.argtypes = [vp, C.c_uint64, i32, C.POINTER(i32)]
            L.pbr_serve_stats.argtypes = [vp, C.POINTER(ServeStats), i32]
            L.pbr_now.restype = C.c_double
            L.pbr_now.argtypes = []
            L.pbr_serve_estimate.argtypes = [vp, C.c_int32, C.POINTER(Camera),
                                             C.POINTER(C.c_size_t)]
            L.pbr_serve_trace.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(i32), i32, C.POINTER(i32), i32]
            L.pbr_default_optimizer.argtypes = [C.POINTER(OptimizerCfg)]
            L.pbr_default_optimizer.restype = None
            L.pbr_image_loss_tv.argtypes = [C.POINTER(Camera), i32, vp, vp, i32, C.c_float, vp, vp,
                                            vp]
            L.pbr_optimizer_step.argtypes = [i32, vp, vp, vp, vp, i64, C.c_float, C.c_float,
                                             C.c_float, C.c_float, i32, vp]
            L.pbr_graph_set_optimizer.argtypes = [vp, C.POINTER(OptimizerCfg), vp]
            L.pbr_graph_set_lr.argtypes = [vp, C.c_float, C.c_float, C.c_float]
            L.pbr_state_stats.argtypes = [vp, C.POINTER(C.c_ulonglong)]
            L.pbr_kernel_launches.restype = C.c_ulonglong
            L.pbr_kernel_launches.argtypes = []
            L.pbr_set_stage_timing.argtypes = [vp, C.c_int]
            L.pbr_stage_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                          C.c_int]
            L.pbr_measure_alu_peaks.argtypes = [C.c_int, C.POINTER(C.c_double),
                                                C.POINTER(C.c_double)]
            L.pbr_default_refine.restype = None
            L.pbr_default_refine.argtypes = [C.POINTER(RefineCfg)]
            L.pbr_refine_points.argtypes = [vp, C.POINTER(Points), C.POINTER(RefineCfg), vp, vp,
                                            vp, vp, i64, C.POINTER(i64), vp]
            L.pbr_knn.argtypes = [vp, vp, i64, vp, i64, i32, i32, i32, vp, vp, vp]
            L.pbr_default_frame_cfg.restype = None
            L.pbr_default_frame_cfg.argtypes = [C.POINTER(FrameCfg)]
            L.pbr_chamfer.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp, vp, vp]
            L.pbr_frame_init.argtypes = [vp, C.POINTER(Points), vp, i64, C.POINTER(FrameCfg), vp,
                                         vp, vp, C.POINTER(C.c_double), vp]
            L.pbr_consistency_check.argtypes = [vp, vp, i64, C.POINTER(Camera), i32, vp,
                                                C.c_float, vp, vp]
            L.pbr_consistency_filter.argtypes = [vp, C.POINTER(Points), C.POINTER(Camera), i32,
                                                 vp, C.c_float, vp, vp, vp, vp, C.POINTER(i64),
                                                 vp]
            L.pbr_visual_hull_init.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                               C.POINTER(Camera), i32, vp, C.c_float,
                                               C.c_uint64, i64, i64, i32, vp, vp,
                                               C.POINTER(i64), C.POINTER(i64), vp]
            _lib = L
    return _lib


def check(rc):
    if rc != PBR_OK:
        raise PBRError(rc, lib().pbr_last_error(None).decode(errors="replace"))
    return rc


# ------------------------------------------------------------ marshalling
def default_opts(**kw) -> Opts:
    o = Opts()
    lib().pbr_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "bg":
            for j in range(3):
                o.bg[j] = float(v[j])
        elif k == "tile":
            o.tile_w, o.tile_h = int(v[0]), int(v[1])
        else:
            cur = getattr(o, k)
            setattr(o, k, float(v) if isinstance(cur, float) else int(v))
    return o


def make_cameras(cams):
    arr = (Camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        a = arr[i]
        a.fx, a.fy, a.cx, a.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
        R = np.asarray(c["R"], np.float32).reshape(9)
        t = np.asarray(c["t"], np.float32).reshape(3)
        for j in range(9):
            a.R[j] = float(R[j])
        for j in range(3):
            a.t[j] = float(t[j])
        a.width, a.height = int(c["width"]), int(c["height"])
    return arr


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Scene:
    """Device-resident point set: pos [n,3], sh [n,K,3], opacity [n], radius [n]."""

    def __init__(self, pos, sh, opacity, radius, deg, device="cuda"):
        def dev(a):
            t = a if torch.is_tensor(a) else torch.from_numpy(np.ascontiguousarray(a))
            return t.to(device=device, dtype=torch.float32).contiguous()
        self.pos, self.sh, self.opacity, self.radius = dev(pos), dev(sh), dev(opacity), dev(radius)
        self.deg = int(deg)
        self.n = int(self.pos.shape[0])
        assert self.sh.shape == (self.n, (self.deg + 1) ** 2, 3)

    def points(self) -> Points:
        return Points(_ptr(self.pos), _ptr(self.sh), _ptr(self.opacity), _ptr(self.radius),
                      self.n, self.deg, 0)


def n_pixels(cams):
    return sum(int(c["width"]) * int(c["height"]) for c in cams)


class State:
    """Forward state needed by the backward pass (freed on close/GC)."""

    def __init__(self, renderer, handle, scenes):
        self.renderer, self.handle, self.scenes = renderer, handle, scenes

    def info(self) -> dict:
        inf = StateInfo()
        check(lib().pbr_state_info(self.handle, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in StateInfo._fields_}

    ARRAYS = {"tile_keys": (0, np.uint32), "tile_vals": (1, np.uint32), "ranges": (2, np.uint32),
              "records": (3, np.float32), "ntiles": (4, np.uint32), "T_final": (5, np.float32),
              "n_contrib": (6, np.uint32), "T_store": (7, np.float32), "n_comp": (8, np.uint32)}

    def read(self, name: str) -> np.ndarray:
        """Host copy of one state array (see pbr_state_read)."""
        which, dt = self.ARRAYS[name]
        size = C.c_size_t()
        check(lib().pbr_state_read(self.handle, which, None, 0, C.byref(size)))
        out = np.empty(size.value // np.dtype(dt).itemsize, dt)
        check(lib().pbr_state_read(self.handle, which, out.ctypes.data, size.value,
                                   C.byref(size)))
        if name == "ranges":
            out = out.reshape(-1, 2)
        elif name == "records":
            out = out.reshape(-1, 8)
        return out

    def stats(self) -> dict:
        """Raster pair counts (the compositing kernels' work units)."""
        out = (C.c_ulonglong * 4)()
        check(lib().pbr_state_stats(self.handle, out))
        return dict(fwd_examined=out[0], fwd_composited=out[1], bwd_examined=out[2],
                    bwd_contributing=out[3])

    def close(self):
        if self.handle:
            lib().pbr_state_free(self.renderer.ctx, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Renderer:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.ctx = C.c_void_p()
        check(lib().pbr_create(C.byref(self.ctx), int(device), int(hbm_budget)))
        self.device = int(device)

    def close(self):
        if self.ctx:
            lib().pbr_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stage_timing(self, enable: bool):
        check(lib().pbr_set_stage_timing(self.ctx, 1 if enable else 0))

    def stage_times(self) -> dict:
        """{stage: (ms, calls)} accumulated since the last call (synchronises)."""
        ms = (C.c_double * len(STAGES))()
        calls = (C.c_longlong * len(STAGES))()
        check(lib().pbr_stage_times(self.ctx, ms, calls, len(STAGES)))
        return {name: (ms[i], calls[i]) for i, name in enumerate(STAGES)}

    def save_tuning(self, path):
        """Writes the autotuner's cached schedules to a JSON file."""
        check(lib().pbr_autotune_save(self.ctx, os.fsencode(path)))

    def load_tuning(self, path) -> int:
        """Merges a file written by save_tuning into the autotuner's cache;
        returns the number of shape classes it held."""
        n = C.c_int32()
        check(lib().pbr_autotune_load(self.ctx, os.fsencode(path), C.byref(n)))
        return n.value

    def forward(self, scenes, cams, opts=None, scene_of_view=None, keep_state=True, out=None):
        """Renders every camera; returns (image [sum H W, 3] fp32 on device, State|None)."""
        scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
        opts = opts or default_opts()
        pts = (Points * len(scenes))(*[s.points() for s in scenes])
        cam_arr = make_cameras(cams)
        sov = None
        if scene_of_view is not None:
            sov = (C.c_int32 * len(cams))(*[int(x) for x in scene_of_view])
        npix = n_pixels(cams)
        if out is None:
            out = torch.empty((npix, 3), dtype=torch.float32, device=f"cuda:{self.device}")
        h = C.c_void_p()
        check(lib().pbr_render_forward(self.ctx, pts, len(scenes), sov, cam_arr, len(cams),
                                       C.byref(opts), _ptr(out), C.byref(h) if keep_state else None,
                                       _stream()))
        return out, (State(self, h, scenes) if keep_state else None)

    def workspace_size(self, scenes, cams, opts=None, scene_of_view=None, keep_state=True):
        """(peak device bytes of forward(...) with these arguments, bytes of its
        stored transmittance list) -- pbr_forward_workspace_size."""
        scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
        opts = opts or default_opts()
        pts = (Points * len(scenes))(*[s.points() for s in scenes])
        sov = None
        if scene_of_view is not None:
            sov = (C.c_int32 * len(cams))(*[int(x) for x in scene_of_view])
        b, sb = C.c_size_t(), C.c_size_t()
        check(lib().pbr_forward_workspace_size(self.ctx, pts, len(scenes), sov, make_cameras(cams),
                                               len(cams), C.byref(opts), 1 if keep_state else 0,
                                               C.byref(b), C.byref(sb), _stream()))
        return b.value, sb.value

    def backward(self, state: State, grad_rgb, want_opacity=True, out=None):
        """Gradients (packed over the state's scenes) for dL/dimage = grad_rgb.
        `out` = (grad_pos [n,3], grad_sh [n_sh], grad_opacity [n] or None):
        preallocated fp32 device buffers to overwrite."""
        scenes = state.scenes
        dev = f"cuda:{self.device}"
        n_tot = sum(s.n for s in scenes)
        n_sh = sum(s.n * (s.deg + 1) ** 2 * 3 for s in scenes)
        if out is not None:
            gpos, gsh, gop = out
            assert gpos.shape == (n_tot, 3) and gsh.numel() == n_sh and gpos.is_contiguous() \
                and gsh.is_contiguous() and gpos.dtype == gsh.dtype == torch.float32
            assert gop is None or (gop.numel() == n_tot and gop.is_contiguous()
                                   and gop.dtype == torch.float32)
        else:
            gpos = torch.empty((n_tot, 3), dtype=torch.float32, device=dev)
            gsh = torch.empty((n_sh,), dtype=torch.float32, device=dev)
            gop = (torch.empty((n_tot,), dtype=torch.float32, device=dev) if want_opacity
                   else None)
        g = grad_rgb.to(dtype=torch.float32).contiguous()
        check(lib().pbr_render_backward(self.ctx, state.handle, _ptr(g), _ptr(gpos), _ptr(gsh),
                                        _ptr(gop) if gop is not None else None, _stream()))
        return gpos, gsh, gop


def render_forward_noalloc(scenes, cams, opts=None, scene_of_view=None, out=None):
    """Forward render through pbr_render_forward_noalloc (the library keeps
    all intermediate buffers in a fixed 16 MiB device array and allocates
    nothing; sizes beyond it raise PBRError CAPACITY)."""
    scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
    opts = opts or default_opts()
    pts = (Points * len(scenes))(*[s.points() for s in scenes])
    cam_arr = make_cameras(cams)
    sov = None
    if scene_of_view is not None:
        sov = (C.c_int32 * len(cams))(*[int(x) for x in scene_of_view])
    if out is None:
        out = torch.empty((n_pixels(cams), 3), dtype=torch.float32, device=scenes[0].pos.device)
    check(lib().pbr_render_forward_noalloc(pts, len(scenes), sov, cam_arr, len(cams),
                                           C.byref(opts), _ptr(out), _stream()))
    return out


class Graph:
    """A batch of views captured as CUDA graphs (see pbr_graph_create).

    Phases: FORWARD (0) writes `out`; BACKWARD (1) reads `grad_rgb`; STEP (2)
    runs forward, the image loss against `target` and backward.  Tensors
    passed here are bound to the graph: update them in place."""

    FORWARD, BACKWARD, STEP, TRAIN = 0, 1, 2, 3

    def __init__(self, renderer, scenes, cams, opts=None, scene_of_view=None, target=None,
                 loss="l2", backward=True, grad_rgb=None, headroom=0.25):
        self.renderer = renderer
        self.scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
        self.cams = list(cams)
        self.opts = opts or default_opts()
        dev = self.scenes[0].pos.device
        self.out = torch.empty((n_pixels(cams), 3), dtype=torch.float32, device=dev)
        self.target = target
        self.grad_rgb = grad_rgb
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        n_tot = sum(s.n for s in self.scenes)
        n_sh = sum(s.sh.numel() for s in self.scenes)
        self.grad_pos = self.grad_sh = self.grad_opacity = None
        if backward:
            self.grad_pos = torch.zeros((n_tot, 3), dtype=torch.float32, device=dev)
            self.grad_sh = torch.zeros((n_sh,), dtype=torch.float32, device=dev)
            self.grad_opacity = torch.zeros((n_tot,), dtype=torch.float32, device=dev)
        pts = (Points * len(self.scenes))(*[s.points() for s in self.scenes])
        sov = None
        if scene_of_view is not None:
            sov = (C.c_int32 * len(cams))(*[int(x) for x in scene_of_view])
        self._keep = (pts, sov)
        self.handle = C.c_void_p()
        check(lib().pbr_graph_create(
            renderer.ctx, pts, len(self.scenes), sov, make_cameras(cams), len(cams),
            C.byref(self.opts), _ptr(self.out), _ptr(target), 0 if loss == "l2" else 1,
            _ptr(self.loss), _ptr(grad_rgb), _ptr(self.grad_pos), _ptr(self.grad_sh),
            _ptr(self.grad_opacity), float(headroom), _stream(), C.byref(self.handle)))

    def launch(self, phase=0):
        check(lib().pbr_graph_launch(self.handle, int(phase), _stream()))

    def check(self):
        """(ok, pairs of the last replay, planned capacity); synchronises."""
        n, cap = C.c_int64(), C.c_int64()
        rc = lib().pbr_graph_check(self.handle, _stream(), C.byref(n), C.byref(cap))
        if rc not in (PBR_OK, -4):
            check(rc)
        return rc == PBR_OK, n.value, cap.value

    def replan(self):
        check(lib().pbr_graph_replan(self.handle, _stream()))

    def set_optimizer(self, cfg=None, **kw):
        """Adds the TRAIN phase (forward, Eq. 8 loss, backward, optimiser
        update of the scenes' arrays in place)."""
        cfg = cfg or default_optimizer(**kw)
        check(lib().pbr_graph_set_optimizer(self.handle, C.byref(cfg), _stream()))
        self.opt = cfg

    def set_lr(self, lr_pos, lr_sh, lr_opacity=0.0):
        check(lib().pbr_graph_set_lr(self.handle, float(lr_pos), float(lr_sh), float(lr_opacity)))

    def set_cameras(self, cams):
        check(lib().pbr_graph_set_cameras(self.handle, make_cameras(cams), len(cams), _stream()))

    def close(self):
        if self.handle:
            lib().pbr_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over resident scenes (pbr_serve_*)."""

    def __init__(self, renderer, opts=None, max_batch_views=64, n_streams=2, hbm_budget=None):
        self.renderer = renderer
        self.ctx = renderer.ctx
        if hbm_budget is not None:
            check(lib().pbr_serve_set_budget(self.ctx, int(hbm_budget)))
        check(lib().pbr_serve_start(self.ctx, C.byref(opts or default_opts()),
                                    int(max_batch_views), int(n_streams)))
        self.running = True
        self._outs = {}

    def set_budget(self, nbytes):
        check(lib().pbr_serve_set_budget(self.ctx, int(nbytes)))

    def upload(self, scene) -> int:
        """Copies a Scene (or dict of numpy arrays with 'deg') into library HBM."""
        if not isinstance(scene, Scene):
            keep = [np.ascontiguousarray(scene[k], np.float32)
                    for k in ("pos", "sh", "opacity", "radius")]
            pts = Points(*[C.c_void_p(a.ctypes.data) for a in keep], len(keep[0]),
                         int(scene["deg"]), 0)
        else:
            pts = scene.points()
        sid = C.c_int32()
        check(lib().pbr_upload_scene(self.ctx, C.byref(pts), C.byref(sid)))
        return sid.value

    def evict(self, scene_id):
        check(lib().pbr_evict_scene(self.ctx, int(scene_id)))

    def submit(self, scene_id, cam, out=None, arrival=0.0):
        """Queues a render; returns (request id, output tensor [H*W, 3])."""
        if out is None:
            out = torch.empty((int(cam["width"]) * int(cam["height"]), 3), dtype=torch.float32,
                              device=f"cuda:{self.renderer.device}")
        rid = C.c_uint64()
        check(lib().pbr_submit_request(self.ctx, int(scene_id), make_cameras([cam]), _ptr(out),
                                       float(arrival), C.byref(rid)))
        self._outs[rid.value] = out
        return rid.value, out

    def poll(self, rid):
        done, st = C.c_int32(), C.c_int32()
        check(lib().pbr_poll(self.ctx, C.c_uint64(rid), C.byref(done), C.byref(st)))
        if done.value:
            self._outs.pop(rid, None)
        return bool(done.value), st.value

    def wait(self, rid, timeout_ms=60000):
        st = C.c_int32()
        check(lib().pbr_wait(self.ctx, C.c_uint64(rid), int(timeout_ms), C.byref(st)))
        self._outs.pop(rid, None)
        return st.value

    def stats(self, reset=False) -> dict:
        s = ServeStats()
        check(lib().pbr_serve_stats(self.ctx, C.byref(s), 1 if reset else 0))
        return {k: getattr(s, k) for k, _ in ServeStats._fields_}

    def estimate(self, scene_id, cam):
        """Bytes a request for scene_id from cam reserves from the HBM budget
        (pbr_serve_estimate)."""
        b = C.c_size_t()
        check(lib().pbr_serve_estimate(self.ctx, int(scene_id), make_cameras([cam]),
                                       C.byref(b)))
        return b.value

    def trace(self, reset=False):
        """Device intervals of the completed batches: a list of (start_ms,
        end_ms, views), milliseconds after the loop started."""
        n = C.c_int32()
        check(lib().pbr_serve_trace(self.ctx, None, None, None, 0, C.byref(n), 0))
        m = n.value
        a, b, v = (C.c_double * max(m, 1))(), (C.c_double * max(m, 1))(), (C.c_int32 * max(m, 1))()
        check(lib().pbr_serve_trace(self.ctx, a, b, v, m, C.byref(n), 1 if reset else 0))
        m = min(m, n.value)
        return [(a[i], b[i], v[i]) for i in range(m)]

    def stop(self):
        if self.running:
            check(lib().pbr_serve_stop(self.ctx))
            self.running = False


def now() -> float:
    """The serving loop's clock (seconds), for request arrival times."""
    return float(lib().pbr_now())


N_TUNE_CANDIDATES = 15
TUNE_CANDIDATES = [(t, d, p) for t in ((16, 16), (8, 8), (16, 32))
                   for (d, p) in ((0, 0), (0, 1), (128, 0), (256, 0), (512, 0))]


def autotune(renderer, scenes, cams, opts=None, scene_of_view=None, backward=True, reps=2,
             report=True, info=None):
    """Times every schedule candidate on this batch and returns (best opts,
    {(tile, batch_depth, persistent): ms}).  Without `report` a shape class
    already in the renderer's cache returns its schedule untimed; `info`
    (a dict) receives the number of candidates timed as "n_timed"."""
    scenes = scenes if isinstance(scenes, (list, tuple)) else [scenes]
    opts = opts or default_opts()
    pts = (Points * len(scenes))(*[s.points() for s in scenes])
    sov = None
    if scene_of_view is not None:
        sov = (C.c_int32 * len(cams))(*[int(x) for x in scene_of_view])
    ms = (C.c_double * N_TUNE_CANDIDATES)()
    n = C.c_int32()
    check(lib().pbr_autotune(renderer.ctx, pts, len(scenes), sov, make_cameras(cams), len(cams),
                             C.byref(opts), 1 if backward else 0, int(reps), ms if report else None,
                             C.byref(n), _stream()))
    table = {TUNE_CANDIDATES[i]: ms[i] for i in range(n.value)} if report else {}
    if info is not None:
        info["n_timed"] = n.value
    return opts, table


def default_optimizer(**kw) -> OptimizerCfg:
    c = OptimizerCfg()
    lib().pbr_default_optimizer(C.byref(c))
    for k, v in kw.items():
        if k == "kind":
            v = {"sgd": 0, "adam": 1}.get(v, v)
        if k == "loss_kind":
            v = {"l2": 0, "l1": 1}.get(v, v)
        cur = getattr(c, k)
        setattr(c, k, float(v) if isinstance(cur, float) else int(v))
    return c


def image_loss_tv(pred, target, cams, lam=0.01, kind="l2"):
    """Eq. 8 objective over packed views: (loss, dL/dpred)."""
    grad = torch.empty_like(pred)
    loss = torch.zeros(1, dtype=torch.float64, device=pred.device)
    check(lib().pbr_image_loss_tv(make_cameras(cams), len(cams), _ptr(pred), _ptr(target),
                                  0 if kind == "l2" else 1, float(lam), _ptr(grad), _ptr(loss),
                                  _stream()))
    return loss, grad


def optimizer_step(param, grad, m=None, v=None, lr=1e-3, step=1, kind="adam", beta1=0.9,
                   beta2=0.999, eps=1e-8):
    """In-place SGD / Adam update of a float32 device tensor."""
    k = 1 if kind == "adam" else 0
    check(lib().pbr_optimizer_step(k, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                                   float(lr), float(beta1), float(beta2), float(eps), int(step),
                                   _stream()))


def image_loss(pred, target, kind="l2"):
    """(loss, dL/dpred) of a sum-of-squares (kind l2) or sum-of-abs (l1) loss."""
    grad = torch.empty_like(pred)
    loss = torch.zeros(1, dtype=torch.float64, device=pred.device)
    check(lib().pbr_image_loss(0 if kind == "l2" else 1, _ptr(pred), _ptr(target), pred.numel(),
                               _ptr(grad), _ptr(loss), _stream()))
    return loss, grad


def kernel_launches() -> int:
    return int(lib().pbr_kernel_launches())


def refine_points(renderer, scene, n_vox=256, k=8, eps=0.01, stages=7):
    """One pass of the coarse-to-fine update (Sec. 3.3, Algorithm 1) of a
    Scene.  Returns (Scene of the result, (after reduction, after outlier
    removal, output) point counts)."""
    cfg = RefineCfg()
    lib().pbr_default_refine(C.byref(cfg))
    cfg.n_vox, cfg.k, cfg.eps, cfg.stages = int(n_vox), int(k), float(eps), int(stages)
    cap = max(1, 2 * scene.n)
    K = (scene.deg + 1) ** 2
    dev = scene.pos.device
    pos = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    sh = torch.empty((cap, K, 3), dtype=torch.float32, device=dev)
    op = torch.empty(cap, dtype=torch.float32, device=dev)
    rad = torch.empty(cap, dtype=torch.float32, device=dev)
    counts = (C.c_int64 * 3)()
    pts = scene.points()
    check(lib().pbr_refine_points(renderer.ctx, C.byref(pts), C.byref(cfg), _ptr(pos), _ptr(sh),
                                  _ptr(op), _ptr(rad), cap, counts, _stream()))
    m = int(counts[2])
    out = Scene(pos[:m], sh[:m], op[:m], rad[:m], scene.deg, device=dev)
    return out, (int(counts[0]), int(counts[1]), m)


def knn(renderer, ref, k, query=None, grid_n=0):
    """k nearest points of `ref` ([n,3] fp32 device) for every query point
    (query None: the points of ref themselves, each skipping itself).
    Returns (idx [nq,k] int32, d2 [nq,k] fp32), padded with -1 / FLT_MAX."""
    ref = ref.contiguous()
    q = ref if query is None else query.contiguous()
    nq = int(q.shape[0])
    idx = torch.empty((nq, k), dtype=torch.int32, device=ref.device)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=ref.device)
    check(lib().pbr_knn(renderer.ctx, _ptr(ref), int(ref.shape[0]), _ptr(q), nq, int(k),
                        1 if query is None else 0, int(grid_n), _ptr(idx), _ptr(d2), _stream()))
    return idx, d2


def chamfer(renderer, p1, p2, grad=True):
    """Chamfer distance of Sec. 3.4 between two [n,3] fp32 device clouds.
    Returns (CD as a 0-d fp64 device tensor, dCD/dp2 or None, nn12, nn21)."""
    p1, p2 = p1.contiguous(), p2.contiguous()
    dev = p1.device
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    g = torch.empty_like(p2) if grad else None
    nn12 = torch.empty(p1.shape[0], dtype=torch.int32, device=dev)
    nn21 = torch.empty(p2.shape[0], dtype=torch.int32, device=dev)
    check(lib().pbr_chamfer(renderer.ctx, _ptr(p1), int(p1.shape[0]), _ptr(p2),
                            int(p2.shape[0]), _ptr(loss), _ptr(g), _ptr(nn12), _ptr(nn21),
                            _stream()))
    return loss, g, nn12, nn21


def frame_init(renderer, prev, pos2, iters=100, lr=1e-3, k=4, beta1=0.9, beta2=0.999,
               eps=1e-8):
    """Initialises the next frame from the Scene `prev` (Sec. 3.4): pos2 ([n2,3]
    fp32 device, updated in place) descends on the Chamfer distance, then the
    new points take the mean parameters of their k closest previous points.
    Returns (Scene of the new frame, loss history as a list)."""
    cfg = FrameCfg()
    lib().pbr_default_frame_cfg(C.byref(cfg))
    cfg.iters, cfg.lr, cfg.k = int(iters), float(lr), int(k)
    cfg.beta1, cfg.beta2, cfg.eps = float(beta1), float(beta2), float(eps)
    n2 = int(pos2.shape[0])
    K = (prev.deg + 1) ** 2
    dev = pos2.device
    sh = torch.empty((n2, K, 3), dtype=torch.float32, device=dev)
    op = torch.empty(n2, dtype=torch.float32, device=dev)
    rad = torch.empty(n2, dtype=torch.float32, device=dev)
    hist = (C.c_double * (int(iters) + 1))()
    pts = prev.points()
    check(lib().pbr_frame_init(renderer.ctx, C.byref(pts), _ptr(pos2), n2, C.byref(cfg),
                               _ptr(sh), _ptr(op), _ptr(rad), hist, _stream()))
    return Scene(pos2, sh, op, rad, prev.deg, device=dev), list(hist)


def pack_masks(masks, device="cuda"):
    """[H, W] foreground masks (one per camera, > 0 = foreground) packed into
    one uint8 device array in camera order."""
    flat = [np.ascontiguousarray(np.asarray(m) > 0, np.uint8).ravel() for m in masks]
    return torch.from_numpy(np.concatenate(flat)).to(device)


def consistency_check(renderer, pos, cams, masks, z_near=0.01):
    """CC of every point of pos ([n,3] fp32 device) against packed masks
    (see pack_masks): uint8 [n] device tensor."""
    pos = pos.contiguous()
    keep = torch.empty(pos.shape[0], dtype=torch.uint8, device=pos.device)
    arr = make_cameras(cams)
    check(lib().pbr_consistency_check(renderer.ctx, _ptr(pos), int(pos.shape[0]), arr, len(cams),
                                      _ptr(masks), float(z_near), _ptr(keep), _stream()))
    return keep


def consistency_filter(renderer, scene, cams, masks, z_near=0.01):
    """The points of a Scene that pass the check, as a new Scene."""
    n = scene.n
    K = (scene.deg + 1) ** 2
    dev = scene.pos.device
    pos = torch.empty((max(n, 1), 3), dtype=torch.float32, device=dev)
    sh = torch.empty((max(n, 1), K, 3), dtype=torch.float32, device=dev)
    op = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    rad = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    m = C.c_int64()
    arr = make_cameras(cams)
    pts = scene.points()
    check(lib().pbr_consistency_filter(renderer.ctx, C.byref(pts), arr, len(cams), _ptr(masks),
                                       float(z_near), _ptr(pos), _ptr(sh), _ptr(op), _ptr(rad),
                                       C.byref(m), _stream()))
    k = m.value
    return Scene(pos[:k], sh[:k], op[:k], rad[:k], scene.deg, device=dev)


def visual_hull_init(renderer, lo, hi, cams, masks, n_target, seed=0, sh_degree=2,
                     max_candidates=0, z_near=0.01):
    """Visual-hull initialisation (Sec. 3.1).  Returns (positions [n,3],
    SH [n,K,3] drawn from N(0, 1), candidates drawn)."""
    pos = torch.empty((max(n_target, 1), 3), dtype=torch.float32, device="cuda")
    K = (sh_degree + 1) ** 2
    sh = torch.empty((max(n_target, 1), K, 3), dtype=torch.float32, device="cuda")
    lo3 = (C.c_float * 3)(*[float(v) for v in lo])
    hi3 = (C.c_float * 3)(*[float(v) for v in hi])
    n_out, n_drawn = C.c_int64(), C.c_int64()
    arr = make_cameras(cams)
    check(lib().pbr_visual_hull_init(renderer.ctx, lo3, hi3, arr, len(cams), _ptr(masks),
                                     float(z_near), int(seed) & (2 ** 64 - 1), int(n_target),
                                     int(max_candidates), int(sh_degree), _ptr(pos), _ptr(sh),
                                     C.byref(n_out), C.byref(n_drawn), _stream()))
    k = n_out.value
    return pos[:k], sh[:k], n_drawn.value


def measure_alu_peaks(device: int = 0):
    f, e = C.c_double(), C.c_double()
    check(lib().pbr_measure_alu_peaks(device, C.byref(f), C.byref(e)))
    return f.value, e.value


# ------------------------------------------------------- autograd wrapper
_default_renderer = {}


def renderer(device: int = 0) -> Renderer:
    r = _default_renderer.get(device)
    if r is None:
        r = _default_renderer[device] = Renderer(device)
    return r


if torch is not None:
    class PBRRenderFn(torch.autograd.Function):
        """Differentiable render of one scene through the library's hand-written
        backward pass (positions, SH coefficients, opacity)."""

        @staticmethod
        def forward(ctx, pos, sh, opacity, radius, deg, cams, opts):
            r = renderer(pos.device.index or 0)
            scene = Scene(pos.detach(), sh.detach(), opacity.detach(), radius.detach(), deg,
                          device=pos.device)
            img, st = r.forward([scene], cams, opts)
            ctx.state = st
            ctx.shapes = (pos.shape, sh.shape, opacity.shape)
            return img

        @staticmethod
        def backward(ctx, grad_img):
            st = ctx.state
            r = st.renderer
            gpos, gsh, gop = r.backward(st, grad_img)
            st.close()
            ps, ss, os_ = ctx.shapes
            return gpos.view(ps), gsh.view(ss), gop.view(os_), None, None, None, None

    def render(pos, sh, opacity, radius, deg, cams, opts=None):
        return PBRRenderFn.apply(pos, sh, opacity, radius, deg, cams, opts or default_opts())
