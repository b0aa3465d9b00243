"""Python binding of libdare (DARE: Directionality-Aware Reslicing, CUDA sm_103a).

Argument marshalling only.  Every step of reconstruction and reslicing runs
in libdare.so's CUDA kernels; there is no CPU fallback: if the library is
missing or cannot be built, importing the binding's functions raises.
PyTorch supplies device memory (tensors) and streams.

The raw entry points keep the C names (``dare_reslice``, ...); ``Session``
wraps a session handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))

# ---------------------------------------------------------------- constants (dare.h)
DARE_OK, DARE_E_INVALID, DARE_E_OOM, DARE_E_CUDA = 0, 1, 2, 3
DARE_E_ADMISSION, DARE_E_CAPACITY, DARE_E_TIMEOUT, DARE_E_STATE, DARE_E_UNSUPPORTED = 4, 5, 6, 7, 8
DARE_U8, DARE_F16, DARE_BF16, DARE_F32 = 0, 1, 2, 3
DARE_TENT, DARE_BOX, DARE_EXP = 0, 1, 2
DARE_NORMAL_BEAM, DARE_NORMAL_ELEVATION = 0, 1
DARE_WEIGHTS_F32, DARE_WEIGHTS_F16 = 0, 1
DARE_PATH_AUTO, DARE_PATH_PLAIN, DARE_PATH_TILED, DARE_PATH_TILED_FIXED = 0, 1, 2, 3
DARE_PROBE_LINEAR, DARE_PROBE_CURVILINEAR = 0, 1
DARE_SAMPLE_MEAN, DARE_SAMPLE_PIXELS = 0, 1
DARE_SESSION_SCALAR = 1
DARE_SESSION_L2_PERSIST = 2
DARE_SESSION_HOST_VOLUME = 4
DARE_EMPTY_FRAME = 0xFFFF
DARE_FIX_BITS = 20
DARE_NOALLOC_MAX_FRAMES = 16384

STATUS_NAMES = {0: "OK", 1: "E_INVALID", 2: "E_OOM", 3: "E_CUDA", 4: "E_ADMISSION", 5: "E_CAPACITY",
                6: "E_TIMEOUT", 7: "E_STATE", 8: "E_UNSUPPORTED"}
VALUE_DTYPES = {DARE_U8: np.uint8, DARE_F16: np.float16, DARE_BF16: np.uint16, DARE_F32: np.float32}


class DareError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: DARE_{STATUS_NAMES.get(status, status)}: {message}")


# ---------------------------------------------------------------- structures (dare.h)
_d16 = ctypes.c_double * 16


class dare_grid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32),
                ("spacing_mm", ctypes.c_double), ("vol_to_world", _d16)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class dare_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class dare_session_config(ctypes.Structure):
    _fields_ = [("grid", dare_grid), ("dtype", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("max_frames", ctypes.c_int32), ("device", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("alloc", dare_allocator)]


class dare_probe(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("apex_mm", ctypes.c_double * 2)]


class dare_params(ctypes.Structure):
    _fields_ = [("k_normal", ctypes.c_double), ("k_inplane", ctypes.c_double),
                ("thr_normal_deg", ctypes.c_double), ("thr_inplane_deg", ctypes.c_double),
                ("k_dist", ctypes.c_double), ("unassigned", ctypes.c_float), ("radius_vox", ctypes.c_int32),
                ("dist_kernel", ctypes.c_int32), ("normal_axis", ctypes.c_int32),
                ("weight_dtype", ctypes.c_int32), ("path", ctypes.c_int32), ("probe", dare_probe),
                ("sample_weight", ctypes.c_int32), ("tile_rows", ctypes.c_int32)]


class dare_plane(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("px_mm", ctypes.c_double * 2),
                ("image_to_world", _d16)]


class dare_reslice_req(ctypes.Structure):
    _fields_ = [("session", ctypes.c_void_p), ("plane", dare_plane), ("out", ctypes.c_void_p),
                ("mask", ctypes.c_void_p)]


class dare_session_info(ctypes.Structure):
    _fields_ = [("volume_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("overflow_voxels", ctypes.c_int64), ("version", ctypes.c_int64), ("n_frames", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("dtype", ctypes.c_int32), ("record_bytes", ctypes.c_int32),
                ("dims", ctypes.c_int32 * 3), ("flags", ctypes.c_int32), ("spacing_mm", ctypes.c_double),
                ("vol_to_world", _d16)]


class dare_plan_info(ctypes.Structure):
    _fields_ = [("n_requests", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("choice", ctypes.c_int32 * 8),
                ("tune_ms", (ctypes.c_float * 4) * 8), ("workspace_bytes", ctypes.c_int64)]


class dare_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("coalesce_us", ctypes.c_int32), ("params", dare_params), ("max_frames", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class dare_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("done_s", ctypes.c_double), ("issue_s", ctypes.c_double),
                ("batch", ctypes.c_int32), ("lane", ctypes.c_int32)]


class dare_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("ingests", ctypes.c_int64), ("max_batch_seen", ctypes.c_int64), ("lanes", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class dare_trace_counters(ctypes.Structure):
    _fields_ = [("tiled_planes", ctypes.c_int64), ("per_pixel_planes", ctypes.c_int64),
                ("fallback_tiles", ctypes.c_int64)]


class dare_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


# ---------------------------------------------------------------- library
_LIB = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p

_SIGNATURES = {
    "dare_last_error": ([], ctypes.c_char_p),
    "dare_abi_version": ([], ctypes.c_int32),
    "dare_params_default": ([_P(dare_params)], ctypes.c_int),
    "dare_grid_from_frames": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_double),
                               _P(ctypes.c_double), ctypes.c_double, ctypes.c_int32, _P(dare_grid)], ctypes.c_int),
    "dare_pixel_affine": ([_P(dare_grid), _P(dare_plane), _P(ctypes.c_int64)], ctypes.c_int),
    "dare_session_create": ([_P(dare_session_config), _P(_vp)], ctypes.c_int),
    "dare_session_destroy": ([_vp], ctypes.c_int),
    "dare_session_sync": ([_vp], ctypes.c_int),
    "dare_session_query": ([_vp, _P(dare_session_info)], ctypes.c_int),
    "dare_session_read_records": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "dare_session_read_frames": ([_vp, _P(ctypes.c_double)], ctypes.c_int),
    "dare_session_set_probe": ([_vp, _P(dare_probe), _vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "dare_fill_holes": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp], ctypes.c_int),
    "dare_session_set_cache": ([_vp, ctypes.c_int64], ctypes.c_int),
    "dare_session_cache_stats": ([_vp, _P(ctypes.c_int64)], ctypes.c_int),
    "dare_reslice_scalar_filled": ([_vp, _P(dare_plane), ctypes.c_float, _vp, _vp, _vp], ctypes.c_int),
    "dare_session_read_filled": ([_vp, _vp], ctypes.c_int),
    "dare_session_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "dare_session_load": ([_P(dare_session_config), ctypes.c_char_p, _P(_vp)], ctypes.c_int),
    "dare_build_volume": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_double),
                           _P(ctypes.c_double), _vp], ctypes.c_int),
    "dare_reslice": ([_vp, _P(dare_plane), _P(dare_params), _vp, _vp, _vp], ctypes.c_int),
    "dare_reslice_batch": ([_P(dare_reslice_req), ctypes.c_int32, _P(dare_params), _vp], ctypes.c_int),
    "dare_build_volume_host": ([_vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_double),
                                _P(ctypes.c_double), ctypes.c_int32, _vp], ctypes.c_int),
    "dare_reslice_batch_host": ([_P(dare_reslice_req), ctypes.c_int32, _P(dare_params), ctypes.c_int32, _vp],
                                ctypes.c_int),
    "dare_reslice_noalloc": ([_vp, _P(dare_plane), _P(dare_params), _vp, _vp, _vp], ctypes.c_int),
    "dare_plan_create": ([_P(dare_reslice_req), ctypes.c_int32, _P(dare_params), _vp, _P(_vp)], ctypes.c_int),
    "dare_plan_set_poses": ([_vp, _P(ctypes.c_double)], ctypes.c_int),
    "dare_plan_launch": ([_vp, _vp], ctypes.c_int),
    "dare_plan_query": ([_vp, _P(dare_plan_info)], ctypes.c_int),
    "dare_plan_destroy": ([_vp], ctypes.c_int),
    "dare_reslice_scalar": ([_vp, _P(dare_plane), ctypes.c_float, _vp, _vp, _vp], ctypes.c_int),
    "dare_footprint": ([_vp, _P(dare_plane), ctypes.c_int32, _P(ctypes.c_int64), _vp], ctypes.c_int),
    "dare_session_reset": ([_vp, _vp], ctypes.c_int),
    "dare_trace_enable": ([ctypes.c_int32], ctypes.c_int),
    "dare_trace_read": ([_P(dare_kernel_time), ctypes.c_int32, _P(ctypes.c_int32)], ctypes.c_int),
    "dare_launch_count": ([], ctypes.c_int64),
    "dare_trace_counters_read": ([_P(dare_trace_counters), ctypes.c_int32], ctypes.c_int),
    "dare_tune_cache_file": ([ctypes.c_char_p], ctypes.c_int),
    "dare_measure_l2_bandwidth": ([ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P(ctypes.c_double)],
                                  ctypes.c_int),
    "dare_clock_seconds": ([], ctypes.c_double),
    "dare_server_create": ([_P(dare_server_config), _P(_vp)], ctypes.c_int),
    "dare_server_submit": ([_vp, _P(dare_reslice_req), ctypes.c_uint64], ctypes.c_int),
    "dare_server_ingest": ([_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_double),
                            _P(ctypes.c_double), ctypes.c_uint64], ctypes.c_int),
    "dare_server_poll": ([_vp, _P(dare_completion), ctypes.c_int32, _P(ctypes.c_int32)], ctypes.c_int),
    "dare_server_drain": ([_vp, ctypes.c_double], ctypes.c_int),
    "dare_server_stats_get": ([_vp, _P(dare_server_stats)], ctypes.c_int),
    "dare_server_destroy": ([_vp], ctypes.c_int),
    "dare_set_memory_budget": ([ctypes.c_int64], ctypes.c_int),
    "dare_memory_in_use": ([], ctypes.c_int64),
}


def library_path():
    return os.path.join(_PKG, "libdare.so")


def lib():
    """Load libdare.so (building it first if the sources are newer).  Raises if
    the library cannot be built or loaded: there is no fallback path."""
    global _LIB
    if _LIB is None:
        from . import _build
        path = _build.build()
        handle = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = handle
    return _LIB


def last_error():
    return lib().dare_last_error().decode(errors="replace")


def check(status, where):
    if status != DARE_OK:
        raise DareError(status, where, last_error())


def __getattr__(name):
    # raw C entry points under their own names: paper_2605_26325_b300.dare_reslice(...)
    if name in _SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


# ---------------------------------------------------------------- marshalling helpers

def _mat16(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return _d16(*a)


def make_grid(dims, spacing_mm, vol_to_world) -> dare_grid:
    g = dare_grid()
    g.dims[:] = [int(x) for x in dims]
    g.spacing_mm = float(spacing_mm)
    g.vol_to_world = _mat16(vol_to_world)
    return g


def fill_plane(p, width, height, px_mm, image_to_world):
    """Write a plane's size, spacing and pose into an existing dare_plane."""
    T = np.ascontiguousarray(image_to_world, dtype=np.float64)
    if T.size != 16:
        raise ValueError("image_to_world must hold 16 values")
    p.width, p.height = int(width), int(height)
    p.px_mm[0], p.px_mm[1] = float(px_mm[0]), float(px_mm[1])
    ctypes.memmove(ctypes.addressof(p.image_to_world), T.ctypes.data, 128)
    return p


def make_plane(width, height, px_mm, image_to_world) -> dare_plane:
    return fill_plane(dare_plane(), width, height, px_mm, image_to_world)


def make_probe(kind=DARE_PROBE_LINEAR, apex_mm=(0.0, 0.0)) -> dare_probe:
    pr = dare_probe()
    pr.kind = int(kind)
    pr.apex_mm[0], pr.apex_mm[1] = float(apex_mm[0]), float(apex_mm[1])
    return pr


def params_default(probe_apex_mm=None, **overrides) -> dare_params:
    """The paper's parameters with overrides by field name; probe_apex_mm=(x, y)
    makes the virtual probe curvilinear with that fan apex (image mm)."""
    p = dare_params()
    check(lib().dare_params_default(ctypes.byref(p)), "dare_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    if probe_apex_mm is not None:
        p.probe = make_probe(DARE_PROBE_CURVILINEAR, probe_apex_mm)
    return p


def pixel_affine(dims, spacing_mm, vol_to_world, width, height, px_mm, image_to_world):
    g = make_grid(dims, spacing_mm, vol_to_world)
    pl = make_plane(width, height, px_mm, image_to_world)
    out = (ctypes.c_int64 * 9)()
    check(lib().dare_pixel_affine(ctypes.byref(g), ctypes.byref(pl), out), "dare_pixel_affine")
    return np.array(out[:], dtype=np.int64)


def grid_from_frames(poses, width, height, px_mm, spacing_mm, margin_vox=1):
    poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 16))
    px = (ctypes.c_double * 2)(float(px_mm[0]), float(px_mm[1]))
    g = dare_grid()
    check(lib().dare_grid_from_frames(poses.shape[0], int(width), int(height), px,
                                      poses.ctypes.data_as(_P(ctypes.c_double)), float(spacing_mm),
                                      int(margin_vox), ctypes.byref(g)), "dare_grid_from_frames")
    T = np.array(g.vol_to_world[:]).reshape(4, 4)
    return tuple(g.dims[:]), g.spacing_mm, T


def mask_words(width):
    return (int(width) + 31) // 32


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _host_ptr(t, name, shape=None):
    """Host buffer (numpy array or CPU torch tensor, contiguous) -> pointer."""
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be contiguous")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return ctypes.c_void_p(t.ctypes.data)
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"expected a host array or CPU tensor for {name}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _dev_shape2(t, name):
    """(rows, columns) of a contiguous 2-D float32 CUDA tensor."""
    import torch
    if type(t) is not torch.Tensor or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or \
            t.dtype is not torch.float32:
        raise TypeError(f"{name} must be a contiguous 2-D float32 CUDA tensor")
    return t.shape


def _dev_addr(t, name, shape):
    """Device address of a contiguous 32-bit CUDA tensor of the given shape, as an int."""
    import torch
    if type(t) is not torch.Tensor or not t.is_cuda or not t.is_contiguous() or t.element_size() != 4:
        raise TypeError(f"{name} must be a contiguous CUDA tensor of 32-bit words")
    if t.shape != shape:
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _stream_addr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _dev_ptr(t, dtype_name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"expected a CUDA tensor for {dtype_name}")
    if not t.is_contiguous():
        raise ValueError(f"{dtype_name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{dtype_name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def trace_enable(on=True):
    check(lib().dare_trace_enable(1 if on else 0), "dare_trace_enable")


def trace_read():
    """{kernel name: (launches, total device ms)} since the last read; waits for the events."""
    cap = 64
    arr = (dare_kernel_time * cap)()
    n = ctypes.c_int32()
    check(lib().dare_trace_read(arr, cap, ctypes.byref(n)), "dare_trace_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, cap))}


def launch_count():
    return int(lib().dare_launch_count())


def trace_counters(reset=False):
    """{tiled_planes, per_pixel_planes, fallback_tiles} (dare_trace_counters_read)."""
    c = dare_trace_counters()
    check(lib().dare_trace_counters_read(ctypes.byref(c), 1 if reset else 0), "dare_trace_counters_read")
    return {k: int(getattr(c, k)) for k, _ in c._fields_}


def measure_l2_bandwidth(device=0, nbytes=32 << 20, reps=200):
    """L2-to-SM read bandwidth of the device in GB/s (dare_measure_l2_bandwidth)."""
    g = ctypes.c_double()
    check(lib().dare_measure_l2_bandwidth(int(device), int(nbytes), int(reps), ctypes.byref(g)),
          "dare_measure_l2_bandwidth")
    return float(g.value)


def tune_cache_file(path):
    """Plan tuning choices read from and written to this JSON file (None: no file)."""
    check(lib().dare_tune_cache_file(None if path is None else os.fsencode(path)), "dare_tune_cache_file")


def set_memory_budget(nbytes):
    check(lib().dare_set_memory_budget(int(nbytes)), "dare_set_memory_budget")


def memory_in_use():
    return int(lib().dare_memory_in_use())


class Session:
    """A directional volume on one device (Sec. 2.1, Fig. 1) and its reslicing."""

    def __init__(self, dims, spacing_mm, vol_to_world, dtype=DARE_F32, max_slots=8, max_frames=65535,
                 device=0, flags=0, allocator=None, _handle=None):
        self._cfg = dare_session_config()
        self._cfg.grid = make_grid(dims, spacing_mm, vol_to_world)
        self._cfg.dtype = int(dtype)
        self._cfg.max_slots = int(max_slots)
        self._cfg.max_frames = int(max_frames)
        self._cfg.device = int(device)
        self._cfg.flags = int(flags)
        self._alloc_keep = None
        if allocator is not None:
            self._alloc_keep = allocator
            self._cfg.alloc = allocator.as_struct()
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            check(lib().dare_session_create(ctypes.byref(self._cfg), ctypes.byref(self._h)), "dare_session_create")
        self.dims = tuple(int(x) for x in dims)
        self.spacing_mm = float(spacing_mm)
        self.vol_to_world = np.array(vol_to_world, dtype=np.float64).reshape(4, 4)
        self.device = int(device)

    @classmethod
    def load(cls, path, device=0, flags=0, allocator=None):
        cfg = dare_session_config()
        cfg.device = int(device)
        cfg.flags = int(flags)
        if allocator is not None:
            cfg.alloc = allocator.as_struct()
        h = ctypes.c_void_p()
        check(lib().dare_session_load(ctypes.byref(cfg), str(path).encode(), ctypes.byref(h)), "dare_session_load")
        info = dare_session_info()
        check(lib().dare_session_query(h, ctypes.byref(info)), "dare_session_query")
        obj = cls.__new__(cls)
        obj._cfg = cfg
        obj._alloc_keep = allocator
        obj._h = h
        obj.dims = tuple(info.dims[:])
        obj.spacing_mm = float(info.spacing_mm)
        obj.vol_to_world = np.array(info.vol_to_world[:], dtype=np.float64).reshape(4, 4)
        obj.device = int(device)
        return obj

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(lib().dare_session_destroy(self._h), "dare_session_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if getattr(self, "_h", None) and self._h.value and _LIB is not None:
                _LIB.dare_session_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- state
    def info(self) -> dare_session_info:
        info = dare_session_info()
        check(lib().dare_session_query(self._h, ctypes.byref(info)), "dare_session_query")
        return info

    def sync(self):
        check(lib().dare_session_sync(self._h), "dare_session_sync")

    def reset(self, stream=None):
        check(lib().dare_session_reset(self._h, _stream_ptr(stream)), "dare_session_reset")

    def set_probe(self, kind=DARE_PROBE_LINEAR, apex_mm=(0.0, 0.0), pixel_mask=None):
        """Probe of the frames built from now on: DARE_PROBE_CURVILINEAR fans the
        beams from apex_mm (image x, y in mm); pixel_mask (H, W), zero bytes
        excluded from voxelisation (e.g. outside the fan)."""
        pr = make_probe(kind, apex_mm)
        if pixel_mask is None:
            check(lib().dare_session_set_probe(self._h, ctypes.byref(pr), None, 0, 0), "dare_session_set_probe")
            return
        m = np.ascontiguousarray(np.asarray(pixel_mask, dtype=np.uint8))
        if m.ndim != 2:
            raise ValueError("pixel_mask must be (H, W)")
        check(lib().dare_session_set_probe(self._h, ctypes.byref(pr), m.ctypes.data_as(ctypes.c_void_p),
                                           m.shape[1], m.shape[0]), "dare_session_set_probe")

    def read_records(self, npix=False, scalar=False):
        """Host copies of the volume: dict(frame_ids (n_vox, K) uint16, values (n_vox, K),
        npix (n_vox, K) uint16, scalar_sum, scalar_count)."""
        info = self.info()
        nv = int(np.prod(info.dims[:]))
        K = info.slots
        ids = np.empty((nv, K), np.uint16)
        vals = np.empty((nv, K), VALUE_DTYPES[info.dtype])
        np_ = np.empty((nv, K), np.uint16) if npix else None
        ss = np.empty(nv, np.uint32) if scalar else None
        sc = np.empty(nv, np.uint32) if scalar else None
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        check(lib().dare_session_read_records(self._h, c(ids), c(vals), c(np_), c(ss), c(sc)),
              "dare_session_read_records")
        return dict(frame_ids=ids, values=vals, npix=np_, scalar_sum=ss, scalar_count=sc)

    def read_frames(self):
        n = self.info().n_frames
        out = np.zeros((n, 9), np.float64)
        check(lib().dare_session_read_frames(self._h, out.ctypes.data_as(_P(ctypes.c_double))),
              "dare_session_read_frames")
        return out.reshape(n, 3, 3)

    def save(self, path):
        check(lib().dare_session_save(self._h, str(path).encode()), "dare_session_save")

    # ---- reconstruction
    def build(self, frames_dev, poses, px_mm, stream=None):
        """Append frames (device uint8 tensor (n, H, W)) with host poses (n, 4, 4)."""
        n, H, W = (int(x) for x in frames_dev.shape)
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(n, 16))
        px = (ctypes.c_double * 2)(float(px_mm[0]), float(px_mm[1]))
        import torch
        if frames_dev.dtype != torch.uint8:
            raise TypeError("frames must be uint8")
        check(lib().dare_build_volume(self._h, _dev_ptr(frames_dev, "frames"), n, W, H, px,
                                      poses.ctypes.data_as(_P(ctypes.c_double)), _stream_ptr(stream)),
              "dare_build_volume")

    def build_host(self, frames_host, poses, px_mm, stream=None, slice_frames=0):
        """Append frames held in host memory (uint8 (n, H, W) numpy array or CPU
        tensor; page-locked memory lets the uploads overlap the scatter)."""
        n, H, W = (int(x) for x in frames_host.shape)
        if str(frames_host.dtype) not in ("uint8", "torch.uint8"):
            raise TypeError("frames must be uint8")
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(n, 16))
        px = (ctypes.c_double * 2)(float(px_mm[0]), float(px_mm[1]))
        check(lib().dare_build_volume_host(self._h, _host_ptr(frames_host, "frames"), n, W, H, px,
                                           poses.ctypes.data_as(_P(ctypes.c_double)), int(slice_frames),
                                           _stream_ptr(stream)), "dare_build_volume_host")

    # ---- reslicing
    def reslice(self, image_to_world, out, mask, px_mm, params=None, stream=None):
        """Reslice one plane into out (H, W) float32 and mask (H, ceil(W/32)) int32 device tensors."""
        fast = self.__dict__.get("_fast")
        if fast is None:
            # one plane struct per session, reused (a session is driven by one thread
            # at a time), with a numpy view of its pose for a cheap copy
            pl = dare_plane()
            fast = self._fast = (pl, ctypes.byref(pl), np.ctypeslib.as_array(pl.image_to_world), lib().dare_reslice)
        pl, pl_ref, pose, fn = fast
        H, W = _dev_shape2(out, "out")
        pose[:] = np.asarray(image_to_world, dtype=np.float64).reshape(16)
        pl.width, pl.height = W, H
        pl.px_mm[0], pl.px_mm[1] = px_mm[0], px_mm[1]
        p = params if params is not None else params_default()
        rc = fn(self._h, pl_ref, ctypes.byref(p), out.data_ptr(), _dev_addr(mask, "mask", (H, (W + 31) >> 5)),
                _stream_addr(stream))
        if rc != DARE_OK:
            raise DareError(rc, "dare_reslice", last_error())

    def reslice_scalar(self, image_to_world, out, mask, px_mm, unassigned=0.0, stream=None):
        H, W = (int(x) for x in out.shape)
        pl = make_plane(W, H, px_mm, image_to_world)
        check(lib().dare_reslice_scalar(self._h, ctypes.byref(pl), float(unassigned), _dev_ptr(out, "out"),
                                        _dev_ptr(mask, "mask", (H, mask_words(W))), _stream_ptr(stream)),
              "dare_reslice_scalar")

    def set_cache(self, nbytes):
        """Brick cache of a host-volume session (0 frees it)."""
        check(lib().dare_session_set_cache(self._h, int(nbytes)), "dare_session_set_cache")

    def cache_stats(self):
        """dict(slots, resident, paged_in, hits) of the brick cache."""
        out = (ctypes.c_int64 * 4)()
        check(lib().dare_session_cache_stats(self._h, out), "dare_session_cache_stats")
        return dict(slots=out[0], resident=out[1], paged_in=out[2], hits=out[3])

    def fill_holes(self, radius_vox=1, min_neighbours=1, stream=None):
        """Hole filling of the compounded volume (the comparator's, Sec. 2.2)."""
        check(lib().dare_fill_holes(self._h, int(radius_vox), int(min_neighbours), _stream_ptr(stream)),
              "dare_fill_holes")

    def reslice_scalar_filled(self, image_to_world, out, mask, px_mm, unassigned=0.0, stream=None):
        H, W = (int(x) for x in out.shape)
        pl = make_plane(W, H, px_mm, image_to_world)
        check(lib().dare_reslice_scalar_filled(self._h, ctypes.byref(pl), float(unassigned), _dev_ptr(out, "out"),
                                               _dev_ptr(mask, "mask", (H, mask_words(W))), _stream_ptr(stream)),
              "dare_reslice_scalar_filled")

    def read_filled(self):
        """Host copy of the hole-filled volume, flat (x fastest), NaN = empty."""
        out = np.empty(int(np.prod(self.info().dims[:])), np.float32)
        check(lib().dare_session_read_filled(self._h, out.ctypes.data_as(ctypes.c_void_p)), "dare_session_read_filled")
        return out

    def footprint(self, poses, width, height, px_mm, stream=None):
        poses = np.asarray(poses, dtype=np.float64).reshape(-1, 4, 4)
        n = poses.shape[0]
        planes = (dare_plane * n)(*[make_plane(width, height, px_mm, T) for T in poses])
        counts = (ctypes.c_int64 * n)()
        check(lib().dare_footprint(self._h, planes, n, counts, _stream_ptr(stream)), "dare_footprint")
        return np.array(counts[:], dtype=np.int64)


def make_requests(items, host=False):
    """items: iterable of (session, image_to_world, out, mask, px_mm) -> ctypes array of dare_reslice_req.
    host: out / mask are host buffers (for reslice_batch_host), else CUDA tensors."""
    items = list(items)
    arr = (dare_reslice_req * len(items))()
    ptr = _host_ptr if host else _dev_ptr
    for i, (s, T, out, mask, px) in enumerate(items):
        H, W = (int(x) for x in out.shape)
        arr[i].session = s.handle.value
        arr[i].plane = make_plane(W, H, px, T)
        arr[i].out = ptr(out, "out").value
        arr[i].mask = ptr(mask, "mask", (H, mask_words(W))).value
    return arr


def reslice_batch(requests, params=None, stream=None):
    """requests: ctypes array from make_requests (or the items list)."""
    if not isinstance(requests, ctypes.Array):
        requests = make_requests(requests)
    p = params if params is not None else params_default()
    check(lib().dare_reslice_batch(requests, len(requests), ctypes.byref(p), _stream_ptr(stream)),
          "dare_reslice_batch")


def reslice_batch_host(requests, params=None, stream=None, group_planes=0):
    """Like reslice_batch, with host outputs: requests from make_requests(..., host=True)."""
    if not isinstance(requests, ctypes.Array):
        requests = make_requests(requests, host=True)
    p = params if params is not None else params_default()
    check(lib().dare_reslice_batch_host(requests, len(requests), ctypes.byref(p), int(group_planes),
                                        _stream_ptr(stream)), "dare_reslice_batch_host")


class Plan:
    """A fixed request set replayed through a CUDA graph (dare_plan_*)."""

    def __init__(self, requests, params=None, stream=None):
        if not isinstance(requests, ctypes.Array):
            requests = make_requests(requests)
        self._reqs = requests  # keeps the descriptors alive
        self.n = len(requests)
        p = params if params is not None else params_default()
        self._h = ctypes.c_void_p()
        check(lib().dare_plan_create(requests, self.n, ctypes.byref(p), _stream_ptr(stream), ctypes.byref(self._h)),
              "dare_plan_create")

    def set_poses(self, poses):
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(self.n, 16))
        check(lib().dare_plan_set_poses(self._h, poses.ctypes.data_as(_P(ctypes.c_double))), "dare_plan_set_poses")

    def launch(self, stream=None):
        check(lib().dare_plan_launch(self._h, _stream_ptr(stream)), "dare_plan_launch")

    def info(self):
        i = dare_plan_info()
        check(lib().dare_plan_query(self._h, ctypes.byref(i)), "dare_plan_query")
        return {"n_requests": i.n_requests, "n_groups": i.n_groups, "choice": list(i.choice[:i.n_groups]),
                "tune_ms": [list(i.tune_ms[g]) for g in range(i.n_groups)], "workspace_bytes": i.workspace_bytes}

    def close(self):
        if self._h and self._h.value:
            check(lib().dare_plan_destroy(self._h), "dare_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h and self._h.value and _LIB is not None:
                _LIB.dare_plan_destroy(self._h)
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop (dare_server_*)."""

    def __init__(self, device=0, lanes=2, max_batch=64, params=None, coalesce_us=0, max_frames=0):
        c = dare_server_config()
        c.device, c.lanes, c.max_batch = int(device), int(lanes), int(max_batch)
        c.coalesce_us, c.max_frames = int(coalesce_us), int(max_frames)
        c.params = params if params is not None else params_default()
        self._h = ctypes.c_void_p()
        check(lib().dare_server_create(ctypes.byref(c), ctypes.byref(self._h)), "dare_server_create")
        self._req = dare_reslice_req()
        self._keep = {}

    def submit(self, session, image_to_world, out, mask, px_mm, tag):
        H, W = (int(x) for x in out.shape)
        r = self._req
        r.session = session.handle.value
        r.plane = make_plane(W, H, px_mm, image_to_world)
        r.out = out.data_ptr()
        r.mask = mask.data_ptr()
        check(lib().dare_server_submit(self._h, ctypes.byref(r), ctypes.c_uint64(tag)), "dare_server_submit")

    def ingest(self, session, frames_dev, poses, px_mm, tag):
        n, H, W = (int(x) for x in frames_dev.shape)
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(n, 16))
        px = (ctypes.c_double * 2)(float(px_mm[0]), float(px_mm[1]))
        self._keep[tag] = frames_dev  # valid until its completion is polled
        check(lib().dare_server_ingest(self._h, session.handle, ctypes.c_void_p(frames_dev.data_ptr()), n, W, H, px,
                                       poses.ctypes.data_as(_P(ctypes.c_double)), ctypes.c_uint64(tag)),
              "dare_server_ingest")

    def poll(self, capacity=4096):
        arr = (dare_completion * capacity)()
        n = ctypes.c_int32()
        check(lib().dare_server_poll(self._h, arr, capacity, ctypes.byref(n)), "dare_server_poll")
        out = [(arr[i].tag, arr[i].status, arr[i].kind, arr[i].submit_s, arr[i].done_s, arr[i].issue_s,
                arr[i].batch, arr[i].lane) for i in range(n.value)]
        for t, _, kind, *_ in out:
            if kind == 1:
                self._keep.pop(t, None)
        return out

    def drain(self, timeout_s=60.0):
        check(lib().dare_server_drain(self._h, float(timeout_s)), "dare_server_drain")

    def stats(self):
        st = dare_server_stats()
        check(lib().dare_server_stats_get(self._h, ctypes.byref(st)), "dare_server_stats_get")
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}

    def close(self):
        if self._h and self._h.value:
            check(lib().dare_server_destroy(self._h), "dare_server_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h and self._h.value and _LIB is not None:
                _LIB.dare_server_destroy(self._h)
        except Exception:
            pass


def clock_seconds():
    return float(lib().dare_clock_seconds())


def unpack_mask(mask_words_np, width):
    """(H, ceil(W/32)) int32/uint32 words -> (H, W) uint8 coverage bits."""
    m = np.ascontiguousarray(mask_words_np).view(np.uint32)
    bits = ((m[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1).astype(np.uint8)
    return bits.reshape(m.shape[0], -1)[:, :width]


class TorchAllocator:
    """Routes a session's device allocations through PyTorch's caching allocator."""

    def __init__(self, device=0):
        import torch
        self._torch = torch
        self.device = device
        self.live = {}
        self.fail_next = 0  # test hook: make the next N allocations fail

        def _alloc(nbytes, stream, ctx):
            if self.fail_next > 0:
                self.fail_next -= 1
                return None
            t = self._torch.empty(int(nbytes) + 256, dtype=self._torch.uint8, device=f"cuda:{self.device}")
            p = (t.data_ptr() + 255) // 256 * 256
            self.live[p] = t
            return p

        def _free(ptr, nbytes, stream, ctx):
            self.live.pop(ptr, None)

        self._alloc_fn = _ALLOC_FN(_alloc)
        self._free_fn = _FREE_FN(_free)

    def as_struct(self):
        a = dare_allocator()
        a.alloc = self._alloc_fn
        a.free = self._free_fn
        a.ctx = None
        return a
