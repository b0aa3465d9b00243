"""DARE CPU oracle (FP64) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``dare_oracle.c``; this file
only marshals numpy arrays.

Every function restates a step of the paper (Sec. 2.1): ``build`` is the
volume reconstruction (Fig. 1), ``reslice``/``reslice_pixels`` the reslicing
with Eq. 1 and Eq. 2 (Fig. 2), ``reslice_scalar`` the mean-compounding
comparator (the scalar reading of the PLUS baseline, Sec. 2.2), and
``footprint`` the count of voxel records one reslice must read.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

U8, F16, BF16, F32 = 0, 1, 2, 3
TENT, BOX, EXP = 0, 1, 2
BEAM, ELEVATION = 0, 1
LINEAR, CURVILINEAR = 0, 1

_LIB = None


class _Params(ctypes.Structure):
    _fields_ = [("k_normal", ctypes.c_double), ("k_inplane", ctypes.c_double),
                ("thr_normal_deg", ctypes.c_double), ("thr_inplane_deg", ctypes.c_double),
                ("k_dist", ctypes.c_double), ("unassigned", ctypes.c_double),
                ("radius", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("normal_axis", ctypes.c_int32), ("use_exact", ctypes.c_int32),
                ("probe", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("apex_x", ctypes.c_double), ("apex_y", ctypes.c_double),
                ("sample_weight", ctypes.c_int32), ("pad2", ctypes.c_int32)]


@dataclass
class Params:
    """Reslicing parameters; defaults are the paper's (Sec. 2.1: k_normal 10,
    k_inplane 5, thresholds 25 and 15 degrees) with radius 1 voxel.  probe
    CURVILINEAR makes the virtual plane a fan of beams from apex_mm (image
    point, mm)."""
    k_normal: float = 10.0
    k_inplane: float = 5.0
    thr_normal_deg: float = 25.0
    thr_inplane_deg: float = 15.0
    k_dist: float = 1.0
    unassigned: float = 0.0
    radius: int = 1
    kernel: int = TENT
    normal_axis: int = BEAM
    use_exact: bool = False
    probe: int = LINEAR
    apex_mm: tuple = (0.0, 0.0)
    per_pixel: bool = False   # every pixel its own sample: merged samples weighted by npix

    def _c(self):
        return _Params(self.k_normal, self.k_inplane, self.thr_normal_deg, self.thr_inplane_deg,
                       self.k_dist, self.unassigned, int(self.radius), int(self.kernel),
                       int(self.normal_axis), int(bool(self.use_exact)), int(self.probe), 0,
                       float(self.apex_mm[0]), float(self.apex_mm[1]), int(bool(self.per_pixel)), 0)


def _P(t):
    return ctypes.POINTER(t)


def _lib():
    global _LIB
    if _LIB is None:
        from . import _build
        # a test may point the oracle at a deliberately broken build to check that the pins catch it
        override = os.environ.get("DARE_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else _build.build())
        i32p, i64p, dp, u8p = _P(ctypes.c_int32), _P(ctypes.c_int64), _P(ctypes.c_double), _P(ctypes.c_uint8)
        vp = ctypes.c_void_p
        lib.ora_pixel_affine.argtypes = [dp, ctypes.c_double, dp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, i64p]
        lib.ora_pixel_affine.restype = ctypes.c_int
        lib.ora_build.argtypes = [i32p, ctypes.c_double, dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_double, u8p, dp, ctypes.c_int32, ctypes.c_int32, u8p]
        lib.ora_build.restype = vp
        lib.ora_build_probe.argtypes = lib.ora_build.argtypes + [i32p, dp, u8p]
        lib.ora_build_probe.restype = vp
        lib.ora_volume_manual.argtypes = [i32p, ctypes.c_double, dp, ctypes.c_int64, i64p, i32p, dp, dp]
        lib.ora_volume_manual.restype = vp
        lib.ora_volume_free.argtypes = [vp]
        lib.ora_volume_free.restype = None
        for f in ("ora_volume_nsamples", "ora_volume_noverflow", "ora_volume_ndropped"):
            getattr(lib, f).argtypes = [vp]
            getattr(lib, f).restype = ctypes.c_int64
        lib.ora_volume_export.argtypes = [vp, i64p, i32p, i64p, i64p, dp, dp, dp, i64p, i64p]
        lib.ora_volume_export.restype = None
        lib.ora_reslice.argtypes = [vp, dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    _P(_Params), dp, u8p]
        lib.ora_reslice.restype = ctypes.c_int
        lib.ora_reslice_pixels.argtypes = [vp, dp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           _P(_Params), ctypes.c_int64, i32p, dp, u8p]
        lib.ora_reslice_pixels.restype = ctypes.c_int
        lib.ora_reslice_scalar.argtypes = [vp, dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp, u8p]
        lib.ora_reslice_scalar.restype = ctypes.c_int
        lib.ora_compounded.argtypes = [vp, dp]
        lib.ora_compounded.restype = None
        lib.ora_fill_holes.argtypes = [vp, dp, ctypes.c_int32, ctypes.c_int32, dp]
        lib.ora_fill_holes.restype = None
        lib.ora_reslice_values.argtypes = [i32p, ctypes.c_double, dp, dp, dp, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, u8p]
        lib.ora_reslice_values.restype = ctypes.c_int
        lib.ora_footprint.argtypes = [i32p, ctypes.c_double, dp, dp, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
        lib.ora_footprint.restype = ctypes.c_int64
        lib.ora_round_stored.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        lib.ora_round_stored.restype = ctypes.c_double
        _LIB = lib
    return _LIB


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a, t):
    return a.ctypes.data_as(_P(t))


def pixel_affine(vol_to_world, spacing, image_to_world, width, px_mm):
    """Quantised pixel->voxel affine [G0, A, B] in units of 2^-20 voxel."""
    V = _arr(vol_to_world, np.float64).reshape(16)
    T = _arr(image_to_world, np.float64).reshape(16)
    out = np.zeros(9, dtype=np.int64)
    rc = _lib().ora_pixel_affine(_ptr(V, ctypes.c_double), float(spacing), _ptr(T, ctypes.c_double),
                                 int(width), float(px_mm[0]), float(px_mm[1]), _ptr(out, ctypes.c_int64))
    if rc:
        raise ValueError("bad geometry")
    return out


def round_stored(total, npix, dtype):
    """RN_fp32(total / npix) rounded to the storage type, as a float."""
    return _lib().ora_round_stored(float(total), float(npix), int(dtype))


class Volume:
    """A reconstructed directional volume held by the oracle (CSR over voxels)."""

    def __init__(self, handle, dims, spacing, vol_to_world):
        if not handle:
            raise ValueError("oracle volume construction failed")
        self._h = ctypes.c_void_p(handle)
        self.dims = tuple(int(d) for d in dims)
        self.spacing = float(spacing)
        self.vol_to_world = np.array(vol_to_world, dtype=np.float64).reshape(4, 4)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.ora_volume_free(h)
            self._h = None

    @property
    def n_samples(self):
        return int(_lib().ora_volume_nsamples(self._h))

    @property
    def n_overflow(self):
        return int(_lib().ora_volume_noverflow(self._h))

    @property
    def n_dropped(self):
        return int(_lib().ora_volume_ndropped(self._h))

    def export(self):
        """dict of numpy arrays: offsets, frame_id, npix, sum, mean_exact, stored,
        quat (n x 4), tot_sum, tot_npix."""
        n = self.n_samples
        nv = self.dims[0] * self.dims[1] * self.dims[2]
        d = dict(offsets=np.zeros(nv + 1, np.int64), frame_id=np.zeros(n, np.int32),
                 npix=np.zeros(n, np.int64), sum=np.zeros(n, np.int64),
                 mean_exact=np.zeros(n, np.float64), stored=np.zeros(n, np.float64),
                 quat=np.zeros((n, 4), np.float64), tot_sum=np.zeros(nv, np.int64),
                 tot_npix=np.zeros(nv, np.int64))
        c = ctypes
        _lib().ora_volume_export(self._h, _ptr(d["offsets"], c.c_int64), _ptr(d["frame_id"], c.c_int32),
                                 _ptr(d["npix"], c.c_int64), _ptr(d["sum"], c.c_int64),
                                 _ptr(d["mean_exact"], c.c_double), _ptr(d["stored"], c.c_double),
                                 _ptr(d["quat"], c.c_double), _ptr(d["tot_sum"], c.c_int64),
                                 _ptr(d["tot_npix"], c.c_int64))
        return d


def build(dims, spacing, vol_to_world, frames, poses, px_mm, dtype=F32, kmax=16, voxel_filter=None,
          probe=None, apex_mm=None, pixel_mask=None):
    """Reconstruct the directional volume from uint8 frames (n, H, W) and poses (n, 4, 4).

    probe: per-frame LINEAR / CURVILINEAR (a scalar applies to every frame),
    apex_mm: the fan apex of curvilinear frames, (2,) or (n, 2) image mm;
    pixel_mask: (H, W), zero excludes that pixel of every frame."""
    frames = _arr(frames, np.uint8)
    n, H, W = frames.shape
    poses = _arr(poses, np.float64).reshape(n, 16)
    dims_a = _arr(dims, np.int32)
    V = _arr(vol_to_world, np.float64).reshape(16)
    filt = None
    if voxel_filter is not None:
        filt = _arr(voxel_filter, np.uint8).reshape(-1)
        if filt.size != int(np.prod(dims)):
            raise ValueError("voxel_filter size")
    kinds = apex = pm = None
    if probe is not None:
        kinds = _arr(np.broadcast_to(np.asarray(probe, np.int32), (n,)), np.int32)
        apex = _arr(np.broadcast_to(np.asarray(apex_mm if apex_mm is not None else (0.0, 0.0), np.float64),
                                    (n, 2)), np.float64)
    if pixel_mask is not None:
        pm = _arr(pixel_mask, np.uint8)
        if pm.shape != (H, W):
            raise ValueError("pixel_mask shape")
    h = _lib().ora_build_probe(_ptr(dims_a, ctypes.c_int32), float(spacing), _ptr(V, ctypes.c_double), n, W, H,
                               float(px_mm[0]), float(px_mm[1]), _ptr(frames, ctypes.c_uint8),
                               _ptr(poses, ctypes.c_double), int(dtype), int(kmax),
                               _ptr(filt, ctypes.c_uint8) if filt is not None else None,
                               _ptr(kinds, ctypes.c_int32) if kinds is not None else None,
                               _ptr(apex, ctypes.c_double) if apex is not None else None,
                               _ptr(pm, ctypes.c_uint8) if pm is not None else None)
    return Volume(h, dims, spacing, vol_to_world)


def volume_from_samples(dims, spacing, vol_to_world, voxel, frame, value, quat):
    """Volume from explicit samples sorted by voxel index; quat is (n, 4) (w, x, y, z)."""
    voxel = _arr(voxel, np.int64)
    frame = _arr(frame, np.int32)
    value = _arr(value, np.float64)
    quat = _arr(quat, np.float64).reshape(-1, 4)
    dims_a = _arr(dims, np.int32)
    V = _arr(vol_to_world, np.float64).reshape(16)
    h = _lib().ora_volume_manual(_ptr(dims_a, ctypes.c_int32), float(spacing), _ptr(V, ctypes.c_double),
                                 voxel.size, _ptr(voxel, ctypes.c_int64), _ptr(frame, ctypes.c_int32),
                                 _ptr(value, ctypes.c_double), _ptr(quat, ctypes.c_double))
    return Volume(h, dims, spacing, vol_to_world)


def reslice(vol: Volume, image_to_world, width, height, px_mm, params: Params = None):
    """FP64 reslice of a whole plane: (out (H, W) float64, mask (H, W) uint8)."""
    p = (params or Params())._c()
    T = _arr(image_to_world, np.float64).reshape(16)
    out = np.zeros((height, width), np.float64)
    mask = np.zeros((height, width), np.uint8)
    rc = _lib().ora_reslice(vol._h, _ptr(T, ctypes.c_double), int(width), int(height), float(px_mm[0]),
                            float(px_mm[1]), ctypes.byref(p), _ptr(out, ctypes.c_double),
                            _ptr(mask, ctypes.c_uint8))
    if rc:
        raise ValueError("bad reslice arguments")
    return out, mask


def reslice_pixels(vol: Volume, image_to_world, width, px_mm, uv, params: Params = None):
    """FP64 reslice of chosen pixels uv (n, 2) = (u, v): (out (n,), mask (n,))."""
    p = (params or Params())._c()
    T = _arr(image_to_world, np.float64).reshape(16)
    uv = _arr(uv, np.int32).reshape(-1, 2)
    out = np.zeros(uv.shape[0], np.float64)
    mask = np.zeros(uv.shape[0], np.uint8)
    rc = _lib().ora_reslice_pixels(vol._h, _ptr(T, ctypes.c_double), int(width), float(px_mm[0]),
                                   float(px_mm[1]), ctypes.byref(p), uv.shape[0], _ptr(uv, ctypes.c_int32),
                                   _ptr(out, ctypes.c_double), _ptr(mask, ctypes.c_uint8))
    if rc:
        raise ValueError("bad reslice arguments")
    return out, mask


def reslice_scalar(vol: Volume, image_to_world, width, height, px_mm, unassigned=0.0):
    T = _arr(image_to_world, np.float64).reshape(16)
    out = np.zeros((height, width), np.float64)
    mask = np.zeros((height, width), np.uint8)
    _lib().ora_reslice_scalar(vol._h, _ptr(T, ctypes.c_double), int(width), int(height), float(px_mm[0]),
                              float(px_mm[1]), float(unassigned), _ptr(out, ctypes.c_double),
                              _ptr(mask, ctypes.c_uint8))
    return out, mask


def compounded(vol: Volume):
    """Mean-compounded value per voxel (flat, x fastest): RN_fp32(sum / npix) over
    every pixel that landed in it, NaN where none did."""
    out = np.zeros(int(np.prod(vol.dims)), np.float64)
    _lib().ora_compounded(vol._h, _ptr(out, ctypes.c_double))
    return out


def fill_holes(vol: Volume, values, radius=1, min_neighbours=1):
    """Hole filling of a compounded volume (the PLUS baseline's, Sec. 2.2): each
    empty voxel takes the 1/distance-weighted mean of the occupied voxels of its
    (2 radius + 1)^3 cube when at least min_neighbours are occupied."""
    values = _arr(values, np.float64).reshape(-1)
    out = np.zeros_like(values)
    _lib().ora_fill_holes(vol._h, _ptr(values, ctypes.c_double), int(radius), int(min_neighbours),
                          _ptr(out, ctypes.c_double))
    return out


def reslice_values(dims, spacing, vol_to_world, values, image_to_world, width, height, px_mm, unassigned=0.0):
    """Trilinear reslice of a scalar volume (NaN = empty), renormalised over the
    non-empty corners: (out (H, W), mask (H, W))."""
    dims_a = _arr(dims, np.int32)
    V = _arr(vol_to_world, np.float64).reshape(16)
    T = _arr(image_to_world, np.float64).reshape(16)
    values = _arr(values, np.float64).reshape(-1)
    out = np.zeros((height, width), np.float64)
    mask = np.zeros((height, width), np.uint8)
    _lib().ora_reslice_values(_ptr(dims_a, ctypes.c_int32), float(spacing), _ptr(V, ctypes.c_double),
                              _ptr(values, ctypes.c_double), _ptr(T, ctypes.c_double), int(width), int(height),
                              float(px_mm[0]), float(px_mm[1]), float(unassigned), _ptr(out, ctypes.c_double),
                              _ptr(mask, ctypes.c_uint8))
    return out, mask


def footprint(dims, spacing, vol_to_world, image_to_world, width, height, px_mm, radius=1, kernel=TENT):
    dims_a = _arr(dims, np.int32)
    V = _arr(vol_to_world, np.float64).reshape(16)
    T = _arr(image_to_world, np.float64).reshape(16)
    return int(_lib().ora_footprint(_ptr(dims_a, ctypes.c_int32), float(spacing), _ptr(V, ctypes.c_double),
                                    _ptr(T, ctypes.c_double), int(width), int(height), float(px_mm[0]),
                                    float(px_mm[1]), int(radius), int(kernel)))
