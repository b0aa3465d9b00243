"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Bit-exact: voxel assignment, frame ids, stored values, npix, coverage masks.
Floating point: |gpu - oracle| <= 1e-5 max(|oracle|, 1) for FP32 weight tables
(FP32 accumulation vs the oracle's FP64 on the same stored values).
"""
import ctypes
import math
import types

import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import (DEV, assert_parity, gpu_reslice, gpu_session, new_outputs, ora_params, oracle_dense,
                         oracle_volume)

pytestmark = pytest.mark.gpu

DTYPES = [dare.DARE_U8, dare.DARE_F16, dare.DARE_BF16, dare.DARE_F32]
PATHS = [dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED]


@pytest.fixture(scope="module")
def tiny_f32(tiny):
    s = gpu_session(tiny, dare.DARE_F32, 8)
    v = oracle_volume(tiny, dare.DARE_F32, 8)
    yield s, v
    s.close()


# ------------------------------------------------------------------ reconstruction

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [4, 8])
def test_build_records_bit_exact(tiny, dtype, K):
    """Fig. 1 voxelisation: every voxel's (frame id, stored value, npix) list equals
    the oracle's, including the capacity rule (tiny has up to 5 samples/voxel)."""
    s = gpu_session(tiny, dtype, K)
    vol = oracle_volume(tiny, dtype, K)
    ids, vals, npix, _ = oracle_dense(vol, K, dtype)
    g = s.read_records(npix=True)
    assert np.array_equal(g["frame_ids"], ids)
    assert np.array_equal(g["values"].view(np.uint8), vals.view(np.uint8))
    assert np.array_equal(g["npix"], npix)
    assert s.info().overflow_voxels == vol.n_overflow
    assert s.info().n_frames == len(tiny.frames)
    s.close()


def test_build_append_equals_one_call(tiny):
    """Appending in chunks (incremental integration, Sec. 4) gives the volume a
    single call gives; scalar totals too."""
    a = gpu_session(tiny, dare.DARE_F16, 4, flags=dare.DARE_SESSION_SCALAR, chunks=[0, 37, 120, 121, 200])
    b = gpu_session(tiny, dare.DARE_F16, 4, flags=dare.DARE_SESSION_SCALAR)
    ra, rb = a.read_records(npix=True, scalar=True), b.read_records(npix=True, scalar=True)
    for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
        assert np.array_equal(ra[k], rb[k]), k
    assert np.array_equal(ra["values"].view(np.uint16), rb["values"].view(np.uint16))
    e = oracle_volume(tiny, dare.DARE_F16, 4).export()
    assert np.array_equal(ra["scalar_sum"].astype(np.int64), e["tot_sum"])
    assert np.array_equal(ra["scalar_count"].astype(np.int64), e["tot_npix"])
    assert a.info().version == 4 and b.info().version == 1
    a.close()
    b.close()


def test_build_fine_pixels_coarse_voxels(tiny):
    """Pixels far finer than voxels (0.1 mm pixels in 4 mm voxels: over a
    thousand pixels of one frame in a voxel, and voxels beyond capacity):
    npix, means and the capacity rule stay bit-exact."""
    w = types.SimpleNamespace(grid=synth.centred_grid((9, 8, 7), 4.0), frames=tiny.frames[:60],
                              frame_poses=tiny.frame_poses[:60], frame_px=(0.1, 0.12))
    for dtype in (dare.DARE_F32, dare.DARE_U8):
        s = gpu_session(w, dtype, 8)
        ids, vals, npix, e = oracle_dense(oracle_volume(w, dtype, 8), 8, dtype)
        assert e["npix"].max() > 255
        g = s.read_records(npix=True)
        assert np.array_equal(g["frame_ids"], ids)
        assert np.array_equal(g["values"].view(np.uint8), vals.view(np.uint8))
        assert np.array_equal(g["npix"], npix)
        s.close()


@pytest.mark.parametrize("case", ["tiny_grid", "coarse_grid"])
def test_build_small_appends_touch_only_their_voxels(tiny, case):
    """Appends of 1 to 4 frames into an existing volume (incremental
    integration, Sec. 4) finalize only the voxels they reach (the listed path):
    records, npix and scalar totals equal one call over all frames, bit for
    bit, including voxels whose entries overflow their bucket (coarse grid:
    each frame splits a voxel over up to four tiles, 4-frame appends give it up
    to 16 entries) and the capacity rule (K = 4)."""
    if case == "tiny_grid":
        w = tiny
        bounds = [0, 40] + list(range(41, 81)) + [80, 200]
    else:
        w = types.SimpleNamespace(grid=synth.centred_grid((9, 8, 7), 4.0), frames=tiny.frames[:60],
                                  frame_poses=tiny.frame_poses[:60], frame_px=(0.1, 0.12))
        bounds = [0, 4, 8, 9, 11, 14, 18, 22, 26, 30, 34, 38, 42, 46, 50, 54, 58, 60]
    bounds = sorted(set(bounds))
    for dtype, K in ((dare.DARE_F32, 8), (dare.DARE_U8, 4)):
        a = gpu_session(w, dtype, K, flags=dare.DARE_SESSION_SCALAR, chunks=bounds)
        b = gpu_session(w, dtype, K, flags=dare.DARE_SESSION_SCALAR)
        ra, rb = a.read_records(npix=True, scalar=True), b.read_records(npix=True, scalar=True)
        for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
            assert np.array_equal(ra[k], rb[k]), k
        assert np.array_equal(ra["values"].view(np.uint8), rb["values"].view(np.uint8))
        a.close()
        b.close()


def test_build_frame_table(tiny, tiny_f32):
    s, _ = tiny_f32
    R = s.read_frames()
    V = tiny.grid.vol_to_world
    ref = np.einsum("ji,njk->nik", V[:3, :3], tiny.frame_poses[:, :3, :3])
    assert np.allclose(R, ref, atol=1e-15)


# ------------------------------------------------------------------ reslicing

@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("dtype", DTYPES)
def test_reslice_parity_tiny(tiny, path, dtype):
    """Eq. 1 / Eq. 2 reslicing of the 16 tiny poses (near-frame, moderately
    rotated, uniformly random -- the last fully unassigned)."""
    s = gpu_session(tiny, dtype, 8)
    vol = oracle_volume(tiny, dtype, 8)
    p = dare.params_default(path=path)
    covered = 0
    for T in tiny.reslice_poses:
        out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
        assert_parity(out, mw, ref, rm, tiny.out_w)
        covered += rm.sum()
    assert covered > 0.4 * 16 * tiny.out_w * tiny.out_h
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_reslice_variants(tiny, tiny_f32, path):
    """Elevation reading of Eq. 1's normal, thresholds off with k = 0
    (orientation-blind), custom constants, NaN for unassigned pixels."""
    s, vol = tiny_f32
    variants = [
        dare.params_default(path=path, normal_axis=dare.DARE_NORMAL_ELEVATION),
        dare.params_default(path=path, k_normal=0.0, k_inplane=0.0, thr_normal_deg=180.0, thr_inplane_deg=180.0),
        dare.params_default(path=path, k_normal=3.0, k_inplane=20.0, thr_normal_deg=40.0, thr_inplane_deg=5.0),
        dare.params_default(path=path, unassigned=float("nan")),
    ]
    for p in variants:
        for T in tiny.reslice_poses[[0, 5, 9, 13]]:
            out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
            ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
            assert_parity(out, mw, ref, rm, tiny.out_w, unassigned=float(p.unassigned))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("K", [4, 8, 12, 16])
def test_reslice_every_record_fill(tiny, K, path):
    """Records holding every sample count from 1 to K, full ones included: 3 mm
    voxels over every 1st, 2nd, 3rd and 5th tiny frame at 0.1 x 0.12 mm pixels
    put 1 to 16 frames in a voxel.  The reslice kernels look the weights of a
    record's samples up in groups of slots and stop at the first empty slot, so
    each count stops at a different place inside or between groups; checked on
    the TENT R = 1 kernels, the general-radius kernels (BOX R = 2) and per-pixel
    sample weighting."""
    g = synth.centred_grid((12, 10, 9), 3.0)
    seen = set()
    for stride in (1, 2, 3, 5):
        w = types.SimpleNamespace(grid=g, frames=tiny.frames[::stride], frame_poses=tiny.frame_poses[::stride],
                                  frame_px=(0.1, 0.12))
        s = gpu_session(w, dare.DARE_F32, K)
        vol = oracle_volume(w, dare.DARE_F32, K)
        seen |= set(np.diff(vol.export()["offsets"]).tolist())
        for p in (dare.params_default(path=path),
                  dare.params_default(path=path, radius_vox=2, dist_kernel=dare.DARE_BOX),
                  dare.params_default(path=path, sample_weight=dare.DARE_SAMPLE_PIXELS)):
            covered = 0
            for T in tiny.reslice_poses[[0, 3, 5, 12]]:
                out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
                ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
                assert_parity(out, mw, ref, rm, tiny.out_w)
                covered += int(rm.sum())
            assert covered > 0
        s.close()
    assert set(range(1, K + 1)) <= seen


@pytest.mark.parametrize("path", PATHS)
def test_reslice_fp16_weights(tiny, path):
    """FP16 weight table: masks stay bit-exact; values within the bound of a
    relative weight error eps = 2^-11: |d out| <= 2 eps / (1 - eps) (max I - min I)."""
    s = gpu_session(tiny, dare.DARE_F16, 8)
    vol = oracle_volume(tiny, dare.DARE_F16, 8)
    p = dare.params_default(path=path, weight_dtype=dare.DARE_WEIGHTS_F16)
    eps = 2.0 ** -11
    bound = 2 * eps / (1 - eps) * 255.0 + 1e-3
    for T in tiny.reslice_poses[:12]:
        out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
        assert np.array_equal(dare.unpack_mask(mw, tiny.out_w), rm)
        cov = rm.astype(bool)
        assert np.max(np.abs(out[cov] - ref[cov]), initial=0) <= bound
    s.close()


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("W,H", [(1, 1), (37, 23), (33, 17), (200, 5), (5, 200), (64, 48)])
def test_reslice_ragged_sizes(tiny, tiny_f32, path, W, H):
    """Output sizes that are not multiples of the 32 x 16 tile or of 32-bit mask words."""
    s, vol = tiny_f32
    p = dare.params_default(path=path)
    px = (0.31, 0.27)
    for T in tiny.reslice_poses[[1, 8]]:
        T = synth.plane_pose_centred(T[:3, :3], np.zeros(3), W, H, *px)
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert_parity(out, mw, ref, rm, W)


@pytest.mark.parametrize("path", PATHS)
def test_reslice_edge_cases(tiny, path):
    """A session with no frames, and a plane entirely outside the grid: every
    pixel unassigned, every mask bit 0."""
    p = dare.params_default(path=path, unassigned=-1.0)
    empty = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world)
    out, mw = gpu_reslice(empty, tiny.reslice_poses[0], 40, 30, tiny.out_px, p)
    assert np.all(out == -1.0) and not mw.any()
    empty.close()
    s = gpu_session(tiny, dare.DARE_F32, 8)
    far = tiny.reslice_poses[0].copy()
    far[:3, 3] += 500.0
    out, mw = gpu_reslice(s, far, 64, 64, tiny.out_px, p)
    assert np.all(out == -1.0) and not mw.any()
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_batch_equals_single(tiny, path):
    """dare_reslice_batch over two sessions of different storage types and
    uneven output sizes: each result equals the request resliced alone, and the
    oracle."""
    s1 = gpu_session(tiny, dare.DARE_F32, 8)
    s2 = gpu_session(tiny, dare.DARE_U8, 4)
    v1 = oracle_volume(tiny, dare.DARE_F32, 8)
    v2 = oracle_volume(tiny, dare.DARE_U8, 4)
    p = dare.params_default(path=path)
    sizes = [(128, 128), (37, 23), (256, 64), (64, 200), (1, 1), (96, 96)]
    items, singles, refs = [], [], []
    for i, (W, H) in enumerate(sizes * 2):
        s, v = (s1, v1) if i % 2 == 0 else (s2, v2)
        T = synth.plane_pose_centred(tiny.reslice_poses[i % 16][:3, :3], np.zeros(3), W, H, *tiny.out_px)
        out, mask = new_outputs(W, H)
        items.append((s, T, out, mask, tiny.out_px))
        singles.append(gpu_reslice(s, T, W, H, tiny.out_px, p))
        refs.append(oracle.reslice(v, T, W, H, tiny.out_px, ora_params(p)) + (W,))
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    for (s, T, out, mask, _), (o1, m1), (ref, rm, W) in zip(items, singles, refs):
        assert np.array_equal(out.cpu().numpy(), o1) or np.allclose(out.cpu().numpy(), o1, rtol=1e-6, atol=1e-6)
        assert np.array_equal(mask.cpu().numpy(), m1)
        assert_parity(out.cpu().numpy(), mask.cpu().numpy(), ref, rm, W)
    s1.close()
    s2.close()


# ------------------------------------------------------------------ comparator, footprint

def test_scalar_comparator(tiny):
    s = gpu_session(tiny, dare.DARE_F32, 8, flags=dare.DARE_SESSION_SCALAR)
    vol = oracle_volume(tiny, dare.DARE_F32, 8)
    for T in tiny.reslice_poses[[0, 3, 12]]:
        out, mask = new_outputs(tiny.out_w, tiny.out_h)
        s.reslice_scalar(T, out, mask, tiny.out_px)
        torch.cuda.synchronize()
        ref, rm = oracle.reslice_scalar(vol, T, tiny.out_w, tiny.out_h, tiny.out_px)
        assert_parity(out.cpu().numpy(), mask.cpu().numpy(), ref, rm, tiny.out_w)
    s.close()


def test_footprint_counts(tiny, tiny_f32):
    s, _ = tiny_f32
    got = s.footprint(tiny.reslice_poses, tiny.out_w, tiny.out_h, tiny.out_px)
    ref = [oracle.footprint(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, T, tiny.out_w, tiny.out_h,
                            tiny.out_px) for T in tiny.reslice_poses]
    assert list(got) == ref


# ------------------------------------------------------------------ checkpoint, memory, capacity

def test_save_load_roundtrip(tiny, tmp_path):
    s = gpu_session(tiny, dare.DARE_BF16, 8, flags=dare.DARE_SESSION_SCALAR)
    path = tmp_path / "vol.dare"
    s.save(path)
    t = dare.Session.load(path)
    assert t.dims == s.dims and t.info().n_frames == s.info().n_frames
    p = dare.params_default()
    for T in tiny.reslice_poses[[0, 9]]:
        a = gpu_reslice(s, T, 96, 80, tiny.out_px, p)
        b = gpu_reslice(t, T, 96, 80, tiny.out_px, p)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0x40
    bad = tmp_path / "bad.dare"
    bad.write_bytes(bytes(raw))
    with pytest.raises(dare.DareError) as ei:
        dare.Session.load(bad)
    assert ei.value.status == dare.DARE_E_INVALID and "CRC" in str(ei.value)
    s.close()
    t.close()


def test_allocator_hook_and_oom(tiny):
    """Volumes and workspace come from PyTorch's caching allocator through the
    callback; a failing allocation returns DARE_E_OOM and leaves the session usable."""
    alloc = dare.TorchAllocator(0)
    alloc.fail_next = 1
    with pytest.raises(dare.DareError) as ei:
        dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, allocator=alloc)
    assert ei.value.status == dare.DARE_E_OOM
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, allocator=alloc)
    assert len(alloc.live) == 1
    ft = torch.from_numpy(tiny.frames).to(DEV)
    alloc.fail_next = 1  # the build's workspace
    with pytest.raises(dare.DareError) as ei:
        s.build(ft, tiny.frame_poses, tiny.frame_px)
    assert ei.value.status == dare.DARE_E_OOM
    s.build(ft, tiny.frame_poses, tiny.frame_px)
    ref = gpu_session(tiny, dare.DARE_F32, 8)
    p = dare.params_default()
    a = gpu_reslice(s, tiny.reslice_poses[2], 64, 64, tiny.out_px, p)
    b = gpu_reslice(ref, tiny.reslice_poses[2], 64, 64, tiny.out_px, p)
    assert np.array_equal(a[0], b[0])
    s.close()
    ref.close()
    assert len(alloc.live) == 0


class _ShiftedAllocator:
    """Caller allocator whose blocks start `shift` bytes past a 256-byte boundary."""

    def __init__(self, shift):
        self.shift, self.live, self.freed = shift, {}, []

        def _alloc(nbytes, stream, ctx):
            t = torch.empty(int(nbytes) + 512, dtype=torch.uint8, device=DEV)
            p = (t.data_ptr() + 255) // 256 * 256 + self.shift
            self.live[p] = t
            return p

        def _free(ptr, nbytes, stream, ctx):
            self.freed.append(ptr)
            self.live.pop(ptr, None)

        self._a, self._f = dare._ALLOC_FN(_alloc), dare._FREE_FN(_free)

    def as_struct(self):
        a = dare.dare_allocator()
        a.alloc, a.free, a.ctx = self._a, self._f, None
        return a


def test_allocator_misaligned_block_refused(tiny):
    """A block off the 256-byte alignment the header asks of a caller allocator
    goes straight back to its free and the call fails with DARE_E_OOM, before
    any kernel could touch it; aligned blocks from the same allocator work."""
    bad = _ShiftedAllocator(16)
    with pytest.raises(dare.DareError) as ei:
        dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, allocator=bad)
    assert ei.value.status == dare.DARE_E_OOM
    assert len(bad.freed) == 1 and not bad.live
    good = _ShiftedAllocator(0)
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, allocator=good)
    s.build(torch.from_numpy(tiny.frames).to(DEV), tiny.frame_poses, tiny.frame_px)
    ref = gpu_session(tiny, dare.DARE_F32, 8)
    p = dare.params_default()
    a = gpu_reslice(s, tiny.reslice_poses[2], 64, 64, tiny.out_px, p)
    b = gpu_reslice(ref, tiny.reslice_poses[2], 64, 64, tiny.out_px, p)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    s.close()
    ref.close()
    assert not good.live


def test_memory_budget_admission(tiny):
    base = dare.memory_in_use()
    dare.set_memory_budget(base + 1024)
    try:
        with pytest.raises(dare.DareError) as ei:
            dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world)
        assert ei.value.status == dare.DARE_E_ADMISSION
    finally:
        dare.set_memory_budget(0)
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world)
    assert dare.memory_in_use() > base
    s.close()
    assert dare.memory_in_use() == base


def test_frame_capacity(tiny):
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, max_frames=150)
    ft = torch.from_numpy(tiny.frames).to(DEV)
    with pytest.raises(dare.DareError) as ei:
        s.build(ft, tiny.frame_poses, tiny.frame_px)
    assert ei.value.status == dare.DARE_E_CAPACITY
    assert s.info().n_frames == 0
    s.build(ft[:150], tiny.frame_poses[:150], tiny.frame_px)
    assert s.info().n_frames == 150
    s.close()


def test_unsupported_radius_is_reported(tiny, tiny_f32):
    s, _ = tiny_f32
    out, mask = new_outputs(8, 8)
    for path in (dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED):
        with pytest.raises(dare.DareError) as ei:
            s.reslice(tiny.reslice_poses[0], out, mask, tiny.out_px, dare.params_default(radius_vox=17, path=path))
        assert ei.value.status == dare.DARE_E_UNSUPPORTED


def test_reset_then_rebuild_equals_fresh(tiny):
    s = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR)
    ft = torch.from_numpy(tiny.frames).to(DEV)
    s.reset()
    info = s.info()
    assert info.n_frames == 0 and info.version == 0
    g = s.read_records(npix=True, scalar=True)
    assert np.all(g["frame_ids"] == 0xFFFF) and not g["npix"].any() and not g["scalar_count"].any()
    s.build(ft, tiny.frame_poses, tiny.frame_px)
    fresh = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR)
    a, b = s.read_records(npix=True, scalar=True), fresh.read_records(npix=True, scalar=True)
    for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["values"].view(np.uint16), b["values"].view(np.uint16))
    s.close()
    fresh.close()


def test_trace_and_launch_count(tiny, tiny_f32):
    s, _ = tiny_f32
    dare.trace_read()
    n0 = dare.launch_count()
    dare.trace_enable(True)
    try:
        p = dare.params_default()
        gpu_reslice(s, tiny.reslice_poses[0], 64, 64, tiny.out_px, p)
        gpu_reslice(s, tiny.reslice_poses[1], 64, 64, tiny.out_px, dare.params_default(path=dare.DARE_PATH_PLAIN))
        t = dare.trace_read()
    finally:
        dare.trace_enable(False)
    assert dare.launch_count() - n0 == 4
    assert t["reslice_tiled"][0] == 1 and t["reslice_plain"][0] == 1 and t["weight_table"][0] == 2
    assert all(ms > 0 for _, ms in t.values())


@pytest.mark.parametrize("path", [dare.DARE_PATH_AUTO, dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED])
def test_plan_graph_replay(tiny, path):
    """A plan (graph capture, autotuned kernels) over two sessions of different
    storage types and uneven sizes equals dare_reslice per request, and a replay
    after set_poses equals the new poses resliced alone."""
    s1 = gpu_session(tiny, dare.DARE_F32, 8)
    s2 = gpu_session(tiny, dare.DARE_F16, 4)
    p = dare.params_default(path=path)
    sizes = [(128, 128), (37, 23), (256, 64), (64, 200), (96, 96), (128, 128), (128, 128)]
    items, poses_a, poses_b = [], [], []
    for i, (W, H) in enumerate(sizes):
        s = s1 if i % 2 == 0 else s2
        Ta = synth.plane_pose_centred(tiny.reslice_poses[i][:3, :3], np.zeros(3), W, H, *tiny.out_px)
        Tb = synth.plane_pose_centred(tiny.reslice_poses[i + 7][:3, :3], np.zeros(3), W, H, *tiny.out_px)
        out, mask = new_outputs(W, H)
        items.append((s, Ta, out, mask, tiny.out_px))
        poses_a.append(Ta)
        poses_b.append(Tb)
    plan = dare.Plan(items, p)
    info = plan.info()
    assert info["n_groups"] == 2 and info["n_requests"] == len(sizes)
    if path == dare.DARE_PATH_AUTO:
        assert all(c in (0, 16, 32, 64) for c in info["choice"])
    for poses in (poses_a, poses_b):
        plan.set_poses(np.stack(poses))
        for _, _, out, mask, _ in items:
            out.fill_(-7.0)
        plan.launch()
        torch.cuda.synchronize()
        for (s, _, out, mask, px), T in zip(items, poses):
            H, W = out.shape
            o1, m1 = gpu_reslice(s, T, W, H, px, dare.params_default())
            assert np.array_equal(mask.cpu().numpy(), m1)
            cov = dare.unpack_mask(m1, W).astype(bool)
            got = out.cpu().numpy()
            assert np.all(np.abs(got[cov] - o1[cov]) <= 1e-5 * np.maximum(np.abs(o1[cov]), 1))
            assert np.all(got[~cov] == 0.0)
    s1.reset()
    with pytest.raises(dare.DareError) as ei:
        plan.launch()
    assert ei.value.status == dare.DARE_E_STATE
    plan.close()
    s1.close()
    s2.close()


def test_l2_persist_mode_same_results(tiny):
    """DARE_SESSION_L2_PERSIST changes cache policy only: results on a side
    stream equal those of an ordinary session, batch and single."""
    a = gpu_session(tiny, dare.DARE_F32, 8, flags=dare.DARE_SESSION_L2_PERSIST)
    b = gpu_session(tiny, dare.DARE_F32, 8)
    side = torch.cuda.Stream()
    p = dare.params_default()
    for T in tiny.reslice_poses[[0, 4, 9]]:
        oa, ma = new_outputs(128, 128)
        with torch.cuda.stream(side):
            a.reslice(T, oa, ma, tiny.out_px, p, stream=side)
        side.synchronize()
        ob, mb = gpu_reslice(b, T, 128, 128, tiny.out_px, p)
        assert np.array_equal(ma.cpu().numpy(), mb) and np.array_equal(oa.cpu().numpy(), ob)
    items = []
    for T in tiny.reslice_poses[:6]:
        o, m = new_outputs(128, 128)
        items.append((a, T, o, m, tiny.out_px))
    dare.reslice_batch(items, p, stream=side)
    side.synchronize()
    for (_, T, o, m, _) in items:
        ob, mb = gpu_reslice(b, T, 128, 128, tiny.out_px, p)
        assert np.array_equal(m.cpu().numpy(), mb) and np.array_equal(o.cpu().numpy(), ob)
    a.close()
    b.close()


def test_host_volume_session_equals_device(tiny):
    """DARE_SESSION_HOST_VOLUME: records in mapped host memory give the
    device-resident session's records and images bit for bit, and the device
    holds only the session's small tables."""
    dev = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR)
    host = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR | dare.DARE_SESSION_HOST_VOLUME,
                       chunks=[0, 77, 200])
    ref = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR, chunks=[0, 77, 200])
    ra, rb = ref.read_records(npix=True, scalar=True), host.read_records(npix=True, scalar=True)
    for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
        assert np.array_equal(ra[k], rb[k]), k
    assert np.array_equal(ra["values"].view(np.uint16), rb["values"].view(np.uint16))
    nv = int(np.prod(tiny.grid.dims))
    assert dev.info().volume_bytes - host.info().volume_bytes >= nv * (dev.info().record_bytes + 2 * 8)
    for path in (dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED):
        p = dare.params_default(path=path)
        for T in tiny.reslice_poses[[0, 4, 9]]:
            o1, m1 = gpu_reslice(ref, T, 96, 80, tiny.out_px, p)
            o2, m2 = gpu_reslice(host, T, 96, 80, tiny.out_px, p)
            assert np.array_equal(m1, m2) and np.array_equal(o1, o2)
    for s in (dev, host, ref):
        s.close()


@pytest.mark.parametrize("flags", [dare.DARE_SESSION_SCALAR, dare.DARE_SESSION_SCALAR | dare.DARE_SESSION_HOST_VOLUME])
def test_reset_is_cleared_by_the_next_call(tiny, tmp_path, flags):
    """dare_session_reset defers the clear: the next build's finalize writes
    every voxel (records, npix, scalar totals), and any other call clears the
    volume first.  Each route gives exactly the volume (or the unassigned
    image) of a session that never held the old frames."""
    ft = torch.from_numpy(tiny.frames).to(DEV)
    a, b = slice(0, 120), slice(80, 200)
    fresh = gpu_session(tiny, dare.DARE_F16, 8, flags=flags, frames=tiny.frames[b], poses=tiny.frame_poses[b])
    ref = fresh.read_records(npix=True, scalar=True)
    s = gpu_session(tiny, dare.DARE_F16, 8, flags=flags, frames=tiny.frames[a], poses=tiny.frame_poses[a])
    # reset + build: the full-write finalize
    s.reset()
    s.build(ft[b], tiny.frame_poses[b], tiny.frame_px)
    got = s.read_records(npix=True, scalar=True)
    for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["values"].view(np.uint16), ref["values"].view(np.uint16))
    T = tiny.reslice_poses[3]
    o1, m1 = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, dare.params_default())
    o2, m2 = gpu_reslice(fresh, T, tiny.out_w, tiny.out_h, tiny.out_px, dare.params_default())
    assert np.array_equal(m1, m2) and np.array_equal(o1, o2)
    # reset + every reading call: an empty volume
    for route in ("reslice", "batch", "scalar", "holes", "save"):
        s.reset()
        out, mask = new_outputs(40, 30)
        if route == "reslice":
            s.reslice(T, out, mask, tiny.out_px)
        elif route == "batch":
            dare.reslice_batch([(s, T, out, mask, tiny.out_px)])
        elif route == "scalar":
            s.reslice_scalar(T, out, mask, tiny.out_px)
        elif route == "holes":
            s.fill_holes(1, 1)
            assert np.all(np.isnan(s.read_filled()))
            s.reslice_scalar_filled(T, out, mask, tiny.out_px)
        else:
            path = str(tmp_path / "reset.dare")
            s.save(path)
            r = dare.Session.load(path)
            e = r.read_records(npix=True, scalar=True)
            assert np.all(e["frame_ids"] == 0xFFFF) and not e["npix"].any() and not e["scalar_count"].any()
            r.close()
            s.reslice(T, out, mask, tiny.out_px)
        torch.cuda.synchronize()
        assert not mask.cpu().numpy().any(), route
        assert np.all(out.cpu().numpy() == 0.0), route
        e = s.read_records(npix=True, scalar=True)
        assert np.all(e["frame_ids"] == 0xFFFF) and not e["npix"].any() and not e["scalar_sum"].any()
        s.build(ft[b], tiny.frame_poses[b], tiny.frame_px)  # merge into the cleared volume: as fresh
        got = s.read_records(npix=True, scalar=True)
        assert np.array_equal(got["frame_ids"], ref["frame_ids"]) and np.array_equal(got["npix"], ref["npix"])
        assert np.array_equal(got["scalar_sum"], ref["scalar_sum"])
    s.close()
    fresh.close()


def test_reset_rebuild_odd_grid_matches_oracle(tiny):
    """Reset + rebuild (the full-write finalize, whole 256-voxel runs stored by
    bulk copies and a shorter tail run thread by thread) on a grid whose voxel
    count is not a multiple of 256: records bit-exact against the oracle."""
    import synth
    g = synth.centred_grid((61, 57, 59), 0.55)
    s = dare.Session(g.dims, g.spacing, g.vol_to_world, dtype=dare.DARE_BF16, max_slots=8,
                     flags=dare.DARE_SESSION_SCALAR)
    ft = torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV)
    s.build(ft[:50], tiny.frame_poses[:50], tiny.frame_px)
    s.reset()
    s.build(ft, tiny.frame_poses, tiny.frame_px)
    got = s.read_records(npix=True, scalar=True)
    vol = oracle.build(g.dims, g.spacing, g.vol_to_world, tiny.frames, tiny.frame_poses, tiny.frame_px, oracle.BF16, 8)
    ids, vals, npix, e = oracle_dense(vol, 8, dare.DARE_BF16)
    assert int(np.prod(g.dims)) % 256 != 0
    assert np.array_equal(got["frame_ids"], ids)
    assert np.array_equal(got["values"].view(np.uint16), vals.view(np.uint16))
    assert np.array_equal(got["npix"], npix)
    assert np.array_equal(got["scalar_count"], e["tot_npix"].astype(np.uint32))
    assert np.array_equal(got["scalar_sum"], e["tot_sum"].astype(np.uint32))
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_reslice_maximum_plane_sizes(tiny, tiny_f32, path):
    """Planes at the largest accepted size along one axis (65535 pixels wide,
    or tall) against the oracle; one past it is refused."""
    s, vol = tiny_f32
    p = dare.params_default(path=path)
    px = (0.0005, 0.0005)  # 65535 pixels span 33 mm: across the whole grid
    for W, H in ((65535, 2), (3, 65535)):
        T = synth.plane_pose_centred(tiny.reslice_poses[4][:3, :3], np.zeros(3), W, H, *px)
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert rm.sum() > 1000
        assert_parity(out, mw, ref, rm, W)
    out, mask = new_outputs(8, 8)
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], torch.empty((1, 65536), device=DEV), torch.empty((1, 2048), dtype=torch.int32,
                                                                                        device=DEV), tiny.out_px, p)
    assert ei.value.status == dare.DARE_E_INVALID


@pytest.mark.parametrize("W,H", [(1, 1), (37, 29), (33, 64), (130, 7)])
def test_build_ragged_frame_sizes(tiny, W, H):
    """Frames that are not whole 32 x 32 scatter tiles (down to one pixel):
    records bit-exact against the oracle."""
    rng = np.random.default_rng(W * 131 + H)
    frames = rng.integers(0, 256, (60, H, W)).astype(np.uint8)
    px = (0.3, 0.3)
    poses = np.stack([synth.plane_pose_centred(tiny.frame_poses[i][:3, :3], rng.uniform(-4, 4, 3), W, H, *px)
                      for i in range(0, 120, 2)])
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=8)
    s.build(torch.from_numpy(frames).to(DEV), poses, px)
    got = s.read_records(npix=True)
    vol = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, frames, poses, px, oracle.F32, 8)
    ids, vals, npix, e = oracle_dense(vol, 8, dare.DARE_F32)
    assert e["npix"].sum() > 0
    assert np.array_equal(got["frame_ids"], ids)
    assert np.array_equal(got["values"].view(np.uint32), vals.view(np.uint32))
    assert np.array_equal(got["npix"], npix)
    s.close()


@pytest.mark.parametrize("W,H", [(130, 37), (64, 64)])
def test_build_frames_at_odd_address(tiny, W, H):
    """Even frame widths let the count pass read a pixel pair with one 16-bit
    load; frames that start at an odd device address take the byte loads.
    Both give the oracle's records bit for bit."""
    rng = np.random.default_rng(W + 7 * H)
    frames = rng.integers(0, 256, (40, H, W)).astype(np.uint8)
    px = (0.3, 0.3)
    poses = np.stack([synth.plane_pose_centred(tiny.frame_poses[i][:3, :3], rng.uniform(-4, 4, 3), W, H, *px)
                      for i in range(0, 120, 3)])
    buf = torch.empty(frames.size + 1, dtype=torch.uint8, device=DEV)
    odd = buf[1:].view(frames.shape)
    odd.copy_(torch.from_numpy(frames))
    assert odd.data_ptr() % 2 == 1
    vol = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, frames, poses, px, oracle.F32, 8)
    ids, vals, npix, e = oracle_dense(vol, 8, dare.DARE_F32)
    assert e["npix"].sum() > 0
    for src in (torch.from_numpy(frames).to(DEV), odd):
        s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=8)
        s.build(src, poses, px)
        got = s.read_records(npix=True)
        assert np.array_equal(got["frame_ids"], ids)
        assert np.array_equal(got["values"].view(np.uint32), vals.view(np.uint32))
        assert np.array_equal(got["npix"], npix)
        s.close()


def test_single_plane_graph_equals_launches(tiny, tiny_f32):
    """A single tiled plane runs as the session's two-node graph (weight table,
    reslice) with its node parameters replaced each call; while tracing it runs
    as two launches instead. Both give the same bits, across plane sizes (the
    reslice node's grid changes), FP16 and FP32 weights (the graph is rebuilt)
    and back."""
    s, vol = tiny_f32
    sizes = [(64, 48), (130, 101), (37, 29), (64, 48)]
    for wd in (dare.DARE_WEIGHTS_F32, dare.DARE_WEIGHTS_F16, dare.DARE_WEIGHTS_F32):
        p = dare.params_default(path=dare.DARE_PATH_TILED, weight_dtype=wd)
        for k, (W, H) in enumerate(sizes):
            T = tiny.reslice_poses[(3 * k + wd) % len(tiny.reslice_poses)]
            n0 = dare.launch_count()
            g = gpu_reslice(s, T, W, H, tiny.out_px, p)
            assert dare.launch_count() - n0 == 2
            dare.trace_read()
            dare.trace_enable(True)
            try:
                d = gpu_reslice(s, T, W, H, tiny.out_px, p)
                t = dare.trace_read()
            finally:
                dare.trace_enable(False)
            assert t["weight_table"][0] == 1 and t["reslice_tiled"][0] == 1
            assert np.array_equal(g[1], d[1]) and np.array_equal(g[0], d[0])
            if wd == dare.DARE_WEIGHTS_F32:
                ref, rm = oracle.reslice(vol, T, W, H, tiny.out_px, ora_params(p))
                assert_parity(g[0], g[1], ref, rm, W)
