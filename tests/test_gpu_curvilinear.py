"""Curvilinear probes (a fan of beams from an apex; the paper's probe is a
linear array) on the CUDA path against the FP64 oracle: curvilinear frames,
a curvilinear virtual probe, both; every distance kernel at radius 1 and 2,
both normals, thresholds on and off, reduced storage; the build's pixel
mask; batches, host buffers and save / load.

Masks are bit-exact: every threshold decision is the FP64 one (FP32 with an
FP64 re-check inside the FP32 error bound).  Values: the weights are FP32
evaluations of Eq. 2 on per-sample axes, each axis within about 3e-7 of the
FP64 one here (|p| >= 20 mm, operand sums <= 100 mm), so a weight is within
(k_normal + k_inplane) |n_s - n_r| 3e-7 <= 15 * 0.43 * 3e-7 = 2e-6 of its FP64
value and a weighted mean within 2e-6 of the sample span (<= 255):
|gpu - oracle| <= 1e-5 max(|oracle|, 1) + 5e-4."""
import ctypes
import math
import types

import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import DEV, ORA_DTYPE, assert_parity, gpu_reslice, new_outputs, ora_params, oracle_dense

pytestmark = pytest.mark.gpu

APEX = (0.0, -20.0)
ATOL = 5e-4


def curv_params(p, out_apex=None):
    op = ora_params(p)
    if out_apex is not None:
        op.probe, op.apex_mm = oracle.CURVILINEAR, tuple(out_apex)
    return op


def check(out, mw, ref, rm, W, unassigned=0.0):
    """mask bit-exact; values within 1e-5 relative plus the weight-rounding term"""
    bits = dare.unpack_mask(mw, W)
    assert np.array_equal(bits, rm.astype(np.uint8)), f"mask mismatch at {np.argwhere(bits != rm)[:5]}"
    cov = rm.astype(bool)
    err = np.abs(out[cov] - ref[cov])
    tol = 1e-5 * np.maximum(np.abs(ref[cov]), 1.0) + ATOL
    assert np.all(err <= tol), f"max err {err.max()}"
    if np.isnan(unassigned):
        assert np.all(np.isnan(out[~cov]))
    else:
        assert np.all(out[~cov] == unassigned)
    return float(err.max(initial=0.0))


def curv_session(w, dtype=dare.DARE_F32, K=8, apex=APEX, pixel_mask=None, frames=None, poses=None):
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=K)
    s.set_probe(dare.DARE_PROBE_CURVILINEAR, apex, pixel_mask)
    frames = w.frames if frames is None else frames
    poses = w.frame_poses if poses is None else poses
    s.build(torch.from_numpy(np.ascontiguousarray(frames)).to(DEV), poses, w.frame_px)
    torch.cuda.synchronize()
    return s


def curv_oracle(w, dtype=dare.DARE_F32, K=8, apex=APEX, pixel_mask=None):
    return oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                        ORA_DTYPE[dtype], K, probe=oracle.CURVILINEAR, apex_mm=apex, pixel_mask=pixel_mask)


@pytest.fixture(scope="module")
def curv_pair(tiny):
    s = curv_session(tiny)
    yield s, curv_oracle(tiny)
    s.close()


@pytest.fixture(scope="module")
def linear_pair(tiny):
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=8)
    s.build(torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV), tiny.frame_poses, tiny.frame_px)
    torch.cuda.synchronize()
    yield s, oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, tiny.frames,
                          tiny.frame_poses, tiny.frame_px, oracle.F32, 8)
    s.close()


def _run(tiny, s, vol, p, out_apex, poses):
    covered, worst = 0, 0.0
    for T in poses:
        out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, curv_params(p, out_apex))
        worst = max(worst, check(out, mw, ref, rm, tiny.out_w, unassigned=float(p.unassigned)))
        covered += int(rm.sum())
    return covered, worst


@pytest.mark.parametrize("normal_axis", [dare.DARE_NORMAL_BEAM, dare.DARE_NORMAL_ELEVATION])
def test_curvilinear_frames_parity(tiny, curv_pair, normal_axis):
    s, vol = curv_pair
    p = dare.params_default(normal_axis=normal_axis)
    covered, _ = _run(tiny, s, vol, p, None, tiny.reslice_poses[[0, 2, 5, 9, 12, 15]])
    assert covered > 0


@pytest.mark.parametrize("normal_axis", [dare.DARE_NORMAL_BEAM, dare.DARE_NORMAL_ELEVATION])
def test_curvilinear_virtual_probe_parity(tiny, linear_pair, normal_axis):
    s, vol = linear_pair
    apex = (1.5, -24.0)
    p = dare.params_default(normal_axis=normal_axis, probe_apex_mm=apex)
    covered, _ = _run(tiny, s, vol, p, apex, tiny.reslice_poses[[1, 3, 6, 10, 13]])
    assert covered > 0


@pytest.mark.parametrize("kernel,R", [(dare.DARE_TENT, 1), (dare.DARE_TENT, 2), (dare.DARE_BOX, 1),
                                      (dare.DARE_EXP, 2)])
def test_both_curvilinear_kernels_and_radii(tiny, curv_pair, kernel, R):
    s, vol = curv_pair
    p = dare.params_default(radius_vox=R, dist_kernel=kernel, k_dist=0.8, probe_apex_mm=APEX)
    covered, _ = _run(tiny, s, vol, p, APEX, tiny.reslice_poses[[0, 7, 14]])
    assert covered > 0


def test_curvilinear_per_pixel_samples(tiny, curv_pair):
    """Per-pixel samples (npix-weighted) under a curvilinear virtual probe."""
    s, vol = curv_pair
    p = dare.params_default(probe_apex_mm=APEX, sample_weight=dare.DARE_SAMPLE_PIXELS)
    assert _run(tiny, s, vol, p, APEX, tiny.reslice_poses[[1, 8]])[0] > 0


def test_curvilinear_thresholds_off_and_nan(tiny, curv_pair):
    s, vol = curv_pair
    for p in (dare.params_default(thr_normal_deg=180.0, thr_inplane_deg=180.0, probe_apex_mm=APEX),
              dare.params_default(thr_normal_deg=10.0, thr_inplane_deg=180.0, unassigned=float("nan")),
              dare.params_default(k_normal=0.0, k_inplane=0.0, thr_inplane_deg=5.0, probe_apex_mm=(-3.0, -15.0))):
        apex = tuple(p.probe.apex_mm) if p.probe.kind else None
        _run(tiny, s, vol, p, apex, tiny.reslice_poses[[4, 11]])


@pytest.mark.parametrize("dtype,K", [(dare.DARE_U8, 4), (dare.DARE_F16, 12), (dare.DARE_BF16, 16)])
def test_curvilinear_reduced_storage(tiny, dtype, K):
    s = curv_session(tiny, dtype, K)
    vol = curv_oracle(tiny, dtype, K)
    p = dare.params_default(probe_apex_mm=APEX)
    _run(tiny, s, vol, p, APEX, tiny.reslice_poses[[2, 8]])
    s.close()


def test_threshold_decisions_are_fp64(tiny):
    """A linear frame resliced at its own pose by a curvilinear virtual probe:
    every sample of pixel p has d_inplane = cos(alpha_p) exactly, so with the
    in-plane threshold set a millionth of a degree either side of some pixels'
    alpha_p, FP32 alone cannot tell; the masks must still be the oracle's."""
    w = tiny
    T = w.frame_poses[60]
    frames = np.repeat(w.frames[60:61], 3, axis=0)
    poses = np.repeat(T[None], 3, axis=0)
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=4)
    s.build(torch.from_numpy(np.ascontiguousarray(frames)).to(DEV), poses, w.frame_px)
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, frames, poses, w.frame_px, oracle.F32, 4)
    W, H = w.frame_w, w.frame_h
    apex = (0.3, -18.0)
    n_flips = 0
    for (x, y) in [(5, 3), (100, 17), (64, 90), (20, 60)]:
        px, py = (x - 0.5 * (W - 1)) * w.frame_px[0] - apex[0], y * w.frame_px[1] - apex[1]
        alpha = math.degrees(math.atan2(abs(px), py))
        masks = []
        for delta in (-1e-6, 1e-6):
            p = dare.params_default(thr_inplane_deg=alpha + delta, thr_normal_deg=180.0, probe_apex_mm=apex)
            out, mw = gpu_reslice(s, T, W, H, w.frame_px, p)
            ref, rm = oracle.reslice(vol, T, W, H, w.frame_px, curv_params(p, apex))
            check(out, mw, ref, rm, W)
            masks.append(rm[y, x])
        n_flips += masks[0] != masks[1]
    assert n_flips >= 3  # the pixel's own decision flips with the threshold
    s.close()


def test_pixel_mask_build_records(tiny):
    """Masked pixels never reach the volume: records, npix and scalar totals
    equal the oracle's masked build bit for bit."""
    H, W = tiny.frames.shape[1:]
    yy, xx = np.mgrid[0:H, 0:W]
    px, py = (xx - 0.5 * (W - 1)) * tiny.frame_px[0] - APEX[0], yy * tiny.frame_px[1] - APEX[1]
    r = np.hypot(px, py)
    fan = ((np.abs(np.arctan2(px, py)) <= math.radians(20.0)) & (r >= 24.0)).astype(np.uint8)
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F16, max_slots=8,
                     flags=dare.DARE_SESSION_SCALAR)
    s.set_probe(dare.DARE_PROBE_CURVILINEAR, APEX, fan)
    s.build(torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV), tiny.frame_poses, tiny.frame_px)
    vol = curv_oracle(tiny, dare.DARE_F16, 8, pixel_mask=fan)
    rec = s.read_records(npix=True, scalar=True)
    ids, vals, npix, e = oracle_dense(vol, 8, dare.DARE_F16)
    assert np.array_equal(rec["frame_ids"], ids)
    assert np.array_equal(rec["values"].view(np.uint16), vals.view(np.uint16))
    assert np.array_equal(rec["npix"], npix)
    assert np.array_equal(rec["scalar_count"], e["tot_npix"].astype(np.uint32))
    assert np.array_equal(rec["scalar_sum"], e["tot_sum"].astype(np.uint32))
    assert 0.3 < fan.mean() < 0.9
    p = dare.params_default(probe_apex_mm=APEX)
    _run(tiny, s, vol, p, APEX, tiny.reslice_poses[[0, 5]])
    with pytest.raises(dare.DareError) as ei:  # frames of another size than the mask
        s.build(torch.zeros((1, H, W + 1), dtype=torch.uint8, device=DEV), tiny.frame_poses[:1], tiny.frame_px)
    assert ei.value.status == dare.DARE_E_INVALID
    s.close()


def test_mixed_batch_single_host_and_reload(tiny, curv_pair, linear_pair, tmp_path):
    """A batch over a curvilinear and a linear session equals the single calls
    bit for bit, through device and host buffers; a saved and reloaded
    curvilinear session reslices identically; plans and the allocation-free
    call refuse curvilinear work."""
    sc, _ = curv_pair
    sl, _ = linear_pair
    rng = np.random.default_rng(5)
    items, outs = [], []
    for i in range(10):
        W, H = int(rng.choice([37, 64, 100])), int(rng.choice([29, 64, 96]))
        o, m = new_outputs(W, H)
        items.append(((sc, sl)[i % 2], tiny.reslice_poses[i], o, m, tiny.out_px))
        outs.append((o, m, W, H))
    p = dare.params_default()
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    host = [(np.zeros((H, W), np.float32), np.zeros((H, dare.mask_words(W)), np.int32)) for _, _, W, H in outs]
    dare.reslice_batch_host(dare.make_requests([(it[0], it[1], ho, hm, it[4]) for it, (ho, hm) in zip(items, host)],
                                               host=True), p, group_planes=3)
    torch.cuda.current_stream().synchronize()
    for it, (o, m, W, H), (ho, hm) in zip(items, outs, host):
        o1, m1 = gpu_reslice(it[0], it[1], W, H, tiny.out_px, p)
        assert np.array_equal(m.cpu().numpy(), m1) and np.array_equal(o.cpu().numpy(), o1)
        assert np.array_equal(hm, m1) and np.array_equal(ho, o1)
    path = str(tmp_path / "curv.dare")
    sc.save(path)
    sr = dare.Session.load(path)
    for i in (3, 9):
        a = gpu_reslice(sc, tiny.reslice_poses[i], 64, 64, tiny.out_px, p)
        b = gpu_reslice(sr, tiny.reslice_poses[i], 64, 64, tiny.out_px, p)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    sr.close()
    with pytest.raises(dare.DareError) as ei:
        dare.Plan(items[:2], p)
    assert ei.value.status == dare.DARE_E_UNSUPPORTED
    o, m = new_outputs(16, 16)
    plane = dare.make_plane(16, 16, tiny.out_px, tiny.reslice_poses[0])
    pc = dare.params_default(probe_apex_mm=APEX)
    status = dare.lib().dare_reslice_noalloc(sl.handle, ctypes.byref(plane), ctypes.byref(pc),
                                             ctypes.c_void_p(o.data_ptr()), ctypes.c_void_p(m.data_ptr()), None)
    assert status == dare.DARE_E_UNSUPPORTED


def test_probe_argument_errors(tiny, linear_pair):
    s, _ = linear_pair
    for kind, apex in ((2, (0.0, -20.0)), (dare.DARE_PROBE_CURVILINEAR, (float("nan"), 0.0))):
        with pytest.raises(dare.DareError) as ei:
            s.set_probe(kind, apex)
        assert ei.value.status == dare.DARE_E_INVALID
    o, m = new_outputs(8, 8)
    p = dare.params_default()
    p.probe.kind = 7
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], o, m, tiny.out_px, p)
    assert ei.value.status == dare.DARE_E_INVALID


@pytest.mark.parametrize("K", [12, 16])
def test_curvilinear_every_record_fill(tiny, K):
    """Curvilinear frames and virtual probe on records of every fill from 1 to
    K (3 mm voxels over every 1st, 2nd, 3rd and 5th tiny frame at 0.1 x 0.12 mm
    pixels): the per-sample loop runs to every stopping point, full records
    included; masks exact, values within the bound above."""
    g = synth.centred_grid((12, 10, 9), 3.0)
    p = dare.params_default(probe_apex_mm=APEX)
    seen = set()
    for stride in (1, 2, 3, 5):
        w = types.SimpleNamespace(grid=g, frames=tiny.frames[::stride], frame_poses=tiny.frame_poses[::stride],
                                  frame_px=(0.1, 0.12))
        s = curv_session(w, K=K)
        vol = curv_oracle(w, K=K)
        seen |= set(np.diff(vol.export()["offsets"]).tolist())
        covered, _ = _run(tiny, s, vol, p, APEX, tiny.reslice_poses[[0, 3, 5]])
        assert covered > 0
        s.close()
    assert set(range(1, K + 1)) <= seen
