"""Pins for the CPU oracle: checks against facts the paper and mathematics fix.

None of these compares the oracle with itself.  Each pin is an independent
derivation -- a closed form, a library routine (scipy / torch), a numpy
re-derivation by different means, a brute force over the whole grid, or an
invariant -- chosen so that a dropped term, a wrong sign, a swapped index or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy import ndimage
from scipy.spatial.transform import Rotation

import _brute
import oracle
import synth

FIX = 2.0 ** 20
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def quat_wxyz(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def voxel_coords(aff, W, H):
    """continuous voxel coordinates of every pixel from a quantised affine, (H, W, 3)"""
    u = np.arange(W, dtype=np.int64)[None, :, None]
    v = np.arange(H, dtype=np.int64)[:, None, None]
    G = aff[0:3][None, None, :] + u * aff[3:6][None, None, :] + v * aff[6:9][None, None, :]
    return G, G.astype(np.float64) / FIX


def flat_index(c, dims):
    return c[..., 0] + dims[0] * (c[..., 1] + dims[1] * c[..., 2])


def rigid(rng, spread=10.0):
    return synth.make_pose(synth.random_rotation(rng), rng.uniform(-spread, spread, 3))


def rot_x(a):
    return synth.rot_axis_angle([1, 0, 0], a)


def rot_y(a):
    return synth.rot_axis_angle([0, 1, 0], a)


def rot_z(a):
    return synth.rot_axis_angle([0, 0, 1], a)


def single_voxel_case(sample_rots, values, plane_R, params):
    """3x3x3 grid at 1 mm, identity volume pose, all samples in voxel (1,1,1),
    a 1x1 plane whose only pixel sits exactly on that voxel centre."""
    dims = (3, 3, 3)
    n = len(values)
    vol = oracle.volume_from_samples(dims, 1.0, np.eye(4), [13] * n, list(range(n)), values,
                                     [quat_wxyz(R) for R in sample_rots])
    P = synth.make_pose(plane_R, [1.0, 1.0, 1.0])
    out, mask = oracle.reslice(vol, P, 1, 1, (1.0, 1.0), params)
    return out[0, 0], mask[0, 0]


# ----------------------------------------------------------------- geometry

def test_affine_axis_aligned_exact():
    """Hand-computed case: volume origin voxel at (-2.5,-2.5,-2.5) mm, h = 0.5 mm,
    identity plane rotation at the world origin, W = 5, 0.5 mm pixels: pixel
    (u, v) lands on voxel (3 + u, 5 + v, 5)."""
    V = synth.make_pose(np.eye(3), [-2.5, -2.5, -2.5])
    T = np.eye(4)
    aff = oracle.pixel_affine(V, 0.5, T, 5, (0.5, 0.5))
    assert list(aff) == [3 * 2**20, 5 * 2**20, 5 * 2**20, 2**20, 0, 0, 0, 2**20, 0]


def test_affine_matches_matrix_inverse():
    """Against numpy's general 4x4 inverse: every coefficient within half a unit
    of 2^-20 voxel, and pixel coordinates within the accumulated rounding."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        V, T = rigid(rng), rigid(rng)
        h = rng.uniform(0.1, 1.0)
        W = int(rng.integers(1, 700))
        sx, sy = rng.uniform(0.05, 0.6, 2)
        aff = oracle.pixel_affine(V, h, T, W, (sx, sy))
        M = np.linalg.inv(V) @ T
        g0 = (M[:3, 3] - 0.5 * (W - 1) * sx * M[:3, 0]) / h
        a = sx * M[:3, 0] / h
        b = sy * M[:3, 1] / h
        ref = np.concatenate([g0, a, b]) * FIX
        assert np.all(np.abs(aff - ref) <= 0.5 + 1e-6 * np.abs(ref).max() * 2**-20 + 1e-6)
        u, v = rng.integers(0, W), rng.integers(0, 600)
        q = np.array([(u - 0.5 * (W - 1)) * sx, v * sy, 0.0, 1.0])
        g_ref = (np.linalg.inv(V) @ T @ q)[:3] / h
        g = (aff[0:3] + u * aff[3:6] + v * aff[6:9]) / FIX
        assert np.all(np.abs(g - g_ref) <= (1 + u + v) * 2.0**-21 + 1e-9)


# ----------------------------------------------------------------- reconstruction

def _numpy_scatter(w, frames, poses):
    """Independent numpy re-derivation of Fig. 1's voxelisation: nearest voxel of
    every pixel, grouped per (voxel, frame)."""
    dims = w.grid.dims
    n, H, W = frames.shape
    vox_all, fr_all, val_all = [], [], []
    for f in range(n):
        aff = oracle.pixel_affine(w.grid.vol_to_world, w.grid.spacing, poses[f], W, w.frame_px)
        G, _ = voxel_coords(aff, W, H)
        c = np.floor_divide(G + 2**19, 2**20)
        ok = np.all((c >= 0) & (c < np.array(dims)), axis=-1)
        vox_all.append(flat_index(c, dims)[ok])
        fr_all.append(np.full(ok.sum(), f))
        val_all.append(frames[f][ok].astype(np.int64))
    return np.concatenate(vox_all), np.concatenate(fr_all), np.concatenate(val_all)


def test_scatter_conservation_and_grouping(tiny):
    """Sum of npix = in-grid pixel count; sum of sums = in-grid pixel total; each
    (voxel, frame) sample equals a numpy group-by; stored values are the storage
    rounding of sum / npix (numpy float32 division)."""
    frames, poses = tiny.frames[:40], tiny.frame_poses[:40]
    vox, fr, val = _numpy_scatter(tiny, frames, poses)
    vol = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, frames, poses,
                       tiny.frame_px, oracle.F32, 64)
    e = vol.export()
    assert e["npix"].sum() == vox.size
    assert e["sum"].sum() == val.sum()
    nv = int(np.prod(tiny.grid.dims))
    assert np.array_equal(e["tot_npix"], np.bincount(vox, minlength=nv))
    assert np.array_equal(e["tot_sum"], np.bincount(vox, weights=val, minlength=nv).astype(np.int64))
    key = vox * 1000 + fr
    uk, inv = np.unique(key, return_inverse=True)
    npix = np.bincount(inv)
    sums = np.bincount(inv, weights=val).astype(np.int64)
    ovox = np.repeat(np.arange(nv), np.diff(e["offsets"]))
    assert np.array_equal(ovox * 1000 + e["frame_id"], uk)  # sorted by voxel then frame id
    assert np.array_equal(e["npix"], npix)
    assert np.array_equal(e["sum"], sums)
    m32 = np.float32(sums) / np.float32(npix)
    assert np.array_equal(e["stored"], m32.astype(np.float64))
    assert np.allclose(e["mean_exact"], sums / npix, rtol=0, atol=0)


@pytest.mark.parametrize("dtype", [oracle.U8, oracle.F16, oracle.BF16, oracle.F32])
def test_storage_rounding(dtype):
    """Storage rounding = round-to-nearest-even of RN_fp32(sum/npix), against
    numpy (float32 division, float16 cast, rint) and torch (bfloat16 cast)."""
    rng = np.random.default_rng(11)
    npix = rng.integers(1, 300, 4000)
    sums = (rng.integers(0, 256, 4000) * npix + rng.integers(0, npix)).clip(0, 255 * npix)
    # exact ties for u8 (x.5) and small-denominator cases
    npix = np.concatenate([npix, [2, 2, 2, 2, 4, 8]])
    sums = np.concatenate([sums, [5, 7, 1, 509, 10, 20]])
    m32 = np.float32(sums) / np.float32(npix)
    if dtype == oracle.F32:
        ref = m32.astype(np.float64)
    elif dtype == oracle.F16:
        ref = m32.astype(np.float16).astype(np.float64)
    elif dtype == oracle.BF16:
        ref = torch.from_numpy(m32).to(torch.bfloat16).double().numpy()
    else:
        ref = np.clip(np.rint(m32), 0, 255).astype(np.float64)
    got = np.array([oracle.round_stored(s, n, dtype) for s, n in zip(sums, npix)])
    assert np.array_equal(got, ref)


def test_identity_scatter():
    """Axis-aligned frames at voxel spacing, one per voxel layer: every voxel
    holds exactly the one pixel that lands on it."""
    dims = (8, 8, 8)
    rng = np.random.default_rng(3)
    frames = rng.integers(0, 256, (8, 8, 8)).astype(np.uint8)
    poses = np.stack([synth.make_pose(np.eye(3), [3.5, 0.0, float(k)]) for k in range(8)])
    for dtype in (oracle.U8, oracle.F16, oracle.BF16, oracle.F32):
        vol = oracle.build(dims, 1.0, np.eye(4), frames, poses, (1.0, 1.0), dtype, 4)
        e = vol.export()
        assert np.array_equal(np.diff(e["offsets"]), np.ones(512, np.int64))
        # voxel (x, y, z) <- frame z, pixel (u = x, v = y)
        vals = e["stored"].reshape(8, 8, 8)  # [z][y][x]
        assert np.array_equal(vals, frames.astype(np.float64))
        assert np.array_equal(e["frame_id"].reshape(8, 8, 8), np.broadcast_to(np.arange(8)[:, None, None], (8, 8, 8)))


def test_capacity_rule(tiny):
    """With kmax = 2 each voxel keeps the 2 samples of largest npix (ties: lower
    frame id), listed by frame id; compared with a numpy group-by + lexsort."""
    frames, poses = tiny.frames, tiny.frame_poses
    vox, fr, val = _numpy_scatter(tiny, frames, poses)
    vol = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, frames, poses,
                       tiny.frame_px, oracle.U8, 2)
    e = vol.export()
    key = vox * 1000 + fr
    uk, inv = np.unique(key, return_inverse=True)
    npix = np.bincount(inv)
    kv, kf = uk // 1000, uk % 1000
    order = np.lexsort((kf, -npix, kv))  # by voxel, then npix desc, then frame asc
    kv_o, kf_o, np_o = kv[order], kf[order], npix[order]
    rank = np.zeros(order.size, np.int64)
    starts = np.r_[0, np.flatnonzero(np.diff(kv_o)) + 1]
    for s, t in zip(starts, np.r_[starts[1:], order.size]):
        rank[s:t] = np.arange(t - s)
    keep = rank < 2
    kept = np.unique(kv_o[keep] * 1000 + kf_o[keep])
    nv = int(np.prod(tiny.grid.dims))
    ovox = np.repeat(np.arange(nv), np.diff(e["offsets"]))
    assert np.array_equal(ovox * 1000 + e["frame_id"], kept)
    assert vol.n_dropped == int((~keep).sum())
    assert vol.n_overflow == int(np.sum(np.bincount(kv) > 2))


# ----------------------------------------------------------------- reslicing

def _one_sample_volume(dims, rng, quat):
    nv = int(np.prod(dims))
    vals = rng.uniform(0, 255, nv)
    vol = oracle.volume_from_samples(dims, 1.0, np.eye(4), np.arange(nv), np.zeros(nv, np.int32), vals,
                                     np.tile(quat, (nv, 1)))
    return vol, vals.reshape(dims[2], dims[1], dims[0]).transpose(2, 1, 0)  # [x, y, z]


def _interior(g, dims):
    f = np.floor(g)
    return np.all((f >= 0) & (f + 1 <= np.array(dims) - 1), axis=-1)


def test_trilinear_reduction_scipy_and_torch():
    """P-1: one sample per voxel, all aligned with the plane (Eq. 1 gives 1, 1 and
    Eq. 2 gives weight 1), TENT R = 1: the reslice equals textbook trilinear
    interpolation of the scalar volume (scipy map_coordinates order 1, and
    torch grid_sample align_corners=True)."""
    rng = np.random.default_rng(21)
    dims = (12, 10, 9)
    R = synth.random_rotation(rng)
    vol, arr = _one_sample_volume(dims, rng, quat_wxyz(R))
    W, H = 23, 17
    P = synth.make_pose(R, [2.0, 1.5, 1.0])
    P[:3, 3] = np.array([5.5, 4.5, 4.0]) - R @ np.array([0.0, 0.5 * (H - 1) * 0.4, 0.0])
    out, mask = oracle.reslice(vol, P, W, H, (0.4, 0.4))
    aff = oracle.pixel_affine(np.eye(4), 1.0, P, W, (0.4, 0.4))
    _, g = voxel_coords(aff, W, H)
    inside = _interior(g, dims)
    assert inside.sum() > 100
    ref = ndimage.map_coordinates(arr, g.reshape(-1, 3).T, order=1, mode="nearest").reshape(H, W)
    assert np.max(np.abs(out - ref)[inside]) < 1e-12 * 255
    assert np.all(mask[inside] == 1)
    # torch: input (N, C, D=z, H=y, W=x), grid (x, y, z) normalised to [-1, 1]
    t_in = torch.from_numpy(arr.transpose(2, 1, 0).copy())[None, None]
    norm = torch.from_numpy(2 * g / (np.array(dims) - 1) - 1)
    t_out = torch.nn.functional.grid_sample(t_in, norm[None, None], mode="bilinear",
                                            align_corners=True)[0, 0, 0].numpy()
    assert np.max(np.abs(out - t_out)[inside]) < 1e-11 * 255


def test_orientation_blind_closed_form():
    """P-2: k_normal = k_inplane = 0 and thresholds off, several samples with
    random orientations per voxel: out = sum_c t_c S_c / sum_c t_c m_c, with
    S_c the sum and m_c the count of voxel c's samples (numpy, vectorised)."""
    rng = np.random.default_rng(8)
    dims = (9, 8, 7)
    nv = int(np.prod(dims))
    counts = rng.integers(0, 4, nv)
    voxel = np.repeat(np.arange(nv), counts)
    vals = rng.uniform(0, 255, voxel.size)
    quats = rng.normal(size=(voxel.size, 4))
    vol = oracle.volume_from_samples(dims, 1.0, np.eye(4), voxel, np.zeros(voxel.size, np.int32), vals, quats)
    S = np.bincount(voxel, weights=vals, minlength=nv)
    m = counts.astype(np.float64)
    p = oracle.Params(k_normal=0, k_inplane=0, thr_normal_deg=180, thr_inplane_deg=180)
    W, H = 19, 15
    P = synth.make_pose(synth.random_rotation(rng), [3.7, 3.1, 2.9])
    out, mask = oracle.reslice(vol, P, W, H, (0.37, 0.41), p)
    aff = oracle.pixel_affine(np.eye(4), 1.0, P, W, (0.37, 0.41))
    _, g = voxel_coords(aff, W, H)
    f = np.floor(g).astype(np.int64)
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = f + np.array([dx, dy, dz])
                ok = np.all((c >= 0) & (c < np.array(dims)), axis=-1)
                t = np.prod(1 - np.abs(g - c), axis=-1)
                idx = np.where(ok, flat_index(c, dims), 0)
                num += np.where(ok, t * S[idx], 0)
                den += np.where(ok, t * m[idx], 0)
    has = den > 0
    assert np.array_equal(mask.astype(bool), has)
    assert np.max(np.abs(out[has] - num[has] / den[has])) < 1e-12 * 255
    assert np.all(out[~has] == 0.0)


def test_frame_self_reproduction():
    """P-3: voxel = pixel spacing, axis-aligned frames lying on voxel planes two
    voxels apart: reslicing a frame's own pose returns its pixels exactly."""
    dims = (32, 32, 32)
    h = 0.5
    rng = np.random.default_rng(4)
    n = 16
    frames = rng.integers(0, 256, (n, 32, 32)).astype(np.uint8)
    R = np.eye(3)
    poses = np.stack([synth.make_pose(R, [15.5 * h, 0.0, 2 * k * h]) for k in range(n)])
    vol = oracle.build(dims, h, np.eye(4), frames, poses, (h, h), oracle.F32, 4)
    for k in (0, 5, 15):
        out, mask = oracle.reslice(vol, poses[k], 32, 32, (h, h))
        assert np.all(mask == 1)
        assert np.array_equal(out, frames[k].astype(np.float64))


def test_rigid_motion_invariance(tiny):
    """P-4: moving the volume and every pose by one rigid transform G leaves the
    reconstruction and every reslice unchanged (orientations are compared in
    the volume frame)."""
    rng = np.random.default_rng(17)
    G = rigid(rng, 40.0)
    frames, poses = tiny.frames[::4], tiny.frame_poses[::4]
    V = tiny.grid.vol_to_world
    a = oracle.build(tiny.grid.dims, tiny.grid.spacing, V, frames, poses, tiny.frame_px, oracle.F32, 16)
    b = oracle.build(tiny.grid.dims, tiny.grid.spacing, G @ V, frames, G @ poses, tiny.frame_px, oracle.F32, 16)
    ea, eb = a.export(), b.export()
    for k in ("offsets", "frame_id", "npix", "sum"):
        assert np.array_equal(ea[k], eb[k])
    for i in (0, 3, 9):
        P = tiny.reslice_poses[i]
        assert np.array_equal(oracle.pixel_affine(V, tiny.grid.spacing, P, tiny.out_w, tiny.out_px),
                              oracle.pixel_affine(G @ V, tiny.grid.spacing, G @ P, tiny.out_w, tiny.out_px))
        oa, ma = oracle.reslice(a, P, tiny.out_w, tiny.out_h, tiny.out_px)
        ob, mb = oracle.reslice(b, G @ P, tiny.out_w, tiny.out_h, tiny.out_px)
        assert np.array_equal(ma, mb)
        assert ma.mean() > 0.05
        assert np.max(np.abs(oa - ob)) < 1e-12 * 255


@pytest.mark.parametrize("kernel,radius", [(oracle.TENT, 1), (oracle.TENT, 2), (oracle.BOX, 1),
                                           (oracle.BOX, 2), (oracle.EXP, 1), (oracle.EXP, 2)])
@pytest.mark.parametrize("normal_axis", [oracle.BEAM, oracle.ELEVATION])
def test_brute_force_8cube(kernel, radius, normal_axis):
    """P-5: the windowed oracle equals a brute force that visits every voxel of
    an 8^3 grid and every stored sample, for each distance kernel and R = 1, 2."""
    rng = np.random.default_rng(100 + 7 * kernel + radius + 31 * normal_axis)
    dims = (8, 8, 8)
    nv = 512
    counts = rng.integers(0, 3, nv)
    voxel = np.repeat(np.arange(nv), counts)
    base = synth.random_rotation(rng)
    # orientations scattered around the plane's so that thresholds both pass and fail
    rots = [synth.rot_axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, 40))) @ base
            for _ in range(voxel.size)]
    quats = np.array([quat_wxyz(R) for R in rots])
    vals = rng.uniform(0, 255, voxel.size)
    Vp = rigid(rng, 3.0)
    vol = oracle.volume_from_samples(dims, 0.9, Vp, voxel, np.arange(voxel.size, dtype=np.int32), vals, quats)
    p = oracle.Params(radius=radius, kernel=kernel, normal_axis=normal_axis, k_dist=0.7)
    W, H = 6, 5
    P = synth.make_pose(Vp[:3, :3] @ base, Vp[:3, :3] @ np.array([3.3, 3.6, 3.4]) * 0.9 + Vp[:3, 3])
    out, mask = oracle.reslice(vol, P, W, H, (0.8, 0.7), p)
    aff = oracle.pixel_affine(Vp, 0.9, P, W, (0.8, 0.7))
    _, g = voxel_coords(aff, W, H)
    samples = {}
    for s, vi in enumerate(voxel):
        key = (vi % 8, (vi // 8) % 8, vi // 64)
        samples.setdefault(key, []).append((vals[s], tuple(quats[s])))
    plane_q = tuple(quat_wxyz(Vp[:3, :3].T @ P[:3, :3]))
    n_masked = 0
    for y in range(H):
        for x in range(W):
            ref, m = _brute.reslice_pixel(dims, samples, g[y, x], plane_q, p)
            assert mask[y, x] == m
            n_masked += m
            assert abs(out[y, x] - ref) < 1e-12 * 255
    assert n_masked > 0


def test_closed_form_weights():
    """P-6 and Eq. 1 signs: values of Eq. 2 with the paper's k_normal = 10,
    k_inplane = 5, thresholds 25 and 15 degrees (Sec. 2.1), read from
    tests/golden/eq2_closed_forms.json."""
    with open(os.path.join(GOLDEN, "eq2_closed_forms.json")) as fh:
        gold = json.load(fh)
    R0 = synth.random_rotation(np.random.default_rng(2))
    I_a, I_b = 40.0, 200.0
    beam = oracle.Params()
    elev = oracle.Params(normal_axis=oracle.ELEVATION)
    # tilt about the elevation axis by 10 deg: beam and lateral both turn by 10 deg
    w10 = gold["tilt10_about_elevation_beam_reading"]
    out, m = single_voxel_case([R0, R0 @ rot_z(math.radians(10))], [I_a, I_b], R0, beam)
    assert m == 1 and abs(out - (I_a + w10 * I_b) / (1 + w10)) < 1e-12
    # elevation reading: the normal is unchanged, only the in-plane term acts
    w10e = gold["tilt10_about_elevation_elevation_reading"]
    out, m = single_voxel_case([R0, R0 @ rot_z(math.radians(10))], [I_a, I_b], R0, elev)
    assert abs(out - (I_a + w10e * I_b) / (1 + w10e)) < 1e-12
    # 20 deg about elevation: in-plane misalignment beyond 15 deg -> discarded
    out, m = single_voxel_case([R0, R0 @ rot_z(math.radians(20))], [I_a, I_b], R0, beam)
    assert m == 1 and abs(out - I_a) < 1e-12
    # a single sample returns its own intensity
    out, m = single_voxel_case([R0 @ rot_z(math.radians(5))], [I_b], R0, beam)
    assert m == 1 and abs(out - I_b) < 1e-12
    # reversed beam (180 deg about elevation): d_normal = -1 is signed -> rejected
    out, m = single_voxel_case([R0 @ rot_z(math.pi)], [I_b], R0, beam)
    assert m == 0 and out == 0.0
    # lateral mirror (180 deg about the beam): |d_inplane| = 1, d_normal = 1 -> weight 1
    out, m = single_voxel_case([R0, R0 @ rot_y(math.pi)], [I_a, I_b], R0, beam)
    assert m == 1 and abs(out - 0.5 * (I_a + I_b)) < 1e-12
    # a pure beam tilt of 20 deg about the lateral axis: weight exp(10 (cos 20 - 1))
    w20n = gold["tilt20_about_lateral_beam_reading"]
    out, m = single_voxel_case([R0, R0 @ rot_x(math.radians(20))], [0.0, 1.0], R0, beam)
    assert abs(out - w20n / (1 + w20n)) < 1e-12
    # unassigned value is configurable (NaN reading)
    out, m = single_voxel_case([R0 @ rot_z(math.pi)], [I_b], R0, oracle.Params(unassigned=float("nan")))
    assert m == 0 and math.isnan(out)


def test_threshold_edges():
    """P-7: orientations 1e-9 rad inside / outside the 25 deg normal and 15 deg
    in-plane thresholds fall on the right side (inclusive reading), and the
    weight at both thresholds is exp(10 (cos 25 - 1) + 5 (cos 15 - 1))."""
    with open(os.path.join(GOLDEN, "eq2_closed_forms.json")) as fh:
        gold = json.load(fh)
    R0 = synth.random_rotation(np.random.default_rng(9))
    p = oracle.Params()
    e = 1e-9
    tn, ti = math.radians(25), math.radians(15)
    for ang, inside in ((tn - e, True), (tn + e, False)):
        _, m = single_voxel_case([R0 @ rot_x(ang)], [1.0], R0, p)  # beam tilts, lateral fixed
        assert m == inside
    for ang, inside in ((ti - e, True), (ti + e, False)):
        _, m = single_voxel_case([R0 @ rot_y(ang)], [1.0], R0, p)  # lateral turns, beam fixed
        assert m == inside
    # both at once: R_x(25) R_y(15) gives d_normal = cos 25, d_inplane = cos 15
    out, m = single_voxel_case([R0, R0 @ rot_x(tn - e) @ rot_y(ti - e)], [0.0, 1.0], R0, p)
    w = out / (1 - out)
    assert m == 1 and abs(w - gold["both_thresholds"]) < 1e-7


def test_convexity_and_constant_field():
    """P-8: each output lies between the smallest and largest contributing
    sample; a constant volume reslices to the constant wherever covered."""
    rng = np.random.default_rng(12)
    dims = (10, 10, 10)
    nv = 1000
    counts = rng.integers(0, 3, nv)
    voxel = np.repeat(np.arange(nv), counts)
    base = synth.random_rotation(rng)
    quats = np.array([quat_wxyz(synth.rot_axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, 30))) @ base)
                      for _ in range(voxel.size)])
    vals = rng.uniform(0, 255, voxel.size)
    P = synth.make_pose(base, [4.5, 4.5, 4.5])
    vol = oracle.volume_from_samples(dims, 1.0, np.eye(4), voxel, np.zeros(voxel.size, np.int32), vals, quats)
    out, mask = oracle.reslice(vol, P, 16, 16, (0.6, 0.6))
    aff = oracle.pixel_affine(np.eye(4), 1.0, P, 16, (0.6, 0.6))
    _, g = voxel_coords(aff, 16, 16)
    lo_v = np.full(nv, np.inf)
    hi_v = np.full(nv, -np.inf)
    np.minimum.at(lo_v, voxel, vals)
    np.maximum.at(hi_v, voxel, vals)
    f = np.floor(g).astype(np.int64)
    lo = np.full((16, 16), np.inf)
    hi = np.full((16, 16), -np.inf)
    for d in np.ndindex(2, 2, 2):
        c = f + np.array(d)
        ok = np.all((c >= 0) & (c < np.array(dims)), axis=-1)
        idx = np.where(ok, flat_index(c, dims), 0)
        lo = np.where(ok, np.minimum(lo, lo_v[idx]), lo)
        hi = np.where(ok, np.maximum(hi, hi_v[idx]), hi)
    mk = mask.astype(bool)
    assert mk.sum() > 50
    assert np.all(out[mk] >= lo[mk] - 1e-9) and np.all(out[mk] <= hi[mk] + 1e-9)
    const = oracle.volume_from_samples(dims, 1.0, np.eye(4), voxel, np.zeros(voxel.size, np.int32),
                                       np.full(voxel.size, 77.25), quats)
    oc, mc = oracle.reslice(const, P, 16, 16, (0.6, 0.6))
    assert np.array_equal(mc, mask)
    assert np.max(np.abs(oc[mk] - 77.25)) < 1e-12


@pytest.mark.parametrize("kernel,radius", [(oracle.TENT, 1), (oracle.TENT, 2), (oracle.BOX, 1)])
def test_footprint_numpy(tiny, kernel, radius):
    """Footprint = distinct in-grid window voxels over all pixels (numpy np.unique)."""
    g = tiny.grid
    for P in tiny.reslice_poses[[0, 9, 14]]:
        aff = oracle.pixel_affine(g.vol_to_world, g.spacing, P, tiny.out_w, tiny.out_px)
        G, _ = voxel_coords(aff, tiny.out_w, tiny.out_h)
        base = np.floor_divide(G + (2**19 if kernel == oracle.BOX else 0), 2**20)
        lo = base - radius if kernel == oracle.BOX else base - radius + 1
        span = 2 * radius + 1 if kernel == oracle.BOX else 2 * radius
        idx = []
        for d in np.ndindex(span, span, span):
            c = lo + np.array(d)
            ok = np.all((c >= 0) & (c < np.array(g.dims)), axis=-1)
            idx.append(flat_index(c, g.dims)[ok])
        ref = np.unique(np.concatenate(idx)).size
        assert oracle.footprint(g.dims, g.spacing, g.vol_to_world, P, tiny.out_w, tiny.out_h, tiny.out_px,
                                radius, kernel) == ref


def test_scalar_comparator(tiny):
    """Mean compounding + trilinear: where all 8 corners are occupied it equals
    scipy's trilinear interpolation of the RN_fp32 mean volume."""
    g = tiny.grid
    vol = oracle.build(g.dims, g.spacing, g.vol_to_world, tiny.frames, tiny.frame_poses, tiny.frame_px)
    e = vol.export()
    occ = e["tot_npix"] > 0
    mean = np.zeros(e["tot_npix"].size)
    mean[occ] = (np.float32(e["tot_sum"][occ]) / np.float32(e["tot_npix"][occ])).astype(np.float64)
    arr = mean.reshape(g.dims[2], g.dims[1], g.dims[0]).transpose(2, 1, 0)
    occ3 = occ.reshape(g.dims[2], g.dims[1], g.dims[0]).transpose(2, 1, 0)
    P = tiny.reslice_poses[2]
    out, mask = oracle.reslice_scalar(vol, P, tiny.out_w, tiny.out_h, tiny.out_px)
    aff = oracle.pixel_affine(g.vol_to_world, g.spacing, P, tiny.out_w, tiny.out_px)
    _, gc = voxel_coords(aff, tiny.out_w, tiny.out_h)
    f = np.floor(gc).astype(np.int64)
    full = _interior(gc, g.dims)
    fi = np.where(full[..., None], f, 0)
    for d in np.ndindex(2, 2, 2):
        c = fi + np.array(d)
        full &= occ3[c[..., 0], c[..., 1], c[..., 2]]
    assert full.sum() > 1000
    ref = ndimage.map_coordinates(arr, gc.reshape(-1, 3).T, order=1).reshape(gc.shape[:2])
    assert np.max(np.abs(out - ref)[full]) < 1e-9
    assert np.all(mask[full] == 1)


# ----------------------------------------------------------------- per-pixel samples

def test_per_pixel_samples_literal(tiny):
    """The per-pixel reading of Sec. 2.1's storage, built literally: a volume
    holding every in-grid pixel as its own sample (numpy voxelisation, the
    frame's quaternion from scipy), resliced one sample per entry, equals the
    merged volume resliced with each sample weighted by its npix."""
    w = tiny
    g = w.grid
    sel = np.arange(0, 200, 7)
    frames, poses = w.frames[sel], w.frame_poses[sel]
    merged = oracle.build(g.dims, g.spacing, g.vol_to_world, frames, poses, w.frame_px, oracle.F32, 16)
    assert merged.n_overflow == 0
    H, W = frames.shape[1:]
    vox, fid, val, quat = [], [], [], []
    for k, T in enumerate(poses):
        aff = oracle.pixel_affine(g.vol_to_world, g.spacing, T, W, w.frame_px)
        G, _ = voxel_coords(aff, W, H)
        c = np.floor_divide(G + 2**19, 2**20)
        ok = np.all((c >= 0) & (c < np.array(g.dims)), axis=-1)
        vi = flat_index(c, g.dims)[ok]
        vox.append(vi)
        fid.append(np.full(vi.size, k, np.int32))
        val.append(frames[k][ok].astype(np.float64))
        q = quat_wxyz(g.vol_to_world[:3, :3].T @ T[:3, :3])
        quat.append(np.repeat(q[None], vi.size, axis=0))
    vox, fid, val, quat = (np.concatenate(x) for x in (vox, fid, val, quat))
    order = np.lexsort((fid, vox))
    literal = oracle.volume_from_samples(g.dims, g.spacing, g.vol_to_world, vox[order], fid[order], val[order],
                                         quat[order])
    n_diff = 0
    for T in w.reslice_poses[[0, 5, 10]]:
        a, am = oracle.reslice(literal, T, w.out_w, w.out_h, w.out_px, oracle.Params(radius=1))
        b, bm = oracle.reslice(merged, T, w.out_w, w.out_h, w.out_px, oracle.Params(per_pixel=True, use_exact=True))
        c_, _ = oracle.reslice(merged, T, w.out_w, w.out_h, w.out_px, oracle.Params(use_exact=True))
        assert np.array_equal(am, bm)
        assert np.max(np.abs(a - b)) < 1e-9
        n_diff += int((np.abs(c_ - b) > 1e-3).sum())
    assert n_diff > 100  # the npix weighting matters: mean-per-frame samples give other images


# ----------------------------------------------------------------- hole filling (comparator)

def test_compounded_and_values_reslice(tiny):
    """The compounded volume is the RN_fp32 mean of every voxel's pixels (NaN
    where empty), and the scalar-volume reslice of it is the mean-compounding
    comparator exactly."""
    g = tiny.grid
    vol = oracle.build(g.dims, g.spacing, g.vol_to_world, tiny.frames[:80], tiny.frame_poses[:80], tiny.frame_px)
    e = vol.export()
    occ = e["tot_npix"] > 0
    vals = oracle.compounded(vol)
    assert np.array_equal(np.isnan(vals), ~occ)
    assert np.array_equal(vals[occ], (np.float32(e["tot_sum"][occ]) / np.float32(e["tot_npix"][occ])).astype(np.float64))
    for P in tiny.reslice_poses[[0, 6, 13]]:
        a, am = oracle.reslice_scalar(vol, P, tiny.out_w, tiny.out_h, tiny.out_px, unassigned=-3.0)
        b, bm = oracle.reslice_values(g.dims, g.spacing, g.vol_to_world, vals, P, tiny.out_w, tiny.out_h,
                                      tiny.out_px, unassigned=-3.0)
        assert np.array_equal(am, bm)
        assert np.max(np.abs(a - b)) < 1e-12


def _empty_volume(dims):
    return oracle.volume_from_samples(dims, 1.0, np.eye(4), np.zeros(0, np.int64), np.zeros(0, np.int32),
                                      np.zeros(0), np.zeros((0, 4)))


def test_fill_holes_closed_forms():
    """Hand-computed fills: one occupied voxel fills its 26 neighbours with its
    value; between two occupied voxels the 1/distance weights give the plain
    mean at equal distances and (10 + 40/sqrt 5)/(1 + 1/sqrt 5) at distances 1
    and sqrt 5; min_neighbours leaves a voxel with fewer occupied neighbours
    empty; occupied voxels keep their value."""
    dims = (7, 7, 7)
    vol = _empty_volume(dims)
    idx = lambda x, y, z: x + 7 * (y + 7 * z)
    one = np.full(343, np.nan)
    one[idx(3, 3, 3)] = 10.0
    f = oracle.fill_holes(vol, one, 1, 1)
    cube = np.zeros(343, bool)
    for d in np.ndindex(3, 3, 3):
        cube[idx(2 + d[0], 2 + d[1], 2 + d[2])] = True
    assert np.all(f[cube] == 10.0)
    assert np.all(np.isnan(f[~cube]))
    two = np.full(343, np.nan)
    two[idx(2, 3, 3)], two[idx(4, 3, 3)] = 10.0, 40.0
    f1 = oracle.fill_holes(vol, two, 1, 1)
    assert f1[idx(2, 3, 3)] == 10.0 and f1[idx(4, 3, 3)] == 40.0
    assert abs(f1[idx(3, 3, 3)] - 25.0) < 1e-13
    assert abs(f1[idx(3, 4, 3)] - 25.0) < 1e-13
    assert f1[idx(2, 4, 3)] == 10.0          # only the near voxel lies in its 3^3 cube
    f2 = oracle.fill_holes(vol, two, 2, 1)
    r5 = 1.0 / math.sqrt(5.0)
    assert abs(f2[idx(2, 4, 3)] - (10.0 + 40.0 * r5) / (1.0 + r5)) < 1e-13
    fm = oracle.fill_holes(vol, two, 1, 2)
    assert np.isnan(fm[idx(2, 4, 3)]) and abs(fm[idx(3, 3, 3)] - 25.0) < 1e-13


@pytest.mark.parametrize("radius,min_nb", [(1, 1), (1, 5), (2, 1), (2, 9)])
def test_fill_holes_convolution(radius, min_nb):
    """Whole-volume check by convolution (scipy): filled = conv(S occ, K) /
    conv(occ, K) with K = 1/distance (0 at the centre), where conv(occ, 1) >=
    min_neighbours; occupied voxels unchanged, the rest empty."""
    rng = np.random.default_rng(70 + 3 * radius + min_nb)
    dims = (12, 10, 9)
    n = int(np.prod(dims))
    occ = rng.random(n) < 0.12
    vals = np.where(occ, rng.uniform(0, 255, n), np.nan)
    got = oracle.fill_holes(_empty_volume(dims), vals, radius, min_nb)
    k = 2 * radius + 1
    dz, dy, dx = np.meshgrid(*(np.arange(k) - radius,) * 3, indexing="ij")
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    K = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    ones = (d > 0).astype(np.float64)
    occ3 = occ.reshape(dims[2], dims[1], dims[0]).astype(np.float64)
    S3 = np.where(occ, vals, 0.0).reshape(dims[2], dims[1], dims[0])
    num = ndimage.convolve(S3 * occ3, K, mode="constant", cval=0.0).reshape(-1)
    den = ndimage.convolve(occ3, K, mode="constant", cval=0.0).reshape(-1)
    cnt = np.rint(ndimage.convolve(occ3, ones, mode="constant", cval=0.0)).reshape(-1)
    fill = (~occ) & (cnt >= max(min_nb, 1))
    ref = np.where(occ, vals, np.nan)
    ref[fill] = num[fill] / den[fill]
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.max(np.abs(got[ok] - ref[ok])) < 1e-10
    assert fill.sum() > 50
    if (radius, min_nb) != (2, 1):  # a 5^3 cube always holds an occupied voxel here
        assert (~occ & ~fill).sum() > 5


# ----------------------------------------------------------------- curvilinear probes
#
# A curvilinear probe's beams fan out from an apex of the image plane: the
# beam through image point p runs along (p - a) / |p - a|.  These pins derive
# the expected axes from positions and plain unit vectors (no angles, no
# quaternion products), the oracle from steering angles and quaternions.

FAN_APEX = (0.7, -12.0)


def fan_beam(px, py, apex):
    """unit beam direction(s) in image coordinates for a fan from apex"""
    dx, dy = np.asarray(px, np.float64) - apex[0], np.asarray(py, np.float64) - apex[1]
    r = np.hypot(dx, dy)
    return dx / r, dy / r


def voxel_centres(idx, dims, spacing, V):
    c = np.stack([idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])], axis=-1)
    return (V[:3, :3] @ (spacing * c.astype(np.float64)).T).T + V[:3, 3]


def quat_matrices(q):
    return Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=-1)).as_matrix()


def test_curvilinear_sample_axes(tiny):
    """Every sample of a curvilinear frame carries its frame's axes turned in
    the image plane so that image y runs from the apex through the voxel
    centre (projected into the frame): beam R (u_x, u_y, 0), lateral
    R (u_y, -u_x, 0), elevation R z, in the volume frame.  Samples, npix and
    sums are those of the linear build."""
    w = tiny
    n = 6
    apex = (1.5, -25.0)
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames[:n], w.frame_poses[:n],
                       w.frame_px, probe=oracle.CURVILINEAR, apex_mm=apex)
    lin = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames[:n], w.frame_poses[:n],
                       w.frame_px)
    e, el = vol.export(), lin.export()
    for k in ("offsets", "frame_id", "npix", "sum", "stored"):
        assert np.array_equal(e[k], el[k]), k
    V = w.grid.vol_to_world
    vox = np.repeat(np.arange(len(e["offsets"]) - 1), np.diff(e["offsets"]))
    ctr = voxel_centres(vox, w.grid.dims, w.grid.spacing, V)
    T = w.frame_poses[:n][e["frame_id"]]
    p = np.einsum("nki,nk->ni", T[:, :3, :3], ctr - T[:, :3, 3])  # R_f^T (c - t_f)
    ux, uy = fan_beam(p[:, 0], p[:, 1], apex)
    zero = np.zeros_like(ux)
    R = np.einsum("ji,njk->nik", V[:3, :3], T[:, :3, :3])        # R_v^T R_f
    beam = np.einsum("nij,nj->ni", R, np.stack([ux, uy, zero], -1))
    lat = np.einsum("nij,nj->ni", R, np.stack([uy, -ux, zero], -1))
    M = quat_matrices(e["quat"])
    assert vox.size > 1000
    assert np.max(np.abs(M[:, :, 1] - beam)) < 1e-12
    assert np.max(np.abs(M[:, :, 0] - lat)) < 1e-12
    assert np.max(np.abs(M[:, :, 2] - R[:, :, 2])) < 1e-12
    # the fan really turns the beams: tens of degrees across the frame
    tilt = np.degrees(np.arccos(np.clip(np.einsum("ni,ni->n", M[:, :, 1], R[:, :, 1]), -1, 1)))
    assert tilt.max() > 15.0


def test_curvilinear_limits_and_mask_identity(tiny):
    """A far apex is the linear probe; an all-ones pixel mask, and an explicit
    LINEAR probe, change nothing."""
    w = tiny
    n = 4
    args = (w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames[:n], w.frame_poses[:n], w.frame_px)
    ref = oracle.build(*args).export()
    far = oracle.build(*args, probe=oracle.CURVILINEAR, apex_mm=(0.0, -1e9)).export()
    assert np.max(np.abs(quat_matrices(far["quat"]) - quat_matrices(ref["quat"]))) < 1e-7
    H, W = w.frames.shape[1:]
    for e in (oracle.build(*args, pixel_mask=np.ones((H, W), np.uint8)).export(),
              oracle.build(*args, probe=oracle.LINEAR, apex_mm=(3.0, -5.0)).export()):
        for k in ref:
            assert np.array_equal(ref[k], e[k]), k


def test_pixel_mask_voxelisation(tiny):
    """Masked pixels are never voxelised: per-voxel totals and per-(voxel, frame)
    samples equal a numpy group-by over the unmasked pixels only."""
    w = tiny
    n = 5
    H, W = w.frames.shape[1:]
    rng = np.random.default_rng(41)
    pm = (rng.random((H, W)) < 0.6).astype(np.uint8)
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames[:n], w.frame_poses[:n],
                       w.frame_px, pixel_mask=pm)
    e = vol.export()
    dims = w.grid.dims
    nv = int(np.prod(dims))
    tot_n, tot_s = np.zeros(nv, np.int64), np.zeros(nv, np.int64)
    keys = {}
    for f in range(n):
        aff = oracle.pixel_affine(w.grid.vol_to_world, w.grid.spacing, w.frame_poses[f], W, w.frame_px)
        G, _ = voxel_coords(aff, W, H)
        c = np.floor_divide(G + 2**19, 2**20)
        ok = np.all((c >= 0) & (c < np.array(dims)), axis=-1) & (pm > 0)
        vi = flat_index(c, dims)[ok]
        val = w.frames[f][ok].astype(np.int64)
        np.add.at(tot_n, vi, 1)
        np.add.at(tot_s, vi, val)
        for a, b in zip(vi, val):
            k = (int(a), f)
            s = keys.setdefault(k, [0, 0])
            s[0] += 1
            s[1] += int(b)
    assert np.array_equal(e["tot_npix"], tot_n)
    assert np.array_equal(e["tot_sum"], tot_s)
    vox = np.repeat(np.arange(nv), np.diff(e["offsets"]))
    got = {(int(a), int(f)): [int(m), int(s)] for a, f, m, s in zip(vox, e["frame_id"], e["npix"], e["sum"])}
    assert got == keys
    assert tot_n.sum() < 0.7 * H * W * n


def _coplanar_case(seed, frame_curv, out_curv):
    """One random frame in a rotated 40^3 grid, resliced at its own pose."""
    rng = np.random.default_rng(seed)
    h, dims = 0.6, (40, 40, 40)
    V = synth.make_pose(synth.random_rotation(rng), rng.uniform(-5, 5, 3))
    W, H, px = 48, 40, (0.3, 0.3)
    Rrel = synth.random_rotation(rng)
    c0 = np.array([12.0, 12.0, 12.0]) + rng.uniform(-0.3, 0.3, 3)
    Tv = synth.make_pose(Rrel, c0 - Rrel @ np.array([0.0, 6.0, 0.0]))
    T = V @ Tv
    frame = rng.integers(0, 256, (1, H, W)).astype(np.uint8)
    vol = oracle.build(dims, h, V, frame, T[None], px, probe=oracle.CURVILINEAR if frame_curv else None,
                       apex_mm=FAN_APEX)
    return vol, V, T, W, H, px, dims, h


@pytest.mark.parametrize("frame_curv,out_curv", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("normal_axis", [oracle.BEAM, oracle.ELEVATION])
def test_curvilinear_coplanar_brute_force(frame_curv, out_curv, normal_axis):
    """Frame and virtual plane share one pose, so every sample's axes and every
    pixel's axes differ by a turn in the plane: d_normal = u_s . u_p (beam) or
    1 (elevation), d_inplane = |u_s . u_p|, with u the unit beams of the fan
    (u = (0, 1) for a linear probe).  Whole plane against a numpy brute force:
    masks exact, values to 1e-12."""
    vol, V, T, W, H, px, dims, h = _coplanar_case(500 + 2 * frame_curv + out_curv, frame_curv, out_curv)
    p = oracle.Params(normal_axis=normal_axis, probe=oracle.CURVILINEAR if out_curv else oracle.LINEAR,
                      apex_mm=FAN_APEX)
    out, mask = oracle.reslice(vol, T, W, H, px, p)
    e = vol.export()
    aff = oracle.pixel_affine(V, h, T, W, px)
    _, g = voxel_coords(aff, W, H)
    # samples: value and beam per voxel (one frame: at most one sample per voxel)
    nv = int(np.prod(dims))
    cnt = np.diff(e["offsets"])
    has = cnt > 0
    val = np.zeros(nv)
    val[has] = e["stored"][e["offsets"][:-1][has]]
    us = np.zeros((nv, 2))
    us[:, 1] = 1.0
    if frame_curv:
        idx = np.nonzero(has)[0]
        ctr = voxel_centres(idx, dims, h, V)
        q = (T[:3, :3].T @ (ctr - T[:3, 3]).T).T
        us[idx] = np.stack(fan_beam(q[:, 0], q[:, 1], FAN_APEX), -1)
    cn, ci = math.cos(math.radians(25.0)), math.cos(math.radians(15.0))
    n_on = 0
    for y in range(H):
        for x in range(W):
            up = (0.0, 1.0)
            if out_curv:
                up = fan_beam((x - 0.5 * (W - 1)) * px[0], y * px[1], FAN_APEX)
            f = np.floor(g[y, x]).astype(np.int64)
            num = den = 0.0
            for k in range(8):
                c = f + np.array([k & 1, (k >> 1) & 1, k >> 2])
                if np.any(c < 0) or np.any(c >= dims):
                    continue
                vi = int(c[0] + dims[0] * (c[1] + dims[1] * c[2]))
                if not has[vi]:
                    continue
                t = np.prod(1.0 - np.abs(g[y, x] - c))
                cosd = us[vi, 0] * up[0] + us[vi, 1] * up[1]
                dn = cosd if normal_axis == oracle.BEAM else 1.0
                di = abs(cosd)
                assert abs(dn - cn) > 1e-9 and abs(di - ci) > 1e-9
                if dn < cn or di < ci:
                    continue
                wgt = math.exp(10.0 * (dn - 1.0) + 5.0 * (di - 1.0))
                num += t * wgt * val[vi]
                den += t * wgt
            m = 1 if den > 0 else 0
            assert mask[y, x] == m, (x, y)
            n_on += m
            if m:
                assert abs(out[y, x] - num / den) < 1e-12 * 255
    # one fan against a linear probe keeps and drops pixels; two matching fans keep all
    assert n_on > 0.2 * W * H
    assert (n_on < 0.95 * W * H) == (frame_curv != out_curv)


@pytest.mark.parametrize("normal_axis,kernel,radius", [(oracle.BEAM, oracle.TENT, 1),
                                                       (oracle.ELEVATION, oracle.BOX, 1),
                                                       (oracle.BEAM, oracle.EXP, 2)])
def test_curvilinear_plane_brute_force_8cube(normal_axis, kernel, radius):
    """A curvilinear virtual plane in general position over hand-made samples:
    each pixel's plane orientation is R_plane times the in-plane turn whose
    columns are (u_y, -u_x, 0), (u_x, u_y, 0), z, built as a matrix and
    handed to the every-voxel brute force."""
    rng = np.random.default_rng(900 + 10 * normal_axis + kernel)
    dims = (8, 8, 8)
    nv = 512
    counts = rng.integers(0, 3, nv)
    voxel = np.repeat(np.arange(nv), counts)
    base = synth.random_rotation(rng)
    rots = [synth.rot_axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, 40))) @ base
            for _ in range(voxel.size)]
    quats = np.array([quat_wxyz(R) for R in rots])
    vals = rng.uniform(0, 255, voxel.size)
    Vp = rigid(rng, 3.0)
    vol = oracle.volume_from_samples(dims, 0.9, Vp, voxel, np.arange(voxel.size, dtype=np.int32), vals, quats)
    apex = (0.4, -2.5)
    p = oracle.Params(radius=radius, kernel=kernel, normal_axis=normal_axis, k_dist=0.7,
                      probe=oracle.CURVILINEAR, apex_mm=apex)
    W, H, px = 6, 5, (0.8, 0.7)
    P = synth.make_pose(Vp[:3, :3] @ base, Vp[:3, :3] @ np.array([3.3, 3.6, 3.4]) * 0.9 + Vp[:3, 3])
    out, mask = oracle.reslice(vol, P, W, H, px, p)
    aff = oracle.pixel_affine(Vp, 0.9, P, W, px)
    _, g = voxel_coords(aff, W, H)
    samples = {}
    for s, vi in enumerate(voxel):
        samples.setdefault((vi % 8, (vi // 8) % 8, vi // 64), []).append((vals[s], tuple(quats[s])))
    Rp = Vp[:3, :3].T @ P[:3, :3]
    n_on = 0
    for y in range(H):
        for x in range(W):
            ux, uy = fan_beam((x - 0.5 * (W - 1)) * px[0], y * px[1], apex)
            turn = np.array([[uy, ux, 0.0], [-ux, uy, 0.0], [0.0, 0.0, 1.0]])
            ref, m = _brute.reslice_pixel(dims, samples, g[y, x], tuple(quat_wxyz(Rp @ turn)), p)
            assert mask[y, x] == m
            n_on += m
            assert abs(out[y, x] - ref) < 1e-12 * 255
    assert n_on > 0
