"""Hole filling of the mean-compounding comparator (the PLUS baseline of
Sec. 2.2 runs mean compounding with hole-filling) on the CUDA path against the
FP64 oracle.  Which voxels get filled is an integer decision: the empty-voxel
pattern must match exactly.  A filled value is an FP32 quotient of two sums of
at most n = (2r+1)^3 - 1 positive FMA terms (the compounded values themselves
are exact RN_fp32 means, the 1/d weights correctly rounded), so it is within
(2n + 2) 2^-24 relative of the FP64 value.  Reslices of the filled volume are
convex blends of those: masks exact, values within 1e-5 plus that bound,
relative."""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
from gpu_helpers import DEV, gpu_session, new_outputs

pytestmark = pytest.mark.gpu


def fill_tol(radius):
    n = (2 * radius + 1) ** 3 - 1
    return (2 * n + 2) * 2.0 ** -24


@pytest.fixture(scope="module")
def scalar_pair(tiny):
    # half the frames: a sparser volume with more holes
    frames, poses = tiny.frames[::2], tiny.frame_poses[::2]
    s = gpu_session(tiny, dare.DARE_U8, 4, flags=dare.DARE_SESSION_SCALAR, frames=frames, poses=poses)
    vol = oracle.build(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, frames, poses, tiny.frame_px,
                       oracle.U8, 4)
    yield s, vol
    s.close()


@pytest.mark.parametrize("radius,min_nb", [(1, 1), (1, 6), (2, 1), (3, 20)])
def test_fill_holes_volume(tiny, scalar_pair, radius, min_nb):
    s, vol = scalar_pair
    s.fill_holes(radius, min_nb)
    got = s.read_filled().astype(np.float64)
    ref = oracle.fill_holes(vol, oracle.compounded(vol), radius, min_nb)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.all(np.abs(got[ok] - ref[ok]) <= fill_tol(radius) * np.maximum(np.abs(ref[ok]), 1.0))
    comp = oracle.compounded(vol)
    n_filled = int((np.isnan(comp) & ok).sum())
    assert n_filled > 1000


@pytest.mark.parametrize("radius,min_nb", [(1, 1), (2, 4)])
def test_reslice_filled_parity(tiny, scalar_pair, radius, min_nb):
    s, vol = scalar_pair
    s.fill_holes(radius, min_nb)
    ref_vals = oracle.fill_holes(vol, oracle.compounded(vol), radius, min_nb)
    g = tiny.grid
    gained = 0
    for T in tiny.reslice_poses[[0, 4, 9, 15]]:
        out, mask = new_outputs(tiny.out_w, tiny.out_h)
        s.reslice_scalar_filled(T, out, mask, tiny.out_px, unassigned=-1.0)
        torch.cuda.synchronize()
        ref, rm = oracle.reslice_values(g.dims, g.spacing, g.vol_to_world, ref_vals, T, tiny.out_w, tiny.out_h,
                                        tiny.out_px, unassigned=-1.0)
        bits = dare.unpack_mask(mask.cpu().numpy(), tiny.out_w)
        assert np.array_equal(bits, rm)
        o = out.cpu().numpy()
        cov = rm.astype(bool)
        assert np.all(np.abs(o[cov] - ref[cov]) <= (1e-5 + fill_tol(radius)) * np.maximum(np.abs(ref[cov]), 1.0))
        assert np.all(o[~cov] == -1.0)
        _, m0 = oracle.reslice_scalar(vol, T, tiny.out_w, tiny.out_h, tiny.out_px)
        gained += int(rm.sum()) - int(m0.sum())
    assert gained > 0  # filling covers pixels the plain comparator leaves unassigned


def test_fill_holes_state_and_errors(tiny, scalar_pair):
    s, _ = scalar_pair
    out, mask = new_outputs(16, 16)
    for args in ((0, 1), (9, 1), (1, 27), (1, -1)):
        with pytest.raises(dare.DareError) as ei:
            s.fill_holes(*args)
        assert ei.value.status == dare.DARE_E_INVALID
    t = gpu_session(tiny, dare.DARE_U8, 4, flags=dare.DARE_SESSION_SCALAR, frames=tiny.frames[:3],
                    poses=tiny.frame_poses[:3])
    with pytest.raises(dare.DareError) as ei:  # never filled
        t.reslice_scalar_filled(tiny.reslice_poses[0], out, mask, tiny.out_px)
    assert ei.value.status == dare.DARE_E_STATE
    t.fill_holes(1, 1)
    t.reslice_scalar_filled(tiny.reslice_poses[0], out, mask, tiny.out_px)
    t.build(torch.from_numpy(np.ascontiguousarray(tiny.frames[3:5])).to(DEV), tiny.frame_poses[3:5], tiny.frame_px)
    with pytest.raises(dare.DareError) as ei:  # stale after a build
        t.reslice_scalar_filled(tiny.reslice_poses[0], out, mask, tiny.out_px)
    assert ei.value.status == dare.DARE_E_STATE
    t.close()
    u = gpu_session(tiny, dare.DARE_U8, 4, frames=tiny.frames[:2], poses=tiny.frame_poses[:2])
    with pytest.raises(dare.DareError) as ei:  # no scalar totals
        u.fill_holes(1, 1)
    assert ei.value.status == dare.DARE_E_STATE
    u.close()
