"""GPU parity of the full rebuild (a reset volume rebuilt from its frames, Fig. 1):
records, npix rows and scalar totals bit-exact against the FP64 oracle.

After a reset the next build's finalize writes every voxel of the volume (empty
ones with the empty record) in whole 256-voxel runs, a shorter tail run thread
by thread.  The cases below cover every storage type and capacity, grids whose
voxel count is not a multiple of the run, thin grids, voxels whose entries
overflow their bucket with the capacity rule, and a rebuild given in two calls.
"""
import types

import numpy as np
import pytest
import torch

import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import DEV, oracle_dense, oracle_volume

pytestmark = pytest.mark.gpu

DTYPES = [dare.DARE_U8, dare.DARE_F16, dare.DARE_BF16, dare.DARE_F32]


def rebuilt(w, dtype, K, first=50, flags=0):
    """A session that held `first` frames, was reset and rebuilt from all of w's frames."""
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=K,
                     flags=dare.DARE_SESSION_SCALAR | flags)
    ft = torch.from_numpy(np.ascontiguousarray(w.frames)).to(DEV)
    s.build(ft[:first], w.frame_poses[:first], w.frame_px)
    s.reset()
    s.build(ft, w.frame_poses, w.frame_px)
    torch.cuda.synchronize()
    return s


def check_against_oracle(s, w, dtype, K):
    vol = oracle_volume(w, dtype, K)
    ids, vals, npix, e = oracle_dense(vol, K, dtype)
    g = s.read_records(npix=True, scalar=True)
    assert np.array_equal(g["frame_ids"], ids)
    assert np.array_equal(g["values"].view(np.uint8), vals.view(np.uint8))
    assert np.array_equal(g["npix"], npix)
    assert np.array_equal(g["scalar_count"], e["tot_npix"].astype(np.uint32))
    assert np.array_equal(g["scalar_sum"], e["tot_sum"].astype(np.uint32))
    assert s.info().overflow_voxels == vol.n_overflow
    return e


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [4, 8, 12, 16])
def test_rebuild_records_bit_exact(tiny, dtype, K):
    """Every storage type and capacity: the capacity rule (K = 4 with up to 5
    samples a voxel) and frames split across tiles (entries of one frame merged)."""
    s = rebuilt(tiny, dtype, K)
    check_against_oracle(s, tiny, dtype, K)
    s.close()


@pytest.mark.parametrize("dims", [(61, 57, 59), (17, 9, 33), (8, 8, 8), (3, 70, 5)])
def test_rebuild_ragged_grids(tiny, dims):
    """Grids whose voxel counts are not multiples of the 256-voxel run (a short
    tail run) and thin grids."""
    g = synth.centred_grid(dims, 32.0 / max(dims))
    w = types.SimpleNamespace(grid=g, frames=tiny.frames, frame_poses=tiny.frame_poses, frame_px=tiny.frame_px)
    s = rebuilt(w, dare.DARE_F32, 8)
    check_against_oracle(s, w, dare.DARE_F32, 8)
    s.close()


@pytest.mark.parametrize("K", [4, 12])
@pytest.mark.parametrize("host", [False, True])
def test_rebuild_dense_voxels(tiny, K, host):
    """Coarse voxels reached by many frames and tiles: entries past a voxel's
    bucket of 8 (its overflow range: about 1000 voxels with 9 to 16 entries, which
    the second finalize pass sorts in registers, and about 300 with up to 54, which
    take the general merge) and more samples than K (the capacity rule); records
    in device memory and in mapped host memory."""
    g = synth.centred_grid((12, 12, 12), 2.5)
    w = types.SimpleNamespace(grid=g, frames=tiny.frames, frame_poses=tiny.frame_poses, frame_px=(0.2, 0.2))
    for dtype in (dare.DARE_F32, dare.DARE_U8):
        s = rebuilt(w, dtype, K, first=10, flags=dare.DARE_SESSION_HOST_VOLUME if host else 0)
        check_against_oracle(s, w, dtype, K)
        assert oracle_volume(w, dtype, 12).n_overflow > 0  # more than 12 samples, so more than 8 entries
        s.close()


def test_rebuild_equals_fresh_build(tiny):
    """A reset + rebuild given in two calls (a full write, then a merge into the
    stored records) and one build into a new session give the same records,
    npix rows and totals, on the working storage (f32, K = 12)."""
    ft = torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV)
    a = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=12,
                     flags=dare.DARE_SESSION_SCALAR)
    a.build(ft, tiny.frame_poses, tiny.frame_px)
    b = rebuilt(tiny, dare.DARE_F32, 12, first=200)
    b.reset()
    b.build(ft[:120], tiny.frame_poses[:120], tiny.frame_px)
    b.build(ft[120:], tiny.frame_poses[120:], tiny.frame_px)
    ra, rb = a.read_records(npix=True, scalar=True), b.read_records(npix=True, scalar=True)
    for k in ("frame_ids", "npix", "scalar_sum", "scalar_count"):
        assert np.array_equal(ra[k], rb[k]), k
    assert np.array_equal(ra["values"].view(np.uint32), rb["values"].view(np.uint32))
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["large_boxes", "large_steps"])
def test_rebuild_fine_grids(tiny, case):
    """Voxels much finer than pixels.  At 2.5 voxels per pixel a 32 x 64 frame
    region spans a voxel box far past 4096 cells, so the count pass sums it in
    the hash table, one 32-row band at a time; at about 36 voxels per pixel the
    pixel steps exceed 2^25 in fixed point, so pixel coordinates are evaluated in
    int64 instead of int32 steps from each band's origin.  A reset + rebuild
    and a build into a new session both equal the oracle."""
    if case == "large_boxes":
        g = synth.centred_grid((96, 96, 96), 0.1)
    else:
        g = synth.centred_grid((160, 160, 160), 0.006)
    w = types.SimpleNamespace(grid=g, frames=tiny.frames, frame_poses=tiny.frame_poses, frame_px=tiny.frame_px)
    s = rebuilt(w, dare.DARE_F32, 8)
    e = check_against_oracle(s, w, dare.DARE_F32, 8)
    assert e["tot_npix"].sum() > 0
    s.close()
    fresh = dare.Session(g.dims, g.spacing, g.vol_to_world, dtype=dare.DARE_F32, max_slots=8,
                         flags=dare.DARE_SESSION_SCALAR)
    fresh.build(torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV), tiny.frame_poses, tiny.frame_px)
    check_against_oracle(fresh, w, dare.DARE_F32, 8)
    fresh.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [4, 12])
def test_rebuild_sparse_build(tiny, dtype, K):
    """A rebuild of fewer than 8 pixels per voxel (7.0 here: the tiny sweep three
    times over a 112^3 grid of 0.3 mm voxels), whose full-write finalize reads a
    bucket only as far as its counter says: about 190 k voxels with 9 to 12
    entries (overflow ranges and the second finalize pass), the capacity rule at
    K = 4, every storage type."""
    g = synth.centred_grid((112, 112, 112), 0.3)
    w = types.SimpleNamespace(grid=g, frames=np.concatenate([tiny.frames] * 3),
                              frame_poses=np.concatenate([tiny.frame_poses] * 3), frame_px=tiny.frame_px)
    assert w.frames.size < 8 * np.prod(g.dims)
    s = rebuilt(w, dtype, K)
    e = check_against_oracle(s, w, dtype, K)
    assert np.diff(e["offsets"]).max() == min(K, 12)
    s.close()
