"""Brick paging for volumes beyond device memory (Sec. 4: growing datasets
despite GPU memory limits): a DARE_SESSION_HOST_VOLUME session with a device
cache of 8^3-voxel bricks.  Results must not depend on what the cache holds
(one slot, a few, all of them: bit-identical), must match the FP64 oracle
(masks exact, values 1e-5 relative), and must follow builds and resets."""
import types

import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import DEV, ORA_DTYPE, assert_parity, gpu_reslice, new_outputs, ora_params, oracle_volume

pytestmark = pytest.mark.gpu


def host_session(w, dtype=dare.DARE_F32, K=8, frames=None, poses=None, cache_bricks=None):
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=K,
                     flags=dare.DARE_SESSION_HOST_VOLUME)
    frames = w.frames if frames is None else frames
    poses = w.frame_poses if poses is None else poses
    s.build(torch.from_numpy(np.ascontiguousarray(frames)).to(DEV), poses, w.frame_px)
    if cache_bricks is not None:
        s.set_cache(cache_bricks * 512 * s.info().record_bytes)
    torch.cuda.synchronize()
    return s


@pytest.fixture(scope="module")
def paged_trio(tiny):
    sessions = [host_session(tiny, cache_bricks=n) for n in (1, 200, 512)]
    yield sessions
    for s in sessions:
        s.close()


@pytest.mark.parametrize("kernel,R,weights", [(dare.DARE_TENT, 1, dare.DARE_WEIGHTS_F32),
                                              (dare.DARE_BOX, 2, dare.DARE_WEIGHTS_F32),
                                              (dare.DARE_EXP, 1, dare.DARE_WEIGHTS_F16)])
def test_paged_results_independent_of_cache(tiny, paged_trio, kernel, R, weights):
    p = dare.params_default(radius_vox=R, dist_kernel=kernel, weight_dtype=weights, k_dist=0.9)
    vol = oracle_volume(tiny, dare.DARE_F32, 8)
    for i in (0, 3, 4, 9, 12, 15):
        T = tiny.reslice_poses[i]
        res = [gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p) for s in paged_trio]
        for o, m in res[1:]:
            assert np.array_equal(m, res[0][1]) and np.array_equal(o, res[0][0])
        if weights == dare.DARE_WEIGHTS_F32:
            ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
            assert_parity(res[2][0], res[2][1], ref, rm, tiny.out_w)
    st = [s.cache_stats() for s in paged_trio]
    assert st[0]["slots"] == 1 and st[1]["slots"] == 200 and st[2]["slots"] == 512
    assert all(x["resident"] <= x["slots"] for x in st)
    assert st[2]["hits"] > 0 and st[1]["paged_in"] > st[1]["slots"]  # the small cache evicts and re-pages


def test_paged_follows_builds_resets_and_batches(tiny):
    half = slice(0, 100)
    s = host_session(tiny, frames=tiny.frames[half], poses=tiny.frame_poses[half], cache_bricks=64)
    T = tiny.reslice_poses[2]
    gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, dare.params_default())  # fill the cache
    s.build(torch.from_numpy(np.ascontiguousarray(tiny.frames[100:])).to(DEV), tiny.frame_poses[100:], tiny.frame_px)
    vol = oracle_volume(tiny, dare.DARE_F32, 8)
    p = dare.params_default()
    for i in (2, 5, 13):
        out, mw = gpu_reslice(s, tiny.reslice_poses[i], tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, tiny.reslice_poses[i], tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
        assert_parity(out, mw, ref, rm, tiny.out_w)
    # a batch runs plane by plane, equal to the single calls
    outs = [new_outputs(64, 48) for _ in range(6)]
    items = [(s, tiny.reslice_poses[i], o, m, tiny.out_px) for i, (o, m) in enumerate(outs)]
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    for i, (o, m) in enumerate(outs):
        o1, m1 = gpu_reslice(s, tiny.reslice_poses[i], 64, 48, tiny.out_px, p)
        assert np.array_equal(m.cpu().numpy(), m1) and np.array_equal(o.cpu().numpy(), o1)
    # reset: the cached bricks are stale, the volume empty
    s.reset()
    out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
    assert not mw.any() and np.all(out == 0.0)
    # the calls that cannot page refuse the session
    host = [(np.zeros((48, 64), np.float32), np.zeros((48, 2), np.int32))]
    with pytest.raises(dare.DareError) as ei:
        dare.reslice_batch_host(dare.make_requests([(s, T, host[0][0], host[0][1], tiny.out_px)], host=True))
    assert ei.value.status == dare.DARE_E_UNSUPPORTED
    with pytest.raises(dare.DareError) as ei:
        dare.Plan(items[:1], p)
    assert ei.value.status == dare.DARE_E_UNSUPPORTED
    s.set_cache(0)
    assert s.cache_stats()["slots"] == 0
    s.close()


def test_cache_arguments(tiny):
    d = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_U8, max_slots=4)
    with pytest.raises(dare.DareError) as ei:
        d.set_cache(1 << 20)
    assert ei.value.status == dare.DARE_E_STATE
    d.close()
    h = host_session(tiny, dare.DARE_U8, 4, frames=tiny.frames[:4], poses=tiny.frame_poses[:4])
    for bad, status in ((-1, dare.DARE_E_INVALID), (100, dare.DARE_E_INVALID)):
        with pytest.raises(dare.DareError) as ei:
            h.set_cache(bad)
        assert ei.value.status == status
    h.set_cache(1 << 40)  # more than the volume: one slot per brick
    assert h.cache_stats()["slots"] == 512
    h.close()


@pytest.mark.parametrize("K", [8, 12, 16])
def test_paged_every_record_fill(tiny, K):
    """The paged gather on records of every fill from 1 to K (3 mm voxels over
    strided frame subsets, as in the device-resident parity test): a 2-brick
    cache (most records over the host link) and a cache of every brick give
    the same bits, and both match the oracle."""
    g = synth.centred_grid((12, 10, 9), 3.0)
    p = dare.params_default()
    for stride in (1, 3, 5):
        w = types.SimpleNamespace(grid=g, frames=tiny.frames[::stride], frame_poses=tiny.frame_poses[::stride],
                                  frame_px=(0.1, 0.12))
        small = host_session(w, dare.DARE_F32, K, cache_bricks=2)
        full = host_session(w, dare.DARE_F32, K, cache_bricks=1 << 12)
        vol = oracle.build(g.dims, g.spacing, g.vol_to_world, w.frames, w.frame_poses, w.frame_px, oracle.F32, K)
        for T in tiny.reslice_poses[[0, 3, 5]]:
            a = gpu_reslice(small, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
            b = gpu_reslice(full, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
            assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0])
            ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
            assert_parity(a[0], a[1], ref, rm, tiny.out_w)
        small.close()
        full.close()
