"""dare_reslice_noalloc: the reslice for callers that must not ask for device
memory while they run (a fixed-latency preview loop, or an application whose
device memory belongs to another component).  It must give what dare_reslice
gives, call after call, without allocating, and refuse sessions whose weight
table does not fit its fixed array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2605_26325_b300 as dare
from gpu_helpers import DEV, gpu_reslice, gpu_session, new_outputs

pytestmark = pytest.mark.gpu


def noalloc_reslice(s, T, W, H, px, params, bufs=None):
    """Call the entry point through the C ABI (into bufs = (out, mask) when given)."""
    out, mask = bufs if bufs is not None else new_outputs(W, H)
    plane = dare.make_plane(W, H, px, T)
    status = dare.lib().dare_reslice_noalloc(s.handle, ctypes.byref(plane), ctypes.byref(params),
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    dare.check(status, "dare_reslice_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy(), mask.cpu().numpy()


@pytest.mark.parametrize("path", [dare.DARE_PATH_TILED, dare.DARE_PATH_PLAIN])
@pytest.mark.parametrize("weights", [dare.DARE_WEIGHTS_F32, dare.DARE_WEIGHTS_F16])
def test_noalloc_matches_reslice_twice(tiny, path, weights):
    alloc = dare.TorchAllocator(0)
    s = gpu_session(tiny, dare.DARE_F32, 8, allocator=alloc)
    p = dare.params_default(path=path, weight_dtype=weights)
    gpu_reslice(s, tiny.reslice_poses[0], tiny.out_w, tiny.out_h, tiny.out_px, p)  # workspace exists already
    # set-up call: the first call on a device looks up the array's address, which
    # may load the library's module that holds it (device memory)
    noalloc_reslice(s, tiny.reslice_poses[3], tiny.out_w, tiny.out_h, tiny.out_px, p)
    live, in_use = len(alloc.live), dare.memory_in_use()
    refs = [gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p) for T in tiny.reslice_poses[[0, 9]]]
    bufs = [new_outputs(tiny.out_w, tiny.out_h) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outs = [noalloc_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p, b)  # two calls in a row, different planes
            for T, b in zip(tiny.reslice_poses[[0, 9]], bufs)]
    assert torch.cuda.mem_get_info()[0] == free0
    assert len(alloc.live) == live and dare.memory_in_use() == in_use
    for (a_out, a_mask), (b_out, b_mask) in zip(outs, refs):
        # same weight-table and reslice kernels with the same launch set-up: bit for bit
        np.testing.assert_array_equal(a_mask, b_mask)
        np.testing.assert_array_equal(a_out, b_out)
        assert dare.unpack_mask(b_mask, tiny.out_w).sum() > 1000
    s.close()


def test_noalloc_rejects_more_frames_than_its_array():
    n = dare.DARE_NOALLOC_MAX_FRAMES + 1
    s = dare.Session((32, 32, 32), 1.0, np.eye(4), max_frames=n)
    frames = torch.full((n, 1, 1), 100, dtype=torch.uint8, device=DEV)
    poses = np.tile(np.eye(4), (n, 1, 1))
    k = np.arange(n)
    poses[:, 0, 3], poses[:, 1, 3], poses[:, 2, 3] = k % 32, (k // 32) % 32, k // 1024  # one frame per voxel
    s.build(frames, poses, (1.0, 1.0))
    out, mask = new_outputs(8, 8)
    plane = dare.make_plane(8, 8, (0.5, 0.5), np.eye(4))
    p = dare.params_default()
    status = dare.lib().dare_reslice_noalloc(s.handle, ctypes.byref(plane), ctypes.byref(p),
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert status == dare.DARE_E_INVALID
    assert str(dare.DARE_NOALLOC_MAX_FRAMES) in dare.last_error()
    s.close()
