"""Host-buffer entry points (dare_build_volume_host, dare_reslice_batch_host):
the same records and images as the device-buffer calls, bit for bit, whatever
the slice and group sizes, host-buffer kind (page-locked or pageable) and
adjacency of the host outputs."""
import numpy as np
import pytest
import torch

import paper_2605_26325_b300 as dare
from gpu_helpers import DEV, gpu_session, new_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def tiny_f32(tiny):
    s = gpu_session(tiny, dare.DARE_F32, 8)
    yield s, None
    s.close()


def _records(s):
    r = s.read_records(npix=True, scalar=bool(s.info().flags & dare.DARE_SESSION_SCALAR))
    return {k: np.asarray(v).view(np.uint8) if k == "values" else np.asarray(v) for k, v in r.items()}


def _host_session(w, frames_host, dtype, K, flags=0, slices=(0,), bounds=None):
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=K, flags=flags)
    bounds = bounds or [0, len(w.frames)]
    for (a, b), sl in zip(zip(bounds[:-1], bounds[1:]), list(slices) * len(bounds)):
        s.build_host(frames_host[a:b], w.frame_poses[a:b], w.frame_px, slice_frames=sl)
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("kind", ["pinned", "pageable"])
@pytest.mark.parametrize("slices", [(0,), (7,), (1, 64)])
def test_build_host_equals_device(tiny, kind, slices):
    frames = np.ascontiguousarray(tiny.frames)
    host = torch.from_numpy(frames).pin_memory() if kind == "pinned" else frames
    ref = gpu_session(tiny, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR)
    got = _host_session(tiny, host, dare.DARE_F16, 8, flags=dare.DARE_SESSION_SCALAR, slices=slices,
                        bounds=[0, 37, 120, 200] if len(slices) > 1 else None)
    ra, rb = _records(ref), _records(got)
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    assert got.info().n_frames == ref.info().n_frames == len(tiny.frames)
    assert got.info().overflow_voxels == ref.info().overflow_voxels
    ref.close()
    got.close()


def _requests(tiny, rng, n):
    sizes = [(int(rng.choice([37, 64, 128])), int(rng.choice([23, 64, 96]))) for _ in range(n)]
    poses = [tiny.reslice_poses[i % len(tiny.reslice_poses)] for i in range(n)]
    return sizes, poses


@pytest.mark.parametrize("layout", ["adjacent", "separate"])
@pytest.mark.parametrize("group", [0, 1, 3])
def test_reslice_batch_host_equals_device(tiny, tiny_f32, layout, group):
    s, _ = tiny_f32
    rng = np.random.default_rng(7)
    sizes, poses = _requests(tiny, rng, 20)
    dev = [new_outputs(W, H) for W, H in sizes]
    dare.reslice_batch([(s, T, o, m, tiny.out_px) for (o, m), T in zip(dev, poses)])
    torch.cuda.synchronize()
    if layout == "adjacent":
        # one page-locked buffer for all images and one for all masks, planes back to back
        n_out = sum(W * H for W, H in sizes)
        n_msk = sum(H * dare.mask_words(W) for W, H in sizes)
        big_o = torch.full((n_out,), -7.0, dtype=torch.float32).pin_memory()
        big_m = torch.full((n_msk,), -1, dtype=torch.int32).pin_memory()
        host, oo, mo = [], 0, 0
        for W, H in sizes:
            host.append((big_o[oo:oo + W * H].view(H, W), big_m[mo:mo + H * dare.mask_words(W)].view(H, -1)))
            oo += W * H
            mo += H * dare.mask_words(W)
    else:
        host = [(np.full((H, W), -7.0, np.float32), np.full((H, dare.mask_words(W)), -1, np.int32))
                for W, H in sizes]
    reqs = dare.make_requests([(s, T, o, m, tiny.out_px) for (o, m), T in zip(host, poses)], host=True)
    dare.reslice_batch_host(reqs, group_planes=group)
    torch.cuda.current_stream().synchronize()
    for (o, m), (ho, hm) in zip(dev, host):
        assert np.array_equal(np.asarray(ho), o.cpu().numpy())
        assert np.array_equal(np.asarray(hm), m.cpu().numpy())


def test_host_calls_keep_session_order(tiny):
    """A host reslice queued between two host builds sees the volume as of its
    call: the second build's uploads run ahead, but its scatter waits."""
    frames = torch.from_numpy(np.ascontiguousarray(tiny.frames)).pin_memory()
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=8)
    half = gpu_session(tiny, dare.DARE_F32, 8, frames=tiny.frames[:100], poses=tiny.frame_poses[:100])
    full = gpu_session(tiny, dare.DARE_F32, 8)
    W, H = 96, 80
    outs = [(np.zeros((H, W), np.float32), np.zeros((H, dare.mask_words(W)), np.int32)) for _ in range(6)]
    s.build_host(frames[:100], tiny.frame_poses[:100], tiny.frame_px, slice_frames=9)
    dare.reslice_batch_host(dare.make_requests([(s, tiny.reslice_poses[i], o, m, tiny.out_px)
                                                for i, (o, m) in enumerate(outs[:3])], host=True), group_planes=1)
    s.build_host(frames[100:], tiny.frame_poses[100:], tiny.frame_px, slice_frames=9)
    dare.reslice_batch_host(dare.make_requests([(s, tiny.reslice_poses[i], o, m, tiny.out_px)
                                                for i, (o, m) in enumerate(outs[3:])], host=True), group_planes=2)
    torch.cuda.current_stream().synchronize()
    for ref, group in ((half, outs[:3]), (full, outs[3:])):
        for i, (o, m) in enumerate(group):
            ro, rm = new_outputs(W, H)
            ref.reslice(tiny.reslice_poses[i], ro, rm, tiny.out_px)
            torch.cuda.synchronize()
            assert np.array_equal(o, ro.cpu().numpy())
            assert np.array_equal(m, rm.cpu().numpy())
    for x in (s, half, full):
        x.close()


def test_host_calls_reject_bad_sizes(tiny, tiny_f32):
    s, _ = tiny_f32
    with pytest.raises(dare.DareError) as ei:
        s.build_host(np.ascontiguousarray(tiny.frames[:2]), tiny.frame_poses[:2], tiny.frame_px, slice_frames=-1)
    assert ei.value.status == dare.DARE_E_INVALID
    o, m = np.zeros((16, 16), np.float32), np.zeros((16, 1), np.int32)
    with pytest.raises(dare.DareError) as ei:
        dare.reslice_batch_host([(s, tiny.reslice_poses[0], o, m, tiny.out_px)], group_planes=-2)
    assert ei.value.status == dare.DARE_E_INVALID
    with pytest.raises(TypeError):
        dare.make_requests([(s, tiny.reslice_poses[0], torch.zeros(16, 16, device=DEV), m, tiny.out_px)], host=True)
