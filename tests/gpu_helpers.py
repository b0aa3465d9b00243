"""Shared helpers of the GPU tests: run the CUDA path through the C-ABI binding
and convert the oracle's results into the library's layouts."""
import numpy as np
import torch

import oracle
import paper_2605_26325_b300 as dare

DEV = "cuda:0"
ORA_DTYPE = {dare.DARE_U8: oracle.U8, dare.DARE_F16: oracle.F16, dare.DARE_BF16: oracle.BF16,
             dare.DARE_F32: oracle.F32}


def gpu_session(w, dtype=dare.DARE_F32, K=8, flags=0, chunks=None, frames=None, poses=None, allocator=None):
    s = dare.Session(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, dtype=dtype, max_slots=K, flags=flags,
                     allocator=allocator)
    frames = w.frames if frames is None else frames
    poses = w.frame_poses if poses is None else poses
    ft = torch.from_numpy(np.ascontiguousarray(frames)).to(DEV)
    bounds = chunks or [0, len(frames)]
    for a, b in zip(bounds[:-1], bounds[1:]):
        s.build(ft[a:b], poses[a:b], w.frame_px)
    torch.cuda.synchronize()
    return s


def oracle_volume(w, dtype=dare.DARE_F32, K=8, voxel_filter=None):
    return oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                        ORA_DTYPE[dtype], K, voxel_filter)


def stored_bits(values, dtype):
    """oracle FP64 stored values -> the storage type's bits as the library lays them out"""
    v = np.asarray(values, dtype=np.float64)
    if dtype == dare.DARE_F32:
        return v.astype(np.float32)
    if dtype == dare.DARE_F16:
        return v.astype(np.float16)
    if dtype == dare.DARE_BF16:
        return torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    return v.astype(np.uint8)


def oracle_dense(vol, K, dtype):
    """oracle CSR -> dense (n_vox, K) frame ids, values (storage type) and npix."""
    e = vol.export()
    counts = np.diff(e["offsets"])
    assert counts.max(initial=0) <= K
    nv = counts.size
    vox = np.repeat(np.arange(nv), counts)
    slot = np.arange(vox.size) - np.repeat(e["offsets"][:-1], counts)
    ids = np.full((nv, K), 0xFFFF, np.uint16)
    vals = np.zeros((nv, K), dare.VALUE_DTYPES[dtype])
    npix = np.zeros((nv, K), np.uint16)
    ids[vox, slot] = e["frame_id"]
    vals[vox, slot] = stored_bits(e["stored"], dtype)
    npix[vox, slot] = np.minimum(e["npix"], 65535)
    return ids, vals, npix, e


def ora_params(p):
    return oracle.Params(k_normal=p.k_normal, k_inplane=p.k_inplane, thr_normal_deg=p.thr_normal_deg,
                         thr_inplane_deg=p.thr_inplane_deg, k_dist=p.k_dist, unassigned=float(p.unassigned),
                         radius=p.radius_vox, kernel=p.dist_kernel, normal_axis=p.normal_axis,
                         per_pixel=p.sample_weight == dare.DARE_SAMPLE_PIXELS)


def new_outputs(W, H):
    out = torch.full((H, W), -12345.0, dtype=torch.float32, device=DEV)
    mask = torch.full((H, dare.mask_words(W)), -1, dtype=torch.int32, device=DEV)
    return out, mask


def gpu_reslice(s, T, W, H, px, params):
    out, mask = new_outputs(W, H)
    s.reslice(T, out, mask, px, params)
    torch.cuda.synchronize()
    return out.cpu().numpy(), mask.cpu().numpy()


def assert_parity(out, mask_words, ref, ref_mask, W, unassigned=0.0, rtol=1e-5):
    """mask bit-exact (padding bits 0), values within rtol * max(|ref|, 1)."""
    bits = dare.unpack_mask(mask_words, W)
    assert np.array_equal(bits, ref_mask.astype(np.uint8)), f"mask mismatch at {np.argwhere(bits != ref_mask)[:5]}"
    full = dare.unpack_mask(mask_words, mask_words.shape[1] * 32)
    assert not full[:, W:].any(), "padding bits set"
    cov = ref_mask.astype(bool)
    err = np.abs(out[cov] - ref[cov])
    tol = rtol * np.maximum(np.abs(ref[cov]), 1.0)
    assert np.all(err <= tol), f"max err {err.max()} (rel {np.max(err / np.maximum(np.abs(ref[cov]), 1))})"
    if np.isnan(unassigned):
        assert np.all(np.isnan(out[~cov]))
    else:
        assert np.all(out[~cov] == unassigned)
    return float(err.max(initial=0.0))
