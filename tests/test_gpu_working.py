"""GPU parity at the working size (256^3 grid, 1600 frames of 256x512, 512x512
planes) in the benchmark's launch configuration, on sampled pixels the oracle
computes one by one; and the storage-precision sweep against the FP64 oracle
on unrounded means."""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import (DEV, assert_parity, gpu_reslice, gpu_session, new_outputs, ora_params, oracle_dense,
                         oracle_volume)

pytestmark = pytest.mark.gpu

K_WORK = 12  # the working-size sweeps put up to 10 samples in a voxel


@pytest.fixture(scope="module")
def working():
    return synth.working_workload(1, n_poses=48)


def _corner_filter(w, poses, uvs):
    nv = int(np.prod(w.grid.dims))
    filt = np.zeros(nv, np.uint8)
    dims = np.array(w.grid.dims)
    for T, uv in zip(poses, uvs):
        aff = oracle.pixel_affine(w.grid.vol_to_world, w.grid.spacing, T, w.out_w, w.out_px)
        G = aff[0:3][None] + uv[:, :1] * aff[3:6][None] + uv[:, 1:2] * aff[6:9][None]
        c0 = np.floor_divide(G, 2**20)
        for d in np.ndindex(2, 2, 2):
            c = c0 + np.array(d)
            ok = np.all((c >= 0) & (c < dims), axis=1)
            c = c[ok]
            filt[c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])] = 1
    return filt


@pytest.mark.parametrize("path", [dare.DARE_PATH_TILED, dare.DARE_PATH_PLAIN])
def test_working_size_sampled(working, path):
    w = working
    s = gpu_session(w, dare.DARE_F32, K_WORK)
    assert s.info().overflow_voxels == 0
    p = dare.params_default(path=path)
    items = []
    for T in w.reslice_poses:
        out, mask = new_outputs(w.out_w, w.out_h)
        items.append((s, T, out, mask, w.out_px))
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    pick = [0, 7, 19, 30, 47]
    uvs = [np.stack([rng.integers(0, w.out_w, 3000), rng.integers(0, w.out_h, 3000)], axis=1) for _ in pick]
    # edges and corners of the image too
    for uv in uvs:
        uv[:4] = [[0, 0], [w.out_w - 1, 0], [0, w.out_h - 1], [w.out_w - 1, w.out_h - 1]]
    filt = _corner_filter(w, w.reslice_poses[pick], uvs)
    vol = oracle_volume(w, dare.DARE_F32, K_WORK, voxel_filter=filt)
    covered = 0
    for k, i in enumerate(pick):
        _, T, out, mask, _ = items[i]
        ref, rm = oracle.reslice_pixels(vol, T, w.out_w, w.out_px, uvs[k], ora_params(p))
        o = out.cpu().numpy()[uvs[k][:, 1], uvs[k][:, 0]]
        bits = dare.unpack_mask(mask.cpu().numpy(), w.out_w)[uvs[k][:, 1], uvs[k][:, 0]]
        assert np.array_equal(bits, rm)
        cov = rm.astype(bool)
        covered += cov.sum()
        assert np.all(np.abs(o[cov] - ref[cov]) <= 1e-5 * np.maximum(np.abs(ref[cov]), 1))
        assert np.all(o[~cov] == 0.0)
    assert covered > 3000
    # the records of every sampled neighbourhood, bit for bit
    ids, vals, npix, _ = oracle_dense(vol, K_WORK, dare.DARE_F32)
    g = s.read_records(npix=True)
    sel = filt.astype(bool)
    assert np.array_equal(g["frame_ids"][sel], ids[sel])
    assert np.array_equal(g["values"][sel].view(np.uint32), vals[sel].view(np.uint32))
    assert np.array_equal(g["npix"][sel], npix[sel])
    s.close()


# storage half-ulp for values in [128, 256) (u8 0.5, f16 2^-4, bf16 2^-1, f32 2^-17) plus FP32
# accumulation of a convex combination of values <= 255 (a few ulp of 255: 4e-5); the FP16-weight
# term is added separately
PRECISION_BOUND = {dare.DARE_U8: 0.5 + 4e-5, dare.DARE_F16: 0.0625 + 4e-5, dare.DARE_BF16: 0.5 + 4e-5,
                   dare.DARE_F32: 2.0 ** -17 + 4e-5}


@pytest.mark.parametrize("dtype", [dare.DARE_U8, dare.DARE_F16, dare.DARE_BF16, dare.DARE_F32])
def test_precision_against_unrounded_oracle(tiny, dtype):
    """Reduced storage types with the FP16 weight table against the FP64 oracle
    on the exact (unrounded) means: the output is a convex combination, so its
    error is at most the storage half-ulp plus 2 eps/(1-eps) (max I - min I)
    for the weights (eps = 2^-11) plus FP32 accumulation."""
    s = gpu_session(tiny, dtype, 8)
    vol = oracle_volume(tiny, dtype, 8)
    wd = dare.DARE_WEIGHTS_F32 if dtype == dare.DARE_F32 else dare.DARE_WEIGHTS_F16
    p = dare.params_default(weight_dtype=wd)
    op = ora_params(p)
    op.use_exact = True
    eps = 2.0 ** -11
    wterm = 0.0 if wd == dare.DARE_WEIGHTS_F32 else 2 * eps / (1 - eps) * 255.0
    worst = 0.0
    sq, n = 0.0, 0
    for T in tiny.reslice_poses[:12]:
        out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, op)
        assert np.array_equal(dare.unpack_mask(mw, tiny.out_w), rm)
        cov = rm.astype(bool)
        e = np.abs(out[cov] - ref[cov])
        worst = max(worst, float(e.max(initial=0)))
        sq += float(np.sum(e.astype(np.float64) ** 2))
        n += int(cov.sum())
    assert worst <= PRECISION_BOUND[dtype] + wterm
    psnr = 10 * np.log10(255.0 ** 2 / max(sq / max(n, 1), 1e-30))
    assert psnr > 40.0
    s.close()


def test_precision_sweep_working_size():
    """Storage precision at the working size over all 1000 planes: every storage
    type (u8, f16 and bf16 with an FP16 weight table; f32 with FP32 weights)
    against the FP64 oracle on the exact means, at 64 covered pixels of every
    512x512 plane (tests/golden/precision_working.npz, written from the oracle
    by tests/golden/make_precision_reference.py; its workload digest must match).
    Masks are 1 there; the max error stays within the storage half-ulp plus the
    weight term.  Reports max abs error and PSNR (peak 255) per type."""
    import json
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_precision_reference as mpr
    w = synth.working_workload(1, n_poses=mpr.N_POSES)
    g = np.load(mpr.OUT)
    assert str(g["workload"]) == mpr.workload_hash(w)
    uv, ref, cnt = g["uv"].astype(np.int64), g["value"], g["count"]
    keep = (np.arange(uv.shape[1])[None, :] < cnt[:, None]).reshape(-1)
    pi = np.repeat(np.arange(uv.shape[0]), uv.shape[1])[keep]
    u, v, refv = uv[:, :, 0].reshape(-1)[keep], uv[:, :, 1].reshape(-1)[keep], ref.reshape(-1)[keep]
    assert refv.size >= 60000
    P = uv.shape[0]
    outs = torch.empty((P, w.out_h, w.out_w), dtype=torch.float32, device=DEV)
    masks = torch.empty((P, w.out_h, dare.mask_words(w.out_w)), dtype=torch.int32, device=DEV)
    ti, tv, tu = (torch.from_numpy(x).to(DEV) for x in (pi, v, u))
    eps = 2.0 ** -11
    report = {}
    for dtype, name in ((dare.DARE_U8, "u8"), (dare.DARE_F16, "f16"), (dare.DARE_BF16, "bf16"), (dare.DARE_F32, "f32")):
        s = gpu_session(w, dtype, K_WORK)
        assert s.info().overflow_voxels == 0
        wd = dare.DARE_WEIGHTS_F32 if dtype == dare.DARE_F32 else dare.DARE_WEIGHTS_F16
        p = dare.params_default(weight_dtype=wd)
        dare.reslice_batch([(s, w.reslice_poses[i], outs[i], masks[i], w.out_px) for i in range(P)], p)
        torch.cuda.synchronize()
        got = outs[ti, tv, tu].double().cpu().numpy()
        words = masks[ti, tv, tu // 32].cpu().numpy().view(np.uint32)
        assert np.all((words >> (u % 32).astype(np.uint32)) & 1)
        e = np.abs(got - refv)
        wterm = 0.0 if wd == dare.DARE_WEIGHTS_F32 else 2 * eps / (1 - eps) * 255.0
        assert e.max() <= PRECISION_BOUND[dtype] + wterm, (name, e.max())
        psnr = float(10 * np.log10(255.0 ** 2 / max(np.mean(e ** 2), 1e-30)))
        report[name] = {"max_abs": float(e.max()), "psnr_db": psnr, "pixels": int(e.size), "planes": P,
                        "weights": "f32" if wd == dare.DARE_WEIGHTS_F32 else "f16",
                        "bound": PRECISION_BOUND[dtype] + wterm}
        s.close()
    print("precision sweep:", json.dumps(report))
    out_dir = os.environ.get("DARE_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "precision_working.json"), "w") as fh:
            json.dump(report, fh, indent=1)
