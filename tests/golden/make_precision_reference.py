"""Write precision_working.npz: the FP64 oracle's reslice of the working-size
workload (256^3 grid at 0.4 mm, 1600 frames of 256 x 512, 1000 planes of
512 x 512 at 0.2 mm, synth.working_workload(seed 1)) on the exact, unrounded
per-(voxel, frame) means, at up to 64 covered pixels of every plane.

These are the reference values of the storage-precision sweep (FP32
accumulation over u8 / f16 / bf16 / f32 stored samples against FP64 on the
exact means; Sec. 2.1 reslicing with Eq. 1 and Eq. 2 at the paper's
constants).  Only the oracle and the seeded input generators are called.

    python tests/golden/make_precision_reference.py
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "precision_working.npz")
N_POSES = 1000
CANDIDATES = 256   # random pixels tried per plane
KEEP = 64          # covered pixels kept per plane
SEED = 2605


def workload_hash(w):
    """Digest of everything the reslices depend on: grid, frames, frame poses, plane poses and sizes."""
    h = hashlib.sha256()
    h.update(np.asarray(w.grid.dims, np.int64).tobytes())
    h.update(np.float64(w.grid.spacing).tobytes())
    h.update(np.ascontiguousarray(w.grid.vol_to_world, np.float64).tobytes())
    h.update(np.ascontiguousarray(w.frames).tobytes())
    h.update(np.ascontiguousarray(w.frame_poses, np.float64).tobytes())
    h.update(np.asarray(w.frame_px, np.float64).tobytes())
    h.update(np.ascontiguousarray(w.reslice_poses, np.float64).tobytes())
    h.update(np.asarray([w.out_w, w.out_h], np.int64).tobytes())
    h.update(np.asarray(w.out_px, np.float64).tobytes())
    return h.hexdigest()[:32]


def support_filter(w, uv):
    """1 for every in-grid voxel of the TENT (R = 1) support of the pixels uv (n_poses, m, 2)."""
    dims = np.array(w.grid.dims)
    filt = np.zeros(int(np.prod(dims)), np.uint8)
    for T, pts in zip(w.reslice_poses, uv):
        aff = oracle.pixel_affine(w.grid.vol_to_world, w.grid.spacing, T, w.out_w, w.out_px)
        G = aff[0:3][None] + pts[:, :1] * aff[3:6][None] + pts[:, 1:2] * aff[6:9][None]
        c0 = np.floor_divide(G, 2**20)
        for d in np.ndindex(2, 2, 2):
            c = c0 + np.array(d)
            ok = np.all((c >= 0) & (c < dims), axis=1)
            c = c[ok]
            filt[c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])] = 1
    return filt


def main():
    t0 = time.time()
    w = synth.working_workload(1, n_poses=N_POSES)
    rng = np.random.default_rng(SEED)
    cand = np.stack([rng.integers(0, w.out_w, (N_POSES, CANDIDATES)),
                     rng.integers(0, w.out_h, (N_POSES, CANDIDATES))], axis=2).astype(np.int64)
    filt = support_filter(w, cand)
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                       oracle.F32, 16, voxel_filter=filt)
    assert vol.n_overflow == 0
    params = oracle.Params(use_exact=True)
    uv = np.zeros((N_POSES, KEEP, 2), np.uint16)
    value = np.full((N_POSES, KEEP), np.nan, np.float64)
    count = np.zeros(N_POSES, np.int32)
    for i, T in enumerate(w.reslice_poses):
        ref, m = oracle.reslice_pixels(vol, T, w.out_w, w.out_px, cand[i], params)
        sel = np.flatnonzero(m)[:KEEP]
        count[i] = sel.size
        uv[i, :sel.size] = cand[i, sel]
        value[i, :sel.size] = ref[sel]
    np.savez_compressed(OUT, uv=uv, value=value, count=count, workload=np.array(workload_hash(w)),
                        seed=np.int64(SEED), max_slots=np.int64(16))
    print(f"{OUT}: {int(count.sum())} pixels over {N_POSES} planes in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
