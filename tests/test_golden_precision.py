"""The stored FP64 reference values of the working-size precision sweep
(tests/golden/precision_working.npz) still describe the current workload and
agree with the oracle: the workload digest matches, and a fresh oracle
reslice of a few planes' stored pixels gives the stored values again."""
import os
import sys

import numpy as np
import pytest

import oracle
import synth

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_precision_reference as mpr  # noqa: E402

pytestmark = pytest.mark.slow


def test_precision_reference_matches_workload_and_oracle():
    w = synth.working_workload(1, n_poses=mpr.N_POSES)
    g = np.load(mpr.OUT)
    assert str(g["workload"]) == mpr.workload_hash(w)
    uv, value, count = g["uv"].astype(np.int64), g["value"], g["count"]
    assert uv.shape == (mpr.N_POSES, mpr.KEEP, 2) and np.all(count == mpr.KEEP)
    assert np.all(np.isfinite(value)) and value.min() >= 0.0 and value.max() <= 255.0
    planes = [0, 333, 999]
    filt = mpr.support_filter(w.__class__(**{**w.__dict__, "reslice_poses": w.reslice_poses[planes]}),
                              uv[planes])
    vol = oracle.build(w.grid.dims, w.grid.spacing, w.grid.vol_to_world, w.frames, w.frame_poses, w.frame_px,
                       oracle.F32, 16, voxel_filter=filt)
    for i in planes:
        ref, m = oracle.reslice_pixels(vol, w.reslice_poses[i], w.out_w, w.out_px, uv[i],
                                       oracle.Params(use_exact=True))
        assert np.all(m == 1)
        np.testing.assert_array_equal(ref, value[i])
