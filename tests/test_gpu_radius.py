"""Distance kernels and interpolation radii beyond TENT at R = 1 (Sec. 2.1
"Reslicing": a cubic neighbourhood of fixed interpolation distance; Sec. 3
times radii of one, two and four voxels): TENT, BOX and EXP at radii 1-5 on
both reslice kernels, against the FP64 oracle.  Masks bit-exact, values within
1e-5 relative; batches, plans and the single-plane call agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
from gpu_helpers import assert_parity, gpu_reslice, gpu_session, new_outputs, ora_params, oracle_volume

pytestmark = pytest.mark.gpu

PATHS = [dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED]
KERNELS = [dare.DARE_TENT, dare.DARE_BOX, dare.DARE_EXP]


@pytest.fixture(scope="module")
def f32_pair(tiny):
    s = gpu_session(tiny, dare.DARE_F32, 8)
    yield s, oracle_volume(tiny, dare.DARE_F32, 8)
    s.close()


def _check(tiny, s, vol, p, poses):
    covered = 0
    for T in poses:
        out, mw = gpu_reslice(s, T, tiny.out_w, tiny.out_h, tiny.out_px, p)
        ref, rm = oracle.reslice(vol, T, tiny.out_w, tiny.out_h, tiny.out_px, ora_params(p))
        assert_parity(out, mw, ref, rm, tiny.out_w, unassigned=float(p.unassigned))
        covered += int(rm.sum())
    return covered


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("R", [1, 2])
def test_kernel_radius_parity(tiny, f32_pair, path, kernel, R):
    if R == 1 and kernel == dare.DARE_TENT:
        pytest.skip("the default kernel: covered by the main parity tests")
    s, vol = f32_pair
    p = dare.params_default(path=path, radius_vox=R, dist_kernel=kernel, k_dist=1.5)
    covered = _check(tiny, s, vol, p, tiny.reslice_poses[[0, 3, 5, 9, 13, 15]])
    assert covered > 0


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kernel,R", [(dare.DARE_TENT, 3), (dare.DARE_TENT, 4), (dare.DARE_BOX, 4),
                                      (dare.DARE_EXP, 4), (dare.DARE_TENT, 5)])
def test_large_radius_parity(tiny, f32_pair, path, kernel, R):
    """R = 3 (TENT factors not exact in FP32), the paper's largest radius
    (4), and R = 5, whose support is too wide for the tiled kernel: those
    planes gather per pixel."""
    s, vol = f32_pair
    p = dare.params_default(path=path, radius_vox=R, dist_kernel=kernel)
    assert _check(tiny, s, vol, p, tiny.reslice_poses[[1, 6]]) > 0


@pytest.mark.parametrize("dtype", [dare.DARE_U8, dare.DARE_F16])
def test_radius_reduced_storage_and_variants(tiny, dtype):
    """Reduced storage with FP16 weight tables, the elevation normal and
    thresholds off, at radius 2."""
    s = gpu_session(tiny, dtype, 4)
    vol = oracle_volume(tiny, dtype, 4)
    for p in (dare.params_default(path=dare.DARE_PATH_TILED, radius_vox=2, dist_kernel=dare.DARE_BOX,
                                  normal_axis=dare.DARE_NORMAL_ELEVATION),
              dare.params_default(path=dare.DARE_PATH_TILED, radius_vox=2, k_normal=0.0, k_inplane=0.0,
                                  thr_normal_deg=180.0, thr_inplane_deg=180.0, unassigned=float("nan"))):
        _check(tiny, s, vol, p, tiny.reslice_poses[[2, 11]])
    s.close()


@pytest.mark.parametrize("path", PATHS)
def test_radius_batch_plan_single_agree(tiny, f32_pair, path):
    s, _ = f32_pair
    p = dare.params_default(path=path, radius_vox=2, dist_kernel=dare.DARE_EXP, k_dist=0.7)
    rng = np.random.default_rng(3)
    sizes = [(int(rng.choice([37, 64, 100])), int(rng.choice([29, 64, 96]))) for _ in range(9)]
    poses = [tiny.reslice_poses[i % 16] for i in range(9)]
    outs = [new_outputs(W, H) for W, H in sizes]
    items = [(s, T, o, m, tiny.out_px) for (o, m), T in zip(outs, poses)]
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    got = [(o.cpu().numpy(), m.cpu().numpy()) for o, m in outs]
    for (W, H), T, (go, gm) in zip(sizes, poses, got):
        o1, m1 = gpu_reslice(s, T, W, H, tiny.out_px, p)
        assert np.array_equal(gm, m1)
        assert np.array_equal(go, o1)
    for o, m in outs:
        o.fill_(-1.0)
        m.fill_(-1)
    plan = dare.Plan(items, p)
    plan.launch()
    torch.cuda.synchronize()
    for (o, m), (go, gm) in zip(outs, got):
        assert np.array_equal(m.cpu().numpy(), gm)
        assert np.array_equal(o.cpu().numpy(), go)
    plan.close()


def test_radius_limits(tiny, f32_pair):
    s, _ = f32_pair
    out, mask = new_outputs(8, 8)
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], out, mask, tiny.out_px, dare.params_default(radius_vox=17))
    assert ei.value.status == dare.DARE_E_UNSUPPORTED
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], out, mask, tiny.out_px,
                  dare.params_default(dist_kernel=dare.DARE_EXP, k_dist=-1.0))
    assert ei.value.status == dare.DARE_E_INVALID


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kernel,R", [(dare.DARE_TENT, 1), (dare.DARE_BOX, 2), (dare.DARE_EXP, 1)])
def test_per_pixel_samples_parity(tiny, f32_pair, path, kernel, R):
    """DARE_SAMPLE_PIXELS (every pixel its own sample: stored samples weighted
    by their npix) on both general kernels against the oracle's reading."""
    s, vol = f32_pair
    p = dare.params_default(path=path, radius_vox=R, dist_kernel=kernel, sample_weight=dare.DARE_SAMPLE_PIXELS)
    assert _check(tiny, s, vol, p, tiny.reslice_poses[[0, 6, 11]]) > 0


def test_per_pixel_samples_u8_batch_and_plan(tiny):
    """Reduced storage, and batches / plans / single calls bit for bit."""
    s = gpu_session(tiny, dare.DARE_U8, 4)
    vol = oracle_volume(tiny, dare.DARE_U8, 4)
    p = dare.params_default(sample_weight=dare.DARE_SAMPLE_PIXELS)
    _check(tiny, s, vol, p, tiny.reslice_poses[[2, 9]])
    outs = [new_outputs(64, 48) for _ in range(5)]
    items = [(s, tiny.reslice_poses[i], o, m, tiny.out_px) for i, (o, m) in enumerate(outs)]
    dare.reslice_batch(items, p)
    torch.cuda.synchronize()
    got = [(o.cpu().numpy(), m.cpu().numpy()) for o, m in outs]
    plan = dare.Plan(items, p)
    for o, m in outs:
        o.fill_(-1.0)
    plan.launch()
    torch.cuda.synchronize()
    for i, ((o, m), (go, gm)) in enumerate(zip(outs, got)):
        o1, m1 = gpu_reslice(s, tiny.reslice_poses[i], 64, 48, tiny.out_px, p)
        assert np.array_equal(gm, m1) and np.array_equal(go, o1)
        assert np.array_equal(m.cpu().numpy(), m1) and np.array_equal(o.cpu().numpy(), o1)
    plan.close()
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], outs[0][0], outs[0][1], tiny.out_px, dare.params_default(sample_weight=5))
    assert ei.value.status == dare.DARE_E_INVALID
    s.close()
