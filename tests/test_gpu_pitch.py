"""GPU parity of the tiled reslice at pixel-to-voxel pitches where a 32 x 64
tile's voxel-column box no longer fits shared memory.

Planes are built on purpose at 0.75, 1.0 and 2.0 voxels per pixel, and at 0.5
voxel with a 45 degree in-plane rotation, both grid-aligned and oblique.  The
automatic tile choice must keep every tile inside shared memory (no per-pixel
fallback inside the kernel) or send the plane to the per-pixel kernel; the
fixed-height path forces the in-kernel per-pixel branch.  Both must equal the
FP64 oracle (Sec. 2.1, Eq. 1 / Eq. 2): masks bit-exact, values within
1e-5 max(|oracle|, 1)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import assert_parity, gpu_reslice, gpu_session, new_outputs, ora_params, oracle_volume

pytestmark = pytest.mark.gpu

H_VOX = 0.5  # tiny grid spacing (mm)


def _rot_z(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])


def _planes(tiny):
    """(name, pose, W, H, px_mm): sizes span several tiles with ragged tails.
    "aligned" planes have their normal on a grid axis (the sweep axis) and the
    +30 degree sweep's in-plane orientation; "rot40" / "rot45" turn the image
    40 / 45 degrees in-plane against the grid axes (10 / 15 degrees from that
    sweep, inside or on Eq. 1's 15 degree threshold); "oblique" is a moderately
    rotated pose of the tiny workload."""
    oblique = tiny.reslice_poses[9][:3, :3]
    out = []
    for name, pitch, W, H in (("p0.75", 0.75, 130, 101), ("p1.0", 1.0, 97, 83), ("p2.0", 2.0, 61, 45)):
        px = pitch * H_VOX
        for tag, R in (("aligned", synth.probe_rotation(30.0)), ("oblique", oblique)):
            out.append((f"{name}_{tag}", synth.plane_pose_centred(R, np.zeros(3), W, H, px, px), W, H, (px, px)))
    px = 0.5 * H_VOX
    for tag, deg in (("rot40", 40.0), ("rot45", 45.0)):
        out.append((f"p0.5_{tag}", synth.plane_pose_centred(synth.probe_rotation(deg), np.array([0.3, -0.2, 0.1]),
                                                             160, 150, px, px), 160, 150, (px, px)))
    return out


@pytest.fixture(scope="module")
def vols(tiny):
    s = gpu_session(tiny, dare.DARE_F32, 8)
    v = oracle_volume(tiny, dare.DARE_F32, 8)
    yield s, v
    s.close()


def test_automatic_tile_rows_never_fall_back(tiny, vols):
    """Single planes and one batch, automatic tile rows: no tile gathers per
    pixel inside the tiled kernel, the grid-aligned 2.0-voxel plane (whose
    smallest tile, 32 x 8 pixels, spans 65 x 17 voxel columns) goes to the
    per-pixel kernel, and every plane equals the oracle."""
    s, vol = vols
    p = dare.params_default(path=dare.DARE_PATH_TILED)
    planes = _planes(tiny)
    dare.trace_counters(reset=True)
    refs = {}
    for name, T, W, H, px in planes:
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        refs[name] = (ref, rm)
        assert rm.sum() > 0.05 * W * H, name
        assert_parity(out, mw, ref, rm, W)
    c = dare.trace_counters(reset=True)
    assert c["fallback_tiles"] == 0
    n_pp = c["per_pixel_planes"]
    assert n_pp >= 1 and c["tiled_planes"] == len(planes) - n_pp
    items = []
    for name, T, W, H, px in planes:
        out, mask = new_outputs(W, H)
        items.append((name, s, T, out, mask, px))
    dare.reslice_batch([it[1:] for it in items], p)
    torch.cuda.synchronize()
    c = dare.trace_counters(reset=True)
    assert c["fallback_tiles"] == 0 and c["per_pixel_planes"] == n_pp
    for name, _, _, out, mask, _ in items:
        ref, rm = refs[name]
        assert_parity(out.cpu().numpy(), mask.cpu().numpy(), ref, rm, out.shape[1])


@pytest.mark.parametrize("rows", [64, 32])
def test_fixed_tile_rows_fall_back_per_pixel(tiny, vols, rows):
    """DARE_PATH_TILED_FIXED keeps 32 x rows tiles at every pitch: tiles whose
    box overflows gather per pixel inside the kernel (counted), with the same
    result as the oracle."""
    s, vol = vols
    p = dare.params_default(path=dare.DARE_PATH_TILED_FIXED, tile_rows=rows)
    dare.trace_counters(reset=True)
    for name, T, W, H, px in _planes(tiny):
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert_parity(out, mw, ref, rm, W)
    c = dare.trace_counters(reset=True)
    assert c["fallback_tiles"] > 0 and c["per_pixel_planes"] == 0


@pytest.mark.parametrize("cap", [0, 16, 8])
def test_tile_row_caps(tiny, vols, cap):
    """tile_rows caps the automatic choice; every cap gives the oracle's result."""
    s, vol = vols
    p = dare.params_default(path=dare.DARE_PATH_TILED, tile_rows=cap)
    dare.trace_counters(reset=True)
    for name, T, W, H, px in _planes(tiny)[::2]:
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert_parity(out, mw, ref, rm, W)
    assert dare.trace_counters(reset=True)["fallback_tiles"] == 0


def test_tile_rows_rejects_other_values(tiny, vols):
    s, _ = vols
    out, mask = new_outputs(16, 16)
    with pytest.raises(dare.DareError) as ei:
        s.reslice(tiny.reslice_poses[0], out, mask, tiny.out_px, dare.params_default(tile_rows=48))
    assert ei.value.status == dare.DARE_E_INVALID


@pytest.mark.parametrize("path", [dare.DARE_PATH_AUTO, dare.DARE_PATH_TILED, dare.DARE_PATH_PLAIN])
def test_plan_replays_follow_tile_rows_of_new_poses(tiny, vols, path):
    """A plan's persistent tiled kernel reads each replay's tile count from the
    work queue: poses that change the planes' tile heights (aligned 0.5-voxel
    planes take 64 rows, 45-degree ones 32) give the results of dare_reslice
    on every replay."""
    s, _ = vols
    # thresholds off: every stored sample counts, whatever the plane's orientation
    off = dict(thr_normal_deg=180.0, thr_inplane_deg=180.0)
    p = dare.params_default(path=path, **off)
    px = 0.5 * H_VOX
    W, H = 160, 150
    pose_sets = [
        [synth.plane_pose_centred(synth.probe_rotation(a), np.array([0.2 * k, 0.0, 0.1]), W, H, px, px)
         for k, a in enumerate((0.0, 10.0, 0.0, 5.0))],
        [synth.plane_pose_centred(synth.probe_rotation(a), np.array([0.0, 0.2 * k, -0.1]), W, H, px, px)
         for k, a in enumerate((45.0, 40.0, 45.0, 50.0))],
        [synth.plane_pose_centred(tiny.reslice_poses[k][:3, :3] @ _rot_z(45.0), np.zeros(3), W, H, px, px)
         for k in (0, 4, 8, 12)],
    ]
    items = []
    for T in pose_sets[0]:
        out, mask = new_outputs(W, H)
        items.append((s, T, out, mask, (px, px)))
    plan = dare.Plan(items, p)
    for poses in pose_sets + pose_sets[:1]:
        plan.set_poses(np.stack(poses))
        for _, _, out, _, _ in items:
            out.fill_(-7.0)
        plan.launch()
        torch.cuda.synchronize()
        for (_, _, out, mask, _), T in zip(items, poses):
            o1, m1 = gpu_reslice(s, T, W, H, (px, px), dare.params_default(**off))
            assert np.array_equal(mask.cpu().numpy(), m1)
            assert dare.unpack_mask(m1, W).sum() > 0.05 * W * H
            cov = dare.unpack_mask(m1, W).astype(bool)
            got = out.cpu().numpy()
            if path == dare.DARE_PATH_TILED:  # same per-voxel sums and blend: bit-identical
                assert np.array_equal(got[cov], o1[cov])
            else:
                assert np.all(np.abs(got[cov] - o1[cov]) <= 1e-5 * np.maximum(np.abs(o1[cov]), 1))
            assert np.all(got[~cov] == 0.0)
    plan.close()


@pytest.mark.parametrize("path", [dare.DARE_PATH_PLAIN, dare.DARE_PATH_TILED])
def test_thresholds_open_parity(tiny, vols, path):
    """Eq. 1's thresholds opened to 180 degrees: every stored sample counts and
    Eq. 2's weights span orders of magnitude between neighbouring voxels, which
    a blend that subtracts neighbouring (A, B) sums would lose to cancellation.
    Both kernels stay within the path's tolerance of the oracle at every
    pitch of this file."""
    s, vol = vols
    p = dare.params_default(path=path, thr_normal_deg=180.0, thr_inplane_deg=180.0)
    for name, T, W, H, px in _planes(tiny):
        out, mw = gpu_reslice(s, T, W, H, px, p)
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert rm.sum() > 0.05 * W * H, name
        assert_parity(out, mw, ref, rm, W)


def test_plan_per_pixel_planes(tiny, vols):
    """Planes that no tile height fits (2.0 voxels per pixel) inside a plan's
    persistent kernel: gathered per pixel, equal to the oracle."""
    s, vol = vols
    p = dare.params_default(path=dare.DARE_PATH_TILED)
    planes = [pl for pl in _planes(tiny) if pl[0].startswith("p2.0") or pl[0].startswith("p0.75")]
    items = []
    for name, T, W, H, px in planes:
        out, mask = new_outputs(W, H)
        items.append((s, T, out, mask, px))
    plan = dare.Plan(items, p)
    plan.launch()
    torch.cuda.synchronize()
    for (name, T, W, H, px), (_, _, out, mask, _) in zip(planes, items):
        ref, rm = oracle.reslice(vol, T, W, H, px, ora_params(p))
        assert_parity(out.cpu().numpy(), mask.cpu().numpy(), ref, rm, W)
    plan.close()


def test_tuning_choices_persist_in_a_file(tiny, vols, tmp_path):
    """Plan tuning writes its choice per shape to the JSON file named by
    dare_tune_cache_file; a later plan of the same shape takes the choice from
    the file (here edited to the plain kernel) without timing anything, and its
    replay still equals dare_reslice."""
    import json
    s, _ = vols
    path = tmp_path / "tune.json"
    px = 0.5 * H_VOX
    W, H = 96, 80
    items = []
    for k in range(3):
        T = synth.plane_pose_centred(synth.probe_rotation(30.0 + 3 * k), np.array([0.0, 0.3 * k, 0.0]), W, H, px, px)
        out, mask = new_outputs(W, H)
        items.append((s, T, out, mask, (px, px)))
    dare.tune_cache_file(str(path))  # writes the choices known so far
    try:
        before = json.loads(path.read_text())
        plan = dare.Plan(items, dare.params_default(path=dare.DARE_PATH_AUTO))
        info = plan.info()
        plan.close()
        assert all(t > 0 for t in info["tune_ms"][0])  # a shape no other test uses: timed now
        saved = json.loads(path.read_text())
        new_keys = set(saved) - set(before)
        assert len(new_keys) == 1
        key = new_keys.pop()
        assert saved[key] == info["choice"][0] in (0, 16, 32, 64)
        saved[key] = 0 if info["choice"][0] != 0 else 32
        path.write_text(json.dumps(saved))
        dare.tune_cache_file(str(path))  # reload
        plan = dare.Plan(items, dare.params_default(path=dare.DARE_PATH_AUTO))
        info2 = plan.info()
        assert info2["choice"][0] == saved[key] and not any(t > 0 for t in info2["tune_ms"][0])
        plan.launch()
        torch.cuda.synchronize()
        for (_, T, out, mask, _) in items:
            o1, m1 = gpu_reslice(s, T, W, H, (px, px), dare.params_default())
            assert np.array_equal(mask.cpu().numpy(), m1)
            cov = dare.unpack_mask(m1, W).astype(bool)
            got = out.cpu().numpy()
            assert np.all(np.abs(got[cov] - o1[cov]) <= 1e-5 * np.maximum(np.abs(o1[cov]), 1))
        plan.close()
    finally:
        dare.tune_cache_file(None)


def test_plan_destroyed_after_its_session(tiny):
    """A plan may outlive its sessions' handles at destruction: dare_plan_destroy
    frees the plan's workspace through the allocator it recorded at creation and
    touches no session."""
    s = gpu_session(tiny, dare.DARE_F32, 8)
    out, mask = new_outputs(64, 48)
    plan = dare.Plan([(s, tiny.reslice_poses[3], out, mask, tiny.out_px)], dare.params_default())
    plan.launch()
    torch.cuda.synchronize()
    s.close()
    plan.close()
    alloc = dare.TorchAllocator(0)
    s = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, allocator=alloc)
    s.build(torch.from_numpy(tiny.frames).to("cuda"), tiny.frame_poses, tiny.frame_px)
    plan = dare.Plan([(s, tiny.reslice_poses[3], out, mask, tiny.out_px)], dare.params_default())
    s.close()
    assert len(alloc.live) == 1  # the plan's workspace, taken from the session's allocator
    plan.close()
    assert len(alloc.live) == 0
