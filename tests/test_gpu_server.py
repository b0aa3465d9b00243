"""Serving loop (dare_server_*): continuous batching over stream lanes gives each
request exactly what it gets resliced alone, and live ingestion is ordered
with the requests around it."""
import numpy as np
import pytest
import torch

import paper_2605_26325_b300 as dare
import synth
from gpu_helpers import DEV, gpu_reslice, gpu_session, new_outputs

pytestmark = pytest.mark.gpu


def _wait_all(server, n, timeout=30.0):
    server.drain(timeout)
    got = []
    while len(got) < n:
        got += server.poll()
    return got


def test_server_mix_equals_alone(tiny):
    s1 = gpu_session(tiny, dare.DARE_F32, 8)
    s2 = gpu_session(tiny, dare.DARE_U8, 4)
    server = dare.Server(lanes=3, max_batch=5)
    rng = np.random.default_rng(0)
    jobs = []
    for i in range(48):
        s = s1 if rng.random() < 0.5 else s2
        W, H = int(rng.choice([37, 64, 128, 160])), int(rng.choice([23, 64, 128]))
        T = synth.plane_pose_centred(tiny.reslice_poses[i % 12][:3, :3], rng.uniform(-2, 2, 3), W, H, *tiny.out_px)
        out, mask = new_outputs(W, H)
        jobs.append((s, T, out, mask))
        server.submit(s, T, out, mask, tiny.out_px, tag=i)
    done = _wait_all(server, len(jobs))
    assert sorted(d[0] for d in done) == list(range(48))
    assert all(d[1] == dare.DARE_OK and d[4] >= d[3] for d in done)
    st = server.stats()
    assert st["submitted"] == st["completed"] == 48 and st["batches"] >= 10 and st["max_batch_seen"] <= 5
    for s, T, out, mask in jobs:
        H, W = out.shape
        o1, m1 = gpu_reslice(s, T, W, H, tiny.out_px, dare.params_default())
        assert np.array_equal(mask.cpu().numpy(), m1)
        cov = dare.unpack_mask(m1, W).astype(bool)
        got = out.cpu().numpy()
        assert np.all(np.abs(got[cov] - o1[cov]) <= 1e-5 * np.maximum(np.abs(o1[cov]), 1))
        assert np.all(got[~cov] == o1[~cov])
    server.close()
    s1.close()
    s2.close()


def test_server_ingest_is_ordered(tiny):
    """Requests submitted before an ingest see the old volume, requests after it
    the grown one."""
    live = gpu_session(tiny, dare.DARE_F16, 8, frames=tiny.frames[:100], poses=tiny.frame_poses[:100])
    half = gpu_session(tiny, dare.DARE_F16, 8, frames=tiny.frames[:100], poses=tiny.frame_poses[:100])
    full = gpu_session(tiny, dare.DARE_F16, 8)
    more = torch.from_numpy(tiny.frames[100:]).to(DEV)
    server = dare.Server(lanes=2, max_batch=4)
    before, after = [], []
    for i in range(8):
        out, mask = new_outputs(96, 96)
        T = tiny.reslice_poses[i]
        before.append((T, out, mask))
        server.submit(live, T, out, mask, tiny.out_px, tag=i)
    server.ingest(live, more, tiny.frame_poses[100:], tiny.frame_px, tag=1000)
    for i in range(8):
        out, mask = new_outputs(96, 96)
        T = tiny.reslice_poses[i]
        after.append((T, out, mask))
        server.submit(live, T, out, mask, tiny.out_px, tag=100 + i)
    done = _wait_all(server, 17)
    assert {d[0] for d in done} == set(range(8)) | set(range(100, 108)) | {1000}
    assert all(d[1] == dare.DARE_OK for d in done)
    p = dare.params_default()
    for ref_session, group in ((half, before), (full, after)):
        for T, out, mask in group:
            o1, m1 = gpu_reslice(ref_session, T, 96, 96, tiny.out_px, p)
            assert np.array_equal(mask.cpu().numpy(), m1)
            assert np.allclose(out.cpu().numpy(), o1, rtol=1e-5, atol=1e-5)
    assert live.info().n_frames == 200
    server.close()
    for s in (live, half, full):
        s.close()


def test_server_rejects_bad_requests(tiny, tmp_path):
    s = gpu_session(tiny, dare.DARE_F32, 8)
    server = dare.Server()
    out, mask = new_outputs(16, 16)
    bad = np.eye(4)
    bad[0, 0] = 3.0
    with pytest.raises(dare.DareError) as ei:
        server.submit(s, bad, out, mask, tiny.out_px, tag=1)
    assert ei.value.status == dare.DARE_E_INVALID
    server.drain(5.0)
    server.close()
    s.close()


def test_server_curvilinear_and_paged_sessions(tiny):
    """A curvilinear session served next to a linear one (the batch groups
    them by kernel family) gives what each request gets alone; a session with
    a brick cache is refused at submission."""
    curv = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_F32, max_slots=8)
    curv.set_probe(dare.DARE_PROBE_CURVILINEAR, (0.0, -20.0))
    curv.build(torch.from_numpy(np.ascontiguousarray(tiny.frames)).to(DEV), tiny.frame_poses, tiny.frame_px)
    lin = gpu_session(tiny, dare.DARE_F32, 8)
    server = dare.Server(lanes=2, max_batch=6)
    jobs = []
    for i in range(24):
        s = curv if i % 3 else lin
        W, H = (64, 48) if i % 2 else (96, 80)
        out, mask = new_outputs(W, H)
        jobs.append((s, tiny.reslice_poses[i % 16], out, mask))
        server.submit(s, tiny.reslice_poses[i % 16], out, mask, tiny.out_px, tag=i)
    done = _wait_all(server, len(jobs))
    assert all(d[1] == dare.DARE_OK for d in done)
    for s, T, out, mask in jobs:
        H, W = out.shape
        o1, m1 = gpu_reslice(s, T, W, H, tiny.out_px, dare.params_default())
        assert np.array_equal(mask.cpu().numpy(), m1) and np.array_equal(out.cpu().numpy(), o1)
    hv = dare.Session(tiny.grid.dims, tiny.grid.spacing, tiny.grid.vol_to_world, dtype=dare.DARE_U8, max_slots=4,
                      flags=dare.DARE_SESSION_HOST_VOLUME)
    hv.set_cache(1 << 22)
    out, mask = new_outputs(16, 16)
    with pytest.raises(dare.DareError) as ei:
        server.submit(hv, tiny.reslice_poses[0], out, mask, tiny.out_px, tag=99)
    assert ei.value.status == dare.DARE_E_UNSUPPORTED
    server.close()
    for x in (curv, lin, hv):
        x.close()


def test_server_coalesces_within_its_window(tiny):
    """With a coalescing window, requests of different sessions and output sizes
    submitted close together go out in few batches (here far fewer than one per
    request), and each result still equals dare_reslice of that request alone."""
    s1 = gpu_session(tiny, dare.DARE_F32, 8)
    s2 = gpu_session(tiny, dare.DARE_F16, 8)
    server = dare.Server(lanes=2, max_batch=64, coalesce_us=200000)
    jobs = []
    for i in range(24):
        s = (s1, s2)[i % 2]
        W, H = (64, 96, 128)[i % 3], (48, 128)[i % 2]
        T = synth.plane_pose_centred(tiny.reslice_poses[i % 16][:3, :3], np.zeros(3), W, H, *tiny.out_px)
        out, mask = new_outputs(W, H)
        jobs.append((s, T, out, mask))
        server.submit(s, T, out, mask, tiny.out_px, tag=i)
    done = _wait_all(server, len(jobs))
    assert sorted(d[0] for d in done) == list(range(24)) and all(d[1] == dare.DARE_OK for d in done)
    st = server.stats()
    assert st["completed"] == 24 and st["batches"] <= 4 and st["max_batch_seen"] >= 8
    for s, T, out, mask in jobs:
        H, W = out.shape
        o1, m1 = gpu_reslice(s, T, W, H, tiny.out_px, dare.params_default())
        assert np.array_equal(mask.cpu().numpy(), m1)
        np.testing.assert_array_equal(out.cpu().numpy(), o1)
    server.close()
    s1.close()
    s2.close()


def test_server_refuses_sessions_beyond_its_frame_budget(tiny):
    """Lane workspaces are sized at creation for sessions of up to max_frames
    frames; a session that allows more is refused at submission."""
    s = gpu_session(tiny, dare.DARE_F32, 8)  # max_frames 65535
    server = dare.Server(lanes=1, max_batch=4, max_frames=1000)
    out, mask = new_outputs(32, 32)
    with pytest.raises(dare.DareError) as ei:
        server.submit(s, tiny.reslice_poses[0], out, mask, tiny.out_px, tag=1)
    assert ei.value.status == dare.DARE_E_INVALID
    server.close()
    s.close()
