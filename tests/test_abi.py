"""The C-ABI boundary on the CPU: the library loads, exports every entry point
include/dare.h declares, its structures have the layout the binding assumes,
and its host-only functions (parameters, fixed-point geometry, bounding box,
argument checks) behave as documented.  No GPU compute is called."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2605_26325_b300 as dare
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dare.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dare_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = dare.lib()
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in dare._SIGNATURES, f"binding lacks {n}"
    out = subprocess.run(["nm", "-D", "--defined-only", dare.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported
    # nothing but the C ABI leaks out (the static CUDA runtime stays private)
    assert all(e.startswith("dare_") for e in exported), sorted(e for e in exported if not e.startswith("dare_"))


def test_abi_version():
    assert dare.lib().dare_abi_version() == 3


def test_struct_layouts_match_c(tmp_path):
    structs = {
        "dare_grid": dare.dare_grid, "dare_allocator": dare.dare_allocator,
        "dare_session_config": dare.dare_session_config, "dare_params": dare.dare_params,
        "dare_plane": dare.dare_plane, "dare_reslice_req": dare.dare_reslice_req,
        "dare_session_info": dare.dare_session_info, "dare_probe": dare.dare_probe,
        "dare_plan_info": dare.dare_plan_info, "dare_trace_counters": dare.dare_trace_counters,
        "dare_server_config": dare.dare_server_config, "dare_server_stats": dare.dare_server_stats,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in got:
        if not line:
            continue
        parts = line.split()
        cls = structs[parts[0]]
        if parts[1] == "size":
            assert ctypes.sizeof(cls) == int(parts[2]), line
        else:
            assert getattr(cls, parts[1]).offset == int(parts[2]), line


def test_params_default_are_the_papers():
    p = dare.params_default()
    assert (p.k_normal, p.k_inplane, p.thr_normal_deg, p.thr_inplane_deg) == (10.0, 5.0, 25.0, 15.0)
    assert p.radius_vox == 1 and p.dist_kernel == dare.DARE_TENT and p.normal_axis == dare.DARE_NORMAL_BEAM
    assert p.unassigned == 0.0 and p.weight_dtype == dare.DARE_WEIGHTS_F32


def test_pixel_affine_bit_identical_to_oracle():
    """The library's FP64 composition and the oracle's, written independently in
    the canonical order, round to the same 2^-20 grid points."""
    rng = np.random.default_rng(0)
    for _ in range(400):
        V = synth.make_pose(synth.random_rotation(rng), rng.uniform(-80, 80, 3))
        T = synth.make_pose(synth.random_rotation(rng), rng.uniform(-80, 80, 3))
        h = rng.uniform(0.1, 1.0)
        W, H = int(rng.integers(1, 1024)), int(rng.integers(1, 1024))
        px = rng.uniform(0.05, 0.8, 2)
        a = dare.pixel_affine((64, 64, 64), h, V, W, H, px, T)
        b = oracle.pixel_affine(V, h, T, W, px)
        assert np.array_equal(a, b)


def test_grid_from_frames_covers_every_corner():
    rng = np.random.default_rng(1)
    poses = np.stack([synth.make_pose(synth.random_rotation(rng), rng.uniform(-20, 20, 3)) for _ in range(30)])
    W, H, px, h = 64, 96, (0.3, 0.25), 0.5
    dims, sp, V = dare.grid_from_frames(poses, W, H, px, h, margin_vox=1)
    assert sp == h and np.allclose(V[:3, :3], np.eye(3))
    for T in poses:
        for u in (0, W - 1):
            for v in (0, H - 1):
                p = T @ np.array([(u - 0.5 * (W - 1)) * px[0], v * px[1], 0, 1])
                g = (p[:3] - V[:3, 3]) / h
                assert np.all(g >= 1 - 1e-9) and np.all(g <= np.array(dims) - 2 + 1e-9)


def test_argument_errors_without_a_device():
    lib = dare.lib()
    cfg = dare.dare_session_config()
    cfg.grid = dare.make_grid((8, 8, 8), 1.0, np.eye(4))
    cfg.dtype, cfg.max_slots, cfg.max_frames = dare.DARE_F32, 7, 10
    h = ctypes.c_void_p()
    assert lib.dare_session_create(ctypes.byref(cfg), ctypes.byref(h)) == dare.DARE_E_INVALID
    assert "max_slots" in dare.last_error()
    cfg.max_slots = 8
    bad = np.eye(4)
    bad[0, 0] = 2.0
    cfg.grid = dare.make_grid((8, 8, 8), 1.0, bad)
    assert lib.dare_session_create(ctypes.byref(cfg), ctypes.byref(h)) == dare.DARE_E_INVALID
    assert "rigid" in dare.last_error()
    g = dare.make_grid((8, 8, 8), 1.0, np.eye(4))
    pl = dare.make_plane(0, 4, (1, 1), np.eye(4))
    out = (ctypes.c_int64 * 9)()
    assert lib.dare_pixel_affine(ctypes.byref(g), ctypes.byref(pl), out) == dare.DARE_E_INVALID
    assert lib.dare_reslice(None, None, None, None, None, None) == dare.DARE_E_INVALID
    assert lib.dare_set_memory_budget(-1) == dare.DARE_E_INVALID
    with pytest.raises(dare.DareError):
        dare.check(dare.DARE_E_INVALID, "x")


def test_tune_cache_file_host_side(tmp_path):
    """dare_tune_cache_file (host only): the file is written at once as a JSON
    object of the choices known to the process; a path that cannot be written
    is refused; None stops using a file."""
    import json
    path = tmp_path / "tune.json"
    path.write_text('{"sm148 t3 K12 w0 px2^20 n2^4 pitch4 l20 f2^11": 32, "broken": "x"}')
    dare.tune_cache_file(str(path))
    got = json.loads(path.read_text())
    assert got.get("sm148 t3 K12 w0 px2^20 n2^4 pitch4 l20 f2^11") == 32 and "broken" not in got
    with pytest.raises(dare.DareError) as ei:
        dare.tune_cache_file(str(tmp_path / "no_such_dir" / "tune.json"))
    assert ei.value.status == dare.DARE_E_INVALID
    dare.tune_cache_file(None)
