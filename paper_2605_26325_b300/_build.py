"""Build libdare.so in place: CUDA kernels for sm_103a plus the C-ABI host code.

    python -m paper_2605_26325_b300._build [--force]

The library links the CUDA runtime statically, binds its own symbols
(-Bsymbolic) and exports only the dare_* entry points, so it cannot clash
with another CUDA runtime loaded in the same process (e.g. PyTorch's).
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
OUT = os.path.join(PKG, "libdare.so")
HEADER = os.path.join(ROOT, "include", "dare.h")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["kernels.cu", "kernels_tiled.cu", "kernels_radius.cu", "kernels_curv.cu", "kernels_paged.cu",
              "kernels_build.cu", "noalloc.cu"]
CPP_SOURCES = ["api.cpp", "server.cpp"]


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
           if f.endswith((".cu", ".cpp", ".h", ".cuh"))]
    return out + [HEADER, os.path.abspath(__file__)]


def _stale():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force=False, verbose=False):
    if not force and not _stale():
        return OUT
    os.makedirs(OBJ, exist_ok=True)
    procs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(OBJ, src + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd[1:1] = ["-Xptxas", "-v"]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(OBJ, src + ".o")
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-Wall",
               "-I", "/usr/local/cuda/include", "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((cmd, text))
        elif verbose and text.strip():
            print(text)
    if failed:
        msg = "\n\n".join(" ".join(c) + "\n" + t for c, t in failed)
        raise RuntimeError("libdare build failed:\n" + msg)
    mapfile = os.path.join(OBJ, "dare.map")
    with open(mapfile, "w") as fh:
        fh.write("{ global: dare_*; local: *; };\n")
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs,
           "-Xlinker", "-Bsymbolic", "-Xlinker", "--exclude-libs,ALL",
           "-Xlinker", f"--version-script={mapfile}"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libdare link failed:\n" + " ".join(cmd) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
