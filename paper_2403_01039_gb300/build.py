"""Builds the in-tree shared library ``_lib/librism3d.so`` for sm_103a with nvcc.

The translation units are compiled in parallel and linked with ``nvcc -shared``; a build
is skipped when the library is newer than every source and header.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "librism3d.so")

SOURCES = ["rism3d_planes_f32.cu", "rism3d_kernels_f32.cu", "rism3d_planes_f64.cu", "rism3d_kernels_f64.cu",
           "rism3d_capi.cu", "rism3d_noalloc.cu", "rism3d_microbench.cu", "unet3d.cu", "unet3d_tc.cu",
           "rism1d.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
# RISM_MINBLOCKS_F32: minimum resident blocks per SM that the FP32 plane, pencil and
# transform kernels are compiled for (their launch bounds; 3 when unset), for occupancy sweeps
if os.environ.get("RISM_MINBLOCKS_F32"):
    FLAGS.append("-DRISM_MINBLOCKS_F32=%d" % int(os.environ["RISM_MINBLOCKS_F32"]))


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = []
    for d in (CSRC, INCLUDE):
        for name in os.listdir(d):
            if name.endswith((".cu", ".cuh", ".h", ".cpp")):
                files.append(os.path.join(d, name))
    return files


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force=False, verbose=False):
    """Compile and link the library; returns its path. Raises RuntimeError on failure."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        cmd = [nvcc] + ARCH + FLAGS + ["-c", path, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + FLAGS + ["-x", "c++", "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
