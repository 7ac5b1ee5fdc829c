"""Host programs built from the sources, run without a GPU.

tests/c_abi_check.c includes every public header, compiles as strict C99 (gcc -std=c99
-pedantic -Werror), links the library and runs the calls that need no GPU (defaults,
workspace sizes, the host 1D solvent solve of Eq. 4, argument checks).
tests/fastdiv_check.cpp checks the kernels' multiply-shift index division."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_headers_compile_as_c99_and_host_calls_behave(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2403_01039_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_check")
    cc = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O1",
          "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_check.c"),
          "-L", libdir, "-lrism3d", "-Wl,-rpath," + libdir, "-lm", "-o", exe]
    r = subprocess.run(cc, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_multiply_shift_division_matches_hardware(tmp_path):
    """tests/fastdiv_check.cpp: the index divisions of the kernels (make_fastdiv of
    rism3d_internal.h) equal n / d for every divisor up to 1024 with n < 2^18 and for every
    2^a 3^b 5^c divisor below 2^27 at quotient boundaries up to 2^31 - 1."""
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not available")
    exe = str(tmp_path / "fastdiv_check")
    cc = ["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror",
          "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2403_01039_gb300", "csrc"),
          "-I", cuda_inc, os.path.join(ROOT, "tests", "fastdiv_check.cpp"), "-o", exe]
    r = subprocess.run(cc, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr
