"""The C ABI from C: tests/c_abi_check.c includes every public header, compiles as strict
C99 (gcc -std=c99 -pedantic -Werror), links the library and runs the calls that need no
GPU (defaults, workspace sizes, the host 1D solvent solve of Eq. 4, argument checks)."""
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
