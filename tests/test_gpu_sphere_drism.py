"""The sphere_32 workload as specified: a neutral LJ sphere (sigma 3.73 A, eps 0.294) at the
grid centre in 3-site water whose susceptibility comes from 1D DRISM (dielectric constant
78.44), 32^3 at 0.5 A, KH, MDIIS 5, tol 1e-6, FP64; the CUDA path against the FP64 oracle
run with the same algorithm (bars: max|dg|, max|dc| <= 1e-6, |dSFE| <= 1e-4 kcal/mol,
iteration counts within one)."""
import numpy as np
import pytest

from oracle import rism3d as orc, closure as cl
from paper_2403_01039_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()


def test_sphere_32_drism_solvent_matches_oracle(water3_drism):
    w = synth.WORKLOADS["sphere_32"]
    grid = synth.cubic_grid(w["n"], w["spacing"])
    sphere = synth.lj_sphere()
    P = orc.Problem(water3_drism, grid, sphere)
    ref = orc.solve(P, cl.KH, 1, tol=1e-6, mdiis_nvec=w["mdiis_nvec"])
    with capi.Solver(water3_drism, grid, precision=64, mdiis_nvec=w["mdiis_nvec"]) as S:
        S.set_solute(sphere["xyz"], sphere["q"], sphere["sigma"], sphere["eps"])
        rep = S.solve("kh", tol=1e-6)
        g = S.get("g")
        c = S.get("c")
        sfe, _ = S.sfe("kh")
    assert rep["converged"] and abs(rep["iterations"] - ref["iterations"]) <= 1, (rep, ref["iterations"])
    assert np.max(np.abs(g - ref["g"])) <= 1e-6
    assert np.max(np.abs(c - ref["c"])) <= 1e-6
    assert abs(sfe - orc.sfe(P, ref, cl.SFE_KH)[0]) <= 1e-4
