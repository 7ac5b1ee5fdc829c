"""The half-integer k grid (kgrid="half", numerical-procedure section) on the CUDA path
against the oracle with the same grid: single steps element by element, whole solves, the
row-chunked planes, and the warp-row kernels of Nz/2 = 64."""
import numpy as np
import pytest

from oracle import closure as cl
from oracle import rism3d as orc
from paper_2403_01039_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()

GRIDS = [
    dict(n=(32, 32, 32), spacing=(0.5, 0.5, 0.5), origin=(-8.0, -8.0, -8.0)),
    # ragged: Kz = 15 (odd, one self-paired column), radices 3 and 5, anisotropic
    dict(n=(24, 20, 30), spacing=(0.55, 0.6, 0.5), origin=(-6.6, -6.0, -7.5)),
    # Nz / 2 = 64: the FP32 warp-row plane kernels
    dict(n=(20, 24, 128), spacing=(0.5, 0.5, 0.25), origin=(-5.0, -6.0, -16.0)),
]


def _solute():
    return synth.random_solute(8, 3.0, 11, net_charge=1.0)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("gi", [0, 1, 2])
def test_half_grid_residual_elementwise(water_nacl, precision, gi):
    grid = GRIDS[gi]
    sol = _solute()
    P = orc.Problem(water_nacl, grid, sol, kgrid="half")
    rng = np.random.default_rng(40 + gi)
    t = P.f + 0.3 * rng.standard_normal(P.f.shape)
    ref, g, _ = P.residual(t, cl.KH, 1)
    with capi.Solver(water_nacl, grid, precision=precision, kgrid="half") as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        got = S.residual(t, "kh", 1)
    scale = max(1.0, float(np.max(np.abs(g))), float(np.max(np.abs(ref))))
    err = float(np.max(np.abs(got - ref)))
    assert err < (1e-10 if precision == 64 else 2e-4) * scale, (err, scale)


@pytest.mark.parametrize("slab_rows", [0, 8])
def test_half_grid_solve_fp64(water_nacl, slab_rows):
    grid = GRIDS[0]
    sol = _solute()
    P = orc.Problem(water_nacl, grid, sol, kgrid="half")
    ref = orc.solve(P, cl.KH, 1, tol=1e-6, mdiis_nvec=5)
    assert ref["converged"]
    with capi.Solver(water_nacl, grid, precision=64, kgrid="half", slab_rows=slab_rows) as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        rep = S.solve("kh", tol=1e-6)
        g = S.get("g")
        sfe, _ = S.sfe("kh")
    assert rep["converged"] and abs(rep["iterations"] - ref["iterations"]) <= 2
    assert np.max(np.abs(g - ref["g"])) <= 1e-6
    assert abs(sfe - orc.sfe(P, ref, cl.SFE_KH)[0]) <= 1e-4


def test_half_grid_solve_fp32(water_nacl):
    """FP32 against the oracle converged to 1e-10 (bars of the FP32 form)."""
    grid = GRIDS[2]
    sol = _solute()
    P = orc.Problem(water_nacl, grid, sol, kgrid="half")
    ref = orc.solve(P, cl.KH, 1, tol=1e-10, mdiis_nvec=5)
    with capi.Solver(water_nacl, grid, precision=32, kgrid="half") as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        rep = S.solve("kh", tol=1e-6)
        g = S.get("g")
        sfe, _ = S.sfe("kh")
    assert rep["converged"]
    assert np.max(np.abs(g - ref["g"])) <= 1e-3
    assert abs(sfe - orc.sfe(P, ref, cl.SFE_KH)[0]) <= 0.05
