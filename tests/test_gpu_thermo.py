"""Thermodynamics on the CUDA path (through the C ABI) against the FP64 oracle: the partial
molar volume of Eq. 19 (grid integrals of c) and the SFE derivative with respect to the
solute atom positions (second Eq. 21, Hybrid implementation section).

Bars: FP64 path, solved to RMS 1e-10 like the oracle, 1e-7 relative on the c integrals and
1e-6 of the largest gradient component; FP32 path (RMS 1e-6 against the oracle at 1e-10)
1e-3 relative and 5e-3 of the largest component, the size of the FP32 solution's
deviation (max |dg| <= 1e-3) carried through the grid sums."""
import numpy as np
import pytest

from oracle import closure as cl
from oracle import rism3d as orc
from oracle import thermo
from paper_2403_01039_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()

GRIDS = [
    dict(n=(20, 20, 20), spacing=(0.5, 0.5, 0.5), origin=(-5.0, -5.0, -5.0)),
    # ragged tiles (Kz = 15, Ny = 20), radices 3 and 5, anisotropic spacing
    dict(n=(24, 20, 30), spacing=(0.55, 0.6, 0.5), origin=(-6.6, -6.0, -7.5)),
]
KT_CHI_T = 2.1763913575    # any positive value: Eq. 19 is linear in it


def _solutes():
    neutral = dict(xyz=np.array([[0.3, -0.2, 0.1], [-1.2, 0.9, -0.4]]), q=np.zeros(2),
                   sigma=np.array([3.2, 3.5]), eps=np.array([0.15, 0.1]))
    # 11 atoms: two full FP32 atom tiles plus a ragged one (FP64: two of four plus three)
    charged = synth.random_solute(11, 3.0, 23, net_charge=1.0)
    return dict(neutral=neutral, charged=charged)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("gi,which,kind,order,name", [
    (0, "neutral", cl.HNC, 0, "hnc"),
    (0, "charged", cl.KH, 1, "kh"),
    (1, "charged", cl.KH, 1, "kh"),
])
def test_pmv_and_sfe_gradient(water3, precision, gi, which, kind, order, name):
    grid = GRIDS[gi]
    sol = _solutes()[which]
    P = orc.Problem(water3, grid, sol)
    ref = orc.solve(P, kind, order, tol=1e-10)
    ref_ci = thermo.c_integrals(P, ref)
    ref_v = thermo.pmv(P, ref, KT_CHI_T)
    ref_grad = thermo.sfe_gradient(P, ref, sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
    with capi.Solver(water3, grid, precision=precision) as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        rep = S.solve(name, tol=1e-10 if precision == 64 else 1e-6)
        v, ci = S.pmv(KT_CHI_T)
        grad = S.sfe_gradient()
        grad2 = S.sfe_gradient()
    assert rep["converged"]
    assert np.array_equal(grad, grad2)                      # fixed-order reductions
    rel_c, rel_g = (1e-7, 1e-6) if precision == 64 else (1e-3, 5e-3)
    assert np.max(np.abs(ci - ref_ci)) <= rel_c * np.max(np.abs(ref_ci)), (ci, ref_ci)
    assert abs(v - ref_v) <= rel_c * KT_CHI_T * (1.0 + np.sum(np.abs(P.rho * ref_ci))), (v, ref_v)
    scale = np.max(np.abs(ref_grad))
    assert np.max(np.abs(grad - ref_grad)) <= rel_g * scale, (np.max(np.abs(grad - ref_grad)), scale)


def test_thermo_requires_solute(water3):
    with capi.Solver(water3, GRIDS[0], precision=64) as S:
        with pytest.raises(capi.RismError):
            S.pmv(KT_CHI_T)
        S.set_solute(np.zeros((1, 3)), [0.0], [3.73], [0.294])
        with pytest.raises(capi.RismError):
            S.pmv(-1.0)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("gi", [0, 1])
def test_sfe_finite_size_matches_oracle(water_nacl, precision, gi):
    """Finite-size correction of the SFE of a charged solute (rism3d_get_sfe_finite_size)
    against oracle.thermo: the DFT of the Eq. 29 field, the lattice sum with the solvent's
    charge response and the orientation-averaged integral (same quadrature: [0, 20] 1/A,
    16385 points). The result is the difference of two sums of similar size (~10x the result),
    so the bars are 1e-9 (FP64) and 2e-4 (FP32 fields and transform) relative to the sums."""
    sol = synth.random_solute(11, 3.0, 23, net_charge=1.0)
    grid = GRIDS[gi]
    P = orc.Problem(water_nacl, grid, sol)
    S_fn = lambda k: thermo.charge_response(P.chi, P.dk, P.site_q, P.rho, k)
    diff = thermo.lattice_minus_integral(P, sol["xyz"], sol["q"], S_fn, box_field=P.phi, k_max=20.0, n_quad=16385)
    ref = -0.5 * P.beta * diff
    scale = 0.5 * P.beta * abs(thermo.lattice_minus_integral(P, sol["xyz"], sol["q"], S_fn, box_field=None,
                                                             k_max=20.0, n_quad=16385))
    with capi.Solver(water_nacl, grid, precision=precision) as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        got = S.sfe_finite_size()
    bar = (1e-9 if precision == 64 else 2e-4) * max(abs(ref), scale, 1.0)
    assert abs(got - ref) <= bar, (got, ref, bar)
