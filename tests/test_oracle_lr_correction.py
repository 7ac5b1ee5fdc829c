"""Finite-size correction of the SFE of a charged solute on the periodic grid (oracle,
oracle/thermo.py: sfe_finite_size; the paper's Eqs. 17-18 are box sums and give none).

Pins: (1) the lattice sum minus the integral of a point charge's 1/k^2 response is the
Ewald-Wigner constant of the simple cubic lattice, xi / (4 pi L) with xi = -2.837297
(mathematics of lattice sums); (2) the orientation average in the integral is the closed
form sin(kR)/(kR) (checked by Gauss-Legendre quadrature over the angle); (3) physics: the
box-sum SFE of a monovalent cation changes by ~15 kcal/mol between boxes of 12 and 24 A
(as Q^2 / L), the corrected one by under 1.5 kcal/mol, and it lands within 2 kcal/mol of
the infinite-dilution radial 1D-RISM SFE (Eq. 8) in both DRISM water and water + 0.1 M NaCl
(the remaining difference is the 0.5 A grid's discretisation of a small ion)."""
import numpy as np
import pytest

from conftest import GOLDEN
from oracle import rism1d, rism3d, thermo, closure as cl
from oracle.units import COULOMB
from paper_2403_01039_gb300 import synth

XI_EW = -2.837297


@pytest.mark.parametrize("L", [32.0, 48.0])
def test_lattice_sum_gives_ewald_wigner_constant(water3, L):
    h = 0.25
    N = int(round(L / h))
    P = rism3d.Problem(water3, synth.cubic_grid(N, h), synth.lj_sphere())
    S2 = 1.0e-4
    xyz = np.array([[0.0, 0.0, 0.0]])
    diff = thermo.lattice_minus_integral(P, xyz, [1.0], lambda k: S2 * np.asarray(k) ** 2)
    # 1 / (k^2 (k^2 + 1)^2) = 1 / k^2 - (k^2 + 2) / (k^2 + 1)^2: the smooth part's lattice sum
    # lacks only its k = 0 value, -2 / V
    V = L ** 3
    expect = (4.0 * np.pi * COULOMB) ** 2 * S2 * (XI_EW / (4.0 * np.pi * L) + 2.0 / V)
    assert abs(diff - expect) <= 5e-3 * abs(expect), (diff, expect)


def test_pair_structure_is_orientation_average():
    rng = np.random.default_rng(3)
    xyz = rng.uniform(-3, 3, (4, 3))
    q = np.array([0.7, -0.3, -0.6, 0.4])
    k = np.array([0.05, 0.7, 2.3, 6.0])
    mu, w = np.polynomial.legendre.leggauss(200)
    ref = np.full(k.shape, float(np.sum(q * q)))
    for a in range(4):
        for b in range(a + 1, 4):
            d = np.linalg.norm(xyz[a] - xyz[b])
            ref += 2 * q[a] * q[b] * np.array([np.sum(w * np.cos(kk * d * mu)) / 2.0 for kk in k])
    assert np.allclose(thermo.pair_structure(xyz, q, k), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,solvent,chi_file", [("DRISM water", "water3", "chi_water3_drism.npz"),
                                                   ("water + NaCl", "water_nacl", "chi_water_nacl.npz")])
def test_corrected_sfe_is_box_independent_and_matches_1d(name, solvent, chi_file):
    d = np.load(GOLDEN + "/" + chi_file)
    s = synth.solvent_sites(solvent)
    s = dict(q=s["q"], sigma=s["sigma"], eps=s["eps"], rho=s["rho"], temperature=s["temperature"],
             chi=d["chi"], dk=float(d["dk"]))
    q_ion, sig, eps = 1.0, 2.6, 0.1
    g1 = rism1d.RadialGrid(int(d["n"]), float(d["dr"]))
    u = rism1d.solute_1d(d["chi"], g1, s["q"], s["sigma"], s["eps"], s["rho"], s["temperature"], q_ion, sig, eps,
                         closure=cl.KH, tol=1e-10, max_iter=50000)
    sfe_1d = rism1d.sfe_1d(u, cl.SFE_KH, s["temperature"])
    xyz = np.array([[0.13, -0.21, 0.07]])
    box, corrected = [], []
    for N in (24, 48):
        P = rism3d.Problem(s, synth.cubic_grid(N, 0.5), dict(xyz=xyz, q=[q_ion], sigma=[sig], eps=[eps]))
        r = rism3d.solve(P, cl.KH, 1, tol=1e-8, mdiis_nvec=5)
        sfe = rism3d.sfe(P, r, cl.SFE_KH)[0]
        box.append(sfe)
        corrected.append(sfe - thermo.sfe_finite_size(P, xyz, [q_ion]))
    assert abs(box[0] - box[1]) > 10.0, box
    assert abs(corrected[0] - corrected[1]) < 1.5, corrected
    assert all(abs(c - sfe_1d) < 2.0 for c in corrected), (corrected, sfe_1d)
