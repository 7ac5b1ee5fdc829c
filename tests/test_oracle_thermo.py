"""Pins of the thermodynamics oracle (Eqs. 19-21 and the SFE derivative of the Hybrid
implementation section) against limits and identities that do not use its formulas:
the second virial coefficient at low density, the test-particle partial molar volume of a
simple fluid (1/rho), the low-density structure factor, and finite differences of the
SFE for the derivative."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import closure as cl
from oracle import rism1d, rism3d, thermo
from oracle.units import KB_KCAL
from paper_2403_01039_gb300 import synth

AR_SIG, AR_EPS = 3.405, 0.2385       # argon-like LJ site (A, kcal/mol)


def _b2(sig, eps, temperature):
    """Second virial coefficient -2 pi int (exp(-beta u) - 1) r^2 dr of an LJ pair (A^3)."""
    beta = 1.0 / (KB_KCAL * temperature)

    def f(r):
        x = (sig / r) ** 6
        return (np.exp(-beta * 4.0 * eps * (x * x - x)) - 1.0) * r * r

    return -2.0 * np.pi * (quad(f, 1e-3, sig, limit=200)[0] + quad(f, sig, 80.0, limit=200)[0])


def _simple_fluid(sig, eps, rho, temperature, closure=cl.HNC):
    n = len(sig)
    return rism1d.xrism_solvent(np.zeros(n), sig, eps, rho, list(range(n)), np.zeros((n, 3)), temperature,
                                closure=closure, charge_steps=(1.0,))


def test_pressure_second_virial_mixture():
    """Eq. 20 for a dilute binary LJ mixture: P / kT = rho_1 + rho_2 + sum_ab rho_a rho_b B2_ab
    up to O(rho^3) (the direct correlation tends to the Mayer function)."""
    T, rho = 120.0, 1e-5
    sig, eps = np.array([AR_SIG, 3.0]), np.array([AR_EPS, 0.15])
    o = _simple_fluid(sig, eps, [rho, rho], T)
    P = thermo.pressure(o["c"], o["grid"].r, [rho, rho], [0, 1], T)
    kT = KB_KCAL * T
    b2 = sum(_b2(0.5 * (sig[a] + sig[b]), np.sqrt(eps[a] * eps[b]), T) for a in range(2) for b in range(2))
    virial = kT * rho * rho * b2
    assert abs((P - 2.0 * rho * kT) - virial) <= 0.01 * abs(virial)


def test_kT_chi_T_low_density():
    """k_B T chi_T = S(0) / rho with S(0) = 1 - 2 B2 rho + O(rho^2) for a dilute simple fluid."""
    T, rho = 120.0, 1e-5
    o = _simple_fluid(np.array([AR_SIG]), np.array([AR_EPS]), [rho], T)
    s0 = thermo.kT_chi_T(o["chi"], [rho]) * rho
    expect = -2.0 * _b2(AR_SIG, AR_EPS, T) * rho
    assert abs((s0 - 1.0) - expect) <= 0.01 * abs(expect)


def test_pmv_test_particle_is_molecular_volume():
    """Eq. 19 for a solute identical to the particles of a one-site fluid: its partial molar
    volume is the volume per particle, 1 / rho (here within the 3D box truncation, 1 %)."""
    T, rho = 500.0, 0.01
    o = _simple_fluid(np.array([AR_SIG]), np.array([AR_EPS]), [rho], T, closure=cl.KH)
    solv = dict(q=np.zeros(1), sigma=np.array([AR_SIG]), eps=np.array([AR_EPS]), rho=np.array([rho]),
                temperature=T, chi=o["chi"], dk=o["dk"])
    P = rism3d.Problem(solv, synth.cubic_grid(64, 0.5),
                       dict(xyz=np.zeros((1, 3)), q=[0.0], sigma=[AR_SIG], eps=[AR_EPS]))
    s = rism3d.solve(P, cl.KH, tol=1e-10)
    V = thermo.pmv(P, s, thermo.kT_chi_T(o["chi"], [rho]))
    assert abs(V - 1.0 / rho) <= 0.01 / rho


@pytest.mark.parametrize("kind,order,sk", [(cl.HNC, 0, cl.SFE_HNC), (cl.KH, 1, cl.SFE_KH)])
def test_sfe_gradient_is_derivative_of_sfe(water3, kind, order, sk):
    """For a neutral solute the HNC / KH SFE is stationary in the correlation functions, so its
    derivative with respect to an atom position is the solvent-averaged force of the second
    Eq. 21; central differences of the converged SFE (delta 1e-4 A) must agree."""
    sol = dict(xyz=np.array([[0.3, -0.2, 0.1], [-1.2, 0.9, -0.4]]), q=np.zeros(2),
               sigma=np.array([3.2, 3.5]), eps=np.array([0.15, 0.1]))
    grid = synth.cubic_grid(20, 0.5)
    P = rism3d.Problem(water3, grid, sol)
    s = rism3d.solve(P, kind, order, tol=1e-11)
    G = thermo.sfe_gradient(P, s, sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
    d = 1e-4
    for atom, dim in [(1, 0), (1, 1), (0, 2)]:
        vals = []
        for sgn in (1, -1):
            x = sol["xyz"].copy()
            x[atom, dim] += sgn * d
            Pq = rism3d.Problem(water3, grid, dict(sol, xyz=x))
            vals.append(rism3d.sfe(Pq, rism3d.solve(Pq, kind, order, tol=1e-11), sk)[0])
        fd = (vals[0] - vals[1]) / (2 * d)
        assert abs(fd - G[atom, dim]) <= 1e-6 * max(1.0, abs(fd)), (atom, dim, fd, G[atom, dim])
