"""Pins for the 1D RISM part of the oracle (Eq. 4 for the solvent, Eq. 8 for a single site)."""
import numpy as np
import pytest

from oracle import rism1d, closure as cl
from oracle.units import COULOMB, beta
from paper_2403_01039_gb300 import synth

from conftest import load_chi, GOLDEN


def test_radial_transform_gaussian():
    g = rism1d.RadialGrid(2048, 0.05)
    f = np.exp(-g.r ** 2)
    F = g.forward(f)
    assert np.max(np.abs(F - np.pi ** 1.5 * np.exp(-g.k ** 2 / 4.0))) < 1e-12
    assert np.max(np.abs(g.inverse(F) - f)) < 1e-13


def test_low_density_limit_hnc():
    """As rho -> 0 the HNC solution tends to h = exp(-beta u) - 1 (first order in rho)."""
    T = 120.0
    r = rism1d.xrism_solvent([0.0], [3.4], [0.238], [1e-7], [0], [[0, 0, 0]], T, closure=cl.HNC,
                             tol=1e-12, charge_steps=(1.0,))
    rr = r["grid"].r
    sr6 = (3.4 / rr) ** 6
    ref = np.exp(-np.minimum(beta(T) * 4 * 0.238 * (sr6 * sr6 - sr6), 1e4)) - 1.0
    assert np.max(np.abs(r["h"][0, 0] - ref)) < 1e-4
    assert np.max(np.abs(r["chi"][0, 0] - 1.0)) < 1e-4       # X -> omega (X - 1 = rho h~, O(rho))


@pytest.fixture(scope="module")
def water_xrism():
    s = synth.water_3site()
    return s, rism1d.xrism_solvent(s["q"], s["sigma"], s["eps"], s["rho"], s["species"],
                                   s["coords"], s["temperature"])


def test_water_converged_and_symmetric(water_xrism):
    s, r = water_xrism
    assert r["rms"] < 1e-10
    chi = r["chi"]
    assert np.max(np.abs(chi[1, 1] - chi[2, 2])) < 1e-8     # H1 and H2 are equivalent
    assert np.max(np.abs(chi - np.swapaxes(chi, 0, 1))) < 1e-8   # equal densities -> symmetric
    assert chi[0, 0, 0] > 0.0                                  # S_OO(0) = rho kT kappa_T > 0


def test_water_dielectric_limit(water_xrism):
    """XRISM's dielectric constant is the ideal-dipole one, eps = 1 + 3y with
    y = 4 pi beta rho mu^2 / 9, so 4 pi beta S_qq(k)/k^2 -> 3y/(1+3y) as k -> 0."""
    s, r = water_xrism
    chi = r["chi"]
    q = s["q"]
    rho = s["rho"][0]
    b = beta(s["temperature"])
    k = np.arange(chi.shape[2]) * r["dk"]
    S = sum(rho * q[a] * q[c] * chi[a, c] for a in range(3) for c in range(3))
    mu = np.linalg.norm(sum(q[a] * s["coords"][a] for a in range(3)))
    y = 4 * np.pi * b * COULOMB * rho * mu * mu / 9.0
    lim = 4 * np.pi * b * COULOMB * S[1] / k[1] ** 2
    assert abs(lim - 3 * y / (1 + 3 * y)) < 2e-3


def _dielectric_limit(s, chi, dk):
    """k -> 0 limit of 4 pi beta S_qq(k) / k^2 for a one-molecule solvent, Richardson-
    extrapolated from k = dk and 2 dk (the leading correction is O(k^2))."""
    q, rho, b = s["q"], s["rho"][0], beta(s["temperature"])
    n = len(q)
    S = sum(rho * q[a] * q[c] * chi[a, c] for a in range(n) for c in range(n))
    lim = [4 * np.pi * b * COULOMB * S[j] / (j * dk) ** 2 for j in (1, 2)]
    return (4 * lim[0] - lim[1]) / 3


@pytest.mark.parametrize("eps_r", [78.44, 40.0])
def test_drism_dielectric_limit(eps_r):
    """DRISM (Perkyns-Pettitt) exists to give the solvent a prescribed dielectric constant:
    4 pi beta S_qq(k) / k^2 -> 1 - 1/eps as k -> 0, where XRISM gives 3y / (1 + 3y)
    (measured: 0.987253 for eps 78.44, 0.975000 for eps 40). A wrong amplitude (eps in
    place of eps - 1 moves it by 1.6e-4), a dropped zeta in omega' or in h, j0 in place of
    j1, or a dipole frame off the dipole each move the limit by more than the bar."""
    s = synth.water_3site()
    r = rism1d.xrism_solvent(s["q"], s["sigma"], s["eps"], s["rho"], s["species"], s["coords"],
                             s["temperature"], dielectric=eps_r)
    assert r["rms"] < 1e-10
    assert abs(_dielectric_limit(s, r["chi"], r["dk"]) - (1.0 - 1.0 / eps_r)) < 3e-5
    if eps_r == synth.WORKLOADS["sphere_32"]["dielectric"]:       # the stored table is this solve
        chi, dk = load_chi("water3_drism")
        assert np.isclose(dk, r["dk"]) and np.max(np.abs(chi - r["chi"])) < 1e-8


def test_xrism_dielectric_limit_extrapolated(water_xrism):
    s, r = water_xrism
    rho, b = s["rho"][0], beta(s["temperature"])
    mu = np.linalg.norm(sum(s["q"][a] * s["coords"][a] for a in range(3)))
    y = 4 * np.pi * b * COULOMB * rho * mu * mu / 9.0
    assert abs(_dielectric_limit(s, r["chi"], r["dk"]) - 3 * y / (1 + 3 * y)) < 3e-5


def test_stored_tables_match_live_solve(water_xrism):
    _, r = water_xrism
    chi, dk = load_chi("water3")
    assert np.isclose(dk, r["dk"]) and np.max(np.abs(chi - r["chi"])) < 1e-8


def test_single_site_solute_equals_solvent_ion():
    """A Na+ solute at infinite dilution in water + NaCl obeys the same equation as the
    solvent's own Na-gamma correlations (omega_NaNa = 1), so Eq. 8 must reproduce the XRISM
    h_Na,gamma. X is not symmetric here (rho_ion != rho_water): a transposed X fails."""
    s = synth.water_nacl_5site()
    d = np.load(GOLDEN + "/chi_water_nacl.npz")
    g = rism1d.RadialGrid(int(d["n"]), float(d["dr"]))
    u = rism1d.solute_1d(d["chi"], g, s["q"], s["sigma"], s["eps"], s["rho"], s["temperature"],
                         1.0, s["sigma"][3], s["eps"][3], tol=1e-11)
    assert np.max(np.abs(u["h"] - d["h"][3])) < 1e-7
