"""Thermodynamics beyond the SFE (oracle, FP64).

* Eq. 19 (PMV):        V = k_B T chi_T (1 - sum_g rho_g int c_g(r) dr)
* Eq. 20 (pressure):   P = sum_G rho_G (n_G + 1) / (2 beta) - sum_{g,l} (2 pi rho_g rho_l / beta)
                           int c_gl(r) r^2 dr        (G: solvent species, n_G their sites)
* Eq. 21:              dmu_PC = -P V
* second "Eq. 21" (Hybrid implementation): the solvent part of the derivative of the free
  energy with respect to a solute atom, d(dmu)/dR_a = sum_g rho_g int du_g(r)/dR_a g_g(r) dr.

Readings (the paper is silent): k_B T chi_T of the solvent is X_OO(0) / rho_O of its first
site (for water, the structure factor of the molecular centre); the integrals are plain grid
sums (dV on the 3D grid, dr on the 1D grid, the same grids as the solve); du/dR is the
analytic derivative of Eq. 22's pair terms evaluated at the grid points (r^2 floored as in
the potential; where beta*u is capped, g = 0 to working precision).
"""
import numpy as np

from .potential import grid_points, lorentz_berthelot
from .units import COULOMB, R2_FLOOR, KB_KCAL

A3_TO_CC_PER_MOL = 0.602214076     # 1 A^3 per molecule = 0.6022 cm^3/mol


def kT_chi_T(chi, rho):
    """k_B T chi_T from the susceptibility at k = 0 of the first solvent site."""
    return float(chi[0, 0, 0] / rho[0])


def c_integrals(problem, sol):
    """int c_g(r) dr per site (A^3) as grid sums."""
    return np.array([problem.dV * float(np.sum(sol["c"][g])) for g in range(problem.n_sites)])


def pmv(problem, sol, kt_chi_t):
    """Partial molar volume of Eq. 19 in A^3 per molecule."""
    return kt_chi_t * (1.0 - float(np.sum(problem.rho * c_integrals(problem, sol))))


def pressure(c_r, r, rho, species, temperature):
    """Bulk pressure of Eq. 20 (kcal/mol/A^3) from the solvent direct correlation c_gl(r)
    ([n, n, len(r)], full c including its Coulomb tail) on the radial grid r."""
    kT = KB_KCAL * temperature
    rho = np.asarray(rho, dtype=np.float64)
    species = np.asarray(species)
    ideal = 0.0
    for sp in np.unique(species):
        sites = np.nonzero(species == sp)[0]
        ideal += rho[sites[0]] * (len(sites) + 1) * kT / 2.0
    dr = r[1] - r[0]
    integ = dr * np.sum(c_r * r * r, axis=-1)                # [n, n]
    return ideal - 2.0 * np.pi * kT * float(rho @ integ @ rho)


def sfe_gradient(problem, sol, xyz, q, sig, eps):
    """d(dmu)/dR_a in kcal/mol/A for every solute atom ([n_atoms, 3]): direct sums over the
    grid of rho_g g_g(r) du_g(r)/dR_a, with
    du/dR = (48 eps s^12 / d^14 - 24 eps s^6 / d^8 + C q_a q_g / d^3) (r - R)."""
    P = problem
    pts = grid_points(P.n, P.spacing, P.origin)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(q), 3))
    for a in range(len(q)):
        e = pts - xyz[a]
        d2 = np.maximum(np.sum(e * e, axis=-1), R2_FLOOR)
        for g in range(P.n_sites):
            s_ag, e_ag = lorentz_berthelot(sig[a], eps[a], P.site_sig[g], P.site_eps[g])
            s6 = (s_ag * s_ag / d2) ** 3
            fac = (48.0 * e_ag * s6 * s6 - 24.0 * e_ag * s6) / d2 + COULOMB * q[a] * P.site_q[g] / (d2 * np.sqrt(d2))
            w = P.rho[g] * P.dV * fac * sol["g"][g]
            out[a] += np.tensordot(w, e, axes=([0, 1, 2], [0, 1, 2]))
    return out
