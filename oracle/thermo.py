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


# ---------------------------------------------------------------------------------------
# Finite-size correction of the SFE of a charged solute (reading: the paper's Eqs. 17-18 are
# evaluated as box sums on the periodic grid, whose long-range field of Eq. 30 has no k = 0
# term; it gives no correction).
#
# At long range the solvent responds linearly to the solute's field: a potential Phi~(k)
# (Eq. 30 without beta q_g) induces the charge density -beta Phi~(k) S(k), with
# S(k) = sum_{a,g} q_a X_ag(k) rho_g q_g the solvent's charge response (Eq. 13 with the
# direct correlation -beta q_a Phi~ of Eq. 32). The electrostatic part of the box-sum SFE is
# half the energy of that induced charge in the solute's potential of Eq. 29 sampled on the
# box, -(beta/2) (1/V) sum_{k != 0} Re(Phi~(k) phi~_box(k)*) S(k), where the periodic grid
# holds the response only at the lattice wave vectors; in infinite space the same energy is
# -(beta/2) int d^3k/(2 pi)^3 |Phi~(k)|^2 S(k). Their difference Delta is the finite-size
# error of the box sum: the infinite-dilution SFE is SFE_box - Delta. It grows as Q^2 / L for
# a net charge Q in a box of side L.


def charge_response(chi, dk, q, rho, kmag):
    """S(k) = sum_{a,g} q_a X_ag(|k|) rho_g q_g on the array kmag. Below the first table point
    k_1 = dk it is continued as S(k_1) (k / k_1)^2: the charge response of an electroneutral
    molecular solvent vanishes as k^2 (its tabulated k = 0 value is the 1D solve's rounding)."""
    from .rism3d import chi_interp
    q = np.asarray(q, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    kmag = np.asarray(kmag, dtype=np.float64)
    S = np.einsum("a,g,g,ag...->...", q, q, rho, chi_interp(chi, dk, kmag))
    S1 = float(np.einsum("a,g,g,ag...->...", q, q, rho, chi_interp(chi, dk, np.array([dk])))[0])
    return np.where(kmag < dk, S1 * (kmag / dk) ** 2, S)


def pair_structure(xyz, q, k):
    """sum_{a,b} q_a q_b sin(k R_ab) / (k R_ab): the orientation average of |sum_a q_a e^{-ik.R_a}|^2."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    out = np.full(k.shape, float(np.sum(q * q)))
    for a in range(len(q)):
        for b in range(a + 1, len(q)):
            R = float(np.linalg.norm(xyz[a] - xyz[b]))
            out += 2.0 * q[a] * q[b] * np.sinc(k * R / np.pi)
    return out


def lattice_minus_integral(problem, xyz, q, S_fn, box_field=None, k_max=40.0, n_quad=40001):
    """(1/V) sum_{k != 0} Re(Phi~(k) F(k)*) S(k) - int d^3k/(2 pi)^3 |Phi~(k)|^2 S(k) for the
    solute (xyz, q) on the problem's integer k grid (half spectrum, Nyquist planes dropped as
    in Phi~), with F = dV * DFT of box_field (the Eq. 29 potential sampled on the grid when
    box_field is the grid field; F = Phi~ when box_field is None). The integral is the radial
    form (1 / 2 pi^2) int k^2 (4 pi C)^2 S(k) pair_structure(k) / (k^2 (k^2 + 1))^2 dk by the
    trapezoidal rule on [0, k_max]."""
    from .potential import kvectors_half, phik_long_range
    P = problem
    if P.kgrid != "integer":
        raise ValueError("the finite-size correction is defined on the periodic (integer) k grid")
    kv, _ = kvectors_half(P.n, P.spacing)
    kmag = np.sqrt(np.sum(kv * kv, axis=-1))
    phik = phik_long_range(P.n, P.spacing, P.origin, xyz, q)
    F = phik if box_field is None else P.dV * np.fft.rfftn(box_field)
    wz = np.full(kmag.shape[2], 2.0)
    wz[0] = 1.0
    if P.n[2] % 2 == 0:
        wz[-1] = 1.0
    V = float(np.prod(P.n)) * P.dV
    lat = float(np.sum(wz[None, None, :] * (phik * np.conj(F)).real * S_fn(kmag))) / V
    k = np.linspace(0.0, k_max, n_quad)
    C4 = (4.0 * np.pi * COULOMB) ** 2
    Sk = S_fn(k)
    Sab = pair_structure(xyz, q, k)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(k > 0, C4 * Sk * Sab / (k * k * (k * k + 1.0) ** 2), 0.0)
    if k[1] > 0:                                   # k -> 0 limit: S(k) / k^2 is finite
        f[0] = C4 * float(S_fn(np.array([k[1]]))[0]) / (k[1] * k[1]) * Sab[0]
    integ = float(np.trapezoid(f, k)) / (2.0 * np.pi ** 2)
    return lat - integ


def sfe_finite_size(problem, xyz, q):
    """Delta (kcal/mol): the SFE box sum minus its infinite-dilution value, from the linear
    response of the solvent to the solute's long-range field (see above); the corrected SFE
    is SFE_box - Delta."""
    P = problem
    S_fn = lambda k: charge_response(P.chi, P.dk, P.site_q, P.rho, k)
    return -0.5 * P.beta * lattice_minus_integral(P, xyz, q, S_fn, box_field=P.phi)
