"""1D RISM (oracle, FP64): solvent susceptibility and the single-site solute check.

* Eq. 4 (RISM theory): h = omega * c * omega + omega * c * rho h for the pure solvent
  ("XRISM"), closed by the closures of ``oracle.closure``; its solution gives the solvent
  susceptibility X_ag = omega_ag + rho_a h_ag (the definition under Eq. 8), the input of
  the 3D-RISM equation (Eq. 13).
* Eq. 8 with a single-site solute: h_g = sum_a c_a * X_ag, the 3D-RISM equation
  under spherical symmetry, solved with the same steps 1-7 as the 3D solve (long-range
  split of Eqs. 29-31 in radial form). Used only to cross-check the 3D oracle.

Readings (the paper defers the 1D method to Kinoshita and is silent on details):
* radial grid r_i = i dr, k_j = j dk, dk = pi / (N dr), i, j = 1..N-1 (sine-transform pairs)
  F(k) = (4 pi dr / k) sum_i r_i f(r_i) sin(k r_i),
  f(r) = (dk / (2 pi^2 r)) sum_j k_j F(k_j) sin(k_j r),
  evaluated as direct matrix sums (the definition);
* Coulomb long range of solvent-solvent pairs split with the same function as Eq. 29,
  u_L = COULOMB q_a q_b (1 - e^{-r}) / r, whose transform is 4 pi COULOMB q_a q_b /
  (k^2 (k^2 + 1)) (Eq. 30); the closure then acts on d = -beta u_s + tau with
  tau = h - c_s, c = c_s - beta u_L;
* intramolecular omega_ab(k) = sin(k l_ab) / (k l_ab) for two sites of one molecule,
  1 on the diagonal, 0 between molecules;
* X at k = 0 from X_ab(0) = omega_ab(0) + rho_a 4 pi dr sum_i r_i^2 h_ab(r_i);
* MDIIS as in ``oracle.mdiis``; the charges are switched on in ten steps (0.1, 0.2, ... 1.0 of
  their values, each solve starting from the previous tau), without which XRISM-KH for
  the 3-site water above diverges from tau = 0;
* DRISM (the dielectrically consistent RISM of Perkyns and Pettitt, which the paper names
  through Kinoshita's 1D method without detail), as an option: the RISM equation above is
  solved with omega' = omega + rho zeta in place of omega for h' = h - zeta, and the
  physical h = h' + zeta; then X = omega + rho h = omega' + rho h'. zeta couples the sites
  of the polar molecules: zeta_ab(k) = d_a(k) d_b(k) h_c(k), d_a = j0(k x_a) j0(k y_a)
  j1(k z_a) with (x, y, z) the site position in its molecule's frame (origin at the
  centroid of its sites, z along the dipole mu, x along the component normal to z of the
  site farthest from the z axis, the first such site on a tie; y = z cross x), h_c(k) =
  h_c0 exp(-a^2 k^2 / 4). The amplitude follows from
  the small-k limit: with j1(x) -> x/3 the polar species' dipole strength
  y = sum_s 4 pi beta COULOMB rho_s mu_s^2 / 9 grows to y + sum_s rho_s y_s h_c0 / 3, and
  the RISM dielectric constant 1 + 3y (the XRISM value) becomes the prescribed eps when
  h_c0 = (eps - 1 - 3y) / sum_s rho_s y_s. The damping length a is a parameter (1 A by
  default; the paper is silent). X is a shared input of both the oracle and the CUDA path,
  so this choice cannot affect their parity.
"""
import numpy as np

from . import closure as cl
from . import mdiis
from .units import COULOMB, R2_FLOOR, BETA_U_CAP, beta as beta_of


class RadialGrid:
    def __init__(self, n=2048, dr=0.05):
        self.N = int(n)
        self.dr = float(dr)
        self.dk = np.pi / (self.N * self.dr)
        idx = np.arange(1, self.N)
        self.r = idx * self.dr
        self.k = idx * self.dk
        self.S = np.sin(np.pi * np.outer(idx, idx) / self.N)   # symmetric DST-I matrix

    def forward(self, f):
        """Radial Fourier transform along the last axis."""
        return (4.0 * np.pi * self.dr / self.k) * ((f * self.r) @ self.S)

    def inverse(self, F):
        return (self.dk / (2.0 * np.pi ** 2 * self.r)) * ((F * self.k) @ self.S)


def omega_matrix(grid, species, coords):
    """omega_ab(k_j), shape [n, n, N-1]."""
    n = len(species)
    W = np.zeros((n, n, grid.N - 1))
    for a in range(n):
        for b in range(n):
            if a == b:
                W[a, b] = 1.0
            elif species[a] == species[b]:
                l = float(np.linalg.norm(np.asarray(coords[a]) - np.asarray(coords[b])))
                W[a, b] = np.sin(grid.k * l) / (grid.k * l)
    return W


def _sph_j0(x):
    xs = np.where(x == 0.0, 1.0, x)
    return np.where(x == 0.0, 1.0, np.sin(xs) / xs)


def _sph_j1(x):
    xs = np.where(x == 0.0, 1.0, x)
    return np.where(x == 0.0, 0.0, np.sin(xs) / (xs * xs) - np.cos(xs) / xs)


def drism_zeta(grid, q, rho, species, coords, temperature, dielectric, a=1.0):
    """zeta_ab(k_j) of DRISM, shape [n, n, N-1] (zero outside the polar molecules), and the
    amplitude h_c0 (module docstring). Raises ValueError when no molecule has a dipole."""
    q = np.asarray(q, dtype=np.float64)
    coords = np.asarray(coords, dtype=np.float64)
    species = np.asarray(species)
    n = len(q)
    b = beta_of(temperature)
    k = grid.k
    d = np.zeros((n, grid.N - 1))
    y_tot, rho_y = 0.0, 0.0
    for s_ in np.unique(species):
        idx = np.flatnonzero(species == s_)
        pos = coords[idx] - coords[idx].mean(axis=0)
        mu = q[idx] @ pos
        m = float(np.linalg.norm(mu))
        if m < 1e-12:
            continue
        z = mu / m
        perp = pos - np.outer(pos @ z, z)                # components normal to z
        pn = np.linalg.norm(perp, axis=1)
        far = int(np.argmax(pn))
        if pn[far] > 1e-12:
            x = perp[far] / pn[far]
        else:                                            # all sites on the dipole axis
            x = np.cross(z, [1.0, 0.0, 0.0] if abs(z[0]) < 0.9 else [0.0, 1.0, 0.0])
            x /= np.linalg.norm(x)
        yax = np.cross(z, x)
        ys = 4.0 * np.pi * b * COULOMB * rho[idx[0]] * m * m / 9.0
        y_tot += ys
        rho_y += rho[idx[0]] * ys
        for i, site in enumerate(idx):
            d[site] = _sph_j0(k * (pos[i] @ x)) * _sph_j0(k * (pos[i] @ yax)) * _sph_j1(k * (pos[i] @ z))
    if rho_y == 0.0:
        raise ValueError("DRISM needs a solvent molecule with a dipole")
    hc0 = (dielectric - 1.0 - 3.0 * y_tot) / rho_y
    hc = hc0 * np.exp(-(a * k) ** 2 / 4.0)
    return d[:, None, :] * d[None, :, :] * hc, hc0


def _pair_params(q, sig, eps):
    s = 0.5 * (sig[:, None] + sig[None, :])
    e = np.sqrt(eps[:, None] * eps[None, :])
    return q[:, None] * q[None, :], s, e


def xrism_solvent(q, sig, eps, rho, species, coords, temperature, n=2048, dr=0.05,
                  closure=cl.KH, tol=1e-10, max_iter=5000, mdiis_nvec=5, mdiis_damp=0.3,
                  charge_steps=tuple(0.1 * i for i in range(1, 11)), verbose=False,
                  dielectric=None, drism_a=1.0):
    """Solve Eq. 4 for the pure solvent (XRISM; DRISM with the given dielectric constant
    when ``dielectric`` is set). Returns dict(chi [n,n,N] at k_j = j dk for j = 0..N-1, dk,
    h, c, grid, iterations, rms)."""
    q, sig, eps, rho = (np.asarray(v, dtype=np.float64) for v in (q, sig, eps, rho))
    grid = RadialGrid(n, dr)
    b = beta_of(temperature)
    ns = len(q)
    r = grid.r
    k = grid.k
    r2 = np.maximum(r * r, R2_FLOOR)
    W = omega_matrix(grid, species, coords)
    Wk = np.moveaxis(W, -1, 0)                           # [N-1, n, n]
    P = np.diag(rho)
    I = np.eye(ns)
    Zk = np.zeros((grid.N - 1, ns, ns))
    if dielectric is not None:
        zeta, _ = drism_zeta(grid, q, rho, species, coords, temperature, dielectric, drism_a)
        Zk = np.moveaxis(zeta, -1, 0)                   # [N-1, n, n]
    Wp = Wk + P[None] @ Zk                               # omega' = omega + rho zeta
    tau = np.zeros((ns, ns, grid.N - 1))
    total_it = 0
    for scale in charge_steps:
        qq, s, e = _pair_params(q * scale, sig, eps)
        sr6 = (s[..., None] ** 2 / r2) ** 3
        u_lj = 4.0 * e[..., None] * (sr6 * sr6 - sr6)
        bu_s = np.minimum(b * (u_lj + COULOMB * qq[..., None] * np.exp(-r) / r), BETA_U_CAP)
        bU_L = b * 4.0 * np.pi * COULOMB * qq[..., None] / (k * k * (k * k + 1.0))

        def step(tau):
            d = -bu_s + tau
            g = cl.closure_g(d, closure)
            h = g - 1.0
            cs = h - tau
            Cs = grid.forward(cs)
            C = np.moveaxis(Cs - bU_L, -1, 0)            # full c = c_s - beta u_L
            WC = Wp @ C
            H = np.linalg.solve(I[None] - WC @ P[None], WC @ Wp) + Zk   # Eq. 4 in k space
            tau_new = grid.inverse(np.moveaxis(H, 0, -1) - Cs)
            return tau_new - tau, h, cs, np.moveaxis(H, 0, -1)

        hist_t, hist_R = [], []
        rms = np.inf
        for it in range(1, max_iter + 1):
            R, h, cs, H = step(tau)
            rms = float(np.sqrt(np.mean(R * R)))
            if verbose and it % 50 == 0:
                print("1d charge scale", scale, "iter", it, rms)
            if not np.isfinite(rms):
                raise FloatingPointError("1D RISM diverged")
            if rms < tol:
                break
            hist_t.append(tau)
            hist_R.append(R)
            if len(hist_R) > mdiis_nvec:
                hist_t.pop(0)
                hist_R.pop(0)
            kk = len(hist_R)
            B = np.array([[float(np.sum(hist_R[i] * hist_R[j])) for j in range(kk)]
                          for i in range(kk)])
            c, dropped = mdiis.coefficients(B)
            for _ in range(dropped):
                hist_t.pop(0)
                hist_R.pop(0)
            tau = sum(ci * (ti + mdiis_damp * Ri) for ci, ti, Ri in zip(c, hist_t, hist_R))
        total_it += it
    chi = np.empty((ns, ns, grid.N))
    chi[:, :, 1:] = W + rho[:, None, None] * H
    h0 = 4.0 * np.pi * grid.dr * np.sum(r * r * h, axis=-1)
    W0 = np.array([[1.0 if species[a] == species[bb] else 0.0 for bb in range(ns)] for a in range(ns)])
    chi[:, :, 0] = W0 + rho[:, None] * h0
    return dict(chi=chi, dk=grid.dk, h=h, c=cs - b * COULOMB * qq[..., None] * (-np.expm1(-r)) / r,
                grid=grid, iterations=total_it, rms=rms, H=H, W=W)


def solute_1d(chi, grid, site_q, site_sig, site_eps, rho, temperature, solute_q, solute_sig,
              solute_eps, closure=cl.KH, pse_order=3, tol=1e-10, max_iter=20000, mdiis_nvec=5,
              mdiis_damp=0.7):
    """Single-site solute in solvent (Eq. 8 with omega_uu = 1), steps 1-7 in radial form.

    chi: [n, n, N] table on k_j = j dk (the entries j >= 1 are used). Returns dict with
    g, h, c, t, d per solvent site on grid.r, and the SFE integrand sums."""
    b = beta_of(temperature)
    r = grid.r
    k = grid.k
    ns = len(site_q)
    site_q, site_sig, site_eps = (np.asarray(v, dtype=np.float64) for v in (site_q, site_sig, site_eps))
    s = 0.5 * (solute_sig + site_sig)
    e = np.sqrt(solute_eps * site_eps)
    r2 = np.maximum(r * r, R2_FLOOR)
    sr6 = (s[:, None] ** 2 / r2) ** 3
    bu = np.minimum(b * (4.0 * e[:, None] * (sr6 * sr6 - sr6)
                         + COULOMB * solute_q * site_q[:, None] / r), BETA_U_CAP)
    f = b * COULOMB * solute_q * site_q[:, None] * (-np.expm1(-r)) / r          # Eq. 29
    ftil = b * 4.0 * np.pi * COULOMB * solute_q * site_q[:, None] / (k * k * (k * k + 1.0))  # Eq. 30
    X = chi[:, :, 1:]

    def step(t):
        d = -bu + t
        g = cl.closure_g(d, closure, pse_order)
        csr = g - 1.0 - t + f
        ctil = grid.forward(csr) - ftil
        htil = np.einsum("aj,agj->gj", ctil, X)
        h = grid.inverse(htil)
        return h + 1.0 - g, g, d

    t = f.copy()
    hist_t, hist_R = [], []
    for it in range(1, max_iter + 1):
        R, g, d = step(t)
        rms = float(np.sqrt(np.mean(R * R)))
        if rms < tol:
            break
        hist_t.append(t)
        hist_R.append(R)
        if len(hist_R) > mdiis_nvec:
            hist_t.pop(0)
            hist_R.pop(0)
        kk = len(hist_R)
        B = np.array([[float(np.sum(hist_R[i] * hist_R[j])) for j in range(kk)] for i in range(kk)])
        c, dropped = mdiis.coefficients(B)
        for _ in range(dropped):
            hist_t.pop(0)
            hist_R.pop(0)
        t = sum(ci * (ti + mdiis_damp * Ri) for ci, ti, Ri in zip(c, hist_t, hist_R))
    d = -bu + t
    g = cl.closure_g(d, closure, pse_order)
    h = g - 1.0
    c = h - t
    return dict(g=g, h=h, c=c, t=t, d=d, r=r, iterations=it, rms=rms, rho=np.asarray(rho))


def sfe_1d(sol, kind, temperature, pse_order=3):
    """SFE of the single-site solute (radial form of Eqs. 17-18), kcal/mol."""
    from .units import KB_KCAL
    kT = KB_KCAL * temperature
    r = sol["r"]
    dr = r[1] - r[0]
    tot = 0.0
    for g_ in range(sol["g"].shape[0]):
        dens = cl.sfe_density(sol["h"][g_], sol["c"][g_], sol["d"][g_], kind, pse_order)
        tot += kT * sol["rho"][g_] * 4.0 * np.pi * dr * float(np.sum(r * r * dens))
    return tot
