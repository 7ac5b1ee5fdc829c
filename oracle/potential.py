"""Solute -> grid potentials (oracle, FP64, direct sums).

Paper passages restated here:
* Eq. 22 (Hybrid implementation, MM/3D-RISM): u_gamma(r) = sum_alpha [ q_alpha q_gamma / |r - R_alpha|
  + 4 eps_ag ((sigma_ag / |r - R_alpha|)^12 - (sigma_ag / |r - R_alpha|)^6) ].
* Eq. 29 (Numerical procedure): long-range part f_gamma(r) = sum_alpha beta q_alpha q_gamma
  (1 - exp(-|r - R_alpha|)) / |r - R_alpha|.
* Eq. 30: its Fourier transform f~_gamma(k) = sum_alpha 4 pi beta q_alpha q_gamma
  exp(-i k.R_alpha) / (k^2 (k^2 + 1)).

Readings (the paper is silent): Lorentz-Berthelot mixing sigma_ag = (sigma_a + sigma_g)/2,
eps_ag = sqrt(eps_a eps_g) ("usual meanings"); no cutoff; r^2 floored at R2_FLOOR and
beta*u capped from above at BETA_U_CAP; f~ on the periodic integer k grid with the
phase taken relative to the grid origin r0, and f~ := 0 at k = 0 and on every plane
whose index is the Nyquist index -N/2 (this keeps the spectrum Hermitian).

The shared solute fields are returned without the solvent factor:
phi(r) = COULOMB sum_alpha q_alpha (1 - exp(-r_alpha)) / r_alpha, so f_gamma = beta q_gamma phi;
Phi~(k) = sum_alpha 4 pi COULOMB q_alpha exp(-i k.(R_alpha - r0)) / (k^2 (k^2 + 1)),
so f~_gamma = beta q_gamma Phi~.
"""
import numpy as np

from .units import COULOMB, R2_FLOOR, BETA_U_CAP, beta as beta_of


def grid_points(n, spacing, origin, x_range=None):
    """Cartesian coordinates of every grid point, shape (Nx, Ny, Nz, 3).

    Grid index (i, j, k) sits at origin + (i dx, j dy, k dz). ``x_range`` = (x0, x1) keeps
    only the planes x0 <= i < x1 (same coordinates as in the whole grid)."""
    axes = [origin[d] + spacing[d] * np.arange(n[d], dtype=np.float64) for d in range(3)]
    if x_range is not None:
        axes[0] = axes[0][x_range[0]:x_range[1]]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def lorentz_berthelot(sig_a, eps_a, sig_g, eps_g):
    """Mixing rule for the LJ pair parameters of Eq. 22 (reading: Lorentz-Berthelot)."""
    return 0.5 * (sig_a + sig_g), np.sqrt(eps_a * eps_g)


def _pair_r2(points, R, box=None):
    d = points - R
    if box is not None:                       # minimum image (shift-invariance test only)
        d = d - box * np.round(d / box)
    return np.maximum(np.sum(d * d, axis=-1), R2_FLOOR)


def beta_u(n, spacing, origin, xyz, q, sig, eps, site_q, site_sig, site_eps, temperature,
           minimum_image=False, x_range=None):
    """Reduced solute-solvent potential beta*u_gamma(r) of Eq. 22 on the grid.

    Direct sum over every solute atom at every grid point, no cutoff.
    Returns an array [n_sites, Nx, Ny, Nz] (only the planes of ``x_range`` if given);
    beta*u is capped above at BETA_U_CAP."""
    b = beta_of(temperature)
    pts = grid_points(n, spacing, origin, x_range)
    box = np.asarray(spacing, dtype=np.float64) * np.asarray(n) if minimum_image else None
    out = np.zeros((len(site_q),) + pts.shape[:3], dtype=np.float64)
    for a in range(len(q)):
        r2 = _pair_r2(pts, np.asarray(xyz[a], dtype=np.float64), box)
        r = np.sqrt(r2)
        for g in range(len(site_q)):
            s_ag, e_ag = lorentz_berthelot(sig[a], eps[a], site_sig[g], site_eps[g])
            sr6 = (s_ag * s_ag / r2) ** 3
            u_lj = 4.0 * e_ag * (sr6 * sr6 - sr6)
            u_coul = COULOMB * q[a] * site_q[g] / r
            out[g] += b * (u_lj + u_coul)
    return np.minimum(out, BETA_U_CAP)


def phi_long_range(n, spacing, origin, xyz, q, minimum_image=False, x_range=None):
    """Shared long-range field phi(r) = COULOMB sum_a q_a (1 - e^{-r_a}) / r_a (Eq. 29 without
    the factor beta q_gamma). 1 - e^{-r} is evaluated as -expm1(-r)."""
    pts = grid_points(n, spacing, origin, x_range)
    box = np.asarray(spacing, dtype=np.float64) * np.asarray(n) if minimum_image else None
    out = np.zeros(pts.shape[:3], dtype=np.float64)
    for a in range(len(q)):
        r = np.sqrt(_pair_r2(pts, np.asarray(xyz[a], dtype=np.float64), box))
        out += COULOMB * q[a] * (-np.expm1(-r)) / r
    return out


def signed_index(N):
    """DFT index m in [-N/2, N/2) for positions 0..N-1 (numpy fftfreq order times N)."""
    m = np.arange(N)
    return np.where(m < (N + 1) // 2, m, m - N) if N % 2 else np.where(m < N // 2, m, m - N)


def kvectors_half(n, spacing):
    """Wave vectors of the real-to-complex half spectrum [Nx, Ny, Nz//2+1, 3] and the mask of
    points that lie on a Nyquist plane (any index equal to -N/2 for even N)."""
    ks, nyq = [], []
    for d in range(3):
        N = n[d]
        m = signed_index(N) if d < 2 else np.arange(N // 2 + 1)
        ks.append(2.0 * np.pi * m / (N * spacing[d]))
        nyq.append((N % 2 == 0) & (np.abs(m) == N // 2))
    KX, KY, KZ = np.meshgrid(*ks, indexing="ij")
    NX, NY, NZ = np.meshgrid(*nyq, indexing="ij")
    return np.stack([KX, KY, KZ], axis=-1), (NX | NY | NZ)


def phik_long_range(n, spacing, origin, xyz, q):
    """Phi~(k) on the half spectrum: sum_a 4 pi COULOMB q_a exp(-i k.(R_a - r0)) / (k^2 (k^2+1))
    (Eq. 30 without beta q_gamma). Zero at k = 0 and on Nyquist planes."""
    kv, nyq = kvectors_half(n, spacing)
    k2 = np.sum(kv * kv, axis=-1)
    zero = (k2 == 0.0) | nyq
    k2s = np.where(zero, 1.0, k2)
    amp = 4.0 * np.pi * COULOMB / (k2s * (k2s + 1.0))
    out = np.zeros(k2.shape, dtype=np.complex128)
    r0 = np.asarray(origin, dtype=np.float64)
    for a in range(len(q)):
        phase = kv @ (np.asarray(xyz[a], dtype=np.float64) - r0)
        out += q[a] * amp * np.exp(-1j * phase)
    out[zero] = 0.0
    return out


def kvectors_shifted(n, spacing):
    """Wave vectors of the half-integer grid k_m = 2 pi (m + 1/2) / (N d), m in [-N/2, N/2)
    per axis (numpy FFT order), on the full spectrum [Nx, Ny, Nz, 3]; no k is zero."""
    ks = [2.0 * np.pi * (signed_index(n[d]) + 0.5) / (n[d] * spacing[d]) for d in range(3)]
    KX, KY, KZ = np.meshgrid(*ks, indexing="ij")
    return np.stack([KX, KY, KZ], axis=-1)


def phik_long_range_shifted(n, spacing, origin, xyz, q):
    """Phi~(k) of Eq. 30 (without beta q_gamma) on the half-integer grid (full spectrum)."""
    kv = kvectors_shifted(n, spacing)
    k2 = np.sum(kv * kv, axis=-1)
    amp = 4.0 * np.pi * COULOMB / (k2 * (k2 + 1.0))
    out = np.zeros(k2.shape, dtype=np.complex128)
    r0 = np.asarray(origin, dtype=np.float64)
    for a in range(len(q)):
        out += q[a] * amp * np.exp(-1j * (kv @ (np.asarray(xyz[a], dtype=np.float64) - r0)))
    return out
