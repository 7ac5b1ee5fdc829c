"""Pins for the oracle's k-space long-range field (Eq. 30) against a real-space
construction that shares nothing with it.

Eq. 30 gives the transform of the long-range function (1 - e^{-r})/r of Eq. 29 as
4 pi / (k^2 (k^2 + 1)) = 4 pi / k^2 - 4 pi / (k^2 + 1). On a periodic box of side L the
Fourier series (1/V) sum_k Phi~(k) e^{ik.(r - R)} over the box's reciprocal lattice is then
the lattice sum of 1/r minus the lattice sum of the Yukawa function e^{-r}/r, each taken
with k = 0 removed (zero mean). The 1/r sum is evaluated by Ewald summation (Gaussian
screening: an erfc real-space sum over images plus a Gaussian-damped reciprocal sum, minus
pi / (alpha^2 V) for the mean), the Yukawa sum directly over images (it decays
exponentially). On the half-integer grid (kgrid = 1) the reciprocal vectors are
2 pi (m + 1/2) / L, the series is anti-periodic, and both sums take the image n with sign
(-1)^(n_x + n_y + n_z) and no mean term.

The grid's series stops at |m| < N/2 on every axis (on the integer grid the Nyquist planes
are zero by reading, which keeps the spectrum Hermitian), so the two agree to a truncation
error that falls as the grid is refined at fixed L. The terms cut on one axis, summed over
the other two, give a field concentrated within ~1/k_max of the line through each charge
along that axis (up to 0.2 of a field of 100 at 0.5 A spacing there, a few 1e-4 of it
elsewhere), so the comparison leaves out points within 1 A of the axis-parallel lines
through the charges; it bounds the error at the 0.5 A spacing of the workloads and checks
that it shrinks from 1 A to 0.5 A. A wrong phase sign, a wrong phase reference, a dropped
"+1", a wrong normalisation or a wrong charge weighting each moves the field by a large
fraction of its size."""
import itertools

import numpy as np
from scipy.special import erfc

from oracle import potential as pot
from oracle.units import COULOMB

ORIGIN = (-3.0, 1.5, 2.25)


def _charges(L, h):
    """Two unequal charges at off-grid points, 3-4 A apart."""
    o = np.asarray(ORIGIN)
    xyz = np.array([o + [L / 2 + 0.3 * h, L / 2 - 0.2 * h, L / 2 + 0.45 * h],
                    o + [L / 2 - 3.0 + 0.15 * h, L / 2 + 1.4 + 0.35 * h, L / 2 - 1.1 + 0.05 * h]])
    return xyz, np.array([1.0, -0.6])


def _lattice_sum(points, xyz, q, L, anti, alpha=0.35, n_img=2, m_rec=12, n_yuk=3):
    """C sum_a q_a [Ewald(1/r) - Yukawa] at each point, periodic (zero mean) or anti-periodic.
    With alpha = 0.35 / A and L = 16 A the omitted real-space images are below erfc(14) and
    the omitted reciprocal terms below exp(-30) of the largest."""
    V = L ** 3
    if anti:
        m = np.arange(-m_rec, m_rec) + 0.5
        M = np.array(list(itertools.product(m, m, m)))
    else:
        m = np.arange(-m_rec, m_rec + 1, dtype=np.float64)
        M = np.array(list(itertools.product(m, m, m)))
        M = M[np.any(M != 0.0, axis=1)]
    K = 2.0 * np.pi * M / L
    k2 = np.sum(K * K, axis=1)
    w_rec = 4.0 * np.pi / V * np.exp(-k2 / (4.0 * alpha ** 2)) / k2
    total = np.zeros(len(points))
    for R, qa in zip(xyz, q):
        d0 = points - R
        ew = np.zeros(len(points))
        for n in itertools.product(range(-n_img, n_img + 1), repeat=3):
            s = (-1.0) ** (sum(n) % 2) if anti else 1.0
            r = np.linalg.norm(d0 + np.asarray(n) * L, axis=1)
            ew += s * erfc(alpha * r) / r
        ew += np.cos(d0 @ K.T) @ w_rec
        yk = np.zeros(len(points))
        for n in itertools.product(range(-n_yuk, n_yuk + 1), repeat=3):
            s = (-1.0) ** (sum(n) % 2) if anti else 1.0
            r = np.linalg.norm(d0 + np.asarray(n) * L, axis=1)
            yk += s * np.exp(-r) / r
        if not anti:
            ew -= np.pi / (alpha ** 2 * V)
            yk -= 4.0 * np.pi / V
        total += COULOMB * qa * (ew - yk)
    return total


def _sample(N, h, count=300):
    """Grid indices and positions origin + index * h of a seeded sample of grid points."""
    rng = np.random.default_rng(11)
    idx = rng.integers(0, N, size=(count, 3))
    return idx, np.asarray(ORIGIN) + h * idx


def _field_error(N, h, anti):
    L = N * h
    n, sp = (N, N, N), (h, h, h)
    xyz, q = _charges(L, h)
    idx, pts = _sample(N, h)
    if anti:
        ph = pot.phik_long_range_shifted(n, sp, ORIGIN, xyz, q)
        # (1/V) sum_k Phi~ e^{ik.(r_n - r0)}, k = 2 pi (m + 1/2) / L: numpy's inverse DFT
        # times N^3 / V, times e^{i pi (n_x + n_y + n_z) / N} for the half-index shift
        full = np.fft.ifftn(ph) * (N ** 3 / L ** 3)
        vals = full[idx[:, 0], idx[:, 1], idx[:, 2]] * np.exp(1j * np.pi * idx.sum(axis=1) / N)
        assert np.max(np.abs(vals.imag)) <= 1e-10 * np.max(np.abs(vals.real))
        vals = vals.real
    else:
        ph = pot.phik_long_range(n, sp, ORIGIN, xyz, q)
        full = np.fft.irfftn(ph, s=n, axes=(0, 1, 2)) / h ** 3
        vals = full[idx[:, 0], idx[:, 1], idx[:, 2]]
    ref = _lattice_sum(pts, xyz, q, L, anti)
    keep = np.ones(len(pts), dtype=bool)
    for R in xyz:
        d = pts - R
        d -= L * np.round(d / L)
        for ax in range(3):
            other = [a for a in range(3) if a != ax]
            keep &= np.hypot(d[:, other[0]], d[:, other[1]]) >= 1.0
    assert keep.sum() >= 100
    return np.max(np.abs(vals - ref)[keep]), np.max(np.abs(ref))


def test_eq30_field_is_the_periodic_lattice_sum():
    err_fine, scale = _field_error(32, 0.5, anti=False)
    err_coarse, _ = _field_error(16, 1.0, anti=False)
    assert err_fine <= 1e-3 * scale, (err_fine, scale)
    assert err_fine < 0.2 * err_coarse, (err_fine, err_coarse)


def test_eq30_half_grid_field_is_the_antiperiodic_lattice_sum():
    err_fine, scale = _field_error(32, 0.5, anti=True)
    err_coarse, _ = _field_error(16, 1.0, anti=True)
    assert err_fine <= 1e-3 * scale, (err_fine, scale)
    assert err_fine < 0.2 * err_coarse, (err_fine, err_coarse)
