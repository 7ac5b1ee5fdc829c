"""Pins for the oracle's transform convention and the Eq. 13 contraction.

The oracle uses numpy's FFT; these tests pin it to the definition of the transform
(c~(k) = dV sum_n c(r_n) exp(-i k.(r_n - r0)), written out as a direct sum) and the
k-space product of Eq. 13 to a brute-force circular convolution in real space."""
import numpy as np

from oracle import rism3d
from oracle.potential import grid_points, kvectors_half, signed_index


def _direct_dft(c, n, spacing, origin):
    pts = grid_points(n, spacing, origin).reshape(-1, 3) - np.asarray(origin)
    kv, _ = kvectors_half(n, spacing)
    kflat = kv.reshape(-1, 3)
    dV = float(np.prod(spacing))
    out = np.exp(-1j * kflat @ pts.T) @ c.reshape(-1)
    return dV * out.reshape(kv.shape[:3])


def test_rfftn_matches_direct_dft():
    rng = np.random.default_rng(1)
    for n, sp in (((8, 8, 8), (0.5, 0.5, 0.5)), ((6, 10, 12), (0.4, 0.5, 0.3))):
        c = rng.standard_normal(n)
        origin = (-1.0, 2.0, 0.3)
        dV = float(np.prod(sp))
        got = dV * np.fft.rfftn(c)
        ref = _direct_dft(c, n, sp, origin)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_kvectors_signed_and_nyquist():
    assert list(signed_index(8)) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert list(signed_index(5)) == [0, 1, 2, -2, -1]
    kv, nyq = kvectors_half((8, 6, 4), (0.5, 1.0, 0.25))
    assert kv.shape == (8, 6, 3, 3)
    assert np.isclose(kv[4, 0, 0, 0], -2 * np.pi * 4 / (8 * 0.5))
    assert nyq[4, 0, 0] and nyq[0, 3, 0] and nyq[0, 0, 2] and not nyq[1, 1, 1]


def _toy_problem(n, spacing, n_sites, rng, nk=400, dk=0.05):
    chi = rng.standard_normal((n_sites, n_sites, nk)) * np.exp(-0.02 * np.arange(nk))
    solv = dict(q=np.zeros(n_sites), sigma=np.ones(n_sites), eps=np.zeros(n_sites),
                rho=np.full(n_sites, 0.03), temperature=300.0, chi=chi, dk=dk)
    grid = dict(n=n, spacing=spacing, origin=(0.0, 0.0, 0.0))
    solute = dict(xyz=np.zeros((1, 3)), q=np.zeros(1), sigma=np.ones(1), eps=np.zeros(1))
    return rism3d.Problem(solv, grid, solute), chi


def test_contraction_is_circular_convolution():
    """h_g = sum_a c_a (*) x_ag with x_ag(n) = N^-1 sum_m X_ag(|k_m|) e^{2 pi i m.n/N}, the
    kernel built by an explicit loop over the FULL integer k grid (not the half spectrum)."""
    rng = np.random.default_rng(2)
    n = (8, 8, 8)
    sp = (0.7, 0.7, 0.7)
    P, chi = _toy_problem(n, sp, 2, rng)
    c = rng.standard_normal((2,) + n)
    got = P.rism_h(c)                          # steps 3-5 with f~ = 0
    N = n[0]
    m = np.array([i if i < N // 2 else i - N for i in range(N)])
    kk = 2 * np.pi * m / (N * sp[0])
    kmag = np.sqrt(kk[:, None, None] ** 2 + kk[None, :, None] ** 2 + kk[None, None, :] ** 2)
    X = rism3d.chi_interp(chi, P.dk, kmag)     # [a][g][N][N][N]
    x = np.real(np.fft.ifftn(X, axes=(2, 3, 4)))
    ref = np.zeros_like(c)
    idx = np.arange(N)
    for g in range(2):
        for a in range(2):
            for i in range(N):
                for j in range(N):
                    for k in range(N):
                        shifted = x[a, g][np.ix_((i - idx) % N, (j - idx) % N, (k - idx) % N)]
                        ref[g, i, j, k] += np.sum(c[a] * shifted)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_chi_interp_linear_and_clamped():
    chi = np.zeros((1, 1, 5))
    chi[0, 0] = [0.0, 1.0, 4.0, 9.0, 16.0]
    k = np.array([[[0.0, 0.25, 1.5]], [[3.9, 4.0, 10.0]]])
    got = rism3d.chi_interp(chi, 0.5, k)[0, 0]
    # x = k / dk = 0, 0.5, 3 | 7.8, 8, 20 -> clamped past index 4
    assert np.allclose(got, [[[0.0, 0.5, 9.0]], [[16.0, 16.0, 16.0]]])


def test_roundtrip_and_parseval():
    rng = np.random.default_rng(3)
    c = rng.standard_normal((12, 10, 8))
    C = np.fft.rfftn(c)
    assert np.max(np.abs(np.fft.irfftn(C, s=c.shape, axes=(0, 1, 2)) - c)) < 1e-14
    full = np.fft.fftn(c)
    assert np.isclose(np.sum(np.abs(full) ** 2) / c.size, np.sum(c * c), rtol=1e-13)
