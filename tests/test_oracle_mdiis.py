"""Pins for the MDIIS coefficients of the oracle (Eq. 40 read as the bordered DIIS system)."""
import numpy as np

from oracle import mdiis


def test_gaussian_elimination_against_lapack():
    rng = np.random.default_rng(5)
    for n in (2, 3, 6, 11):
        A = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal(n)
        x, ok = mdiis.gaussian_elimination(A, b)
        assert ok
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    # a zero leading entry needs the row swap
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    x, ok = mdiis.gaussian_elimination(A, np.array([2.0, 3.0]))
    assert ok and np.allclose(x, [3.0, 2.0])


def test_single_vector_is_damped_picard():
    c, dropped = mdiis.coefficients(np.array([[4.0]]))
    assert dropped == 0 and np.array_equal(c, [1.0])


def test_orthogonal_residuals_closed_form():
    # minimise |sum c_i R_i|^2 with sum c_i = 1 and <R_i,R_j> = n_i delta_ij: c_i ∝ 1/n_i
    norms = np.array([4.0, 1.0, 0.25, 2.0])
    c, dropped = mdiis.coefficients(np.diag(norms))
    ref = (1.0 / norms) / np.sum(1.0 / norms)
    assert dropped == 0 and np.allclose(c, ref, rtol=1e-14)


def test_minimiser_property():
    rng = np.random.default_rng(6)
    R = rng.standard_normal((5, 50))
    B = R @ R.T
    c, dropped = mdiis.coefficients(B)
    assert dropped == 0 and np.isclose(np.sum(c), 1.0)
    best = np.sum((c @ R) ** 2)
    for _ in range(200):
        v = rng.standard_normal(5) * 0.05
        v -= v.mean()
        assert np.sum(((c + v) @ R) ** 2) >= best - 1e-12


def test_duplicate_history_drops_oldest():
    r1 = np.array([1.0, 0.0, 0.0])
    r2 = np.array([0.0, 1.0, 0.5])
    R = np.stack([r1, r1, r2])                  # oldest two identical -> singular
    B = R @ R.T
    c, dropped = mdiis.coefficients(B)
    assert dropped == 1
    Rs = R[1:]
    n = np.sum(Rs * Rs, axis=1)
    # remaining two are orthogonal: c ∝ 1/n
    assert np.allclose(c, (1 / n) / np.sum(1 / n))


def test_dynamic_damping():
    assert mdiis.damping(1e-3, 0.7, False) == 0.7
    assert np.isclose(mdiis.damping(1e-3, 0.7, True), 0.6)
    assert mdiis.damping(10.0, 0.7, True) == 0.1
    assert mdiis.damping(1e-9, 0.7, True) == 1.0
