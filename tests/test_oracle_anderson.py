"""Pins for the modified Anderson coefficients (Eqs. 34-39)."""
import numpy as np

from oracle import anderson, mdiis, rism3d, closure as cl
from paper_2403_01039_gb300 import synth


def _direct(Rs, s1, s2):
    """Eqs. 34-36 written on the vectors themselves (not the Gram matrix)."""
    R2, R1, R0 = Rs                         # oldest -> newest
    D = [R0 - R1, R0 - R2]
    M = np.array([[D[j] @ D[i] for j in range(2)] for i in range(2)])
    rhs = np.array([R0 @ D[i] for i in range(2)])
    th = np.linalg.solve(M, rhs)
    a1, a2 = th[0] + s1, th[1] + s2
    return np.array([a2, a1, 1 - a1 - a2])


def test_matches_vector_form():
    rng = np.random.default_rng(7)
    Rs = rng.standard_normal((3, 40))
    B = Rs @ Rs.T
    for s1, s2 in ((0.2, 0.0), (0.0, 0.0), (0.3, 0.4)):
        assert np.allclose(anderson.coefficients(B, s1, s2), _direct(Rs, s1, s2), rtol=1e-12)


def test_zero_shift_is_diis_minimiser():
    """With s = 0, theta minimises |(1 - sum theta) R0 + sum theta_j R_j|: the DIIS problem
    over the same three vectors."""
    rng = np.random.default_rng(8)
    Rs = rng.standard_normal((3, 25))
    B = Rs @ Rs.T
    c_diis, dropped = mdiis.coefficients(B)
    assert dropped == 0
    assert np.allclose(anderson.coefficients(B, 0.0, 0.0), c_diis, rtol=1e-10, atol=1e-12)


def test_picard_for_first_two_steps_and_sum():
    assert np.array_equal(anderson.coefficients(np.eye(1)), [1.0])
    assert np.array_equal(anderson.coefficients(np.diag([1.0, 2.0])), [0.0, 1.0])
    rng = np.random.default_rng(9)
    Rs = rng.standard_normal((3, 10))
    assert np.isclose(np.sum(anderson.coefficients(Rs @ Rs.T, 0.2, 0.0)), 1.0)


def test_anderson_solve_reaches_the_same_fixed_point(water3):
    """The accelerator changes the path, not the solution (paper's parameters s1 = 0.2,
    s2 = 0, b = 0.6)."""
    P = rism3d.Problem(water3, synth.cubic_grid(16, 0.5), synth.lj_sphere())
    a = rism3d.solve(P, cl.KH, tol=1e-10, accel="anderson", mdiis_damp=0.6)
    m = rism3d.solve(P, cl.KH, tol=1e-10)
    assert a["converged"] and m["converged"]
    assert np.max(np.abs(a["g"] - m["g"])) < 1e-8
