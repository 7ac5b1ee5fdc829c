"""MDIIS coefficients (oracle, FP64).

Eq. 40 (Convergence acceleration, Modified DIIS) mixes the stored iterates with
coefficients c_i "decided by the Lagrange multiplier technique". As printed the
update adds b * sum c_i (X - Y) to Y, which has the wrong sign for a residual
R = Y - X. Reading (the standard MDIIS the paper cites): minimise
|| sum_i c_i R_i ||^2 subject to sum_i c_i = 1, i.e. solve the bordered system

    [ B   1 ] [ c      ]   [ 0 ]
    [ 1^T 0 ] [ lambda ] = [ 1 ],      B_ij = <R_i, R_j>,

then form the new input t_new = sum_i c_i (t_i + eta R_i).

Policies (the paper is silent; the CUDA path follows the same ones):
* the inner product is the plain sum over all sites and grid points (Eq. 38's
  weight w = 1/rho is read as one scalar, which cancels in c);
* B is divided by its largest diagonal entry before the solve;
* Gaussian elimination with partial pivoting; if a pivot falls below
  PIVOT_MIN in magnitude the oldest stored vector is dropped and the solve is
  repeated (a single vector always gives c = [1]).
"""
import numpy as np

PIVOT_MIN = 1.0e-12


def gaussian_elimination(A, b):
    """Solve A x = b by Gaussian elimination with partial pivoting, written out.

    Returns (x, ok); ok is False when a pivot is smaller than PIVOT_MIN."""
    A = np.array(A, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    n = A.shape[0]
    for col in range(n):
        p = col + int(np.argmax(np.abs(A[col:, col])))
        if abs(A[p, col]) < PIVOT_MIN:
            return None, False
        if p != col:
            A[[col, p]] = A[[p, col]]
            b[[col, p]] = b[[p, col]]
        for row in range(col + 1, n):
            f = A[row, col] / A[col, col]
            A[row, col:] -= f * A[col, col:]
            b[row] -= f * b[col]
    x = np.zeros(n)
    for row in range(n - 1, -1, -1):
        x[row] = (b[row] - np.dot(A[row, row + 1:], x[row + 1:])) / A[row, row]
    return x, True


def bordered_solve(B):
    """Coefficients c (sum c = 1) minimising the residual norm for Gram matrix B (k x k).

    Returns (c, ok)."""
    k = B.shape[0]
    scale = np.max(np.diag(B))
    Bs = B / scale if scale > 0.0 else B
    A = np.zeros((k + 1, k + 1))
    A[:k, :k] = Bs
    A[:k, k] = 1.0
    A[k, :k] = 1.0
    rhs = np.zeros(k + 1)
    rhs[k] = 1.0
    x, ok = gaussian_elimination(A, rhs)
    return (x[:k] if ok else None), ok


def coefficients(B):
    """Solve for the MDIIS coefficients, dropping the oldest vectors while singular.

    B is the Gram matrix of the stored residuals ordered oldest -> newest.
    Returns (c, n_dropped): c applies to the newest len(c) vectors."""
    k = B.shape[0]
    for drop in range(k):
        sub = B[drop:, drop:]
        if sub.shape[0] == 1:
            return np.ones(1), drop
        c, ok = bordered_solve(sub)
        if ok:
            return c, drop
    return np.ones(1), k - 1


def damping(rms, static_eta, dynamic):
    """Mixing factor eta. Static by default; the dynamic option restates b = -0.2 log(R) of the
    Modified DIIS passage with log base 10 (base not stated), clamped to [0.1, 1]."""
    if not dynamic:
        return static_eta
    return float(min(max(-0.2 * np.log10(rms), 0.1), 1.0))
