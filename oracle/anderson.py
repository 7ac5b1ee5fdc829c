"""Modified Anderson mixing with two histories (oracle, FP64).

Eqs. 34-39 (Convergence acceleration, Modified Anderson): with X the inputs, Y the outputs,
R^{n-1} = Y^n - X^{n-1} (Eq. 37) and D_i = R^{n-1} - R^{n-1-i} (i = 1, 2), theta solves the
2 x 2 system of Eq. 36,  sum_j <D_j, D_i> theta_j = <R^{n-1}, D_i>,  and with a_i = theta_i + s_i

    u   = X^{n-1} + sum_i a_i (X^{n-1-i} - X^{n-1})                       (Eq. 34)
    v   = Y^n     + sum_i a_i (Y^{n-i}   - Y^n)                           (Eq. 35)
    X^n = u + b (v - u)                                                    (Eq. 39).

Since Y^{n-i} = X^{n-1-i} + R^{n-1-i}, this is X^n = sum_k c_k (X_k + b R_k) over the last
three stored pairs with c_{n-1} = 1 - a_1 - a_2 and c_{n-1-i} = a_i: the same update form as
MDIIS (``oracle.mdiis``) with its own coefficients. Readings: the inner product of Eq. 38
with w = 1/rho read as one scalar (it cancels in theta); the first two steps are Picard
(X^n = X^{n-1} + b R^{n-1}), as the passage states; if the 2 x 2 system is singular (pivot
below ``mdiis.PIVOT_MIN`` after scaling by its largest diagonal entry) the step is Picard.
"""
import numpy as np

from . import mdiis


def coefficients(B, s1=0.2, s2=0.0):
    """Coefficients over the stored residuals ordered oldest -> newest, from their Gram
    matrix B. Returns c (same length as B) with sum(c) = 1."""
    k = B.shape[0]
    if k < 3:
        c = np.zeros(k)
        c[-1] = 1.0
        return c
    n0, n1, n2 = k - 1, k - 2, k - 3          # newest, previous, the one before
    idx = (n1, n2)
    M = np.empty((2, 2))
    rhs = np.empty(2)
    for i in range(2):
        di = idx[i]
        rhs[i] = B[n0, n0] - B[n0, di]
        for j in range(2):
            dj = idx[j]
            M[i, j] = B[n0, n0] - B[n0, dj] - B[n0, di] + B[di, dj]
    scale = max(M[0, 0], M[1, 1])
    c = np.zeros(k)
    if not scale > 0.0:
        c[-1] = 1.0
        return c
    theta, ok = mdiis.gaussian_elimination(M / scale, rhs / scale)
    if not ok:
        c[-1] = 1.0
        return c
    a1, a2 = theta[0] + s1, theta[1] + s2
    c[n0] = 1.0 - a1 - a2
    c[n1] = a1
    c[n2] = a2
    return c
