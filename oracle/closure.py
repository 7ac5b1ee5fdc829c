"""Closures and SFE integrands (oracle, FP64).

* HNC, Eq. 14: g = exp(d), with d = -beta u + h - c = -beta u + t (Eq. 16).
* KH, Eq. 15-16. As printed, Eq. 15 swaps the two branches (and the 1D form, Eq. 6,
  switches at d = 1). Reading: the Kovalenko-Hirata form g = exp(d) for d <= 0 and
  g = 1 + d for d > 0, the only one continuous at d = 0, non-negative, and consistent
  with the Theta(-h) of Eq. 18.
* PSE-n (partial series expansion; not in the paper, required as a third closure):
  g = exp(d) for d <= 0, g = sum_{i=0..n} d^i / i! for d > 0. PSE-1 is KH.

SFE integrands per site (multiply by k_B T rho_gamma dV and sum over the grid):
* HNC, Eq. 17:  -c - h c / 2 + h^2 / 2
* KH,  Eq. 18:  -c - h c / 2 + Theta(-h) h^2 / 2
* GF (Gaussian fluctuation; not in the paper): -c - h c / 2
* PSE-n (not in the paper): -c - h c / 2 + h^2 / 2 - Theta(d) d^(n+1) / (n+1)!
"""
import math
import numpy as np

KH, HNC, PSE = 1, 2, 3
SFE_KH, SFE_HNC, SFE_GF, SFE_PSE = 1, 2, 3, 4


def closure_g(d, kind, pse_order=3):
    """g(d) for the given closure; d = -beta u + t."""
    d = np.asarray(d, dtype=np.float64)
    if kind == HNC:
        return np.exp(d)
    if kind == KH:
        return np.where(d <= 0.0, np.exp(np.minimum(d, 0.0)), 1.0 + d)
    if kind == PSE:
        if pse_order < 1:
            raise ValueError("PSE order must be >= 1")
        series = np.ones_like(d)
        term = np.ones_like(d)
        for i in range(1, pse_order + 1):
            term = term * d / i
            series = series + term
        return np.where(d <= 0.0, np.exp(np.minimum(d, 0.0)), series)
    raise ValueError("unknown closure %r" % (kind,))


def sfe_density(h, c, d, kind, pse_order=3):
    """Integrand of the SFE for one site (dimensionless; times k_B T rho dV gives kcal/mol)."""
    base = -c - 0.5 * h * c
    if kind == SFE_HNC:
        return base + 0.5 * h * h
    if kind == SFE_KH:
        return base + np.where(h < 0.0, 0.5 * h * h, 0.0)
    if kind == SFE_GF:
        return base
    if kind == SFE_PSE:
        n1 = pse_order + 1
        tail = np.where(d > 0.0, d ** n1 / math.factorial(n1), 0.0)
        return base + 0.5 * h * h - tail
    raise ValueError("unknown SFE kind %r" % (kind,))
