"""Pins for the closures (Eqs. 14-16, PSE-n) and the SFE integrands (Eqs. 17-18, GF, PSE-n)."""
import math

import numpy as np

from oracle import closure as cl


def test_closed_forms():
    d = np.array([-2.0, -0.5, 0.0, 0.5, 2.0])
    assert np.allclose(cl.closure_g(d, cl.HNC), np.exp(d), rtol=0, atol=0)
    kh = cl.closure_g(d, cl.KH)
    assert np.allclose(kh, [math.exp(-2.0), math.exp(-0.5), 1.0, 1.5, 3.0], rtol=1e-15)
    pse3 = cl.closure_g(d, cl.PSE, 3)
    assert np.allclose(pse3[:3], np.exp(d[:3]))
    assert np.isclose(pse3[4], 1 + 2 + 2 + 8 / 6.0)


def test_kh_is_pse1_and_continuous():
    d = np.linspace(-5, 5, 1001)
    assert np.array_equal(cl.closure_g(d, cl.KH), cl.closure_g(d, cl.PSE, 1))
    eps = 1e-9
    for kind, n in ((cl.KH, 1), (cl.PSE, 2), (cl.PSE, 5)):
        lo, hi = cl.closure_g(np.array([-eps, eps]), kind, n)
        assert abs(hi - lo) < 3 * eps
        # first derivative also continuous at 0 (both branches have slope 1)
        lo2, hi2 = cl.closure_g(np.array([-2 * eps, 2 * eps]), kind, n)
        assert abs((hi2 - hi) - (lo - lo2)) < 1e-12


def test_pse_tends_to_hnc():
    d = np.linspace(0, 2, 21)
    assert np.max(np.abs(cl.closure_g(d, cl.PSE, 30) - np.exp(d))) < 1e-12
    errs = [np.max(np.abs(cl.closure_g(d, cl.PSE, n) - np.exp(d))) for n in (1, 2, 3, 4, 6)]
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_sfe_integrands():
    rng = np.random.default_rng(0)
    h = rng.uniform(-1, 3, 200)
    c = rng.uniform(-3, 1, 200)
    d = rng.uniform(-3, 3, 200)
    gf = cl.sfe_density(h, c, d, cl.SFE_GF)
    assert np.allclose(gf, -c - 0.5 * h * c)
    hnc = cl.sfe_density(h, c, d, cl.SFE_HNC)
    kh = cl.sfe_density(h, c, d, cl.SFE_KH)
    assert np.allclose(hnc - gf, 0.5 * h * h)
    assert np.allclose(hnc - kh, np.where(h > 0, 0.5 * h * h, 0.0))
    # with h, d taken from the KH closure itself, the PSE-1 SFE integrand equals KH's
    dd = np.linspace(-4, 4, 401)
    hh = cl.closure_g(dd, cl.KH) - 1.0
    cc = rng.uniform(-2, 2, dd.size)
    assert np.allclose(cl.sfe_density(hh, cc, dd, cl.SFE_PSE, 1),
                       cl.sfe_density(hh, cc, dd, cl.SFE_KH), atol=1e-14)
    assert np.allclose(cl.sfe_density(h, c, d, cl.SFE_PSE, 3),
                       hnc - np.where(d > 0, d ** 4 / 24.0, 0.0))
