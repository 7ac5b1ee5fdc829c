"""Pins for the potential builder of the oracle (Eq. 22, Eq. 29)."""
import numpy as np

from oracle import potential as pot
from oracle.units import COULOMB, BETA_U_CAP, beta


def _one(sig_a, eps_a, q_a, sig_g, eps_g, q_g, r, T=300.0):
    n = (4, 1, 1)
    sp = (r, 1.0, 1.0)
    bu = pot.beta_u(n, sp, (0.0, 0.0, 0.0), np.zeros((1, 3)), [q_a], [sig_a], [eps_a],
                    [q_g], [sig_g], [eps_g], T)
    return bu[0, 1, 0, 0] / beta(T)          # grid point 1 sits at distance r


def test_lj_closed_forms():
    s_ag, e_ag = pot.lorentz_berthelot(3.0, 0.2, 3.4, 0.05)
    assert np.isclose(s_ag, 3.2) and np.isclose(e_ag, 0.1)
    assert abs(_one(3.0, 0.2, 0.0, 3.4, 0.05, 0.0, s_ag)) < 1e-12
    assert np.isclose(_one(3.0, 0.2, 0.0, 3.4, 0.05, 0.0, 2 ** (1 / 6) * s_ag), -e_ag, rtol=1e-12)


def test_coulomb_closed_form():
    u = _one(1.0, 0.0, 0.5, 1.0, 0.0, -0.8, 2.5)
    assert np.isclose(u, COULOMB * 0.5 * -0.8 / 2.5, rtol=1e-14)


def test_cap_and_floor():
    bu = pot.beta_u((3, 3, 3), (1.0,) * 3, (-1.0,) * 3, np.zeros((1, 3)), [0.0], [3.0], [0.2],
                    [0.0], [3.0], [0.2], 300.0)
    assert bu[0, 1, 1, 1] == BETA_U_CAP
    assert np.all(bu <= BETA_U_CAP)


def test_phi_closed_form_and_superposition():
    xyz = np.array([[0.3, -0.2, 0.1], [1.1, 0.4, -0.7]])
    q = np.array([0.7, -0.25])
    n = (5, 4, 3)
    sp = (0.5, 0.6, 0.7)
    org = (-1.0, -1.0, -1.0)
    phi = pot.phi_long_range(n, sp, org, xyz, q)
    pts = pot.grid_points(n, sp, org)
    ref = np.zeros(n)
    for a in range(2):
        r = np.sqrt(np.sum((pts - xyz[a]) ** 2, axis=-1))
        ref += COULOMB * q[a] * (1.0 - np.exp(-r)) / r
    assert np.max(np.abs(phi - ref)) < 1e-11


def test_whole_cell_shift_is_index_roll():
    rng = np.random.default_rng(4)
    xyz = rng.uniform(-1.5, 1.5, (4, 3))
    q = rng.normal(0, 0.3, 4)
    sig = rng.uniform(2.5, 3.8, 4)
    eps = rng.uniform(0.05, 0.2, 4)
    n = (12, 10, 8)
    sp = (0.5, 0.5, 0.5)
    org = (-3.0, -2.5, -2.0)
    args = ([0.4, -0.8], [1.0, 3.2], [0.05, 0.15], 298.15)
    a = pot.beta_u(n, sp, org, xyz, q, sig, eps, *args, minimum_image=True)
    shift = np.array([2, -3, 1])
    b = pot.beta_u(n, sp, org, xyz + shift * 0.5, q, sig, eps, *args, minimum_image=True)
    assert np.max(np.abs(np.roll(a, tuple(shift), axis=(1, 2, 3)) - b)) < 1e-9 * np.max(np.abs(a))
