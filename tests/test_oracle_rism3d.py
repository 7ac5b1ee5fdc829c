"""Pins for the 3D-RISM solve of the oracle (steps 1-7, Eqs. 13, 17-18, 29-33, 40-41)."""
import numpy as np
import pytest

from oracle import rism1d, rism3d, closure as cl
from oracle.potential import grid_points
from paper_2403_01039_gb300 import synth

from conftest import GOLDEN


def _solvent(name, water3, water_nacl):
    return water3 if name == "water3" else water_nacl


def test_zero_potential_gives_zero_correlations(water3):
    solute = dict(xyz=np.zeros((1, 3)), q=np.zeros(1), sigma=np.ones(1), eps=np.zeros(1))
    P = rism3d.Problem(water3, synth.cubic_grid(16, 0.5), solute)
    assert np.all(P.bu == 0.0) and np.all(P.f == 0.0)
    sol = rism3d.solve(P, cl.KH, tol=1e-12)
    assert sol["converged"] and sol["iterations"] == 1
    assert np.all(sol["t"] == 0.0) and np.all(sol["g"] == 1.0)
    assert np.all(sol["h"] == 0.0) and np.all(sol["c"] == 0.0)
    for kind in (cl.SFE_KH, cl.SFE_HNC, cl.SFE_GF, cl.SFE_PSE):
        assert rism3d.sfe(P, sol, kind)[0] == 0.0


@pytest.fixture(scope="module")
def sphere32(water3):
    P = rism3d.Problem(water3, synth.cubic_grid(32, 0.5), synth.lj_sphere())
    return P, rism3d.solve(P, cl.KH, tol=1e-9)


def test_sphere_cubic_symmetry(sphere32):
    """A sphere on grid index N/2 is invariant under axis permutations and the reflections
    n -> (N - n) mod N, so g must be too (to rounding)."""
    P, sol = sphere32
    g = sol["g"]
    assert sol["converged"]
    for perm in ((0, 2, 1, 3), (0, 3, 2, 1), (0, 2, 3, 1)):
        assert np.max(np.abs(np.transpose(g, perm) - g)) < 1e-10
    refl = np.roll(np.flip(g, axis=1), 1, axis=1)
    assert np.max(np.abs(refl - g)) < 1e-10
    assert np.max(np.abs(g[1] - g[2])) < 1e-8          # H1 and H2 equivalent


def test_sphere_matches_1d_rism(sphere32):
    """Under spherical symmetry Eq. 13 is the single-site Eq. 8: the 3D grid solution must
    match the 1D solution on 2048 x 0.05 A up to discretisation and box images
    (measured: max|dg| 0.027 (O), 0.094 (H); SFE 8.31 vs 8.05 kcal/mol)."""
    P, sol = sphere32
    d = np.load(GOLDEN + "/chi_water3.npz")
    g1 = rism1d.RadialGrid(int(d["n"]), float(d["dr"]))
    s = synth.water_3site()
    u = rism1d.solute_1d(d["chi"], g1, s["q"], s["sigma"], s["eps"], s["rho"], s["temperature"],
                         0.0, 3.73, 0.294, tol=1e-11)
    r = np.sqrt(np.sum(grid_points(P.n, P.spacing, P.origin) ** 2, axis=-1))
    m = r < 6.0
    for site, tol in ((0, 0.05), (1, 0.15), (2, 0.15)):
        gi = np.interp(r, u["r"], u["g"][site])
        assert np.max(np.abs(sol["g"][site][m] - gi[m])) < tol
    e3 = rism3d.sfe(P, sol, cl.SFE_KH)[0]
    e1 = rism1d.sfe_1d(u, cl.SFE_KH, s["temperature"])
    assert abs(e3 - e1) < 0.5


def test_sfe_tolerance_dependence(water3):
    """SFE at residual 1e-6 and 1e-9 agree within 0.02 kcal/mol (Performance section, Fig. 5)."""
    P = rism3d.Problem(water3, synth.cubic_grid(32, 0.5), synth.lj_sphere())
    a = rism3d.sfe(P, rism3d.solve(P, cl.KH, tol=1e-6), cl.SFE_KH)[0]
    b = rism3d.sfe(P, rism3d.solve(P, cl.KH, tol=1e-9), cl.SFE_KH)[0]
    assert abs(a - b) < 0.02


def _ion(xyz, s):
    return dict(xyz=np.asarray(xyz, dtype=float).reshape(1, 3), q=[1.0], sigma=[s["sigma"][3]],
                eps=[s["eps"][3]])


def test_ion_matches_1d_rism(water_nacl):
    """Na+ slightly off a grid point: Eqs. 29-32 in 3D against the radial solution. Measured
    max|dg_O| 0.75 at r < 6 A; dropping, doubling or conjugating f~, or losing the grid-origin
    phase, each gives > 3.4."""
    s = water_nacl
    off = np.array([0.13, -0.21, 0.07])
    P = rism3d.Problem(s, synth.cubic_grid(32, 0.5), _ion(off, s))
    sol = rism3d.solve(P, cl.KH, tol=1e-8)
    d = np.load(GOLDEN + "/chi_water_nacl.npz")
    g1 = rism1d.RadialGrid(int(d["n"]), float(d["dr"]))
    u = rism1d.solute_1d(d["chi"], g1, s["q"], s["sigma"], s["eps"], s["rho"], s["temperature"],
                         1.0, s["sigma"][3], s["eps"][3], tol=1e-11)
    r = np.sqrt(np.sum((grid_points(P.n, P.spacing, P.origin) - off) ** 2, axis=-1))
    m = r < 6.0
    gi = np.interp(r, u["r"], u["g"][0])
    assert np.max(np.abs(sol["g"][0][m] - gi[m])) < 1.5


def test_whole_cell_shift_charged(water_nacl):
    """Moving a charged solute by whole grid cells (minimum-image real-space fields) rolls the
    solution by the same cells: pins the exp(-i k.(R - r0)) phase of Eq. 30."""
    s = water_nacl
    shift = np.array([2, -3, 1])
    grid = synth.cubic_grid(24, 0.5)
    xyz = np.array([0.3, 0.2, -0.1])
    P1 = rism3d.Problem(s, grid, _ion(xyz, s), minimum_image=True)
    P2 = rism3d.Problem(s, grid, _ion(xyz + 0.5 * shift, s), minimum_image=True)
    a = rism3d.solve(P1, cl.KH, tol=1e-10)
    b = rism3d.solve(P2, cl.KH, tol=1e-10)
    assert a["converged"] and b["converged"]
    assert np.max(np.abs(np.roll(a["g"], tuple(shift), axis=(1, 2, 3)) - b["g"])) < 1e-8


def test_closure_continuation_and_pse1(water3):
    P = rism3d.Problem(water3, synth.cubic_grid(16, 0.5), synth.lj_sphere())
    kh = rism3d.solve(P, cl.KH, tol=1e-10)
    p1 = rism3d.solve(P, cl.PSE, 1, tol=1e-10)
    assert np.array_equal(kh["g"], p1["g"]) and kh["iterations"] == p1["iterations"]
    assert rism3d.closure_stages(cl.PSE, 3) == [(cl.KH, 1), (cl.PSE, 2), (cl.PSE, 3)]
    p3 = rism3d.solve(P, cl.PSE, 3, tol=1e-10)
    assert p3["converged"]
    # the returned fields satisfy the PSE-3 closure and the step-5 fixed point
    R, g, d = P.residual(p3["t"], cl.PSE, 3)
    assert np.sqrt(np.mean(R * R)) < 1e-10 and np.array_equal(g, p3["g"])
