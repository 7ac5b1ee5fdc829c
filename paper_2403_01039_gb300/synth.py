"""Seeded synthetic inputs: solvent models, solutes and grids.

This module holds parameter tables and random draws only, none of the solver's
arithmetic. The CUDA path and the FP64 oracle both receive what it returns as
plain arrays. Recipes (lengths in Angstrom, energies in kcal/mol, charges in e):

* water, 3 sites (O, H1, H2): O sigma 3.166, eps 0.1553, q -0.8476; H sigma 1.0,
  eps 0.046, q +0.4238; OH 1.0, HOH 109.47 degrees; rho 0.0334 / A^3; T 298.15 K.
* water + NaCl at 0.1 M (5 sites): the water above plus Na+ (sigma 2.1595,
  eps 0.3526418, q +1) and Cl- (sigma 4.8305, eps 0.0127850, q -1), the
  Joung-Cheatham SPC/E ion set; rho_ion = 0.1 mol/L = 6.0221e-5 / A^3.
* random solute: atoms drawn uniformly in a sphere by random sequential addition
  (reject a draw closer than 1.0 A to any accepted atom), sigma ~ U(2.5, 3.8),
  eps ~ U(0.05, 0.2), q ~ N(0, 0.3) shifted so the charges sum to the requested net
  charge; centroid moved to the origin. numpy Generator(PCG64(seed)).
* grid: N^3 points at spacing d with grid index N/2 on the origin, so the solute
  centroid sits at the box centre.
"""
import math
import numpy as np

AVOGADRO_PER_L_TO_A3 = 6.02214076e-4   # mol/L -> molecules / A^3


def water_geometry():
    th = math.radians(109.47)
    return np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [math.cos(th), math.sin(th), 0.0]])


def water_3site(rho=0.0334, temperature=298.15):
    return dict(names=["O", "H1", "H2"],
                q=np.array([-0.8476, 0.4238, 0.4238]),
                sigma=np.array([3.166, 1.0, 1.0]),
                eps=np.array([0.1553, 0.046, 0.046]),
                rho=np.full(3, rho),
                species=np.array([0, 0, 0]),
                coords=water_geometry(),
                temperature=temperature)


def water_nacl_5site(conc_molar=0.1, rho_water=0.0334, temperature=298.15):
    w = water_3site(rho_water, temperature)
    rho_ion = conc_molar * AVOGADRO_PER_L_TO_A3
    return dict(names=w["names"] + ["Na", "Cl"],
                q=np.concatenate([w["q"], [1.0, -1.0]]),
                sigma=np.concatenate([w["sigma"], [2.1595, 4.8305]]),
                eps=np.concatenate([w["eps"], [0.3526418, 0.0127850]]),
                rho=np.concatenate([w["rho"], [rho_ion, rho_ion]]),
                species=np.array([0, 0, 0, 1, 2]),
                coords=np.concatenate([w["coords"], np.zeros((2, 3))]),
                temperature=temperature)


def lj_sphere(sigma=3.73, eps=0.294, q=0.0):
    return dict(xyz=np.zeros((1, 3)), q=np.array([float(q)]), sigma=np.array([float(sigma)]),
                eps=np.array([float(eps)]))


def random_solute(n_atoms, radius, seed, net_charge=0.0, min_dist=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    tries = 0
    while len(pts) < n_atoms:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("could not pack %d atoms in radius %g" % (n_atoms, radius))
        p = rng.uniform(-radius, radius, 3)
        if p @ p > radius * radius:
            continue
        if pts and np.min(np.sum((np.asarray(pts) - p) ** 2, axis=1)) < min_dist * min_dist:
            continue
        pts.append(p)
    xyz = np.asarray(pts)
    xyz -= xyz.mean(axis=0)
    sigma = rng.uniform(2.5, 3.8, n_atoms)
    eps = rng.uniform(0.05, 0.2, n_atoms)
    q = rng.normal(0.0, 0.3, n_atoms)
    q = q - q.mean() + net_charge / n_atoms
    return dict(xyz=xyz, q=q, sigma=sigma, eps=eps)


def cubic_grid(n, spacing):
    """Grid of n^3 points with index n/2 at the origin."""
    return dict(n=(n, n, n), spacing=(spacing,) * 3, origin=(-(n // 2) * spacing,) * 3)


# dielectric constant of water for the DRISM solvent (298 K)
WATER_DIELECTRIC = 78.44


# Workloads ------------------------------------------------------------------
# sphere_32: one neutral LJ sphere in 3-site water (X from 1D DRISM, dielectric constant
#            78.44), 32^3 at 0.5 A, KH, MDIIS 5, FP64.
# solute50_128: 50-atom solute (10 A sphere, seed 2001) in water + 0.1 M NaCl,
#               128^3 at 0.5 A, KH and PSE-3, FP32 and FP64, MDIIS 5.
# globule2000_256: 2000-atom globule (radius 16 A, seed 3001, net +8) in water + NaCl,
#               256^3 at 0.375 A, KH, MDIIS 10.
# globule12877_512: 12877 atoms (radius 32 A, seed 5001, net 0) in water + NaCl, 512^3 at
#               0.5 A, KH, MDIIS 10.
WORKLOADS = {
    "sphere_32": dict(n=32, spacing=0.5, solvent="water3", mdiis_nvec=5, dielectric=WATER_DIELECTRIC),
    "solute50_128": dict(n=128, spacing=0.5, solvent="water_nacl", mdiis_nvec=5,
                         atoms=50, radius=10.0, seed=2001, net_charge=0.0),
    "globule2000_256": dict(n=256, spacing=0.375, solvent="water_nacl", mdiis_nvec=10,
                            atoms=2000, radius=16.0, seed=3001, net_charge=8.0),
    # the paper's grid (512^3 over a 256 A box) and atom count (12 877), net charge 0
    "globule12877_512": dict(n=512, spacing=0.5, solvent="water_nacl", mdiis_nvec=10,
                             atoms=12877, radius=32.0, seed=5001, net_charge=0.0),
}


def smooth_even(n):
    """Smallest m >= n that is even with m / 2 free of prime factors above 5 (the grid sizes
    the transform passes take)."""
    m = int(n) + (int(n) & 1)
    while True:
        k = m // 2
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 2


def batch_workload(count=64, seed0=4000, spacing=0.5):
    """Many small solutes on uneven grids: for seed s = seed0 .. seed0 + count - 1, draw with
    PCG64(s) the atom count n ~ U{20..120} and the grid size N ~ U{64..128} rounded up by
    smooth_even; the solute is random_solute(n, 10 (n/50)^(1/3), s), net charge 0; 3-site
    water, spacing 0.5 A. Returns a list of dict(seed, grid, solute)."""
    out = []
    for s in range(seed0, seed0 + count):
        rng = np.random.Generator(np.random.PCG64(s))
        n_atoms = int(rng.integers(20, 121))
        N = smooth_even(int(rng.integers(64, 129)))
        sol = random_solute(n_atoms, 10.0 * (n_atoms / 50.0) ** (1.0 / 3.0), s)
        out.append(dict(seed=s, grid=cubic_grid(N, spacing), solute=sol))
    return out


def solvent_sites(name):
    return water_3site() if name == "water3" else water_nacl_5site()


def workload_solute(name):
    w = WORKLOADS[name]
    if "atoms" not in w:
        return lj_sphere()
    return random_solute(w["atoms"], w["radius"], w["seed"], w["net_charge"])
