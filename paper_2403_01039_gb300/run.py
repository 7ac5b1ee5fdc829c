"""Command-line 3D-RISM solve: one solute from a text file, a named solvent, a cubic grid.

    python -m paper_2403_01039_gb300.run atoms.txt --solvent water_nacl --n 128 --spacing 0.5 \\
        --closure kh --tol 1e-6 --precision 32 --out result.npz [--dielectric 78.44] [--fields g c]

atoms.txt holds one atom per line, "x y z q sigma eps" (A, e, A, kcal/mol); blank lines and
lines starting with '#' are skipped. The grid is centred on the solute's centroid. The
solvent's susceptibility comes from the library's host 1D solver (XRISM, or DRISM when
--dielectric is given). The output .npz holds the SFE (kcal/mol, total and per site), the
iteration count and final residual, the grid, and the requested fields as float32
[n_sites, N, N, N] arrays. Every step of the solve runs in the library's CUDA kernels; this
module only reads, validates and writes.
"""
import argparse
import json
import sys

import numpy as np

SOLVENTS = ("water3", "water_nacl")
FIELDS = ("g", "c", "h", "t", "u")


def read_atoms(path):
    """(xyz [n, 3], q, sigma, eps) from a whitespace-separated text file."""
    rows = []
    with open(path) as f:
        for lineno, line in enumerate(f, 1):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) != 6:
                raise ValueError("%s:%d: expected 'x y z q sigma eps', got %d fields" % (path, lineno, len(parts)))
            try:
                rows.append([float(v) for v in parts])
            except ValueError:
                raise ValueError("%s:%d: not a number in %r" % (path, lineno, line)) from None
    if not rows:
        raise ValueError("%s: no atoms" % path)
    a = np.array(rows, dtype=np.float64)
    if not np.all(np.isfinite(a)):
        raise ValueError("%s: non-finite value" % path)
    if np.any(a[:, 4] < 0) or np.any(a[:, 5] < 0):
        raise ValueError("%s: sigma and eps must be >= 0" % path)
    return a[:, :3].copy(), a[:, 3].copy(), a[:, 4].copy(), a[:, 5].copy()


def centred_grid(xyz, n, spacing):
    """Cubic grid of n^3 points whose index n/2 sits on the centroid of xyz."""
    c = xyz.mean(axis=0)
    return dict(n=(n, n, n), spacing=(spacing,) * 3, origin=tuple(float(v) - (n // 2) * spacing for v in c))


def parse(argv=None):
    p = argparse.ArgumentParser(prog="python -m paper_2403_01039_gb300.run", description=__doc__.split("\n")[0])
    p.add_argument("atoms", help="text file: x y z q sigma eps per line")
    p.add_argument("--solvent", default="water_nacl", choices=SOLVENTS)
    p.add_argument("--dielectric", type=float, default=None, help="DRISM with this dielectric constant")
    p.add_argument("--n", type=int, default=128, help="grid points per axis (even; N and N/2 5-smooth)")
    p.add_argument("--spacing", type=float, default=0.5)
    p.add_argument("--closure", default="kh", choices=("kh", "hnc", "pse"))
    p.add_argument("--pse-order", type=int, default=3)
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--precision", type=int, default=32, choices=(32, 64))
    p.add_argument("--mdiis", type=int, default=5, help="stored MDIIS vectors")
    p.add_argument("--max-iter", type=int, default=10000)
    p.add_argument("--fields", nargs="*", default=["g"], choices=FIELDS)
    p.add_argument("--out", default="rism3d_result.npz")
    a = p.parse_args(argv)
    if a.n < 2 or a.n % 2:
        p.error("--n must be even")
    if not a.spacing > 0 or not a.tol > 0:
        p.error("--spacing and --tol must be positive")
    return a


def main(argv=None):
    a = parse(argv)
    xyz, q, sigma, eps = read_atoms(a.atoms)
    from . import capi, synth
    sites = synth.solvent_sites(a.solvent)
    chi, dk, _, _ = capi.xrism(sites, dielectric=a.dielectric)
    solvent = dict(sites, chi=chi, dk=dk)
    grid = centred_grid(xyz, a.n, a.spacing)
    sfe_kind = {"kh": "kh", "hnc": "hnc", "pse": "pse"}[a.closure]
    with capi.Solver(solvent, grid, precision=a.precision, mdiis_nvec=a.mdiis, max_iter=a.max_iter) as S:
        S.set_solute(xyz, q, sigma, eps)
        rep = S.solve(a.closure, a.pse_order, a.tol, check=False)
        total, per_site = S.sfe(sfe_kind, a.pse_order)
        out = {f: S.get(f).astype(np.float32) for f in a.fields}
    status = capi.STATUS_NAMES[rep["status"]] if 0 <= rep["status"] < len(capi.STATUS_NAMES) else str(rep["status"])
    np.savez_compressed(a.out, sfe=total, sfe_per_site=per_site, site_names=np.array(sites["names"]),
                        iterations=rep["iterations"], rms=rep["rms"], status=status,
                        n=np.array(grid["n"]), spacing=np.array(grid["spacing"]), origin=np.array(grid["origin"]),
                        **out)
    print(json.dumps(dict(status=status, iterations=rep["iterations"], rms=rep["rms"], sfe_kcal_mol=total,
                          out=a.out)))
    return 0 if status == "OK" else 1


if __name__ == "__main__":
    sys.exit(main())
