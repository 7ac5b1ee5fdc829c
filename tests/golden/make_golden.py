"""Writes the stored inputs and expected values under tests/golden/.

Calls only the FP64 oracle (``oracle/``) and the seeded input generators; nothing here
touches the CUDA path. Run from the repository root:

    python tests/golden/make_golden.py chi          # solvent susceptibility tables (XRISM)
    python tests/golden/make_golden.py drism        # 3-site water from DRISM (eps 78.44)
    python tests/golden/make_golden.py thermo       # bulk pressure, kT chi_T, c(r) of water
    python tests/golden/make_golden.py solute50_128 # full-size reference (slow, ~minutes)
    python tests/golden/make_golden.py globule2000_256  # protein-scale reference (hours)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import rism1d, rism3d, thermo, closure as cl   # noqa: E402
from paper_2403_01039_gb300 import synth           # noqa: E402


def make_chi():
    for name in ("water3", "water_nacl"):
        s = synth.solvent_sites(name)
        t0 = time.time()
        r = rism1d.xrism_solvent(s["q"], s["sigma"], s["eps"], s["rho"], s["species"],
                                 s["coords"], s["temperature"])
        np.savez_compressed(os.path.join(HERE, "chi_%s.npz" % name), chi=r["chi"], dk=r["dk"], h=r["h"],
                            n=2048, dr=0.05, iterations=r["iterations"], rms=r["rms"])
        print(name, "iterations", r["iterations"], "rms %.2e" % r["rms"], "%.1f s" % (time.time() - t0))


def make_drism():
    """X of 3-site water from the oracle's DRISM with the dielectric constant of the
    sphere_32 workload."""
    s = synth.solvent_sites("water3")
    eps_r = synth.WORKLOADS["sphere_32"]["dielectric"]
    t0 = time.time()
    r = rism1d.xrism_solvent(s["q"], s["sigma"], s["eps"], s["rho"], s["species"], s["coords"],
                             s["temperature"], dielectric=eps_r)
    np.savez_compressed(os.path.join(HERE, "chi_water3_drism.npz"), chi=r["chi"], dk=r["dk"], n=2048,
                        dr=0.05, dielectric=eps_r, iterations=r["iterations"], rms=r["rms"])
    print("water3 DRISM iterations", r["iterations"], "rms %.2e" % r["rms"], "%.1f s" % (time.time() - t0))


def make_thermo():
    """Bulk pressure (Eq. 20), k_B T chi_T and the full direct correlation c(r) (every 8th
    radial point from r = dr) of 3-site water from the oracle's 1D solve."""
    s = synth.solvent_sites("water3")
    r = rism1d.xrism_solvent(s["q"], s["sigma"], s["eps"], s["rho"], s["species"], s["coords"],
                             s["temperature"])
    P = thermo.pressure(r["c"], r["grid"].r, s["rho"], s["species"], s["temperature"])
    kt = thermo.kT_chi_T(r["chi"], s["rho"])
    np.savez_compressed(os.path.join(HERE, "thermo_water3.npz"), pressure=P, kT_chi_T=kt,
                        c_every8=r["c"][:, :, ::8])
    print("water3 pressure %.10g kcal/mol/A^3, kT chi_T %.10g A^3" % (P, kt))


def sample_points(n, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n, size=(count, 3))


def make_full(workload, closures=((cl.KH, 3, "kh"), (cl.PSE, 3, "pse3")), tols=(1e-6, 1e-10)):
    """Oracle solves of a full-size workload; stores the solution at 1024 seeded grid points
    (all sites), g on the whole x = N/2 plane (all sites; float64 at 1e-6, float32 at tighter
    tolerances) plus SFEs and iteration counts in tests/golden/<workload>_reference.npz."""
    w = synth.WORKLOADS[workload]
    s = synth.solvent_sites(w["solvent"])
    chi = np.load(os.path.join(HERE, "chi_%s.npz" % w["solvent"]))
    solv = dict(q=s["q"], sigma=s["sigma"], eps=s["eps"], rho=s["rho"],
                temperature=s["temperature"], chi=chi["chi"], dk=float(chi["dk"]))
    grid = synth.cubic_grid(w["n"], w["spacing"])
    P = rism3d.Problem(solv, grid, synth.workload_solute(workload), workers=8, threads=5)
    pts = sample_points(w["n"], 1024, 7)
    idx = (slice(None), pts[:, 0], pts[:, 1], pts[:, 2])
    xp = w["n"] // 2
    out = dict(points=pts, plane_x=xp)
    for kind, order, tag in closures:
        for tol in tols:
            t0 = time.time()
            sol = rism3d.solve(P, kind, order, tol=tol, mdiis_nvec=w["mdiis_nvec"], verbose=True)
            sfe_kind = {cl.KH: cl.SFE_KH, cl.HNC: cl.SFE_HNC, cl.PSE: cl.SFE_PSE}[kind]
            tot, per = rism3d.sfe(P, sol, sfe_kind, order)
            gf, _ = rism3d.sfe(P, sol, cl.SFE_GF, order)
            key = "%s_%g" % (tag, tol)
            out[key + "_iterations"] = sol["iterations"]
            out[key + "_rms"] = sol["rms"]
            out[key + "_sfe"] = tot
            out[key + "_sfe_per_site"] = per
            out[key + "_sfe_gf"] = gf
            out[key + "_g"] = sol["g"][idx]
            out[key + "_c"] = sol["c"][idx]
            out[key + "_t"] = sol["t"][idx]
            out[key + "_g_max"] = float(sol["g"].max())
            plane = sol["g"][:, xp]
            out[key + "_g_plane"] = plane if tol >= 1e-6 else plane.astype(np.float32)
            print(workload, tag, tol, sol["iterations"], sol["converged"], tot,
                  "%.0f s" % (time.time() - t0), flush=True)
            np.savez_compressed(os.path.join(HERE, "%s_reference.npz" % workload), **out)


def make_globule(workload="globule2000_256", tol=1e-10, snapshots=(1e-6, 1e-8), workers=8, threads=5):
    """One KH oracle solve of the protein-scale workload to ``tol``, with the solutions a
    solve stopped at each of ``snapshots`` returns (the same run). Stores, for each
    tolerance, g, c and t at 4096 seeded grid points (all sites), the whole x = N/2 plane
    of g (all sites; float64 at the loosest tolerance, float32 otherwise), the KH and GF
    SFE (total and per site) and the iteration count, in tests/golden/<workload>_reference.npz."""
    w = synth.WORKLOADS[workload]
    s = synth.solvent_sites(w["solvent"])
    chi = np.load(os.path.join(HERE, "chi_%s.npz" % w["solvent"]))
    solv = dict(q=s["q"], sigma=s["sigma"], eps=s["eps"], rho=s["rho"],
                temperature=s["temperature"], chi=chi["chi"], dk=float(chi["dk"]))
    grid = synth.cubic_grid(w["n"], w["spacing"])
    t0 = time.time()
    P = rism3d.Problem(solv, grid, synth.workload_solute(workload), workers=workers, threads=threads)
    print("setup %.0f s" % (time.time() - t0), flush=True)
    pts = sample_points(w["n"], 4096, 7)
    idx = (slice(None), pts[:, 0], pts[:, 1], pts[:, 2])
    xp = w["n"] // 2
    sol = rism3d.solve(P, cl.KH, 1, tol=tol, mdiis_nvec=w["mdiis_nvec"], verbose=True,
                       snapshots=snapshots)
    print("solve %.0f s, %d iterations, converged %s" % (time.time() - t0, sol["iterations"], sol["converged"]),
          flush=True)
    out = dict(points=pts, plane_x=xp)
    loosest = max(snapshots) if snapshots else tol
    runs = [(tol, sol["t"], sol["iterations"], sol["rms"])]
    runs += [(k, v["t"], v["iterations"], v["rms"]) for k, v in sol["snapshots"].items()]
    for tl, t, iters, rms in runs:
        r = rism3d.solution_from_t(P, t, cl.KH, 1)
        tot, per = rism3d.sfe(P, r, cl.SFE_KH, 1)
        gf, gf_per = rism3d.sfe(P, r, cl.SFE_GF, 1)
        key = "kh_%g" % tl
        out[key + "_iterations"] = iters
        out[key + "_rms"] = rms
        out[key + "_sfe"] = tot
        out[key + "_sfe_per_site"] = per
        out[key + "_sfe_gf"] = gf
        out[key + "_g"] = r["g"][idx]
        out[key + "_c"] = r["c"][idx]
        out[key + "_t"] = r["t"][idx]
        out[key + "_g_max"] = float(r["g"].max())
        plane = r["g"][:, xp]
        out[key + "_g_plane"] = plane if tl == loosest else plane.astype(np.float32)
        print(workload, tl, iters, tot, gf, flush=True)
    np.savez_compressed(os.path.join(HERE, "%s_reference.npz" % workload), **out)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "chi"
    if what == "chi":
        make_chi()
    elif what == "thermo":
        make_thermo()
    elif what == "drism":
        make_drism()
    elif what.startswith("globule"):
        make_globule(what)
    else:
        make_full(what)
