"""FP64 CPU oracle for the 3D-RISM fixed-point solve (RISMiCal, arXiv 2403.01039).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it. It shares no code, tables or constants with the
CUDA path; both sides receive the same seeded synthetic inputs (plain arrays)
and nothing else.

The oracle is deliberately plain and slow: direct sums for the potential,
numpy's FFT as the transform primitive (pinned against the direct DFT sum),
dense loops for the closure, Gaussian elimination for the MDIIS system. Every
function cites the paper passage it restates.

Modules
-------
units      physical constants and unit conventions (the paper is silent on them)
potential  Eq. 22 (solute-solvent LJ + Coulomb), Eq. 29 / Eq. 30 (long-range split)
closure    Eqs. 14-16 (HNC, KH) and PSE-n; SFE integrands of Eqs. 17-18, GF, PSE-n
mdiis      Eq. 40 (MDIIS coefficients: bordered Gram system, Gaussian elimination)
rism3d     the solve procedure (steps 1-7 of the Numerical procedure section,
           Eqs. 13, 31-33, 41) and the SFE sums
rism1d     Eq. 4 (XRISM for the pure solvent -> susceptibility X of Eq. 8) and the
           single-site solute-solvent RISM of Eq. 8 used to cross-check 3D
anderson   Eqs. 34-39 (the modified Anderson coefficients with two histories)
thermo     Eq. 19 (partial molar volume), Eq. 20 (pressure), the second Eq. 21
           (solvation force as the SFE gradient)
unet       the learned-guess network (no counterpart in the paper): 3x3x3
           convolutions, pooling, upsampling, MSE and the chain rule, in FP64

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
except the 1D solvent susceptibility values themselves ("parity unpinned"
beyond the low-density limit, the k -> 0 dielectric limits of XRISM and DRISM,
and a single-site solute reproducing the solvent's own ion correlations); chi is
a shared input of both sides, so it cannot break parity.
"""
