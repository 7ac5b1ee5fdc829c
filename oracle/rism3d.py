"""3D-RISM fixed-point solve (oracle, FP64), in the paper's step order.

Numerical procedure section, steps 1-7:
  1. t_gamma = f_gamma (Eq. 29) as the initial guess (or a supplied guess);
  2. closure (Eqs. 14-16, PSE-n) gives g; c^sr = g - 1 - t + f (Eq. 31);
  3. Fourier transform, c~ = c~^sr - f~ (Eq. 32, f~ from Eq. 30);
  4. 3D-RISM equation h~_gamma = sum_alpha c~_alpha X_alpha,gamma(|k|) (Eq. 13);
  5. inverse transform; t' = t + h + 1 - g (Eq. 33), i.e. residual R = t' - t;
  6. new input from MDIIS (Eq. 40, read as in ``oracle.mdiis``);
  7. repeat until the RMS residual is below the tolerance.
PSE-n and HNC are reached by closure continuation (``closure_stages``).

Readings (the paper is silent or garbled):
* transform convention: c~(k) = dV sum_n c(r_n) exp(-i k.(r_n - r0)) and
  h(r) = (N dV)^-1 sum_k h~(k) exp(i k.(r - r0)) on the periodic integer k grid
  k_m = 2 pi m / (N d), m in [-N/2, N/2); numpy's FFT is the transform primitive
  (pinned against the direct DFT sum by the tests);
* X(|k|) by linear interpolation in k on the tabulated X(k_j), k_j = j dk,
  clamped to the last entry past the table end;
* residual: Eq. 41 prints the mean of sqrt((t^j - t^{j-1})^2); the oracle stops on
  RMS = sqrt(sum R^2 / (N n_v)) with R = t' - t (Eq. 33) and also records the printed
  mean-absolute form;
* the returned solution is the last input t with g, c from its closure and h = g - 1;
* half-integer grid (option kgrid="half"; the numerical-procedure section places k at
  half-integers): k_m = 2 pi (m + 1/2) / (N d) on every axis, c~(k) = dV sum_n c(r_n)
  exp(-i k.(r_n - r0)) evaluated as the DFT of c(r_n) exp(-i pi sum_d n_d / N_d), and the
  inverse with the conjugate factor; no k is zero, so Phi~ needs no special points.
"""
import numpy as np

from . import anderson
from . import closure as cl
from . import mdiis
from .potential import (beta_u, phi_long_range, phik_long_range, kvectors_half, kvectors_shifted,
                        phik_long_range_shifted)
from .units import beta as beta_of, KB_KCAL


def chi_interp(chi, dk, kmag):
    """X_ag(|k|) by linear interpolation on the table chi[a][g][j] at k_j = j dk.

    Past the last table point the last value is used. Returns [n_a, n_g] + kmag.shape."""
    nk = chi.shape[2]
    x = np.asarray(kmag, dtype=np.float64) / dk
    j = np.minimum(np.floor(x).astype(np.int64), nk - 2)
    w = np.clip(x - j, 0.0, 1.0)
    return chi[:, :, j] * (1.0 - w) + chi[:, :, j + 1] * w


class Problem:
    """All inputs of one solve: solvent, grid and solute, plus the fields derived from them
    once per solute (beta*u, f, f~, X on the half spectrum).

    ``minimum_image`` evaluates the real-space potentials with the minimum-image
    convention; it exists only for the whole-cell shift test. ``kgrid`` = "integer" (the
    periodic grid) or "half" (half-integer k on every axis). ``workers`` > 1 evaluates the
    direct potential sums of Eqs. 22 and 29 over slabs of x planes in that many processes
    (each grid point's sum is the same as in one process); ``threads`` > 1 runs the steps of
    an iteration site by site in that many threads (the same operations per site; only the
    order of the contraction's sum over sites may differ in rounding)."""

    def __init__(self, solvent, grid, solute, minimum_image=False, kgrid="integer", workers=1, threads=1):
        self.threads = int(threads)
        self.n = tuple(int(v) for v in grid["n"])
        self.spacing = tuple(float(v) for v in grid["spacing"])
        self.origin = tuple(float(v) for v in grid["origin"])
        self.site_q = np.asarray(solvent["q"], dtype=np.float64)
        self.site_sig = np.asarray(solvent["sigma"], dtype=np.float64)
        self.site_eps = np.asarray(solvent["eps"], dtype=np.float64)
        self.rho = np.asarray(solvent["rho"], dtype=np.float64)
        self.temperature = float(solvent["temperature"])
        self.chi = np.asarray(solvent["chi"], dtype=np.float64)
        self.dk = float(solvent["dk"])
        self.beta = beta_of(self.temperature)
        self.dV = float(np.prod(self.spacing))
        self.n_sites = len(self.site_q)
        xyz = np.asarray(solute["xyz"], dtype=np.float64).reshape(-1, 3)
        q = np.asarray(solute["q"], dtype=np.float64)
        sig = np.asarray(solute["sigma"], dtype=np.float64)
        eps = np.asarray(solute["eps"], dtype=np.float64)
        # Eq. 22 and Eq. 29 on the grid
        args = (self.n, self.spacing, self.origin, xyz, q, sig, eps, self.site_q, self.site_sig,
                self.site_eps, self.temperature, minimum_image)
        if workers > 1:
            self.bu, self.phi = _potentials_parallel(args, int(workers))
        else:
            self.bu, self.phi = _potentials_slab(args + (None,))
        # Eq. 30: f_gamma = beta q_gamma phi, f~_gamma = beta q_gamma Phi~
        if kgrid not in ("integer", "half"):
            raise ValueError("kgrid must be 'integer' or 'half'")
        self.kgrid = kgrid
        if kgrid == "half":
            self.phik = phik_long_range_shifted(self.n, self.spacing, self.origin, xyz, q)
            kv = kvectors_shifted(self.n, self.spacing)
            ph = [np.exp(-1j * np.pi * np.arange(N) / N) for N in self.n]
            self.shift = ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
        else:
            self.phik = phik_long_range(self.n, self.spacing, self.origin, xyz, q)
            kv, _ = kvectors_half(self.n, self.spacing)
        bq = self.beta * self.site_q
        self.f = bq[:, None, None, None] * self.phi[None]
        self.ftil = bq[:, None, None, None] * self.phik[None]
        self.kmag = np.sqrt(np.sum(kv * kv, axis=-1))
        self.chik = chi_interp(self.chi, self.dk, self.kmag)   # [a][g][kx][ky][kz]

    # ---- step 2
    def closure(self, t, kind, pse_order):
        d = -self.bu + t
        g = cl.closure_g(d, kind, pse_order)
        return d, g

    # ---- steps 3-5
    def rism_h(self, csr):
        """h_gamma(r) from c^sr via Eqs. 32 and 13 (steps 3-5)."""
        axes = (1, 2, 3)
        if self.kgrid == "half":
            ctil = self.dV * np.fft.fftn(csr * self.shift, axes=axes) - self.ftil
            htil = np.einsum("a...,ag...->g...", ctil, self.chik)
            return (np.fft.ifftn(htil, axes=axes) * np.conj(self.shift)).real / self.dV
        ctil = self.dV * np.fft.rfftn(csr, axes=axes) - self.ftil            # Eq. 32
        htil = np.einsum("a...,ag...->g...", ctil, self.chik)                 # Eq. 13
        return np.fft.irfftn(htil, s=self.n, axes=axes) / self.dV           # step 5

    def map_sites(self, fn, n_sites=None):
        """[fn(site) for every site], in ``threads`` threads when more than one."""
        n = self.n_sites if n_sites is None else n_sites
        if self.threads <= 1:
            return [fn(g) for g in range(n)]
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(min(self.threads, n)) as ex:
            return list(ex.map(fn, range(n)))

    def residual_threaded(self, t, kind, pse_order):
        """residual() with every step split by site over ``threads`` threads (integer k grid)."""
        axes = (0, 1, 2)
        d = np.empty_like(t)
        g = np.empty_like(t)
        csr = np.empty_like(t)

        def close(a):
            d[a] = -self.bu[a] + t[a]
            g[a] = cl.closure_g(d[a], kind, pse_order)
            csr[a] = g[a] - 1.0 - t[a] + self.f[a]                          # Eq. 31
        self.map_sites(close)
        ctil = self.map_sites(lambda a: self.dV * np.fft.rfftn(csr[a], axes=axes) - self.ftil[a])   # Eq. 32
        R = np.empty_like(t)

        def contract(gam):
            htil = sum(ctil[a] * self.chik[a, gam] for a in range(self.n_sites))   # Eq. 13
            R[gam] = np.fft.irfftn(htil, s=self.n, axes=axes) / self.dV + 1.0 - g[gam]   # Eq. 33
        self.map_sites(contract)
        return R, g, d

    def residual(self, t, kind, pse_order):
        """One application of steps 2-5: returns (R, g, d) with R = t' - t = h + 1 - g."""
        if self.threads > 1 and self.kgrid == "integer":
            return self.residual_threaded(t, kind, pse_order)
        d, g = self.closure(t, kind, pse_order)
        csr = g - 1.0 - t + self.f                                           # Eq. 31
        h = self.rism_h(csr)
        return h + 1.0 - g, g, d                                             # Eq. 33


def _potentials_slab(args):
    """beta*u (Eq. 22) and phi (Eq. 29) on the x planes args[-1] = (x0, x1) (None: all)."""
    n, spacing, origin, xyz, q, sig, eps, sq, ss, se, temp, mi, xr = args
    bu = beta_u(n, spacing, origin, xyz, q, sig, eps, sq, ss, se, temp, minimum_image=mi, x_range=xr)
    phi = phi_long_range(n, spacing, origin, xyz, q, minimum_image=mi, x_range=xr)
    return bu, phi


def _potentials_parallel(args, workers):
    import multiprocessing as mp
    nx = args[0][0]
    edges = np.linspace(0, nx, min(workers, nx) + 1).astype(int)
    jobs = [args + ((int(a), int(b)),) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_potentials_slab, jobs)
    return (np.concatenate([p[0] for p in parts], axis=1), np.concatenate([p[1] for p in parts], axis=0))


def closure_stages(kind, pse_order):
    """Closure continuation (the paper is silent): an exponential closure started from
    t = f overflows for charged solutes, so PSE-n is reached through PSE-1 (= KH), PSE-2, ...,
    PSE-n and HNC through KH, each stage starting from the previous stage's solution."""
    if kind == cl.KH:
        return [(cl.KH, 1)]
    if kind == cl.PSE:
        return [(cl.KH, 1)] + [(cl.PSE, n) for n in range(2, pse_order + 1)]
    if kind == cl.HNC:
        return [(cl.KH, 1), (cl.HNC, 0)]
    raise ValueError("unknown closure %r" % (kind,))


STAGE_TOL = 1.0e-4   # tolerance of every stage but the last one (the last uses tol)


def solve(problem, kind=cl.KH, pse_order=3, tol=1e-6, max_iter=10000, mdiis_nvec=5,
          mdiis_damp=0.7, dynamic_damp=False, t_guess=None, verbose=False, accel="mdiis",
          anderson_s=(0.2, 0.0), snapshots=()):
    """Run steps 1-7 (per closure stage) and return a dict with t, g, h, c, d, the total
    iteration count and the RMS history. ``accel`` is "mdiis" (Eq. 40) or "anderson" (the
    modified Anderson method of Eqs. 34-39 with two histories, shifts ``anderson_s`` and
    mixing b = ``mdiis_damp``).

    ``snapshots``: tolerances above ``tol``; for each, the result also holds (under
    ``"snapshots"``, keyed by the tolerance) the input t of the first iteration of the last
    closure stage whose RMS residual fell below it, with its iteration count: the solution a
    solve stopped at that tolerance returns, taken from the same run.

    The Gram entries <R_i, R_j> of the stored residuals do not change while the pair stays
    in the history, so each iteration computes only the new residual's row (the same sums
    a full recomputation gives)."""
    if accel == "anderson":
        mdiis_nvec = 3
    P = problem
    t = P.f.copy() if t_guess is None else np.array(t_guess, dtype=np.float64, copy=True)  # step 1
    stages = closure_stages(kind, pse_order)
    rms_log, mad_log = [], []
    snaps = {}
    pending = sorted((float(s) for s in snapshots if s > tol), reverse=True)
    converged = False
    total = 0
    for si, (skind, sorder) in enumerate(stages):
        last = si == len(stages) - 1
        stol = tol if last else max(tol, STAGE_TOL)
        hist_t, hist_R = [], []
        gram = np.zeros((0, 0))
        converged = False
        while total < max_iter:
            total += 1
            R, g, d = P.residual(t, skind, sorder)
            rms = float(np.sqrt(np.mean(R * R)))
            rms_log.append(rms)
            mad_log.append(float(np.mean(np.abs(R))))
            if verbose and (total % 20 == 0 or total < 5):
                print("iter %d stage %d rms %.3e" % (total, si, rms), flush=True)
            if not np.isfinite(rms):
                break
            while last and pending and rms < pending[0]:
                snaps[pending.pop(0)] = dict(t=t.copy(), iterations=total, rms=rms)
            if rms < stol:
                converged = True
                break
            if total >= max_iter:
                break
            # step 6: MDIIS
            if P.threads > 1:
                row = np.array([sum(P.map_sites(lambda a: float(np.sum(Ri[a] * R[a])))) for Ri in hist_R + [R]])
            else:
                row = np.array([float(np.sum(Ri * R)) for Ri in hist_R] + [float(np.sum(R * R))])
            hist_t.append(t)
            hist_R.append(R)
            k = len(hist_R)
            grown = np.empty((k, k))
            grown[:k - 1, :k - 1] = gram
            grown[k - 1, :] = row
            grown[:, k - 1] = row
            gram = grown
            if k > mdiis_nvec:
                hist_t.pop(0)
                hist_R.pop(0)
                gram = gram[1:, 1:]
            B = gram.copy()
            if accel == "anderson":
                c, dropped = anderson.coefficients(B, *anderson_s), 0
            else:
                c, dropped = mdiis.coefficients(B)
            for _ in range(dropped):
                hist_t.pop(0)
                hist_R.pop(0)
            gram = gram[dropped:, dropped:]
            eta = mdiis.damping(rms, mdiis_damp, dynamic_damp)
            if P.threads > 1:
                tn = np.empty_like(t)

                def update(a):
                    tn[a] = sum(ci * (ti[a] + eta * Ri[a]) for ci, ti, Ri in zip(c, hist_t, hist_R))
                P.map_sites(update)
                t = tn
            else:
                t = sum(ci * (ti + eta * Ri) for ci, ti, Ri in zip(c, hist_t, hist_R))
        if not converged:
            break
    d, g = P.closure(t, kind, pse_order)
    h = g - 1.0
    c = h - t
    return dict(t=t, g=g, h=h, c=c, d=d, iterations=total, converged=converged,
                rms=rms_log[-1] if rms_log else float("nan"), rms_log=rms_log, mad_log=mad_log,
                snapshots=snaps)


def solution_from_t(problem, t, kind, pse_order=3):
    """The returned fields of a solve stopped at input t: g, d from its closure, h = g - 1,
    c = h - t (the returned-solution reading)."""
    d, g = problem.closure(t, kind, pse_order)
    h = g - 1.0
    return dict(t=t, g=g, h=h, c=h - t, d=d)


def sfe(problem, sol, kind, pse_order=3):
    """Solvation free energy in kcal/mol: k_B T sum_gamma rho_gamma dV sum_grid (integrand),
    Eq. 17 (HNC), Eq. 18 (KH), GF and PSE-n. Returns (total, per_site)."""
    P = problem
    kT = KB_KCAL * P.temperature
    per = np.empty(P.n_sites)
    for g_ in range(P.n_sites):
        dens = cl.sfe_density(sol["h"][g_], sol["c"][g_], sol["d"][g_], kind, pse_order)
        per[g_] = kT * P.rho[g_] * P.dV * float(np.sum(dens))
    return float(np.sum(per)), per
