#!/usr/bin/env python
"""Benchmark: converged 3D-RISM solves/s (and site-gridpoint-iterations/s) at 1e-6 residual.

Workload (default ``globule2000_256``, the largest configuration that fits one GPU): a
seeded 2000-atom synthetic globule (16 A sphere, net charge +8) in 3-site water + 0.1 M NaCl
(5 sites), 256^3 grid at 0.375 A, KH closure, MDIIS with 10 vectors, FP32 form (FP64 Gram,
MDIIS solve, SFE and Coulomb sums), tolerance 1e-6. ``--workload solute50_128`` is the
50-atom, 128^3 x 0.5 A, MDIIS-5 configuration. One step is one whole solve through the C ABI:
rism3d_set_solute (potential + long-range field + initial guess), rism3d_solve (all
iterations), rism3d_get_sfe. The solvent susceptibility comes from the library's own 1D
solver (rism1d_xrism) once, before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own copy of the workload (independent solves,
no collective on the data path: "replicas only"); value = all ranks' solves / the slowest
rank's time. ``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only), on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged 3D-RISM solves/s & site-gridpoint-iters/s at 1e-6 residual"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="globule2000_256")
    p.add_argument("--no-cufft", action="store_true",
                   help="skip the cuFFT comparison (torch.fft transforms of the same fields)")
    p.add_argument("--precision", type=int, default=32, choices=[32, 64])
    p.add_argument("--closure", default="kh", choices=["kh", "pse", "hnc"])
    p.add_argument("--pse-order", type=int, default=3)
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-sample-iters", type=int, default=2)
    p.add_argument("--cpu-sample-atoms", type=int, default=4,
                   help="atoms whose direct potential sums the CPU baseline times (scaled to all)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--inflight", type=int, default=8, help="batch64: jobs in flight")
    p.add_argument("--no-forms", action="store_true",
                   help="skip the batched and learned-guess forms measured after the main line")
    p.add_argument("--split-passes", action="store_true",
                   help="run the plane passes as split element/transform kernels")
    p.add_argument("--no-kernel-events", action="store_true",
                   help="time the solves without per-kernel CUDA events (no roofline)")
    p.add_argument("--profile-iters", type=int, default=0,
                   help="profiling case for ncu: one solve of the workload capped at this many "
                        "iterations, no timing, no JSON line")
    p.add_argument("--nx", type=int, default=0,
                   help="with --profile-iters: grid planes along x (0: the workload's own), a "
                        "smaller case with the same per-plane launch shapes")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_inputs(name, chi_source):
    from paper_2403_01039_gb300 import synth
    w = synth.WORKLOADS[name]
    sites = synth.solvent_sites(w["solvent"])
    chi, dk = chi_source(sites, w.get("dielectric"))
    solv = dict(sites)
    solv.update(chi=chi, dk=dk)
    grid = synth.cubic_grid(w["n"], w["spacing"])
    solute = synth.workload_solute(name)
    return w, solv, grid, solute


def product_chi(sites, dielectric=None):
    """X of the solvent from the library's host 1D solver (XRISM; DRISM when the workload
    names a dielectric constant)."""
    from paper_2403_01039_gb300 import capi
    chi, dk, _, _ = capi.xrism(sites, dielectric=dielectric)
    return chi, dk


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            out_dir = os.environ.get("RISM_BENCH_OUT", tempfile.gettempdir())
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, "bench_clocks_rank%d.csv" % self.index)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits", "-lms",
                 "200", "-i", str(self.index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm),
                    reasons=sorted(reasons))


NOMINAL_HBM_GBS = 7900.0        # GB300 HBM3e nominal bandwidth, for context beside the measured peak


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s, one earlier GB300 copy measurement; MEASURED_PEAKS.json absent)"


def ncu_traffic(kernel, workload):
    """dram bytes per launch from a committed ncu summary, if it was taken on the current
    kernel source (its hash is stored beside the figure); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    src = os.path.join(ROOT, "paper_2403_01039_gb300", "csrc", "rism3d_kernels.cuh")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("kernels_sha") != h:
        return None
    return e.get("dram_bytes_per_launch")


class _HostClock:
    """Wall and CPU time (all threads of this process and its finished children) of a host region: their ratio is the number
    of host cores the oracle kept busy, which numpy's BLAS may make more than one."""

    @staticmethod
    def _cpu():
        t = os.times()           # this process (all threads) and its finished child processes
        return t.user + t.system + t.children_user + t.children_system

    def __enter__(self):
        self.w0, self.c0 = time.perf_counter(), self._cpu()
        return self

    def __exit__(self, *exc):
        self.wall = time.perf_counter() - self.w0
        self.cpu = self._cpu() - self.c0
        return False


def _cores_used(*clocks):
    wall = sum(c.wall for c in clocks)
    cpu = sum(c.cpu for c in clocks)
    ratio = cpu / wall if wall > 0 else 1.0
    return max(1, int(round(ratio))), ratio


def oracle_sample(solv, grid, solute, closure, pse_order, mdiis_nvec, n_iter, n_atoms_sample, warm=0, par=1,
                  budget_s=0.0):
    """The FP64 oracle as it stands, timed on a bounded sample of one solve of a workload.

    Setup: the oracle's Problem built with the first a = n_atoms_sample atoms (its direct
    potential sums of Eqs. 22, 29 and 30 grow with the atom count, the rest does not), plus
    those a atoms' sums timed alone; the whole solute's setup is then
    T_problem(a) + (n / a - 1) T_sums(a). With a >= n the whole solute is built and timed.
    Iterations: n_iter iterations of steps 2-6 on that Problem (their cost does not depend on
    the atoms), after ``warm`` untimed ones; with ``budget_s`` > 0 the iterations continue
    past n_iter until they have taken that long (at most 20). ``par`` > 1 runs the oracle's
    parallel forms on that many host cores (potential sums over x-plane slabs in processes,
    iteration steps site by site in threads). Returns (t_setup, t_iter, clocks, description)."""
    from oracle import rism3d as orc, closure as cl, potential as pot
    kinds = {"kh": cl.KH, "pse": cl.PSE, "hnc": cl.HNC}
    n = len(solute["q"])
    a = min(n, max(1, int(n_atoms_sample)) * max(1, par))     # a few atoms per core
    sub = {k: solute[k][:a] for k in ("xyz", "q", "sigma", "eps")}
    with _HostClock() as cs:
        P = orc.Problem(solv, grid, sub, workers=par, threads=par)
    clocks = [cs]
    t_setup = cs.wall
    how = "setup of all %d atoms %.1f s" % (n, t_setup)
    if a < n:
        with _HostClock() as ca:
            args = (P.n, P.spacing, P.origin, sub["xyz"], sub["q"], sub["sigma"], sub["eps"], P.site_q,
                    P.site_sig, P.site_eps, P.temperature, False)
            if par > 1:
                orc._potentials_parallel(args, par)
            else:
                orc._potentials_slab(args + (None,))
            pot.phik_long_range(P.n, P.spacing, P.origin, sub["xyz"], sub["q"])
        clocks.append(ca)
        t_setup = cs.wall + (n / a - 1.0) * ca.wall
        how = ("setup with %d of %d atoms %.1f s, of which the atom sums %.1f s, scaled to all atoms "
               "%.1f s" % (a, n, cs.wall, ca.wall, t_setup))
    if warm:
        orc.solve(P, kinds[closure], pse_order, tol=1e-300, max_iter=warm, mdiis_nvec=mdiis_nvec)
    with _HostClock() as ci:
        orc.solve(P, kinds[closure], pse_order, tol=1e-300, max_iter=n_iter, mdiis_nvec=mdiis_nvec)
    if budget_s > 0 and ci.wall < budget_s and n_iter < 20:
        # time again with as many iterations as fit the budget (the history is rebuilt)
        n_iter = int(min(20, max(n_iter + 1, n_iter * budget_s / max(ci.wall, 1e-9))))
        with _HostClock() as ci:
            orc.solve(P, kinds[closure], pse_order, tol=1e-300, max_iter=n_iter, mdiis_nvec=mdiis_nvec)
    clocks.append(ci)
    t_iter = ci.wall / n_iter
    return t_setup, t_iter, clocks, how + "; %d iterations %.2f s each" % (n_iter, t_iter)


def oracle_iterations(workload, closure, tol, fallback):
    """The oracle's own iteration count to ``tol`` for a workload (stored reference), else
    ``fallback`` = (count, source)."""
    import numpy as np
    ref = os.path.join(ROOT, "tests", "golden", "%s_reference.npz" % workload)
    key = "%s_%g_iterations" % ({"kh": "kh", "pse": "pse3"}.get(closure, closure), tol)
    if os.path.exists(ref):
        d = np.load(ref)
        if key in d:
            return int(d[key]), "the oracle's own iteration count (stored reference)"
    return fallback


def cpu_baseline(args, w, solv, grid, solute, n_iter_gpu):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the same
    workload (oracle_sample), extrapolated to a whole solve with the iteration count the
    oracle needs for this workload (stored reference), else the GPU solve's count: once on
    one core (the line's value) and once with the oracle's parallel forms on every core."""
    import numpy as np
    n_full, src = oracle_iterations(args.workload, args.closure, args.tol,
                                    (n_iter_gpu, "the GPU solve's iteration count"))
    legs = []
    ncpu = os.cpu_count() or 1
    for par in (1, ncpu):
        t_setup, t_iter, clocks, how = oracle_sample(solv, grid, solute, args.closure, args.pse_order,
                                                     w["mdiis_nvec"], args.cpu_sample_iters,
                                                     args.cpu_sample_atoms, par=par, budget_s=10.0)
        cores, ratio = _cores_used(*clocks)
        legs.append(dict(value=1.0 / (t_setup + n_full * t_iter), unit="solves/s", cores=cores, kind="oracle",
                         sample="%s of %s; host CPU time / wall time %.2f (%d cores available, %d used by "
                                "the oracle's parallel forms); extrapolated to %d iterations (%s)"
                                % (how, args.workload, ratio, ncpu, par, n_full, src),
                         site_gridpoint_iters_per_s=len(solv["q"]) * float(np.prod(grid["n"])) / t_iter))
        if ncpu == 1:
            break
    out = dict(legs[0])
    if len(legs) > 1:
        out["all_cores"] = legs[1]
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_2403_01039_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    sites = synth.solvent_sites(w["solvent"])
    # the oracle's own 1D solver provides its susceptibility
    from oracle import rism1d
    r1 = rism1d.xrism_solvent(sites["q"], sites["sigma"], sites["eps"], sites["rho"], sites["species"],
                              sites["coords"], sites["temperature"], dielectric=w.get("dielectric"))
    solv = dict(sites)
    solv.update(chi=r1["chi"], dk=r1["dk"])
    grid = synth.cubic_grid(w["n"], w["spacing"])
    solute = synth.workload_solute(args.workload)
    # one step = one iteration of steps 2-6 (a bounded sample of the solve)
    t_setup, t_iter, clocks, how = oracle_sample(solv, grid, solute, args.closure, args.pse_order,
                                                 w["mdiis_nvec"], args.steps, args.cpu_sample_atoms,
                                                 warm=args.warmup)
    cores, ratio = _cores_used(*clocks)
    n_full, src = oracle_iterations(args.workload, args.closure, args.tol, (None, None))
    if n_full is None:
        if len(sites["q"]) * int(np.prod(grid["n"])) <= 1 << 20:       # small: count them
            from oracle import rism3d as orc, closure as cl
            P = orc.Problem(solv, grid, solute)
            kind = {"kh": cl.KH, "pse": cl.PSE, "hnc": cl.HNC}[args.closure]
            n_full = orc.solve(P, kind, args.pse_order, tol=args.tol, mdiis_nvec=w["mdiis_nvec"])["iterations"]
            src = "counted by an untimed oracle solve"
        else:
            n_full, src = 569, "assumed (the FP64 GPU solve's count on globule2000_256; no stored reference)"
    value = 1.0 / (t_setup + n_full * t_iter)
    sample = ("%s; host CPU time / wall time %.2f (%d cores available); extrapolated to the %d "
              "iterations of a converged solve (%s)" % (how, ratio, os.cpu_count() or 0, n_full, src))
    line = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=t_iter * 1e3, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, grid="%d^3 x %.3g A" % (w["n"], w["spacing"]),
                            sites=len(sites["q"]), atoms=len(solute["q"]), closure=args.closure,
                            tol=args.tol, mdiis=w["mdiis_nvec"]),
                site_gridpoint_iters_per_s=len(sites["q"]) * float(np.prod(grid["n"])) / t_iter,
                cpu_baseline=dict(value=value, unit="solves/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def replica_totals(secs, iters, device):
    """Replicas only: every rank solved its own copies; the job took as long as its slowest
    rank and did the sum of all ranks' iterations. One all-reduce of two scalars per
    quantity, on the timing path only (no collective touches the solver's data)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    n = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t[0]), float(n[0])


def cufft_comparison(nv, n, precision, iteration_ms, pairs=20, warmup=3):
    """cuFFT (through torch.fft) timed as a comparison only: the forward R2C and inverse C2R
    3D transforms of all solvent sites on the same grid and precision, which is the FFT part
    of one iteration; the solver's iteration also does the closure, the contraction, the
    residual, the Gram products and the update. The L2 is flushed (a 256 MB write) before
    each timed pair, as the solver's fields do not fit in L2 either. Never fails the bench:
    an error is reported in the result instead."""
    try:
        import torch
        dt = torch.float32 if precision == 32 else torch.float64
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        x = torch.randn((nv,) + tuple(n), dtype=dt, device="cuda", generator=gen)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        dims = (1, 2, 3)
        for _ in range(warmup):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=dims), s=tuple(n), dim=dims)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(pairs)]
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record()
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=dims), s=tuple(n), dim=dims)
            e1.record()
        torch.cuda.synchronize()
        ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs)
        err = float((y - x).abs().max())
        del x, y, flush
        return dict(what="torch.fft.rfftn + irfftn over all %d sites (cuFFT), %s, L2 flushed before "
                         "each pair; comparison only, not on the solve path" % (nv, "FP32" if precision == 32 else "FP64"),
                    ms_per_pair=ms, iteration_ms=iteration_ms,
                    iteration_over_pair=(iteration_ms / ms) if (iteration_ms and ms) else None,
                    roundtrip_max_err=err, pairs=pairs)
    except Exception as exc:          # the comparison is optional context for the line
        return dict(error="%s: %s" % (type(exc).__name__, exc))


def run_ours(args):
    import numpy as np
    import torch

    from paper_2403_01039_gb300 import build, capi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w, solv, grid, solute = workload_inputs(args.workload, product_chi)
    G = int(np.prod(grid["n"]))
    nv = len(solv["q"])
    # per-kernel CUDA events on the first iteration of every 8-iteration graph (a sample
    # spread over the whole timed region; every-iteration events cost ~5 % of the time)
    S = capi.Solver(solv, grid, precision=args.precision, mdiis_nvec=w["mdiis_nvec"],
                    timing=False if args.no_kernel_events else "sampled", split_passes=args.split_passes)

    def step():
        S.set_solute(solute["xyz"], solute["q"], solute["sigma"], solute["eps"])
        rep = S.solve(args.closure, args.pse_order, args.tol)
        S.sfe(args.closure, args.pse_order)
        return rep

    for _ in range(args.warmup):
        step()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    S.reset_stats()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(S.stream)
    reps = [step() for _ in range(args.steps)]
    ev1.record(S.stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    stats = S.stats()
    iters = sum(r["iterations"] for r in reps)
    secs, iters_all = replica_totals(ms / 1e3, iters, "cuda")
    value = world * args.steps / secs
    sgi = iters_all * nv * G / secs

    # end to end through the C ABI with host buffers: atoms in from pinned host memory,
    # g (all sites, FP64) and the SFE back to pinned host memory, every step
    pinned = {k: torch.from_numpy(np.ascontiguousarray(solute[k], dtype=np.float64)).pin_memory()
              for k in ("xyz", "q", "sigma", "eps")}
    g_host = torch.empty(S.field_shape, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        S.set_solute(pinned["xyz"].numpy(), pinned["q"].numpy(), pinned["sigma"].numpy(),
                     pinned["eps"].numpy())
        S.solve(args.closure, args.pse_order, args.tol)
        S.sfe(args.closure, args.pse_order)
        S.get("g", out=g_host.numpy())
    barrier()
    e2e_s, _ = replica_totals(time.perf_counter() - t0, 0, "cuda")
    e2e_val = world * args.e2e_steps / e2e_s
    h2d = int(len(solute["q"]) * (3 + 3) * 8)
    d2h = int(nv * G * 8 + nv * 152 * 8)

    # roofline of the dominant kernel (largest share of device time in the timed region)
    peak, peak_src = measured_peaks()
    kern = stats["kernels"]
    # launches that did work: every iteration for the iteration kernels, every timed launch
    # for the once-per-solve ones
    per_iter = ("plane_fwd", "pencil", "plane_inv", "mdiis", "ypencil_fwd", "ypencil_inv")
    per_iter2 = ("fwd_elem", "fft_fwd", "fft_inv", "inv_elem")          # two launches per iteration
    worked = {k: (stats["iterations"] if k in per_iter else 2 * stats["iterations"] if k in per_iter2
                  else kern[k]["timed"]) for k in kern}
    avg_ms = {k: (v["ms"] / v["timed"] if v["timed"] else 0.0) for k, v in kern.items()}
    share_ms = {k: avg_ms[k] * worked[k] for k in kern}       # estimated device time in the region
    dom = max(kern, key=lambda k: share_ms[k])
    kd = kern[dom]
    per_launch_s = avg_ms[dom] / 1e3
    total_ms = sum(share_ms.values())
    # algorithmic bytes of the iteration's byte model (s bytes per real, per site-point and
    # iteration): closure read 2s, two-pass transform 4s, residual and Gram (M + 2)s, update
    # (2M + 1)s, in all (3M + 9)s; split by kernel as plane_fwd = update + closure + plane
    # write (2M + 4)s, pencil 2s, plane_inv = plane read + residual (M + 3)s, and 2s for each
    # y-pencil pass of the row-chunked planes (the third transform pass, outside the base model)
    sb = 4.0 if args.precision == 32 else 8.0
    M = w["mdiis_nvec"]
    P = nv * float(G)
    model_units = {"plane_fwd": 2 * M + 4, "pencil": 2, "plane_inv": M + 3, "ypencil_fwd": 2, "ypencil_inv": 2}
    model_bytes = {k: u * sb * P for k, u in model_units.items()}
    lib_bytes_per_launch = kd["bytes"] / max(worked[dom], 1)
    bytes_per_launch = model_bytes.get(dom, lib_bytes_per_launch)
    achieved = bytes_per_launch / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    it_keys = [k for k in per_iter + per_iter2 if k in kern]
    it_ms = sum(share_ms[k] for k in it_keys) / stats["iterations"] if stats["iterations"] else None
    iter_bytes = (3 * M + 9) * sb * P
    iter_gbs = iter_bytes / (it_ms / 1e3) / 1e9 if it_ms else None
    traffic = ncu_traffic(dom, args.workload)
    roofline = dict(bound="hbm", kernel=dom, achieved=achieved, peak=peak, unit="GB/s",
                    frac=achieved / peak, peak_source=peak_src,
                    frac_of_nominal=achieved / NOMINAL_HBM_GBS, nominal_peak=NOMINAL_HBM_GBS,
                    traffic=traffic,
                    frac_by_traffic=(traffic / per_launch_s / 1e9 / peak) if traffic and per_launch_s > 0 else None,
                    model_note=("the (3M+9)s byte model counts 2M history fields for the update of plane_fwd; "
                                "storing Y = t + eta R lets the kernel read M, so its DRAM traffic is below the "
                                "model and frac_by_traffic (ncu bytes / launch time) is the bandwidth it sustains"
                                if dom == "plane_fwd" else None),
                    algorithmic_bytes_per_launch=bytes_per_launch,
                    bytes_model="(3M+9)s per site-point and iteration; %s: %s" % (
                        dom, "%ds" % model_units[dom] if dom in model_units else "library counter"),
                    library_bytes_per_launch=lib_bytes_per_launch,
                    library_frac=(lib_bytes_per_launch / per_launch_s / 1e9 / peak) if per_launch_s > 0 else None,
                    avg_launch_ms=per_launch_s * 1e3,
                    timed_launches=kd["timed"], share=share_ms[dom] / total_ms if total_ms else None,
                    iteration=dict(model_bytes=iter_bytes, ms=it_ms, achieved=iter_gbs,
                                   frac=(iter_gbs / peak) if iter_gbs else None,
                                   step_frac=iter_bytes * iters_all / (world * secs) / 1e9 / peak))
    launches = int(sum(k["launches"] for k in kern.values()))
    kernels_out = {k: dict(launches=v["launches"], timed=v["timed"],
                           ms_per_launch=avg_ms[k] if v["timed"] else None,
                           GBps=(v["bytes"] / max(worked[k], 1) / (avg_ms[k] / 1e3) / 1e9) if avg_ms[k] else None,
                           model_GBps=(model_bytes[k] / (avg_ms[k] / 1e3) / 1e9) if (avg_ms[k] and k in model_bytes) else None,
                           share=(share_ms[k] / total_ms) if total_ms else None)
                   for k, v in kern.items() if v["launches"]}

    cufft = None
    if rank == 0 and not args.no_cufft:
        cufft = cufft_comparison(nv, grid["n"], args.precision, it_ms)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w, solv, grid, solute, reps[-1]["iterations"])

    # measured FMA rates of this GPU; the FP64 form is bound by FP64 arithmetic rather than HBM
    fma = None
    if rank == 0:
        try:
            fma = {"fp32_tflops": capi.fma_rate(32) / 1e12, "fp64_tflops": capi.fma_rate(64) / 1e12}
        except Exception as exc:
            fma = dict(error="%s: %s" % (type(exc).__name__, exc))
    alu = None
    if fma and "fp64_tflops" in fma and args.precision == 64:
        # the arithmetic model per site-point and iteration: the R2C + C2R pair
        # 5 log2(N^3), closure ~20, contraction 2 n_v, MDIIS ~6M
        flops = 5.0 * np.log2(float(G)) + 20.0 + 2.0 * nv + 6.0 * w["mdiis_nvec"]
        ach = flops * sgi / 1e12
        alu = dict(bound="fp64 alu", flops_per_site_point_iteration=flops, achieved=ach,
                   peak=fma["fp64_tflops"], unit="TFLOP/s", frac=ach / fma["fp64_tflops"],
                   peak_source="measured FP64 FMA rate (rism3d_fma_rate)")

    # the batched and learned-guess forms, each against the plain solve of its own workload
    forms = None
    ws_gb = S.workspace.numel() / 1e9
    if rank == 0 and not args.no_forms:
        S.close()
        S.workspace = None                    # the forms create their own contexts
        torch.cuda.empty_cache()
        forms = {}
        for name, fn in (("batch64", lambda: batch_measure(32, 1e-6, args.inflight, 1, 1)),
                         ("learned_guess_solute50_128", lambda: learned_guess_measure())):
            try:
                forms[name] = fn()
            except Exception as exc:          # context for the line, never fails the bench
                forms[name] = dict(error="%s: %s" % (type(exc).__name__, exc))

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=secs * 1e3 / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32" if args.precision == 32 else "f64",
                    data="synthetic",
                    config=dict(workload=args.workload, grid="%d^3 x %.3g A" % (w["n"], w["spacing"]),
                                sites=nv, atoms=len(solute["q"]), closure=args.closure, tol=args.tol,
                                mdiis=w["mdiis_nvec"], parallelism="replicas" if world > 1 else "single",
                                l2="inputs larger than L2 (working set %.2f GB)" % ws_gb),
                    site_gridpoint_iters_per_s=sgi, iterations_per_solve=iters_all / (world * args.steps),
                    roofline=roofline, cpu_baseline=cpu,
                    e2e=dict(value=e2e_val, unit="solves/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    gpu_launches=launches, clocks=clk, kernels=kernels_out, cufft_comparison=cufft,
                    fma_rates=fma, roofline_fp64_alu=alu, forms=forms)
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile_case(args):
    """One solve of the workload (its grid, or --nx planes of it), capped at --profile-iters
    iterations: the kernels a profiler captures, with the same per-plane launch shapes."""
    from paper_2403_01039_gb300 import build, capi
    build.build()
    w, solv, grid, solute = workload_inputs(args.workload, product_chi)
    if args.nx:
        grid = dict(grid, n=(args.nx,) + tuple(grid["n"][1:]),
                    origin=(-(args.nx // 2) * grid["spacing"][0],) + tuple(grid["origin"][1:]))
    with capi.Solver(solv, grid, precision=args.precision, mdiis_nvec=w["mdiis_nvec"],
                     max_iter=args.profile_iters) as S:
        S.set_solute(solute["xyz"], solute["q"], solute["sigma"], solute["eps"])
        rep = S.solve(args.closure, args.pse_order, args.tol, check=False)
        print("profile case %s grid %s: %d iterations, rms %.3e, workspace %.2f GB"
              % (args.workload, grid["n"], rep["iterations"], rep["rms"], S.workspace.numel() / 1e9))


def batch_measure(precision, tol, inflight, steps, warmup, with_clocks=False):
    """The batch64 form: 64 seeded solutes (20-120 atoms) on uneven cubic grids (64-128, sizes
    with factors 2, 3, 5 only) in 3-site water, KH, MDIIS 5. A step is the whole batch: every
    job's set_solute + solve + SFE, once one at a time, once through rism3d_solve_batch (host
    scheduler, ``inflight`` jobs at a time) and once through rism3d_solve_batch_graph (all jobs
    as device loops in one graph launch). Contexts are created (one per grid) and their pencil
    tiles tuned before timing; the plane tiles stay the default (tiles picked by
    rism3d_tune_planes for a grid alone made the batch 5 % slower: a tile that fills the GPU
    alone is not the one that shares it best)."""
    import numpy as np
    import torch

    from paper_2403_01039_gb300 import capi, synth

    sites = synth.water_3site()
    chi, dk, _, _ = capi.xrism(sites)
    solv = dict(sites, chi=chi, dk=dk)
    work = synth.batch_workload()
    solvers = [capi.Solver(solv, w["grid"], precision=precision, mdiis_nvec=5) for w in work]
    try:
        tuned = []
        for S, w in zip(solvers, work):
            sol = w["solute"]
            S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            tuned.append(S.tune()[0])

        def one_at_a_time():
            its = 0
            for S, w in zip(solvers, work):
                sol = w["solute"]
                S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
                its += S.solve("kh", tol=tol)["iterations"]
                S.sfe("kh")
            return its

        site_points = [len(sites["q"]) * float(np.prod(w["grid"]["n"])) for w in work]
        spi = []

        def batched(one_graph=False):
            jobs = [dict(solver=S, solute=w["solute"], closure="kh", tol=tol, sfe="kh")
                    for S, w in zip(solvers, work)]
            res = capi.solve_batch(jobs, max_inflight=inflight, one_graph=one_graph)
            bad = [r for r in res if r["status"] != "OK"]
            if bad:
                raise RuntimeError("batch job failed: %s" % bad[0])
            spi.append(sum(p * r["iterations"] for p, r in zip(site_points, res)))
            return sum(r["iterations"] for r in res)

        def timed(fn):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = sum(fn() for _ in range(steps))
            torch.cuda.synchronize()
            return time.perf_counter() - t0, its

        t_seq, it_seq = timed(one_at_a_time)
        clocks = ClockSampler(0) if with_clocks else None
        if clocks:
            clocks.start()
        t_bat, it_bat = timed(batched)
        t_graph, it_graph = timed(lambda: batched(one_graph=True))
        clk = clocks.stop() if clocks else None
    finally:
        for S in solvers:
            S.close()
    n = len(work) * steps
    return dict(batched=n / t_bat, one_at_a_time=n / t_seq, speedup=t_seq / t_bat, unit="solves/s",
                one_graph=n / t_graph, one_graph_speedup=t_seq / t_graph, one_graph_iterations=it_graph,
                jobs=len(work), steps=steps, warmup=warmup, inflight=inflight, tol=tol,
                batched_iterations=it_bat, one_at_a_time_iterations=it_seq, t_batched_s=t_bat,
                site_gridpoint_iters_per_s=sum(spi[-steps:]) / t_bat,
                pencil_widths={str(k): tuned.count(k) for k in sorted(set(tuned))},
                clocks=clk)


def learned_guess_measure(n_seeds=8, tol=1e-6):
    """The learned-initial-guess form on held-out solutes of the solute50_128 kind (seeds
    60000..): set_solute + solve from the zero guess against set_solute + network + solve
    from the network's guess, with the stored trained weights; FP32, 128^3, KH."""
    import numpy as np
    import torch

    from paper_2403_01039_gb300 import capi, guess, synth

    wpath = os.path.join(ROOT, "paper_2403_01039_gb300", "data", "guess_unet_solute50_128.npz")
    W = np.load(wpath)
    crop = int(W["crop"])
    solv = guess._solvent()
    arith = str(W["arith"]) if "arith" in W else "bf16"
    net = capi.UNet3D(5, 5, crop, tuple(int(c) for c in W["channels"]), arith=arith)
    try:
        net.set_params(W["params"])
        with capi.Solver(solv, synth.cubic_grid(128, 0.5), precision=32, mdiis_nvec=5) as S:
            seeds = [guess.TEST_SEED0 + i for i in range(n_seeds)]
            guess.evaluate(S, net, seeds[:1], tol=tol, crop=crop)       # warm-up
            ev = guess.evaluate(S, net, seeds, tol=tol, crop=crop)
    finally:
        net.close()
    zi, gi = np.array(ev["zero_iters"]), np.array(ev["guess_iters"])
    return dict(seeds="%d held-out solutes, seeds %d-%d" % (n_seeds, seeds[0], seeds[-1]), crop=crop,
                network="%s form" % arith,
                zero_guess=dict(iterations_mean=float(zi.mean()), solves_per_s=len(zi) / float(np.sum(ev["zero_s"]))),
                learned_guess=dict(iterations_mean=float(gi.mean()), solves_per_s=len(gi) / float(np.sum(ev["guess_s"]))),
                fewer_iterations=int(np.sum(gi < zi)), more_iterations=int(np.sum(gi > zi)),
                speedup=float(np.sum(ev["zero_s"]) / np.sum(ev["guess_s"])), unit="solves/s", tol=tol)


def run_batch(args):
    """--workload batch64 (batch_measure): value is the batched solves/s, the one-at-a-time
    rate is reported beside it."""
    import torch

    from paper_2403_01039_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    m = batch_measure(args.precision, args.tol, args.inflight, args.steps, args.warmup, with_clocks=True)
    line = dict(metric=METRIC, value=m["batched"], unit="solves/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=m["t_batched_s"] * 1e3 / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32" if args.precision == 32 else "f64",
                data="synthetic",
                config=dict(workload="batch64", jobs=m["jobs"], grids="64-128 cubic (2,3,5 sizes) x 0.5 A",
                            sites=3, atoms="20-120", closure="kh", tol=args.tol, mdiis=5,
                            inflight=args.inflight, parallelism="single", pencil_widths=m["pencil_widths"]),
                one_at_a_time=dict(value=m["one_at_a_time"], unit="solves/s", iterations=m["one_at_a_time_iterations"]),
                one_graph=dict(value=m["one_graph"], unit="solves/s", iterations=m["one_graph_iterations"],
                               what="rism3d_solve_batch_graph: every job a device loop, one graph launch"),
                batched_iterations=m["batched_iterations"],
                site_gridpoint_iters_per_s=m["site_gridpoint_iters_per_s"], clocks=m["clocks"])
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        from paper_2403_01039_gb300 import synth
        if args.workload not in synth.WORKLOADS:
            sys.exit("--impl reference times the oracle on one solve of a single-solute workload "
                     "(%s); %s has no such form" % (", ".join(sorted(synth.WORKLOADS)), args.workload))
        run_reference(args)
    elif args.profile_iters > 0:
        run_profile_case(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
