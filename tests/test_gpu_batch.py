"""The batched form (rism3d_solve_batch with its host scheduler, rism3d_solve_batch_graph as
one graph launch of device loops): independent solutes on uneven grids solved concurrently
must give exactly what one-at-a-time solves give, match the FP64 oracle on every distinct
grid, honour the time limit and reject job lists it cannot schedule."""
import numpy as np
import pytest

from paper_2403_01039_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()

# uneven grids: powers of two, radix 3 and 5 sizes, anisotropic, and one row-chunked plane
JOBS = [
    (dict(n=(32, 32, 32), spacing=(0.5,) * 3, origin=(-8.0,) * 3), 20, 0),
    (dict(n=(24, 20, 30), spacing=(0.55, 0.6, 0.5), origin=(-6.6, -6.0, -7.5)), 31, 0),
    (dict(n=(36, 36, 36), spacing=(0.5,) * 3, origin=(-9.0,) * 3), 45, 0),
    (dict(n=(40, 36, 48), spacing=(0.45, 0.5, 0.4), origin=(-9.0, -9.0, -9.6)), 27, 0),
    (dict(n=(30, 30, 30), spacing=(0.5,) * 3, origin=(-7.5,) * 3), 24, 0),
    (dict(n=(32, 32, 32), spacing=(0.5,) * 3, origin=(-8.0,) * 3), 38, 8),
]


def _solute(k, n_atoms):
    return synth.random_solute(n_atoms, 10.0 * (n_atoms / 50.0) ** (1.0 / 3.0) * 0.5, 4100 + k)


@pytest.mark.parametrize("precision,one_graph", [(64, False), (32, False), (64, True), (32, True)])
def test_batch_equals_sequential(water3, precision, one_graph):
    tol = 1e-6
    seq = []
    for k, (grid, n_atoms, slab) in enumerate(JOBS):
        sol = _solute(k, n_atoms)
        with capi.Solver(water3, grid, precision=precision, slab_rows=slab) as S:
            S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            rep = S.solve("kh", tol=tol)
            sfe, _ = S.sfe("kh")
            seq.append((rep, sfe, S.get("g")))
    solvers = [capi.Solver(water3, grid, precision=precision, slab_rows=slab) for grid, _, slab in JOBS]
    try:
        jobs = [dict(solver=S, solute=_solute(k, JOBS[k][1]), closure="kh", tol=tol, sfe="kh")
                for k, S in enumerate(solvers)]
        res = capi.solve_batch(jobs, max_inflight=3, one_graph=one_graph)
        for k, (r, S) in enumerate(zip(res, solvers)):
            rep, sfe, g = seq[k]
            assert r["status"] == "OK" and r["converged"], r
            assert r["iterations"] == rep["iterations"]
            assert r["sfe"] == sfe
            assert np.array_equal(S.get("g"), g)
    finally:
        for S in solvers:
            S.close()


def test_batch_graph_device_deadline(water3):
    """One graph launch: each job's loop test stops the job on the device once the GPU's
    global timer passes the job's deadline (set by its first loop test); the jobs report
    ETIMEOUT after two body passes of check_every iterations, and the contexts stay usable."""
    grid, n_atoms, _ = JOBS[0]
    sol = _solute(0, n_atoms)
    with capi.Solver(water3, grid, precision=64) as A, capi.Solver(water3, grid, precision=32) as B:
        jobs = [dict(solver=S, solute=sol, closure="kh", tol=1e-10) for S in (A, B)]
        res = capi.solve_batch(jobs, time_limit=1e-9, one_graph=True)
        for r in res:
            assert r["status"] == "ETIMEOUT" and not r["converged"] and r["iterations"] == 16, r
        assert np.all(np.isfinite(A.get("g")))
        rep = A.solve("kh", tol=1e-6)
        assert rep["converged"]
        res = capi.solve_batch([dict(solver=S, solute=sol, closure="kh", tol=1e-6) for S in (A, B)], time_limit=60.0,
                               one_graph=True)
        assert all(r["status"] == "OK" and r["converged"] for r in res), res


def test_batch_time_limit_and_reuse(water3):
    grid, n_atoms, _ = JOBS[0]
    sol = _solute(0, n_atoms)
    with capi.Solver(water3, grid, precision=64) as A, capi.Solver(water3, grid, precision=64) as B:
        jobs = [dict(solver=S, solute=sol, closure="kh", tol=1e-10) for S in (A, B)]
        res = capi.solve_batch(jobs, max_inflight=2, time_limit=1e-9)
        for r in res:
            assert r["status"] == "ETIMEOUT" and not r["converged"] and r["iterations"] > 0, r
        assert np.all(np.isfinite(A.get("g")))
        # the contexts stay usable
        rep = A.solve("kh", tol=1e-6)
        assert rep["converged"]


def test_batch_shared_stream_and_rejected_context(water3):
    """Jobs whose contexts share a stream run in turn and still match one-at-a-time solves;
    a context listed twice makes the list invalid (nothing runs)."""
    grid = JOBS[0][0]
    sol = _solute(0, JOBS[0][1])
    st = torch.cuda.Stream()
    with capi.Solver(water3, grid, precision=64) as R:
        R.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        ref = R.solve("kh", tol=1e-6)
        g_ref = R.get("g")
    with capi.Solver(water3, grid, precision=64, stream=st) as A, \
            capi.Solver(water3, grid, precision=64, stream=st) as B:
        res = capi.solve_batch([dict(solver=A, solute=sol), dict(solver=B, solute=sol)])
        for r, S in zip(res, (A, B)):
            assert r["status"] == "OK" and r["iterations"] == ref["iterations"], r
            assert np.array_equal(S.get("g"), g_ref)
    with capi.Solver(water3, grid, precision=64) as A:
        res = capi.solve_batch([dict(solver=A, solute=sol), dict(solver=A, solute=sol)])
        assert all(r["status"] == "ESTATE" for r in res)
        with pytest.raises(capi.RismError):
            A.solve("kh")                                          # no solute was set


@pytest.mark.parametrize("precision,one_graph", [(64, False), (32, False), (32, True)])
def test_batch_matches_oracle(water3, precision, one_graph):
    """Every job of the uneven-grid batch against the oracle: FP64 against the oracle run with
    the same algorithm and tolerance (max|dg| <= 1e-6, |dSFE| <= 1e-4 kcal/mol, iterations
    +-2), FP32 (converged to 1e-7) against the oracle at 1e-10 (1e-3, 0.05 kcal/mol)."""
    from oracle import rism3d as orc, closure as cl
    tol = 1e-6 if precision == 64 else 1e-7
    solvers = [capi.Solver(water3, grid, precision=precision, slab_rows=slab) for grid, _, slab in JOBS]
    try:
        jobs = [dict(solver=S, solute=_solute(k, JOBS[k][1]), closure="kh", tol=tol, sfe="kh")
                for k, S in enumerate(solvers)]
        res = capi.solve_batch(jobs, max_inflight=3, one_graph=one_graph)
        for k, (r, S) in enumerate(zip(res, solvers)):
            grid, n_atoms, _ = JOBS[k]
            P = orc.Problem(water3, grid, _solute(k, n_atoms))
            ref = orc.solve(P, cl.KH, 1, tol=1e-6 if precision == 64 else 1e-10, mdiis_nvec=5)
            sref = orc.sfe(P, ref, cl.SFE_KH)[0]
            assert r["status"] == "OK" and r["converged"], r
            dg = float(np.max(np.abs(S.get("g") - ref["g"])))
            if precision == 64:
                assert dg <= 1e-6 and abs(r["sfe"] - sref) <= 1e-4, (k, dg, r["sfe"], sref)
                assert abs(r["iterations"] - ref["iterations"]) <= 2, (k, r["iterations"], ref["iterations"])
            else:
                assert dg <= 1e-3 and abs(r["sfe"] - sref) <= 0.05, (k, dg, r["sfe"], sref)
    finally:
        for S in solvers:
            S.close()


def test_tune_planes_picks_a_working_shape(water_nacl):
    """rism3d_tune_planes times the plane-pass tiles the grid admits on temporary contexts and
    returns the fastest; a solve with that tile gives the default tile's result to rounding
    (FP64: 1e-8 in g) and the same iteration count."""
    grid = dict(n=(24, 32, 32), spacing=(0.5, 0.5, 0.5), origin=(-6.0, -8.0, -8.0))
    t = capi.tune_planes(water_nacl, grid, precision=64, mdiis_nvec=5, iters=8)
    assert t["slab_rows"] in (0, 16, 8, 4) and t["ms_per_iter"] > 0.0, t
    sol = synth.random_solute(8, 3.0, 11, net_charge=1.0)
    out = []
    for kw in (dict(), dict(slab_rows=t["slab_rows"], ypencil_pass=t["ypencil_pass"])):
        with capi.Solver(water_nacl, grid, precision=64, **kw) as S:
            S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            rep = S.solve("kh", tol=1e-8)
            out.append((rep["iterations"], S.get("g")))
    assert out[0][0] == out[1][0]
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-8
