"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads,
exports every entry point declared in include/*.h, and validates its inputs without
touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2403_01039_gb300 import build, capi
    build.build()
    return capi.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b((?:rism3d|rism1d|unet3d)_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "rism3d_solve" in names and "unet3d_forward" in names and len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n


def _inputs(n=(32, 32, 32), sites=3, precision=64):
    from paper_2403_01039_gb300 import capi
    rng = np.random.default_rng(0)
    sv = dict(q=np.zeros(sites), sigma=np.ones(sites), eps=np.ones(sites), rho=np.full(sites, 0.03),
              temperature=300.0, chi=rng.standard_normal((sites, sites, 64)), dk=0.05)
    grid = dict(n=n, spacing=(0.5, 0.5, 0.5), origin=(0.0, 0.0, 0.0))
    opt = capi.default_options()
    opt.precision = precision
    return sv, grid, opt


def _ws(lib, sv, grid, opt):
    from paper_2403_01039_gb300 import capi
    s, keep = capi.make_solvent(sv)
    g = capi.make_grid(grid)
    nbytes = ctypes.c_size_t(0)
    st = lib.rism3d_workspace_bytes(ctypes.byref(s), ctypes.byref(g), ctypes.byref(opt), ctypes.byref(nbytes))
    return st, nbytes.value


def test_defaults_and_workspace_size(lib):
    from paper_2403_01039_gb300 import capi
    o = capi.default_options()
    assert (o.precision, o.mdiis_nvec, o.max_iter, o.check_every) == (32, 5, 10000, 8)
    assert abs(o.mdiis_damp - 0.7) < 1e-15
    sv, grid, opt = _inputs()
    st, nb = _ws(lib, sv, grid, opt)
    G = 32 ** 3
    # at least: beta*u, ring of 2 M fields, spectrum, staging (FP64)
    assert st == capi.OK and nb >= (3 * G * 8) * (1 + 2 * 5) + 3 * 32 * 32 * 17 * 16 + 3 * G * 8
    opt.precision = 32
    st, nb32 = _ws(lib, sv, grid, opt)
    assert st == capi.OK and nb32 < nb


@pytest.mark.parametrize("mutate,code", [
    (lambda sv, g, o: sv.update(rho=np.array([0.03, -1.0, 0.03])), 1),
    (lambda sv, g, o: sv.update(temperature=0.0), 1),
    (lambda sv, g, o: g.update(n=(32, 32, 31)), 8),
    (lambda sv, g, o: g.update(n=(14, 32, 32)), 8),
    (lambda sv, g, o: g.update(n=(32, 32, 28)), 8),          # Nz/2 = 14 has the factor 7
    (lambda sv, g, o: g.update(n=(8, 8, 30000)), 8),         # one FP64 row exceeds shared memory
    (lambda sv, g, o: setattr(o, "precision", 16), 1),
    (lambda sv, g, o: setattr(o, "mdiis_nvec", 17), 1),
    (lambda sv, g, o: setattr(o, "max_iter", 0), 1),
])
def test_validation(lib, mutate, code):
    sv, grid, opt = _inputs()
    mutate(sv, grid, opt)
    st, _ = _ws(lib, sv, grid, opt)
    assert st == code
    assert len(lib.rism3d_last_error(None)) > 0


def test_null_context_calls(lib):
    from paper_2403_01039_gb300 import capi
    rep = capi.Report()
    assert lib.rism3d_solve(None, 1, 1, 1e-6, ctypes.byref(rep)) == capi.EINVAL
    lib.rism3d_destroy(None)
    assert b"rism3d" in lib.rism3d_version()


def test_product_xrism_matches_oracle_table(lib):
    """The library's host 1D solver (solvent preparation, Eq. 4) against the oracle's
    susceptibility table for 3-site water (both converged to RMS 1e-10)."""
    from paper_2403_01039_gb300 import capi, synth
    from conftest import load_chi
    chi, dk, its, rms = capi.xrism(synth.water_3site())
    ref, rdk = load_chi("water3")
    assert dk == rdk and rms < 1e-10
    assert np.max(np.abs(chi - ref)) < 1e-7


def test_product_drism_matches_oracle(lib):
    """The library's host DRISM (dielectric 78.44) against the oracle's stored table (both to
    RMS 1e-10; measured max|dX| 1.6e-9), and its refusals: a dielectric constant at or below
    the XRISM value, a solvent without a dipole."""
    from paper_2403_01039_gb300 import capi, synth
    from conftest import load_chi
    s = synth.water_3site()
    ref, rdk = load_chi("water3_drism")
    chi, dk, its, rms = capi.xrism(s, dielectric=synth.WORKLOADS["sphere_32"]["dielectric"])
    assert dk == rdk and rms < 1e-10
    assert np.max(np.abs(chi - ref)) < 1e-7
    with pytest.raises(RuntimeError, match="XRISM value"):
        capi.xrism(s, dielectric=5.0)
    lj = dict(q=np.zeros(1), sigma=np.array([3.4]), eps=np.array([0.2]), rho=np.array([0.02]),
              species=np.zeros(1, dtype=np.int32), coords=np.zeros((1, 3)), temperature=120.0)
    with pytest.raises(RuntimeError, match="dipole"):
        capi.xrism(lj, dielectric=2.0)


def test_product_xrism_thermo_matches_oracle(lib):
    """Bulk pressure (Eq. 20), k_B T chi_T and the full direct correlation of 3-site water
    from the library's host 1D solver against the oracle's stored values."""
    import os
    from paper_2403_01039_gb300 import capi, synth
    chi, dk, its, rms, th = capi.xrism(synth.water_3site(), thermo=True)
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "thermo_water3.npz"))
    assert abs(th["pressure"] - float(ref["pressure"])) <= 1e-7 * abs(float(ref["pressure"]))
    assert abs(th["kT_chi_T"] - float(ref["kT_chi_T"])) <= 1e-6 * float(ref["kT_chi_T"])
    assert np.max(np.abs(th["c"][:, :, ::8] - ref["c_every8"])) <= 1e-6


@pytest.mark.parametrize("mutate,msg", [
    (lambda s: s["coords"].__setitem__((2, slice(None)), s["coords"][1]), "same position"),
    (lambda s: s["sigma"].__setitem__(0, -1.0), "sigma"),
    (lambda s: s["q"].__setitem__(1, np.nan), "q finite"),
    (lambda s: s["coords"].__setitem__((0, 0), np.inf), "position"),
])
def test_product_xrism_validates_sites(lib, mutate, msg):
    """The host 1D solver refuses sites it cannot represent (coincident sites of one
    molecule make omega = sin(kl)/(kl) undefined) before it iterates."""
    from paper_2403_01039_gb300 import capi, synth
    sv = synth.water_3site()
    sv = {k: (np.array(v, dtype=np.float64) if k in ("q", "sigma", "eps", "rho", "coords") else v)
          for k, v in sv.items()}
    mutate(sv)
    with pytest.raises(RuntimeError, match=msg):
        capi.xrism(sv)


def test_new_entry_points_validate_without_a_device(lib):
    """Batch, tuning, learned-guess and network entry points reject bad arguments before
    any CUDA call."""
    from paper_2403_01039_gb300 import capi
    P = ctypes.POINTER
    # batch: null list with jobs, bad max_inflight; an empty list is fine
    assert lib.rism3d_solve_batch(None, 2, 4, 0.0) == 1
    jobs = (capi.BatchJob * 1)()
    assert lib.rism3d_solve_batch(jobs, 1, 0, 0.0) == 1
    assert lib.rism3d_solve_batch(jobs, 1, 4, 0.0) == 1          # job without a context
    assert jobs[0].status == 4                                     # ESTATE: never started
    assert lib.rism3d_solve_batch(jobs, 0, 4, 0.0) == 0
    # null contexts
    w, ms = ctypes.c_int(), ctypes.c_double()
    assert lib.rism3d_tune(None, ctypes.byref(w), ctypes.byref(ms)) == 1
    corner = (ctypes.c_int * 3)(0, 0, 0)
    assert lib.rism3d_guess_input(None, corner, 8, None) == 1
    assert lib.rism3d_set_guess_crop(None, corner, 8, None) == 1
    assert lib.rism3d_get_pmv(None, 1.0, ctypes.byref(ms), None) == 1
    assert lib.rism3d_get_sfe_gradient(None, None) == 1
    # network: sizes are checked before any allocation
    net = ctypes.c_void_p()
    assert lib.unet3d_create(5, 5, 30, 16, 32, 64, None, ctypes.byref(net)) == 1     # crop % 4
    assert lib.unet3d_create(0, 5, 32, 16, 32, 64, None, ctypes.byref(net)) == 1
    assert not net.value
    assert lib.unet3d_param_count(None) == 0


def test_option_validation(lib):
    """kgrid, split_passes and timing outside their ranges are rejected by the size query."""
    sv, grid, opt = _inputs()
    for field, bad in (("kgrid", 2), ("split_passes", 3), ("timing", 5)):
        o = type(opt)()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opt), ctypes.sizeof(opt))
        setattr(o, field, bad)
        st, _ = _ws(lib, sv, grid, o)
        assert st == 1, field


def test_device_tensor_arguments_are_checked_before_the_call():
    """Crop and network entry points take raw device pointers: the binding refuses host
    tensors, other dtypes and non-tensors before anything reaches the library."""
    torch = pytest.importorskip("torch")
    from paper_2403_01039_gb300 import capi
    for bad in (torch.zeros(8), torch.zeros(8, dtype=torch.float64), np.zeros(8, dtype=np.float32), None):
        with pytest.raises(ValueError):
            capi._f32_cuda(bad, 8, "x")


def test_solute_arrays_must_agree_in_length():
    """The binding refuses a solute whose arrays disagree in length: the library reads
    n_atoms values from each pointer."""
    from paper_2403_01039_gb300 import capi
    (xyz, q, s, e), _ = capi._solute_arrays(np.zeros((4, 3)), np.zeros(4), np.ones(4), np.ones(4))
    assert xyz.shape == (4, 3) and q.shape == s.shape == e.shape == (4,)
    with pytest.raises(ValueError):
        capi._solute_arrays(np.zeros((3, 3)), np.zeros(4), np.ones(4), np.ones(4))
    with pytest.raises(ValueError):
        capi._solute_arrays(np.zeros((4, 3)), np.zeros(4), np.ones(5), np.ones(4))


def test_workloads_fit_one_gb300(lib):
    """The device workspace of every named workload, in both precisions, fits one GB300
    (284,208 MiB of HBM) with room to spare for the CUDA context and the caller."""
    from paper_2403_01039_gb300 import capi, synth
    hbm = 284208 * 2 ** 20
    for name, w in synth.WORKLOADS.items():
        sites = synth.solvent_sites(w["solvent"])
        nv = len(sites["q"])
        s, keep = capi.make_solvent(dict(sites, chi=np.zeros((nv, nv, 64)), dk=0.05))
        g = capi.make_grid(synth.cubic_grid(w["n"], w["spacing"]))
        for prec in (32, 64):
            o = capi.default_options()
            o.precision, o.mdiis_nvec = prec, w["mdiis_nvec"]
            nb = ctypes.c_size_t()
            st = lib.rism3d_workspace_bytes(ctypes.byref(s), ctypes.byref(g), ctypes.byref(o), ctypes.byref(nb))
            assert st == capi.OK and 0 < nb.value < 0.6 * hbm, (name, prec, nb.value)


def test_tune_planes_validates_before_any_device_work(lib):
    """rism3d_tune_planes refuses iters < 2 without touching the GPU."""
    from paper_2403_01039_gb300 import capi, synth
    d = np.load(os.path.join(ROOT, "tests", "golden", "chi_water3.npz"))
    s = synth.water_3site()
    s.update(chi=d["chi"], dk=float(d["dk"]))
    with pytest.raises(capi.RismError) as e:
        capi.tune_planes(s, synth.cubic_grid(16, 0.5), iters=1)
    assert e.value.status == capi.EINVAL
