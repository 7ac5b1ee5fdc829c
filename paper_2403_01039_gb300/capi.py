"""ctypes binding of the C ABI in include/rism3d.h (argument marshalling only).

Every step of the solve runs in the library's CUDA kernels. PyTorch supplies the device
memory of the workspace and the CUDA stream the library runs on. Importing this module
does not load the library; the first use does, and fails loudly (``RuntimeError``) when the
compiled library is missing - there is no fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "librism3d.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ENOTCONV, EDIVERGED, ETIMEOUT, EUNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ESTATE", "ENOTCONV", "EDIVERGED", "ETIMEOUT",
                "EUNSUPPORTED"]
CLOSURES = {"kh": 1, "hnc": 2, "pse": 3}
SFE_KINDS = {"kh": 1, "hnc": 2, "gf": 3, "pse": 4}
FIELDS = {"g": 1, "c": 2, "h": 3, "t": 4, "u": 5, "phi": 6, "r": 7}

_dp = ctypes.POINTER(ctypes.c_double)


class Solvent(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int), ("q", _dp), ("sigma", _dp), ("eps", _dp), ("rho", _dp),
                ("temperature", ctypes.c_double), ("n_k", ctypes.c_int), ("dk", ctypes.c_double),
                ("chi", _dp)]


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("spacing", ctypes.c_double * 3),
                ("origin", ctypes.c_double * 3)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mdiis_nvec", ctypes.c_int),
                ("mdiis_damp", ctypes.c_double), ("dynamic_damp", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("max_atoms", ctypes.c_int), ("timing", ctypes.c_int),
                ("accelerator", ctypes.c_int), ("anderson_s1", ctypes.c_double),
                ("anderson_s2", ctypes.c_double), ("slab_rows", ctypes.c_int),
                ("split_passes", ctypes.c_int), ("kgrid", ctypes.c_int), ("ypencil_pass", ctypes.c_int),
                ("anchor_ratio", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


N_KERNELS = 14
KERNEL_NAMES = ["plane_fwd", "pencil", "plane_inv", "mdiis", "potential", "long_range", "sfe", "other",
                "ypencil_fwd", "ypencil_inv", "fwd_elem", "fft_fwd", "fft_inv", "inv_elem"]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * N_KERNELS), ("timed", ctypes.c_longlong * N_KERNELS),
                ("ms", ctypes.c_double * N_KERNELS), ("bytes", ctypes.c_double * N_KERNELS),
                ("iterations", ctypes.c_longlong), ("solves", ctypes.c_longlong)]


class Report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("rms_residual", ctypes.c_double), ("seconds_iter", ctypes.c_double)]


class BatchJob(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("n_atoms", ctypes.c_int), ("xyz", _dp), ("q", _dp),
                ("sigma", _dp), ("eps", _dp), ("closure", ctypes.c_int), ("pse_order", ctypes.c_int),
                ("tol", ctypes.c_double), ("sfe_kind", ctypes.c_int), ("report", Report),
                ("sfe", ctypes.c_double), ("status", ctypes.c_int)]


_lib = None


def load():
    """Load the compiled library (once). Raises RuntimeError when it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("the CUDA library %s is missing: run __graft_entry__.build() "
                           "(or python -m paper_2403_01039_gb300.build) first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "rism3d_version": (ctypes.c_char_p, []),
        "rism3d_options_default": (None, [P(Options)]),
        "rism3d_workspace_bytes": (c_int, [P(Solvent), P(Grid), P(Options), P(c_size_t)]),
        "rism3d_create": (c_int, [P(Solvent), P(Grid), P(Options), P(c_void_p)]),
        "rism3d_set_solute": (c_int, [c_void_p, c_int, _dp, _dp, _dp, _dp]),
        "rism3d_set_guess": (c_int, [c_void_p, c_void_p, c_int]),
        "rism3d_solve": (c_int, [c_void_p, c_int, c_int, c_double, P(Report)]),
        "rism3d_residual": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
        "rism3d_get": (c_int, [c_void_p, c_int, c_void_p, c_size_t, c_int]),
        "rism3d_get_sfe": (c_int, [c_void_p, c_int, c_int, P(c_double), _dp]),
        "rism3d_solve_batch": (c_int, [P(BatchJob), c_int, c_int, c_double]),
        "rism3d_solve_batch_graph": (c_int, [P(BatchJob), c_int, c_double]),
        "rism3d_get_sfe_finite_size": (c_int, [c_void_p, P(c_double)]),
        "rism3d_tune_planes": (c_int, [c_void_p, c_void_p, P(Options), c_int, P(Options), P(c_double)]),
        "rism3d_tune": (c_int, [c_void_p, P(c_int), P(c_double)]),
        "rism3d_guess_input": (c_int, [c_void_p, P(c_int), c_int, c_void_p]),
        "rism3d_guess_target": (c_int, [c_void_p, P(c_int), c_int, c_void_p]),
        "rism3d_set_guess_crop": (c_int, [c_void_p, P(c_int), c_int, c_void_p]),
        "unet3d_create": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, P(c_void_p)]),
        "unet3d_create_ex": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, P(c_void_p)]),
        "unet3d_conv3_bf16": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                      c_void_p, c_void_p]),
        "unet3d_param_count": (c_size_t, [c_void_p]),
        "unet3d_set_params": (c_int, [c_void_p, P(ctypes.c_float)]),
        "unet3d_get_params": (c_int, [c_void_p, P(ctypes.c_float)]),
        "unet3d_forward": (c_int, [c_void_p, c_void_p, c_void_p]),
        "unet3d_backward": (c_int, [c_void_p, c_void_p]),
        "unet3d_get_grads": (c_int, [c_void_p, P(ctypes.c_float)]),
        "unet3d_mse": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, P(c_double), c_void_p]),
        "unet3d_mse_core": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_float, ctypes.c_float, P(c_double),
                                    c_void_p]),
        "unet3d_adam": (c_int, [c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, c_int]),
        "unet3d_last_error": (ctypes.c_char_p, []),
        "unet3d_destroy": (None, [c_void_p]),
        "rism3d_get_pmv": (c_int, [c_void_p, c_double, P(c_double), _dp]),
        "rism3d_get_sfe_gradient": (c_int, [c_void_p, _dp]),
        "rism3d_get_stats": (c_int, [c_void_p, P(Stats)]),
        "rism3d_reset_stats": (c_int, [c_void_p]),
        "rism3d_last_error": (ctypes.c_char_p, [c_void_p]),
        "rism3d_destroy": (None, [c_void_p]),
    }
    sig.update({
        "rism3d_sfe_noalloc": (c_int, [c_int, ctypes.c_longlong, c_void_p, c_void_p, c_void_p, _dp,
                                       c_double, c_double, c_int, c_int, P(c_double), _dp, c_void_p]),
        "rism3d_fma_rate": (c_int, [c_int, P(c_double)]),
        "rism1d_options_default": (None, [P(Rism1dOptions)]),
        "rism1d_xrism": (c_int, [P(Rism1dSolvent), P(Rism1dOptions), _dp, _dp, P(c_int), _dp]),
        "rism1d_xrism_ex": (c_int, [P(Rism1dSolvent), P(Rism1dOptions), _dp, _dp, _dp, _dp, _dp,
                                    P(c_int), _dp]),
        "rism1d_last_error": (ctypes.c_char_p, []),
    })
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class Rism1dSolvent(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int), ("q", _dp), ("sigma", _dp), ("eps", _dp), ("rho", _dp),
                ("species", ctypes.POINTER(ctypes.c_int)), ("coords", _dp),
                ("temperature", ctypes.c_double)]


class Rism1dOptions(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("dr", ctypes.c_double), ("closure", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mdiis_nvec", ctypes.c_int),
                ("mdiis_damp", ctypes.c_double), ("charge_steps", ctypes.c_int),
                ("dielectric", ctypes.c_double), ("drism_damping", ctypes.c_double)]


class RismError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message))


def _arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _solute_arrays(xyz, q, sigma, eps):
    """Contiguous float64 copies of a solute and their pointers; the library reads n_atoms
    values from each, so the lengths must agree (checked here: it cannot check a pointer)."""
    xyz, pxyz = _arr(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    q, pq = _arr(np.ravel(q))
    s, ps = _arr(np.ravel(sigma))
    e, pe = _arr(np.ravel(eps))
    if not (len(xyz) == len(q) == len(s) == len(e)):
        raise ValueError("solute arrays disagree: %d positions, %d charges, %d sigma, %d eps"
                         % (len(xyz), len(q), len(s), len(e)))
    return (xyz, q, s, e), (pxyz, pq, ps, pe)


def make_solvent(sites):
    """Marshal a solvent dict (q, sigma, eps, rho, temperature, chi [n,n,nk], dk)."""
    keep = {}
    for k in ("q", "sigma", "eps", "rho", "chi"):
        keep[k] = _arr(sites[k])
    n = len(keep["q"][0])
    chi = keep["chi"][0]
    if chi.shape[:2] != (n, n):
        raise ValueError("chi must be [n_sites][n_sites][n_k]")
    s = Solvent(n, keep["q"][1], keep["sigma"][1], keep["eps"][1], keep["rho"][1],
                float(sites["temperature"]), chi.shape[2], float(sites["dk"]), keep["chi"][1])
    return s, keep


def make_grid(grid):
    g = Grid()
    for d in range(3):
        g.n[d] = int(grid["n"][d])
        g.spacing[d] = float(grid["spacing"][d])
        g.origin[d] = float(grid["origin"][d])
    return g


def default_options():
    o = Options()
    load().rism3d_options_default(ctypes.byref(o))
    return o


def _f32_cuda(t, count, name):
    """Device pointer of a contiguous float32 CUDA tensor of exactly ``count`` values: the
    kernels behind it read and write that many values, so anything else is refused here."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)
    if t.numel() != count:
        raise ValueError("%s has %d values, expected %d" % (name, t.numel(), count))
    return ctypes.c_void_p(t.data_ptr())


def _check(lib, ctx, st):
    if st != OK:
        raise RismError(st, lib.rism3d_last_error(ctx).decode())


def sfe_noalloc(h, c, rho, temperature, dV, kind="kh", pse_order=3, d=None, stream=None):
    """rism3d_sfe_noalloc on CUDA float64 tensors h, c (and d for PSE) of shape
    [n_sites, ...]: the SFE with the library's static scratch, no device allocation.
    Returns (total, per_site)."""
    import torch
    lib = load()
    n_sites = h.shape[0]
    n_points = h.numel() // n_sites
    for x in (h, c) + ((d,) if d is not None else ()):
        if x.dtype.itemsize != 8 or not x.is_cuda or not x.is_contiguous() or x.numel() != h.numel():
            raise ValueError("h, c, d must be contiguous float64 CUDA tensors of one shape")
        if x.device != h.device:
            raise ValueError("h, c, d must be on one device")
    rho_a, prho = _arr(rho)
    tot = ctypes.c_double()
    per = np.zeros(n_sites)
    with torch.cuda.device(h.device):
        st = lib.rism3d_sfe_noalloc(n_sites, n_points, ctypes.c_void_p(h.data_ptr()),
                                    ctypes.c_void_p(c.data_ptr()),
                                    ctypes.c_void_p(d.data_ptr() if d is not None else 0), prho,
                                    float(temperature), float(dV), SFE_KINDS[kind], int(pse_order),
                                    ctypes.byref(tot), per.ctypes.data_as(_dp),
                                    ctypes.c_void_p(stream.cuda_stream if stream is not None else 0))
    if st != OK:
        raise RismError(st, lib.rism3d_last_error(None).decode())
    return tot.value, per


def fma_rate(precision):
    """FP32 (32) or FP64 (64) FMA throughput of the current device in flop/s (rism3d_fma_rate)."""
    lib = load()
    r = ctypes.c_double()
    st = lib.rism3d_fma_rate(int(precision), ctypes.byref(r))
    if st != OK:
        raise RismError(st, "rism3d_fma_rate failed")
    return r.value


def xrism(sites, n_r=2048, dr=0.05, closure="kh", tol=1e-10, charge_steps=10, thermo=False,
          dielectric=None, drism_damping=1.0):
    """Solvent susceptibility X_ag(k_j), k_j = j dk, of a pure solvent (Eq. 4) from the
    library's host 1D-RISM solver (XRISM, or DRISM with the given dielectric constant).
    Returns (chi [n][n][n_r], dk, iterations, rms); with
    thermo=True also a dict with the full direct correlation c [n][n][n_r - 1] at r_i = i dr,
    the bulk pressure of Eq. 20 (kcal/mol/A^3) and k_B T chi_T (A^3)."""
    lib = load()
    keep = {k: _arr(sites[k]) for k in ("q", "sigma", "eps", "rho")}
    species = np.ascontiguousarray(sites["species"], dtype=np.int32)
    coords, pc = _arr(np.asarray(sites["coords"], dtype=np.float64).reshape(-1, 3))
    n = len(keep["q"][0])
    sv = Rism1dSolvent(n, keep["q"][1], keep["sigma"][1], keep["eps"][1], keep["rho"][1],
                       species.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), pc,
                       float(sites["temperature"]))
    o = Rism1dOptions()
    lib.rism1d_options_default(ctypes.byref(o))
    o.n_r, o.dr, o.tol, o.charge_steps = int(n_r), float(dr), float(tol), int(charge_steps)
    o.closure = {"kh": 1, "hnc": 2}[closure]
    o.dielectric = 0.0 if dielectric is None else float(dielectric)
    o.drism_damping = float(drism_damping)
    chi = np.zeros((n, n, n_r))
    c_r = np.zeros((n, n, n_r - 1))
    dk, pres, ktchi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    its = ctypes.c_int()
    rms = ctypes.c_double()
    st = lib.rism1d_xrism_ex(ctypes.byref(sv), ctypes.byref(o), chi.ctypes.data_as(_dp), ctypes.byref(dk),
                             c_r.ctypes.data_as(_dp) if thermo else None,
                             ctypes.byref(pres) if thermo else None,
                             ctypes.byref(ktchi) if thermo else None, ctypes.byref(its), ctypes.byref(rms))
    if st != 0:
        raise RuntimeError("rism1d_xrism failed (%d): %s" % (st, lib.rism1d_last_error().decode()))
    if thermo:
        return chi, dk.value, its.value, rms.value, dict(c=c_r, pressure=pres.value, kT_chi_T=ktchi.value)
    return chi, dk.value, its.value, rms.value


def tune_planes(solvent, grid, precision=32, mdiis_nvec=5, iters=16, kgrid="integer"):
    """rism3d_tune_planes: the fastest plane-pass tile (slab_rows, ypencil_pass) for this
    solvent, grid and precision, timed on temporary contexts. Returns dict(slab_rows,
    ypencil_pass, ms_per_iter), ready to pass to Solver."""
    lib = load()
    solv, keep = make_solvent(solvent)
    gr = make_grid(grid)
    o = default_options()
    o.precision = precision
    o.mdiis_nvec = mdiis_nvec
    o.kgrid = {"integer": 0, "half": 1}[kgrid]
    best = Options()
    ms = ctypes.c_double()
    st = lib.rism3d_tune_planes(ctypes.byref(solv), ctypes.byref(gr), ctypes.byref(o), int(iters), ctypes.byref(best),
                                ctypes.byref(ms))
    if st != OK:
        raise RismError(st, lib.rism3d_last_error(None).decode())
    del keep
    return dict(slab_rows=best.slab_rows, ypencil_pass=bool(best.ypencil_pass), ms_per_iter=ms.value)


def solve_batch(jobs, max_inflight=8, time_limit=0.0, one_graph=False):
    """Solve independent problems concurrently (``rism3d_solve_batch``, or with one_graph
    ``rism3d_solve_batch_graph``: all jobs as device loops in one graph launch). jobs: list
    of dicts with keys solver (a Solver of its own), solute (dict xyz/q/sigma/eps, or None to
    keep the solver's current solute), closure ("kh"), pse_order (3), tol (1e-6), sfe (None or
    an SFE kind). Returns a list of dicts (status name, iterations, converged, rms, sfe)."""
    lib = load()
    arr = (BatchJob * len(jobs))()
    keep = []
    for J, d in zip(arr, jobs):
        S = d["solver"]
        J.ctx = S.ctx
        sol = d.get("solute")
        if sol is not None:
            arrays, (pxyz, pq, ps, pe) = _solute_arrays(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            keep += list(arrays)
            J.n_atoms, J.xyz, J.q, J.sigma, J.eps = len(arrays[1]), pxyz, pq, ps, pe
            S.n_atoms = len(arrays[1])
        else:
            J.n_atoms = 0
        J.closure = CLOSURES[d.get("closure", "kh")]
        J.pse_order = int(d.get("pse_order", 3))
        J.tol = float(d.get("tol", 1e-6))
        J.sfe_kind = SFE_KINDS[d["sfe"]] if d.get("sfe") else 0
    if one_graph:
        lib.rism3d_solve_batch_graph(arr, len(jobs), float(time_limit))
    else:
        lib.rism3d_solve_batch(arr, len(jobs), int(max_inflight), float(time_limit))
    out = []
    for J in arr:
        name = STATUS_NAMES[J.status] if 0 <= J.status < len(STATUS_NAMES) else str(J.status)
        out.append(dict(status=name, iterations=J.report.iterations,
                        converged=bool(J.report.converged), rms=J.report.rms_residual, sfe=J.sfe,
                        seconds=J.report.seconds_iter))
    return out


class Solver:
    """One solvent on one grid (``rism3d_create``); solutes are set and solved in turn."""

    def __init__(self, solvent, grid, precision=32, mdiis_nvec=5, mdiis_damp=0.7,
                 dynamic_damp=False, max_iter=10000, check_every=8, max_atoms=100000,
                 timing=False, accelerator="mdiis", anderson_s=(0.2, 0.0), slab_rows=0,
                 kgrid="integer", split_passes=False, ypencil_pass=False, anchor_ratio=None, stream=None,
                 device=None):
        import torch
        self._torch = torch
        lib = load()
        self.lib = lib
        self.device = torch.device("cuda" if device is None else device)
        self.n = tuple(int(v) for v in grid["n"])
        self.n_sites = len(solvent["q"])
        self.precision = precision
        self._solv, self._keep = make_solvent(solvent)
        self._grid = make_grid(grid)
        o = default_options()
        o.precision = precision
        o.mdiis_nvec = mdiis_nvec
        o.mdiis_damp = mdiis_damp
        o.dynamic_damp = int(bool(dynamic_damp))
        o.max_iter = max_iter
        o.check_every = check_every
        o.max_atoms = max_atoms
        o.timing = 2 if timing == "sampled" else int(bool(timing))
        o.accelerator = {"mdiis": 0, "anderson": 1}[accelerator]
        o.anderson_s1, o.anderson_s2 = float(anderson_s[0]), float(anderson_s[1])
        o.slab_rows = int(slab_rows)
        o.kgrid = {"integer": 0, "half": 1}[kgrid]
        o.split_passes = int(bool(split_passes))
        o.ypencil_pass = int(bool(ypencil_pass))
        if anchor_ratio is not None:
            o.anchor_ratio = float(anchor_ratio)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
            nbytes = ctypes.c_size_t()
            _check(lib, None, lib.rism3d_workspace_bytes(ctypes.byref(self._solv), ctypes.byref(self._grid),
                                                         ctypes.byref(o), ctypes.byref(nbytes)))
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            o.workspace = ctypes.c_void_p(self.workspace.data_ptr())
            o.workspace_bytes = nbytes.value
            self._opt = o
            ctx = ctypes.c_void_p()
            _check(lib, None, lib.rism3d_create(ctypes.byref(self._solv), ctypes.byref(self._grid),
                                                ctypes.byref(o), ctypes.byref(ctx)))
        self.ctx = ctx

    # -- helpers
    @property
    def field_shape(self):
        return (self.n_sites,) + self.n

    def _field_arg(self, x):
        """(pointer, on_device, keepalive) for a full field [n_sites][Nx][Ny][Nz] given as a
        numpy array or a contiguous float64 CUDA tensor; the size is checked here because
        the library cannot check a raw pointer."""
        torch = self._torch
        need = int(np.prod(self.field_shape))
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
                raise ValueError("device arrays must be contiguous float64 CUDA tensors")
            if x.numel() != need:
                raise ValueError("field has %d values, expected %d" % (x.numel(), need))
            return ctypes.c_void_p(x.data_ptr()), 1, x
        a = np.ascontiguousarray(x, dtype=np.float64)
        if a.size != need:
            raise ValueError("field has %d values, expected %d" % (a.size, need))
        return ctypes.c_void_p(a.ctypes.data), 0, a

    def _sync_torch(self):
        # device inputs produced on torch's current stream must be ready for the library stream
        self.stream.wait_stream(self._torch.cuda.current_stream(self.device))

    # -- API
    def set_solute(self, xyz, q, sigma, eps):
        arrays, (pxyz, pq, ps, pe) = _solute_arrays(xyz, q, sigma, eps)
        n = len(arrays[1])
        _check(self.lib, self.ctx, self.lib.rism3d_set_solute(self.ctx, n, pxyz, pq, ps, pe))
        self.n_atoms = n

    def set_guess(self, t):
        p, dev, keep = self._field_arg(t)
        if dev:
            self._sync_torch()
        _check(self.lib, self.ctx, self.lib.rism3d_set_guess(self.ctx, p, dev))

    def solve(self, closure="kh", pse_order=3, tol=1e-6, check=True):
        rep = Report()
        st = self.lib.rism3d_solve(self.ctx, CLOSURES[closure], int(pse_order), float(tol),
                                   ctypes.byref(rep))
        out = dict(status=st, iterations=rep.iterations, converged=bool(rep.converged),
                   rms=rep.rms_residual, seconds=rep.seconds_iter)
        if check and st not in (OK,):
            raise RismError(st, self.lib.rism3d_last_error(self.ctx).decode())
        return out

    def residual(self, t, closure="kh", pse_order=3):
        torch = self._torch
        p, dev, keep = self._field_arg(t)
        if dev:
            out = torch.empty_like(t)
            self._sync_torch()
            st = self.lib.rism3d_residual(self.ctx, CLOSURES[closure], int(pse_order), p,
                                          ctypes.c_void_p(out.data_ptr()), 1)
        else:
            out = np.empty(keep.shape, dtype=np.float64)
            st = self.lib.rism3d_residual(self.ctx, CLOSURES[closure], int(pse_order), p,
                                          ctypes.c_void_p(out.ctypes.data), 0)
        _check(self.lib, self.ctx, st)
        return out

    def get(self, field, out=None):
        """Field as a float64 numpy array, or into ``out`` (numpy or CUDA tensor)."""
        shape = self.n if field == "phi" else self.field_shape
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        torch = self._torch
        if isinstance(out, torch.Tensor):
            if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
                raise ValueError("out must be a contiguous float64 CUDA tensor")
            st = self.lib.rism3d_get(self.ctx, FIELDS[field], ctypes.c_void_p(out.data_ptr()), out.numel(), 1)
        else:
            if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a contiguous float64 numpy array")
            st = self.lib.rism3d_get(self.ctx, FIELDS[field], ctypes.c_void_p(out.ctypes.data), out.size, 0)
        _check(self.lib, self.ctx, st)
        return out

    def sfe(self, kind="kh", pse_order=3):
        tot = ctypes.c_double()
        per = np.zeros(self.n_sites)
        _check(self.lib, self.ctx, self.lib.rism3d_get_sfe(self.ctx, SFE_KINDS[kind], int(pse_order),
                                                           ctypes.byref(tot), per.ctypes.data_as(_dp)))
        return tot.value, per

    def tune(self):
        """Pick the pencil tile width by measurement (rism3d_tune); returns (W, ms)."""
        w, ms = ctypes.c_int(), ctypes.c_double()
        _check(self.lib, self.ctx, self.lib.rism3d_tune(self.ctx, ctypes.byref(w), ctypes.byref(ms)))
        return w.value, ms.value

    def _corner(self, corner):
        return (ctypes.c_int * 3)(*[int(v) for v in corner])

    def _crop_arg(self, t, crop, name):
        return _f32_cuda(t, self.n_sites * int(crop) ** 3, name)

    def guess_input(self, corner, crop, out):
        """Network input tanh(beta u / 4) on the crop into ``out`` (float32 CUDA tensor
        [n_sites, crop, crop, crop])."""
        p = self._crop_arg(out, crop, "out")
        _check(self.lib, self.ctx, self.lib.rism3d_guess_input(self.ctx, self._corner(corner), int(crop), p))

    def guess_target(self, corner, crop, out):
        """The current iterate tau = t - f on the crop into ``out`` (float32 CUDA tensor)."""
        p = self._crop_arg(out, crop, "out")
        _check(self.lib, self.ctx, self.lib.rism3d_guess_target(self.ctx, self._corner(corner), int(crop), p))

    def set_guess_crop(self, corner, crop, tau):
        """Start the next solve from tau on the crop (float32 CUDA tensor) and 0 elsewhere."""
        p = self._crop_arg(tau, crop, "tau")
        self._sync_torch()
        _check(self.lib, self.ctx, self.lib.rism3d_set_guess_crop(self.ctx, self._corner(corner), int(crop), p))

    def pmv(self, kT_chi_T):
        """Partial molar volume (Eq. 19, A^3) and the per-site c integrals of the current
        iterate, given the solvent's k_B T chi_T (A^3)."""
        v = ctypes.c_double()
        ci = np.zeros(self.n_sites)
        _check(self.lib, self.ctx, self.lib.rism3d_get_pmv(self.ctx, float(kT_chi_T), ctypes.byref(v),
                                                           ci.ctypes.data_as(_dp)))
        return v.value, ci

    def sfe_gradient(self):
        """dSFE/dR of every solute atom (kcal/mol/A), [n_atoms, 3]."""
        g = np.zeros((getattr(self, "n_atoms", 0), 3))
        _check(self.lib, self.ctx, self.lib.rism3d_get_sfe_gradient(self.ctx, g.ctypes.data_as(_dp)))
        return g

    def sfe_finite_size(self):
        """Finite-size error of the SFE box sum for the current solute (kcal/mol,
        rism3d_get_sfe_finite_size): the infinite-dilution SFE is the box SFE minus it."""
        d = ctypes.c_double()
        _check(self.lib, self.ctx, self.lib.rism3d_get_sfe_finite_size(self.ctx, ctypes.byref(d)))
        return d.value

    def stats(self):
        st = Stats()
        _check(self.lib, self.ctx, self.lib.rism3d_get_stats(self.ctx, ctypes.byref(st)))
        out = dict(iterations=st.iterations, solves=st.solves, kernels={})
        for k, name in enumerate(KERNEL_NAMES):
            out["kernels"][name] = dict(launches=st.launches[k], timed=st.timed[k], ms=st.ms[k],
                                        bytes=st.bytes[k])
        return out

    def reset_stats(self):
        _check(self.lib, self.ctx, self.lib.rism3d_reset_stats(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.rism3d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class UNet3D:
    """The learned-guess network of ``unet3d.h`` (device kernels of the library); tensors
    are float32 CUDA tensors, parameters a flat float32 numpy vector. ``arith`` is "fp32"
    (UNET3D_FP32) or "bf16" (UNET3D_BF16: tensor-core convolutions, BF16 activations)."""

    ARITH = {"fp32": 0, "bf16": 1}

    def __init__(self, n_in, n_out, crop, channels=(16, 32, 64), stream=None, arith="fp32"):
        import torch
        self._torch = torch
        self.lib = load()
        self.n_in, self.n_out, self.crop = n_in, n_out, crop
        self.arith = arith
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        net = ctypes.c_void_p()
        st = self.lib.unet3d_create_ex(n_in, n_out, crop, channels[0], channels[1], channels[2], self.ARITH[arith],
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(net))
        if st != 0:
            raise RuntimeError("unet3d_create: " + self.lib.unet3d_last_error().decode())
        self.net = net
        self.n_params = int(self.lib.unet3d_param_count(net))

    def _ok(self, st):
        if st != 0:
            raise RuntimeError("unet3d: " + self.lib.unet3d_last_error().decode())

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError("parameter vector has %d values, expected %d" % (a.size, self.n_params))
        self._ok(self.lib.unet3d_set_params(self.net, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._ok(self.lib.unet3d_get_params(self.net, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def get_grads(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._ok(self.lib.unet3d_get_grads(self.net, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def forward(self, x, y):
        px = _f32_cuda(x, self.n_in * self.crop ** 3, "x")
        py = _f32_cuda(y, self.n_out * self.crop ** 3, "y")
        self._ok(self.lib.unet3d_forward(self.net, px, py))

    def backward(self, gy):
        self._ok(self.lib.unet3d_backward(self.net, _f32_cuda(gy, self.n_out * self.crop ** 3, "gy")))

    def mse(self, y, target, gy):
        n = y.numel() if hasattr(y, "numel") else 0
        py = _f32_cuda(y, n, "y")
        pt = _f32_cuda(target, n, "target")
        pg = _f32_cuda(gy, n, "gy")
        loss = ctypes.c_double()
        self._ok(self.lib.unet3d_mse(self.net, py, pt, n, ctypes.byref(loss), pg))
        return loss.value

    def mse_core(self, y, target, gy, core_x, core_weight):
        """Weighted squared error (unet3d_mse_core): weight core_weight where the last
        input's first channel is at least core_x."""
        n = self.n_out * self.crop ** 3
        loss = ctypes.c_double()
        self._ok(self.lib.unet3d_mse_core(self.net, _f32_cuda(y, n, "y"), _f32_cuda(target, n, "target"),
                                          float(core_x), float(core_weight), ctypes.byref(loss), _f32_cuda(gy, n, "gy")))
        return loss.value

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        self._ok(self.lib.unet3d_adam(self.net, float(lr), float(beta1), float(beta2), float(eps), int(t)))

    def close(self):
        if getattr(self, "net", None):
            self.lib.unet3d_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def conv3_bf16(mode, n, cin, cout, inp, w, b=None, relu=False, in2=None, out=None):
    """unet3d_conv3_bf16 on torch CUDA tensors: ``inp`` (and ``in2``) bfloat16 channels-last
    [n^3, channels], ``w`` float32 [cout, cin, 27], ``b`` float32 [cout] or None. Mode 0
    returns y [n^3, cout] (bfloat16), mode 1 dL/dx [n^3, cin] (bfloat16), mode 2 dL/dw
    [cout, cin, 27] (float32)."""
    import torch
    lib = load()
    dev = inp.device
    for name, t, dt in (("inp", inp, torch.bfloat16), ("in2", in2, torch.bfloat16), ("w", w, torch.float32),
                        ("b", b, torch.float32)):
        if t is not None and (t.device != dev or t.dtype != dt or not t.is_contiguous()):
            raise ValueError("%s must be a contiguous %s tensor on %s" % (name, dt, dev))
    if mode == 0:
        out = torch.empty((n ** 3, cout), dtype=torch.bfloat16, device=dev) if out is None else out
    elif mode == 1:
        out = torch.empty((n ** 3, cin), dtype=torch.bfloat16, device=dev) if out is None else out
    else:
        out = torch.empty((cout, cin, 27), dtype=torch.float32, device=dev) if out is None else out
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream()
        st = lib.unet3d_conv3_bf16(int(mode), int(n), int(cin), int(cout), ctypes.c_void_p(inp.data_ptr()),
                                   ctypes.c_void_p(in2.data_ptr() if in2 is not None else 0),
                                   ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(b.data_ptr() if b is not None else 0),
                                   int(bool(relu)), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise RuntimeError("unet3d_conv3_bf16: " + lib.unet3d_last_error().decode())
    return out


def flatten_params(params):
    """Per-layer parameters [[w, b], ...] (w [out][in][3][3][3] or [out][in]) to the
    library's flat float32 vector, layer by layer, weights before biases."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def unflatten(flat, like):
    """Flat vector back to per-layer [[w, b], ...] with the shapes of ``like``."""
    out, o = [], 0
    for w, b in like:
        gw = flat[o:o + w.size].reshape(w.shape)
        o += w.size
        gb = flat[o:o + b.size]
        o += b.size
        out.append([gw, gb])
    return out
