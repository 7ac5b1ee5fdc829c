"""rism3d_sfe_noalloc: the SFE entry point that allocates no device memory.

Some callers cannot allocate: a host framework that owns every device allocation, or a
latency-critical loop in which cudaMalloc would synchronise the device. This test checks, on
the GPU and through the C ABI, that the no-allocation entry point gives the same SFE as the
context's rism3d_get_sfe, on two calls in a row (the static scratch is shared between
calls), that it rejects more sites than its static scratch holds, and that it rejects
fields outside device memory before launching anything. The file is named so that pytest
collects it last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi, synth  # noqa: E402

build.build()


def test_noalloc_sfe_matches_context_sfe(water_nacl):
    grid = synth.cubic_grid(32, 0.5)
    sol = synth.random_solute(8, 3.0, 11, net_charge=1.0)
    dV = 0.5 ** 3
    with capi.Solver(water_nacl, grid, precision=64) as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        S.solve("pse", pse_order=3, tol=1e-6)
        shape = S.field_shape
        h = torch.empty(shape, dtype=torch.float64, device="cuda")
        c = torch.empty(shape, dtype=torch.float64, device="cuda")
        t = torch.empty(shape, dtype=torch.float64, device="cuda")
        u = torch.empty(shape, dtype=torch.float64, device="cuda")
        S.get("h", out=h)
        S.get("c", out=c)
        S.get("t", out=t)
        S.get("u", out=u)
        d = t - u
        torch.cuda.synchronize()
        for kind in ("kh", "hnc", "gf", "pse"):
            ref_total, ref_per = S.sfe(kind, 3)
            for _ in range(2):                       # two calls in a row share the scratch
                tot, per = capi.sfe_noalloc(h, c, water_nacl["rho"], water_nacl["temperature"], dV,
                                            kind=kind, pse_order=3, d=d)
                assert abs(tot - ref_total) <= 1e-9 * max(1.0, abs(ref_total)), (kind, tot, ref_total)
                assert np.allclose(per, ref_per, rtol=1e-9, atol=1e-9)


def test_noalloc_rejects_too_many_sites():
    n = 9
    h = torch.zeros((n, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(capi.RismError) as e:
        capi.sfe_noalloc(h, h, np.full(n, 0.03), 298.15, 0.125)
    assert e.value.status == capi.EINVAL and "static scratch" in str(e.value)


def test_noalloc_rejects_host_memory():
    """Pinned host memory (which the GPU could even read) is refused by the pointer check,
    before any kernel runs."""
    import ctypes
    lib = capi.load()
    h = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    host = torch.zeros((1, 64), dtype=torch.float64).pin_memory()
    rho = np.full(1, 0.03)
    tot = ctypes.c_double()
    for hp, cp in ((host, h), (h, host)):
        st = lib.rism3d_sfe_noalloc(1, 64, ctypes.c_void_p(hp.data_ptr()), ctypes.c_void_p(cp.data_ptr()),
                                    None, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 298.15, 0.125,
                                    capi.SFE_KINDS["kh"], 1, ctypes.byref(tot), None, None)
        assert st == capi.EINVAL
        assert "device memory" in lib.rism3d_last_error(None).decode()
