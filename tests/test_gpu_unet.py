"""The learned-guess network on the GPU (unet3d.h kernels) against the FP64 oracle of
oracle/unet.py, and the solver's crop entry points.

Bars (FP32 kernels with FP32 accumulation against FP64): outputs within 2e-5 of their
largest magnitude, every layer's weight and bias gradient within 1e-4 of its largest
magnitude (sums of up to 27 x 96 products per output and 16^3 positions per gradient)."""
import numpy as np
import pytest

from oracle import rism3d as orc
from oracle import unet as ounet
from paper_2403_01039_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()


@pytest.mark.parametrize("channels,crop", [((4, 6, 8), 16), ((16, 32, 64), 12)])
def test_unet_forward_backward_match_oracle(channels, crop):
    rng = np.random.default_rng(8)
    n_in, n_out = 5, 5
    params = ounet.init_params(n_in, n_out, seed=3, channels=channels)
    for p in params:
        p[1] += 0.05 * rng.standard_normal(p[1].shape)
    flat = capi.flatten_params(params)
    params64 = capi.unflatten(flat.astype(np.float64), params)       # the FP32-rounded values
    x = rng.standard_normal((n_in, crop, crop, crop)).astype(np.float32)
    target = rng.standard_normal((n_out, crop, crop, crop)).astype(np.float32)
    y_ref, cache = ounet.forward(params64, x.astype(np.float64))
    loss_ref, gy_ref = ounet.mse(y_ref, target.astype(np.float64))
    g_ref = ounet.backward(params64, cache, gy_ref)

    net = capi.UNet3D(n_in, n_out, crop, channels)
    try:
        assert net.n_params == flat.size
        net.set_params(flat)
        assert np.array_equal(net.get_params(), flat)
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(target).cuda()
        yd = torch.empty_like(td)
        gyd = torch.empty_like(td)
        net.forward(xd, yd)
        loss = net.mse(yd, td, gyd)
        net.backward(gyd)
        g = capi.unflatten(net.get_grads().astype(np.float64), params)
    finally:
        net.close()
    y = yd.cpu().numpy()
    assert np.max(np.abs(y - y_ref)) <= 2e-5 * np.max(np.abs(y_ref))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    for k in range(len(params)):
        for j in range(2):
            ref = g_ref[k][j]
            scale = max(np.max(np.abs(ref)), 1e-30)
            assert np.max(np.abs(g[k][j] - ref)) <= 1e-4 * scale, (k, j, np.max(np.abs(g[k][j] - ref)), scale)


def test_guess_crops(water3):
    """Network input on a crop equals tanh(beta u / 4) of the oracle's potential; the
    converged iterate put back as a guess (whole-grid crop) restarts at the fixed point."""
    grid = synth.cubic_grid(32, 0.5)
    sol = synth.random_solute(6, 2.5, 17, net_charge=0.0)
    P = orc.Problem(water3, grid, sol)
    corner, crop = (4, 8, 0), 24
    with capi.Solver(water3, grid, precision=64) as S:
        S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
        x = torch.empty((3, crop, crop, crop), dtype=torch.float32, device="cuda")
        S.guess_input(corner, crop, x)
        ref = np.tanh(P.bu[:, 4:28, 8:32, 0:24] / 4.0)
        assert np.max(np.abs(x.cpu().numpy() - ref)) < 1e-6
        rep = S.solve("kh", tol=1e-6)
        full = torch.empty((3, 32, 32, 32), dtype=torch.float32, device="cuda")
        S.guess_target((0, 0, 0), 32, full)
        S.set_guess_crop((0, 0, 0), 32, full)
        rep2 = S.solve("kh", tol=1e-6)
        assert rep["converged"] and rep2["converged"] and rep2["iterations"] <= 3, (rep, rep2)
        with pytest.raises(capi.RismError):
            S.guess_input((10, 10, 10), 24, x)                       # outside the grid


def test_learned_guess_solve_matches_oracle(water_nacl):
    """solute50_128 (FP32, KH, tol 1e-6) started from the trained network's guess: the
    solve still ends at the oracle's fixed point (bars of the FP32 form against the oracle
    converged to 1e-10, at the 1024 stored sample points) in fewer iterations than from
    the zero guess."""
    import os
    from conftest import GOLDEN
    from paper_2403_01039_gb300 import guess
    wpath = os.path.join(os.path.dirname(capi.__file__), "data", "guess_unet_solute50_128.npz")
    ref = np.load(os.path.join(GOLDEN, "solute50_128_reference.npz"))
    W = np.load(wpath)
    crop = int(W["crop"])
    grid = synth.cubic_grid(128, 0.5)
    sol = synth.workload_solute("solute50_128")
    pts = ref["points"]
    net = capi.UNet3D(5, 5, crop, tuple(int(c) for c in W["channels"]))
    try:
        net.set_params(W["params"])
        with capi.Solver(water_nacl, grid, precision=32) as S:
            S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            zero = S.solve("kh", tol=1e-6)
            S.set_solute(sol["xyz"], sol["q"], sol["sigma"], sol["eps"])
            x = torch.empty((5, crop, crop, crop), dtype=torch.float32, device="cuda")
            y = torch.empty_like(x)
            c = guess.corner(128, crop)
            S.guess_input(c, crop, x)
            net.forward(x, y)
            S.set_guess_crop(c, crop, y)
            rep = S.solve("kh", tol=1e-6)
            g = S.get("g")[:, pts[:, 0], pts[:, 1], pts[:, 2]]
            sfe, _ = S.sfe("kh")
    finally:
        net.close()
    assert rep["converged"] and rep["iterations"] < zero["iterations"], (rep, zero)
    assert np.max(np.abs(g - ref["kh_1e-10_g"])) <= 1e-3
    assert abs(sfe - float(ref["kh_1e-10_sfe"])) <= 0.05
