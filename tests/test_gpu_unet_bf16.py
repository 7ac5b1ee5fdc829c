"""BF16 tensor-core form of the learned-guess network (unet3d.h, UNET3D_BF16) against the
FP64 oracle of oracle/unet.py.

Single layers (unet3d_conv3_bf16, the tcgen05 kernels alone): inputs and weights are BF16
values, so the oracle's FP64 convolution of those same values is the exact answer. The
tensor cores accumulate in FP32 and the forward and data-gradient results are rounded to
BF16 once, so the bar is one BF16 rounding, |y - ref| <= 2^-8 |ref|, plus 1e-5 of the
output's scale for the FP32 accumulation; the weight gradient is an FP32 result (sums over
up to 20^3 voxels, FP32 accumulation in the tensor core and a fixed-order sum of chunks):
1e-5 of its scale. Grids of 12^3 and 20^3 leave ragged tiles (a tile is 2 x 16 x 8 voxels).

Whole network: an exact reference does not exist, because the GPU accumulates in FP32
before each BF16 rounding and the oracle in FP64; the rare values near a rounding tie then
round differently (about 1e-3 of a layer's outputs, measured), and each such step perturbs
the next layer's values, which round differently in turn, so two BF16 computations of the
same network drift apart to about the size of their rounding error. The test therefore
holds the GPU to the accuracy of exact BF16 storage: its distance from the FP64 oracle
(relative Frobenius norm) for the output and for every parameter gradient is at most 1.5
times (+2e-3) the distance of the oracle's BF16 storage form (oracle.unet with
store=bf16_round: the same roundings at the same points, FP64 sums) from FP64, which is
about 7e-3 for the output and up to 7.5e-2 for the first layer's weight gradient, whose
sums over the crop cancel. A transposed tap, a wrong channel offset or a lost ReLU mask
gives errors of order one."""
import numpy as np
import pytest

from oracle import unet as ounet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2403_01039_gb300 import build, capi  # noqa: E402

build.build()


def _bf16(rng, shape, scale=1.0):
    """Random values that are exactly representable in BF16 (a CUDA bfloat16 tensor and its
    FP64 copy)."""
    t = torch.from_numpy((scale * rng.standard_normal(shape)).astype(np.float32)).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()


def _cf(a_cl, n):
    """channels-last [n^3, C] -> channels-first [C, n, n, n]"""
    return np.ascontiguousarray(a_cl.T).reshape(-1, n, n, n)


@pytest.mark.parametrize("n,cin,cout", [(12, 16, 16), (20, 48, 16), (12, 32, 64), (12, 96, 32), (8, 64, 128),
                                        (4, 64, 64), (3, 32, 64), (6, 96, 32)])
def test_conv3_bf16_layer_matches_oracle(n, cin, cout):
    rng = np.random.default_rng(n * 1000 + cin + cout)
    x_d, x = _bf16(rng, (n ** 3, cin))
    gy_d, gy = _bf16(rng, (n ** 3, cout))
    w32 = (rng.standard_normal((cout, cin, 27)) / np.sqrt(27 * cin)).astype(np.float32)
    b32 = rng.standard_normal(cout).astype(np.float32)
    wb = torch.from_numpy(w32).to(torch.bfloat16).to(torch.float64).numpy()     # the products' weights
    w_d, b_d = torch.from_numpy(w32).cuda(), torch.from_numpy(b32).cuda()
    w5 = wb.reshape(cout, cin, 3, 3, 3)
    xc, gyc = _cf(x, n), _cf(gy, n)

    # forward, with bias and ReLU
    y = capi.conv3_bf16(0, n, cin, cout, x_d, w_d, b_d, relu=True).to(torch.float64).cpu().numpy()
    ref = np.maximum(ounet.conv3(xc, w5, b32.astype(np.float64)), 0.0).reshape(cout, -1).T
    scale = np.max(np.abs(ref))
    err = np.abs(y - ref) - 2.0 ** -8 * np.abs(ref)
    assert np.max(err) <= 1e-5 * scale, ("forward", float(np.max(err)), scale)

    # data gradient (transposed, flipped taps)
    gx = capi.conv3_bf16(1, n, cin, cout, gy_d, w_d).to(torch.float64).cpu().numpy()
    gref, gwref, _ = ounet.conv3_backward(xc, w5, gyc)
    gref = gref.reshape(cin, -1).T
    scale = np.max(np.abs(gref))
    err = np.abs(gx - gref) - 2.0 ** -8 * np.abs(gref)
    assert np.max(err) <= 1e-5 * scale, ("data gradient", float(np.max(err)), scale)

    # weight gradient (FP32 result)
    gw = capi.conv3_bf16(2, n, cin, cout, x_d, w_d, in2=gy_d).cpu().numpy().astype(np.float64)
    gwref = gwref.reshape(cout, cin, 27)
    scale = np.max(np.abs(gwref))
    assert np.max(np.abs(gw - gwref)) <= 1e-5 * scale, ("weight gradient", float(np.max(np.abs(gw - gwref))), scale)


def test_conv3_bf16_rejects_shapes():
    x = torch.zeros((8 ** 3, 24), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((16, 24, 27), dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        capi.conv3_bf16(0, 8, 24, 16, x, w)            # 24 input channels: not a multiple of 16
    with pytest.raises(RuntimeError):
        capi.UNet3D(5, 5, 16, (4, 6, 8), arith="bf16")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("crop", [16, 12])
def test_unet_bf16_forward_backward_match_oracle(crop):
    rng = np.random.default_rng(9)
    n_in, n_out, channels = 5, 5, (16, 32, 64)
    params = ounet.init_params(n_in, n_out, seed=4, channels=channels)
    for p in params:
        p[1] += 0.05 * rng.standard_normal(p[1].shape)
    flat = capi.flatten_params(params)
    params64 = capi.unflatten(flat.astype(np.float64), params)
    x = rng.standard_normal((n_in, crop, crop, crop)).astype(np.float32)
    target = rng.standard_normal((n_out, crop, crop, crop)).astype(np.float32)
    y_ref, cache = ounet.forward(params64, x.astype(np.float64))
    loss_ref, gy_ref = ounet.mse(y_ref, target.astype(np.float64))
    g_ref = ounet.backward(params64, cache, gy_ref)
    st = ounet.bf16_round
    y_b, cache_b = ounet.forward(params64, x.astype(np.float64), store=st)
    _, gy_b = ounet.mse(y_b, target.astype(np.float64))
    g_b = ounet.backward(params64, cache_b, gy_b, store=st)

    net = capi.UNet3D(n_in, n_out, crop, channels, arith="bf16")
    try:
        assert net.n_params == flat.size
        net.set_params(flat)
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
    y = yd.cpu().numpy().astype(np.float64)
    assert _rel(y, y_ref) <= 1.5 * _rel(y_b, y_ref) + 2e-3, (_rel(y, y_ref), _rel(y_b, y_ref))
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    for k in range(len(params)):
        for j in range(2):
            own = _rel(g_b[k][j], g_ref[k][j])
            assert _rel(g[k][j], g_ref[k][j]) <= 1.5 * own + 2e-3, (k, j, _rel(g[k][j], g_ref[k][j]), own)


def test_learned_guess_bf16_solve_matches_oracle(water_nacl):
    """The stored network (trained in FP32; the parameters are the same flat FP32 vector in
    both forms) run in the BF16 form as the starting iterate of solute50_128 (FP32, KH, tol
    1e-6): the solve ends at the oracle's fixed point (FP32 bars against the oracle at 1e-10,
    1024 stored sample points) in fewer iterations than from the zero guess."""
    import os
    from conftest import GOLDEN
    from paper_2403_01039_gb300 import guess, synth
    wpath = os.path.join(os.path.dirname(capi.__file__), "data", "guess_unet_solute50_128.npz")
    ref = np.load(os.path.join(GOLDEN, "solute50_128_reference.npz"))
    W = np.load(wpath)
    crop = int(W["crop"])
    grid = synth.cubic_grid(128, 0.5)
    sol = synth.workload_solute("solute50_128")
    pts = ref["points"]
    net = capi.UNet3D(5, 5, crop, tuple(int(c) for c in W["channels"]), arith="bf16")
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
