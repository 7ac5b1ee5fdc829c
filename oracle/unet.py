"""3D U-Net of the learned initial guess (oracle, FP64; test infrastructure only).

The network maps the solute-solvent potential on a cubic crop to the initial iterate
tau = t - f of the 3D-RISM solve (step 1 of the numerical procedure takes t = f, i.e.
tau = 0; a learned guess starts closer to the fixed point). The paper has no learned
component: the architecture and its readings are this project's.

Architecture (channels C = (16, 32, 64)), on crops of side n divisible by 4:
  enc1 = relu(conv(relu(conv(x, w0)), w1))                      [C0, n]
  enc2 = relu(conv(relu(conv(pool(enc1), w2)), w3))              [C1, n/2]
  mid  = relu(conv(relu(conv(pool(enc2), w4)), w5))              [C2, n/4]
  dec2 = relu(conv(relu(conv(cat(up(mid), enc2), w6)), w7))     [C1, n/2]
  dec1 = relu(conv(relu(conv(cat(up(dec2), enc1), w8)), w9))     [C0, n]
  y    = conv1(dec1, w10)                                        [n_out, n]
conv: 3x3x3, zero padding 1, stride 1, with bias; pool: 2x2x2 mean; up: nearest, x2;
cat: channel concatenation (upsampled first); conv1: 1x1x1 with bias.
Loss: mean squared error over all outputs.

Every routine is a plain definition (direct sums over the 27 taps); the backward pass is
the chain rule through the same definitions.

BF16 storage form (``store=bf16_round``): the network of the BF16 configuration keeps its
activations and their gradients as bfloat16 values and multiplies BF16 weights; forward()
and backward() then round, at the points where that form stores a value, with the plain
definition of bfloat16 rounding (the FP32 value rounded to 8 significand bits, to nearest,
ties to even). Sums and products stay FP64.
"""
import numpy as np

CHANNELS = (16, 32, 64)


def bf16_round(a):
    """a rounded to the nearest bfloat16 value (ties to even), returned as float64: the
    float32 value of a keeps its upper 16 bits after adding half of the dropped range."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _keep(a):
    return a


def conv3(x, w, b):
    """y[o, i, j, k] = b[o] + sum_{c, a, d, e} w[o, c, a, d, e] x[c, i+a-1, j+d-1, k+e-1]
    (zero outside the crop). x [Ci, n, n, n], w [Co, Ci, 3, 3, 3]."""
    ci, n1, n2, n3 = x.shape
    xp = np.zeros((ci, n1 + 2, n2 + 2, n3 + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], n1, n2, n3))
    for a in range(3):
        for d in range(3):
            for e in range(3):
                y += np.einsum("oc,cijk->oijk", w[:, :, a, d, e], xp[:, a:a + n1, d:d + n2, e:e + n3])
    return y + b[:, None, None, None]


def conv3_backward(x, w, gy):
    """Gradients of conv3 with respect to x, w and b given dL/dy."""
    ci, n1, n2, n3 = x.shape
    xp = np.zeros((ci, n1 + 2, n2 + 2, n3 + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for a in range(3):
        for d in range(3):
            for e in range(3):
                win = xp[:, a:a + n1, d:d + n2, e:e + n3]
                gw[:, :, a, d, e] = np.einsum("oijk,cijk->oc", gy, win)
                gxp[:, a:a + n1, d:d + n2, e:e + n3] += np.einsum("oc,oijk->cijk", w[:, :, a, d, e], gy)
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gy.sum(axis=(1, 2, 3))


def conv1(x, w, b):
    """1x1x1 convolution: y[o] = b[o] + sum_c w[o, c] x[c]; w [Co, Ci]."""
    return np.einsum("oc,cijk->oijk", w, x) + b[:, None, None, None]


def pool(x):
    c, n1, n2, n3 = x.shape
    return x.reshape(c, n1 // 2, 2, n2 // 2, 2, n3 // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(gy):
    c, n1, n2, n3 = gy.shape
    return gy.reshape(c, n1 // 2, 2, n2 // 2, 2, n3 // 2, 2).sum(axis=(2, 4, 6))


def init_params(n_in, n_out, seed, channels=CHANNELS):
    """He-normal weights, zero biases (PCG64(seed)); the list order is w0..w10 as above."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c0, c1, c2 = channels
    shapes = [(c0, n_in), (c0, c0), (c1, c0), (c1, c1), (c2, c1), (c2, c2),
              (c1, c2 + c1), (c1, c1), (c0, c1 + c0), (c0, c0)]
    params = []
    for co, ci in shapes:
        params.append([rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co)])
    params.append([rng.standard_normal((n_out, c0)) * np.sqrt(1.0 / c0), np.zeros(n_out)])
    return params


def forward(params, x, store=None):
    """Returns (y, cache) for one crop x [n_in, n, n, n]. ``store`` (e.g. bf16_round) is
    applied to the input, to the 3x3x3 weights and to every stored activation."""
    st = store or _keep
    cache = {}

    def block(name, inp, k):
        a = conv3(inp, st(params[k][0]), params[k][1])
        ra = st(np.maximum(a, 0.0))
        b = conv3(ra, st(params[k + 1][0]), params[k + 1][1])
        rb = st(np.maximum(b, 0.0))
        cache[name] = (inp, a, ra, b)
        return rb

    e1 = block("e1", st(x), 0)
    e2 = block("e2", st(pool(e1)), 2)
    m = block("m", st(pool(e2)), 4)
    d2 = block("d2", np.concatenate([up(m), e2]), 6)
    d1 = block("d1", np.concatenate([up(d2), e1]), 8)
    y = conv1(d1, *params[10])
    cache["out"] = d1
    return y, cache


def backward(params, cache, gy, store=None):
    """Gradients [[gw, gb], ...] of the loss given dL/dy, in the order of params. With
    ``store``, the data gradients of the 3x3x3 layers use the stored (rounded) weights and
    every stored activation gradient is rounded; weight and bias gradients are not."""
    st = store or _keep
    grads = [None] * len(params)
    d1 = cache["out"]
    grads[10] = [np.einsum("oijk,cijk->oc", gy, d1), gy.sum(axis=(1, 2, 3))]
    g = st(np.einsum("oc,oijk->cijk", params[10][0], gy))

    def block_back(name, g_out, k):
        inp, a, ra, b = cache[name]
        gb_ = g_out * (b > 0)
        gra, gw1, gbias1 = conv3_backward(ra, st(params[k + 1][0]), gb_)
        ga = st(gra) * (a > 0)
        ginp, gw0, gbias0 = conv3_backward(inp, st(params[k][0]), ga)
        grads[k] = [gw0, gbias0]
        grads[k + 1] = [gw1, gbias1]
        return st(ginp)

    c0, c1, c2 = params[0][0].shape[0], params[2][0].shape[0], params[4][0].shape[0]
    gcat1 = block_back("d1", g, 8)                     # [c1 + c0]
    g_d2 = st(up_backward(gcat1[:c1]))
    g_e1 = gcat1[c1:].copy()
    gcat2 = block_back("d2", g_d2, 6)                  # [c2 + c1]
    g_m = st(up_backward(gcat2[:c2]))
    g_e2 = gcat2[c2:].copy()
    g_e2 = st(g_e2 + pool_backward(block_back("m", g_m, 4)))
    g_e1 = st(g_e1 + pool_backward(block_back("e2", g_e2, 2)))
    block_back("e1", g_e1, 0)
    return grads


def mse(y, target):
    """Loss and dL/dy of the mean squared error."""
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size
