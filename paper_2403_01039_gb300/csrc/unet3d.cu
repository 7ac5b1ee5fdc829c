// 3D U-Net of the learned initial guess: forward, backward, loss and Adam. The network is
// described in unet3d.h; the gradient is the chain rule through the same operations in
// reverse. Two arithmetic forms share the parameters, loss and optimiser: FP32 (direct
// convolutions over shared-memory tiles, channels-first activations) and BF16 (implicit-GEMM
// convolutions on the tensor cores with FP32 accumulation, channels-last BF16 activations;
// unet3d_tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "unet3d.h"
#include "unet3d_tc.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define UNET_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(3, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kTile = 8;              // output tile edge of the 3x3x3 convolutions
constexpr int kHalo = kTile + 2;
constexpr int kCob = 16;              // output channels per block
constexpr int kCib = 4;               // input channels per shared-memory stage

// ------------------------------------------------------------------ 3x3x3 convolution
// y[o][p] = b[o] + sum_c sum_tap w[o][c][tap] x[c][p + tap - 1] (zero outside), optional
// ReLU. One block per 8x8x8 output tile and kCob output channels; each thread owns two
// voxels (z and z + 4) of one (x, y) column and accumulates kCob channels.
__global__ void __launch_bounds__(256) k_conv3(const float *x, int ci, int n1, int n2, int n3, const float *w,
                                               const float *b, int co, int relu, float *y) {
    __shared__ float xs[kCib][kHalo][kHalo][kHalo];
    __shared__ float ws[kCib][27][kCob];
    const int t3n = (n3 + kTile - 1) / kTile, t2n = (n2 + kTile - 1) / kTile;
    int t = blockIdx.x;
    const int t3 = t % t3n;
    t /= t3n;
    const int t2 = t % t2n, t1 = t / t2n;
    const int i0 = t1 * kTile, j0 = t2 * kTile, k0 = t3 * kTile, o0 = blockIdx.y * kCob;
    const int tid = threadIdx.x;
    const int lk = tid & 3, lj = (tid >> 2) & 7, li = tid >> 5;
    const long long plane = (long long)n2 * n3, vol = (long long)n1 * plane;
    float acc[2][kCob];
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
        for (int o = 0; o < kCob; ++o) acc[v][o] = 0.f;
    for (int c0 = 0; c0 < ci; c0 += kCib) {
        __syncthreads();
        for (int e = tid; e < kCib * kHalo * kHalo * kHalo; e += blockDim.x) {
            const int cc = e / (kHalo * kHalo * kHalo), r = e - cc * (kHalo * kHalo * kHalo);
            const int a = r / (kHalo * kHalo), r2 = r - a * (kHalo * kHalo);
            const int d = r2 / kHalo, f = r2 - d * kHalo;
            const int gi = i0 - 1 + a, gj = j0 - 1 + d, gk = k0 - 1 + f;
            float v = 0.f;
            if (c0 + cc < ci && gi >= 0 && gi < n1 && gj >= 0 && gj < n2 && gk >= 0 && gk < n3)
                v = x[(long long)(c0 + cc) * vol + gi * plane + (long long)gj * n3 + gk];
            xs[cc][a][d][f] = v;
        }
        for (int e = tid; e < kCib * 27 * kCob; e += blockDim.x) {
            const int oo = e % kCob, r = e / kCob, tap = r % 27, cc = r / 27;
            float v = 0.f;
            if (c0 + cc < ci && o0 + oo < co) v = w[((long long)(o0 + oo) * ci + (c0 + cc)) * 27 + tap];
            ws[cc][tap][oo] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int cc = 0; cc < kCib; ++cc)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const int tap = (a * 3 + d) * 3 + f;
                        const float x0 = xs[cc][li + a][lj + d][lk + f];
                        const float x1 = xs[cc][li + a][lj + d][lk + 4 + f];
#pragma unroll
                        for (int o = 0; o < kCob; ++o) {
                            const float wv = ws[cc][tap][o];
                            acc[0][o] = fmaf(wv, x0, acc[0][o]);
                            acc[1][o] = fmaf(wv, x1, acc[1][o]);
                        }
                    }
    }
    const int gi = i0 + li, gj = j0 + lj;
    if (gi >= n1 || gj >= n2) return;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const int gk = k0 + lk + 4 * v;
        if (gk >= n3) continue;
#pragma unroll
        for (int o = 0; o < kCob; ++o) {
            if (o0 + o >= co) break;
            float r = acc[v][o] + (b ? b[o0 + o] : 0.f);
            if (relu) r = fmaxf(r, 0.f);
            y[(long long)(o0 + o) * vol + gi * plane + (long long)gj * n3 + gk] = r;
        }
    }
}

// wt[c][o][26 - tap] = w[o][c][tap]: the convolution that maps dL/dy to dL/dx.
__global__ void k_flip_transpose(const float *w, int co, int ci, float *wt) {
    const long long n = (long long)co * ci * 27;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int tap = (int)(i % 27);
        const long long oc = i / 27;
        const int c = (int)(oc % ci), o = (int)(oc / ci);
        wt[((long long)c * co + o) * 27 + (26 - tap)] = w[i];
    }
}

// Weight gradient partial sums: part[chunk][o][c][tap] = sum over the chunk's tiles of
// gy[o][p] x[c][p + tap - 1]. Block = (chunk, output-channel group, input-channel group);
// thread = (o, c) pair of the groups and a quarter of the 27 taps.
__global__ void __launch_bounds__(256) k_conv3_wgrad(const float *x, int ci, int n1, int n2, int n3, const float *gy,
                                                     int co, int tiles_per_chunk, float *part) {
    __shared__ float xs[kCib][kHalo][kHalo][kHalo];
    __shared__ float gs[kCob][kTile][kTile][kTile];
    const int t3n = (n3 + kTile - 1) / kTile, t2n = (n2 + kTile - 1) / kTile, t1n = (n1 + kTile - 1) / kTile;
    const int ntiles = t1n * t2n * t3n;
    const int chunk = blockIdx.x, o0 = blockIdx.y * kCob, c0 = blockIdx.z * kCib;
    const int tid = threadIdx.x;
    const int pair = tid >> 2, tg = tid & 3;           // 64 pairs: o = pair / kCib, c = pair % kCib
    const int oo = pair / kCib, cc = pair - oo * kCib;
    const long long plane = (long long)n2 * n3, vol = (long long)n1 * plane;
    float acc[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] = 0.f;
    const int tbeg = chunk * tiles_per_chunk, tend = min(ntiles, tbeg + tiles_per_chunk);
    for (int tile = tbeg; tile < tend; ++tile) {
        int t = tile;
        const int t3 = t % t3n;
        t /= t3n;
        const int t2 = t % t2n, t1 = t / t2n;
        const int i0 = t1 * kTile, j0 = t2 * kTile, k0 = t3 * kTile;
        __syncthreads();
        for (int e = tid; e < kCib * kHalo * kHalo * kHalo; e += blockDim.x) {
            const int c = e / (kHalo * kHalo * kHalo), r = e - c * (kHalo * kHalo * kHalo);
            const int a = r / (kHalo * kHalo), r2 = r - a * (kHalo * kHalo);
            const int d = r2 / kHalo, f = r2 - d * kHalo;
            const int gi = i0 - 1 + a, gj = j0 - 1 + d, gk = k0 - 1 + f;
            float v = 0.f;
            if (c0 + c < ci && gi >= 0 && gi < n1 && gj >= 0 && gj < n2 && gk >= 0 && gk < n3)
                v = x[(long long)(c0 + c) * vol + gi * plane + (long long)gj * n3 + gk];
            xs[c][a][d][f] = v;
        }
        for (int e = tid; e < kCob * kTile * kTile * kTile; e += blockDim.x) {
            const int o = e / (kTile * kTile * kTile), r = e - o * (kTile * kTile * kTile);
            const int a = r / (kTile * kTile), r2 = r - a * (kTile * kTile);
            const int d = r2 / kTile, f = r2 - d * kTile;
            const int gi = i0 + a, gj = j0 + d, gk = k0 + f;
            float v = 0.f;
            if (o0 + o < co && gi < n1 && gj < n2 && gk < n3)
                v = gy[(long long)(o0 + o) * vol + gi * plane + (long long)gj * n3 + gk];
            gs[o][a][d][f] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int p = 0; p < kTile * kTile * kTile; ++p) {
            const int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
            const float g = gs[oo][li][lj][lk];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const int tap = tg + 4 * q;
                if (tap < 27) {
                    const int a = tap / 9, d = (tap / 3) % 3, f = tap % 3;
                    acc[q] = fmaf(g, xs[cc][li + a][lj + d][lk + f], acc[q]);
                }
            }
        }
    }
    if (o0 + oo < co && c0 + cc < ci) {
        float *dst = part + ((long long)chunk * co + (o0 + oo)) * ci * 27 + (long long)(c0 + cc) * 27;
#pragma unroll
        for (int q = 0; q < 7; ++q)
            if (tg + 4 * q < 27) dst[tg + 4 * q] = acc[q];
    }
}

// out[i] = sum_{k < nk} part[k][i] in order (reproducible).
__global__ void k_sum_parts(const float *part, int nk, long long n, float *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < nk; ++k) s += part[(long long)k * n + i];
        out[i] = s;
    }
}

// gb[o] = sum_p gy[o][p] (one block per channel, fixed reduction order).
__global__ void k_bias_grad(const float *gy, long long vol, float *gb) {
    __shared__ float red[8];
    const float *g = gy + (long long)blockIdx.x * vol;
    float s = 0.f;
    for (long long p = threadIdx.x; p < vol; p += blockDim.x) s += g[p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        gb[blockIdx.x] = t;
    }
}

// g *= (y > 0): ReLU backward from the ReLU output.
__global__ void k_relu_back(float *g, const float *y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) g[i] = 0.f;
}

// ------------------------------------------------------------------ 1x1x1 convolution
__global__ void k_conv1(const float *x, int ci, long long vol, const float *w, const float *b, int co, float *y) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < vol; p += (long long)gridDim.x * blockDim.x)
        for (int o = 0; o < co; ++o) {
            float s = b[o];
            for (int c = 0; c < ci; ++c) s = fmaf(w[o * ci + c], x[c * vol + p], s);
            y[o * vol + p] = s;
        }
}

// gx[c][p] = sum_o w[o][c] gy[o][p]
__global__ void k_conv1_dgrad(const float *gy, int co, long long vol, const float *w, int ci, float *gx) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < vol; p += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < ci; ++c) {
            float s = 0.f;
            for (int o = 0; o < co; ++o) s = fmaf(w[o * ci + c], gy[o * vol + p], s);
            gx[c * vol + p] = s;
        }
}

// gw[o][c] = sum_p gy[o][p] x[c][p] (one block per (o, c), fixed order)
__global__ void k_conv1_wgrad(const float *gy, const float *x, long long vol, int ci, float *gw) {
    __shared__ float red[8];
    const int o = blockIdx.x / ci, c = blockIdx.x - o * ci;
    float s = 0.f;
    for (long long p = threadIdx.x; p < vol; p += blockDim.x) s = fmaf(gy[o * vol + p], x[c * vol + p], s);
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        gw[blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ pool / up
// y[c][i][j][k] = mean of x[c][2i..2i+1][2j..][2k..]; x side n, y side n/2
__global__ void k_pool(const float *x, int C, int n, float *y) {
    const int m = n / 2;
    const long long total = (long long)C * m * m * m;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % m);
        r /= m;
        const int j = (int)(r % m);
        r /= m;
        const int i = (int)(r % m);
        const int c = (int)(r / m);
        const float *s = x + (long long)c * n * n * n;
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 2; ++d)
                for (int f = 0; f < 2; ++f) acc += s[((long long)(2 * i + a) * n + (2 * j + d)) * n + (2 * k + f)];
        y[id] = 0.125f * acc;
    }
}

// gx[c][p] += gy[c][p / 2] / 8 (pool backward, accumulating)
__global__ void k_pool_back_add(const float *gy, int C, int n, float *gx) {
    const int m = n / 2;
    const long long total = (long long)C * n * n * n;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % n);
        r /= n;
        const int j = (int)(r % n);
        r /= n;
        const int i = (int)(r % n);
        const int c = (int)(r / n);
        gx[id] += 0.125f * gy[(((long long)c * m + i / 2) * m + j / 2) * m + k / 2];
    }
}

// y[c][p] = x[c][p / 2] (nearest upsampling, side m -> 2m)
__global__ void k_up(const float *x, int C, int m, float *y) {
    const int n = 2 * m;
    const long long total = (long long)C * n * n * n;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % n);
        r /= n;
        const int j = (int)(r % n);
        r /= n;
        const int i = (int)(r % n);
        const int c = (int)(r / n);
        y[id] = x[(((long long)c * m + i / 2) * m + j / 2) * m + k / 2];
    }
}

// gx[c][q] = sum of gy[c] over the 8 children of q (up backward; side 2m -> m)
__global__ void k_up_back(const float *gy, int C, int m, float *gx) {
    const int n = 2 * m;
    const long long total = (long long)C * m * m * m;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % m);
        r /= m;
        const int j = (int)(r % m);
        r /= m;
        const int i = (int)(r % m);
        const int c = (int)(r / m);
        const float *s = gy + (long long)c * n * n * n;
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 2; ++d)
                for (int f = 0; f < 2; ++f) acc += s[((long long)(2 * i + a) * n + (2 * j + d)) * n + (2 * k + f)];
        gx[id] = acc;
    }
}

// ------------------------------------------------------------------ loss and optimiser
__global__ void k_mse(const float *y, const float *t, long long n, float scale, float *gy, double *part) {
    __shared__ double red[8];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        gy[i] = scale * d;
        s += (double)d * (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) acc += red[i];
        part[blockIdx.x] = acc;
    }
}

// Weighted squared error: weight cw where the first input channel x0[p] >= cx (p = i % vol),
// else 1. part[block] = (sum w d^2, sum w) in FP64; gy written by k_wmse_grad.
__global__ void k_wmse_part(const float *y, const float *t, const float *x0, long long vol, long long n, float cx,
                            float cw, double *part) {
    __shared__ double red[2][8];
    double s = 0.0, sw = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        const double w = x0[i % vol] >= cx ? (double)cw : 1.0;
        s += w * (double)d * (double)d;
        sw += w;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = s, red[1][threadIdx.x >> 5] = sw;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[0][i], b += red[1][i];
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_wmse_grad(const float *y, const float *t, const float *x0, long long vol, long long n, float cx,
                            float cw, float scale, float *gy) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float w = x0[i % vol] >= cx ? cw : 1.f;
        gy[i] = scale * w * (y[i] - t[i]);
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

constexpr int kMseBlocks = 304;

}  // namespace

// ------------------------------------------------------------------ network
struct unet3d {
    int n_in = 0, n_out = 0, n = 0, c0 = 0, c1 = 0, c2 = 0;
    cudaStream_t stream = nullptr;
    std::vector<size_t> woff, boff, wsize;   // per layer, offsets into the flat vector
    std::vector<int> lco, lci;               // per layer channels
    size_t nparam = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    std::vector<float *> bufs;               // every device allocation but the above
    float *x = nullptr;                      // copy of the last input
    bool have_forward = false;               // activations of a forward pass are stored
    float *cat1 = nullptr, *e1a = nullptr, *p1 = nullptr, *cat2 = nullptr, *e2a = nullptr, *p2 = nullptr;
    float *ma = nullptr, *mid = nullptr, *d2a = nullptr, *dec2 = nullptr, *d1a = nullptr, *dec1 = nullptr;
    // gradients of activations
    float *g_dec1 = nullptr, *g_d1a = nullptr, *g_cat1 = nullptr, *g_dec2 = nullptr, *g_d2a = nullptr;
    float *g_cat2 = nullptr, *g_mid = nullptr, *g_ma = nullptr, *g_p2 = nullptr, *g_e2a = nullptr;
    float *g_p1 = nullptr, *g_e1a = nullptr, *g_x = nullptr;
    float *wt = nullptr, *part = nullptr;
    size_t part_floats = 0;
    double *mse_part = nullptr, *mse_host = nullptr;
    double *mse_blocks2 = nullptr, *mse_host2 = nullptr;   // weighted loss: (sum w d^2, sum w) per block
    // BF16 form (arith = UNET3D_BF16): channels-last BF16 activations and their gradients
    int arith = UNET3D_FP32, cin0 = 0;       // cin0: input channels padded to a multiple of 16
    int *status = nullptr;                   // first failure reported by a tensor-core kernel
    __nv_bfloat16 *bx = nullptr, *bcat1 = nullptr, *be1a = nullptr, *bp1 = nullptr, *bcat2 = nullptr;
    __nv_bfloat16 *be2a = nullptr, *bp2 = nullptr, *bma = nullptr, *bmid = nullptr, *bd2a = nullptr;
    __nv_bfloat16 *bdec2 = nullptr, *bd1a = nullptr, *bdec1 = nullptr;
    __nv_bfloat16 *gb_dec1 = nullptr, *gb_d1a = nullptr, *gb_cat1 = nullptr, *gb_dec2 = nullptr, *gb_d2a = nullptr;
    __nv_bfloat16 *gb_cat2 = nullptr, *gb_mid = nullptr, *gb_ma = nullptr, *gb_p2 = nullptr, *gb_e2a = nullptr;
    __nv_bfloat16 *gb_p1 = nullptr, *gb_e1a = nullptr;
    __nv_bfloat16 *wprep = nullptr;          // prepared BF16 weights of the layer being run
    float *tpart = nullptr;                  // weight- and bias-gradient partial sums
};

namespace {

long long cube(int n) { return (long long)n * n * n; }

int alloc(unet3d *net, float **p, long long count) {
    if (cudaMalloc(p, (size_t)count * sizeof(float)) != cudaSuccess) return fail(2, "cudaMalloc failed");
    net->bufs.push_back(*p);
    return 0;
}

int alloc_b(unet3d *net, __nv_bfloat16 **p, long long count) {
    float *q = nullptr;
    const int e = alloc(net, &q, (count + 1) / 2);
    *p = reinterpret_cast<__nv_bfloat16 *>(q);
    return e;
}

#define UNET_TRY_TC(call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(3, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// Failure recorded by a tensor-core kernel (a wait on a barrier that ran out), read at the
// synchronous calls.
int tc_status(const unet3d *net) {
    if (!net->status) return 0;
    int st = 0;
    UNET_TRY(cudaMemcpyAsync(&st, net->status, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    if (st) return fail(3, "a tensor-core convolution gave up waiting on a barrier (code " + std::to_string(st) + ")");
    return 0;
}

tcnet::CLView cv(__nv_bfloat16 *p, int ld, int off = 0) { return tcnet::CLView{p, ld, off}; }

// BF16 form: y = relu(conv3(x)) of one layer (x with cin channels, padded for layer 0)
int conv3_tc(unet3d *net, int layer, tcnet::CLView x, int cin, int n, tcnet::CLView y) {
    const int co = net->lco[layer];
    UNET_TRY_TC(tcnet::prep_fwd(net->stream, net->params + net->woff[layer], co, net->lci[layer], cin, net->wprep));
    UNET_TRY_TC(tcnet::conv3(net->stream, x, cin, net->wprep, net->params + net->boff[layer], y, co, n, 1, net->status));
    return 0;
}

// BF16 form of conv3_back: gy (layer output gradient, masked in place), x the layer input
// (cin channels), y the layer output; gx (cin channels) when wanted.
int conv3_back_tc(unet3d *net, int layer, tcnet::CLView x, int cin, tcnet::CLView y, tcnet::CLView gy, int n,
                  const tcnet::CLView *gx) {
    const int co = net->lco[layer];
    const long long vol = cube(n);
    cudaStream_t s = net->stream;
    UNET_TRY_TC(tcnet::relu_back(s, gy, y, co, vol));
    UNET_TRY_TC(tcnet::conv3_wgrad(s, x, cin, net->lci[layer], gy, co, n, net->tpart, net->grads + net->woff[layer],
                                   net->status));
    UNET_TRY_TC(tcnet::bias_grad(s, gy, co, vol, net->tpart, net->grads + net->boff[layer]));
    if (gx) {
        UNET_TRY_TC(tcnet::prep_dgrad(s, net->params + net->woff[layer], co, cin, net->wprep));
        UNET_TRY_TC(tcnet::conv3(s, gy, co, net->wprep, nullptr, *gx, cin, n, 0, net->status));
    }
    return 0;
}

int conv3(unet3d *net, int layer, const float *x, int n, float *y, int relu) {
    const int ci = net->lci[layer], co = net->lco[layer];
    const int tn = (n + kTile - 1) / kTile;
    const dim3 grid((unsigned)(tn * tn * tn), (unsigned)((co + kCob - 1) / kCob));
    k_conv3<<<grid, 256, 0, net->stream>>>(x, ci, n, n, n, net->params + net->woff[layer],
                                           net->params + net->boff[layer], co, relu, y);
    UNET_TRY(cudaGetLastError());
    return 0;
}

// Backward of y = relu(conv3(x)) given dL/dy in gy (modified in place by the ReLU mask):
// parameter gradients of the layer, and dL/dx into gx when gx is not null.
int conv3_back(unet3d *net, int layer, const float *x, const float *y, float *gy, int n, float *gx) {
    const int ci = net->lci[layer], co = net->lco[layer];
    const long long vol = cube(n);
    k_relu_back<<<grid_for((long long)co * vol), 256, 0, net->stream>>>(gy, y, (long long)co * vol);
    UNET_TRY(cudaGetLastError());
    const int tn = (n + kTile - 1) / kTile, ntiles = tn * tn * tn;
    const int cog = (co + kCob - 1) / kCob, cig = (ci + kCib - 1) / kCib;
    int chunks = 600 / (cog * cig);
    chunks = chunks < 1 ? 1 : (chunks > ntiles ? ntiles : chunks);
    const int per = (ntiles + chunks - 1) / chunks;
    chunks = (ntiles + per - 1) / per;
    const long long nw = (long long)co * ci * 27;
    if ((size_t)(chunks * nw) > net->part_floats) return fail(4, "weight-gradient scratch too small");
    k_conv3_wgrad<<<dim3(chunks, cog, cig), 256, 0, net->stream>>>(x, ci, n, n, n, gy, co, per, net->part);
    UNET_TRY(cudaGetLastError());
    k_sum_parts<<<grid_for(nw), 256, 0, net->stream>>>(net->part, chunks, nw, net->grads + net->woff[layer]);
    UNET_TRY(cudaGetLastError());
    k_bias_grad<<<co, 256, 0, net->stream>>>(gy, vol, net->grads + net->boff[layer]);
    UNET_TRY(cudaGetLastError());
    if (gx) {
        k_flip_transpose<<<grid_for(nw), 256, 0, net->stream>>>(net->params + net->woff[layer], co, ci, net->wt);
        UNET_TRY(cudaGetLastError());
        const dim3 grid((unsigned)ntiles, (unsigned)((ci + kCob - 1) / kCob));
        k_conv3<<<grid, 256, 0, net->stream>>>(gy, co, n, n, n, net->wt, nullptr, ci, 0, gx);
        UNET_TRY(cudaGetLastError());
    }
    return 0;
}

// BF16 form: the same network with channels-last BF16 activations (views into the
// concatenation buffers as in the FP32 form: cat1 = [up(dec2), enc1], cat2 = [up(mid), enc2]).
int forward_tc(unet3d *net, const float *x, float *y) {
    const int n = net->n, h = n / 2, q = n / 4;
    const long long V = cube(n);
    const int c0 = net->c0, c1 = net->c1, c2 = net->c2, ci0 = net->cin0;
    cudaStream_t s = net->stream;
    const tcnet::CLView xb = cv(net->bx, ci0), e1a = cv(net->be1a, c0), enc1 = cv(net->bcat1, c1 + c0, c1);
    const tcnet::CLView p1 = cv(net->bp1, c0), e2a = cv(net->be2a, c1), enc2 = cv(net->bcat2, c2 + c1, c2);
    const tcnet::CLView p2 = cv(net->bp2, c1), ma = cv(net->bma, c2), mid = cv(net->bmid, c2);
    const tcnet::CLView cat2 = cv(net->bcat2, c2 + c1), d2a = cv(net->bd2a, c1), dec2 = cv(net->bdec2, c1);
    const tcnet::CLView cat1 = cv(net->bcat1, c1 + c0), d1a = cv(net->bd1a, c0), dec1 = cv(net->bdec1, c0);
    UNET_TRY_TC(tcnet::to_cl(s, x, net->n_in, V, net->bx, ci0));
    int e;
    if ((e = conv3_tc(net, 0, xb, ci0, n, e1a))) return e;
    if ((e = conv3_tc(net, 1, e1a, c0, n, enc1))) return e;
    UNET_TRY_TC(tcnet::pool(s, enc1, c0, n, p1));
    if ((e = conv3_tc(net, 2, p1, c0, h, e2a))) return e;
    if ((e = conv3_tc(net, 3, e2a, c1, h, enc2))) return e;
    UNET_TRY_TC(tcnet::pool(s, enc2, c1, h, p2));
    if ((e = conv3_tc(net, 4, p2, c1, q, ma))) return e;
    if ((e = conv3_tc(net, 5, ma, c2, q, mid))) return e;
    UNET_TRY_TC(tcnet::up(s, mid, c2, q, cat2));
    if ((e = conv3_tc(net, 6, cat2, c2 + c1, h, d2a))) return e;
    if ((e = conv3_tc(net, 7, d2a, c1, h, dec2))) return e;
    UNET_TRY_TC(tcnet::up(s, dec2, c1, h, cat1));
    if ((e = conv3_tc(net, 8, cat1, c1 + c0, n, d1a))) return e;
    if ((e = conv3_tc(net, 9, d1a, c0, n, dec1))) return e;
    UNET_TRY_TC(tcnet::conv1(s, dec1, c0, V, net->params + net->woff[10], net->params + net->boff[10], net->n_out, y));
    return 0;
}

int backward_tc(unet3d *net, const float *gy) {
    const int n = net->n, h = n / 2, q = n / 4;
    const long long V = cube(n);
    const int c0 = net->c0, c1 = net->c1, c2 = net->c2, ci0 = net->cin0;
    cudaStream_t s = net->stream;
    const tcnet::CLView xb = cv(net->bx, ci0), e1a = cv(net->be1a, c0), enc1 = cv(net->bcat1, c1 + c0, c1);
    const tcnet::CLView p1 = cv(net->bp1, c0), e2a = cv(net->be2a, c1), enc2 = cv(net->bcat2, c2 + c1, c2);
    const tcnet::CLView p2 = cv(net->bp2, c1), ma = cv(net->bma, c2), mid = cv(net->bmid, c2);
    const tcnet::CLView cat2 = cv(net->bcat2, c2 + c1), d2a = cv(net->bd2a, c1), dec2 = cv(net->bdec2, c1);
    const tcnet::CLView cat1 = cv(net->bcat1, c1 + c0), d1a = cv(net->bd1a, c0), dec1 = cv(net->bdec1, c0);
    const tcnet::CLView g_dec1 = cv(net->gb_dec1, c0), g_d1a = cv(net->gb_d1a, c0), g_cat1 = cv(net->gb_cat1, c1 + c0);
    const tcnet::CLView g_enc1 = cv(net->gb_cat1, c1 + c0, c1), g_dec2 = cv(net->gb_dec2, c1), g_d2a = cv(net->gb_d2a, c1);
    const tcnet::CLView g_cat2 = cv(net->gb_cat2, c2 + c1), g_enc2 = cv(net->gb_cat2, c2 + c1, c2);
    const tcnet::CLView g_mid = cv(net->gb_mid, c2), g_ma = cv(net->gb_ma, c2), g_p2 = cv(net->gb_p2, c1);
    const tcnet::CLView g_e2a = cv(net->gb_e2a, c1), g_p1 = cv(net->gb_p1, c0), g_e1a = cv(net->gb_e1a, c0);
    // output layer (FP32 arithmetic)
    UNET_TRY_TC(tcnet::conv1_wgrad(s, gy, net->n_out, dec1, V, c0, net->grads + net->woff[10]));
    k_bias_grad<<<net->n_out, 256, 0, s>>>(gy, V, net->grads + net->boff[10]);
    UNET_TRY(cudaGetLastError());
    UNET_TRY_TC(tcnet::conv1_dgrad(s, gy, net->n_out, V, net->params + net->woff[10], c0, g_dec1));
    int e;
    if ((e = conv3_back_tc(net, 9, d1a, c0, dec1, g_dec1, n, &g_d1a))) return e;
    if ((e = conv3_back_tc(net, 8, cat1, c1 + c0, d1a, g_d1a, n, &g_cat1))) return e;
    UNET_TRY_TC(tcnet::up_back(s, g_cat1, c1, h, g_dec2));
    if ((e = conv3_back_tc(net, 7, d2a, c1, dec2, g_dec2, h, &g_d2a))) return e;
    if ((e = conv3_back_tc(net, 6, cat2, c2 + c1, d2a, g_d2a, h, &g_cat2))) return e;
    UNET_TRY_TC(tcnet::up_back(s, g_cat2, c2, q, g_mid));
    if ((e = conv3_back_tc(net, 5, ma, c2, mid, g_mid, q, &g_ma))) return e;
    if ((e = conv3_back_tc(net, 4, p2, c1, ma, g_ma, q, &g_p2))) return e;
    UNET_TRY_TC(tcnet::pool_back_add(s, g_p2, c1, h, g_enc2));
    if ((e = conv3_back_tc(net, 3, e2a, c1, enc2, g_enc2, h, &g_e2a))) return e;
    if ((e = conv3_back_tc(net, 2, p1, c0, e2a, g_e2a, h, &g_p1))) return e;
    UNET_TRY_TC(tcnet::pool_back_add(s, g_p1, c0, n, g_enc1));
    if ((e = conv3_back_tc(net, 1, e1a, c0, enc1, g_enc1, n, &g_e1a))) return e;
    if ((e = conv3_back_tc(net, 0, xb, ci0, e1a, g_e1a, n, nullptr))) return e;
    return 0;
}

}  // namespace

extern "C" {

const char *unet3d_last_error(void) { return g_err.c_str(); }

int unet3d_create(int n_in, int n_out, int crop, int c0, int c1, int c2, void *stream, unet3d **out) {
    return unet3d_create_ex(n_in, n_out, crop, c0, c1, c2, UNET3D_FP32, stream, out);
}

int unet3d_create_ex(int n_in, int n_out, int crop, int c0, int c1, int c2, int arith, void *stream, unet3d **out) {
    if (!out) return fail(1, "null out");
    *out = nullptr;
    if (n_in < 1 || n_out < 1 || crop < 4 || crop % 4 || c0 < 1 || c1 < 1 || c2 < 1)
        return fail(1, "bad sizes (crop must be a positive multiple of 4)");
    if (arith != UNET3D_FP32 && arith != UNET3D_BF16) return fail(1, "arith must be UNET3D_FP32 or UNET3D_BF16");
    const int cin0 = (n_in + 15) / 16 * 16;
    unet3d *net = new unet3d();
    net->arith = arith, net->cin0 = cin0;
    net->n_in = n_in, net->n_out = n_out, net->n = crop, net->c0 = c0, net->c1 = c1, net->c2 = c2;
    net->stream = static_cast<cudaStream_t>(stream);
    const int lco[11] = {c0, c0, c1, c1, c2, c2, c1, c1, c0, c0, n_out};
    const int lci[11] = {n_in, c0, c0, c1, c1, c2, c2 + c1, c1, c1 + c0, c0, c0};
    if (arith == UNET3D_BF16) {
        bool ok = c0 % 16 == 0 && c1 % 16 == 0 && c2 % 16 == 0;
        for (int l = 0; l < 10 && ok; ++l) {
            const int ci = l == 0 ? cin0 : lci[l];
            ok = tcnet::conv_shape_ok(ci, lco[l]) && tcnet::wgrad_shape_ok(ci, lco[l]) &&
                 (l == 0 || tcnet::conv_shape_ok(lco[l], ci));
        }
        if (!ok) {
            delete net;
            return fail(1, "the BF16 form needs channel counts that are multiples of 16 within the tensor-core "
                           "tile limits");
        }
    }
    size_t off = 0, maxw = 0;
    for (int l = 0; l < 11; ++l) {
        const size_t nw = (size_t)lco[l] * lci[l] * (l < 10 ? 27 : 1);
        net->lco.push_back(lco[l]);
        net->lci.push_back(lci[l]);
        net->woff.push_back(off);
        net->wsize.push_back(nw);
        off += nw;
        net->boff.push_back(off);
        off += lco[l];
        maxw = nw > maxw ? nw : maxw;
    }
    net->nparam = off;
    const long long V = cube(crop), V2 = cube(crop / 2), V4 = cube(crop / 4);
    int e = 0;
    auto A = [&](float **p, long long count) {
        if (!e) e = alloc(net, p, count);
    };
    A(&net->params, (long long)off);
    A(&net->grads, (long long)off);
    A(&net->m, (long long)off);
    A(&net->v, (long long)off);
    A(&net->x, (long long)n_in * V);
    if (arith == UNET3D_BF16) {
        auto B = [&](__nv_bfloat16 **p, long long count) {
            if (!e) e = alloc_b(net, p, count);
        };
        B(&net->bx, (long long)cin0 * V);
        B(&net->bcat1, (long long)(c1 + c0) * V);
        B(&net->be1a, (long long)c0 * V);
        B(&net->bp1, (long long)c0 * V2);
        B(&net->bcat2, (long long)(c2 + c1) * V2);
        B(&net->be2a, (long long)c1 * V2);
        B(&net->bp2, (long long)c1 * V4);
        B(&net->bma, (long long)c2 * V4);
        B(&net->bmid, (long long)c2 * V4);
        B(&net->bd2a, (long long)c1 * V2);
        B(&net->bdec2, (long long)c1 * V2);
        B(&net->bd1a, (long long)c0 * V);
        B(&net->bdec1, (long long)c0 * V);
        B(&net->gb_dec1, (long long)c0 * V);
        B(&net->gb_d1a, (long long)c0 * V);
        B(&net->gb_cat1, (long long)(c1 + c0) * V);
        B(&net->gb_dec2, (long long)c1 * V2);
        B(&net->gb_d2a, (long long)c1 * V2);
        B(&net->gb_cat2, (long long)(c2 + c1) * V2);
        B(&net->gb_mid, (long long)c2 * V4);
        B(&net->gb_ma, (long long)c2 * V4);
        B(&net->gb_p2, (long long)c1 * V4);
        B(&net->gb_e2a, (long long)c1 * V2);
        B(&net->gb_p1, (long long)c0 * V2);
        B(&net->gb_e1a, (long long)c0 * V);
        size_t wmax = 0, pmax = 0;
        const int side[10] = {crop, crop, crop / 2, crop / 2, crop / 4, crop / 4, crop / 2, crop / 2, crop, crop};
        for (int l = 0; l < 10; ++l) {
            const int ci = l == 0 ? cin0 : lci[l];
            wmax = std::max(wmax, tcnet::prep_elems(ci, lco[l]));
            pmax = std::max(pmax, tcnet::wgrad_part_floats(side[l], ci, lco[l]));
            pmax = std::max(pmax, tcnet::bias_part_floats(lco[l]));
        }
        B(&net->wprep, (long long)wmax);
        A(&net->tpart, (long long)pmax);
        if (!e && cudaMalloc(&net->status, sizeof(int)) != cudaSuccess) e = fail(2, "cudaMalloc failed");
        if (!e && cudaMemset(net->status, 0, sizeof(int)) != cudaSuccess) e = fail(3, "cudaMemset failed");
    } else {
    A(&net->cat1, (long long)(c1 + c0) * V);
    A(&net->e1a, (long long)c0 * V);
    A(&net->p1, (long long)c0 * V2);
    A(&net->cat2, (long long)(c2 + c1) * V2);
    A(&net->e2a, (long long)c1 * V2);
    A(&net->p2, (long long)c1 * V4);
    A(&net->ma, (long long)c2 * V4);
    A(&net->mid, (long long)c2 * V4);
    A(&net->d2a, (long long)c1 * V2);
    A(&net->dec2, (long long)c1 * V2);
    A(&net->d1a, (long long)c0 * V);
    A(&net->dec1, (long long)c0 * V);
    A(&net->g_dec1, (long long)c0 * V);
    A(&net->g_d1a, (long long)c0 * V);
    A(&net->g_cat1, (long long)(c1 + c0) * V);
    A(&net->g_dec2, (long long)c1 * V2);
    A(&net->g_d2a, (long long)c1 * V2);
    A(&net->g_cat2, (long long)(c2 + c1) * V2);
    A(&net->g_mid, (long long)c2 * V4);
    A(&net->g_ma, (long long)c2 * V4);
    A(&net->g_p2, (long long)c1 * V4);
    A(&net->g_e2a, (long long)c1 * V2);
    A(&net->g_p1, (long long)c0 * V2);
    A(&net->g_e1a, (long long)c0 * V);
    A(&net->g_x, (long long)n_in * V);
    A(&net->wt, (long long)maxw);
    net->part_floats = (size_t)600 * maxw;
    A(&net->part, (long long)net->part_floats);
    }
    if (!e && cudaMalloc(&net->mse_part, kMseBlocks * sizeof(double)) != cudaSuccess) e = fail(2, "cudaMalloc failed");
    if (!e && cudaMallocHost(&net->mse_host, kMseBlocks * sizeof(double)) != cudaSuccess) e = fail(2, "cudaMallocHost failed");
    if (!e && (cudaMemset(net->m, 0, off * sizeof(float)) != cudaSuccess ||
               cudaMemset(net->v, 0, off * sizeof(float)) != cudaSuccess ||
               cudaMemset(net->params, 0, off * sizeof(float)) != cudaSuccess))
        e = fail(3, "cudaMemset failed");
    if (e) {
        unet3d_destroy(net);
        return e;
    }
    *out = net;
    return 0;
}

size_t unet3d_param_count(const unet3d *net) { return net ? net->nparam : 0; }

int unet3d_set_params(unet3d *net, const float *host) {
    if (!net || !host) return fail(1, "null argument");
    UNET_TRY(cudaMemcpyAsync(net->params, host, net->nparam * sizeof(float), cudaMemcpyHostToDevice, net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    return 0;
}

int unet3d_get_params(const unet3d *net, float *host) {
    if (!net || !host) return fail(1, "null argument");
    UNET_TRY(cudaMemcpyAsync(host, net->params, net->nparam * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    return 0;
}

int unet3d_get_grads(const unet3d *net, float *host) {
    if (!net || !host) return fail(1, "null argument");
    UNET_TRY(cudaMemcpyAsync(host, net->grads, net->nparam * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    return tc_status(net);
}

int unet3d_forward(unet3d *net, const float *x, float *y) {
    if (!net || !x || !y) return fail(1, "null argument");
    net->have_forward = false;
    const int n = net->n, h = n / 2, q = n / 4;
    const long long V = cube(n), V2 = cube(h), V4 = cube(q);
    const int c0 = net->c0, c1 = net->c1, c2 = net->c2;
    cudaStream_t s = net->stream;
    UNET_TRY(cudaMemcpyAsync(net->x, x, (size_t)net->n_in * V * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (net->arith == UNET3D_BF16) {
        const int e = forward_tc(net, net->x, y);
        if (e) return e;
        net->have_forward = true;
        return 0;
    }
    float *enc1 = net->cat1 + (long long)c1 * V, *enc2 = net->cat2 + (long long)c2 * V2;
    int e;
    if ((e = conv3(net, 0, net->x, n, net->e1a, 1))) return e;
    if ((e = conv3(net, 1, net->e1a, n, enc1, 1))) return e;
    k_pool<<<grid_for(c0 * V2), 256, 0, s>>>(enc1, c0, n, net->p1);
    if ((e = conv3(net, 2, net->p1, h, net->e2a, 1))) return e;
    if ((e = conv3(net, 3, net->e2a, h, enc2, 1))) return e;
    k_pool<<<grid_for(c1 * V4), 256, 0, s>>>(enc2, c1, h, net->p2);
    if ((e = conv3(net, 4, net->p2, q, net->ma, 1))) return e;
    if ((e = conv3(net, 5, net->ma, q, net->mid, 1))) return e;
    k_up<<<grid_for(c2 * V2), 256, 0, s>>>(net->mid, c2, q, net->cat2);
    if ((e = conv3(net, 6, net->cat2, h, net->d2a, 1))) return e;
    if ((e = conv3(net, 7, net->d2a, h, net->dec2, 1))) return e;
    k_up<<<grid_for(c1 * V), 256, 0, s>>>(net->dec2, c1, h, net->cat1);
    if ((e = conv3(net, 8, net->cat1, n, net->d1a, 1))) return e;
    if ((e = conv3(net, 9, net->d1a, n, net->dec1, 1))) return e;
    k_conv1<<<grid_for(V), 256, 0, s>>>(net->dec1, c0, V, net->params + net->woff[10], net->params + net->boff[10],
                                         net->n_out, y);
    UNET_TRY(cudaGetLastError());
    net->have_forward = true;
    return 0;
}

int unet3d_backward(unet3d *net, const float *gy) {
    if (!net || !gy) return fail(1, "null argument");
    if (!net->have_forward) return fail(4, "backward before a successful forward");
    if (net->arith == UNET3D_BF16) return backward_tc(net, gy);
    const int n = net->n, h = n / 2, q = n / 4;
    const long long V = cube(n), V2 = cube(h), V4 = cube(q);
    const int c0 = net->c0, c1 = net->c1, c2 = net->c2;
    cudaStream_t s = net->stream;
    float *enc1 = net->cat1 + (long long)c1 * V, *enc2 = net->cat2 + (long long)c2 * V2;
    // output layer
    k_conv1_wgrad<<<net->n_out * c0, 256, 0, s>>>(gy, net->dec1, V, c0, net->grads + net->woff[10]);
    k_bias_grad<<<net->n_out, 256, 0, s>>>(gy, V, net->grads + net->boff[10]);
    k_conv1_dgrad<<<grid_for(V), 256, 0, s>>>(gy, net->n_out, V, net->params + net->woff[10], c0, net->g_dec1);
    UNET_TRY(cudaGetLastError());
    int e;
    // decoder level 1: cat1 -> d1a -> dec1
    if ((e = conv3_back(net, 9, net->d1a, net->dec1, net->g_dec1, n, net->g_d1a))) return e;
    if ((e = conv3_back(net, 8, net->cat1, net->d1a, net->g_d1a, n, net->g_cat1))) return e;
    float *g_enc1 = net->g_cat1 + (long long)c1 * V;
    k_up_back<<<grid_for(c1 * V2), 256, 0, s>>>(net->g_cat1, c1, h, net->g_dec2);
    // decoder level 2: cat2 -> d2a -> dec2
    if ((e = conv3_back(net, 7, net->d2a, net->dec2, net->g_dec2, h, net->g_d2a))) return e;
    if ((e = conv3_back(net, 6, net->cat2, net->d2a, net->g_d2a, h, net->g_cat2))) return e;
    float *g_enc2 = net->g_cat2 + (long long)c2 * V2;
    k_up_back<<<grid_for(c2 * V4), 256, 0, s>>>(net->g_cat2, c2, q, net->g_mid);
    // middle: p2 -> ma -> mid
    if ((e = conv3_back(net, 5, net->ma, net->mid, net->g_mid, q, net->g_ma))) return e;
    if ((e = conv3_back(net, 4, net->p2, net->ma, net->g_ma, q, net->g_p2))) return e;
    k_pool_back_add<<<grid_for(c1 * V2), 256, 0, s>>>(net->g_p2, c1, h, g_enc2);
    // encoder level 2: p1 -> e2a -> enc2
    if ((e = conv3_back(net, 3, net->e2a, enc2, g_enc2, h, net->g_e2a))) return e;
    if ((e = conv3_back(net, 2, net->p1, net->e2a, net->g_e2a, h, net->g_p1))) return e;
    k_pool_back_add<<<grid_for(c0 * V), 256, 0, s>>>(net->g_p1, c0, n, g_enc1);
    // encoder level 1: x -> e1a -> enc1 (no input gradient needed)
    if ((e = conv3_back(net, 1, net->e1a, enc1, g_enc1, n, net->g_e1a))) return e;
    if ((e = conv3_back(net, 0, net->x, net->e1a, net->g_e1a, n, nullptr))) return e;
    UNET_TRY(cudaGetLastError());
    return 0;
}

int unet3d_mse(unet3d *net, const float *y, const float *target, size_t count, double *loss, float *gy) {
    if (!net || !y || !target || !gy || count == 0) return fail(1, "bad argument");
    k_mse<<<kMseBlocks, 256, 0, net->stream>>>(y, target, (long long)count, 2.0f / (float)count, gy, net->mse_part);
    UNET_TRY(cudaGetLastError());
    UNET_TRY(cudaMemcpyAsync(net->mse_host, net->mse_part, kMseBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                             net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    if (int e = tc_status(net)) return e;
    double s = 0.0;
    for (int i = 0; i < kMseBlocks; ++i) s += net->mse_host[i];
    if (loss) *loss = s / (double)count;
    return 0;
}

int unet3d_mse_core(unet3d *net, const float *y, const float *target, float core_x, float core_weight,
                    double *loss, float *gy) {
    if (!net || !y || !target || !gy || !(core_weight > 0.f)) return fail(1, "bad argument");
    if (!net->have_forward) return fail(4, "loss before a successful forward");
    const long long vol = cube(net->n), count = (long long)net->n_out * vol;
    if (net->mse_blocks2 == nullptr) {
        UNET_TRY(cudaMalloc(&net->mse_blocks2, 2 * kMseBlocks * sizeof(double)));
        UNET_TRY(cudaMallocHost(&net->mse_host2, 2 * kMseBlocks * sizeof(double)));
    }
    k_wmse_part<<<kMseBlocks, 256, 0, net->stream>>>(y, target, net->x, vol, count, core_x, core_weight, net->mse_blocks2);
    UNET_TRY(cudaGetLastError());
    UNET_TRY(cudaMemcpyAsync(net->mse_host2, net->mse_blocks2, 2 * kMseBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                             net->stream));
    UNET_TRY(cudaStreamSynchronize(net->stream));
    if (int e = tc_status(net)) return e;
    double s = 0.0, sw = 0.0;
    for (int i = 0; i < kMseBlocks; ++i) s += net->mse_host2[2 * i], sw += net->mse_host2[2 * i + 1];
    if (loss) *loss = s / sw;
    k_wmse_grad<<<grid_for(count), 256, 0, net->stream>>>(y, target, net->x, vol, count, core_x, core_weight,
                                                         (float)(2.0 / sw), gy);
    UNET_TRY(cudaGetLastError());
    return 0;
}

int unet3d_adam(unet3d *net, float lr, float beta1, float beta2, float eps, int t) {
    if (!net || t < 1) return fail(1, "bad argument");
    const float bc1 = 1.f - powf(beta1, (float)t), bc2 = 1.f - powf(beta2, (float)t);
    k_adam<<<grid_for((long long)net->nparam), 256, 0, net->stream>>>(net->params, net->grads, net->m, net->v,
                                                                      (long long)net->nparam, lr, beta1, beta2,
                                                                      eps, bc1, bc2);
    UNET_TRY(cudaGetLastError());
    return 0;
}

int unet3d_conv3_bf16(int mode, int n, int cin, int cout, const void *in, const void *in2, const float *w,
                      const float *b, int relu, void *out, void *stream) {
    if (mode < 0 || mode > 2 || n < 1 || !in || !w || !out || (mode == 2 && !in2)) return fail(1, "bad argument");
    const bool ok = mode == 0 ? tcnet::conv_shape_ok(cin, cout)
                    : mode == 1 ? tcnet::conv_shape_ok(cout, cin)
                                : tcnet::wgrad_shape_ok(cin, cout);
    if (!ok) return fail(1, "channel counts outside the tensor-core tile limits");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    __nv_bfloat16 *wp = nullptr;
    float *part = nullptr;
    int *status = nullptr;
    int rc = 0;
    auto run = [&]() -> int {
        UNET_TRY(cudaMalloc(&status, sizeof(int)));
        UNET_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
        __nv_bfloat16 *src = const_cast<__nv_bfloat16 *>(static_cast<const __nv_bfloat16 *>(in));
        if (mode == 0 || mode == 1) {
            UNET_TRY(cudaMalloc(&wp, tcnet::prep_elems(cin, cout) * sizeof(__nv_bfloat16)));
            if (mode == 0) {
                UNET_TRY(tcnet::prep_fwd(s, w, cout, cin, cin, wp));
                UNET_TRY(tcnet::conv3(s, cv(src, cin), cin, wp, b, cv(static_cast<__nv_bfloat16 *>(out), cout), cout, n,
                                      relu, status));
            } else {
                UNET_TRY(tcnet::prep_dgrad(s, w, cout, cin, wp));
                UNET_TRY(tcnet::conv3(s, cv(src, cout), cout, wp, nullptr, cv(static_cast<__nv_bfloat16 *>(out), cin), cin,
                                      n, 0, status));
            }
        } else {
            UNET_TRY(cudaMalloc(&part, tcnet::wgrad_part_floats(n, cin, cout) * sizeof(float)));
            __nv_bfloat16 *g = const_cast<__nv_bfloat16 *>(static_cast<const __nv_bfloat16 *>(in2));
            UNET_TRY(tcnet::conv3_wgrad(s, cv(src, cin), cin, cin, cv(g, cout), cout, n, part, static_cast<float *>(out),
                                        status));
        }
        int st = 0;
        UNET_TRY(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        UNET_TRY(cudaStreamSynchronize(s));
        if (st) return fail(3, "a tensor-core convolution gave up waiting on a barrier (code " + std::to_string(st) + ")");
        return 0;
    };
    rc = run();
    if (wp) cudaFree(wp);
    if (part) cudaFree(part);
    if (status) cudaFree(status);
    return rc;
}

void unet3d_destroy(unet3d *net) {
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    for (float *p : net->bufs) cudaFree(p);
    if (net->mse_part) cudaFree(net->mse_part);
    if (net->mse_host) cudaFreeHost(net->mse_host);
    if (net->status) cudaFree(net->status);
    if (net->mse_blocks2) cudaFree(net->mse_blocks2);
    if (net->mse_host2) cudaFreeHost(net->mse_host2);
    delete net;
}

}  // extern "C"
