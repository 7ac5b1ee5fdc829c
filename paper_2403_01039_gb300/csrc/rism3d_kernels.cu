// CUDA kernels of the 3D-RISM solve (sm_103a). One iteration of the procedure of the
// "Numerical procedure" section (steps 2-6) is four launches:
//
//   plane_fwd  : [MDIIS update, Eq. 40] -> closure (Eqs. 14-16, PSE-n) -> c^sr (Eq. 31)
//                -> real-to-complex FFT along z and complex FFT along y of one x-plane
//   pencil     : FFT along x -> 3D-RISM contraction h~_g = sum_a c~_a X_ag(|k|) with
//                c~ = c~^sr - f~ (Eqs. 13, 32) -> inverse FFT along x
//   plane_inv  : inverse FFT along y and complex-to-real along z -> residual
//                R = h + 1 - g (Eq. 33) -> FP64 Gram-row partials <R, R_i> and sum R^2
//   mdiis      : reduce the partials, update the Gram matrix, solve the bordered MDIIS
//                system (Eq. 40), convergence test on the RMS residual (Eq. 41 read as RMS)
//
// Every field stays in HBM between launches; the solver state lives in a device struct
// (Ctrl) so that one captured CUDA graph replays any number of iterations.
//
// The iterate is stored as tau = t - f (f = beta q phi of Eq. 29) and the potential as
// w = f - beta*u, so that d = -beta*u + t = w + tau and c^sr = g - 1 - t + f = g - 1 - tau
// (Eq. 31) without the large long-range parts of t and beta*u; since the MDIIS weights sum
// to one, iterating on tau is the same iteration as on t.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rism3d_internal.h"

namespace rism {

// ------------------------------------------------------------------ complex helpers
__host__ __device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return cmk(a.x, -a.y); }
// multiply by s * i (s = +1 or -1)
template <typename C> __host__ __device__ __forceinline__ C cmuli(C a, int s) {
    return s > 0 ? cmk(-a.y, a.x) : cmk(a.y, -a.x);
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
    return cmk(a.x * s, a.y * s);
}

// ------------------------------------------------------------------ small DFTs
// X_k = sum_n v_n exp(s 2 pi i n k / R), s = -1 forward, +1 inverse.
template <int R> struct Dft;

template <> struct Dft<2> {
    template <typename C> __device__ __forceinline__ static void run(C *v, int) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <> struct Dft<4> {
    template <typename C> __device__ __forceinline__ static void run(C *v, int s) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = cmuli(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <> struct Dft<8> {
    template <typename C> __device__ __forceinline__ static void run(C *v, int s) {
        typedef decltype(v[0].x) Rt;
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4>::run(e, s);
        Dft<4>::run(o, s);
        const Rt h = (Rt)0.70710678118654752440;   // sqrt(1/2)
        // w8^k = exp(s 2 pi i k / 8)
        C o1 = cmul(o[1], cmk(h, (Rt)s * h));
        C o2 = cmuli(o[2], s);
        C o3 = cmul(o[3], cmk(-h, (Rt)s * h));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <> struct Dft<3> {
    template <typename C> __device__ __forceinline__ static void run(C *v, int s) {
        typedef decltype(v[0].x) Rt;
        const Rt c = (Rt)0.86602540378443864676;   // sin(2 pi / 3)
        C t = cadd(v[1], v[2]);
        C u = cscale(cmuli(csub(v[1], v[2]), s), c);
        C m = csub(v[0], cscale(t, (Rt)0.5));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    }
};

template <> struct Dft<5> {
    template <typename C> __device__ __forceinline__ static void run(C *v, int s) {
        typedef decltype(v[0].x) Rt;
        const Rt c1 = (Rt)0.30901699437494742410, c2 = (Rt)-0.80901699437494742410;
        const Rt s1 = (Rt)0.95105651629515357212, s2 = (Rt)0.58778525229247312917;
        C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        C u1 = csub(v[1], v[4]), u2 = csub(v[2], v[3]);
        C a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
        C a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
        C b1 = cmuli(cadd(cscale(u1, s1), cscale(u2, s2)), s);
        C b2 = cmuli(csub(cscale(u1, s2), cscale(u2, s1)), s);
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

// ------------------------------------------------------------------ batched in-place FFT
// Self-sorting (Stockham) mixed-radix transform of nb sequences of length L held in
// shared memory (element stride es, sequence stride bs). All threads of the block take
// part; each stage loads every butterfly input into registers, synchronises, then writes,
// so the transform runs in place. MAXI bounds the butterflies a thread holds per stage;
// the host picks the batch chunk so that this bound holds.
template <typename C, int R, int MAXI>
__device__ __forceinline__ void fft_stage(C *buf, int L, int es, int nb, int bs, int Ns,
                                          const C *tw, int sign) {
    const int LR = L / R;
    const int items = nb * LR;
    const int step = L / (Ns * R);
    C v[MAXI][R];
#pragma unroll
    for (int m = 0; m < MAXI; ++m) {
        const int it = threadIdx.x + m * blockDim.x;
        if (it < items) {
            const int b = it / LR, j = it - b * LR;
            const C *src = buf + (long)b * bs;
            const int k = j % Ns;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C a = src[(j + r * LR) * es];
                if (r > 0) {
                    C w = tw[k * r * step];
                    if (sign > 0) w.y = -w.y;
                    a = cmul(a, w);
                }
                v[m][r] = a;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MAXI; ++m) {
        const int it = threadIdx.x + m * blockDim.x;
        if (it < items) {
            const int b = it / LR, j = it - b * LR;
            const int k = j % Ns;
            Dft<R>::run(v[m], sign);
            const int d0 = (j / Ns) * Ns * R + k;
            C *dst = buf + (long)b * bs;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[(d0 + r * Ns) * es] = v[m][r];
        }
    }
    __syncthreads();
}

template <typename C, int MAXC>
__device__ void fft_smem(C *buf, const FftPlan &p, int es, int nb, int bs, int chunk, const C *tw,
                         int sign) {
    for (int b0 = 0; b0 < nb; b0 += chunk) {
        const int nbc = min(chunk, nb - b0);
        C *base = buf + (long)b0 * bs;
        int Ns = 1;
        for (int st = 0; st < p.nst; ++st) {
            const int R = p.radix[st];
            switch (R) {
                case 8: fft_stage<C, 8, MAXC / 8>(base, p.L, es, nbc, bs, Ns, tw, sign); break;
                case 4: fft_stage<C, 4, MAXC / 4>(base, p.L, es, nbc, bs, Ns, tw, sign); break;
                case 2: fft_stage<C, 2, MAXC / 2>(base, p.L, es, nbc, bs, Ns, tw, sign); break;
                case 3: fft_stage<C, 3, MAXC / 3>(base, p.L, es, nbc, bs, Ns, tw, sign); break;
                case 5: fft_stage<C, 5, MAXC / 5>(base, p.L, es, nbc, bs, Ns, tw, sign); break;
                default: break;
            }
            Ns *= R;
        }
    }
}

template <typename T> struct MaxC;
template <> struct MaxC<float> { static constexpr int v = 8; };
template <> struct MaxC<double> { static constexpr int v = 8; };

// ------------------------------------------------------------------ closure
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }

// g(d), d = -beta u + t: HNC (Eq. 14), KH (Eqs. 15-16 read as exp(d) for d <= 0, 1 + d
// otherwise), PSE-n (exp(d) for d <= 0, sum_{i<=n} d^i / i! otherwise).
template <typename T>
__device__ __forceinline__ T closure_g(T d, int kind, int order) {
    if (kind == kHNC || d <= (T)0) return dexp(d);
    if (kind == kKH) return (T)1 + d;
    T term = (T)1, s = (T)1;
    for (int i = 1; i <= order; ++i) {
        term = term * d / (T)i;
        s += term;
    }
    return s;
}

// Error-free FP32 dot-product accumulation (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005): the rounding error of each product (recovered
// with an FMA) and of each sum (TwoSum) is carried in a second FP32 word, so the pair
// (hi, lo) holds the FP32 dot product to about FP64 accuracy without FP64 arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename T> struct GramAcc;
template <> struct GramAcc<float> {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float x, float y) {
        const float p = x * y;
        const float pe = __fmaf_rn(x, y, -p);
        float sm, e;
        two_sum(hi, p, sm, e);
        hi = sm;
        lo += e + pe;
    }
    __device__ __forceinline__ void merge(float h2, float l2) {
        float sm, e;
        two_sum(hi, h2, sm, e);
        hi = sm;
        lo += l2 + e;
    }
    __device__ __forceinline__ void warp_reduce() {
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            merge(h2, l2);
        }
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <> struct GramAcc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x, double y) { s += x * y; }
    __device__ __forceinline__ void warp_reduce() {
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

// ------------------------------------------------------------------ pass 1: plane_fwd
// One block per (x plane, site). MAXH bounds the stored MDIIS pairs (8 or 16) so the update
// coefficients and slots live in registers.
template <typename T, int MAXH>
__global__ void __launch_bounds__(kThreadsPlane, sizeof(T) == 4 ? 3 : 2)
k_plane_fwd(Fields<T> f) {
    typedef typename Cx<T>::type C;
    typedef typename Vec2<T>::type V2;
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = f.Kz, pitch = f.pitch;
    C *tw_h = buf + (long)Ny * pitch;
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];

    const int x = blockIdx.x, gam = blockIdx.y;
    const int stage = ctl->stage;
    const int kind = ctl->stage_kind[stage], order = ctl->stage_order[stage];
    const int cur = ctl->cur;
    const int do_update = ctl->do_update;
    const int upd_n = ctl->upd_n;
    const T eta = (T)ctl->eta;
    const long long ring = (long long)f.nv * f.G;
    const long long siteoff = (long long)gam * f.G + (long long)x * Ny * f.Nz;
    T coef[MAXH];
    int slot[MAXH];
#pragma unroll
    for (int i = 0; i < MAXH; ++i) {
        coef[i] = i < upd_n ? (T)ctl->upd_coef[i] : (T)0;
        slot[i] = i < upd_n ? ctl->upd_slot[i] : 0;
    }
    T *tcur = f.X + (long long)cur * ring + siteoff;
    const T *wp = f.w + siteoff;
    const int anchor = ctl->anchor_valid, refresh = ctl->refresh;
    T *ca = f.csr_a + siteoff;

    // update (Eq. 40) + closure + c^sr (Eq. 31), packed two reals per complex along z
    const int npairs = Ny * Kz;
    for (int idx = threadIdx.x; idx < npairs; idx += blockDim.x) {
        const int y = idx / Kz, m = idx - y * Kz;
        const long long o = (long long)y * f.Nz + 2 * m;
        V2 t;
        if (do_update) {
            t.x = (T)0;
            t.y = (T)0;
#pragma unroll
            for (int i = 0; i < MAXH; ++i) {
                if (i < upd_n) {
                    const long long base = (long long)slot[i] * ring + siteoff + o;
                    const V2 xv = *reinterpret_cast<const V2 *>(f.X + base);
                    const V2 rv = *reinterpret_cast<const V2 *>(f.R + base);
                    t.x += coef[i] * (xv.x + eta * rv.x);
                    t.y += coef[i] * (xv.y + eta * rv.y);
                }
            }
            *reinterpret_cast<V2 *>(tcur + o) = t;
        } else {
            t = *reinterpret_cast<const V2 *>(tcur + o);
        }
        const V2 wv = *reinterpret_cast<const V2 *>(wp + o);
        const T g0 = closure_g(wv.x + t.x, kind, order);
        const T g1 = closure_g(wv.y + t.y, kind, order);
        V2 c;
        c.x = g0 - (T)1 - t.x;
        c.y = g1 - (T)1 - t.y;
        C dc = cmk(c.x, c.y);
        if (anchor) {                          // transform only c^sr - c^sr_a
            const V2 a = *reinterpret_cast<const V2 *>(ca + o);
            dc.x -= a.x;
            dc.y -= a.y;
        }
        if (refresh) *reinterpret_cast<V2 *>(ca + o) = c;
        buf[y * pitch + m] = dc;
    }
    __syncthreads();
    // rows: complex FFT of length Kz
    fft_smem<C, MaxC<T>::v>(buf, f.ph, 1, Ny, pitch, f.chunk_rows, tw_h, -1);
    // real-to-complex post-processing: X[k] = E[k] + w^k O[k], k = 0..Kz
    const int half = Kz / 2;
    for (int idx = threadIdx.x; idx < Ny * (half + 1); idx += blockDim.x) {
        const int y = idx / (half + 1), k = idx - y * (half + 1);
        C *row = buf + y * pitch;
        if (k == 0) {
            C z = row[0];
            row[0] = cmk(z.x + z.y, (T)0);
            row[Kz] = cmk(z.x - z.y, (T)0);
        } else {
            const int k2 = Kz - k;
            C a = row[k], b = row[k2];
            C e1 = cscale(cadd(a, cconj(b)), (T)0.5);
            C o1 = cscale(csub(a, cconj(b)), (T)0.5);
            C X1 = cadd(e1, cmul(cmuli(o1, -1), tw_z[k]));
            if (k2 != k) {
                C e2 = cscale(cadd(b, cconj(a)), (T)0.5);
                C o2 = cscale(csub(b, cconj(a)), (T)0.5);
                row[k2] = cadd(e2, cmul(cmuli(o2, -1), tw_z[k2]));
            }
            row[k] = X1;
        }
    }
    __syncthreads();
    // columns: complex FFT of length Ny for kz = 0..Kz
    fft_smem<C, MaxC<T>::v>(buf, f.py, pitch, Kz + 1, 1, f.chunk_cols_fwd, tw_y, -1);
    C *dst = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;
    for (int idx = threadIdx.x; idx < Ny * Kz; idx += blockDim.x) {
        const int y = idx / Kz, k = idx - y * Kz;
        dst[idx] = buf[y * pitch + k];
    }
    C *dn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) dn[y] = buf[y * pitch + Kz];
}

// ------------------------------------------------------------------ pass 2: pencil
__device__ __forceinline__ int signed_index(int i, int N) { return (2 * i < N) ? i : i - N; }

// One block per tile of W spectrum columns (all x, all NV sites). NV is a template argument
// so the contraction unrolls over exactly the solvent sites.
template <typename T, int NV>
__global__ void __launch_bounds__(kThreadsPencil, sizeof(T) == 4 ? 3 : 2)
k_pencil(Fields<T> f) {
    typedef typename Cx<T>::type C;
    if (f.ctrl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Nx = f.Nx, Ny = f.Ny, Kz = f.Kz, W = f.W, pp = f.pencil_pitch;
    C *tw_x = buf + (long)NV * W * pp;
    for (int i = threadIdx.x; i < Nx; i += blockDim.x) tw_x[i] = f.tw_x[i];

    // main tiles cover (y, kz0 .. kz0+W) with kz < Kz; Nyquist tiles (y0 .. y0+W, kz = Kz)
    int tile = blockIdx.x;
    const bool nyq = tile >= f.tiles_main;
    int y = 0, kz0 = 0, y0 = 0, ncol;
    long long col_base, xstride;
    if (!nyq) {
        const int per = (Kz + W - 1) / W;
        y = tile / per;
        kz0 = (tile - y * per) * W;
        ncol = min(W, Kz - kz0);
        col_base = (long long)y * Kz + kz0;
        xstride = (long long)Ny * Kz;
    } else {
        tile -= f.tiles_main;
        y0 = tile * W;
        ncol = min(W, Ny - y0);
        col_base = y0;
        xstride = Ny;
    }
    const C *src_base = nyq ? f.spec_nyq : f.spec;
    const long long site_stride = (long long)Nx * xstride;
    const int nload = NV * Nx * ncol;
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int c = idx % ncol;
        const int rest = idx / ncol;
        const int xx = rest % Nx, a = rest / Nx;
        buf[(a * W + c) * pp + xx] = src_base[a * site_stride + xx * xstride + col_base + c];
    }
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, f.px, 1, NV * W, pp, f.chunk_x, tw_x, -1);
    // contraction (Eq. 13 with Eq. 32): E_g = sum_a D_a A_ag(|k|) [+ Psi A_{nv,g} before the
    // first anchor, after which f~ is part of h_a]
    const C *psi = nyq ? f.psi_nyq : f.psi;
    const bool psi_on = f.ctrl->anchor_valid == 0;
    const int npts = Nx * ncol;
    constexpr int rowlen = (NV + 1) * NV;
    const T ks0 = (T)f.ks[0], ks1 = (T)f.ks[1], ks2 = (T)f.ks[2], inv_dk = (T)f.inv_dk;
    for (int idx = threadIdx.x; idx < npts; idx += blockDim.x) {
        const int c = idx % ncol, xx = idx / ncol;
        const int yy = nyq ? y0 + c : y;
        const int kz = nyq ? Kz : kz0 + c;
        const T kx = ks0 * (T)signed_index(xx, Nx);
        const T ky = ks1 * (T)signed_index(yy, Ny);
        const T kzv = ks2 * (T)kz;
        const T xk = sqrt(kx * kx + ky * ky + kzv * kzv) * inv_dk;
        int j = (int)floor(xk);
        if (j > f.nk - 2) j = f.nk - 2;
        T w = xk - (T)j;
        w = w < (T)0 ? (T)0 : (w > (T)1 ? (T)1 : w);
        const T *A0 = f.table + (long long)j * rowlen;
        const T *A1 = A0 + rowlen;
        C D[NV];
#pragma unroll
        for (int a = 0; a < NV; ++a) D[a] = buf[(a * W + c) * pp + xx];
        const C Psi = psi_on ? psi[xx * xstride + col_base + c] : cmk((T)0, (T)0);
#pragma unroll
        for (int g = 0; g < NV; ++g) {
            T ar = (T)0, ai = (T)0;
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                const T coef = __ldg(A0 + a * NV + g) * ((T)1 - w) + __ldg(A1 + a * NV + g) * w;
                ar += coef * D[a].x;
                ai += coef * D[a].y;
            }
            if (psi_on) {
                const T coef = __ldg(A0 + NV * NV + g) * ((T)1 - w) + __ldg(A1 + NV * NV + g) * w;
                ar += coef * Psi.x;
                ai += coef * Psi.y;
            }
            buf[(g * W + c) * pp + xx] = cmk(ar, ai);
        }
    }
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, f.px, 1, NV * W, pp, f.chunk_x, tw_x, +1);
    C *dst_base = nyq ? f.spec_nyq : f.spec;
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int c = idx % ncol;
        const int rest = idx / ncol;
        const int xx = rest % Nx, a = rest / Nx;
        dst_base[a * site_stride + xx * xstride + col_base + c] = buf[(a * W + c) * pp + xx];
    }
}

// ------------------------------------------------------------------ pass 3: plane_inv
// One block per (x plane, site): inverse y and z transforms, residual, and the block's
// contribution to <R_cur, R_i> and sum R^2 (Dot2 accumulation, FP64 across threads).
// Partials are stored value-major: partials[i * n_blocks + block].
template <typename T, int MAXH>
__global__ void __launch_bounds__(kThreadsPlane, sizeof(T) == 4 ? 3 : 2)
k_plane_inv(Fields<T> f) {
    typedef typename Cx<T>::type C;
    typedef typename Vec2<T>::type V2;
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = f.Kz, pitch = f.pitch;
    C *tw_h = buf + (long)Ny * pitch;
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    double *red = reinterpret_cast<double *>(tw_z + (Kz + 1));
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];
    const int x = blockIdx.x, gam = blockIdx.y;

    const C *src = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;
    for (int idx = threadIdx.x; idx < Ny * Kz; idx += blockDim.x) {
        const int y = idx / Kz, k = idx - y * Kz;
        buf[y * pitch + k] = src[idx];
    }
    const C *sn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) buf[y * pitch + Kz] = sn[y];
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, f.py, pitch, Kz + 1, 1, f.chunk_cols_fwd, tw_y, +1);
    // complex-to-real pre-processing: Z[k] = (X[k] + conj X[Kz-k]) + i w^-k (X[k] - conj X[Kz-k])
    const int half = Kz / 2;
    for (int idx = threadIdx.x; idx < Ny * (half + 1); idx += blockDim.x) {
        const int y = idx / (half + 1), k = idx - y * (half + 1);
        C *row = buf + y * pitch;
        const int k2 = Kz - k;
        C a = row[k], b = row[k2];
        C Z1 = cadd(cadd(a, cconj(b)), cmuli(cmul(csub(a, cconj(b)), cconj(tw_z[k])), +1));
        if (k != 0 && k2 != k)
            row[k2] = cadd(cadd(b, cconj(a)), cmuli(cmul(csub(b, cconj(a)), cconj(tw_z[k2])), +1));
        row[k] = Z1;
    }
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, f.ph, 1, Ny, pitch, f.chunk_rows, tw_h, +1);

    const int stage = ctl->stage;
    const int kind = ctl->stage_kind[stage], order = ctl->stage_order[stage];
    const int cur = ctl->cur;
    const int hist_n = ctl->hist_n;
    const long long ring = (long long)f.nv * f.G;
    const long long siteoff = (long long)gam * f.G + (long long)x * Ny * f.Nz;
    const T *tcur = f.X + (long long)cur * ring + siteoff;
    T *rcur = f.R + (long long)cur * ring + siteoff;
    const T *wp = f.w + siteoff;
    const int anchor = ctl->anchor_valid, refresh = ctl->refresh;
    T *ha = f.h_a + siteoff;
    int hslot[MAXH];
#pragma unroll
    for (int i = 0; i < MAXH; ++i) hslot[i] = i < hist_n ? ctl->hist_slot[i] : 0;
    GramAcc<T> acc[MAXH + 1];
#pragma unroll
    for (int i = 0; i <= MAXH; ++i) acc[i].zero();
    for (int idx = threadIdx.x; idx < Ny * Kz; idx += blockDim.x) {
        const int y = idx / Kz, m = idx - y * Kz;
        const long long o = (long long)y * f.Nz + 2 * m;
        const C hc = buf[y * pitch + m];
        const V2 t = *reinterpret_cast<const V2 *>(tcur + o);
        const V2 wv = *reinterpret_cast<const V2 *>(wp + o);
        const T g0 = closure_g(wv.x + t.x, kind, order);
        const T g1 = closure_g(wv.y + t.y, kind, order);
        // R = h + 1 - g (Eq. 33) with h = h_a + dh; (h_a - g) first: near association peaks
        // both are large and close, and the difference is then exact
        V2 r, h;
        if (anchor) {
            const V2 a = *reinterpret_cast<const V2 *>(ha + o);
            r.x = ((a.x - g0) + (T)1) + hc.x;
            r.y = ((a.y - g1) + (T)1) + hc.y;
            h.x = a.x + hc.x;
            h.y = a.y + hc.y;
        } else {
            r.x = (hc.x - g0) + (T)1;
            r.y = (hc.y - g1) + (T)1;
            h.x = hc.x;
            h.y = hc.y;
        }
        if (refresh) *reinterpret_cast<V2 *>(ha + o) = h;
        *reinterpret_cast<V2 *>(rcur + o) = r;
        acc[0].add(r.x, r.x);
        acc[0].add(r.y, r.y);
#pragma unroll
        for (int i = 0; i < MAXH; ++i) {
            if (i < hist_n) {
                const V2 q = *reinterpret_cast<const V2 *>(f.R + (long long)hslot[i] * ring + siteoff + o);
                acc[i + 1].add(r.x, q.x);
                acc[i + 1].add(r.y, q.y);
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long nblocks = (long long)f.nv * f.Nx;
    const long long blk = (long long)gam * f.Nx + x;
#pragma unroll
    for (int i = 0; i <= MAXH; ++i) {
        if (i <= hist_n) {
            acc[i].warp_reduce();
            if (lane == 0) red[i * nw + warp] = acc[i].value();
        }
    }
    __syncthreads();
    if (threadIdx.x <= hist_n) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += red[threadIdx.x * nw + k];
        f.partials[threadIdx.x * nblocks + blk] = s;
    }
}

// ------------------------------------------------------------------ MDIIS (one block)
// Reduce the Gram partials in a fixed order (bit-reproducible), update B, then one thread
// solves the bordered system [B 1; 1^T 0][c; l] = [0; 1] by Gaussian elimination with
// partial pivoting (B scaled by its largest diagonal entry; pivots below 1e-12 drop the
// oldest vector and retry), and prepares the next update (Eq. 40).
__global__ void k_mdiis(Ctrl *ctl, const double *partials, int nblocks) {
    __shared__ double sums[kMaxHist + 1];
    if (ctl->status != kRunning) return;
    const int hist_n = ctl->hist_n;
    __syncthreads();
    if (threadIdx.x == 0) {           // what this iteration's kernels moved (byte model)
        ctl->acc_iters += 1;
        ctl->acc_fwd_units += ctl->do_update ? 2 * ctl->upd_n + 1 : 1;
        ctl->acc_hist += hist_n;
        ctl->acc_anchor += ctl->anchor_valid;
        ctl->acc_refresh += ctl->refresh;
        ctl->acc_psi += ctl->anchor_valid == 0;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp <= hist_n) {
        const double *pv = partials + (long long)warp * nblocks;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = lane;
        for (; b + 96 < nblocks; b += 128) {
            s0 += pv[b];
            s1 += pv[b + 32];
            s2 += pv[b + 64];
            s3 += pv[b + 96];
        }
        for (; b < nblocks; b += 32) s0 += pv[b];
        double s = (s0 + s1) + (s2 + s3);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sums[warp] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;

    const int M = ctl->M;
    const int cur = ctl->cur;
    const double rr = sums[0];
    const double rms = sqrt(rr * ctl->inv_count);
    ctl->rms = rms;
    ctl->iter += 1;
    if (ctl->refresh) {               // this iteration wrote c^sr_a and h_a
        ctl->refresh = 0;
        ctl->anchor_valid = 1;
    }
    if (!isfinite(rms)) {
        ctl->status = kDiverged;
        return;
    }
    if (rms < ctl->next_refresh) {    // next iteration re-anchors the transform
        ctl->refresh = 1;
        ctl->next_refresh = rms * 1e-2;
    }
    const int st = ctl->stage;
    if (rms < ctl->stage_tol[st]) {
        if (st + 1 >= ctl->n_stages) {
            ctl->status = kConverged;
        } else if (ctl->iter >= ctl->max_iter) {
            ctl->status = kMaxIter;
        } else {                      // closure continuation: next stage from this t
            ctl->stage = st + 1;
            ctl->hist_n = 0;
            ctl->do_update = 0;
            ctl->upd_n = 0;
        }
        return;
    }
    if (ctl->iter >= ctl->max_iter) {
        ctl->status = kMaxIter;
        return;
    }
    // Gram row of the new residual
    for (int i = 0; i < hist_n; ++i) {
        const int s = ctl->hist_slot[i];
        ctl->B[cur * kMaxHist + s] = sums[i + 1];
        ctl->B[s * kMaxHist + cur] = sums[i + 1];
    }
    ctl->B[cur * kMaxHist + cur] = rr;
    int H[kMaxHist];
    int k = 0;
    for (int i = 0; i < hist_n; ++i) H[k++] = ctl->hist_slot[i];
    H[k++] = cur;
    double c[kMaxHist];
    int first = 0;
    if (ctl->accel == 1) {
        // modified Anderson, two histories (Eqs. 34-39): theta from the 2 x 2 system of
        // Eq. 36 on D_i = R_new - R_{new-i}; a_i = theta_i + s_i; Picard while fewer than
        // three pairs are stored or if the system is singular
        for (int i = 0; i < k; ++i) c[i] = 0.0;
        c[k - 1] = 1.0;
        if (k >= 3) {
            const int n0 = H[k - 1], n1 = H[k - 2], n2 = H[k - 3];
            const int di[2] = {n1, n2};
            double Mm[2][2], rhs[2];
            const double b00 = ctl->B[n0 * kMaxHist + n0];
            for (int i = 0; i < 2; ++i) {
                rhs[i] = b00 - ctl->B[n0 * kMaxHist + di[i]];
                for (int j = 0; j < 2; ++j)
                    Mm[i][j] = b00 - ctl->B[n0 * kMaxHist + di[j]] - ctl->B[n0 * kMaxHist + di[i]] +
                               ctl->B[di[i] * kMaxHist + di[j]];
            }
            const double sc = fmax(Mm[0][0], Mm[1][1]);
            if (sc > 0.0) {
                for (int i = 0; i < 2; ++i) {
                    rhs[i] /= sc;
                    for (int j = 0; j < 2; ++j) Mm[i][j] /= sc;
                }
                // 2 x 2 Gaussian elimination with partial pivoting
                int p = fabs(Mm[1][0]) > fabs(Mm[0][0]) ? 1 : 0;
                if (fabs(Mm[p][0]) >= 1e-12) {
                    if (p == 1) {
                        double t0 = Mm[0][0], t1 = Mm[0][1], tr = rhs[0];
                        Mm[0][0] = Mm[1][0]; Mm[0][1] = Mm[1][1]; rhs[0] = rhs[1];
                        Mm[1][0] = t0; Mm[1][1] = t1; rhs[1] = tr;
                    }
                    const double fct = Mm[1][0] / Mm[0][0];
                    const double m11 = Mm[1][1] - fct * Mm[0][1];
                    const double r1 = rhs[1] - fct * rhs[0];
                    if (fabs(m11) >= 1e-12) {
                        const double th1 = r1 / m11;
                        const double th0 = (rhs[0] - Mm[0][1] * th1) / Mm[0][0];
                        const double a1 = th0 + ctl->s1, a2 = th1 + ctl->s2;
                        c[k - 1] = 1.0 - a1 - a2;
                        c[k - 2] = a1;
                        c[k - 3] = a2;
                    }
                }
            }
        }
    } else for (;;) {                 // MDIIS: bordered solve with drop-oldest retry
        const int n = k - first;
        if (n == 1) {
            c[0] = 1.0;
            break;
        }
        double A[kMaxHist + 1][kMaxHist + 2];
        double scale = 0.0;
        for (int i = 0; i < n; ++i) scale = fmax(scale, ctl->B[H[first + i] * kMaxHist + H[first + i]]);
        const double inv = scale > 0.0 ? 1.0 / scale : 1.0;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) A[i][j] = ctl->B[H[first + i] * kMaxHist + H[first + j]] * inv;
            A[i][n] = 1.0;
            A[i][n + 1] = 0.0;
        }
        for (int j = 0; j < n; ++j) A[n][j] = 1.0;
        A[n][n] = 0.0;
        A[n][n + 1] = 1.0;
        const int dim = n + 1;
        bool ok = true;
        for (int col = 0; col < dim && ok; ++col) {
            int p = col;
            double best = fabs(A[col][col]);
            for (int r = col + 1; r < dim; ++r)
                if (fabs(A[r][col]) > best) {
                    best = fabs(A[r][col]);
                    p = r;
                }
            if (best < 1e-12) {
                ok = false;
                break;
            }
            if (p != col)
                for (int j = col; j <= dim; ++j) {
                    const double tmp = A[col][j];
                    A[col][j] = A[p][j];
                    A[p][j] = tmp;
                }
            for (int r = col + 1; r < dim; ++r) {
                const double fct = A[r][col] / A[col][col];
                for (int j = col; j <= dim; ++j) A[r][j] -= fct * A[col][j];
            }
        }
        if (ok) {
            double xsol[kMaxHist + 1];
            for (int r = dim - 1; r >= 0; --r) {
                double s = A[r][dim];
                for (int j = r + 1; j < dim; ++j) s -= A[r][j] * xsol[j];
                xsol[r] = s / A[r][r];
            }
            for (int i = 0; i < n; ++i) c[i] = xsol[i];
            break;
        }
        ++first;
    }
    const int n = k - first;
    double eta = ctl->damp;
    if (ctl->dynamic) eta = fmin(fmax(-0.2 * log10(rms), 0.1), 1.0);
    ctl->eta = eta;
    ctl->upd_n = n;
    for (int i = 0; i < n; ++i) {
        ctl->upd_slot[i] = H[first + i];
        ctl->upd_coef[i] = c[i];
    }
    // slot for the next iterate: a free one while the history is short, else the oldest,
    // which then leaves the history
    int next;
    if (n < M) {
        int used = 0;
        for (int i = 0; i < n; ++i) used |= 1 << H[first + i];
        next = 0;
        while (used & (1 << next)) ++next;
        ctl->hist_n = n;
        for (int i = 0; i < n; ++i) ctl->hist_slot[i] = H[first + i];
    } else {
        next = H[first];
        ctl->hist_n = n - 1;
        for (int i = 1; i < n; ++i) ctl->hist_slot[i - 1] = H[first + i];
    }
    ctl->cur = next;
    ctl->do_update = 1;
}

// ------------------------------------------------------------------ potential (Eq. 22, 29)
// One thread per grid point and all sites; atoms staged through shared memory. For the
// FP32 form, far pairs are evaluated in FP32 (their Coulomb and phi terms accumulated in
// FP64) and near pairs (r < 1.5 max sigma_ag, where the r^-12 term is large enough for FP32
// coordinate rounding to show) entirely in FP64. Writes beta*u (capped at 1e4), phi and
// w = beta q phi - beta*u.
template <typename T>
__global__ void __launch_bounds__(256)
k_potential(Fields<T> f, const double *atoms, int n_atoms, const double *site_sig,
            const double *site_eps, const double *site_q, double beta, double ox, double oy,
            double oz, double dx, double dy, double dz) {
    constexpr int TILE = 64;
    constexpr bool kMixed = sizeof(T) == 4;
    __shared__ double ax[TILE], ay[TILE], az[TILE], aq[TILE], anear2[TILE];
    __shared__ double dsig2[TILE][kMaxSites], deps4[TILE][kMaxSites];
    __shared__ T sx[TILE], sy[TILE], sz[TILE], sq[TILE];
    __shared__ T ssig2[TILE][kMaxSites], seps4[TILE][kMaxSites];
    const int nv = f.nv;
    const long long G = f.G;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < G;
    const int NyNz = f.Ny * f.Nz;
    int ix = 0, iy = 0, iz = 0;
    if (active) {
        ix = (int)(p / NyNz);
        const int rem = (int)(p - (long long)ix * NyNz);
        iy = rem / f.Nz;
        iz = rem - iy * f.Nz;
    }
    // grid point relative to the origin
    const double pxd = ix * dx, pyd = iy * dy, pzd = iz * dz;
    const T px = (T)pxd, py = (T)pyd, pz = (T)pzd;
    T lj[kMaxSites];
    double ljd[kMaxSites];
#pragma unroll
    for (int g = 0; g < kMaxSites; ++g) {
        lj[g] = (T)0;
        ljd[g] = 0.0;
    }
    double coul = 0.0, phi = 0.0;
    for (int a0 = 0; a0 < n_atoms; a0 += TILE) {
        const int na = min(TILE, n_atoms - a0);
        __syncthreads();
        for (int i = threadIdx.x; i < na; i += blockDim.x) {
            const double *at = atoms + (long long)(a0 + i) * kAtomStride;
            ax[i] = at[0] - ox;
            ay[i] = at[1] - oy;
            az[i] = at[2] - oz;
            aq[i] = at[3];
            sx[i] = (T)ax[i];
            sy[i] = (T)ay[i];
            sz[i] = (T)az[i];
            sq[i] = (T)at[3];
            double smax = 0.0;
            for (int g = 0; g < nv; ++g) {
                const double s = 0.5 * (at[4] + site_sig[g]);
                smax = fmax(smax, s);
                dsig2[i][g] = s * s;
                deps4[i][g] = 4.0 * sqrt(at[5] * site_eps[g]);
                ssig2[i][g] = (T)dsig2[i][g];
                seps4[i][g] = (T)deps4[i][g];
            }
            anear2[i] = kMixed ? 2.25 * smax * smax : -1.0;
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < na; ++i) {
                const T ddx = px - sx[i], ddy = py - sy[i], ddz = pz - sz[i];
                const T r2f = ddx * ddx + ddy * ddy + ddz * ddz;
                if (kMixed && (double)r2f < anear2[i]) {
                    const double ex = pxd - ax[i], ey = pyd - ay[i], ez = pzd - az[i];
                    double r2 = ex * ex + ey * ey + ez * ez;
                    r2 = r2 < 1e-8 ? 1e-8 : r2;
                    const double r = sqrt(r2);
                    const double ir = 1.0 / r, ir2 = 1.0 / r2;
                    coul += aq[i] * ir;
                    phi += aq[i] * (-expm1(-r)) * ir;
#pragma unroll
                    for (int g = 0; g < kMaxSites; ++g) {
                        if (g < nv) {
                            const double s2 = dsig2[i][g] * ir2;
                            const double s6 = s2 * s2 * s2;
                            ljd[g] += deps4[i][g] * (s6 * s6 - s6);
                        }
                    }
                } else {
                    const T r2 = r2f < (T)1e-8 ? (T)1e-8 : r2f;
                    const T ir2 = (T)1 / r2;
                    const T r = sqrt(r2);
                    const T ir = (T)1 / r;
                    coul += (double)(sq[i] * ir);
                    phi += (double)(sq[i] * (T)(-expm1(-r)) * ir);
#pragma unroll
                    for (int g = 0; g < kMaxSites; ++g) {
                        if (g < nv) {
                            const T s2 = ssig2[i][g] * ir2;
                            const T s6 = s2 * s2 * s2;
                            lj[g] += seps4[i][g] * (s6 * s6 - s6);
                        }
                    }
                }
            }
        }
    }
    if (!active) return;
    const double C = 332.0637;
    const double phiv = C * phi;
    for (int g = 0; g < nv; ++g) {
        double v = beta * ((double)lj[g] + ljd[g] + C * site_q[g] * coul);
        v = v > 1e4 ? 1e4 : v;
        f.bu[(long long)g * G + p] = (T)v;
        f.w[(long long)g * G + p] = (T)(beta * site_q[g] * phiv - v);
    }
    f.phi[p] = (T)phiv;
}

// ------------------------------------------------------------------ long range (Eq. 30)
// Psi(k) = beta Phi~(k) / dV = amp0 / (k^2 (k^2 + 1)) sum_a q_a exp(-i k.(R_a - r0)),
// zero at k = 0 and on Nyquist planes. The phase is evaluated in FP64 as
// sincospi(2 (mx ux + my uy + mz uz)) with u = (R - r0) / L.
template <typename T>
__global__ void __launch_bounds__(256)
k_longrange(Fields<T> f, const double *atoms, int n_atoms, double amp0) {
    typedef typename Cx<T>::type C;
    const long long nmain = (long long)f.Nx * f.Ny * f.Kz;
    const long long total = nmain + (long long)f.Nx * f.Ny;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total) return;
    int ix, iy, iz;
    if (id < nmain) {
        ix = (int)(id / ((long long)f.Ny * f.Kz));
        const long long rem = id - (long long)ix * f.Ny * f.Kz;
        iy = (int)(rem / f.Kz);
        iz = (int)(rem - (long long)iy * f.Kz);
    } else {
        const long long r = id - nmain;
        ix = (int)(r / f.Ny);
        iy = (int)(r - (long long)ix * f.Ny);
        iz = f.Kz;
    }
    const int mx = signed_index(ix, f.Nx), my = signed_index(iy, f.Ny), mz = iz;
    const bool nyq = ((f.Nx % 2 == 0) && 2 * abs(mx) == f.Nx) ||
                     ((f.Ny % 2 == 0) && 2 * abs(my) == f.Ny) || (2 * mz == f.Nz);
    const double kx = f.ks[0] * mx, ky = f.ks[1] * my, kz = f.ks[2] * mz;
    const double k2 = kx * kx + ky * ky + kz * kz;
    double re = 0.0, im = 0.0;
    if (!nyq && k2 > 0.0) {
        for (int a = 0; a < n_atoms; ++a) {
            const double *at = atoms + (long long)a * kAtomStride;
            const double ph = 2.0 * (mx * at[6] + my * at[7] + mz * at[8]);
            double s, c;
            sincospi(ph, &s, &c);
            re += at[3] * c;
            im -= at[3] * s;
        }
        const double amp = amp0 / (k2 * (k2 + 1.0));
        re *= amp;
        im *= amp;
    }
    C v = cmk((T)re, (T)im);
    if (id < nmain)
        f.psi[id] = v;
    else
        f.psi_nyq[id - nmain] = v;
}

// ------------------------------------------------------------------ small helpers
// Step 1: t = f, i.e. tau = 0.
template <typename T>
__global__ void k_init_guess(Fields<T> f, int slot) {
    const long long n = (long long)f.nv * f.G;
    const long long base = (long long)slot * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        f.X[base + i] = (T)0;
}

// tau = t - beta q phi from a caller field t (FP64), into ring slot `slot`.
template <typename T>
__global__ void k_guess_from_t(Fields<T> f, int slot, const double *src) {
    const long long n = (long long)f.nv * f.G;
    const long long base = (long long)slot * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / f.G);
        const long long p = i - (long long)g * f.G;
        f.X[base + i] = (T)(src[i] - f.bq[g] * (double)f.phi[p]);
    }
}

template <typename T>
__global__ void k_get_field(Fields<T> f, int field, int slot, int kind, int order, double *dst) {
    const long long ring = (long long)f.nv * f.G;
    const long long n = field == 6 ? f.G : ring;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double v;
        if (field == 6) {
            v = (double)f.phi[i];
        } else if (field == 5) {
            v = (double)f.bu[i];
        } else if (field == 7) {
            v = (double)f.R[(long long)slot * ring + i];
        } else {
            const int g = (int)(i / f.G);
            const long long p = i - (long long)g * f.G;
            const T tau = f.X[(long long)slot * ring + i];
            const double fq = f.bq[g] * (double)f.phi[p];
            if (field == 4) {
                v = (double)tau + fq;
            } else {
                const T gv = closure_g(f.w[i] + tau, kind, order);
                if (field == 1) v = (double)gv;
                else if (field == 3) v = (double)(gv - (T)1);
                else v = (double)(gv - (T)1 - tau) - fq;      // c = h - t
            }
        }
        dst[i] = v;
    }
}

// Block-wide FP64 sum (result valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// SFE integrands (Eqs. 17-18, GF, PSE-n) accumulated in FP64, per site and block.
template <typename T>
__global__ void __launch_bounds__(256)
k_sfe(Fields<T> f, int slot, int kind, int order, int sfe_kind, int sfe_order, double *partials) {
    __shared__ double red[32];
    const int g = blockIdx.y;
    const long long ring = (long long)f.nv * f.G;
    const T *tt = f.X + (long long)slot * ring + (long long)g * f.G;
    const T *wp = f.w + (long long)g * f.G;
    const double bq = f.bq[g];
    double acc = 0.0;
    double fact = 1.0;
    for (int i = 2; i <= sfe_order + 1; ++i) fact *= i;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < f.G;
         p += (long long)gridDim.x * blockDim.x) {
        const T tau = tt[p];
        const T d = wp[p] + tau;
        const T gv = closure_g(d, kind, order);
        const double h = (double)(gv - (T)1);
        const double c = (double)(gv - (T)1 - tau) - bq * (double)f.phi[p];   // c = h - t
        double v = -c - 0.5 * h * c;
        if (sfe_kind == 2) v += 0.5 * h * h;                     // HNC, Eq. 17
        else if (sfe_kind == 1) v += h < 0.0 ? 0.5 * h * h : 0.0;  // KH, Eq. 18
        else if (sfe_kind == 4) {                                // PSE-n
            v += 0.5 * h * h;
            if ((double)d > 0.0) v -= pow((double)d, (double)(sfe_order + 1)) / fact;
        }
        acc += v;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(long long)g * gridDim.x + blockIdx.x] = s;
}

// ------------------------------------------------------------------ launchers
template <typename T> size_t plane_smem_bytes(const Fields<T> &f) {
    typedef typename Cx<T>::type C;
    return sizeof(C) * ((size_t)f.Ny * f.pitch + f.Kz + f.Ny + f.Kz + 1) +
           (kMaxHist + 1) * (kThreadsPlane / 32) * sizeof(double) + 16;
}
template <typename T> size_t pencil_smem_bytes(const Fields<T> &f) {
    typedef typename Cx<T>::type C;
    return sizeof(C) * ((size_t)f.nv * f.W * f.pencil_pitch + f.Nx);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T> cudaError_t prepare_kernels(const Fields<T> &f) {
    const size_t pl = plane_smem_bytes(f), pe = pencil_smem_bytes(f);
    cudaError_t e = set_smem(k_plane_fwd<T, 8>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_fwd<T, kMaxHist>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_inv<T, 8>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_inv<T, kMaxHist>, pl);
    if (e != cudaSuccess) return e;
    switch (f.nv) {
        case 1: return set_smem(k_pencil<T, 1>, pe);
        case 2: return set_smem(k_pencil<T, 2>, pe);
        case 3: return set_smem(k_pencil<T, 3>, pe);
        case 4: return set_smem(k_pencil<T, 4>, pe);
        case 5: return set_smem(k_pencil<T, 5>, pe);
        case 6: return set_smem(k_pencil<T, 6>, pe);
        case 7: return set_smem(k_pencil<T, 7>, pe);
        case 8: return set_smem(k_pencil<T, 8>, pe);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T> cudaError_t launch_plane_fwd(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = plane_smem_bytes(f);
    const dim3 grid(f.Nx, f.nv);
    if (f.M <= 8)
        k_plane_fwd<T, 8><<<grid, kThreadsPlane, sm, s>>>(f);
    else
        k_plane_fwd<T, kMaxHist><<<grid, kThreadsPlane, sm, s>>>(f);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_plane_inv(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = plane_smem_bytes(f);
    const dim3 grid(f.Nx, f.nv);
    if (f.M <= 8)
        k_plane_inv<T, 8><<<grid, kThreadsPlane, sm, s>>>(f);
    else
        k_plane_inv<T, kMaxHist><<<grid, kThreadsPlane, sm, s>>>(f);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_pencil(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = pencil_smem_bytes(f);
    const unsigned grid = f.tiles_main + f.tiles_nyq;
    switch (f.nv) {
        case 1: k_pencil<T, 1><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 2: k_pencil<T, 2><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 3: k_pencil<T, 3><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 4: k_pencil<T, 4><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 5: k_pencil<T, 5><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 6: k_pencil<T, 6><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 7: k_pencil<T, 7><<<grid, kThreadsPencil, sm, s>>>(f); break;
        case 8: k_pencil<T, 8><<<grid, kThreadsPencil, sm, s>>>(f); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_mdiis(const Fields<T> &f, cudaStream_t s) {
    k_mdiis<<<1, 32 * (kMaxHist + 1), 0, s>>>(f.ctrl, f.partials, f.nv * f.Nx);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_potential(const Fields<T> &f, const double *atoms, int n_atoms,
                             const double *site_sig, const double *site_eps, const double *site_q,
                             double beta, const double *origin, const double *spacing,
                             cudaStream_t s) {
    const long long blocks = (f.G + 255) / 256;
    k_potential<T><<<(unsigned)blocks, 256, 0, s>>>(f, atoms, n_atoms, site_sig, site_eps, site_q, beta,
                                                     origin[0], origin[1], origin[2], spacing[0],
                                                     spacing[1], spacing[2]);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_longrange(const Fields<T> &f, const double *atoms, int n_atoms, double amp0,
                             cudaStream_t s) {
    const long long total = (long long)f.Nx * f.Ny * (f.Kz + 1);
    k_longrange<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(f, atoms, n_atoms, amp0);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_init_guess(const Fields<T> &f, int slot, cudaStream_t s) {
    k_init_guess<T><<<152 * 8, 256, 0, s>>>(f, slot);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_guess_from_t(const Fields<T> &f, int slot, const double *src, cudaStream_t s) {
    k_guess_from_t<T><<<152 * 8, 256, 0, s>>>(f, slot, src);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_get_field(const Fields<T> &f, int field, int slot, int kind, int order,
                             double *dst, cudaStream_t s) {
    k_get_field<T><<<152 * 8, 256, 0, s>>>(f, field, slot, kind, order, dst);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_sfe(const Fields<T> &f, int slot, int kind, int order, int sfe_kind,
                       int sfe_order, double *partials, int blocks_per_site, cudaStream_t s) {
    k_sfe<T><<<dim3(blocks_per_site, f.nv), 256, 0, s>>>(f, slot, kind, order, sfe_kind, sfe_order,
                                                        partials);
    return cudaGetLastError();
}

#define RISM_INSTANTIATE(T)                                                                     \
    template size_t plane_smem_bytes<T>(const Fields<T> &);                                      \
    template cudaError_t prepare_kernels<T>(const Fields<T> &);                                  \
    template size_t pencil_smem_bytes<T>(const Fields<T> &);                                     \
    template cudaError_t launch_plane_fwd<T>(const Fields<T> &, cudaStream_t);                   \
    template cudaError_t launch_plane_inv<T>(const Fields<T> &, cudaStream_t);                   \
    template cudaError_t launch_pencil<T>(const Fields<T> &, cudaStream_t);                      \
    template cudaError_t launch_mdiis<T>(const Fields<T> &, cudaStream_t);                       \
    template cudaError_t launch_potential<T>(const Fields<T> &, const double *, int,            \
                                             const double *, const double *, const double *,    \
                                             double, const double *, const double *,            \
                                             cudaStream_t);                                     \
    template cudaError_t launch_longrange<T>(const Fields<T> &, const double *, int, double,    \
                                             cudaStream_t);                                     \
    template cudaError_t launch_init_guess<T>(const Fields<T> &, int, cudaStream_t);            \
    template cudaError_t launch_guess_from_t<T>(const Fields<T> &, int, const double *, cudaStream_t); \
    template cudaError_t launch_get_field<T>(const Fields<T> &, int, int, int, int, double *,   \
                                             cudaStream_t);                                     \
    template cudaError_t launch_sfe<T>(const Fields<T> &, int, int, int, int, int, double *,    \
                                       int, cudaStream_t);

RISM_INSTANTIATE(float)
RISM_INSTANTIATE(double)

}  // namespace rism
