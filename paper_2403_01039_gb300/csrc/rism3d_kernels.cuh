// CUDA kernels of the 3D-RISM solve (sm_103a). One iteration of the procedure of the
// "Numerical procedure" section (steps 2-6) is four launches:
//
//   plane_fwd  : [MDIIS update, Eq. 40] -> closure (Eqs. 14-16, PSE-n) -> c^sr (Eq. 31)
//                -> real-to-complex FFT along z and complex FFT along y of one x-plane
//   pencil     : FFT along x -> 3D-RISM contraction h~_g = sum_a c~_a X_ag(|k|) with
//                c~ = c~^sr - f~ (Eqs. 13, 32) -> inverse FFT along x
//   plane_inv  : inverse FFT along y and complex-to-real along z -> residual
//                R = h + 1 - g (Eq. 33) -> stored pair (Y = tau + eta R, R) -> Gram-row
//                partials <R, R_i> and sum R^2 (Dot2 in FP32, FP64 across threads)
//   mdiis      : reduce the partials, update the Gram matrix, solve the bordered MDIIS
//                system (Eq. 40), convergence test on the RMS residual (Eq. 41 read as RMS)
//
// Planes too large for shared memory take row chunks plus y-pencil passes (k_ypencil); the
// split option runs each plane pass as a streaming element kernel and a transform kernel
// on two graph branches. Every field stays in HBM between launches; the solver state lives
// in a device struct (Ctrl) so that one captured CUDA graph replays any number of
// iterations. The shared-memory transforms are compile-time radix-8 passes for power-of-two
// lengths 16-256 and mixed-radix (2, 3, 4, 5, 8) Stockham stages otherwise.
//
// The iterate is stored as tau = t - f (f = beta q phi of Eq. 29) and the potential as
// w = f - beta*u, so that d = -beta*u + t = w + tau and c^sr = g - 1 - t + f = g - 1 - tau
// (Eq. 31) without the large long-range parts of t and beta*u; since the MDIIS weights sum
// to one, iterating on tau is the same iteration as on t.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rism3d_internal.h"

// Resident blocks per SM the FP32 plane and pencil kernels are compiled for (register budget
// 65536 / (256 x this)); 3 (80 registers, a few hundred bytes of spills) measured faster
// than 2 (no spills): these kernels are latency-bound and need the resident warps.
#ifndef RISM_MINBLOCKS_F32
#define RISM_MINBLOCKS_F32 3
#endif

namespace rism {
namespace cg = cooperative_groups;

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
// Self-sorting (Stockham) mixed-radix transform of nb sequences of length L held in shared
// memory (element stride es, sequence stride bs). A stage loads every butterfly input into
// registers, synchronises, then writes, so the transform runs in place. For power-of-two
// lengths the index arithmetic uses shifts and masks.
struct StageIdx {
    int LR, Ns, step;
    bool pow2;
    int lgLR, lgNs;
    FastDiv dLR, dNs;
    __device__ __forceinline__ void split(int it, int &b, int &j, int &k, int &jq) const {
        if (pow2) {
            b = it >> lgLR;
            j = it & (LR - 1);
            k = j & (Ns - 1);
            jq = j >> lgNs;
        } else {
            b = fdiv(it, dLR);
            j = it - b * LR;
            jq = fdiv(j, dNs);
            k = j - jq * Ns;
        }
    }
};

__device__ __forceinline__ StageIdx make_stage(const FftPlan &p, int st, int Ns) {
    StageIdx s;
    const int L = p.L, R = p.radix[st];
    s.LR = L / R;
    s.Ns = Ns;
    s.step = L / (Ns * R);
    s.pow2 = ((L & (L - 1)) == 0) && ((R & (R - 1)) == 0);
    s.lgLR = __ffs(s.LR) - 1;
    s.lgNs = __ffs(Ns) - 1;
    s.dLR = p.dlr[st];
    s.dNs = p.dns[st];
    return s;
}

// One stage over `items` butterflies of nb sequences, shared by `nthr` threads with index
// `tid`; `bar` is the barrier of that group (block or warp).
template <typename C, int R, int MAXI, bool WARP>
__device__ __forceinline__ void fft_stage(C *buf, const StageIdx &si, int es, int nb, int bs,
                                          const C *tw, int sign, int tid, int nthr) {
    const int items = nb * si.LR;
    C v[MAXI][R];
#pragma unroll
    for (int m = 0; m < MAXI; ++m) {
        const int it = tid + m * nthr;
        if (it < items) {
            int b, j, k, jq;
            si.split(it, b, j, k, jq);
            const C *src = buf + (long)b * bs;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C a = src[(j + r * si.LR) * es];
                if (r > 0) {
                    C w = tw[k * r * si.step];
                    if (sign > 0) w.y = -w.y;
                    a = cmul(a, w);
                }
                v[m][r] = a;
            }
        }
    }
    if (WARP) __syncwarp(); else __syncthreads();
#pragma unroll
    for (int m = 0; m < MAXI; ++m) {
        const int it = tid + m * nthr;
        if (it < items) {
            int b, j, k, jq;
            si.split(it, b, j, k, jq);
            Dft<R>::run(v[m], sign);
            const int d0 = jq * si.Ns * R + k;
            C *dst = buf + (long)b * bs;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[(d0 + r * si.Ns) * es] = v[m][r];
        }
    }
    if (WARP) __syncwarp(); else __syncthreads();
}

template <typename C, int MAXC, bool WARP>
__device__ __forceinline__ void fft_stages_inl(C *base, const FftPlan &p, int es, int nbc, int bs,
                                           const C *tw, int sign, int tid, int nthr) {
    int Ns = 1;
    for (int st = 0; st < p.nst; ++st) {
        const int R = p.radix[st];
        const StageIdx si = make_stage(p, st, Ns);
        switch (R) {
            case 8: fft_stage<C, 8, MAXC / 8, WARP>(base, si, es, nbc, bs, tw, sign, tid, nthr); break;
            case 4: fft_stage<C, 4, MAXC / 4, WARP>(base, si, es, nbc, bs, tw, sign, tid, nthr); break;
            case 2: fft_stage<C, 2, MAXC / 2, WARP>(base, si, es, nbc, bs, tw, sign, tid, nthr); break;
            case 3: fft_stage<C, 3, MAXC / 3, WARP>(base, si, es, nbc, bs, tw, sign, tid, nthr); break;
            case 5: fft_stage<C, 5, MAXC / 5, WARP>(base, si, es, nbc, bs, tw, sign, tid, nthr); break;
            default: break;
        }
        Ns *= R;
    }
}

// Power-of-two lengths 16..256 take a transform whose passes are fixed at compile time:
// radix 8 passes, then one pass of the remaining radix (2, 4 or 8). T = L/8 threads share a
// sequence (all within one warp, so passes are separated by warp barriers) and each holds 8
// values per pass; the first pass needs no twiddles. Its outputs are written stride-8
// apart, which would put several lanes on one shared-memory bank, so the hand-off between
// the first and second pass uses the permuted position i ^ ((i >> 3) & 7) (a bijection of
// 0..L-1 that only permutes within groups of 8); every other layout is the natural one.
__host__ __device__ constexpr int p2_pow8(int p) { return p == 0 ? 1 : 8 * p2_pow8(p - 1); }
__host__ __device__ constexpr int p2_npass(int L) { return L <= 8 ? 1 : 1 + p2_npass(L / 8); }
__host__ __device__ constexpr int p2_radix(int L, int p) {
    return p + 1 < p2_npass(L) ? 8 : L / p2_pow8(p);
}
__device__ __forceinline__ int p2_swz(int i) { return i ^ ((i >> 3) & 7); }

template <typename C, int L, int P>
__device__ __forceinline__ void p2_pass(C *seq, int es, int u, const C *tw, int sign, bool act) {
    constexpr int NP = p2_npass(L);
    constexpr int R = p2_radix(L, P);
    constexpr int NS = p2_pow8(P);
    constexpr int T = L / 8, LR = L / R, NB = 8 / R;
    constexpr bool SWZ_IN = P == 1;
    constexpr bool SWZ_OUT = P == 0 && NP > 1;
    C v[8];
    if (act) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int j = u + q * T;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int li = j + r * LR;
                C a = seq[(SWZ_IN ? p2_swz(li) : li) * es];
                if (NS > 1 && r > 0) {
                    C w = tw[(j & (NS - 1)) * r * (L / (NS * R))];
                    if (sign > 0) w.y = -w.y;
                    a = cmul(a, w);
                }
                v[q * R + r] = a;
            }
        }
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int j = u + q * T;
            Dft<R>::run(&v[q * R], sign);
            const int d0 = (j / NS) * (NS * R) + (j & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int li = d0 + r * NS;
                seq[(SWZ_OUT ? p2_swz(li) : li) * es] = v[q * R + r];
            }
        }
    }
    __syncwarp();
}

template <typename C, int L>
__device__ __forceinline__ void p2_seq(C *seq, int es, int u, const C *tw, int sign, bool act) {
    p2_pass<C, L, 0>(seq, es, u, tw, sign, act);
    if constexpr (p2_npass(L) > 1) p2_pass<C, L, 1>(seq, es, u, tw, sign, act);
    if constexpr (p2_npass(L) > 2) p2_pass<C, L, 2>(seq, es, u, tw, sign, act);
}

// nb sequences of length L (element stride es, sequence stride bs); ends with a block
// barrier like fft_smem.
template <typename C, int L>
__device__ void fft_p2(C *buf, int es, int nb, int bs, const C *tw, int sign) {
    static_assert(L >= 16 && L <= 256, "warp-resident power-of-two lengths only");
    constexpr int T = L / 8, SPW = 32 / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int u = lane & (T - 1), sl = lane / T;
    for (int g0 = warp * SPW; g0 < nb; g0 += nw * SPW) {
        const int b = g0 + sl;
        p2_seq<C, L>(buf + (long)(b < nb ? b : 0) * bs, es, u, tw, sign, b < nb);
    }
    __syncthreads();
}

// Transform the nb sequences. When the plan allows (seq_per_warp > 0), each warp takes its
// own groups of seq_per_warp sequences and separates stages with warp barriers only;
// otherwise the whole block takes chunks of `chunk` sequences with block barriers.
// GENERIC = false compiles only the power-of-two lengths 16..256 (the caller guarantees
// one), which keeps the mixed-radix stages and their registers out of the kernel.
template <typename C, int MAXC, bool GENERIC = true>
__device__ void fft_smem(C *buf, const FftPlan &p, int es, int nb, int bs, int chunk, const C *tw,
                         int sign) {
    switch (p.L) {
        case 16: fft_p2<C, 16>(buf, es, nb, bs, tw, sign); return;
        case 32: fft_p2<C, 32>(buf, es, nb, bs, tw, sign); return;
        case 64: fft_p2<C, 64>(buf, es, nb, bs, tw, sign); return;
        case 128: fft_p2<C, 128>(buf, es, nb, bs, tw, sign); return;
        case 256: fft_p2<C, 256>(buf, es, nb, bs, tw, sign); return;
        default: break;
    }
    if constexpr (!GENERIC) return;
    if (p.seq_per_warp > 0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int S = p.seq_per_warp;
        for (int g0 = warp * S; g0 < nb; g0 += nw * S)
            fft_stages_inl<C, MAXC, true>(buf + (long)g0 * bs, p, es, min(S, nb - g0), bs, tw, sign, lane, 32);
        __syncthreads();
        return;
    }
    for (int b0 = 0; b0 < nb; b0 += chunk)
        fft_stages_inl<C, MAXC, false>(buf + (long)b0 * bs, p, es, min(chunk, nb - b0), bs, tw, sign,
                                       threadIdx.x, blockDim.x);
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

// Sum of many terms in the working precision carried to about FP64 accuracy: FP32 keeps the
// TwoSum error of every addition in a second word; FP64 adds directly.
template <typename T> struct SumAcc;
template <> struct SumAcc<float> {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float sm, e;
        two_sum(hi, x, sm, e);
        hi = sm;
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <> struct SumAcc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

// Read-only-path load of two consecutive reals. Used for fields that no other thread writes
// during the pass (each element is read, and possibly rewritten, by one thread only).
__device__ __forceinline__ float2 ld2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ double2 ld2(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }

// ------------------------------------------------------------------ row helpers
// z transform of nr <= 256 / L rows (row stride bs) by one warp with the power-of-two
// transform of length L (L/8 lanes per row).
template <typename C, int L>
__device__ __forceinline__ void fft_rows_warp(C *rows, int nr, int bs, const C *tw, int sign, int lane) {
    constexpr int T = L / 8;
    constexpr int LG = L == 16 ? 1 : (L == 32 ? 2 : (L == 64 ? 3 : (L == 128 ? 4 : 5)));
    const int sl = lane >> LG;
    p2_seq<C, L>(rows + (long)min(sl, nr - 1) * bs, 1, lane & (T - 1), tw, sign, sl < nr);
}

// Real-to-complex post-processing of nr rows after the half-length complex transform:
// X[k] = E[k] + w^k O[k] for k = 0..Kz. X[0] and X[Kz] are real; packed = true stores them
// as one complex value X[0] + i X[Kz] in row[0] (the y transform then takes both real
// columns as one complex column), else row[0] = X[0] and row[Kz] = X[Kz].
template <typename C>
__device__ __forceinline__ void r2c_rows(C *rows, int nr, int Kz, int pitch, const C *tw_z, const FastDiv &dh1,
                                         int tid, int nthr, bool packed) {
    typedef decltype(rows[0].x) R;
    const int half = Kz / 2;
    for (int idx = tid; idx < nr * (half + 1); idx += nthr) {
        const int y = fdiv(idx, dh1), k = idx - y * (half + 1);
        C *row = rows + y * pitch;
        if (k == 0) {
            C z = row[0];
            if (packed) {
                row[0] = cmk(z.x + z.y, z.x - z.y);
            } else {
                row[0] = cmk(z.x + z.y, (R)0);
                row[Kz] = cmk(z.x - z.y, (R)0);
            }
        } else {
            const int k2 = Kz - k;
            C a = row[k], b = row[k2];
            C e1 = cscale(cadd(a, cconj(b)), (R)0.5);
            C o1 = cscale(csub(a, cconj(b)), (R)0.5);
            C X1 = cadd(e1, cmul(cmuli(o1, -1), tw_z[k]));
            if (k2 != k) {
                C e2 = cscale(cadd(b, cconj(a)), (R)0.5);
                C o2 = cscale(csub(b, cconj(a)), (R)0.5);
                row[k2] = cadd(e2, cmul(cmuli(o2, -1), tw_z[k2]));
            }
            row[k] = X1;
        }
    }
}

// Complex-to-real pre-processing of nr rows before the inverse half-length transform:
// Z[k] = (X[k] + conj X[Kz-k]) + i w^-k (X[k] - conj X[Kz-k]). packed = true: row[0] holds
// X[0] + i X[Kz] (both real), as r2c_rows writes it.
template <typename C>
__device__ __forceinline__ void c2r_rows(C *rows, int nr, int Kz, int pitch, const C *tw_z, const FastDiv &dh1,
                                         int tid, int nthr, bool packed) {
    typedef decltype(rows[0].x) R;
    const int half = Kz / 2;
    for (int idx = tid; idx < nr * (half + 1); idx += nthr) {
        const int y = fdiv(idx, dh1), k = idx - y * (half + 1);
        C *row = rows + y * pitch;
        const int k2 = Kz - k;
        C a = row[k], b = row[k2];
        if (packed && k == 0) {
            b = cmk(a.y, (R)0);
            a = cmk(a.x, (R)0);
        }
        C Z1 = cadd(cadd(a, cconj(b)), cmuli(cmul(csub(a, cconj(b)), cconj(tw_z[k])), +1));
        if (k != 0 && k2 != k)
            row[k2] = cadd(cadd(b, cconj(a)), cmuli(cmul(csub(b, cconj(a)), cconj(tw_z[k2])), +1));
        row[k] = Z1;
    }
}

// Half-integer grid, real-to-complex step of nr rows: with Z the half-length transform of
// the pre-twiddled packed row, X(m + 1/2) = E(m) + exp(-i pi (2m + 1) / Nz) O(m),
// E(m) = (Z(m) + conj Z(M-1-m)) / 2, O(m) = -i (Z(m) - conj Z(M-1-m)) / 2 (M = Kz values, no
// real or Nyquist terms); the result is multiplied by the row's y and x shift factors ph.
template <typename C>
__device__ __forceinline__ void r2c_rows_half(C *rows, int nr, int yg, int Kz, int pitch, const C *tw_q,
                                              const C *tw_ys, C phx, const FastDiv &dp, int tid, int nthr) {
    typedef decltype(rows[0].x) R;
    const int np = (Kz + 1) / 2;
    for (int idx = tid; idx < nr * np; idx += nthr) {
        const int y = fdiv(idx, dp), m = idx - y * np, m2 = Kz - 1 - m;
        C *row = rows + y * pitch;
        const C ph = cmul(tw_ys[yg + y], phx);
        const C a = row[m], b = row[m2];
        const C X1 = cadd(cscale(cadd(a, cconj(b)), (R)0.5), cmul(tw_q[m], cscale(cmuli(csub(a, cconj(b)), -1), (R)0.5)));
        if (m2 != m)
            row[m2] = cmul(cadd(cscale(cadd(b, cconj(a)), (R)0.5),
                                cmul(tw_q[m2], cscale(cmuli(csub(b, cconj(a)), -1), (R)0.5))), ph);
        row[m] = cmul(X1, ph);
    }
}

// Half-integer grid, complex-to-real step of nr rows (inverse of r2c_rows_half, up to the
// factor Nz of the unnormalised transforms): the row is first multiplied by conj(ph), then
// Z(m) = (X(m) + conj X(M-1-m)) + i conj(exp(-i pi (2m + 1) / Nz)) (X(m) - conj X(M-1-m)).
template <typename C>
__device__ __forceinline__ void c2r_rows_half(C *rows, int nr, int yg, int Kz, int pitch, const C *tw_q,
                                              const C *tw_ys, C phx, const FastDiv &dp, int tid, int nthr) {
    const int np = (Kz + 1) / 2;
    for (int idx = tid; idx < nr * np; idx += nthr) {
        const int y = fdiv(idx, dp), m = idx - y * np, m2 = Kz - 1 - m;
        C *row = rows + y * pitch;
        const C ph = cconj(cmul(tw_ys[yg + y], phx));
        const C a = cmul(row[m], ph), b = cmul(row[m2], ph);
        const C Z1 = cadd(cadd(a, cconj(b)), cmuli(cmul(csub(a, cconj(b)), cconj(tw_q[m])), +1));
        if (m2 != m)
            row[m2] = cadd(cadd(b, cconj(a)), cmuli(cmul(csub(b, cconj(a)), cconj(tw_q[m2])), +1));
        row[m] = Z1;
    }
}

// Asynchronous 8-byte global -> shared copy (no register staging: every copy of a loop is
// in flight at once); cp_async_wait() waits for the calling thread's copies.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------------------ y transform across a cluster
// When a y-z plane exceeds one block's shared memory, its R = Ny / S row chunks of S rows go
// to the R blocks of a thread-block cluster (block rank r holds rows r S .. r S + S - 1) and
// the length-Ny y transform is split as Ny = R x S (decimation in frequency): with
// y = n + S j and k = R k' + r,
//   X[R k' + r] = sum_n exp(-2 pi i n k' / S) [exp(-2 pi i n r / Ny) sum_j x_j[n] W_R^{j r}],
// so a radix-R step across the cluster (distributed shared memory) followed by a local
// length-S transform leaves X[R k' + r] in row k' of block r; the inverse runs the local
// transform first and the cross-block step last. Each row position (n, column) is owned by
// one block, which reads the R values from the R blocks and writes the R results back, so
// no position is read after another block has written it; a cluster barrier before and
// after orders the step against the local work.
template <typename C, int R>
__device__ __forceinline__ void cluster_radix(C *buf, int S, int K1, int pitch, const FastDiv &dK1,
                                              const C *tw_y, int sign) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int P = S * K1;
    const int p0 = (int)((long long)P * rank / R), p1 = (int)((long long)P * (rank + 1) / R);
    C *rb[R];
#pragma unroll
    for (int j = 0; j < R; ++j) rb[j] = cl.map_shared_rank(buf, j);
    cl.sync();
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int n = fdiv(p, dK1), col = p - n * K1;
        const int off = n * pitch + col;
        C v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = rb[j][off];
        if (sign > 0) {                      // inverse: B_r[n] exp(+2 pi i n r / Ny), then the DFT
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], cconj(tw_y[n * r]));
        }
        Dft<R>::run(v, sign);
        if (sign < 0) {                      // forward: the DFT, then exp(-2 pi i n r / Ny)
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_y[n * r]);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) rb[j][off] = v[j];
    }
    cl.sync();
}

template <typename C>
__device__ __forceinline__ void cluster_y_step(C *buf, int R, int S, int K1, int pitch, const FastDiv &dK1,
                                               const C *tw_y, int sign) {
    switch (R) {
        case 2: cluster_radix<C, 2>(buf, S, K1, pitch, dK1, tw_y, sign); break;
        case 4: cluster_radix<C, 4>(buf, S, K1, pitch, dK1, tw_y, sign); break;
        default: cluster_radix<C, 8>(buf, S, K1, pitch, dK1, tw_y, sign); break;
    }
}

// ------------------------------------------------------------------ pass 1: plane_fwd
// Per-launch values of the update and closure, shared by the element loops.
template <typename T, int MAXH>
struct FwdArgs {
    const T *coef;               // [MAXH] update coefficients of Y_i (shared memory)
    const T *dcoef;              // [MAXH] coefficients of R_i (dynamic damping only)
    const long long *slot_off;   // [MAXH] ring offsets of the combined pairs (shared memory)
    int upd_n, upd_r, do_update, kind, order, anchor, refresh;
    T *tcur, *ga;                // this block's part of the iterate offset delta and of g_a
    T *wp;                       // this block's part of w = f - beta u + tau0 (d = w + delta)
    T *t0;                       // this block's part of tau0 (written on refresh)
    const typename Cx<T>::type *pre;   // half grid: exp(-i pi p / Kz) per packed element, else null
};

// Update (Eq. 40) + closure + c^sr (Eq. 31) of the elements e in [e0, e1) of the block's
// rows (e = row * Kz + m; complex element m packs the reals 2m, 2m + 1), written into the
// row buffer. tid / nthr split them, two elements per thread and step with every load
// issued before any store.
//
// The iterate is tau = tau0 + delta: the stored history Y_i and the current field hold
// delta, w holds f - beta u + tau0 and the anchor holds g_a, the closure's g at the anchor
// point. With c^sr = g - 1 - tau (Eq. 31) the transform input c^sr - c^sr_a is then
// (g - g_a) - delta, which stays exact where the solute core makes g = g_a = 0 and |tau| is
// in the hundreds: no rounding at the size of tau enters the iteration. A refresh moves the
// offset to the current iterate (tau0 += delta, w += delta, Y_i -= delta, delta = 0) and
// stores g_a = g.
// Refresh of one packed pair at offset o: the offset moves to the current iterate.
template <typename T, int MAXH>
__device__ __forceinline__ void fwd_refresh(const Fields<T> &f, const FwdArgs<T, MAXH> &A, long long o,
                                            typename Vec2<T>::type t, typename Vec2<T>::type dv,
                                            typename Vec2<T>::type g) {
    typedef typename Vec2<T>::type V2;
    V2 t0 = ld2(A.t0 + o);
    t0.x += t.x;
    t0.y += t.y;
    *reinterpret_cast<V2 *>(A.t0 + o) = t0;
    *reinterpret_cast<V2 *>(A.wp + o) = dv;       // w + delta: the new anchor point's d
    *reinterpret_cast<V2 *>(A.ga + o) = g;
    V2 z;
    z.x = z.y = (T)0;
    *reinterpret_cast<V2 *>(A.tcur + o) = z;
    if (A.do_update)
        for (int i = 0; i < A.upd_n; ++i) {       // the stored pairs in the new coordinates
            T *yb = f.X + A.slot_off[i];
            V2 y = ld2(yb + o);
            y.x -= t.x;
            y.y -= t.y;
            *reinterpret_cast<V2 *>(yb + o) = y;
        }
}

template <typename T, int MAXH>
__device__ __forceinline__ void fwd_elements(const Fields<T> &f, const FwdArgs<T, MAXH> &A,
                                             typename Cx<T>::type *buf, int y0, int e0, int e1, int tid,
                                             int nthr) {
    typedef typename Cx<T>::type C;
    typedef typename Vec2<T>::type V2;
    const int Kz = f.Kz, pitch = f.pitch;
    for (int i0 = e0 + tid; i0 < e1; i0 += 2 * nthr) {
        const int i1 = i0 + nthr;
        const bool has1 = i1 < e1;
        const int yA = fdiv(i0, f.dKz), mA = i0 - yA * Kz;
        const int yB = has1 ? fdiv(i1, f.dKz) : yA, mB = has1 ? i1 - yB * Kz : mA;
        const long long oA = (long long)(y0 + yA) * f.Nz + 2 * mA;
        const long long oB = (long long)(y0 + yB) * f.Nz + 2 * mB;
        V2 tA, tB;
        if (A.do_update) {
            // t = sum_i c_i Y_i (+ sum_i d_i R_i when the damping changed since Y_i was
            // stored), Y_i = t_i + eta_i R_i: one stored field per pair
            tA.x = tA.y = tB.x = tB.y = (T)0;
#pragma unroll
            for (int i = 0; i < MAXH; ++i) {
                if (i < A.upd_n) {
                    const T *yb = f.X + A.slot_off[i];
                    const V2 ya = ld2(yb + oA), yv = ld2(yb + oB);
                    const T c = A.coef[i];
                    tA.x += c * ya.x;
                    tA.y += c * ya.y;
                    tB.x += c * yv.x;
                    tB.y += c * yv.y;
                }
            }
            if (A.upd_r) {
                for (int i = 0; i < A.upd_n; ++i) {
                    const T *rb = f.R + A.slot_off[i];
                    const V2 ra = ld2(rb + oA), rv = ld2(rb + oB);
                    const T d = A.dcoef[i];
                    tA.x += d * ra.x;
                    tA.y += d * ra.y;
                    tB.x += d * rv.x;
                    tB.y += d * rv.y;
                }
            }
        } else {
            tA = ld2(A.tcur + oA);
            tB = ld2(A.tcur + oB);
        }
        const V2 wA = ld2(A.wp + oA), wB = ld2(A.wp + oB);
        V2 aA, aB;
        if (A.anchor) {
            aA = ld2(A.ga + oA);
            aB = ld2(A.ga + oB);
        } else {
            aA.x = aA.y = aB.x = aB.y = (T)1;   // no anchor: c^sr = (g - 1) - tau
        }
        V2 dvA, dvB, gA, gB;
        dvA.x = wA.x + tA.x;
        dvA.y = wA.y + tA.y;
        dvB.x = wB.x + tB.x;
        dvB.y = wB.y + tB.y;
        gA.x = closure_g(dvA.x, A.kind, A.order);
        gA.y = closure_g(dvA.y, A.kind, A.order);
        gB.x = closure_g(dvB.x, A.kind, A.order);
        gB.y = closure_g(dvB.y, A.kind, A.order);
        C dA = cmk((gA.x - aA.x) - tA.x, (gA.y - aA.y) - tA.y);
        C dB = cmk((gB.x - aB.x) - tB.x, (gB.y - aB.y) - tB.y);
        if (A.pre) {                           // half grid: z shift of the packed element
            dA = cmul(dA, A.pre[mA]);
            dB = cmul(dB, A.pre[mB]);
        }
        if (A.refresh) {
            fwd_refresh<T, MAXH>(f, A, oA, tA, dvA, gA);
            if (has1) fwd_refresh<T, MAXH>(f, A, oB, tB, dvB, gB);
        } else if (A.do_update) {
            *reinterpret_cast<V2 *>(A.tcur + oA) = tA;
            if (has1) *reinterpret_cast<V2 *>(A.tcur + oB) = tB;
        }
        buf[yA * pitch + mA] = dA;
        if (has1) buf[yB * pitch + mB] = dB;
    }
}

// One block per (x plane or row chunk of one, site). MAXH bounds the stored MDIIS pairs the
// update combines (5, 8 or 16), so the loop over them unrolls. LZ = Nz / 2 when the kernel is
// specialised for that power-of-two length (64 or 128): each warp then takes its own
// 256 / LZ rows at a time through update, closure, z transform and real-to-complex step
// with warp barriers only, so that its loads overlap other warps' arithmetic. LZ = 0 is the
// block-wide form for any length. The y transform needs the whole plane in both.
template <typename T, int MAXH, int LZ>
__global__ void __launch_bounds__(kThreadsPlane, sizeof(T) == 4 ? RISM_MINBLOCKS_F32 : 2)
k_plane_fwd(Fields<T> f) {
    typedef typename Cx<T>::type C;
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = f.Kz, pitch = f.pitch;
    C *tw_h = buf + (long)f.slab_rows * pitch;    // after the block's rows
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    C *tw_q = tw_z + (Kz + 1);
    C *tw_s = reinterpret_cast<C *>(reinterpret_cast<double *>(tw_q + Kz) + (kMaxHist + 1) * (kThreadsPlane / 32));
    const bool half = f.half;
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];
    if (half)
        for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_q[i] = f.tw_q[i];
    if (f.cl > 1)              // length-S twiddles of the local y transform: W_Ny^(R m)
        for (int i = threadIdx.x; i < f.slab_rows; i += blockDim.x) tw_s[i] = f.tw_y[i * f.cl];

    // block = (x plane, row chunk yc, site): rows y0 .. y0 + nyb of plane x
    const int nyc = f.nyc;
    const int x = blockIdx.x / nyc, yc = blockIdx.x - (blockIdx.x / nyc) * nyc, gam = blockIdx.y;
    const int y0 = yc * f.slab_rows, nyb = min(f.slab_rows, Ny - y0);
    const int stage = ctl->stage;
    const long long ring = (long long)f.nv * f.G;
    const long long siteoff = (long long)gam * f.G + (long long)x * Ny * f.Nz;
    __shared__ T coef[MAXH], dcoef[MAXH];
    __shared__ long long slot_off[MAXH];
    FwdArgs<T, MAXH> A;
    A.upd_n = ctl->upd_n;
    if (threadIdx.x < MAXH) {
        const int i = threadIdx.x;
        coef[i] = i < A.upd_n ? (T)ctl->upd_coef[i] : (T)0;
        dcoef[i] = i < A.upd_n ? (T)ctl->upd_dcoef[i] : (T)0;
        slot_off[i] = i < A.upd_n ? (long long)ctl->upd_slot[i] * ring + siteoff : 0;
    }
    A.coef = coef;
    A.dcoef = dcoef;
    A.slot_off = slot_off;
    A.upd_r = ctl->upd_r;
    A.do_update = ctl->do_update;
    A.kind = ctl->stage_kind[stage];
    A.order = ctl->stage_order[stage];
    A.anchor = ctl->anchor_valid;
    A.refresh = ctl->refresh;
    A.tcur = f.Tc + (long long)gam * f.G + (long long)x * Ny * f.Nz;
    A.ga = f.g_a + siteoff;
    A.wp = f.w + siteoff;
    A.t0 = f.tau0 + siteoff;
    A.pre = half ? tw_z : nullptr;
    const C phx = half ? f.tw_xs[x] : cmk((T)1, (T)0);
    __syncthreads();

    if constexpr (LZ > 0) {
        constexpr int RW = 256 / LZ;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r0 = warp * RW; r0 < nyb; r0 += nw * RW) {
            const int nr = min(RW, nyb - r0);
            fwd_elements<T, MAXH>(f, A, buf, y0, r0 * LZ, (r0 + nr) * LZ, lane, 32);
            __syncwarp();
            fft_rows_warp<C, LZ>(buf + (long)r0 * pitch, nr, pitch, tw_h, -1, lane);
            if (half)
                r2c_rows_half(buf + (long)r0 * pitch, nr, y0 + r0, LZ, pitch, tw_q, f.tw_ys, phx, f.dKzp, lane, 32);
            else
                r2c_rows(buf + (long)r0 * pitch, nr, LZ, pitch, tw_z, f.dKz1h, lane, 32, nyc == 1);
            __syncwarp();
        }
        __syncthreads();
    } else {
        fwd_elements<T, MAXH>(f, A, buf, y0, 0, nyb * Kz, threadIdx.x, blockDim.x);
        __syncthreads();
        fft_smem<C, MaxC<T>::v>(buf, f.ph, 1, nyb, pitch, f.chunk_rows, tw_h, -1);
        if (half)
            r2c_rows_half(buf, nyb, y0, Kz, pitch, tw_q, f.tw_ys, phx, f.dKzp, threadIdx.x, blockDim.x);
        else
            r2c_rows(buf, nyb, Kz, pitch, tw_z, f.dKz1h, threadIdx.x, blockDim.x, nyc == 1);
        __syncthreads();
    }
    // columns: complex FFT of length Ny for kz = 0..Kz (whole planes only; a split plane
    // leaves the y transform to the y-pencil pass). The real columns kz = 0 and Kz travel
    // as one complex column P = A + iB and are separated afterwards with the Hermitian
    // symmetry of a real sequence's transform: A[k] = (P[k] + conj P[-k]) / 2,
    // B[k] = -i (P[k] - conj P[-k]) / 2.
    if (nyc == 1 && half) {
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, -1);
    } else if (nyc == 1) {
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, -1);
        for (int k = threadIdx.x; k <= Ny / 2; k += blockDim.x) {
            const int k2 = k == 0 ? 0 : Ny - k;
            const C P = buf[k * pitch], Q = buf[k2 * pitch];
            buf[k * pitch] = cscale(cadd(P, cconj(Q)), (T)0.5);
            buf[k * pitch + Kz] = cscale(cmuli(csub(P, cconj(Q)), -1), (T)0.5);
            if (k2 != k) {
                buf[k2 * pitch] = cscale(cadd(Q, cconj(P)), (T)0.5);
                buf[k2 * pitch + Kz] = cscale(cmuli(csub(Q, cconj(P)), -1), (T)0.5);
            }
        }
        __syncthreads();
    } else if (f.cl > 1) {
        // the y transform across the cluster (all Kz + 1 columns, unpacked): the cross-block
        // radix step, then the local length-S transform; row y then holds ky = R y + yc
        cluster_y_step<C>(buf, f.cl, nyb, Kz + 1, pitch, f.dK1, tw_y, -1);
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.pys, pitch, Kz + 1, 1, f.chunk_ys, tw_s, -1);
        C *dst = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;
        for (int idx = threadIdx.x; idx < nyb * Kz; idx += blockDim.x) {
            const int y = fdiv(idx, f.dKz), k = idx - y * Kz;
            dst[(long long)(f.cl * y + yc) * Kz + k] = buf[y * pitch + k];
        }
        C *dn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
        for (int y = threadIdx.x; y < nyb; y += blockDim.x) dn[f.cl * y + yc] = buf[y * pitch + Kz];
        return;
    }
    C *dst = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz + (long long)y0 * Kz;
    for (int idx = threadIdx.x; idx < nyb * Kz; idx += blockDim.x) {
        const int y = fdiv(idx, f.dKz), k = idx - y * Kz;
        dst[idx] = buf[y * pitch + k];
    }
    if (!half) {
        C *dn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny + y0;
        for (int y = threadIdx.x; y < nyb; y += blockDim.x) dn[y] = buf[y * pitch + Kz];
    }
}

// ------------------------------------------------------------------ pass 2: pencil
__device__ __forceinline__ int signed_index(int i, int N) { return (2 * i < N) ? i : i - N; }

// One block per tile of W spectrum columns (all x, all NV sites). NV is a template argument
// so the contraction unrolls over exactly the solvent sites; P2 compiles only the
// power-of-two x transforms (Nx = 16..256).
template <typename T, int NV, bool P2>
__global__ void __launch_bounds__(kThreadsPencil, sizeof(T) == 4 ? RISM_MINBLOCKS_F32 : 2)
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
    // element loops run over whole tiles (W columns) and skip the columns past a ragged
    // tile's end, so that the index split is a multiply by constants
    const int nload = NV * Nx * W;
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int rest = fdiv(idx, f.dW), c = idx - rest * W;
        const int a = fdiv(rest, f.dNx), xx = rest - a * Nx;
        if (c < ncol) {
            const C *g = &src_base[a * site_stride + xx * xstride + col_base + c];
            if (sizeof(T) == 4) cp_async8(&buf[(a * W + c) * pp + xx], g);   // in flight together
            else buf[(a * W + c) * pp + xx] = *g;
        }
    }
    if (sizeof(T) == 4) cp_async_wait();
    __syncthreads();
    fft_smem<C, MaxC<T>::v, !P2>(buf, f.px, 1, NV * W, pp, f.chunk_x, tw_x, -1);
    // contraction (Eq. 13 with Eq. 32): E_g = sum_a D_a A_ag(|k|) [+ Psi A_{nv,g} before the
    // first anchor, after which f~ is part of h_a]
    const C *psi = nyq ? f.psi_nyq : f.psi;
    const bool psi_on = f.ctrl->anchor_valid == 0;
    const int npts = Nx * W;
    constexpr int rowlen = (NV + 1) * NV;
    const T ks0 = (T)f.ks[0], ks1 = (T)f.ks[1], ks2 = (T)f.ks[2], inv_dk = (T)f.inv_dk;
    const T hs = f.half ? (T)0.5 : (T)0;
    if (P2 || (Nx & 1) == 0) {
        // kx and -kx (on the half grid kx and -kx of the shifted frequencies) have the same
        // |k|: one thread contracts both points (xx, its mirror xp) with one interpolation of
        // the table. Even Nx (always so for the power-of-two form): xx = 0 .. Nx/2 on the
        // integer grid (0 and Nx/2 are their own mirrors), xx = 0 .. Nx/2 - 1 on the half
        // grid. Odd Nx takes the per-point loop below.
        const int nxh = f.half ? Nx / 2 : Nx / 2 + 1;
        for (int idx = threadIdx.x; idx < nxh * W; idx += blockDim.x) {
            const int xx = fdiv(idx, f.dW), c = idx - xx * W;
            if (c >= ncol) continue;
            const int xp = f.half ? Nx - 1 - xx : (xx == 0 ? 0 : Nx - xx);
            const bool two = xp != xx;
            const int yy = nyq ? y0 + c : y;
            const int kz = nyq ? Kz : kz0 + c;
            const T kx = ks0 * ((T)signed_index(xx, Nx) + hs);
            const T ky = ks1 * ((T)signed_index(yy, Ny) + hs);
            const T kzv = ks2 * ((T)kz + hs);
            const T xk = sqrt(kx * kx + ky * ky + kzv * kzv) * inv_dk;
            int j = (int)floor(xk);
            if (j > f.nk - 2) j = f.nk - 2;
            T w = xk - (T)j;
            w = w < (T)0 ? (T)0 : (w > (T)1 ? (T)1 : w);
            const T *A0 = f.table + (long long)j * rowlen;
            const T *A1 = A0 + rowlen;
            C D[NV], E[NV];
#pragma unroll
            for (int a = 0; a < NV; ++a) {
                D[a] = buf[(a * W + c) * pp + xx];
                E[a] = two ? buf[(a * W + c) * pp + xp] : cmk((T)0, (T)0);
            }
            const C Psi = psi_on ? psi[xx * xstride + col_base + c] : cmk((T)0, (T)0);
            const C Psp = psi_on && two ? psi[xp * xstride + col_base + c] : cmk((T)0, (T)0);
#pragma unroll
            for (int g = 0; g < NV; ++g) {
                T ar = (T)0, ai = (T)0, br = (T)0, bi = (T)0;
#pragma unroll
                for (int a = 0; a < NV; ++a) {
                    const T coef = __ldg(A0 + a * NV + g) * ((T)1 - w) + __ldg(A1 + a * NV + g) * w;
                    ar += coef * D[a].x;
                    ai += coef * D[a].y;
                    br += coef * E[a].x;
                    bi += coef * E[a].y;
                }
                if (psi_on) {
                    const T coef = __ldg(A0 + NV * NV + g) * ((T)1 - w) + __ldg(A1 + NV * NV + g) * w;
                    ar += coef * Psi.x;
                    ai += coef * Psi.y;
                    br += coef * Psp.x;
                    bi += coef * Psp.y;
                }
                buf[(g * W + c) * pp + xx] = cmk(ar, ai);
                if (two) buf[(g * W + c) * pp + xp] = cmk(br, bi);
            }
        }
    } else
    for (int idx = threadIdx.x; idx < npts; idx += blockDim.x) {
        const int xx = fdiv(idx, f.dW), c = idx - xx * W;
        if (c >= ncol) continue;
        const int yy = nyq ? y0 + c : y;
        const int kz = nyq ? Kz : kz0 + c;
        const T kx = ks0 * ((T)signed_index(xx, Nx) + hs);   // hs = 1/2 on the half grid
        const T ky = ks1 * ((T)signed_index(yy, Ny) + hs);
        const T kzv = ks2 * ((T)kz + hs);
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
    fft_smem<C, MaxC<T>::v, !P2>(buf, f.px, 1, NV * W, pp, f.chunk_x, tw_x, +1);
    C *dst_base = nyq ? f.spec_nyq : f.spec;
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int rest = fdiv(idx, f.dW), c = idx - rest * W;
        const int a = fdiv(rest, f.dNx), xx = rest - a * Nx;
        if (c < ncol) dst_base[a * site_stride + xx * xstride + col_base + c] = buf[(a * W + c) * pp + xx];
    }
}

// ------------------------------------------------------------------ y pencils (split planes)
// When a y-z plane does not fit in shared memory the plane passes work on row chunks and
// this pass does the y transform: a tile holds W spectrum columns of one x plane for all y
// and all sites (main tiles: kz0 .. kz0+W; Nyquist tiles: the kz = Kz values of W planes).
template <typename T>
__global__ void __launch_bounds__(kThreadsPencil)
k_ypencil(Fields<T> f, int sign) {
    typedef typename Cx<T>::type C;
    if (f.ctrl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Nx = f.Nx, Ny = f.Ny, Kz = f.Kz, W = f.Wy, pp = f.ypitch, nv = f.nv;
    C *tw_y = buf + (long)nv * W * pp;
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    int tile = blockIdx.x;
    const bool nyq = tile >= f.ytiles_main;
    long long col_base, col_stride, ystride, site_stride;
    int ncol;
    const C *base;
    if (!nyq) {
        const int per = (Kz + W - 1) / W;
        const int x = tile / per, kz0 = (tile - x * per) * W;
        ncol = min(W, Kz - kz0);
        col_base = (long long)x * Ny * Kz + kz0;
        col_stride = 1;
        ystride = Kz;
        site_stride = (long long)Nx * Ny * Kz;
        base = f.spec;
    } else {
        tile -= f.ytiles_main;
        const int x0 = tile * W;
        ncol = min(W, Nx - x0);
        col_base = (long long)x0 * Ny;
        col_stride = Ny;
        ystride = 1;
        site_stride = (long long)Nx * Ny;
        base = f.spec_nyq;
    }
    C *gbase = const_cast<C *>(base);
    const int nload = nv * Ny * W;
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int rest = fdiv(idx, f.dWy), c = idx - rest * W;
        const int a = fdiv(rest, f.dNy), y = rest - a * Ny;
        if (c < ncol) buf[(a * W + c) * pp + y] = gbase[a * site_stride + col_base + c * col_stride + y * ystride];
    }
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, f.py, 1, nv * W, pp, f.chunk_y, tw_y, sign);
    for (int idx = threadIdx.x; idx < nload; idx += blockDim.x) {
        const int rest = fdiv(idx, f.dWy), c = idx - rest * W;
        const int a = fdiv(rest, f.dNy), y = rest - a * Ny;
        if (c < ncol) gbase[a * site_stride + col_base + c * col_stride + y * ystride] = buf[(a * W + c) * pp + y];
    }
}

// ------------------------------------------------------------------ pass 3: plane_inv
// Per-launch values of the residual pass.
template <typename T>
struct InvArgs {
    const long long *hoff;       // [MAXH] ring offsets of the stored residuals (shared memory)
    int hist_n, kind, order, anchor, refresh;
    const T *tcur, *wp;
    T *rcur, *ycur, *ha;         // residual and Y = t + eta R of the new history pair
    T eta;
    const typename Cx<T>::type *post;   // half grid: conj of exp(-i pi p / Kz) applies, else null
};

// Residual R = h + 1 - g (Eq. 33) of the elements e in [e0, e1) of the block's rows, stored
// into the ring and back into the row buffer (in place of h, for the Gram pass that follows),
// with the thread's sum of R^2 in acc.
template <typename T>
__device__ __forceinline__ void inv_elements(const Fields<T> &f, const InvArgs<T> &A,
                                             typename Cx<T>::type *buf, int y0, int e0, int e1,
                                             int tid, int nthr, GramAcc<T> &acc) {
    typedef typename Cx<T>::type C;
    typedef typename Vec2<T>::type V2;
    const int Kz = f.Kz, pitch = f.pitch;
    for (int i0 = e0 + tid; i0 < e1; i0 += 2 * nthr) {
        const int i1 = i0 + nthr;
        const bool has1 = i1 < e1;
        const int yA = fdiv(i0, f.dKz), mA = i0 - yA * Kz;
        const int yB = has1 ? fdiv(i1, f.dKz) : yA, mB = has1 ? i1 - yB * Kz : mA;
        const long long oA = (long long)(y0 + yA) * f.Nz + 2 * mA;
        const long long oB = (long long)(y0 + yB) * f.Nz + 2 * mB;
        // loads of both elements first: delta, w, anchor
        const V2 tA = ld2(A.tcur + oA), tB = ld2(A.tcur + oB);
        const V2 wA = ld2(A.wp + oA), wB = ld2(A.wp + oB);
        V2 aA, aB;
        if (A.anchor) {
            aA = ld2(A.ha + oA);
            aB = ld2(A.ha + oB);
        }
        C hcA = buf[yA * pitch + mA], hcB = buf[yB * pitch + mB];
        if (A.post) {                          // half grid: undo the z shift
            hcA = cmul(hcA, cconj(A.post[mA]));
            hcB = cmul(hcB, cconj(A.post[mB]));
        }
        const T gA0 = closure_g(wA.x + tA.x, A.kind, A.order), gA1 = closure_g(wA.y + tA.y, A.kind, A.order);
        const T gB0 = closure_g(wB.x + tB.x, A.kind, A.order), gB1 = closure_g(wB.y + tB.y, A.kind, A.order);
        // R = h + 1 - g (Eq. 33) with h = h_a + dh; (h_a - g) first: near association peaks
        // both are large and close, and the difference is then exact
        V2 rA, rB, hA, hB;
        if (A.anchor) {
            rA.x = ((aA.x - gA0) + (T)1) + hcA.x;
            rA.y = ((aA.y - gA1) + (T)1) + hcA.y;
            rB.x = ((aB.x - gB0) + (T)1) + hcB.x;
            rB.y = ((aB.y - gB1) + (T)1) + hcB.y;
            hA.x = aA.x + hcA.x;
            hA.y = aA.y + hcA.y;
            hB.x = aB.x + hcB.x;
            hB.y = aB.y + hcB.y;
        } else {
            rA.x = (hcA.x - gA0) + (T)1;
            rA.y = (hcA.y - gA1) + (T)1;
            rB.x = (hcB.x - gB0) + (T)1;
            rB.y = (hcB.y - gB1) + (T)1;
            hA.x = hcA.x;
            hA.y = hcA.y;
            hB.x = hcB.x;
            hB.y = hcB.y;
        }
        acc.add(rA.x, rA.x);
        acc.add(rA.y, rA.y);
        if (A.refresh) *reinterpret_cast<V2 *>(A.ha + oA) = hA;
        *reinterpret_cast<V2 *>(A.rcur + oA) = rA;
        V2 ysA;
        ysA.x = tA.x + A.eta * rA.x;
        ysA.y = tA.y + A.eta * rA.y;
        *reinterpret_cast<V2 *>(A.ycur + oA) = ysA;
        buf[yA * pitch + mA] = cmk(rA.x, rA.y);
        if (has1) {
            acc.add(rB.x, rB.x);
            acc.add(rB.y, rB.y);
            if (A.refresh) *reinterpret_cast<V2 *>(A.ha + oB) = hB;
            *reinterpret_cast<V2 *>(A.rcur + oB) = rB;
            V2 ysB;
            ysB.x = tB.x + A.eta * rB.x;
            ysB.y = tB.y + A.eta * rB.y;
            *reinterpret_cast<V2 *>(A.ycur + oB) = ysB;
            buf[yB * pitch + mB] = cmk(rB.x, rB.y);
        }
    }
}

// Gram row of the new residual, <R, R_i> for each stored residual i, over the block's rows:
// R from the row buffer, R_i streamed from the ring, one history value at a time (one
// accumulator in registers, G = 16 (FP32) or 8 (FP64) loads in flight per thread, issued
// before the shared-memory reads of R so that only the loads occupy registers). The warp
// sums go to red[(i + 1) * nw + warp].
template <typename T>
__device__ __forceinline__ void gram_row(const Fields<T> &f, const InvArgs<T> &A,
                                         const typename Cx<T>::type *buf, int y0, int nyb, double *red) {
    typedef typename Cx<T>::type C;
    typedef typename Vec2<T>::type V2;
    constexpr int G = sizeof(T) == 4 ? 16 : 8;
    const int Kz = f.Kz, pitch = f.pitch;
    const int n = nyb * Kz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nthr = blockDim.x;
    for (int h = 0; h < A.hist_n; ++h) {
        const T *q = f.R + A.hoff[h];
        GramAcc<T> acc;
        acc.zero();
        // whole batches of G elements per thread, then the rest one at a time; summed in
        // element order
        int e = threadIdx.x;
        for (; e + (G - 1) * nthr < n; e += G * nthr) {
            V2 qv[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int ei = e + u * nthr;
                const int y = fdiv(ei, f.dKz), m = ei - y * Kz;
                qv[u] = ld2(q + (long long)(y0 + y) * f.Nz + 2 * m);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int ei = e + u * nthr;
                const int y = fdiv(ei, f.dKz), m = ei - y * Kz;
                const C rv = buf[y * pitch + m];
                acc.add(rv.x, qv[u].x);
                acc.add(rv.y, qv[u].y);
            }
        }
        for (; e < n; e += nthr) {
            const int y = fdiv(e, f.dKz), m = e - y * Kz;
            const V2 qv = ld2(q + (long long)(y0 + y) * f.Nz + 2 * m);
            const C rv = buf[y * pitch + m];
            acc.add(rv.x, qv.x);
            acc.add(rv.y, qv.y);
        }
        acc.warp_reduce();
        if (lane == 0) red[(h + 1) * nw + warp] = acc.value();
    }
}

// One block per (x plane or row chunk of one, site): inverse y and z transforms, residual,
// and the block's contribution to <R_cur, R_i> and sum R^2 (Dot2 accumulation, FP64 across
// threads). Partials are stored value-major: partials[i * n_blocks + block]. With LZ > 0
// (as for plane_fwd) each warp takes its own rows through the complex-to-real step, the z
// transform and the residual after the block-wide y transform.
template <typename T, int MAXH, int LZ>
__global__ void __launch_bounds__(kThreadsPlane, sizeof(T) == 4 ? RISM_MINBLOCKS_F32 : 2)
k_plane_inv(Fields<T> f) {
    typedef typename Cx<T>::type C;
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = f.Kz, pitch = f.pitch;
    C *tw_h = buf + (long)f.slab_rows * pitch;    // after the block's rows
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    C *tw_q = tw_z + (Kz + 1);
    double *red = reinterpret_cast<double *>(tw_q + Kz);
    const bool half = f.half;
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];
    if (half)
        for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_q[i] = f.tw_q[i];
    const int nyc = f.nyc;
    const int x = blockIdx.x / nyc, yc = blockIdx.x - (blockIdx.x / nyc) * nyc, gam = blockIdx.y;
    const int y0 = yc * f.slab_rows, nyb = min(f.slab_rows, Ny - y0);
    const long long ring = (long long)f.nv * f.G;
    const long long siteoff = (long long)gam * f.G + (long long)x * Ny * f.Nz;
    __shared__ long long hoff[MAXH];
    InvArgs<T> A;
    A.hist_n = ctl->hist_n;
    if (threadIdx.x < MAXH)
        hoff[threadIdx.x] = threadIdx.x < A.hist_n ? (long long)ctl->hist_slot[threadIdx.x] * ring + siteoff : 0;
    const int stage = ctl->stage;
    A.hoff = hoff;
    A.kind = ctl->stage_kind[stage];
    A.order = ctl->stage_order[stage];
    A.anchor = ctl->anchor_valid;
    A.refresh = ctl->refresh;
    A.tcur = f.Tc + (long long)gam * f.G + (long long)x * Ny * f.Nz;
    A.rcur = f.R + (long long)ctl->cur * ring + siteoff;
    A.ycur = f.X + (long long)ctl->cur * ring + siteoff;
    A.eta = (T)ctl->eta;
    A.wp = f.w + siteoff;
    A.ha = f.h_a + siteoff;
    A.post = half ? tw_z : nullptr;
    const C phx = half ? f.tw_xs[x] : cmk((T)1, (T)0);

    const bool clus = f.cl > 1;
    // row y of the block takes spectrum row ky = y0 + y, or ky = R y + yc across a cluster
    const int rstride = clus ? f.cl : 1, roff = clus ? yc : y0;
    if (clus) {
        C *tw_s = reinterpret_cast<C *>(red + (kMaxHist + 1) * (kThreadsPlane / 32));
        for (int i = threadIdx.x; i < nyb; i += blockDim.x) tw_s[i] = f.tw_y[i * f.cl];
    }
    const C *src = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;
    if (sizeof(T) == 4) {                     // 8-byte elements: asynchronous copies
        for (int idx = threadIdx.x; idx < nyb * Kz; idx += blockDim.x) {
            const int y = fdiv(idx, f.dKz), k = idx - y * Kz;
            cp_async8(&buf[y * pitch + k], &src[(long long)(rstride * y + roff) * Kz + k]);
        }
        if (!half) {
            const C *sn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
            for (int y = threadIdx.x; y < nyb; y += blockDim.x)
                cp_async8(&buf[y * pitch + Kz], &sn[rstride * y + roff]);
        }
        cp_async_wait();
    } else if (clus) {
        for (int idx = threadIdx.x; idx < nyb * Kz; idx += blockDim.x) {
            const int y = fdiv(idx, f.dKz), k = idx - y * Kz;
            buf[y * pitch + k] = src[(long long)(rstride * y + roff) * Kz + k];
        }
        const C *sn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
        for (int y = threadIdx.x; y < nyb; y += blockDim.x) buf[y * pitch + Kz] = sn[rstride * y + roff];
    } else {
        src += (long long)y0 * Kz;
        for (int idx = threadIdx.x; idx < nyb * Kz; idx += blockDim.x) {
            const int y = fdiv(idx, f.dKz), k = idx - y * Kz;
            buf[y * pitch + k] = src[idx];
        }
        if (!half) {
            const C *sn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny + y0;
            for (int y = threadIdx.x; y < nyb; y += blockDim.x) buf[y * pitch + Kz] = sn[y];
        }
    }
    __syncthreads();
    if (nyc == 1 && half) {
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, +1);
    } else if (nyc == 1) {
        // columns kz = 0 and Kz (transforms of real sequences) as one: P = A + iB
        for (int y = threadIdx.x; y < Ny; y += blockDim.x) {
            const C A0 = buf[y * pitch], B0 = buf[y * pitch + Kz];
            buf[y * pitch] = cmk(A0.x - B0.y, A0.y + B0.x);
        }
        __syncthreads();
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, +1);
    } else if (clus) {
        // inverse y transform across the cluster: the local length-S transform (it ends with
        // a block barrier), then the cross-block radix step
        C *tw_s = reinterpret_cast<C *>(red + (kMaxHist + 1) * (kThreadsPlane / 32));
        fft_smem<C, MaxC<T>::v, LZ == 0>(buf, f.pys, pitch, Kz + 1, 1, f.chunk_ys, tw_s, +1);
        cluster_y_step<C>(buf, f.cl, nyb, Kz + 1, pitch, f.dK1, tw_y, +1);
    }

    GramAcc<T> acc;
    acc.zero();
    if constexpr (LZ > 0) {
        constexpr int RW = 256 / LZ;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r0 = warp * RW; r0 < nyb; r0 += nw * RW) {
            const int nr = min(RW, nyb - r0);
            if (half)
                c2r_rows_half(buf + (long)r0 * pitch, nr, y0 + r0, LZ, pitch, tw_q, f.tw_ys, phx, f.dKzp, lane, 32);
            else
                c2r_rows(buf + (long)r0 * pitch, nr, LZ, pitch, tw_z, f.dKz1h, lane, 32, nyc == 1);
            __syncwarp();
            fft_rows_warp<C, LZ>(buf + (long)r0 * pitch, nr, pitch, tw_h, +1, lane);
            inv_elements<T>(f, A, buf, y0, r0 * LZ, (r0 + nr) * LZ, lane, 32, acc);
        }
    } else {
        if (half)
            c2r_rows_half(buf, nyb, y0, Kz, pitch, tw_q, f.tw_ys, phx, f.dKzp, threadIdx.x, blockDim.x);
        else
            c2r_rows(buf, nyb, Kz, pitch, tw_z, f.dKz1h, threadIdx.x, blockDim.x, nyc == 1);
        __syncthreads();
        fft_smem<C, MaxC<T>::v>(buf, f.ph, 1, nyb, pitch, f.chunk_rows, tw_h, +1);
        inv_elements<T>(f, A, buf, y0, 0, nyb * Kz, threadIdx.x, blockDim.x, acc);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long nblocks = (long long)f.nv * f.Nx * nyc;
    const long long blk = ((long long)gam * f.Nx + x) * nyc + yc;
    acc.warp_reduce();
    if (lane == 0) red[warp] = acc.value();
    __syncthreads();                       // every row's R is in the buffer
    gram_row<T>(f, A, buf, y0, nyb, red);
    __syncthreads();
    if (threadIdx.x <= A.hist_n) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += red[threadIdx.x * nw + k];
        f.partials[threadIdx.x * nblocks + blk] = s;
    }
}

// ------------------------------------------------------------------ MDIIS (one block)
// Reduce the Gram partials in a fixed order (bit-reproducible), update the Gram matrix,
// solve for the accelerator's coefficients (Eq. 40 as the bordered DIIS system, or the
// modified Anderson rule of Eqs. 34-39) and prepare the next update. The control block is
// staged in shared memory: the bookkeeping is a short serial chain, and on this GPU a chain
// of FP64 operations on global memory costs tens of microseconds.

// Scratch of the MDIIS kernel in shared memory.
struct MdiisScratch {
    double A[kMaxHist + 1][kMaxHist + 2];    // bordered system, augmented with its rhs
    double fcol[kMaxHist + 1];
    double inv_diag[kMaxHist + 1];
    double c[kMaxHist];
    int H[kMaxHist];
    int k, first, mode;
};

// Bookkeeping before the coefficient solve (thread 0): byte counters, RMS, convergence and
// closure stages, the Gram row of the new residual, and the candidate history H (oldest
// first). mode: 0 = nothing more to do, 1 = MDIIS bordered solve, 2 = modified Anderson.
static __device__ void mdiis_pre(Ctrl *ctl, const double *sums, MdiisScratch &sc) {
    const int hist_n = ctl->hist_n;
    sc.mode = 0;
    ctl->acc_iters += 1;
    ctl->acc_fwd_units += ctl->do_update ? ctl->upd_n + 1 : 1;
    ctl->acc_upd_r += ctl->do_update && ctl->upd_r ? ctl->upd_n : 0;
    ctl->acc_hist += hist_n;
    ctl->acc_anchor += ctl->anchor_valid;
    ctl->acc_refresh += ctl->refresh;
    ctl->acc_shift += ctl->refresh && ctl->do_update ? ctl->upd_n : 0;
    ctl->acc_psi += ctl->anchor_valid == 0;
    const int cur = ctl->cur;
    ctl->eta_slot[cur] = ctl->eta;    // plane_inv stored Y_cur = t + eta R_cur
    const double rr = sums[0];
    const double rms = sqrt(rr * ctl->inv_count);
    ctl->rms = rms;
    ctl->iter += 1;
    if (ctl->refresh) {               // this iteration wrote g_a, h_a and moved the offset
        ctl->refresh = 0;
        ctl->anchor_valid = 1;
    }
    if (!isfinite(rms)) {
        ctl->status = kDiverged;
        return;
    }
    if (rms < ctl->next_refresh) {    // next iteration re-anchors the transform
        ctl->refresh = 1;
        ctl->next_refresh = rms * ctl->anchor_ratio;
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
    for (int i = 0; i < hist_n; ++i) {
        const int s = ctl->hist_slot[i];
        ctl->B[cur * kMaxHist + s] = sums[i + 1];
        ctl->B[s * kMaxHist + cur] = sums[i + 1];
    }
    ctl->B[cur * kMaxHist + cur] = rr;
    int k = 0;
    for (int i = 0; i < hist_n; ++i) sc.H[k++] = ctl->hist_slot[i];
    sc.H[k++] = cur;
    sc.k = k;
    sc.first = 0;
    sc.mode = ctl->accel == 1 ? 2 : 1;
}

// Modified Anderson coefficients (Eqs. 34-39, two histories): theta from the 2 x 2 system
// of Eq. 36 on D_i = R_new - R_{new-i}, a_i = theta_i + s_i; Picard while fewer than three
// pairs are stored or if the system is singular.
static __device__ void anderson_coef(const Ctrl *ctl, MdiisScratch &sc) {
    const int k = sc.k;
    for (int i = 0; i < k; ++i) sc.c[i] = 0.0;
    sc.c[k - 1] = 1.0;
    if (k < 3) return;
    const int n0 = sc.H[k - 1], n1 = sc.H[k - 2], n2 = sc.H[k - 3];
    const int di[2] = {n1, n2};
    double Mm[2][2], rhs[2];
    const double b00 = ctl->B[n0 * kMaxHist + n0];
    for (int i = 0; i < 2; ++i) {
        rhs[i] = b00 - ctl->B[n0 * kMaxHist + di[i]];
        for (int j = 0; j < 2; ++j)
            Mm[i][j] = b00 - ctl->B[n0 * kMaxHist + di[j]] - ctl->B[n0 * kMaxHist + di[i]] +
                       ctl->B[di[i] * kMaxHist + di[j]];
    }
    const double sc0 = fmax(Mm[0][0], Mm[1][1]);
    if (!(sc0 > 0.0)) return;
    const double is = 1.0 / sc0;
    for (int i = 0; i < 2; ++i) {
        rhs[i] *= is;
        for (int j = 0; j < 2; ++j) Mm[i][j] *= is;
    }
    const int p = fabs(Mm[1][0]) > fabs(Mm[0][0]) ? 1 : 0;
    if (fabs(Mm[p][0]) < 1e-12) return;
    if (p == 1) {
        const double t0 = Mm[0][0], t1 = Mm[0][1], tr = rhs[0];
        Mm[0][0] = Mm[1][0];
        Mm[0][1] = Mm[1][1];
        rhs[0] = rhs[1];
        Mm[1][0] = t0;
        Mm[1][1] = t1;
        rhs[1] = tr;
    }
    const double fct = Mm[1][0] / Mm[0][0];
    const double m11 = Mm[1][1] - fct * Mm[0][1];
    const double r1 = rhs[1] - fct * rhs[0];
    if (fabs(m11) < 1e-12) return;
    const double th1 = r1 / m11;
    const double th0 = (rhs[0] - Mm[0][1] * th1) / Mm[0][0];
    const double a1 = th0 + ctl->s1, a2 = th1 + ctl->s2;
    sc.c[k - 1] = 1.0 - a1 - a2;
    sc.c[k - 2] = a1;
    sc.c[k - 3] = a2;
}

// MDIIS coefficients by one warp: lane j owns column j of [B / max diag, 1; 1^T, 0 | rhs];
// Gaussian elimination with partial pivoting (pivot search by shuffles, one reciprocal per
// pivot); a pivot below 1e-12 drops the oldest vector and retries. Every branch decision is
// lane 0's (broadcast), a NaN entry counts as a zero pivot, and there are at most k
// attempts, so the warp stays converged and the loop ends whatever the Gram entries are.
static __device__ void mdiis_coef_warp(const Ctrl *ctl, MdiisScratch &sc, int lane) {
    for (int attempt = 0; attempt < kMaxHist + 1; ++attempt) {
        const int n = sc.k - sc.first;
        if (n == 1) {
            if (lane == 0) sc.c[0] = 1.0;
            __syncwarp();
            return;
        }
        const int dim = n + 1;
        const int *H = sc.H + sc.first;
        double scale = 0.0;
        for (int i = 0; i < n; ++i) scale = fmax(scale, ctl->B[H[i] * kMaxHist + H[i]]);
        const double inv = scale > 0.0 ? 1.0 / scale : 1.0;
        if (lane <= dim)                       // lane j fills column j (j = dim: the rhs)
            for (int i = 0; i < dim; ++i) {
                double v;
                if (lane == dim) v = (i == n) ? 1.0 : 0.0;
                else if (i == n) v = (lane == n) ? 0.0 : 1.0;
                else if (lane == n) v = 1.0;
                else v = ctl->B[H[i] * kMaxHist + H[lane]] * inv;
                sc.A[i][lane] = v;
            }
        __syncwarp();
        bool ok = true;
        for (int col = 0; col < dim; ++col) {
            double v = (lane >= col && lane < dim) ? fabs(sc.A[lane][col]) : -1.0;
            if (!(v == v)) v = 0.0;                          // NaN: no usable pivot
            int p = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int p2 = __shfl_xor_sync(0xffffffffu, p, o);
                if (v2 > v || (v2 == v && p2 < p)) {
                    v = v2;
                    p = p2;
                }
            }
            v = __shfl_sync(0xffffffffu, v, 0);             // one decision for the warp
            p = __shfl_sync(0xffffffffu, p, 0);
            if (!(v >= 1e-12)) {
                ok = false;
                break;
            }
            if (p != col && lane <= dim) {
                const double t = sc.A[col][lane];
                sc.A[col][lane] = sc.A[p][lane];
                sc.A[p][lane] = t;
            }
            __syncwarp();
            const double id = 1.0 / sc.A[col][col];
            if (lane == 0) sc.inv_diag[col] = id;
            if (lane > col && lane < dim) sc.fcol[lane] = sc.A[lane][col] * id;
            __syncwarp();
            if (lane > col && lane <= dim)
                for (int r = col + 1; r < dim; ++r) sc.A[r][lane] -= sc.fcol[r] * sc.A[col][lane];
            __syncwarp();
        }
        if (ok) {
            if (lane == 0) {
                double xs[kMaxHist + 1];
                for (int r = dim - 1; r >= 0; --r) {
                    double s = sc.A[r][dim];
                    for (int j = r + 1; j < dim; ++j) s -= sc.A[r][j] * xs[j];
                    xs[r] = s * sc.inv_diag[r];
                }
                for (int i = 0; i < n; ++i) sc.c[i] = xs[i];
            }
            __syncwarp();
            return;
        }
        if (lane == 0) sc.first += 1;
        __syncwarp();
    }
    if (lane == 0) {                          // not reached for valid input: keep the newest
        sc.first = sc.k - 1;
        sc.c[0] = 1.0;
    }
    __syncwarp();
}

// After the solve (thread 0): damping, the update list and the ring slot of the next
// iterate (a free slot while the history is short, else the oldest, which leaves it).
static __device__ void mdiis_post(Ctrl *ctl, MdiisScratch &sc) {
    const int M = ctl->M;
    const int n = sc.k - sc.first;
    const int *H = sc.H + sc.first;
    double eta = ctl->damp;
    if (ctl->dynamic) eta = fmin(fmax(-0.2 * log10(ctl->rms), 0.1), 1.0);
    ctl->eta = eta;
    ctl->upd_n = n;
    ctl->upd_r = 0;
    for (int i = 0; i < n; ++i) {
        ctl->upd_slot[i] = H[i];
        ctl->upd_coef[i] = sc.c[i];
        // sum c_i (t_i + eta R_i) = sum c_i Y_i + sum c_i (eta - eta_i) R_i
        const double d = sc.c[i] * (eta - ctl->eta_slot[H[i]]);
        ctl->upd_dcoef[i] = d;
        if (d != 0.0) ctl->upd_r = 1;
    }
    int next;
    if (n < M) {
        int used = 0;
        for (int i = 0; i < n; ++i) used |= 1 << H[i];
        next = 0;
        while (used & (1 << next)) ++next;
        ctl->hist_n = n;
        for (int i = 0; i < n; ++i) ctl->hist_slot[i] = H[i];
    } else {
        next = H[0];
        ctl->hist_n = n - 1;
        for (int i = 1; i < n; ++i) ctl->hist_slot[i - 1] = H[i];
    }
    ctl->cur = next;
    ctl->do_update = 1;
}

static __global__ void k_mdiis(Ctrl *ctl_g, const double *partials, int nblocks) {
    __shared__ double sums[kMaxHist + 1];
    __shared__ double part[kMaxHist + 1][kThreadsMdiis / 32];
    __shared__ Ctrl ctl_s;
    __shared__ MdiisScratch sc;
    if (ctl_g->status != kRunning) return;
    const int hist_n = ctl_g->hist_n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    {   // the control block to shared memory, while the partial sums are being loaded
        const int n = (int)(sizeof(Ctrl) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(ctl_g);
        int *dst = reinterpret_cast<int *>(&ctl_s);
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
    // value v = <R_cur, R_v-1> (v > 0) or sum R^2 (v = 0): wpv warps per value, each summing
    // a fixed stride of block partials; the warps' sums are then added in a fixed order
    const int nval = hist_n + 1, wpv = nw / nval;
    const int v = warp / wpv, sub = warp - v * wpv;
    if (v < nval) {
        const double *pv = partials + (long long)v * nblocks;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        const int st = 32 * wpv;
        int b = sub * 32 + lane;
        for (; b + 3 * st < nblocks; b += 4 * st) {
            s0 += pv[b];
            s1 += pv[b + st];
            s2 += pv[b + 2 * st];
            s3 += pv[b + 3 * st];
        }
        for (; b < nblocks; b += st) s0 += pv[b];
        double s = (s0 + s1) + (s2 + s3);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[v][sub] = s;
    }
    __syncthreads();
    if (threadIdx.x < nval) {
        double s = 0.0;
        for (int k = 0; k < wpv; ++k) s += part[threadIdx.x][k];
        sums[threadIdx.x] = s;
    }
    Ctrl *ctl = &ctl_s;
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) mdiis_pre(ctl, sums, sc);
        __syncwarp();
        if (sc.mode == 1) mdiis_coef_warp(ctl, sc, lane);
        if (sc.mode == 2 && lane == 0) anderson_coef(ctl, sc);
        __syncwarp();
        if (sc.mode != 0 && lane == 0) mdiis_post(ctl, sc);
    }
    __syncthreads();
    {
        const int n = (int)(sizeof(Ctrl) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(&ctl_s);
        int *dst = reinterpret_cast<int *>(ctl_g);
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
}

// ------------------------------------------------------------------ potential (Eq. 22, 29)
// One thread per grid point and all sites; atoms staged through shared memory. For the
// FP32 form, far pairs are evaluated in FP32 (their Coulomb and phi terms accumulated in
// FP64) and near pairs (r < 1.5 max sigma_ag, where the r^-12 term is large enough for FP32
// coordinate rounding to show) entirely in FP64. Writes beta*u (capped at 1e4), phi and
// w = beta q phi - beta*u (both the kept copy wref and the working field w, whose offset
// tau0 is zero until a solve refreshes it).
template <typename T>
__global__ void __launch_bounds__(256)
k_potential(Fields<T> f, const double *atoms, int n_atoms, const double *site_sig,
            const double *site_eps, const double *site_q, double beta, double ox, double oy,
            double oz, double dx, double dy, double dz) {
    constexpr int TILE = 64;
    constexpr bool kMixed = sizeof(T) == 4;
    __shared__ double ax[TILE], ay[TILE], az[TILE], aq[TILE];
    __shared__ T anear2[TILE];
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
    double coul = 0.0, phi = 0.0;            // near pairs (FP64)
    SumAcc<T> coul_f, phi_f;                 // far pairs
    coul_f.zero();
    phi_f.zero();
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
            anear2[i] = kMixed ? (T)(2.25 * smax * smax) : (T)-1;
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < na; ++i) {
                const T ddx = px - sx[i], ddy = py - sy[i], ddz = pz - sz[i];
                const T r2f = ddx * ddx + ddy * ddy + ddz * ddz;
                if (kMixed && r2f < anear2[i]) {
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
                    T ir, ir2, r, om;
                    if constexpr (kMixed) {
                        // far pairs (r above 1.5 sigma_ag >= 2.6 A): 1 - e^{-r} >= 0.93, so the
                        // fast exponential keeps ~1e-7; 1/r stays correctly rounded, since the
                        // Coulomb and phi sums of a charged solute cancel to a few % of the sum
                        // of their magnitudes and a biased 1/r would show at 1e-5
                        r = sqrtf(r2);
                        ir = 1.f / r;
                        ir2 = ir * ir;
                        om = 1.f - __expf(-r);
                    } else {
                        ir2 = (T)1 / r2;
                        r = sqrt(r2);
                        ir = (T)1 / r;
                        om = (T)(-expm1(-r));
                    }
                    coul_f.add(sq[i] * ir);
                    phi_f.add(sq[i] * om * ir);
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
    coul += coul_f.value();
    phi += phi_f.value();
    const double C = 332.0637;
    const double phiv = C * phi;
    for (int g = 0; g < nv; ++g) {
        double v = beta * ((double)lj[g] + ljd[g] + C * site_q[g] * coul);
        v = v > 1e4 ? 1e4 : v;
        const T wv = (T)(beta * site_q[g] * phiv - v);
        f.bu[(long long)g * G + p] = (T)v;
        f.wref[(long long)g * G + p] = wv;
        f.w[(long long)g * G + p] = wv;
    }
    f.phi[p] = (T)phiv;
}

// ------------------------------------------------------------------ long range (Eq. 30)
// Psi(k) = beta Phi~(k) / dV = amp0 / (k^2 (k^2 + 1)) sum_a q_a exp(-i k.(R_a - r0)), zero at
// k = 0 and on Nyquist planes. The phase factorises over the axes,
// exp(-i k.u) = E_x(a, mx) E_y(a, my) E_z(a, mz) with E(a, m) = exp(-2 pi i m u_a) and
// u = (R - r0) / L; the tables are evaluated once per atom chunk in FP64 (sincospi) and
// rounded to the working precision, so each (atom, k) pair costs two complex products and
// a compensated sum.
template <typename T>
__global__ void k_phase_tables(Fields<T> f, const double *atoms, int a0, int na,
                               typename Cx<T>::type *tab) {
    typedef typename Cx<T>::type C;
    const int per = f.Nx + f.Ny + f.Kz + 1;
    const long long n = (long long)na * per;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(id / per), e = (int)(id - (long long)a * per);
        const double *at = atoms + (long long)(a0 + a) * kAtomStride;
        double u;
        int m;
        if (e < f.Nx) {
            m = signed_index(e, f.Nx);
            u = at[6];
        } else if (e < f.Nx + f.Ny) {
            m = signed_index(e - f.Nx, f.Ny);
            u = at[7];
        } else {
            m = e - f.Nx - f.Ny;
            u = at[8];
        }
        double sn, cs;
        sincospi(2.0 * (m + (f.half ? 0.5 : 0.0)) * u, &sn, &cs);
        C v;
        v.x = (T)cs;
        v.y = (T)(-sn);
        tab[id] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_longrange(Fields<T> f, const double *atoms, int a0, int na, const typename Cx<T>::type *tab,
            double amp0, int accumulate) {
    typedef typename Cx<T>::type C;
    __shared__ T qs[kPhaseChunk];
    for (int i = threadIdx.x; i < na; i += blockDim.x) qs[i] = (T)atoms[(long long)(a0 + i) * kAtomStride + 3];
    __syncthreads();
    const long long nmain = (long long)f.Nx * f.Ny * f.Kz;
    const long long total = nmain + (f.half ? 0 : (long long)f.Nx * f.Ny);
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
    // integer grid: zero at k = 0 and on Nyquist planes; the half grid has neither
    const bool nyq = !f.half && (((f.Nx % 2 == 0) && 2 * abs(mx) == f.Nx) ||
                                 ((f.Ny % 2 == 0) && 2 * abs(my) == f.Ny) || (2 * mz == f.Nz));
    const double hs = f.half ? 0.5 : 0.0;
    const double kx = f.ks[0] * (mx + hs), ky = f.ks[1] * (my + hs), kz = f.ks[2] * (mz + hs);
    const double k2 = kx * kx + ky * ky + kz * kz;
    double re = 0.0, im = 0.0;
    if (!nyq && k2 > 0.0) {
        const int per = f.Nx + f.Ny + f.Kz + 1;
        const C *ex = tab + ix, *ey = tab + f.Nx + iy, *ez = tab + f.Nx + f.Ny + iz;
        SumAcc<T> sr, si;
        sr.zero();
        si.zero();
        for (int a = 0; a < na; ++a) {
            const long long o = (long long)a * per;
            const C xy = cmul(__ldg(ex + o), __ldg(ey + o));
            const C e = cmul(xy, __ldg(ez + o));
            sr.add(qs[a] * e.x);
            si.add(qs[a] * e.y);
        }
        const double amp = amp0 / (k2 * (k2 + 1.0));
        re = amp * sr.value();
        im = amp * si.value();
    }
    C *dst = id < nmain ? f.psi + id : f.psi_nyq + (id - nmain);
    C v = cmk((T)re, (T)im);
    if (accumulate) {
        const C o = *dst;
        v.x += o.x;
        v.y += o.y;
    }
    *dst = v;
}

// ------------------------------------------------------------------ learned guess crops
// Crop of side n at grid index (i0, j0, k0) (inside the grid), FP32 [nv][n^3]:
// mode 0: network input tanh(beta u / 4); mode 1: the iterate tau of `slot`.
template <typename T>
__global__ void k_guess_crop_out(Fields<T> f, int mode, int slot, int i0, int j0, int k0, int n, float *out) {
    const long long V = (long long)n * n * n, total = (long long)f.nv * V;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % n);
        r /= n;
        const int j = (int)(r % n);
        r /= n;
        const int i = (int)(r % n);
        const int g = (int)(r / n);
        const long long src = (long long)g * f.G + ((long long)(i0 + i) * f.Ny + (j0 + j)) * f.Nz + (k0 + k);
        if (mode == 0)
            out[id] = tanhf((float)f.bu[src] * 0.25f);
        else
            out[id] = (float)((double)f.tau0[src] + (double)f.Tc[src]);
    }
}

// The iterate of `slot` (whole field): tau = crop values inside the crop, 0 outside (offset
// tau0 = 0, w = wref).
template <typename T>
__global__ void k_guess_crop_in(Fields<T> f, int slot, int i0, int j0, int k0, int n, const float *in) {
    const long long total = (long long)f.nv * f.G;
    T *dst = f.Tc;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        long long r = id;
        const int k = (int)(r % f.Nz);
        r /= f.Nz;
        const int j = (int)(r % f.Ny);
        r /= f.Ny;
        const int i = (int)(r % f.Nx);
        const int g = (int)(r / f.Nx);
        const int ci = i - i0, cj = j - j0, ck = k - k0;
        T v = (T)0;
        if (ci >= 0 && ci < n && cj >= 0 && cj < n && ck >= 0 && ck < n)
            v = (T)in[(((long long)g * n + ci) * n + cj) * n + ck];
        dst[id] = v;
        f.tau0[id] = (T)0;
        f.w[id] = f.wref[id];
    }
}

template <typename T>
cudaError_t launch_guess_crop(const Fields<T> &f, int mode, int slot, const int *corner, int n, float *out,
                              const float *in, cudaStream_t s) {
    if (mode == 2)
        k_guess_crop_in<T><<<152 * 8, 256, 0, s>>>(f, slot, corner[0], corner[1], corner[2], n, in);
    else
        k_guess_crop_out<T><<<152 * 8, 256, 0, s>>>(f, mode, slot, corner[0], corner[1], corner[2], n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ small helpers
// Step 1: t = f, i.e. tau = 0: delta = 0 in the current-iterate field, offset tau0 = 0 and
// w = wref (the ring slot argument of the launcher only names where the next residual goes).
template <typename T>
__global__ void k_init_guess(Fields<T> f) {
    const long long n = (long long)f.nv * f.G;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        f.Tc[i] = (T)0;
        f.tau0[i] = (T)0;
        f.w[i] = f.wref[i];
    }
}

// tau = t - beta q phi from a caller field t (FP64) as delta, with offset tau0 = 0.
template <typename T>
__global__ void k_guess_from_t(Fields<T> f, const double *src) {
    const long long n = (long long)f.nv * f.G;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / f.G);
        const long long p = i - (long long)g * f.G;
        f.Tc[i] = (T)(src[i] - f.bq[g] * (double)f.phi[p]);
        f.tau0[i] = (T)0;
        f.w[i] = f.wref[i];
    }
}

// Before a solve restarts from the last iterate: tau = tau0 + delta becomes delta with
// tau0 = 0 and w = wref, so that the unanchored first iterations transform c^sr whole.
template <typename T>
__global__ void k_flatten(Fields<T> f) {
    const long long n = (long long)f.nv * f.G;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        f.Tc[i] = f.tau0[i] + f.Tc[i];
        f.tau0[i] = (T)0;
        f.w[i] = f.wref[i];
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
            const T delta = f.Tc[i];
            const double tau = (double)f.tau0[i] + (double)delta;
            const double fq = f.bq[g] * (double)f.phi[p];
            if (field == 4) {
                v = tau + fq;
            } else {
                const T gv = closure_g(f.w[i] + delta, kind, order);
                if (field == 1) v = (double)gv;
                else if (field == 3) v = (double)(gv - (T)1);
                else v = ((double)gv - 1.0 - tau) - fq;      // c = h - t
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
    const T *tt = f.Tc + (long long)g * f.G;
    const T *t0 = f.tau0 + (long long)g * f.G;
    const T *wp = f.w + (long long)g * f.G;
    const double bq = f.bq[g];
    double acc = 0.0;
    double fact = 1.0;
    for (int i = 2; i <= sfe_order + 1; ++i) fact *= i;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < f.G;
         p += (long long)gridDim.x * blockDim.x) {
        const T delta = tt[p];
        const T d = wp[p] + delta;
        const T gv = closure_g(d, kind, order);
        const double h = (double)(gv - (T)1);
        const double tau = (double)t0[p] + (double)delta;
        const double c = ((double)gv - 1.0 - tau) - bq * (double)f.phi[p];   // c = h - t
        double v = -c - 0.5 * h * c;
        if (sfe_kind == 5) v = c;                                // int c dr (PMV, Eq. 19)
        else if (sfe_kind == 2) v += 0.5 * h * h;                // HNC, Eq. 17
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


// ------------------------------------------------------------------ SFE gradient (second Eq. 21)
// d(dmu)/dR_a = sum_g rho_g int g_g(r) du_g(r)/dR_a dr with
// du/dR = (48 eps s^12 / d^14 - 24 eps s^6 / d^8 + C q_a q_g / d^3) (r - R), d = |r - R_a|.
// Pass 1 stores rho_g dV g_g(r) (the spectrum buffer is free after a solve); pass 2 takes a
// tile of atoms per block row and a range of grid points per block, with per-thread partial
// sums and a block reduction into partials[(atom * 3 + component) * nblk + block]; pass 3
// sums the blocks in a fixed order.
template <typename T>
__global__ void k_grad_weights(Fields<T> f, int slot, int kind, int order, const double *rho_dV) {
    T *wg = reinterpret_cast<T *>(f.spec);
    const long long ring = (long long)f.nv * f.G;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ring;
         i += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(i / f.G);
        const T tau = f.Tc[i];
        wg[i] = (T)rho_dV[g] * closure_g(f.w[i] + tau, kind, order);
    }
}

template <typename T> struct GradTile;
template <> struct GradTile<float> { static constexpr int v = 8; };
template <> struct GradTile<double> { static constexpr int v = 4; };

template <typename T>
__global__ void __launch_bounds__(256)
k_sfe_gradient(Fields<T> f, const double *atoms, int n_atoms, const double *site_sig,
               const double *site_eps, const double *site_q, double ox, double oy, double oz,
               double dx, double dy, double dz, double *partials) {
    constexpr int AT = GradTile<T>::v;
    __shared__ T ax[AT], ay[AT], az[AT], aq[AT];
    __shared__ T s2[AT][kMaxSites], e48[AT][kMaxSites], e24[AT][kMaxSites];
    __shared__ double red[8][3 * AT];
    const int nv = f.nv;
    const int a0 = blockIdx.y * AT;
    const int na = min(AT, n_atoms - a0);
    for (int i = threadIdx.x; i < AT; i += blockDim.x) {
        if (i < na) {
            const double *at = atoms + (long long)(a0 + i) * kAtomStride;
            ax[i] = (T)(at[0] - ox);
            ay[i] = (T)(at[1] - oy);
            az[i] = (T)(at[2] - oz);
            aq[i] = (T)(332.0637 * at[3]);
            for (int g = 0; g < nv; ++g) {
                const double sg = 0.5 * (at[4] + site_sig[g]), eg = sqrt(at[5] * site_eps[g]);
                s2[i][g] = (T)(sg * sg);
                e48[i][g] = (T)(48.0 * eg);
                e24[i][g] = (T)(24.0 * eg);
            }
        }
    }
    __syncthreads();
    const T *wg = reinterpret_cast<const T *>(f.spec);
    T acc[3 * AT];
#pragma unroll
    for (int k = 0; k < 3 * AT; ++k) acc[k] = (T)0;
    const int NyNz = f.Ny * f.Nz;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < f.G;
         p += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(p / NyNz);
        const int rem = (int)(p - (long long)ix * NyNz);
        const int iy = rem / f.Nz, iz = rem - (rem / f.Nz) * f.Nz;
        const T px = (T)(ix * dx), py = (T)(iy * dy), pz = (T)(iz * dz);
        T wv[kMaxSites];
#pragma unroll
        for (int g = 0; g < kMaxSites; ++g) wv[g] = g < nv ? wg[(long long)g * f.G + p] : (T)0;
#pragma unroll
        for (int i = 0; i < AT; ++i) {
            if (i < na) {
                const T ex = px - ax[i], ey = py - ay[i], ez = pz - az[i];
                T d2 = ex * ex + ey * ey + ez * ez;
                d2 = d2 < (T)1e-8 ? (T)1e-8 : d2;
                const T id2 = (T)1 / d2;
                const T id3 = id2 * ((T)1 / sqrt(d2));
                T fac = (T)0;
#pragma unroll
                for (int g = 0; g < kMaxSites; ++g) {
                    if (g < nv) {
                        const T q = s2[i][g] * id2;
                        const T s6 = q * q * q;
                        fac += wv[g] * ((e48[i][g] * s6 * s6 - e24[i][g] * s6) * id2 +
                                        aq[i] * (T)site_q[g] * id3);
                    }
                }
                acc[3 * i] += fac * ex;
                acc[3 * i + 1] += fac * ey;
                acc[3 * i + 2] += fac * ez;
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 3 * AT; ++k) {
        double v = (double)acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3 * na) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w][threadIdx.x];
        const int i = threadIdx.x / 3, comp = threadIdx.x - 3 * (threadIdx.x / 3);
        partials[((long long)(a0 + i) * 3 + comp) * gridDim.x + blockIdx.x] = sum;
    }
}

static __global__ void k_sum_rows(const double *partials, int rows, int cols, double *out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < cols; ++c) s += partials[(long long)r * cols + c];
        out[r] = s;
    }
}

template <typename T>
cudaError_t launch_sfe_gradient(const Fields<T> &f, int slot, int kind, int order, const double *rho_dV,
                                const double *atoms, int n_atoms, const double *site_sig,
                                const double *site_eps, const double *site_q, const double *origin,
                                const double *spacing, double *partials, double *out, cudaStream_t s) {
    k_grad_weights<T><<<152 * 8, 256, 0, s>>>(f, slot, kind, order, rho_dV);
    constexpr int AT = GradTile<T>::v;
    const int nblk = kGradBlocks;
    const dim3 grid(nblk, (n_atoms + AT - 1) / AT);
    k_sfe_gradient<T><<<grid, 256, 0, s>>>(f, atoms, n_atoms, site_sig, site_eps, site_q, origin[0],
                                           origin[1], origin[2], spacing[0], spacing[1], spacing[2],
                                           partials);
    k_sum_rows<<<(3 * n_atoms + 255) / 256, 256, 0, s>>>(partials, 3 * n_atoms, nblk, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ split plane passes
// The plane passes in two kernels each, for x planes [x0, x1), so that the streaming
// element work of one half of the planes can run beside the transforms of the other:
//   fwd_elem : MDIIS update, closure, c^sr - c^sr_a (refresh of the iterate offset)
//              -> the spectrum buffer (real layout)
//   fft_fwd  : z and y transforms of those planes, in place (spectrum layout)
//   fft_inv  : inverse y and z transforms, in place back to the real layout
//   inv_elem : residual, Y, Gram-row partial sums
// The spectrum buffer holds n_v * Nx * Ny * Nz reals, so plane (site, x) occupies the same
// bytes in both layouts and each transform block works in place on its own plane. FP32,
// whole planes, integer grid and Nz/2 = LZ in {64, 128}.

// Four consecutive reals (two packed complex elements) per thread and step.
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

template <int MAXH>
__global__ void __launch_bounds__(256) k_fwd_elem(Fields<float> f, int x0, int x1) {
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    __shared__ float coef[MAXH], dcoef[MAXH];
    __shared__ long long slot_off[MAXH];
    const long long ring = (long long)f.nv * f.G;
    const int upd_n = ctl->upd_n;
    if (threadIdx.x < MAXH) {
        const int i = threadIdx.x;
        coef[i] = i < upd_n ? (float)ctl->upd_coef[i] : 0.f;
        dcoef[i] = i < upd_n ? (float)ctl->upd_dcoef[i] : 0.f;
        slot_off[i] = i < upd_n ? (long long)ctl->upd_slot[i] * ring : 0;
    }
    const int do_update = ctl->do_update, upd_r = ctl->upd_r;
    const int stage = ctl->stage, kind = ctl->stage_kind[stage], order = ctl->stage_order[stage];
    const int anchor = ctl->anchor_valid, refresh = ctl->refresh;
    __syncthreads();
    const int g = blockIdx.y;
    const long long plane = (long long)f.Ny * f.Nz;
    const long long base = (long long)g * f.G + (long long)x0 * plane;
    const long long nq = (long long)(x1 - x0) * plane / 4;
    float *cs = reinterpret_cast<float *>(f.spec);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        const long long o = base + 4 * q;
        float4 t;
        if (do_update) {
            t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < MAXH; ++i) {
                if (i < upd_n) {
                    const float4 y = ld4(f.X + slot_off[i] + o);
                    const float c = coef[i];
                    t.x += c * y.x;
                    t.y += c * y.y;
                    t.z += c * y.z;
                    t.w += c * y.w;
                }
            }
            if (upd_r)
                for (int i = 0; i < upd_n; ++i) {
                    const float4 r = ld4(f.R + slot_off[i] + o);
                    const float d = dcoef[i];
                    t.x += d * r.x;
                    t.y += d * r.y;
                    t.z += d * r.z;
                    t.w += d * r.w;
                }
        } else {
            t = ld4(f.Tc + o);
        }
        const float4 w = ld4(f.w + o);
        // c^sr - c^sr_a = (g - g_a) - delta (g_a = 1 before the first anchor), as in plane_fwd
        float4 a = make_float4(1.f, 1.f, 1.f, 1.f);
        if (anchor) a = ld4(f.g_a + o);
        const float4 dv = make_float4(w.x + t.x, w.y + t.y, w.z + t.z, w.w + t.w);
        const float4 gv = make_float4(closure_g(dv.x, kind, order), closure_g(dv.y, kind, order),
                                      closure_g(dv.z, kind, order), closure_g(dv.w, kind, order));
        if (refresh) {
            float4 t0 = ld4(f.tau0 + o);
            t0 = make_float4(t0.x + t.x, t0.y + t.y, t0.z + t.z, t0.w + t.w);
            *reinterpret_cast<float4 *>(f.tau0 + o) = t0;
            *reinterpret_cast<float4 *>(f.w + o) = dv;
            *reinterpret_cast<float4 *>(f.g_a + o) = gv;
            *reinterpret_cast<float4 *>(f.Tc + o) = make_float4(0.f, 0.f, 0.f, 0.f);
            if (do_update)
                for (int i = 0; i < upd_n; ++i) {
                    float *yb = f.X + slot_off[i] + o;
                    const float4 y = ld4(yb);
                    *reinterpret_cast<float4 *>(yb) = make_float4(y.x - t.x, y.y - t.y, y.z - t.z, y.w - t.w);
                }
        } else if (do_update) {
            *reinterpret_cast<float4 *>(f.Tc + o) = t;
        }
        *reinterpret_cast<float4 *>(cs + o) = make_float4((gv.x - a.x) - t.x, (gv.y - a.y) - t.y,
                                                          (gv.z - a.z) - t.z, (gv.w - a.w) - t.w);
    }
}

template <int MAXH>
__global__ void __launch_bounds__(256) k_inv_elem(Fields<float> f, int x0, int x1, int part0, int nparts) {
    const Ctrl *ctl = f.ctrl;
    if (ctl->status != kRunning) return;
    __shared__ long long hoff[MAXH];
    __shared__ double red[(MAXH + 1) * 8];
    const long long ring = (long long)f.nv * f.G;
    const int hist_n = ctl->hist_n;
    if (threadIdx.x < MAXH) hoff[threadIdx.x] = threadIdx.x < hist_n ? (long long)ctl->hist_slot[threadIdx.x] * ring : 0;
    const int stage = ctl->stage, kind = ctl->stage_kind[stage], order = ctl->stage_order[stage];
    const int anchor = ctl->anchor_valid, refresh = ctl->refresh;
    const float eta = (float)ctl->eta;
    const long long cur = (long long)ctl->cur * ring;
    __syncthreads();
    const int g = blockIdx.y;
    const long long plane = (long long)f.Ny * f.Nz;
    const long long base = (long long)g * f.G + (long long)x0 * plane;
    const long long nq = (long long)(x1 - x0) * plane / 4;
    const float *dh = reinterpret_cast<const float *>(f.spec);
    GramAcc<float> acc[MAXH + 1];
#pragma unroll
    for (int i = 0; i <= MAXH; ++i) acc[i].zero();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        const long long o = base + 4 * q;
        const float4 t = ld4(f.Tc + o), w = ld4(f.w + o), hc = ld4(dh + o);
        float4 ha = make_float4(0.f, 0.f, 0.f, 0.f);
        if (anchor) ha = ld4(f.h_a + o);
        float4 qv[MAXH];
#pragma unroll
        for (int i = 0; i < MAXH; ++i)
            if (i < hist_n) qv[i] = ld4(f.R + hoff[i] + o);
        const float g0 = closure_g(w.x + t.x, kind, order), g1 = closure_g(w.y + t.y, kind, order);
        const float g2 = closure_g(w.z + t.z, kind, order), g3 = closure_g(w.w + t.w, kind, order);
        // R = h + 1 - g (Eq. 33) with h = h_a + dh, (h_a - g) first as in plane_inv
        float4 r;
        if (anchor) {
            r.x = ((ha.x - g0) + 1.f) + hc.x;
            r.y = ((ha.y - g1) + 1.f) + hc.y;
            r.z = ((ha.z - g2) + 1.f) + hc.z;
            r.w = ((ha.w - g3) + 1.f) + hc.w;
        } else {
            r.x = (hc.x - g0) + 1.f;
            r.y = (hc.y - g1) + 1.f;
            r.z = (hc.z - g2) + 1.f;
            r.w = (hc.w - g3) + 1.f;
        }
        acc[0].add(r.x, r.x);
        acc[0].add(r.y, r.y);
        acc[0].add(r.z, r.z);
        acc[0].add(r.w, r.w);
#pragma unroll
        for (int i = 0; i < MAXH; ++i)
            if (i < hist_n) {
                acc[i + 1].add(r.x, qv[i].x);
                acc[i + 1].add(r.y, qv[i].y);
                acc[i + 1].add(r.z, qv[i].z);
                acc[i + 1].add(r.w, qv[i].w);
            }
        if (refresh)
            *reinterpret_cast<float4 *>(f.h_a + o) =
                make_float4(ha.x + hc.x, ha.y + hc.y, ha.z + hc.z, ha.w + hc.w);
        *reinterpret_cast<float4 *>(f.R + cur + o) = r;
        *reinterpret_cast<float4 *>(f.X + cur + o) =
            make_float4(t.x + eta * r.x, t.y + eta * r.y, t.z + eta * r.z, t.w + eta * r.w);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i <= MAXH; ++i)
        if (i <= hist_n) {
            acc[i].warp_reduce();
            if (lane == 0) red[i * 8 + warp] = acc[i].value();
        }
    __syncthreads();
    if (threadIdx.x <= hist_n) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += red[threadIdx.x * 8 + k];
        const int blk = part0 + blockIdx.y * gridDim.x + blockIdx.x;
        f.partials[(long long)threadIdx.x * nparts + blk] = s;
    }
}

// z and y transforms of planes [x0, x1) in place: the block's plane is read as packed rows
// (real layout), transformed, and written back in the spectrum layout.
template <int LZ>
__global__ void __launch_bounds__(kThreadsPlane, RISM_MINBLOCKS_F32) k_fft_fwd(Fields<float> f, int x0) {
    typedef float2 C;
    if (f.ctrl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = LZ, pitch = f.pitch;
    C *tw_h = buf + (long)Ny * pitch;
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];
    const int x = x0 + blockIdx.x, gam = blockIdx.y;
    C *plane = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;     // same bytes in both layouts
    __syncthreads();
    constexpr int RW = 256 / LZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r0 = warp * RW; r0 < Ny; r0 += nw * RW) {
        const int nr = min(RW, Ny - r0);
        for (int e = lane; e < nr * Kz; e += 32) {            // packed row element m of row r0 + e / Kz
            const int y = e / Kz, m = e - y * Kz;
            cp_async8(&buf[(r0 + y) * pitch + m], &plane[(long long)(r0 + y) * Kz + m]);
        }
        cp_async_wait();
        __syncwarp();
        fft_rows_warp<C, LZ>(buf + (long)r0 * pitch, nr, pitch, tw_h, -1, lane);
        r2c_rows(buf + (long)r0 * pitch, nr, Kz, pitch, tw_z, f.dKz1h, lane, 32, true);
        __syncwarp();
    }
    __syncthreads();
    fft_smem<C, MaxC<float>::v>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, -1);
    for (int k = threadIdx.x; k <= Ny / 2; k += blockDim.x) {     // split the real columns
        const int k2 = k == 0 ? 0 : Ny - k;
        const C P = buf[k * pitch], Q = buf[k2 * pitch];
        buf[k * pitch] = cscale(cadd(P, cconj(Q)), 0.5f);
        buf[k * pitch + Kz] = cscale(cmuli(csub(P, cconj(Q)), -1), 0.5f);
        if (k2 != k) {
            buf[k2 * pitch] = cscale(cadd(Q, cconj(P)), 0.5f);
            buf[k2 * pitch + Kz] = cscale(cmuli(csub(Q, cconj(P)), -1), 0.5f);
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Ny * Kz; idx += blockDim.x) {
        const int y = idx / Kz, k = idx - y * Kz;
        plane[idx] = buf[y * pitch + k];
    }
    C *dn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) dn[y] = buf[y * pitch + Kz];
}

template <int LZ>
__global__ void __launch_bounds__(kThreadsPlane, RISM_MINBLOCKS_F32) k_fft_inv(Fields<float> f, int x0) {
    typedef float2 C;
    if (f.ctrl->status != kRunning) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int Ny = f.Ny, Kz = LZ, pitch = f.pitch;
    C *tw_h = buf + (long)Ny * pitch;
    C *tw_y = tw_h + Kz;
    C *tw_z = tw_y + Ny;
    for (int i = threadIdx.x; i < Kz; i += blockDim.x) tw_h[i] = f.tw_h[i];
    for (int i = threadIdx.x; i < Ny; i += blockDim.x) tw_y[i] = f.tw_y[i];
    for (int i = threadIdx.x; i <= Kz; i += blockDim.x) tw_z[i] = f.tw_z[i];
    const int x = x0 + blockIdx.x, gam = blockIdx.y;
    C *plane = f.spec + ((long long)gam * f.Nx + x) * Ny * Kz;
    for (int idx = threadIdx.x; idx < Ny * Kz; idx += blockDim.x) {
        const int y = idx / Kz, k = idx - y * Kz;
        cp_async8(&buf[y * pitch + k], &plane[idx]);
    }
    const C *sn = f.spec_nyq + ((long long)gam * f.Nx + x) * Ny;
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) cp_async8(&buf[y * pitch + Kz], &sn[y]);
    cp_async_wait();
    __syncthreads();
    for (int y = threadIdx.x; y < Ny; y += blockDim.x) {           // real columns as one
        const C A0 = buf[y * pitch], B0 = buf[y * pitch + Kz];
        buf[y * pitch] = cmk(A0.x - B0.y, A0.y + B0.x);
    }
    __syncthreads();
    fft_smem<C, MaxC<float>::v>(buf, f.py, pitch, Kz, 1, f.chunk_cols_fwd, tw_y, +1);
    constexpr int RW = 256 / LZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r0 = warp * RW; r0 < Ny; r0 += nw * RW) {
        const int nr = min(RW, Ny - r0);
        c2r_rows(buf + (long)r0 * pitch, nr, Kz, pitch, tw_z, f.dKz1h, lane, 32, true);
        __syncwarp();
        fft_rows_warp<C, LZ>(buf + (long)r0 * pitch, nr, pitch, tw_h, +1, lane);
        for (int e = lane; e < nr * Kz; e += 32) {
            const int y = e / Kz, m = e - y * Kz;
            plane[(long long)(r0 + y) * Kz + m] = buf[(r0 + y) * pitch + m];
        }
    }
}

// ------------------------------------------------------------------ launchers
template <typename T> size_t plane_smem_bytes(const Fields<T> &f) {
    typedef typename Cx<T>::type C;
    return sizeof(C) * ((size_t)f.slab_rows * f.pitch + f.Kz + f.Ny + f.Kz + 1 + f.Kz +
                        (f.cl > 1 ? f.slab_rows : 0)) +
           (kMaxHist + 1) * (kThreadsPlane / 32) * sizeof(double) + 16;
}
template <typename T> size_t pencil_smem_bytes(const Fields<T> &f) {
    typedef typename Cx<T>::type C;
    return sizeof(C) * ((size_t)f.nv * f.W * f.pencil_pitch + f.Nx);
}
template <typename T> size_t ypencil_smem_bytes(const Fields<T> &f) {
    typedef typename Cx<T>::type C;
    return sizeof(C) * ((size_t)f.nv * f.Wy * f.ypitch + f.Ny);
}

// The dynamic shared memory cap is a property of the kernel function, shared by every
// context in the process: each kernel gets the device's opt-in maximum (occupancy follows
// the amount a launch asks for, not the cap), so contexts of different grid sizes coexist.
// The size check of a context is on its own needs against that maximum.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const size_t cap = (size_t)optin - fa.sharedSizeBytes;   // less the kernel's static arrays
    if (bytes > cap) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

// z-row length classes with a specialised plane kernel (FP32 only; FP64 and other lengths
// take the block-wide form). The specialised kernels compile only the power-of-two
// transforms, so every y transform they run (whole columns of Ny, or the local length of
// a cluster's row chunks) must be one of those too.
inline bool p2_length(int L) { return L >= 16 && L <= 256 && (L & (L - 1)) == 0; }
template <typename T> int plane_lz(const Fields<T> &f) {
    if (sizeof(T) != 4 || !(f.Kz == 64 || f.Kz == 128)) return 0;
    if (f.nyc == 1 && !p2_length(f.py.L)) return 0;
    if (f.nyc > 1 && f.cl > 1 && !p2_length(f.pys.L)) return 0;
    return f.Kz;
}

template <typename T, int LZ> cudaError_t prepare_planes(size_t pl) {
    cudaError_t e = set_smem(k_plane_fwd<T, 5, LZ>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_fwd<T, 8, LZ>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_fwd<T, kMaxHist, LZ>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_inv<T, 4, LZ>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_inv<T, 8, LZ>, pl);
    if (e == cudaSuccess) e = set_smem(k_plane_inv<T, kMaxHist, LZ>, pl);
    return e;
}

// The plane kernels (fused and split) are compiled in their own translation units.
template <typename T> cudaError_t prepare_plane_kernels(const Fields<T> &f) {
    const size_t pl = plane_smem_bytes(f);
    cudaError_t e;
    switch (plane_lz(f)) {
        case 64: e = prepare_planes<T, sizeof(T) == 4 ? 64 : 0>(pl); break;
        case 128: e = prepare_planes<T, sizeof(T) == 4 ? 128 : 0>(pl); break;
        default: e = prepare_planes<T, 0>(pl); break;
    }
    if (e == cudaSuccess && split_planes(f)) {
        if constexpr (sizeof(T) == 4) {
            if (f.Kz == 64) {
                e = set_smem(k_fft_fwd<64>, pl);
                if (e == cudaSuccess) e = set_smem(k_fft_inv<64>, pl);
            } else {
                e = set_smem(k_fft_fwd<128>, pl);
                if (e == cudaSuccess) e = set_smem(k_fft_inv<128>, pl);
            }
        }
    }
    return e;
}

// The pencil kernel for the x length: the power-of-two form (FP32 only) or the generic one.
template <typename T> bool pencil_p2(const Fields<T> &f) { return sizeof(T) == 4 && p2_length(f.px.L); }
template <typename T, int NV> cudaError_t prepare_pencil(const Fields<T> &f, size_t pe) {
    if constexpr (sizeof(T) == 4)
        if (pencil_p2(f)) return set_smem(k_pencil<T, NV, true>, pe);
    return set_smem(k_pencil<T, NV, false>, pe);
}
template <typename T, int NV> void pencil_go(const Fields<T> &f, unsigned grid, size_t sm, cudaStream_t s) {
    if constexpr (sizeof(T) == 4)
        if (pencil_p2(f)) {
            k_pencil<T, NV, true><<<grid, kThreadsPencil, sm, s>>>(f);
            return;
        }
    k_pencil<T, NV, false><<<grid, kThreadsPencil, sm, s>>>(f);
}

template <typename T> cudaError_t prepare_kernels(const Fields<T> &f) {
    const size_t pe = pencil_smem_bytes(f);
    cudaError_t e = prepare_plane_kernels(f);
    if (e == cudaSuccess) e = set_smem(k_ypencil<T>, f.nyc > 1 ? ypencil_smem_bytes(f) : 0);
    if (e != cudaSuccess) return e;
    switch (f.nv) {
        case 1: return prepare_pencil<T, 1>(f, pe);
        case 2: return prepare_pencil<T, 2>(f, pe);
        case 3: return prepare_pencil<T, 3>(f, pe);
        case 4: return prepare_pencil<T, 4>(f, pe);
        case 5: return prepare_pencil<T, 5>(f, pe);
        case 6: return prepare_pencil<T, 6>(f, pe);
        case 7: return prepare_pencil<T, 7>(f, pe);
        case 8: return prepare_pencil<T, 8>(f, pe);
        default: return cudaErrorInvalidValue;
    }
}

// Split plane passes (see above): FP32, whole planes, integer grid, Nz/2 in {64, 128}.
template <typename T> bool split_planes(const Fields<T> &f) {
    return f.split && sizeof(T) == 4 && f.nyc == 1 && !f.half && (f.Kz == 64 || f.Kz == 128) && f.Nx >= 2;
}

// Element-kernel blocks per site for one half of the planes (about 4 blocks per SM).
inline int split_elem_blocks(int nv) { return (kSplitBlocks + nv - 1) / nv; }

template <typename T>
cudaError_t launch_split(const Fields<T> &f, int which, int x0, int x1, int part0, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
        const dim3 eg(split_elem_blocks(f.nv), f.nv), pg(x1 - x0, f.nv);
        const size_t sm = plane_smem_bytes(f);
        switch (which) {
            case 0:
                if (f.M <= 5) k_fwd_elem<5><<<eg, 256, 0, s>>>(f, x0, x1);
                else if (f.M <= 8) k_fwd_elem<8><<<eg, 256, 0, s>>>(f, x0, x1);
                else k_fwd_elem<kMaxHist><<<eg, 256, 0, s>>>(f, x0, x1);
                break;
            case 1:
                if (f.Kz == 64) k_fft_fwd<64><<<pg, kThreadsPlane, sm, s>>>(f, x0);
                else k_fft_fwd<128><<<pg, kThreadsPlane, sm, s>>>(f, x0);
                break;
            case 2:
                if (f.Kz == 64) k_fft_inv<64><<<pg, kThreadsPlane, sm, s>>>(f, x0);
                else k_fft_inv<128><<<pg, kThreadsPlane, sm, s>>>(f, x0);
                break;
            default:
                if (f.M <= 5) k_inv_elem<4><<<eg, 256, 0, s>>>(f, x0, x1, part0, f.nparts);
                else if (f.M <= 8) k_inv_elem<8><<<eg, 256, 0, s>>>(f, x0, x1, part0, f.nparts);
                else k_inv_elem<kMaxHist><<<eg, 256, 0, s>>>(f, x0, x1, part0, f.nparts);
                break;
        }
        return cudaGetLastError();
    }
}

template <typename T> cudaError_t launch_ypencil(const Fields<T> &f, int sign, cudaStream_t s) {
    k_ypencil<T><<<f.ytiles_main + f.ytiles_nyq, kThreadsPencil, ypencil_smem_bytes(f), s>>>(f, sign);
    return cudaGetLastError();
}
// A plane kernel launch; with f.cl > 1 the row chunks of each plane are launched as one
// thread-block cluster of f.cl blocks (grid x = Nx * nyc, consecutive blocks of one plane).
template <typename T>
cudaError_t plane_launch(void (*kernel)(Fields<T>), const Fields<T> &f, dim3 grid, size_t sm, cudaStream_t s) {
    if (f.cl > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(kThreadsPlane);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)f.cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, f);
    }
    kernel<<<grid, kThreadsPlane, sm, s>>>(f);
    return cudaGetLastError();
}
template <typename T, int LZ> cudaError_t plane_fwd_lz(const Fields<T> &f, dim3 grid, size_t sm, cudaStream_t s) {
    // the update combines up to M stored pairs
    if (f.M <= 5) return plane_launch<T>(k_plane_fwd<T, 5, LZ>, f, grid, sm, s);
    if (f.M <= 8) return plane_launch<T>(k_plane_fwd<T, 8, LZ>, f, grid, sm, s);
    return plane_launch<T>(k_plane_fwd<T, kMaxHist, LZ>, f, grid, sm, s);
}
template <typename T, int LZ> cudaError_t plane_inv_lz(const Fields<T> &f, dim3 grid, size_t sm, cudaStream_t s) {
    // the Gram row pairs the new residual with at most M - 1 stored ones
    if (f.M <= 5) return plane_launch<T>(k_plane_inv<T, 4, LZ>, f, grid, sm, s);
    if (f.M <= 8) return plane_launch<T>(k_plane_inv<T, 8, LZ>, f, grid, sm, s);
    return plane_launch<T>(k_plane_inv<T, kMaxHist, LZ>, f, grid, sm, s);
}
template <typename T> cudaError_t launch_plane_fwd(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = plane_smem_bytes(f);
    const dim3 grid(f.Nx * f.nyc, f.nv);
    switch (plane_lz(f)) {
        case 64: return plane_fwd_lz<T, sizeof(T) == 4 ? 64 : 0>(f, grid, sm, s);
        case 128: return plane_fwd_lz<T, sizeof(T) == 4 ? 128 : 0>(f, grid, sm, s);
        default: return plane_fwd_lz<T, 0>(f, grid, sm, s);
    }
}
template <typename T> cudaError_t launch_plane_inv(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = plane_smem_bytes(f);
    const dim3 grid(f.Nx * f.nyc, f.nv);
    switch (plane_lz(f)) {
        case 64: return plane_inv_lz<T, sizeof(T) == 4 ? 64 : 0>(f, grid, sm, s);
        case 128: return plane_inv_lz<T, sizeof(T) == 4 ? 128 : 0>(f, grid, sm, s);
        default: return plane_inv_lz<T, 0>(f, grid, sm, s);
    }
}
template <typename T> cudaError_t launch_pencil(const Fields<T> &f, cudaStream_t s) {
    const size_t sm = pencil_smem_bytes(f);
    const unsigned grid = f.tiles_main + f.tiles_nyq;
    switch (f.nv) {
        case 1: pencil_go<T, 1>(f, grid, sm, s); break;
        case 2: pencil_go<T, 2>(f, grid, sm, s); break;
        case 3: pencil_go<T, 3>(f, grid, sm, s); break;
        case 4: pencil_go<T, 4>(f, grid, sm, s); break;
        case 5: pencil_go<T, 5>(f, grid, sm, s); break;
        case 6: pencil_go<T, 6>(f, grid, sm, s); break;
        case 7: pencil_go<T, 7>(f, grid, sm, s); break;
        case 8: pencil_go<T, 8>(f, grid, sm, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_mdiis(const Fields<T> &f, cudaStream_t s) {
    k_mdiis<<<1, kThreadsMdiis, 0, s>>>(f.ctrl, f.partials, f.nparts);
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
    for (int a0 = 0; a0 < n_atoms; a0 += kPhaseChunk) {
        const int na = min(kPhaseChunk, n_atoms - a0);
        k_phase_tables<T><<<152 * 4, 256, 0, s>>>(f, atoms, a0, na, f.phase);
        k_longrange<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(f, atoms, a0, na, f.phase, amp0,
                                                                       a0 > 0);
    }
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_init_guess(const Fields<T> &f, int, cudaStream_t s) {
    k_init_guess<T><<<152 * 8, 256, 0, s>>>(f);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_guess_from_t(const Fields<T> &f, int, const double *src, cudaStream_t s) {
    k_guess_from_t<T><<<152 * 8, 256, 0, s>>>(f, src);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_flatten(const Fields<T> &f, cudaStream_t s) {
    k_flatten<T><<<152 * 8, 256, 0, s>>>(f);
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

// ------------------------------------------------------------------ finite-size correction
// The correction of a charged solute's SFE needs three reductions (the energy of the
// solvent's linear response to the long-range field of Eq. 30 on the box's k lattice with the
// box-sampled Eq. 29 potential, and in infinite space):
//   1. phi~_box = DFT of the grid field phi (three in-place axis passes over a complex copy);
//   2. sum over the half spectrum of w_z Re(Psi conj(phi~_box)) S(|k|), with Psi = beta Phi~ / dV
//      and S(k) = sum_g rho_g q_g sum_a q_a X_ag(k) from the charge row of the table;
//   3. the radial integral of (4 pi C)^2 S(k) P(k) / (k^2 (k^2 + 1)^2), P(k) = sum_ab q_a q_b
//      sin(k R_ab) / (k R_ab) (the orientation average of |sum_a q_a exp(-i k.R_a)|^2).

// a[p] = phi[p] + 0i over the grid
template <typename T>
__global__ void k_lr_load_phi(Fields<T> f, typename Cx<T>::type *a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < f.G; i += (long long)gridDim.x * blockDim.x)
        a[i] = cmk(f.phi[i], (T)0);
}

// One axis of the forward 3D DFT of a[Nx][Ny][Nz] in place. A block loads W lines of length
// L (z: W consecutive (x, y) lines; y and x: the lines at W consecutive z of one x or one y
// plane, so that each row of the tile is W contiguous values), transforms them in shared
// memory with the engine of the plane passes and writes them back.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_dft_axis(typename Cx<T>::type *a, int Nx, int Ny, int Nz, int axis,
                                                     FftPlan p, int W, int pitch, int chunk) {
    typedef typename Cx<T>::type C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *buf = reinterpret_cast<C *>(smraw);
    const int L = p.L;
    C *tw = buf + (long)W * pitch;
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)m / (double)L, &sn, &cs);
        tw[m] = cmk((T)cs, (T)sn);
    }
    long long base;
    long long estride;
    int nw;
    if (axis == 2) {                                   // lines (x, y), contiguous
        const long long line0 = (long long)blockIdx.x * W;
        nw = (int)min((long long)W, (long long)Nx * Ny - line0);
        base = line0 * Nz;
        estride = 1;
    } else {
        const int zt = (Nz + W - 1) / W;
        const int z0 = (blockIdx.x % zt) * W, o = blockIdx.x / zt;
        nw = min(W, Nz - z0);
        base = axis == 1 ? (long long)o * Ny * Nz + z0 : (long long)o * Nz + z0;
        estride = axis == 1 ? (long long)Nz : (long long)Ny * Nz;
    }
    const long long wstride = axis == 2 ? (long long)Nz : 1;
    for (int idx = threadIdx.x; idx < W * L; idx += blockDim.x) {
        int e, w;
        if (axis == 2) {
            w = idx / L;
            e = idx - w * L;
        } else {
            e = idx / W;
            w = idx - e * W;
        }
        if (w < nw) buf[w * pitch + e] = a[base + w * wstride + e * estride];
    }
    __syncthreads();
    fft_smem<C, MaxC<T>::v>(buf, p, 1, W, pitch, chunk, tw, -1);
    for (int idx = threadIdx.x; idx < W * L; idx += blockDim.x) {
        int e, w;
        if (axis == 2) {
            w = idx / L;
            e = idx - w * L;
        } else {
            e = idx / W;
            w = idx - e * W;
        }
        if (w < nw) a[base + w * wstride + e * estride] = buf[w * pitch + e];
    }
}

// S(|k|) from the charge row of the interpolation table (continued as S(k_1) (k / k_1)^2
// below the first table point k_1 = dk); rq[g] = rho_g q_g.
template <typename T>
__device__ double lr_charge_response(const Fields<T> &f, const double *rq, double kmag) {
    const int nv = f.nv;
    const int rowlen = (nv + 1) * nv;
    double xk = kmag * f.inv_dk, scale = 1.0;
    if (xk < 1.0) {
        scale = xk * xk;
        xk = 1.0;
    }
    int j = (int)floor(xk);
    if (j > f.nk - 2) j = f.nk - 2;
    double w = xk - (double)j;
    w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
    const T *A0 = f.table + (long long)j * rowlen + nv * nv, *A1 = A0 + rowlen;
    double s = 0.0;
    for (int g = 0; g < nv; ++g) s += rq[g] * ((double)A0[g] * (1.0 - w) + (double)A1[g] * w);
    return -(double)f.G * s * scale;             // the table holds -Q_g / G
}

struct LrSites {
    double rq[kMaxSites];
};

// part[block] = sum over the block's half-spectrum points of w_z Re(Psi conj(F)) S(|k|),
// F = DFT(phi) (full complex array [Nx][Ny][Nz]).
template <typename T>
__global__ void __launch_bounds__(256) k_lr_lattice(Fields<T> f, const typename Cx<T>::type *F, LrSites sites,
                                                    double *part) {
    __shared__ double red[8];
    const int Nx = f.Nx, Ny = f.Ny, Nz = f.Nz, Kz = f.Kz;
    const long long npts = (long long)Nx * Ny * (Kz + 1);
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(i % (Kz + 1));
        const long long xy = i / (Kz + 1);
        const int y = (int)(xy % Ny), x = (int)(xy / Ny);
        typename Cx<T>::type psi;
        if (kz < Kz) psi = f.psi[xy * Kz + kz];
        else psi = f.psi_nyq[xy];
        if (psi.x == (T)0 && psi.y == (T)0) continue;
        const typename Cx<T>::type Fk = F[xy * Nz + kz];
        const double kx = f.ks[0] * (double)signed_index(x, Nx), ky = f.ks[1] * (double)signed_index(y, Ny);
        const double kzv = f.ks[2] * (double)kz;
        const double S = lr_charge_response(f, sites.rq, sqrt(kx * kx + ky * ky + kzv * kzv));
        const double wz = (kz == 0 || 2 * kz == Nz) ? 1.0 : 2.0;
        acc += wz * ((double)psi.x * (double)Fk.x + (double)psi.y * (double)Fk.y) * S;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// pairs[c][i] = sum over the atom pairs (a, b > a) with a in chunk c of q_a q_b
// sin(k_i R_ab) / (k_i R_ab), k_i = i dk (the i = 0 value is the limit q_a q_b); atoms
// [n][kAtomStride] (x, y, z, q, ...). A thread takes kLrRun consecutive k_i and, per pair,
// starts sin(i x) at its first two indices with sincos and continues with the recurrence
// sin((i + 1) x) = 2 cos(x) sin(i x) - sin((i - 1) x), x = dk R_ab.
constexpr int kLrRun = 16;
static __global__ void __launch_bounds__(256) k_lr_pairs(const double *atoms, int n, int rows_per_chunk, double dk, int nq,
                                                  double *pairs) {
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * kLrRun;
    if (i0 >= nq) return;
    const int c = blockIdx.y;
    const int a0 = c * rows_per_chunk, a1 = min(n, a0 + rows_per_chunk);
    double acc[kLrRun];
#pragma unroll
    for (int j = 0; j < kLrRun; ++j) acc[j] = 0.0;
    double acc0 = 0.0;                                 // the k = 0 limit
    for (int a = a0; a < a1; ++a) {
        const double *A = atoms + (size_t)a * kAtomStride;
        for (int b = a + 1; b < n; ++b) {
            const double *B = atoms + (size_t)b * kAtomStride;
            const double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
            const double x = dk * sqrt(dx * dx + dy * dy + dz * dz);
            const double qq = A[3] * B[3];
            acc0 += qq;
            if (!(x > 1e-300)) continue;
            const double cp = qq / x;
            double sc = sin((double)i0 * x), sp = sin((double)(i0 - 1) * x);
            const double cx = cos(x);
#pragma unroll
            for (int j = 0; j < kLrRun; ++j) {
                acc[j] += cp * sc;
                const double sn = 2.0 * cx * sc - sp;
                sp = sc;
                sc = sn;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kLrRun; ++j) {
        const int i = i0 + j;
        if (i < nq) pairs[(size_t)c * nq + i] = i == 0 ? acc0 : acc[j] / (double)i;
    }
}

// part[block] = sum over the block's quadrature points of the trapezoid weight times
// (4 pi C)^2 S(k) P(k) / (k^2 (k^2 + 1)^2), P(k) = sum_a q_a^2 + 2 sum_c pairs[c][i]; the
// k = 0 point takes its limit S(k_1) / k_1^2 P(0) (4 pi C)^2.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_integral(Fields<T> f, LrSites sites, const double *pairs, int chunks,
                                                     int nq, double k_max, double q2, double c4, double *part) {
    __shared__ double red[8];
    const double dk = k_max / (double)(nq - 1);
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        double P = 0.0;
        for (int c = 0; c < chunks; ++c) P += pairs[(size_t)c * nq + i];
        P = q2 + 2.0 * P;
        double v;
        if (i == 0) {
            const double k1 = 1.0 / f.inv_dk;
            v = c4 * lr_charge_response(f, sites.rq, k1) / (k1 * k1) * P;
        } else {
            const double k = dk * (double)i, k2 = k * k;
            v = c4 * lr_charge_response(f, sites.rq, k) * P / (k2 * (k2 + 1.0) * (k2 + 1.0));
        }
        acc += (i == 0 || i == nq - 1 ? 0.5 : 1.0) * dk * v;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
cudaError_t launch_lr_parts(const Fields<T> &f, typename Cx<T>::type *scratch, const FftPlan *plans,
                            const double *rq, const double *atoms, int n_atoms, double k_max, int nq, int chunks,
                            double *pairs, double *lat_part, int lat_blocks, double *int_part, int int_blocks,
                            double c4, double q2, cudaStream_t s) {
    typedef typename Cx<T>::type C;
    k_lr_load_phi<T><<<152 * 8, 256, 0, s>>>(f, scratch);
    cudaError_t e = cudaGetLastError();
    const int n[3] = {f.Nx, f.Ny, f.Nz};
    for (int axis = 2; axis >= 0 && e == cudaSuccess; --axis) {
        const FftPlan &p = plans[axis];
        const int W = 8, pitch = p.L + 1;
        int chunk = 1 << 30;
        for (int st = 0; st < p.nst; ++st) {
            const int c = 256 * (MaxC<T>::v / p.radix[st]) / (p.L / p.radix[st]);
            chunk = c < chunk ? c : chunk;
        }
        const size_t smem = sizeof(C) * ((size_t)W * pitch + p.L);
        e = cudaFuncSetAttribute(k_lr_dft_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) break;
        const long long blocks = axis == 2 ? ((long long)n[0] * n[1] + W - 1) / W
                                           : (long long)(axis == 1 ? n[0] : n[1]) * ((n[2] + W - 1) / W);
        k_lr_dft_axis<T><<<(unsigned)blocks, 256, smem, s>>>(scratch, n[0], n[1], n[2], axis, p, W, pitch, chunk);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    LrSites sites;
    for (int g = 0; g < kMaxSites; ++g) sites.rq[g] = g < f.nv ? rq[g] : 0.0;
    k_lr_lattice<T><<<lat_blocks, 256, 0, s>>>(f, scratch, sites, lat_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rows = (n_atoms + chunks - 1) / chunks;
    if (n_atoms > 1) {
        const unsigned kb = (unsigned)((nq + 256 * kLrRun - 1) / (256 * kLrRun));
        k_lr_pairs<<<dim3(kb, (unsigned)chunks), 256, 0, s>>>(atoms, n_atoms, rows, k_max / (double)(nq - 1), nq, pairs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        if ((e = cudaMemsetAsync(pairs, 0, sizeof(double) * (size_t)chunks * nq, s)) != cudaSuccess) return e;
    }
    k_lr_integral<T><<<int_blocks, 256, 0, s>>>(f, sites, pairs, chunks, nq, k_max, q2, c4, int_part);
    return cudaGetLastError();
}

// Explicit instantiations, in two groups compiled in separate translation units: the plane
// kernels (fused and split) and everything else.
#define RISM_INSTANTIATE_PLANES(T)                                                              \
    template size_t plane_smem_bytes<T>(const Fields<T> &);                                      \
    template cudaError_t prepare_plane_kernels<T>(const Fields<T> &);                            \
    template cudaError_t launch_plane_fwd<T>(const Fields<T> &, cudaStream_t);                   \
    template cudaError_t launch_plane_inv<T>(const Fields<T> &, cudaStream_t);                   \
    template bool split_planes<T>(const Fields<T> &);                                            \
    template cudaError_t launch_split<T>(const Fields<T> &, int, int, int, int, cudaStream_t);

#define RISM_EXTERN_PLANES(T)                                                                   \
    extern template size_t plane_smem_bytes<T>(const Fields<T> &);                               \
    extern template cudaError_t prepare_plane_kernels<T>(const Fields<T> &);                     \
    extern template bool split_planes<T>(const Fields<T> &);

#define RISM_INSTANTIATE_REST(T)                                                                \
    template cudaError_t prepare_kernels<T>(const Fields<T> &);                                  \
    template size_t pencil_smem_bytes<T>(const Fields<T> &);                                     \
    template cudaError_t launch_ypencil<T>(const Fields<T> &, int, cudaStream_t);                \
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
    template cudaError_t launch_flatten<T>(const Fields<T> &, cudaStream_t);                     \
    template cudaError_t launch_get_field<T>(const Fields<T> &, int, int, int, int, double *,   \
                                             cudaStream_t);                                     \
    template cudaError_t launch_sfe<T>(const Fields<T> &, int, int, int, int, int, double *,    \
                                       int, cudaStream_t);                                     \
    template cudaError_t launch_sfe_gradient<T>(const Fields<T> &, int, int, int, const double *, \
                                                const double *, int, const double *,           \
                                                const double *, const double *, const double *, \
                                                const double *, double *, double *, cudaStream_t);    \
    template cudaError_t launch_guess_crop<T>(const Fields<T> &, int, int, const int *, int, float *,  \
                                              const float *, cudaStream_t);                    \
    template cudaError_t launch_lr_parts<T>(const Fields<T> &, typename Cx<T>::type *, const FftPlan *, \
                                            const double *, const double *, int, double, int, int, \
                                            double *, double *, int, double *, int, double, double, \
                                            cudaStream_t);

}  // namespace rism
