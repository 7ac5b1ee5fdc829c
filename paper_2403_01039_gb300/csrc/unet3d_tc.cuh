// BF16 form of the U-Net: 3x3x3 convolutions as implicit GEMMs on the fifth-generation
// tensor cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in tensor
// memory) and the channels-last element kernels around them.
//
// Activations are BF16, channels-last: voxel p of an n^3 volume holds its channels at
// a[p * ld + off + c] (ld, off multiples of 8, so every 8 channels are one 16-byte chunk).
//
// Operand layouts (no swizzle). A tcgen05 shared-memory operand is a grid of "core
// matrices", each 8 rows of 16 contiguous bytes; the descriptor gives the start address,
// the byte distance between core matrices along K (leading byte offset) and along M or N
// (stride byte offset). K-major: a row holds 8 consecutive K values of one M/N index.
// MN-major: a row holds 8 consecutive M/N values of one K index.
//
// Convolution tile: one CTA computes TX x-planes x 16 y x 8 z output voxels; one MMA row
// block (M = 128) is one x-plane of the tile, M index m = 8 * y_local + z_local. The input
// halo of the tile, for 8 channels at a time, is stored [x][y][z] with 16 bytes per voxel,
// so the 8 voxels z..z+7 of one (x, y) are one core matrix, the y rows are 160 bytes apart,
// and a tap (dx, dy, dz) of the 3x3x3 stencil is only a different start address: the
// stencil needs no im2col copy.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace tc {

constexpr int kHY = 18, kHZ = 10;                 // halo extent in y and z (16 + 2, 8 + 2)
constexpr int kRowBytes = kHZ * 16;                // one halo y row of 8 channels
constexpr int kTimeoutNs = 1000000000;             // bound of every wait on a barrier (1 s)

// status codes written by the kernels (first failure wins)
constexpr int kErrWaitWeights = 1, kErrWaitMma = 2;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);     // version bits 46-48 = 0b001
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

// Wait for the phase with the given parity to complete; false after kTimeoutNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    const uint32_t a = smem_u32(b);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            const uint64_t t = globaltimer();
            if (it == 0) t0 = t;
            else if (t - t0 > (uint64_t)kTimeoutNs) return false;
        }
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion
// counted on the barrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 fills zeros without reading
__device__ __forceinline__ void cp16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp-wide)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr uint32_t tmem_cols(int need) {
    return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : need <= 256 ? 256u : 512u;
}

// ------------------------------------------------------------------ shared-memory plans
// Forward / data-gradient convolution: halo of 16 channels (two 8-channel halves) then the
// 16-channel slice of the weights for all 27 taps.
__host__ __device__ constexpr uint32_t fwd_half_bytes(int tx) { return (uint32_t)(tx + 2) * kHY * kRowBytes + 64; }
__host__ __device__ constexpr uint32_t fwd_w_bytes(int cout) { return 27u * 2u * (uint32_t)cout * 16u; }
__host__ __device__ constexpr uint32_t fwd_smem(int tx, int cout) { return 2 * fwd_half_bytes(tx) + fwd_w_bytes(cout); }

// Weight gradient: the output-gradient tile [cout/8][tx][16][8] x 16 B, padded so that the
// 16 row blocks of an M = 128 operand stay inside the CTA's shared memory (rows beyond cout
// read other data and give accumulator rows that are never read), then the input halo of
// all cin channels.
__host__ __device__ constexpr uint32_t wg_gy_bytes(int tx, int cout) { return (uint32_t)cout / 8u * (uint32_t)tx * 2048u; }
__host__ __device__ constexpr uint32_t wg_cb_bytes(int tx) { return (uint32_t)(tx + 2) * kHY * kRowBytes + 64; }
__host__ __device__ constexpr uint32_t wg_smem(int tx, int cin, int cout) {
    return (wg_gy_bytes(tx, cout) + (uint32_t)cin / 8u * wg_cb_bytes(tx)) > 16u * (uint32_t)tx * 2048u
               ? wg_gy_bytes(tx, cout) + (uint32_t)cin / 8u * wg_cb_bytes(tx)
               : 16u * (uint32_t)tx * 2048u;
}

struct ConvArgs {
    const __nv_bfloat16 *x;     // input view: x[p * ldx + xoff + c], c < cin
    int ldx, xoff, cin;
    const __nv_bfloat16 *w;     // prepared weights [cin/16][27][2][cout/8][8][8]
    const float *bias;          // [cout] or null
    __nv_bfloat16 *y;           // output view: y[p * ldy + yoff + o], o < cout
    int ldy, yoff, cout;
    int n, relu;
    int *status;
};

// y = conv3x3x3(x) (+ bias, ReLU). Block of 128 threads; thread 0 issues the MMAs.
template <int TX>
__global__ void __launch_bounds__(128) k_conv3_tc(ConvArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[2];           // 0: weight slice landed, 1: MMAs done
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, tyn = (n + 15) >> 4, tzn = (n + 7) >> 3;
    int b = blockIdx.x;
    const int tz = b % tzn;
    b /= tzn;
    const int ty = b % tyn, tx = b / tyn;
    const int x0 = tx * TX, y0 = ty * 16, z0 = tz * 8;
    const uint32_t H = fwd_half_bytes(TX), WB = fwd_w_bytes(a.cout);
    unsigned char *halo = sm, *wsm = sm + 2 * H;
    const uint32_t ncols = tmem_cols(TX * a.cout);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(128, a.cout, 0, 0);
    const long long plane = (long long)n * n;
    const int nk = a.cin >> 4;
    bool ok = true;
    for (int kk = 0; kk < nk; ++kk) {
        if (kk > 0 && !mbar_wait(&bars[1], (uint32_t)(kk - 1) & 1u)) {
            ok = false;
            if (tid == 0) atomicCAS(a.status, 0, kErrWaitMma);
        }
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (tid == 0) {
            mbar_expect_tx(&bars[0], WB);
            bulk_g2s(wsm, a.w + (size_t)kk * (WB / 2), WB, &bars[0]);
        }
        // halo of channels [16 kk, 16 kk + 16): [half][x][y][z] x 16 B
        const int total = 2 * (TX + 2) * kHY * kHZ;
        for (int i = tid; i < total; i += 128) {
            int r = i;
            const int half = r & 1;
            r >>= 1;
            const int zh = r % kHZ;
            r /= kHZ;
            const int yh = r % kHY, xh = r / kHY;
            const int gx = x0 + xh - 1, gy = y0 + yh - 1, gz = z0 + zh - 1;
            const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n;
            const __nv_bfloat16 *src =
                in ? a.x + ((long long)gx * plane + (long long)gy * n + gz) * a.ldx + a.xoff + kk * 16 + half * 8 : a.x;
            cp16(halo + half * H + ((xh * kHY + yh) * kHZ + zh) * 16, src, in ? 16u : 0u);
        }
        cp_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(&bars[0], (uint32_t)kk & 1u)) {
                atomicCAS(a.status, 0, kErrWaitWeights);
                ok = false;
            } else {
                tc_fence_after();
                const uint32_t hb = smem_u32(halo), wb = smem_u32(wsm);
                const uint32_t nb = (uint32_t)a.cout / 8u;
                for (int t = 0; t < TX; ++t)
                    for (int tap = 0; tap < 27; ++tap) {
                        const int da = tap / 9, dd = (tap / 3) % 3, df = tap % 3;
                        const uint32_t aaddr = hb + (uint32_t)(((t + da) * kHY + dd) * kRowBytes + df * 16);
                        const uint64_t ad = sdesc(aaddr, H, kRowBytes);
                        const uint64_t bd = sdesc(wb + (uint32_t)tap * 2u * nb * 128u, nb * 128u, 128u);
                        mma_bf16(tmem + (uint32_t)(t * a.cout), ad, bd, idesc, (kk > 0 || tap > 0) ? 1u : 0u);
                    }
                mma_commit(&bars[1]);
            }
        }
        if (!__syncthreads_and(ok)) { ok = false; break; }
    }
    if (ok && !mbar_wait(&bars[1], (uint32_t)(nk - 1) & 1u)) {
        ok = false;
        if (tid == 0) atomicCAS(a.status, 0, kErrWaitMma);
    }
    tc_fence_after();
    if (__syncthreads_and(ok)) {
        const int m = warp * 32 + lane, yl = m >> 3, zl = m & 7;
        for (int t = 0; t < TX; ++t) {
            const int gx = x0 + t, gy = y0 + yl, gz = z0 + zl;
            const bool in = gx < n && gy < n && gz < n;
            __nv_bfloat16 *dst = a.y + ((long long)gx * plane + (long long)gy * n + gz) * a.ldy + a.yoff;
            for (int c0 = 0; c0 < a.cout; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * a.cout + c0), v);
                if (in) {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float u0 = v[2 * j] + (a.bias ? a.bias[c0 + 2 * j] : 0.f);
                        float u1 = v[2 * j + 1] + (a.bias ? a.bias[c0 + 2 * j + 1] : 0.f);
                        if (a.relu) u0 = fmaxf(u0, 0.f), u1 = fmaxf(u1, 0.f);
                        const __nv_bfloat162 h = __floats2bfloat162_rn(u0, u1);
                        pk[j] = *reinterpret_cast<const uint32_t *>(&h);
                    }
                    reinterpret_cast<uint4 *>(dst + c0)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    reinterpret_cast<uint4 *>(dst + c0)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, ncols);
}

struct WgradArgs {
    const __nv_bfloat16 *x;     // layer input view, cin channels
    int ldx, xoff, cin;
    const __nv_bfloat16 *gy;    // gradient of the layer output (after the ReLU mask), cout channels
    int ldg, goff, cout;
    int n, tiles_per_chunk, taps_per_group;
    float *part;                // [chunk][27][cin][cout]
    int *status;
};

// part[chunk][tap][c][o] = sum over the chunk's output voxels p of gy[p][o] x[p + tap][c].
// D[o][c] (M = 128 rows of o, N = cin) per tap, K = voxels; both operands MN-major.
template <int TX>
__global__ void __launch_bounds__(128) k_conv3_wgrad_tc(WgradArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bars[1];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, tyn = (n + 15) >> 4, tzn = (n + 7) >> 3, txn = (n + TX - 1) / TX;
    const int ntiles = txn * tyn * tzn;
    const int chunk = blockIdx.x, group = blockIdx.y;
    const int tap0 = group * a.taps_per_group, tap1 = min(27, tap0 + a.taps_per_group);
    const int tbeg = chunk * a.tiles_per_chunk, tend = min(ntiles, tbeg + a.tiles_per_chunk);
    const uint32_t GB = wg_gy_bytes(TX, a.cout), CB = wg_cb_bytes(TX);
    unsigned char *gys = sm, *halo = sm + GB;
    const uint32_t ncols = tmem_cols(a.taps_per_group * a.cin);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(128, a.cin, 1, 1);
    const long long plane = (long long)n * n;
    const int ob = a.cout >> 3, cb = a.cin >> 3;
    bool ok = true;
    int issued = 0;
    for (int tile = tbeg; tile < tend; ++tile) {
        if (issued > 0 && !mbar_wait(&bars[0], (uint32_t)(issued - 1) & 1u)) {
            ok = false;
            if (tid == 0) atomicCAS(a.status, 0, kErrWaitMma);
        }
        if (!__syncthreads_and(ok)) { ok = false; break; }
        int b = tile;
        const int tz = b % tzn;
        b /= tzn;
        const int ty = b % tyn, tx = b / tyn;
        const int x0 = tx * TX, y0 = ty * 16, z0 = tz * 8;
        // output-gradient tile: [o-block][t][y][z] x 16 B, zero outside the volume
        const int gtotal = ob * TX * 128;
        for (int i = tid; i < gtotal; i += 128) {
            int r = i;
            const int obk = r % ob;
            r /= ob;
            const int zl = r & 7, yl = (r >> 3) & 15, t = r >> 7;
            const int gx = x0 + t, gyy = y0 + yl, gz = z0 + zl;
            const bool in = gx < n && gyy < n && gz < n;
            const __nv_bfloat16 *src =
                in ? a.gy + ((long long)gx * plane + (long long)gyy * n + gz) * a.ldg + a.goff + obk * 8 : a.gy;
            cp16(gys + (((obk * TX + t) * 16 + yl) * 8 + zl) * 16, src, in ? 16u : 0u);
        }
        // input halo, all cin channels: [c-block][x][y][z] x 16 B
        const int htotal = cb * (TX + 2) * kHY * kHZ;
        for (int i = tid; i < htotal; i += 128) {
            int r = i;
            const int cbk = r % cb;
            r /= cb;
            const int zh = r % kHZ;
            r /= kHZ;
            const int yh = r % kHY, xh = r / kHY;
            const int gx = x0 + xh - 1, gyy = y0 + yh - 1, gz = z0 + zh - 1;
            const bool in = gx >= 0 && gx < n && gyy >= 0 && gyy < n && gz >= 0 && gz < n;
            const __nv_bfloat16 *src =
                in ? a.x + ((long long)gx * plane + (long long)gyy * n + gz) * a.ldx + a.xoff + cbk * 8 : a.x;
            cp16(halo + cbk * CB + ((xh * kHY + yh) * kHZ + zh) * 16, src, in ? 16u : 0u);
        }
        cp_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t gb = smem_u32(gys), hb = smem_u32(halo);
            for (int t = 0; t < TX; ++t)
                for (int tap = tap0; tap < tap1; ++tap) {
                    const int da = tap / 9, dd = (tap / 3) % 3, df = tap % 3;
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint64_t ad = sdesc(gb + (uint32_t)((t * 16 + 2 * ks) * 128), 128u, (uint32_t)TX * 2048u);
                        const uint32_t baddr = hb + (uint32_t)(((t + da) * kHY + 2 * ks + dd) * kRowBytes + df * 16);
                        const uint64_t bd = sdesc(baddr, (uint32_t)kRowBytes, CB);
                        const uint32_t acc = (tile > tbeg || t > 0 || ks > 0) ? 1u : 0u;
                        mma_bf16(tmem + (uint32_t)((tap - tap0) * a.cin), ad, bd, idesc, acc);
                    }
                }
            mma_commit(&bars[0]);
        }
        ++issued;
    }
    if (ok && issued > 0 && !mbar_wait(&bars[0], (uint32_t)(issued - 1) & 1u)) {
        ok = false;
        if (tid == 0) atomicCAS(a.status, 0, kErrWaitMma);
    }
    tc_fence_after();
    if (__syncthreads_and(ok) && warp * 32 < a.cout) {
        const int o = warp * 32 + lane;
        for (int tap = tap0; tap < tap1; ++tap)
            for (int c0 = 0; c0 < a.cin; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((tap - tap0) * a.cin + c0), v);
                if (o < a.cout) {
                    float *dst = a.part + (((long long)chunk * 27 + tap) * a.cin + c0) * a.cout + o;
#pragma unroll
                    for (int j = 0; j < 16; ++j) dst[(long long)j * a.cout] = issued > 0 ? v[j] : 0.f;
                }
            }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, ncols);
}

// gw[o][c][tap] = sum over chunks of part[chunk][tap][c][o], in chunk order.
__global__ void k_wgrad_sum(const float *part, int chunks, int cin, int cout, int cin_real, float *gw) {
    const long long n = (long long)cout * cin_real * 27;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int tap = (int)(i % 27);
        const long long oc = i / 27;
        const int c = (int)(oc % cin_real), o = (int)(oc / cin_real);
        float s = 0.f;
        for (int k = 0; k < chunks; ++k) s += part[(((long long)k * 27 + tap) * cin + c) * cout + o];
        gw[i] = s;
    }
}

// Prepared forward weights from w[o][c][tap] (FP32, cin_real input channels): element
// (o, c, tap) goes to [c/16][tap][(c/8)%2][o/8][o%8][c%8], zero for c >= cin_real.
__global__ void k_prep_fwd(const float *w, int cout, int cin_real, int cin, __nv_bfloat16 *wp) {
    const long long n = (long long)cin * 27 * cout;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        const int e = (int)(r % 8);
        r /= 8;
        const int ro = (int)(r % 8);
        r /= 8;
        const int nb = (int)(r % (cout / 8));
        r /= cout / 8;
        const int kb = (int)(r % 2);
        r /= 2;
        const int tap = (int)(r % 27);
        const int kk = (int)(r / 27);
        const int o = nb * 8 + ro, c = kk * 16 + kb * 8 + e;
        wp[i] = __float2bfloat16_rn(c < cin_real ? w[((long long)o * cin_real + c) * 27 + tap] : 0.f);
    }
}

// Prepared data-gradient weights: the convolution that maps dL/dy (cout channels) to dL/dx
// (cin channels) has weights w'[c][o][26 - tap] = w[o][c][tap]; laid out as k_prep_fwd with
// the roles of o and c exchanged.
__global__ void k_prep_dgrad(const float *w, int cout, int cin, __nv_bfloat16 *wp) {
    const long long n = (long long)cout * 27 * cin;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long r = i;
        const int e = (int)(r % 8);
        r /= 8;
        const int rc = (int)(r % 8);
        r /= 8;
        const int nb = (int)(r % (cin / 8));
        r /= cin / 8;
        const int kb = (int)(r % 2);
        r /= 2;
        const int tap = (int)(r % 27);
        const int kk = (int)(r / 27);
        const int c = nb * 8 + rc, o = kk * 16 + kb * 8 + e;
        wp[i] = __float2bfloat16_rn(w[((long long)o * cin + c) * 27 + (26 - tap)]);
    }
}

// ------------------------------------------------------------------ channels-last element kernels
struct View {
    __nv_bfloat16 *p;
    int ld, off;
};

// x FP32 [c_real][vol] -> BF16 channels-last [vol][ld], channels c_real.. ld-1 zero
__global__ void k_to_cl(const float *x, int c_real, long long vol, __nv_bfloat16 *y, int ld) {
    const long long n = vol * ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ld);
        const long long p = i / ld;
        y[i] = __float2bfloat16_rn(c < c_real ? x[(long long)c * vol + p] : 0.f);
    }
}

__device__ __forceinline__ long long cl_parent(long long p, int n) {
    const int k = (int)(p % n);
    const long long r = p / n;
    const int j = (int)(r % n), i = (int)(r / n);
    const int m = n / 2;
    return ((long long)(i / 2) * m + j / 2) * m + k / 2;
}

// y[q][c] = mean over the 8 children of q of x[child][c]; x side n, y side n/2
__global__ void k_pool_cl(View x, int C, int n, View y) {
    const int m = n / 2;
    const long long total = (long long)m * m * m * C;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(id % C);
        long long q = id / C;
        const int k = (int)(q % m);
        q /= m;
        const int j = (int)(q % m), i = (int)(q / m);
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 2; ++d)
                for (int f = 0; f < 2; ++f) {
                    const long long p = ((long long)(2 * i + a) * n + (2 * j + d)) * n + (2 * k + f);
                    acc += __bfloat162float(x.p[p * x.ld + x.off + c]);
                }
        y.p[(id / C) * y.ld + y.off + c] = __float2bfloat16_rn(0.125f * acc);
    }
}

// y[p][c] = x[parent(p)][c] (nearest upsampling, side m -> 2m)
__global__ void k_up_cl(View x, int C, int m, View y) {
    const int n = 2 * m;
    const long long total = (long long)n * n * n * C;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(id % C);
        const long long p = id / C;
        y.p[p * y.ld + y.off + c] = x.p[cl_parent(p, n) * x.ld + x.off + c];
    }
}

// g[p][c] = 0 where y[p][c] <= 0 (ReLU backward from the ReLU output)
__global__ void k_relu_back_cl(View g, View y, int C, long long vol) {
    const long long total = vol * C;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(id % C);
        const long long p = id / C;
        if (!(__bfloat162float(y.p[p * y.ld + y.off + c]) > 0.f)) g.p[p * g.ld + g.off + c] = __float2bfloat16_rn(0.f);
    }
}

// gx[p][c] += gy[parent(p)][c] / 8 (pool backward, accumulating; gx side n)
__global__ void k_pool_back_add_cl(View gy, int C, int n, View gx) {
    const long long total = (long long)n * n * n * C;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(id % C);
        const long long p = id / C;
        __nv_bfloat16 &d = gx.p[p * gx.ld + gx.off + c];
        d = __float2bfloat16_rn(__bfloat162float(d) + 0.125f * __bfloat162float(gy.p[cl_parent(p, n) * gy.ld + gy.off + c]));
    }
}

// gx[q][c] = sum over the 8 children of q of gy[child][c] (upsampling backward; side 2m -> m)
__global__ void k_up_back_cl(View gy, int C, int m, View gx) {
    const int n = 2 * m;
    const long long total = (long long)m * m * m * C;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(id % C);
        long long q = id / C;
        const int k = (int)(q % m);
        q /= m;
        const int j = (int)(q % m), i = (int)(q / m);
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 2; ++d)
                for (int f = 0; f < 2; ++f) {
                    const long long p = ((long long)(2 * i + a) * n + (2 * j + d)) * n + (2 * k + f);
                    acc += __bfloat162float(gy.p[p * gy.ld + gy.off + c]);
                }
        gx.p[(id / C) * gx.ld + gx.off + c] = __float2bfloat16_rn(acc);
    }
}

// part[block][c] = sum over the block's voxel range of g[p][c] (C <= 256, 256 threads:
// thread = (voxel lane, channel)); the caller sums the blocks in order.
__global__ void k_bias_part_cl(View g, int C, long long vol, long long per_block, float *part) {
    __shared__ float red[256];
    const int lanes = 256 / C;
    const int c = threadIdx.x % C, l = threadIdx.x / C;
    const long long p0 = (long long)blockIdx.x * per_block, p1 = min(vol, p0 + per_block);
    float s = 0.f;
    if (l < lanes)
        for (long long p = p0 + l; p < p1; p += lanes) s += __bfloat162float(g.p[p * g.ld + g.off + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int k = 0; k < lanes; ++k) t += red[k * C + threadIdx.x];
        part[(long long)blockIdx.x * C + threadIdx.x] = t;
    }
}

// out[c] = sum over blocks of part[block][c], in block order
__global__ void k_sum_rows_f(const float *part, int blocks, int C, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += part[(long long)b * C + c];
    out[c] = s;
}

// Output layer (1x1x1): y[o][p] = b[o] + sum_c w[o][c] x[p][c] (FP32 result)
__global__ void k_conv1_cl(View x, int ci, long long vol, const float *w, const float *b, int co, float *y) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < vol; p += (long long)gridDim.x * blockDim.x)
        for (int o = 0; o < co; ++o) {
            float s = b[o];
            for (int c = 0; c < ci; ++c) s = fmaf(w[o * ci + c], __bfloat162float(x.p[p * x.ld + x.off + c]), s);
            y[(long long)o * vol + p] = s;
        }
}

// gx[p][c] = sum_o w[o][c] gy[o][p] (gy FP32 [co][vol])
__global__ void k_conv1_dgrad_cl(const float *gy, int co, long long vol, const float *w, int ci, View gx) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < vol; p += (long long)gridDim.x * blockDim.x)
        for (int c = 0; c < ci; ++c) {
            float s = 0.f;
            for (int o = 0; o < co; ++o) s = fmaf(w[o * ci + c], gy[(long long)o * vol + p], s);
            gx.p[p * gx.ld + gx.off + c] = __float2bfloat16_rn(s);
        }
}

// gw[o][c] = sum_p gy[o][p] x[p][c] (one block per (o, c), fixed order)
__global__ void k_conv1_wgrad_cl(const float *gy, View x, long long vol, int ci, float *gw) {
    __shared__ float red[8];
    const int o = blockIdx.x / ci, c = blockIdx.x - o * ci;
    float s = 0.f;
    for (long long p = threadIdx.x; p < vol; p += blockDim.x)
        s = fmaf(gy[(long long)o * vol + p], __bfloat162float(x.p[p * x.ld + x.off + c]), s);
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        gw[blockIdx.x] = t;
    }
}

}  // namespace tc
