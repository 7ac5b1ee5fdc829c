// Launchers of the BF16 tensor-core U-Net kernels (unet3d_tc.cuh).
#include "unet3d_tc.h"

#include "unet3d_tc.cuh"

namespace tcnet {

namespace {

constexpr int kTX = 2;                  // x planes per convolution tile
constexpr int kWgradCtas = 296;         // target CTAs of one weight-gradient launch (2 per SM)
constexpr int kBiasBlocks = 256;

unsigned grid_for(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

int tiles(int n) { return cdiv(n, kTX) * cdiv(n, 16) * cdiv(n, 8); }

struct WgradPlan {
    int groups, taps_per_group, chunks, per;
};

WgradPlan wgrad_plan(int n, int cin) {
    WgradPlan p;
    p.groups = cdiv(27LL * cin, 512);
    p.taps_per_group = cdiv(27, p.groups);
    p.groups = cdiv(27, p.taps_per_group);
    const int nt = tiles(n);
    int chunks = kWgradCtas / p.groups;
    chunks = chunks < 1 ? 1 : (chunks > nt ? nt : chunks);
    p.per = cdiv(nt, chunks);
    p.chunks = cdiv(nt, p.per);
    return p;
}

constexpr unsigned kSmemLimit = 227u * 1024u - 1024u;   // dynamic bytes, below the opt-in maximum

// raise the kernel's dynamic shared-memory cap to the device's opt-in maximum minus its
// static shared memory
cudaError_t set_smem(const void *fn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

tc::View tv(CLView v) { return tc::View{v.p, v.ld, v.off}; }

}  // namespace

bool conv_shape_ok(int cin, int cout) {
    return cin >= 16 && cin % 16 == 0 && cout >= 16 && cout % 16 == 0 && cout <= 128 &&
           tc::fwd_smem(kTX, cout) <= kSmemLimit;
}

bool wgrad_shape_ok(int cin, int cout) {
    return cin >= 16 && cin % 16 == 0 && cin <= 256 && cout >= 16 && cout % 16 == 0 && cout <= 128 &&
           tc::wg_smem(kTX, cin, cout) <= kSmemLimit;
}

size_t prep_elems(int cin, int cout) { return (size_t)cin * 27 * cout; }

size_t wgrad_part_floats(int n, int cin, int cout) {
    const WgradPlan p = wgrad_plan(n, cin);
    return (size_t)p.chunks * 27 * cin * cout;
}

size_t bias_part_floats(int cout) { return (size_t)kBiasBlocks * cout; }

cudaError_t prep_fwd(cudaStream_t s, const float *w, int cout, int cin_real, int cin, __nv_bfloat16 *wp) {
    tc::k_prep_fwd<<<grid_for((long long)prep_elems(cin, cout)), 256, 0, s>>>(w, cout, cin_real, cin, wp);
    return cudaGetLastError();
}

cudaError_t prep_dgrad(cudaStream_t s, const float *w, int cout, int cin, __nv_bfloat16 *wp) {
    tc::k_prep_dgrad<<<grid_for((long long)prep_elems(cin, cout)), 256, 0, s>>>(w, cout, cin, wp);
    return cudaGetLastError();
}

cudaError_t conv3(cudaStream_t s, CLView x, int cin, const __nv_bfloat16 *wp, const float *bias, CLView y, int cout,
                  int n, int relu, int *status) {
    if (!conv_shape_ok(cin, cout) || n < 1) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = set_smem((const void *)tc::k_conv3_tc<kTX>);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc::ConvArgs a;
    a.x = x.p, a.ldx = x.ld, a.xoff = x.off, a.cin = cin;
    a.w = wp, a.bias = bias;
    a.y = y.p, a.ldy = y.ld, a.yoff = y.off, a.cout = cout;
    a.n = n, a.relu = relu, a.status = status;
    tc::k_conv3_tc<kTX><<<tiles(n), 128, tc::fwd_smem(kTX, cout), s>>>(a);
    return cudaGetLastError();
}

cudaError_t conv3_wgrad(cudaStream_t s, CLView x, int cin, int cin_real, CLView gy, int cout, int n, float *part,
                        float *gw, int *status) {
    if (!wgrad_shape_ok(cin, cout) || n < 1 || cin_real > cin) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = set_smem((const void *)tc::k_conv3_wgrad_tc<kTX>);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const WgradPlan p = wgrad_plan(n, cin);
    tc::WgradArgs a;
    a.x = x.p, a.ldx = x.ld, a.xoff = x.off, a.cin = cin;
    a.gy = gy.p, a.ldg = gy.ld, a.goff = gy.off, a.cout = cout;
    a.n = n, a.tiles_per_chunk = p.per, a.taps_per_group = p.taps_per_group;
    a.part = part, a.status = status;
    tc::k_conv3_wgrad_tc<kTX><<<dim3((unsigned)p.chunks, (unsigned)p.groups), 128, tc::wg_smem(kTX, cin, cout), s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc::k_wgrad_sum<<<grid_for((long long)cout * cin_real * 27), 256, 0, s>>>(part, p.chunks, cin, cout, cin_real, gw);
    return cudaGetLastError();
}

cudaError_t bias_grad(cudaStream_t s, CLView g, int cout, long long vol, float *part, float *gb) {
    if (cout > 256) return cudaErrorInvalidValue;
    const long long per = (vol + kBiasBlocks - 1) / kBiasBlocks;
    tc::k_bias_part_cl<<<kBiasBlocks, 256, 0, s>>>(tv(g), cout, vol, per, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc::k_sum_rows_f<<<(cout + 127) / 128, 128, 0, s>>>(part, kBiasBlocks, cout, gb);
    return cudaGetLastError();
}

cudaError_t to_cl(cudaStream_t s, const float *x, int c_real, long long vol, __nv_bfloat16 *y, int ld) {
    tc::k_to_cl<<<grid_for(vol * ld), 256, 0, s>>>(x, c_real, vol, y, ld);
    return cudaGetLastError();
}

cudaError_t pool(cudaStream_t s, CLView x, int C, int n, CLView y) {
    const long long m = n / 2;
    tc::k_pool_cl<<<grid_for(m * m * m * C), 256, 0, s>>>(tv(x), C, n, tv(y));
    return cudaGetLastError();
}

cudaError_t up(cudaStream_t s, CLView x, int C, int m, CLView y) {
    const long long n = 2LL * m;
    tc::k_up_cl<<<grid_for(n * n * n * C), 256, 0, s>>>(tv(x), C, m, tv(y));
    return cudaGetLastError();
}

cudaError_t relu_back(cudaStream_t s, CLView g, CLView y, int C, long long vol) {
    tc::k_relu_back_cl<<<grid_for(vol * C), 256, 0, s>>>(tv(g), tv(y), C, vol);
    return cudaGetLastError();
}

cudaError_t pool_back_add(cudaStream_t s, CLView gy, int C, int n, CLView gx) {
    tc::k_pool_back_add_cl<<<grid_for((long long)n * n * n * C), 256, 0, s>>>(tv(gy), C, n, tv(gx));
    return cudaGetLastError();
}

cudaError_t up_back(cudaStream_t s, CLView gy, int C, int m, CLView gx) {
    tc::k_up_back_cl<<<grid_for((long long)m * m * m * C), 256, 0, s>>>(tv(gy), C, m, tv(gx));
    return cudaGetLastError();
}

cudaError_t conv1(cudaStream_t s, CLView x, int ci, long long vol, const float *w, const float *b, int co, float *y) {
    tc::k_conv1_cl<<<grid_for(vol), 256, 0, s>>>(tv(x), ci, vol, w, b, co, y);
    return cudaGetLastError();
}

cudaError_t conv1_dgrad(cudaStream_t s, const float *gy, int co, long long vol, const float *w, int ci, CLView gx) {
    tc::k_conv1_dgrad_cl<<<grid_for(vol), 256, 0, s>>>(gy, co, vol, w, ci, tv(gx));
    return cudaGetLastError();
}

cudaError_t conv1_wgrad(cudaStream_t s, const float *gy, int co, CLView x, long long vol, int ci, float *gw) {
    tc::k_conv1_wgrad_cl<<<co * ci, 256, 0, s>>>(gy, tv(x), vol, ci, gw);
    return cudaGetLastError();
}

}  // namespace tcnet
