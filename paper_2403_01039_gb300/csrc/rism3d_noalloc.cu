// Solvation free energy from caller-supplied fields, for callers that cannot allocate
// device memory.
//
// rism3d_get_sfe reduces into per-block partial sums held in the context's workspace. Some
// callers have no context and cannot obtain scratch memory: code whose device memory
// budget is fixed in advance by a host framework that owns every allocation (a memory pool
// that hands out all of the device), and latency-critical loops where a cudaMalloc or
// cudaFree would synchronise the device. rism3d_sfe_noalloc serves them: its scratch is the
// file-scope array below, which every GPU that loads the library holds until the process
// exits. The call waits for its stream to finish before it returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "rism3d.h"
#include "rism3d_internal.h"

namespace {

constexpr int kScratchSites = 8;       // largest n_sites the static scratch can hold
constexpr int kScratchBlocks = 152;    // partial sums per site (one per block)
constexpr int kScratchDoubles = kScratchSites * kScratchBlocks + kScratchSites;
constexpr int kMaxDevices = 64;

// [site][block] partial sums, then one total per site. Shared by every call: each call
// writes every slot it later reads, so nothing has to start at zero, and two calls whose
// kernels overlap on the GPU race on it.
static __device__ __align__(256) double g_sfe_scratch[kScratchDoubles];

double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

constexpr double kKB = 0.0019872041;   // kcal / (mol K)

// Integrand of the SFE per site (Eqs. 17-18, GF, PSE-n), accumulated in FP64 per block.
__global__ void __launch_bounds__(256)
k_sfe_fields(const double *h, const double *c, const double *d, long long n_points, int kind,
             int order, double *scratch) {
    __shared__ double red[8];
    const int site = blockIdx.y;
    const double *hs = h + (long long)site * n_points;
    const double *cs = c + (long long)site * n_points;
    const double *ds = d ? d + (long long)site * n_points : nullptr;
    double fact = 1.0;
    for (int i = 2; i <= order + 1; ++i) fact *= i;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_points;
         p += (long long)gridDim.x * blockDim.x) {
        const double hv = hs[p], cv = cs[p];
        double v = -cv - 0.5 * hv * cv;
        if (kind == RISM3D_SFE_HNC) {
            v += 0.5 * hv * hv;
        } else if (kind == RISM3D_SFE_KH) {
            v += hv < 0.0 ? 0.5 * hv * hv : 0.0;
        } else if (kind == RISM3D_SFE_PSE) {
            v += 0.5 * hv * hv;
            const double dv = ds[p];
            if (dv > 0.0) v -= pow(dv, (double)(order + 1)) / fact;
        }
        acc += v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        scratch[site * kScratchBlocks + blockIdx.x] = s;
    }
}

// Per-site totals in a fixed order (bit-reproducible), after the partials.
__global__ void k_sfe_fields_finish(double *scratch, int n_sites) {
    const int site = threadIdx.x;
    if (site >= n_sites) return;
    double s = 0.0;
    for (int b = 0; b < kScratchBlocks; ++b) s += scratch[site * kScratchBlocks + b];
    scratch[kScratchSites * kScratchBlocks + site] = s;
}

rism3d_status bad(rism3d_status st, const char *msg) {
    rism::set_global_error(msg);
    return st;
}

// True if p is device (or managed) memory that device dev can read.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();     // clear the error this query left
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" rism3d_status rism3d_sfe_noalloc(int n_sites, long long n_points, const double *h,
                                            const double *c, const double *d, const double *rho,
                                            double temperature, double dV, int kind, int pse_order,
                                            double *total, double *per_site, void *cuda_stream) {
    if (n_sites < 1) return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: n_sites must be >= 1");
    if (n_sites > kScratchSites) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "rism3d_sfe_noalloc: n_sites %d exceeds the static scratch capacity of %d sites",
                 n_sites, kScratchSites);
        return bad(RISM3D_EINVAL, msg);
    }
    if (n_points < 1) return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: n_points must be >= 1");
    if (!h || !c || !rho || !total) return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: null h, c, rho or total");
    if (kind < RISM3D_SFE_KH || kind > RISM3D_SFE_PSE) return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: bad kind");
    if (kind == RISM3D_SFE_PSE && (pse_order < 1 || !d))
        return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: PSE needs pse_order >= 1 and the d field");
    if (!(temperature > 0.0) || !(dV > 0.0))
        return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: temperature and dV must be positive");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return bad(RISM3D_ECUDA, "rism3d_sfe_noalloc: no usable current device");
    if (!on_device(h, dev) || !on_device(c, dev) || (kind == RISM3D_SFE_PSE && !on_device(d, dev)))
        return bad(RISM3D_EINVAL, "rism3d_sfe_noalloc: h, c and d must be device memory of the current device");
    double *scratch = nullptr;
    {
        // One-time set-up per device, with that device current: the device address of the
        // static array (its name in host code is only a host-side stand-in).
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_sfe_scratch);
            if (e != cudaSuccess) {
                char msg[200];
                snprintf(msg, sizeof(msg), "rism3d_sfe_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return bad(RISM3D_ECUDA, msg);
            }
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_sfe_fields<<<dim3(kScratchBlocks, n_sites), 256, 0, s>>>(h, c, kind == RISM3D_SFE_PSE ? d : nullptr,
                                                              n_points, kind, pse_order, scratch);
    k_sfe_fields_finish<<<1, 32, 0, s>>>(scratch, n_sites);
    cudaError_t e = cudaGetLastError();        // launch errors, before anything is copied
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "rism3d_sfe_noalloc: launch: %s", cudaGetErrorString(e));
        return bad(RISM3D_ECUDA, msg);
    }
    double sums[kScratchSites];
    e = cudaMemcpyAsync(sums, scratch + kScratchSites * kScratchBlocks, (size_t)n_sites * sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "rism3d_sfe_noalloc: %s", cudaGetErrorString(e));
        return bad(RISM3D_ECUDA, msg);
    }
    const double kT = kKB * temperature;
    double tot = 0.0;
    for (int g = 0; g < n_sites; ++g) {
        const double v = kT * rho[g] * dV * sums[g];
        if (per_site) per_site[g] = v;
        tot += v;
    }
    *total = tot;
    return RISM3D_OK;
}
