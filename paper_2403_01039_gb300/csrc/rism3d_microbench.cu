// FP32 and FP64 fused multiply-add throughput of the device (a measurement of the machine,
// no counterpart in the paper): the FP64 form of the solve is expected to be bound by FP64
// arithmetic rather than by HBM on this GPU, and its roofline needs the measured rate.
#include <cuda_runtime.h>

#include <cstdio>

#include "rism3d.h"
#include "rism3d_internal.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread (hides the latency)
constexpr int kThreads = 256;

// Every thread runs kChains dependent chains of `iters` FMAs each; the result is written only
// if it is the impossible value -1, so the work cannot be removed and nothing is stored.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma(int iters, T a, T b, T *sink) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == (T)-1) sink[0] = s;
}

template <typename T>
rism3d_status run(int sms, double *rate) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RISM3D_ECUDA;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (sms > 0 ? sms : nsm) * 8;
    const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 12;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RISM3D_ECUDA;
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma<T><<<blocks, kThreads>>>(iters / 16, a, b, nullptr);      // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_fma<T><<<blocks, kThreads>>>(iters, a, b, nullptr);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || best >= 1e30f) return RISM3D_ECUDA;
    const double fmas = (double)blocks * kThreads * kChains * (double)iters;
    *rate = 2.0 * fmas / (best * 1e-3);
    return RISM3D_OK;
}

}  // namespace

extern "C" rism3d_status rism3d_fma_rate(int precision, double *flops_per_s) {
    if (!flops_per_s || (precision != 32 && precision != 64)) return RISM3D_EINVAL;
    return precision == 32 ? run<float>(0, flops_per_s) : run<double>(0, flops_per_s);
}
