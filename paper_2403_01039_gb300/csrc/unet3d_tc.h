// Host launchers of the BF16 tensor-core form of the U-Net (unet3d_tc.cu), used by
// unet3d.cu. Library-internal: not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace tcnet {

// channels-last BF16 view: voxel p holds its channels at p[q * ld + off + c]
struct CLView {
    __nv_bfloat16 *p;
    int ld, off;
};

// limits of the tensor-core convolutions
bool conv_shape_ok(int cin, int cout);          // forward / data gradient (cin -> cout)
bool wgrad_shape_ok(int cin, int cout);

size_t prep_elems(int cin, int cout);           // prepared BF16 weights of one layer
size_t wgrad_part_floats(int n, int cin, int cout);
size_t bias_part_floats(int cout);

cudaError_t prep_fwd(cudaStream_t s, const float *w, int cout, int cin_real, int cin, __nv_bfloat16 *wp);
cudaError_t prep_dgrad(cudaStream_t s, const float *w, int cout, int cin, __nv_bfloat16 *wp);
// y = conv3x3x3(x) (+ bias, ReLU) with prepared weights
cudaError_t conv3(cudaStream_t s, CLView x, int cin, const __nv_bfloat16 *wp, const float *bias, CLView y, int cout,
                  int n, int relu, int *status);
// gw[o][c][tap] (FP32, cin_real input channels) = sum_p gy[p][o] x[p + tap][c]
cudaError_t conv3_wgrad(cudaStream_t s, CLView x, int cin, int cin_real, CLView gy, int cout, int n, float *part,
                        float *gw, int *status);
// gb[o] = sum_p g[p][o]
cudaError_t bias_grad(cudaStream_t s, CLView g, int cout, long long vol, float *part, float *gb);

cudaError_t to_cl(cudaStream_t s, const float *x, int c_real, long long vol, __nv_bfloat16 *y, int ld);
cudaError_t pool(cudaStream_t s, CLView x, int C, int n, CLView y);
cudaError_t up(cudaStream_t s, CLView x, int C, int m, CLView y);
cudaError_t relu_back(cudaStream_t s, CLView g, CLView y, int C, long long vol);
cudaError_t pool_back_add(cudaStream_t s, CLView gy, int C, int n, CLView gx);
cudaError_t up_back(cudaStream_t s, CLView gy, int C, int m, CLView gx);
cudaError_t conv1(cudaStream_t s, CLView x, int ci, long long vol, const float *w, const float *b, int co, float *y);
cudaError_t conv1_dgrad(cudaStream_t s, const float *gy, int co, long long vol, const float *w, int ci, CLView gx);
cudaError_t conv1_wgrad(cudaStream_t s, const float *gy, int co, CLView x, long long vol, int ci, float *gw);

}  // namespace tcnet
