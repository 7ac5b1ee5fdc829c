/*
 * unet3d.h - the 3D U-Net of the learned initial guess for the 3D-RISM solve.
 *
 * The paper has no learned component: it starts every solve from t = f (step 1 of the
 * "Numerical procedure" section). This network predicts the starting iterate
 * tau = t - f on a cubic crop around the solute from the potential beta*u on that crop,
 * so that the fixed-point iteration starts closer to its solution; the solve itself is
 * unchanged (its result is the same fixed point). rism3d.h has the entry points that
 * cut the network's input out of a solver context and put its output back as the guess.
 *
 * Architecture (channels c0, c1, c2; crop side n divisible by 4):
 *   enc1 = relu(conv(relu(conv(x))))                              [c0, n^3]
 *   enc2 = relu(conv(relu(conv(pool(enc1)))))                      [c1, (n/2)^3]
 *   mid  = relu(conv(relu(conv(pool(enc2)))))                      [c2, (n/4)^3]
 *   dec2 = relu(conv(relu(conv([up(mid), enc2]))))                 [c1, (n/2)^3]
 *   dec1 = relu(conv(relu(conv([up(dec2), enc1]))))                [c0, n^3]
 *   y    = conv1x1(dec1)                                           [n_out, n^3]
 * conv: 3x3x3, zero padding, bias; pool: 2x2x2 mean; up: nearest x2; [a, b]: channel
 * concatenation. Parameters are one flat FP32 vector, layer by layer, each layer's weights
 * ([out][in][3][3][3], or [out][in] for the last) followed by its biases.
 *
 * Arithmetic, chosen at creation (unet3d_create_ex):
 *   UNET3D_FP32  FP32 activations, FP32 direct convolutions over shared-memory tiles.
 *   UNET3D_BF16  BF16 activations (channels-last inside the network), the 3x3x3
 *                convolutions, their data gradients and their weight gradients as implicit
 *                GEMMs on the tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation in
 *                tensor memory); the 1x1x1 output layer, loss and Adam in FP32. Parameters,
 *                gradients and moments stay FP32 in both forms (the same flat vector), so
 *                parameters trained in one form run in the other. Needs c0, c1, c2 multiples
 *                of 16 with c2 + c1 <= 256; the input channels are padded to a multiple of 16.
 * Every array argument is device memory of the current CUDA device unless stated; every
 * call returns 0 on success, else a nonzero code with a message in unet3d_last_error():
 * 1 bad arguments, 2 allocation failure, 3 a CUDA error, 4 a call out of order.
 * Calls enqueue on the network's stream and return without synchronising unless stated.
 */
#ifndef UNET3D_PUBLIC_API_H_
#define UNET3D_PUBLIC_API_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet3d unet3d;

enum { UNET3D_FP32 = 0, UNET3D_BF16 = 1 };

/* Allocates parameters, gradients, Adam moments and the activations of one crop.
 * n_in, n_out >= 1; crop >= 4 and divisible by 4; channels >= 1. stream: cudaStream_t or
 * NULL (the legacy default stream). Returns 1 on bad arguments, 2 on allocation failure. */
int unet3d_create(int n_in, int n_out, int crop, int c0, int c1, int c2, void *stream, unet3d **out);

/* unet3d_create with the arithmetic form (UNET3D_FP32 or UNET3D_BF16); returns 1 when the
 * channels do not suit the form. unet3d_create is unet3d_create_ex(..., UNET3D_FP32, ...). */
int unet3d_create_ex(int n_in, int n_out, int crop, int c0, int c1, int c2, int arith, void *stream,
                     unet3d **out);

/* Number of FP32 parameters (weights and biases of all layers). */
size_t unet3d_param_count(const unet3d *net);

/* Copy the flat parameter vector in or out (host memory; synchronous). */
int unet3d_set_params(unet3d *net, const float *host_params);
int unet3d_get_params(const unet3d *net, float *host_params);

/* y [n_out][crop^3] = network(x [n_in][crop^3]); keeps the activations for backward. */
int unet3d_forward(unet3d *net, const float *x, float *y);

/* Parameter gradient of a loss with dL/dy = gy [n_out][crop^3] at the last forward's
 * input, written into the network's gradient vector (overwritten, not accumulated).
 * Returns 4 when no forward pass has completed since creation (or the last one failed). */
int unet3d_backward(unet3d *net, const float *gy);

/* Copy the gradient vector to host memory (synchronous). */
int unet3d_get_grads(const unet3d *net, float *host_grads);

/* Mean squared error of y against target (count values): loss to host (synchronous,
 * FP64 sum in a fixed order) and gy = 2 (y - target) / count on the device. */
int unet3d_mse(unet3d *net, const float *y, const float *target, size_t count, double *loss, float *gy);

/* Weighted mean squared error of y [n_out][crop^3] against target at the last forward's
 * input x: weight core_weight (> 0) where the first input channel x[0][p] >= core_x, else 1;
 * loss = sum w (y - target)^2 / sum w to host (synchronous, FP64 sums in a fixed order) and
 * gy = 2 w (y - target) / sum w on the device. For the learned guess the first input channel
 * is tanh(beta u / 4) of the first solvent site, so core_x near 1 selects the solute core,
 * where the target iterate is large and the solve settles it within a few iterations.
 * Returns 4 when no forward pass has completed. */
int unet3d_mse_core(unet3d *net, const float *y, const float *target, float core_x, float core_weight,
                    double *loss, float *gy);

/* One Adam step on the parameters with the current gradient: step t >= 1, moments with
 * decay beta1, beta2, bias-corrected; p -= lr m^ / (sqrt(v^) + eps). */
int unet3d_adam(unet3d *net, float lr, float beta1, float beta2, float eps, int t);

const char *unet3d_last_error(void);

/* One 3x3x3 convolution of the BF16 form on caller buffers (device memory; BF16 arrays are
 * channels-last, voxel p of the n^3 volume at [p][channels]), for callers that run single
 * layers and for checking the tensor-core kernels against a reference convolution:
 *   mode 0: out[p][o] = bf16(b[o] + sum_c sum_tap w[o][c][tap] in[p + tap - 1][c]), in
 *           [n^3][cin], out [n^3][cout], b FP32 [cout] or NULL, ReLU when relu != 0;
 *   mode 1: data gradient, in = dL/dy [n^3][cout], out = dL/dx [n^3][cin] (BF16);
 *   mode 2: weight gradient, in = x [n^3][cin], in2 = dL/dy [n^3][cout],
 *           out = dL/dw FP32 [cout][cin][27].
 * w is FP32 [cout][cin][27] (rounded to BF16 for the products); zero padding outside the
 * volume. cin and cout multiples of 16 (cout <= 128; cin <= 128 in mode 1). Allocates its
 * scratch on the device and returns after the stream has finished (synchronous). */
int unet3d_conv3_bf16(int mode, int n, int cin, int cout, const void *in, const void *in2, const float *w,
                      const float *b, int relu, void *out, void *stream);

void unet3d_destroy(unet3d *net);

#ifdef __cplusplus
}
#endif

#endif /* UNET3D_PUBLIC_API_H_ */
