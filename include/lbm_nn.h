/*
 * lbm_nn.h -- C ABI of the kernels of the learned fast-forward: a small
 * convolutional encoder-decoder trained on coarse-grained (phi, u, v)
 * snapshots that the lattice Boltzmann solver (lbm.h) generates, used to
 * predict the coarse fields K steps ahead; the solver restarts from the
 * prediction and judges it.  The paper has no counterpart: this is the third
 * extension of the hot path (learned parts of a sweep).
 *
 * Conventions
 *  - Activations are bfloat16, channels last: element (m, c) of a tensor with
 *    channel stride s and channel offset o is at [m * s + o + c], m = (b * H +
 *    y) * W + x.  A channel offset lets a convolution write into, or read
 *    from, a slice of a wider tensor (the concatenations of the decoder).
 *  - Convolution weights are bfloat16 [co][taps * ci] with k = tap * ci + c
 *    and tap = 3 ky + kx (3 x 3, zero padding 1: output (y, x) reads input
 *    (y + ky - 1, x + kx - 1)) or taps = 1 (1 x 1).  Biases, gradients of
 *    weights and the optimiser state are float32.
 *  - Tensor-core operands are moved as 16-byte vectors: ci, the input channel
 *    stride and (for the weight gradient) co and the gradient stride must be
 *    multiples of 8, and those tensors 16-byte aligned; violations return
 *    LBM_NN_ERR_ARG.
 *  - All pointers are device pointers owned by the caller; every call only
 *    enqueues kernels on `stream` (NULL = legacy default stream) and returns.
 *    Launch failures return LBM_NN_ERR_CUDA; the text of the last error of
 *    the calling thread is lbm_nn_last_error().
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LBM_NN_OK = 0, LBM_NN_ERR_ARG = -1, LBM_NN_ERR_CUDA = -2 } lbm_nn_status;

const char* lbm_nn_last_error(void);

/* y[m][y_offset + co] (bf16, may be NULL) and yf[m][co] (f32, may be NULL) =
 * relu?(sum_k patch(x)[m][k] wt[co][k] + bias[co]) for the nb * h * w
 * positions; bias may be NULL.  When the output tiles alone would leave most
 * of the GPU idle (few positions, many channels), the k range is split over
 * blocks: their float32 partial sums go to scratch allocated on `stream`
 * (cudaMallocAsync, at most 16 MB, freed on `stream`) and are added in a fixed
 * order, so results do not depend on scheduling. */
int lbm_nn_conv_fwd(const void* x, int32_t x_stride, int32_t ci, int32_t taps, const void* wt, const float* bias,
                    int32_t co, void* y, int32_t y_stride, int32_t y_offset, float* yf, int32_t yf_stride,
                    int32_t relu, int32_t nb, int32_t h, int32_t w, void* stream);

/* The contraction lbm_nn_conv_fwd (and with it the backward-data pass, the
 * same call on flipped weights) runs on: 0 the fifth-generation tensor cores
 * -- tcgen05.mma with the float32 accumulator in tensor memory,
 * 128-position x 32/64/128-channel tiles, operands brought into shared
 * memory by asynchronous copies three k-tiles deep; 1 the warp-level
 * mma.sync kernels; 2 (default) tcgen05 for calls of at least 4 GFLOP
 * (2 positions x co x taps x ci), else mma.sync.  All sum in float32 over bfloat16 products; they may differ in
 * the order of the sums.  Process-wide; LBM_NN_ERR_ARG for other values. */
int lbm_nn_set_conv_path(int32_t path);

/* Whether a bounded wait of the tcgen05 convolution kernels gave up since the
 * last call (*timed_out = 1; the outputs of that call are not valid), then
 * clears the flag.  The flag is a 4-byte device word allocated on the first
 * convolution call on each device.  Synchronises the device's legacy default
 * stream. */
int lbm_nn_conv_status(int32_t* timed_out);

/* Gradients of a convolution from the gradient dz of its pre-activation
 * output: dwt[co][k] += sum_m dz[m][co] patch(x)[m][k], dbias[co] += sum_m
 * dz[m][co] (dbias may be NULL).  Accumulates: zero the outputs first.  The
 * sums over positions are split into chunks whose partial sums go to scratch
 * allocated on `stream` (cudaMallocAsync, at most 16 MB, freed on `stream`)
 * and are added in chunk order: the result does not depend on scheduling. */
int lbm_nn_conv_wgrad(const void* x, int32_t x_stride, int32_t ci, int32_t taps, const void* dz, int32_t dz_stride,
                      int32_t co, float* dwt, float* dbias, int32_t nb, int32_t h, int32_t w, void* stream);

/* wflip[c][tap' * co + o] = wt[o][(taps - 1 - tap') * ci + c]: the weights of
 * the convolution that maps the output gradient to the input gradient
 * (lbm_nn_conv_fwd with ci and co exchanged). */
int lbm_nn_flip_weights(const void* wt, int32_t ci, int32_t co, int32_t taps, void* wflip, void* stream);

/* dz[m][c] = dy[m][dy_offset + c] where y[m][y_offset + c] > 0, else 0. */
int lbm_nn_relu_bwd(const void* dy, int32_t dy_stride, int32_t dy_offset, const void* y, int32_t y_stride,
                    int32_t y_offset, void* dz, int32_t dz_stride, int32_t c, int64_t m, void* stream);

/* 2 x 2 average pooling of an h x w tensor (h, w even) and its adjoint; the
 * adjoint adds into dx. */
int lbm_nn_pool(const void* x, int32_t x_stride, int32_t x_offset, void* y, int32_t y_stride, int32_t y_offset,
                int32_t c, int32_t nb, int32_t h, int32_t w, void* stream);
int lbm_nn_pool_bwd(const void* dy, int32_t dy_stride, void* dx, int32_t dx_stride, int32_t dx_offset, int32_t c,
                    int32_t nb, int32_t h, int32_t w, void* stream);

/* Nearest 2x upsampling to an h x w tensor (h, w even) and its adjoint (the
 * sum over the 2 x 2 children; written, not added). */
int lbm_nn_upsample(const void* x, int32_t x_stride, void* y, int32_t y_stride, int32_t y_offset, int32_t c,
                    int32_t nb, int32_t h, int32_t w, void* stream);
int lbm_nn_upsample_bwd(const void* dy, int32_t dy_stride, int32_t dy_offset, void* dx, int32_t dx_stride, int32_t c,
                        int32_t nb, int32_t h, int32_t w, void* stream);

/* Residual head and loss over m positions and the first c channels: pred =
 * x[:, :c] + d[:, :c] (d f32 with stride d_stride; pred f32 [m][c], may be
 * NULL); with a target (f32 [m][c]): *loss += mean of (pred - target)^2 (loss
 * may be NULL) and dd[m][ch] = its gradient wrt d[m][ch] for ch < c (bf16
 * with stride dd_stride, may be NULL; other channels untouched). */
int lbm_nn_mse(const float* d, int32_t d_stride, const void* x, int32_t x_stride, const float* target, int32_t c,
               int64_t m, float* pred, void* dd, int32_t dd_stride, float* loss, void* stream);

/* Adam step t >= 1 on f32 weights w with moments m, v and gradient g; writes
 * the bf16 copy w_bf16 (may be NULL). */
int lbm_nn_adam(float* w, float* m, float* v, const float* g, void* w_bf16, int64_t n, float lr, float beta1,
                float beta2, float eps, int32_t t, void* stream);

/* b = bf16(a), n elements. */
int lbm_nn_to_bf16(const float* a, void* b, int64_t n, void* stream);

/* dst[m][dst_offset + c] += src[m][src_offset + c] (bf16). */
int lbm_nn_add(const void* src, int32_t src_stride, int32_t src_offset, void* dst, int32_t dst_stride,
               int32_t dst_offset, int32_t c, int64_t m, void* stream);

/* Network input from solver fields phi, u, v (f32 planes [hf][wf]): means
 * over factor x factor cells; x[m][0..x_channels) = (phi, u u_scale, v
 * u_scale, cond, 0 ...) in bf16 (may be NULL) and xf[m][0..3) the first
 * three in f32 (may be NULL). */
int lbm_nn_coarsen(const float* phi, const float* u, const float* v, int32_t hf, int32_t wf, int32_t factor,
                   float u_scale, float cond, void* x, int32_t x_channels, float* xf, void* stream);

/* Solver fields from a coarse prediction pred[m][3] = (phi, u u_scale, v
 * u_scale) of an hc x wc grid: bilinear interpolation between coarse cell
 * centres (clamped at the edges) onto the hc factor x wc factor grid, phi
 * clamped to [0, 1] and the speed limited to u_max (a restart state the
 * solver can take). */
int lbm_nn_refine(const float* pred, int32_t hc, int32_t wc, int32_t factor, float u_scale, float u_max, float* phi,
                  float* u, float* v, void* stream);

/* Re-sharpening of a phase field refined from a coarse grid (n values, in
 * place): phi <- 1/2 + 1/2 tanh(ratio atanh(2 q - 1)), q = phi clamped to
 * [1e-6, 1 - 1e-6].  A tanh interface profile of width W' becomes one of
 * width W' / ratio with the same phi = 1/2 level set; for a profile of width W
 * coarse-grained by 4 and refined bilinearly ratio ~ 1.35 restores W.
 * Restarting the solver from a field refined from a coarse grid otherwise
 * starts from a too-wide interface (the phase-field equation of
 * eq:lbe_interface relaxes it back, moving the interface while it does).
 * No counterpart in the paper.  Errors: LBM_NN_ERR_ARG (null, n < 1,
 * ratio <= 0). */
int lbm_nn_sharpen(float* phi, int64_t n, float ratio, void* stream);

/* Interface-localised mass projection of a phase field (n values): phi +=
 * c 4 q (1 - q), q = phi clamped to [0, 1], with c such that sum phi =
 * target before rounding (the correction vanishes in the pure phases).  sums: 2 doubles of scratch; on
 * return (after the stream completes) they hold sum phi and sum 4 phi (1 -
 * phi) of the field before the correction, summed in a fixed order (block
 * partials in scratch allocated and freed on `stream`), so the projection
 * is the same on every run. */
int lbm_nn_mass_project(float* phi, int64_t n, double target, double* sums, void* stream);

/* Comparison of the phase fields a (e.g. a prediction) and b (the solver's)
 * on an ny x nx grid (x fastest): out[0] = cells on different sides of
 * phi = 1/2, out[1] = grid edges across which b crosses 1/2 (x-neighbours
 * periodic), out[2] = sum a, out[3] = sum b.  out[0] / out[1] is the mean
 * distance between the two interfaces in cells. */
int lbm_nn_interface_stats(const float* a, const float* b, int32_t ny, int32_t nx, double* out, void* stream);

/* Intact length of a jet issued along y from y = 0 (the quantity behind a
 * breakup length): per column x in [x0, x1) the number of cells from y = 0
 * up to the first phi <= 1/2; out[0] / out[1] = its largest value over the
 * columns for a / b (int32). */
int lbm_nn_jet_length(const float* a, const float* b, int32_t ny, int32_t nx, int32_t x0, int32_t x1, int32_t* out,
                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_NN_H */
