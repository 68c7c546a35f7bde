/*
 * vds_score.h -- C ABI of the learned score surrogate: an MLP
 * s_theta: R^D -> R^D (D -> 256 -> 256 -> 256 -> D, SiLU hidden layers) that
 * approximates the score grad ln f of the particle density, trained by
 * denoising score matching (noise level sigma = the kernel bandwidth h) on
 * particle configurations produced by VDS itself, and used in place of the
 * O(N^2) entropy gradient inside the reduced-order step.  Not in the paper;
 * an extension of its Sec. 2.4 acceleration.  BF16 weights and activations
 * with FP32 accumulation on the tensor cores; FP32 master weights and Adam.
 *
 * Parameters (host, FP32, flat): W1 (256 x D, row-major), b1 (256),
 * W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (D x 256), b4 (D); see
 * vds_score_param_count.  Same status codes and conventions as vds.h.
 */
#ifndef VDS_SCORE_H
#define VDS_SCORE_H

#include "vds.h"

#ifdef __cplusplus
extern "C" {
#endif

#ifndef VDS_SCORE_TYPEDEF
#define VDS_SCORE_TYPEDEF
typedef struct vds_score vds_score;
#endif

VDS_API long vds_score_param_count(int D, int width);
/* Create a network with input/output dimension D (<= 16), width 256, from
 * the given initial parameters (host).  Adam state starts at zero. */
VDS_API int vds_score_create(vds_ctx *ctx, int D, int width, const float *params, vds_score **out);
VDS_API void vds_score_free(vds_score *s);
VDS_API int vds_score_set_params(vds_ctx *ctx, vds_score *s, const float *params);
VDS_API int vds_score_get_params(vds_ctx *ctx, const vds_score *s, float *params);
/* out (device, N x D) = s_theta(x) for x (device, N x D), all four layers
 * in one persistent tensor-core launch (the activations of each 128-row
 * tile stay on chip).  Its SiLU uses the hardware tanh, z sigma(z) =
 * h (1 + tanh h) with h = z/2, so outputs differ from the training forward's
 * by far less than the BF16 rounding of the activations.  The first call
 * after the parameters change repacks the BF16 weights (one extra launch). */
VDS_API int vds_score_eval(vds_ctx *ctx, vds_score *s, const float *x, int N, float *out);
/* Denoising score-matching loss on a batch of M rows (M a multiple of 128):
 * L = (1/M) sum_m |s_theta(x_m + sigma eps_m) + eps_m/sigma|^2 and its
 * gradient (host, flat as the parameters, may be NULL); *loss host.  The
 * batch rows are x[rows[m]] when rows (device, M ints) is given, else x[m]
 * (x device, rows x D); eps device M x D. */
VDS_API int vds_score_loss_grad(vds_ctx *ctx, vds_score *s, const float *x, const int *rows,
                                const float *eps, int M, double sigma, double *loss, float *grads);
/* One Adam step (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the
 * gradient of the DSM loss of the batch; *loss (host, may be NULL). */
VDS_API int vds_score_train(vds_ctx *ctx, vds_score *s, const float *x, const int *rows,
                            const float *eps, int M, double sigma, double lr, double *loss);

/* Supervised fit to given target scores (e.g. the exact VDS entropy gradient
 * of the same particles, which carries the second, 1/rho_J term of
 * Eq. model_DymRepPar that the denoising objective does not see):
 *   L = (1/M) sum_m |s_theta(x_m) - t_m|^2,
 * rows as in vds_score_loss_grad (t_m = target[rows[m]] when rows is given).
 * lr > 0 takes one Adam step; grads (host, may be NULL) as in
 * vds_score_loss_grad; *loss host (may be NULL). */
VDS_API int vds_score_fit(vds_ctx *ctx, vds_score *s, const float *x, const int *rows,
                          const float *target, int M, double lr, double *loss, float *grads);

#ifdef __cplusplus
}
#endif
#endif /* VDS_SCORE_H */
