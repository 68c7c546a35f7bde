/*
 * vds_pod.h -- C ABI of the POD model-order reduction (Sec. 2.3-2.4, Sec. 3.1)
 * of the VDS hot path: snapshot Gram, FP64 eigensolve, rank rule, basis, the
 * project / lift maps of Eq. model_pq and the reduced-order step of
 * Eq. model_DymReduced.  Same conventions as vds.h.
 */
#ifndef VDS_POD_H
#define VDS_POD_H

#include "vds.h"

#ifdef __cplusplus
extern "C" {
#endif

/* POD by the method of snapshots (Sec. 2.3, Sec. 3.1).
 * X: device, column-major (N s) x M snapshot matrix, one column per
 * (snapshot l, bond k) = q_k(t_l) flattened over rows (I, alpha).
 * C = X^T X (M x M) on the tensor cores: TF32 with one refinement step (each
 * FP32 value split into two TF32 parts, three products per pair), FP32
 * tensor-memory sums over 32-row chunks, Kahan-compensated FP32 across
 * chunks and FP64 across K splits; C = V Lambda V^T by cyclic Jacobi in FP64;
 * rank r = r_fixed if > 0, else
 * the smallest r with sum_{i<=r} lambda_i >= energy * sum_i lambda_i,
 * capped at r_max (<= 64), and reduced to the number of leading eigenvalues
 * that are positive and above 1e-13 lambda_1 (a rank beyond them cannot be
 * normalised; *r reports the rank used); Phi = X V_r Lambda_r^(-1/2), re-orthonormalised
 * by one Cholesky-QR pass; sign: the largest-magnitude entry of each column
 * is positive (ties: lowest row).  kappa (host, s x s) gives
 * X^H = Phi^T (I (x) kappa) Phi (Sec. 2.4).  *out receives a new basis owned
 * by the caller (pod_free); *r (host) the rank.  M <= 2048. */
VDS_API int pod_build(vds_ctx *ctx, const float *X, long Ns, int M, int s,
              double energy, int r_max, int r_fixed, const double *kappa,
              pod_basis **out, int *r);
/* A basis supplied by the caller (one stored from an earlier pod_build, or
 * computed elsewhere): phi device, (N s) x r row-major FP32 with orthonormal
 * columns (not checked), 1 <= r <= 64; kappa (host, s x s) gives X^H as in
 * pod_build.  The basis holds no eigenvalues (pod_eigenvalues copies none).
 * *out receives a new basis owned by the caller (pod_free). */
VDS_API int pod_load(vds_ctx *ctx, const float *phi, long Ns, int r, int s, const double *kappa,
                     pod_basis **out);
/* Basis accessors: Phi (device, (N s) x r row-major, leading dimension *ld),
 * eigenvalues (host copy, M values, descending), X^H (host, r x r). */
VDS_API int pod_info(const pod_basis *b, int *r, int *ld, const float **phi_dev,
             long *Ns);
VDS_API int pod_eigenvalues(const pod_basis *b, double *lam_host, int M);
/* Number of cyclic Jacobi sweeps pod_build ran (0 for pod_load, VDS_EARG for
 * NULL); the eigensolve stops when every off-diagonal entry is below
 * 1e-11 ||C||_F or the off-diagonal norm stops falling. */
VDS_API int pod_sweeps(const pod_basis *b);
VDS_API int pod_xh(const pod_basis *b, double *xh_host);
/* p_{k:} = Phi^T q_{k:} (Eq. model_pq).  q: device N x D; p: device r x nb
 * row-major (p[t*nb + k]). */
VDS_API int pod_project(vds_ctx *ctx, const pod_basis *b, const float *q, int N, int D,
                float *p);
/* q~_{k:} = Phi p_{k:} (Eq. model_pq).  p: device r x nb; q: device N x D. */
VDS_API int pod_lift(vds_ctx *ctx, const pod_basis *b, const float *p, int N, int D,
             float *q);
VDS_API void pod_free(pod_basis *b);

/* Frozen Brownian matrices of Sec. 2.4 at the lifted state q~ = Phi P
 * (P: device r x nb):
 *   X^B1_st = -(1/h^2) sum_(I a) Phi_(Ia)s sum_K Z_IK (Phi_(Ia)t - Phi_(Ka)t) / rho_I
 *   X^B2_st = -(1/h^2) sum_(I a) Phi_(Ia)s sum_K Z_IK (Phi_(Ia)t - Phi_(Ka)t) / rho_K
 * with Z_IK = exp(-|q~_I - q~_K|^2 / 2h^2) and rho_I = sum_J Z_IJ at q~.
 * xb1, xb2: host r x r row-major (either may be NULL). */
VDS_API int pod_brownian(vds_ctx *ctx, const pod_basis *b, const float *P, int N, int D,
                         const vds_params *p, double *xb1, double *xb2);

/* Reduced-order stepping of P (device r x nb, in/out) by nsteps explicit
 * Euler steps of size p->dt.
 * mode 1, Galerkin projection (Eq. model_DymRepParPod): Pdot = Phi^T v(Phi P)
 *   with v the full-order particle velocity of Eq. model_DymRepPar.
 * mode 2, the accelerated POD-MOR of Eq. model_DymReduced:
 *   Pdot = X^H P - (kBT/zeta)(X^B1 + X^B2) P A - (1/zeta) P diag(H) A,
 *   X^B1 + X^B2 rebuilt at the lifted state every refresh_every steps and
 *   frozen in between (Hookean springs only; FENE returns VDS_EARG).
 * The basis must come from snapshots of N particles of the same s. */
VDS_API int pod_step(vds_ctx *ctx, const pod_basis *b, float *P, int N, int D,
                     const vds_params *p, int nsteps, int refresh_every, int mode);

/* Reduced-order stepping with the learned score surrogate (include/
 * vds_score.h; not in the paper): as pod_step mode 1 but with the O(N^2)
 * entropy gradient S replaced by the network's score at the lifted state,
 * mean-centred over the particles (the exact S sums to zero):
 *   Pdot = Phi^T [kappa q~ - (1/zeta)(A (x) I)(kBT (s - mean s) + grad Psi(q~))].
 * Every check_every steps (0: never) the exact S of check_n particles (every
 * (N/check_n)-th) is evaluated (a full density pass, then the gradient of
 * those rows only) and compared by ||s - mean s - S|| / ||S||; above
 * check_tol that step uses the exact S of every particle (fallback).
 * check_err (host, may be NULL) receives the largest relative error seen,
 * fallbacks (host, may be NULL) their number.  The steps between checks
 * (after the first step of the call) replay one CUDA graph captured on a
 * private stream and launched on the context's stream. */
#ifndef VDS_SCORE_TYPEDEF
#define VDS_SCORE_TYPEDEF
typedef struct vds_score vds_score;
#endif
VDS_API int pod_step_score(vds_ctx *ctx, const pod_basis *b, vds_score *score, float *P, int N,
                           int D, const vds_params *p, int nsteps, int check_every, int check_n,
                           double check_tol, double *check_err, int *fallbacks);

#ifdef __cplusplus
}
#endif
#endif /* VDS_POD_H */
