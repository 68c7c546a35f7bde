// pod_internal.cuh -- the POD basis object and helpers shared by pod.cu and
// reduced.cu (not part of the public ABI).
#pragma once
#include "../../include/vds_pod.h"
#include "vds_internal.cuh"

struct pod_basis {
  int device = 0;
  long Ns = 0;
  int M = 0, r = 0, ld = 0, s = 0;
  int sweeps = 0;              // Jacobi sweeps of the eigensolve (0 for pod_load)
  float *phi = nullptr;        // device, Ns x ld row-major (columns >= r zero)
  double *lam = nullptr;       // host, M eigenvalues descending
  double *xh = nullptr;        // host, r x r
};

// C (device, M x M FP64) = X^T X for column-major FP32 X (Ns x M) on the
// tensor cores (3xTF32, FP64 across 512-row segments; gram_tc.cu); `part` is
// device workspace of pod_gram_tc_workspace bytes.
size_t pod_gram_tc_workspace(const vds_ctx *c, long Ns, int M);
int pod_gram_tc(vds_ctx *c, const float *X, long Ns, int M, double *part, double *C);
// G (device, r x r FP64) = A^T B for row-major Ns x ld FP32 matrices.
int pod_tsgram(vds_ctx *c, const float *A, const float *B, long Ns, int ld, int r, double *G);
// P = Phi^T q (r x nb) into pd (FP64, may be NULL) and/or pf (FP32, may be NULL).
int pod_project_dev(vds_ctx *c, const pod_basis *b, const float *q, int N, int D, double *pd, float *pf);
// The projection's split over CTAs (nblk CTAs of per_cta contiguous
// particles) and its final step: per-CTA FP64 partials [nblk][n] in
// ctx->gbuf summed in a fixed order into pd and/or pf (n = r nb values), for
// kernels that compute the projected field themselves (reduced.cu).
void pod_project_grid(const vds_ctx *c, int N, long &nblk, long &per_cta);
int pod_project_finish(vds_ctx *c, int n, long nblk, double *pd, float *pf);
// U1, U2 (Ns x ld, FP32) of the X^B refresh at the records in ctx->rec
// (refresh.cu); time kind PK_REFRESH.
int pod_refresh_dev(vds_ctx *c, const pod_basis *b, int N, int D, float *U1, float *U2);
// q = Phi P from FP32 P (r x nb).
int pod_lift_dev(vds_ctx *c, const pod_basis *b, const float *p, int N, int D, float *q);
