// pair.cu -- dispatch of the pair passes over the supported D = nb*s and the
// parameters they take; the kernels themselves are in pair_impl.cuh,
// instantiated once per D in pair_d<D>.cu.
#include <math.h>

#include "pair.cuh"
#include "pair_impl.cuh"

namespace {
__global__ void k_axpy(int n, const float *__restrict__ a, const float *__restrict__ b,
                       float *__restrict__ o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] + b[i];
}

}  // namespace

// Supported D = nb * s with s in {2,3}, nb <= 8, D <= 16.
#define VDS_DISPATCH_D(D, CALL)                          \
  switch (D) {                                           \
    case 2: return CALL(2);                              \
    case 3: return CALL(3);                              \
    case 4: return CALL(4);                              \
    case 6: return CALL(6);                              \
    case 8: return CALL(8);                              \
    case 9: return CALL(9);                              \
    case 10: return CALL(10);                            \
    case 12: return CALL(12);                            \
    case 14: return CALL(14);                            \
    case 15: return CALL(15);                            \
    case 16: return CALL(16);                            \
    default: return VDS_EARG;                            \
  }

int vds_prep_2(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_2(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_2(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_2(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_2(vds_ctx *, const KParams &, const float *, float *);
int vds_query_2(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_3(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_3(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_3(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_3(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_3(vds_ctx *, const KParams &, const float *, float *);
int vds_query_3(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_4(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_4(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_4(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_4(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_4(vds_ctx *, const KParams &, const float *, float *);
int vds_query_4(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_6(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_6(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_6(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_6(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_6(vds_ctx *, const KParams &, const float *, float *);
int vds_query_6(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_8(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_8(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_8(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_8(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_8(vds_ctx *, const KParams &, const float *, float *);
int vds_query_8(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_9(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_9(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_9(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_9(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_9(vds_ctx *, const KParams &, const float *, float *);
int vds_query_9(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_10(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_10(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_10(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_10(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_10(vds_ctx *, const KParams &, const float *, float *);
int vds_query_10(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_12(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_12(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_12(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_12(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_12(vds_ctx *, const KParams &, const float *, float *);
int vds_query_12(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_14(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_14(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_14(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_14(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_14(vds_ctx *, const KParams &, const float *, float *);
int vds_query_14(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_15(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_15(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_15(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_15(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_15(vds_ctx *, const KParams &, const float *, float *);
int vds_query_15(vds_ctx *, const KParams &, const float *, const float *, int, float *);
int vds_prep_16(vds_ctx *, const KParams &, const float *, const float *, const float *, float, float *);
int vds_density_16(vds_ctx *, const KParams &, float *, bool, const float *, const float *, const float *, const float *, bool);
int vds_grad_16(vds_ctx *, const KParams &, int, float *, const float *, const float *, const float *, const float *, float *);
int vds_stress_16(vds_ctx *, const KParams &, const float *, double *, double *);
int vds_flow_16(vds_ctx *, const KParams &, const float *, float *);
int vds_query_16(vds_ctx *, const KParams &, const float *, const float *, int, float *);

int vds_rowsdens_2(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_2(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_3(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_3(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_4(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_4(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_6(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_6(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_8(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_8(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_9(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_9(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_10(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_10(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_12(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_12(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_14(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_14(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_15(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_15(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);
int vds_rowsdens_16(vds_ctx *, const KParams &, const float *, int, int, float *);
int vds_rowsgrad_16(vds_ctx *, const KParams &, const float *, const float *, int, int, int, float *);

KParams make_kparams(const vds_params *p, int N, int D) {
  KParams k;
  k.N = N;
  k.D = D;
  k.nb = p->nb;
  k.s = p->s;
  k.spring = p->spring;
  k.h = p->h;
  k.kBT = p->kBT;
  k.zeta = p->zeta;
  k.dt = p->dt;
  k.b = p->b;
  for (int j = 0; j < 8; ++j) k.H[j] = p->H[j];
  for (int j = 0; j < 9; ++j) k.kappa[j] = p->kappa[j];
  const double c = sqrt(1.4426950408889634 / (2.0 * p->h * p->h));  // log2(e)/(2h^2)
  k.c = (float)c;
  k.sfac = 1.0 / (p->h * p->h * (double)k.c);
  k.lnorm = -log((double)N) - 0.5 * D * log(2.0 * 3.14159265358979323846 * p->h * p->h);
  return k;
}

int pass_npad(int N) { return (N + vds_pair::TJ - 1) / vds_pair::TJ * vds_pair::TJ; }

int pass_prep(vds_ctx *c, const KParams &kp, const float *base, const float *delta,
              const float *dir, float alpha, float *delta_out) {
#define CALL(DD) vds_prep_##DD(c, kp, base, delta, dir, alpha, delta_out)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_density(vds_ctx *c, const KParams &kp, float *rho_out, bool want_energy,
                 const float *ybase, const float *ydelta, const float *qa, const float *qb, bool expand) {
#define CALL(DD) vds_density_##DD(c, kp, rho_out, want_energy, ybase, ydelta, qa, qb, expand)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_grad(vds_ctx *c, const KParams &kp, int mode, float *out, const float *ybase,
              const float *ydelta, const float *qa, const float *qb, float *q_io) {
#define CALL(DD) vds_grad_##DD(c, kp, mode, out, ybase, ydelta, qa, qb, q_io)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_stress(vds_ctx *c, const KParams &kp, const float *q, double *tau, double *qq) {
#define CALL(DD) vds_stress_##DD(c, kp, q, tau, qq)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_flow(vds_ctx *c, const KParams &kp, const float *q, float *qs) {
#define CALL(DD) vds_flow_##DD(c, kp, q, qs)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_density_at(vds_ctx *c, const KParams &kp, const float *q, const float *y, int M, float *f_out) {
#define CALL(DD) vds_query_##DD(c, kp, q, y, M, f_out)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_density_rows(vds_ctx *c, const KParams &kp, const float *q, int row0, int nrows, float *rho) {
#define CALL(DD) vds_rowsdens_##DD(c, kp, q, row0, nrows, rho)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_grad_rows(vds_ctx *c, const KParams &kp, const float *q, const float *rho, int row0, int nrows,
                   int mode, float *out) {
#define CALL(DD) vds_rowsgrad_##DD(c, kp, q, rho, row0, nrows, mode, out)
  VDS_DISPATCH_D(kp.D, CALL)
#undef CALL
}

int pass_axpy(vds_ctx *c, int n, const float *base, const float *delta, float *out) {
  k_axpy<<<(n + 255) / 256, 256, 0, c->stream>>>(n, base, delta, out);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}
