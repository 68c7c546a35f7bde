// reduced.cu -- the reduced-order (POD-MOR) steps of Sec. 2.3-2.4 on GB300.
//
// Mode 1, Galerkin (Eq. model_DymRepParPod): Pdot = Phi^T v(Phi P), the
//   full-order particle velocity at the lifted state, projected; explicit
//   Euler on P.  Costs a full density + gradient evaluation per step.
// Mode 2, frozen linearised Brownian terms (Eq. model_DymReduced):
//   Pdot = X^H P - (kBT/zeta)(X^B1 + X^B2) P A - (1/zeta) P diag(H) A,
//   with X^B1, X^B2 rebuilt every `refresh_every` steps at the lifted state
//   ("mapping back and forth", Sec. 2.4, Sec. 3.2) and frozen in between.
//
// The refresh is a pair pass over the lifted particles (refresh.cu) that
// writes U1 = Phi - W1 / rho_I and U2 = c Phi - W2 per particle, so that
//   X^B1 = -(1/h^2) Phi^T U1,  X^B2 = -(1/h^2) Phi^T U2;
// both contractions are FP64-accumulated tall-skinny Grams.
#include <math.h>

#include "../../include/vds_score.h"
#include "pair.cuh"
#include "pod_internal.cuh"

namespace {

struct RedParams {
  double kBT, zeta, dt;
  double H[8];
};

__device__ __forceinline__ double rA(int j, int k) {
  return j == k ? 2.0 : ((j - k == 1 || k - j == 1) ? -1.0 : 0.0);
}

// nsteps explicit Euler steps of Eq. model_DymReduced with frozen X^B, one
// block; P kept in FP64 (shared memory), written back to Pd and Pf.
__global__ void __launch_bounds__(512)
    k_reduced_euler(double *__restrict__ Pd, float *__restrict__ Pf, const double *__restrict__ XH,
                    const double *__restrict__ XB, int r, int nb, RedParams rp, int nsteps) {
  __shared__ double P[64 * 8], Pdot[64 * 8], Y[64 * 8];
  const int n = r * nb;
  for (int o = threadIdx.x; o < n; o += blockDim.x) P[o] = Pd[o];
  __syncthreads();
  for (int step = 0; step < nsteps; ++step) {
    // Y = X^B P
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
      const int t = o / nb, j = o - t * nb;
      double y = 0.0;
      for (int u = 0; u < r; ++u) y += XB[t * r + u] * P[u * nb + j];
      Y[o] = y;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
      const int t = o / nb, k = o - t * nb;
      double a = 0.0, b = 0.0, cc = 0.0;
      for (int u = 0; u < r; ++u) a += XH[t * r + u] * P[u * nb + k];
      for (int j = 0; j < nb; ++j) {
        const double A = rA(j, k);
        b += Y[t * nb + j] * A;
        cc += P[t * nb + j] * rp.H[j] * A;
      }
      Pdot[o] = a - (rp.kBT / rp.zeta) * b - cc / rp.zeta;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < n; o += blockDim.x) P[o] += rp.dt * Pdot[o];
    __syncthreads();
  }
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    Pd[o] = P[o];
    Pf[o] = (float)P[o];
  }
}

__global__ void k_f2d(const float *__restrict__ a, double *__restrict__ b, int n) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n) b[o] = (double)a[o];
}

__global__ void k_euler_p(double *__restrict__ Pd, float *__restrict__ Pf, const double *__restrict__ Pdot,
                          double dt, int n) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n) {
    const double v = Pd[o] + dt * Pdot[o];
    Pd[o] = v;
    Pf[o] = (float)v;
  }
}

__global__ void k_combine_xb(const double *__restrict__ G1, const double *__restrict__ G2, double scale,
                             double *__restrict__ XB, int n) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n) XB[o] = scale * (G1[o] + G2[o]);
}

// column means of an N x D matrix (D <= 16): up to CM_BLK CTAs, each over a
// contiguous range of rows; a thread sums the rows I0 + tid, I0 + tid + 256,
// ... in FP32 (a handful per thread), the CTA combines them in a fixed order
// (warp shuffle tree in FP32, then the warps in order in FP64), and one warp
// adds the CTA sums in order: the result does not depend on the schedule.
constexpr int CM_NT = 256;
constexpr int CM_BLK = 256;
__global__ void __launch_bounds__(CM_NT)
    k_colmean_part(const float *__restrict__ s, int N, int D, long per_cta, double *__restrict__ part) {
  __shared__ double red[CM_NT / 32][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long I0 = (long)blockIdx.x * per_cta, I1 = min((long)N, I0 + per_cta);
  float acc[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) acc[a] = 0.f;
  for (long I = I0 + threadIdx.x; I < I1; I += CM_NT) {
#pragma unroll
    for (int a = 0; a < 16; ++a)
      if (a < D) acc[a] += s[(size_t)I * D + a];
  }
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    float v = acc[a];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][a] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < D) {
    double v = 0.0;
    for (int w = 0; w < CM_NT / 32; ++w) v += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * 16 + threadIdx.x] = v;
  }
}
// one warp per column: lanes take every 32nd CTA sum, then a fixed shuffle tree
__global__ void k_colmean(const double *__restrict__ part, int nblk, int N, int D, double *__restrict__ mean,
                          float *__restrict__ meanf) {
  const int a = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a >= D) return;
  double v = 0.0;
  for (int b = lane; b < nblk; b += 32) v += part[(size_t)b * 16 + a];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    mean[a] = v / (double)N;
    meanf[a] = (float)(v / (double)N);
  }
}
// the grid of k_colmean_part for N rows
inline void colmean_grid(const vds_ctx *c, int N, int &nblk, long &per_cta) {
  long nb = (N + CM_NT - 1) / CM_NT;
  const long cap = 2L * c->num_sms < CM_BLK ? 2L * c->num_sms : CM_BLK;
  if (nb > cap) nb = cap;
  per_cta = (N + nb - 1) / nb;
  nblk = (int)((N + per_cta - 1) / per_cta);
}

// particle velocity with the entropy gradient replaced by the surrogate
// (mean-centred): v = kappa q - (1/zeta)(A (x) I)(kBT (s - mean s) + grad Psi),
// in FP32 (the inputs and the output are FP32); A is the Rouse matrix, so
// (A g)_k = 2 g_k - g_(k-1) - g_(k+1) per bond k.
// the step's constants in FP32, converted once on the host (a conversion
// from FP64 per particle would run on this GPU's narrow FP64 pipe)
struct VelF {
  float kappa[9];
  float H[8];
  float kBT, izeta, b;
  int spring, N;
};

// v of one particle from its connectors y and its score (FP32)
template <int D, int S>
__device__ __forceinline__ void score_velocity(const VelF &vf, const float (&y)[D], const float *__restrict__ si,
                                               const float *__restrict__ smean, float (&v)[D], int *err) {
  constexpr int NB = D / S;
  float g[D];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    float f = vf.H[k];
    if (vf.spring != 0) {
      float n2 = 0.f;
#pragma unroll
      for (int al = 0; al < S; ++al) n2 = fmaf(y[k * S + al], y[k * S + al], n2);
      const float x = 1.f - n2 / vf.b;
      if (!(x > 0.f)) vds_flag(err, VDS_EDOMAIN);
      f = x > 0.f ? f / x : 0.f;
    }
#pragma unroll
    for (int al = 0; al < S; ++al) {
      const int a = k * S + al;
      const float sm = smean ? smean[a] : 0.f;
      g[a] = fmaf(vf.kBT, si[a] - sm, f * y[a]);
    }
  }
#pragma unroll
  for (int k = 0; k < NB; ++k)
#pragma unroll
    for (int al = 0; al < S; ++al) {
      const int a = k * S + al;
      float vv = 0.f;
#pragma unroll
      for (int be = 0; be < S; ++be) vv = fmaf(vf.kappa[al * S + be], y[k * S + be], vv);
      float m = 2.f * g[a];
      if (k > 0) m -= g[a - S];
      if (k < NB - 1) m -= g[a + S];
      v[a] = fmaf(-vf.izeta, m, vv);
    }
}

constexpr int VP_NT = 256;  // threads per CTA
constexpr int VP_TT = 8;    // basis columns per pass

// The surrogate step's velocity and its projection in one pass: per-CTA
// partials part[blk][t nb + k] = sum over the CTA's particles I (a
// contiguous range of per_cta) of sum_a Phi[(I s + a), t] v_I[s k + a], with
// v_I the velocity above; the velocity is never written to memory.  Each
// thread keeps VP_TT x nb FP32 sums per pass over the basis columns; the CTA
// combines them in a fixed order (warp shuffle tree, then the warps in order
// in FP64), so the result does not depend on the schedule.
template <int D, int S>
__global__ void __launch_bounds__(VP_NT)
    k_vel_project(VelF vf, const float *__restrict__ q, const float *__restrict__ sc,
                  const float *__restrict__ smean, const float *__restrict__ phi, int ld, int r, long per_cta,
                  double *__restrict__ part, int *err) {
  constexpr int NB = D / S;
  __shared__ double red[VP_NT / 32][VP_TT * NB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long I0 = (long)blockIdx.x * per_cta, I1 = min((long)vf.N, I0 + per_cta);
  for (int t0 = 0; t0 < r; t0 += VP_TT) {
    float acc[VP_TT][NB];
#pragma unroll
    for (int tt = 0; tt < VP_TT; ++tt)
#pragma unroll
      for (int k = 0; k < NB; ++k) acc[tt][k] = 0.f;
    for (long I = I0 + threadIdx.x; I < I1; I += VP_NT) {
      float y[D], v[D];
#pragma unroll
      for (int a = 0; a < D; ++a) y[a] = q[(size_t)I * D + a];
      score_velocity<D, S>(vf, y, sc + (size_t)I * D, smean, v, err);
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const float *row = phi + ((size_t)I * S + a) * ld + t0;
        float ph[VP_TT];
#pragma unroll
        for (int tt = 0; tt < VP_TT; ++tt) ph[tt] = t0 + tt < r ? row[tt] : 0.f;
#pragma unroll
        for (int tt = 0; tt < VP_TT; ++tt)
#pragma unroll
          for (int k = 0; k < NB; ++k) acc[tt][k] = fmaf(ph[tt], v[k * S + a], acc[tt][k]);
      }
    }
#pragma unroll
    for (int tt = 0; tt < VP_TT; ++tt)
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        float x = acc[tt][k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][tt * NB + k] = (double)x;
      }
    __syncthreads();
    if (threadIdx.x < VP_TT * NB) {
      const int tt = threadIdx.x / NB, k = threadIdx.x % NB;
      if (t0 + tt < r) {
        double x = 0.0;
        for (int w = 0; w < VP_NT / 32; ++w) x += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * (r * NB) + (t0 + tt) * NB + k] = x;
      }
    }
    __syncthreads();
  }
}

// The exact entropy gradient S of the checked particles only (every
// stride-th, nrows of them) from records that carry w = 1/rho of all N: the
// gradient pair pass restricted to those rows.  grid.x covers the rows (128
// per CTA), grid.y splits the j range into segments whose FP64 partials are
// summed in a fixed order by k_grad_rows_sum; inside a segment FP32 sums per
// 128-record tile with Kahan compensation across tiles.
constexpr int GR_NT = 128;
constexpr int GR_TJ = 128;

template <int D>
__global__ void __launch_bounds__(GR_NT)
    k_grad_rows(const float *__restrict__ rec, int Npad, int stride, int nrows, int jseg,
                double *__restrict__ part) {
  constexpr int DP = Rec<D>::DP;
  __shared__ __align__(16) float srec[GR_TJ * DP];
  const int r = blockIdx.x * GR_NT + threadIdx.x;
  const long i = (long)(r < nrows ? r : nrows - 1) * stride;
  float xi[D];
#pragma unroll
  for (int d = 0; d < D; ++d) xi[d] = rec[i * DP + d];
  const float wi = rec[i * DP + D];
  float sum[D], cmp[D];
#pragma unroll
  for (int d = 0; d < D; ++d) sum[d] = cmp[d] = 0.f;
  const int j0 = blockIdx.y * jseg, j1 = min(Npad, j0 + jseg);
  for (int jt = j0; jt < j1; jt += GR_TJ) {
    __syncthreads();
    const float4 *src = reinterpret_cast<const float4 *>(rec + (size_t)jt * DP);
    float4 *dst = reinterpret_cast<float4 *>(srec);
    for (int e = threadIdx.x; e < GR_TJ * DP / 4; e += GR_NT) dst[e] = src[e];
    __syncthreads();
    float acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.f;
#pragma unroll 2
    for (int j = 0; j < GR_TJ; ++j) {
      const float *rj = srec + j * DP;
      float dd[D], r2 = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        dd[d] = xi[d] - rj[d];
        r2 = fmaf(dd[d], dd[d], r2);
      }
      const float u = ex2_approx(-r2) * (wi + rj[D]);
#pragma unroll
      for (int d = 0; d < D; ++d) acc[d] = fmaf(u, dd[d], acc[d]);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float y = acc[d] - cmp[d];
      const float t = sum[d] + y;
      cmp[d] = (t - sum[d]) - y;
      sum[d] = t;
    }
  }
  if (r >= nrows) return;
#pragma unroll
  for (int d = 0; d < D; ++d)
    part[((size_t)blockIdx.y * nrows + r) * D + d] = (double)sum[d] - (double)cmp[d];
}

// S_rows = -sfac * (sum over the j segments, in order); sfac = 1/(h^2 c)
__global__ void k_grad_rows_sum(const double *__restrict__ part, int nseg, int nrows, int D, double sfac,
                                float *__restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nrows * D) return;
  double v = 0.0;
  for (int k = 0; k < nseg; ++k) v += part[(size_t)k * nrows * D + e];
  S[e] = (float)(-sfac * v);
}

// sums over the checked particles of |s - mean s - S|^2 and |S|^2, with S
// given for the checked rows only (row r is particle r * stride)
__global__ void k_check_err(const float *__restrict__ sc, const double *__restrict__ smean,
                            const float *__restrict__ S, int nrows, int D, int stride, double *__restrict__ out) {
  __shared__ double sh[2][256];
  double e = 0.0, n = 0.0;
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    const long i = (long)r * stride;
    for (int a = 0; a < D; ++a) {
      const double Sv = (double)S[(size_t)r * D + a];
      const double d = (double)sc[i * D + a] - smean[a] - Sv;
      e += d * d;
      n += Sv * Sv;
    }
  }
  sh[0][threadIdx.x] = e;
  sh[1][threadIdx.x] = n;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
  }
}

// j segments of the checked-row gradient: about four CTAs per SM over the row
// blocks, segment length a multiple of the tile
void grad_rows_split(const vds_ctx *c, int N, int nrows, int &nseg, int &jseg) {
  const int Npad = pass_npad(N);
  const int rb = (nrows + GR_NT - 1) / GR_NT;
  nseg = (4 * c->num_sms + rb - 1) / rb;
  jseg = (Npad + nseg - 1) / nseg;
  jseg = (jseg + GR_TJ - 1) / GR_TJ * GR_TJ;
  nseg = (Npad + jseg - 1) / jseg;
}

size_t grad_rows_part_bytes(const vds_ctx *c, int N, int nrows, int D) {
  int nseg, jseg;
  grad_rows_split(c, N, nrows, nseg, jseg);
  return (size_t)nseg * nrows * D * sizeof(double);
}

template <int D>
int grad_rows_impl(vds_ctx *c, const KParams &kS, int stride, int nrows, double *part, float *Srows) {
  const int Npad = pass_npad(kS.N);
  const int rb = (nrows + GR_NT - 1) / GR_NT;
  int nseg, jseg;
  grad_rows_split(c, kS.N, nrows, nseg, jseg);
  k_grad_rows<D><<<dim3(rb, nseg), GR_NT, 0, c->stream>>>((const float *)c->rec.ptr, Npad, stride, nrows, jseg,
                                                          part);
  k_grad_rows_sum<<<(nrows * D + 255) / 256, 256, 0, c->stream>>>(part, nseg, nrows, D, kS.sfac, Srows);
  VDS_CUDA_TRY(cudaGetLastError());
  c->launches += 2;
  return VDS_OK;
}

int grad_rows(vds_ctx *c, const KParams &kS, int stride, int nrows, double *part, float *Srows) {
  switch (kS.D) {
    case 2: return grad_rows_impl<2>(c, kS, stride, nrows, part, Srows);
    case 3: return grad_rows_impl<3>(c, kS, stride, nrows, part, Srows);
    case 4: return grad_rows_impl<4>(c, kS, stride, nrows, part, Srows);
    case 6: return grad_rows_impl<6>(c, kS, stride, nrows, part, Srows);
    case 8: return grad_rows_impl<8>(c, kS, stride, nrows, part, Srows);
    case 9: return grad_rows_impl<9>(c, kS, stride, nrows, part, Srows);
    case 12: return grad_rows_impl<12>(c, kS, stride, nrows, part, Srows);
    default: return VDS_EARG;
  }
}

// Pdot (FP64 and/or FP32, r x nb) = Phi^T v, v the surrogate velocity of
// every particle (scores sc, mean-centred by smean when given)
template <int D, int S>
int vel_project_impl(vds_ctx *c, const KParams &kp, const pod_basis *b, const float *q, const float *sc,
                     const float *smean, double *pd) {
  VelF vf;
  for (int k = 0; k < 9; ++k) vf.kappa[k] = (float)kp.kappa[k];
  for (int k = 0; k < 8; ++k) vf.H[k] = (float)kp.H[k];
  vf.kBT = (float)kp.kBT;
  vf.izeta = (float)(1.0 / kp.zeta);
  vf.b = (float)kp.b;
  vf.spring = kp.spring;
  vf.N = kp.N;
  long nblk, per_cta;
  pod_project_grid(c, kp.N, nblk, per_cta);
  const int n = b->r * (D / S);
  VDS_TRY(vds_ensure(c, c->gbuf, (size_t)nblk * n * sizeof(double)));
  k_vel_project<D, S><<<(unsigned)nblk, VP_NT, 0, c->stream>>>(vf, q, sc, smean, b->phi, b->ld, b->r, per_cta,
                                                               (double *)c->gbuf.ptr, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return pod_project_finish(c, n, nblk, pd, nullptr);
}

int vel_project(vds_ctx *c, const KParams &kp, const pod_basis *b, const float *q, const float *sc,
                const float *smean, double *pd) {
  const int key = kp.D * 4 + kp.s;
  switch (key) {
    case 2 * 4 + 2: return vel_project_impl<2, 2>(c, kp, b, q, sc, smean, pd);
    case 3 * 4 + 3: return vel_project_impl<3, 3>(c, kp, b, q, sc, smean, pd);
    case 4 * 4 + 2: return vel_project_impl<4, 2>(c, kp, b, q, sc, smean, pd);
    case 6 * 4 + 2: return vel_project_impl<6, 2>(c, kp, b, q, sc, smean, pd);
    case 6 * 4 + 3: return vel_project_impl<6, 3>(c, kp, b, q, sc, smean, pd);
    case 8 * 4 + 2: return vel_project_impl<8, 2>(c, kp, b, q, sc, smean, pd);
    case 9 * 4 + 3: return vel_project_impl<9, 3>(c, kp, b, q, sc, smean, pd);
    case 12 * 4 + 2: return vel_project_impl<12, 2>(c, kp, b, q, sc, smean, pd);
    case 12 * 4 + 3: return vel_project_impl<12, 3>(c, kp, b, q, sc, smean, pd);
    default: return VDS_EARG;
  }
}

int check(const vds_params *p, const pod_basis *b, int N, int D) {
  if (!p || !b || N < 1 || D < 2 || D > VDS_MAXD) return VDS_EARG;
  if (p->s != b->s || p->nb * p->s != D || (long)N * b->s != b->Ns || p->nb > 8) return VDS_EARG;
  if (!(p->h > 0.0) || !(p->zeta > 0.0) || !(p->kBT >= 0.0)) return VDS_EARG;
  if (p->spring != 0 && p->spring != 1) return VDS_EARG;
  if (p->spring == 1 && !(p->b > 0.0)) return VDS_EARG;
  return VDS_OK;
}

struct Dev {
  int prev = -1, dev;
  explicit Dev(int d) : dev(d) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Dev() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

// The density of every particle of the records in ctx->rec for the passes
// held to 1e-4 or looser (the refresh's lifted state, the surrogate's
// subset check): the pair dot products on the tensor cores where the records
// allow it (D = 6, 9), else the expanded distances on the CUDA cores.  The
// tensor-core sums lose more to the |q|^2 terms at single particles (3.4e-4
// at the worst particle of a cloud stretched five-fold), but X^B, a sum over
// all particles, stays as close to the oracle as with the FP32 expanded form
// (N = 65536, r = 10: 3.8e-6 and 1.2e-5 relative at equilibrium and at a
// three-fold stretch, against 4.5e-6 and 1.5e-5).
int density_1e4(vds_ctx *c, const KParams &kp, const float *qt) {
  const int st = pass_density_tc(c, kp, nullptr);
  if (st != VDS_EARG) return st;
  return pass_density(c, kp, nullptr, false, qt, nullptr, nullptr, nullptr, true);
}

// Lift P, evaluate the density at the lifted state, run the refresh pass and
// the two contractions: G1 = Phi^T U1, G2 = Phi^T U2 (device FP64 r x r).
int brownian_dev(vds_ctx *c, const pod_basis *b, const float *P, int N, int D, const KParams &kp,
                 float *qt, float *U1, float *U2, double *G1, double *G2) {
  VDS_TRY(pod_lift_dev(c, b, P, N, D, qt));
  VDS_TRY(pass_prep(c, kp, qt, nullptr, nullptr, 0.f, nullptr));
  // the density at the lifted state feeds only the frozen terms (X^B within
  // 1e-4 of the FP64 oracle)
  VDS_TRY(density_1e4(c, kp, qt));
  VDS_TRY(pod_refresh_dev(c, b, N, D, U1, U2));
  VDS_TRY(pod_tsgram(c, b->phi, U1, b->Ns, b->ld, b->r, G1));
  VDS_TRY(pod_tsgram(c, b->phi, U2, b->Ns, b->ld, b->r, G2));
  return VDS_OK;
}

}  // namespace

extern "C" {

int pod_brownian(vds_ctx *c, const pod_basis *b, const float *P, int N, int D, const vds_params *p,
                 double *xb1, double *xb2) {
  if (!c || !P) return VDS_EARG;
  VDS_TRY(check(p, b, N, D));
  Dev dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  const size_t nd = (size_t)N * D, nu = (size_t)b->Ns * b->ld;
  const int r = b->r;
  VDS_TRY(vds_ensure(c, c->vecs, nd * sizeof(float)));
  VDS_TRY(vds_ensure(c, c->ubuf, 2 * nu * sizeof(float) + 2 * 4096 * sizeof(double)));
  float *U1 = (float *)c->ubuf.ptr, *U2 = U1 + nu;
  double *G1 = (double *)(U2 + nu), *G2 = G1 + 4096;
  VDS_TRY(brownian_dev(c, b, P, N, D, kp, (float *)c->vecs.ptr, U1, U2, G1, G2));
  const double scale = -1.0 / (p->h * p->h);
  if (xb1) VDS_CUDA_TRY(cudaMemcpyAsync(xb1, G1, sizeof(double) * r * r, cudaMemcpyDeviceToHost, c->stream));
  if (xb2) VDS_CUDA_TRY(cudaMemcpyAsync(xb2, G2, sizeof(double) * r * r, cudaMemcpyDeviceToHost, c->stream));
  VDS_TRY(vds_sync_status(c));
  for (int k = 0; k < r * r; ++k) {
    if (xb1) xb1[k] *= scale;
    if (xb2) xb2[k] *= scale;
  }
  return VDS_OK;
}

int pod_step(vds_ctx *c, const pod_basis *b, float *P, int N, int D, const vds_params *p, int nsteps,
             int refresh_every, int mode) {
  if (!c || !P || nsteps < 0 || (mode != 1 && mode != 2)) return VDS_EARG;
  VDS_TRY(check(p, b, N, D));
  if (!(p->dt > 0.0)) return VDS_EARG;
  if (mode == 2 && (p->spring != 0 || refresh_every < 1)) return VDS_EARG;
  if (nsteps == 0) return VDS_OK;
  Dev dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  const int r = b->r, nb = p->nb, n = r * nb;
  const size_t nd = (size_t)N * D, nu = (size_t)b->Ns * b->ld;
  VDS_TRY(vds_ensure(c, c->vecs, 2 * nd * sizeof(float)));
  float *qt = (float *)c->vecs.ptr, *vel = qt + nd;
  // small FP64 state: Pd, Pdot, XH, XB, G1, G2
  VDS_TRY(vds_ensure(c, c->ubuf, (mode == 2 ? 2 * nu * sizeof(float) : 0) + (2 * 512 + 4 * 4096) * sizeof(double)));
  float *U1 = (float *)c->ubuf.ptr, *U2 = U1 + (mode == 2 ? nu : 0);
  double *Pd = (double *)(U2 + (mode == 2 ? nu : 0));
  double *Pdot = Pd + 512, *XH = Pdot + 512, *XB = XH + 4096, *G1 = XB + 4096, *G2 = G1 + 4096;
  k_f2d<<<(n + 255) / 256, 256, 0, c->stream>>>(P, Pd, n);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  RedParams rp;
  rp.kBT = p->kBT;
  rp.zeta = p->zeta;
  rp.dt = p->dt;
  for (int j = 0; j < 8; ++j) rp.H[j] = p->H[j];
  if (mode == 2) {
    VDS_CUDA_TRY(cudaMemcpyAsync(XH, b->xh, sizeof(double) * r * r, cudaMemcpyHostToDevice, c->stream));
    const double scale = -1.0 / (p->h * p->h);
    for (int n0 = 0; n0 < nsteps;) {
      VDS_TRY(brownian_dev(c, b, P, N, D, kp, qt, U1, U2, G1, G2));
      k_combine_xb<<<(r * r + 255) / 256, 256, 0, c->stream>>>(G1, G2, scale, XB, r * r);
      const int m = (nsteps - n0) < refresh_every ? (nsteps - n0) : refresh_every;
      k_reduced_euler<<<1, 512, 0, c->stream>>>(Pd, P, XH, XB, r, nb, rp, m);
      VDS_CUDA_TRY(cudaGetLastError());
      c->launches += 2;
      n0 += m;
    }
  } else {
    for (int n0 = 0; n0 < nsteps; ++n0) {
      VDS_TRY(pod_lift_dev(c, b, P, N, D, qt));
      VDS_TRY(pass_prep(c, kp, qt, nullptr, nullptr, 0.f, nullptr));
      VDS_TRY(pass_density(c, kp, nullptr, false, qt, nullptr, nullptr, nullptr));
      VDS_TRY(pass_grad(c, kp, GM_VEL, vel, qt, nullptr, nullptr, nullptr, nullptr));
      VDS_TRY(pod_project_dev(c, b, vel, N, D, Pdot, nullptr));
      k_euler_p<<<(n + 255) / 256, 256, 0, c->stream>>>(Pd, P, Pdot, p->dt, n);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
    }
  }
  return vds_sync_status(c);
}

int pod_step_score(vds_ctx *c, const pod_basis *b, vds_score *sc, float *P, int N, int D, const vds_params *p,
                   int nsteps, int check_every, int check_n, double check_tol, double *check_err,
                   int *fallbacks) {
  if (!c || !P || !sc || nsteps < 0 || check_every < 0 || (check_every > 0 && check_n < 1)) return VDS_EARG;
  VDS_TRY(check(p, b, N, D));
  if (!(p->dt > 0.0)) return VDS_EARG;
  if (D != 2 && D != 3 && D != 4 && D != 6 && D != 8 && D != 9 && D != 12) return VDS_EARG;
  if (check_err) *check_err = 0.0;
  if (fallbacks) *fallbacks = 0;
  if (nsteps == 0) return VDS_OK;
  Dev dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  vds_params pS = *p;  // exact entropy gradient alone: kBT = 1, no springs
  pS.kBT = 1.0;
  pS.spring = 0;
  for (int j = 0; j < 8; ++j) pS.H[j] = 0.0;
  const KParams kS = make_kparams(&pS, N, D);
  const int r = b->r, nb = p->nb, n = r * nb;
  const size_t nd = (size_t)N * D;
  VDS_TRY(vds_ensure(c, c->vecs, 3 * nd * sizeof(float)));
  float *qt = (float *)c->vecs.ptr, *sbuf = qt + nd, *Sx = sbuf + nd;
  VDS_TRY(vds_ensure(c, c->ubuf, (2 * 512 + 64 + 16 * CM_BLK) * sizeof(double)));
  double *Pd = (double *)c->ubuf.ptr, *Pdot = Pd + 512, *smean = Pdot + 512, *errs = smean + 32,
         *cpart = errs + 32;
  float *smeanf = (float *)(smean + 16);  // FP32 copy of the means (D <= 16)
  k_f2d<<<(n + 255) / 256, 256, 0, c->stream>>>(P, Pd, n);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  const int stride = check_n >= N ? 1 : N / check_n;
  const int nrows = (N + stride - 1) / stride;
  int cm_nblk;
  long cm_per;
  colmean_grid(c, N, cm_nblk, cm_per);
  double worst = 0.0;
  int nfall = 0;
  // one surrogate step without a check: lift, network, mean, velocity and
  // projection (one pass), Euler update of P
  auto plain_step = [&]() -> int {
    VDS_TRY(pod_lift_dev(c, b, P, N, D, qt));
    VDS_TRY(vds_score_eval(c, sc, qt, N, sbuf));
    k_colmean_part<<<cm_nblk, CM_NT, 0, c->stream>>>(sbuf, N, D, cm_per, cpart);
    k_colmean<<<1, 32 * D, 0, c->stream>>>(cpart, cm_nblk, N, D, smean, smeanf);
    VDS_CUDA_TRY(cudaGetLastError());
    c->launches += 2;
    VDS_TRY(vel_project(c, kp, b, qt, sbuf, smeanf, Pdot));
    k_euler_p<<<(n + 255) / 256, 256, 0, c->stream>>>(Pd, P, Pdot, p->dt, n);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    return VDS_OK;
  };
  // Steps without a check replay one captured CUDA graph of plain_step (its
  // buffers are all sized by then: the first step runs uncaptured); if the
  // capture fails they are launched one by one.
  cudaGraphExec_t gexec = nullptr;
  long graph_kernels = 0;
  const void *graph_gbuf = nullptr;  // scratch the captured projection uses
  bool try_graph = true;
  struct GraphGuard {
    cudaGraphExec_t *g;
    ~GraphGuard() {
      if (*g) cudaGraphExecDestroy(*g);
    }
  } gguard{&gexec};
  for (int step = 0; step < nsteps; ++step) {
    const bool check_step = check_every > 0 && step % check_every == 0;
    if (!check_step && step > 0 && try_graph) {
      if (!gexec) {
        // captured on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured); nothing runs while
        // capturing, and the graph is then launched on the caller's stream
        const long l0 = c->launches;
        cudaGraph_t g = nullptr;
        int st = VDS_OK;
        cudaStream_t cs = nullptr, user = c->stream;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
          st = VDS_ECUDA;
        } else if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          st = VDS_ECUDA;
        } else {
          c->stream = cs;
          st = plain_step();
          c->stream = user;
          const cudaError_t ec = cudaStreamEndCapture(cs, &g);
          if (st == VDS_OK && ec != cudaSuccess) st = VDS_ECUDA;
        }
        c->stream = user;
        if (cs) cudaStreamDestroy(cs);
        if (st == VDS_OK && cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess) {
          gexec = nullptr;
          st = VDS_ECUDA;
        }
        if (g) cudaGraphDestroy(g);
        graph_kernels = c->launches - l0;
        c->launches = l0;
        graph_gbuf = c->gbuf.ptr;
        if (st != VDS_OK) {
          (void)cudaGetLastError();  // a failed capture leaves its status behind; launch directly instead
          try_graph = false;
        }
      }
      if (gexec) {
        VDS_CUDA_TRY(cudaGraphLaunch(gexec, c->stream));
        c->launches += graph_kernels;
        continue;
      }
    }
    if (!check_step) {
      VDS_TRY(plain_step());
      continue;
    }
    VDS_TRY(pod_lift_dev(c, b, P, N, D, qt));
    VDS_TRY(vds_score_eval(c, sc, qt, N, sbuf));
    k_colmean_part<<<cm_nblk, CM_NT, 0, c->stream>>>(sbuf, N, D, cm_per, cpart);
    k_colmean<<<1, 32 * D, 0, c->stream>>>(cpart, cm_nblk, N, D, smean, smeanf);
    VDS_CUDA_TRY(cudaGetLastError());
    c->launches += 2;
    bool exact = false;
    {
      // full density (every 1/rho_J enters S_I), gradient of the checked rows;
      // the density within about 1e-4 (against a check threshold of order 0.1
      // and a fallback step held to 1e-3)
      VDS_TRY(pass_prep(c, kS, qt, nullptr, nullptr, 0.f, nullptr));
      VDS_TRY(density_1e4(c, kS, qt));
      // compact exact S of the checked rows (after the FP64 segment partials)
      // in the shared scratch, taken afresh at every check
      const size_t rows_bytes = ((size_t)nrows * D * sizeof(float) + 255) / 256 * 256;
      VDS_TRY(vds_ensure(c, c->gbuf, rows_bytes + grad_rows_part_bytes(c, N, nrows, D)));
      float *Srows = (float *)c->gbuf.ptr;
      double *rows_part = (double *)((char *)c->gbuf.ptr + rows_bytes);
      VDS_TRY(grad_rows(c, kS, stride, nrows, rows_part, Srows));
      k_check_err<<<1, 256, 0, c->stream>>>(sbuf, smean, Srows, nrows, D, stride, errs);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
      double h_err[2];
      VDS_CUDA_TRY(cudaMemcpyAsync(h_err, errs, sizeof(h_err), cudaMemcpyDeviceToHost, c->stream));
      VDS_TRY(vds_sync_status(c));
      const double rel = h_err[1] > 0.0 ? sqrt(h_err[0] / h_err[1]) : 0.0;
      if (rel > worst) worst = rel;
      if (!(rel <= check_tol)) {
        // fall back: the exact gradient of every particle for this step
        VDS_TRY(pass_grad(c, kS, GM_OUT, Sx, qt, nullptr, nullptr, nullptr, nullptr));
        exact = true;
        ++nfall;
      }
    }
    VDS_TRY(vel_project(c, kp, b, qt, exact ? Sx : sbuf, exact ? nullptr : smeanf, Pdot));
    k_euler_p<<<(n + 255) / 256, 256, 0, c->stream>>>(Pd, P, Pdot, p->dt, n);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    if (gexec && c->gbuf.ptr != graph_gbuf) {
      // the check grew the scratch the captured projection writes into:
      // capture again before the next plain step
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
  }
  if (check_err) *check_err = worst;
  if (fallbacks) *fallbacks = nfall;
  return vds_sync_status(c);
}

}  // extern "C"
