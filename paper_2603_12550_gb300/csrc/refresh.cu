// refresh.cu -- the pair pass that rebuilds the linearised Brownian terms of
// the reduced model (Sec. 2.4, Eq. model_DymReduced) at a lifted state.
//
// For each particle I and basis column t it accumulates
//   W1_(Ia)t = sum_K Z_IK Phi_(Ka)t,  W2_(Ia)t = sum_K Z_IK Phi_(Ka)t / rho_K,
//   c_I = sum_K Z_IK / rho_K,
// and writes U1 = Phi - W1 / rho_I and U2 = c Phi - W2, so that
//   X^B1 = -(1/h^2) Phi^T U1,  X^B2 = -(1/h^2) Phi^T U2
// (the row sum of Z is rho_I).
//
// Per pair the kernel value Z_IK costs 2D FP32 ops and one ex2; the 2 s r
// FMAs that follow dominate.  One CTA column chunk carries RT basis columns
// (RT in {4, 8, 12, 16}, chosen at launch to cover r with the fewest wasted
// columns), so for r <= 16 the kernel value is evaluated once per pair.
// Sums run in FP32: per 32-record j-tile into registers, then into per-
// particle totals (two-level summation; a single running FP32 sum over all
// N = 65536 terms loses about two more digits).
#include <math.h>

#include "pair.cuh"
#include "pod_internal.cuh"

namespace {

constexpr int RF_NT = 64;   // threads (particles) per CTA
constexpr int RF_TJ = 32;   // j records per shared-memory tile (divides the record padding)

// Resident CTAs per SM: 8 (128 registers) when the per-tile partials fit,
// else 6 (170 registers), or 5 (204) for the widest rows.
template <int D, int S, int RT>
struct RfOcc {
  static constexpr int value = (2 * S * RT <= 72) ? 8 : (D + 2 * S * RT <= 105 ? 6 : 5);
};

// One thread per particle I, RT columns of one chunk.  Per j-tile the sums go
// to register partials a1, a2; the per-particle totals live in shared memory
// (thread-private columns), which keeps the register count at the occupancy
// target.
template <int D, int S, int RT>
__global__ void __launch_bounds__(RF_NT, RfOcc<D, S, RT>::value)
    k_refresh(const float *__restrict__ rec, int N, const float *__restrict__ phi, int ld, int r,
              float *__restrict__ U1, float *__restrict__ U2) {
  constexpr int DP = Rec<D>::DP;
  constexpr int NC = S * RT;
  __shared__ __align__(16) float srec[RF_TJ * DP];
  __shared__ __align__(16) float sphi[RF_TJ][S][RT];
  __shared__ float W1s[NC][RF_NT], W2s[NC][RF_NT];
  const int tid = threadIdx.x;
  const int i = blockIdx.x * RF_NT + tid;
  const int t0 = blockIdx.y * RT;
  const bool vi = i < N;
  const int ic = vi ? i : N - 1;
  float xi[D];
#pragma unroll
  for (int d = 0; d < D; ++d) xi[d] = rec[(size_t)ic * DP + d];
  const float wi = rec[(size_t)ic * DP + D];
#pragma unroll
  for (int k = 0; k < NC; ++k) W1s[k][tid] = W2s[k][tid] = 0.f;
  float cs = 0.f;

  for (int jt = 0; jt < N; jt += RF_TJ) {
    __syncthreads();
    {
      const float4 *src = reinterpret_cast<const float4 *>(rec + (size_t)jt * DP);
      float4 *dst = reinterpret_cast<float4 *>(srec);
      for (int e = tid; e < RF_TJ * DP / 4; e += RF_NT) dst[e] = src[e];
    }
    // basis rows of the tile: RT consecutive columns of row (J, a), as float4
    // (ld and t0 are multiples of 4; columns r..ld-1 of Phi are zero)
    for (int e = tid; e < RF_TJ * S * (RT / 4); e += RF_NT) {
      const int row = e / (RT / 4), v = e - row * (RT / 4);
      const int jj = row / S, a = row - jj * S;
      const int J = jt + jj;
      float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (J < N && t0 + 4 * v < ld)
        f = *reinterpret_cast<const float4 *>(phi + ((size_t)J * S + a) * ld + t0 + 4 * v);
      *reinterpret_cast<float4 *>(&sphi[jj][a][4 * v]) = f;
    }
    __syncthreads();
    float a1[S][RT], a2[S][RT], ac = 0.f;
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int t = 0; t < RT; ++t) a1[a][t] = a2[a][t] = 0.f;
#pragma unroll 2
    for (int j = 0; j < RF_TJ; ++j) {
      const float *rj = srec + j * DP;
      float r2 = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float dd = xi[d] - rj[d];
        r2 = fmaf(dd, dd, r2);
      }
      const float K = ex2_approx(-r2);
      const float kw = K * rj[D];
      ac += kw;
#pragma unroll
      for (int a = 0; a < S; ++a)
#pragma unroll
        for (int t = 0; t < RT; ++t) {
          const float f = sphi[j][a][t];
          a1[a][t] = fmaf(K, f, a1[a][t]);
          a2[a][t] = fmaf(kw, f, a2[a][t]);
        }
    }
    cs += ac;
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        W1s[a * RT + t][tid] += a1[a][t];
        W2s[a * RT + t][tid] += a2[a][t];
      }
  }
  if (!vi) return;
#pragma unroll
  for (int a = 0; a < S; ++a)
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      if (t0 + t >= r) continue;
      const size_t o = ((size_t)i * S + a) * ld + t0 + t;
      const float f = phi[o];
      U1[o] = f - W1s[a * RT + t][tid] * wi;
      U2[o] = cs * f - W2s[a * RT + t][tid];
    }
}

template <int D, int S, int RT>
int refresh_launch(vds_ctx *c, const pod_basis *b, int N, float *U1, float *U2) {
  dim3 grid((N + RF_NT - 1) / RF_NT, (b->r + RT - 1) / RT);
  k_refresh<D, S, RT><<<grid, RF_NT, 0, c->stream>>>((const float *)c->rec.ptr, N, b->phi, b->ld, b->r,
                                                     U1, U2);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// Column chunk width for r columns: the fewest issue slots per pair, counting
// 2 S RT FMAs, S RT / 4 shared loads and 2D + 3 kernel-value ops per chunk.
int choose_rt(int r, int S, int D) {
  int best = 16;
  double best_cost = 1e300;
  for (int rt : {4, 8, 12, 16}) {
    const int chunks = (r + rt - 1) / rt;
    const double cost = chunks * (2.0 * S * rt + S * rt / 4.0 + 2.0 * D + 3.0);
    if (cost < best_cost) {
      best_cost = cost;
      best = rt;
    }
  }
  return best;
}

template <int D, int S>
int refresh_impl(vds_ctx *c, const pod_basis *b, int N, float *U1, float *U2) {
  switch (choose_rt(b->r, S, D)) {
    case 4: return refresh_launch<D, S, 4>(c, b, N, U1, U2);
    case 8: return refresh_launch<D, S, 8>(c, b, N, U1, U2);
    case 12: return refresh_launch<D, S, 12>(c, b, N, U1, U2);
    default: return refresh_launch<D, S, 16>(c, b, N, U1, U2);
  }
}

}  // namespace

int pod_refresh_dev(vds_ctx *c, const pod_basis *b, int N, int D, float *U1, float *U2) {
  const int s = b->s;
  VDS_TRY(vds_time_begin(c, PK_REFRESH));
  int st = VDS_EARG;
#define RF(DD, SS) \
  else if (D == DD && s == SS) st = refresh_impl<DD, SS>(c, b, N, U1, U2);
  if (false) {
  }
  RF(2, 2) RF(3, 3) RF(4, 2) RF(6, 2) RF(6, 3) RF(8, 2) RF(9, 3) RF(10, 2) RF(12, 2) RF(12, 3)
  RF(14, 2) RF(15, 3) RF(16, 2)
#undef RF
  VDS_TRY(st);
  VDS_TRY(vds_time_end(c, PK_REFRESH));
  return VDS_OK;
}
