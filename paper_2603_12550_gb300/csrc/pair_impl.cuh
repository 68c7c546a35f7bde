#pragma once
// pair_impl.cuh -- the O(N^2) Gaussian-kernel pair passes of the VDS hot path and
// their fused O(N) epilogues, for GB300 (sm_103a).
//
// Density pass (Eq. model_DeteParAppr, denominators of Eq. model_DymRepPar):
//   rho_I = sum_J exp2(-|qhat_I - qhat_J|^2),  qhat = c q,  c^2 = log2(e)/(2h^2)
// Gradient pass (Eq. model_DymRepPar with grad K = -(x/h^2) K):
//   S_I = -(1/(h^2 c)) sum_J khat_IJ (w_I + w_J)(qhat_I - qhat_J),  w = 1/rho.
//
// Each CTA owns a contiguous range of (i-tile, j-chunk) items (stream-K),
// keeps RI particles per thread in registers and streams j-tiles of particle
// records through a ring of shared-memory stages filled by TMA bulk copies
// (cp.async.bulk + mbarrier transaction counts) issued by one thread.  All
// threads read the same record at a time (shared-memory broadcast).  Inside a
// j-tile sums are plain FP32; across tiles they are Kahan-compensated; across
// CTAs they are combined in FP64 by the epilogue in a fixed order.
#include <math.h>

#include "pair.cuh"

namespace vds_pair {

// Tile shape (overridable at build time for tuning sweeps).
#ifndef VDS_PAIR_TJ
#define VDS_PAIR_TJ 256
#endif
#ifndef VDS_PAIR_NSTAGE
#define VDS_PAIR_NSTAGE 3
#endif
constexpr int TJ = VDS_PAIR_TJ;          // records per j-tile (= j-chunk)
constexpr int NSTAGE = VDS_PAIR_NSTAGE;  // shared-memory ring depth

// Threads per CTA and particles per thread of each pass.  D = 9 takes the
// fastest shapes of a sweep on GB300 at N = 65536 (density 512 x 4, gradient
// 384 x 3: 2.46 + 3.86 ms against 2.51 + 3.99 ms for 256 x 4 in both); other
// D keep 256 threads, 4 particles per thread, 2 for the gradient above D = 9
// (255 registers).
template <int D>
struct PairCfg {
  static constexpr int NT_DENS = (D == 9) ? 512 : 256;
  static constexpr int RI_DENS = 4;
  static constexpr int NT_GRAD = (D == 9) ? 384 : 256;
  static constexpr int RI_GRAD = (D <= 6) ? 4 : (D == 9 ? 3 : (D <= 9 ? 4 : 2));
};

// Small clouds (the paper's P = 1000 workloads, the 2D dumbbell): with the
// shapes above the (i-tile, j-chunk) items would cover fewer than half the
// SMs (N = 1000 gives 4 items), so such passes take 128 threads of one
// particle and 64-record j-tiles instead (N = 1000: 128 items).  Explicit
// step on GB300: N = 1000, D = 9 131 -> 50 us; N = 512, D = 2 40 -> 23 us;
// N = 4096, D = 9 142 -> 102 us.
constexpr int NT_SMALL = 128, RI_SMALL = 1, TJ_SMALL = 64;

// ------------------------------------------------------------- pair kernel

// EXP (density pass only, records with their squared norm in slot D + 1):
// the squared distance through the norms, |x|^2 + |y|^2 - 2 x.y, D + 2 FP32
// operations per pair instead of 2D + 1, with an absolute error of a few
// units of FP32 rounding of |x|^2 + |y|^2 (1e-6 relative in the kernel value
// for the bulk of a cloud).  Only the reduced model's refresh cycle takes
// it; the full-order path keeps the differences its 1e-5 bar needs.
template <int D>
struct HasNorm {
  static constexpr bool value = Rec<D>::DP >= D + 2;
};

template <int D, int RI, int NT, bool GRAD, int TJK = TJ, bool EXP = false>
__global__ void __launch_bounds__(NT)
    k_pair(const float *__restrict__ rec, const float *__restrict__ reci, Sched sc,
           double *__restrict__ part, int *__restrict__ err) {
  static_assert(!EXP || (!GRAD && HasNorm<D>::value), "expanded distances: density pass, norm slot");
  static_assert(TJ % TJK == 0, "j-tiles divide the record padding");
  constexpr int DP = Rec<D>::DP;
  constexpr int ACC = GRAD ? D : 1;
  constexpr uint32_t TILE_FLOATS = TJK * DP;
  constexpr uint32_t TILE_BYTES = TILE_FLOATS * 4;
  extern __shared__ __align__(128) float tiles[];  // NSTAGE * TILE_FLOATS
  __shared__ __align__(8) uint64_t full[NSTAGE];

  const int tid = threadIdx.x;
  const long long it0 = (long long)blockIdx.x * sc.items / sc.G;
  const long long it1 = (long long)(blockIdx.x + 1) * sc.items / sc.G;
  if (it0 >= it1) return;  // uniform over the CTA

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < NSTAGE && it0 + s < it1; ++s) {
      const int ch = (int)((it0 + s) % sc.nchunk);
      mbar_arrive_expect_tx(&full[s], TILE_BYTES);
      bulk_g2s(tiles + s * TILE_FLOATS, rec + (size_t)ch * TILE_FLOATS, TILE_BYTES, &full[s]);
    }
  }

  float xi[RI][D];
  float wi[RI];
  float ni[RI];
  float sum[RI][ACC], cmp[RI][ACC];
  int cur = -1, seg = 0;
  long long it_fail = -1;

  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < RI; ++k) {
      const int il = tid + k * NT;
      double *dst = part + (((size_t)cur * sc.maxseg + seg) * sc.TI + il) * ACC;
#pragma unroll
      for (int a = 0; a < ACC; ++a) dst[a] = (double)sum[k][a] - (double)cmp[k][a];
    }
  };

  for (long long it = it0; it < it1; ++it) {
    const int t = (int)(it / sc.nchunk);
    if (t != cur) {
      if (cur >= 0) flush();
      cur = t;
      seg = (int)blockIdx.x - sched_first_cta((long long)t * sc.nchunk, sc);
#pragma unroll
      for (int k = 0; k < RI; ++k) {
        int i = t * sc.TI + tid + k * NT;
        i = i < sc.Nipad ? i : sc.Nipad - 1;
        const float *r = reci + (size_t)i * DP;
#pragma unroll
        for (int d = 0; d < D; ++d) xi[k][d] = r[d];
        wi[k] = GRAD ? r[D] : 0.f;
        ni[k] = EXP ? r[D + 1] : 0.f;
#pragma unroll
        for (int a = 0; a < ACC; ++a) sum[k][a] = cmp[k][a] = 0.f;
      }
    }
    const int stage = (int)((it - it0) % NSTAGE);
    const uint32_t parity = (uint32_t)(((it - it0) / NSTAGE) & 1);
    const bool got = mbar_wait_bounded(&full[stage], parity, VDS_WAIT_LIMIT_NS);
    if (__syncthreads_or(!got)) {
      it_fail = it;
      break;
    }

    const float *tj = tiles + stage * TILE_FLOATS;
    float acc[RI][ACC];
#pragma unroll
    for (int k = 0; k < RI; ++k)
#pragma unroll
      for (int a = 0; a < ACC; ++a) acc[k][a] = 0.f;

#pragma unroll 2
    for (int j = 0; j < TJK; ++j) {
      float xj[DP];
      const float4 *pj = reinterpret_cast<const float4 *>(tj + j * DP);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 f = pj[v];
        xj[4 * v + 0] = f.x;
        xj[4 * v + 1] = f.y;
        xj[4 * v + 2] = f.z;
        xj[4 * v + 3] = f.w;
      }
#pragma unroll
      for (int k = 0; k < RI; ++k) {
        float dd[D];
        float r2;
        if constexpr (EXP) {
          float dot = xi[k][0] * xj[0];
#pragma unroll
          for (int d = 1; d < D; ++d) dot = fmaf(xi[k][d], xj[d], dot);
          r2 = fmaf(-2.f, dot, ni[k] + xj[(D + 1) % DP]);
        } else {
          dd[0] = xi[k][0] - xj[0];
          r2 = dd[0] * dd[0];
#pragma unroll
          for (int d = 1; d < D; ++d) {
            dd[d] = xi[k][d] - xj[d];
            r2 = fmaf(dd[d], dd[d], r2);
          }
        }
        const float e = ex2_approx(-r2);
        if constexpr (!GRAD) {
          acc[k][0] += e;
        } else {
          const float u = e * (wi[k] + xj[D]);
#pragma unroll
          for (int d = 0; d < D; ++d) acc[k][d] = fmaf(u, dd[d], acc[k][d]);
        }
      }
    }
    // Kahan-compensated accumulation of the tile sums
#pragma unroll
    for (int k = 0; k < RI; ++k)
#pragma unroll
      for (int a = 0; a < ACC; ++a) {
        const float y = acc[k][a] - cmp[k][a];
        const float tt = sum[k][a] + y;
        cmp[k][a] = (tt - sum[k][a]) - y;
        sum[k][a] = tt;
      }
    __syncthreads();  // stage fully consumed
    if (tid == 0 && it + NSTAGE < it1) {
      fence_proxy_async_smem();
      const int ch = (int)((it + NSTAGE) % sc.nchunk);
      mbar_arrive_expect_tx(&full[stage], TILE_BYTES);
      bulk_g2s(tiles + stage * TILE_FLOATS, rec + (size_t)ch * TILE_FLOATS, TILE_BYTES,
               &full[stage]);
    }
  }
  if (it_fail >= 0) {
    if (tid == 0) {
      vds_flag(err, VDS_ETIMEOUT);
      // copies for items it_fail .. it_fail+NSTAGE-1 may still be in flight:
      // give each a bounded chance to land before shared memory is released
      for (long long k = it_fail; k < it_fail + NSTAGE && k < it1; ++k)
        mbar_wait_bounded(&full[(k - it0) % NSTAGE], (uint32_t)(((k - it0) / NSTAGE) & 1),
                          VDS_WAIT_LIMIT_NS / 8);
    }
    return;
  }
  if (cur >= 0) flush();
}

// --------------------------------------------------------- small device math

__device__ __forceinline__ double rouse_A(int j, int k) {
  return j == k ? 2.0 : ((j - k == 1 || k - j == 1) ? -1.0 : 0.0);
}

// inverse of the tridiagonal Rouse matrix: min(j,k)(nb+1-max(j,k))/(nb+1), 1-based
__device__ __forceinline__ double rouse_Ainv(int j, int k, int nb) {
  const int lo = (j < k ? j : k) + 1, hi = (j > k ? j : k) + 1;
  return (double)lo * (double)(nb + 1 - hi) / (double)(nb + 1);
}

// Spring energy and force factor per bond: grad Psi_k = f_k q_k.
template <int D>
__device__ __forceinline__ bool spring_eval(const KParams &kp, const double (&y)[D], double &psi,
                                            double (&f)[8]) {
  psi = 0.0;
  bool ok = true;
  for (int k = 0; k < kp.nb; ++k) {
    double n2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a / kp.s == k) n2 += y[a] * y[a];
    if (kp.spring == 0) {
      psi += 0.5 * kp.H[k] * n2;
      f[k] = kp.H[k];
    } else {
      const double x = 1.0 - n2 / kp.b;
      if (!(x > 0.0)) {
        ok = false;
        f[k] = 0.0;
      } else {
        psi += -0.5 * kp.H[k] * kp.b * log(x);
        f[k] = kp.H[k] / x;
      }
    }
  }
  return ok;
}

// --------------------------------------------------------------- prep kernel

template <int D>
__global__ void k_prep(int N, int Npad, float c, const float *__restrict__ base,
                       const float *__restrict__ delta, const float *__restrict__ dir,
                       float alpha, float *__restrict__ delta_out, float *__restrict__ rec) {
  constexpr int DP = Rec<D>::DP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  float o[DP];
  if (i < N) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float dl = 0.f;
      if (delta) {
        dl = delta[(size_t)i * D + d];
        if (dir) dl = dl - alpha * dir[(size_t)i * D + d];
        if (delta_out) delta_out[(size_t)i * D + d] = dl;
      }
      o[d] = c * (base[(size_t)i * D + d] + dl);
    }
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) o[d] = VDS_PAD_COORD;
  }
#pragma unroll
  for (int d = D; d < DP; ++d) o[d] = 0.f;
  if constexpr (HasNorm<D>::value) {
    // the squared norm, rounded as the expanded density pass forms x.x
    float nrm = o[0] * o[0];
#pragma unroll
    for (int d = 1; d < D; ++d) nrm = fmaf(o[d], o[d], nrm);
    o[D + 1] = nrm;
  }
  float4 *dst = reinterpret_cast<float4 *>(rec + (size_t)i * DP);
#pragma unroll
  for (int v = 0; v < DP / 4; ++v) dst[v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
}

// ------------------------------------------------------------- epilogues

constexpr int NT_FIN = 256;

// Deterministic grid reduction: every block stores its partial, the last
// block to arrive (ticket) sums them in block order.  Returns true in the
// thread that holds the final value.
template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], const bool (&is_max)[K], double *red,
                                            unsigned *ticket, double (&out)[K]) {
  __shared__ double sh[NT_FIN / 32][K];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = is_max[k] ? fmax(x, y) : x + y;
    }
    if (lane == 0) sh[w][k] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = is_max[k] ? 0.0 : 0.0;
      for (int q = 0; q < NT_FIN / 32; ++q) x = is_max[k] ? fmax(x, sh[q][k]) : x + sh[q][k];
      red[(size_t)blockIdx.x * K + k] = x;
    }
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      const double y = __ldcg(red + (size_t)b * K + k);
      x = is_max[k] ? fmax(x, y) : x + y;
    }
    out[k] = x;
  }
  *ticket = 0u;
  return true;
}

template <int D>
__device__ __forceinline__ void load_y(const float *ybase, const float *ydelta, int i, double (&y)[D],
                                       float (&yf)[D]) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float v = ybase[(size_t)i * D + d];
    if (ydelta) v = v + ydelta[(size_t)i * D + d];
    yf[d] = v;
    y[d] = (double)v;
  }
}

template <int D>
__global__ void __launch_bounds__(NT_FIN)
    k_dens_finish(Sched sc, const double *__restrict__ part, float *__restrict__ rec,
                  float *__restrict__ rho_out, KParams kp, int want_energy,
                  const float *__restrict__ ybase, const float *__restrict__ ydelta,
                  const float *__restrict__ qa, const float *__restrict__ qb, double *red,
                  unsigned *ticket, double *scal, int *err) {
  constexpr int DP = Rec<D>::DP;
  const int i = blockIdx.x * NT_FIN + threadIdx.x;
  double e = 0.0;
  if (i < kp.N) {
    const int t = i / sc.TI, il = i - t * sc.TI;
    const int f = sched_first_cta((long long)t * sc.nchunk, sc);
    const int l = sched_first_cta((long long)(t + 1) * sc.nchunk - 1, sc);
    double rho = 0.0;
    for (int g = 0; g <= l - f; ++g) rho += part[((size_t)t * sc.maxseg + g) * sc.TI + il];
    if (!(rho >= 0.5 && rho <= 1e300)) vds_flag(err, VDS_ENAN);
    rec[(size_t)i * DP + D] = (float)(1.0 / rho);
    if (rho_out) rho_out[i] = (float)rho;
    if (want_energy) {
      double y[D];
      float yf[D];
      load_y<D>(ybase, ydelta, i, y, yf);
      double psi, fk[8];
      if (!spring_eval<D>(kp, y, psi, fk)) vds_flag(err, VDS_EDOMAIN);
      e = kp.kBT * (log(rho) + kp.lnorm) + psi;
      if (qa) {
        double dl[D];
#pragma unroll
        for (int d = 0; d < D; ++d)
          dl[d] = (double)qa[(size_t)i * D + d] - (qb ? (double)qb[(size_t)i * D + d] : 0.0);
        double quad = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (a % kp.s == b % kp.s) quad += dl[a] * rouse_Ainv(a / kp.s, b / kp.s, kp.nb) * dl[b];
        e += kp.zeta / (2.0 * kp.dt) * quad;
      }
    }
  }
  if (want_energy) {
    double v[1] = {e}, out[1];
    const bool mx[1] = {false};
    if (grid_reduce<1>(v, mx, red, ticket, out)) {
      scal[SC_E] = out[0] / (double)kp.N;
      if (!(fabs(scal[SC_E]) <= 1e300)) vds_flag(err, VDS_ENAN);
    }
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(NT_FIN)
    k_grad_finish(Sched sc, const double *__restrict__ part, float *__restrict__ rec, KParams kp,
                  float *__restrict__ out, const float *ybase,
                  const float *__restrict__ ydelta, const float *__restrict__ qa,
                  const float *__restrict__ qb, float *q_io, double *red,
                  unsigned *ticket, double *scal, int *err) {
  constexpr int DP = Rec<D>::DP;
  const int i = blockIdx.x * NT_FIN + threadIdx.x;
  double dec = 0.0, dmax = 0.0, ymax = 0.0;
  if (i < kp.N) {
    const int t = i / sc.TI, il = i - t * sc.TI;
    const int f = sched_first_cta((long long)t * sc.nchunk, sc);
    const int l = sched_first_cta((long long)(t + 1) * sc.nchunk - 1, sc);
    double g[D];
#pragma unroll
    for (int a = 0; a < D; ++a) g[a] = 0.0;
    for (int s = 0; s <= l - f; ++s) {
      const double *p = part + (((size_t)t * sc.maxseg + s) * sc.TI + il) * D;
#pragma unroll
      for (int a = 0; a < D; ++a) g[a] += p[a];
    }
    double y[D];
    float yf[D];
    load_y<D>(ybase, ydelta, i, y, yf);
    double psi, fk[8];
    if (!spring_eval<D>(kp, y, psi, fk)) vds_flag(err, VDS_EDOMAIN);
#pragma unroll
    for (int a = 0; a < D; ++a) g[a] = kp.kBT * (-kp.sfac * g[a]) + fk[a / kp.s] * y[a];

    if constexpr (MODE == GM_OUT) {
      if (qa) {
        double dl[D];
#pragma unroll
        for (int d = 0; d < D; ++d)
          dl[d] = (double)qa[(size_t)i * D + d] - (qb ? (double)qb[(size_t)i * D + d] : 0.0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double v = 0.0;
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (a % kp.s == b % kp.s) v += rouse_Ainv(a / kp.s, b / kp.s, kp.nb) * dl[b];
          g[a] += kp.zeta / kp.dt * v;
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) out[(size_t)i * D + a] = (float)g[a];
    } else if constexpr (MODE == GM_VEL) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int k = a / kp.s, al = a - k * kp.s;
        double v = 0.0, m = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const int kb = b / kp.s, be = b - kb * kp.s;
          if (kb == k) v += kp.kappa[al * kp.s + be] * y[b];
          if (be == al) m += rouse_A(k, kb) * g[b];
        }
        out[(size_t)i * D + a] = (float)(v - m / kp.zeta);
      }
    } else if constexpr (MODE == GM_EXPLICIT) {
      float yn[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int k = a / kp.s, al = a - k * kp.s;
        double v = 0.0, m = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const int kb = b / kp.s, be = b - kb * kp.s;
          if (kb == k) v += kp.kappa[al * kp.s + be] * y[b];
          if (be == al) m += rouse_A(k, kb) * g[b];
        }
        yn[a] = (float)(y[a] + kp.dt * (v - m / kp.zeta));
      }
      if (kp.spring == 1) {
        for (int k = 0; k < kp.nb; ++k) {
          double n2 = 0.0;
#pragma unroll
          for (int a = 0; a < D; ++a)
            if (a / kp.s == k) n2 += (double)yn[a] * yn[a];
          if (!(n2 < kp.b)) vds_flag(err, VDS_EDOMAIN);
        }
      }
      float o[DP];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        q_io[(size_t)i * D + a] = yn[a];
        o[a] = kp.c * yn[a];
      }
#pragma unroll
      for (int a = D; a < DP; ++a) o[a] = 0.f;
      float4 *dst = reinterpret_cast<float4 *>(rec + (size_t)i * DP);
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) dst[v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
    } else {  // GM_IMPLICIT_DIR
      double dl[D];
#pragma unroll
      for (int d = 0; d < D; ++d) dl[d] = (double)ydelta[(size_t)i * D + d];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int k = a / kp.s, al = a - k * kp.s;
        double ag = 0.0, aid = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const int kb = b / kp.s, be = b - kb * kp.s;
          if (be == al) {
            ag += rouse_A(k, kb) * g[b];
            aid += rouse_Ainv(k, kb, kp.nb) * dl[b];
          }
        }
        const double dr = dl[a] + kp.dt / kp.zeta * ag;
        const double G = kp.zeta / kp.dt * aid + g[a];
        const float drf = (float)dr;
        out[(size_t)i * D + a] = drf;
        dec += G * dr;
        dmax = fmax(dmax, fabs((double)drf));
        ymax = fmax(ymax, fabs((double)yf[a]));
      }
    }
  }
  if constexpr (MODE == GM_IMPLICIT_DIR) {
    double v[3] = {dec, dmax, ymax}, o[3];
    const bool mx[3] = {false, true, true};
    if (grid_reduce<3>(v, mx, red, ticket, o)) {
      scal[SC_DEC] = o[0] / (double)kp.N;
      scal[SC_DMAX] = o[1];
      scal[SC_YMAX] = o[2];
      if (!(fabs(o[0]) <= 1e300)) vds_flag(err, VDS_ENAN);
    }
  }
}

// ------------------------------------------------------------ stress kernel

constexpr int STRESS_BP = 128;  // particles staged per block iteration

template <int D>
__global__ void __launch_bounds__(256)
    k_stress(KParams kp, const float *__restrict__ q, double *red, unsigned *ticket, double *scal,
             int *err) {
  __shared__ float ys[STRESS_BP][D];
  const int s = kp.s, ne_tau = s * s, ne = ne_tau + D * D;
  double acc[2] = {0.0, 0.0};  // entries tid and tid+256
  for (int base = blockIdx.x * STRESS_BP; base < kp.N; base += gridDim.x * STRESS_BP) {
    __syncthreads();
    for (int x = threadIdx.x; x < STRESS_BP * D; x += blockDim.x) {
      const int p = x / D, d = x - p * D;
      ys[p][d] = (base + p < kp.N) ? q[(size_t)(base + p) * D + d] : 0.f;
    }
    __syncthreads();
    if (kp.spring == 1 && threadIdx.x < STRESS_BP && base + threadIdx.x < kp.N) {
      const int p = threadIdx.x;
      for (int k = 0; k < kp.nb; ++k) {
        double n2 = 0.0;
        for (int a = 0; a < s; ++a) n2 += (double)ys[p][s * k + a] * ys[p][s * k + a];
        if (!(n2 < kp.b)) vds_flag(err, VDS_EDOMAIN);
      }
    }
    const int np = min(STRESS_BP, kp.N - base);
    for (int r = 0; r < 2; ++r) {
      const int e = threadIdx.x + r * 256;
      if (e >= ne) continue;
      double a = 0.0;
      if (e < ne_tau) {
        const int al = e / s, be = e - al * s;
        for (int p = 0; p < np; ++p) {
          for (int k = 0; k < kp.nb; ++k) {
            double f = kp.H[k];
            if (kp.spring == 1) {
              double n2 = 0.0;
              for (int c = 0; c < s; ++c) n2 += (double)ys[p][s * k + c] * ys[p][s * k + c];
              f = kp.H[k] / (1.0 - n2 / kp.b);
            }
            a += (double)ys[p][s * k + al] * f * (double)ys[p][s * k + be];
          }
        }
      } else {
        const int x = e - ne_tau, ra = x / D, rb = x - ra * D;
        for (int p = 0; p < np; ++p) a += (double)ys[p][ra] * (double)ys[p][rb];
      }
      acc[r] += a;
    }
  }
  // block partials of all entries, then ticketed final sum in block order
  __shared__ bool last;
  for (int r = 0; r < 2; ++r) {
    const int e = threadIdx.x + r * 256;
    if (e < ne) red[(size_t)blockIdx.x * ne + e] = acc[r];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    double x = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) x += __ldcg(red + (size_t)b * ne + e);
    scal[SC_AUX + e] = x / (double)kp.N;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0u;
}

template <int D>
__global__ void k_flow(KParams kp, const float *__restrict__ q, float *__restrict__ qs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kp.N) return;
  float y[D];
#pragma unroll
  for (int a = 0; a < D; ++a) y[a] = q[(size_t)i * D + a];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int k = a / kp.s, al = a - k * kp.s;
    double v = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b / kp.s == k) v += kp.kappa[al * kp.s + (b - k * kp.s)] * (double)y[b];
    qs[(size_t)i * D + a] = (float)((double)y[a] + kp.dt * v);
  }
}

// ------------------------------------------------------------ host plumbing

// i points: the Ni records at reci (the particles themselves unless a query
// pass); j points: the N particle records in c->rec.
template <int D, int RI, int NT, bool GRAD, int TJK = TJ, bool EXP = false>
int launch_pair(vds_ctx *c, int N, Sched &sc, int Ni, const float *reci) {
  constexpr int DP = Rec<D>::DP;
  constexpr int ACC = GRAD ? D : 1;
  constexpr int TI = NT * RI;
  const size_t smem = (size_t)NSTAGE * TJK * DP * sizeof(float);
  // per device: the attribute is a property of the function on that device
  static int occ_dev[VDS_MAX_DEVICES] = {};
  int &occ = occ_dev[c->device < VDS_MAX_DEVICES ? c->device : 0];
  if (occ <= 0 || c->device >= VDS_MAX_DEVICES) {
    // large D needs more than the default 48 KB of dynamic shared memory
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_pair<D, RI, NT, GRAD, TJK, EXP>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int o = 0;
    VDS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_pair<D, RI, NT, GRAD, TJK, EXP>, NT, smem));
    occ = o > 0 ? o : 1;
  }
  sc.TI = TI;
  sc.Npad = (N + TJ - 1) / TJ * TJ;
  sc.Nipad = (Ni + TJ - 1) / TJ * TJ;
  sc.nchunk = sc.Npad / TJK;
  sc.n_itiles = (Ni + TI - 1) / TI;
  sc.items = (long long)sc.n_itiles * sc.nchunk;
  const long long cap = (long long)c->num_sms * occ;
  sc.G = (int)(sc.items < cap ? sc.items : cap);
  int maxseg = 1;
  for (int t = 0; t < sc.n_itiles; ++t) {
    const int f = sched_first_cta((long long)t * sc.nchunk, sc);
    const int l = sched_first_cta((long long)(t + 1) * sc.nchunk - 1, sc);
    if (l - f + 1 > maxseg) maxseg = l - f + 1;
  }
  sc.maxseg = maxseg;
  VDS_TRY(vds_ensure(c, c->part, (size_t)sc.n_itiles * maxseg * TI * ACC * sizeof(double)));
  const int pk = GRAD ? PK_GRADIENT : PK_DENSITY;
  VDS_TRY(vds_time_begin(c, pk));
  k_pair<D, RI, NT, GRAD, TJK, EXP><<<sc.G, NT, smem, c->stream>>>((const float *)c->rec.ptr, reci, sc,
                                                                     (double *)c->part.ptr, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  VDS_TRY(vds_time_end(c, pk));
  ++c->launches;
  return VDS_OK;
}

template <int D>
int prep_impl(vds_ctx *c, const KParams &kp, const float *base, const float *delta,
              const float *dir, float alpha, float *delta_out) {
  const int Npad = (kp.N + TJ - 1) / TJ * TJ;
  VDS_TRY(vds_ensure(c, c->rec, (size_t)Npad * Rec<D>::DP * sizeof(float)));
  k_prep<D><<<(Npad + 255) / 256, 256, 0, c->stream>>>(kp.N, Npad, kp.c, base, delta, dir, alpha,
                                                       delta_out, (float *)c->rec.ptr);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// One pair pass with the pass's shape, or the small-cloud shape when the
// former's items would cover fewer than half the SMs.  Between the two
// (fewer than 8 items per SM), the pass's shape takes 64-record j-chunks:
// four times the items, so that the last round of the stream-K split is
// not a large fraction of the pass (N = 10000 at D = 9: 200 and 360 items
// per pass at 256 records).
// EXP: the expanded distances of the density pass, for large clouds only
// (small clouds keep the direct form: their passes are latency bound).
template <int D, bool GRAD, bool EXP = false>
int launch_pass(vds_ctx *c, int N, Sched &sc, int Ni, const float *reci) {
  constexpr int RI = GRAD ? PairCfg<D>::RI_GRAD : PairCfg<D>::RI_DENS;
  constexpr int NT = GRAD ? PairCfg<D>::NT_GRAD : PairCfg<D>::NT_DENS;
  const long long items = (long long)((Ni + NT * RI - 1) / (NT * RI)) * ((N + TJ - 1) / TJ);
  if (2 * items < c->num_sms) return launch_pair<D, RI_SMALL, NT_SMALL, GRAD, TJ_SMALL>(c, N, sc, Ni, reci);
  if (items < 8LL * c->num_sms) return launch_pair<D, RI, NT, GRAD, TJ_SMALL>(c, N, sc, Ni, reci);
  if constexpr (EXP && !GRAD && HasNorm<D>::value) return launch_pair<D, RI, NT, GRAD, TJ, true>(c, N, sc, Ni, reci);
  else return launch_pair<D, RI, NT, GRAD>(c, N, sc, Ni, reci);
}

template <int D>
int density_impl(vds_ctx *c, const KParams &kp, float *rho_out, bool want_energy,
                 const float *ybase, const float *ydelta, const float *qa, const float *qb, bool expand) {
  Sched sc;
  if (expand)
    VDS_TRY((launch_pass<D, false, true>(c, kp.N, sc, kp.N, (const float *)c->rec.ptr)));
  else
    VDS_TRY((launch_pass<D, false>(c, kp.N, sc, kp.N, (const float *)c->rec.ptr)));
  const int nb = (kp.N + NT_FIN - 1) / NT_FIN;
  VDS_TRY(vds_ensure(c, c->red, (size_t)nb * 4 * sizeof(double)));
  k_dens_finish<D><<<nb, NT_FIN, 0, c->stream>>>(sc, (const double *)c->part.ptr, (float *)c->rec.ptr,
                                                 rho_out, kp, want_energy ? 1 : 0, ybase, ydelta, qa,
                                                 qb, (double *)c->red.ptr, c->ticket + TK_DENS,
                                                 c->scal, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

template <int D>
int grad_impl(vds_ctx *c, const KParams &kp, int mode, float *out, const float *ybase,
              const float *ydelta, const float *qa, const float *qb, float *q_io) {
  Sched sc;
  VDS_TRY((launch_pass<D, true>(c, kp.N, sc, kp.N, (const float *)c->rec.ptr)));
  const int nb = (kp.N + NT_FIN - 1) / NT_FIN;
  VDS_TRY(vds_ensure(c, c->red, (size_t)nb * 4 * sizeof(double)));
  const double *pp = (const double *)c->part.ptr;
  float *rp = (float *)c->rec.ptr;
  double *red = (double *)c->red.ptr;
  unsigned *tk = c->ticket + TK_GRAD;
  if (mode == GM_OUT)
    k_grad_finish<D, GM_OUT><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rp, kp, out, ybase, ydelta, qa, qb,
                                                          q_io, red, tk, c->scal, c->err);
  else if (mode == GM_EXPLICIT)
    k_grad_finish<D, GM_EXPLICIT><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rp, kp, out, ybase, ydelta, qa,
                                                               qb, q_io, red, tk, c->scal, c->err);
  else if (mode == GM_VEL)
    k_grad_finish<D, GM_VEL><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rp, kp, out, ybase, ydelta, qa, qb,
                                                          q_io, red, tk, c->scal, c->err);
  else
    k_grad_finish<D, GM_IMPLICIT_DIR><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rp, kp, out, ybase, ydelta,
                                                                   qa, qb, q_io, red, tk, c->scal,
                                                                   c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// f at the query points: the segment partials of each query summed in a
// fixed order (FP64), times (1/N)(2 pi h^2)^(-D/2).
template <int D>
__global__ void __launch_bounds__(NT_FIN)
    k_query_finish(Sched sc, const double *__restrict__ part, int M, double scale, float *__restrict__ f_out,
                   int *err) {
  const int i = blockIdx.x * NT_FIN + threadIdx.x;
  if (i >= M) return;
  const int t = i / sc.TI, il = i - t * sc.TI;
  const int f = sched_first_cta((long long)t * sc.nchunk, sc);
  const int l = sched_first_cta((long long)(t + 1) * sc.nchunk - 1, sc);
  double s = 0.0;
  for (int g = 0; g <= l - f; ++g) s += part[((size_t)t * sc.maxseg + g) * sc.TI + il];
  if (!(s >= 0.0 && s <= 1e300)) vds_flag(err, VDS_ENAN);
  f_out[i] = (float)(s * scale);
}

template <int D>
int query_impl(vds_ctx *c, const KParams &kp, const float *q, const float *y, int M, float *f_out) {
  VDS_TRY(prep_impl<D>(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  const int Mpad = (M + TJ - 1) / TJ * TJ;
  VDS_TRY(vds_ensure(c, c->recq, (size_t)Mpad * Rec<D>::DP * sizeof(float)));
  k_prep<D><<<(Mpad + 255) / 256, 256, 0, c->stream>>>(M, Mpad, kp.c, y, nullptr, nullptr, 0.f, nullptr,
                                                       (float *)c->recq.ptr);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  Sched sc;
  VDS_TRY((launch_pass<D, false>(c, kp.N, sc, M, (const float *)c->recq.ptr)));
  k_query_finish<D><<<(M + NT_FIN - 1) / NT_FIN, NT_FIN, 0, c->stream>>>(sc, (const double *)c->part.ptr, M,
                                                                         exp(kp.lnorm), f_out, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// ------------------------------------------------- row-range passes
//
// The pair passes restricted to the particles row0 .. row0 + nrows - 1 as
// the rows I (all N particles as the columns J): the pieces of one
// evaluation split over ranks by rows (each rank holds all of q, and all of
// rho before its gradient pass).

// w = 1/rho of every particle into its record, from a gathered rho array.
template <int D>
__global__ void k_set_w(int N, const float *__restrict__ rho, float *__restrict__ rec, int *err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float r = rho[i];
  if (!(r >= 0.5f && r <= 3.0e38f)) vds_flag(err, VDS_ENAN);
  rec[(size_t)i * Rec<D>::DP + D] = (float)(1.0 / (double)r);
}

// The records of nrows consecutive particles (src already offset to row0)
// copied into their own array padded to Mpad rows, so a pass reads its i
// records from a buffer whose padding rows are far away (kernel value 0).
template <int D>
__global__ void k_copy_rows(int nrows, int Mpad, const float *__restrict__ src, float *__restrict__ dst) {
  constexpr int DP = Rec<D>::DP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Mpad) return;
  float4 *d = reinterpret_cast<float4 *>(dst + (size_t)i * DP);
  if (i < nrows) {
    const float4 *s = reinterpret_cast<const float4 *>(src + (size_t)i * DP);
#pragma unroll
    for (int v = 0; v < DP / 4; ++v) d[v] = s[v];
  } else {
    float o[DP];
#pragma unroll
    for (int a = 0; a < D; ++a) o[a] = VDS_PAD_COORD;
#pragma unroll
    for (int a = D; a < DP; ++a) o[a] = 0.f;
#pragma unroll
    for (int v = 0; v < DP / 4; ++v) d[v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
  }
}

template <int D>
int rows_records(vds_ctx *c, int row0, int nrows) {
  const int Mpad = (nrows + TJ - 1) / TJ * TJ;
  VDS_TRY(vds_ensure(c, c->recq, (size_t)Mpad * Rec<D>::DP * sizeof(float)));
  k_copy_rows<D><<<(Mpad + 255) / 256, 256, 0, c->stream>>>(nrows, Mpad, (const float *)c->rec.ptr +
                                                                             (size_t)row0 * Rec<D>::DP,
                                                           (float *)c->recq.ptr);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// rho of the rows (FP32) from the density pass over all N columns.
template <int D>
int rows_density_impl(vds_ctx *c, const KParams &kp, const float *q, int row0, int nrows, float *rho_rows) {
  VDS_TRY(prep_impl<D>(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  VDS_TRY(rows_records<D>(c, row0, nrows));
  Sched sc;
  VDS_TRY((launch_pass<D, false>(c, kp.N, sc, nrows, (const float *)c->recq.ptr)));
  k_query_finish<D><<<(nrows + NT_FIN - 1) / NT_FIN, NT_FIN, 0, c->stream>>>(sc, (const double *)c->part.ptr,
                                                                             nrows, 1.0, rho_rows, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

// With rho of all N particles: the gradient pass for the rows, then either
// g = kBT S + grad Psi of the rows (mode 0) or their explicit Euler update
// (mode 1) into out (nrows x D).
template <int D>
int rows_grad_impl(vds_ctx *c, const KParams &kp, const float *q, const float *rho, int row0, int nrows,
                   int mode, float *out) {
  VDS_TRY(prep_impl<D>(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  k_set_w<D><<<(kp.N + 255) / 256, 256, 0, c->stream>>>(kp.N, rho, (float *)c->rec.ptr, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_TRY(rows_records<D>(c, row0, nrows));
  Sched sc;
  VDS_TRY((launch_pass<D, true>(c, kp.N, sc, nrows, (const float *)c->recq.ptr)));
  KParams kl = kp;
  kl.N = nrows;
  const int nb = (nrows + NT_FIN - 1) / NT_FIN;
  const double *pp = (const double *)c->part.ptr;
  float *rq = (float *)c->recq.ptr;
  const float *y = q + (size_t)row0 * D;
  if (mode == 0)
    k_grad_finish<D, GM_OUT><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rq, kl, out, y, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, nullptr, c->scal, c->err);
  else
    k_grad_finish<D, GM_EXPLICIT><<<nb, NT_FIN, 0, c->stream>>>(sc, pp, rq, kl, nullptr, y, nullptr, nullptr,
                                                               nullptr, out, nullptr, nullptr, c->scal, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

template <int D>
int stress_impl(vds_ctx *c, const KParams &kp, const float *q, double *tau, double *qq) {
  const int ne = kp.s * kp.s + D * D;
  int nblk = (kp.N + STRESS_BP - 1) / STRESS_BP;
  if (nblk > 2 * c->num_sms) nblk = 2 * c->num_sms;
  VDS_TRY(vds_ensure(c, c->red, (size_t)nblk * ne * sizeof(double)));
  k_stress<D><<<nblk, 256, 0, c->stream>>>(kp, q, (double *)c->red.ptr, c->ticket + TK_STRESS, c->scal,
                                          c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  VDS_TRY(vds_sync_status(c));
  for (int e = 0; e < kp.s * kp.s; ++e) tau[e] = c->h_scal[SC_AUX + e];
  if (qq)
    for (int e = 0; e < D * D; ++e) qq[e] = c->h_scal[SC_AUX + kp.s * kp.s + e];
  return VDS_OK;
}

template <int D>
int flow_impl(vds_ctx *c, const KParams &kp, const float *q, float *qs) {
  k_flow<D><<<(kp.N + 255) / 256, 256, 0, c->stream>>>(kp, q, qs);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

}  // namespace vds_pair

// One translation unit per supported D (pair_d<D>.cu) instantiates the passes
// through this macro, so the library builds in parallel.
#define VDS_PAIR_INSTANTIATE(DD)                                                              \
  int vds_prep_##DD(vds_ctx *c, const KParams &kp, const float *base, const float *delta,     \
                    const float *dir, float alpha, float *delta_out) {                        \
    return vds_pair::prep_impl<DD>(c, kp, base, delta, dir, alpha, delta_out);                \
  }                                                                                           \
  int vds_density_##DD(vds_ctx *c, const KParams &kp, float *rho_out, bool want_energy,       \
                       const float *ybase, const float *ydelta, const float *qa,              \
                       const float *qb, bool expand) {                                        \
    return vds_pair::density_impl<DD>(c, kp, rho_out, want_energy, ybase, ydelta, qa, qb,     \
                                      expand);                                                \
  }                                                                                           \
  int vds_grad_##DD(vds_ctx *c, const KParams &kp, int mode, float *out, const float *ybase,  \
                    const float *ydelta, const float *qa, const float *qb, float *q_io) {     \
    return vds_pair::grad_impl<DD>(c, kp, mode, out, ybase, ydelta, qa, qb, q_io);            \
  }                                                                                           \
  int vds_stress_##DD(vds_ctx *c, const KParams &kp, const float *q, double *tau, double *qq) { \
    return vds_pair::stress_impl<DD>(c, kp, q, tau, qq);                                      \
  }                                                                                           \
  int vds_flow_##DD(vds_ctx *c, const KParams &kp, const float *q, float *qs) {               \
    return vds_pair::flow_impl<DD>(c, kp, q, qs);                                             \
  }                                                                                           \
  int vds_query_##DD(vds_ctx *c, const KParams &kp, const float *q, const float *y, int M,     \
                     float *f) {                                                              \
    return vds_pair::query_impl<DD>(c, kp, q, y, M, f);                                       \
  }                                                                                           \
  int vds_rowsdens_##DD(vds_ctx *c, const KParams &kp, const float *q, int row0, int nrows,    \
                        float *rho) {                                                         \
    return vds_pair::rows_density_impl<DD>(c, kp, q, row0, nrows, rho);                       \
  }                                                                                           \
  int vds_rowsgrad_##DD(vds_ctx *c, const KParams &kp, const float *q, const float *rho,       \
                        int row0, int nrows, int mode, float *out) {                          \
    return vds_pair::rows_grad_impl<DD>(c, kp, q, rho, row0, nrows, mode, out);               \
  }
