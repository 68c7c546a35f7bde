// batched.cu -- many independent VDS ensembles of uneven size advanced
// together (include/vds_batch.h).
//
// One persistent pair kernel per pass: each CTA pops (ensemble, i-tile) work
// items, in longest-processing-time order, from an atomic counter and streams
// all j-tiles of that ensemble through a shared-memory ring filled by TMA bulk
// copies.  An item covers the whole j range, so every particle's sums are
// formed by one CTA in a fixed order (plain FP32 inside a j-tile, Kahan across
// tiles): results are independent of which CTA took which item.
//
// Implicit steps run every ensemble's minimiser (the single-ensemble
// algorithm of vds_step, scheme 1) in lockstep rounds.  Per-ensemble state
// lives on the device; a round is
//   prep     -> records of each ensemble's current trial point / final q
//   pair     -> density pass for ensembles in a line-search trial, gradient
//               pass for ensembles that need a new direction (one launch)
//   finish   -> w = 1/rho and energy terms, or g and the new direction
//   reduce   -> per-ensemble FP64 sums in a fixed order and the state update
// captured once as a CUDA graph and replayed until every ensemble is done.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/vds_batch.h"
#include "vds_internal.cuh"

namespace {

constexpr int BTJ = 128;  // records per j-tile
constexpr int BNS = 3;    // ring stages
constexpr int RNT = 256;  // threads of the per-ensemble reduction

// Candidate pair-kernel shapes of the tile autotuner (vds_batch_autotune):
// threads per CTA and particles per thread; the i-tile of a work item is
// their product.  j-tiles and summation order are the same in every shape.
constexpr int kCfgNT[VDS_BATCH_CONFIGS] = {128, 128, 256, 256};
constexpr int kCfgRI[VDS_BATCH_CONFIGS] = {2, 4, 2, 4};
constexpr int kMinTile = 256;  // smallest i-tile over the candidates
inline int default_config(int D) { return D <= 6 ? 1 : 0; }

struct EParam {
  float c;
  float pad_;
  double h, sfac, lnorm;
  double kappa[9];
};

struct BCommon {
  int nb, s, spring, max_iter;
  double H[8];
  double b, kBT, zeta, dt, tol, jfloor;
};

enum { ST_TRIAL = 0, ST_GRAD = 1, ST_FINAL = 2, ST_DONE = 3 };

struct BState {
  double J, alpha, dec;
  int phase, it, ls, status, cur, fin_dir;
};

// ------------------------------------------------------------ pair kernel

template <int D, int RI, int NT, bool GRAD>
__device__ __forceinline__ bool bitem(float *tiles, uint64_t *full, const float *__restrict__ recE, int Ne,
                                      int t, long long gtile, double *__restrict__ outE) {
  constexpr int DP = Rec<D>::DP;
  constexpr int ACC = GRAD ? D : 1;
  constexpr int TILE = BTJ * DP;
  constexpr int TI = NT * RI;
  const int tid = threadIdx.x;
  const int ntile = (Ne + BTJ - 1) / BTJ;
  if (tid == 0) {
    for (int s = 0; s < BNS && s < ntile; ++s) {
      const int stage = (int)((gtile + s) % BNS);
      const uint32_t bytes = (uint32_t)(min(BTJ, Ne - s * BTJ) * DP * 4);
      mbar_arrive_expect_tx(&full[stage], bytes);
      bulk_g2s(tiles + stage * TILE, recE + (size_t)s * TILE, bytes, &full[stage]);
    }
  }
  float xi[RI][D], wi[RI], sum[RI][ACC], cmp[RI][ACC];
#pragma unroll
  for (int k = 0; k < RI; ++k) {
    int i = t * TI + tid + k * NT;
    i = i < Ne ? i : Ne - 1;
    const float *r = recE + (size_t)i * DP;
#pragma unroll
    for (int d = 0; d < D; ++d) xi[k][d] = r[d];
    wi[k] = GRAD ? r[D] : 0.f;
#pragma unroll
    for (int a = 0; a < ACC; ++a) sum[k][a] = cmp[k][a] = 0.f;
  }
  for (int kt = 0; kt < ntile; ++kt) {
    const long long g = gtile + kt;
    const int stage = (int)(g % BNS);
    const bool got = mbar_wait_bounded(&full[stage], (uint32_t)((g / BNS) & 1), VDS_WAIT_LIMIT_NS);
    if (__syncthreads_or(!got)) {
      if (tid == 0)
        for (int k2 = kt; k2 < kt + BNS && k2 < ntile; ++k2)
          mbar_wait_bounded(&full[(gtile + k2) % BNS], (uint32_t)(((gtile + k2) / BNS) & 1),
                            VDS_WAIT_LIMIT_NS / 8);
      return false;
    }
    const float *tj = tiles + stage * TILE;
    const int cnt = min(BTJ, Ne - kt * BTJ);
    float acc[RI][ACC];
#pragma unroll
    for (int k = 0; k < RI; ++k)
#pragma unroll
      for (int a = 0; a < ACC; ++a) acc[k][a] = 0.f;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
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
        dd[0] = xi[k][0] - xj[0];
        float r2 = dd[0] * dd[0];
#pragma unroll
        for (int d = 1; d < D; ++d) {
          dd[d] = xi[k][d] - xj[d];
          r2 = fmaf(dd[d], dd[d], r2);
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
#pragma unroll
    for (int k = 0; k < RI; ++k)
#pragma unroll
      for (int a = 0; a < ACC; ++a) {
        const float y = acc[k][a] - cmp[k][a];
        const float tt = sum[k][a] + y;
        cmp[k][a] = (tt - sum[k][a]) - y;
        sum[k][a] = tt;
      }
    __syncthreads();
    if (tid == 0 && kt + BNS < ntile) {
      fence_proxy_async_smem();
      const uint32_t bytes = (uint32_t)(min(BTJ, Ne - (kt + BNS) * BTJ) * DP * 4);
      mbar_arrive_expect_tx(&full[stage], bytes);
      bulk_g2s(tiles + stage * TILE, recE + (size_t)(kt + BNS) * TILE, bytes, &full[stage]);
    }
  }
#pragma unroll
  for (int k = 0; k < RI; ++k) {
    const int i = t * TI + tid + k * NT;
    if (i < Ne)
#pragma unroll
      for (int a = 0; a < ACC; ++a) outE[(size_t)i * D + a] = (double)sum[k][a] - (double)cmp[k][a];
  }
  return true;
}

// mode 0: density for every item; 1: gradient for every item; 2: by the
// ensemble's minimiser state (trial -> density, direction -> gradient).
template <int D, int RI, int NT>
__global__ void __launch_bounds__(NT)
    k_bpair(const float *__restrict__ rec, const long long *__restrict__ off, const int *__restrict__ sizes,
            const int2 *__restrict__ queue, int nitems, unsigned *counter, int mode,
            const BState *__restrict__ st, double *__restrict__ acc_out, int *err) {
  constexpr int DP = Rec<D>::DP;
  extern __shared__ __align__(128) float tiles[];
  __shared__ __align__(8) uint64_t full[BNS];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < BNS; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long gtile = 0;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    const int2 w = queue[item];
    const int e = w.x, t = w.y;
    bool grad = (mode == 1);
    if (mode == 2) {
      const int ph = st[e].phase;
      if (ph != ST_TRIAL && ph != ST_GRAD) continue;
      grad = ph == ST_GRAD;
    }
    const int Ne = sizes[e];
    const long long base = off[e];
    const bool ok = grad ? bitem<D, RI, NT, true>(tiles, full, rec + base * DP, Ne, t, gtile, acc_out + base * D)
                         : bitem<D, RI, NT, false>(tiles, full, rec + base * DP, Ne, t, gtile, acc_out + base * D);
    if (!ok) {
      if (tid == 0) vds_flag(err, VDS_ETIMEOUT);
      return;
    }
    gtile += (Ne + BTJ - 1) / BTJ;
  }
}

// ------------------------------------------------------ per-particle kernels

__device__ __forceinline__ double bA(int j, int k) {
  return j == k ? 2.0 : ((j - k == 1 || k - j == 1) ? -1.0 : 0.0);
}
__device__ __forceinline__ double bAinv(int j, int k, int nb) {
  const int lo = (j < k ? j : k) + 1, hi = (j > k ? j : k) + 1;
  return (double)lo * (double)(nb + 1 - hi) / (double)(nb + 1);
}

template <int D>
__device__ __forceinline__ bool bspring(const BCommon &cm, const double (&y)[D], double &psi, double (&f)[8]) {
  psi = 0.0;
  bool ok = true;
  for (int k = 0; k < cm.nb; ++k) {
    double n2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a / cm.s == k) n2 += y[a] * y[a];
    if (cm.spring == 0) {
      psi += 0.5 * cm.H[k] * n2;
      f[k] = cm.H[k];
    } else {
      const double x = 1.0 - n2 / cm.b;
      if (!(x > 0.0)) {
        ok = false;
        f[k] = 0.0;
      } else {
        psi += -0.5 * cm.H[k] * cm.b * log(x);
        f[k] = cm.H[k] / x;
      }
    }
  }
  return ok;
}

template <int D>
__device__ __forceinline__ void write_rec(float *rec, long i, float c, const float (&y)[D]) {
  constexpr int DP = Rec<D>::DP;
  float o[DP];
#pragma unroll
  for (int d = 0; d < D; ++d) o[d] = c * y[d];
#pragma unroll
  for (int d = D; d < DP; ++d) o[d] = 0.f;
  float4 *dst = reinterpret_cast<float4 *>(rec + (size_t)i * DP);
#pragma unroll
  for (int v = 0; v < DP / 4; ++v) dst[v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
}

// mode 0: records from q for every particle.
// mode 1: implicit round: trial records y = q* + (d_cur - alpha dir) (the
//         trial displacement stored in the other buffer), or the final q.
// mode 2: start of an implicit step: q* = q + dt kappa_e q, zero buffers.
template <int D>
__global__ void k_bprep(long total, const int *__restrict__ ens, const EParam *__restrict__ ep,
                        const BState *__restrict__ st, const BCommon cm, int mode, float *q, float *qs,
                        float *dA, float *dB, float *dir, float *dprev, float *__restrict__ rec) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int e = ens[i];
  const float c = ep[e].c;
  float y[D];
  if (mode == 0) {
#pragma unroll
    for (int d = 0; d < D; ++d) y[d] = q[(size_t)i * D + d];
    write_rec<D>(rec, i, c, y);
    return;
  }
  if (mode == 2) {
    float x[D];
#pragma unroll
    for (int d = 0; d < D; ++d) x[d] = q[(size_t)i * D + d];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int k = a / cm.s, al = a - k * cm.s;
      double v = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b)
        if (b / cm.s == k) v += ep[e].kappa[al * cm.s + (b - k * cm.s)] * (double)x[b];
      qs[(size_t)i * D + a] = (float)((double)x[a] + cm.dt * v);
      dB[(size_t)i * D + a] = 0.f;
      dir[(size_t)i * D + a] = 0.f;
    }
    // start from q* + the previous step's correction of this call (zero at
    // its first step); a particle whose start would leave the FENE domain
    // starts from q*
    bool inside = true;
    if (cm.spring == 1)
      for (int k = 0; k < cm.nb; ++k) {
        double n2 = 0.0;
        for (int a = 0; a < cm.s; ++a) {
          const double y = (double)qs[(size_t)i * D + cm.s * k + a] + dprev[(size_t)i * D + cm.s * k + a];
          n2 += y * y;
        }
        if (!(n2 < cm.b)) inside = false;
      }
#pragma unroll
    for (int a = 0; a < D; ++a) dA[(size_t)i * D + a] = inside ? dprev[(size_t)i * D + a] : 0.f;
    return;
  }
  const BState s = st[e];
  const float *dcur = s.cur ? dB : dA;
  float *doth = s.cur ? dA : dB;
  if (s.phase == ST_TRIAL) {
    const float al = (float)s.alpha;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float dl = dcur[(size_t)i * D + d] - al * dir[(size_t)i * D + d];
      doth[(size_t)i * D + d] = dl;
      y[d] = qs[(size_t)i * D + d] + dl;
    }
    write_rec<D>(rec, i, c, y);
  } else if (s.phase == ST_FINAL) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float dl = dcur[(size_t)i * D + d];
      if (s.fin_dir) dl = dl - 1.f * dir[(size_t)i * D + d];
      q[(size_t)i * D + d] = qs[(size_t)i * D + d] + dl;
      dprev[(size_t)i * D + d] = dl;
    }
  }
}

// mode 0: density finish (w, rho_out, energy terms in contrib[3i]);
// mode 1: gradient output g; mode 2: explicit Euler update + records;
// mode 3: implicit round (trial: w and J terms; gradient: g -> direction).
template <int D>
__global__ void k_bfin(long total, const int *__restrict__ ens, const EParam *__restrict__ ep,
                       const BState *__restrict__ st, const BCommon cm, int mode, int want_energy,
                       const double *__restrict__ acc, float *rec, float *q, const float *__restrict__ qs,
                       const float *dA, const float *dB, float *dir, float *__restrict__ out,
                       double *__restrict__ contrib, int *err) {
  constexpr int DP = Rec<D>::DP;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int e = ens[i];
  const EParam &P = ep[e];
  int phase = -1;
  const float *dcur = nullptr, *doth = nullptr;
  if (mode == 3) {
    const BState s = st[e];
    phase = s.phase;
    dcur = s.cur ? dB : dA;
    doth = s.cur ? dA : dB;
    if (phase != ST_TRIAL && phase != ST_GRAD) return;
  }
  const bool dens = mode == 0 || (mode == 3 && phase == ST_TRIAL);
  double y[D];
  float yf[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float v;
    if (mode == 3) v = qs[(size_t)i * D + d] + (phase == ST_TRIAL ? doth : dcur)[(size_t)i * D + d];
    else v = q[(size_t)i * D + d];
    yf[d] = v;
    y[d] = (double)v;
  }
  double psi, fk[8];
  const bool ok = bspring<D>(cm, y, psi, fk);
  if (dens) {
    const double rho = acc[(size_t)i * D];
    if (!(rho >= 0.5 && rho <= 1e300)) vds_flag(err, VDS_ENAN);
    rec[(size_t)i * DP + D] = (float)(1.0 / rho);
    if (mode == 0 && out) out[i] = (float)rho;
    if (mode == 0 && !ok && want_energy) vds_flag(err, VDS_EDOMAIN);
    if (want_energy || mode == 3) {
      double en = cm.kBT * (log(rho) + P.lnorm) + psi;
      if (mode == 3) {
        double quad = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (a % cm.s == b % cm.s)
              quad += (double)doth[(size_t)i * D + a] * bAinv(a / cm.s, b / cm.s, cm.nb) *
                      (double)doth[(size_t)i * D + b];
        en += cm.zeta / (2.0 * cm.dt) * quad;
      }
      contrib[3 * i] = en;
      contrib[3 * i + 1] = ok ? 0.0 : 1.0;
      contrib[3 * i + 2] = 0.0;
    }
    return;
  }
  if (!ok) vds_flag(err, VDS_EDOMAIN);
  double g[D];
#pragma unroll
  for (int a = 0; a < D; ++a) g[a] = cm.kBT * (-P.sfac * acc[(size_t)i * D + a]) + fk[a / cm.s] * y[a];
  if (mode == 1) {
#pragma unroll
    for (int a = 0; a < D; ++a) out[(size_t)i * D + a] = (float)g[a];
    return;
  }
  if (mode == 2) {
    float yn[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int k = a / cm.s, al = a - k * cm.s;
      double v = 0.0, m = 0.0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int kb = b / cm.s, be = b - kb * cm.s;
        if (kb == k) v += P.kappa[al * cm.s + be] * y[b];
        if (be == al) m += bA(k, kb) * g[b];
      }
      yn[a] = (float)(y[a] + cm.dt * (v - m / cm.zeta));
    }
    if (cm.spring == 1)
      for (int k = 0; k < cm.nb; ++k) {
        double n2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
          if (a / cm.s == k) n2 += (double)yn[a] * yn[a];
        if (!(n2 < cm.b)) vds_flag(err, VDS_EDOMAIN);
      }
#pragma unroll
    for (int a = 0; a < D; ++a) q[(size_t)i * D + a] = yn[a];
    write_rec<D>(rec, i, P.c, yn);
    return;
  }
  // mode 3, new direction
  double dec = 0.0, dmax = 0.0, ymax = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int k = a / cm.s, al = a - k * cm.s;
    double ag = 0.0, aid = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const int kb = b / cm.s, be = b - kb * cm.s;
      if (be == al) {
        ag += bA(k, kb) * g[b];
        aid += bAinv(k, kb, cm.nb) * (double)dcur[(size_t)i * D + b];
      }
    }
    const double dr = (double)dcur[(size_t)i * D + a] + cm.dt / cm.zeta * ag;
    const double G = cm.zeta / cm.dt * aid + g[a];
    const float drf = (float)dr;
    dir[(size_t)i * D + a] = drf;
    dec += G * dr;
    dmax = fmax(dmax, fabs((double)drf));
    ymax = fmax(ymax, fabs((double)yf[a]));
  }
  contrib[3 * i] = dec;
  contrib[3 * i + 1] = dmax;
  contrib[3 * i + 2] = ymax;
}

// One CTA per ensemble: fixed-order sums of the particles' contributions.
// mode 0: energies E_e -> eout[e].  mode 3: implicit state machine.
__global__ void __launch_bounds__(RNT)
    k_breduce(int E, const long long *__restrict__ off, const int *__restrict__ sizes, BState *st,
              const BCommon cm, int mode, const double *__restrict__ contrib, double *eout, int *active) {
  __shared__ double sh[3][RNT];
  const int e = blockIdx.x;
  if (e >= E) return;
  BState s = st[e];
  if (mode == 3 && s.phase == ST_FINAL) {
    if (threadIdx.x == 0) {
      s.phase = ST_DONE;
      st[e] = s;
    }
    return;
  }
  if (mode == 3 && s.phase == ST_DONE) return;
  const long long base = off[e];
  const int Ne = sizes[e];
  const bool gradphase = mode == 3 && s.phase == ST_GRAD;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int k = threadIdx.x; k < Ne; k += RNT) {
    const double *c = contrib + 3 * (base + k);
    a0 += c[0];
    if (gradphase) {
      a1 = fmax(a1, c[1]);
      a2 = fmax(a2, c[2]);
    } else {
      a1 += c[1];
    }
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int o = RNT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      if (gradphase) {
        sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
        sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
      } else {
        sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    eout[e] = sh[0][0] / (double)Ne;
    return;
  }
  if (s.phase == ST_TRIAL) {
    const double Jn = sh[0][0] / (double)Ne;
    const bool bad = sh[1][0] > 0.0;
    if (!bad && Jn <= s.J - 1e-4 * s.alpha * s.dec + cm.jfloor * (1.0 + fabs(s.J))) {
      s.J = Jn;
      s.cur ^= 1;
      if (s.it >= cm.max_iter) {
        s.status = VDS_ENOCONV;
        s.phase = ST_FINAL;
        s.fin_dir = 0;
      } else {
        s.phase = ST_GRAD;
      }
    } else {
      s.alpha *= 0.5;
      s.ls += 1;
      if (s.ls > 30) {
        s.status = VDS_ENOCONV;
        s.phase = ST_FINAL;
        s.fin_dir = 0;
      }
    }
  } else {  // ST_GRAD: direction computed
    s.it += 1;
    s.dec = sh[0][0] / (double)Ne;
    const double dmax = sh[1][0], ymax = sh[2][0];
    if (!(fabs(s.dec) <= 1e300)) {
      s.status = VDS_ENAN;
      s.phase = ST_FINAL;
      s.fin_dir = 0;
    } else if (dmax <= cm.tol * (1.0 + ymax)) {
      s.phase = ST_FINAL;
      s.fin_dir = 1;
    } else {
      s.alpha = 1.0;
      s.ls = 0;
      s.phase = ST_TRIAL;
    }
  }
  st[e] = s;
  if (s.phase != ST_DONE) atomicAdd(active, 1);
}

__global__ void k_binit(int E, BState *st) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  BState s;
  s.J = __longlong_as_double(0x7ff0000000000000ll);  // +inf: the first trial (y = q*) is accepted
  s.alpha = 1.0;
  s.dec = 0.0;
  s.phase = ST_TRIAL;
  s.it = 0;
  s.ls = 0;
  s.status = 0;
  s.cur = 0;
  s.fin_dir = 0;
  st[e] = s;
}

// tau_e = (1/N_e) sum_I sum_k q_k (x) grad Psi_k(q_k) for ensemble e = block;
// FP64, fixed per-thread assignment and tree order (deterministic).
template <int D>
__global__ void __launch_bounds__(256)
    k_bstress(const float *__restrict__ q, const long long *__restrict__ off, const int *__restrict__ sizes,
              const BCommon cm, double *__restrict__ tau, int *err) {
  __shared__ double sh[9][256];
  const int e = blockIdx.x, s = cm.s;
  const long long base = off[e];
  const int Ne = sizes[e];
  double acc[9];
#pragma unroll
  for (int x = 0; x < 9; ++x) acc[x] = 0.0;
  for (int i = threadIdx.x; i < Ne; i += blockDim.x) {
    float y[D];
#pragma unroll
    for (int d = 0; d < D; ++d) y[d] = q[(size_t)(base + i) * D + d];
    for (int k = 0; k < cm.nb; ++k) {
      double f = cm.H[k];
      if (cm.spring == 1) {
        double n2 = 0.0;
        for (int a = 0; a < s; ++a) n2 += (double)y[s * k + a] * y[s * k + a];
        if (!(n2 < cm.b)) vds_flag(err, VDS_EDOMAIN);
        f = cm.H[k] / (1.0 - n2 / cm.b);
      }
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) acc[a * s + b] += (double)y[s * k + a] * f * (double)y[s * k + b];
    }
  }
#pragma unroll
  for (int x = 0; x < 9; ++x) sh[x][threadIdx.x] = acc[x];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int x = 0; x < 9; ++x) sh[x][threadIdx.x] += sh[x][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < s * s) tau[(size_t)e * s * s + threadIdx.x] = sh[threadIdx.x][0] / (double)Ne;
}

__global__ void k_bset_kappa(EParam *ep, const double *__restrict__ kappa, int E, int ss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int k = 0; k < 9; ++k) ep[e].kappa[k] = k < ss ? kappa[(size_t)e * ss + k] : 0.0;
}

}  // namespace

// ------------------------------------------------------------------ host

struct vds_batch {
  int device = 0, E = 0, D = 0, tile = 0, nitems = 0, grid = 0, scheme = 0, cfg = 0, max_items = 0;
  long total = 0;
  BCommon cm;
  std::vector<int> sizes;
  std::vector<long long> off;
  std::vector<int> items;  // host copy of the queue
  long long *d_off = nullptr;
  int *d_sizes = nullptr, *d_ens = nullptr, *d_active = nullptr, *h_active = nullptr;
  int2 *d_queue = nullptr;
  unsigned *d_counter = nullptr;
  EParam *d_ep = nullptr;
  BState *d_st = nullptr;
  float *rec = nullptr, *qs = nullptr, *dA = nullptr, *dB = nullptr, *dir = nullptr, *dprev = nullptr;
  double *acc = nullptr, *contrib = nullptr, *eout = nullptr;
  size_t smem = 0;
  cudaGraphExec_t round_exec = nullptr;
  cudaGraph_t round_graph = nullptr;
  cudaStream_t graph_stream = nullptr;  // stream the round graph was captured for
  float *graph_q = nullptr;
};

namespace {

template <int D, int RI, int NT>
int b_launch_cfg(vds_ctx *c, vds_batch *b, int mode) {
  k_bpair<D, RI, NT><<<b->grid, NT, b->smem, c->stream>>>(b->rec, b->d_off, b->d_sizes, b->d_queue, b->nitems,
                                                           b->d_counter, mode, b->d_st, b->acc, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  return VDS_OK;
}

template <int D>
int b_launch_pair(vds_ctx *c, vds_batch *b, int mode) {
  VDS_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), c->stream));
  VDS_TRY(vds_time_begin(c, mode == 1 ? PK_GRADIENT : PK_DENSITY));
  switch (b->cfg) {
    case 0: VDS_TRY((b_launch_cfg<D, kCfgRI[0], kCfgNT[0]>(c, b, mode))); break;
    case 1: VDS_TRY((b_launch_cfg<D, kCfgRI[1], kCfgNT[1]>(c, b, mode))); break;
    case 2: VDS_TRY((b_launch_cfg<D, kCfgRI[2], kCfgNT[2]>(c, b, mode))); break;
    default: VDS_TRY((b_launch_cfg<D, kCfgRI[3], kCfgNT[3]>(c, b, mode))); break;
  }
  VDS_TRY(vds_time_end(c, mode == 1 ? PK_GRADIENT : PK_DENSITY));
  ++c->launches;
  return VDS_OK;
}

template <int D>
int b_prep(vds_ctx *c, vds_batch *b, int mode, float *q) {
  k_bprep<D><<<(unsigned)((b->total + 255) / 256), 256, 0, c->stream>>>(
      b->total, b->d_ens, b->d_ep, b->d_st, b->cm, mode, q, b->qs, b->dA, b->dB, b->dir, b->dprev, b->rec);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

template <int D>
int b_fin(vds_ctx *c, vds_batch *b, int mode, int want_energy, float *q, float *out) {
  k_bfin<D><<<(unsigned)((b->total + 255) / 256), 256, 0, c->stream>>>(
      b->total, b->d_ens, b->d_ep, b->d_st, b->cm, mode, want_energy, b->acc, b->rec, q, b->qs, b->dA, b->dB,
      b->dir, out, b->contrib, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

int b_reduce(vds_ctx *c, vds_batch *b, int mode) {
  k_breduce<<<b->E, RNT, 0, c->stream>>>(b->E, b->d_off, b->d_sizes, b->d_st, b->cm, mode, b->contrib, b->eout,
                                         b->d_active);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

#define VDS_BATCH_D(D, CALL)     \
  switch (D) {                   \
    case 2: return CALL(2);      \
    case 3: return CALL(3);      \
    case 4: return CALL(4);      \
    case 6: return CALL(6);      \
    case 8: return CALL(8);      \
    case 9: return CALL(9);      \
    case 12: return CALL(12);    \
    default: return VDS_EARG;    \
  }

template <int D, int RI, int NT>
int b_setup_cfg(vds_ctx *c, vds_batch *b) {
  b->tile = NT * RI;
  b->smem = (size_t)BNS * BTJ * Rec<D>::DP * sizeof(float);
  VDS_CUDA_TRY(cudaFuncSetAttribute(k_bpair<D, RI, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int occ = 0;
  VDS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bpair<D, RI, NT>, NT, b->smem));
  b->grid = c->num_sms * (occ > 0 ? occ : 1);
  return VDS_OK;
}

// Select pair-kernel shape b->cfg: i-tile, shared memory, grid (resident CTAs
// on every SM, at most one per work item) and the work queue for that tile.
template <int D>
int b_setup_kernel(vds_ctx *c, vds_batch *b) {
  switch (b->cfg) {
    case 0: VDS_TRY((b_setup_cfg<D, kCfgRI[0], kCfgNT[0]>(c, b))); break;
    case 1: VDS_TRY((b_setup_cfg<D, kCfgRI[1], kCfgNT[1]>(c, b))); break;
    case 2: VDS_TRY((b_setup_cfg<D, kCfgRI[2], kCfgNT[2]>(c, b))); break;
    default: VDS_TRY((b_setup_cfg<D, kCfgRI[3], kCfgNT[3]>(c, b))); break;
  }
  return VDS_OK;
}

// Work queue in longest-processing-time order for the current tile: cost N_e
// descending, then ensemble, then tile ascending.
void b_build_queue(vds_batch *b) {
  struct It {
    int n, e, t;
  };
  std::vector<It> its;
  for (int e = 0; e < b->E; ++e)
    for (int t = 0; t < (b->sizes[e] + b->tile - 1) / b->tile; ++t) its.push_back({b->sizes[e], e, t});
  std::sort(its.begin(), its.end(), [](const It &a, const It &bb) {
    if (a.n != bb.n) return a.n > bb.n;
    if (a.e != bb.e) return a.e < bb.e;
    return a.t < bb.t;
  });
  b->nitems = (int)its.size();
  b->items.resize(2 * its.size());
  for (size_t k = 0; k < its.size(); ++k) {
    b->items[2 * k] = its[k].e;
    b->items[2 * k + 1] = its[k].t;
  }
  if (b->grid > b->nitems) b->grid = b->nitems;
}

void b_drop_graph(vds_batch *b) {
  if (b->round_exec) cudaGraphExecDestroy(b->round_exec);
  if (b->round_graph) cudaGraphDestroy(b->round_graph);
  b->round_exec = nullptr;
  b->round_graph = nullptr;
  b->graph_stream = nullptr;
  b->graph_q = nullptr;
}

// Switch to shape cfg: kernel setup, queue, upload; the round graph is
// captured again at the next implicit step.
int b_apply_config(vds_ctx *c, vds_batch *b, int cfg) {
  b->cfg = cfg;
  int st;
#define SETUP(DD) b_setup_kernel<DD>(c, b)
  st = [&]() -> int { VDS_BATCH_D(b->D, SETUP) }();
#undef SETUP
  VDS_TRY(st);
  b_build_queue(b);
  if (b->nitems > b->max_items) return VDS_EARG;
  VDS_CUDA_TRY(cudaMemcpyAsync(b->d_queue, b->items.data(), sizeof(int2) * b->nitems, cudaMemcpyHostToDevice,
                               c->stream));
  VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  b_drop_graph(b);
  return VDS_OK;
}

template <int D>
int b_round(vds_ctx *c, vds_batch *b, float *q) {
  VDS_TRY(b_prep<D>(c, b, 1, q));
  VDS_TRY(b_launch_pair<D>(c, b, 2));
  VDS_TRY(b_fin<D>(c, b, 3, 0, q, nullptr));
  VDS_CUDA_TRY(cudaMemsetAsync(b->d_active, 0, sizeof(int), c->stream));
  VDS_TRY(b_reduce(c, b, 3));
  VDS_CUDA_TRY(cudaMemcpyAsync(b->h_active, b->d_active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return VDS_OK;
}

template <int D>
int b_energy_grad(vds_ctx *c, vds_batch *b, const float *q, double *E, float *g, float *rho) {
  VDS_TRY(b_prep<D>(c, b, 0, (float *)q));
  VDS_TRY(b_launch_pair<D>(c, b, 0));
  VDS_TRY(b_fin<D>(c, b, 0, E ? 1 : 0, (float *)q, rho));
  if (E) VDS_TRY(b_reduce(c, b, 0));
  if (g) {
    VDS_TRY(b_launch_pair<D>(c, b, 1));
    VDS_TRY(b_fin<D>(c, b, 1, 0, (float *)q, g));
  }
  if (E) VDS_CUDA_TRY(cudaMemcpyAsync(E, b->eout, sizeof(double) * b->E, cudaMemcpyDeviceToHost, c->stream));
  return vds_sync_status(c);
}

template <int D>
int b_step(vds_ctx *c, vds_batch *b, float *q, int nsteps, int *iters_out, int scheme) {
  if (scheme == 0) {
    VDS_TRY(b_prep<D>(c, b, 0, q));
    for (int n = 0; n < nsteps; ++n) {
      VDS_TRY(b_launch_pair<D>(c, b, 0));
      VDS_TRY(b_fin<D>(c, b, 0, 0, q, nullptr));
      VDS_TRY(b_launch_pair<D>(c, b, 1));
      VDS_TRY(b_fin<D>(c, b, 2, 0, q, nullptr));
    }
    return vds_sync_status(c);
  }
  // implicit: capture one round as a graph (per stream and q), replay until done
  const bool timing = c->timing && c->timing->on;
  if (!timing && (!b->round_exec || b->graph_stream != c->stream || b->graph_q != q)) {
    if (b->round_exec) {
      cudaGraphExecDestroy(b->round_exec);
      cudaGraphDestroy(b->round_graph);
      b->round_exec = nullptr;
      b->round_graph = nullptr;
    }
    cudaStream_t cap;
    VDS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    c->stream = cap;
    const long saved_launches = c->launches;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int st = VDS_OK;
    if (e == cudaSuccess) st = b_round<D>(c, b, q);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    c->stream = saved;
    c->launches = saved_launches;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess || st != VDS_OK) {
      if (graph) cudaGraphDestroy(graph);
      vds_last_cuda_error(e != cudaSuccess ? e : e2);
      return st != VDS_OK ? st : VDS_ECUDA;
    }
    VDS_CUDA_TRY(cudaGraphInstantiate(&b->round_exec, graph, 0));
    b->round_graph = graph;
    b->graph_stream = c->stream;
    b->graph_q = q;
  }
  const int round_launches = 4;
  const int max_rounds = 32 * (b->cm.max_iter + 1) + 4;
  std::vector<BState> hs(b->E);
  int status = VDS_OK;
  // the first step of a call starts every minimiser from q*
  VDS_CUDA_TRY(cudaMemsetAsync(b->dprev, 0, sizeof(float) * (size_t)b->total * D, c->stream));
  for (int n = 0; n < nsteps; ++n) {
    k_binit<<<(b->E + 255) / 256, 256, 0, c->stream>>>(b->E, b->d_st);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    VDS_TRY(b_prep<D>(c, b, 2, q));
    int rounds = 0;
    for (;;) {
      if (timing) {
        VDS_TRY(b_round<D>(c, b, q));
      } else {
        VDS_CUDA_TRY(cudaGraphLaunch(b->round_exec, c->stream));
        c->launches += round_launches;
      }
      ++rounds;
      VDS_TRY(vds_sync_status(c));
      if (*b->h_active == 0) break;
      if (rounds >= max_rounds) return VDS_ENOCONV;
    }
    // final rounds move FINAL -> DONE; q is written in the round that saw FINAL
    VDS_CUDA_TRY(cudaMemcpyAsync(hs.data(), b->d_st, sizeof(BState) * b->E, cudaMemcpyDeviceToHost, c->stream));
    VDS_TRY(vds_sync_status(c));
    for (int e = 0; e < b->E; ++e) {
      if (iters_out) iters_out[(size_t)n * b->E + e] = hs[e].it;
      if (hs[e].status != 0 && status == VDS_OK) status = hs[e].status;
    }
    if (status != VDS_OK) return status;
  }
  return VDS_OK;
}

template <int D>
int b_autotune(vds_ctx *c, vds_batch *b, const float *q, int reps, int *best_cfg, double *ms_out) {
  // records of q with w = 1/rho, from one density pass in the current shape
  VDS_TRY(b_prep<D>(c, b, 0, (float *)q));
  VDS_TRY(b_launch_pair<D>(c, b, 0));
  VDS_TRY(b_fin<D>(c, b, 0, 0, (float *)q, nullptr));
  VDS_TRY(vds_sync_status(c));
  struct Ev {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Ev() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  VDS_CUDA_TRY(cudaEventCreate(&ev.e[0]));
  VDS_CUDA_TRY(cudaEventCreate(&ev.e[1]));
  double best = 1e300;
  int bi = b->cfg;
  for (int k = 0; k < VDS_BATCH_CONFIGS; ++k) {
    VDS_TRY(b_apply_config(c, b, k));
    VDS_TRY(b_launch_pair<D>(c, b, 0));  // warm-up
    VDS_TRY(b_launch_pair<D>(c, b, 1));
    double tmin = 1e300;
    for (int r = 0; r < reps; ++r) {
      VDS_CUDA_TRY(cudaEventRecord(ev.e[0], c->stream));
      VDS_TRY(b_launch_pair<D>(c, b, 0));
      VDS_TRY(b_launch_pair<D>(c, b, 1));
      VDS_CUDA_TRY(cudaEventRecord(ev.e[1], c->stream));
      VDS_TRY(vds_sync_status(c));
      float ms = 0.f;
      VDS_CUDA_TRY(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
      if (ms < tmin) tmin = ms;
    }
    if (ms_out) ms_out[k] = tmin;
    if (tmin < best) {
      best = tmin;
      bi = k;
    }
  }
  VDS_TRY(b_apply_config(c, b, bi));
  if (best_cfg) *best_cfg = bi;
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

}  // namespace

extern "C" {

void vds_batch_free(vds_batch *b) {
  if (!b) return;
  Dev dg(b->device);
  b_drop_graph(b);
  void *ptrs[] = {b->d_off, b->d_sizes, b->d_ens, b->d_active, b->d_queue, b->d_counter, b->d_ep, b->d_st,
                  b->rec, b->qs, b->dA, b->dB, b->dir, b->dprev, b->acc, b->contrib, b->eout};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (b->h_active) cudaFreeHost(b->h_active);
  delete b;
}

int vds_batch_create(vds_ctx *c, int E, const int *sizes, int D, const vds_params *p, const double *h,
                     const double *kappa, vds_batch **out) {
  if (!c || !out || !sizes || !p || !h || !kappa || E < 1) return VDS_EARG;
  if (p->s < 2 || p->s > 3 || p->nb < 1 || p->nb > 8 || p->nb * p->s != D) return VDS_EARG;
  if (D != 2 && D != 3 && D != 4 && D != 6 && D != 8 && D != 9 && D != 12) return VDS_EARG;
  if (!(p->zeta > 0.0) || !(p->kBT >= 0.0) || (p->spring != 0 && p->spring != 1)) return VDS_EARG;
  if (p->spring == 1 && !(p->b > 0.0)) return VDS_EARG;
  for (int e = 0; e < E; ++e)
    if (sizes[e] < 1 || !(h[e] > 0.0)) return VDS_EARG;
  *out = nullptr;
  Dev dg(c->device);
  vds_batch *b = new vds_batch();
  b->device = c->device;
  b->E = E;
  b->D = D;
  b->cm.nb = p->nb;
  b->cm.s = p->s;
  b->cm.spring = p->spring;
  b->cm.max_iter = p->max_iter;
  for (int j = 0; j < 8; ++j) b->cm.H[j] = p->H[j];
  b->cm.b = p->b;
  b->cm.kBT = p->kBT;
  b->cm.zeta = p->zeta;
  b->cm.dt = p->dt;
  b->cm.tol = p->tol;
  b->cm.jfloor = p->jfloor;
  b->scheme = p->scheme;
  b->sizes.assign(sizes, sizes + E);
  b->off.resize(E);
  long tot = 0;
  for (int e = 0; e < E; ++e) {
    b->off[e] = tot;
    tot += sizes[e];
  }
  b->total = tot;
  b->max_items = 0;
  for (int e = 0; e < E; ++e) b->max_items += (sizes[e] + kMinTile - 1) / kMinTile;
  std::vector<int> ens(tot);
  for (int e = 0; e < E; ++e)
    for (int k = 0; k < sizes[e]; ++k) ens[b->off[e] + k] = e;
  std::vector<EParam> ep(E);
  for (int e = 0; e < E; ++e) {
    const double cc = sqrt(1.4426950408889634 / (2.0 * h[e] * h[e]));
    ep[e].c = (float)cc;
    ep[e].pad_ = 0.f;
    ep[e].h = h[e];
    ep[e].sfac = 1.0 / (h[e] * h[e] * (double)ep[e].c);
    ep[e].lnorm = -log((double)sizes[e]) - 0.5 * D * log(2.0 * 3.14159265358979323846 * h[e] * h[e]);
    for (int k = 0; k < 9; ++k) ep[e].kappa[k] = 0.0;
    for (int k = 0; k < p->s * p->s; ++k) ep[e].kappa[k] = kappa[(size_t)e * p->s * p->s + k];
  }
  const size_t nd = (size_t)tot * D;
  cudaError_t ce = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMalloc(ptr, bytes);
  };
  A((void **)&b->d_off, sizeof(long long) * E);
  A((void **)&b->d_sizes, sizeof(int) * E);
  A((void **)&b->d_ens, sizeof(int) * tot);
  A((void **)&b->d_active, sizeof(int));
  A((void **)&b->d_queue, sizeof(int2) * b->max_items);
  A((void **)&b->d_counter, sizeof(unsigned));
  A((void **)&b->d_ep, sizeof(EParam) * E);
  A((void **)&b->d_st, sizeof(BState) * E);
  A((void **)&b->rec, sizeof(float) * (size_t)tot * Rec<12>::DP);
  A((void **)&b->qs, sizeof(float) * nd);
  A((void **)&b->dA, sizeof(float) * nd);
  A((void **)&b->dB, sizeof(float) * nd);
  A((void **)&b->dir, sizeof(float) * nd);
  A((void **)&b->dprev, sizeof(float) * nd);
  A((void **)&b->acc, sizeof(double) * nd);
  A((void **)&b->contrib, sizeof(double) * 3 * tot);
  A((void **)&b->eout, sizeof(double) * E);
  if (ce == cudaSuccess) ce = cudaMallocHost((void **)&b->h_active, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemcpy(b->d_off, b->off.data(), sizeof(long long) * E, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(b->d_sizes, sizes, sizeof(int) * E, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(b->d_ens, ens.data(), sizeof(int) * tot, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(b->d_ep, ep.data(), sizeof(EParam) * E, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    vds_last_cuda_error(ce);
    vds_batch_free(b);
    return ce == cudaErrorMemoryAllocation ? VDS_ENOMEM : VDS_ECUDA;
  }
  const int st = b_apply_config(c, b, default_config(D));
  if (st != VDS_OK) {
    vds_batch_free(b);
    return st;
  }
  *out = b;
  return VDS_OK;
}

int vds_batch_info(const vds_batch *b, long *total, int *tile, int *n_items) {
  if (!b) return VDS_EARG;
  if (total) *total = b->total;
  if (tile) *tile = b->tile;
  if (n_items) *n_items = b->nitems;
  return VDS_OK;
}

int vds_batch_queue(const vds_batch *b, int *items, int n_items) {
  if (!b || !items || n_items < b->nitems) return VDS_EARG;
  memcpy(items, b->items.data(), sizeof(int) * 2 * b->nitems);
  return VDS_OK;
}

int vds_batch_stress(vds_ctx *c, vds_batch *b, const float *q, double *tau) {
  if (!c || !b || !q || !tau || b->device != c->device) return VDS_EARG;
  Dev dg(c->device);
  const int ss = b->cm.s * b->cm.s;
  VDS_TRY(vds_ensure(c, c->red, (size_t)b->E * ss * sizeof(double)));
  double *dt = (double *)c->red.ptr;
#define CALL(DD) (k_bstress<DD><<<b->E, 256, 0, c->stream>>>(q, b->d_off, b->d_sizes, b->cm, dt, c->err), VDS_OK)
  const int st = [&]() -> int { VDS_BATCH_D(b->D, CALL) }();
#undef CALL
  VDS_TRY(st);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_CUDA_TRY(cudaMemcpyAsync(tau, dt, (size_t)b->E * ss * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return vds_sync_status(c);
}

int vds_batch_set_kappa(vds_ctx *c, vds_batch *b, const double *kappa) {
  if (!c || !b || !kappa || b->device != c->device) return VDS_EARG;
  Dev dg(c->device);
  const int ss = b->cm.s * b->cm.s;
  VDS_TRY(vds_ensure(c, c->red, (size_t)b->E * ss * sizeof(double)));
  double *dk = (double *)c->red.ptr;
  VDS_CUDA_TRY(cudaMemcpyAsync(dk, kappa, (size_t)b->E * ss * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  k_bset_kappa<<<(b->E + 255) / 256, 256, 0, c->stream>>>(b->d_ep, dk, b->E, ss);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return vds_sync_status(c);
}

int vds_batch_set_config(vds_ctx *c, vds_batch *b, int config) {
  if (!c || !b || config < 0 || config >= VDS_BATCH_CONFIGS || b->device != c->device) return VDS_EARG;
  Dev dg(c->device);
  return b_apply_config(c, b, config);
}

int vds_batch_get_config(const vds_batch *b, int *config) {
  if (!b || !config) return VDS_EARG;
  *config = b->cfg;
  return VDS_OK;
}

int vds_batch_autotune(vds_ctx *c, vds_batch *b, const float *q, int reps, int *config, double *ms) {
  if (!c || !b || !q || reps < 1 || b->device != c->device) return VDS_EARG;
  Dev dg(c->device);
#define CALL(DD) b_autotune<DD>(c, b, q, reps, config, ms)
  VDS_BATCH_D(b->D, CALL)
#undef CALL
}

int vds_batch_energy_grad(vds_ctx *c, vds_batch *b, const float *q, double *E, float *g, float *rho) {
  if (!c || !b || !q || b->device != c->device) return VDS_EARG;
  Dev dg(c->device);
#define CALL(DD) b_energy_grad<DD>(c, b, q, E, g, rho)
  VDS_BATCH_D(b->D, CALL)
#undef CALL
}

int vds_batch_step(vds_ctx *c, vds_batch *b, float *q, int nsteps, int *iters_out) {
  if (!c || !b || !q || nsteps < 0 || b->device != c->device) return VDS_EARG;
  if (!(b->cm.dt > 0.0) || (b->scheme != 0 && b->scheme != 1)) return VDS_EARG;
  if (b->scheme == 1 && (b->cm.max_iter < 1 || !(b->cm.tol >= 0.0))) return VDS_EARG;
  if (nsteps == 0) return VDS_OK;
  Dev dg(c->device);
#define CALL(DD) b_step<DD>(c, b, q, nsteps, iters_out, b->scheme)
  VDS_BATCH_D(b->D, CALL)
#undef CALL
}

}  // extern "C"
