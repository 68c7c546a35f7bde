// refresh.cu -- the pair pass that rebuilds the linearised Brownian terms of
// the reduced model (Sec. 2.4, Eq. model_DymReduced) at a lifted state.
//
// For each particle I and basis column t it needs
//   W1_(Ia)t = sum_K Z_IK Phi_(Ka)t,  W2_(Ia)t = sum_K Z_IK Phi_(Ka)t / rho_K,
//   c_I = sum_K Z_IK / rho_K,
// and writes U1 = Phi - W1 / rho_I and U2 = c Phi - W2, so that
//   X^B1 = -(1/h^2) Phi^T U1,  X^B2 = -(1/h^2) Phi^T U2
// (the row sum of Z is rho_I).
//
// All three are one dense contraction W = Z B of the N x N kernel matrix
// with the N x (2 s r + 1) matrix B = [Phi, Phi / rho, 1 / rho] (one row per
// particle K): the shape of attention's P V.  Z never exists in memory: per
// CTA of 128 particles I and per chunk of 32 particles K the CUDA cores form
// Z_IK = exp2(-|q^_I - q^_K|^2) (2D FP32 ops and one ex2 per pair), split it
// into two TF32 parts and store them in shared memory in the tensor cores'
// K-major layout; one thread then issues tcgen05.mma of kind::tf32 against
// the matching 32-row slice of B (pre-split into TF32 parts in global memory,
// staged by cp.async).  TF32 with one refinement step: every product is
// Z_hi B_hi + Z_hi B_lo + Z_lo B_hi (relative error about 2^-21).  The
// accumulator (FP32, tensor memory) covers 512 particles K; after each such
// segment it is added into FP32 registers (two-level summation, as in the
// CUDA-core pair passes), so no FP32 sum runs over more than 512 terms.
// Basis columns beyond 256 accumulator columns are split across grid.y.
#include <math.h>

#include "pair.cuh"
#include "pod_internal.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int RC_M = 128;    // particles I per CTA (MMA M, tensor-memory lanes)
constexpr int RC_KC = 32;    // particles K per chunk (MMA K = 4 x 8)
constexpr int RC_NT = 256;   // threads: 4 x 4 blocks of Z per chunk; two per TMEM lane in the flush
constexpr int RC_SEG = 16;   // chunks per FP32 accumulator segment (512 K)
constexpr int RC_ZOP = RC_M * RC_KC * 4;  // bytes of one Z operand tile (16 KB)

// Shared memory: two Z slots (hi and lo tiles each), a 2-stage ring of B
// slices (hi, lo) and a 3-stage ring of record tiles; the epilogue reuses it
// for the per-particle totals.
template <int D, int NCP>
struct RcLayout {
  static constexpr int DP = Rec<D>::DP;
  static constexpr int BOP = NCP * RC_KC * 4;          // one B operand tile
  static constexpr int REC = ((RC_KC * DP * 4 + 127) / 128) * 128;
  static constexpr int ZOFF = 0;                       // slot z: + z * 2 ZOP (hi), + ZOP (lo)
  static constexpr int BOFF = 4 * RC_ZOP;              // stage b: + b * 2 BOP (hi), + BOP (lo)
  static constexpr int ROFF = BOFF + 4 * BOP;          // stage k: + k * REC
  static constexpr int TOT_LD = NCP + 1;               // epilogue row stride (floats)
  static constexpr size_t RING = (size_t)ROFF + 3 * REC;
  static constexpr size_t SMEM = RING > (size_t)RC_M * TOT_LD * 4 ? RING : (size_t)RC_M * TOT_LD * 4;
  // resident CTAs per SM (two need <= 128 registers: 4 rows of D <= 12 coordinates)
  static constexpr int OCC = (SMEM <= 110 * 1024 && D <= 12) ? 2 : 1;
};

// Column layout of B for column chunk cb (rc basis columns t0 .. t0+rc-1,
// t0 = cb rr):
//   c = a rc + u          -> Phi_(K a)(t0+u)
//   c = s rc + a rc + u   -> Phi_(K a)(t0+u) / rho_K
//   c = 2 s rc            -> 1 / rho_K
// zero elsewhere and for K >= N.  Stored transposed (row c, K contiguous) as
// TF32 hi and lo parts: bt[(cb * NCP + c) * Npad + K].
__global__ void k_rc_bt(const float *__restrict__ phi, int ld, int r, int s, int rr, const float *__restrict__ rec,
                        int DP, int D, int N, int Npad, int NCP, float *__restrict__ bt_hi,
                        float *__restrict__ bt_lo) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y, cb = blockIdx.z;
  if (K >= Npad) return;
  const int t0 = cb * rr;
  const int rc = min(rr, r - t0);
  float v = 0.f;
  if (K < N) {
    const float w = rec[(size_t)K * DP + D];
    if (c < 2 * s * rc) {
      const int cc = c < s * rc ? c : c - s * rc;
      const int a = cc / rc, u = cc - a * rc;
      v = phi[((size_t)K * s + a) * ld + t0 + u];
      if (c >= s * rc) v *= w;
    } else if (c == 2 * s * rc) {
      v = w;
    }
  }
  const float h = to_tf32(v);
  const size_t o = ((size_t)cb * NCP + c) * Npad + K;
  bt_hi[o] = h;
  bt_lo[o] = to_tf32(v - h);
}

// 16-byte cp.async staging of the record tile of chunk K0..K0+31, and of the
// B^T slice (NCP rows x 32 K, hi and lo) in the tensor cores' K-major layout:
// element (row c, k) at (c/8)*1024 + (k/4)*128 + (c%8)*16 + (k%4)*4.
template <int DP>
__device__ __forceinline__ void rc_load_rec(uint32_t dst, const float *__restrict__ rec, int K0) {
  for (int idx = threadIdx.x; idx < RC_KC * DP / 4; idx += RC_NT)
    cp_async16(dst + idx * 16, rec + (size_t)K0 * DP + idx * 4, true);
}
template <int NCP>
__device__ __forceinline__ void rc_load_b(uint32_t dst, const float *__restrict__ bh, const float *__restrict__ bl,
                                          int Npad, int K0) {
  constexpr int BOP = NCP * RC_KC * 4;
  for (int idx = threadIdx.x; idx < NCP * 8; idx += RC_NT) {
    const int r8 = idx & 7, kc = (idx >> 3) & 7, g = idx >> 6;
    const int row = g * 8 + r8;
    const uint32_t off = g * 1024 + kc * 128 + r8 * 16;
    const size_t src = (size_t)row * Npad + K0 + 4 * kc;
    cp_async16(dst + off, bh + src, true);
    cp_async16(dst + BOP + off, bl + src, true);
  }
}

// Per chunk ch: wait for the MMAs of chunk ch-1 (their B stage is refilled
// next), stage B(ch+1) and the records of ch+2, form Z(ch) in Z slot ch % 2
// while the tensor cores may still run nothing of this CTA (the other
// resident CTA fills the gap), then one thread issues the 12 MMAs of ch.
template <int D, int NCP>
__global__ void __launch_bounds__(RC_NT, RcLayout<D, NCP>::OCC)
    k_refresh_tc(const float *__restrict__ rec, int N, int Npad, const float *__restrict__ bt_hi,
                 const float *__restrict__ bt_lo, const float *__restrict__ phi, int ld, int r, int s, int rr,
                 float *__restrict__ U1, float *__restrict__ U2, int *err) {
  using L = RcLayout<D, NCP>;
  constexpr int DP = L::DP;
  constexpr int HALF = NCP / 2;  // accumulator columns per thread
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int il = (warp & 3) * 32 + lane;  // row of the tile = tensor-memory lane
  const int kh = warp >> 2;               // which 16 K of a chunk, and which column half
  const int i0 = blockIdx.x * RC_M;
  const int cb = blockIdx.y;
  const float *bh = bt_hi + (size_t)cb * NCP * Npad, *bl = bt_lo + (size_t)cb * NCP * Npad;
  const int nch = Npad / RC_KC;
  if (warp == 0) tc_alloc(&s_tmem, NCP);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc(TC_FMT_TF32, RC_M, NCP);
  const uint32_t sbase = smem_u32(sm);
  // Z is formed in 4 x 4 blocks: rows rg + 32 m (m < 4) and the 4 K of
  // k-group jg of the chunk, so each staged record is read once per 4 pairs
  const int rg = tid & 31, jg = tid >> 5;
  float xi[4][D];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int i = min(i0 + rg + 32 * m, Npad - 1);
#pragma unroll
    for (int d = 0; d < D; ++d) xi[m][d] = rec[(size_t)i * DP + d];
  }
  float tot[HALF];
#pragma unroll
  for (int j = 0; j < HALF; ++j) tot[j] = 0.f;

  // prologue: records of chunks 0 and 1, B of chunk 0
  rc_load_rec<DP>(sbase + L::ROFF, rec, 0);
  if (nch > 1) rc_load_rec<DP>(sbase + L::ROFF + L::REC, rec, RC_KC);
  rc_load_b<NCP>(sbase + L::BOFF, bh, bl, Npad, 0);
  cp_async_commit();
  bool ok = true;
  int last = -1;
  for (int ch = 0; ch < nch; ++ch) {
    if (ch >= 1) {
      const int pc = ch - 1;
      const bool got = mbar_wait_bounded(&bars[pc & 1], (uint32_t)((pc >> 1) & 1), VDS_WAIT_LIMIT_NS);
      if (__syncthreads_or(!got)) {
        ok = false;
        break;
      }
    }
    if (ch + 1 < nch) rc_load_b<NCP>(sbase + L::BOFF + ((ch + 1) & 1) * 2 * L::BOP, bh, bl, Npad, (ch + 1) * RC_KC);
    if (ch + 2 < nch) rc_load_rec<DP>(sbase + L::ROFF + ((ch + 2) % 3) * L::REC, rec, (ch + 2) * RC_KC);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    // Z block of this thread as TF32 hi / lo; element (row i, k) of a Z tile
    // at (i/8)*1024 + (k/4)*128 + (i%8)*16 + (k%4)*4, so a row's 4 K of one
    // k-group are one float4
    uint8_t *zslot = sm + L::ZOFF + (ch & 1) * 2 * RC_ZOP;
    {
      const float *rs = reinterpret_cast<const float *>(sm + L::ROFF + (ch % 3) * L::REC) + jg * 4 * DP;
      float z[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float xj[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xj[d] = rs[u * DP + d];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          float r2 = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float dd = xi[m][d] - xj[d];
            r2 = fmaf(dd, dd, r2);
          }
          z[m][u] = ex2_approx(-r2);
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int row = rg + 32 * m;
        const size_t off = (size_t)(row >> 3) * 1024 + (row & 7) * 16 + jg * 128;
        float4 h, l;
        h.x = to_tf32(z[m][0]);
        h.y = to_tf32(z[m][1]);
        h.z = to_tf32(z[m][2]);
        h.w = to_tf32(z[m][3]);
        l.x = to_tf32(z[m][0] - h.x);
        l.y = to_tf32(z[m][1] - h.y);
        l.z = to_tf32(z[m][2] - h.z);
        l.w = to_tf32(z[m][3] - h.w);
        *reinterpret_cast<float4 *>(zslot + off) = h;
        *reinterpret_cast<float4 *>(zslot + RC_ZOP + off) = l;
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t zh = sbase + L::ZOFF + (ch & 1) * 2 * RC_ZOP, zl = zh + RC_ZOP;
      const uint32_t b_hi = sbase + L::BOFF + (ch & 1) * 2 * L::BOP, b_lo = b_hi + L::BOP;
#pragma unroll
      for (int k = 0; k < RC_KC / 8; ++k) {
        const uint32_t o = (uint32_t)k * 256u;
        const int first = (ch % RC_SEG == 0 && k == 0) ? 0 : 1;
        tc_mma_tf32(tmem, tc_sdesc(zl + o), tc_sdesc(b_hi + o), idesc, first);
        tc_mma_tf32(tmem, tc_sdesc(zh + o), tc_sdesc(b_lo + o), idesc, 1);
        tc_mma_tf32(tmem, tc_sdesc(zh + o), tc_sdesc(b_hi + o), idesc, 1);
      }
      tc_commit(&bars[ch & 1]);
    }
    last = ch;
    if (ch % RC_SEG == RC_SEG - 1 || ch == nch - 1) {
      const bool got = mbar_wait_bounded(&bars[ch & 1], (uint32_t)((ch >> 1) & 1), VDS_WAIT_LIMIT_NS);
      if (__syncthreads_or(!got)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < HALF; c0 += 16) {
        uint32_t v[16];
        tc_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(kh * HALF + c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[c0 + j] += __uint_as_float(v[j]);
      }
      tc_fence_before();
    }
  }
  cp_async_wait<0>();
  if (!ok) {
    if (tid == 0 && last >= 0)
      mbar_wait_bounded(&bars[last & 1], (uint32_t)((last >> 1) & 1), VDS_WAIT_LIMIT_NS / 8);
    if (tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, NCP);
  if (!ok) return;
  // epilogue: totals through shared memory, then U1, U2 per (I, a, t)
  float *T = reinterpret_cast<float *>(sm);
#pragma unroll
  for (int j = 0; j < HALF; ++j) T[il * L::TOT_LD + kh * HALF + j] = tot[j];
  __syncthreads();
  const int t0 = cb * rr;
  const int rc = min(rr, r - t0);
  const int per = s * rc;
  for (int e = tid; e < RC_M * per; e += RC_NT) {
    const int row = e / per, rem = e - row * per;
    const int a = rem / rc, u = rem - a * rc;
    const int I = i0 + row;
    if (I >= N) continue;
    const float *Tr = T + row * L::TOT_LD;
    const float wI = rec[(size_t)I * DP + D];
    const size_t o = ((size_t)I * s + a) * ld + t0 + u;
    const float f = phi[o];
    U1[o] = f - Tr[a * rc + u] * wI;
    U2[o] = Tr[2 * per] * f - Tr[per + a * rc + u];
  }
}

template <int D, int NCP>
int refresh_launch(vds_ctx *c, const pod_basis *b, int N, int Npad, int rr, int ncb, const float *bh,
                   const float *bl, float *U1, float *U2) {
  using L = RcLayout<D, NCP>;
  VDS_CUDA_TRY(cudaFuncSetAttribute(k_refresh_tc<D, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)L::SMEM));
  dim3 grid((N + RC_M - 1) / RC_M, ncb);
  k_refresh_tc<D, NCP><<<grid, RC_NT, L::SMEM, c->stream>>>((const float *)c->rec.ptr, N, Npad, bh, bl, b->phi,
                                                             b->ld, b->r, b->s, rr, U1, U2, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

template <int D>
int refresh_impl(vds_ctx *c, const pod_basis *b, int N, float *U1, float *U2) {
  const int s = b->s, r = b->r;
  // basis columns per column chunk: 2 s rr + 1 accumulator columns <= 256
  const int rr_max = (256 - 1) / (2 * s);
  const int ncb = (r + rr_max - 1) / rr_max;
  const int rr = (r + ncb - 1) / ncb;
  const int need = 2 * s * rr + 1;
  const int NCP = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : 256;
  // record rows as written by pass_prep (a multiple of 256 >= RC_KC)
  const int Npad = pass_npad(N);
  const size_t nbt = (size_t)ncb * NCP * Npad;
  VDS_TRY(vds_ensure(c, c->gbuf, 2 * nbt * sizeof(float)));
  float *bh = (float *)c->gbuf.ptr, *bl = bh + nbt;
  k_rc_bt<<<dim3((Npad + 255) / 256, NCP, ncb), 256, 0, c->stream>>>(b->phi, b->ld, r, s, rr,
                                                                     (const float *)c->rec.ptr, Rec<D>::DP, D,
                                                                     N, Npad, NCP, bh, bl);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  switch (NCP) {
    case 32: return refresh_launch<D, 32>(c, b, N, Npad, rr, ncb, bh, bl, U1, U2);
    case 64: return refresh_launch<D, 64>(c, b, N, Npad, rr, ncb, bh, bl, U1, U2);
    case 128: return refresh_launch<D, 128>(c, b, N, Npad, rr, ncb, bh, bl, U1, U2);
    default: return refresh_launch<D, 256>(c, b, N, Npad, rr, ncb, bh, bl, U1, U2);
  }
}

}  // namespace

int pod_refresh_dev(vds_ctx *c, const pod_basis *b, int N, int D, float *U1, float *U2) {
  VDS_TRY(vds_time_begin(c, PK_REFRESH));
  int st = VDS_EARG;
  switch (D) {
    case 2: st = refresh_impl<2>(c, b, N, U1, U2); break;
    case 3: st = refresh_impl<3>(c, b, N, U1, U2); break;
    case 4: st = refresh_impl<4>(c, b, N, U1, U2); break;
    case 6: st = refresh_impl<6>(c, b, N, U1, U2); break;
    case 8: st = refresh_impl<8>(c, b, N, U1, U2); break;
    case 9: st = refresh_impl<9>(c, b, N, U1, U2); break;
    case 10: st = refresh_impl<10>(c, b, N, U1, U2); break;
    case 12: st = refresh_impl<12>(c, b, N, U1, U2); break;
    case 14: st = refresh_impl<14>(c, b, N, U1, U2); break;
    case 15: st = refresh_impl<15>(c, b, N, U1, U2); break;
    case 16: st = refresh_impl<16>(c, b, N, U1, U2); break;
    default: break;
  }
  VDS_TRY(st);
  VDS_TRY(vds_time_end(c, PK_REFRESH));
  return VDS_OK;
}
