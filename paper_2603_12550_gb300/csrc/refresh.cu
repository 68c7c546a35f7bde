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
// particle K): the shape of attention's P V.  Z never exists in memory.  One
// CTA per 128 particles I (and per column chunk of B), warp-specialised:
//   warps 0-15  form Z_IK = exp2(-|q^_I - q^_K|^2) for chunks of 32
//               particles K on the CUDA cores (one ex2 per pair, two pairs
//               per f32x2 instruction) and put them where the tensor cores
//               read them;
//   warp 16     stages the records and B slices (hi and lo TF32 parts,
//               pre-arranged in global memory as the exact shared-memory
//               images) with 1-D bulk copies (TMA engine);
//   warp 17     issues tcgen05.mma of kind::tf32 (M = 128, K = 8) into an
//               FP32 accumulator in tensor memory.
// Two kernels share this plan.  k_refresh_ta (2 s r + 1 <= 64, the common
// case: r <= 10 at s = 3) keeps Z in tensor memory, one row per thread, as
// the MMAs' A operand, rounded to TF32 once against B_hi + B_lo; the wide
// kernel k_refresh_tc (up to 256 columns) keeps Z in shared memory in the
// tensor cores' K-major layout and forms Z_hi B_hi + Z_hi B_lo + Z_lo B_hi
// (TF32 with a refinement step on both operands, relative error about
// 2^-21).  mbarrier rings connect the roles; nothing waits on a CTA-wide
// barrier inside the loop.  The accumulator covers one segment of 512
// particles K and is double-buffered: warps 0-15 add a finished segment into
// FP32 registers while the tensor cores fill the other buffer (two-level
// summation, as in the CUDA-core pair passes: no FP32 sum runs over more
// than 512 terms).  Every wait is bounded; a wait that runs out raises the
// abort flag, every role leaves its loop, copies and MMAs in flight are
// waited for and the tensor memory is freed.
#include <cuda_fp16.h>
#include <math.h>

#include "pair.cuh"
#include "pod_internal.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int RC_M = 128;    // particles I per CTA (MMA M, tensor-memory lanes)
constexpr int RC_KC = 32;    // particles K per chunk (MMA K = 4 x 8)
constexpr int RC_PW = 16;    // Z-forming warps: 2 rows x 4 K blocks of Z per thread and chunk
constexpr int RC_PT = RC_PW * 32;
constexpr int RC_NT = RC_PT + 64;  // + one warp of bulk copies + one warp of MMA issue
constexpr int RC_SEG = 16;   // chunks per FP32 accumulator segment (512 K)
constexpr int RC_FLUSH = 7;  // chunk of the next segment at which a segment is flushed
constexpr int RC_ZOP = RC_M * RC_KC * 4;  // bytes of one Z operand tile (16 KB)
// k_refresh_ta works in FP16 (kind::f16, K = 16 per MMA) on chunks of 64
// particles K, eight to the same 512-particle segment; B is scaled by 2^12
// on its way to FP16 (|Phi| <= 1 and rho >= 1 put every entry of
// [Phi, Phi/rho, 1/rho] below 4096, and the small ones above FP16's smallest
// normal), the totals by 2^-12 on the way out (both exact)
constexpr int TA_KC = 64;
constexpr int TA_SEGC = 8;
constexpr float TA_BSCALE = 4096.f;

// Shared memory of the wide-B kernel (2 s r + 1 > 64): NZ slots of
// [Z hi | Z lo | B hi | B lo | records]; the epilogue reuses it for the
// per-particle totals.
template <int D, int NCP>
struct RcLayout {
  static constexpr int DP = Rec<D>::DP;
  static constexpr int BOP = NCP * RC_KC * 4;            // one B operand tile
  // records of one chunk as staged, every coordinate duplicated, so that a
  // 64-bit shared load is a ready f32x2 operand against a pair of rows
  static constexpr int REC_BYTES = RC_KC * DP * 4 * 2;
  static constexpr int REC = ((REC_BYTES + 127) / 128) * 128;
  static constexpr int ZB = 2 * RC_ZOP;                  // Z tiles of a slot
  static constexpr int BOFF = ZB;                        // B hi, then B lo
  static constexpr int ROFF = ZB + 2 * BOP;              // records
  static constexpr int SLOT = ((ZB + 2 * BOP + REC + 1023) / 1024) * 1024;
  static constexpr int NZ = (216 * 1024 / SLOT) < 4 ? (216 * 1024 / SLOT) : 4;
  static constexpr int TOT_LD = NCP + 1;                 // epilogue row stride (floats)
  static constexpr size_t RING = (size_t)NZ * SLOT;
  static constexpr size_t SMEM = RING > (size_t)RC_M * TOT_LD * 4 ? RING : (size_t)RC_M * TOT_LD * 4;
  static_assert(NZ >= 2, "refresh ring depth");
  static_assert(SMEM <= 227 * 1024 - 1024, "refresh shared memory");
};

// Column layout of B for column chunk cb (rc basis columns t0 .. t0+rc-1,
// t0 = cb rr):
//   c = a rc + u          -> Phi_(K a)(t0+u)
//   c = s rc + a rc + u   -> Phi_(K a)(t0+u) / rho_K
//   c = 2 s rc            -> 1 / rho_K
// zero elsewhere and for K >= N.  Stored as TF32 hi and lo parts, per
// (column chunk, 32-particle chunk of K) the shared-memory image of the
// tensor cores' K-major operand: element (c, k) at byte (c/8)*1024 +
// (k/4)*128 + (c%8)*16 + (k%4)*4 of the hi tile, the lo tile BOP bytes after
// it; image (cb, ch) at float offset ((cb * nch + ch) * 2 NCP RC_KC).
//
// recs receives the records again as the refresh stages them.  NCP <= 64
// (Z in tensor memory, one row per thread): interleaved by pairs of
// particles, particle k of a 32-particle chunk, pair p = k/2, half k%2,
// coordinate d at float (chunk * 32 + 2 p) * DP + 2 d + k%2, so that one
// 64-bit shared load gives coordinate d of both particles of a pair as the
// two halves of an f32x2 operand.  NCP > 64 (two rows per thread): every
// coordinate duplicated, particle K's coordinate d at floats
// 2 (K DP + d) and 2 (K DP + d) + 1, the operand against a pair of rows.
__global__ void k_rc_bt(const float *__restrict__ phi, int ld, int r, int s, int rr, const float *__restrict__ rec,
                        int DP, int D, int N, int Npad, int NCP, float *__restrict__ bimg, float *__restrict__ recs) {
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
  if (NCP <= 64) {
    // FP16, chunks of TA_KC particles: element (c, k) of the hi tile at byte
    // (c/8)*1024 + (k/8)*128 + (c%8)*16 + (k%8)*2, the lo tile NCP*128 bytes on
    const int nch = Npad / TA_KC, ch = K / TA_KC, k = K - ch * TA_KC;
    __half *img = reinterpret_cast<__half *>(bimg);
    const size_t tile = (size_t)NCP * TA_KC;  // halves per tile
    const size_t o = ((size_t)cb * nch + ch) * 2 * tile +
                     (size_t)(((c >> 3) * 1024 + (k >> 3) * 128 + (c & 7) * 16 + (k & 7) * 2) >> 1);
    const float vs = v * TA_BSCALE;
    const __half h = __float2half_rn(vs);
    img[o] = h;
    img[o + tile] = __float2half_rn(vs - __half2float(h));
  } else {
    const int nch = Npad / RC_KC, ch = K / RC_KC, k = K - ch * RC_KC;
    const size_t tile = (size_t)NCP * RC_KC;
    const size_t o = ((size_t)cb * nch + ch) * 2 * tile +
                     (size_t)(((c >> 3) * 1024 + (k >> 2) * 128 + (c & 7) * 16 + (k & 3) * 4) >> 2);
    const float h = to_tf32(v);
    bimg[o] = h;
    bimg[o + tile] = to_tf32(v - h);
  }
  const int ch = K / RC_KC, k = K - ch * RC_KC;
  if (c == 0 && cb == 0) {
    if (NCP <= 64) {
      // coordinates, then |q^_K|^2 in place of w (FP32, d ascending: the same
      // sequence of roundings as the row's own norm in k_refresh_ta)
      float *dst = recs + ((size_t)ch * RC_KC + (k & ~1)) * DP + (k & 1);
      float nrm = 0.f;
      for (int d = 0; d < D; ++d) {
        const float x = rec[(size_t)K * DP + d];
        dst[2 * d] = x;
        nrm = fmaf(x, x, nrm);
      }
      dst[2 * D] = nrm;
      for (int d = D + 1; d < DP; ++d) dst[2 * d] = rec[(size_t)K * DP + d];
    } else {
      float *dst = recs + (size_t)K * 2 * DP;
      for (int d = 0; d < DP; ++d) dst[2 * d] = dst[2 * d + 1] = rec[(size_t)K * DP + d];
    }
  }
}

// Packed pairs of FP32 values (f32x2 instructions: one issue slot for two
// lanes' worth of FP32 work, each half rounded as the scalar instruction).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// One probe of an mbarrier phase that may suspend the thread (up to 20 us)
// until the phase completes, so that waiting roles do not take issue slots
// from the warps sharing their scheduler.
__device__ __forceinline__ bool rc_try_wait_sleep(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
// Wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool rc_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    if (rc_try_wait_sleep(bar, parity)) return true;
    if (*abort) return false;
    if (global_timer_ns() - t0 > VDS_WAIT_LIMIT_NS) {
      *abort = 1;
      return false;
    }
  }
}

// Epilogue of a refresh CTA: the Z-forming threads' totals (row 32 (warp %
// 4) + lane, column quarter warp / 4) through shared memory, then U1, U2 per
// (I, a, t), or this K split's totals into part (summed over the splits by
// k_rc_fin).
template <int D, int NCP, int QC>
__device__ __forceinline__ void rc_epilogue(uint8_t *sm, int tot_ld, const float (&tot)[QC], int tid, int warp,
                                            int lane, int i0, int cb, int N, const float *__restrict__ rec,
                                            const float *__restrict__ phi, int ld, int r, int s, int rr,
                                            float *__restrict__ U1, float *__restrict__ U2,
                                            float *__restrict__ part, float scale) {
  constexpr int DP = Rec<D>::DP;
  float *T = reinterpret_cast<float *>(sm);
  if (tid < RC_PT) {
    const int il = (warp & 3) * 32 + lane, cq = warp >> 2;
#pragma unroll
    for (int j = 0; j < QC; ++j) T[il * tot_ld + cq * QC + j] = tot[j] * scale;
  }
  __syncthreads();
  if (part) {
    float *dst = part + (((size_t)cb * gridDim.x + blockIdx.x) * RC_M) * NCP;
    for (int e = tid; e < RC_M * NCP; e += RC_NT) dst[e] = T[(e / NCP) * tot_ld + e % NCP];
    return;
  }
  const int t0 = cb * rr;
  const int rc = min(rr, r - t0);
  const int per = s * rc;
  for (int e = tid; e < RC_M * per; e += RC_NT) {
    const int row = e / per, rem = e - row * per;
    const int a = rem / rc, u = rem - a * rc;
    const int I = i0 + row;
    if (I >= N) continue;
    const float *Tr = T + row * tot_ld;
    const float wI = rec[(size_t)I * DP + D];
    const size_t o = ((size_t)I * s + a) * ld + t0 + u;
    const float f = phi[o];
    U1[o] = f - Tr[a * rc + u] * wI;
    U2[o] = Tr[2 * per] * f - Tr[per + a * rc + u];
  }
}

// Synchronisation per ring slot z (chunk ch uses slot ch % NZ; counts are
// completions, u = ch / NZ):
//   full[z]   bulk-copy bytes of records + B of chunk ch (completion u);
//   zready[z] RC_PT arrivals: Z of chunk ch stored (completion u);
//   sfree[z]  tcgen05.commit after the MMAs of chunk ch (completion u).
// Per accumulator buffer b (segment g uses b = g & 1, v = g >> 1):
//   segdone[b] commit after the last MMA of segment g (completion v);
//   accfree[b] RC_PT arrivals: segment g added into registers (completion v).
template <int D, int NCP>
__global__ void __launch_bounds__(RC_NT, 1)
    k_refresh_tc(const float *__restrict__ rec, const float *__restrict__ recs, int N, int Npad,
                 const float *__restrict__ bimg,
                 const float *__restrict__ phi, int ld, int r, int s, int rr, float *__restrict__ U1,
                 float *__restrict__ U2, int nsplit, float *__restrict__ part, int *err) {
  using L = RcLayout<D, NCP>;
  constexpr int DP = L::DP;
  constexpr int NZ = L::NZ;
  constexpr int QC = NCP / 4;  // accumulator columns per thread in a flush
  // NCP <= 128: one MMA takes Z_hi against [B_hi; B_lo] (N = 2 NCP), so Z_hi
  // is read from shared memory once per K step; the two halves of the
  // accumulator are added at the flush.  NCP = 256: three MMAs of N = NCP.
  constexpr bool FB = NCP <= 128;
  constexpr int ACW = FB ? 2 * NCP : NCP;  // accumulator columns per buffer
  static_assert(NCP >= 128, "narrower B slices run k_refresh_ta");
  constexpr int TCOLS = 2 * ACW;
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t full[NZ], zready[NZ], sfree[NZ], segdone[2], accfree[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // CTA = (row tile, split of the K range into whole segments, column chunk)
  const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
  const int i0 = tile * RC_M;
  const int cb = blockIdx.y;
  const int nch_all = Npad / RC_KC, nseg_all = (nch_all + RC_SEG - 1) / RC_SEG;
  const int sg0 = split * nseg_all / nsplit, sg1 = (split + 1) * nseg_all / nsplit;
  const int c0 = sg0 * RC_SEG;                                  // first chunk of this CTA
  const int nch = min(sg1 * RC_SEG, nch_all) - c0;              // chunks of this CTA (local index ch)
  const int nseg = sg1 - sg0;
  volatile int *abort = &s_abort;
  if (warp == 0) tc_alloc(&s_tmem, TCOLS);
  if (tid == 0) {
    for (int z = 0; z < NZ; ++z) {
      mbar_init(&full[z], 1);
      mbar_init(&zready[z], RC_PT);
      mbar_init(&sfree[z], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&segdone[b], 1);
      mbar_init(&accfree[b], RC_PT);
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_u32(sm);
  float tot[QC];
  bool ok = true;

  if (warp == RC_PW) {
    // ---------------------------------------------------- bulk copies
    if (lane == 0) {
      const float *bsrc = bimg + ((size_t)cb * nch_all + c0) * 2 * NCP * RC_KC;
      int ch = 0;
      for (; ch < nch; ++ch) {
        const int z = ch % NZ;
        if (ch >= NZ && !rc_wait(&sfree[z], (uint32_t)((ch / NZ - 1) & 1), abort)) {
          ok = false;
          break;
        }
        uint8_t *slot = sm + (size_t)z * L::SLOT;
        mbar_arrive_expect_tx(&full[z], (uint32_t)(L::REC_BYTES + 2 * L::BOP));
        // the records as staged for the producers' f32x2 operands (k_rc_bt)
        bulk_g2s(slot + L::ROFF, reinterpret_cast<const uint8_t *>(recs) + (size_t)(c0 + ch) * L::REC_BYTES,
                 L::REC_BYTES, &full[z]);
        bulk_g2s(slot + L::BOFF, bsrc + (size_t)ch * 2 * NCP * RC_KC, 2 * L::BOP, &full[z]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // the copies still in flight land before the CTA may exit
      for (int k = ch > NZ ? ch - NZ : 0; k < ch; ++k)
        mbar_wait_bounded(&full[k % NZ], (uint32_t)((k / NZ) & 1), VDS_WAIT_LIMIT_NS);
    }
  } else if (warp == RC_PW + 1) {
    // ---------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc = tc_idesc(TC_FMT_TF32, RC_M, NCP), idesc2 = tc_idesc(TC_FMT_TF32, RC_M, ACW);
      for (int ch = 0; ch < nch && ok; ++ch) {
        const int z = ch % NZ, g = ch / RC_SEG, b = g & 1;
        if (ch % RC_SEG == 0 && g >= 2 && !rc_wait(&accfree[b], (uint32_t)(((g >> 1) - 1) & 1), abort)) {
          ok = false;
          break;
        }
        if (!rc_wait(&zready[z], (uint32_t)((ch / NZ) & 1), abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t zh = sbase + (uint32_t)(z * L::SLOT), zl = zh + RC_ZOP;
        const uint32_t b_hi = zh + L::BOFF, b_lo = b_hi + L::BOP;
        const uint32_t acc = tmem + (uint32_t)(b * ACW);
#pragma unroll
        for (int k = 0; k < RC_KC / 8; ++k) {
          const uint32_t o = (uint32_t)k * 256u;
          const int first = (ch % RC_SEG == 0 && k == 0) ? 0 : 1;
          if constexpr (FB) {
            // B_lo's rows follow B_hi's at the next 8-row group: one operand of 2 NCP rows
            tc_mma_tf32(acc, tc_sdesc(zh + o), tc_sdesc(b_hi + o), idesc2, first);
            tc_mma_tf32(acc, tc_sdesc(zl + o), tc_sdesc(b_hi + o), idesc, 1);
          } else {
            tc_mma_tf32(acc, tc_sdesc(zl + o), tc_sdesc(b_hi + o), idesc, first);
            tc_mma_tf32(acc, tc_sdesc(zh + o), tc_sdesc(b_lo + o), idesc, 1);
            tc_mma_tf32(acc, tc_sdesc(zh + o), tc_sdesc(b_hi + o), idesc, 1);
          }
        }
        tc_commit(&sfree[z]);
        if (ch % RC_SEG == RC_SEG - 1 || ch == nch - 1) tc_commit(&segdone[b]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
    }
  } else {
    // ---------------------------------------------------- Z formation
    // rows rg + 32 (2 mh + m) (m < 2) and the 4 K of k-group jg of each
    // chunk; element (row i, k) of a shared-memory Z tile at (i/8)*1024 +
    // (k/4)*128 + (i%8)*16 + (k%4)*4, so a row's 4 K of one k-group are one
    // float4
    constexpr int RPT = 2;  // rows per thread
    const int rg = lane, jg = warp & 7, mh = warp >> 3;
    const int q4 = warp & 3, cq = warp >> 2;  // flush: TMEM lanes 32 q4 .., column quarter cq
    float xi[RPT][D];
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int i = min(i0 + rg + 32 * (2 * mh + m), Npad - 1);
#pragma unroll
      for (int d = 0; d < D; ++d) xi[m][d] = rec[(size_t)i * DP + d];
    }
#pragma unroll
    for (int j = 0; j < QC; ++j) tot[j] = 0.f;
    // the two rows of the thread side by side
    unsigned long long xi2r[D];
#pragma unroll
    for (int d = 0; d < D; ++d) xi2r[d] = f2_pack(xi[0][d], xi[RPT - 1][d]);
    auto flush = [&](int g) -> bool {
      const int b = g & 1;
      if (!__all_sync(0xffffffffu, rc_wait(&segdone[b], (uint32_t)((g >> 1) & 1), abort))) return false;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * ACW + cq * QC);
#pragma unroll
      for (int c0 = 0; c0 < QC; c0 += 16) {
        uint32_t v[16];
        tc_ld16(ta + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[c0 + j] += __uint_as_float(v[j]);
        if constexpr (FB) {
          tc_ld16(ta + (uint32_t)(NCP + c0), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) tot[c0 + j] += __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
      mbar_arrive(&accfree[b]);
      return true;
    };
    int flushed = 0;  // segments added into registers
    {
      for (int ch = 0; ch < nch && ok; ++ch) {
        const int z = ch % NZ;
        if (!__all_sync(0xffffffffu, rc_wait(&full[z], (uint32_t)((ch / NZ) & 1), abort))) {
          ok = false;
          break;
        }
        uint8_t *slot = sm + (size_t)z * L::SLOT;
        // the thread's two rows in the halves of one f32x2 operand against
        // the duplicated coordinates of each record
        const unsigned long long *rs =
            reinterpret_cast<const unsigned long long *>(slot + L::ROFF) + jg * 4 * DP;
        float zz[2][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          unsigned long long r2 = f2_pack(0.f, 0.f);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const unsigned long long dd = f2_sub(xi2r[d], rs[u * DP + d]);
            r2 = f2_fma(dd, dd, r2);
          }
          float r2a, r2b;
          f2_unpack(r2, r2a, r2b);
          zz[0][u] = ex2_approx(-r2a);
          zz[1][u] = ex2_approx(-r2b);
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const int row = rg + 32 * (2 * mh + m);
          const size_t off = (size_t)(row >> 3) * 1024 + (row & 7) * 16 + jg * 128;
          float4 h, l;
          h.x = to_tf32(zz[m][0]);
          h.y = to_tf32(zz[m][1]);
          h.z = to_tf32(zz[m][2]);
          h.w = to_tf32(zz[m][3]);
          // low parts unrounded, as on the tensor-memory path
          l.x = zz[m][0] - h.x;
          l.y = zz[m][1] - h.y;
          l.z = zz[m][2] - h.z;
          l.w = zz[m][3] - h.w;
          *reinterpret_cast<float4 *>(slot + off) = h;
          *reinterpret_cast<float4 *>(slot + RC_ZOP + off) = l;
        }
        fence_proxy_async_smem();
        mbar_arrive(&zready[z]);
        // segment g - 1 is added into registers part-way through segment g
        if (ch % RC_SEG == RC_FLUSH && ch / RC_SEG >= 1) {
          if (!flush(ch / RC_SEG - 1)) {
            ok = false;
            break;
          }
          ++flushed;
        }
      }
    }
    for (; ok && flushed < nseg; ++flushed)
      if (!flush(flushed)) ok = false;
    if (!ok && tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  // every role has left its loop; the MMAs issued are complete before the
  // tensor memory and shared memory are released
  tc_fence_before();
  __syncthreads();
  if (warp == 9 && lane == 0) {
    tc_commit(&fin);
    mbar_wait_bounded(&fin, 0, VDS_WAIT_LIMIT_NS);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, TCOLS);
  if (*abort) return;
  rc_epilogue<D, NCP, QC>(sm, L::TOT_LD, tot, tid, warp, lane, i0, cb, N, rec, phi, ld, r, s, rr, U1, U2, part,
                          1.f);
}

// ------------------------------------------------ Z in tensor memory (NCP <= 64)
//
// The same contraction with Z in tensor memory, in FP16 (kind::f16, K = 16
// per MMA: half the accumulator updates of K = 8 TF32 steps at the same
// 11-bit significand), and the staging decoupled from it: shared memory
// holds NS2 pair slots, each the B images of two consecutive 64-particle
// chunks (one 32 KB bulk copy at NCP = 64) and their 128 records (one copy),
// each with its own mbarrier, so the Z-forming warps wait only for the
// records and the tensor cores only for B; tensor memory holds four pair
// slots of Z (8 chunks, two halves per column).  The copies run up to NS2
// pairs of chunks ahead of the tensor cores, the Z-forming warps up to four.
//
// Precision: Z is rounded to FP16 once (relative error at most 2^-11 per
// kernel value, unbiased; below FP16's smallest normal an absolute error of
// at most 2^-25) and B carries the refinement step (B_hi + B_lo, each FP16,
// of B scaled by 2^12), so one MMA of N = 2 NCP per K step forms
// Z (B_hi + B_lo).  Z's own low part (the third product of the wide kernel)
// is left out: with it the tensor cores' accumulator updates, not the kernel
// values, set the pace; without it X^B moved by at most 1e-6 relative against
// the FP64 oracle's, far inside the 1e-4 the tests demand.  The squared
// distance of a pair is expanded, |x - y|^2 = |x|^2 + |y|^2 - 2 x.y: D + 2
// FP32 operations instead of 2D + 1 (k_rc_bt stores each staged record's
// norm; the row's own is rounded the same way, so coincident points give
// exactly 0).
//
// Barriers (pass c2 = chunks 2 c2 and 2 c2 + 1; pair slot j = c2 % NS2,
// completion u = c2 / NS2; Z pair zp = c2 % NZP, completion c2 / NZP):
//   rfull[j]  bulk-copy bytes of the pass's records;
//   bfull[j]  bulk-copy bytes of the pass's B images;
//   sfree[j]  tcgen05.commit after the pass's MMAs (slot j may be refilled);
//   zready[zp] one arrival per Z-forming warp: Z of the pass stored;
//   zfree[zp]  tcgen05.commit after the pass's MMAs (Z pair may be rewritten);
//   segdone[b], accfree[b] as in k_refresh_tc (accfree: one per warp).
template <int D, int NCP>
struct TaLayout {
  static constexpr int DP = Rec<D>::DP;
  static constexpr int BOP = NCP * TA_KC * 2;        // one FP16 B operand tile
  static constexpr int BCH = 2 * BOP;                // B hi + lo of one chunk
  static constexpr int REC_BYTES = TA_KC * DP * 4;   // one chunk's records
  static constexpr int ROFF = 2 * BCH;               // records of the pair
  static constexpr int SLOT = ((2 * BCH + 2 * REC_BYTES + 1023) / 1024) * 1024;
  static constexpr int NS2 = (200 * 1024 / SLOT) < 8 ? (200 * 1024 / SLOT) : 8;
  static constexpr int TOT_LD = NCP + 1;
  static constexpr size_t RING = (size_t)NS2 * SLOT;
  static constexpr size_t SMEM = RING > (size_t)RC_M * TOT_LD * 4 ? RING : (size_t)RC_M * TOT_LD * 4;
  static_assert(NCP <= 64, "Z in tensor memory needs 2 s r + 1 <= 64");
  static_assert(NS2 >= 2, "refresh ring depth");
  static_assert(SMEM <= 227 * 1024 - 1024, "refresh shared memory");
};

template <int D, int NCP>
__global__ void __launch_bounds__(RC_NT, 1)
    k_refresh_ta(const float *__restrict__ rec, const float *__restrict__ recs, int N, int Npad,
                 const float *__restrict__ bimg,
                 const float *__restrict__ phi, int ld, int r, int s, int rr, float *__restrict__ U1,
                 float *__restrict__ U2, int nsplit, float *__restrict__ part, int *err) {
  using L = TaLayout<D, NCP>;
  constexpr int DP = L::DP;
  constexpr int NS2 = L::NS2;
  constexpr int QC = NCP / 4;           // accumulator columns per thread in a flush
  constexpr int ACW = 2 * NCP;          // Z against [B_hi; B_lo]: N = 2 NCP
  constexpr int NZP = 4;                // Z pair slots: 2 chunks x 32 columns each
  constexpr int TCOLS = 512;            // 2 ACW accumulator columns + NZP x 64 Z columns
  static_assert(2 * ACW + NZP * 64 <= TCOLS, "tensor memory columns");
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t rfull[NS2], bfull[NS2], sfree[NS2], zready[NZP], zfree[NZP], segdone[2],
      accfree[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
  const int i0 = tile * RC_M;
  const int cb = blockIdx.y;
  const int nch_all = Npad / TA_KC, nseg_all = (nch_all + TA_SEGC - 1) / TA_SEGC;
  const int sg0 = split * nseg_all / nsplit, sg1 = (split + 1) * nseg_all / nsplit;
  const int c0 = sg0 * TA_SEGC;                      // first chunk of this CTA
  const int nch = min(sg1 * TA_SEGC, nch_all) - c0;  // a multiple of 4: Npad is of 256
  const int npass = nch / 2;
  const int nseg = sg1 - sg0;
  volatile int *abort = &s_abort;
  if (warp == 0) tc_alloc(&s_tmem, TCOLS);
  if (tid == 0) {
    for (int j = 0; j < NS2; ++j) {
      mbar_init(&rfull[j], 1);
      mbar_init(&bfull[j], 1);
      mbar_init(&sfree[j], 1);
    }
    for (int b = 0; b < NZP; ++b) {
      mbar_init(&zready[b], RC_PW);
      mbar_init(&zfree[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&segdone[b], 1);
      mbar_init(&accfree[b], RC_PW);
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_u32(sm);
  float tot[QC];
  bool ok = true;

  if (warp == RC_PW) {
    // ---------------------------------------------------- bulk copies
    if (lane == 0) {
      const uint8_t *bsrc = reinterpret_cast<const uint8_t *>(bimg) + ((size_t)cb * nch_all + c0) * L::BCH;
      const uint8_t *rsrc = reinterpret_cast<const uint8_t *>(recs) + (size_t)c0 * L::REC_BYTES;
      int c2 = 0;
      for (; c2 < npass; ++c2) {
        const int j = c2 % NS2;
        if (c2 >= NS2 && !rc_wait(&sfree[j], (uint32_t)((c2 / NS2 - 1) & 1), abort)) {
          ok = false;
          break;
        }
        uint8_t *slot = sm + (size_t)j * L::SLOT;
        // records first: the Z-forming warps wait for them only
        mbar_arrive_expect_tx(&rfull[j], (uint32_t)(2 * L::REC_BYTES));
        bulk_g2s(slot + L::ROFF, rsrc + (size_t)(2 * c2) * L::REC_BYTES, 2 * L::REC_BYTES, &rfull[j]);
        mbar_arrive_expect_tx(&bfull[j], (uint32_t)(2 * L::BCH));
        bulk_g2s(slot, bsrc + (size_t)(2 * c2) * L::BCH, 2 * L::BCH, &bfull[j]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // the copies still in flight land before the CTA may exit
      for (int k = c2 > NS2 ? c2 - NS2 : 0; k < c2; ++k) {
        mbar_wait_bounded(&rfull[k % NS2], (uint32_t)((k / NS2) & 1), VDS_WAIT_LIMIT_NS);
        mbar_wait_bounded(&bfull[k % NS2], (uint32_t)((k / NS2) & 1), VDS_WAIT_LIMIT_NS);
      }
    }
  } else if (warp == RC_PW + 1) {
    // ---------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc2 = tc_idesc(TC_FMT_F16, RC_M, ACW);
      for (int c2 = 0; c2 < npass && ok; ++c2) {
        const int j = c2 % NS2, zp = c2 % NZP;
        if (!rc_wait(&zready[zp], (uint32_t)((c2 / NZP) & 1), abort) ||
            !rc_wait(&bfull[j], (uint32_t)((c2 / NS2) & 1), abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int e = 0; e < 2 && ok; ++e) {
          const int ch = 2 * c2 + e, g = ch / TA_SEGC, b = g & 1;
          if (ch % TA_SEGC == 0 && g >= 2 && !rc_wait(&accfree[b], (uint32_t)(((g >> 1) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          const uint32_t b_hi = sbase + (uint32_t)(j * L::SLOT + e * L::BCH);
          const uint32_t zt = tmem + (uint32_t)(2 * ACW + 64 * zp + 32 * e);
          const uint32_t acc = tmem + (uint32_t)(b * ACW);
          // four K = 16 steps: 8 Z columns (16 halves) and 256 bytes of B each
#pragma unroll
          for (int k = 0; k < TA_KC / 16; ++k) {
            const uint32_t o = (uint32_t)k * 256u;
            const int first = (ch % TA_SEGC == 0 && k == 0) ? 0 : 1;
            // B_lo's rows follow B_hi's at the next 8-row group: one operand of 2 NCP rows
            tc_mma_f16_ta(acc, zt + (uint32_t)(8 * k), tc_sdesc(b_hi + o), idesc2, first);
          }
          if (ch % TA_SEGC == TA_SEGC - 1 || ch == nch - 1) tc_commit(&segdone[b]);
        }
        tc_commit(&sfree[j]);
        tc_commit(&zfree[zp]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // every MMA this thread issued has completed before the tensor memory
      // and shared memory are released (also after an abort)
      tc_commit(&fin);
      mbar_wait_bounded(&fin, 0, VDS_WAIT_LIMIT_NS);
    }
  } else {
    // ---------------------------------------------------- Z formation
    // thread = row 32 (warp % 4) + lane (its tensor-memory lane), the 8 K of
    // quarter warp / 4 of each chunk
    const int q4 = warp & 3, cq = warp >> 2;
    float xi[D];
    {
      const int i = min(i0 + 32 * q4 + lane, Npad - 1);
#pragma unroll
      for (int d = 0; d < D; ++d) xi[d] = rec[(size_t)i * DP + d];
    }
#pragma unroll
    for (int j = 0; j < QC; ++j) tot[j] = 0.f;
    unsigned long long xi2[D];
#pragma unroll
    for (int d = 0; d < D; ++d) xi2[d] = f2_pack(xi[d], xi[d]);
    float ni = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) ni = fmaf(xi[d], xi[d], ni);
    const unsigned long long ni2 = f2_pack(ni, ni), m2 = f2_pack(-2.f, -2.f);
    auto flush = [&](int g) -> bool {
      const int b = g & 1;
      if (!__all_sync(0xffffffffu, rc_wait(&segdone[b], (uint32_t)((g >> 1) & 1), abort))) return false;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * ACW + cq * QC);
      // the two halves of the accumulator (Z_hi B_hi + Z_lo B_hi, Z_hi B_lo)
      if constexpr (QC == 16) {
        uint32_t v[16];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          tc_ld16(ta + (uint32_t)(hf * NCP), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) tot[j] += __uint_as_float(v[j]);
        }
      } else {
        static_assert(QC == 8, "accumulator columns per thread");
        uint32_t v[8];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          tc_ld8(ta + (uint32_t)(hf * NCP), v);
#pragma unroll
          for (int j = 0; j < 8; ++j) tot[j] += __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[b]);
      return true;
    };
    int flushed = 0;  // segments added into registers
    // Z of one chunk for this thread's row and 16 K, rounded to FP16, two K
    // per f32x2 instruction: the squared distances to records u and u + 1 in
    // the two halves of a packed register (records interleaved by particle
    // pairs), expanded through the norms (see above)
    auto z_chunk = [&](const uint8_t *recs_ch, uint32_t (&hv)[8]) {
      const unsigned long long *rs = reinterpret_cast<const unsigned long long *>(recs_ch) + cq * 8 * DP;
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const unsigned long long *rp = rs + (u / 2) * DP;
        // coordinates d, d + 1 (and the norms in slot D) of the pair in
        // 128-bit shared loads
        unsigned long long dot = f2_pack(0.f, 0.f), nk = 0ull;
#pragma unroll
        for (int d = 0; d <= D; d += 2) {
          if (d + 1 <= D) {
            const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(rp + d);
            if (d + 1 < D) {
              dot = f2_fma(xi2[d], w.x, dot);
              dot = f2_fma(xi2[d + 1], w.y, dot);
            } else {
              dot = f2_fma(xi2[d], w.x, dot);
              nk = w.y;
            }
          } else {
            nk = rp[D];
          }
        }
        const unsigned long long r2 = f2_fma(m2, dot, f2_add(ni2, nk));
        float r2a, r2b;
        f2_unpack(r2, r2a, r2b);
        // particles u and u + 1 as two halves of one tensor-memory column
        const __half2 z2 = __floats2half2_rn(ex2_approx(-r2a), ex2_approx(-r2b));
        hv[u / 2] = *reinterpret_cast<const uint32_t *>(&z2);
      }
    };
    for (int c2 = 0; c2 < npass && ok; ++c2) {
      const int j = c2 % NS2, zp = c2 % NZP;
      if (!__all_sync(0xffffffffu, rc_wait(&rfull[j], (uint32_t)((c2 / NS2) & 1), abort) &&
                                       (c2 < NZP || rc_wait(&zfree[zp], (uint32_t)((c2 / NZP - 1) & 1), abort)))) {
        ok = false;
        break;
      }
      tc_fence_after();  // the MMAs that read this Z pair have completed
      const uint8_t *rp = sm + (size_t)j * L::SLOT + L::ROFF;
      uint32_t hv0[8], hv1[8];
      z_chunk(rp, hv0);
      z_chunk(rp + L::REC_BYTES, hv1);
      const uint32_t zt = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(2 * ACW + 64 * zp + 8 * cq);
      tc_st8(zt, hv0);
      tc_st8(zt + 32u, hv1);
      tc_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&zready[zp]);
      // segment g - 1 is added into registers at the third pass of segment g
      const int ch = 2 * c2;
      if (ch % TA_SEGC == 4 && ch / TA_SEGC >= 1) {
        if (!flush(ch / TA_SEGC - 1)) {
          ok = false;
          break;
        }
        ++flushed;
      }
    }
    for (; ok && flushed < nseg; ++flushed)
      if (!flush(flushed)) ok = false;
    if (!ok && tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  // every role has left its loop (the MMA issuer after its MMAs completed,
  // the copy issuer after its copies landed)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, TCOLS);
  if (*abort) return;
  rc_epilogue<D, NCP, QC>(sm, L::TOT_LD, tot, tid, warp, lane, i0, cb, N, rec, phi, ld, r, s, rr, U1, U2, part,
                          1.f / TA_BSCALE);
}

// ---------------------------------------------------------------------------
// The refresh with the kernel values' dot products on the tensor cores as
// well (D = 6, 9; 2 s r + 1 <= 64): per pass of two 64-particle chunks K, one
// group of tcgen05.mma kind::tf32 forms a_I . b_K = 2 qh_I . qh_K - |qh_K|^2
// (the density pass's operand images: TF32 hi/lo split, three products per
// K = 8 step) into a 128-column tensor-memory buffer; the 16 warps that formed
// Z from the records on the CUDA cores now read those sums (tcgen05.ld),
// subtract |qh_I|^2, take ex2 and round to FP16 (one ex2, one FP32 operation
// and a half conversion per pair instead of D + 2 operations), and the MMA
// warp runs Z against [B_hi; B_lo] as in k_refresh_ta.
// Tensor memory: the two segment accumulators (2 x 2 NCP columns) and two
// 128-column pass buffers X_0, X_1.  Pass c's dot products land in
// X_(c mod 2); each thread reads its sums 16 columns at a time and writes
// their 8 FP16 pairs back over the first 8 of the 16 columns, so Z of pass c is
// the A operand of the Z.B MMAs in place (16 particles per 16 columns).  The
// dot products of pass c + 2 go into the same buffer once the Z.B MMAs of
// pass c have completed, so the tensor pipe holds the next pass's dot
// products while the warps form Z.  The 16 warps form Z in two groups of eight
// on alternate passes (buffers), so one group's tensor-memory traffic and
// waits overlap the other's exponentials.
template <int NCP>
struct DtLayout {
  static constexpr int BOP = NCP * TA_KC * 2;       // one FP16 B operand tile
  static constexpr int BCH = 2 * BOP;               // B hi + lo of one chunk
  static constexpr int DOT = 2 * TA_KC * 128;       // dot-product B image of a pass (128 rows)
  static constexpr int AIMG = RC_M * 128;           // dot-product A image of the row tile
  static constexpr int SLOT = ((2 * BCH + DOT + 1023) / 1024) * 1024;
  static constexpr int NS2 = ((200 * 1024 - AIMG) / SLOT) < 8 ? ((200 * 1024 - AIMG) / SLOT) : 8;
  static constexpr int TOT_LD = NCP + 1;
  static constexpr size_t RING = (size_t)AIMG + (size_t)NS2 * SLOT;
  static constexpr size_t SMEM = RING > (size_t)RC_M * TOT_LD * 4 ? RING : (size_t)RC_M * TOT_LD * 4;
  static_assert(NCP <= 64, "Z in tensor memory needs 2 s r + 1 <= 64");
  static_assert(NS2 >= 2, "refresh ring depth");
  static_assert(SMEM <= 227 * 1024 - 1024, "refresh shared memory");
};

template <int D, int NCP>
__global__ void __launch_bounds__(RC_NT, 1)
    k_refresh_dt(const float *__restrict__ rec, int N, int Npad, const float *__restrict__ bimg,
                 const uint8_t *__restrict__ daimg, const uint8_t *__restrict__ dbimg,
                 const float *__restrict__ phi, int ld, int r, int s, int rr, float *__restrict__ U1,
                 float *__restrict__ U2, int nsplit, float *__restrict__ part, int *err) {
  using L = DtLayout<NCP>;
  constexpr int DP = Rec<D>::DP;
  constexpr int NS2 = L::NS2;
  constexpr int QC = NCP / 4;   // accumulator columns per thread in a flush
  constexpr int ACW = 2 * NCP;  // Z against [B_hi; B_lo]: N = 2 NCP
  constexpr int XCOL = 2 * ACW;  // the two pass buffers
  constexpr int TCOLS = 512;
  static_assert(XCOL + 2 * 128 <= TCOLS, "tensor memory columns");
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t afull, sfull[NS2], sfree[NS2], dotready[2], zready[2], xfree[2], segdone[2],
      accfree[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x / nsplit, split = blockIdx.x - tile * nsplit;
  const int i0 = tile * RC_M;
  const int cb = blockIdx.y;
  const int nch_all = Npad / TA_KC, nseg_all = (nch_all + TA_SEGC - 1) / TA_SEGC;
  const int sg0 = split * nseg_all / nsplit, sg1 = (split + 1) * nseg_all / nsplit;
  const int c0 = sg0 * TA_SEGC;                      // first chunk of this CTA
  const int nch = min(sg1 * TA_SEGC, nch_all) - c0;  // a multiple of 4: Npad is of 256
  const int npass = nch / 2;
  const int nseg = sg1 - sg0;
  volatile int *abort = &s_abort;
  if (warp == 0) tc_alloc(&s_tmem, TCOLS);
  if (tid == 0) {
    mbar_init(&afull, 1);
    for (int j = 0; j < NS2; ++j) {
      mbar_init(&sfull[j], 1);
      mbar_init(&sfree[j], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&dotready[b], 1);
      mbar_init(&zready[b], RC_PW / 2);  // the eight warps of group b
      mbar_init(&xfree[b], 1);
      mbar_init(&segdone[b], 1);
      mbar_init(&accfree[b], RC_PW);
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_u32(sm);
  float tot[QC];
  bool ok = true;

  if (warp == RC_PW) {
    // ---------------------------------------------------- bulk copies
    if (lane == 0) {
      mbar_arrive_expect_tx(&afull, (uint32_t)L::AIMG);
      bulk_g2s(sm, daimg + (size_t)tile * L::AIMG, L::AIMG, &afull);
      const uint8_t *bsrc = reinterpret_cast<const uint8_t *>(bimg) + ((size_t)cb * nch_all + c0) * L::BCH;
      const uint8_t *dsrc = dbimg + (size_t)c0 * TA_KC * 128;
      int c2 = 0;
      for (; c2 < npass; ++c2) {
        const int j = c2 % NS2;
        if (c2 >= NS2 && !rc_wait(&sfree[j], (uint32_t)((c2 / NS2 - 1) & 1), abort)) {
          ok = false;
          break;
        }
        uint8_t *slot = sm + L::AIMG + (size_t)j * L::SLOT;
        mbar_arrive_expect_tx(&sfull[j], (uint32_t)(2 * L::BCH + L::DOT));
        bulk_g2s(slot + 2 * L::BCH, dsrc + (size_t)c2 * L::DOT, L::DOT, &sfull[j]);
        bulk_g2s(slot, bsrc + (size_t)(2 * c2) * L::BCH, 2 * L::BCH, &sfull[j]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // the copies still in flight land before the CTA may exit
      for (int k = c2 > NS2 ? c2 - NS2 : 0; k < c2; ++k)
        mbar_wait_bounded(&sfull[k % NS2], (uint32_t)((k / NS2) & 1), VDS_WAIT_LIMIT_NS);
      mbar_wait_bounded(&afull, 0, VDS_WAIT_LIMIT_NS);
    }
  } else if (warp == RC_PW + 1) {
    // ---------------------------------------------------- MMA issue
    if (lane == 0) {
      const uint32_t idesc2 = tc_idesc(TC_FMT_F16, RC_M, ACW);
      const uint32_t idot = tc_idesc(TC_FMT_TF32, RC_M, 2 * TA_KC);
      const uint32_t a0 = sbase;
      // the dot products of pass c2 into X_(c2 mod 2), once the Z.B MMAs of
      // pass c2 - 2 (which read Z from that buffer) have completed
      auto issue_dot = [&](int c2) -> bool {
        const int j = c2 % NS2, x = c2 & 1;
        if (!rc_wait(&sfull[j], (uint32_t)((c2 / NS2) & 1), abort)) return false;
        if (c2 >= 2 && !rc_wait(&xfree[x], (uint32_t)(((c2 >> 1) - 1) & 1), abort)) return false;
        tc_fence_after();
        const uint32_t b0 = sbase + (uint32_t)(L::AIMG + j * L::SLOT + 2 * L::BCH);
        const uint32_t d = tmem + (uint32_t)(XCOL + 128 * x);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t o = (uint32_t)(kk * 256);
          tc_mma_tf32(d, tc_sdesc(a0 + o), tc_sdesc(b0 + o), idot, kk > 0 ? 1 : 0);
          tc_mma_tf32(d, tc_sdesc(a0 + o), tc_sdesc(b0 + 512 + o), idot, 1);
          tc_mma_tf32(d, tc_sdesc(a0 + 512 + o), tc_sdesc(b0 + o), idot, 1);
        }
        tc_commit(&dotready[x]);
        return true;
      };
      ok = rc_wait(&afull, 0, abort) && (npass < 1 || issue_dot(0)) && (npass < 2 || issue_dot(1));
      for (int c2 = 0; c2 < npass && ok; ++c2) {
        const int j = c2 % NS2, x = c2 & 1;
        if (!rc_wait(&zready[x], (uint32_t)((c2 >> 1) & 1), abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int e = 0; e < 2 && ok; ++e) {
          const int ch = 2 * c2 + e, g = ch / TA_SEGC, b = g & 1;
          if (ch % TA_SEGC == 0 && g >= 2 && !rc_wait(&accfree[b], (uint32_t)(((g >> 1) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          const uint32_t b_hi = sbase + (uint32_t)(L::AIMG + j * L::SLOT + e * L::BCH);
          const uint32_t zt = tmem + (uint32_t)(XCOL + 128 * x + 64 * e);
          const uint32_t acc = tmem + (uint32_t)(b * ACW);
#pragma unroll
          for (int k = 0; k < TA_KC / 16; ++k) {
            const uint32_t o = (uint32_t)k * 256u;
            const int first = (ch % TA_SEGC == 0 && k == 0) ? 0 : 1;
            tc_mma_f16_ta(acc, zt + (uint32_t)(16 * k), tc_sdesc(b_hi + o), idesc2, first);
          }
          if (ch % TA_SEGC == TA_SEGC - 1 || ch == nch - 1) tc_commit(&segdone[b]);
        }
        if (!ok) break;
        tc_commit(&sfree[j]);
        tc_commit(&xfree[x]);
        if (c2 + 2 < npass && !issue_dot(c2 + 2)) {
          ok = false;
          break;
        }
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      tc_commit(&fin);
      mbar_wait_bounded(&fin, 0, VDS_WAIT_LIMIT_NS);
    }
  } else {
    // ---------------------------------------------------- Z from the dot products
    // thread = row 32 (warp % 4) + lane (its tensor-memory lane), the 16 K of
    // quarter warp / 4 of each chunk
    const int q4 = warp & 3, cq = warp >> 2;
    const float ni = rec[(size_t)min(i0 + 32 * q4 + lane, Npad - 1) * DP + D + 1];
#pragma unroll
    for (int j = 0; j < QC; ++j) tot[j] = 0.f;
    auto flush = [&](int g) -> bool {
      const int b = g & 1;
      if (!__all_sync(0xffffffffu, rc_wait(&segdone[b], (uint32_t)((g >> 1) & 1), abort))) return false;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * ACW + cq * QC);
      if constexpr (QC == 16) {
        uint32_t v[16];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          tc_ld16(ta + (uint32_t)(hf * NCP), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) tot[j] += __uint_as_float(v[j]);
        }
      } else {
        static_assert(QC == 8, "accumulator columns per thread");
        uint32_t v[8];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          tc_ld8(ta + (uint32_t)(hf * NCP), v);
#pragma unroll
          for (int j = 0; j < 8; ++j) tot[j] += __uint_as_float(v[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[b]);
      return true;
    };
    int flushed = 0;
    const uint32_t lbase = (uint32_t)(q4 * 32) << 16;
    // two groups of eight warps take alternate passes: group gp the passes
    // c2 = gp mod 2, so always pass buffer X_gp, and one group's
    // tensor-memory loads and stores overlap the other's exponentials.  A
    // warp covers its lane quarter and the 16-column blocks 2 h and 2 h + 1
    // of each chunk, one block after the other.
    const int gp = cq >> 1, h = cq & 1;
    static_assert(RC_PW == 16 && TA_KC == 64,
                  "two groups x 4 lane quarters x 2 column halves; 4 blocks of 16 particles per chunk");
    for (int c2 = gp; c2 < npass && ok; c2 += 2) {
      if (!__all_sync(0xffffffffu, rc_wait(&dotready[gp], (uint32_t)((c2 >> 1) & 1), abort))) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int blk = 0; blk < 2; ++blk) {
        // the block's 16 particles of each chunk: columns 16 (2 h + blk).. of
        // the chunk's 64; Z goes back over the first 8 of them, two halves a
        // column, where the Z.B MMA of K block 2 h + blk takes it
        const uint32_t xt = tmem + lbase + (uint32_t)(XCOL + 128 * gp + 16 * (2 * h + blk));
        uint32_t v0[16], v1[16];
        tc_ld16x2(xt, xt + (uint32_t)TA_KC, v0, v1);
        uint32_t hv0[8], hv1[8];
#pragma unroll
        for (int u = 0; u < 16; u += 2) {
          const __half2 z0 = __floats2half2_rn(ex2_approx(__uint_as_float(v0[u]) - ni),
                                               ex2_approx(__uint_as_float(v0[u + 1]) - ni));
          const __half2 z1 = __floats2half2_rn(ex2_approx(__uint_as_float(v1[u]) - ni),
                                               ex2_approx(__uint_as_float(v1[u + 1]) - ni));
          hv0[u / 2] = *reinterpret_cast<const uint32_t *>(&z0);
          hv1[u / 2] = *reinterpret_cast<const uint32_t *>(&z1);
        }
        tc_st8(xt, hv0);
        tc_st8(xt + (uint32_t)TA_KC, hv1);
      }
      tc_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&zready[gp]);
      // segment sg - 1 is flushed after this group's pass in the middle of
      // segment sg (pass 2 of its 4 for group 0, pass 3 for group 1)
      constexpr int PPS = TA_SEGC / 2;  // passes per segment
      static_assert(PPS == 4, "flush schedule: four passes per segment");
      if (c2 % PPS == 2 + gp && c2 / PPS >= 1) {
        if (!flush(c2 / PPS - 1)) {
          ok = false;
          break;
        }
        ++flushed;
      }
    }
    for (; ok && flushed < nseg; ++flushed)
      if (!flush(flushed)) ok = false;
    if (!ok && tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, TCOLS);
  if (*abort) return;
  rc_epilogue<D, NCP, QC>(sm, L::TOT_LD, tot, tid, warp, lane, i0, cb, N, rec, phi, ld, r, s, rr, U1, U2, part,
                          1.f / TA_BSCALE);
}

// U1, U2 from the totals of the nsplit K splits of every row tile, summed in
// split order (FP64): one thread per (I, a, u).
__global__ void k_rc_fin(const float *__restrict__ part, int nsplit, int NCP, int ncta_x, const float *__restrict__ rec,
                         int DP, int D, int N, const float *__restrict__ phi, int ld, int r, int s, int rr,
                         float *__restrict__ U1, float *__restrict__ U2) {
  const int cb = blockIdx.y;
  const int t0 = cb * rr;
  const int rc = min(rr, r - t0);
  const int per = s * rc;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)N * per) return;
  const int I = (int)(e / per), rem = (int)(e - (long)I * per);
  const int a = rem / rc, u = rem - a * rc;
  const int tile = I / RC_M, row = I - tile * RC_M;
  double w1 = 0.0, w2 = 0.0, cs = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) {
    const float *Tr = part + (((size_t)cb * ncta_x + (size_t)tile * nsplit + sp) * RC_M + row) * NCP;
    w1 += Tr[a * rc + u];
    w2 += Tr[per + a * rc + u];
    cs += Tr[2 * per];
  }
  const float wI = rec[(size_t)I * DP + D];
  const size_t o = ((size_t)I * s + a) * ld + t0 + u;
  const float f = phi[o];
  U1[o] = f - (float)w1 * wI;
  U2[o] = (float)cs * f - (float)w2;
}

// the K splits' totals summed into U1, U2 (when the row tiles were split)
template <int D, int NCP>
int refresh_finish(vds_ctx *c, const pod_basis *b, int N, int rr, int ncb, int nsplit, float *part, float *U1,
                   float *U2) {
  if (nsplit <= 1) return VDS_OK;
  const int ntiles = (N + RC_M - 1) / RC_M;
  const int per = b->s * rr;
  k_rc_fin<<<dim3((unsigned)(((long)N * per + 255) / 256), ncb), 256, 0, c->stream>>>(
      part, nsplit, NCP, ntiles * nsplit, (const float *)c->rec.ptr, Rec<D>::DP, D, N, b->phi, b->ld, b->r, b->s,
      rr, U1, U2);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

template <int D, int NCP>
int refresh_launch(vds_ctx *c, const pod_basis *b, int N, int Npad, int rr, int ncb, const float *bimg,
                   const float *recs, int nsplit, float *part, float *U1, float *U2, const uint8_t *daimg,
                   const uint8_t *dbimg) {
  const int ntiles = (N + RC_M - 1) / RC_M;
  dim3 grid(ntiles * nsplit, ncb);
  float *pp = nsplit > 1 ? part : nullptr;
  if constexpr (NCP <= 64 && (D == 6 || D == 9)) {
    if (daimg && dbimg) {
      using L = DtLayout<NCP>;
      VDS_CUDA_TRY(cudaFuncSetAttribute(k_refresh_dt<D, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)L::SMEM));
      k_refresh_dt<D, NCP><<<grid, RC_NT, L::SMEM, c->stream>>>((const float *)c->rec.ptr, N, Npad, bimg, daimg,
                                                                 dbimg, b->phi, b->ld, b->r, b->s, rr, U1, U2,
                                                                 nsplit, pp, c->err);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
      return refresh_finish<D, NCP>(c, b, N, rr, ncb, nsplit, part, U1, U2);
    }
  }
  if constexpr (NCP <= 64) {
    using L = TaLayout<D, NCP>;
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_refresh_ta<D, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)L::SMEM));
    k_refresh_ta<D, NCP><<<grid, RC_NT, L::SMEM, c->stream>>>((const float *)c->rec.ptr, recs, N, Npad, bimg,
                                                               b->phi, b->ld, b->r, b->s, rr, U1, U2, nsplit, pp,
                                                               c->err);
  } else {
    using L = RcLayout<D, NCP>;
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_refresh_tc<D, NCP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)L::SMEM));
    k_refresh_tc<D, NCP><<<grid, RC_NT, L::SMEM, c->stream>>>((const float *)c->rec.ptr, recs, N, Npad, bimg,
                                                               b->phi, b->ld, b->r, b->s, rr, U1, U2, nsplit, pp,
                                                               c->err);
  }
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return refresh_finish<D, NCP>(c, b, N, rr, ncb, nsplit, part, U1, U2);
}

// K splits per row tile: whole segments, chosen so that the CTAs (one per
// SM) fill their last wave; each CTA costs its segments plus a fixed start
// and finish of about 1.5 segments.
int refresh_splits(int ntiles, int ncb, int nseg, int nsm) {
  int best = 1;
  double best_cost = 1e300;
  for (int ns = 1; ns <= 8 && ns <= nseg; ++ns) {
    const long items = (long)ntiles * ncb * ns;
    const long waves = (items + nsm - 1) / nsm;
    const double cost = (double)waves * ((nseg + ns - 1) / ns + 1.5);
    if (cost < best_cost * 0.995) {
      best_cost = cost;
      best = ns;
    }
  }
  return best;
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
  const int ntiles = (N + RC_M - 1) / RC_M;
  const int nsplit = refresh_splits(ntiles, ncb, (Npad / RC_KC + RC_SEG - 1) / RC_SEG, c->num_sms);
  const size_t npart = nsplit > 1 ? (size_t)ncb * ntiles * nsplit * RC_M * NCP : 0;
  // records as staged: pair-interleaved (NCP <= 64) or duplicated (NCP > 64)
  const size_t nrecs = (size_t)Npad * Rec<D>::DP * (NCP <= 64 ? 1 : 2);
  VDS_TRY(vds_ensure(c, c->gbuf, (2 * nbt + npart + nrecs) * sizeof(float)));
  float *bimg = (float *)c->gbuf.ptr, *part = bimg + 2 * nbt, *recs = part + npart;
  k_rc_bt<<<dim3((Npad + 255) / 256, NCP, ncb), 256, 0, c->stream>>>(b->phi, b->ld, r, s, rr,
                                                                     (const float *)c->rec.ptr, Rec<D>::DP, D,
                                                                     N, Npad, NCP, bimg, recs);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  // the dot products of the kernel values on the tensor cores where the
  // density pass's operand images exist for this D (the same layout and
  // padding as the records: Npad rows)
  const uint8_t *daimg = nullptr, *dbimg = nullptr;
  if (NCP <= 64 && (D == 6 || D == 9)) VDS_TRY(pass_density_tc_images(c, N, D, &daimg, &dbimg));
  switch (NCP) {
    case 32: return refresh_launch<D, 32>(c, b, N, Npad, rr, ncb, bimg, recs, nsplit, part, U1, U2, daimg, dbimg);
    case 64: return refresh_launch<D, 64>(c, b, N, Npad, rr, ncb, bimg, recs, nsplit, part, U1, U2, daimg, dbimg);
    case 128:
      return refresh_launch<D, 128>(c, b, N, Npad, rr, ncb, bimg, recs, nsplit, part, U1, U2, nullptr, nullptr);
    default:
      return refresh_launch<D, 256>(c, b, N, Npad, rr, ncb, bimg, recs, nsplit, part, U1, U2, nullptr, nullptr);
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
