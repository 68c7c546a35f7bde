// gram_tc.cu -- the POD snapshot Gram C = X^T X (Sec. 2.3, method of
// snapshots) on the 5th-generation tensor cores, TF32 with one refinement
// step (3xTF32), compensated FP32 across chunks, FP64 across K splits.
//
// Every FP32 snapshot value x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi) (round to nearest), so x = x_hi + x_lo up to 2^-22 |x|,
// and each product is formed as x_hi y_hi + x_hi y_lo + x_lo y_hi (the
// dropped x_lo y_lo is below 2^-22 |x y|): three tcgen05.mma of kind::tf32
// per K step, accumulating in FP32 in tensor memory: x_hi y_hi in one
// accumulator, the two correction products (2^-11 smaller) in another, so the
// rounding of the large running sum is confined to the 4 MMAs of one 32-row
// chunk.  After each chunk both accumulators are read back (tcgen05.ld) and
// added into per-thread FP32 totals with Kahan compensation (each of the 8
// warps holds 64 columns of its 32 rows) while the next chunk accumulates into
// a second accumulator pair.  Per-CTA FP64 partial tiles are summed over the
// K splits in a fixed order: the result does not depend on the schedule.
//
// Layout: X is column-major (Ns x M), so a tile row (one snapshot column) is
// contiguous along K; chunks of 32 rows are staged by cp.async into the
// K-major canonical layout (8-row x 16-byte core matrices) in a 3-stage ring,
// split into hi/lo in shared memory, and consumed by one thread issuing the
// MMAs.  Only tiles on or above the diagonal are computed.
#include <math.h>

#include "pod_internal.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int TG_M = 128;                 // C tile (rows = cols)
constexpr int TG_KC = 32;                 // snapshot rows per chunk (128 B per tile row)
constexpr int TG_ST = 3;                  // ring stages
constexpr int TG_NT = 256;                // threads (8 warps)
constexpr int TG_OP = TG_M * TG_KC * 4;   // bytes of one operand tile (16 KB)
constexpr int TG_STAGE = 4 * TG_OP;       // A hi, A lo, B hi, B lo
constexpr size_t TG_SMEM = (size_t)TG_ST * TG_STAGE;
constexpr uint32_t TG_TMEM_COLS = 512;     // two (big, small) accumulator pairs; one CTA per SM

// Copy tile rows (snapshot columns col0..col0+127) x chunk rows
// [kr0, kr0 + 32) of X into the canonical layout at dst; zero outside
// [0, M) x [kr0, k1).  Byte offset of element (r, k): (r/8)*1024 +
// (k/4)*128 + (r%8)*16 + (k%4)*4.
__device__ __forceinline__ void tg_load(uint32_t dst, const float *__restrict__ X, long Ns, int M, int col0,
                                        long kr0, long k1, bool aligned) {
  if (aligned) {
    // 16-byte granules (4 rows of one column); Ns and every chunk start are
    // multiples of 4, so a granule is either inside [kr0, k1) or outside
    for (int idx = threadIdx.x; idx < TG_M * 8; idx += TG_NT) {
      const int r8 = idx & 7, c = (idx >> 3) & 7, g = idx >> 6;
      const int r = g * 8 + r8;
      const long kk = kr0 + 4 * c;
      const bool ok = (col0 + r < M) && (kk < k1);
      const float *p = X + (ok ? (size_t)(col0 + r) * Ns + kk : 0);
      cp_async16(dst + g * 1024 + c * 128 + r8 * 16, p, ok);
    }
  } else {
    for (int idx = threadIdx.x; idx < TG_M * TG_KC; idx += TG_NT) {
      const int r8 = idx & 7, q = (idx >> 3) & 3, c = (idx >> 5) & 7, g = idx >> 8;
      const int r = g * 8 + r8;
      const long kk = kr0 + 4 * c + q;
      const bool ok = (col0 + r < M) && (kk < k1);
      const float *p = X + (ok ? (size_t)(col0 + r) * Ns + kk : 0);
      cp_async4(dst + g * 1024 + c * 128 + r8 * 16 + q * 4, p, ok);
    }
  }
}

// In place x -> tf32(x) and lo slot <- tf32(x - tf32(x)) over one operand tile.
__device__ __forceinline__ void tg_split(uint8_t *tile) {
  float4 *hi = reinterpret_cast<float4 *>(tile);
  float4 *lo = reinterpret_cast<float4 *>(tile + TG_OP);
#pragma unroll
  for (int u = 0; u < TG_OP / 16 / TG_NT; ++u) {
    const int e = threadIdx.x + u * TG_NT;
    const float4 x = hi[e];
    float4 h, l;
    h.x = to_tf32(x.x);
    h.y = to_tf32(x.y);
    h.z = to_tf32(x.z);
    h.w = to_tf32(x.w);
    l.x = to_tf32(x.x - h.x);
    l.y = to_tf32(x.y - h.y);
    l.z = to_tf32(x.z - h.z);
    l.w = to_tf32(x.w - h.w);
    hi[e] = h;
    lo[e] = l;
  }
}

// part[split][tile][128][128] (FP64) for tiles (bi <= bj) of C.
__global__ void __launch_bounds__(TG_NT, 1)
    k_gram_tc(const float *__restrict__ X, long Ns, int M, int nbt, long kchunk, int aligned,
              double *__restrict__ part, int *err) {
  const int bi = blockIdx.x / nbt, bj = blockIdx.x - (blockIdx.x / nbt) * nbt;
  if (bi > bj) return;
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t bars[TG_ST];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool diag = bi == bj;
  const long k0 = (long)blockIdx.y * kchunk;
  const long k1 = min(Ns, k0 + kchunk);
  const int nch = k1 > k0 ? (int)((k1 - k0 + TG_KC - 1) / TG_KC) : 0;
  if (warp == 0) tc_alloc(&s_tmem, TG_TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < TG_ST; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc(TC_FMT_TF32, TG_M, TG_M);
  const uint32_t sbase = smem_u32(gsm);
  // tensor memory: per chunk parity b, x_hi y_hi into columns 256 b and the
  // two correction products into columns 256 b + 128; warp w reads lanes
  // 32 (w % 4) .. (its rows) and columns 64 (w / 4) .. of both
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32);
  const int col_half = (warp >> 2) * 64;
  float tot[64], cmp[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) tot[j] = cmp[j] = 0.f;
  // chunk c's FP32 tile into the compensated per-thread totals
  auto flush = [&](int c) {
    const uint32_t base = tmem + (lane_base << 16) + (uint32_t)((c & 1) * 256 + col_half);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t vb[16], vs[16];
      tc_ld16(base + 16 * q, vb);
      tc_ld16(base + 128 + 16 * q, vs);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float y = (__uint_as_float(vb[j]) + __uint_as_float(vs[j])) - cmp[16 * q + j];
        const float t = tot[16 * q + j] + y;
        cmp[16 * q + j] = (t - tot[16 * q + j]) - y;
        tot[16 * q + j] = t;
      }
    }
  };

  auto issue_loads = [&](int ch) {
    if (ch < nch) {
      const uint32_t st = sbase + (ch % TG_ST) * TG_STAGE;
      const long kr0 = k0 + (long)ch * TG_KC;
      tg_load(st, X, Ns, M, bi * TG_M, kr0, k1, aligned != 0);
      if (!diag) tg_load(st + 2 * TG_OP, X, Ns, M, bj * TG_M, kr0, k1, aligned != 0);
    }
    cp_async_commit();
  };
  for (int ch = 0; ch < TG_ST - 1; ++ch) issue_loads(ch);
  bool ok = true;
  int last_committed = -1;
  for (int ch = 0; ch < nch; ++ch) {
    const int stage = ch % TG_ST;
    uint8_t *stp = gsm + (size_t)stage * TG_STAGE;
    cp_async_wait<TG_ST - 2>();
    __syncthreads();
    tg_split(stp);
    if (!diag) tg_split(stp + 2 * TG_OP);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_hi = sbase + stage * TG_STAGE, a_lo = a_hi + TG_OP;
      const uint32_t b_hi = diag ? a_hi : a_hi + 2 * TG_OP, b_lo = diag ? a_lo : a_hi + 3 * TG_OP;
      const uint32_t d_big = tmem + (uint32_t)((ch & 1) * 256), d_small = d_big + 128;
#pragma unroll
      for (int k = 0; k < TG_KC / 8; ++k) {
        const uint32_t o = (uint32_t)k * 256u;  // 8 TF32 of K = two core matrices
        tc_mma_tf32(d_small, tc_sdesc(a_lo + o), tc_sdesc(b_hi + o), idesc, k > 0 ? 1 : 0);
        tc_mma_tf32(d_small, tc_sdesc(a_hi + o), tc_sdesc(b_lo + o), idesc, 1);
        tc_mma_tf32(d_big, tc_sdesc(a_hi + o), tc_sdesc(b_hi + o), idesc, k > 0 ? 1 : 0);
      }
      tc_commit(&bars[stage]);
    }
    last_committed = ch;
    // chunk ch - 1: its MMAs are done before its stage is refilled and its
    // accumulators are read (chunk ch runs meanwhile on the other pair)
    if (ch >= 1) {
      const int pc = ch - 1;
      const bool got = mbar_wait_bounded(&bars[pc % TG_ST], (uint32_t)((pc / TG_ST) & 1), VDS_WAIT_LIMIT_NS);
      if (__syncthreads_or(!got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      flush(pc);
      tc_fence_before();
    }
    issue_loads(ch + TG_ST - 1);
  }
  if (ok && nch > 0) {
    const int pc = nch - 1;
    const bool got = mbar_wait_bounded(&bars[pc % TG_ST], (uint32_t)((pc / TG_ST) & 1), VDS_WAIT_LIMIT_NS);
    if (__syncthreads_or(!got)) {
      ok = false;
    } else {
      tc_fence_after();
      flush(pc);
    }
  }
  cp_async_wait<0>();
  if (!ok) {
    // let the MMAs already issued finish (bounded) before releasing TMEM
    if (tid == 0 && last_committed >= 0)
      mbar_wait_bounded(&bars[last_committed % TG_ST], (uint32_t)((last_committed / TG_ST) & 1),
                        VDS_WAIT_LIMIT_NS / 8);
    if (tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, TG_TMEM_COLS);
  if (!ok) return;
  const int row = (int)lane_base + lane;
  double *dst = part + (((size_t)blockIdx.y * nbt * nbt + blockIdx.x) * TG_M + row) * TG_M + col_half;
#pragma unroll
  for (int j = 0; j < 64; ++j) dst[j] = (double)tot[j] - (double)cmp[j];
}

// C (M x M, FP64) = sum over K splits (in order) of the tile partials,
// upper triangle mirrored.
__global__ void k_gram_tc_reduce(const double *__restrict__ part, int M, int nbt, int nks, double *__restrict__ C) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  const int i = (int)(idx / M), j = (int)(idx - (long)(idx / M) * M);
  const int ii = i <= j ? i : j, jj = i <= j ? j : i;
  const int bi = ii / TG_M, bj = jj / TG_M;
  const size_t off = ((size_t)(bi * nbt + bj) * TG_M + (ii - bi * TG_M)) * TG_M + (jj - bj * TG_M);
  const size_t tstride = (size_t)nbt * nbt * TG_M * TG_M;
  double v = 0.0;
  for (int k = 0; k < nks; ++k) v += part[(size_t)k * tstride + off];
  C[idx] = v;
}

}  // namespace

size_t pod_gram_tc_workspace(const vds_ctx *c, long Ns, int M) {
  const int nbt = (M + TG_M - 1) / TG_M;
  const int ntiles = nbt * (nbt + 1) / 2;
  int nks = c->num_sms / ntiles;
  if (nks < 1) nks = 1;
  if ((long)nks * TG_KC > Ns) nks = (int)((Ns + TG_KC - 1) / TG_KC);
  return (size_t)nks * nbt * nbt * TG_M * TG_M * sizeof(double);
}

int pod_gram_tc(vds_ctx *c, const float *X, long Ns, int M, double *part, double *C) {
  const int nbt = (M + TG_M - 1) / TG_M;
  const int ntiles = nbt * (nbt + 1) / 2;
  // K splits: one wave of one CTA per SM over the upper-triangle tiles
  int nks = c->num_sms / ntiles;
  if (nks < 1) nks = 1;
  if ((long)nks * TG_KC > Ns) nks = (int)((Ns + TG_KC - 1) / TG_KC);
  long kchunk = (Ns + nks - 1) / nks;
  kchunk = (kchunk + TG_KC - 1) / TG_KC * TG_KC;
  const int aligned = (Ns % 4 == 0 && ((uintptr_t)X & 15) == 0) ? 1 : 0;
  VDS_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
  k_gram_tc<<<dim3(nbt * nbt, nks), TG_NT, TG_SMEM, c->stream>>>(X, Ns, M, nbt, kchunk, aligned, part, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  k_gram_tc_reduce<<<(unsigned)(((long)M * M + 255) / 256), 256, 0, c->stream>>>(part, M, nbt, nks, C);
  VDS_CUDA_TRY(cudaGetLastError());
  c->launches += 2;
  return VDS_OK;
}
