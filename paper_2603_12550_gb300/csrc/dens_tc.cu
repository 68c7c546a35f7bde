// dens_tc.cu -- the density pass rho_I = sum_J exp2(-|qh_I - qh_J|^2)
// (Sec. 2.2's kernel density, qh the connectors scaled by sqrt(log2 e / 2h^2))
// with the pair dot products on the 5th-generation tensor cores, for passes
// held to 1e-4 rather than the full-order path's 1e-5: the density at the
// lifted state of the frozen reduced step's refresh, and the density of all
// particles that the surrogate's subset check needs.
//
// -|qh_I - qh_J|^2 = a_I . b_J - |qh_I|^2 with a_I = (qh_I, 1, 0...) and
// b_J = (2 qh_J, -|qh_J|^2, 0...), K = 16 columns.  One tcgen05.mma of kind
// tf32 (M = 128 rows I, N = 256 columns J, K = 8) takes TF32 operands, so each
// value is split into hi = tf32(x) and lo = tf32(x - hi) and the product is
// formed as hi.hi + hi.lo + lo.hi (six MMAs per 128 x 256 tile).  The tensor
// cores accumulate in FP32 rounding toward zero, so the large terms of the
// expansion (|qh|^2 of tens to hundreds) leave an error of a few FP32 ulps of
// them in the exponent: 1e-5 relative for the median particle of an
// equilibrium cloud, 3e-4 at the worst particle of a cloud stretched
// five-fold.  The products land in tensor memory; the epilogue warps read them
// (tcgen05.ld), subtract |qh_I|^2, take ex2 and sum, so the CUDA cores do two
// FP32 operations and one ex2 per pair instead of D + 2 operations and one
// ex2.  Two 256-column accumulators alternate, so the MMAs of one tile run
// while the epilogue reads the previous one.
//
// Operand images (one per 8-row group, 1024 bytes: the hi values in bytes
// 0..511 as K-major core matrices of 8 rows x 4 values, the lo values in
// bytes 512..1023 the same way), written by k_dt_prep from the pass records:
// element (r, k) of the hi part at (r/8)*1024 + (k/4)*128 + (r%8)*16 +
// (k%4)*4.  So one descriptor layout (core matrices 128 bytes apart along K,
// 8-row groups 1024 bytes apart) serves hi and lo, 512 bytes apart.  Rows
// past N: a_I = 0 (their sums are discarded), b_J with -1e30 in column D
// (exp2 of it is 0).
//
// Roles per CTA (one 128-row tile of I, a range of 256-column tiles of J):
// one thread bulk-copies the A image once and the B images through a
// DT_NS-stage ring; one thread issues the MMAs; 16 warps read the
// accumulators (warp w: rows 32 (w % 4) + lane, columns 64 (w / 4) ..),
// keep FP32 sums per tile and Kahan-compensated FP32 totals across tiles.
// Every wait is bounded; a wait that runs out sets the abort flag and the
// error status, and every role leaves its loop.  Partial sums per column
// split go to part[split][row] (FP64) and k_dt_finish adds them in a fixed
// order, so the result does not depend on the schedule.
#include "pair_impl.cuh"
#include "tcgen05.cuh"

namespace {

constexpr int DT_M = 128;                  // rows I per CTA (tensor-memory lanes)
constexpr int DT_N = 256;                  // columns J per MMA tile
constexpr int DT_K = 16;                   // padded dot-product length
constexpr int DT_NS = 4;                   // B ring stages
constexpr int DT_EW = 16;                  // epilogue warps (4 per tensor-memory lane quarter)
constexpr int DT_CW = DT_N / (DT_EW / 4);   // accumulator columns per epilogue warp
constexpr int DT_NT = (DT_EW + 2) * 32;    // + copy warp + MMA warp
constexpr int DT_RB = 128;                 // image bytes per row (hi 64 + lo 64, interleaved by row group)
constexpr int DT_AB = DT_M * DT_RB;        // 16 KB
constexpr int DT_BB = DT_N * DT_RB;        // 32 KB
constexpr size_t DT_SMEM = (size_t)DT_AB + (size_t)DT_NS * DT_BB;

__device__ __forceinline__ uint32_t dt_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// A and B images of rows [0, Npad) from the pass records (qh in slots 0..D-1,
// |qh|^2 in slot D + 1), one thread per (row, column k).
template <int D>
__global__ void k_dt_prep(const float *__restrict__ rec, int N, int Npad, uint8_t *__restrict__ aimg,
                          uint8_t *__restrict__ bimg) {
  constexpr int DP = Rec<D>::DP;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)Npad * DT_K) return;
  const int r = (int)(e / DT_K), k = (int)(e % DT_K);
  float a = 0.f, b = 0.f;
  if (r < N) {
    const float *x = rec + (size_t)r * DP;
    if (k < D) {
      a = x[k];
      b = 2.f * x[k];
    } else if (k == D) {
      a = 1.f;
      b = -x[D + 1];
    }
  } else if (k == D) {
    b = -1e30f;
  }
  const float ah = to_tf32(a), bh = to_tf32(b);
  const size_t o = (size_t)dt_off(r, k);
  *reinterpret_cast<float *>(aimg + o) = ah;
  *reinterpret_cast<float *>(aimg + o + 512) = to_tf32(a - ah);
  *reinterpret_cast<float *>(bimg + o) = bh;
  *reinterpret_cast<float *>(bimg + o + 512) = to_tf32(b - bh);
}

// rho_I = sum over the splits (in order) of the partial sums; the pass
// records' weight slot gets 1/rho (what the gradient passes read), rho_out rho.
__global__ void k_dt_finish(const double *__restrict__ part, int nsplit, int Nrow, int N, int DP, int wslot,
                            float *__restrict__ rec, float *__restrict__ rho_out, int *err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double rho = 0.0;
  for (int s = 0; s < nsplit; ++s) rho += part[(size_t)s * Nrow + i];
  if (!(rho >= 0.5 && rho <= 1e300)) vds_flag(err, VDS_ENAN);
  rec[(size_t)i * DP + wslot] = (float)(1.0 / rho);
  if (rho_out) rho_out[i] = (float)rho;
}

// Wait for a barrier phase, giving up when another role has aborted or after
// the library's wait limit (then setting the abort flag).
__device__ __forceinline__ bool dt_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t n = 0;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 15u) == 15u) {
      if (*abort) return false;
      if (global_timer_ns() - t0 > VDS_WAIT_LIMIT_NS) {
        *abort = 1;
        return false;
      }
    }
  }
}

// part[split][row] = sum over the split's column tiles [c0, c1) of
// exp2(a_row . b_J - |qh_row|^2), rows of row tile blockIdx.x.
__global__ void __launch_bounds__(DT_NT, 1)
    k_dens_tc(const uint8_t *__restrict__ aimg, const uint8_t *__restrict__ bimg, const float *__restrict__ rec,
              int DP, int nslot, int N, int ntc, int tpc, double *__restrict__ part, int *err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ __align__(8) uint64_t abar, full[DT_NS], empty[DT_NS], accfull[2], accfree[2], fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ float s_tot[DT_EW / 4][DT_M], s_cmp[DT_EW / 4][DT_M];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tr = blockIdx.x, split = blockIdx.y;
  const int c0 = split * tpc, c1 = min(ntc, c0 + tpc);
  const int nt = c1 > c0 ? c1 - c0 : 0;
  uint8_t *sa = dsm, *ring = dsm + DT_AB;
  volatile int *abort = &s_abort;
  if (warp == 0) tc_alloc(&s_tmem, 512);
  if (tid == 0) {
    mbar_init(&abar, 1);
    for (int k = 0; k < DT_NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&accfull[k], 1);
      mbar_init(&accfree[k], DT_EW);  // one arrival per epilogue warp
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == DT_EW) {
    // ------------------------------------------------ bulk copies
    if (lane == 0) {
      mbar_arrive_expect_tx(&abar, DT_AB);
      bulk_g2s(sa, aimg + (size_t)tr * DT_AB, DT_AB, &abar);
      int g = 0;
      bool ok = true;
      for (; g < nt; ++g) {
        const int st = g % DT_NS;
        if (g >= DT_NS && !dt_wait(&empty[st], (uint32_t)(((g / DT_NS) - 1) & 1), abort)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[st], DT_BB);
        bulk_g2s(ring + st * DT_BB, bimg + (size_t)(c0 + g) * DT_BB, DT_BB, &full[st]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // the copies still in flight land before the CTA may exit
      for (int k = g > DT_NS ? g - DT_NS : 0; k < g; ++k)
        mbar_wait_bounded(&full[k % DT_NS], (uint32_t)((k / DT_NS) & 1), VDS_WAIT_LIMIT_NS);
      mbar_wait_bounded(&abar, 0, VDS_WAIT_LIMIT_NS);
    }
  } else if (warp == DT_EW + 1) {
    // ------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = tc_idesc(TC_FMT_TF32, DT_M, DT_N);
      const uint32_t a0 = smem_u32(sa), rb = smem_u32(ring);
      bool ok = dt_wait(&abar, 0, abort);
      for (int g = 0; g < nt && ok; ++g) {
        const int st = g % DT_NS, b = g & 1;
        if (!dt_wait(&full[st], (uint32_t)((g / DT_NS) & 1), abort)) {
          ok = false;
          break;
        }
        // the epilogue has read this accumulator's previous tile
        if (g >= 2 && !dt_wait(&accfree[b], (uint32_t)(((g >> 1) - 1) & 1), abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * DT_N);
        const uint32_t b0 = rb + (uint32_t)(st * DT_BB);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t o = (uint32_t)(kk * 256);  // 8 TF32 of K = two core matrices
          tc_mma_tf32(d, tc_sdesc(a0 + o), tc_sdesc(b0 + o), idesc, kk > 0 ? 1 : 0);   // hi . hi
          tc_mma_tf32(d, tc_sdesc(a0 + o), tc_sdesc(b0 + 512 + o), idesc, 1);         // hi . lo
          tc_mma_tf32(d, tc_sdesc(a0 + 512 + o), tc_sdesc(b0 + o), idesc, 1);         // lo . hi
        }
        tc_commit(&empty[st]);
        tc_commit(&accfull[b]);
      }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
    }
  } else {
    // ------------------------------------------------ epilogue warps 0-7
    const int q = warp & 3, hc = warp >> 2;
    const int rl = q * 32 + lane;
    const int row = tr * DT_M + rl;
    const float nI = row < N ? rec[(size_t)row * DP + nslot] : 0.f;
    float tot = 0.f, cmp = 0.f;
    bool ok = true;
    for (int g = 0; g < nt && ok; ++g) {
      const int b = g & 1;
      ok = __all_sync(0xffffffffu, dt_wait(&accfull[b], (uint32_t)((g >> 1) & 1), abort));
      if (!ok) break;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * DT_N + hc * DT_CW);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
      for (int c = 0; c < DT_CW / 32; ++c) {
        uint32_t v[32];
        tc_ld32(ta + (uint32_t)(c * 32), v);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          s0 += ex2_approx(__uint_as_float(v[j]) - nI);
          s1 += ex2_approx(__uint_as_float(v[j + 1]) - nI);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[b]);
      const float y = (s0 + s1) - cmp;
      const float t = tot + y;
      cmp = (t - tot) - y;
      tot = t;
    }
    // the two column halves of a row: warp pairs (w, w + 4) through shared memory
    s_tot[hc][rl] = tot;
    s_cmp[hc][rl] = cmp;
    asm volatile("bar.sync 1, %0;" ::"r"(DT_EW * 32) : "memory");
    if (hc == 0 && row < N) {
      double v = 0.0;
      for (int k = 0; k < DT_EW / 4; ++k) v += (double)s_tot[k][rl] - (double)s_cmp[k][rl];
      part[(size_t)split * N + row] = v;
    }
    if (!ok && lane == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  // every role has left its loop; the MMAs issued are complete before the
  // tensor memory is released
  tc_fence_before();
  __syncthreads();
  if (warp == DT_EW + 1 && lane == 0) {
    tc_commit(&fin);
    mbar_wait_bounded(&fin, 0, VDS_WAIT_LIMIT_NS);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, 512);
}

}  // namespace

// ------------------------------------------------------------------ host

namespace {

// column splits: the CTAs (row tiles x splits, one per SM at a time) in
// whole waves as nearly as possible, at least 8 column tiles per split
int dt_splits(int ntr, int ntc, int nsm) {
  int best = 1;
  double best_eff = 0.0;
  for (int ns = 1; ns <= 16; ++ns) {
    const int tpc = (ntc + ns - 1) / ns;
    if (ns > 1 && tpc < 8) break;
    const int nsr = (ntc + tpc - 1) / tpc;
    const long ctas = (long)ntr * nsr;
    const long waves = (ctas + nsm - 1) / nsm;
    const double eff = (double)ctas / (double)(waves * nsm);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = nsr;
    }
  }
  return best;
}

template <int D>
int dens_tc_impl(vds_ctx *c, int N, float *rho_out) {
  constexpr int DP = Rec<D>::DP;
  const int Npad = (N + DT_N - 1) / DT_N * DT_N;
  const int ntr = (N + DT_M - 1) / DT_M, ntc = Npad / DT_N;
  const int nsplit = dt_splits(ntr, ntc, c->num_sms);
  const int tpc = (ntc + nsplit - 1) / nsplit;
  const size_t img = (size_t)Npad * DT_RB;
  VDS_TRY(vds_ensure(c, c->dtbuf, 2 * img + (size_t)nsplit * N * sizeof(double)));
  uint8_t *aimg = (uint8_t *)c->dtbuf.ptr, *bimg = aimg + img;
  double *part = (double *)(bimg + img);
  const float *rec = (const float *)c->rec.ptr;
  const long ne = (long)Npad * DT_K;
  k_dt_prep<D><<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(rec, N, Npad, aimg, bimg);
  VDS_CUDA_TRY(cudaGetLastError());
  static bool attr[VDS_MAX_DEVICES] = {};
  if (c->device >= VDS_MAX_DEVICES || !attr[c->device]) {
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_dens_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DT_SMEM));
    if (c->device < VDS_MAX_DEVICES) attr[c->device] = true;
  }
  k_dens_tc<<<dim3((unsigned)ntr, (unsigned)nsplit), DT_NT, DT_SMEM, c->stream>>>(
      aimg, bimg, rec, DP, D + 1, N, ntc, tpc, part, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  k_dt_finish<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(part, nsplit, N, N, DP, D,
                                                                  (float *)c->rec.ptr, rho_out, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  c->launches += 3;
  return VDS_OK;
}

}  // namespace

int pass_density_tc(vds_ctx *c, const KParams &kp, float *rho_out) {
  if (kp.N < 1) return VDS_EARG;
  switch (kp.D) {
    case 6: return dens_tc_impl<6>(c, kp.N, rho_out);
    case 9: return dens_tc_impl<9>(c, kp.N, rho_out);
    default: return VDS_EARG;  // no norm slot in the records, or D + 1 > 16
  }
}

int pass_density_tc_images(vds_ctx *c, int N, int D, const uint8_t **aimg, const uint8_t **bimg) {
  if (N < 1 || (D != 6 && D != 9)) return VDS_EARG;
  const int Npad = (N + DT_N - 1) / DT_N * DT_N;
  const size_t img = (size_t)Npad * DT_RB;
  VDS_TRY(vds_ensure(c, c->dtbuf, 2 * img));
  uint8_t *a = (uint8_t *)c->dtbuf.ptr, *b = a + img;
  const long ne = (long)Npad * DT_K;
  if (D == 6)
    k_dt_prep<6><<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>((const float *)c->rec.ptr, N, Npad, a, b);
  else
    k_dt_prep<9><<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>((const float *)c->rec.ptr, N, Npad, a, b);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  *aimg = a;
  *bimg = b;
  return VDS_OK;
}
