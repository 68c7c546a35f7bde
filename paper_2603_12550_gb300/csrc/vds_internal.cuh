// vds_internal.cuh -- shared device helpers and the context of the CUDA
// library.  Not part of the public ABI (include/vds.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vds.h"

#define VDS_MAXD 16

// ----------------------------------------------------------------- status

#define VDS_CUDA_TRY(x)                                   \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) {                              \
      vds_last_cuda_error(e_);                            \
      return e_ == cudaErrorMemoryAllocation ? VDS_ENOMEM \
                                             : VDS_ECUDA; \
    }                                                     \
  } while (0)

#define VDS_TRY(x)          \
  do {                      \
    int st_ = (x);          \
    if (st_ != VDS_OK)      \
      return st_;           \
  } while (0)

void vds_last_cuda_error(cudaError_t e);

// Device error flag: first error wins.
__device__ __forceinline__ void vds_flag(int *err, int code) {
  atomicCAS(err, 0, code);
}

// ----------------------------------------------------------- particle records
// A record holds one particle's scaled coordinates qhat = c q (c chosen so
// that the unnormalised kernel is exp2(-|qhat_I - qhat_J|^2)), then the
// weight w = 1/rho, zero-padded to a multiple of 4 floats (16 B) so that tiles
// of records can be moved by bulk copies and read as float4.
template <int D>
struct Rec {
  static constexpr int DP = ((D + 1 + 3) / 4) * 4;
};

// Padding records sit at this coordinate: every kernel value against them is
// exp2(-huge) = +0 exactly, so they contribute nothing to any pair sum.
#define VDS_PAD_COORD 1.0e15f

// --------------------------------------------------------- inline PTX utils

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit_ns` nanoseconds of
// globaltimer time and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t n = 0;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
  }
}

// 1-D bulk copy global -> shared (TMA engine, no tensor map), completion
// signalled on `bar` as transaction bytes.  dst, src 16-B aligned; bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

#define VDS_WAIT_LIMIT_NS 2000000000ull  // 2 s

// Per-device caches of launch attributes cover devices 0 .. VDS_MAX_DEVICES-1.
constexpr int VDS_MAX_DEVICES = 64;

// ------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide FP64 sum in a fixed order (deterministic); result valid in
// thread 0.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double *sh) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;
}

// --------------------------------------------------------------- context

struct DevBuf {
  void *ptr = nullptr;
  size_t cap = 0;
};

// Optional instrumentation of pair-pass launches and POD phases (vds_timing).
enum {
  PK_DENSITY = 0,
  PK_GRADIENT = 1,
  PK_BANDWIDTH = 2,
  PK_REFRESH = 3,
  PK_GRAM = 4,
  PK_EIGEN = 5,
  PK_BASIS = 6,
  PK_COUNT = 7
};
static_assert(PK_COUNT == VDS_TIMING_KINDS, "timing kinds");
struct TimingPool {
  bool on = false;
  cudaEvent_t ev[PK_COUNT][2][256] = {};
  int used[PK_COUNT] = {};
  double ms[PK_COUNT] = {};
  long count[PK_COUNT] = {};
};

struct vds_ctx {
  long launches = 0;  // kernels launched by the library (all kinds)
  TimingPool *timing = nullptr;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  // workspace, grown on demand
  DevBuf rec;      // records (N_pad x DP floats)
  DevBuf recq;     // records of query points (vds_density_at)
  DevBuf part;     // pair-pass partial sums (FP64)
  DevBuf red;      // block partials of reductions (FP64)
  DevBuf vecs;     // minimiser vectors / scratch (FP32)
  DevBuf gbuf;     // Gram / projection partials (FP64)
  DevBuf ubuf;     // reduced-order scratch (refresh outputs, reduced state)
  DevBuf dtbuf;    // tensor-core density: operand images and split partials
  int *err = nullptr;          // device error flag
  unsigned *ticket = nullptr;  // last-block tickets (zeroed, self-resetting)
  double *scal = nullptr;      // device scalars
  double *h_scal = nullptr;    // pinned host mirror of scal
  int *h_err = nullptr;        // pinned host mirror of err
};

int vds_ensure(vds_ctx *c, DevBuf &b, size_t bytes);
// Bracket a pair-pass launch of kind `pk` with timing events (no-op unless
// instrumentation is on).
int vds_time_begin(vds_ctx *c, int pk);
int vds_time_end(vds_ctx *c, int pk);
int vds_sync_status(vds_ctx *c);  // synchronise the stream, read+clear err

// Scalar slots in ctx->scal
enum { SC_E = 0, SC_DEC = 1, SC_DMAX = 2, SC_YMAX = 3, SC_H = 4, SC_AUX = 5, SC_COUNT = 320 };
// Ticket slots
enum { TK_DENS = 0, TK_GRAD = 1, TK_STRESS = 2, TK_MISC = 3, TK_COUNT = 16 };
