// mlp.cu -- learned score surrogate s_theta ~ grad ln f (include/vds_score.h):
// an MLP D -> W -> W -> W -> D with SiLU hidden layers, BF16 weights and
// activations, FP32 accumulation, trained by denoising score matching with
// Adam; forward and backward GEMMs on the 5th-generation tensor cores.
//
// GEMM (k_gemm_tma): C[M x N] = A[M x K] . B[N x K]^T, A and B row-major
// BF16 (K contiguous).  One CTA per 128-row tile (and per K split), 8 warps.
// K is consumed in chunks of 64: one thread loads the A (128 x 64) and B
// (N x 64) chunks with tensor-map TMA copies (128-byte swizzle) into a ring of
// stages, one thread issues four tcgen05.mma (M=128, N, K=16, kind::f16 with
// BF16 inputs) per chunk accumulating in tensor memory and frees the stage
// with a commit.  The epilogue reads the accumulator with tcgen05.ld (warp w
// owns lanes 32 (w % 4).. = rows) and applies the layer's bias/activation,
// writing row-major and, where the backward pass needs it, transposed copies.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/vds_score.h"
#include "tcgen05.cuh"
#include "vds_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int GM = 128;   // rows per CTA tile
constexpr int KC = 64;    // K per chunk
constexpr int TMEM_COLS = 128;

// Logistic sigma(z) = 1 / (1 + e^-z) with the hardware 2^x (e^-z = 2^(-z log2 e))
// and a fast reciprocal: about 1e-7 relative, far below the BF16 rounding of
// the activations it feeds.
__device__ __forceinline__ float sigmoid_f(float z) {
  return __fdividef(1.f, 1.f + ex2_approx(-1.4426950408889634f * z));
}
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = sigmoid_f(z);
  return s * (1.f + z * (1.f - s));
}

enum { EPI_F32 = 0, EPI_SILU = 1, EPI_DSILU = 2 };

struct Epi {
  int mode;
  int rows;          // valid rows of C
  int ncols;         // valid columns written
  int ldc;           // row stride of outf / h / zf
  long long split_stride;  // element offset of a K split's output (EPI_F32)
  const float *bias;       // per column (may be null)
  float *outf;             // EPI_F32 output, or FP32 copy (z for SILU, dz for DSILU)
  bf16 *h;                 // BF16 row-major output
  bf16 *ht;                // BF16 transposed output (may be null)
  int ldt;                 // row stride of ht
  const float *zin;        // pre-activation for DSILU (stride ldc)
};

constexpr int GBN = 128;   // columns of C per CTA
constexpr int GNT = 256;   // threads: warps w and w + 4 share TMEM lanes 32 (w % 4), split the columns
constexpr int GSTAGE = GM * KC * 2 + GBN * KC * 2;  // bytes per stage (A 16 KB + B <= 16 KB)

// C tile [128 rows x BN cols] = A[m0:, K-split] . B[n0:n0+BN, K-split]^T.
// A and B come in by tensor-map TMA loads (2-D boxes of 64 K x 128 (or BN)
// rows, 128-byte swizzled, rows past the tensor zero-filled) issued by one
// thread into a GS-stage ring; one thread issues four tcgen05.mma per chunk
// (M=128, N=BN, K=16, kind::f16 with BF16 inputs) and frees each stage with a
// commit; all 8 warps then run the epilogue (warps w and w + 4 share tensor
// memory lanes 32 (w % 4).., splitting the columns).
template <int GS>
__global__ void __launch_bounds__(GNT)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int N,
               int Ksplit, int boxB, Epi ep, int *err) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t full[GS], empty[GS], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * GM;
  const int kbase = blockIdx.y * Ksplit;
  const int n0 = blockIdx.z * GBN;
  const int BN = min(GBN, N - n0);
  if (warp == 0) tc_alloc(&s_tmem, TMEM_COLS);
  if (tid == 0) {
    for (int k = 0; k < GS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    mbar_init(&done, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int nch = Ksplit / KC;
  const uint32_t sbase = smem_u32(gsm);
  const uint32_t txbytes = (uint32_t)(GM * KC * 2 + boxB * KC * 2);
  // this thread's epilogue share: row `row`, columns [cb, ce) of the tile
  const int row = m0 + (warp & 3) * 32 + lane;
  const bool vrow = row < ep.rows;
  const int half = ((BN + 31) / 32) * 16;
  const int cb = (warp >> 2) * half, ce = min(BN, cb + half);
  // the pre-activations the derivative epilogue multiplies by are loaded
  // before the main loop, so their latency hides behind it
  constexpr int HMAX = GBN / 2;
  float zpre[HMAX];
  if (ep.mode == EPI_DSILU) {
    const bool vec = (ep.ldc & 3) == 0 && ((uintptr_t)ep.zin & 15) == 0;
#pragma unroll
    for (int c4 = 0; c4 < HMAX; c4 += 4) {
      const int colb = n0 + cb + c4;
      const bool in = vrow && cb + c4 < ce;
      if (in && vec && colb + 4 <= ep.ncols) {
        const float4 z4 = *reinterpret_cast<const float4 *>(ep.zin + (size_t)row * ep.ldc + colb);
        zpre[c4] = z4.x;
        zpre[c4 + 1] = z4.y;
        zpre[c4 + 2] = z4.z;
        zpre[c4 + 3] = z4.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          zpre[c4 + u] = (in && cb + c4 + u < ce && colb + u < ep.ncols) ? ep.zin[(size_t)row * ep.ldc + colb + u]
                                                                        : 0.f;
      }
    }
  }
  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int ch = 0;
    for (; ch < nch; ++ch) {
      const int st = ch % GS;
      if (ch >= GS && !mbar_wait_bounded(&empty[st], (uint32_t)((ch / GS - 1) & 1), VDS_WAIT_LIMIT_NS)) {
        s_abort = 1;
        break;
      }
      const uint32_t a0 = sbase + st * GSTAGE, b0 = a0 + GM * KC * 2;
      mbar_arrive_expect_tx(&full[st], txbytes);
      tma_load_2d(a0, &tmA, kbase + ch * KC, m0, &full[st]);
      tma_load_2d(b0, &tmB, kbase + ch * KC, n0, &full[st]);
    }
    // the loads still in flight land before the CTA may exit
    for (int k = ch > GS ? ch - GS : 0; k < ch; ++k)
      mbar_wait_bounded(&full[k % GS], (uint32_t)((k / GS) & 1), VDS_WAIT_LIMIT_NS);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issue
    const uint32_t idesc = tc_idesc(TC_FMT_BF16, GM, BN);
    for (int ch = 0; ch < nch; ++ch) {
      const int st = ch % GS;
      if (!mbar_wait_bounded(&full[st], (uint32_t)((ch / GS) & 1), VDS_WAIT_LIMIT_NS)) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = sbase + st * GSTAGE, b0 = a0 + GM * KC * 2;
#pragma unroll
      for (int k = 0; k < KC / 16; ++k)
        tc_mma_bf16(tmem, tc_sdesc_sw128(a0 + k * 32), tc_sdesc_sw128(b0 + k * 32), idesc,
                    (ch > 0 || k > 0) ? 1 : 0);
      tc_commit(&empty[st]);
    }
    // every MMA issued is complete before the epilogue reads the accumulator
    tc_commit(&done);
  }
  __syncwarp();
  const bool got = mbar_wait_bounded(&done, 0, VDS_WAIT_LIMIT_NS);
  const bool ok = !__syncthreads_or(!got || s_abort);
  tc_fence_after();
  if (!ok) {
    if (tid == 0) vds_flag(err, VDS_ETIMEOUT);
  } else {
    // warp w: rows 32 (w % 4) + lane, columns [cb, ce) of the tile
#pragma unroll
    for (int cc = 0; cc < HMAX; cc += 16) {
      const int c0 = cb + cc;
      if (c0 >= ce) break;
      uint32_t v[16];
      tc_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
      if (!vrow) continue;
      const int colb = n0 + c0;
      const bool full = colb + 16 <= ep.ncols;
      float a[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] = __uint_as_float(v[j]);
      if (ep.mode == EPI_F32) {
        float *o = ep.outf + (long long)blockIdx.y * ep.split_stride + (size_t)row * ep.ldc + colb;
        if (full && (ep.ldc & 3) == 0 && (ep.split_stride & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (ep.bias) a[j] += ep.bias[colb + j];
#pragma unroll
          for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(o + j) = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (colb + j < ep.ncols) o[j] = a[j] + (ep.bias ? ep.bias[colb + j] : 0.f);
        }
        continue;
      }
      float y[16];
      if (ep.mode == EPI_SILU) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float z = a[j] + ((ep.bias && (full || colb + j < ep.ncols)) ? ep.bias[colb + j] : 0.f);
          a[j] = z;
          y[j] = silu_f(z);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          y[j] = a[j] * dsilu_f(zpre[cc + j]);
          a[j] = y[j];
        }
      }
      // FP32 copy (z, or dz) and BF16 activations, row-major; transposed copy
      if (full && (ep.ldc & 7) == 0) {
        if (ep.outf) {
          float *o = ep.outf + (size_t)row * ep.ldc + colb;
#pragma unroll
          for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(o + j) = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
        }
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const __nv_bfloat162 t = __floats2bfloat162_rn(y[2 * j], y[2 * j + 1]);
          pk[j] = *reinterpret_cast<const uint32_t *>(&t);
        }
        uint4 *hp = reinterpret_cast<uint4 *>(ep.h + (size_t)row * ep.ldc + colb);
        hp[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        hp[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (colb + j >= ep.ncols) continue;
          if (ep.outf) ep.outf[(size_t)row * ep.ldc + colb + j] = a[j];
          ep.h[(size_t)row * ep.ldc + colb + j] = __float2bfloat16_rn(y[j]);
        }
      }
      if (ep.ht) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (colb + j < ep.ncols) ep.ht[(size_t)(colb + j) * ep.ldt + row] = __float2bfloat16_rn(y[j]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    tc_dealloc(tmem, TMEM_COLS);
}


// ------------------------------------------------------------ small kernels

// A0 = bf16(x + sigma eps) padded to Dp columns (and its transpose)
__global__ void k_input(const float *__restrict__ x, const int *__restrict__ rows, const float *__restrict__ eps,
                        float sigma, int M, int D, int Dp, bf16 *__restrict__ a0, bf16 *__restrict__ a0t, int ldt) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * Dp) return;
  const int m = (int)(idx / Dp), k = (int)(idx - (long)m * Dp);
  float v = 0.f;
  if (k < D) {
    v = x[(size_t)(rows ? rows[m] : m) * D + k];
    if (eps) v += sigma * eps[(size_t)m * D + k];
  }
  const bf16 b = __float2bfloat16_rn(v);
  a0[idx] = b;
  if (a0t) a0t[(size_t)k * ldt + m] = b;
}

// dS = (2/M)(s + eps/sigma) (first D columns), padded BF16 copies; loss terms
__global__ void k_dsm_out(const float *__restrict__ S, int ldS, const float *__restrict__ eps, float sigma, int M,
                          int D, float *__restrict__ dSf, int Op, bf16 *__restrict__ dSb, int ldb,
                          bf16 *__restrict__ dSt, int ldt, double *__restrict__ lossp) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (m < M) {
    for (int k = 0; k < ldb; ++k) {
      float g = 0.f;
      if (k < D) {
        const float r = S[(size_t)m * ldS + k] + eps[(size_t)m * D + k] / sigma;
        l += (double)r * r;
        g = 2.f * r / (float)M;
      }
      if (k < Op) {
        dSf[(size_t)m * Op + k] = g;
        dSt[(size_t)k * ldt + m] = __float2bfloat16_rn(g);
      }
      dSb[(size_t)m * ldb + k] = __float2bfloat16_rn(g);
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lossp[blockIdx.x] = sh[0];
}

// regression: dS = (2/M)(s - t), t = target[rows[m]] (or target[m])
__global__ void k_fit_out(const float *__restrict__ S, int ldS, const float *__restrict__ target,
                          const int *__restrict__ rows, int M, int D, float *__restrict__ dSf, int Op,
                          bf16 *__restrict__ dSb, int ldb, bf16 *__restrict__ dSt, int ldt,
                          double *__restrict__ lossp) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (m < M) {
    const size_t tr = (size_t)(rows ? rows[m] : m) * D;
    for (int k = 0; k < ldb; ++k) {
      float g = 0.f;
      if (k < D) {
        const float r = S[(size_t)m * ldS + k] - target[tr + k];
        l += (double)r * r;
        g = 2.f * r / (float)M;
      }
      if (k < Op) {
        dSf[(size_t)m * Op + k] = g;
        dSt[(size_t)k * ldt + m] = __float2bfloat16_rn(g);
      }
      dSb[(size_t)m * ldb + k] = __float2bfloat16_rn(g);
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lossp[blockIdx.x] = sh[0];
}

// column sums of an M x n FP32 matrix in a fixed order -> out[n]
__global__ void k_colsum(const float *__restrict__ X, int M, int n, int ld, float *__restrict__ out) {
  const int col = blockIdx.x;
  double a = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) a += X[(size_t)m * ld + col];
  __shared__ double sh[512];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 256; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && col < n) out[col] = (float)sh[0];
}

// out[i] = sum over splits of part[s * stride + i]
__global__ void k_split_reduce(const float *__restrict__ part, int splits, long long stride, long long n,
                               float *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = 0.f;
  for (int s = 0; s < splits; ++s) a += part[s * stride + i];
  out[i] = a;
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copy of a rows x cols FP32 matrix and (optionally) its transpose
// padded to tcols columns (zeros beyond rows).
__global__ void k_to_bf16(const float *__restrict__ W, int rows, int cols, bf16 *__restrict__ Wb,
                          bf16 *__restrict__ Wt, int tcols) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long)rows * cols) {
    const int r = (int)(idx / cols), c = (int)(idx - (long)r * cols);
    const bf16 b = __float2bfloat16_rn(W[idx]);
    Wb[idx] = b;
    if (Wt) Wt[(size_t)c * tcols + r] = b;
  }
  if (Wt && idx < (long)cols * tcols) {
    const int c = (int)(idx / tcols), r = (int)(idx - (long)c * tcols);
    if (r >= rows) Wt[idx] = __float2bfloat16_rn(0.f);
  }
}

// ------------------------------------------------- fused inference forward
//
// k_mlp_fwd evaluates all four layers of the width-256 network for 128-row
// tiles in one persistent launch (one CTA per SM, 576 threads): the hidden
// activations of a tile never leave shared memory.  Roles:
//   warp 16, one lane  streams the packed weights (F_NCOPY copies per tile,
//                      each the exact shared-memory image of the two 128-row
//                      x 64-K operand blocks of one K-chunk) through an
//                      F_STAGES-deep ring with 1-D bulk copies (TMA engine);
//   warp 17, one lane  issues the tcgen05.mma (M=128, N=256: the two 128-row
//                      weight blocks of a K-chunk are adjacent and form one
//                      B operand; K=16; N=16 for the output layer);
//   warps 0-15         read the accumulator (warp w: rows 32 (w % 4) + lane,
//                      16 columns (w / 4) of each 64-column K-chunk), add the
//                      bias, apply SiLU and write BF16 activations back in
//                      place as the next layer's A operand; for the output
//                      layer they add b4 and store the first D columns.
// One tile is in flight, with two 256-column accumulators: layer L writes
// accumulator L % 2, so the MMAs of layer L + 1 start on K-chunk kc as soon
// as the epilogue of layer L has written it (barrier hb[kc]) while the
// epilogue goes on with the next chunks.  Shared memory holds one tile's
// activations (64 KB) and the weight ring.  The weights (the same 296 KB for
// every tile, read by every SM from L2) move in 32 KB copies: on GB300 one
// SM's bulk copies complete one after another at about a quarter
// microsecond each up to tens of KB, so per-SM throughput grows with the copy
// size (16 KB copies: about 63 KB/us, 32 KB: about 130 KB/us), not with the
// number in flight.  The CTA takes tiles b, b + G, b + 2G, ...
//
// Synchronisation (L = 4 i + l: layer l of the CTA's i-th tile):
//   afull      tcgen05.commit after the MMAs of layer L (completion L);
//   accfree[b] 512 arrivals: accumulator b read by the epilogue of layer L
//              (b = L % 2, completion L / 2);
//   hb[kc]     512 arrivals: K-chunk kc of the activations written by a
//              hidden-layer epilogue (completion 3 i + l);
//   a0r        512 arrivals: the tile's input block written (completion i);
//   full/empty[stage]  weight ring (bulk-copy bytes / MMA commit).
// Every wait is bounded: a wait that runs out sets the abort flag and the
// error flag, every role then leaves its loop, the copies and MMAs in flight
// are waited for (again bounded) and the tensor memory is freed.
//
// SiLU here is z sigma(z) = h (1 + tanh h) with h = z / 2 and the hardware
// tanh approximation (relative error about 2^-11, far below the BF16
// rounding of the activation it produces).

constexpr int F_EW = 16;                         // epilogue warps
constexpr int F_ET = F_EW * 32;                  // epilogue threads
constexpr int F_THREADS = F_ET + 64;             // + weight producer warp + MMA warp
constexpr int F_CHUNK = 16384;                   // bytes of one 128-row x 64-K weight block
constexpr int F_NCHUNK = 19;                     // blocks: W1 2, W2 8, W3 8, W4 1 (8 KB)
constexpr int F_COPY = 2 * F_CHUNK;              // bytes of one copy: both 128-row halves of a K-chunk
constexpr int F_NCOPY = 10;                      // copies per tile: W1 1, W2 4, W3 4, W4 1 (8 KB)
constexpr int F_HBYTES = 4 * 16384;              // activations of one tile: 4 K-chunks of 128 x 64 BF16
constexpr int F_BIAS_FLOATS = 3 * 256 + 16;
constexpr int F_STAGES = (227 * 1024 - 1024 - F_HBYTES - F_BIAS_FLOATS * 4) / F_COPY;
constexpr size_t F_SMEM = F_HBYTES + F_STAGES * F_COPY + F_BIAS_FLOATS * 4;
constexpr size_t F_WPACK_BYTES = 18 * (size_t)F_CHUNK + 8192;

// Packed pairs of FP32 values (f32x2 instructions; each half rounded as the
// scalar instruction).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


// Wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool fwait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t n = 0;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 63u) == 63u) {
      if (*abort) return false;
      if (global_timer_ns() - t0 > VDS_WAIT_LIMIT_NS) {
        *abort = 1;
        return false;
      }
    }
  }
}

// copies of layer l: 1, 4, 4, 1 (copy j covers blocks 2j and 2j + 1)
__host__ __device__ constexpr int f_ncopies(int l) { return (l == 0 || l == 3) ? 1 : 4; }
static_assert(2 * (F_NCOPY - 1) + 1 == F_NCHUNK, "weight stream length");
static_assert(F_STAGES >= 4, "weight ring depth");
static_assert(F_SMEM <= 227 * 1024 - 1024, "shared memory of k_mlp_fwd");

// Packed weight stream: chunk j holds, in the canonical K-major layout
// ((r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2 bytes), rows 128 nh .. of W1
// (j = nh), of W2 (j = 2 + 2 kc + nh, K columns 64 kc ..) or W3 (j = 10 +
// ...); chunk 18 is W4 (16 rows) as four 2 KB blocks of 64 K columns.
__global__ void k_pack_w(const bf16 *__restrict__ w1, const bf16 *__restrict__ w2, const bf16 *__restrict__ w3,
                         const bf16 *__restrict__ w4, int Dp, int W, bf16 *__restrict__ pack) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)(F_WPACK_BYTES / 2)) return;
  const int j = (int)(e / (F_CHUNK / 2));
  int b = (int)(e - (long)j * (F_CHUNK / 2)) * 2;  // byte inside the chunk
  int sub = 0;
  if (j == 18) {
    sub = b >> 11;
    b &= 2047;
  }
  const int g = b >> 10, c = (b >> 7) & 7, r8 = (b >> 4) & 7, k8 = (b >> 1) & 7;
  const int r = g * 8 + r8, k = c * 8 + k8;
  bf16 v;
  if (j < 2) {
    v = w1[(size_t)(j * 128 + r) * Dp + k];
  } else if (j < 18) {
    const int jj = (j - 2) & 7, kc = jj >> 1, nh = jj & 1;
    const bf16 *w = j < 10 ? w2 : w3;
    v = w[(size_t)(nh * 128 + r) * W + kc * 64 + k];
  } else {
    v = w4[(size_t)r * W + sub * 64 + k];
  }
  pack[e] = v;
}

__global__ void __launch_bounds__(F_THREADS, 1)
    k_mlp_fwd(const float *__restrict__ x, int N, int D, const bf16 *__restrict__ wpack,
              const float *__restrict__ b1, const float *__restrict__ b2, const float *__restrict__ b3,
              const float *__restrict__ b4, float *__restrict__ out, int *err) {
  extern __shared__ __align__(1024) uint8_t fsm[];
  __shared__ __align__(8) uint64_t full[F_STAGES], empty[F_STAGES], afull, accfree[2], hb[4], a0r, fin;
  static_assert(F_STAGES <= 8, "barrier array size");
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (N + GM - 1) / GM;
  const int G = gridDim.x;
  const int nk = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;  // tiles of this CTA
  uint8_t *hbuf = fsm;                                  // 64 KB activations
  uint8_t *ring = fsm + F_HBYTES;                       // weight stages
  float *sbias = reinterpret_cast<float *>(ring + F_STAGES * F_COPY);
  volatile int *abort = &s_abort;

  if (warp == 0) tc_alloc(&s_tmem, 512);
  if (tid == 0) {
    for (int k = 0; k < F_STAGES; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    mbar_init(&afull, 1);
    // one arrival per epilogue warp (its lanes synchronised first): 16
    // arrivals per barrier phase instead of 512 atomics on one word
    for (int k = 0; k < 2; ++k) mbar_init(&accfree[k], F_EW);
    for (int k = 0; k < 4; ++k) mbar_init(&hb[k], F_EW);
    mbar_init(&a0r, F_EW);
    mbar_init(&fin, 1);
    s_abort = 0;
    fence_mbar_init();
  }
  for (int i = tid; i < F_BIAS_FLOATS; i += F_THREADS)
    sbias[i] = i < 256 ? b1[i] : (i < 512 ? b2[i - 256] : (i < 768 ? b3[i - 512] : (i - 768 < D ? b4[i - 768] : 0.f)));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto tile_of = [&](int i) { return (int)blockIdx.x + i * G; };

  if (warp == F_EW) {
    // ------------------------------------------------ weight producer
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int i = 0; i < nk && ok; ++i)
        for (int j = 0; j < F_NCOPY; ++j, ++g) {
          const uint32_t st = g % F_STAGES;
          if (g >= F_STAGES && !fwait(&empty[st], ((g / F_STAGES) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          const uint32_t bytes = j == F_NCOPY - 1 ? 8192u : (uint32_t)F_COPY;
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(ring + st * F_COPY, reinterpret_cast<const uint8_t *>(wpack) + (size_t)j * F_COPY, bytes,
                   &full[st]);
        }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
      // the copies still in flight land before the CTA may exit
      for (uint32_t k = g > F_STAGES ? g - F_STAGES : 0; k < g; ++k)
        mbar_wait_bounded(&full[k % F_STAGES], (k / F_STAGES) & 1, VDS_WAIT_LIMIT_NS);
    }
  } else if (warp == F_EW + 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id256 = tc_idesc(TC_FMT_BF16, GM, 256), id16 = tc_idesc(TC_FMT_BF16, GM, 16);
      const uint32_t hb0 = smem_u32(hbuf), rb = smem_u32(ring);
      uint32_t g = 0;
      bool ok = true;
      for (int i = 0; i < nk && ok; ++i)
        for (int l = 0; l < 4 && ok; ++l) {
          const int L = 4 * i + l, b = L & 1;
          const uint32_t d = tmem + (uint32_t)(b * 256);
          // the epilogue of layer L - 2 has read this accumulator
          if (L >= 2 && !fwait(&accfree[b], (uint32_t)(((L >> 1) - 1) & 1), abort)) {
            ok = false;
            break;
          }
          if (l == 0 && !fwait(&a0r, (uint32_t)(i & 1), abort)) {
            ok = false;
            break;
          }
          const uint32_t hpar = (uint32_t)((3 * i + l - 1) & 1);  // hidden epilogue 3 i + l - 1
          for (int jj = 0; jj < f_ncopies(l) && ok; ++jj, ++g) {
            const uint32_t st = g % F_STAGES;
            if (!fwait(&full[st], (g / F_STAGES) & 1, abort)) {
              ok = false;
              break;
            }
            const uint32_t wb = rb + st * F_COPY;
            if (l == 3) {
#pragma unroll 1
              for (int kc = 0; kc < 4 && ok; ++kc) {
                if (!fwait(&hb[kc], hpar, abort)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  tc_mma_bf16(d, tc_sdesc(hb0 + kc * 16384 + k * 256), tc_sdesc(wb + kc * 2048 + k * 256), id16,
                              (kc > 0 || k > 0) ? 1 : 0);
              }
            } else {
              const int kc = jj;  // K-chunk; the copy holds both 128-row halves of the weights
              if (l > 0 && !fwait(&hb[kc], hpar, abort)) {
                ok = false;
                break;
              }
              tc_fence_after();
              // rows 128..255 of the weights follow rows 0..127 at the next
              // 8-row group (F_CHUNK bytes on): one operand of 256 rows
#pragma unroll
              for (int k = 0; k < 4; ++k)
                tc_mma_bf16(d, tc_sdesc(hb0 + kc * 16384 + k * 256), tc_sdesc(wb + k * 256), id256,
                            (kc > 0 || k > 0) ? 1 : 0);
            }
            tc_commit(&empty[st]);
          }
          if (ok) tc_commit(&afull);
        }
      if (!ok) vds_flag(err, VDS_ETIMEOUT);
    }
  } else {
    // ------------------------------------------------ epilogue warps 0-15
    const int q = warp & 3, cp = warp >> 2;
    const int rl = q * 32 + lane;                       // accumulator row of this thread
    const int ar = tid & 127, ag = tid >> 7;            // input row and 8-column group (ag, ag + 4)
    float xp[8];
    auto fetch_x = [&](int tile) {
      const int row = tile * GM + ar;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = ag * 8 + u;
        xp[u] = (row < N && k < D && ag < 2) ? x[(size_t)row * D + k] : 0.f;
      }
    };
    // A0 = bf16(x) padded to 64 columns, into K-chunk 0 of the activations
    auto put_a0 = [&]() {
      uint8_t *h = hbuf + (ar >> 3) * 1024 + (ar & 7) * 16;
      uint32_t pk[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 t = __floats2bfloat162_rn(xp[2 * u], xp[2 * u + 1]);
        pk[u] = *reinterpret_cast<const uint32_t *>(&t);
      }
      *reinterpret_cast<uint4 *>(h + ag * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      *reinterpret_cast<uint4 *>(h + (ag + 4) * 128) = make_uint4(0, 0, 0, 0);
    };
    auto warp_arrive = [&](uint64_t *bar) {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar);
    };
    if (nk > 0) {
      fetch_x(tile_of(0));
      put_a0();
      fence_proxy_async_smem();
      warp_arrive(&a0r);
    }
    bool ok = true;
    for (int i = 0; i < nk && ok; ++i)
      for (int l = 0; l < 4 && ok; ++l) {
        const int L = 4 * i + l, b = L & 1;
        ok = __all_sync(0xffffffffu, fwait(&afull, (uint32_t)(L & 1), abort));
        if (!ok) break;
        tc_fence_after();
        const uint32_t ta = tmem + (uint32_t)(b * 256) + ((uint32_t)(q * 32) << 16);
        const bool next = i + 1 < nk;
        if (l < 3) {
          if (l == 2 && next) fetch_x(tile_of(i + 1));
          const float *bias = sbias + l * 256;
          uint8_t *h = hbuf + (rl >> 3) * 1024 + (rl & 7) * 16 + cp * 2 * 128;
#pragma unroll 1
          for (int kc = 0; kc < 4; ++kc) {
            uint32_t v[16];
            const int c0 = kc * 64 + cp * 16;
            tc_ld16(ta + (uint32_t)c0, v);
            uint32_t pk[8];
            // two columns per f32x2 instruction (each half rounded as the
            // scalar operation): adjacent accumulator columns and biases
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const unsigned long long b2 = *reinterpret_cast<const unsigned long long *>(bias + c0 + 2 * u);
              const unsigned long long h2 =
                  f2_mul(f2_add(f2_pack(__uint_as_float(v[2 * u]), __uint_as_float(v[2 * u + 1])), b2),
                         f2_pack(0.5f, 0.5f));
              float h0, h1;
              f2_unpack(h2, h0, h1);
              float y0, y1;
              f2_unpack(f2_fma(h2, f2_pack(tanh_approx(h0), tanh_approx(h1)), h2), y0, y1);
              const __nv_bfloat162 t = __floats2bfloat162_rn(y0, y1);
              pk[u] = *reinterpret_cast<const uint32_t *>(&t);
            }
            uint8_t *hk = h + kc * 16384;
            *reinterpret_cast<uint4 *>(hk) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4 *>(hk + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            // this K-chunk is the next layer's operand as soon as every thread wrote it
            fence_proxy_async_smem();
            warp_arrive(&hb[kc]);
          }
        } else {
          // the output layer's MMAs have read the activations: the next tile's input may go in
          if (next) {
            put_a0();
            fence_proxy_async_smem();
            warp_arrive(&a0r);
          }
          if (cp == 0) {
            uint32_t v[16];
            tc_ld16(ta, v);
            const int row = tile_of(i) * GM + rl;
            if (row < N) {
              const float *bias = sbias + 768;
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (j < D) out[(size_t)row * D + j] = __uint_as_float(v[j]) + bias[j];
            }
          }
        }
        tc_fence_before();
        warp_arrive(&accfree[b]);
      }
    if (!ok && tid == 0) vds_flag(err, VDS_ETIMEOUT);
  }
  // every role has left its loop; the MMAs issued are complete before the
  // tensor memory is released
  tc_fence_before();
  __syncthreads();
  if (warp == F_EW + 1 && lane == 0) {
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

struct vds_score {
  int device = 0, D = 0, W = 0, Dp = 64, Op = 16;
  long long off[8] = {};  // W1 b1 W2 b2 W3 b3 W4 b4 in the flat padded parameter vector
  long long np = 0;
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  bf16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w4b = nullptr;
  bf16 *w2t = nullptr, *w3t = nullptr, *w4t = nullptr;  // transposes (w4t: W x 64, K padded)
  bf16 *wpack = nullptr;  // weight stream of the fused inference kernel (F_WPACK_BYTES)
  bool packed = false;    // wpack matches the current BF16 weights
  int t = 0;
  int mcap = 0;
  // activations for up to mcap rows
  bf16 *a0 = nullptr, *a0t = nullptr, *h[3] = {}, *ht[3] = {}, *dzb[2] = {}, *dzt[2] = {}, *dsb = nullptr,
       *dst = nullptr;
  float *z[3] = {}, *dzf[2] = {}, *sf = nullptr, *dsf = nullptr, *part = nullptr;
  double *lossp = nullptr, *h_loss = nullptr;
};

namespace {

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

// Tensor map of a row-major BF16 matrix (rows x K used, row stride ld
// elements) in boxes of 64 K x box_rows rows, 128-byte swizzled, rows and K
// past the matrix read as zeros.
// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library does not link the driver library itself, so it loads without one)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int make_tmap(CUtensorMap *m, const bf16 *base, int rows, int K, int ld, int box_rows) {
  if (((uintptr_t)base & 15) != 0 || (ld * 2) % 16 != 0) return VDS_EARG;
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return VDS_ECUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(base), dims,
                                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? VDS_OK : VDS_ECUDA;
}

int gemm(vds_ctx *c, const bf16 *A, int lda, const bf16 *B, int ldb, int rows, int N, int K, int splits,
         const Epi &ep) {
  if (N % 16 != 0 || N < 16 || N > 256 || K % (KC * splits) != 0) return VDS_EARG;
  // per device: the shared-memory attribute is a property of the function on that device
  static bool attr[VDS_MAX_DEVICES] = {};
  if (c->device >= VDS_MAX_DEVICES || !attr[c->device]) {
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * GSTAGE));
    VDS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * GSTAGE));
    if (c->device < VDS_MAX_DEVICES) attr[c->device] = true;
  }
  const int boxB = N < GBN ? N : GBN;
  CUtensorMap tA, tB;
  VDS_TRY(make_tmap(&tA, A, rows, K, lda, GM));
  VDS_TRY(make_tmap(&tB, B, N, K, ldb, boxB));
  dim3 grid((rows + GM - 1) / GM, splits, (N + GBN - 1) / GBN);
  const int nch = K / splits / KC;
  if (nch <= 4)
    k_gemm_tma<2><<<grid, GNT, 2 * GSTAGE, c->stream>>>(tA, tB, N, K / splits, boxB, ep, c->err);
  else
    k_gemm_tma<4><<<grid, GNT, 4 * GSTAGE, c->stream>>>(tA, tB, N, K / splits, boxB, ep, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

Epi epi_f32(int rows, int ncols, int ldc, const float *bias, float *out, long long split_stride = 0) {
  Epi e;
  memset(&e, 0, sizeof(e));
  e.mode = EPI_F32;
  e.rows = rows;
  e.ncols = ncols;
  e.ldc = ldc;
  e.bias = bias;
  e.outf = out;
  e.split_stride = split_stride;
  return e;
}

Epi epi_act(int mode, int rows, int ncols, int ldc, const float *bias, float *outf, bf16 *h, bf16 *ht, int ldt,
            const float *zin) {
  Epi e;
  memset(&e, 0, sizeof(e));
  e.mode = mode;
  e.rows = rows;
  e.ncols = ncols;
  e.ldc = ldc;
  e.bias = bias;
  e.outf = outf;
  e.h = h;
  e.ht = ht;
  e.ldt = ldt;
  e.zin = zin;
  return e;
}

void free_acts(vds_score *s) {
  void *ptrs[] = {s->a0, s->a0t, s->h[0], s->h[1], s->h[2], s->ht[0], s->ht[1], s->ht[2], s->dzb[0], s->dzb[1],
                  s->dzt[0], s->dzt[1], s->dsb, s->dst, s->z[0], s->z[1], s->z[2], s->dzf[0], s->dzf[1], s->sf,
                  s->dsf, s->part, s->lossp};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  s->a0 = s->a0t = s->dsb = s->dst = nullptr;
  for (int k = 0; k < 3; ++k) s->h[k] = s->ht[k] = nullptr, s->z[k] = nullptr;
  for (int k = 0; k < 2; ++k) s->dzb[k] = s->dzt[k] = nullptr, s->dzf[k] = nullptr;
  s->sf = s->dsf = s->part = nullptr;
  s->lossp = nullptr;
  s->mcap = 0;
}

int ensure_acts(vds_score *s, int M) {
  if (M <= s->mcap) return VDS_OK;
  free_acts(s);
  const int Mc = (M + 127) / 128 * 128;
  const size_t W = s->W;
  cudaError_t ce = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMalloc(p, bytes);
  };
  A((void **)&s->a0, sizeof(bf16) * Mc * s->Dp);
  A((void **)&s->a0t, sizeof(bf16) * Mc * s->Dp);
  for (int k = 0; k < 3; ++k) {
    A((void **)&s->h[k], sizeof(bf16) * Mc * W);
    A((void **)&s->ht[k], sizeof(bf16) * Mc * W);
    A((void **)&s->z[k], sizeof(float) * Mc * W);
  }
  for (int k = 0; k < 2; ++k) {
    A((void **)&s->dzb[k], sizeof(bf16) * Mc * W);
    A((void **)&s->dzt[k], sizeof(bf16) * Mc * W);
    A((void **)&s->dzf[k], sizeof(float) * Mc * W);
  }
  A((void **)&s->dsb, sizeof(bf16) * Mc * 64);
  A((void **)&s->dst, sizeof(bf16) * Mc * s->Op);
  A((void **)&s->sf, sizeof(float) * Mc * s->Op);
  A((void **)&s->dsf, sizeof(float) * Mc * s->Op);
  A((void **)&s->part, sizeof(float) * 64 * W * W);
  A((void **)&s->lossp, sizeof(double) * (Mc / 256 + 1));
  if (ce != cudaSuccess) {
    vds_last_cuda_error(ce);
    free_acts(s);
    return ce == cudaErrorMemoryAllocation ? VDS_ENOMEM : VDS_ECUDA;
  }
  s->mcap = Mc;
  return VDS_OK;
}

int refresh_bf16(vds_ctx *c, vds_score *s) {
  const int W = s->W;
  auto conv = [&](const float *src, int rows, int cols, bf16 *dst, bf16 *dt, int tcols) -> int {
    const long n = (long)rows * cols > (long)cols * tcols ? (long)rows * cols : (long)cols * tcols;
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(src, rows, cols, dst, dt, tcols);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    return VDS_OK;
  };
  VDS_TRY(conv(s->p + s->off[0], W, s->Dp, s->w1b, nullptr, 0));
  VDS_TRY(conv(s->p + s->off[2], W, W, s->w2b, s->w2t, W));
  VDS_TRY(conv(s->p + s->off[4], W, W, s->w3b, s->w3t, W));
  VDS_TRY(conv(s->p + s->off[6], s->Op, W, s->w4b, s->w4t, 64));
  s->packed = false;  // repacked by the next inference call
  return VDS_OK;
}

// forward for M rows (A0 built); train keeps Z/H^T for the backward pass
int forward(vds_ctx *c, vds_score *s, int M, bool train, float *out, int ldo, int ncols_out) {
  const int W = s->W;
  const float *b1 = s->p + s->off[1], *b2 = s->p + s->off[3], *b3 = s->p + s->off[5], *b4 = s->p + s->off[7];
  const int Mc = s->mcap;
  VDS_TRY(gemm(c, s->a0, s->Dp, s->w1b, s->Dp, M, W, s->Dp, 1,
               epi_act(EPI_SILU, M, W, W, b1, train ? s->z[0] : nullptr, s->h[0], train ? s->ht[0] : nullptr, Mc,
                       nullptr)));
  VDS_TRY(gemm(c, s->h[0], W, s->w2b, W, M, W, W, 1,
               epi_act(EPI_SILU, M, W, W, b2, train ? s->z[1] : nullptr, s->h[1], train ? s->ht[1] : nullptr, Mc,
                       nullptr)));
  VDS_TRY(gemm(c, s->h[1], W, s->w3b, W, M, W, W, 1,
               epi_act(EPI_SILU, M, W, W, b3, train ? s->z[2] : nullptr, s->h[2], train ? s->ht[2] : nullptr, Mc,
                       nullptr)));
  VDS_TRY(gemm(c, s->h[2], W, s->w4b, W, M, s->Op, W, 1, epi_f32(M, ncols_out, ldo, b4, out)));
  return VDS_OK;
}

// loss and gradients (flat padded vector s->g) for a batch of M rows
int loss_grad(vds_ctx *c, vds_score *s, const float *x, const int *rows, const float *eps, int M, double sigma,
              double *loss, const float *target = nullptr) {
  const int W = s->W, Mc = s->mcap;
  k_input<<<(unsigned)(((long)M * s->Dp + 255) / 256), 256, 0, c->stream>>>(x, rows, target ? nullptr : eps,
                                                                           (float)sigma, M, s->D, s->Dp, s->a0,
                                                                           s->a0t, Mc);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_TRY(forward(c, s, M, true, s->sf, s->Op, s->Op));
  const int nb = (M + 255) / 256;
  if (target)
    k_fit_out<<<nb, 256, 0, c->stream>>>(s->sf, s->Op, target, rows, M, s->D, s->dsf, s->Op, s->dsb, 64, s->dst,
                                         Mc, s->lossp);
  else
    k_dsm_out<<<nb, 256, 0, c->stream>>>(s->sf, s->Op, eps, (float)sigma, M, s->D, s->dsf, s->Op, s->dsb, 64,
                                         s->dst, Mc, s->lossp);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  // split-K over the batch for the weight gradients
  // (at most 16 splits: more write more FP32 partials than their MMAs save)
  int splits = M / KC;
  while (splits > 16 || (M % (KC * splits)) != 0) --splits;
  if (splits < 1) splits = 1;
  auto wgrad = [&](const bf16 *At, int rows, const bf16 *Bt, int N, float *dst) -> int {
    const long long stride = (long long)rows * N;
    VDS_TRY(gemm(c, At, Mc, Bt, Mc, rows, N, M, splits, epi_f32(rows, N, N, nullptr, s->part, stride)));
    k_split_reduce<<<(unsigned)((stride + 255) / 256), 256, 0, c->stream>>>(s->part, splits, stride, stride, dst);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    return VDS_OK;
  };
  auto bgrad = [&](const float *X, int n, int ld, float *dst) -> int {
    k_colsum<<<n, 512, 0, c->stream>>>(X, M, n, ld, dst);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    return VDS_OK;
  };
  // layer 4
  VDS_TRY(wgrad(s->dst, s->Op, s->ht[2], W, s->g + s->off[6]));
  VDS_TRY(bgrad(s->dsf, s->Op, s->Op, s->g + s->off[7]));
  // dZ3 = (dS W4) * silu'(Z3)
  VDS_TRY(gemm(c, s->dsb, 64, s->w4t, 64, M, W, 64, 1,
               epi_act(EPI_DSILU, M, W, W, nullptr, s->dzf[0], s->dzb[0], s->dzt[0], Mc, s->z[2])));
  VDS_TRY(wgrad(s->dzt[0], W, s->ht[1], W, s->g + s->off[4]));
  VDS_TRY(bgrad(s->dzf[0], W, W, s->g + s->off[5]));
  // dZ2 = (dZ3 W3) * silu'(Z2)
  VDS_TRY(gemm(c, s->dzb[0], W, s->w3t, W, M, W, W, 1,
               epi_act(EPI_DSILU, M, W, W, nullptr, s->dzf[1], s->dzb[1], s->dzt[1], Mc, s->z[1])));
  VDS_TRY(wgrad(s->dzt[1], W, s->ht[0], W, s->g + s->off[2]));
  VDS_TRY(bgrad(s->dzf[1], W, W, s->g + s->off[3]));
  // dZ1 = (dZ2 W2) * silu'(Z1)
  VDS_TRY(gemm(c, s->dzb[1], W, s->w2t, W, M, W, W, 1,
               epi_act(EPI_DSILU, M, W, W, nullptr, s->dzf[0], s->dzb[0], s->dzt[0], Mc, s->z[0])));
  VDS_TRY(wgrad(s->dzt[0], W, s->a0t, s->Dp, s->g + s->off[0]));
  VDS_TRY(bgrad(s->dzf[0], W, W, s->g + s->off[1]));
  if (loss) {
    std::vector<double> lp(nb);
    VDS_CUDA_TRY(cudaMemcpyAsync(lp.data(), s->lossp, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
    VDS_TRY(vds_sync_status(c));
    double a = 0.0;
    for (int k = 0; k < nb; ++k) a += lp[k];
    *loss = a / (double)M;
  }
  return VDS_OK;
}

// flat unpadded parameter layout: W1 (W x D), b1 (W), W2 (W x W), b2, W3, b3,
// W4 (D x W), b4 (D)
long long flat_count(int D, int W) { return (long long)W * D + W + 2LL * (W * W + W) + (long long)D * W + D; }

void pad_params(const vds_score *s, const float *in, std::vector<float> &out) {
  const int D = s->D, W = s->W;
  out.assign(s->np, 0.f);
  long long k = 0;
  for (int r = 0; r < W; ++r)
    for (int cc = 0; cc < D; ++cc) out[s->off[0] + (long long)r * s->Dp + cc] = in[k++];
  for (int r = 0; r < W; ++r) out[s->off[1] + r] = in[k++];
  for (int l = 0; l < 2; ++l) {
    for (long long e = 0; e < (long long)W * W; ++e) out[s->off[2 + 2 * l] + e] = in[k++];
    for (int r = 0; r < W; ++r) out[s->off[3 + 2 * l] + r] = in[k++];
  }
  for (int r = 0; r < D; ++r)
    for (int cc = 0; cc < W; ++cc) out[s->off[6] + (long long)r * W + cc] = in[k++];
  for (int r = 0; r < D; ++r) out[s->off[7] + r] = in[k++];
}

void unpad_params(const vds_score *s, const std::vector<float> &in, float *out) {
  const int D = s->D, W = s->W;
  long long k = 0;
  for (int r = 0; r < W; ++r)
    for (int cc = 0; cc < D; ++cc) out[k++] = in[s->off[0] + (long long)r * s->Dp + cc];
  for (int r = 0; r < W; ++r) out[k++] = in[s->off[1] + r];
  for (int l = 0; l < 2; ++l) {
    for (long long e = 0; e < (long long)W * W; ++e) out[k++] = in[s->off[2 + 2 * l] + e];
    for (int r = 0; r < W; ++r) out[k++] = in[s->off[3 + 2 * l] + r];
  }
  for (int r = 0; r < D; ++r)
    for (int cc = 0; cc < W; ++cc) out[k++] = in[s->off[6] + (long long)r * W + cc];
  for (int r = 0; r < D; ++r) out[k++] = in[s->off[7] + r];
}

}  // namespace

extern "C" {

int vds_score_create(vds_ctx *c, int D, int width, const float *params, vds_score **out) {
  if (!c || !out || !params || D < 1 || D > 16 || width != 256) return VDS_EARG;
  *out = nullptr;
  Dev dg(c->device);
  vds_score *s = new vds_score();
  s->device = c->device;
  s->D = D;
  s->W = width;
  const int W = width;
  long long o = 0;
  s->off[0] = o; o += (long long)W * s->Dp;
  s->off[1] = o; o += W;
  s->off[2] = o; o += (long long)W * W;
  s->off[3] = o; o += W;
  s->off[4] = o; o += (long long)W * W;
  s->off[5] = o; o += W;
  s->off[6] = o; o += (long long)s->Op * W;
  s->off[7] = o; o += s->Op;
  s->np = o;
  cudaError_t ce = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (ce == cudaSuccess) ce = cudaMalloc(p, bytes);
  };
  A((void **)&s->p, sizeof(float) * o);
  A((void **)&s->m, sizeof(float) * o);
  A((void **)&s->v, sizeof(float) * o);
  A((void **)&s->g, sizeof(float) * o);
  A((void **)&s->w1b, sizeof(bf16) * W * s->Dp);
  A((void **)&s->w2b, sizeof(bf16) * W * W);
  A((void **)&s->w3b, sizeof(bf16) * W * W);
  A((void **)&s->w4b, sizeof(bf16) * s->Op * W);
  A((void **)&s->w2t, sizeof(bf16) * W * W);
  A((void **)&s->w3t, sizeof(bf16) * W * W);
  A((void **)&s->w4t, sizeof(bf16) * W * 64);
  A((void **)&s->wpack, F_WPACK_BYTES);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->m, 0, sizeof(float) * o, c->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->v, 0, sizeof(float) * o, c->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->g, 0, sizeof(float) * o, c->stream);
  if (ce != cudaSuccess) {
    vds_last_cuda_error(ce);
    vds_score_free(s);
    return ce == cudaErrorMemoryAllocation ? VDS_ENOMEM : VDS_ECUDA;
  }
  int st = vds_score_set_params(c, s, params);
  if (st != VDS_OK) {
    vds_score_free(s);
    return st;
  }
  *out = s;
  return VDS_OK;
}

void vds_score_free(vds_score *s) {
  if (!s) return;
  Dev dg(s->device);
  free_acts(s);
  void *ptrs[] = {s->p, s->m, s->v, s->g, s->w1b, s->w2b, s->w3b, s->w4b, s->w2t, s->w3t, s->w4t, s->wpack};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

long vds_score_param_count(int D, int width) { return (long)flat_count(D, width); }

int vds_score_set_params(vds_ctx *c, vds_score *s, const float *params) {
  if (!c || !s || !params) return VDS_EARG;
  Dev dg(c->device);
  std::vector<float> pad;
  pad_params(s, params, pad);
  VDS_CUDA_TRY(cudaMemcpyAsync(s->p, pad.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice, c->stream));
  VDS_CUDA_TRY(cudaMemsetAsync(s->m, 0, sizeof(float) * s->np, c->stream));
  VDS_CUDA_TRY(cudaMemsetAsync(s->v, 0, sizeof(float) * s->np, c->stream));
  s->t = 0;
  VDS_TRY(refresh_bf16(c, s));
  return vds_sync_status(c);
}

int vds_score_get_params(vds_ctx *c, const vds_score *s, float *params) {
  if (!c || !s || !params) return VDS_EARG;
  Dev dg(c->device);
  std::vector<float> pad(s->np);
  VDS_CUDA_TRY(cudaMemcpyAsync(pad.data(), s->p, sizeof(float) * s->np, cudaMemcpyDeviceToHost, c->stream));
  VDS_TRY(vds_sync_status(c));
  unpad_params(s, pad, params);
  return VDS_OK;
}

int vds_score_eval(vds_ctx *c, vds_score *s, const float *x, int N, float *out) {
  if (!c || !s || !x || !out || N < 1) return VDS_EARG;
  Dev dg(c->device);
  if (s->W == 256 && s->Dp == 64 && s->Op == 16) {
    // all four layers in one persistent launch (k_mlp_fwd)
    static bool attr[VDS_MAX_DEVICES] = {};
    if (c->device >= VDS_MAX_DEVICES || !attr[c->device]) {
      VDS_CUDA_TRY(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F_SMEM));
      if (c->device < VDS_MAX_DEVICES) attr[c->device] = true;
    }
    if (!s->packed) {
      const long ne = (long)(F_WPACK_BYTES / 2);
      k_pack_w<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>(s->w1b, s->w2b, s->w3b, s->w4b, s->Dp, s->W,
                                                                    s->wpack);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
      s->packed = true;
    }
    const int ntiles = (N + GM - 1) / GM;
    const int grid = ntiles < c->num_sms ? ntiles : c->num_sms;
    k_mlp_fwd<<<grid, F_THREADS, F_SMEM, c->stream>>>(x, N, s->D, s->wpack, s->p + s->off[1], s->p + s->off[3],
                                                      s->p + s->off[5], s->p + s->off[7], out, c->err);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    return VDS_OK;
  }
  const int chunk = 65536;
  VDS_TRY(ensure_acts(s, N < chunk ? N : chunk));
  for (int n0 = 0; n0 < N; n0 += chunk) {
    const int M = (N - n0) < chunk ? (N - n0) : chunk;
    k_input<<<(unsigned)(((long)M * s->Dp + 255) / 256), 256, 0, c->stream>>>(x + (size_t)n0 * s->D, nullptr,
                                                                             nullptr, 0.f, M, s->D, s->Dp, s->a0,
                                                                             nullptr, 0);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    VDS_TRY(forward(c, s, M, false, out + (size_t)n0 * s->D, s->D, s->D));
  }
  return VDS_OK;
}

int vds_score_loss_grad(vds_ctx *c, vds_score *s, const float *x, const int *rows, const float *eps, int M,
                        double sigma, double *loss, float *grads) {
  if (!c || !s || !x || !eps || M < 128 || M % 128 != 0 || !(sigma > 0.0)) return VDS_EARG;
  Dev dg(c->device);
  VDS_TRY(ensure_acts(s, M));
  VDS_TRY(loss_grad(c, s, x, rows, eps, M, sigma, loss));
  if (grads) {
    std::vector<float> pad(s->np);
    VDS_CUDA_TRY(cudaMemcpyAsync(pad.data(), s->g, sizeof(float) * s->np, cudaMemcpyDeviceToHost, c->stream));
    VDS_TRY(vds_sync_status(c));
    unpad_params(s, pad, grads);
  }
  return vds_sync_status(c);
}

int vds_score_train(vds_ctx *c, vds_score *s, const float *x, const int *rows, const float *eps, int M,
                    double sigma, double lr, double *loss) {
  if (!c || !s || !x || !eps || M < 128 || M % 128 != 0 || !(sigma > 0.0) || !(lr > 0.0)) return VDS_EARG;
  Dev dg(c->device);
  VDS_TRY(ensure_acts(s, M));
  VDS_TRY(loss_grad(c, s, x, rows, eps, M, sigma, loss));
  s->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)s->t), c2 = 1.f - powf(b2, (float)s->t);
  k_adam<<<(unsigned)((s->np + 255) / 256), 256, 0, c->stream>>>(s->p, s->m, s->v, s->g, s->np, (float)lr, b1, b2,
                                                                1e-8f, c1, c2);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_TRY(refresh_bf16(c, s));
  return loss ? vds_sync_status(c) : VDS_OK;
}

int vds_score_fit(vds_ctx *c, vds_score *s, const float *x, const int *rows, const float *target, int M, double lr,
                  double *loss, float *grads) {
  if (!c || !s || !x || !target || M < 128 || M % 128 != 0 || !(lr >= 0.0)) return VDS_EARG;
  Dev dg(c->device);
  VDS_TRY(ensure_acts(s, M));
  VDS_TRY(loss_grad(c, s, x, rows, nullptr, M, 1.0, loss, target));
  if (grads) {
    std::vector<float> pad(s->np);
    VDS_CUDA_TRY(cudaMemcpyAsync(pad.data(), s->g, sizeof(float) * s->np, cudaMemcpyDeviceToHost, c->stream));
    VDS_TRY(vds_sync_status(c));
    unpad_params(s, pad, grads);
  }
  if (lr > 0.0) {
    s->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)s->t), c2 = 1.f - powf(b2, (float)s->t);
    k_adam<<<(unsigned)((s->np + 255) / 256), 256, 0, c->stream>>>(s->p, s->m, s->v, s->g, s->np, (float)lr, b1,
                                                                  b2, 1e-8f, c1, c2);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    VDS_TRY(refresh_bf16(c, s));
  }
  return loss ? vds_sync_status(c) : VDS_OK;
}

}  // extern "C"
