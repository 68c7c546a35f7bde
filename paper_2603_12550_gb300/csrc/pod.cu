// pod.cu -- POD by the method of snapshots (Sec. 2.3, Sec. 3.1) and the
// project / lift maps of Eq. model_pq, for GB300 (sm_103a).
//
// pod_build:
//   C = X^T X            tensor cores, TF32 with one refinement step
//                        (3xTF32 split of every snapshot value) and FP64
//                        sums across 512-row segments (gram_tc.cu)
//   C = V Lambda V^T     two-sided cyclic Jacobi in FP64 with the round-robin
//                        ordering, one launch per round: each CTA computes
//                        the few of the round's M/2 disjoint rotations its
//                        tile needs (angles to FP32 accuracy, orthogonal to
//                        FP64 rounding), then applies them (blocks (a,b) of
//                        A' = R_a^T A_ab R_b, a <= b, with their mirror
//                        images; columns of V' = V R)
//   r                    energy rule on the sorted eigenvalues (FP64 prefix
//                        sums in descending order), or r_fixed
//   Phi = X V_r Lambda_r^(-1/2)   FP64 accumulation, stored FP32
//   Cholesky-QR          G = Phi^T Phi, G = L L^T, Phi <- Phi L^-T
//   sign                 largest-|.| entry of each column made positive
//   X^H = Phi^T (I (x) kappa) Phi (Sec. 2.4)
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pod_internal.cuh"



namespace {

struct KappaArg {
  double k[9];
};

// ------------------------------------------------------------------ Jacobi

__device__ __forceinline__ void jac_pair(int a, int rnd, int Mp, int &p, int &q) {
  if (a == 0) {
    p = rnd;
    q = Mp - 1;
  } else {
    p = (rnd + a) % (Mp - 1);
    q = (rnd - a + Mp - 1) % (Mp - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Rotation R = [[c, s], [-s, c]] on (p, q), the classical Jacobi rotation
// (the smaller angle, R^T A R zeroing the (p, q) entry) with its angle taken
// to FP32 accuracy: tan(theta) comes from the FP64 entries scaled by a power
// of two and rounded to FP32 (the FP64 divide and square root of this GPU are
// slow and on the critical path of every round); c and s are then promoted
// and normalised in FP64 by the series (c^2 + s^2)^(-1/2) = 1 - d/2 + 3d^2/8,
// d = c^2 + s^2 - 1 (|d| ~ 1e-7, the truncation ~ d^3 is below FP64
// rounding), so R is orthogonal to FP64 rounding and R^T A R a similarity.
// The (p, q) entry drops to ~1e-7 of itself instead of to zero; the next
// sweeps take it further, at the pace of the exact rotation's convergence.
__device__ __forceinline__ double2 jac_rot(const double *A, int M, int p, int q) {
  if (q >= M) return make_double2(1.0, 0.0);
  const double apq = A[(size_t)p * M + q];
  if (apq == 0.0) return make_double2(1.0, 0.0);
  const double dqp = A[(size_t)q * M + q] - A[(size_t)p * M + p];
  // scale both by 2^-e, e the exponent of apq (|apq 2^-e| in [1, 2)); the
  // scale is built from its bits (e in [-1022, 1022]; outside, apq is
  // subnormal or within a factor 2 of overflow, and the pair is left alone)
  const int e = ((__double2hiint(apq) >> 20) & 0x7ff) - 1023;
  if (e < -1022 || e > 1022) return make_double2(1.0, 0.0);
  const double sc = __hiloint2double((1023 - e) << 20, 0);
  const float a32 = (float)(apq * sc), d32 = (float)(dqp * sc);
  const float theta = d32 / (2.f * a32);
  float t;
  if (fabsf(theta) > 1e18f) t = 0.5f / theta;  // also theta = +-inf: t = 0
  else t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
  const float cf = 1.f / sqrtf(t * t + 1.f), sf = t * cf;
  const double c = cf, s = sf;
  const double d = (c * c + s * s) - 1.0;
  const double f = 1.0 + d * (-0.5 + 0.375 * d);
  return make_double2(c * f, s * f);
}

constexpr int JR_NT = 256;  // threads per CTA
constexpr int JT = 16;       // pairs per tile side
constexpr int JV_ROWS = 32;  // rows of V per tile (two per thread)

// One round of the cyclic Jacobi sweep in one launch.  The work is cut into
// tiles that need few rotations, so each CTA computes only those (into
// shared memory, one per thread, every CTA the same values for a pair):
//   CTAs [0, nAt): the JT x JT tiles (ta, tb), ta <= tb, of 2x2 blocks (a, b)
//     of A2 = R^T A R (rows of pair a, columns of pair b); a thread takes one
//     block with a <= b and writes it with its mirror image (A2 exactly
//     symmetric; a diagonal block writes its (p, q) value to (q, p));
//   CTAs [nAt, nAt + nVt): the JV_ROWS x JT tiles (rows i, pairs b) of
//     V2 = V R, two rows per thread.
__global__ void __launch_bounds__(JR_NT)
    k_jacobi_round(const double *__restrict__ A, double *__restrict__ A2, const double *__restrict__ V,
                   double *__restrict__ V2, int M, int Mp, int rnd, int nT, int nAt) {
  __shared__ double2 rot[2 * JT];
  constexpr int VR = JV_ROWS / (JR_NT / JT);  // rows of V per thread
  const int H = Mp / 2, tid = threadIdx.x;
  int bt = blockIdx.x;
  // Each thread loads its entries first; the rotations are computed while
  // those loads are in flight (the round's critical path is one L2 round
  // trip plus the rotation arithmetic, not their sum).
  if (bt < nAt) {
    int ta = 0;
    while (bt >= nT - ta) {  // upper-triangle tile index -> (ta, tb)
      bt -= nT - ta;
      ++ta;
    }
    const int tb = ta + bt;
    const int a = ta * JT + tid / JT, b = tb * JT + tid % JT;
    const bool act = a < H && b < H && a <= b;
    int p = 0, q = 0, p2 = 0, q2 = 0;
    double x00 = 0.0, x01 = 0.0, x10 = 0.0, x11 = 0.0;
    auto get = [&](int i, int j) -> double { return (i < M && j < M) ? A[(size_t)i * M + j] : 0.0; };
    if (act) {
      jac_pair(a, rnd, Mp, p, q);
      jac_pair(b, rnd, Mp, p2, q2);
      x00 = get(p, p2);
      x01 = get(p, q2);
      x10 = get(q, p2);
      x11 = get(q, q2);
    }
    if (tid < 2 * JT) {
      const int ar = (tid < JT ? ta : tb) * JT + (tid % JT);
      double2 r = make_double2(1.0, 0.0);
      if (ar < H) {
        int pr, qr;
        jac_pair(ar, rnd, Mp, pr, qr);
        r = jac_rot(A, M, pr, qr);
      }
      rot[tid] = r;
    }
    __syncthreads();
    if (!act) return;
    const double2 ra = rot[tid / JT], rb = rot[JT + tid % JT];
    const double ca = ra.x, sa = ra.y, cb = rb.x, sb = rb.y;
    const double t00 = ca * x00 - sa * x10, t01 = ca * x01 - sa * x11;
    const double t10 = sa * x00 + ca * x10, t11 = sa * x01 + ca * x11;
    const double y00 = t00 * cb - t01 * sb, y01 = t00 * sb + t01 * cb;
    const double y10 = t10 * cb - t11 * sb, y11 = t10 * sb + t11 * cb;
    auto put = [&](int i, int j, double v) {
      if (i < M && j < M) {
        A2[(size_t)i * M + j] = v;
        A2[(size_t)j * M + i] = v;
      }
    };
    if (a == b) {
      put(p, p, y00);
      put(p, q, y01);
      put(q, q, y11);
    } else {
      put(p, p2, y00);
      put(p, q2, y01);
      put(q, p2, y10);
      put(q, q2, y11);
    }
  } else {
    bt -= nAt;
    const int tb = bt % nT, ti = bt / nT;
    const int b = tb * JT + tid % JT;
    int p2 = 0, q2 = 0;
    double vp[VR], vq[VR];
    if (b < H) jac_pair(b, rnd, Mp, p2, q2);
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int i = ti * JV_ROWS + tid / JT + k * (JR_NT / JT);
      const bool ok = b < H && i < M;
      vp[k] = (ok && p2 < M) ? V[(size_t)i * M + p2] : 0.0;
      vq[k] = (ok && q2 < M) ? V[(size_t)i * M + q2] : 0.0;
    }
    if (tid < JT) {
      const int br = tb * JT + tid;
      double2 r = make_double2(1.0, 0.0);
      if (br < H) {
        int pr, qr;
        jac_pair(br, rnd, Mp, pr, qr);
        r = jac_rot(A, M, pr, qr);
      }
      rot[tid] = r;
    }
    __syncthreads();
    if (b >= H) return;
    const double2 rb = rot[tid % JT];
    const double cb = rb.x, sb = rb.y;
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int i = ti * JV_ROWS + tid / JT + k * (JR_NT / JT);
      if (i >= M) break;
      if (q2 >= M) {  // the dummy index of odd M: column p2 is carried over
        if (p2 < M) V2[(size_t)i * M + p2] = vp[k];
        continue;
      }
      V2[(size_t)i * M + p2] = vp[k] * cb - vq[k] * sb;
      V2[(size_t)i * M + q2] = vp[k] * sb + vq[k] * cb;
    }
  }
}

__global__ void k_identity(double *V, int M) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long)M * M) V[idx] = (idx / M == idx % M) ? 1.0 : 0.0;
}

// off-diagonal and total squared Frobenius norms -> scal[SC_AUX], scal[SC_AUX+1]
// (M <= 2048: int indices; the last CTA sums the per-CTA partials in a fixed
// order, one warp, lanes striding over the CTAs, then a fixed shuffle tree)
__global__ void __launch_bounds__(256)
    k_offnorm(const double *__restrict__ A, int M, double *red, unsigned *ticket, double *scal) {
  __shared__ double sh[8][2];
  __shared__ bool last;
  double off = 0.0, tot = 0.0;
  const int MM = M * M;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < MM; idx += gridDim.x * blockDim.x) {
    const double v = A[idx];
    const int i = idx / M;
    tot += v * v;
    if (idx != i * M + i) off += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5][0] = off;
    sh[threadIdx.x >> 5][1] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double o = 0.0, t = 0.0;
    for (int w = 0; w < 8; ++w) {
      o += sh[w][0];
      t += sh[w][1];
    }
    red[2 * blockIdx.x] = o;
    red[2 * blockIdx.x + 1] = t;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  double o = 0.0, t = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) {
    o += __ldcg(red + 2 * b);
    t += __ldcg(red + 2 * b + 1);
  }
  for (int k = 16; k > 0; k >>= 1) {
    o += __shfl_xor_sync(0xffffffffu, o, k);
    t += __shfl_xor_sync(0xffffffffu, t, k);
  }
  if (threadIdx.x == 0) {
    scal[SC_AUX] = o;
    scal[SC_AUX + 1] = t;
    *ticket = 0u;
  }
}

// ------------------------------------------------------- sort and rank rule

// Sort eigenvalues descending (ties: lower index first), choose r, and build
// W = V[:, order[t]] / sqrt(lambda_t) for t < r (M x 64, FP64).
__global__ void __launch_bounds__(1024)
    k_eig_sort(const double *__restrict__ A, const double *__restrict__ V, int M, double energy,
               int r_max, int r_fixed, double *lam_sorted, int *order, double *W, double *scal) {
  __shared__ int r_sh;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double li = A[(size_t)i * M + i];
    int rank = 0;
    for (int j = 0; j < M; ++j) {
      const double lj = A[(size_t)j * M + j];
      rank += (lj > li) || (lj == li && j < i);
    }
    order[rank] = i;
    lam_sorted[rank] = li;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < M; ++k) tot += lam_sorted[k];
    int r;
    if (r_fixed > 0) {
      r = r_fixed < M ? r_fixed : M;
    } else {
      r = M;
      double cum = 0.0;
      for (int k = 0; k < M; ++k) {
        cum += lam_sorted[k];
        if (cum >= energy * tot) {
          r = k + 1;
          break;
        }
      }
      if (r > r_max) r = r_max;
    }
    // modes whose eigenvalue is not resolved in FP64 cannot be normalised
    int rp = 0;
    while (rp < r && lam_sorted[rp] > 1e-13 * lam_sorted[0] && lam_sorted[rp] > 0.0) ++rp;
    scal[SC_AUX + 2] = (double)r;
    scal[SC_AUX + 3] = (double)rp;
    r_sh = rp;
  }
  __syncthreads();
  const int r = r_sh;
  for (int idx = threadIdx.x; idx < M * 64; idx += blockDim.x) {
    const int m = idx / 64, t = idx - (idx / 64) * 64;
    W[idx] = t < r ? V[(size_t)m * M + order[t]] / sqrt(lam_sorted[t]) : 0.0;
  }
}

// ---------------------------------------------------------------- basis

constexpr int BT = 16;  // basis columns per CTA
constexpr int BM = 128; // W rows staged per step

// Phi[row, t] = sum_m X[row + m Ns] W[m, t]  (FP64 accumulation)
__global__ void __launch_bounds__(256)
    k_basis(const float *__restrict__ X, long Ns, int M, const double *__restrict__ W, int r, int ld,
            float *__restrict__ phi) {
  __shared__ double Ws[BM][BT];
  const long row = (long)blockIdx.x * 256 + threadIdx.x;
  const int t0 = blockIdx.y * BT;
  double acc[BT];
#pragma unroll
  for (int t = 0; t < BT; ++t) acc[t] = 0.0;
  for (int m0 = 0; m0 < M; m0 += BM) {
    __syncthreads();
    for (int e = threadIdx.x; e < BM * BT; e += 256) {
      const int mm = e / BT, t = e - (e / BT) * BT;
      Ws[mm][t] = (m0 + mm < M) ? W[(size_t)(m0 + mm) * 64 + t0 + t] : 0.0;
    }
    __syncthreads();
    if (row < Ns) {
      const int mend = min(BM, M - m0);
      for (int mm = 0; mm < mend; ++mm) {
        const double x = (double)X[row + (long)(m0 + mm) * Ns];
#pragma unroll
        for (int t = 0; t < BT; ++t) acc[t] = fma(x, Ws[mm][t], acc[t]);
      }
    }
  }
  if (row < Ns) {
#pragma unroll
    for (int t = 0; t < BT; ++t)
      if (t0 + t < ld) phi[row * ld + t0 + t] = (t0 + t < r) ? (float)acc[t] : 0.f;
  }
}

// ------------------------------------------------- tall-skinny Gram A^T B

constexpr int TR = 32;  // rows per tile

// partial[blk][64x64] = sum over the block's rows of A[row,:]^T B[row,:] for
// the leading W x W corner, W = 4 TT >= r (the rest of the 64 x 64 slot is
// left unwritten).  TT x TT threads of 4 x 4 outputs each cover the corner;
// the 256 / TT^2 such groups take every RG-th row of a tile and are summed
// in a fixed order at the end, so the FP64 work per row is W^2 rather than
// 64^2 for small r.  Rows are staged in shared memory already in FP64.
template <int TT>
__global__ void __launch_bounds__(256)
    k_tsgram(const float *__restrict__ A, const float *__restrict__ B, long Ns, int ld, long rchunk,
             double *__restrict__ part) {
  constexpr int W = 4 * TT, NG = TT * TT, RG = 256 / NG;
  static_assert(2 * TR * W <= 4096 && RG * W * W == 4096, "tsgram shared memory");
  __shared__ double sm[4096];  // As, Bs while accumulating, then the group partials
  double *As = sm, *Bs = sm + TR * W;
  const int tid = threadIdx.x, g = tid % NG, tx = g % TT, ty = g / TT, rg = tid / NG;
  const int wc = min(ld, W);
  const long r0 = (long)blockIdx.x * rchunk, r1 = min(Ns, r0 + rchunk);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long rb = r0; rb < r1; rb += TR) {
    for (int e = tid; e < TR * W; e += 256) {
      const int rr = e / W, c = e - (e / W) * W;
      const long row = rb + rr;
      const bool ok = row < r1 && c < wc;
      As[e] = ok ? (double)A[row * ld + c] : 0.0;
      Bs[e] = ok ? (double)B[row * ld + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = rg; rr < TR; rr += RG) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[rr * W + tx * 4 + i];
        b[i] = Bs[rr * W + ty * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double *red = sm + (size_t)rg * W * W;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) red[(tx * 4 + i) * W + ty * 4 + j] = acc[i][j];
  __syncthreads();
  double *dst = part + (size_t)blockIdx.x * 4096;
  for (int o = tid; o < W * W; o += 256) {
    double v = 0.0;
    for (int q = 0; q < RG; ++q) v += sm[(size_t)q * W * W + o];
    dst[(o / W) * 64 + o % W] = v;
  }
}

// G[i][j] = sum over the blocks' partials: one warp per output, the lanes
// taking every 32nd block and a fixed shuffle tree combining them, so the
// order (and the result) does not depend on scheduling.
__global__ void k_tsgram_reduce(const double *__restrict__ part, int nblk, int r,
                                double *__restrict__ G) {
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (idx >= r * r) return;
  const int i = idx / r, j = idx - (idx / r) * r;
  double v = 0.0;
  for (int b = lane; b < nblk; b += 32) v += part[(size_t)b * 4096 + i * 64 + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) G[idx] = v;
}

// Cholesky G = L L^T (FP64, one thread) and Linv = L^-1; failure flags.
__global__ void k_chol_inv(const double *__restrict__ G, int r, double *__restrict__ Linv,
                           int *err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[64 * 64];
  for (int i = 0; i < r * r; ++i) L[i] = 0.0;
  for (int j = 0; j < r; ++j) {
    double d = G[j * r + j];
    for (int k = 0; k < j; ++k) d -= L[j * r + k] * L[j * r + k];
    if (!(d > 0.0)) {
      vds_flag(err, VDS_ENAN);
      return;
    }
    const double ljj = sqrt(d);
    L[j * r + j] = ljj;
    for (int i = j + 1; i < r; ++i) {
      double v = G[i * r + j];
      for (int k = 0; k < j; ++k) v -= L[i * r + k] * L[j * r + k];
      L[i * r + j] = v / ljj;
    }
  }
  // forward substitution column by column: L X = I
  for (int c = 0; c < r; ++c) {
    for (int i = 0; i < r; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= L[i * r + k] * Linv[k * r + c];
      Linv[i * r + c] = (i >= c) ? v / L[i * r + i] : 0.0;
    }
  }
}

// Phi[row, t] <- sum_{u <= t} Phi[row, u] Linv[t, u]  (Phi L^-T)
__global__ void __launch_bounds__(256)
    k_apply_linv(float *__restrict__ phi, long Ns, int ld, int r, const double *__restrict__ Linv) {
  __shared__ double Ls[64 * 64];
  for (int e = threadIdx.x; e < r * r; e += 256) Ls[e] = Linv[e];
  __syncthreads();
  const long row = (long)blockIdx.x * 256 + threadIdx.x;
  if (row >= Ns) return;
  float x[64];
  for (int u = 0; u < r; ++u) x[u] = phi[row * ld + u];
  for (int t = 0; t < r; ++t) {
    double v = 0.0;
    for (int u = 0; u <= t; ++u) v = fma((double)x[u], Ls[t * r + u], v);
    phi[row * ld + t] = (float)v;
  }
}

// --------------------------------------------------------------- sign fix

// per block and column: largest |phi| and its (lowest) row
__global__ void __launch_bounds__(256)
    k_colmax(const float *__restrict__ phi, long Ns, int ld, int r, long rchunk, float *bmax,
             long *brow) {
  __shared__ float sv[256];
  __shared__ long sr[256];
  const long r0 = (long)blockIdx.x * rchunk, r1 = min(Ns, r0 + rchunk);
  for (int t = 0; t < r; ++t) {
    float best = -1.f;
    long brw = 0x7fffffffffffffffL;
    for (long row = r0 + threadIdx.x; row < r1; row += 256) {
      const float v = fabsf(phi[row * ld + t]);
      if (v > best) {
        best = v;
        brw = row;
      }
    }
    sv[threadIdx.x] = best;
    sr[threadIdx.x] = brw;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const float v2 = sv[threadIdx.x + o];
        const long r2 = sr[threadIdx.x + o];
        if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && r2 < sr[threadIdx.x])) {
          sv[threadIdx.x] = v2;
          sr[threadIdx.x] = r2;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      bmax[(size_t)blockIdx.x * 64 + t] = sv[0];
      brow[(size_t)blockIdx.x * 64 + t] = sr[0];
    }
    __syncthreads();
  }
}

__global__ void k_colsign(const float *__restrict__ phi, int ld, int r, int nblk,
                          const float *__restrict__ bmax, const long *__restrict__ brow,
                          float *__restrict__ sgn) {
  const int t = threadIdx.x;
  if (t >= r) return;
  float best = -1.f;
  long brw = 0x7fffffffffffffffL;
  for (int b = 0; b < nblk; ++b) {
    const float v = bmax[(size_t)b * 64 + t];
    const long rw = brow[(size_t)b * 64 + t];
    if (v > best || (v == best && rw < brw)) {
      best = v;
      brw = rw;
    }
  }
  sgn[t] = (best > 0.f && phi[brw * ld + t] < 0.f) ? -1.f : 1.f;
}

__global__ void k_colscale(float *__restrict__ phi, long Ns, int ld, int r, const float *__restrict__ sgn) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * ld) return;
  const int t = (int)(idx % ld);
  if (t < r) phi[idx] *= sgn[t];
}

// (I (x) kappa) Phi: out[(I a), t] = sum_b kappa[a][b] Phi[(I b), t]
__global__ void k_kappa_phi(const float *__restrict__ phi, long Ns, int ld, int s, KappaArg kap,
                            float *__restrict__ out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * ld) return;
  const long row = idx / ld;
  const int t = (int)(idx - row * ld);
  const long I = row / s;
  const int a = (int)(row - I * s);
  double v = 0.0;
  for (int b = 0; b < s; ++b) v += kap.k[a * s + b] * (double)phi[(I * s + b) * ld + t];
  out[idx] = (float)v;
}

// ------------------------------------------------------- project and lift

constexpr int PJ_NT = 256;   // threads per CTA
constexpr int PJ_TT = 8;     // basis columns per pass

// partial[blk][t*nb + k] = sum over the block's particles of
//   sum_a Phi[(I s + a), t] q[I D + s k + a]
// (PJ_NB >= nb bonds, a compile-time bound).
// Each thread takes particles I = I0 + tid, I0 + tid + 256, ... of the
// block's contiguous range and keeps PJ_TT x nb FP32 sums per pass over the
// basis columns; the block combines them in a fixed order (warp shuffle tree,
// then the warps in order, in FP64), so the result does not depend on the
// schedule.  Phi rows and q rows are read once per pass.
template <int S, int PJ_NB>
__global__ void __launch_bounds__(PJ_NT)
    k_project(const float *__restrict__ phi, int ld, int r, const float *__restrict__ q, int N, int nb,
              long per_cta, double *__restrict__ part) {
  __shared__ double red[PJ_NT / 32][PJ_TT * PJ_NB];
  const int D = nb * S, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long I0 = (long)blockIdx.x * per_cta, I1 = min((long)N, I0 + per_cta);
  for (int t0 = 0; t0 < r; t0 += PJ_TT) {
    float acc[PJ_TT][PJ_NB];
#pragma unroll
    for (int tt = 0; tt < PJ_TT; ++tt)
#pragma unroll
      for (int k = 0; k < PJ_NB; ++k) acc[tt][k] = 0.f;
    for (long I = I0 + threadIdx.x; I < I1; I += PJ_NT) {
      float qv[PJ_NB * S];
#pragma unroll
      for (int e = 0; e < PJ_NB * S; ++e) qv[e] = e < D ? q[(size_t)I * D + e] : 0.f;
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const float *row = phi + ((size_t)I * S + a) * ld + t0;
        float ph[PJ_TT];
#pragma unroll
        for (int tt = 0; tt < PJ_TT; ++tt) ph[tt] = t0 + tt < r ? row[tt] : 0.f;
#pragma unroll
        for (int tt = 0; tt < PJ_TT; ++tt)
#pragma unroll
          for (int k = 0; k < PJ_NB; ++k) acc[tt][k] = fmaf(ph[tt], qv[k * S + a], acc[tt][k]);
      }
    }
#pragma unroll
    for (int tt = 0; tt < PJ_TT; ++tt)
#pragma unroll
      for (int k = 0; k < PJ_NB; ++k) {
        float v = acc[tt][k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][tt * PJ_NB + k] = (double)v;
      }
    __syncthreads();
    if (threadIdx.x < PJ_TT * PJ_NB) {
      const int tt = threadIdx.x / PJ_NB, k = threadIdx.x % PJ_NB;
      if (t0 + tt < r && k < nb) {
        double v = 0.0;
        for (int w = 0; w < PJ_NT / 32; ++w) v += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * (r * nb) + (t0 + tt) * nb + k] = v;
      }
    }
    __syncthreads();
  }
}

// one block per output: strided partial sums over the CTA partials, then a
// fixed-order tree (deterministic)
__global__ void k_project_reduce2(const double *__restrict__ part, int nblk, int n, double *__restrict__ pd,
                                  float *__restrict__ pf) {
  __shared__ double sh[256];
  const int o = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += part[(size_t)b * n + o];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (pd) pd[o] = sh[0];
    if (pf) pf[o] = (float)sh[0];
  }
}

// q[I D + s k + a] = sum_t Phi[(I s + a), t] p[t nb + k]
__global__ void __launch_bounds__(256)
    k_lift(const float *__restrict__ phi, int ld, int r, const float *__restrict__ p, int N, int D,
           int s, int nb, float *__restrict__ q) {
  __shared__ float ps[64 * 8];
  for (int e = threadIdx.x; e < r * nb; e += 256) ps[e] = p[e];
  __syncthreads();
  const long row = (long)blockIdx.x * 256 + threadIdx.x;
  if (row >= (long)N * s) return;
  const long I = row / s;
  const int a = (int)(row - I * s);
  float acc[8];
  for (int k = 0; k < nb; ++k) acc[k] = 0.f;
  // ld is a multiple of 4 (columns r..ld-1 hold zeros): the row in float4s
  const float4 *row4 = reinterpret_cast<const float4 *>(phi + row * ld);
  for (int t4 = 0; t4 < (r + 3) / 4; ++t4) {
    const float4 f4 = row4[t4];
    const float f[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = 4 * t4 + u;
      if (t >= r) break;
      for (int k = 0; k < nb; ++k) acc[k] = fmaf(f[u], ps[t * nb + k], acc[k]);
    }
  }
  for (int k = 0; k < nb; ++k) q[I * D + s * k + a] = acc[k];
}

struct TmpBufs {
  void *p[12] = {};
  ~TmpBufs() {
    for (void *x : p)
      if (x) cudaFree(x);
  }
};

int tsgram(vds_ctx *c, const float *A, const float *B, long Ns, int ld, int r, double *part,
           int nblk, long rchunk, double *G) {
  if (r <= 16)
    k_tsgram<4><<<nblk, 256, 0, c->stream>>>(A, B, Ns, ld, rchunk, part);
  else if (r <= 32)
    k_tsgram<8><<<nblk, 256, 0, c->stream>>>(A, B, Ns, ld, rchunk, part);
  else
    k_tsgram<16><<<nblk, 256, 0, c->stream>>>(A, B, Ns, ld, rchunk, part);
  VDS_CUDA_TRY(cudaGetLastError());
  k_tsgram_reduce<<<(r * r + 7) / 8, 256, 0, c->stream>>>(part, nblk, r, G);
  VDS_CUDA_TRY(cudaGetLastError());
  c->launches += 2;
  return VDS_OK;
}

}  // namespace

int pod_tsgram(vds_ctx *c, const float *A, const float *B, long Ns, int ld, int r, double *G) {
  int nblk = 4 * c->num_sms;
  long rchunk = (Ns + nblk - 1) / nblk;
  rchunk = (rchunk + TR - 1) / TR * TR;
  nblk = (int)((Ns + rchunk - 1) / rchunk);
  VDS_TRY(vds_ensure(c, c->gbuf, (size_t)nblk * 4096 * sizeof(double)));
  return tsgram(c, A, B, Ns, ld, r, (double *)c->gbuf.ptr, nblk, rchunk, G);
}

void pod_project_grid(const vds_ctx *c, int N, long &nblk, long &per_cta) {
  // about two CTAs per SM, each a contiguous range of particles
  nblk = (N + PJ_NT - 1) / PJ_NT;
  if (nblk > 2L * c->num_sms) nblk = 2L * c->num_sms;
  per_cta = (N + nblk - 1) / nblk;
  nblk = (N + per_cta - 1) / per_cta;
}

int pod_project_finish(vds_ctx *c, int n, long nblk, double *pd, float *pf) {
  k_project_reduce2<<<n, 256, 0, c->stream>>>((const double *)c->gbuf.ptr, (int)nblk, n, pd, pf);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

int pod_project_dev(vds_ctx *c, const pod_basis *b, const float *q, int N, int D, double *pd, float *pf) {
  const int nb = D / b->s;
  if (nb > 8) return VDS_EARG;
  long nblk, per_cta;
  pod_project_grid(c, N, nblk, per_cta);
  const int n = b->r * nb;
  VDS_TRY(vds_ensure(c, c->gbuf, (size_t)nblk * n * sizeof(double)));
  auto launch = [&](auto kern) {
    kern<<<(unsigned)nblk, PJ_NT, 0, c->stream>>>(b->phi, b->ld, b->r, q, N, nb, per_cta, (double *)c->gbuf.ptr);
  };
  if (b->s == 3) {
    if (nb <= 1) launch(k_project<3, 1>);
    else if (nb <= 2) launch(k_project<3, 2>);
    else if (nb <= 3) launch(k_project<3, 3>);
    else if (nb <= 4) launch(k_project<3, 4>);
    else launch(k_project<3, 8>);
  } else {
    if (nb <= 1) launch(k_project<2, 1>);
    else if (nb <= 2) launch(k_project<2, 2>);
    else if (nb <= 3) launch(k_project<2, 3>);
    else if (nb <= 4) launch(k_project<2, 4>);
    else launch(k_project<2, 8>);
  }
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return pod_project_finish(c, n, nblk, pd, pf);
}

int pod_lift_dev(vds_ctx *c, const pod_basis *b, const float *p, int N, int D, float *q) {
  const int nb = D / b->s;
  k_lift<<<(unsigned)(((long)N * b->s + 255) / 256), 256, 0, c->stream>>>(b->phi, b->ld, b->r, p, N, D, b->s,
                                                                         nb, q);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return VDS_OK;
}

extern "C" {

int pod_build(vds_ctx *c, const float *X, long Ns, int M, int s, double energy, int r_max,
              int r_fixed, const double *kappa, pod_basis **out, int *r_out) {
  if (!c || !X || !out || Ns < 1 || M < 1 || M > 2048 || (s != 2 && s != 3) || Ns % s != 0)
    return VDS_EARG;
  if (r_max < 1 || r_max > 64 || r_fixed < 0 || r_fixed > 64 || !(energy > 0.0 && energy <= 1.0))
    return VDS_EARG;
  *out = nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, c->device};

  TmpBufs tb;
  const size_t MM = (size_t)M * M;
  double *gpart, *A0, *A1, *V0, *V1, *W, *lam_s, *G, *Linv;
  int *order;
  VDS_CUDA_TRY(cudaMalloc(&tb.p[0], pod_gram_tc_workspace(c, Ns, M)));
  gpart = (double *)tb.p[0];
  VDS_CUDA_TRY(cudaMalloc(&tb.p[1], 4 * MM * sizeof(double)));
  A0 = (double *)tb.p[1];
  A1 = A0 + MM;
  V0 = A1 + MM;
  V1 = V0 + MM;
  VDS_CUDA_TRY(cudaMalloc(&tb.p[2], (size_t)M * 64 * sizeof(double) + (size_t)M * sizeof(double) +
                                        2 * 64 * 64 * sizeof(double)));
  W = (double *)tb.p[2];
  lam_s = W + (size_t)M * 64;
  G = lam_s + M;
  Linv = G + 64 * 64;
  VDS_CUDA_TRY(cudaMalloc(&tb.p[3], (size_t)M * sizeof(int)));
  order = (int *)tb.p[3];

  // 1. Gram
  VDS_TRY(vds_time_begin(c, PK_GRAM));
  VDS_TRY(pod_gram_tc(c, X, Ns, M, gpart, A0));
  VDS_TRY(vds_time_end(c, PK_GRAM));
  VDS_TRY(vds_time_begin(c, PK_EIGEN));
  k_identity<<<(unsigned)((MM + 255) / 256), 256, 0, c->stream>>>(V0, M);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;

  // 2. cyclic Jacobi, round-robin ordering
  VDS_TRY(vds_ensure(c, c->red, 2 * 1024 * sizeof(double)));
  const int Mpe = (M % 2 == 0) ? M : M + 1;  // odd M: one dummy index
  const int H = Mpe / 2;
  const int nT = (H + JT - 1) / JT;                                // <= 64 (M <= 2048)
  const int nAt = nT * (nT + 1) / 2, nVt = ((M + JV_ROWS - 1) / JV_ROWS) * nT;
  const unsigned nblk_round = (unsigned)(nAt + nVt);
  int offblk = (int)((MM + 255) / 256);
  if (offblk > 256) offblk = 256;
  // One sweep (Mpe - 1 rounds, one launch each) is captured as a CUDA graph
  // per starting buffer pair (the buffers swap once per round).
  struct SweepGraphs {
    cudaGraphExec_t g[2] = {nullptr, nullptr};
    ~SweepGraphs() {
      for (cudaGraphExec_t x : g)
        if (x) cudaGraphExecDestroy(x);
    }
  } sg;
  double *Ab[2] = {A0, A1}, *Vb[2] = {V0, V1};
  auto capture = [&](int par) -> int {
    cudaStream_t cap;
    VDS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int cur = par;
    for (int rnd = 0; rnd < Mpe - 1 && e == cudaSuccess; ++rnd) {
      k_jacobi_round<<<nblk_round, JR_NT, 0, cap>>>(Ab[cur], Ab[cur ^ 1], Vb[cur], Vb[cur ^ 1], M, Mpe, rnd,
                                                    nT, nAt);
      e = cudaGetLastError();
      cur ^= 1;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&sg.g[par], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      vds_last_cuda_error(e != cudaSuccess ? e : e2);
      return VDS_ECUDA;
    }
    return VDS_OK;
  };
  int par = 0;  // buffers holding the current A, V
  int sweeps = 0;
  double prev_off = -1.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (!sg.g[par]) VDS_TRY(capture(par));
    VDS_CUDA_TRY(cudaGraphLaunch(sg.g[par], c->stream));
    c->launches += Mpe - 1;
    if ((Mpe - 1) % 2 == 1) par ^= 1;
    k_offnorm<<<offblk, 256, 0, c->stream>>>(Ab[par], M, (double *)c->red.ptr, c->ticket + TK_MISC, c->scal);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    VDS_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
    VDS_TRY(vds_sync_status(c));
    const double off = c->h_scal[SC_AUX], tot = c->h_scal[SC_AUX + 1];
    ++sweeps;
    // converged once every off-diagonal entry is below 1e-11 ||C||_F: the
    // eigenvalues then move by less than that, four orders below the error
    // of the TF32 Gram itself; or when the off-norm stops falling (it cannot
    // rise in exact arithmetic: the rotations of a round are disjoint)
    if (off <= 1e-22 * tot || (prev_off >= 0.0 && off >= prev_off)) break;
    prev_off = off;
  }
  A0 = Ab[par];
  V0 = Vb[par];

  // 3. sort, rank rule, W = V_r Lambda_r^-1/2
  k_eig_sort<<<1, 1024, 0, c->stream>>>(A0, V0, M, energy, r_max, r_fixed, lam_s, order, W, c->scal);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  VDS_TRY(vds_time_end(c, PK_EIGEN));
  VDS_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  VDS_TRY(vds_sync_status(c));
  // the rank of the rule (or r_fixed), reduced to the leading eigenvalues
  // that are positive and above 1e-13 lambda_1 (the others cannot be
  // normalised); *r_out reports it
  const int r = (int)c->h_scal[SC_AUX + 3];
  if (r < 1) return VDS_EARG;
  const int ld = (r + 3) / 4 * 4;

  pod_basis *b = new pod_basis();
  b->device = c->device;
  b->sweeps = sweeps;
  b->Ns = Ns;
  b->M = M;
  b->r = r;
  b->ld = ld;
  b->s = s;
  int st = VDS_OK;
  do {
    if (cudaMalloc(&b->phi, (size_t)Ns * ld * sizeof(float)) != cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    b->lam = (double *)malloc(sizeof(double) * M);
    b->xh = (double *)malloc(sizeof(double) * r * r);
    if (!b->lam || !b->xh) {
      st = VDS_ENOMEM;
      break;
    }
    // 4. basis
    if ((st = vds_time_begin(c, PK_BASIS)) != VDS_OK) break;
    k_basis<<<dim3((unsigned)((Ns + 255) / 256), (ld + BT - 1) / BT), 256, 0, c->stream>>>(X, Ns, M, W, r,
                                                                                         ld, b->phi);
    if (cudaGetLastError() != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    ++c->launches;
    // 5. Cholesky-QR
    int nblk = 4 * c->num_sms;
    long rchunk = (Ns + nblk - 1) / nblk;
    rchunk = (rchunk + TR - 1) / TR * TR;
    nblk = (int)((Ns + rchunk - 1) / rchunk);
    if (cudaMalloc(&tb.p[4], (size_t)nblk * 4096 * sizeof(double)) != cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    double *tpart = (double *)tb.p[4];
    if ((st = tsgram(c, b->phi, b->phi, Ns, ld, r, tpart, nblk, rchunk, G)) != VDS_OK) break;
    k_chol_inv<<<1, 1, 0, c->stream>>>(G, r, Linv, c->err);
    k_apply_linv<<<(unsigned)((Ns + 255) / 256), 256, 0, c->stream>>>(b->phi, Ns, ld, r, Linv);
    if (cudaGetLastError() != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    c->launches += 2;
    // 6. sign fix
    if (cudaMalloc(&tb.p[5], (size_t)nblk * 64 * (sizeof(float) + sizeof(long)) + 64 * sizeof(float)) !=
        cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    float *bmax = (float *)tb.p[5];
    long *brow = (long *)(bmax + (size_t)nblk * 64);
    float *sgn = (float *)(brow + (size_t)nblk * 64);
    k_colmax<<<nblk, 256, 0, c->stream>>>(b->phi, Ns, ld, r, rchunk, bmax, brow);
    k_colsign<<<1, 64, 0, c->stream>>>(b->phi, ld, r, nblk, bmax, brow, sgn);
    k_colscale<<<(unsigned)((Ns * ld + 255) / 256), 256, 0, c->stream>>>(b->phi, Ns, ld, r, sgn);
    if (cudaGetLastError() != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    c->launches += 3;
    // 7. X^H = Phi^T (I (x) kappa) Phi
    if (cudaMalloc(&tb.p[6], (size_t)Ns * ld * sizeof(float)) != cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    KappaArg ka;
    for (int k = 0; k < 9; ++k) ka.k[k] = 0.0;
    if (kappa)
      for (int k = 0; k < s * s; ++k) ka.k[k] = kappa[k];
    k_kappa_phi<<<(unsigned)((Ns * ld + 255) / 256), 256, 0, c->stream>>>(b->phi, Ns, ld, s, ka,
                                                                         (float *)tb.p[6]);
    if (cudaGetLastError() != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    ++c->launches;
    if ((st = tsgram(c, b->phi, (const float *)tb.p[6], Ns, ld, r, tpart, nblk, rchunk, G)) != VDS_OK) break;
    if ((st = vds_time_end(c, PK_BASIS)) != VDS_OK) break;
    if (cudaMemcpyAsync(b->xh, G, sizeof(double) * r * r, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->lam, lam_s, sizeof(double) * M, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    st = vds_sync_status(c);
  } while (0);
  if (st != VDS_OK) {
    pod_free(b);
    return st;
  }
  *out = b;
  if (r_out) *r_out = r;
  return VDS_OK;
}

int pod_load(vds_ctx *c, const float *phi, long Ns, int r, int s, const double *kappa, pod_basis **out) {
  if (!c || !phi || !out || Ns < 1 || r < 1 || r > 64 || (s != 2 && s != 3) || Ns % s != 0) return VDS_EARG;
  *out = nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, c->device};
  TmpBufs tb;
  const int ld = (r + 3) / 4 * 4;
  pod_basis *b = new pod_basis();
  b->device = c->device;
  b->Ns = Ns;
  b->M = 0;
  b->r = r;
  b->ld = ld;
  b->s = s;
  int st = VDS_OK;
  do {
    b->xh = (double *)malloc(sizeof(double) * r * r);
    if (!b->xh || cudaMalloc(&b->phi, (size_t)Ns * ld * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tb.p[0], (size_t)Ns * ld * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tb.p[1], (size_t)r * r * sizeof(double)) != cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    if (cudaMemsetAsync(b->phi, 0, (size_t)Ns * ld * sizeof(float), c->stream) != cudaSuccess ||
        cudaMemcpy2DAsync(b->phi, (size_t)ld * sizeof(float), phi, (size_t)r * sizeof(float),
                          (size_t)r * sizeof(float), (size_t)Ns, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    KappaArg ka;
    for (int k = 0; k < 9; ++k) ka.k[k] = 0.0;
    if (kappa)
      for (int k = 0; k < s * s; ++k) ka.k[k] = kappa[k];
    k_kappa_phi<<<(unsigned)((Ns * ld + 255) / 256), 256, 0, c->stream>>>(b->phi, Ns, ld, s, ka,
                                                                         (float *)tb.p[0]);
    if (cudaGetLastError() != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    ++c->launches;
    double *G = (double *)tb.p[1];
    if ((st = pod_tsgram(c, b->phi, (const float *)tb.p[0], Ns, ld, r, G)) != VDS_OK) break;
    if (cudaMemcpyAsync(b->xh, G, sizeof(double) * r * r, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    st = vds_sync_status(c);
  } while (0);
  if (st != VDS_OK) {
    pod_free(b);
    return st;
  }
  *out = b;
  return VDS_OK;
}

int pod_info(const pod_basis *b, int *r, int *ld, const float **phi, long *Ns) {
  if (!b) return VDS_EARG;
  if (r) *r = b->r;
  if (ld) *ld = b->ld;
  if (phi) *phi = b->phi;
  if (Ns) *Ns = b->Ns;
  return VDS_OK;
}

int pod_sweeps(const pod_basis *b) { return b ? b->sweeps : VDS_EARG; }

int pod_eigenvalues(const pod_basis *b, double *lam, int M) {
  if (!b || !lam || M < b->M) return VDS_EARG;
  if (b->M > 0) memcpy(lam, b->lam, sizeof(double) * b->M);
  return VDS_OK;
}

int pod_xh(const pod_basis *b, double *xh) {
  if (!b || !xh) return VDS_EARG;
  memcpy(xh, b->xh, sizeof(double) * b->r * b->r);
  return VDS_OK;
}

void pod_free(pod_basis *b) {
  if (!b) return;
  if (b->phi) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaFree(b->phi);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  }
  free(b->lam);
  free(b->xh);
  delete b;
}

int pod_project(vds_ctx *c, const pod_basis *b, const float *q, int N, int D, float *p) {
  if (!c || !b || !q || !p || N < 1 || D % b->s != 0 || (long)N * b->s != b->Ns) return VDS_EARG;
  const int nb = D / b->s;
  if (nb < 1 || nb > 8) return VDS_EARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  const int st = pod_project_dev(c, b, q, N, D, nullptr, p);
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return st;
}

int pod_lift(vds_ctx *c, const pod_basis *b, const float *p, int N, int D, float *q) {
  if (!c || !b || !q || !p || N < 1 || D % b->s != 0 || (long)N * b->s != b->Ns) return VDS_EARG;
  const int nb = D / b->s;
  if (nb < 1 || nb > 8) return VDS_EARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  k_lift<<<(unsigned)(((long)N * b->s + 255) / 256), 256, 0, c->stream>>>(b->phi, b->ld, b->r, p, N, D, b->s,
                                                                         nb, q);
  ++c->launches;
  const int st = cudaGetLastError() == cudaSuccess ? VDS_OK : VDS_ECUDA;
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return st;
}

}  // extern "C"
