// bandwidth.cu -- kernel bandwidth selection (Sec. 2.2).
//
// Median rule (Eq. model_bandwidth): h = med / sqrt(2 ln N), med the lower
// middle order statistic of the N(N-1)/2 distances |q_J - q_K|, J < K.  The
// selection is exact on FP32 squared distances (their bit patterns order like
// the values): a radix select over the N^2 ordered pairs, diagonal included,
// where every unordered distance appears twice and the diagonal adds N zeros,
// so the wanted element has ordered rank N + 2 k, k = (M-1)/2, M = N(N-1)/2.
// Three histogram passes (11 + 11 + 10 key bits) over all pairs, each followed
// by a one-block digit selection, entirely on the device.
//
// Silverman rule: h = sigma (4 / ((D+2) N))^(1/(D+4)), sigma the mean over
// coordinates of the sample standard deviation (two FP64 passes).
#include <math.h>

#include "vds_internal.cuh"

namespace {

struct SelState {
  unsigned long long rank;  // rank still to find inside the current prefix
  unsigned prefix;          // key bits selected so far
  unsigned pad;
};

constexpr int BW_NT = 256;
constexpr int NBINS = 2048;

__host__ __device__ constexpr int pass_shift(int pass) { return pass == 0 ? 21 : (pass == 1 ? 10 : 0); }
__host__ __device__ constexpr int pass_bits(int pass) { return pass == 2 ? 10 : 11; }

template <int D>
__global__ void __launch_bounds__(BW_NT)
    k_hist(const float *__restrict__ q, int N, int jchunk, const SelState *__restrict__ st, int pass,
           unsigned long long *__restrict__ ghist) {
  __shared__ unsigned hist[NBINS];
  __shared__ float tile[BW_NT * D];
  const int tid = threadIdx.x;
  const int shift = pass_shift(pass), bits = pass_bits(pass);
  const unsigned mask = (1u << bits) - 1u;
  const int hi = shift + bits;
  const unsigned prefix = st->prefix;
  for (int b = tid; b < NBINS; b += BW_NT) hist[b] = 0u;
  const int i = blockIdx.x * BW_NT + tid;
  const bool vi = i < N;
  float xi[D];
#pragma unroll
  for (int d = 0; d < D; ++d) xi[d] = vi ? q[(size_t)i * D + d] : 0.f;
  const int j0 = blockIdx.y * jchunk;
  const int j1 = min(N, j0 + jchunk);
  for (int jt = j0; jt < j1; jt += BW_NT) {
    const int cnt = min(BW_NT, j1 - jt);
    __syncthreads();
    for (int x = tid; x < cnt * D; x += BW_NT) tile[x] = q[(size_t)jt * D + x];
    __syncthreads();
    if (vi) {
      for (int j = 0; j < cnt; ++j) {
        float r2 = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float dd = xi[d] - tile[j * D + d];
          r2 = fmaf(dd, dd, r2);
        }
        const unsigned key = __float_as_uint(r2);
        if (pass == 0 || (key >> hi) == prefix) atomicAdd(&hist[(key >> shift) & mask], 1u);
      }
    }
  }
  __syncthreads();
  for (int b = tid; b < NBINS; b += BW_NT)
    if (hist[b]) atomicAdd(&ghist[b], (unsigned long long)hist[b]);
}

__global__ void k_sel_init(SelState *st, long long N, unsigned long long *ghist) {
  for (int b = threadIdx.x; b < NBINS; b += blockDim.x) ghist[b] = 0ull;
  if (threadIdx.x == 0) {
    const unsigned long long M = (unsigned long long)N * (unsigned long long)(N - 1) / 2ull;
    st->rank = (unsigned long long)N + 2ull * ((M - 1ull) / 2ull);
    st->prefix = 0u;
  }
}

__global__ void k_sel_digit(SelState *st, unsigned long long *ghist, int pass, long long N,
                            double *scal, int *err) {
  __shared__ int found;
  __shared__ unsigned long long below;
  if (threadIdx.x == 0) {
    const int nb = 1 << pass_bits(pass);
    unsigned long long cum = 0ull;
    found = -1;
    for (int b = 0; b < nb; ++b) {
      const unsigned long long c = ghist[b];
      if (st->rank < cum + c) {
        found = b;
        break;
      }
      cum += c;
    }
    below = cum;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < NBINS; b += blockDim.x) ghist[b] = 0ull;
  if (threadIdx.x == 0) {
    if (found < 0) {
      vds_flag(err, VDS_ENAN);
      return;
    }
    st->rank -= below;
    st->prefix = (st->prefix << pass_bits(pass)) | (unsigned)found;
    if (pass == 2) {
      const float r2 = __uint_as_float(st->prefix);
      const double med = sqrt((double)r2);
      scal[SC_H] = med / sqrt(2.0 * log((double)N));
      scal[SC_AUX] = (double)r2;
      if (!(med > 0.0) || !(med < 1e300)) vds_flag(err, VDS_ENAN);
    }
  }
}

// Silverman: per-coordinate FP64 mean, then sum of squared deviations.
template <int D>
__global__ void __launch_bounds__(256)
    k_moments(const float *__restrict__ q, int N, int pass, double *red, unsigned *ticket,
              double *scal) {
  __shared__ double sh[8][D];
  __shared__ bool last;
  double acc[D];
#pragma unroll
  for (int d = 0; d < D; ++d) acc[d] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double v = (double)q[(size_t)i * D + d];
      if (pass == 0) acc[d] += v;
      else {
        const double x = v - scal[SC_AUX + d];
        acc[d] += x * x;
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    double v = acc[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w][d] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int d = 0; d < D; ++d) {
      double v = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += sh[k][d];
      red[(size_t)blockIdx.x * D + d] = v;
    }
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double sig = 0.0;
  for (int d = 0; d < D; ++d) {
    double v = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(red + (size_t)b * D + d);
    if (pass == 0) scal[SC_AUX + d] = v / (double)N;
    else sig += sqrt(v / (double)(N - 1));
  }
  if (pass == 1) {
    sig /= (double)D;
    scal[SC_H] = sig * pow(4.0 / ((double)(D + 2) * (double)N), 1.0 / (double)(D + 4));
  }
  *ticket = 0u;
}

template <int D>
int bandwidth_impl(vds_ctx *c, const float *q, int N, int rule, double *h) {
  if (rule == 1) {
    int nblk = (N + 255) / 256;
    if (nblk > 2 * c->num_sms) nblk = 2 * c->num_sms;
    VDS_TRY(vds_ensure(c, c->red, (size_t)nblk * D * sizeof(double)));
    for (int pass = 0; pass < 2; ++pass) {
      k_moments<D><<<nblk, 256, 0, c->stream>>>(q, N, pass, (double *)c->red.ptr, c->ticket + TK_MISC,
                                                c->scal);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
    }
  } else {
    // state + global histogram live in the reduction scratch
    VDS_TRY(vds_ensure(c, c->red, sizeof(SelState) + NBINS * sizeof(unsigned long long)));
    SelState *st = (SelState *)c->red.ptr;
    unsigned long long *gh = (unsigned long long *)((char *)c->red.ptr + sizeof(SelState));
    k_sel_init<<<1, 256, 0, c->stream>>>(st, N, gh);
    VDS_CUDA_TRY(cudaGetLastError());
    ++c->launches;
    const int n_itiles = (N + BW_NT - 1) / BW_NT;
    // split j so that the grid covers the GPU a few times over
    int nsplit = (4 * c->num_sms + n_itiles - 1) / n_itiles;
    if (nsplit < 1) nsplit = 1;
    int jchunk = (N + nsplit - 1) / nsplit;
    jchunk = (jchunk + BW_NT - 1) / BW_NT * BW_NT;
    nsplit = (N + jchunk - 1) / jchunk;
    for (int pass = 0; pass < 3; ++pass) {
      VDS_TRY(vds_time_begin(c, PK_BANDWIDTH));
      k_hist<D><<<dim3(n_itiles, nsplit), BW_NT, 0, c->stream>>>(q, N, jchunk, st, pass, gh);
      VDS_CUDA_TRY(cudaGetLastError());
      VDS_TRY(vds_time_end(c, PK_BANDWIDTH));
      ++c->launches;
      k_sel_digit<<<1, 256, 0, c->stream>>>(st, gh, pass, N, c->scal, c->err);
      VDS_CUDA_TRY(cudaGetLastError());
      ++c->launches;
    }
  }
  VDS_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  VDS_TRY(vds_sync_status(c));
  *h = c->h_scal[SC_H];
  return VDS_OK;
}

}  // namespace

extern "C" int vds_bandwidth(vds_ctx *c, const float *q, int N, int D, int rule, double *h) {
  if (!c || !q || !h || N < 2 || (rule != 0 && rule != 1)) return VDS_EARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  int st;
  switch (D) {
    case 2: st = bandwidth_impl<2>(c, q, N, rule, h); break;
    case 3: st = bandwidth_impl<3>(c, q, N, rule, h); break;
    case 4: st = bandwidth_impl<4>(c, q, N, rule, h); break;
    case 6: st = bandwidth_impl<6>(c, q, N, rule, h); break;
    case 8: st = bandwidth_impl<8>(c, q, N, rule, h); break;
    case 9: st = bandwidth_impl<9>(c, q, N, rule, h); break;
    case 10: st = bandwidth_impl<10>(c, q, N, rule, h); break;
    case 12: st = bandwidth_impl<12>(c, q, N, rule, h); break;
    case 14: st = bandwidth_impl<14>(c, q, N, rule, h); break;
    case 15: st = bandwidth_impl<15>(c, q, N, rule, h); break;
    case 16: st = bandwidth_impl<16>(c, q, N, rule, h); break;
    default: st = VDS_EARG;
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return st;
}
