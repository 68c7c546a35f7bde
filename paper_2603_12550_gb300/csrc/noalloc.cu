// noalloc.cu -- vds_energy_grad_noalloc: the density + free-energy gradient
// evaluation of vds_energy_grad for callers that cannot allocate device
// memory (see include/vds.h).
//
// All scratch (particle records, pair-pass partial sums, reduction slots, the
// error flag and the result scalars) lives in one fixed-size file-scope
// __device__ array.  Every GPU that loads the library holds it (about 4.7 MiB)
// until the process exits.  No function here calls cudaMalloc, cudaFree or an
// allocating library routine.
//
// Host code never uses the array's name as an address: at its first call on a
// device, with that device current, the entry point asks the runtime for the
// array's device address (cudaGetSymbolAddress) and caches it per device.
// Calls that overlap on the GPU share the array and race; the entry point
// synchronises its stream before returning, on success and on every error
// return, so calls made one after another from one thread do not overlap.
//
// Pass shapes follow vds_energy_grad's choice (small clouds take the
// 128-thread, 64-record shape; mid-size clouds 64-record j-chunks when their
// partial sums fit), except that a stream-K grid whose partial sums would not
// fit the fixed buffer is cut down until they do: at N near
// VDS_NOALLOC_MAX_N the gradient pass runs on fewer CTAs than the context
// path (about a quarter of the SMs at D = 9), so it is slower there.
#include <mutex>

#include "pair_impl.cuh"

#define VDS_NOALLOC_MAX_DEVICES 64

namespace {

constexpr size_t kHeadBytes = 8192;  // err | tickets | scalars | reduction slots
constexpr size_t kErrOff = 0, kTicketOff = 256, kScalOff = 512, kRedOff = 512 + SC_COUNT * 8;
constexpr int kMaxDP = Rec<VDS_MAXD>::DP;  // widest record of any accepted D
constexpr size_t kRecBytes =
    (size_t)((VDS_NOALLOC_MAX_N + vds_pair::TJ - 1) / vds_pair::TJ * vds_pair::TJ) * kMaxDP * sizeof(float);
constexpr size_t kPartBytes = (size_t)4 << 20;
constexpr size_t kScratchBytes = kHeadBytes + kRecBytes + kPartBytes;
static_assert(kRedOff + (VDS_NOALLOC_MAX_N / 256 + 1) * 4 * 8 <= kHeadBytes, "head layout");

}  // namespace

// The scratch array.  Zero at module load; the entry point clears the error
// flag and the reduction tickets at the start of every call, and every other
// byte it reads is written earlier in the same call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

struct DevState {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_noalloc_scratch
  int num_sms = 0;
};
DevState g_dev[VDS_NOALLOC_MAX_DEVICES];
std::mutex g_mu;

int setup_device(int dev, DevState **out) {
  if (dev < 0 || dev >= VDS_NOALLOC_MAX_DEVICES) return VDS_EARG;
  std::lock_guard<std::mutex> lk(g_mu);
  DevState &s = g_dev[dev];
  if (!s.ready) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      vds_last_cuda_error(e);
      return VDS_ECUDA;
    }
    int sms = 0;
    const cudaError_t e2 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e2 != cudaSuccess) {
      vds_last_cuda_error(e2);
      return VDS_ECUDA;
    }
    s.base = (unsigned char *)p;
    s.num_sms = sms;
    s.ready = true;
  }
  *out = &s;
  return VDS_OK;
}

// Plans one pass shape's stream-K grid over the fixed partial buffer and
// launches it.  With `shrink` the grid is cut by a quarter at a time until
// the partial sums fit; without it a shape whose partials do not fit at the
// full grid is declined (done = false, nothing launched).
template <int D, int RI, int NT, bool GRAD, int TJK>
int na_try(const DevState &s, int N, cudaStream_t st, const float *rec, double *part, int *err,
           Sched &sc, bool shrink, bool &done) {
  using namespace vds_pair;
  static_assert(Rec<D>::DP <= kMaxDP, "record area sized for the widest D");
  constexpr int DP = Rec<D>::DP;
  constexpr int ACC = GRAD ? D : 1;
  constexpr int TI = NT * RI;
  const size_t smem = (size_t)NSTAGE * TJK * DP * sizeof(float);
  done = false;
  int occ = 0;
  VDS_CUDA_TRY(cudaFuncSetAttribute(k_pair<D, RI, NT, GRAD, TJK>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  VDS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair<D, RI, NT, GRAD, TJK>, NT, smem));
  if (occ < 1) occ = 1;
  sc.TI = TI;
  sc.Npad = (N + TJ - 1) / TJ * TJ;
  sc.Nipad = sc.Npad;
  sc.nchunk = sc.Npad / TJK;
  sc.n_itiles = (N + TI - 1) / TI;
  sc.items = (long long)sc.n_itiles * sc.nchunk;
  long long G = (long long)s.num_sms * occ;
  if (G > sc.items) G = sc.items;
  for (;;) {
    sc.G = (int)G;
    int maxseg = 1;
    for (int t = 0; t < sc.n_itiles; ++t) {
      const int f = sched_first_cta((long long)t * sc.nchunk, sc);
      const int l = sched_first_cta((long long)(t + 1) * sc.nchunk - 1, sc);
      if (l - f + 1 > maxseg) maxseg = l - f + 1;
    }
    sc.maxseg = maxseg;
    if ((size_t)sc.n_itiles * maxseg * TI * ACC * sizeof(double) <= kPartBytes) break;
    if (!shrink) return VDS_OK;
    if (G == 1) return VDS_ESIZE;
    G = G * 3 / 4;
    if (G < 1) G = 1;
  }
  k_pair<D, RI, NT, GRAD, TJK><<<sc.G, NT, smem, st>>>(rec, rec, sc, part, err);
  VDS_CUDA_TRY(cudaGetLastError());
  done = true;
  return VDS_OK;
}

// One pair pass, shaped as vds_energy_grad shapes it (small-cloud shape below
// half the SMs' worth of items, 64-record j-chunks below 8 items per SM if
// their partials fit, otherwise 256-record j-chunks).
template <int D, bool GRAD>
int na_pair(const DevState &s, int N, cudaStream_t st, const float *rec, double *part, int *err,
            Sched &sc) {
  using namespace vds_pair;
  constexpr int RI = GRAD ? PairCfg<D>::RI_GRAD : PairCfg<D>::RI_DENS;
  constexpr int NT = GRAD ? PairCfg<D>::NT_GRAD : PairCfg<D>::NT_DENS;
  const long long items = (long long)((N + NT * RI - 1) / (NT * RI)) * ((N + TJ - 1) / TJ);
  bool done = false;
  if (2 * items < s.num_sms)
    return na_try<D, RI_SMALL, NT_SMALL, GRAD, TJ_SMALL>(s, N, st, rec, part, err, sc, true, done);
  if (items < 8LL * s.num_sms) {
    VDS_TRY((na_try<D, RI, NT, GRAD, TJ_SMALL>(s, N, st, rec, part, err, sc, false, done)));
    if (done) return VDS_OK;
  }
  return na_try<D, RI, NT, GRAD, TJ>(s, N, st, rec, part, err, sc, true, done);
}

template <int D>
int na_energy_grad(const DevState &s, const float *q, const KParams &kp, double *E, float *g,
                   float *rho, cudaStream_t st) {
  using namespace vds_pair;
  unsigned char *base = s.base;
  int *err = (int *)(base + kErrOff);
  unsigned *ticket = (unsigned *)(base + kTicketOff);
  double *scal = (double *)(base + kScalOff);
  double *red = (double *)(base + kRedOff);
  float *rec = (float *)(base + kHeadBytes);
  double *part = (double *)(base + kHeadBytes + kRecBytes);
  const int N = kp.N;
  const int Npad = (N + TJ - 1) / TJ * TJ;
  // error flag and tickets must start at zero
  VDS_CUDA_TRY(cudaMemsetAsync(base, 0, kScalOff, st));
  k_prep<D><<<(Npad + 255) / 256, 256, 0, st>>>(N, Npad, kp.c, q, nullptr, nullptr, 0.f, nullptr, rec);
  VDS_CUDA_TRY(cudaGetLastError());
  Sched sd, sg;
  VDS_TRY((na_pair<D, false>(s, N, st, rec, part, err, sd)));
  const int nb = (N + NT_FIN - 1) / NT_FIN;
  k_dens_finish<D><<<nb, NT_FIN, 0, st>>>(sd, part, rec, rho, kp, E ? 1 : 0, q, nullptr, nullptr, nullptr,
                                         red, ticket + TK_DENS, scal, err);
  VDS_CUDA_TRY(cudaGetLastError());
  if (g) {
    VDS_TRY((na_pair<D, true>(s, N, st, rec, part, err, sg)));
    k_grad_finish<D, GM_OUT><<<nb, NT_FIN, 0, st>>>(sg, part, rec, kp, g, q, nullptr, nullptr, nullptr,
                                                   nullptr, red, ticket + TK_GRAD, scal, err);
    VDS_CUDA_TRY(cudaGetLastError());
  }
  double e_host = 0.0;
  int err_host = 0;
  if (E) VDS_CUDA_TRY(cudaMemcpyAsync(&e_host, scal + SC_E, sizeof(double), cudaMemcpyDeviceToHost, st));
  VDS_CUDA_TRY(cudaMemcpyAsync(&err_host, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  VDS_CUDA_TRY(cudaStreamSynchronize(st));
  if (err_host != 0) return err_host;
  if (E) *E = e_host;
  return VDS_OK;
}

}  // namespace

extern "C" int vds_energy_grad_noalloc(const float *q, int N, int D, const vds_params *p, double *E,
                                       float *g, float *rho, void *cuda_stream) {
  if (!q || !p || N < 1 || D < 2 || D > VDS_MAXD) return VDS_EARG;
  if (p->s < 2 || p->s > 3 || p->nb < 1 || p->nb > 8 || p->nb * p->s != D) return VDS_EARG;
  if (!(p->h > 0.0) || !(p->zeta > 0.0) || !(p->kBT >= 0.0)) return VDS_EARG;
  if ((p->spring != 0 && p->spring != 1) || (p->spring == 1 && !(p->b > 0.0))) return VDS_EARG;
  if (N > VDS_NOALLOC_MAX_N) return VDS_ESIZE;
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    vds_last_cuda_error(e);
    return VDS_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the call copies a status word to the host and synchronises its stream,
  // neither of which a stream capture allows: refuse before touching it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return VDS_EARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return VDS_EARG;
  DevState *s = nullptr;
  VDS_TRY(setup_device(dev, &s));
  const KParams kp = make_kparams(p, N, D);
  int r = VDS_EARG;
  switch (D) {
    case 2: r = na_energy_grad<2>(*s, q, kp, E, g, rho, st); break;
    case 3: r = na_energy_grad<3>(*s, q, kp, E, g, rho, st); break;
    case 4: r = na_energy_grad<4>(*s, q, kp, E, g, rho, st); break;
    case 6: r = na_energy_grad<6>(*s, q, kp, E, g, rho, st); break;
    case 8: r = na_energy_grad<8>(*s, q, kp, E, g, rho, st); break;
    case 9: r = na_energy_grad<9>(*s, q, kp, E, g, rho, st); break;
    case 10: r = na_energy_grad<10>(*s, q, kp, E, g, rho, st); break;
    case 12: r = na_energy_grad<12>(*s, q, kp, E, g, rho, st); break;
    case 14: r = na_energy_grad<14>(*s, q, kp, E, g, rho, st); break;
    case 15: r = na_energy_grad<15>(*s, q, kp, E, g, rho, st); break;
    case 16: r = na_energy_grad<16>(*s, q, kp, E, g, rho, st); break;
    default: return VDS_EARG;
  }
  // An error after the first launch can leave kernels queued on the shared
  // scratch: wait for them, so that the next call cannot race with them.
  if (r != VDS_OK) (void)cudaStreamSynchronize(st);
  return r;
}
