// vds_capi.cu -- the C ABI (include/vds.h): context, energy/gradient
// evaluation, explicit and implicit time steps, stress.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "pair.cuh"

namespace {
thread_local cudaError_t g_last_cuda = cudaSuccess;

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int check_params(const vds_params *p, int N, int D) {
  if (!p || N < 1 || D < 2 || D > VDS_MAXD) return VDS_EARG;
  if (p->s < 2 || p->s > 3 || p->nb < 1 || p->nb > 8 || p->nb * p->s != D) return VDS_EARG;
  if (!(p->h > 0.0) || !(p->zeta > 0.0) || !(p->kBT >= 0.0)) return VDS_EARG;
  if (p->spring != 0 && p->spring != 1) return VDS_EARG;
  if (p->spring == 1 && !(p->b > 0.0)) return VDS_EARG;
  return VDS_OK;
}

// Copy the device scalars to the pinned mirror, synchronise, collect status.
int read_scalars(vds_ctx *c) {
  VDS_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  return vds_sync_status(c);
}

float *vec(vds_ctx *c, int k, size_t nd) { return (float *)c->vecs.ptr + (size_t)k * nd; }

}  // namespace

void vds_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

int vds_ensure(vds_ctx *c, DevBuf &b, size_t bytes) {
  if (bytes <= b.cap) return VDS_OK;
  if (b.ptr) {
    VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
  }
  const size_t want = bytes + bytes / 4 + 256;
  VDS_CUDA_TRY(cudaMalloc(&b.ptr, want));
  b.cap = want;
  return VDS_OK;
}

static int timing_harvest(vds_ctx *c) {
  TimingPool *t = c->timing;
  if (!t) return VDS_OK;
  VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < PK_COUNT; ++k) {
    for (int i = 0; i < t->used[k]; ++i) {
      float ms = 0.f;
      VDS_CUDA_TRY(cudaEventElapsedTime(&ms, t->ev[k][0][i], t->ev[k][1][i]));
      t->ms[k] += ms;
      t->count[k] += 1;
    }
    t->used[k] = 0;
  }
  return VDS_OK;
}

int vds_time_begin(vds_ctx *c, int pk) {
  TimingPool *t = c->timing;
  if (!t || !t->on) return VDS_OK;
  if (t->used[pk] == 256) VDS_TRY(timing_harvest(c));
  cudaEvent_t &e = t->ev[pk][0][t->used[pk]];
  if (!e) VDS_CUDA_TRY(cudaEventCreate(&e));
  VDS_CUDA_TRY(cudaEventRecord(e, c->stream));
  return VDS_OK;
}

int vds_time_end(vds_ctx *c, int pk) {
  TimingPool *t = c->timing;
  if (!t || !t->on) return VDS_OK;
  cudaEvent_t &e = t->ev[pk][1][t->used[pk]];
  if (!e) VDS_CUDA_TRY(cudaEventCreate(&e));
  VDS_CUDA_TRY(cudaEventRecord(e, c->stream));
  t->used[pk] += 1;
  return VDS_OK;
}

int vds_sync_status(vds_ctx *c) {
  VDS_CUDA_TRY(cudaMemcpyAsync(c->h_err, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int e = *c->h_err;
  if (e != 0) {
    VDS_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return e;
}

namespace {
// The library's bounded-wait pattern run on waits that nothing completes:
// an mbarrier phase no thread arrives on, and a flag in global memory no
// thread sets.  Each gives up after limit_ns of globaltimer time and raises
// VDS_ETIMEOUT, as every wait in the pair, refresh, Gram and network kernels
// does; the kernel then returns normally.
__global__ void k_wait_selftest(unsigned long long limit_ns, const volatile int *flag, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) vds_flag(err, VDS_ETIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_timer_ns();
    while (*flag == 0) {
      if (global_timer_ns() - t0 > limit_ns) {
        vds_flag(err, VDS_ETIMEOUT);
        break;
      }
    }
  }
}
}  // namespace

extern "C" {

int vds_wait_selftest(vds_ctx *c, double limit_s) {
  if (!c || !(limit_s > 0.0) || !(limit_s <= 1.0)) return VDS_EARG;
  DeviceGuard dg(c->device);
  // the flag: a zeroed word of the reduction scratch that no kernel sets
  VDS_TRY(vds_ensure(c, c->red, sizeof(double)));
  VDS_CUDA_TRY(cudaMemsetAsync(c->red.ptr, 0, sizeof(double), c->stream));
  k_wait_selftest<<<1, 32, 0, c->stream>>>((unsigned long long)(limit_s * 1e9),
                                           (const volatile int *)c->red.ptr, c->err);
  VDS_CUDA_TRY(cudaGetLastError());
  ++c->launches;
  return vds_sync_status(c);
}

const char *vds_strerror(int st) {
  switch (st) {
    case VDS_OK: return "ok";
    case VDS_EARG: return "invalid argument";
    case VDS_ECUDA: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
    case VDS_EDOMAIN: return "FENE bond outside |q|^2 < b";
    case VDS_ENOCONV: return "implicit minimiser did not converge";
    case VDS_ENAN: return "non-finite density or energy";
    case VDS_ETIMEOUT: return "bounded device wait gave up";
    case VDS_ENOMEM: return "device allocation failed";
    case VDS_ESURROGATE: return "surrogate check failed";
    case VDS_ESIZE: return "problem larger than the fixed-size scratch allows";
    default: return "unknown status";
  }
}

int vds_create(vds_ctx **out, void *stream, int device) {
  if (!out) return VDS_EARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VDS_EARG;
  DeviceGuard g(device);
  if (!g.ok) return VDS_ECUDA;
  vds_ctx *c = new vds_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  int st = VDS_OK;
  do {
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    if (cudaMalloc(&c->err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->ticket, TK_COUNT * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&c->scal, SC_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_scal, SC_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
      st = VDS_ENOMEM;
      break;
    }
    if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ticket, 0, TK_COUNT * sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->scal, 0, SC_COUNT * sizeof(double), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
  } while (0);
  if (st != VDS_OK) {
    vds_destroy(c);
    return st;
  }
  *out = c;
  return VDS_OK;
}

void vds_destroy(vds_ctx *c) {
  if (!c) return;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  DevBuf *bufs[] = {&c->rec, &c->recq, &c->part, &c->red, &c->vecs, &c->gbuf, &c->ubuf, &c->dtbuf};
  for (DevBuf *b : bufs)
    if (b->ptr) cudaFree(b->ptr);
  if (c->err) cudaFree(c->err);
  if (c->ticket) cudaFree(c->ticket);
  if (c->scal) cudaFree(c->scal);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->timing) {
    for (int k = 0; k < PK_COUNT; ++k)
      for (int p = 0; p < 2; ++p)
        for (int i = 0; i < 256; ++i)
          if (c->timing->ev[k][p][i]) cudaEventDestroy(c->timing->ev[k][p][i]);
    delete c->timing;
  }
  delete c;
}

int vds_set_stream(vds_ctx *c, void *stream) {
  if (!c) return VDS_EARG;
  DeviceGuard g(c->device);
  VDS_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)stream;
  return VDS_OK;
}

int vds_timing(vds_ctx *c, int enable) {
  if (!c) return VDS_EARG;
  DeviceGuard dg(c->device);
  if (!c->timing) c->timing = new TimingPool();
  VDS_TRY(timing_harvest(c));
  TimingPool *t = c->timing;
  for (int k = 0; k < PK_COUNT; ++k) {
    t->ms[k] = 0.0;
    t->count[k] = 0;
  }
  t->on = enable != 0;
  c->launches = 0;
  return VDS_OK;
}

int vds_timing_read(vds_ctx *c, double *ms, long *launches, long *total_launches) {
  if (!c) return VDS_EARG;
  DeviceGuard dg(c->device);
  if (c->timing) VDS_TRY(timing_harvest(c));
  for (int k = 0; k < PK_COUNT; ++k) {
    if (ms) ms[k] = c->timing ? c->timing->ms[k] : 0.0;
    if (launches) launches[k] = c->timing ? c->timing->count[k] : 0;
  }
  if (total_launches) *total_launches = c->launches;
  return VDS_OK;
}

int vds_energy_grad(vds_ctx *c, const float *q, int N, int D, const vds_params *p,
                    const float *q_star, double *E, float *g, float *rho) {
  if (!c || !q) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  if (q_star && !(p->dt > 0.0)) return VDS_EARG;
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  const float *qa = q_star ? q : nullptr;
  VDS_TRY(pass_prep(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  VDS_TRY(pass_density(c, kp, rho, E != nullptr, q, nullptr, qa, q_star));
  if (g) VDS_TRY(pass_grad(c, kp, GM_OUT, g, q, nullptr, qa, q_star, nullptr));
  if (E) {
    VDS_TRY(read_scalars(c));
    *E = c->h_scal[SC_E];
  }
  return VDS_OK;
}

int vds_density_rows(vds_ctx *c, const float *q, int N, int D, const vds_params *p, int row0, int nrows,
                     float *rho_rows) {
  if (!c || !q || !rho_rows || row0 < 0 || nrows < 1) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  if ((long)row0 + nrows > N) return VDS_EARG;
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  VDS_TRY(pass_density_rows(c, kp, q, row0, nrows, rho_rows));
  return VDS_OK;
}

int vds_grad_rows(vds_ctx *c, const float *q, int N, int D, const vds_params *p, const float *rho, int row0,
                  int nrows, int mode, float *out) {
  if (!c || !q || !rho || !out || row0 < 0 || nrows < 1 || (mode != 0 && mode != 1)) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  if ((long)row0 + nrows > N) return VDS_EARG;
  if (mode == 1 && !(p->dt > 0.0)) return VDS_EARG;
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  VDS_TRY(pass_grad_rows(c, kp, q, rho, row0, nrows, mode, out));
  return VDS_OK;
}

int vds_density_tc(vds_ctx *c, const float *q, int N, int D, const vds_params *p, float *rho) {
  if (!c || !q || !rho) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  if (D != 6 && D != 9) return VDS_EARG;
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  VDS_TRY(pass_prep(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  return pass_density_tc(c, kp, rho);
}

int vds_density_at(vds_ctx *c, const float *q, int N, int D, const vds_params *p, const float *y, int M,
                   float *f) {
  if (!c || !q || !y || !f || M < 1) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  return pass_density_at(c, kp, q, y, M, f);
}

// Explicit steps.  After the first (launched directly; it sizes every buffer
// a step uses), the steps replay one captured CUDA graph of a step (density
// pass, its epilogue, gradient pass, the fused update: four kernels with the
// same arguments every step), which takes the per-launch host cost out of
// small clouds.  With phase timing on (its events belong to single
// launches), or if the capture fails, the steps are launched one by one.
static int step_explicit(vds_ctx *c, float *q, const KParams &kp, int nsteps) {
  VDS_TRY(pass_prep(c, kp, q, nullptr, nullptr, 0.f, nullptr));
  auto one_step = [&]() -> int {
    VDS_TRY(pass_density(c, kp, nullptr, false, q, nullptr, nullptr, nullptr));
    return pass_grad(c, kp, GM_EXPLICIT, nullptr, q, nullptr, nullptr, nullptr, q);
  };
  int n = 0;
  if (nsteps > 0) {
    VDS_TRY(one_step());
    ++n;
  }
  cudaGraphExec_t gexec = nullptr;
  long per_step = 0;
  if (nsteps - n >= 2 && !(c->timing && c->timing->on)) {
    // captured on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured), launched on the caller's stream
    const long l0 = c->launches;
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr, user = c->stream;
    int st = VDS_OK;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      st = VDS_ECUDA;
    } else if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = VDS_ECUDA;
    } else {
      c->stream = cs;
      st = one_step();
      c->stream = user;
      const cudaError_t ec = cudaStreamEndCapture(cs, &g);
      if (st == VDS_OK && ec != cudaSuccess) st = VDS_ECUDA;
    }
    c->stream = user;
    if (cs) cudaStreamDestroy(cs);
    if (st == VDS_OK && cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess) {
      gexec = nullptr;
      st = VDS_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    per_step = c->launches - l0;
    c->launches = l0;
    if (st != VDS_OK) {
      (void)cudaGetLastError();  // a failed capture leaves its status behind
      if (gexec) cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
  }
  int st = VDS_OK;
  for (; n < nsteps && gexec; ++n) {
    if (cudaGraphLaunch(gexec, c->stream) != cudaSuccess) {
      st = VDS_ECUDA;
      break;
    }
    c->launches += per_step;
  }
  for (; st == VDS_OK && n < nsteps; ++n) st = one_step();
  const int sst = vds_sync_status(c);  // the replays have finished before the graph goes
  if (gexec) cudaGraphExecDestroy(gexec);
  return st != VDS_OK ? st : sst;
}

// Implicit Euler step as the minimiser of J (see vds.h).  y = q* + d is
// carried through d = y - q*, which keeps the dissipation term of J accurate
// in FP32.
static int step_implicit(vds_ctx *c, float *q, const KParams &kp, const vds_params *p, int nsteps,
                         int *iters_out) {
  const size_t nd = (size_t)kp.N * kp.D;
  VDS_TRY(vds_ensure(c, c->vecs, 4 * nd * sizeof(float)));
  float *qs = vec(c, 0, nd), *d0 = vec(c, 1, nd), *d1 = vec(c, 2, nd), *dir = vec(c, 3, nd);
  for (int n = 0; n < nsteps; ++n) {
    VDS_TRY(pass_flow(c, kp, q, qs));
    // start from y = q* + (the previous step's solution - its q*): the
    // correction varies slowly between steps, so the minimiser usually needs
    // one gradient evaluation fewer; q* itself for the first step of a call or
    // when that start leaves the FENE domain
    double J = 0.0;
    bool warm = n > 0;
    for (;;) {
      if (!warm) VDS_CUDA_TRY(cudaMemsetAsync(d0, 0, nd * sizeof(float), c->stream));
      VDS_TRY(pass_prep(c, kp, qs, d0, nullptr, 0.f, nullptr));
      VDS_TRY(pass_density(c, kp, nullptr, true, qs, d0, d0, nullptr));
      const int st = read_scalars(c);
      if (st == VDS_EDOMAIN && warm) {
        warm = false;
        continue;
      }
      VDS_TRY(st);
      J = c->h_scal[SC_E];
      break;
    }
    int it = 0;
    bool converged = false;
    while (it < p->max_iter) {
      ++it;
      VDS_TRY(pass_grad(c, kp, GM_IMPLICIT_DIR, dir, qs, d0, nullptr, nullptr, nullptr));
      VDS_TRY(read_scalars(c));
      const double dec = c->h_scal[SC_DEC], dmax = c->h_scal[SC_DMAX], ymax = c->h_scal[SC_YMAX];
      if (dmax <= p->tol * (1.0 + ymax)) {
        VDS_TRY(pass_prep(c, kp, qs, d0, dir, 1.f, d1));
        float *t = d0;
        d0 = d1;
        d1 = t;
        converged = true;
        break;
      }
      double alpha = 1.0, Jn = 0.0;
      bool acc = false;
      for (int ls = 0; ls <= 30; ++ls) {
        VDS_TRY(pass_prep(c, kp, qs, d0, dir, (float)alpha, d1));
        VDS_TRY(pass_density(c, kp, nullptr, true, qs, d1, d1, nullptr));
        const int st = read_scalars(c);
        if (st != VDS_OK && st != VDS_EDOMAIN) return st;
        Jn = c->h_scal[SC_E];
        if (st == VDS_OK && Jn <= J - 1e-4 * alpha * dec + p->jfloor * (1.0 + fabs(J))) {
          acc = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!acc) return VDS_ENOCONV;
      float *t = d0;
      d0 = d1;
      d1 = t;
      J = Jn;
    }
    if (iters_out) iters_out[n] = it;
    VDS_TRY(pass_axpy(c, (int)nd, qs, d0, q));
    if (!converged) {
      VDS_TRY(vds_sync_status(c));
      return VDS_ENOCONV;
    }
  }
  return vds_sync_status(c);
}

int vds_step(vds_ctx *c, float *q, int N, int D, const vds_params *p, int nsteps, int *iters_out) {
  if (!c || !q || nsteps < 0) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  if (!(p->dt > 0.0)) return VDS_EARG;
  if (p->scheme == 1 && (p->max_iter < 1 || !(p->tol >= 0.0))) return VDS_EARG;
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  if (nsteps == 0) return VDS_OK;
  if (p->scheme == 0) return step_explicit(c, q, kp, nsteps);
  if (p->scheme == 1) return step_implicit(c, q, kp, p, nsteps, iters_out);
  return VDS_EARG;
}

int vds_stress(vds_ctx *c, const float *q, int N, int D, const vds_params *p, double *tau,
               double *qq) {
  if (!c || !q || !tau) return VDS_EARG;
  VDS_TRY(check_params(p, N, D));
  DeviceGuard dg(c->device);
  const KParams kp = make_kparams(p, N, D);
  return pass_stress(c, kp, q, tau, qq);
}

}  // extern "C"
