/*
 * vds.h -- C ABI of the GB300 (sm_103a) hot path of the reduced-order
 * variational deterministic-particle scheme (VDS with POD) for the
 * microscopic Fokker-Planck equation of bead-spring chains in homogeneous
 * flow (Fang, Bao, Song, Xu, Huang, arXiv 2603.12550).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Notation: N representative particles (the paper's P); nb bonds per chain
 *    (the paper's N-1); s spatial dimension (the paper's d); D = nb*s
 *    coordinates per particle (the paper's (N-1)d).  1 <= D <= 16, s in {2,3},
 *    1 <= nb <= 8.
 *  - Particle arrays are DEVICE pointers to row-major N x D FP32, contiguous;
 *    bond k of particle I is q[I*D + s*k + alpha].  The caller owns them.
 *  - Scalars written to the host (E, h, tau, r, iters) are HOST pointers; the
 *    call synchronises the context stream before returning them.  Every other
 *    call is asynchronous on the context stream.
 *  - The library owns the context (its stream binding and device workspace)
 *    and pod_basis objects.
 *  - Return value: VDS_OK or a negative status; on error the outputs are
 *    unspecified and no memory is leaked.  Device-side failures (a FENE bond
 *    leaving |q|^2 < b, a NaN, a wait that gave up) are reported by the next
 *    call that synchronises (every call returning host scalars, and vds_step).
 */
#ifndef VDS_H
#define VDS_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define VDS_API __attribute__((visibility("default")))
#else
#define VDS_API
#endif

typedef struct vds_ctx vds_ctx;
typedef struct pod_basis pod_basis;

enum {
  VDS_OK = 0,
  VDS_EARG = -1,      /* invalid argument (size, pointer, parameter) */
  VDS_ECUDA = -2,     /* CUDA runtime error */
  VDS_EDOMAIN = -3,   /* FENE bond with |q_j|^2 >= b */
  VDS_ENOCONV = -4,   /* implicit minimiser did not converge */
  VDS_ENAN = -5,      /* non-finite density / energy */
  VDS_ETIMEOUT = -6,  /* a bounded device-side wait gave up */
  VDS_ENOMEM = -7,    /* device allocation failed */
  VDS_ESURROGATE = -8, /* surrogate check failed */
  VDS_ESIZE = -9       /* problem larger than a fixed-size buffer allows */
};

/* Physical and numerical parameters (Sec. 2.1-2.2, Sec. 3.1, Appendix A). */
typedef struct {
  int spring;       /* 0: Hookean Psi_j = H_j|q_j|^2/2 (Eq. model_Hookean);
                       1: FENE Psi_j = -(H_j b/2) ln(1-|q_j|^2/b) */
  int nb;           /* bonds per chain */
  int s;            /* spatial dimension */
  int max_iter;     /* implicit minimiser: max gradient evaluations per step */
  double H[8];      /* spring constants H_j, j < nb */
  double b;         /* FENE extensibility */
  double kBT;       /* thermal energy */
  double zeta;      /* friction */
  double h;         /* kernel bandwidth (Eq. model_bandwidth or given) */
  double dt;        /* time step */
  double kappa[9];  /* s x s row-major velocity gradient G = (grad u)^T,
                       acting as qdot = kappa q */
  double tol;       /* minimiser stop: max|dir| <= tol (1 + max|y|) */
  double jfloor;    /* Armijo round-off allowance, relative to 1 + |J| */
  int scheme;       /* vds_step: 0 explicit Euler, 1 implicit Euler */
  int reserved;
} vds_params;

/* Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream). */
VDS_API int vds_create(vds_ctx **ctx, void *cuda_stream, int device);
VDS_API void vds_destroy(vds_ctx *ctx);
/* Rebind the context to another stream of the same device. */
VDS_API int vds_set_stream(vds_ctx *ctx, void *cuda_stream);
VDS_API const char *vds_strerror(int status);

/* Kernel bandwidth (Sec. 2.2).  rule 0: median rule of Eq. model_bandwidth,
 * h = med_{J<K} |q_J - q_K| / sqrt(2 ln N), med the lower middle order
 * statistic of the N(N-1)/2 distances (exact selection on FP32 squared
 * distances).  rule 1: Silverman, h = sigma (4/((D+2)N))^(1/(D+4)) with sigma
 * the mean per-coordinate sample standard deviation.  N >= 2.  *h: host. */
VDS_API int vds_bandwidth(vds_ctx *ctx, const float *q, int N, int D, int rule,
                  double *h);

/* Density and free-energy gradient (Eq. model_DeteParAppr, Eq. model_DymRepPar).
 *   rho_I = sum_J exp(-|q_I - q_J|^2 / 2h^2)   (self term included)
 *   S_I   = -(1/h^2) sum_J khat_IJ (q_I - q_J)(1/rho_I + 1/rho_J)
 *   E     = (1/N) sum_I [kBT ln f_h(q_I) + Psi(q_I)],
 *           f_h(q_I) = (2 pi h^2)^(-D/2) rho_I / N
 *   g_I   = N dE/dq_I = kBT S_I + grad Psi(q_I)
 * With q_star != NULL (device, N x D) and p->dt > 0 it evaluates instead the
 * implicit-step objective (Appendix A, implicit scheme)
 *   J = (1/N) sum_I (zeta/2dt)(q_I - q*_I)^T (A^-1 (x) I_s)(q_I - q*_I) + E
 * and G_I = N dJ/dq_I = (zeta/dt)(A^-1 (x) I_s)(q_I - q*_I) + g_I.
 * E: host (may be NULL); g: device N x D (may be NULL); rho: device N
 * (may be NULL). */
VDS_API int vds_energy_grad(vds_ctx *ctx, const float *q, int N, int D,
                    const vds_params *p, const float *q_star, double *E,
                    float *g, float *rho);

/* Advance q (device, N x D, in place) by nsteps time steps.
 * scheme 0, explicit Euler (Appendix A):
 *   q_{k,I} += dt [kappa q_{k,I} - (1/zeta) sum_j A_kj g_{I,j}],
 *   A_jk = 2[j=k] - [|j-k|=1] the Rouse matrix (Sec. 2.1).
 * scheme 1, implicit Euler (Appendix A), flow at t and the rest at t+dt,
 *   q+ = q* - (dt/zeta)(A (x) I_s) g(q+),  q* = q + dt kappa q,
 * solved as the minimiser of J above by preconditioned descent with FP64
 * Armijo acceptance (unit step = fixed-point iteration).  iters_out (host,
 * nsteps ints, may be NULL) receives gradient evaluations per step.
 * Explicit calls of three or more steps capture the second step as a CUDA
 * graph (on a private stream) and replay it for the rest, launched on the
 * context stream; results are bit-identical to launching every step, which
 * is what happens while vds_timing is on.  The call synchronises the
 * context stream before it returns. */
VDS_API int vds_step(vds_ctx *ctx, float *q, int N, int D, const vds_params *p,
             int nsteps, int *iters_out);

/* Polymer stress (Sec. 2.1, discrete form of Appendix A, n = 1):
 *   tau = (1/N) sum_I sum_k q_{k,I} (x) grad Psi_k(q_{k,I})   (s x s, host)
 * and second moments qq = (1/N) sum_I q_I q_I^T (D x D, host, may be NULL).
 * The Kramers form is tau - nb kBT Id. */
VDS_API int vds_stress(vds_ctx *ctx, const float *q, int N, int D, const vds_params *p,
               double *tau, double *qq);

/* Kernel density estimate of the particle cloud at M query points
 * (Eq. model_DeteParAppr; Appendix A compares runs through it on the grid
 * {-2, 0, 2}^D):
 *   f[J] = (1/N) sum_I (2 pi h^2)^(-D/2) exp(-|y_J - q_I|^2 / (2 h^2)),
 * the same Gaussian kernel and bandwidth p->h as the pair passes (which take
 * the query points to be the particles themselves: f(q_I) = rho_I (1/N)
 * (2 pi h^2)^(-D/2)).  q: device N x D, y: device M x D, f: device M (FP32);
 * p->nb, p->s give D.  One query-particle pair pass (query points as its
 * rows, counted as a density pass by vds_timing) with FP64 sums across
 * particle tiles.  Asynchronous on the context stream.  VDS_EARG for a NULL
 * pointer, N < 1, M < 1 or invalid parameters. */
VDS_API int vds_density_at(vds_ctx *ctx, const float *q, int N, int D, const vds_params *p,
                           const float *y, int M, float *f);

/* Density of every particle, rho[I] = sum_J exp(-|q_I - q_J|^2 / 2h^2)
 * (Sec. 2.2, self term included), with the pair dot products on the tensor
 * cores: -|qh_I - qh_J|^2 = 2 qh_I . qh_J - |qh_I|^2 - |qh_J|^2 as MMAs of
 * TF32 operands split into two TF32 parts each (three products per pair), the
 * exponentials on the CUDA cores.  For passes held to 1e-4 (the library
 * uses it for the density at the lifted state of the frozen reduced step's
 * refresh and for the density of the surrogate's subset check): within
 * 1e-5 relative of the exact kernel sum for the median particle of an
 * equilibrium cloud and 1e-4 at its outermost particles; the error grows with
 * |q|^2 / h^2 (3.4e-4 at the worst particle of a cloud stretched five-fold
 * along one axis at h = 0.7), faster than for the expanded form on the CUDA
 * cores, because the tensor cores accumulate the large |q|^2 terms in FP32
 * with rounding toward zero.
 * q: device N x D FP32; rho: device N FP32.  D = 6 or 9 (records with a norm
 * slot and D + 1 <= 16); VDS_EARG otherwise, for NULL pointers or invalid
 * parameters; VDS_ENAN (at the next synchronising call) for a non-finite
 * density.  Asynchronous on the context stream. */
VDS_API int vds_density_tc(vds_ctx *ctx, const float *q, int N, int D, const vds_params *p, float *rho);

/* Row-range evaluation: the pieces of one evaluation split over ranks by
 * particle rows.  The paper's cost is the O(P^2) pair sums (Sec. 1.2, The
 * VDS Scheme and its Limitation); each of G ranks takes a contiguous range
 * of rows I against all N columns J, and two all-gathers per evaluation
 * (q before the density pass, rho before the gradient pass) give every rank
 * the whole state.  The library does the per-rank pair work; the exchange is
 * the caller's (paper_2603_12550_gb300/shard.py uses torch.distributed).
 *
 * vds_density_rows: rho_rows[i] = sum_J exp(-|q_(row0+i) - q_J|^2 / 2h^2)
 * (self term included) for i < nrows, from the device array q (N x D, all
 * particles).  rho_rows: device, nrows FP32.
 * vds_grad_rows: given rho (device, N FP32: the density of every particle),
 * the gradient pass for the rows row0 .. row0+nrows-1, then
 *   mode 0: out = kBT S + grad Psi of those rows (Eq. model_DymRepPar);
 *   mode 1: out = their explicit Euler update q + dt [kappa q - (1/zeta)
 *           (A (x) I) g] (Appendix A, explicit scheme);
 * out: device nrows x D FP32 (must not overlap q).
 * Both are asynchronous on the context stream; VDS_EARG for NULL pointers,
 * nrows < 1, a range outside [0, N) or invalid parameters; VDS_ENAN (at the
 * next synchronising call) for a non-finite density.  Row-range sums are
 * split over CTAs differently from vds_energy_grad's, so results agree with
 * it within FP32 rounding, not bit for bit. */
VDS_API int vds_density_rows(vds_ctx *ctx, const float *q, int N, int D, const vds_params *p, int row0,
                             int nrows, float *rho_rows);
VDS_API int vds_grad_rows(vds_ctx *ctx, const float *q, int N, int D, const vds_params *p, const float *rho,
                          int row0, int nrows, int mode, float *out);

/* Allocation-free density and gradient evaluation.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory at the point of the call: a flow solver that couples one VDS
 * ensemble per grid point and reserves its whole device-memory budget up
 * front, a host that forbids allocation after initialisation (real-time or
 * plugin integrations), or code that must not take the allocator's locks and
 * implicit synchronisation.  It computes what vds_energy_grad computes
 * (q_star = NULL): E (host, may be NULL), g (device N x D, may be NULL) and
 * rho (device N, may be NULL) for the device array q (N x D), on the given
 * stream (a cudaStream_t of the current device; NULL = legacy default
 * stream), and synchronises that stream before returning, also when it
 * returns an error.
 *  - No context and no allocation: all scratch lives in one fixed-size static
 *    device array of the library (about 4.7 MiB, held by every GPU that loads
 *    the library until the process exits); the caller passes inputs and
 *    outputs only.
 *  - N must not exceed VDS_NOALLOC_MAX_N; larger N returns VDS_ESIZE.  Near
 *    that limit the gradient pass runs on fewer CTAs than vds_energy_grad
 *    uses (its partial sums must fit the fixed array), so it is slower there;
 *    results agree within the library's FP32 tolerance.
 *  - The first call on each device looks up the array's device address with
 *    that device current (the call's one-time set-up).
 *  - No call can be captured into a CUDA graph: each copies a status word to
 *    the host and synchronises its stream.  A call on a stream that is being
 *    captured returns VDS_EARG without enqueuing work.
 *  - Every call shares the one array: calls that overlap on the GPU (from
 *    several host threads, or on several streams) race and give wrong results.
 *    Calls made one after another do not overlap, because each synchronises
 *    its stream before returning. */
#define VDS_NOALLOC_MAX_N 8192
VDS_API int vds_energy_grad_noalloc(const float *q, int N, int D, const vds_params *p,
                                    double *E, float *g, float *rho, void *cuda_stream);

/* Instrumentation (no counterpart in the paper; used to report a kernel's
 * achieved rate).  vds_timing(ctx, 1) clears the counters and starts
 * recording the device duration of every pair-pass launch and POD phase on
 * the context stream (CUDA events around it); vds_timing(ctx, 0) stops.  The
 * library's total kernel-launch count is cleared by either call.
 * vds_timing_read synchronises and returns, per kind, the summed milliseconds
 * ms[VDS_TIMING_KINDS] and event-pair counts launches[VDS_TIMING_KINDS] (host
 * arrays of that length, may be NULL), and the number of kernels launched
 * since the last vds_timing call.  Kinds: 0 density pass, 1 gradient pass,
 * 2 bandwidth selection, 3 POD refresh pass (X^B), 4 POD Gram X^T X, 5 POD
 * eigensolve (Jacobi sweeps, sort and rank rule), 6 POD basis (Phi, Cholesky-QR,
 * sign fix, X^H). */
#define VDS_TIMING_KINDS 7
VDS_API int vds_timing(vds_ctx *ctx, int enable);
VDS_API int vds_timing_read(vds_ctx *ctx, double *ms, long *launches, long *total_launches);

/* Failure detection check (no counterpart in the paper).  Every device-side
 * wait of the library (bulk-copy and tensor-core completion barriers in the
 * pair, refresh, Gram and network kernels; the batched queue) is bounded: it
 * gives up after a time limit, raises VDS_ETIMEOUT in the context's error
 * flag and lets the kernel return, so the context stays usable.
 * vds_wait_selftest runs that pattern on two waits that nothing completes
 * (an mbarrier phase with no arrival, a device flag that no thread sets),
 * each limited to limit_s seconds (0 < limit_s <= 1), synchronises, and
 * returns the status the host reads: VDS_ETIMEOUT when the mechanism works. */
VDS_API int vds_wait_selftest(vds_ctx *ctx, double limit_s);

#ifdef __cplusplus
}
#endif
#endif /* VDS_H */
