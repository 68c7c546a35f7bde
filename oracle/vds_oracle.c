/*
 * vds_oracle.c -- plain FP64 CPU oracle for the VDS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA
 * library: every formula below is written out again from the paper.
 *
 * Paper: Fang, Bao, Song, Xu, Huang, "Reduced-Order Variational
 * Deterministic-Particle-Based Scheme for Fokker-Planck Equations in
 * Microscopic Polymer Dynamics" (arXiv 2603.12550).
 *
 * Notation (paper -> here):  P representative particles -> N;
 * (N-1) bonds -> nb;  spatial dimension d -> s;  per-particle configuration
 * dimension (N-1)d -> D = nb*s.  q is row-major N x D; bond k of particle I
 * occupies q[I*D + s*k + alpha], alpha < s.
 *
 * Everything is evaluated literally: O(N^2) double loops, sequential FP64
 * sums over J for each I, OpenMP only across independent I.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define OR_OK 0
#define OR_EARG (-1)
#define OR_EDOMAIN (-3)
#define OR_ENOCONV (-4)

typedef struct {
  int spring;       /* 0 Hookean (Eq. model_Hookean), 1 FENE */
  int nb;           /* bonds per chain (paper N-1) */
  int s;            /* spatial dimension (paper d) */
  int max_iter;     /* implicit minimiser: max gradient evaluations */
  double H[8];      /* spring constants H_j */
  double b;         /* FENE extensibility (|q_j|^2 < b) */
  double kBT, zeta, h, dt;
  double kappa[9];  /* s x s row-major; qdot = kappa q (velocity gradient G) */
  double tol;       /* implicit minimiser stopping tolerance */
  double jfloor;    /* Armijo round-off allowance, relative to 1 + |J| */
} or_params;

/* ---------------------------------------------------------------- kernel */

/* Unnormalised Gaussian kernel exp(-|x|^2 / (2 h^2)), Sec. 2.2 (K_h without
 * its (sqrt(2 pi) h)^{-D} prefactor, which cancels in every ratio of
 * Eq. model_DymRepPar). */
static double khat(const double *a, const double *b, int D, double h) {
  double r2 = 0.0;
  for (int c = 0; c < D; ++c) {
    double d = a[c] - b[c];
    r2 += d * d;
  }
  return exp(-r2 / (2.0 * h * h));
}

/* rho_I = sum_J khat(q_I - q_J), J over all particles including I
 * (the denominators of Eq. model_DymRepPar). */
int or_density(const double *q, long N, int D, double h, double *rho) {
  if (N < 0 || D < 1 || !(h > 0)) return OR_EARG;
#pragma omp parallel for schedule(dynamic, 16)
  for (long I = 0; I < N; ++I) {
    double acc = 0.0;
    for (long J = 0; J < N; ++J) acc += khat(q + I * D, q + J * D, D, h);
    rho[I] = acc;
  }
  return OR_OK;
}

/* Entropy gradient of Eq. model_DymRepPar with grad K_h(x) = -(x/h^2) K_h(x):
 *   S_I = -(1/h^2) sum_J khat_IJ (q_I - q_J) (1/rho_I + 1/rho_J).
 * The first term is the ratio sum_K grad K / sum_J K at I, the second the sum
 * over K of grad K(q_I - q_K) / sum_J K(q_J - q_K). */
int or_entropy_grad(const double *q, long N, int D, double h, const double *rho,
                    double *S) {
  if (N < 0 || D < 1 || !(h > 0)) return OR_EARG;
  const double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(dynamic, 16)
  for (long I = 0; I < N; ++I) {
    double acc[64];
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    for (long J = 0; J < N; ++J) {
      double k = khat(q + I * D, q + J * D, D, h);
      double w = k * (1.0 / rho[I] + 1.0 / rho[J]);
      for (int c = 0; c < D; ++c) acc[c] += w * (q[I * D + c] - q[J * D + c]);
    }
    for (int c = 0; c < D; ++c) S[I * D + c] = -ih2 * acc[c];
  }
  return OR_OK;
}

/* ---------------------------------------------------------------- springs */

/* Spring energy Psi(q_I) and its gradient for one particle.
 * Hookean (Eq. model_Hookean): Psi_j = H_j/2 |q_j|^2, grad = H_j q_j.
 * FENE (not in the paper; standard FENE law): Psi_j = -(H_j b/2) ln(1-|q_j|^2/b),
 * grad = H_j q_j / (1 - |q_j|^2/b), defined only for |q_j|^2 < b. */
static int spring_one(const double *qI, const or_params *p, double *psi,
                      double *grad) {
  const int s = p->s;
  double e = 0.0;
  for (int j = 0; j < p->nb; ++j) {
    const double *qj = qI + s * j;
    double n2 = 0.0;
    for (int a = 0; a < s; ++a) n2 += qj[a] * qj[a];
    double f;
    if (p->spring == 0) {
      e += 0.5 * p->H[j] * n2;
      f = p->H[j];
    } else {
      double x = 1.0 - n2 / p->b;
      if (!(x > 0.0)) return OR_EDOMAIN;
      e += -0.5 * p->H[j] * p->b * log(x);
      f = p->H[j] / x;
    }
    if (grad)
      for (int a = 0; a < s; ++a) grad[s * j + a] = f * qj[a];
  }
  if (psi) *psi = e;
  return OR_OK;
}

/* Rouse matrix A_jk = 2 [j=k] - [|j-k|=1] (Sec. 2.1). */
static double rouse(int j, int k) {
  if (j == k) return 2.0;
  if (j - k == 1 || k - j == 1) return -1.0;
  return 0.0;
}

/* Closed-form inverse of the tridiagonal Rouse matrix, 0-based indices:
 * (A^-1)_jk = min(j+1,k+1) (nb+1-max(j+1,k+1)) / (nb+1). */
static double rouse_inv(int j, int k, int nb) {
  int a = (j < k ? j : k) + 1, b = (j > k ? j : k) + 1;
  return (double)a * (double)(nb + 1 - b) / (double)(nb + 1);
}

double or_rouse(int j, int k) { return rouse(j, k); }
double or_rouse_inv(int j, int k, int nb) { return rouse_inv(j, k, nb); }

/* ------------------------------------------------------- energy, gradient */

/* Discrete free energy E = (1/N) sum_I [kBT ln f_h(q_I) + Psi(q_I)] with
 * f_h(q_I) = (2 pi h^2)^{-D/2} rho_I / N (Eq. model_DeteParAppr with the
 * Gaussian K_h), and g_I = N dE/dq_I = kBT S_I + grad Psi(q_I).
 * rho (optional) receives rho_I; g may be NULL for energy only. */
int or_energy_grad(const double *q, long N, int D, const or_params *p,
                   double *E, double *g, double *rho_out) {
  if (N < 1 || D != p->nb * p->s || D > 64) return OR_EARG;
  double *rho = (double *)malloc(sizeof(double) * (size_t)N);
  if (!rho) return OR_EARG;
  int st = or_density(q, N, D, p->h, rho);
  if (st) { free(rho); return st; }
  const double lnorm = -log((double)N) - 0.5 * D * log(2.0 * M_PI * p->h * p->h);
  double esum = 0.0;
  int bad = 0;
  for (long I = 0; I < N; ++I) {
    double psi;
    if (spring_one(q + I * D, p, &psi, NULL)) { bad = 1; break; }
    esum += p->kBT * (log(rho[I]) + lnorm) + psi;
  }
  if (bad) { free(rho); return OR_EDOMAIN; }
  if (E) *E = esum / (double)N;
  if (g) {
    st = or_entropy_grad(q, N, D, p->h, rho, g);
    if (st) { free(rho); return st; }
    double gs[64];
    for (long I = 0; I < N; ++I) {
      spring_one(q + I * D, p, NULL, gs);
      for (int c = 0; c < D; ++c) g[I * D + c] = p->kBT * g[I * D + c] + gs[c];
    }
  }
  if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)N);
  free(rho);
  return OR_OK;
}

/* ---------------------------------------------------------- explicit step */

/* Flow term kappa q_k per bond (G q_{k,I} in Eq. model_DymRepPar). */
static void flow(const double *qI, const or_params *p, double *out) {
  const int s = p->s;
  for (int k = 0; k < p->nb; ++k)
    for (int a = 0; a < s; ++a) {
      double v = 0.0;
      for (int b = 0; b < s; ++b) v += p->kappa[a * s + b] * qI[s * k + b];
      out[s * k + a] = v;
    }
}

/* First-order explicit Euler of Eq. model_DymRepPar (Appendix A, explicit
 * scheme):  q_{k,I} += dt [kappa q_{k,I} - (1/zeta) sum_j A_kj g_{I,j}]. */
int or_explicit_steps(double *q, long N, int D, const or_params *p, int nsteps) {
  if (N < 1 || D != p->nb * p->s) return OR_EARG;
  double *g = (double *)malloc(sizeof(double) * (size_t)N * D);
  if (!g) return OR_EARG;
  const int s = p->s, nb = p->nb;
  for (int n = 0; n < nsteps; ++n) {
    int st = or_energy_grad(q, N, D, p, NULL, g, NULL);
    if (st) { free(g); return st; }
    for (long I = 0; I < N; ++I) {
      double fl[64], v[64];
      flow(q + I * D, p, fl);
      for (int k = 0; k < nb; ++k)
        for (int a = 0; a < s; ++a) {
          double m = 0.0;
          for (int j = 0; j < nb; ++j) m += rouse(k, j) * g[I * D + s * j + a];
          v[s * k + a] = fl[s * k + a] - m / p->zeta;
        }
      for (int c = 0; c < D; ++c) q[I * D + c] += p->dt * v[c];
    }
  }
  free(g);
  return OR_OK;
}

/* ---------------------------------------------------------- implicit step */

/* Objective of one implicit step (Appendix A, implicit scheme, read as a
 * minimising movement):
 *   J(y) = (1/N) sum_I (zeta/(2 dt)) (y_I - q*_I)^T (A^-1 (x) I_s) (y_I - q*_I) + E(y),
 * q* = q + dt kappa q.  Its stationarity condition
 *   y_I = q*_I - (dt/zeta) (A (x) I_s) g_I(y)
 * is the appendix's implicit equation with the flow at t and the rest at t+. */
static int objective(const double *y, const double *qs, long N, int D,
                     const or_params *p, double *J, double *g, double *E_out) {
  double E;
  int st = or_energy_grad(y, N, D, p, &E, g, NULL);
  if (st) return st;
  const int s = p->s, nb = p->nb;
  double quad = 0.0;
  for (long I = 0; I < N; ++I) {
    double acc = 0.0;
    for (int j = 0; j < nb; ++j)
      for (int k = 0; k < nb; ++k) {
        double ai = rouse_inv(j, k, nb);
        for (int a = 0; a < s; ++a)
          acc += (y[I * D + s * j + a] - qs[I * D + s * j + a]) * ai *
                 (y[I * D + s * k + a] - qs[I * D + s * k + a]);
      }
    quad += acc;
  }
  *J = (p->zeta / (2.0 * p->dt)) * quad / (double)N + E;
  if (E_out) *E_out = E;
  return OR_OK;
}

/* Minimiser (the paper solves the implicit equation "by iteration"):
 * preconditioned descent on J,
 *   dir_I = (y_I - q*_I) + (dt/zeta) (A (x) I_s) g_I(y)   [= (dt/zeta)(A(x)I) G_I],
 *   G_I   = N dJ/dy_I = (zeta/dt)(A^-1 (x) I)(y_I - q*_I) + g_I,
 * starting at y = q*.  When max|dir| <= tol (1 + max|y|) the unit step is
 * taken and the iteration stops.  Otherwise y' = y - alpha dir with Armijo
 * acceptance J(y') <= J(y) - 1e-4 alpha (1/N) sum_I <G_I, dir_I>, alpha halved
 * on rejection (at most 30 halvings).  The test allows a round-off floor of
 * jfloor (1 + |J(y)|), so that steps whose true decrease lies below the
 * precision of J are not rejected.  alpha = 1 is the plain fixed-point
 * (Picard) iteration of the implicit equation.  iters counts gradient
 * evaluations. */
int or_implicit_steps(double *q, long N, int D, const or_params *p, int nsteps,
                      int *iters_out) {
  if (N < 1 || D != p->nb * p->s || p->dt <= 0) return OR_EARG;
  const size_t ND = (size_t)N * D;
  double *qs = malloc(sizeof(double) * ND), *y = malloc(sizeof(double) * ND);
  double *g = malloc(sizeof(double) * ND), *dir = malloc(sizeof(double) * ND);
  double *yn = malloc(sizeof(double) * ND), *gn = malloc(sizeof(double) * ND);
  int ret = OR_OK;
  if (!qs || !y || !g || !dir || !yn || !gn) { ret = OR_EARG; goto done; }
  const int s = p->s, nb = p->nb;
  for (int n = 0; n < nsteps; ++n) {
    for (long I = 0; I < N; ++I) {
      double fl[64];
      flow(q + I * D, p, fl);
      for (int c = 0; c < D; ++c) qs[I * D + c] = q[I * D + c] + p->dt * fl[c];
    }
    memcpy(y, qs, sizeof(double) * ND);
    double Jy;
    int st = objective(y, qs, N, D, p, &Jy, g, NULL);
    if (st) { ret = st; goto done; }
    int it = 0, converged = 0;
    while (it < p->max_iter) {
      ++it;
      double dec = 0.0, dmax = 0.0, ymax = 0.0;
      for (long I = 0; I < N; ++I) {
        for (int k = 0; k < nb; ++k)
          for (int a = 0; a < s; ++a) {
            double ag = 0.0, aid = 0.0;
            for (int j = 0; j < nb; ++j) {
              ag += rouse(k, j) * g[I * D + s * j + a];
              aid += rouse_inv(k, j, nb) * (y[I * D + s * j + a] - qs[I * D + s * j + a]);
            }
            double d = (y[I * D + s * k + a] - qs[I * D + s * k + a]) + (p->dt / p->zeta) * ag;
            double G = (p->zeta / p->dt) * aid + g[I * D + s * k + a];
            dir[I * D + s * k + a] = d;
            dec += G * d;
            if (fabs(d) > dmax) dmax = fabs(d);
            if (fabs(y[I * D + s * k + a]) > ymax) ymax = fabs(y[I * D + s * k + a]);
          }
      }
      dec /= (double)N;
      if (dmax <= p->tol * (1.0 + ymax)) {
        for (size_t c = 0; c < ND; ++c) y[c] -= dir[c];
        converged = 1;
        break;
      }
      double alpha = 1.0, Jn = 0.0;
      int acc = 0;
      for (int ls = 0; ls <= 30; ++ls) {
        for (size_t c = 0; c < ND; ++c) yn[c] = y[c] - alpha * dir[c];
        st = objective(yn, qs, N, D, p, &Jn, gn, NULL);
        if (st == OR_OK && Jn <= Jy - 1e-4 * alpha * dec + p->jfloor * (1.0 + fabs(Jy))) {
          acc = 1;
          break;
        }
        if (st != OR_OK && st != OR_EDOMAIN) { ret = st; goto done; }
        alpha *= 0.5;
      }
      if (!acc) { ret = OR_ENOCONV; goto done; }
      memcpy(y, yn, sizeof(double) * ND);
      memcpy(g, gn, sizeof(double) * ND);
      Jy = Jn;
    }
    if (iters_out) iters_out[n] = it;
    memcpy(q, y, sizeof(double) * ND);
    if (!converged) { ret = OR_ENOCONV; goto done; }
  }
done:
  free(qs); free(y); free(g); free(dir); free(yn); free(gn);
  return ret;
}

/* ----------------------------------------------------------------- stress */

/* Discrete polymer stress (Appendix A, with n = 1):
 *   tau = (1/N) sum_I sum_k q_{k,I} (x) grad Psi_k(q_{k,I})    (s x s)
 * and the second moments qq = (1/N) sum_I q_I q_I^T (D x D). */
int or_stress(const double *q, long N, int D, const or_params *p, double *tau,
              double *qq) {
  if (N < 1 || D != p->nb * p->s) return OR_EARG;
  const int s = p->s;
  for (int c = 0; c < s * s; ++c) tau[c] = 0.0;
  if (qq) for (int c = 0; c < D * D; ++c) qq[c] = 0.0;
  for (long I = 0; I < N; ++I) {
    double gs[64];
    if (spring_one(q + I * D, p, NULL, gs)) return OR_EDOMAIN;
    for (int k = 0; k < p->nb; ++k)
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) tau[a * s + b] += q[I * D + s * k + a] * gs[s * k + b];
    if (qq)
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) qq[a * D + b] += q[I * D + a] * q[I * D + b];
  }
  for (int c = 0; c < s * s; ++c) tau[c] /= (double)N;
  if (qq) for (int c = 0; c < D * D; ++c) qq[c] /= (double)N;
  return OR_OK;
}

/* -------------------------------------------------------------- bandwidth */

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Median pairwise distance of Eq. model_bandwidth over distinct unordered
 * pairs J < K; for an even count the lower middle order statistic
 * (0-based rank (M-1)/2 of the M = N(N-1)/2 sorted distances). */
int or_median_pairdist(const double *q, long N, int D, double *med) {
  if (N < 2) return OR_EARG;
  long M = N * (N - 1) / 2;
  double *r = (double *)malloc(sizeof(double) * (size_t)M);
  if (!r) return OR_EARG;
  long t = 0;
  for (long J = 0; J < N; ++J)
    for (long K = J + 1; K < N; ++K) {
      double r2 = 0.0;
      for (int c = 0; c < D; ++c) {
        double d = q[J * D + c] - q[K * D + c];
        r2 += d * d;
      }
      r[t++] = sqrt(r2);
    }
  qsort(r, (size_t)M, sizeof(double), cmp_double);
  *med = r[(M - 1) / 2];
  free(r);
  return OR_OK;
}

/* Pair counts for checking an order statistic at sizes where sorting all
 * N(N-1)/2 distances does not fit: number of unordered pairs J < K with
 * |q_J - q_K|^2 < r2 (n_lt) and <= r2 (n_le). */
int or_count_pairs(const double *q, long N, int D, double r2, long *n_lt, long *n_le) {
  long lt = 0, le = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : lt, le)
  for (long J = 0; J < N; ++J)
    for (long K = J + 1; K < N; ++K) {
      double d2 = 0.0;
      for (int c = 0; c < D; ++c) {
        double d = q[J * D + c] - q[K * D + c];
        d2 += d * d;
      }
      lt += (d2 < r2);
      le += (d2 <= r2);
    }
  *n_lt = lt;
  *n_le = le;
  return OR_OK;
}

/* Same counts with the squared distances rounded to FP32 before comparing
 * against an FP32 threshold: the order statistic the single-precision path
 * selects is defined on these rounded keys. */
int or_count_pairs_f32(const float *q, long N, int D, float r2, long *n_lt, long *n_le) {
  long lt = 0, le = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : lt, le)
  for (long J = 0; J < N; ++J)
    for (long K = J + 1; K < N; ++K) {
      double d2 = 0.0;
      for (int c = 0; c < D; ++c) {
        double d = (double)q[J * D + c] - (double)q[K * D + c];
        d2 += d * d;
      }
      float f = (float)d2;
      lt += (f < r2);
      le += (f <= r2);
    }
  *n_lt = lt;
  *n_le = le;
  return OR_OK;
}

/* ------------------------------------------ reduced-order pair quantities */

/* Pair sums behind the frozen Brownian terms of Eq. model_DymReduced
 * (Sec. 2.4): for each particle I and column t of the basis block
 * Phi_K = U_{(K alpha) t} (rows K*s + alpha),
 *   W1_(I alpha) t = sum_K Z_IK U_(K alpha) t,
 *   W2_(I alpha) t = sum_K Z_IK U_(K alpha) t / rho_K,
 *   c_I            = sum_K Z_IK / rho_K,
 * with Z_IK = khat(q_I - q_K) evaluated at the given state q (N x D). */
int or_refresh_sums(const double *q, long N, int D, double h, const double *rho,
                    const double *U, int s, int r, double *W1, double *W2,
                    double *c) {
#pragma omp parallel for schedule(dynamic, 16)
  for (long I = 0; I < N; ++I) {
    double ci = 0.0;
    for (int a = 0; a < s; ++a)
      for (int t = 0; t < r; ++t) {
        W1[(I * s + a) * r + t] = 0.0;
        W2[(I * s + a) * r + t] = 0.0;
      }
    for (long K = 0; K < N; ++K) {
      double z = khat(q + I * D, q + K * D, D, h);
      ci += z / rho[K];
      for (int a = 0; a < s; ++a)
        for (int t = 0; t < r; ++t) {
          double u = U[(K * s + a) * r + t];
          W1[(I * s + a) * r + t] += z * u;
          W2[(I * s + a) * r + t] += z * u / rho[K];
        }
    }
    c[I] = ci;
  }
  return OR_OK;
}

/* Entropy gradient S_I (as or_entropy_grad) for a subset of particles only:
 * rows[0..nrows) index particles, S is nrows x D.  rho must hold the density
 * of every particle (the second term of Eq. model_DymRepPar needs all of
 * them). */
/* rho_I (Eq. model_DeteParAppr without the normalisation) for the particles
 * in rows only: the same sum as or_density, O(N) per row. */
int or_density_rows(const double *q, long N, int D, double h, const long *rows, long nrows,
                    double *rho) {
  if (N < 0 || D < 1 || !(h > 0)) return OR_EARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (long r = 0; r < nrows; ++r) {
    const long I = rows[r];
    double acc = 0.0;
    for (long J = 0; J < N; ++J) acc += khat(q + I * D, q + J * D, D, h);
    rho[r] = acc;
  }
  return OR_OK;
}

int or_entropy_grad_rows(const double *q, long N, int D, double h, const double *rho,
                         const long *rows, long nrows, double *S) {
  if (N < 0 || D < 1 || D > 64 || !(h > 0)) return OR_EARG;
  const double ih2 = 1.0 / (h * h);
#pragma omp parallel for schedule(dynamic, 1)
  for (long r = 0; r < nrows; ++r) {
    const long I = rows[r];
    double acc[64];
    for (int c = 0; c < D; ++c) acc[c] = 0.0;
    for (long J = 0; J < N; ++J) {
      double k = khat(q + I * D, q + J * D, D, h);
      double w = k * (1.0 / rho[I] + 1.0 / rho[J]);
      for (int c = 0; c < D; ++c) acc[c] += w * (q[I * D + c] - q[J * D + c]);
    }
    for (int c = 0; c < D; ++c) S[r * D + c] = -ih2 * acc[c];
  }
  return OR_OK;
}
