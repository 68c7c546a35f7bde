// pair.cuh -- host-side interface of the O(N^2) Gaussian-kernel pair passes
// and their fused epilogues (pair.cu).
#pragma once
#include "vds_internal.cuh"

// Stream-K schedule of a pair pass: the (i-tile, j-chunk) items of the N x N
// pair square, flattened i-tile major, are split into G contiguous equal
// ranges, one per CTA of a grid sized to the resident capacity of the GPU.
// A CTA accumulates in registers while its i-tile is unchanged and writes one
// FP64 partial per (i-tile, segment); an epilogue sums the segments of each
// i-tile in a fixed order, so results do not depend on timing.
struct Sched {
  long long items;  // n_itiles * nchunk
  int G;            // CTAs
  int nchunk;       // j-chunks (tiles of TJ records) per i-tile
  int n_itiles;
  int maxseg;       // max segments per i-tile
  int TI;           // particles per i-tile
  int Npad;         // N rounded up to a multiple of TJ (j records)
  int Nipad;        // rows of the i-record array (= Npad unless the i points
                    // are other points than the particles, as for queries)
};

__host__ __device__ __forceinline__ int sched_first_cta(long long x, const Sched &s) {
  return (int)(((x + 1) * (long long)s.G + s.items - 1) / s.items - 1);
}

// Physical parameters as the kernels see them.
struct KParams {
  int N, D, nb, s, spring;
  float c;          // coordinate scale: qhat = c q, khat = exp2(-|dqhat|^2)
  double h, kBT, zeta, dt, b;
  double H[8];
  double kappa[9];
  double lnorm;     // -ln N - (D/2) ln(2 pi h^2)
  double sfac;      // S = -sfac * sum u dqhat, sfac = 1/(h^2 c)
};

KParams make_kparams(const vds_params *p, int N, int D);

// Records of y = base + delta (delta may be NULL) scaled by c, with w = 0,
// padded to Npad with padding records.  If delta_out != NULL it receives
// delta - alpha*dir (and the record is built from base + that).
// Rows of the record array written by pass_prep for N particles: N rounded
// up to the pair passes' j-tile, the rows beyond N far away (kernel value 0)
// with w = 0.
int pass_npad(int N);
int pass_prep(vds_ctx *c, const KParams &kp, const float *base, const float *delta,
              const float *dir, float alpha, float *delta_out);

// Density pass: rho_I over all J, then the epilogue: w_I = 1/rho_I into the
// records, optional rho output, and when want_energy, the FP64 energy
//   (1/N) sum_I [kBT (ln rho_I + lnorm) + Psi(y_I)]
//   + (zeta/2dt)(1/N) sum_I dI^T (A^-1 (x) I) dI,   dI = qa_I - qb_I
// (the quadratic term only when qa != NULL; qb may be NULL) into scal[SC_E].
// y_I = ybase_I + ydelta_I (ydelta may be NULL).  expand: large clouds take
// the squared distances through the records' norms (D + 2 instead of 2D + 1
// FP32 operations per pair; 1e-6 relative in the kernel values), for the
// reduced model's refresh cycle; the records must come from pass_prep.
int pass_density(vds_ctx *c, const KParams &kp, float *rho_out, bool want_energy,
                 const float *ybase, const float *ydelta, const float *qa,
                 const float *qb, bool expand = false);

// The same density without the energy, with the pair dot products on the
// tensor cores (dens_tc.cu: 3xTF32; 1e-5 relative for the median particle of
// an equilibrium cloud, 1e-4 at its outermost, more on stretched clouds): w_I = 1/rho_I
// into the records (which must come from pass_prep), optional rho output.
// D = 6 and 9 only; VDS_EARG otherwise, and the caller takes pass_density.
int pass_density_tc(vds_ctx *c, const KParams &kp, float *rho_out);
// The operand images of that density (a_I rows and b_J rows, TF32 hi/lo
// split, 128 bytes per row, rows [0, pass_npad(N)) in 8-row groups of 1024
// bytes) from the records in ctx->rec, into the context's workspace: for the
// refresh, which forms its kernel values from the same dot products.  D = 6
// and 9 only (VDS_EARG otherwise).
int pass_density_tc_images(vds_ctx *c, int N, int D, const uint8_t **aimg, const uint8_t **bimg);

// Gradient pass (records must hold w from pass_density) and its epilogues.
enum GradMode { GM_OUT = 0, GM_EXPLICIT = 1, GM_IMPLICIT_DIR = 2, GM_VEL = 3 };
// GM_OUT: g = kBT S + grad Psi(y) (+ (zeta/dt)(A^-1 (x) I)(qa - qb) if qa).
// GM_EXPLICIT: q_io += dt [kappa q - (1/zeta)(A (x) I) g]; rebuild records.
// GM_VEL: out = kappa y - (1/zeta)(A (x) I) g (the particle velocity).
// GM_IMPLICIT_DIR: dir = d + (dt/zeta)(A (x) I) g with d = ydelta, and
//   scal[SC_DEC] = (1/N) sum <G, dir>, G = (zeta/dt)(A^-1 (x) I) d + g,
//   scal[SC_DMAX] = max|dir|, scal[SC_YMAX] = max|y|.
int pass_grad(vds_ctx *c, const KParams &kp, int mode, float *out,
              const float *ybase, const float *ydelta, const float *qa,
              const float *qb, float *q_io);

// Stress and second moments (FP64) into host arrays.
int pass_stress(vds_ctx *c, const KParams &kp, const float *q, double *tau, double *qq);

// Kernel density estimate at M query points y (M x D):
//   f_out[J] = (1/N)(2 pi h^2)^(-D/2) sum_I exp(-|y_J - q_I|^2 / (2 h^2)),
// the particles' records built from q, the queries' in their own buffer.
int pass_density_at(vds_ctx *c, const KParams &kp, const float *q, const float *y, int M, float *f_out);

// y = base + delta -> out (element-wise, N x D).
int pass_axpy(vds_ctx *c, int n, const float *base, const float *delta, float *out);
// qs = q + dt kappa q (per bond).
int pass_flow(vds_ctx *c, const KParams &kp, const float *q, float *qs);

// Row-range passes (rows row0 .. row0 + nrows - 1 against all N columns):
// rho of the rows; and, given rho of all N particles, g of the rows (mode 0)
// or their explicit Euler update (mode 1) into out (nrows x D).
int pass_density_rows(vds_ctx *c, const KParams &kp, const float *q, int row0, int nrows, float *rho);
int pass_grad_rows(vds_ctx *c, const KParams &kp, const float *q, const float *rho, int row0, int nrows,
                   int mode, float *out);
