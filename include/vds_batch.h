/*
 * vds_batch.h -- C ABI of the batched form of the VDS hot path: many
 * independent particle ensembles of uneven size (one per macroscopic grid
 * point of a micro-macro solver, the coupling the paper motivates in Sec. 1
 * and Sec. 2.1) advanced together.  Not in the paper's experiments; each
 * ensemble follows exactly the single-ensemble definitions of vds.h.
 *
 * Layout: the ensembles' particles are concatenated, ensemble e occupying
 * rows [off_e, off_e + N_e) of one device array q_all (sum N_e) x D, with
 * off_e = N_0 + ... + N_{e-1}.  Every ensemble has its own bandwidth h_e and
 * velocity gradient kappa_e; the other parameters (springs, kBT, zeta, dt,
 * scheme, tolerances) are shared.  Same status codes as vds.h.
 *
 * Work distribution: one persistent kernel per pair pass pops work items
 * (e, i-tile) from a queue in longest-processing-time order -- cost N_e
 * descending, then e ascending, then tile ascending -- with an atomic
 * counter; an item covers all j of its ensemble, so every particle's sums are
 * formed by one CTA in a fixed order and the results do not depend on the
 * schedule.
 */
#ifndef VDS_BATCH_H
#define VDS_BATCH_H

#include "vds.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vds_batch vds_batch;

/* Set up a batch of E ensembles: sizes (host, E ints, each >= 1), h (host,
 * E doubles > 0), kappa (host, E x s x s doubles, row-major per ensemble),
 * shared parameters p (p->h and p->kappa are ignored).  D = p->nb * p->s.
 * The batch owns its device workspace. */
VDS_API int vds_batch_create(vds_ctx *ctx, int E, const int *sizes, int D, const vds_params *p,
                             const double *h, const double *kappa, vds_batch **out);
VDS_API void vds_batch_free(vds_batch *b);
/* Total particle count and tile size (particles per work item). */
VDS_API int vds_batch_info(const vds_batch *b, long *total, int *tile, int *n_items);
/* Work items in queue order: items[2k] = ensemble, items[2k+1] = tile
 * (host, 2 * n_items ints). */
VDS_API int vds_batch_queue(const vds_batch *b, int *items, int n_items);

/* Per-ensemble energies E_e (host, E doubles, may be NULL), gradients g_all
 * (device, total x D, may be NULL) and densities rho_all (device, total, may
 * be NULL) of vds_energy_grad for every ensemble. */
VDS_API int vds_batch_energy_grad(vds_ctx *ctx, vds_batch *b, const float *q_all, double *E,
                                  float *g_all, float *rho_all);
/* Advance every ensemble by nsteps steps of p->scheme (as vds_step).
 * Implicit steps run all ensembles' minimisers in lockstep rounds (one
 * persistent pair pass per round, each ensemble in its own state: gradient
 * and new direction, or line-search trial), one CUDA graph per round,
 * replayed until every ensemble has converged.  iters_out (host,
 * nsteps x E ints, may be NULL) receives gradient evaluations per ensemble
 * and step; status of the first failing ensemble is returned. */
VDS_API int vds_batch_step(vds_ctx *ctx, vds_batch *b, float *q_all, int nsteps, int *iters_out);

/* Micro-macro coupling (Sec. 1: one ensemble per grid point of a
 * macroscopic solver).  vds_batch_stress: the polymer stress of every
 * ensemble, tau_e = (1/N_e) sum_I sum_k q_k (x) grad Psi_k (as vds_stress),
 * from q_all (device, total x D) into tau (host, E x s x s doubles, row-major
 * per ensemble); FP64 sums in a fixed order; synchronises.
 * vds_batch_set_kappa: new velocity gradients for every ensemble (host,
 * E x s x s doubles, qdot = kappa q), e.g. the macroscopic velocity field at
 * the ensembles' grid points, used from the next step on. */
VDS_API int vds_batch_stress(vds_ctx *ctx, vds_batch *b, const float *q_all, double *tau);
VDS_API int vds_batch_set_kappa(vds_ctx *ctx, vds_batch *b, const double *kappa);

/* Convection (the u . grad_x q term of Eq. model_DymRepPar; for reduced
 * coordinates the u . grad_x p term of Eq. model_DymReduced).  The
 * homogeneous-flow experiments of Sec. 3 drop it; a grid of ensembles needs
 * it.  One first-order upwind step of  dQ/dt + u . grad_x Q = 0  for a field
 * held at the nodes of a structured macroscopic grid nx x ny x nz, node
 * g = ix + nx (iy + ny iz), M FP32 values per node, node-major: q_in[g M + m]
 * (device).  For particle ensembles the field is q_all of ensembles of equal
 * size N, particle I being the same label at every node (M = N D); for
 * reduced coordinates it is each node's p (M = r nb).
 *   q_out[g] = q_in[g] - dt sum_b ( max(u_b,0) (q_in[g] - q_in[g - e_b])
 *                                  + min(u_b,0) (q_in[g + e_b] - q_in[g]) ) / dx_b
 * u: device G x 3 FP32 (the velocity at each node; axes of extent 1 are
 * skipped); dx: host, 3 doubles > 0; dt > 0; bc: 0 periodic, 1 zero gradient
 * (the node beyond a boundary takes the boundary node's value).  FP32
 * arithmetic; q_out (device, G x M) must not overlap q_in (VDS_EARG).
 * Asynchronous on the context stream. */
VDS_API int vds_convect(vds_ctx *ctx, const float *q_in, float *q_out, int nx, int ny, int nz, long M,
                        const float *u, const double *dx, double dt, int bc);

/* Tile autotuner (no counterpart in the paper).  The batched pair kernel has
 * VDS_BATCH_CONFIGS candidate shapes: config k runs 128 << (k >> 1) threads
 * per CTA with 2 << (k & 1) particles per thread, so a work item's i-tile is
 * 256, 512, 512 or 1024 particles.  The j-tiles and the order of every sum
 * are the same in all of them, so results are bit-identical across configs;
 * only the queue (its items follow the tile) and the speed change.  A batch
 * starts in config 1 for D <= 6 and config 0 otherwise.
 *
 * vds_batch_autotune times one density and one gradient pass of every
 * candidate on the batch's particles q_all (device, total x D; reps >= 1
 * timed repetitions each, the fastest kept), selects the fastest candidate,
 * rebuilds the work queue for its tile and returns its index in config
 * (host, may be NULL) and each candidate's milliseconds in ms (host,
 * VDS_BATCH_CONFIGS doubles, may be NULL).  Synchronises.
 * vds_batch_set_config selects a candidate directly; vds_batch_get_config
 * reads the current one.  Either invalidates the captured implicit round. */
#define VDS_BATCH_CONFIGS 4
VDS_API int vds_batch_autotune(vds_ctx *ctx, vds_batch *b, const float *q_all, int reps, int *config,
                               double *ms);
VDS_API int vds_batch_set_config(vds_ctx *ctx, vds_batch *b, int config);
VDS_API int vds_batch_get_config(const vds_batch *b, int *config);

#ifdef __cplusplus
}
#endif
#endif /* VDS_BATCH_H */
