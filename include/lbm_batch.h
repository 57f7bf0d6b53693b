/*
 * lbm_batch.h -- batched ensemble of independent periodic lattices advanced
 * together by liblbm.so.
 *
 * Every instance runs the same method (stencil, collision space, storage)
 * as a single-domain context (include/lbm.h, Eq. 2.1 with the collision of
 * Eq. 2.4-2.6) on its own periodic box; instances differ in their
 * dimensions and their shear relaxation rate.  One step of the whole
 * ensemble is ONE persistent kernel launch: its grid (blocks_per_sm x SM
 * count blocks) walks a list of equal-size tiles of cells, each tile inside
 * one instance, in a fixed round-robin order (no atomics, no inter-block
 * waits).  lbm_batch_step replays the launches from captured CUDA graphs.
 * The tile shape (threads per block, cells per thread) and the grid size
 * are the tuning parameters; lbm_batch_autotune picks them by timing.
 *
 * Conventions are those of include/lbm.h (return codes, ownership, field
 * layouts, velocity order, canonical pre-collision state f(n)).  Only pull
 * streaming, zero-centered storage, deviation arithmetic and the Maxwellian
 * equilibria are served (in-place patterns, LBM_STORE_F64_ABSOLUTE,
 * LBM_ARITH_AS_WRITTEN or LBM_EQ_DISCRETE2 -> LBM_ERR_UNSUPPORTED); every
 * collision space is.  Instance k stores
 * its populations as a structure of arrays at element offset off_k of one
 * device buffer per pull buffer (the library owns them).
 */
#ifndef LBM_BATCH_H
#define LBM_BATCH_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_batch lbm_batch;

typedef struct {
  int threads;          /* threads per block: 32..256, multiple of 32       */
  int cells_per_thread; /* 1..16; tile = threads * cells_per_thread cells    */
  int blocks_per_sm;    /* 1..32; persistent grid = blocks_per_sm * #SMs     */
  int per_instance;     /* 0: one persistent launch per step (default);
                           1: one single-domain launch per instance per step
                              (the unbatched comparison)                     */
} lbm_batch_tuning;

/* Create an ensemble of n >= 1 instances.  proto gives the method, storage,
 * bulk and higher-order rates and the stream (proto->dims is ignored);
 * dims[3*k..3*k+2] the box of instance k (same limits as lbm_create);
 * shear_rates[k] its shear rate in (0, 2] (NULL: proto->rates[0]).
 * Populations start at zero.  Default tuning: 128 threads, 4 cells per
 * thread, 8 blocks per SM, persistent.  Errors: INVALID, INADMISSIBLE,
 * UNSUPPORTED, OOM, CUDA. */
int lbm_batch_create(lbm_batch** out, const lbm_params* proto, int n,
                     const int64_t* dims, const double* shear_rates);

/* Install f(0) = the method's equilibrium of rho[N_k] (NULL: 1) and
 * u[D*N_k] for instance k (FP64, field layout of lbm.h).  Step counter
 * reset to 0.  Errors: INVALID, CUDA. */
int lbm_batch_init_velocity(lbm_batch* b, int k, const double* rho,
                            const double* u, int on_device);

/* Install f(0) for every instance from the Taylor-Green vortex of Eq. 5.1
 * at t = 0 (u0[k] the amplitude of instance k, host array of n doubles,
 * wavenumber 2 pi / N_axis, u_z = 0), evaluated on the device.  Errors:
 * INVALID, CUDA. */
int lbm_batch_init_tgv(lbm_batch* b, const double* u0);

/* Advance every instance n >= 0 steps (asynchronous, graph replay).
 * Errors: INVALID, CUDA. */
int lbm_batch_step(lbm_batch* b, int64_t n);

/* Read-out of instance k, as lbm_get_populations / lbm_macroscopic. */
int lbm_batch_get_populations(lbm_batch* b, int k, double* df, int on_device);
int lbm_batch_macroscopic(lbm_batch* b, int k, double* rho, double* u,
                          int on_device);

/* Total number of cells over all instances, and the instance count. */
int64_t lbm_batch_cells(const lbm_batch* b);
int lbm_batch_size(const lbm_batch* b);

/* Set / get the launch shape.  Errors: INVALID. */
int lbm_batch_set_tuning(lbm_batch* b, const lbm_batch_tuning* t);
int lbm_batch_get_tuning(const lbm_batch* b, lbm_batch_tuning* t);

/* Time every candidate shape (threads in {64, 128, 256}, cells per thread
 * in {1, 2, 4, 8}, blocks per SM in {4, 6, 8, 10, 12, 16}) over trial_steps >= 1
 * steps (rounded up to even), then time the four fastest three more times
 * each and keep the one with the best median; returns it with that median
 * cell-update rate in MLUPS.  The trial steps advance the ensemble: call it
 * before the lbm_batch_init_* calls.  Synchronises the stream.  Errors:
 * INVALID, CUDA. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_tuning* best,
                       double* best_mlups);

/* Current step counter. */
int lbm_batch_get_time(const lbm_batch* b, int64_t* step);

void lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_BATCH_H */
