/*
 * lbm.h -- C ABI of the B300 (sm_103a) zero-centered MRT lattice Boltzmann
 * library (liblbm.so).  Method: Hennig, Holzer, Ruede, "Advanced Automatic
 * Code Generation for Multiple Relaxation-Time Lattice Boltzmann Methods"
 * (arXiv 2211.02435).
 *
 * One call of lbm_step advances every cell by the fused stream + collide
 * update of Eq. 2.1: gather the populations (Eq. 2.1b: pull, or the in-place
 * AA, Esoteric Twist, Esoteric Pull or Esoteric Push patterns, Sec. 4.3),
 * collide (Eq. 2.4-2.6) in population (SRT, TRT), raw-moment (O-MRT,
 * WO-MRT), central-moment or cumulant space (Sec. 2.3) using the raw-moment
 * Chimera (Eq. 4.1), the binomial raw<->central Chimera (Eq. 4.3-4.4), the
 * central<->cumulant relations (Eq. 4.5) and the split backward transform
 * (Eq. 4.2), with an optional body force (Eq. 2.1a source term, Guo or He),
 * and store.
 * Populations are stored zero-centered, df_i = f_i - w_i (Sec. 2.1), or
 * absolute for the round-off studies and the shallow-water methods.
 *
 * Conventions shared by every call
 *  - Return value: LBM_OK (0) or a negative LBM_ERR_* code.  No C++
 *    exception crosses the ABI.  lbm_error_string() names a code.
 *  - Ownership: the library owns the device state it allocates in
 *    lbm_create and the staging buffers it keeps for host transfers (all
 *    freed by lbm_destroy).  The caller owns every buffer it passes in; the
 *    library keeps no pointer to it after the call returns.
 *  - on_device = 1: the pointer is device memory of the context's GPU (e.g.
 *    torch tensor.data_ptr()); 0: host memory.  Host-pointer calls copy
 *    (large arrays in slabs, on copy streams the context owns, ordered
 *    after the work already queued on its stream) and synchronise before
 *    returning.
 *  - All device work is enqueued on params.stream (a cudaStream_t; NULL =
 *    legacy default stream).  lbm_step returns without synchronising
 *    (unless its divergence watch is on).
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns LBM_ERR_CUDA.
 *  - Populations read or written through this interface are always the
 *    zero-centered df = f - w, also for LBM_STORE_F64_ABSOLUTE.
 *  - Field layout (inputs and outputs): structure of arrays with x fastest,
 *    cell index c = (z*Ny + y)*Nx + x.  Scalars: a[c]; vectors: a[d*N + c]
 *    with d = 0..D-1 (D = 2 for D2Q9, 3 otherwise); populations: a[i*N + c].
 *  - Velocity order i (opposite pairs adjacent):
 *      D2Q9 : 0 (0,0); 1 (1,0); 2 (-1,0); 3 (0,1); 4 (0,-1);
 *             5 (1,1); 6 (-1,-1); 7 (1,-1); 8 (-1,1)
 *      D3Q19: 0 rest; 1..6 (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1);
 *             7..18 (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *                   (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *      D3Q27: the D3Q19 order followed by 19..26 (1,1,1) (-1,-1,-1) (1,1,-1)
 *             (-1,-1,1) (1,-1,1) (-1,1,-1) (1,-1,-1) (-1,1,1)
 *  - Time: after n steps the canonical state is the pre-collision
 *    (post-streaming) f(n) of Eq. 2.1, f(0) being what lbm_init_velocity or
 *    lbm_set_populations installed.  Every read-out call returns f(n) or
 *    quantities of f(n), whatever the streaming pattern and its parity.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LBM_OK 0
#define LBM_ERR_INVALID -1        /* bad argument, size or NULL pointer      */
#define LBM_ERR_UNSUPPORTED -2    /* valid request this build does not serve */
#define LBM_ERR_INADMISSIBLE -3   /* combination the method forbids (Sec. 3) */
#define LBM_ERR_OOM -4            /* device allocation failed                */
#define LBM_ERR_CUDA -5           /* CUDA runtime error / no device          */
#define LBM_ERR_DIVERGED -6       /* non-finite populations detected         */
#define LBM_ERR_STATE_MISMATCH -7 /* checkpoint does not fit this context    */
#define LBM_ERR_TIMEOUT -8        /* a kernel's bounded wait ran out         */

/* ---- method specification (Sec. 3, Fig. 2) ---- */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 } lbm_stencil;

/* Collision space (Sec. 2.3).  POPULATIONS is single relaxation time (BGK)
 * in population space, f* = f + omega (f_eq - f) with omega = rates[0] and
 * f_eq = M^-1 m_eq (the raw-moment equilibrium below). */
typedef enum {
  LBM_SPACE_POPULATIONS = 0,
  LBM_SPACE_RAW = 1,      /* orthogonal raw moments, unweighted (O-MRT)  */
  LBM_SPACE_CENTRAL = 2,  /* polynomial central moments (CM)             */
  LBM_SPACE_CUMULANT = 3, /* polynomial cumulants (K)                    */
  LBM_SPACE_TRT = 4,      /* two relaxation times in population space:
                             per opposite pair the even part
                             (f_i + f_ibar)/2 relaxes with rates[0], the
                             odd part with rates[2]; the same method as
                             LBM_SPACE_RAW with even orders at rates[0] and
                             odd orders at rates[2].  Deviation arithmetic
                             only (not with LBM_STORE_F64_ABSOLUTE or
                             LBM_ARITH_AS_WRITTEN: UNSUPPORTED) */
  LBM_SPACE_RAW_WEIGHTED = 5 /* raw moments in the weighted orthogonal
                                basis (WO-MRT, Sec. 4.2): the same rows
                                orthogonalised under sum_i w_i p(xi_i)
                                q(xi_i); equal to LBM_SPACE_RAW when every
                                rate is 1 */
} lbm_space;

/* Equilibrium format (Sec. 2.2): relax deviations against the
 * delta-equilibrium (Eq. 2.5) or the absolute equilibrium (Eq. 2.6).
 * Cumulant space admits only LBM_EQ_ABSOLUTE (Sec. 2.4): the other is
 * rejected with LBM_ERR_INADMISSIBLE.  Raw-moment methods use the
 * continuous Maxwellian truncated at second order in u (Sec. 4.2);
 * central-moment and cumulant methods the untruncated Maxwellian.
 *
 * LBM_EQ_DISCRETE2: the equilibrium prescribed as a discrete population
 * vector (Sec. 2.4), the second-order polynomial
 *   f_eq_i = w_i rho (1 + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u),
 * transformed into the collision space, q_eq = T(f_eq), in every space
 * (SRT and TRT relax against f_eq itself).  Its raw moments equal the
 * truncated Maxwellian's on D2Q9 and D3Q27 and differ on D3Q19 in the
 * x^2 y^2-type moments (by -rho u_k^2 / 6), so raw-moment MRT with equal
 * rates is the textbook BGK there; its central moments and cumulants of
 * order >= 3 are nonzero (central and cumulant methods run their general
 * instance).  lbm_init_velocity sets f_eq.  Served for LBM_STORE_F64 /
 * LBM_STORE_F32, pull streaming and LBM_ARITH_DEVIATION, without a body
 * force or a closure; otherwise LBM_ERR_UNSUPPORTED. */
typedef enum {
  LBM_EQ_DELTA = 0,
  LBM_EQ_ABSOLUTE = 1,
  LBM_EQ_DISCRETE2 = 2
} lbm_equilibrium;

/* Population storage.  F64 computes in FP64, the others in FP32.  The
 * *_DELTA forms store h_i = round_rn(df_i * 2^s_i) in FP16 / BF16 with the
 * per-direction scale exponent s_i = round(-log2 w_i):
 *   D2Q9 1,3,5; D3Q19 2,4,5; D3Q27 2,4,6,8 (rest, |xi|^2 = 1, 2, 3). */
typedef enum {
  LBM_STORE_F64 = 0,
  LBM_STORE_F32 = 1,
  LBM_STORE_F16_DELTA = 2,
  LBM_STORE_BF16_DELTA = 3,
  LBM_STORE_F64_ABSOLUTE = 4 /* absolute populations f, not df (Sec. 2.1):
                                collides with Eq. 2.4 in absolute FP64
                                arithmetic; needs LBM_EQ_ABSOLUTE (Sec. 3);
                                pull streaming only */
} lbm_storage;

/* Collision arithmetic.  DEVIATION (default): every moment, central moment
 * and cumulant is carried as a deviation from the rest state, whichever
 * equilibrium format is chosen (algebraically Eq. 2.5 / 2.6).  AS_WRITTEN:
 * the arithmetic the paper writes, for round-off studies (Sec. 5.1):
 * LBM_EQ_DELTA relaxes deviations against the delta-equilibrium (Eq. 2.5),
 * LBM_EQ_ABSOLUTE evaluates Eq. 2.6: q = T(df + f0) is formed as the
 * nonlinear part of T (shift to central moments, cumulants) applied to the
 * raw moments M df plus the constant background moments M f0, the collision
 * runs on these absolute quantities, and T^-1(q*) - f0 is formed as M^-1 of
 * the post-collision raw moments minus M f0 (M is linear).  Population-space
 * SRT (T = identity) adds f0 = w to df and subtracts it again.  AS_WRITTEN
 * is served for FP64 storage with pull streaming. */
typedef enum { LBM_ARITH_DEVIATION = 0, LBM_ARITH_AS_WRITTEN = 1 } lbm_arithmetic;

/* Streaming pattern (Sec. 4.3): pull with two buffers, or one of the
 * in-place patterns with one buffer: AA (even steps local, odd steps across
 * all neighbours) or one of the esoteric patterns, in which every opposite
 * pair (p, pbar), p the member whose first nonzero component is +1 (odd
 * index), occupies the two elements (x + a_p, slot p) and
 * (x + a_p + xi_p, slot pbar) of cell x at even times and the same elements
 * with the slots swapped at odd times:
 *   Esoteric Twist: a_p = max(-xi_p, 0) per component (the cell and its
 *                   positive neighbours);
 *   Esoteric Pull:  a_p = 0 (p at the own node, pbar at x - xi_pbar);
 *   Esoteric Push:  a_p = -xi_p (pbar at the own node, p at x - xi_p).
 * Each step a cell reads and overwrites exactly its own elements.  All
 * patterns give identical states f(n); lbm_get_time reports the in-place
 * parity. */
typedef enum {
  LBM_PULL = 0,
  LBM_AA = 1,
  LBM_ESOTERIC_TWIST = 2,
  LBM_ESOTERIC_PULL = 3,
  LBM_ESOTERIC_PUSH = 4
} lbm_streaming;

#define LBM_PERIODIC 0 /* the only boundary; others -> LBM_ERR_UNSUPPORTED */

/* Relaxation-rate slots (Sec. 2.2 matrix S, grouped): the rate of the
 * traceless second-order quantities (shear), of the second-order trace
 * (bulk), and of all quantities of order 3, 4, 5 and 6.  Conserved
 * quantities are not relaxed.  Shear rate from viscosity:
 * nu = (1/omega - 1/2) / 3. */
enum {
  LBM_RATE_SHEAR = 0,
  LBM_RATE_BULK = 1,
  LBM_RATE_ORDER3 = 2,
  LBM_RATE_ORDER4 = 3,
  LBM_RATE_ORDER5 = 4,
  LBM_RATE_ORDER6 = 5
};

typedef struct {
  int stencil;      /* lbm_stencil                                       */
  int space;        /* lbm_space                                         */
  int equilibrium;  /* lbm_equilibrium                                   */
  int storage;      /* lbm_storage                                       */
  int streaming;    /* lbm_streaming                                     */
  double rates[6];  /* see LBM_RATE_*; each in (0, 2]                     */
  int64_t dims[3];  /* Nx, Ny, Nz (Nz = 1 for D2Q9); each >= 1, Ny, Nz <=
                       65535, Nx*Ny*Nz + Nx*Ny + 2*Nx + 4096 < 2^31 on
                       D3Q19 / D3Q27 and Nx*Ny + 2*Nx + 4096 < 2^31 on
                       D2Q9 (the kernels' 32-bit cell indices with their
                       periodic wrap corrections); else LBM_ERR_INVALID  */
  int boundary;     /* LBM_PERIODIC                                      */
  void* stream;     /* cudaStream_t for every enqueue; NULL = default     */
  int arithmetic;   /* lbm_arithmetic (0 = deviations throughout)         */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Create a context and allocate its device state (pull: 2 buffers, AA: 1,
 * each q*N elements of the storage type).  Populations start at zero
 * (rest state rho = 1, u = 0).  Errors: INVALID (NULL, bad enum, dims or
 * rates), INADMISSIBLE (cumulant + delta equilibrium), UNSUPPORTED
 * (boundary), OOM, CUDA. */
int lbm_create(lbm_ctx** out, const lbm_params* params);

/* Install f(0) = the method's equilibrium (the collision's fixed point)
 * for density rho[N] (NULL: rho = 1) and velocity u[D*N], FP64, field
 * layout above.  Resets the step counter to 0.  Errors: INVALID, CUDA. */
int lbm_init_velocity(lbm_ctx* ctx, const double* rho, const double* u,
                      int on_device);

/* Advance n >= 0 steps on the context's stream (asynchronous unless the
 * divergence watch of lbm_set_divergence_check is on).
 * Errors: INVALID, CUDA, DIVERGED (watch on). */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Density rho[N] and velocity u[D*N] of f(n), Eq. 2.3, written as FP64.
 * Either pointer may be NULL.  Errors: INVALID, CUDA. */
int lbm_macroscopic(lbm_ctx* ctx, double* rho, double* u, int on_device);

/* One job from host memory to host memory: f(0) from rho[N] (NULL: 1) and
 * u[D*N] as lbm_init_velocity, n >= 0 steps as lbm_step, then rho_out[N]
 * and u_out[D*N] of f(n) as lbm_macroscopic (either may be NULL), all host
 * FP64 arrays in the field layout above; synchronises.  The result equals
 * that sequence bit for bit.  With pull streaming, zero-centered storage,
 * deviation arithmetic, no body force or closure, the direct step kernel
 * and Nz >= 3, the job runs pipelined: the lattice is cut into `slabs` runs
 * of z-planes (0: about 64 MB of rho and u each, at least 3; capped at Nz)
 * and the host-to-device copies, the steps (Eq. 2.1, a slab taking step
 * k + 1 once both neighbouring slabs have taken step k) and the
 * device-to-host copies of different slabs overlap, on two copy streams
 * the library creates for the call and the context's stream.  The device
 * staging (one slot per slab and direction, 2 x 8 (1 + D) N bytes, or a
 * ring of 4 slots per direction when the device lacks the room) is kept
 * by the context for the next call and freed by lbm_destroy.  Otherwise
 * (or with fewer than 3 slabs, or with the divergence watch of
 * lbm_set_divergence_check on) the three calls run one after the other.
 * Errors: INVALID, OOM, CUDA. */
int lbm_run_host(lbm_ctx* ctx, const double* rho, const double* u, int64_t n,
                 double* rho_out, double* u_out, int slabs);

/* Read / write the canonical zero-centered populations df[q*N] of f(n)
 * in FP64 (writing encodes them into the storage type and resets the AA
 * parity; the step counter is kept).  Errors: INVALID, CUDA. */
int lbm_get_populations(lbm_ctx* ctx, double* df, int on_device);
int lbm_set_populations(lbm_ctx* ctx, const double* df, int on_device);

/* Global FP64 reductions over f(n), deterministic (fixed-order two-pass):
 * out[0] sum(rho - 1), out[1..3] sum(rho u_d), out[4] sum(rho |u|^2 / 2),
 * out[5] max |u|, out[6] number of cells with a non-finite population,
 * out[7] number of cells.  Synchronises the stream.  Uses a per-context
 * device scratch buffer allocated at create time.  Errors: INVALID, CUDA,
 * DIVERGED (out is still filled when out[6] > 0). */
int lbm_invariants(lbm_ctx* ctx, double out[8]);

/* Allocation-free variant of lbm_invariants for callers that must not
 * allocate device memory (a host framework that owns the whole device pool,
 * a real-time loop where an allocation could stall or fail, or a caller that
 * only hands this library existing buffers).  The paper has no counterpart;
 * this is a convenience of the library.
 *
 * df: device pointer to the caller's zero-centered populations in the
 * storage type `storage`, structure of arrays df[i*N + c] with slot i of
 * cell c holding f_i of that cell (the canonical f(n), as an AA context holds
 * it at even parity).  dims: Nx, Ny, Nz (Nz = 1 for D2Q9), at most
 * LBM_STATIC_MAX_CELLS cells in all; larger or non-positive sizes are
 * rejected with LBM_ERR_INVALID.  out: 8 doubles as lbm_invariants; a device
 * pointer when on_device = 1 (the call then returns without synchronising
 * and cannot report DIVERGED), else host memory (the call synchronises
 * `stream` and returns LBM_ERR_DIVERGED when out[6] > 0).  stream: a
 * cudaStream_t, NULL = legacy default stream.
 *
 * The partial sums live in one static device array of
 * LBM_STATIC_SCRATCH_ROWS * 8 + 8 doubles (75,840 bytes) that every GPU
 * which loads liblbm.so keeps until the process exits; no cudaMalloc,
 * cudaFree or other allocating routine is called.  The first call on a
 * device looks up that array's device address (with the device current),
 * so make the first call before any stream capture.  All calls on a device
 * share the array: calls whose work overlaps on the GPU (other streams, or
 * other host threads) race and must be serialised by the caller.  Each call
 * overwrites every partial row it reads, so no state carries over.
 * Errors: INVALID, CUDA, DIVERGED. */
#define LBM_STATIC_SCRATCH_ROWS 1184
#define LBM_STATIC_MAX_CELLS 2147483647LL
int lbm_invariants_noalloc(int stencil, int storage, const void* df,
                           const int64_t dims[3], double out[8], int on_device,
                           void* stream);

/* Checkpoint: the raw device buffer plus a header (method, dims, storage,
 * parity, step counter).  lbm_state_bytes gives the size; get/set copy
 * through host memory.  A state from a context with other parameters is
 * refused with STATE_MISMATCH. */
int64_t lbm_state_bytes(const lbm_ctx* ctx);
int lbm_get_state(lbm_ctx* ctx, void* buf, size_t bytes);
int lbm_set_state(lbm_ctx* ctx, const void* buf, size_t bytes);

/* Current step counter and AA parity (0 even, 1 odd). */
int lbm_get_time(const lbm_ctx* ctx, int64_t* step, int* parity);

/* Change the relaxation rates (Sec. 3: rates may stay symbolic until run
 * time).  Errors: INVALID. */
int lbm_set_rates(lbm_ctx* ctx, const double rates[6]);

/* Change the stream later work is enqueued on. */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Body force: the source term f^F of Eq. 2.1a / q^F of Eq. 2.4.  The paper
 * names Guo's and He's models without writing them out; this library
 * implements Guo's: the equilibrium velocity is u = (j + F/2) / rho and,
 * with S_i = w_i [(xi_i - u).F / c_s^2 + (xi_i.u)(xi_i.F) / c_s^4],
 *   POPULATIONS (SRT): f* = f + w (f_eq - f) + (1 - w/2) S
 *   RAW:      q^F = (I - S/2) P M S in the orthogonal basis
 *   CENTRAL:  central moments about u; the first-order central moments
 *             leave the collision as +F/2 (they enter as -F/2, Sec. 4.2)
 *   CUMULANT: cumulants of order >= 2 (shift invariant) relax as without
 *             force; the mean velocity leaves as (j + F) / rho.
 * The total force on a cell is the uniform part plus the field's entry.
 *   lbm_set_force: uniform F[D] (D = 2 for D2Q9, else 3); NULL = none.
 *   lbm_set_force_field: per-cell F[d*N + c], d < D, FP64, host memory or
 *     (on_device = 1) device memory; copied (FP32 storage: rounded to FP32)
 *     into a device array the context owns; NULL removes it.
 * Under a force, lbm_macroscopic returns the fluid velocity (j + F/2) / rho;
 * lbm_invariants keeps reporting sums of rho - 1 and j = sum xi_i f_i.
 * Served for LBM_STORE_F64 / LBM_STORE_F32 with deviation arithmetic, pull
 * or AA, without a learned closure (then LBM_STEP_DIRECT runs); otherwise
 * LBM_ERR_UNSUPPORTED.  Errors: INVALID (non-finite F), UNSUPPORTED, OOM,
 * CUDA. */
int lbm_set_force(lbm_ctx* ctx, const double* F);
int lbm_set_force_field(lbm_ctx* ctx, const double* F, int on_device);

/* Force model of the source term: LBM_FORCE_GUO (default, above) or
 * LBM_FORCE_HE: He's model with the same velocity shift and (I - S/2)
 * weighting but the source S_i = (xi_i - u).F / (rho c_s^2) f_eq_i, f_eq_i
 * the method's absolute equilibrium populations (truncated raw moments for
 * POPULATIONS, TRT, RAW, RAW_WEIGHTED; the full Maxwellian for CENTRAL, where
 * q^F = (I - S/2) P K(u) S).  He's model is not defined for cumulants:
 * LBM_ERR_UNSUPPORTED.  Errors: INVALID, UNSUPPORTED. */
#define LBM_FORCE_GUO 0
#define LBM_FORCE_HE 1
int lbm_set_force_model(lbm_ctx* ctx, int model);

/* Shallow-water methods (Sec. 5.2), g > 0 the gravity in lattice units
 * (g = 0 returns to the context's own method).  The context must be D2Q9,
 * LBM_STORE_F64_ABSOLUTE, LBM_EQ_ABSOLUTE, pull, space CENTRAL or CUMULANT,
 * without a body force; otherwise LBM_ERR_UNSUPPORTED.  The conserved density
 * becomes the water depth h = sum f and the velocity u = sum xi f / h;
 *   CENTRAL  (de Rosis): central moments relax towards those of Zhou's
 *            discrete equilibrium f0 = h (1 - 5gh/6 - 2u.u/3),
 *            f_i = l_i h (gh/6 + xi.u/3 + (xi.u)^2/2 - u.u/6),
 *            l_i = 1 on the axes, 1/4 on the diagonals;
 *   CUMULANT (Venturi): the cumulant collision whose second-order
 *            equilibrium cumulants are h * g h / 2 (the continuous Maxwellian
 *            with c_s^2 = g h / 2), higher ones 0.
 * rates[0] relaxes xy and x^2 - y^2, rates[1] x^2 + y^2, rates[2..3] orders
 * 3 and 4.  lbm_init_velocity(rho = h, u) installs the method's equilibrium;
 * lbm_macroscopic returns (h, u); populations read or written are still
 * f - w.  Errors: INVALID, UNSUPPORTED. */
int lbm_set_shallow_water(lbm_ctx* ctx, double g);

/* Pull step kernel.  Both compute the same per-cell arithmetic (FP16/BF16
 * storage: bitwise-identical states; FP32/FP64: equal up to the compiler's
 * choice of multiply-add contractions); they differ in how the gather of
 * Eq. 2.1b reaches the cell:
 *   LBM_STEP_DIRECT: each thread loads its cells' q populations from
 *     global memory (one grid of 128-thread CTAs over all cells).
 *   LBM_STEP_STAGED: a persistent CTA copies, per x-row of cells, the q
 *     source rows into shared memory with bulk asynchronous copies (two
 *     rows in flight) and collides from there.  Measured slower than
 *     LBM_STEP_DIRECT on B300, so AUTO does not choose it.  Needs pull streaming,
 *     deviation arithmetic, Nx * element size a multiple of 16 bytes and
 *     2 * q * Nx * element size <= 110 KiB (FP16/BF16: Nx <= 1024 for D3Q27;
 *     FP32: Nx <= 512); otherwise LBM_ERR_UNSUPPORTED.
 *   LBM_STEP_AUTO (default): the faster of the two for the context.
 * The paper has no counterpart (its kernels are generated per platform).
 * A staged kernel whose bounded wait ran out makes the next synchronising
 * call (lbm_macroscopic / lbm_get_populations into host memory,
 * lbm_invariants, lbm_get_state) return LBM_ERR_TIMEOUT (once: the report
 * clears the condition; see lbm_set_wait_limit).
 * Errors: INVALID, UNSUPPORTED. */
#define LBM_STEP_AUTO 0
#define LBM_STEP_DIRECT 1
#define LBM_STEP_STAGED 2
int lbm_set_step_kernel(lbm_ctx* ctx, int kernel);

/* Bound of every device wait of the context's kernels (the staged kernel's
 * waits for its rows' bulk copies): `cycles` SM clock cycles, default
 * LBM_WAIT_LIMIT_DEFAULT (2^31, about 1 s at 2 GHz); 0 gives up at the first
 * unsuccessful test.  A wait that runs out abandons the rest of that step
 * (the state is then undefined until lbm_set_populations / lbm_init_velocity
 * / lbm_set_state), lets the copies already issued land (waiting with the
 * default bound) and makes the next synchronising call return
 * LBM_ERR_TIMEOUT once; the context stays usable.  The paper has no
 * counterpart (failure detection of this library).  Errors: INVALID. */
#define LBM_WAIT_LIMIT_DEFAULT 2147483648LL
int lbm_set_wait_limit(lbm_ctx* ctx, int64_t cycles);

/* Divergence watch of lbm_step: every `every` >= 1 steps (counted by the
 * context's step counter) the step call runs the FP64 invariants of f(n)
 * (as lbm_invariants, which synchronises the stream) and returns
 * LBM_ERR_DIVERGED, with the step counter at that step, as soon as a cell
 * holds a non-finite population; 0 turns the watch off (default).
 * Errors: INVALID. */
int lbm_set_divergence_check(lbm_ctx* ctx, int64_t every);

/* Free the context and its device memory.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

const char* lbm_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
