/*
 * lbm_oracle.h -- plain, slow FP64 CPU oracle for the zero-centered MRT
 * lattice Boltzmann step (Hennig, Holzer, Ruede, arXiv 2211.02435).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or generator with
 * the CUDA library.  Where the two must agree on an interface (enum codes,
 * velocity order, array layout) each side writes its own copy of that
 * documented interface.
 *
 * Every function follows the paper's definitions literally, with explicit
 * dense matrices (M, M^-1, K(u), basis matrices) instead of the Chimera
 * transforms the GPU path uses:
 *   populations, zero-centering, conserved quantities   Sec. 2.1, Eq. 2.2-2.3
 *   MRT collision (general / deviation-only / absolute)  Sec. 2.2, Eq. 2.4-2.6
 *   raw moments, central moments, cumulants              Sec. 2.3, Eq. 2.7-2.11
 *   Maxwellian equilibrium and background                Sec. 2.4, Eq. 2.12
 *   second-order truncation of raw equilibrium moments   Sec. 4.2 (Table 1 setup)
 *   streaming                                            Eq. 2.1b
 *
 * Layout: populations are zero-centered deviations df_i = f_i - w_i stored
 * structure-of-arrays, df[i*N + (z*Ny + y)*Nx + x], i in the velocity order
 * below.  The state passed to lbm_oracle_step is the pre-collision f(t).
 *
 * Velocity order (shared interface, documented in include/lbm.h too):
 *   D2Q9 : 0 (0,0); 1 (1,0); 2 (-1,0); 3 (0,1); 4 (0,-1);
 *          5 (1,1); 6 (-1,-1); 7 (1,-1); 8 (-1,1)
 *   D3Q19: 0 rest; 1..6 faces (+x,-x,+y,-y,+z,-z);
 *          7..18 edges (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *                      (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *   D3Q27: D3Q19 followed by corners 19..26 (1,1,1) (-1,-1,-1) (1,1,-1)
 *          (-1,-1,1) (1,-1,1) (-1,1,-1) (1,-1,-1) (-1,1,1)
 *   Opposite pairs are adjacent: for i > 0, ibar = i + 1 if i is odd, i - 1
 *   if i is even.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* stencils */
#define LBM_ORACLE_D2Q9 0
#define LBM_ORACLE_D3Q19 1
#define LBM_ORACLE_D3Q27 2
/* collision spaces; NONE = identity collision (pure streaming) */
#define LBM_ORACLE_SPACE_POPULATIONS 0
#define LBM_ORACLE_SPACE_RAW 1
#define LBM_ORACLE_SPACE_CENTRAL 2
#define LBM_ORACLE_SPACE_CUMULANT 3
/* two-relaxation-time collision in population space: even part with
 * rates[0], odd part with rates[2] (the order-3 slot) */
#define LBM_ORACLE_SPACE_TRT 4
/* raw moments in the weighted orthogonal basis (WO-MRT): the same rows
 * Gram-Schmidt-orthogonalised under <p,q> = sum_i w_i p(xi_i) q(xi_i) */
#define LBM_ORACLE_SPACE_RAW_WEIGHTED 5
#define LBM_ORACLE_SPACE_NONE 6
/* equilibrium format: deviation-only (Eq. 2.5) or absolute (Eq. 2.6) */
#define LBM_ORACLE_EQ_DELTA 0
#define LBM_ORACLE_EQ_ABSOLUTE 1
/* the discrete second-order polynomial equilibrium given as populations,
 * f_eq_i = w_i rho (1 + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u), whose collision-
 * space quantities are q_eq = T(f_eq) (Sec. 2.4: an equilibrium may be
 * prescribed as a discrete population vector and transformed); absolute
 * collision (Eq. 2.6) */
#define LBM_ORACLE_EQ_DISCRETE2 2
/* rate groups (row groups of the polynomial bases) */
#define LBM_ORACLE_GROUP_CONSERVED -1
#define LBM_ORACLE_GROUP_SHEAR 0
#define LBM_ORACLE_GROUP_BULK 1
#define LBM_ORACLE_GROUP_ORDER3 2 /* order k -> group k - 1 */

typedef struct {
  int stencil;     /* LBM_ORACLE_D2Q9 / D3Q19 / D3Q27 */
  int space;       /* LBM_ORACLE_SPACE_* */
  int equilibrium; /* LBM_ORACLE_EQ_* */
  double rates[6]; /* shear, bulk, order 3, order 4, order 5, order 6 */
} lbm_oracle_method;

/* Error codes: 0 ok, -1 invalid argument, -3 inadmissible combination. */

/* Lattice description: q, d, velocities xi[q][3], weights w[q] computed as
 * M^-1 m0 (Sec. 2.4), monomial exponents expo[q][3] ordered by degree. */
int lbm_oracle_lattice(int stencil, int* q, int* d, int* xi, double* w,
                       int* expo);

/* Dense matrices, row-major q x q: monomial raw-moment matrix M (Eq. 2.8),
 * its inverse, the orthogonal raw basis Praw (rows = polynomials in monomial
 * coordinates, unweighted Gram-Schmidt), the homogeneous basis Pcm used for
 * central moments and cumulants, and the rate group of each basis row. */
int lbm_oracle_matrices(int stencil, double* M, double* Minv, double* Praw,
                        double* Pcm, int* group);

/* Weighted orthogonal raw basis (WO-MRT), row-major q x q, rows in the
 * order and groups of the unweighted basis. */
int lbm_oracle_weighted_basis(int stencil, double* Pw);
/* Central-moment matrix K(u)[k][i] = prod_d (xi_{i,d} - u_d)^{e_{k,d}}
 * (Sec. 2.3.2), row-major q x q. */
int lbm_oracle_central_matrix(int stencil, const double* u, double* K);

/* Cumulants of one absolute population vector f (Eq. 2.11, via the
 * set-partition form of log M).  out[k] for monomial k: order 0 -> rho,
 * order 1 -> u_d, order >= 2 -> rescaled cumulant C = rho * c. */
int lbm_oracle_cumulants(int stencil, const double* f, double* out);

/* Inverse: monomial raw moments m from (rho, u, C) in the layout above. */
int lbm_oracle_moments_from_cumulants(int stencil, const double* c_in,
                                      double* m);

/* Joint cumulant of a multiset given normalized raw moments mu[a][b][c]
 * (a,b,c in 0..2, mu[0][0][0] = 1), exponents (a,b,c). */
double lbm_oracle_cumulant_of(const double* mu27, int a, int b, int c);

/* One collision of ncells independent cells.  df_in/df_out are cell-major
 * [ncells][q] zero-centered deviations (may alias). */
int lbm_oracle_collide(const lbm_oracle_method* m, int64_t ncells,
                       const double* df_in, double* df_out);

/* The method's equilibrium, as deviations from w, for given rho and u
 * (cell-major: rho[ncells], u[ncells][3], df_out[ncells][q]). */
int lbm_oracle_equilibrium(const lbm_oracle_method* m, int64_t ncells,
                           const double* rho, const double* u, double* df_out);

/* Fill an SoA state df[q][N] with the equilibrium of rho[N], u[3][N]
 * (u SoA: u[d*N + cell]). */
int lbm_oracle_init(const lbm_oracle_method* m, const int64_t* dims,
                    const double* rho, const double* u, double* df);

/* nsteps of collide (Eq. 2.1a) then stream (Eq. 2.1b) with periodic wrap,
 * in place on the SoA pre-collision state df[q][N]. */
int lbm_oracle_step(const lbm_oracle_method* m, const int64_t* dims,
                    double* df, int64_t nsteps, int nthreads);

/* Density and velocity (Eq. 2.3) of the SoA state: rho[N], u[3][N]. */
int lbm_oracle_macroscopic(const lbm_oracle_method* m, const int64_t* dims,
                           const double* df, double* rho, double* u);

/* Body force (source term f^F of Eq. 2.1a, q^F of Eq. 2.4).  The paper
 * names Guo's and He's models without writing them out; this oracle follows
 * Guo: equilibrium velocity u = (j + F/2) / rho and the population source
 * S_i = w_i [(xi_i - u).F / c_s^2 + (xi_i.u)(xi_i.F) / c_s^4], entering as
 *   SRT:        f* = f + w (f_eq - f) + (1 - w/2) S
 *   raw MRT:    q^F = (I - S/2) P M S   (conserved rows: factor 1)
 *   central:    moments about u, q^F = F on the first-order rows only
 *               (kappa_1 = -F/2 before and +F/2 after the collision)
 *   cumulant:   cumulants of order >= 2 relax as without force; the
 *               first-order cumulant (mean velocity) leaves as (j + F)/rho.
 * model 0 is Guo's model above; model 1 is He's: the same velocity shift and
 * (I - S/2) weighting with the source S_i = (xi_i - u).F / (rho c_s^2)
 * f_eq_i (the method's absolute equilibrium populations), entering central
 * space as q^F = (I - S/2) P K(u) S; not defined for cumulants (-1).
 * collide: force[ncells][3] cell-major (z ignored for D2Q9).  step /
 * macroscopic: force SoA [D][N] (D = 2 for D2Q9, else 3), constant in time,
 * NULL = none; macroscopic then returns the fluid velocity (j + F/2)/rho. */
int lbm_oracle_collide_forced(const lbm_oracle_method* m, int64_t ncells,
                              const double* df_in, const double* force,
                              int model, double* df_out);
int lbm_oracle_step_forced(const lbm_oracle_method* m, const int64_t* dims,
                           double* df, const double* force, int model,
                           int64_t nsteps, int nthreads);
int lbm_oracle_macroscopic_forced(const lbm_oracle_method* m,
                                  const int64_t* dims, const double* df,
                                  const double* force, double* rho, double* u);

/* Shallow-water methods (Sec. 5.2), D2Q9 only, depth h = sum f and
 * h u = sum xi f, gravity g in lattice units, absolute equilibrium:
 *   space CENTRAL  (de Rosis): central moments relax towards those of
 *                  Zhou's discrete equilibrium
 *                  f0 = h (1 - 5gh/6 - 2u.u/3),
 *                  f_i = l_i h (gh/6 + xi.u/3 + (xi.u)^2/2 - u.u/6),
 *                  l_i = 1 (axes), 1/4 (diagonals);
 *   space CUMULANT (Venturi): the cumulant collision with the continuous
 *                  Maxwellian of c_s^2 = g h / 2 (second-order equilibrium
 *                  cumulants h * g h / 2, higher ones 0).
 * Populations in and out are still df = f - w (w the D2Q9 weights), so
 * lbm_oracle_macroscopic returns (h, u).  swe_equilibrium: absolute f[9]
 * of the method's equilibrium at (h, u[2]). */
int lbm_oracle_swe_equilibrium(int space, double g, double h, const double* u,
                               double* f);
int lbm_oracle_swe_collide(const lbm_oracle_method* m, double g, int64_t ncells,
                           const double* df_in, double* df_out);
int lbm_oracle_swe_init(const lbm_oracle_method* m, double g,
                        const int64_t* dims, const double* h, const double* u,
                        double* df);
int lbm_oracle_swe_step(const lbm_oracle_method* m, double g,
                        const int64_t* dims, double* df, int64_t nsteps,
                        int nthreads);

/* ------------------------------------------------------------------ */
/* Learned closure (not in the paper): a per-cell MLP 7 -> 32 -> 32 -> 4 */
/* sets the relaxation rates of orders 3..6 of the cumulant collision.    */
/* ------------------------------------------------------------------ */
#define LBM_ORACLE_CLOSURE_NIN 7
#define LBM_ORACLE_CLOSURE_NH 32
#define LBM_ORACLE_CLOSURE_NOUT 4
#define LBM_ORACLE_CLOSURE_NPARAM 1444 /* W1[32][7] b1 W2[32][32] b2 W3[4][32] b3 */

/* Raw features of one cell from its zero-centered populations df[q]:
 * with Pi = kappa_2 / rho - I/3 (second-order central moments, Sec. 2.3.2),
 * S = -(3 omega_shear / 2) Pi and D = Pi - tr(Pi)/3 I:
 * out = {tr S, I2(S)/|S|, det S/|S|^2, I2(D)/|D|, det D/|D|^2, |Pi|, rho - 1},
 * where I2(A) = ((tr A)^2 - tr(A A)) / 2, |.| is the Frobenius norm and a
 * quotient is 0 where its norm is 0: the principal invariants, each divided
 * by a power of its tensor's norm so that all but the last are of degree 1
 * in Pi.  3-D stencils only. */
int lbm_oracle_closure_features(int stencil, const double* df,
                                double omega_shear, double out[7]);

/* omega[4] (orders 3..6) = clamp(2 sigmoid(W3 tanh(W2 tanh(W1 x + b1) + b2)
 * + b3), 1e-3, 1.999) with x_i = (raw_i - shift_i) * scale_i; all four are 1
 * if any x_i is not finite or |x_i| > 65504 (the FP16 range of the GPU
 * network's operands), or any output is not finite. */
int lbm_oracle_closure_mlp(const double* params, const double* shift,
                           const double* scale, const double raw[7],
                           double omega[4]);

/* One step (collide with per-cell rates of orders 3..6 from the MLP, then
 * stream) of the SoA pre-collision state df[q][N], in place.  base gives
 * the stencil, space and the shear / bulk rates. */
int lbm_oracle_closure_step(const lbm_oracle_method* base,
                            const int64_t* dims, double* df,
                            const double* params, const double* shift,
                            const double* scale, int nthreads);

/* One-step loss: mean over cells of |u(step(df_s)) - u(df_t)|^2 (Eq. 2.3
 * velocities).  Returns NaN on error. */
double lbm_oracle_closure_loss(const lbm_oracle_method* base,
                               const int64_t* dims, const double* df_s,
                               const double* df_t, const double* params,
                               const double* shift, const double* scale,
                               int nthreads);

/* K-step rollout loss: starting from df[0] (K + 1 SoA states df[k][q][N]
 * laid out one after the other, df[k] the target after k steps), run K
 * learned-rate steps and return (1/K) sum_k mean over cells of
 * |u(step^k(df[0])) - u(df[k])|^2.  K = 1 is lbm_oracle_closure_loss.
 * Returns NaN on error. */
double lbm_oracle_closure_rollout_loss(const lbm_oracle_method* base,
                                       const int64_t* dims, const double* df,
                                       int K, const double* params,
                                       const double* shift, const double* scale,
                                       int nthreads);

#ifdef __cplusplus
}
#endif
#endif
