/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * lbm_oracle.h).  Slow on purpose: dense matrices, a generic set-partition
 * cumulant formula and per-cell Gauss-Jordan inverses, so that each step can
 * be checked against the paper by eye.  Shares nothing with the CUDA path.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 27
#define MAXPART 203 /* Bell(6): set partitions of the largest monomial */

typedef struct {
  int nblocks;
  unsigned char e[6][3]; /* exponent of each block */
} partition_t;

typedef struct {
  int ready;
  int q, d;
  int xi[QMAX][3];
  int opp[QMAX]; /* index of -xi_i */
  int expo[QMAX][3];
  int deg[QMAX];
  int mono[3][3][3]; /* exponent -> monomial index, -1 if not in the set */
  double w[QMAX];
  double M[QMAX][QMAX], Minv[QMAX][QMAX];
  double Praw[QMAX][QMAX], Prawinv[QMAX][QMAX];
  double Pw[QMAX][QMAX], Pwinv[QMAX][QMAX]; /* weighted orthogonal (WO-MRT) */
  double Pcm[QMAX][QMAX], Pcminv[QMAX][QMAX];
  int group[QMAX];
  int npart[QMAX];
  partition_t part[QMAX][MAXPART];
} lattice_t;

static lattice_t g_lat[3];

/* ------------------------------------------------------------------ */
/* velocity sets (Sec. 2.1), documented order                          */
/* ------------------------------------------------------------------ */
static const int V2[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0}, {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const int V3[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},
    {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
    {1, -1, -1}, {-1, 1, 1}};

static double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

/* Moments of the 1-D normal distribution with variance c_s^2 = 1/3
 * (the rest-state Maxwellian, Eq. 2.12): E[X^n]. */
static double gauss_moment(int n) {
  if (n % 2) return 0.0;
  double r = 1.0;
  for (int k = n - 1; k > 0; k -= 2) r *= (double)k; /* (n-1)!! */
  return r * ipow(1.0 / 3.0, n / 2);
}

static double binom(int n, int k) {
  double r = 1.0;
  for (int j = 1; j <= k; ++j) r = r * (double)(n - k + j) / (double)j;
  return r;
}

/* Gauss-Jordan inverse with partial pivoting of the leading n x n block of
 * a QMAX x QMAX array.  Returns 0 on success, -1 if singular. */
static int invert(int n, const double A[QMAX][QMAX], double Ainv[QMAX][QMAX]) {
  double a[QMAX][2 * QMAX];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      a[r][c] = c < n ? A[r][c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (fabs(a[piv][col]) < 1e-300) return -1;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    double inv = 1.0 / a[col][col];
    for (int c = 0; c < 2 * n; ++c) a[col][c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) a[r][c] -= f * a[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r][c] = a[r][c + n];
  return 0;
}

static void matvec(int n, const double A[QMAX][QMAX], const double* x,
                   double* y) {
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += A[r][c] * x[c];
    y[r] = s;
  }
}

/* Enumerate the set partitions of the multiset of axis labels given by
 * exponent (a,b,c): positions 0..n-1 carry labels x..x y..y z..z; every
 * partition of the positions is a restricted growth string. */
static void enumerate_partitions(lattice_t* L, int k) {
  int lab[6], n = 0;
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < L->expo[k][d]; ++t) lab[n++] = d;
  L->npart[k] = 0;
  if (n == 0) return;
  int rgs[6] = {0};
  for (;;) {
    partition_t* p = &L->part[k][L->npart[k]++];
    int nb = 0;
    for (int j = 0; j < n; ++j)
      if (rgs[j] + 1 > nb) nb = rgs[j] + 1;
    p->nblocks = nb;
    memset(p->e, 0, sizeof(p->e));
    for (int j = 0; j < n; ++j) p->e[rgs[j]][lab[j]]++;
    /* next restricted growth string */
    int j = n - 1;
    for (; j > 0; --j) {
      int mx = 0;
      for (int t = 0; t < j; ++t)
        if (rgs[t] > mx) mx = rgs[t];
      if (rgs[j] <= mx) {
        rgs[j]++;
        for (int t = j + 1; t < n; ++t) rgs[t] = 0;
        break;
      }
    }
    if (j == 0) break;
  }
}

static int in_set(int stencil, int a, int b, int c) {
  if (stencil == LBM_ORACLE_D2Q9) return c == 0;
  if (stencil == LBM_ORACLE_D3Q19) return (a > 0) + (b > 0) + (c > 0) <= 2;
  return 1;
}

/* Gram-Schmidt of the rows of B (polynomials in monomial coordinates) under
 * the inner product <p,q> = sum_i wt_i p(xi_i) q(xi_i) (wt = 1: unweighted;
 * wt = lattice weights: the weighted product of WO-MRT). */
static void gram_schmidt(lattice_t* L, double B[QMAX][QMAX], const double* wt) {
  int q = L->q;
  double V[QMAX][QMAX]; /* V[r][i] = p_r(xi_i) */
  for (int r = 0; r < q; ++r)
    for (int i = 0; i < q; ++i) {
      double s = 0.0;
      for (int k = 0; k < q; ++k) s += B[r][k] * L->M[k][i];
      V[r][i] = s;
    }
  for (int r = 0; r < q; ++r)
    for (int j = 0; j < r; ++j) {
      double num = 0.0, den = 0.0;
      for (int i = 0; i < q; ++i) {
        num += wt[i] * V[r][i] * V[j][i];
        den += wt[i] * V[j][i] * V[j][i];
      }
      double c = num / den;
      for (int i = 0; i < q; ++i) V[r][i] -= c * V[j][i];
      for (int k = 0; k < q; ++k) B[r][k] -= c * B[j][k];
    }
}

static void add_row(lattice_t* L, double B[QMAX][QMAX], int* r, int grp,
                    const int e[][3], const double* coef, int nterms) {
  for (int k = 0; k < L->q; ++k) B[*r][k] = 0.0;
  for (int t = 0; t < nterms; ++t)
    B[*r][L->mono[e[t][0]][e[t][1]][e[t][2]]] += coef[t];
  L->group[*r] = grp;
  (*r)++;
}

static int build_lattice(int stencil) {
  if (stencil < 0 || stencil > 2) return -1;
  lattice_t* L = &g_lat[stencil];
  if (L->ready) return 0;
  memset(L, 0, sizeof(*L));
  L->q = stencil == LBM_ORACLE_D2Q9 ? 9 : (stencil == LBM_ORACLE_D3Q19 ? 19 : 27);
  L->d = stencil == LBM_ORACLE_D2Q9 ? 2 : 3;
  for (int i = 0; i < L->q; ++i)
    for (int d = 0; d < 3; ++d)
      L->xi[i][d] = stencil == LBM_ORACLE_D2Q9 ? V2[i][d] : V3[i][d];
  for (int i = 0; i < L->q; ++i)
    for (int k = 0; k < L->q; ++k)
      if (L->xi[k][0] == -L->xi[i][0] && L->xi[k][1] == -L->xi[i][1] &&
          L->xi[k][2] == -L->xi[i][2])
        L->opp[i] = k;
  /* monomial exponent set, ordered by total degree then lexicographically */
  int n = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) L->mono[a][b][c] = -1;
  for (int deg = 0; deg <= 6; ++deg)
    for (int a = 2; a >= 0; --a)
      for (int b = 2; b >= 0; --b)
        for (int c = 2; c >= 0; --c) {
          if (a + b + c != deg || !in_set(stencil, a, b, c)) continue;
          L->expo[n][0] = a;
          L->expo[n][1] = b;
          L->expo[n][2] = c;
          L->deg[n] = deg;
          L->mono[a][b][c] = n++;
        }
  if (n != L->q) return -1;
  /* M[k][i] = prod_d xi_{i,d}^{e_{k,d}}  (Eq. 2.8) */
  for (int k = 0; k < L->q; ++k)
    for (int i = 0; i < L->q; ++i)
      L->M[k][i] = ipow(L->xi[i][0], L->expo[k][0]) *
                   ipow(L->xi[i][1], L->expo[k][1]) *
                   ipow(L->xi[i][2], L->expo[k][2]);
  if (invert(L->q, L->M, L->Minv)) return -1;
  /* background f0 = M^-1 m0 with m0 the moments of Psi(1, 0) (Sec. 2.4) */
  double m0[QMAX];
  for (int k = 0; k < L->q; ++k)
    m0[k] = gauss_moment(L->expo[k][0]) * gauss_moment(L->expo[k][1]) *
            gauss_moment(L->expo[k][2]);
  matvec(L->q, L->Minv, m0, L->w);

  /* homogeneous basis: 1 | x y z | shear (traceless 2nd order) | bulk
   * (trace) | every monomial of order 3, 4, 5, 6 */
  int r = 0;
  {
    static const int e0[1][3] = {{0, 0, 0}};
    static const double one[1] = {1.0};
    add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_CONSERVED, e0, one, 1);
    for (int d = 0; d < L->d; ++d) {
      int e1[1][3] = {{d == 0, d == 1, d == 2}};
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_CONSERVED, e1, one, 1);
    }
    static const double pm[2] = {1.0, -1.0}, pp[3] = {1.0, 1.0, 1.0};
    if (L->d == 2) {
      static const int xx_yy[2][3] = {{2, 0, 0}, {0, 2, 0}};
      static const int xy[1][3] = {{1, 1, 0}};
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xx_yy, pm, 2);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xy, one, 1);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_BULK, xx_yy, pp, 2);
    } else {
      static const int xx_yy[2][3] = {{2, 0, 0}, {0, 2, 0}};
      static const int xx_zz[2][3] = {{2, 0, 0}, {0, 0, 2}};
      static const int xy[1][3] = {{1, 1, 0}}, xz[1][3] = {{1, 0, 1}},
                       yz[1][3] = {{0, 1, 1}};
      static const int tr[3][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}};
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xx_yy, pm, 2);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xx_zz, pm, 2);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xy, one, 1);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, xz, one, 1);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_SHEAR, yz, one, 1);
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_BULK, tr, pp, 3);
    }
    for (int k = 0; k < L->q; ++k) {
      if (L->deg[k] < 3) continue;
      int ek[1][3] = {{L->expo[k][0], L->expo[k][1], L->expo[k][2]}};
      add_row(L, L->Pcm, &r, LBM_ORACLE_GROUP_ORDER3 + L->deg[k] - 3, ek, one,
              1);
    }
  }
  if (r != L->q) return -1;
  if (invert(L->q, L->Pcm, L->Pcminv)) return -1;
  /* orthogonal raw-moment basis (O-MRT, Sec. 4.2): same rows, unweighted
   * Gram-Schmidt in degree order */
  double ones[QMAX];
  for (int i = 0; i < QMAX; ++i) ones[i] = 1.0;
  memcpy(L->Praw, L->Pcm, sizeof(L->Praw));
  gram_schmidt(L, L->Praw, ones);
  if (invert(L->q, L->Praw, L->Prawinv)) return -1;
  /* weighted orthogonal raw basis (WO-MRT): Gram-Schmidt of the same rows
   * under the lattice-weight inner product */
  memcpy(L->Pw, L->Pcm, sizeof(L->Pw));
  gram_schmidt(L, L->Pw, L->w);
  if (invert(L->q, L->Pw, L->Pwinv)) return -1;
  for (int k = 0; k < L->q; ++k) enumerate_partitions(L, k);
  L->ready = 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* equilibria (Sec. 2.4, Eq. 2.12)                                      */
/* ------------------------------------------------------------------ */

/* Raw moment of Psi(rho, u) for exponent e:  rho prod_d E[(u_d + X)^e_d]
 * with X ~ N(0, 1/3).  truncate != 0 drops every term of total degree > 2
 * in u (the default second-order equilibrium, Sec. 4.2). */
static double maxwell_raw_moment(const int* e, double rho, const double* u,
                                 int truncate) {
  double s = 0.0;
  for (int ka = 0; ka <= e[0]; ++ka)
    for (int kb = 0; kb <= e[1]; ++kb)
      for (int kc = 0; kc <= e[2]; ++kc) {
        int udeg = (e[0] - ka) + (e[1] - kb) + (e[2] - kc);
        if (truncate && udeg > 2) continue;
        s += binom(e[0], ka) * ipow(u[0], e[0] - ka) * gauss_moment(ka) *
             binom(e[1], kb) * ipow(u[1], e[1] - kb) * gauss_moment(kb) *
             binom(e[2], kc) * ipow(u[2], e[2] - kc) * gauss_moment(kc);
      }
  return rho * s;
}

/* Central moment of Psi(rho, u): rho prod_d E[X^e_d], velocity-free. */
static double maxwell_central_moment(const int* e, double rho) {
  return rho * gauss_moment(e[0]) * gauss_moment(e[1]) * gauss_moment(e[2]);
}

/* The discrete second-order equilibrium as populations (Sec. 2.4, an
 * equilibrium prescribed as a discrete distribution):
 * f_eq_i = w_i rho (1 + 3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u), c_s^2 = 1/3. */
static void discrete_feq(const lattice_t* L, double rho, const double* u, double* feq) {
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < L->q; ++i) {
    const double xu = L->xi[i][0] * u[0] + L->xi[i][1] * u[1] + L->xi[i][2] * u[2];
    feq[i] = L->w[i] * rho * (1.0 + 3.0 * xu + 4.5 * xu * xu - 1.5 * uu);
  }
}

/* ------------------------------------------------------------------ */
/* cumulants (Eq. 2.11): c(S) = sum over set partitions pi of S of      */
/* (-1)^(|pi|-1) (|pi|-1)! prod_{B in pi} mu(B)  -- the coefficient     */
/* extraction of log M; inverse mu(S) = sum_pi prod_B c(B).             */
/* ------------------------------------------------------------------ */
static double fact(int n) {
  double r = 1.0;
  for (int k = 2; k <= n; ++k) r *= k;
  return r;
}

static double cumulant_from_mu(const partition_t* parts, int np,
                               const double mu[3][3][3]) {
  double s = 0.0;
  for (int p = 0; p < np; ++p) {
    int k = parts[p].nblocks;
    double prod = ((k - 1) % 2 ? -1.0 : 1.0) * fact(k - 1);
    for (int b = 0; b < k; ++b)
      prod *= mu[parts[p].e[b][0]][parts[p].e[b][1]][parts[p].e[b][2]];
    s += prod;
  }
  return s;
}

static double mu_from_cumulants(const partition_t* parts, int np,
                                const double c[3][3][3]) {
  double s = 0.0;
  for (int p = 0; p < np; ++p) {
    double prod = 1.0;
    for (int b = 0; b < parts[p].nblocks; ++b)
      prod *= c[parts[p].e[b][0]][parts[p].e[b][1]][parts[p].e[b][2]];
    s += prod;
  }
  return s;
}

/* ------------------------------------------------------------------ */
/* collision (Eq. 2.4-2.6)                                              */
/* ------------------------------------------------------------------ */
static double rate_of(const lbm_oracle_method* m, int grp) {
  return grp < 0 ? 0.0 : m->rates[grp];
}

/* q* = q + S (q_eq - q) in the basis P, acting on monomial quantities v:
 * v_out = P^-1 (P v + S P (v_eq - v)) */
static void relax(const lattice_t* L, const lbm_oracle_method* m,
                  const double P[QMAX][QMAX], const double Pinv[QMAX][QMAX],
                  const double* v, const double* veq, double* vout) {
  double qv[QMAX], qe[QMAX], qs[QMAX];
  matvec(L->q, P, v, qv);
  matvec(L->q, P, veq, qe);
  for (int r = 0; r < L->q; ++r)
    qs[r] = qv[r] + rate_of(m, L->group[r]) * (qe[r] - qv[r]);
  matvec(L->q, Pinv, qs, vout);
}

static void central_matrix(const lattice_t* L, const double* u,
                           double K[QMAX][QMAX]) {
  for (int k = 0; k < L->q; ++k)
    for (int i = 0; i < L->q; ++i)
      K[k][i] = ipow(L->xi[i][0] - u[0], L->expo[k][0]) *
                ipow(L->xi[i][1] - u[1], L->expo[k][1]) *
                ipow(L->xi[i][2] - u[2], L->expo[k][2]);
}

/* Guo's discrete source term of a body force F at velocity u:
 * S_i = w_i [ (xi_i - u).F / c_s^2 + (xi_i.u)(xi_i.F) / c_s^4 ],  c_s^2 = 1/3.
 * Its zeroth moment is 0 and its first moment F. */
static void guo_source(const lattice_t* L, const double* u, const double* F,
                       double* S) {
  for (int i = 0; i < L->q; ++i) {
    double cu = 0.0, cf = 0.0, uf = 0.0;
    for (int d = 0; d < 3; ++d) {
      cu += L->xi[i][d] * u[d];
      cf += L->xi[i][d] * F[d];
      uf += u[d] * F[d];
    }
    S[i] = L->w[i] * (3.0 * (cf - uf) + 9.0 * cu * cf);
  }
}

/* relax() plus the collision-space source of Eq. 2.4:
 * q* = q + S (q_eq - q) + (I - S/2) P sF, with sF the monomial moments of the
 * population source (conserved rows: rate 0, factor 1) */
static void relax_forced(const lattice_t* L, const lbm_oracle_method* m,
                         const double P[QMAX][QMAX],
                         const double Pinv[QMAX][QMAX], const double* v,
                         const double* veq, const double* sF, double* vout) {
  double qv[QMAX], qe[QMAX], qf[QMAX], qs[QMAX];
  matvec(L->q, P, v, qv);
  matvec(L->q, P, veq, qe);
  matvec(L->q, P, sF, qf);
  for (int r = 0; r < L->q; ++r) {
    const double om = rate_of(m, L->group[r]);
    qs[r] = qv[r] + om * (qe[r] - qv[r]) + (1.0 - 0.5 * om) * qf[r];
  }
  matvec(L->q, Pinv, qs, vout);
}

/* central-moment force (first-order rows only): v_k += F_d for the
 * monomial x_d of degree 1 */
static void add_first_order(const lattice_t* L, const double* F, double* v) {
  for (int k = 0; k < L->q; ++k)
    if (L->deg[k] == 1) {
      const int* e = L->expo[k];
      v[k] += F[e[0] ? 0 : (e[1] ? 1 : 2)];
    }
}

/* One cell.  F = NULL: no force.  With a body force F (Eq. 2.1a source term,
 * Eq. 2.4 q^F), the equilibrium velocity is u = (j + F/2) / rho and
 *   populations (SRT): f* = f + w (f_eq - f) + (1 - w/2) S      (Guo)
 *   raw moments:       q^F = (I - S/2) P M S                   (Guo, MRT)
 *   central moments:   moments about u; q^F = F on the first-order rows
 *                      only (kappa_1 = -F/2 before, +F/2 after, Sec. 4.2)
 *   cumulants:         orders >= 2 are translation invariant and relax as
 *                      without force; the first-order cumulant (the mean
 *                      velocity) leaves the collision as (j + F) / rho. */
static void swe_zhou_feq(const lattice_t* L, double h, const double* u,
                         double g, double* feq);

/* He's population source of a body force F at velocity u: the equilibrium
 * populations f_eq (absolute) weighted by (xi_i - u).F / (rho c_s^2) */
static void he_source(const lattice_t* L, double rho, const double* u,
                      const double* F, const double* feq, double* S) {
  for (int i = 0; i < L->q; ++i) {
    double cf = 0.0;
    for (int d = 0; d < 3; ++d) cf += (L->xi[i][d] - u[d]) * F[d];
    S[i] = 3.0 * cf / rho * feq[i];
  }
}

static int collide_cell_f(const lattice_t* L, const lbm_oracle_method* m,
                          const double* df, const double* F, double swe_g,
                          int model, double* out) {
  const int q = L->q;
  /* conserved quantities from the deviations, Eq. 2.3, rho0 = 1 */
  double drho = 0.0, j[3] = {0, 0, 0}, u[3];
  for (int i = 0; i < q; ++i) {
    drho += df[i];
    for (int d = 0; d < 3; ++d) j[d] += L->xi[i][d] * df[i];
  }
  const double rho = 1.0 + drho;
  static const double zero_F[3] = {0, 0, 0};
  const int forced = F != NULL;
  if (!forced) F = zero_F;
  const int shift = forced && m->space != LBM_ORACLE_SPACE_CUMULANT;
  for (int d = 0; d < 3; ++d) u[d] = (j[d] + (shift ? 0.5 * F[d] : 0.0)) / rho;
  double S[QMAX] = {0}, sF[QMAX] = {0};
  const int he = forced && model == 1;
  if (he && m->space == LBM_ORACLE_SPACE_CUMULANT) return -1;
  if (he) {
    /* the method's own equilibrium populations (absolute) at u */
    const int full = m->space == LBM_ORACLE_SPACE_CENTRAL;
    double meq[QMAX], feq[QMAX];
    for (int k = 0; k < q; ++k) meq[k] = maxwell_raw_moment(L->expo[k], rho, u, !full);
    matvec(q, L->Minv, meq, feq);
    he_source(L, rho, u, F, feq, S);
    matvec(q, L->M, S, sF);
  } else if (forced) {
    guo_source(L, u, F, S);
    matvec(q, L->M, S, sF);
  }
  const int delta = m->equilibrium == LBM_ORACLE_EQ_DELTA;
  const int disc = m->equilibrium == LBM_ORACLE_EQ_DISCRETE2; /* absolute path */
  if (disc && (forced || swe_g > 0.0)) return -1; /* not defined with a force */
  double f[QMAX] = {0}, tmp[QMAX] = {0}, tmp2[QMAX] = {0}, veq[QMAX] = {0},
         vout[QMAX] = {0};
  static const double zero_u[3] = {0, 0, 0};

  switch (m->space) {
    case LBM_ORACLE_SPACE_NONE:
      for (int i = 0; i < q; ++i) out[i] = df[i];
      return 0;
    case LBM_ORACLE_SPACE_TRT: {
      /* two relaxation times: the even part f+_i = (f_i + f_ibar)/2 relaxes
       * with w+ = rates[0], the odd part f-_i = (f_i - f_ibar)/2 with
       * w- = rates[2]; equilibrium and Guo source split the same way */
      if (disc) {
        discrete_feq(L, rho, u, tmp);
      } else {
        for (int k = 0; k < q; ++k)
          veq[k] = maxwell_raw_moment(L->expo[k], rho, u, 1) -
                   (delta ? maxwell_raw_moment(L->expo[k], 1.0, zero_u, 1) : 0.0);
        matvec(q, L->Minv, veq, tmp); /* delta: df_eq ; absolute: f_eq */
      }
      const double wp = m->rates[0], wm = m->rates[2];
      for (int i = 0; i < q; ++i) {
        const int ib = L->opp[i];
        const double fi = df[i] + (delta ? 0.0 : L->w[i]);
        const double fb = df[ib] + (delta ? 0.0 : L->w[ib]);
        const double fp = 0.5 * (fi + fb), fm = 0.5 * (fi - fb);
        const double ep = 0.5 * (tmp[i] + tmp[ib]), em = 0.5 * (tmp[i] - tmp[ib]);
        double o = fi - wp * (fp - ep) - wm * (fm - em);
        if (forced)
          o += (1.0 - 0.5 * wp) * 0.5 * (S[i] + S[ib]) +
               (1.0 - 0.5 * wm) * 0.5 * (S[i] - S[ib]);
        out[i] = o - (delta ? 0.0 : L->w[i]);
      }
      return 0;
    }
    case LBM_ORACLE_SPACE_POPULATIONS: {
      /* SRT: f* = f + w (f_eq - f), f_eq = M^-1 m_eq (truncated), or the
       * discrete f_eq itself */
      if (disc) {
        discrete_feq(L, rho, u, tmp);
      } else {
        for (int k = 0; k < q; ++k)
          veq[k] = maxwell_raw_moment(L->expo[k], rho, u, 1) -
                   (delta ? maxwell_raw_moment(L->expo[k], 1.0, zero_u, 1) : 0.0);
        matvec(q, L->Minv, veq, tmp); /* delta: df_eq ; absolute: f_eq */
      }
      const double om = m->rates[0];
      for (int i = 0; i < q; ++i) {
        if (delta)
          out[i] = df[i] + om * (tmp[i] - df[i]);
        else {
          double fi = df[i] + L->w[i];
          out[i] = fi + om * (tmp[i] - fi) - L->w[i];
        }
        if (forced) out[i] += (1.0 - 0.5 * om) * S[i];
      }
      return 0;
    }
    case LBM_ORACLE_SPACE_RAW:
    case LBM_ORACLE_SPACE_RAW_WEIGHTED: {
      /* O-MRT: unweighted orthogonal basis; WO-MRT: weighted (Sec. 4.2) */
      const int wo = m->space == LBM_ORACLE_SPACE_RAW_WEIGHTED;
      const double(*PR)[QMAX] = wo ? L->Pw : L->Praw;
      const double(*PRinv)[QMAX] = wo ? L->Pwinv : L->Prawinv;
      if (delta) { /* Eq. 2.5: dq = T(df), dq_eq = q_eq - q0 */
        matvec(q, L->M, df, tmp);
        for (int k = 0; k < q; ++k)
          veq[k] = maxwell_raw_moment(L->expo[k], rho, u, 1) -
                   maxwell_raw_moment(L->expo[k], 1.0, zero_u, 1);
        relax_forced(L, m, PR, PRinv, tmp, veq, sF, vout);
        matvec(q, L->Minv, vout, out);
      } else { /* Eq. 2.6 */
        for (int i = 0; i < q; ++i) f[i] = df[i] + L->w[i];
        matvec(q, L->M, f, tmp);
        if (disc) { /* q_eq = T(f_eq) */
          double fd[QMAX];
          discrete_feq(L, rho, u, fd);
          matvec(q, L->M, fd, veq);
        } else {
          for (int k = 0; k < q; ++k)
            veq[k] = maxwell_raw_moment(L->expo[k], rho, u, 1);
        }
        relax_forced(L, m, PR, PRinv, tmp, veq, sF, vout);
        matvec(q, L->Minv, vout, tmp2);
        for (int i = 0; i < q; ++i) out[i] = tmp2[i] - L->w[i];
      }
      return 0;
    }
    case LBM_ORACLE_SPACE_CENTRAL: {
      double K[QMAX][QMAX], Kinv[QMAX][QMAX];
      central_matrix(L, u, K);
      if (invert(q, K, Kinv)) return -1;
      if (delta) { /* Eq. 2.5 with T = K(u): q0 = K(u) f0 */
        double k0[QMAX];
        matvec(q, K, df, tmp);
        matvec(q, K, L->w, k0);
        for (int k = 0; k < q; ++k)
          veq[k] = maxwell_central_moment(L->expo[k], rho) - k0[k];
        if (he) { /* q^F = (I - S/2) P K(u) S */
          double sK[QMAX];
          matvec(q, K, S, sK);
          relax_forced(L, m, L->Pcm, L->Pcminv, tmp, veq, sK, vout);
        } else {
          relax(L, m, L->Pcm, L->Pcminv, tmp, veq, vout);
          add_first_order(L, F, vout);
        }
        matvec(q, Kinv, vout, out);
      } else { /* Eq. 2.6 */
        for (int i = 0; i < q; ++i) f[i] = df[i] + L->w[i];
        matvec(q, K, f, tmp);
        if (swe_g > 0.0) { /* shallow water: central moments of Zhou's f_eq */
          double fz[QMAX];
          swe_zhou_feq(L, rho, u, swe_g, fz);
          matvec(q, K, fz, veq);
        } else if (disc) { /* q_eq = K(u) f_eq */
          double fd[QMAX];
          discrete_feq(L, rho, u, fd);
          matvec(q, K, fd, veq);
        } else {
          for (int k = 0; k < q; ++k)
            veq[k] = maxwell_central_moment(L->expo[k], rho);
        }
        if (he) {
          double sK[QMAX];
          matvec(q, K, S, sK);
          relax_forced(L, m, L->Pcm, L->Pcminv, tmp, veq, sK, vout);
        } else {
          relax(L, m, L->Pcm, L->Pcminv, tmp, veq, vout);
          add_first_order(L, F, vout);
        }
        matvec(q, Kinv, vout, tmp2);
        for (int i = 0; i < q; ++i) out[i] = tmp2[i] - L->w[i];
      }
      return 0;
    }
    case LBM_ORACLE_SPACE_CUMULANT: {
      if (delta) return -3; /* no zero-centered cumulants (Sec. 2.4, 3) */
      double mu[3][3][3], c[3][3][3];
      for (int a = 0; a < 27; ++a) (&mu[0][0][0])[a] = NAN, (&c[0][0][0])[a] = NAN;
      for (int i = 0; i < q; ++i) f[i] = df[i] + L->w[i];
      matvec(q, L->M, f, tmp);
      const double rho_a = tmp[0]; /* = m_000 */
      double v[QMAX] = {0};
      for (int k = 0; k < q; ++k) {
        const int* e = L->expo[k];
        mu[e[0]][e[1]][e[2]] = tmp[k] / rho_a;
      }
      double mueq[3][3][3]; /* discrete equilibrium: its own cumulants */
      if (disc) {
        double fd[QMAX], md[QMAX];
        for (int a = 0; a < 27; ++a) (&mueq[0][0][0])[a] = NAN;
        discrete_feq(L, rho, u, fd);
        matvec(q, L->M, fd, md);
        for (int k = 0; k < q; ++k) {
          const int* e = L->expo[k];
          mueq[e[0]][e[1]][e[2]] = md[k] / md[0];
        }
      }
      for (int k = 0; k < q; ++k) {
        const int* e = L->expo[k];
        if (L->deg[k] == 0)
          v[k] = rho_a;
        else if (L->deg[k] == 1)
          v[k] = mu[e[0]][e[1]][e[2]];
        else
          v[k] = rho_a * cumulant_from_mu(L->part[k], L->npart[k], mu);
        /* equilibrium cumulants of Psi: C_eq = rho c_s^2 on the diagonal
         * of order 2, zero above; orders 0 and 1 are conserved */
        if (L->deg[k] <= 1)
          veq[k] = v[k];
        else if (disc)
          veq[k] = rho_a * cumulant_from_mu(L->part[k], L->npart[k], mueq);
        else
          veq[k] = (L->deg[k] == 2 && (e[0] == 2 || e[1] == 2 || e[2] == 2))
                       ? rho_a * (swe_g > 0.0 ? 0.5 * swe_g * rho_a : 1.0 / 3.0)
                       : 0.0;
      }
      relax(L, m, L->Pcm, L->Pcminv, v, veq, vout);
      for (int k = 0; k < q; ++k) {
        const int* e = L->expo[k];
        double mean = 0.0; /* post-collision mean velocity (j + F) / rho */
        if (L->deg[k] == 1)
          mean = forced ? v[k] + F[e[0] ? 0 : (e[1] ? 1 : 2)] / rho_a : v[k];
        c[e[0]][e[1]][e[2]] =
            L->deg[k] >= 2 ? vout[k] / rho_a : (L->deg[k] == 1 ? mean : 1.0);
      }
      for (int k = 0; k < q; ++k) {
        tmp2[k] = L->deg[k] == 0
                      ? rho_a
                      : rho_a * mu_from_cumulants(L->part[k], L->npart[k], c);
      }
      matvec(q, L->Minv, tmp2, f);
      for (int i = 0; i < q; ++i) out[i] = f[i] - L->w[i];
      return 0;
    }
  }
  return -1;
}

static int collide_cell(const lattice_t* L, const lbm_oracle_method* m,
                        const double* df, double* out) {
  return collide_cell_f(L, m, df, NULL, 0.0, 0, out);
}

static int check_method(const lbm_oracle_method* m) {
  if (!m || build_lattice(m->stencil)) return -1;
  if (m->space < 0 || m->space > 6) return -1;
  if (m->equilibrium != LBM_ORACLE_EQ_DELTA &&
      m->equilibrium != LBM_ORACLE_EQ_ABSOLUTE &&
      m->equilibrium != LBM_ORACLE_EQ_DISCRETE2)
    return -1;
  if (m->space == LBM_ORACLE_SPACE_CUMULANT &&
      m->equilibrium == LBM_ORACLE_EQ_DELTA)
    return -3;
  return 0;
}

/* ------------------------------------------------------------------ */
/* exported API                                                         */
/* ------------------------------------------------------------------ */
int lbm_oracle_lattice(int stencil, int* q, int* d, int* xi, double* w,
                       int* expo) {
  if (build_lattice(stencil)) return -1;
  const lattice_t* L = &g_lat[stencil];
  if (q) *q = L->q;
  if (d) *d = L->d;
  for (int i = 0; i < L->q; ++i)
    for (int k = 0; k < 3; ++k) {
      if (xi) xi[i * 3 + k] = L->xi[i][k];
      if (expo) expo[i * 3 + k] = L->expo[i][k];
    }
  if (w)
    for (int i = 0; i < L->q; ++i) w[i] = L->w[i];
  return 0;
}

int lbm_oracle_matrices(int stencil, double* M, double* Minv, double* Praw,
                        double* Pcm, int* group) {
  if (build_lattice(stencil)) return -1;
  const lattice_t* L = &g_lat[stencil];
  int q = L->q;
  for (int r = 0; r < q; ++r) {
    for (int c = 0; c < q; ++c) {
      if (M) M[r * q + c] = L->M[r][c];
      if (Minv) Minv[r * q + c] = L->Minv[r][c];
      if (Praw) Praw[r * q + c] = L->Praw[r][c];
      if (Pcm) Pcm[r * q + c] = L->Pcm[r][c];
    }
    if (group) group[r] = L->group[r];
  }
  return 0;
}

int lbm_oracle_weighted_basis(int stencil, double* Pw) {
  if (build_lattice(stencil) || !Pw) return -1;
  const lattice_t* L = &g_lat[stencil];
  for (int r = 0; r < L->q; ++r)
    for (int c = 0; c < L->q; ++c) Pw[r * L->q + c] = L->Pw[r][c];
  return 0;
}

int lbm_oracle_central_matrix(int stencil, const double* u, double* K) {
  if (build_lattice(stencil) || !u || !K) return -1;
  const lattice_t* L = &g_lat[stencil];
  double Km[QMAX][QMAX];
  central_matrix(L, u, Km);
  for (int r = 0; r < L->q; ++r)
    for (int c = 0; c < L->q; ++c) K[r * L->q + c] = Km[r][c];
  return 0;
}

int lbm_oracle_cumulants(int stencil, const double* f, double* out) {
  if (build_lattice(stencil) || !f || !out) return -1;
  const lattice_t* L = &g_lat[stencil];
  double m[QMAX], mu[3][3][3];
  for (int a = 0; a < 27; ++a) (&mu[0][0][0])[a] = NAN;
  matvec(L->q, L->M, f, m);
  for (int k = 0; k < L->q; ++k)
    mu[L->expo[k][0]][L->expo[k][1]][L->expo[k][2]] = m[k] / m[0];
  for (int k = 0; k < L->q; ++k) {
    const int* e = L->expo[k];
    if (L->deg[k] == 0)
      out[k] = m[0];
    else if (L->deg[k] == 1)
      out[k] = mu[e[0]][e[1]][e[2]];
    else
      out[k] = m[0] * cumulant_from_mu(L->part[k], L->npart[k], mu);
  }
  return 0;
}

int lbm_oracle_moments_from_cumulants(int stencil, const double* c_in,
                                      double* m) {
  if (build_lattice(stencil) || !c_in || !m) return -1;
  const lattice_t* L = &g_lat[stencil];
  double c[3][3][3];
  for (int a = 0; a < 27; ++a) (&c[0][0][0])[a] = NAN;
  const double rho = c_in[0];
  for (int k = 0; k < L->q; ++k) {
    const int* e = L->expo[k];
    c[e[0]][e[1]][e[2]] = L->deg[k] >= 2 ? c_in[k] / rho : c_in[k];
  }
  c[0][0][0] = 1.0;
  for (int k = 0; k < L->q; ++k)
    m[k] = L->deg[k] == 0
               ? rho
               : rho * mu_from_cumulants(L->part[k], L->npart[k], c);
  return 0;
}

double lbm_oracle_cumulant_of(const double* mu27, int a, int b, int c) {
  if (build_lattice(LBM_ORACLE_D3Q27)) return NAN;
  if (a < 0 || a > 2 || b < 0 || b > 2 || c < 0 || c > 2) return NAN;
  const lattice_t* L = &g_lat[LBM_ORACLE_D3Q27];
  double mu[3][3][3];
  memcpy(mu, mu27, sizeof(mu));
  int k = L->mono[a][b][c];
  if (L->deg[k] == 0) return 0.0;
  return cumulant_from_mu(L->part[k], L->npart[k], mu);
}

int lbm_oracle_collide(const lbm_oracle_method* m, int64_t ncells,
                       const double* df_in, double* df_out) {
  int rc = check_method(m);
  if (rc) return rc;
  const lattice_t* L = &g_lat[m->stencil];
  for (int64_t c = 0; c < ncells; ++c) {
    double tmp[QMAX];
    rc = collide_cell(L, m, df_in + c * L->q, tmp);
    if (rc) return rc;
    memcpy(df_out + c * L->q, tmp, sizeof(double) * L->q);
  }
  return 0;
}

int lbm_oracle_collide_forced(const lbm_oracle_method* m, int64_t ncells,
                              const double* df_in, const double* force,
                              int model, double* df_out) {
  int rc = check_method(m);
  if (rc) return rc;
  if (!force || m->space == LBM_ORACLE_SPACE_NONE || model < 0 || model > 1)
    return -1;
  const lattice_t* L = &g_lat[m->stencil];
  for (int64_t c = 0; c < ncells; ++c) {
    double tmp[QMAX], F[3] = {0, 0, 0};
    for (int d = 0; d < L->d; ++d) F[d] = force[c * 3 + d];
    rc = collide_cell_f(L, m, df_in + c * L->q, F, 0.0, model, tmp);
    if (rc) return rc;
    memcpy(df_out + c * L->q, tmp, sizeof(double) * L->q);
  }
  return 0;
}

static void equilibrium_cell(const lattice_t* L, const lbm_oracle_method* m,
                             double rho, const double* u, double* out) {
  /* raw-moment methods relax to the truncated equilibrium; central-moment
   * and cumulant methods to the full Maxwellian (velocity-free central
   * moments), so each method's own equilibrium is a collision fixed point */
  static const double zero_u[3] = {0, 0, 0};
  const int trunc = m->space == LBM_ORACLE_SPACE_RAW ||
                    m->space == LBM_ORACLE_SPACE_RAW_WEIGHTED ||
                    m->space == LBM_ORACLE_SPACE_POPULATIONS ||
                    m->space == LBM_ORACLE_SPACE_TRT ||
                    m->space == LBM_ORACLE_SPACE_NONE;
  if (m->equilibrium == LBM_ORACLE_EQ_DISCRETE2) { /* the discrete f_eq - w */
    discrete_feq(L, rho, u, out);
    for (int i = 0; i < L->q; ++i) out[i] -= L->w[i];
    return;
  }
  double dm[QMAX];
  for (int k = 0; k < L->q; ++k)
    dm[k] = maxwell_raw_moment(L->expo[k], rho, u, trunc) -
            maxwell_raw_moment(L->expo[k], 1.0, zero_u, trunc);
  matvec(L->q, L->Minv, dm, out);
}

int lbm_oracle_equilibrium(const lbm_oracle_method* m, int64_t ncells,
                           const double* rho, const double* u, double* df_out) {
  int rc = check_method(m);
  if (rc) return rc;
  const lattice_t* L = &g_lat[m->stencil];
  for (int64_t c = 0; c < ncells; ++c)
    equilibrium_cell(L, m, rho[c], u + 3 * c, df_out + c * L->q);
  return 0;
}

int lbm_oracle_init(const lbm_oracle_method* m, const int64_t* dims,
                    const double* rho, const double* u, double* df) {
  int rc = check_method(m);
  if (rc) return rc;
  const lattice_t* L = &g_lat[m->stencil];
  const int64_t N = dims[0] * dims[1] * dims[2];
  for (int64_t c = 0; c < N; ++c) {
    double uc[3] = {u[c], u[N + c], L->d == 3 ? u[2 * N + c] : 0.0}, out[QMAX];
    equilibrium_cell(L, m, rho[c], uc, out);
    for (int i = 0; i < L->q; ++i) df[i * N + c] = out[i];
  }
  return 0;
}

int lbm_oracle_step(const lbm_oracle_method* m, const int64_t* dims,
                    double* df, int64_t nsteps, int nthreads) {
  return lbm_oracle_step_forced(m, dims, df, NULL, 0, nsteps, nthreads);
}

static int step_impl(const lbm_oracle_method* m, const int64_t* dims,
                     double* df, const double* force, double swe_g, int model,
                     int64_t nsteps, int nthreads);

int lbm_oracle_step_forced(const lbm_oracle_method* m, const int64_t* dims,
                           double* df, const double* force, int model,
                           int64_t nsteps, int nthreads) {
  if (model < 0 || model > 1) return -1;
  return step_impl(m, dims, df, force, 0.0, model, nsteps, nthreads);
}

static int step_impl(const lbm_oracle_method* m, const int64_t* dims,
                     double* df, const double* force, double swe_g, int model,
                     int64_t nsteps, int nthreads) {
  int rc = check_method(m);
  if (rc) return rc;
  if (force && m->space == LBM_ORACLE_SPACE_NONE) return -1;
  const lattice_t* L = &g_lat[m->stencil];
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
  if (L->d == 2 && nz != 1) return -1;
  const int64_t N = nx * ny * nz;
  const int q = L->q;
  double* out = (double*)malloc(sizeof(double) * q * N);
  if (!out) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int err = 0;
  for (int64_t s = 0; s < nsteps && !err; ++s) {
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int64_t c = 0; c < N; ++c) {
      const int64_t x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
      double in[QMAX], post[QMAX], F[3] = {0, 0, 0};
      for (int i = 0; i < q; ++i) in[i] = df[i * N + c];
      if (force)
        for (int d = 0; d < L->d; ++d) F[d] = force[d * N + c];
      if (collide_cell_f(L, m, in, force ? F : NULL, swe_g, model, post)) err |= 1;
      /* Eq. 2.1b: f_i(x + xi_i, t + 1) = f*_i(x, t), periodic */
      for (int i = 0; i < q; ++i) {
        int64_t xd = (x + L->xi[i][0] + nx) % nx;
        int64_t yd = (y + L->xi[i][1] + ny) % ny;
        int64_t zd = (z + L->xi[i][2] + nz) % nz;
        out[i * N + (zd * ny + yd) * nx + xd] = post[i];
      }
    }
    memcpy(df, out, sizeof(double) * q * N);
  }
  free(out);
  return err ? -1 : 0;
}

int lbm_oracle_macroscopic(const lbm_oracle_method* m, const int64_t* dims,
                           const double* df, double* rho, double* u) {
  return lbm_oracle_macroscopic_forced(m, dims, df, NULL, rho, u);
}

int lbm_oracle_macroscopic_forced(const lbm_oracle_method* m,
                                  const int64_t* dims, const double* df,
                                  const double* force, double* rho, double* u) {
  if (!m || build_lattice(m->stencil)) return -1;
  const lattice_t* L = &g_lat[m->stencil];
  const int64_t N = dims[0] * dims[1] * dims[2];
  for (int64_t c = 0; c < N; ++c) {
    double drho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < L->q; ++i) {
      drho += df[i * N + c];
      for (int d = 0; d < 3; ++d) j[d] += L->xi[i][d] * df[i * N + c];
    }
    rho[c] = 1.0 + drho;
    /* with a body force the fluid velocity is (j + F/2) / rho (Guo) */
    for (int d = 0; d < L->d; ++d)
      u[d * N + c] = (j[d] + (force ? 0.5 * force[d * N + c] : 0.0)) / rho[c];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* learned closure (test infrastructure for the GPU closure kernels)   */
/* ------------------------------------------------------------------ */
static double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

static double inv2(const double A[3][3]) { /* second principal invariant */
  double tr = A[0][0] + A[1][1] + A[2][2], trsq = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) trsq += A[a][b] * A[b][a];
  return 0.5 * (tr * tr - trsq);
}

static int features_cell(const lattice_t* L, const double* df, double omega_s,
                         double* out) {
  double f[QMAX], K[QMAX][QMAX], kappa[QMAX], u[3], drho = 0.0, j[3] = {0, 0, 0};
  for (int i = 0; i < L->q; ++i) {
    f[i] = df[i] + L->w[i];
    drho += df[i];
    for (int d = 0; d < 3; ++d) j[d] += L->xi[i][d] * df[i];
  }
  const double rho = 1.0 + drho;
  for (int d = 0; d < 3; ++d) u[d] = j[d] / rho;
  central_matrix(L, u, K);
  matvec(L->q, K, f, kappa);
  double Pi[3][3], S[3][3], D[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      int e[3] = {0, 0, 0};
      e[a]++;
      e[b]++;
      const int k = L->mono[e[0]][e[1]][e[2]];
      if (k < 0) return -1;
      Pi[a][b] = kappa[k] / rho - (a == b ? 1.0 / 3.0 : 0.0);
      S[a][b] = -1.5 * omega_s * Pi[a][b];
    }
  const double trP = Pi[0][0] + Pi[1][1] + Pi[2][2];
  double fro = 0.0, nS2 = 0.0, nD2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      D[a][b] = Pi[a][b] - (a == b ? trP / 3.0 : 0.0);
      fro += Pi[a][b] * Pi[a][b];
      nS2 += S[a][b] * S[a][b];
      nD2 += D[a][b] * D[a][b];
    }
  /* conditioning: an invariant of degree k in its tensor is divided by the
   * (k-1)-th power of that tensor's Frobenius norm (0 where the norm is 0),
   * so every feature but drho is of degree 1 in Pi and Lipschitz */
  const double nS = sqrt(nS2), nD = sqrt(nD2);
  out[0] = S[0][0] + S[1][1] + S[2][2];
  out[1] = nS > 0.0 ? inv2(S) / nS : 0.0;
  out[2] = nS > 0.0 ? det3(S) / nS2 : 0.0;
  out[3] = nD > 0.0 ? inv2(D) / nD : 0.0;
  out[4] = nD > 0.0 ? det3(D) / nD2 : 0.0;
  out[5] = sqrt(fro);
  out[6] = drho;
  return 0;
}

int lbm_oracle_closure_features(int stencil, const double* df,
                                double omega_shear, double out[7]) {
  if (build_lattice(stencil) || stencil == LBM_ORACLE_D2Q9 || !df || !out) return -1;
  return features_cell(&g_lat[stencil], df, omega_shear, out);
}

int lbm_oracle_closure_mlp(const double* P, const double* shift,
                           const double* scale, const double raw[7],
                           double omega[4]) {
  enum { NI = LBM_ORACLE_CLOSURE_NIN, NH = LBM_ORACLE_CLOSURE_NH, NO = LBM_ORACLE_CLOSURE_NOUT };
  const double* W1 = P;
  const double* b1 = W1 + NH * NI;
  const double* W2 = b1 + NH;
  const double* b2 = W2 + NH * NH;
  const double* W3 = b2 + NH;
  const double* b3 = W3 + NO * NH;
  double x[NI], h1[NH], h2[NH];
  int ok = 1;
  for (int i = 0; i < NI; ++i) {
    x[i] = (raw[i] - shift[i]) * scale[i];
    /* usable input: finite and within FP16's range (|x| <= 65504), the
       operand range of the GPU network; otherwise the cell keeps rates 1 */
    ok = ok && x[i] <= 65504.0 && x[i] >= -65504.0;
  }
  for (int r = 0; r < NH; ++r) {
    double a = b1[r];
    for (int c = 0; c < NI; ++c) a += W1[r * NI + c] * x[c];
    h1[r] = tanh(a);
  }
  for (int r = 0; r < NH; ++r) {
    double a = b2[r];
    for (int c = 0; c < NH; ++c) a += W2[r * NH + c] * h1[c];
    h2[r] = tanh(a);
  }
  for (int r = 0; r < NO; ++r) {
    double z = b3[r];
    for (int c = 0; c < NH; ++c) z += W3[r * NH + c] * h2[c];
    double om = 2.0 / (1.0 + exp(-z));
    if (om < 1e-3) om = 1e-3;
    if (om > 1.999) om = 1.999;
    omega[r] = om;
    ok = ok && isfinite(om);
  }
  if (!ok)
    for (int r = 0; r < NO; ++r) omega[r] = 1.0;
  return 0;
}

int lbm_oracle_closure_step(const lbm_oracle_method* base,
                            const int64_t* dims, double* df,
                            const double* params, const double* shift,
                            const double* scale, int nthreads) {
  int rc = check_method(base);
  if (rc) return rc;
  const lattice_t* L = &g_lat[base->stencil];
  if (L->d != 3) return -1;
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2], N = nx * ny * nz;
  const int q = L->q;
  double* out = (double*)malloc(sizeof(double) * q * N);
  if (!out) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t c = 0; c < N; ++c) {
    const int64_t x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    double in[QMAX], post[QMAX], raw[7], om[4];
    for (int i = 0; i < q; ++i) in[i] = df[i * N + c];
    lbm_oracle_method m = *base;
    if (features_cell(L, in, base->rates[0], raw)) err |= 1;
    lbm_oracle_closure_mlp(params, shift, scale, raw, om);
    for (int k = 0; k < 4; ++k) m.rates[2 + k] = om[k];
    if (collide_cell(L, &m, in, post)) err |= 1;
    for (int i = 0; i < q; ++i) {
      int64_t xd = (x + L->xi[i][0] + nx) % nx;
      int64_t yd = (y + L->xi[i][1] + ny) % ny;
      int64_t zd = (z + L->xi[i][2] + nz) % nz;
      out[i * N + (zd * ny + yd) * nx + xd] = post[i];
    }
  }
  memcpy(df, out, sizeof(double) * q * N);
  free(out);
  return err ? -1 : 0;
}

double lbm_oracle_closure_loss(const lbm_oracle_method* base,
                               const int64_t* dims, const double* df_s,
                               const double* df_t, const double* params,
                               const double* shift, const double* scale,
                               int nthreads) {
  if (check_method(base)) return NAN;
  const lattice_t* L = &g_lat[base->stencil];
  const int64_t N = dims[0] * dims[1] * dims[2];
  double* work = (double*)malloc(sizeof(double) * L->q * N);
  double *r1 = (double*)malloc(sizeof(double) * N), *r2 = (double*)malloc(sizeof(double) * N);
  double *u1 = (double*)malloc(sizeof(double) * 3 * N), *u2 = (double*)malloc(sizeof(double) * 3 * N);
  double loss = NAN;
  if (work && r1 && r2 && u1 && u2) {
    memcpy(work, df_s, sizeof(double) * L->q * N);
    if (lbm_oracle_closure_step(base, dims, work, params, shift, scale, nthreads) == 0 &&
        lbm_oracle_macroscopic(base, dims, work, r1, u1) == 0 &&
        lbm_oracle_macroscopic(base, dims, df_t, r2, u2) == 0) {
      double s = 0.0;
      for (int64_t k = 0; k < 3 * N; ++k) s += (u1[k] - u2[k]) * (u1[k] - u2[k]);
      loss = s / (double)N;
    }
  }
  free(work);
  free(r1);
  free(r2);
  free(u1);
  free(u2);
  return loss;
}

double lbm_oracle_closure_rollout_loss(const lbm_oracle_method* base,
                                       const int64_t* dims, const double* df,
                                       int K, const double* params,
                                       const double* shift, const double* scale,
                                       int nthreads) {
  if (check_method(base) || K < 1) return NAN;
  const lattice_t* L = &g_lat[base->stencil];
  const int64_t N = dims[0] * dims[1] * dims[2];
  const int64_t QN = (int64_t)L->q * N;
  double* work = (double*)malloc(sizeof(double) * QN);
  double *r1 = (double*)malloc(sizeof(double) * N), *r2 = (double*)malloc(sizeof(double) * N);
  double *u1 = (double*)malloc(sizeof(double) * 3 * N), *u2 = (double*)malloc(sizeof(double) * 3 * N);
  double loss = NAN;
  if (work && r1 && r2 && u1 && u2) {
    memcpy(work, df, sizeof(double) * QN);
    double s = 0.0;
    int k = 1;
    for (; k <= K; ++k) {
      if (lbm_oracle_closure_step(base, dims, work, params, shift, scale, nthreads) != 0 ||
          lbm_oracle_macroscopic(base, dims, work, r1, u1) != 0 ||
          lbm_oracle_macroscopic(base, dims, df + k * QN, r2, u2) != 0)
        break;
      double sk = 0.0;
      for (int64_t c = 0; c < 3 * N; ++c) sk += (u1[c] - u2[c]) * (u1[c] - u2[c]);
      s += sk / (double)N;
    }
    if (k > K) loss = s / (double)K;
  }
  free(work);
  free(r1);
  free(r2);
  free(u1);
  free(u2);
  return loss;
}

/* ------------------------------------------------------------------ */
/* shallow water (Sec. 5.2): D2Q9, depth h = sum f, h u = sum xi f       */
/* ------------------------------------------------------------------ */
/* Zhou's discrete equilibrium (Sec. 5.2): rest f0 = h (1 - 5gh/6 - 2u.u/3),
 * moving f_i = l_i h (gh/6 + xi.u/3 + (xi.u)^2/2 - u.u/6), l_i = 1 on the
 * axes and 1/4 on the diagonals. */
static void swe_zhou_feq(const lattice_t* L, double h, const double* u,
                         double g, double* feq) {
  const double uu = u[0] * u[0] + u[1] * u[1];
  for (int i = 0; i < L->q; ++i) {
    const int s = abs(L->xi[i][0]) + abs(L->xi[i][1]);
    const double cu = L->xi[i][0] * u[0] + L->xi[i][1] * u[1];
    if (s == 0)
      feq[i] = h * (1.0 - 5.0 * g * h / 6.0 - 2.0 * uu / 3.0);
    else
      feq[i] = (s == 1 ? 1.0 : 0.25) * h *
               (g * h / 6.0 + cu / 3.0 + 0.5 * cu * cu - uu / 6.0);
  }
}

/* continuous Maxwellian of variance c2 per axis (the cumulant method's
 * equilibrium with c_s^2 = g h / 2), as D2Q9 populations */
static void swe_maxwell_feq(const lattice_t* L, double h, const double* u,
                            double c2, double* feq) {
  double m[QMAX];
  for (int k = 0; k < L->q; ++k) {
    double p = h;
    for (int d = 0; d < 2; ++d) {
      const int e = L->expo[k][d];
      p *= e == 0 ? 1.0 : (e == 1 ? u[d] : u[d] * u[d] + c2);
    }
    m[k] = p;
  }
  matvec(L->q, L->Minv, m, feq);
}

static int swe_check(const lbm_oracle_method* m, double g) {
  int rc = check_method(m);
  if (rc) return rc;
  if (m->stencil != LBM_ORACLE_D2Q9 || !(g > 0.0) ||
      m->equilibrium != LBM_ORACLE_EQ_ABSOLUTE ||
      (m->space != LBM_ORACLE_SPACE_CENTRAL &&
       m->space != LBM_ORACLE_SPACE_CUMULANT))
    return -1;
  return 0;
}

int lbm_oracle_swe_equilibrium(int space, double g, double h, const double* u,
                               double* f) {
  if (build_lattice(LBM_ORACLE_D2Q9) || !u || !f || !(g > 0.0)) return -1;
  const lattice_t* L = &g_lat[LBM_ORACLE_D2Q9];
  const double uu[3] = {u[0], u[1], 0.0};
  if (space == LBM_ORACLE_SPACE_CENTRAL)
    swe_zhou_feq(L, h, uu, g, f);
  else if (space == LBM_ORACLE_SPACE_CUMULANT)
    swe_maxwell_feq(L, h, uu, 0.5 * g * h, f);
  else
    return -1;
  return 0;
}

int lbm_oracle_swe_collide(const lbm_oracle_method* m, double g, int64_t ncells,
                           const double* df_in, double* df_out) {
  int rc = swe_check(m, g);
  if (rc) return rc;
  const lattice_t* L = &g_lat[m->stencil];
  for (int64_t c = 0; c < ncells; ++c) {
    double tmp[QMAX];
    rc = collide_cell_f(L, m, df_in + c * L->q, NULL, g, 0, tmp);
    if (rc) return rc;
    memcpy(df_out + c * L->q, tmp, sizeof(double) * L->q);
  }
  return 0;
}

int lbm_oracle_swe_init(const lbm_oracle_method* m, double g,
                        const int64_t* dims, const double* h, const double* u,
                        double* df) {
  int rc = swe_check(m, g);
  if (rc) return rc;
  const lattice_t* L = &g_lat[m->stencil];
  const int64_t N = dims[0] * dims[1] * dims[2];
  for (int64_t c = 0; c < N; ++c) {
    const double uc[3] = {u[c], u[N + c], 0.0};
    double fe[QMAX];
    if (m->space == LBM_ORACLE_SPACE_CENTRAL)
      swe_zhou_feq(L, h[c], uc, g, fe);
    else
      swe_maxwell_feq(L, h[c], uc, 0.5 * g * h[c], fe);
    for (int i = 0; i < L->q; ++i) df[i * N + c] = fe[i] - L->w[i];
  }
  return 0;
}

int lbm_oracle_swe_step(const lbm_oracle_method* m, double g,
                        const int64_t* dims, double* df, int64_t nsteps,
                        int nthreads) {
  int rc = swe_check(m, g);
  if (rc) return rc;
  return step_impl(m, dims, df, NULL, g, 0, nsteps, nthreads);
}
