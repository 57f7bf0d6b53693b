// lbm_device.cuh -- per-cell collision arithmetic of the zero-centered MRT
// lattice Boltzmann step, unrolled at compile time into registers.
//
// All quantities are carried as deviations from the rest-state background
// (rho0 = 1, u = 0), the paper's zero-centering (Sec. 2.1) extended through
// every transform: raw moments dm, central moments dkappa, normalised
// central moments dk = kappa/rho - k0 and cumulants dc = c - c0 are all
// small numbers, so FP32 registers keep their full relative precision.  The
// rest-state background of every monomial quantity is the product of the
// per-axis factors b = (1, 0, 1/3) (Maxwellian moments, Eq. 2.12).
//
// Steps (Sec. 4.1):
//   fwd_raw_chimera   f -> dm           Eq. 4.1 (three 3-point passes)
//   binomial<-1>      dm -> dkappa      Eq. 4.3 left column (powers of -u)
//   cumulant_fwd/bwd  dk <-> dc         Eq. 4.5 (orders 4-6 nonlinear)
//   relax             q* = q + S(q_eq - q), per rate group   Eq. 2.4
//   binomial<+1>      dkappa* -> dm*    Eq. 4.3 right column (powers of +u)
//   bwd_raw           dm* -> f*         Eq. 4.2 (symmetric/antisymmetric)
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#define LBM_HD __host__ __device__ __forceinline__
// per-cell math is host-callable too (used by host-side unit checks)
#define LBM_D __host__ __device__ __forceinline__
#define CI(K) (decltype(K)::value)

namespace lbm {

enum { D2Q9 = 0, D3Q19 = 1, D3Q27 = 2 };
enum { SP_SRT = 0, SP_RAW = 1, SP_CENTRAL = 2, SP_CUMULANT = 3, SP_TRT = 4, SP_RAW_W = 5 };

// ---------------------------------------------------------------- helpers
template <class F, int... Is>
LBM_HD void sfor_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
// compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1
template <int N, class F>
LBM_HD void sfor(F&& f) {
  sfor_impl(f, std::make_integer_sequence<int, N>{});
}

LBM_HD constexpr int q_of(int st) { return st == D2Q9 ? 9 : (st == D3Q19 ? 19 : 27); }
LBM_HD constexpr int dim_of(int st) { return st == D2Q9 ? 2 : 3; }

// velocity components in the documented order (include/lbm.h)
LBM_HD constexpr int vel(int st, int i, int d) {
  constexpr int v2[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},
                            {0, 1, 0},  {0, -1, 0},  {1, 1, 0},
                            {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
  constexpr int v3[27][3] = {
      {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
      {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
      {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
      {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},
      {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
      {1, -1, -1}, {-1, 1, 1}};
  return st == D2Q9 ? v2[i][d] : v3[i][d];
}
LBM_HD constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// monomial x^a y^b z^c belongs to the stencil's exponent set
LBM_HD constexpr bool has_mono(int st, int a, int b, int c) {
  return st == D2Q9 ? (c == 0) : (st == D3Q19 ? ((a > 0) + (b > 0) + (c > 0)) <= 2 : true);
}

// per-direction power-of-two scale exponent of the FP16/BF16 delta storage,
// round(-log2 w_i)
LBM_HD constexpr int scale_exp(int st, int i) {
  int n2 = vel(st, i, 0) * vel(st, i, 0) + vel(st, i, 1) * vel(st, i, 1) +
           vel(st, i, 2) * vel(st, i, 2);
  if (st == D2Q9) return n2 == 0 ? 1 : (n2 == 1 ? 3 : 5);
  if (st == D3Q19) return n2 == 0 ? 2 : (n2 == 1 ? 4 : 5);
  return n2 == 0 ? 2 : (n2 == 1 ? 4 : (n2 == 2 ? 6 : 8));
}

// lattice weight w_i = f0_i (Sec. 2.4) by speed class |xi_i|^2
LBM_HD constexpr double weight(int st, int i) {
  int n2 = vel(st, i, 0) * vel(st, i, 0) + vel(st, i, 1) * vel(st, i, 1) +
           vel(st, i, 2) * vel(st, i, 2);
  if (st == D2Q9) return n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  if (st == D3Q19) return n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  return n2 == 0 ? 8.0 / 27.0 : (n2 == 1 ? 2.0 / 27.0 : (n2 == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
}

// rest-state background factor of one axis exponent: (1, 0, 1/3)
LBM_HD constexpr double bg1(int e) { return e == 0 ? 1.0 : (e == 1 ? 0.0 : 1.0 / 3.0); }
LBM_HD constexpr double bg3(int a, int b, int c) { return bg1(a) * bg1(b) * bg1(c); }

// "keep" factors (1 - omega_g): [0] shear, [1] bulk, [2..5] orders 3..6
template <class T>
struct Rates {
  T om[6];
};

// ------------------------------------------------------ raw Chimera (4.1)
// one 3-point pass: (f(-1), f(0), f(+1)) -> (m0, m1, m2)
template <class T>
LBM_D void fwd3(T& v0, T& v1, T& v2) {
  const T s = v2 + v0;
  const T d = v2 - v0;
  v0 = s + v1;
  v1 = d;
  v2 = s;
}
// inverse pass: (m0, m1, m2) -> (f(-1), f(0), f(+1)); the +/- split of
// Eq. 4.2: f(+-1) = (m2 +- m1) / 2
template <class T>
LBM_D void bwd3(T& v0, T& v1, T& v2) {
  const T h2 = T(0.5) * v2;
  const T h1 = T(0.5) * v1;
  const T f0 = v0 - v2;
  v0 = h2 - h1;
  v1 = f0;
  v2 = h2 + h1;
}

// zero-centered populations -> raw monomial moment deviations A[a][b][c]
template <int ST, class T>
LBM_D void fwd_raw_chimera(const T (&f)[q_of(ST)], T (&A)[3][3][3]) {
  sfor<27>([&](auto K) { A[CI(K) / 9][(CI(K) / 3) % 3][CI(K) % 3] = T(0); });
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int x = vel(ST, i, 0) + 1, y = vel(ST, i, 1) + 1;
    constexpr int z = dim_of(ST) == 3 ? vel(ST, i, 2) + 1 : 0;
    A[x][y][z] = f[i];
  });
  if constexpr (dim_of(ST) == 3) {
    sfor<9>([&](auto K) {
      constexpr int x = CI(K) / 3, y = CI(K) % 3;
      fwd3(A[x][y][0], A[x][y][1], A[x][y][2]);
    });
  }
  sfor<9>([&](auto K) {
    constexpr int x = CI(K) / 3, c = CI(K) % 3;
    if constexpr (dim_of(ST) == 3 || c == 0) fwd3(A[x][0][c], A[x][1][c], A[x][2][c]);
  });
  sfor<9>([&](auto K) {
    constexpr int b = CI(K) / 3, c = CI(K) % 3;
    if constexpr (dim_of(ST) == 3 || c == 0) fwd3(A[0][b][c], A[1][b][c], A[2][b][c]);
  });
}

// inverse pass without the 1/2: (m0, m1, m2) -> (2 f(-1), f(0), 2 f(+1))
template <class T>
LBM_D void bwd3_x2(T& v0, T& v1, T& v2) {
  const T f0 = v0 - v2;
  const T fm = v2 - v1;
  v2 = v2 + v1;
  v0 = fm;
  v1 = f0;
}

// raw monomial moment deviations -> zero-centered populations.  DEFER
// leaves out the exact power-of-two factors of the split: population i is
// then returned multiplied by 2^(|xi_i|^2), for callers that rescale anyway.
template <int ST, class T, bool DEFER = false>
LBM_D void bwd_raw(T (&A)[3][3][3], T (&f)[q_of(ST)]) {
  if constexpr (ST == D3Q19) {
    // D3Q19 is no tensor product: solve M f = m in closed form, plane by
    // plane, with the symmetric / antisymmetric split of Eq. 4.2
    const T q4 = T(DEFER ? 1.0 : 0.25);
    auto edge = [&](T m22, T m21, T m12, T m11, T& fpp, T& fpm, T& fmp, T& fmm) {
      T s, a2, a1, c;
      if constexpr (DEFER) {
        s = m22, a2 = m21, a1 = m12, c = m11;
      } else {
        s = q4 * m22, a2 = q4 * m21, a1 = q4 * m12, c = q4 * m11;
      }
      const T sp = s + a1, sm = s - a1;  // first axis +1 / -1
      fpp = sp + a2 + c;
      fpm = sp - a2 - c;
      fmp = sm + a2 - c;
      fmm = sm - a2 + c;
    };
    // xy edges: 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
    edge(A[2][2][0], A[2][1][0], A[1][2][0], A[1][1][0], f[7], f[9], f[10], f[8]);
    // xz edges: 11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1)
    edge(A[2][0][2], A[2][0][1], A[1][0][2], A[1][0][1], f[11], f[13], f[14], f[12]);
    // yz edges: 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
    edge(A[0][2][2], A[0][2][1], A[0][1][2], A[0][1][1], f[15], f[17], f[18], f[16]);
    const T h = T(0.5);
    (void)h;
    const T sx = A[2][0][0] - A[2][2][0] - A[2][0][2];
    const T ax = A[1][0][0] - A[1][2][0] - A[1][0][2];
    const T sy = A[0][2][0] - A[2][2][0] - A[0][2][2];
    const T ay = A[0][1][0] - A[2][1][0] - A[0][1][2];
    const T sz = A[0][0][2] - A[2][0][2] - A[0][2][2];
    const T az = A[0][0][1] - A[2][0][1] - A[0][2][1];
    if constexpr (DEFER) {
      f[1] = sx + ax;
      f[2] = sx - ax;
      f[3] = sy + ay;
      f[4] = sy - ay;
      f[5] = sz + az;
      f[6] = sz - az;
    } else {
      f[1] = h * (sx + ax);
      f[2] = h * (sx - ax);
      f[3] = h * (sy + ay);
      f[4] = h * (sy - ay);
      f[5] = h * (sz + az);
      f[6] = h * (sz - az);
    }
    f[0] = A[0][0][0] - (A[2][0][0] + A[0][2][0] + A[0][0][2]) +
           (A[2][2][0] + A[2][0][2] + A[0][2][2]);
  } else {
    auto pass = [](T& v0, T& v1, T& v2) {
      if constexpr (DEFER) bwd3_x2(v0, v1, v2);
      else bwd3(v0, v1, v2);
    };
    sfor<9>([&](auto K) {
      constexpr int b = CI(K) / 3, c = CI(K) % 3;
      if constexpr (dim_of(ST) == 3 || c == 0) pass(A[0][b][c], A[1][b][c], A[2][b][c]);
    });
    sfor<9>([&](auto K) {
      constexpr int x = CI(K) / 3, c = CI(K) % 3;
      if constexpr (dim_of(ST) == 3 || c == 0) pass(A[x][0][c], A[x][1][c], A[x][2][c]);
    });
    if constexpr (dim_of(ST) == 3) {
      sfor<9>([&](auto K) {
        constexpr int x = CI(K) / 3, y = CI(K) % 3;
        pass(A[x][y][0], A[x][y][1], A[x][y][2]);
      });
    }
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      constexpr int x = vel(ST, i, 0) + 1, y = vel(ST, i, 1) + 1;
      constexpr int z = dim_of(ST) == 3 ? vel(ST, i, 2) + 1 : 0;
      f[i] = A[x][y][z];
    });
  }
}

// ------------------------------------------- binomial Chimera (Eq. 4.3)
// One pass along an axis of the deviation quantities (v0, v1, v2) whose
// other indices carry the constant background B0.  Forward (SIGN = -1):
// k1 = m1 - u m0, k2 = m2 - 2u m1 + u^2 m0; backward (SIGN = +1) with +u.
// Only m0 carries a background (b1 = 0, and the b2 terms cancel).
template <int SIGN, class T, int B0NZ>
LBM_D void binom3(T& v0, T& v1, T& v2, T u, T u2, T B0) {
  T full0 = v0;
  if constexpr (B0NZ) full0 = B0 + v0;
  const T su = SIGN > 0 ? u : -u;
  const T t2 = v2 + T(2) * su * v1 + u2 * full0;
  v1 = v1 + su * full0;
  v2 = t2;
}

template <int ST, int SIGN, class T>
LBM_D void binomial(T (&A)[3][3][3], const T (&u)[3], const T (&u2)[3]) {
  if constexpr (dim_of(ST) == 3) {
    sfor<9>([&](auto K) {  // along z
      constexpr int a = CI(K) / 3, b = CI(K) % 3;
      constexpr double B0 = bg3(a, b, 0);
      binom3<SIGN, T, (B0 != 0.0)>(A[a][b][0], A[a][b][1], A[a][b][2], u[2], u2[2], T(B0));
    });
  }
  sfor<9>([&](auto K) {  // along y
    constexpr int a = CI(K) / 3, c = CI(K) % 3;
    constexpr double B0 = bg3(a, 0, c);
    if constexpr (dim_of(ST) == 3 || c == 0)
      binom3<SIGN, T, (B0 != 0.0)>(A[a][0][c], A[a][1][c], A[a][2][c], u[1], u2[1], T(B0));
  });
  sfor<9>([&](auto K) {  // along x
    constexpr int b = CI(K) / 3, c = CI(K) % 3;
    constexpr double B0 = bg3(0, b, c);
    if constexpr (dim_of(ST) == 3 || c == 0)
      binom3<SIGN, T, (B0 != 0.0)>(A[0][b][c], A[1][b][c], A[2][b][c], u[0], u2[0], T(B0));
  });
}

template <class T>
LBM_D T rcp(T x) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, float>::value) return __frcp_rn(x);
#endif
  return T(1) / x;
}

// ------------------------------------------------ relaxation, raw moments
// Deviation of the raw equilibrium moment (Maxwellian truncated at O(u^2),
// Sec. 4.2): dm_eq = drho * b(e) + rho * [terms of degree 1 and 2 in u].
// Per axis the factor of exponent 0 is 1, of 1 is u, of 2 is 1/3 + u^2.
template <class T>
LBM_D T raw_eq_dev(int a, int b, int c, T drho, T rho, const T (&u)[3]) {
  const int e[3] = {a, b, c};
  int n1 = 0, n2 = 0, d1[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    if (e[d] == 1) d1[n1++] = d;
    if (e[d] == 2) ++n2;
  }
  const T third = T(1.0 / 3.0);
  T pw = T(1);
  for (int k = 0; k < n2; ++k) pw *= third;  // (1/3)^n2
  if (n1 == 0) {
    if (n2 == 0) return drho;  // order 0
    T s = T(0);
    for (int d = 0; d < 3; ++d)
      if (e[d] == 2) s += u[d] * u[d];
    T pw1 = T(1);
    for (int k = 0; k < n2 - 1; ++k) pw1 *= third;
    return drho * T(bg3(a, b, c)) + rho * pw1 * s;
  }
  if (n1 == 1) return rho * pw * u[d1[0]];
  if (n1 == 2) return rho * pw * u[d1[0]] * u[d1[1]];
  return T(0);
}

// Orthogonal-basis transform of non-equilibrium raw moments (O-MRT).
// D2Q9 / D3Q27: per axis x^2 -> x^2 - 2/3 (tensor products of the 1-D
// orthogonal polynomials 1, x, x^2 - 2/3).  D3Q19: once the conserved
// parts are zero only the fourth-order polynomials differ from monomials:
// x^2y^2 - (10/21)(x^2 + y^2) + (4/21) z^2 + 4/21.  SIGN = -1 forward.
// W: the weighted orthogonal basis of WO-MRT (inner product with the lattice
// weights): D2Q9 / D3Q27 tensor products of 1, x, x^2 - 1/3; D3Q19
// x^2 y^2 - (x^2 + y^2)/3 + z^2/6 (the unweighted basis: x^2 - 2/3 and
// x^2 y^2 - 10/21 (x^2 + y^2) + 4/21 z^2).  Lower-order and same-group
// terms of the full Gram-Schmidt rows do not change the relaxation and are
// left out.
template <int ST, int SIGN, class T, bool W = false>
LBM_D void ortho_raw(T (&N)[3][3][3]) {
  if constexpr (ST == D3Q19) {
    const T c10 = T(W ? 1.0 / 3.0 : 10.0 / 21.0), c4 = T(W ? 1.0 / 6.0 : 4.0 / 21.0);
    const T s = T(SIGN);
    N[2][2][0] += s * (c10 * (N[2][0][0] + N[0][2][0]) - c4 * N[0][0][2]);
    N[2][0][2] += s * (c10 * (N[2][0][0] + N[0][0][2]) - c4 * N[0][2][0]);
    N[0][2][2] += s * (c10 * (N[0][2][0] + N[0][0][2]) - c4 * N[2][0][0]);
  } else {
    const T t = T(-SIGN) * T(W ? -1.0 / 3.0 : -2.0 / 3.0);
    if constexpr (dim_of(ST) == 3) {
      sfor<9>([&](auto K) { N[CI(K) / 3][CI(K) % 3][2] += t * N[CI(K) / 3][CI(K) % 3][0]; });
    }
    sfor<9>([&](auto K) {
      constexpr int a = CI(K) / 3, c = CI(K) % 3;
      if constexpr (dim_of(ST) == 3 || c == 0) N[a][2][c] += t * N[a][0][c];
    });
    sfor<9>([&](auto K) {
      constexpr int b = CI(K) / 3, c = CI(K) % 3;
      if constexpr (dim_of(ST) == 3 || c == 0) N[2][b][c] += t * N[0][b][c];
    });
  }
}

// Relax the second-order block of deviation quantities X: trace with the
// bulk factor, traceless part and off-diagonals with the shear factor.
// REG: bulk rate fixed at 1 (factor 0).
template <int ST, class T, bool REG>
LBM_D void relax_order2(T (&X)[3][3][3], T ks, T kb) {
  if constexpr (dim_of(ST) == 3) {
    const T m3 = (X[2][0][0] + X[0][2][0] + X[0][0][2]) * T(1.0 / 3.0);
    T mt;
    if constexpr (REG) mt = T(0);
    else mt = kb * m3;
    X[2][0][0] = mt + ks * (X[2][0][0] - m3);
    X[0][2][0] = mt + ks * (X[0][2][0] - m3);
    X[0][0][2] = mt + ks * (X[0][0][2] - m3);
    X[1][1][0] *= ks;
    X[1][0][1] *= ks;
    X[0][1][1] *= ks;
  } else {
    const T m2 = T(0.5) * (X[2][0][0] + X[0][2][0]);
    T mt;
    if constexpr (REG) mt = T(0);
    else mt = kb * m2;
    X[2][0][0] = mt + ks * (X[2][0][0] - m2);
    X[0][2][0] = mt + ks * (X[0][2][0] - m2);
    X[1][1][0] *= ks;
  }
}

// ------------------------------------------------ cumulants (Eq. 4.5)
// K: normalised central-moment deviations dk = kappa/rho - k0 (k0 the
// rest-state Gaussian moments: 1/3, 1/9, 1/27 on the even diagonals).
// Writes cumulant deviations dc = c - c0 (c0: 1/3 on the second-order
// diagonal, 0 elsewhere) of orders 4-6 into C; orders 2-3 are identical.
// Each order-n formula is the sum over the set partitions of the index
// multiset into blocks of size >= 2 (central moments have no first order).
// ABS: K holds absolute normalised central moments and C receives absolute
// cumulants (the same relations with the background constant A = 0).
template <int ST, class T, bool ABS = false>
LBM_D void cumulant_fwd(const T (&K)[3][3][3], T (&C)[3][3][3]) {
  const T A = T(ABS ? 0.0 : 1.0 / 3.0);
  const T a = K[2][0][0], b = K[0][2][0], c = K[0][0][2];
  const T k110 = K[1][1][0], k101 = K[1][0][1], k011 = K[0][1][1];
  C[2][2][0] = K[2][2][0] - A * (a + b) - a * b - T(2) * k110 * k110;
  if constexpr (dim_of(ST) == 3) {
    C[2][0][2] = K[2][0][2] - A * (a + c) - a * c - T(2) * k101 * k101;
    C[0][2][2] = K[0][2][2] - A * (b + c) - b * c - T(2) * k011 * k011;
  }
  if constexpr (ST == D3Q27) {
    const T k111 = K[1][1][1];
    C[2][1][1] = K[2][1][1] - (A + a) * k011 - T(2) * k110 * k101;
    C[1][2][1] = K[1][2][1] - (A + b) * k101 - T(2) * k110 * k011;
    C[1][1][2] = K[1][1][2] - (A + c) * k110 - T(2) * k101 * k011;
    C[2][2][1] = K[2][2][1] - (A + a) * K[0][2][1] - (A + b) * K[2][0][1] -
                 T(4) * k110 * k111 - T(2) * k101 * K[1][2][0] - T(2) * k011 * K[2][1][0];
    C[2][1][2] = K[2][1][2] - (A + a) * K[0][1][2] - (A + c) * K[2][1][0] -
                 T(4) * k101 * k111 - T(2) * k110 * K[1][0][2] - T(2) * k011 * K[2][0][1];
    C[1][2][2] = K[1][2][2] - (A + b) * K[1][0][2] - (A + c) * K[1][2][0] -
                 T(4) * k011 * k111 - T(2) * k110 * K[0][1][2] - T(2) * k101 * K[0][2][1];
    const T d4 = K[0][2][2] + K[2][0][2] + K[2][2][0];
    C[2][2][2] = K[2][2][2] - A * d4 + A * A * (a + b + c) -
                 (a * K[0][2][2] + b * K[2][0][2] + c * K[2][2][0]) +
                 T(2) * A * (a * b + b * c + c * a) + T(2) * a * b * c -
                 T(4) * (k110 * K[1][1][2] + k101 * K[1][2][1] + k011 * K[2][1][1]) -
                 T(2) * (K[2][1][0] * K[0][1][2] + K[2][0][1] * K[0][2][1] +
                         K[1][2][0] * K[1][0][2]) -
                 T(4) * k111 * k111 +
                 T(4) * ((A + a) * k011 * k011 + (A + b) * k101 * k101 + (A + c) * k110 * k110) +
                 T(16) * k110 * k101 * k011;
  }
}

// Inverse of cumulant_fwd for post-collision values.  C holds the relaxed
// cumulant deviations of orders 2..6; writes normalised central-moment
// deviations of orders 4..6 into K.  REG: every cumulant of order >= 3 is
// zero (rates 1), so only Gaussian products of second-order cumulants stay.
template <int ST, class T, bool REG, bool ABS = false>
LBM_D void cumulant_bwd(const T (&C)[3][3][3], T (&K)[3][3][3]) {
  const T A = T(ABS ? 0.0 : 1.0 / 3.0);
  const T a = C[2][0][0], b = C[0][2][0], c = C[0][0][2];
  const T c110 = C[1][1][0], c101 = C[1][0][1], c011 = C[0][1][1];
  const T g220 = A * (a + b) + a * b + T(2) * c110 * c110;
  if constexpr (REG) K[2][2][0] = g220;
  else K[2][2][0] = C[2][2][0] + g220;
  if constexpr (dim_of(ST) == 3) {
    const T g202 = A * (a + c) + a * c + T(2) * c101 * c101;
    const T g022 = A * (b + c) + b * c + T(2) * c011 * c011;
    if constexpr (REG) {
      K[2][0][2] = g202;
      K[0][2][2] = g022;
    } else {
      K[2][0][2] = C[2][0][2] + g202;
      K[0][2][2] = C[0][2][2] + g022;
    }
  }
  if constexpr (ST == D3Q27) {
    const T g211 = (A + a) * c011 + T(2) * c110 * c101;
    const T g121 = (A + b) * c101 + T(2) * c110 * c011;
    const T g112 = (A + c) * c110 + T(2) * c101 * c011;
    const T g222 = A * A * (a + b + c) + A * (a * b + b * c + c * a) + a * b * c +
                   T(2) * ((A + a) * c011 * c011 + (A + b) * c101 * c101 +
                           (A + c) * c110 * c110) +
                   T(8) * c110 * c101 * c011;
    if constexpr (REG) {
      K[2][1][1] = g211;
      K[1][2][1] = g121;
      K[1][1][2] = g112;
      K[2][2][1] = T(0);
      K[2][1][2] = T(0);
      K[1][2][2] = T(0);
      K[2][2][2] = g222;
    } else {
      const T c111 = C[1][1][1];
      K[2][1][1] = C[2][1][1] + g211;
      K[1][2][1] = C[1][2][1] + g121;
      K[1][1][2] = C[1][1][2] + g112;
      K[2][2][1] = C[2][2][1] + (A + a) * C[0][2][1] + (A + b) * C[2][0][1] +
                   T(4) * c110 * c111 + T(2) * c101 * C[1][2][0] + T(2) * c011 * C[2][1][0];
      K[2][1][2] = C[2][1][2] + (A + a) * C[0][1][2] + (A + c) * C[2][1][0] +
                   T(4) * c101 * c111 + T(2) * c110 * C[1][0][2] + T(2) * c011 * C[2][0][1];
      K[1][2][2] = C[1][2][2] + (A + b) * C[1][0][2] + (A + c) * C[1][2][0] +
                   T(4) * c011 * c111 + T(2) * c110 * C[0][1][2] + T(2) * c101 * C[0][2][1];
      K[2][2][2] = C[2][2][2] + A * (C[0][2][2] + C[2][0][2] + C[2][2][0]) +
                   a * C[0][2][2] + b * C[2][0][2] + c * C[2][2][0] +
                   T(4) * (c110 * C[1][1][2] + c101 * C[1][2][1] + c011 * C[2][1][1]) +
                   T(2) * (C[2][1][0] * C[0][1][2] + C[2][0][1] * C[0][2][1] +
                           C[1][2][0] * C[1][0][2]) +
                   T(4) * c111 * c111 + g222;
    }
  }
}

template <int ST, class T, int SPACE>
LBM_D void equilibrium(T drho, const T (&u)[3], T (&f)[q_of(ST)]);

// ---------------------------------- discrete second-order equilibrium
// An equilibrium prescribed as populations (Sec. 2.4): f_eq_i = w_i rho
// (1 + P_i), P_i = 3 xi.u + 9/2 (xi.u)^2 - 3/2 u.u; its collision-space
// quantities are q_eq = T(f_eq).  As deviations: df_eq_i = w_i (drho +
// rho P_i).
template <int ST, int i, class T>
LBM_D T disc_poly(const T (&u)[3], T uu) {
  T xu = T(0);
  if constexpr (vel(ST, i, 0) != 0) xu += T(vel(ST, i, 0)) * u[0];
  if constexpr (vel(ST, i, 1) != 0) xu += T(vel(ST, i, 1)) * u[1];
  if constexpr (vel(ST, i, 2) != 0) xu += T(vel(ST, i, 2)) * u[2];
  return T(3) * xu + T(4.5) * (xu * xu) - T(1.5) * uu;
}
template <int ST, class T>
LBM_D void disc_feq(T drho, T rho, const T (&u)[3], T (&f)[q_of(ST)]) {
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    f[i] = T(weight(ST, i)) * (drho + rho * disc_poly<ST, i, T>(u, uu));
  });
}
// Raw moments of f_eq differ from the truncated Maxwellian's only on D3Q19,
// in the fourth-order x^2 y^2-type moments: by -rho u_k^2 / 6, k the third
// axis (D2Q9 and D3Q27 have product weights, for which they agree).
template <int ST, class T>
LBM_D T disc_raw_corr(int a, int b, int c, T rho, const T (&u)[3]) {
  if (ST != D3Q19 || a + b + c != 4 || a == 1 || b == 1 || c == 1) return T(0);
  const int k = a == 0 ? 0 : (b == 0 ? 1 : 2);
  return -rho * u[k] * u[k] * T(1.0 / 6.0);
}
// Normalised central-moment deviations of f_eq (they depend on u only:
// f_eq / rho = w (1 + P)): the same Chimera passes as for f, applied to
// w_i P_i, whose sum is zero.
template <int ST, class T>
LBM_D void disc_central_eq(const T (&u)[3], const T (&u2)[3], T (&E)[3][3][3]) {
  T g[q_of(ST)];
  const T uu = u2[0] + u2[1] + u2[2];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    g[i] = T(weight(ST, i)) * disc_poly<ST, i, T>(u, uu);
  });
  fwd_raw_chimera<ST, T>(g, E);
  E[0][0][0] = T(0);
  binomial<ST, -1, T>(E, u, u2);
}

// ------------------------------------------------------------ collision
// In: zero-centered pre-collision populations f.  Out: zero-centered
// post-collision populations f*.  keep.om[g] = 1 - omega_g.
// DISC: relax toward the discrete second-order equilibrium (q_eq = T(f_eq))
// instead of the Maxwellian's moments (general instance for central moments
// and cumulants, whose equilibria of order >= 3 are then nonzero).
// population-space collisions under DEFER: scale population i by
// 2^(|xi_i|^2) as the deferred backward transform would have left it
template <int ST, class T>
LBM_D void defer_scale(T (&f)[q_of(ST)]) {
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                      vel(ST, i, 2) * vel(ST, i, 2);
    if constexpr (k > 0) f[i] = f[i] * T(float(1 << k));
  });
}

// Guo's population source of a body force F at velocity u (c_s^2 = 1/3):
// S_i = w_i [3 (xi_i.F - u.F) + 9 (xi_i.u)(xi_i.F)]
template <int ST, class T>
LBM_D void guo_source(const T (&u)[3], const T (&F)[3], T (&S)[q_of(ST)]) {
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
    T cu = T(0), cf = T(0);
    if constexpr (cx != 0) cu += T(cx) * u[0], cf += T(cx) * F[0];
    if constexpr (cy != 0) cu += T(cy) * u[1], cf += T(cy) * F[1];
    if constexpr (cz != 0) cu += T(cz) * u[2], cf += T(cz) * F[2];
    S[i] = T(weight(ST, i)) * (T(3) * (cf - uF) + T(9) * cu * cf);
  });
}

// He's population source: S_i = 3 (xi_i - u).F / rho * f_eq_i with the
// method's absolute equilibrium populations f_eq (truncated raw moments for
// SRT / TRT / raw spaces, the full Maxwellian for central moments).
template <int ST, class T, int SPACE>
LBM_D void he_source(T drho, T inv, const T (&u)[3], const T (&F)[3], T (&S)[q_of(ST)]) {
  T feq[q_of(ST)];
  equilibrium<ST, T, (SPACE == SP_CENTRAL ? SP_CENTRAL : SP_RAW)>(drho, u, feq);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
    const T cf = (T(cx) - u[0]) * F[0] + (T(cy) - u[1]) * F[1] + (T(cz) - u[2]) * F[2];
    S[i] = T(3) * cf * inv * (feq[i] + T(weight(ST, i)));
  });
}

// FORCED: a body force F per cell (source term of Eq. 2.1a, q^F of Eq. 2.4;
// Guo's model, or He's with HE: the same velocity shift and (I - S/2)
// weighting with he_source for S, in central space q^F = (I - S/2) K(u) S).  The equilibrium velocity is u = (j + F/2) / rho and
//   SRT: f* = f + w (f_eq - f) + (1 - w/2) S
//   raw: q^F = (I - S/2) P M S in the orthogonal basis (general path only)
//   central: moments about u, first-order central moments leave as +F/2
//   cumulant: cumulants relax about the mean j / rho; the mean leaves as
//             (j + F) / rho (cumulants of order >= 2 are shift invariant).
template <int ST, class T, int SPACE, bool REG, bool DEFER = false, bool FORCED = false,
          bool HE = false, bool DISC = false>
LBM_D void collide(T (&f)[q_of(ST)], const Rates<T>& keep, const T* F = nullptr) {
  static_assert(!(HE && SPACE == SP_CUMULANT), "He's model is not defined for cumulants");
  static_assert(!(DISC && (FORCED || (REG && (SPACE == SP_CENTRAL || SPACE == SP_CUMULANT)))),
                "the discrete equilibrium runs unforced; central / cumulant: general path");
  static_assert(!(FORCED && REG && (SPACE == SP_RAW || SPACE == SP_RAW_W)),
                "forced raw moments use the general path");
  constexpr bool WO = SPACE == SP_RAW_W;
  T A[3][3][3];
  fwd_raw_chimera<ST, T>(f, A);
  const T drho = A[0][0][0];
  const T rho = T(1) + drho;
  const T inv = rcp(rho);
  const T j[3] = {A[1][0][0], A[0][1][0], dim_of(ST) == 3 ? A[0][0][1] : T(0)};
  T Fv[3] = {T(0), T(0), T(0)};
  if constexpr (FORCED) {
    Fv[0] = F[0];
    Fv[1] = F[1];
    if constexpr (dim_of(ST) == 3) Fv[2] = F[2];
  }
  constexpr bool SHIFT = FORCED && SPACE != SP_CUMULANT;
  const T u[3] = {SHIFT ? (j[0] + T(0.5) * Fv[0]) * inv : j[0] * inv,
                  SHIFT ? (j[1] + T(0.5) * Fv[1]) * inv : j[1] * inv,
                  SHIFT ? (j[2] + T(0.5) * Fv[2]) * inv : j[2] * inv};
  const T u2[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};
  auto force_source = [&](T (&S)[q_of(ST)]) {
    if constexpr (HE) he_source<ST, T, SPACE>(drho, inv, u, Fv, S);
    else guo_source<ST, T>(u, Fv, S);
  };

  // population-space equilibrium f_eq = M^-1 m_eq.  On D3Q27 (product
  // weights) the truncated Maxwellian's raw moments are those of the
  // second-order polynomial, so f_eq is that polynomial, evaluated in closed
  // form; on D2Q9 / D3Q19 the backward transform of m_eq measured faster in
  // the packed FP16 kernel (D3Q27 SRT 47.6 -> 51.6 GLUPS, D2Q9 163.7 ->
  // 154.0, D3Q19 75.1 -> 66.3 with the closed form)
  constexpr bool POLY = DISC || ST == D3Q27;
  if constexpr (SPACE == SP_SRT) {
    // single relaxation time in population space against f_eq
    T feq[q_of(ST)];
    if constexpr (POLY) disc_feq<ST, T>(drho, rho, u, feq);
    else equilibrium<ST, T, SP_RAW>(drho, u, feq);
    if constexpr (FORCED) {
      T S[q_of(ST)];
      force_source(S);
      const T half = T(0.5) * (T(1) + keep.om[0]);  // 1 - w/2
      sfor<q_of(ST)>([&](auto I) {
        constexpr int i = CI(I);
        f[i] = feq[i] + keep.om[0] * (f[i] - feq[i]) + half * S[i];
      });
    } else {
      sfor<q_of(ST)>([&](auto I) {
        constexpr int i = CI(I);
        f[i] = feq[i] + keep.om[0] * (f[i] - feq[i]);
      });
    }
    if constexpr (DEFER) defer_scale<ST, T>(f);
    return;
  } else if constexpr (SPACE == SP_TRT) {
    // two relaxation times: per opposite pair the even part relaxes with
    // keep.om[0] = 1 - w+, the odd part with keep.om[2] = 1 - w-
    T feq[q_of(ST)], S[q_of(ST)];
    if constexpr (POLY) disc_feq<ST, T>(drho, rho, u, feq);
    else equilibrium<ST, T, SP_RAW>(drho, u, feq);
    if constexpr (FORCED) force_source(S);
    const T kp = keep.om[0], km = keep.om[2];
    const T hp = T(0.5) * kp, hm = T(0.5) * km;
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      constexpr int b = opp(i);
      if constexpr (i == b) {
        f[i] = feq[i] + kp * (f[i] - feq[i]);
        if constexpr (FORCED) f[i] += T(0.5) * (T(1) + kp) * S[i];
      } else if constexpr (i < b) {
        // with d = f - f_eq: f*_i = f_eq_i + (1 - w+)(d_i + d_b)/2 +
        // (1 - w-)(d_i - d_b)/2, f*_b the same with the odd part negated
        const T di = f[i] - feq[i], db = f[b] - feq[b];
        const T a = hp * (di + db), c = hm * (di - db);
        T fi = feq[i] + (a + c), fb = feq[b] + (a - c);
        if constexpr (FORCED) {
          const T sp = T(0.25) * (T(1) + kp) * (S[i] + S[b]);
          const T sm = T(0.25) * (T(1) + km) * (S[i] - S[b]);
          fi += sp + sm;
          fb += sp - sm;
        }
        f[i] = fi;
        f[b] = fb;
      }
    });
    if constexpr (DEFER) defer_scale<ST, T>(f);
    return;
  } else if constexpr (SPACE == SP_RAW || SPACE == SP_RAW_W) {
    // non-equilibrium parts in the orthogonal basis, relax, transform back
    T E[3][3][3], N[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      if constexpr (has_mono(ST, a, b, c)) {
        E[a][b][c] = raw_eq_dev<T>(a, b, c, drho, rho, u);
        if constexpr (DISC && ST == D3Q19 && a + b + c == 4)
          E[a][b][c] += disc_raw_corr<ST, T>(a, b, c, rho, u);
        // forced: the first-order non-equilibrium part is -F/2
        if constexpr (o == 0 || (o == 1 && !FORCED) || (REG && o != 2)) N[a][b][c] = T(0);
        else N[a][b][c] = A[a][b][c] - E[a][b][c];
      } else {
        E[a][b][c] = T(0);
        N[a][b][c] = T(0);
      }
    });
    if constexpr (!REG) ortho_raw<ST, -1, T, WO>(N);
    relax_order2<ST, T, REG>(N, keep.om[0], keep.om[1]);
    if constexpr (!REG) {
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        if constexpr (has_mono(ST, a, b, c) && o >= 3) N[a][b][c] *= keep.om[o - 1];
      });
    }
    if constexpr (FORCED) {
      // q^F = (I - S/2) P M S: the source's raw moments in the orthogonal
      // basis, each rate group scaled by 1 - w/2 (conserved rows by 1)
      T S[q_of(ST)], G[3][3][3];
      force_source(S);
      fwd_raw_chimera<ST, T>(S, G);
      G[0][0][0] = T(0);
      ortho_raw<ST, -1, T, WO>(G);
      relax_order2<ST, T, false>(G, T(0.5) * (T(1) + keep.om[0]), T(0.5) * (T(1) + keep.om[1]));
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        if constexpr (has_mono(ST, a, b, c) && o >= 1) {
          if constexpr (o >= 3) N[a][b][c] += T(0.5) * (T(1) + keep.om[o - 1]) * G[a][b][c];
          else N[a][b][c] += G[a][b][c];
        }
      });
    }
    ortho_raw<ST, +1, T, WO>(N);
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) A[a][b][c] = E[a][b][c] + N[a][b][c];
    });
  } else {
    // central moments (binomial Chimera with -u) as deviations
    binomial<ST, -1, T>(A, u, u2);
    // normalised deviations dk = (dkappa - drho * k0) / rho
    T Kn[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr double B = bg3(a, b, c);
      if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) {
        if constexpr (B != 0.0) Kn[a][b][c] = (A[a][b][c] - drho * T(B)) * inv;
        else Kn[a][b][c] = A[a][b][c] * inv;
      } else {
        Kn[a][b][c] = T(0);
      }
    });
    // DISC: the equilibrium's normalised deviations Eq; the Maxwellian's are 0
    T Eq[3][3][3];
    if constexpr (DISC) disc_central_eq<ST, T>(u, u2, Eq);
    auto shift_eq = [&](T (&X)[3][3][3], T sign) {
      if constexpr (DISC) {
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) X[a][b][c] += sign * Eq[a][b][c];
        });
      }
    };
    if constexpr (SPACE == SP_CENTRAL) {
      // dk* = dk_eq + (1 - w) (dk - dk_eq), dk_eq = 0 for the Maxwellian
      shift_eq(Kn, T(-1));
      relax_order2<ST, T, REG>(Kn, keep.om[0], keep.om[1]);
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        if constexpr (has_mono(ST, a, b, c) && o >= 3) {
          if constexpr (REG) Kn[a][b][c] = T(0);
          else Kn[a][b][c] *= keep.om[o - 1];
        }
      });
      shift_eq(Kn, T(1));
      if constexpr (FORCED && HE) {
        // q^F = (I - S/2) K(u) S: central moments of He's source about u,
        // scaled per rate group, added to the normalised deviations
        T S[q_of(ST)], G[3][3][3];
        force_source(S);
        fwd_raw_chimera<ST, T>(S, G);
        if constexpr (dim_of(ST) == 3) {
          sfor<9>([&](auto K) {
            binom3<-1, T, 0>(G[CI(K) / 3][CI(K) % 3][0], G[CI(K) / 3][CI(K) % 3][1],
                             G[CI(K) / 3][CI(K) % 3][2], u[2], u2[2], T(0));
          });
        }
        sfor<9>([&](auto K) {
          constexpr int a = CI(K) / 3, c = CI(K) % 3;
          if constexpr (dim_of(ST) == 3 || c == 0)
            binom3<-1, T, 0>(G[a][0][c], G[a][1][c], G[a][2][c], u[1], u2[1], T(0));
        });
        sfor<9>([&](auto K) {
          constexpr int b = CI(K) / 3, c = CI(K) % 3;
          if constexpr (dim_of(ST) == 3 || c == 0)
            binom3<-1, T, 0>(G[0][b][c], G[1][b][c], G[2][b][c], u[0], u2[0], T(0));
        });
        relax_order2<ST, T, false>(G, T(0.5) * (T(1) + keep.om[0]), T(0.5) * (T(1) + keep.om[1]));
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          constexpr int o = a + b + c;
          if constexpr (has_mono(ST, a, b, c) && o >= 2) {
            if constexpr (o >= 3) Kn[a][b][c] += T(0.5) * (T(1) + keep.om[o - 1]) * G[a][b][c] * inv;
            else Kn[a][b][c] += G[a][b][c] * inv;
          }
        });
      }
    } else {  // cumulants; equilibrium deviations are all 0 as well
      T Cm[3][3][3];
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        Cm[a][b][c] = Kn[a][b][c];
      });
      if constexpr (!REG) cumulant_fwd<ST, T>(Kn, Cm);
      // DISC: relax about the cumulants of f_eq (those of its normalised
      // central moments Eq)
      T Ceq[3][3][3];
      if constexpr (DISC) {
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          Ceq[a][b][c] = Eq[a][b][c];
        });
        cumulant_fwd<ST, T>(Eq, Ceq);
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) Cm[a][b][c] -= Ceq[a][b][c];
        });
      }
      relax_order2<ST, T, REG>(Cm, keep.om[0], keep.om[1]);
      if constexpr (!REG) {
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          constexpr int o = a + b + c;
          if constexpr (has_mono(ST, a, b, c) && o >= 3) Cm[a][b][c] *= keep.om[o - 1];
        });
      }
      if constexpr (DISC) {
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) Cm[a][b][c] += Ceq[a][b][c];
        });
      }
      // orders 2 and 3: central = cumulant; 4..6 from the inverse relations
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        if constexpr (o == 2) Kn[a][b][c] = Cm[a][b][c];
        if constexpr (o == 3) Kn[a][b][c] = REG ? T(0) : Cm[a][b][c];
      });
      cumulant_bwd<ST, T, REG>(Cm, Kn);
    }
    // back to unnormalised deviations: dkappa* = drho k0 + rho dk*
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      constexpr double B = bg3(a, b, c);
      if constexpr (o == 0) {
        A[a][b][c] = drho;
      } else if constexpr (o == 1) {
        // central moments about u leave as F/2; cumulants rebuild about the
        // advanced mean, where the first-order central moments are 0
        if constexpr (FORCED && SPACE == SP_CENTRAL)
          A[a][b][c] = T(0.5) * Fv[a == 1 ? 0 : (b == 1 ? 1 : 2)];
        else
          A[a][b][c] = T(0);
      } else if constexpr (has_mono(ST, a, b, c)) {
        if constexpr (B != 0.0) A[a][b][c] = drho * T(B) + rho * Kn[a][b][c];
        else A[a][b][c] = rho * Kn[a][b][c];
      } else {
        A[a][b][c] = T(0);
      }
    });
    if constexpr (FORCED && SPACE == SP_CUMULANT) {
      const T v[3] = {(j[0] + Fv[0]) * inv, (j[1] + Fv[1]) * inv, (j[2] + Fv[2]) * inv};
      const T v2[3] = {v[0] * v[0], v[1] * v[1], v[2] * v[2]};
      binomial<ST, +1, T>(A, v, v2);
    } else {
      binomial<ST, +1, T>(A, u, u2);
    }
  }
  // conserved moments pass through exactly (plus the force's momentum)
  A[0][0][0] = drho;
  if constexpr (FORCED) {
    A[1][0][0] = j[0] + Fv[0];
    A[0][1][0] = j[1] + Fv[1];
    if constexpr (dim_of(ST) == 3) A[0][0][1] = j[2] + Fv[2];
  } else {
    A[1][0][0] = j[0];
    A[0][1][0] = j[1];
    if constexpr (dim_of(ST) == 3) A[0][0][1] = j[2];
  }
  bwd_raw<ST, T, DEFER>(A, f);
}

// The method's equilibrium as zero-centered populations (the collision's
// fixed point): raw methods use the truncated Maxwellian moments, central
// and cumulant methods the full Maxwellian (velocity-free central moments).
template <int ST, class T, int SPACE>
LBM_D void equilibrium(T drho, const T (&u)[3], T (&f)[q_of(ST)]) {
  T A[3][3][3];
  const T rho = T(1) + drho;
  if constexpr (SPACE == SP_RAW) {
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c)) A[a][b][c] = raw_eq_dev<T>(a, b, c, drho, rho, u);
      else A[a][b][c] = T(0);
    });
  } else {
    const T u2[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr double B = bg3(a, b, c);
      if constexpr ((a + b + c) != 1 && has_mono(ST, a, b, c) && B != 0.0)
        A[a][b][c] = drho * T(B);
      else
        A[a][b][c] = T(0);
    });
    binomial<ST, +1, T>(A, u, u2);
  }
  bwd_raw<ST, T>(A, f);
}

// ----------------------------------------- collision in absolute arithmetic
// The paper's Eq. 2.4 in absolute arithmetic: every moment, central moment
// and cumulant is carried with its background, q* = q_eq + (1 - omega)(q -
// q_eq).  For round-off studies; FP64.
//   ZC = false: in / out absolute populations f (absolute storage).
//   ZC = true : Eq. 2.6 on zero-centered storage, in / out df.  T(df + f0)
//     is evaluated as the nonlinear part of T applied to M df + M f0, with
//     the background raw moments M f0 = (1, 0, 1/3, ...) added as constants
//     (M is linear), and T^-1(q*) - f0 as M^-1 (raw moments of q* - M f0);
//     the conserved moments keep their deviation values.  Population-space
//     SRT (T = identity) adds and subtracts f0 = w itself.
// Absolute equilibrium populations of the shallow-water methods (D2Q9,
// Sec. 5.2): CENTRAL -> Zhou's discrete equilibrium
// f0 = h (1 - 5gh/6 - 2u.u/3), f_i = l_i h (gh/6 + xi.u/3 + (xi.u)^2/2 -
// u.u/6) with l_i = 1 on the axes and 1/4 on the diagonals; CUMULANT -> the
// continuous Maxwellian of c_s^2 = g h / 2 (per axis E[1] = 1, E[x] = u,
// E[x^2] = u^2 + c_s^2).
template <int ST, class T, int SPACE>
LBM_D void swe_feq(T h, const T (&u)[3], T g, T (&f)[q_of(ST)]) {
  static_assert(ST == D2Q9, "shallow water is two-dimensional");
  if constexpr (SPACE == SP_CENTRAL) {
    const T uu = u[0] * u[0] + u[1] * u[1];
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1);
      constexpr int sabs = (cx < 0 ? -cx : cx) + (cy < 0 ? -cy : cy);
      const T cu = T(cx) * u[0] + T(cy) * u[1];
      if constexpr (sabs == 0)
        f[i] = h * (T(1) - T(5.0 / 6.0) * g * h - T(2.0 / 3.0) * uu);
      else
        f[i] = T(sabs == 1 ? 1.0 : 0.25) * h *
               (g * h * T(1.0 / 6.0) + cu * T(1.0 / 3.0) + T(0.5) * cu * cu - uu * T(1.0 / 6.0));
    });
  } else {
    const T c2 = T(0.5) * g * h;
    const T e[3][2] = {{T(1), T(1)}, {u[0], u[1]}, {u[0] * u[0] + c2, u[1] * u[1] + c2}};
    T A[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      A[a][b][c] = c == 0 ? h * e[a][0] * e[b][1] : T(0);
    });
    bwd_raw<ST, T>(A, f);
  }
}

template <int ST, class T, int SPACE, bool REG, bool ZC = false, bool SWE = false>
LBM_D void collide_abs(T (&f)[q_of(ST)], const Rates<T>& keep, T swe_g = T(0)) {
  if constexpr (ZC && SPACE == SP_SRT) {
    sfor<q_of(ST)>([&](auto I) { f[CI(I)] += T(weight(ST, CI(I))); });
  }
  T A[3][3][3];
  fwd_raw_chimera<ST, T>(f, A);
  T drho0 = T(0);  // ZC: the deviation density, kept through the collision
  if constexpr (ZC && SPACE != SP_SRT) {
    drho0 = A[0][0][0];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c) && a + b + c != 1)
        A[a][b][c] += T(a + b + c == 0 ? 1.0 : bg3(a, b, c));
    });
  }
  const T rho = A[0][0][0];
  const T drho = rho - T(1);
  const T inv = rcp(rho);
  const T j[3] = {A[1][0][0], A[0][1][0], dim_of(ST) == 3 ? A[0][0][1] : T(0)};
  const T u[3] = {j[0] * inv, j[1] * inv, j[2] * inv};
  const T u2[3] = {u[0] * u[0], u[1] * u[1], u[2] * u[2]};
  // absolute raw equilibrium moments (truncated Maxwellian, Sec. 4.2)
  auto raw_eq_abs = [&](int a, int b, int c) -> T {
    return raw_eq_dev<T>(a, b, c, drho, rho, u) + T(a + b + c == 0 ? 1.0 : bg3(a, b, c));
  };
  if constexpr (SPACE == SP_SRT) {
    T Me[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c)) {
        if constexpr (a + b + c == 0) Me[a][b][c] = rho;
        else if constexpr (a + b + c == 1) Me[a][b][c] = A[a][b][c];
        else Me[a][b][c] = raw_eq_abs(a, b, c);
      } else {
        Me[a][b][c] = T(0);
      }
    });
    T feq[q_of(ST)];
    bwd_raw<ST, T>(Me, feq);
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      f[i] = feq[i] + keep.om[0] * (f[i] - feq[i]);
      if constexpr (ZC) f[i] -= T(weight(ST, i));
    });
    return;
  } else if constexpr (SPACE == SP_RAW || SPACE == SP_RAW_W) {
    constexpr bool WO = SPACE == SP_RAW_W;
    T E[3][3][3], N[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      if constexpr (has_mono(ST, a, b, c) && o >= 2) {
        E[a][b][c] = raw_eq_abs(a, b, c);
        if constexpr (REG && o != 2) N[a][b][c] = T(0);
        else N[a][b][c] = A[a][b][c] - E[a][b][c];
      } else {
        E[a][b][c] = T(0);
        N[a][b][c] = T(0);
      }
    });
    if constexpr (!REG) ortho_raw<ST, -1, T, WO>(N);
    relax_order2<ST, T, REG>(N, keep.om[0], keep.om[1]);
    if constexpr (!REG) {
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        if constexpr (has_mono(ST, a, b, c) && o >= 3) N[a][b][c] *= keep.om[o - 1];
      });
    }
    ortho_raw<ST, +1, T, WO>(N);
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) A[a][b][c] = E[a][b][c] + N[a][b][c];
    });
  } else {
    // absolute central moments: the binomial passes without background
    auto binom_abs = [&](auto sign_tag) {
      constexpr int SIGN = decltype(sign_tag)::value;
      if constexpr (dim_of(ST) == 3) {
        sfor<9>([&](auto K) {
          binom3<SIGN, T, 0>(A[CI(K) / 3][CI(K) % 3][0], A[CI(K) / 3][CI(K) % 3][1],
                             A[CI(K) / 3][CI(K) % 3][2], u[2], u2[2], T(0));
        });
      }
      sfor<9>([&](auto K) {
        constexpr int a = CI(K) / 3, c = CI(K) % 3;
        if constexpr (dim_of(ST) == 3 || c == 0)
          binom3<SIGN, T, 0>(A[a][0][c], A[a][1][c], A[a][2][c], u[1], u2[1], T(0));
      });
      sfor<9>([&](auto K) {
        constexpr int b = CI(K) / 3, c = CI(K) % 3;
        if constexpr (dim_of(ST) == 3 || c == 0)
          binom3<SIGN, T, 0>(A[0][b][c], A[1][b][c], A[2][b][c], u[0], u2[0], T(0));
      });
    };
    binom_abs(std::integral_constant<int, -1>{});
    T Kn[3][3][3];  // absolute normalised central moments kappa / rho
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) Kn[a][b][c] = A[a][b][c] * inv;
      else Kn[a][b][c] = T(0);
    });
    // equilibrium: Gaussian moments bg3 (central) / 1/3 on the 2nd-order
    // diagonal and 0 above (cumulants)
    T X[3][3][3], Xeq[3][3][3];
    if constexpr (SPACE == SP_CENTRAL && SWE) {
      // shallow water (de Rosis): normalised central moments of Zhou's
      // discrete equilibrium about the same u
      T fe[q_of(ST)];
      swe_feq<ST, T, SP_CENTRAL>(rho, u, swe_g, fe);
      T E[3][3][3];
      fwd_raw_chimera<ST, T>(fe, E);
      if constexpr (dim_of(ST) == 3) {
        sfor<9>([&](auto K) {
          binom3<-1, T, 0>(E[CI(K) / 3][CI(K) % 3][0], E[CI(K) / 3][CI(K) % 3][1],
                           E[CI(K) / 3][CI(K) % 3][2], u[2], u2[2], T(0));
        });
      }
      sfor<9>([&](auto K) {
        constexpr int a = CI(K) / 3, c = CI(K) % 3;
        if constexpr (dim_of(ST) == 3 || c == 0)
          binom3<-1, T, 0>(E[a][0][c], E[a][1][c], E[a][2][c], u[1], u2[1], T(0));
      });
      sfor<9>([&](auto K) {
        constexpr int b = CI(K) / 3, c = CI(K) % 3;
        if constexpr (dim_of(ST) == 3 || c == 0)
          binom3<-1, T, 0>(E[0][b][c], E[1][b][c], E[2][b][c], u[0], u2[0], T(0));
      });
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        X[a][b][c] = Kn[a][b][c];
        Xeq[a][b][c] = (has_mono(ST, a, b, c) && a + b + c >= 2) ? E[a][b][c] * inv : T(0);
      });
    } else if constexpr (SPACE == SP_CENTRAL) {
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        X[a][b][c] = Kn[a][b][c];
        Xeq[a][b][c] = T(bg3(a, b, c));
      });
    } else {
      // cumulants: c_s^2 on the second-order diagonal (1/3, or g h / 2 for
      // the shallow-water method of Venturi), 0 above
      const T cs2 = SWE ? T(0.5) * swe_g * rho : T(1.0 / 3.0);
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        X[a][b][c] = Kn[a][b][c];
        Xeq[a][b][c] = (o == 2 && bg3(a, b, c) != 0.0) ? cs2 : T(0);
      });
      cumulant_fwd<ST, T, true>(Kn, X);
    }
    T N[3][3][3];
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      if constexpr (has_mono(ST, a, b, c) && o >= 2) N[a][b][c] = X[a][b][c] - Xeq[a][b][c];
      else N[a][b][c] = T(0);
    });
    relax_order2<ST, T, REG>(N, keep.om[0], keep.om[1]);
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      if constexpr (has_mono(ST, a, b, c) && o >= 2) {
        if constexpr (o == 2) X[a][b][c] = Xeq[a][b][c] + N[a][b][c];
        else if constexpr (REG) X[a][b][c] = Xeq[a][b][c];
        else X[a][b][c] = Xeq[a][b][c] + keep.om[o - 1] * N[a][b][c];
      }
    });
    if constexpr (SPACE == SP_CUMULANT) {
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        constexpr int o = a + b + c;
        Kn[a][b][c] = (o == 2 || o == 3) ? X[a][b][c] : T(0);
      });
      cumulant_bwd<ST, T, REG, true>(X, Kn);
      if constexpr (REG) {
        sfor<27>([&](auto K) {
          constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
          if constexpr (a + b + c == 3) Kn[a][b][c] = T(0);
        });
      }
    } else {
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
        Kn[a][b][c] = X[a][b][c];
      });
    }
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      constexpr int o = a + b + c;
      if constexpr (o == 0) A[a][b][c] = rho;
      else if constexpr (o == 1) A[a][b][c] = T(0);
      else if constexpr (has_mono(ST, a, b, c)) A[a][b][c] = rho * Kn[a][b][c];
      else A[a][b][c] = T(0);
    });
    binom_abs(std::integral_constant<int, +1>{});
  }
  A[0][0][0] = rho;
  A[1][0][0] = j[0];
  A[0][1][0] = j[1];
  if constexpr (dim_of(ST) == 3) A[0][0][1] = j[2];
  if constexpr (ZC) {
    A[0][0][0] = drho0;
    sfor<27>([&](auto K) {
      constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
      if constexpr (has_mono(ST, a, b, c) && a + b + c >= 2) A[a][b][c] -= T(bg3(a, b, c));
    });
  }
  bwd_raw<ST, T>(A, f);
}

// ------------------------------------------------------- storage codecs
template <class S>
struct Codec;
template <>
struct Codec<double> {
  template <class T>
  LBM_D static T dec(double v, int) { return T(v); }
  template <class T>
  LBM_D static double enc(T v, int) { return double(v); }
};
template <>
struct Codec<float> {
  template <class T>
  LBM_D static T dec(float v, int) { return T(v); }
  template <class T>
  LBM_D static float enc(T v, int) { return float(v); }
};
// FP16 / BF16 deltas: h = round_rn(df * 2^s); powers of two are exact
template <>
struct Codec<__half> {
  template <class T>
  LBM_D static T dec(__half v, int s) { return T(__half2float(v) * (1.0f / float(1u << s))); }
  template <class T>
  LBM_D static __half enc(T v, int s) { return __float2half_rn(float(v) * float(1u << s)); }
};
template <>
struct Codec<__nv_bfloat16> {
  template <class T>
  LBM_D static T dec(__nv_bfloat16 v, int s) {
    return T(__bfloat162float(v) * (1.0f / float(1u << s)));
  }
  template <class T>
  LBM_D static __nv_bfloat16 enc(T v, int s) {
    return __float2bfloat16_rn(float(v) * float(1u << s));
  }
};

}  // namespace lbm
