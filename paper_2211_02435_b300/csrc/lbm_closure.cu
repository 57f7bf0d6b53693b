// lbm_closure.cu -- learned closure (include/lbm_closure.h): the D3Q27
// cumulant collision with per-cell rates of orders 3..6 from a fused MLP,
// and the hand-written training kernels (forward with activations, loss and
// adjoint of streaming, forward-mode tangents of the collision with respect
// to the four rates, MLP backward, deterministic weight-gradient reduction,
// Adam).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_closure.h"
#include "lbm_kernels.cuh"
#include "lbm_umma.cuh"

namespace lbm {

// FP32 inference network of the fused step, a compile-time choice measured
// on B300: 0 CUDA cores (packed FFMA2), 1 warp-level tensor-core MMAs
// (mma.sync, activations in registers between layers), 2 CTA-level
// tcgen05 MMAs with the accumulators in tensor memory
#ifndef LBM_CLOSURE_NET
#define LBM_CLOSURE_NET 1
#endif
// minimum resident CTAs per SM asked of the fused learned-rate step kernel
// (0: the compiler's choice, measured fastest on B300; 4 and 5 spill)
#ifndef LBM_CLOSURE_MINB
#define LBM_CLOSURE_MINB 0
#endif
#if LBM_CLOSURE_MINB > 0
#define LBM_CLOSURE_BOUNDS __launch_bounds__(128, LBM_CLOSURE_MINB)
#else
#define LBM_CLOSURE_BOUNDS __launch_bounds__(128)
#endif

constexpr int NIN = LBM_CLOSURE_NIN, NH = LBM_CLOSURE_NHIDDEN, NOUT = LBM_CLOSURE_NOUT;
constexpr int NPARAM = LBM_CLOSURE_NPARAM;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH;
constexpr int OW3 = OB2 + NH, OB3 = OW3 + NOUT * NH;
static_assert(OB3 + NOUT == NPARAM, "parameter layout");
constexpr int NSMEM = NPARAM + 2 * NIN;  // parameters, shift, scale

// FP32 tanh from the identity tanh|x| = (1 - t) / (1 + t), t = e^(-2|x|) in
// (0, 1], with the sign of x restored: the fast exponential never overflows
// and the quotient's denominator stays in [1, 2].  Absolute error a few 1e-8
// on the whole line (near 0 the relative error grows while the absolute error
// stays at the rounding of 1), exactly +-1 once t underflows, NaN for NaN.
// A third of the instructions of the library tanhf, which was a large part
// of the network's cost.  FP64 keeps tanh.
template <class T>
LBM_D T tanh_t(T x) {
  if constexpr (std::is_same<T, float>::value) {
#ifdef __CUDA_ARCH__
    const float t = __expf(-2.0f * fabsf(x));
    return copysignf(__fdividef(1.0f - t, 1.0f + t), x);
#else
    return tanhf(x);
#endif
  } else {
    return tanh(x);
  }
}
template <class T>
LBM_D T exp_t(T x) {
  if constexpr (std::is_same<T, float>::value) return expf(x);
  else return exp(x);
}
template <class T>
LBM_D T sqrt_t(T x) {
  if constexpr (std::is_same<T, float>::value) return sqrtf(x);
  else return sqrt(x);
}

// ------------------------------------------------ forward-mode dual number
// A value and one tangent.  The collision's templates run on it unchanged,
// so one pass seeded with the unit tangent on population j gives column j of
// the per-cell Jacobian d f* / d f (and d features / d f) exactly, up to
// FP32 rounding; the training backward pass takes 27 such passes per cell.
struct Dual {
  float v, d;
  Dual() = default;
  LBM_D constexpr Dual(double x) : v(float(x)), d(0.f) {}
  LBM_D constexpr Dual(float a, float b) : v(a), d(b) {}
};
LBM_D Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
LBM_D Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
LBM_D Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
LBM_D Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
LBM_D Dual operator/(Dual a, Dual b) {
  const float q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
LBM_D Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
LBM_D Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
LBM_D Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
LBM_D bool operator>(Dual a, Dual b) { return a.v > b.v; }
LBM_D bool operator<(Dual a, Dual b) { return a.v < b.v; }
// d sqrt(x) = dx / (2 sqrt(x)); the features only take it of a sum of
// squares, whose zero is handled by the caller
LBM_D Dual sqrt_t(Dual x) {
  const float r = sqrtf(x.v);
  return Dual(r, r > 0.f ? 0.5f * x.d / r : 0.f);
}

// A cell's normalised input is usable when it is finite and within FP16's
// range, the operand type of the tensor-core network (|x| <= 65504; NaN
// fails both comparisons); a cell with an unusable input keeps rates 1.
template <class T>
LBM_D bool input_ok(T x) {
  return x <= T(65504) && x >= T(-65504);
}

// ----------------------------------------------------------- network
// P points to NSMEM values: parameters, then shift[7], then scale[7].
// Returns the rates omega[4] and d omega / d z (0 where clamped or on the
// non-finite fallback), keeping the activations for the backward pass.
template <class T>
LBM_D void mlp_forward(const T* P, const T (&raw)[NIN], T (&x)[NIN], T (&h1)[NH], T (&h2)[NH],
                       T (&om)[NOUT], T (&dom)[NOUT]) {
  const T* shift = P + NPARAM;
  const T* scale = shift + NIN;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < NIN; ++i) {
    x[i] = (raw[i] - shift[i]) * scale[i];
    ok = ok && input_ok(x[i]);
  }
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int r = 0; r < NH; r += 2) {
      float2 a = make_float2(P[OB1 + r], P[OB1 + r + 1]);
#pragma unroll
      for (int c = 0; c < NIN; ++c)
        a = ffma2(make_float2(P[OW1 + r * NIN + c], P[OW1 + (r + 1) * NIN + c]),
                  make_float2(x[c], x[c]), a);
      h1[r] = tanh_t(a.x);
      h1[r + 1] = tanh_t(a.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < NH; ++r) {
      T a = P[OB1 + r];
#pragma unroll
      for (int c = 0; c < NIN; ++c) a += P[OW1 + r * NIN + c] * x[c];
      h1[r] = tanh_t(a);
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    // two rows per packed fused multiply-add: each lane runs the same FP32
    // chain as the scalar loop, so the results are bitwise equal
#pragma unroll
    for (int r = 0; r < NH; r += 2) {
      float2 a = make_float2(P[OB2 + r], P[OB2 + r + 1]);
#pragma unroll
      for (int c = 0; c < NH; ++c)
        a = ffma2(make_float2(P[OW2 + r * NH + c], P[OW2 + (r + 1) * NH + c]),
                  make_float2(h1[c], h1[c]), a);
      h2[r] = tanh_t(a.x);
      h2[r + 1] = tanh_t(a.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < NH; ++r) {
      T a = P[OB2 + r];
#pragma unroll
      for (int c = 0; c < NH; ++c) a += P[OW2 + r * NH + c] * h1[c];
      h2[r] = tanh_t(a);
    }
  }
#pragma unroll
  for (int k = 0; k < NOUT; ++k) {
    T z = P[OB3 + k];
#pragma unroll
    for (int c = 0; c < NH; ++c) z += P[OW3 + k * NH + c] * h2[c];
    const T sg = T(1) / (T(1) + exp_t(-z));
    T o = T(2) * sg, d = T(2) * sg * (T(1) - sg);
    if (o < T(1e-3)) { o = T(1e-3); d = T(0); }
    if (o > T(1.999)) { o = T(1.999); d = T(0); }
    om[k] = o;
    dom[k] = d;
    ok = ok && isfinite(o);
  }
  if (!ok) {
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      om[k] = T(1);
      dom[k] = T(0);
    }
  }
}

// ----------------------------------------------------------- features
// raw inputs from the normalised second-order central deviations
// (Pi = kappa_2/rho - I/3) and the density deviation: the principal
// invariants of S = -(3 omega_s / 2) Pi and of its deviator D, each of degree
// k divided by the (k-1)-th power of its tensor's Frobenius norm (0 where the
// norm is 0), so that all but the density are of degree 1 in Pi and
// Lipschitz:  {tr S, I2(S)/|S|, det S/|S|^2, I2(D)/|D|, det D/|D|^2, |Pi|, drho}.
// With |S| = (3 omega_s / 2)|Pi| the S quotients are formed from Pi's.
template <class T>
LBM_D void closure_features(const T (&K)[3][3][3], T drho, T omega_s, T (&raw)[NIN]) {
  const T a = K[2][0][0], b = K[0][2][0], c = K[0][0][2];
  const T p = K[1][1][0], q = K[1][0][1], r = K[0][1][1];
  const T s = T(-1.5) * omega_s;  // S = s Pi, s < 0
  const T off = p * p + q * q + r * r;
  const T trP = a + b + c;
  const T i2P = a * b + b * c + c * a - off;
  const T detP = a * (b * c - r * r) - p * (p * c - r * q) + q * (p * r - b * q);
  const T n2P = a * a + b * b + c * c + T(2) * off;
  const T t3 = trP * T(1.0 / 3.0);
  const T da = a - t3, db = b - t3, dc = c - t3;
  const T i2D = da * db + db * dc + dc * da - off;
  const T detD = da * (db * dc - r * r) - p * (p * dc - r * q) + q * (p * r - db * q);
  const T n2D = da * da + db * db + dc * dc + T(2) * off;
  const bool zP = !(n2P > T(0)), zD = !(n2D > T(0));
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, float>::value) {
    // FP32 on the device: one reciprocal square root per norm (the special
    // function unit's, a few ulp) in place of a square root and IEEE
    // divisions; 3 % of the fused learned-rate step
    const float rP = rsqrtf(n2P), rD = rsqrtf(n2D);
    raw[0] = s * trP;
    raw[1] = zP ? 0.f : -s * i2P * rP;
    raw[2] = zP ? 0.f : s * detP * (rP * rP);
    raw[3] = zD ? 0.f : i2D * rD;
    raw[4] = zD ? 0.f : detD * (rD * rD);
    raw[5] = zP ? 0.f : n2P * rP;
    raw[6] = drho;
    return;
  }
#endif
  const T nP = sqrt_t(n2P), nD = sqrt_t(n2D);
  raw[0] = s * trP;
  raw[1] = zP ? T(0) : -s * i2P / nP;    // s^2 I2(Pi) / (|s| |Pi|)
  raw[2] = zP ? T(0) : s * detP / n2P;   // s^3 det(Pi) / (s^2 |Pi|^2)
  raw[3] = zD ? T(0) : i2D / nD;
  raw[4] = zD ? T(0) : detD / n2D;
  raw[5] = nP;
  raw[6] = drho;
}

// ------------------------------------------- cumulant collision, split
template <class T>
struct CumState {
  T drho, rho, inv, j[3], u[3], u2[3];
  T Kn[3][3][3];  // normalised central deviations, orders >= 2
  T Cm[3][3][3];  // pre-collision cumulant deviations, orders 2..6
};

template <class T>
LBM_D void cum_forward(const T (&f)[27], CumState<T>& s) {
  T A[3][3][3];
  fwd_raw_chimera<D3Q27, T>(f, A);
  s.drho = A[0][0][0];
  s.rho = T(1) + s.drho;
  s.inv = rcp(s.rho);
  s.j[0] = A[1][0][0];
  s.j[1] = A[0][1][0];
  s.j[2] = A[0][0][1];
  for (int d = 0; d < 3; ++d) {
    s.u[d] = s.j[d] * s.inv;
    s.u2[d] = s.u[d] * s.u[d];
  }
  binomial<D3Q27, -1, T>(A, s.u, s.u2);
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    constexpr double B = bg3(a, b, c);
    if constexpr (a + b + c >= 2) {
      if constexpr (B != 0.0) s.Kn[a][b][c] = (A[a][b][c] - s.drho * T(B)) * s.inv;
      else s.Kn[a][b][c] = A[a][b][c] * s.inv;
    } else {
      s.Kn[a][b][c] = T(0);
    }
    s.Cm[a][b][c] = s.Kn[a][b][c];
  });
  cumulant_fwd<D3Q27, T>(s.Kn, s.Cm);
}

// relax with keep factors (1 - omega) and return the post-collision
// populations; Cs receives the post-collision cumulant deviations
template <class T>
LBM_D void cum_backward(const CumState<T>& s, const Rates<T>& keep, T (&Cs)[3][3][3],
                        T (&f)[27]) {
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    Cs[a][b][c] = s.Cm[a][b][c];
  });
  relax_order2<D3Q27, T, false>(Cs, keep.om[0], keep.om[1]);
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    constexpr int o = a + b + c;
    if constexpr (o >= 3) Cs[a][b][c] *= keep.om[o - 1];
  });
  T Kp[3][3][3];
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    constexpr int o = a + b + c;
    Kp[a][b][c] = (o == 2 || o == 3) ? Cs[a][b][c] : T(0);
  });
  cumulant_bwd<D3Q27, T, false>(Cs, Kp);
  T A[3][3][3];
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    constexpr int o = a + b + c;
    constexpr double B = bg3(a, b, c);
    if constexpr (o == 0) A[a][b][c] = s.drho;
    else if constexpr (o == 1) A[a][b][c] = T(0);
    else if constexpr (B != 0.0) A[a][b][c] = s.drho * T(B) + s.rho * Kp[a][b][c];
    else A[a][b][c] = s.rho * Kp[a][b][c];
  });
  binomial<D3Q27, +1, T>(A, s.u, s.u2);
  A[0][0][0] = s.drho;
  A[1][0][0] = s.j[0];
  A[0][1][0] = s.j[1];
  A[0][0][1] = s.j[2];
  bwd_raw<D3Q27, T>(A, f);
}

// the binomial Chimera as a pure linear map (no background): used for
// tangents, where the constant background drops out
template <int SIGN, class T>
LBM_D void binomial_linear(T (&A)[3][3][3], const T (&u)[3], const T (&u2)[3]) {
  sfor<9>([&](auto K) {
    constexpr int a = CI(K) / 3, b = CI(K) % 3;
    binom3<SIGN, T, 0>(A[a][b][0], A[a][b][1], A[a][b][2], u[2], u2[2], T(0));
  });
  sfor<9>([&](auto K) {
    constexpr int a = CI(K) / 3, c = CI(K) % 3;
    binom3<SIGN, T, 0>(A[a][0][c], A[a][1][c], A[a][2][c], u[1], u2[1], T(0));
  });
  sfor<9>([&](auto K) {
    constexpr int b = CI(K) / 3, c = CI(K) % 3;
    binom3<SIGN, T, 0>(A[0][b][c], A[1][b][c], A[2][b][c], u[0], u2[0], T(0));
  });
}

// d f* / d omega_ORDER: the post-collision cumulants of order ORDER change
// by -C (pre-collision); the inverse cumulant relations (linearised at the
// post-collision state Cs), the binomial and the raw backward transforms
// are then applied to that direction.
template <int ORDER, class T>
LBM_D void cum_tangent(const CumState<T>& s, const T (&Cs)[3][3][3], T (&t)[27]) {
  const T A3 = T(1.0 / 3.0);
  T dC[3][3][3], dK[3][3][3];
  sfor<27>([&](auto K) {
    constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, c = CI(K) % 3;
    dC[a][b][c] = (a + b + c == ORDER) ? -s.Cm[a][b][c] : T(0);
    dK[a][b][c] = dC[a][b][c];
  });
  const T a = Cs[2][0][0], b = Cs[0][2][0], c = Cs[0][0][2];
  const T c110 = Cs[1][1][0], c101 = Cs[1][0][1], c011 = Cs[0][1][1];
  if constexpr (ORDER == 3) {
    dK[2][2][1] = (A3 + a) * dC[0][2][1] + (A3 + b) * dC[2][0][1] + T(4) * c110 * dC[1][1][1] +
                  T(2) * c101 * dC[1][2][0] + T(2) * c011 * dC[2][1][0];
    dK[2][1][2] = (A3 + a) * dC[0][1][2] + (A3 + c) * dC[2][1][0] + T(4) * c101 * dC[1][1][1] +
                  T(2) * c110 * dC[1][0][2] + T(2) * c011 * dC[2][0][1];
    dK[1][2][2] = (A3 + b) * dC[1][0][2] + (A3 + c) * dC[1][2][0] + T(4) * c011 * dC[1][1][1] +
                  T(2) * c110 * dC[0][1][2] + T(2) * c101 * dC[0][2][1];
    dK[2][2][2] = T(2) * (dC[2][1][0] * Cs[0][1][2] + Cs[2][1][0] * dC[0][1][2] +
                          dC[2][0][1] * Cs[0][2][1] + Cs[2][0][1] * dC[0][2][1] +
                          dC[1][2][0] * Cs[1][0][2] + Cs[1][2][0] * dC[1][0][2]) +
                  T(8) * Cs[1][1][1] * dC[1][1][1];
  } else if constexpr (ORDER == 4) {
    dK[2][2][2] = A3 * (dC[0][2][2] + dC[2][0][2] + dC[2][2][0]) + a * dC[0][2][2] +
                  b * dC[2][0][2] + c * dC[2][2][0] +
                  T(4) * (c110 * dC[1][1][2] + c101 * dC[1][2][1] + c011 * dC[2][1][1]);
  }
  T A[3][3][3];
  sfor<27>([&](auto K) {
    constexpr int a_ = CI(K) / 9, b_ = (CI(K) / 3) % 3, c_ = CI(K) % 3;
    A[a_][b_][c_] = (a_ + b_ + c_ >= 3) ? s.rho * dK[a_][b_][c_] : T(0);
  });
  binomial_linear<+1, T>(A, s.u, s.u2);
  bwd_raw<D3Q27, T>(A, t);
}

// ------------------------------------------------------------ kernels
template <class T>
__device__ __forceinline__ void load_params(T* sp, const T* gp) {
  for (int k = threadIdx.x; k < NSMEM; k += blockDim.x) sp[k] = gp[k];
  __syncthreads();
}

// fused pull step of a context with the learned rates
template <class S, class T>
__global__ void LBM_CLOSURE_BOUNDS
    k_closure_pull(const S* __restrict__ src, S* __restrict__ dst, Geo g, Rates<T> keep,
                   const T* __restrict__ params) {
  __shared__ T sp[NSMEM];
  load_params(sp, params);
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const Nbr n = neighbours(x, y, z, g);
  const int c = (z * g.ny + y) * g.nx + x;
  T f[27];
  load_pops<D3Q27, S, T, G_PULL>(src, g, n, c, f);
  CumState<T> s;
  cum_forward<T>(f, s);
  T raw[NIN], xin[NIN], h1[NH], h2[NH], om[NOUT], dom[NOUT];
  closure_features<T>(s.Kn, s.drho, T(1) - keep.om[0], raw);
  mlp_forward<T>(sp, raw, xin, h1, h2, om, dom);
  Rates<T> k = keep;
#pragma unroll
  for (int o = 0; o < NOUT; ++o) k.om[2 + o] = T(1) - om[o];
  T Cs[3][3][3];
  cum_backward<T>(s, k, Cs, f);
  sfor<27>([&](auto I) {
    constexpr int i = CI(I);
    dst[(int64_t)i * g.N + c] = Codec<S>::template enc<T>(f[i], scale_exp(D3Q27, i));
  });
}

// ------------------------------------------- tensor-core network (FP32)
// The three layers run on the tensor cores for the 128 cells of a CTA at
// once: layer l is D = A * B^T with A = [a_0 | a_1 | a_2] (128 x 3K, row =
// cell) and B = [W | W | W] (N x 3K), where a_0 = bf16(a), a_1 = bf16(a -
// a_0), a_2 = bf16(a - a_0 - a_1) split each FP32 activation into three
// BF16 values.  The weights are BF16 values, so every product is exact and
// the sum runs in FP32 in tensor memory; the split leaves a relative
// residual below 2^-26 per activation, under FP32's own rounding.  Layer 1
// pads the 7 inputs to 8 and its K = 24 to 32 (zero columns), layer 3 pads
// the 4 outputs to N = 16.
constexpr int TC_K1 = 32, TC_K2 = 3 * NH, TC_N3 = 16;
constexpr int TC_B1 = 0, TC_B2 = TC_B1 + NH * TC_K1, TC_B3 = TC_B2 + NH * TC_K2;
constexpr int TC_BELEMS = TC_B3 + TC_N3 * TC_K2;
// packed B operands after the floats and the lane table of the mma.sync network
constexpr int TC_BOFF_BYTES = ((NSMEM * 4 + 127) / 128) * 128 + ((42 * 32 * 4 + 127) / 128) * 128;
constexpr int TC_TMEM_COLS = 32;

// Pack the weights (FP32 values of BF16 numbers) into the three B operands.
inline void pack_tc_weights(const float* P, uint16_t* out) {
  auto bits = [](float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    return uint16_t(u >> 16);  // exact: v is a BF16 value
  };
  for (int k = 0; k < TC_BELEMS; ++k) out[k] = 0;
  for (int n = 0; n < NH; ++n)
    for (int k = 0; k < NIN; ++k)
      for (int h = 0; h < 3; ++h)
        out[TC_B1 + umma::kmajor_offset(n, h * 8 + k, TC_K1)] = bits(P[OW1 + n * NIN + k]);
  for (int n = 0; n < NH; ++n)
    for (int k = 0; k < NH; ++k)
      for (int h = 0; h < 3; ++h)
        out[TC_B2 + umma::kmajor_offset(n, h * NH + k, TC_K2)] = bits(P[OW2 + n * NH + k]);
  for (int n = 0; n < NOUT; ++n)
    for (int k = 0; k < NH; ++k)
      for (int h = 0; h < 3; ++h)
        out[TC_B3 + umma::kmajor_offset(n, h * NH + k, TC_K2)] = bits(P[OW3 + n * NH + k]);
}

// row `r` of an A operand with K columns: the three BF16 parts of v in
// columns [0, KH), [KH, 2 KH), [2 KH, 3 KH); columns from 3 KH on are zero
template <int KH, int K>
__device__ __forceinline__ void write_split(__nv_bfloat16* A, int r, const float (&v)[KH]) {
#pragma unroll
  for (int kc = 0; kc < KH / 8; ++kc) {
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float a = v[kc * 8 + e];
      p0[e] = __float2bfloat16_rn(a);
      const float r1 = a - __bfloat162float(p0[e]);  // exact
      p1[e] = __float2bfloat16_rn(r1);
      p2[e] = __float2bfloat16_rn(r1 - __bfloat162float(p1[e]));
    }
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, kc * 8, K)) =
        *reinterpret_cast<const uint4*>(p0);
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, KH + kc * 8, K)) =
        *reinterpret_cast<const uint4*>(p1);
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, 2 * KH + kc * 8, K)) =
        *reinterpret_cast<const uint4*>(p2);
  }
#pragma unroll
  for (int kc = 3 * KH / 8; kc < K / 8; ++kc)
    *reinterpret_cast<uint4*>(A + umma::kmajor_offset(r, kc * 8, K)) = make_uint4(0, 0, 0, 0);
}

// One layer: every thread has written its A row; thread 0 issues the K/16
// MMAs into tensor-memory columns [0, N) and commits them to `bar`; every
// thread waits (bounded) for the given phase.  Returns false on a timeout.
template <int K, int N>
__device__ __forceinline__ bool tc_layer(const __nv_bfloat16* A, const __nv_bfloat16* B,
                                         uint32_t tmem, uint64_t* bar, uint32_t phase) {
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    umma::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t ad = umma::smem_desc(A + kk * 128, 128, (K / 8) * 128);
      const uint64_t bd = umma::smem_desc(B + kk * 128, 128, (K / 8) * 128);
      umma::mma_bf16(tmem, ad, bd, umma::idesc_bf16_f32(N), kk > 0);
    }
    umma::commit(bar);
  }
  const bool ok = tma::mbar_wait(bar, phase);
  __syncwarp();  // reconverge after the wait loop for the .sync.aligned load
  umma::fence_after_sync();
  return ok;
}

// fused pull step with the learned rates, FP32, network on the tensor cores
__global__ void __launch_bounds__(128)
    k_closure_pull_tc(const float* __restrict__ src, float* __restrict__ dst, Geo g,
                      Rates<float> keep, const float* __restrict__ params, int* status) {
  __shared__ float sp[NSMEM];
  __shared__ __align__(128) __nv_bfloat16 sB[TC_BELEMS];
  __shared__ __align__(128) __nv_bfloat16 sA[128 * TC_K2];  // A of every layer
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, warp = t / 32;
  for (int k = t; k < NSMEM; k += 128) sp[k] = params[k];
  {
    const uint4* gB =
        reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(params) + TC_BOFF_BYTES);
    uint4* sB4 = reinterpret_cast<uint4*>(sB);
    for (int k = t; k < TC_BELEMS / 8; k += 128) sB4[k] = gB[k];
  }
  __syncwarp();  // the tcgen05 .sync.aligned forms need converged warps
  if (warp == 0) umma::tmem_alloc(&tmem_base, TC_TMEM_COLS);
  if (t == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);

  const int x = blockIdx.x * 128 + t;
  const bool active = x < g.nx;
  const int y = blockIdx.y, z = blockIdx.z;
  const int c = (z * g.ny + y) * g.nx + (active ? x : 0);
  float f[27];
  CumState<float> s;
  float xin[8];
  bool ok = true;
  if (active) {
    const Nbr n = neighbours(x, y, z, g);
    load_pops<D3Q27, float, float, G_PULL>(src, g, n, c, f);
    cum_forward<float>(f, s);
    float raw[NIN];
    closure_features<float>(s.Kn, s.drho, 1.0f - keep.om[0], raw);
#pragma unroll
    for (int i = 0; i < NIN; ++i) {
      xin[i] = (raw[i] - sp[NPARAM + i]) * sp[NPARAM + NIN + i];
      ok = ok && input_ok(xin[i]);
    }
    xin[7] = 0.0f;
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) xin[i] = 0.0f;
  }
  bool waited = true;
  float acc[32], h[32];
  write_split<8, TC_K1>(sA, t, xin);
  waited &= tc_layer<TC_K1, NH>(sA, sB + TC_B1, tmem, &bar, 0);
  umma::tmem_ld32(tlane, acc);
#pragma unroll
  for (int j = 0; j < NH; ++j) h[j] = tanh_t(acc[j] + sp[OB1 + j]);
  write_split<NH, TC_K2>(sA, t, h);
  waited &= tc_layer<TC_K2, NH>(sA, sB + TC_B2, tmem, &bar, 1);
  umma::tmem_ld32(tlane, acc);
#pragma unroll
  for (int j = 0; j < NH; ++j) h[j] = tanh_t(acc[j] + sp[OB2 + j]);
  write_split<NH, TC_K2>(sA, t, h);
  waited &= tc_layer<TC_K2, TC_N3>(sA, sB + TC_B3, tmem, &bar, 0);
  float z16[16];
  umma::tmem_ld16(tlane, z16);
  Rates<float> k = keep;
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    const float zz = z16[o] + sp[OB3 + o];
    const float sg = 1.0f / (1.0f + expf(-zz));
    float om = 2.0f * sg;
    if (om < 1e-3f) om = 1e-3f;
    if (om > 1.999f) om = 1.999f;
    ok = ok && isfinite(om);
    k.om[2 + o] = 1.0f - om;
  }
  if (!ok) {
#pragma unroll
    for (int o = 0; o < NOUT; ++o) k.om[2 + o] = 0.0f;  // rates 1
  }
  if (active) {
    float Cs[3][3][3];
    cum_backward<float>(s, k, Cs, f);
    sfor<27>([&](auto I) {
      constexpr int i = CI(I);
      dst[(int64_t)i * g.N + c] = f[i];
    });
  }
  umma::fence_before_sync();
  if (__syncthreads_or(!waited)) {
    // a bounded wait ran out: record it and let the last MMAs finish
    if (t == 0) {
      atomicExch(status, 1);
      tma::mbar_wait(&bar, 0);
    }
    __syncthreads();
  }
  __syncwarp();
  if (warp == 0) umma::tmem_dealloc(tmem, TC_TMEM_COLS);
}

// --------------------------------- warp-level tensor-core network (FP32)
// A warp's 32 cells (one per lane) are two 16-row tiles.  Layer l computes
// D = A B + bias with A the activations and B[k][n] = W_l[n][k] by mma.sync
// (m16n8k8 for the 7 inputs padded to 8, m16n8k16 above), FP16 operands and
// FP32 accumulation.  The weights are BF16 numbers, whose 8 significant bits
// FP16 holds exactly (down to |w| = 2^-17; below that the FP16 subnormal
// spacing 2^-24 bounds the change); the host refuses weights beyond FP16's
// range.  Each FP32 activation enters as two FP16 parts, hi = fp16(a) and
// lo = fp16(a - hi) (|a - hi - lo| <= 2^-22 |a|, plus 2^-25 where lo is
// subnormal), each multiplied by the same B, so every product is exact.
// Two BF16 parts (2^-17) measured a fused-step error of up to 1.2e-5 of the
// FP64 oracle on strongly non-equilibrium states, two FP16 parts 2.7e-6;
// with the residual a - hi formed by one mixed-precision FMA per value, the
// FP16 split is also the cheaper one (16.4 against 16.2 GLUPS at 128^3).
// The accumulator fragments of two adjacent n8 tiles are, element for
// element, the A fragment of the next layer's k16 tile: the hidden
// activations never leave the registers; only the 7 inputs and the 4 outputs
// pass through shared memory.
namespace wmn {
// per-lane table, word w of lane l at [w * 32 + l]
constexpr int L1_B = 0;       // layer 1, n-tiles 0..3: B (k 2t, 2t+1; n 8j + g);
                              // input 7 is the constant 1 and its weight the bias
constexpr int L2_B = 4;       // layer 2, (k-tile kk, n-tile j): 2 words at 4 + 2 (4 kk + j)
constexpr int L3_B = 20;      // layer 3, k-tile kk: 2 words at 20 + 2 kk
constexpr int L2_BIAS = 24;   // layer 2 bias of columns 8j + 2t + e at 24 + 2j + e
constexpr int L3_BIAS = 32;   // layer 3 bias of columns 2t + e (0 for t >= 2)
constexpr int WORDS = 34;
// byte offset of the table in the device parameter image (after the floats)
constexpr int TAB_OFF_BYTES = ((NSMEM * 4 + 127) / 128) * 128;
constexpr int TAB_BYTES = WORDS * 32 * 4;

// two floats as an FP16 pair: first element in the low half (the lower k)
__device__ __forceinline__ uint32_t f16x2(float first, float second) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
  return r;
}
// hi and lo parts of a pair; a - hi is exact (Sterbenz: hi is a's nearest
// FP16 number) and comes from one mixed-precision FMA, hi * (-1) + a, that
// reads hi's half of the packed register as its FP16 operand
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = f16x2(a, b);
  float ra, rb;
  asm("{\n .reg .b16 h0, h1;\n mov.b32 {h0, h1}, %2;\n"
      " fma.rn.f32.f16 %0, h0, %5, %3;\n fma.rn.f32.f16 %1, h1, %5, %4;\n}"
      : "=f"(ra), "=f"(rb)
      : "r"(hi), "f"(a), "f"(b), "h"((unsigned short)0xBC00));  // FP16 -1
  lo = f16x2(ra, rb);
}
__device__ __forceinline__ void mma_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                        uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
      "{%4, %5}, {%6}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}
// the hidden activation: the special-function unit's tanh (one instruction,
// relative error about 2^-11).  Against the FP64 oracle the fused step's
// relative L-infinity error changed little with an accurate tanh from ex2
// and rcp (9.5e-6 against 1.1e-5 with two BF16 parts, the largest case),
// which ran 16 % slower.
__device__ __forceinline__ float tanh_mma(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// the next layer's A fragments (hi and lo parts) of k-tile kk from the
// accumulators D[mt][n-tile][4]
__device__ __forceinline__ void next_a(const float (&D)[4][4], int kk, uint32_t (&ah)[4],
                                       uint32_t (&al)[4]) {
  split2(D[2 * kk][0], D[2 * kk][1], ah[0], al[0]);
  split2(D[2 * kk][2], D[2 * kk][3], ah[1], al[1]);
  split2(D[2 * kk + 1][0], D[2 * kk + 1][1], ah[2], al[2]);
  split2(D[2 * kk + 1][2], D[2 * kk + 1][3], ah[3], al[3]);
}

// The network of the warp's 32 cells: x this lane's normalised inputs (x[7]
// = 1, the input that carries layer 1's bias), tab the lane table (shared
// memory), st 256 words of per-warp shared staging; z receives this lane's 4
// outputs.  All 32 lanes must call it.
__device__ __forceinline__ void mlp_warp(const float (&x)[8], const uint32_t* __restrict__ tab,
                                         uint32_t* st, float (&z)[4]) {
  const int lane = threadIdx.x & 31, t = lane & 3, g = lane >> 2;
  const uint32_t* T = tab + lane;
  // layer 1: the inputs of every row to the fragment layout
  {
    uint4 h, l;
    split2(x[0], x[1], h.x, l.x);
    split2(x[2], x[3], h.y, l.y);
    split2(x[4], x[5], h.z, l.z);
    split2(x[6], x[7], h.w, l.w);
    reinterpret_cast<uint4*>(st)[2 * lane] = h;
    reinterpret_cast<uint4*>(st)[2 * lane + 1] = l;
  }
  __syncwarp();
  float D[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    const uint32_t h0 = st[8 * r0 + t], h1 = st[8 * r1 + t];
    const uint32_t l0 = st[8 * r0 + 4 + t], l1 = st[8 * r1 + 4 + t];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      D[mt][j][0] = D[mt][j][1] = D[mt][j][2] = D[mt][j][3] = 0.f;
      const uint32_t B = T[32 * (L1_B + j)];
      mma_k8(D[mt][j], h0, h1, B);
      mma_k8(D[mt][j], l0, l1, B);
    }
  }
  __syncwarp();  // st is reused below
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) D[mt][j][e] = tanh_mma(D[mt][j][e]);
  // layer 2
  float E[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float b0 = __uint_as_float(T[32 * (L2_BIAS + 2 * j)]);
      const float b1 = __uint_as_float(T[32 * (L2_BIAS + 2 * j + 1)]);
      E[mt][j][0] = b0, E[mt][j][1] = b1, E[mt][j][2] = b0, E[mt][j][3] = b1;
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t ah[4], al[4];
      next_a(D[mt], kk, ah, al);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t B0 = T[32 * (L2_B + 2 * (4 * kk + j))];
        const uint32_t B1 = T[32 * (L2_B + 2 * (4 * kk + j) + 1)];
        mma_k16(E[mt][j], ah, B0, B1);
        mma_k16(E[mt][j], al, B0, B1);
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) E[mt][j][e] = tanh_mma(E[mt][j][e]);
  // layer 3 (outputs in columns 0..3 of one n8 tile)
  float F[2][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const float b0 = __uint_as_float(T[32 * L3_BIAS]), b1 = __uint_as_float(T[32 * (L3_BIAS + 1)]);
    F[mt][0] = b0, F[mt][1] = b1, F[mt][2] = b0, F[mt][3] = b1;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t ah[4], al[4];
      next_a(E[mt], kk, ah, al);
      const uint32_t B0 = T[32 * (L3_B + 2 * kk)], B1 = T[32 * (L3_B + 2 * kk + 1)];
      mma_k16(F[mt], ah, B0, B1);
      mma_k16(F[mt], al, B0, B1);
    }
  }
  // back to one row per lane: lane (g, t) holds row g (F[..][0..1]) and row
  // g + 8 (F[..][2..3]) at columns 2t, 2t + 1
  float* sf = reinterpret_cast<float*>(st);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int e = 0; e < 4; ++e) sf[8 * lane + 4 * mt + e] = F[mt][e];
  __syncwarp();
  {
    const int mt = lane >> 4, r = lane & 15, gg = r & 7, hf = r >> 3;
    const float* a = sf + 8 * (4 * gg) + 4 * mt + 2 * hf;      // t = 0: columns 0, 1
    const float* b = sf + 8 * (4 * gg + 1) + 4 * mt + 2 * hf;  // t = 1: columns 2, 3
    z[0] = a[0], z[1] = a[1], z[2] = b[0], z[3] = b[1];
  }
  __syncwarp();
}
}  // namespace wmn

// Pack the weights (FP32 values of BF16 numbers, |w| <= 65504) as FP16 and
// the biases into the lane table of mlp_warp.
inline void pack_lane_table(const float* P, uint32_t* tab) {
  auto bits = [](float v) { return uint32_t(__half_as_ushort(__float2half_rn(v))); };
  auto pair = [&](float first, float second) { return bits(first) | (bits(second) << 16); };
  auto fbits = [](float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    return u;
  };
  // input column 7 is the constant 1: its weights are layer 1's biases
  auto W1 = [&](int n, int k) { return k < NIN ? P[OW1 + n * NIN + k] : P[OB1 + n]; };
  auto W2 = [&](int n, int k) { return P[OW2 + n * NH + k]; };
  auto W3 = [&](int n, int k) { return n < NOUT ? P[OW3 + n * NH + k] : 0.f; };
  for (int l = 0; l < 32; ++l) {
    const int g = l >> 2, t = l & 3;
    auto at = [&](int w) -> uint32_t& { return tab[w * 32 + l]; };
    for (int j = 0; j < 4; ++j) at(wmn::L1_B + j) = pair(W1(8 * j + g, 2 * t), W1(8 * j + g, 2 * t + 1));
    for (int kk = 0; kk < 2; ++kk)
      for (int j = 0; j < 4; ++j) {
        const int n = 8 * j + g, k = 16 * kk + 2 * t;
        at(wmn::L2_B + 2 * (4 * kk + j)) = pair(W2(n, k), W2(n, k + 1));
        at(wmn::L2_B + 2 * (4 * kk + j) + 1) = pair(W2(n, k + 8), W2(n, k + 9));
      }
    for (int kk = 0; kk < 2; ++kk) {
      const int k = 16 * kk + 2 * t;
      at(wmn::L3_B + 2 * kk) = pair(W3(g, k), W3(g, k + 1));
      at(wmn::L3_B + 2 * kk + 1) = pair(W3(g, k + 8), W3(g, k + 9));
    }
    for (int j = 0; j < 4; ++j)
      for (int e = 0; e < 2; ++e) at(wmn::L2_BIAS + 2 * j + e) = fbits(P[OB2 + 8 * j + 2 * t + e]);
    for (int e = 0; e < 2; ++e)
      at(wmn::L3_BIAS + e) = fbits(2 * t + e < NOUT ? P[OB3 + 2 * t + e] : 0.f);
  }
}

// fused pull step with the learned rates, FP32, the network on warp-level
// MMAs; a persistent grid walks tiles of 128 cells of one x-row.  The
// gather uses per-plane pointers pre-shifted by the interior stencil offset
// (as the plain pull kernel), so a load is src_i[c + wrap_i].
__global__ void LBM_CLOSURE_BOUNDS
    k_closure_pull_mma(const __grid_constant__ PullPtrs<float> P, Geo g, Rates<float> keep,
                       const float* __restrict__ params, int tiles_x, int ntiles) {
  __shared__ __align__(16) uint32_t tab[wmn::WORDS * 32];
  __shared__ __align__(16) uint32_t stage[4][256];
  __shared__ float nrm[2 * NIN];
  {
    const uint32_t* gt = reinterpret_cast<const uint32_t*>(
        reinterpret_cast<const char*>(params) + wmn::TAB_OFF_BYTES);
    for (int k = threadIdx.x; k < wmn::WORDS * 32; k += 128) tab[k] = gt[k];
    if (threadIdx.x < 2 * NIN) nrm[threadIdx.x] = params[NPARAM + threadIdx.x];
  }
  __syncthreads();
  uint32_t* st = stage[threadIdx.x >> 5];
  const float omega_s = 1.0f - keep.om[0];
  const int nxy = g.nx * g.ny;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x = (tile % tiles_x) * 128 + int(threadIdx.x);
    const int row = tile / tiles_x;
    const int y = row % g.ny, z = row / g.ny;
    const bool active = x < g.nx;
    const int c = row * g.nx + (active ? x : 0);
    float f[27];
    CumState<float> s;
    float xin[8];
    bool ok = true;
    if (active) {
      // wrap corrections for a read at x - xi (xi = +1 reads x - 1)
      const int wxp = x == 0 ? g.nx : 0, wxm = x == g.nx - 1 ? -g.nx : 0;
      const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
      const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
      sfor<27>([&](auto I) {
        constexpr int i = CI(I);
        constexpr int cx = vel(D3Q27, i, 0), cy = vel(D3Q27, i, 1), cz = vel(D3Q27, i, 2);
        const int w = (cx > 0 ? wxp : (cx < 0 ? wxm : 0)) + (cy > 0 ? wyp : (cy < 0 ? wym : 0)) +
                      (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
        f[i] = P.src[i][c + w];
      });
      cum_forward<float>(f, s);
      float raw[NIN];
      closure_features<float>(s.Kn, s.drho, omega_s, raw);
#pragma unroll
      for (int i = 0; i < NIN; ++i) {
        xin[i] = (raw[i] - nrm[i]) * nrm[NIN + i];
        ok = ok && input_ok(xin[i]);
      }
      if (!ok)
#pragma unroll
        for (int i = 0; i < NIN; ++i) xin[i] = 0.f;
    } else {
#pragma unroll
      for (int i = 0; i < NIN; ++i) xin[i] = 0.f;
    }
    xin[7] = 1.f;  // the bias input
    float zz[4];
    wmn::mlp_warp(xin, tab, st, zz);
    if (active) {
      Rates<float> k = keep;
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        const float sg = __fdividef(1.0f, 1.0f + __expf(-zz[o]));
        float om = 2.0f * sg;
        om = om < 1e-3f ? 1e-3f : om;
        om = om > 1.999f ? 1.999f : om;
        ok = ok && isfinite(om);
        k.om[2 + o] = 1.0f - om;
      }
      if (!ok)
#pragma unroll
        for (int o = 0; o < NOUT; ++o) k.om[2 + o] = 0.0f;  // rates 1
      float Cs[3][3][3];
      cum_backward<float>(s, k, Cs, f);
      sfor<27>([&](auto I) { P.dst[CI(I)][c] = f[CI(I)]; });
    }
  }
}

// The same step with two cells (x, x + 1) per thread for even Nx: the
// cumulant transforms run on packed FP32 pairs (FFMA2 / FADD2 / FMUL2, each
// lane the FP32 arithmetic of the one-cell kernel), which halves the
// collision's instruction count per cell; the features and the sigmoid stay
// per cell and the warp's network runs twice, once per cell of the pair.  A
// tile is 256 consecutive cells (a pair never straddles a row).  Measured on
// B300 at 128^3: 16.1 GLUPS against 13.8 for the one-cell kernel, 16.3 with
// the register cap of four CTAs per SM (84 bytes of spills).
__global__ void __launch_bounds__(128, 4)
    k_closure_pull_mma2(const __grid_constant__ PullPtrs<float> P, Geo g, Rates<float> keep,
                        const float* __restrict__ params, int ntiles) {
  __shared__ __align__(16) uint32_t tab[wmn::WORDS * 32];
  __shared__ __align__(16) uint32_t stage[4][256];
  __shared__ float nrm[2 * NIN];
  {
    const uint32_t* gt = reinterpret_cast<const uint32_t*>(
        reinterpret_cast<const char*>(params) + wmn::TAB_OFF_BYTES);
    for (int k = threadIdx.x; k < wmn::WORDS * 32; k += 128) tab[k] = gt[k];
    if (threadIdx.x < 2 * NIN) nrm[threadIdx.x] = params[NPARAM + threadIdx.x];
  }
  __syncthreads();
  uint32_t* st = stage[threadIdx.x >> 5];
  const float omega_s = 1.0f - keep.om[0];
  const int nxy = g.nx * g.ny;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile * 256 + 2 * int(threadIdx.x);
    const bool active = c0 < int(g.N);
    const int c = active ? c0 : 0;
    const int row = c / g.nx, x = c - row * g.nx;
    const int y = row % g.ny, z = row / g.ny;
    P2 f[27];
    CumState<P2> s;
    float xa[8], xb[8];  // the two cells' normalised inputs
    bool oka = true, okb = true;
    if (active) {
      // wrap corrections: cell x reading x - 1, cell x + 1 reading x + 2
      const int wx0 = x == 0 ? g.nx : 0, wx1 = x + 2 == g.nx ? -g.nx : 0;
      const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
      const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
      sfor<27>([&](auto I) {
        constexpr int i = CI(I);
        constexpr int cx = vel(D3Q27, i, 0), cy = vel(D3Q27, i, 1), cz = vel(D3Q27, i, 2);
        const int w = (cy > 0 ? wyp : (cy < 0 ? wym : 0)) + (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
        const float* p = P.src[i] + (c + w);  // cell x's source element
        if constexpr (cx == 0) f[i] = P2(*reinterpret_cast<const float2*>(p));
        else if constexpr (cx > 0) f[i] = P2(make_float2(p[wx0], p[1]));
        else f[i] = P2(make_float2(p[0], p[1 + wx1]));
      });
      cum_forward<P2>(f, s);
      float Ka[3][3][3], Kb[3][3][3];
      sfor<27>([&](auto K) {
        constexpr int a = CI(K) / 9, b = (CI(K) / 3) % 3, cc = CI(K) % 3;
        Ka[a][b][cc] = s.Kn[a][b][cc].v.x;
        Kb[a][b][cc] = s.Kn[a][b][cc].v.y;
      });
      float ra[NIN], rb[NIN];
      closure_features<float>(Ka, s.drho.v.x, omega_s, ra);
      closure_features<float>(Kb, s.drho.v.y, omega_s, rb);
#pragma unroll
      for (int i = 0; i < NIN; ++i) {
        xa[i] = (ra[i] - nrm[i]) * nrm[NIN + i];
        xb[i] = (rb[i] - nrm[i]) * nrm[NIN + i];
        oka = oka && input_ok(xa[i]);
        okb = okb && input_ok(xb[i]);
      }
      if (!oka)
#pragma unroll
        for (int i = 0; i < NIN; ++i) xa[i] = 0.f;
      if (!okb)
#pragma unroll
        for (int i = 0; i < NIN; ++i) xb[i] = 0.f;
    } else {
#pragma unroll
      for (int i = 0; i < NIN; ++i) xa[i] = xb[i] = 0.f;
    }
    xa[7] = xb[7] = 1.f;  // the bias input
    float za[4], zb[4];
    wmn::mlp_warp(xa, tab, st, za);
    wmn::mlp_warp(xb, tab, st, zb);
    if (active) {
      Rates<P2> k;
#pragma unroll
      for (int o = 0; o < 6; ++o) k.om[o] = P2(keep.om[o]);
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        float oa = 2.0f * __fdividef(1.0f, 1.0f + __expf(-za[o]));
        float ob = 2.0f * __fdividef(1.0f, 1.0f + __expf(-zb[o]));
        oa = oa < 1e-3f ? 1e-3f : (oa > 1.999f ? 1.999f : oa);
        ob = ob < 1e-3f ? 1e-3f : (ob > 1.999f ? 1.999f : ob);
        oka = oka && isfinite(oa);
        okb = okb && isfinite(ob);
        k.om[2 + o] = P2(make_float2(1.0f - oa, 1.0f - ob));
      }
      // a cell whose inputs or rates are not finite relaxes with rates 1
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        if (!oka) k.om[2 + o].v.x = 0.0f;
        if (!okb) k.om[2 + o].v.y = 0.0f;
      }
      P2 Cs[3][3][3];
      cum_backward<P2>(s, k, Cs, f);
      sfor<27>([&](auto I) { *reinterpret_cast<float2*>(P.dst[CI(I)] + c) = f[CI(I)].v; });
    }
  }
}

// 4^3 block average of the canonical populations of a fine lattice
template <class S, class T, int MODE>
__global__ void __launch_bounds__(128)
    k_restrict(const S* __restrict__ fine, Geo gf, float* __restrict__ snap, Geo gc) {
  const int64_t C = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (C >= gc.N) return;
  int X, Y, Z;
  cell_xyz(int(C), gc, X, Y, Z);
  T acc[27];
  for (int i = 0; i < 27; ++i) acc[i] = T(0);
  for (int dz = 0; dz < 4; ++dz)
    for (int dy = 0; dy < 4; ++dy)
      for (int dx = 0; dx < 4; ++dx) {
        const int x = 4 * X + dx, y = 4 * Y + dy, z = 4 * Z + dz;
        const Nbr n = neighbours(x, y, z, gf);
        T f[27];
        load_pops<D3Q27, S, T, MODE>(fine, gf, n, (z * gf.ny + y) * gf.nx + x, f);
        sfor<27>([&](auto I) { acc[CI(I)] += f[CI(I)]; });
      }
  sfor<27>([&](auto I) { snap[(int64_t)CI(I) * gc.N + C] = float(acc[CI(I)] * T(1.0 / 64.0)); });
}

__global__ void __launch_bounds__(128)
    k_closure_features(const float* __restrict__ snap, Geo g, float omega_s,
                       double* __restrict__ feat) {
  const int64_t c = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= g.N) return;
  float f[27];
  sfor<27>([&](auto I) { f[CI(I)] = snap[(int64_t)CI(I) * g.N + c]; });
  CumState<float> s;
  cum_forward<float>(f, s);
  float raw[NIN];
  closure_features<float>(s.Kn, s.drho, omega_s, raw);
  for (int k = 0; k < NIN; ++k) feat[(int64_t)k * g.N + c] = raw[k];
}

// training forward, step k of the unrolled rollout: post-collision
// populations f* of every cell, from the snapshot itself (SRC_PULL false, the
// first step) or from the pull gather of the previous step's f* (the
// pre-collision state of the next step).  Written in the pull layout of the
// next step.
template <bool SRC_PULL>
__global__ void __launch_bounds__(128)
    k_closure_fwd(const float* __restrict__ fsrc, Geo g, Rates<float> keep,
                  const float* __restrict__ params, float* __restrict__ fstar) {
  __shared__ float sp[NSMEM];
  load_params(sp, params);
  const int64_t c = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= g.N) return;
  int x, y, z;
  cell_xyz(int(c), g, x, y, z);
  const Nbr n = neighbours(x, y, z, g);
  float f[27];
  load_pops<D3Q27, float, float, SRC_PULL ? G_PULL : G_LOCAL>(fsrc, g, n, int(c), f);
  CumState<float> s;
  cum_forward<float>(f, s);
  float raw[NIN], xin[NIN], h1[NH], h2[NH], om[NOUT], dom[NOUT];
  closure_features<float>(s.Kn, s.drho, 1.0f - keep.om[0], raw);
  mlp_forward<float>(sp, raw, xin, h1, h2, om, dom);
  Rates<float> k = keep;
  for (int o = 0; o < NOUT; ++o) k.om[2 + o] = 1.0f - om[o];
  float Cs[3][3][3];
  cum_backward<float>(s, k, Cs, f);
  sfor<27>([&](auto I) { fstar[(int64_t)CI(I) * g.N + c] = f[CI(I)]; });
}

// loss of one step and its adjoint seed: per cell y of the streamed state,
// r(y) = 2 wk/N (u - u_target) / rho and u(y) (6 floats, SoA), plus per-block
// partial sums of wk |u - u_target|^2 / N (wk: the step's weight, 1/K)
constexpr int LOSS_THREADS = 256;
__global__ void __launch_bounds__(LOSS_THREADS)
    k_closure_loss(const float* __restrict__ fstar, const float* __restrict__ target, Geo g,
                   float* __restrict__ r6, double* __restrict__ part, double wk) {
  __shared__ double sh[LOSS_THREADS];
  double acc = 0.0;
  const double invN = 1.0 / double(g.N);
  for (int64_t c = (int64_t)blockIdx.x * LOSS_THREADS + threadIdx.x; c < g.N;
       c += (int64_t)gridDim.x * LOSS_THREADS) {
    int x, y, z;
    cell_xyz(int(c), g, x, y, z);
    const Nbr n = neighbours(x, y, z, g);
    float f[27];
    load_pops<D3Q27, float, float, G_PULL>(fstar, g, n, int(c), f);
    double dr = 0, j[3] = {0, 0, 0}, drt = 0, jt[3] = {0, 0, 0};
    sfor<27>([&](auto I) {
      constexpr int i = CI(I);
      const double v = f[i], vt = target[(int64_t)i * g.N + c];
      dr += v;
      drt += vt;
      if constexpr (vel(D3Q27, i, 0) != 0) { j[0] += vel(D3Q27, i, 0) * v; jt[0] += vel(D3Q27, i, 0) * vt; }
      if constexpr (vel(D3Q27, i, 1) != 0) { j[1] += vel(D3Q27, i, 1) * v; jt[1] += vel(D3Q27, i, 1) * vt; }
      if constexpr (vel(D3Q27, i, 2) != 0) { j[2] += vel(D3Q27, i, 2) * v; jt[2] += vel(D3Q27, i, 2) * vt; }
    });
    const double rho = 1.0 + dr, rhot = 1.0 + drt;
    for (int d = 0; d < 3; ++d) {
      const double u = j[d] / rho, ut = jt[d] / rhot;
      acc += (u - ut) * (u - ut);
      r6[(int64_t)d * g.N + c] = float(2.0 * wk * invN * (u - ut) / rho);
      r6[(int64_t)(3 + d) * g.N + c] = float(u);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = LOSS_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0] * invN * wk;
}

__global__ void k_fold_sum(const double* __restrict__ part, int n, int stride, int width,
                           double* __restrict__ out) {
  // out[k] = sum_r part[r * stride + k] for k < width, rows in fixed order
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= width) return;
  double s = 0.0;
  for (int r = 0; r < n; ++r) s += part[(int64_t)r * stride + k];
  out[k] = s;
}

// dL/df_j of one cell through its collision: sum_i lam_i d f*_i / d f_j at
// the cell's rates held fixed, plus sum_m lraw_m d raw_m / d f_j (the path
// through the rates, lraw = dL/d raw from the network's input gradient).
// One dual-number pass per j.
__device__ __noinline__ void collision_vjp(const float (&f)[27], const Rates<float>& k,
                                           float omega_s, const float (&lam)[27],
                                           const float (&lraw)[NIN], float* out,
                                           int64_t stride) {
  Rates<Dual> kd;
#pragma unroll
  for (int q = 0; q < 6; ++q) kd.om[q] = Dual(k.om[q], 0.f);
#pragma unroll 1
  for (int j = 0; j < 27; ++j) {
    Dual fd[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) fd[i] = Dual(f[i], i == j ? 1.f : 0.f);
    CumState<Dual> sd;
    cum_forward<Dual>(fd, sd);
    Dual rawd[NIN];
    closure_features<Dual>(sd.Kn, sd.drho, Dual(omega_s, 0.f), rawd);
    Dual Csd[3][3][3];
    cum_backward<Dual>(sd, kd, Csd, fd);
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 27; ++i) acc += lam[i] * fd[i].d;
#pragma unroll
    for (int m = 0; m < NIN; ++m) acc += lraw[m] * rawd[m].d;
    out[(int64_t)j * stride] = acc;
  }
}

// training backward, step k of the unrolled rollout (the steps are taken
// from the last back to the first).  64 threads per block; every thread
// takes one cell x per round:
//   f      = f(t+k)(x), the snapshot (SRC_PULL false) or the pull gather of
//            the previous step's f*, and its collision with the network
//   lam_i  = dL/df*_i(x) = lnext_i(x + xi_i) + the seed of the velocity loss
//            of step k+1 at x + xi_i (lnext: dL/df(t+k+1), null for the
//            last step)
//   dL/domega through the tangents d f*/d omega_k, then the MLP backward;
//   every thread accumulates the products of the parameters it owns over
//   the round's 64 cells (activations and deltas staged in shared memory).
//   lout (not null): dL/df(t+k)(x) for the step before (collision_vjp).
// One partial row of NPARAM doubles per block, written or accumulated.
constexpr int BWD_THREADS = 64;
constexpr int BWD_PER_THREAD = (NPARAM + BWD_THREADS - 1) / BWD_THREADS;  // 23
template <bool SRC_PULL>
__global__ void __launch_bounds__(BWD_THREADS)
    k_closure_bwd(const float* __restrict__ fsrc, const float* __restrict__ r6,
                  const float* __restrict__ lnext, float* __restrict__ lout, Geo g,
                  Rates<float> keep, const float* __restrict__ params,
                  double* __restrict__ gpart, int accumulate) {
  __shared__ float sp[NSMEM];
  __shared__ float s_x[BWD_THREADS][NIN + 1];
  __shared__ float s_h1[BWD_THREADS][NH + 1];
  __shared__ float s_h2[BWD_THREADS][NH + 1];
  __shared__ float s_d1[BWD_THREADS][NH + 1];
  __shared__ float s_d2[BWD_THREADS][NH + 1];
  __shared__ float s_dz[BWD_THREADS][NOUT];
  load_params(sp, params);
  double acc[BWD_PER_THREAD];
  for (int k = 0; k < BWD_PER_THREAD; ++k) acc[k] = 0.0;
  const int tid = threadIdx.x;
  const float omega_s = 1.0f - keep.om[0];
  const int64_t rounds = (g.N + (int64_t)gridDim.x * BWD_THREADS - 1) / ((int64_t)gridDim.x * BWD_THREADS);
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t c = (rd * gridDim.x + blockIdx.x) * BWD_THREADS + tid;
    float xin[NIN], h1[NH], h2[NH], dz[NOUT], d1[NH], d2[NH];
    for (int i = 0; i < NIN; ++i) xin[i] = 0.f;
    for (int i = 0; i < NH; ++i) h1[i] = h2[i] = d1[i] = d2[i] = 0.f;
    for (int i = 0; i < NOUT; ++i) dz[i] = 0.f;
    if (c < g.N) {
      int x, y, z;
      cell_xyz(int(c), g, x, y, z);
      const Nbr n = neighbours(x, y, z, g);
      float f[27];
      load_pops<D3Q27, float, float, SRC_PULL ? G_PULL : G_LOCAL>(fsrc, g, n, int(c), f);
      CumState<float> s;
      cum_forward<float>(f, s);
      float raw[NIN], om[NOUT], dom[NOUT];
      closure_features<float>(s.Kn, s.drho, omega_s, raw);
      mlp_forward<float>(sp, raw, xin, h1, h2, om, dom);
      Rates<float> k = keep;
      for (int o = 0; o < NOUT; ++o) k.om[2 + o] = 1.0f - om[o];
      float Cs[3][3][3], post[27];
      cum_backward<float>(s, k, Cs, post);
      // adjoint of streaming and of the velocity: lam_i = dL/df*_i(x)
      float lam[27];
      sfor<27>([&](auto I) {
        constexpr int i = CI(I);
        const int yc = cell_at(n, g, vel(D3Q27, i, 0), vel(D3Q27, i, 1), vel(D3Q27, i, 2));
        float l = lnext ? lnext[(int64_t)i * g.N + yc] : 0.f;
        for (int d = 0; d < 3; ++d)
          l += r6[(int64_t)d * g.N + yc] *
               (float(vel(D3Q27, i, d)) - r6[(int64_t)(3 + d) * g.N + yc]);
        lam[i] = l;
      });
      float t[27], gk[NOUT];
      cum_tangent<3, float>(s, Cs, t);
      gk[0] = 0.f;
      for (int i = 0; i < 27; ++i) gk[0] += lam[i] * t[i];
      cum_tangent<4, float>(s, Cs, t);
      gk[1] = 0.f;
      for (int i = 0; i < 27; ++i) gk[1] += lam[i] * t[i];
      cum_tangent<5, float>(s, Cs, t);
      gk[2] = 0.f;
      for (int i = 0; i < 27; ++i) gk[2] += lam[i] * t[i];
      cum_tangent<6, float>(s, Cs, t);
      gk[3] = 0.f;
      for (int i = 0; i < 27; ++i) gk[3] += lam[i] * t[i];
      for (int o = 0; o < NOUT; ++o) dz[o] = gk[o] * dom[o];
      for (int j = 0; j < NH; ++j) {
        float a = 0.f;
        for (int o = 0; o < NOUT; ++o) a += sp[OW3 + o * NH + j] * dz[o];
        d2[j] = a * (1.f - h2[j] * h2[j]);
      }
      for (int i = 0; i < NH; ++i) {
        float a = 0.f;
        for (int j = 0; j < NH; ++j) a += sp[OW2 + j * NH + i] * d2[j];
        d1[i] = a * (1.f - h1[i] * h1[i]);
      }
      if (lout) {
        // the network's input gradient: x = (raw - shift) * scale
        float lraw[NIN];
        for (int m = 0; m < NIN; ++m) {
          float a = 0.f;
          for (int r = 0; r < NH; ++r) a += sp[OW1 + r * NIN + m] * d1[r];
          lraw[m] = a * sp[NPARAM + NIN + m];
        }
        collision_vjp(f, k, omega_s, lam, lraw, lout + c, g.N);
      }
    }
    for (int i = 0; i < NIN; ++i) s_x[tid][i] = xin[i];
    for (int i = 0; i < NH; ++i) {
      s_h1[tid][i] = h1[i];
      s_h2[tid][i] = h2[i];
      s_d1[tid][i] = d1[i];
      s_d2[tid][i] = d2[i];
    }
    for (int o = 0; o < NOUT; ++o) s_dz[tid][o] = dz[o];
    __syncthreads();
    for (int kk = 0; kk < BWD_PER_THREAD; ++kk) {
      const int p = tid + kk * BWD_THREADS;
      if (p >= NPARAM) break;
      float sum = 0.f;
      if (p < OB1) {
        const int r = p / NIN, cc = p % NIN;
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_d1[e][r] * s_x[e][cc];
      } else if (p < OW2) {
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_d1[e][p - OB1];
      } else if (p < OB2) {
        const int r = (p - OW2) / NH, cc = (p - OW2) % NH;
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_d2[e][r] * s_h1[e][cc];
      } else if (p < OW3) {
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_d2[e][p - OB2];
      } else if (p < OB3) {
        const int r = (p - OW3) / NH, cc = (p - OW3) % NH;
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_dz[e][r] * s_h2[e][cc];
      } else {
        for (int e = 0; e < BWD_THREADS; ++e) sum += s_dz[e][p - OB3];
      }
      acc[kk] += double(sum);
    }
    __syncthreads();
  }
  for (int kk = 0; kk < BWD_PER_THREAD; ++kk) {
    const int p = tid + kk * BWD_THREADS;
    if (p >= NPARAM) continue;
    double* dst = gpart + (int64_t)blockIdx.x * NPARAM + p;
    *dst = accumulate ? *dst + acc[kk] : acc[kk];
  }
}

__global__ void k_round_bf16(const float* __restrict__ master, float* __restrict__ rounded) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NPARAM) rounded[k] = __bfloat162float(__float2bfloat16_rn(master[k]));
}

__global__ void k_adam(float* __restrict__ master, float* __restrict__ m1, float* __restrict__ m2,
                       const double* __restrict__ grad, float* __restrict__ rounded, float lr,
                       float bc1, float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float gk = float(grad[k]);
  const float a = 0.9f * m1[k] + 0.1f * gk;
  const float b = 0.999f * m2[k] + 0.001f * gk * gk;
  m1[k] = a;
  m2[k] = b;
  const float mh = a / bc1, vh = b / bc2;
  const float w = master[k] - lr * mh / (sqrtf(vh) + 1e-8f);
  master[k] = w;
  rounded[k] = __bfloat162float(__float2bfloat16_rn(w));
}

template <class T>
struct ClosureDev {
  T p[NSMEM];
};

void launch_closure_step(const StepArgs& a, const void* closure) {
  const dim3 grid((a.g.nx + 127) / 128, a.g.ny, a.g.nz);
  if (a.storage == STORE_F64) {
    Rates<double> keep;
    for (int k = 0; k < 6; ++k) keep.om[k] = 1.0 - a.rates[k];
    k_closure_pull<double, double><<<grid, 128, 0, a.stream>>>(
        (const double*)a.src, (double*)a.dst, a.g, keep, (const double*)closure);
  } else {
    Rates<float> keep;
    for (int k = 0; k < 6; ++k) keep.om[k] = float(1.0 - a.rates[k]);
#if LBM_CLOSURE_NET == 2
    k_closure_pull_tc<<<grid, 128, 0, a.stream>>>((const float*)a.src, (float*)a.dst, a.g, keep,
                                                   (const float*)closure, a.status);
#elif LBM_CLOSURE_NET == 1
    // persistent grids: CTAs per SM x SMs, once per process and kernel
    auto resident_of = [](auto kernel) {
      int dev = 0, sms = 0, occ = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, 0) != cudaSuccess ||
          occ < 1)
        occ = 1;
      return sms * occ;
    };
    PullPtrs<float> P;
    const int64_t nx = a.g.nx, nxy = int64_t(a.g.nx) * a.g.ny;
    for (int i = 0; i < 27; ++i) {
      const int64_t delta = -(vel(D3Q27, i, 2) * nxy + vel(D3Q27, i, 1) * nx + vel(D3Q27, i, 0));
      P.src[i] = (const float*)a.src + (int64_t(i) * a.g.N + delta);
      P.dst[i] = (float*)a.dst + int64_t(i) * a.g.N;
    }
    if (a.g.nx % 2 == 0) {
      static const int resident2 = resident_of(k_closure_pull_mma2);
      const int ntiles = int((a.g.N + 255) / 256);  // N < 2^31
      k_closure_pull_mma2<<<ntiles < resident2 ? ntiles : resident2, 128, 0, a.stream>>>(
          P, a.g, keep, (const float*)closure, ntiles);
    } else {
      static const int resident = resident_of(k_closure_pull_mma);
      const int tiles_x = (a.g.nx + 127) / 128;
      const int ntiles = tiles_x * a.g.ny * a.g.nz;  // < 2^31: N < 2^31
      k_closure_pull_mma<<<ntiles < resident ? ntiles : resident, 128, 0, a.stream>>>(
          P, a.g, keep, (const float*)closure, tiles_x, ntiles);
    }
#else
    k_closure_pull<float, float><<<grid, 128, 0, a.stream>>>((const float*)a.src, (float*)a.dst,
                                                             a.g, keep, (const float*)closure);
#endif
  }
}

void free_closure(void* closure) { cudaFree(closure); }

}  // namespace lbm

// ------------------------------------------------------------ host side
namespace {

using lbm::Geo;
using lbm::NPARAM;
using lbm::NIN;

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

float bf16_bits_to_float(uint16_t h) {
  uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
uint16_t float_to_bf16_bits(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return uint16_t((u >> 16) | 0x40);
  u += 0x7fffu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}

}  // namespace

struct lbm_trainer {
  Geo g;
  double omega_s, omega_b;
  int cap, count;
  int unroll;      // K: steps of the rollout loss
  float* snaps;
  float* fstar;    // K post-collision fields, 27 N each
  float* r6;       // K loss seeds, 6 N each
  float* lam[2];   // dL/df of two consecutive steps (K > 1), 27 N each
  double* lpart;   // K rows of lblocks loss partials
  int lblocks;
  double* gpart;
  int gblocks;
  double* grad;
  double* loss;
  float* master;  // NSMEM values: params, shift, scale (shift/scale fixed)
  float* rounded;
  float* m1;
  float* m2;
  int adam_t;
  float shift[NIN], scale[NIN];
  cudaStream_t stream;
};

extern "C" {

int lbm_set_closure(lbm_ctx* c, const lbm_closure_weights* w) {
  if (!c) return LBM_ERR_INVALID;
  if (!w) {
    if (c->closure) {
      if (c->stream) cudaStreamSynchronize(c->stream);
      lbm::free_closure(c->closure);
      c->closure = nullptr;
    }
    return LBM_OK;
  }
  if (c->p.stencil != LBM_D3Q27 || c->p.space != LBM_SPACE_CUMULANT ||
      c->p.streaming != LBM_PULL ||
      (c->p.storage != LBM_STORE_F32 && c->p.storage != LBM_STORE_F64) ||
      c->p.arithmetic != LBM_ARITH_DEVIATION || c->force_mode != lbm::FORCE_NONE)
    return LBM_ERR_UNSUPPORTED;
  const bool dbl = c->p.storage == LBM_STORE_F64;
  std::vector<double> hd(lbm::NSMEM);
  for (int k = 0; k < NPARAM; ++k) {
    hd[k] = bf16_bits_to_float(w->w[k]);
    // the FP32 network's FP16 operands hold every finite weight up to 65504
    if (!(hd[k] <= 65504.0 && hd[k] >= -65504.0)) return LBM_ERR_INVALID;
  }
  for (int k = 0; k < NIN; ++k) {
    hd[NPARAM + k] = w->shift[k];
    hd[NPARAM + NIN + k] = w->scale[k];
  }
  // FP32: the float parameters, the lane table of the warp-level network,
  // then the packed B operands of the tcgen05 network
  const size_t bytes = dbl ? lbm::NSMEM * sizeof(double)
                           : size_t(lbm::TC_BOFF_BYTES) + lbm::TC_BELEMS * sizeof(uint16_t);
  static_assert(lbm::wmn::TAB_OFF_BYTES + lbm::wmn::TAB_BYTES <= lbm::TC_BOFF_BYTES, "layout");
  void* dev = nullptr;
  if (cudaMalloc(&dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  int rc;
  if (dbl) {
    rc = cuda_err(cudaMemcpy(dev, hd.data(), bytes, cudaMemcpyHostToDevice));
  } else {
    std::vector<unsigned char> img(bytes, 0);
    std::vector<float> hf(hd.begin(), hd.end());
    std::memcpy(img.data(), hf.data(), hf.size() * sizeof(float));
    lbm::pack_lane_table(hf.data(),
                         reinterpret_cast<uint32_t*>(img.data() + lbm::wmn::TAB_OFF_BYTES));
    lbm::pack_tc_weights(hf.data(),
                         reinterpret_cast<uint16_t*>(img.data() + lbm::TC_BOFF_BYTES));
    rc = cuda_err(cudaMemcpy(dev, img.data(), bytes, cudaMemcpyHostToDevice));
  }
  if (rc != LBM_OK) {
    cudaFree(dev);
    return rc;
  }
  if (c->closure) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    lbm::free_closure(c->closure);
  }
  c->closure = dev;
  return LBM_OK;
}

void lbm_trainer_destroy(lbm_trainer* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  else cudaDeviceSynchronize();
  void* ptrs[] = {t->snaps, t->fstar, t->r6, t->lam[0], t->lam[1], t->lpart, t->gpart,
                  t->grad, t->loss, t->master, t->rounded, t->m1, t->m2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete t;
}

int lbm_trainer_create(lbm_trainer** out, const int64_t dims[3], double omega_s, double omega_b,
                       int max_snapshots, void* stream) {
  if (!out || !dims || max_snapshots < 2 || !(omega_s > 0 && omega_s <= 2) ||
      !(omega_b > 0 && omega_b <= 2))
    return LBM_ERR_INVALID;
  *out = nullptr;
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > 65535) return LBM_ERR_INVALID;
  const int64_t N = dims[0] * dims[1] * dims[2];
  if (N >= (int64_t(1) << 31) || int64_t(max_snapshots) * 27 * N >= (int64_t(1) << 40))
    return LBM_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  lbm_trainer* t = new (std::nothrow) lbm_trainer();
  if (!t) return LBM_ERR_OOM;
  t->g.nx = int(dims[0]);
  t->g.ny = int(dims[1]);
  t->g.nz = int(dims[2]);
  t->g.N = N;
  t->omega_s = omega_s;
  t->omega_b = omega_b;
  t->cap = max_snapshots;
  t->unroll = 1;
  t->stream = (cudaStream_t)stream;
  const int64_t lb = (N + lbm::LOSS_THREADS - 1) / lbm::LOSS_THREADS;
  t->lblocks = int(lb < 1184 ? lb : 1184);
  const int64_t gb = (N + lbm::BWD_THREADS - 1) / lbm::BWD_THREADS;
  t->gblocks = int(gb < 1184 ? gb : 1184);
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      ok = false;
    }
  };
  alloc((void**)&t->snaps, sizeof(float) * 27 * size_t(N) * max_snapshots);
  alloc((void**)&t->fstar, sizeof(float) * 27 * size_t(N));
  alloc((void**)&t->r6, sizeof(float) * 6 * size_t(N));
  alloc((void**)&t->lpart, sizeof(double) * t->lblocks);
  alloc((void**)&t->gpart, sizeof(double) * size_t(t->gblocks) * NPARAM);
  alloc((void**)&t->grad, sizeof(double) * NPARAM);
  alloc((void**)&t->loss, sizeof(double));
  alloc((void**)&t->master, sizeof(float) * lbm::NSMEM);
  alloc((void**)&t->rounded, sizeof(float) * lbm::NSMEM);
  alloc((void**)&t->m1, sizeof(float) * NPARAM);
  alloc((void**)&t->m2, sizeof(float) * NPARAM);
  if (!ok) {
    lbm_trainer_destroy(t);
    return LBM_ERR_OOM;
  }
  std::vector<float> zeros(NPARAM, 0.f), sh(NIN, 0.f), sc(NIN, 1.f);
  int rc = lbm_trainer_set_params(t, zeros.data(), sh.data(), sc.data());
  if (rc != LBM_OK) {
    lbm_trainer_destroy(t);
    return rc;
  }
  *out = t;
  return LBM_OK;
}

int lbm_trainer_set_unroll(lbm_trainer* t, int K) {
  if (!t || K < 1 || K > LBM_CLOSURE_MAX_UNROLL || K + 1 > t->cap) return LBM_ERR_INVALID;
  if (K == t->unroll) return LBM_OK;
  if (t->stream) cudaStreamSynchronize(t->stream);
  else cudaDeviceSynchronize();
  const size_t N = size_t(t->g.N);
  float *fstar = nullptr, *r6 = nullptr, *lam0 = nullptr, *lam1 = nullptr;
  double* lpart = nullptr;
  bool ok = cudaMalloc((void**)&fstar, sizeof(float) * 27 * N * K) == cudaSuccess &&
            cudaMalloc((void**)&r6, sizeof(float) * 6 * N * K) == cudaSuccess &&
            cudaMalloc((void**)&lpart, sizeof(double) * size_t(t->lblocks) * K) == cudaSuccess;
  if (ok && K > 1)
    ok = cudaMalloc((void**)&lam0, sizeof(float) * 27 * N) == cudaSuccess &&
         cudaMalloc((void**)&lam1, sizeof(float) * 27 * N) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    void* ptrs[] = {fstar, r6, lpart, lam0, lam1};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    return LBM_ERR_OOM;  // the trainer keeps its previous unroll
  }
  void* old[] = {t->fstar, t->r6, t->lpart, t->lam[0], t->lam[1]};
  for (void* p : old)
    if (p) cudaFree(p);
  t->fstar = fstar;
  t->r6 = r6;
  t->lpart = lpart;
  t->lam[0] = lam0;
  t->lam[1] = lam1;
  t->unroll = K;
  return LBM_OK;
}

int lbm_trainer_set_params(lbm_trainer* t, const float* params, const float shift[7],
                           const float scale[7]) {
  if (!t || !params || !shift || !scale) return LBM_ERR_INVALID;
  std::vector<float> h(lbm::NSMEM), hr(lbm::NSMEM);
  for (int k = 0; k < NPARAM; ++k) {
    h[k] = params[k];
    hr[k] = bf16_bits_to_float(float_to_bf16_bits(params[k]));
  }
  for (int k = 0; k < NIN; ++k) {
    h[NPARAM + k] = hr[NPARAM + k] = shift[k];
    h[NPARAM + NIN + k] = hr[NPARAM + NIN + k] = scale[k];
    t->shift[k] = shift[k];
    t->scale[k] = scale[k];
  }
  int rc = cuda_err(cudaMemcpy(t->master, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice));
  if (rc == LBM_OK)
    rc = cuda_err(cudaMemcpy(t->rounded, hr.data(), sizeof(float) * hr.size(), cudaMemcpyHostToDevice));
  if (rc == LBM_OK) rc = cuda_err(cudaMemset(t->m1, 0, sizeof(float) * NPARAM));
  if (rc == LBM_OK) rc = cuda_err(cudaMemset(t->m2, 0, sizeof(float) * NPARAM));
  t->adam_t = 0;
  return rc;
}

int lbm_trainer_get_params(lbm_trainer* t, float* params) {
  if (!t || !params) return LBM_ERR_INVALID;
  if (t->stream) cudaStreamSynchronize(t->stream);
  return cuda_err(cudaMemcpy(params, t->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
}

int lbm_trainer_snapshot_count(const lbm_trainer* t) { return t ? t->count : LBM_ERR_INVALID; }

int lbm_trainer_add_restricted(lbm_trainer* t, lbm_ctx* fine) {
  if (!t || !fine || t->count >= t->cap) return LBM_ERR_INVALID;
  if (fine->p.stencil != LBM_D3Q27 || fine->g.nx != 4 * t->g.nx || fine->g.ny != 4 * t->g.ny ||
      fine->g.nz != 4 * t->g.nz || fine->p.storage > LBM_STORE_BF16_DELTA)
    return LBM_ERR_INVALID;
  if (fine->p.streaming != LBM_PULL && fine->p.streaming != LBM_AA) return LBM_ERR_UNSUPPORTED;
  const int mode = fine->p.streaming == LBM_PULL ? lbm::G_PULL
                                                 : (fine->parity ? lbm::G_AAODD : lbm::G_LOCAL);
  const void* buf = fine->p.streaming == LBM_PULL ? fine->buf[fine->cur] : fine->buf[0];
  float* snap = t->snaps + size_t(t->count) * 27 * t->g.N;
  const int blocks = int((t->g.N + 127) / 128);
  cudaStream_t s = fine->stream;
#define LBM_RESTRICT(S, T)                                                                       \
  if (mode == lbm::G_PULL)                                                                       \
    lbm::k_restrict<S, T, lbm::G_PULL><<<blocks, 128, 0, s>>>((const S*)buf, fine->g, snap, t->g); \
  else if (mode == lbm::G_LOCAL)                                                                 \
    lbm::k_restrict<S, T, lbm::G_LOCAL><<<blocks, 128, 0, s>>>((const S*)buf, fine->g, snap, t->g); \
  else                                                                                           \
    lbm::k_restrict<S, T, lbm::G_AAODD><<<blocks, 128, 0, s>>>((const S*)buf, fine->g, snap, t->g);
  switch (fine->p.storage) {
    case LBM_STORE_F64: LBM_RESTRICT(double, double) break;
    case LBM_STORE_F32: LBM_RESTRICT(float, float) break;
    case LBM_STORE_F16_DELTA: LBM_RESTRICT(__half, float) break;
    default: LBM_RESTRICT(__nv_bfloat16, float) break;
  }
#undef LBM_RESTRICT
  int rc = cuda_err(cudaGetLastError());
  if (rc == LBM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = LBM_ERR_CUDA;
  if (rc == LBM_OK) t->count++;
  return rc;
}

int lbm_trainer_add_snapshot(lbm_trainer* t, const double* df, int on_device) {
  if (!t || !df || t->count >= t->cap) return LBM_ERR_INVALID;
  const size_t n = 27 * size_t(t->g.N);
  std::vector<double> h;
  const double* src = df;
  if (on_device) {
    h.resize(n);
    if (cudaMemcpy(h.data(), df, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return LBM_ERR_CUDA;
    src = h.data();
  }
  std::vector<float> f(src, src + n);
  int rc = cuda_err(cudaMemcpy(t->snaps + size_t(t->count) * n, f.data(), n * sizeof(float),
                               cudaMemcpyHostToDevice));
  if (rc == LBM_OK) t->count++;
  return rc;
}

int lbm_trainer_get_snapshot(lbm_trainer* t, int s, double* df, int on_device) {
  if (!t || !df || s < 0 || s >= t->count) return LBM_ERR_INVALID;
  const size_t n = 27 * size_t(t->g.N);
  std::vector<float> f(n);
  if (t->stream) cudaStreamSynchronize(t->stream);
  if (cudaMemcpy(f.data(), t->snaps + size_t(s) * n, n * sizeof(float), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return LBM_ERR_CUDA;
  std::vector<double> d(f.begin(), f.end());
  return cuda_err(cudaMemcpy(df, d.data(), n * sizeof(double),
                             on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
}

int lbm_trainer_features(lbm_trainer* t, int s, double* feat, int on_device) {
  if (!t || !feat || s < 0 || s >= t->count) return LBM_ERR_INVALID;
  const size_t n = size_t(NIN) * t->g.N;
  double* dev = feat;
  if (!on_device && cudaMalloc((void**)&dev, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  const int blocks = int((t->g.N + 127) / 128);
  lbm::k_closure_features<<<blocks, 128, 0, t->stream>>>(t->snaps + size_t(s) * 27 * t->g.N, t->g,
                                                         float(t->omega_s), dev);
  int rc = cuda_err(cudaGetLastError());
  if (!on_device) {
    if (rc == LBM_OK)
      rc = cuda_err(cudaMemcpyAsync(feat, dev, n * sizeof(double), cudaMemcpyDeviceToHost, t->stream));
    if (cudaStreamSynchronize(t->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    cudaFree(dev);
  }
  return rc;
}

static int enqueue_loss_grad(lbm_trainer* t, int s) {
  lbm::Rates<float> keep;
  keep.om[0] = float(1.0 - t->omega_s);
  keep.om[1] = float(1.0 - t->omega_b);
  for (int k = 2; k < 6; ++k) keep.om[k] = 0.f;
  const int K = t->unroll;
  const size_t n = 27 * size_t(t->g.N);
  const float* snap = t->snaps + size_t(s) * n;
  const int blocks = int((t->g.N + 127) / 128);
  auto fst = [&](int k) { return t->fstar + size_t(k) * n; };
  auto r6k = [&](int k) { return t->r6 + size_t(k) * 6 * t->g.N; };
  // forward: K learned-rate steps from snapshot s, the loss of each against
  // snapshot s + k + 1 with weight 1/K
  for (int k = 0; k < K; ++k) {
    if (k == 0)
      lbm::k_closure_fwd<false><<<blocks, 128, 0, t->stream>>>(snap, t->g, keep, t->rounded, fst(0));
    else
      lbm::k_closure_fwd<true><<<blocks, 128, 0, t->stream>>>(fst(k - 1), t->g, keep, t->rounded,
                                                              fst(k));
    lbm::k_closure_loss<<<t->lblocks, lbm::LOSS_THREADS, 0, t->stream>>>(
        fst(k), snap + size_t(k + 1) * n, t->g, r6k(k), t->lpart + size_t(k) * t->lblocks,
        1.0 / K);
  }
  lbm::k_fold_sum<<<1, 32, 0, t->stream>>>(t->lpart, t->lblocks * K, 1, 1, t->loss);
  // backward: the steps from the last to the first; dL/df of the state a
  // step starts from goes to the step before it
  for (int k = K - 1; k >= 0; --k) {
    const float* lnext = k == K - 1 ? nullptr : t->lam[(k + 1) & 1];
    float* lout = k == 0 ? nullptr : t->lam[k & 1];
    const int acc = k != K - 1;
    if (k == 0)
      lbm::k_closure_bwd<false><<<t->gblocks, lbm::BWD_THREADS, 0, t->stream>>>(
          snap, r6k(0), lnext, lout, t->g, keep, t->rounded, t->gpart, acc);
    else
      lbm::k_closure_bwd<true><<<t->gblocks, lbm::BWD_THREADS, 0, t->stream>>>(
          fst(k - 1), r6k(k), lnext, lout, t->g, keep, t->rounded, t->gpart, acc);
  }
  lbm::k_fold_sum<<<(NPARAM + 127) / 128, 128, 0, t->stream>>>(t->gpart, t->gblocks, NPARAM,
                                                                NPARAM, t->grad);
  return cuda_err(cudaGetLastError());
}

int lbm_trainer_loss_grad(lbm_trainer* t, int s, double* loss, double* grad) {
  if (!t || s < 0 || s + t->unroll >= t->count) return LBM_ERR_INVALID;
  int rc = enqueue_loss_grad(t, s);
  if (rc == LBM_OK && loss)
    rc = cuda_err(cudaMemcpyAsync(loss, t->loss, sizeof(double), cudaMemcpyDeviceToHost, t->stream));
  if (rc == LBM_OK && grad)
    rc = cuda_err(cudaMemcpyAsync(grad, t->grad, sizeof(double) * NPARAM, cudaMemcpyDeviceToHost,
                                  t->stream));
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  return rc;
}

int lbm_trainer_adam_step(lbm_trainer* t, int s, double lr, double* loss) {
  if (!t || s < 0 || s + t->unroll >= t->count || !(lr > 0)) return LBM_ERR_INVALID;
  int rc = enqueue_loss_grad(t, s);
  if (rc != LBM_OK) return rc;
  t->adam_t++;
  const float bc1 = float(1.0 - std::pow(0.9, t->adam_t));
  const float bc2 = float(1.0 - std::pow(0.999, t->adam_t));
  lbm::k_adam<<<(NPARAM + 127) / 128, 128, 0, t->stream>>>(t->master, t->m1, t->m2, t->grad,
                                                            t->rounded, float(lr), bc1, bc2);
  rc = cuda_err(cudaGetLastError());
  if (rc == LBM_OK && loss)
    rc = cuda_err(cudaMemcpyAsync(loss, t->loss, sizeof(double), cudaMemcpyDeviceToHost, t->stream));
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  return rc;
}

int lbm_trainer_export(lbm_trainer* t, lbm_closure_weights* out) {
  if (!t || !out) return LBM_ERR_INVALID;
  std::vector<float> p(NPARAM);
  int rc = lbm_trainer_get_params(t, p.data());
  if (rc != LBM_OK) return rc;
  for (int k = 0; k < NPARAM; ++k) out->w[k] = float_to_bf16_bits(p[k]);
  for (int k = 0; k < NIN; ++k) {
    out->shift[k] = t->shift[k];
    out->scale[k] = t->scale[k];
  }
  return LBM_OK;
}

}  // extern "C"
