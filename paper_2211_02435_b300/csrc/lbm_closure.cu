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

// FP32 inference network: tensor cores (1) or CUDA cores (0); a compile-time
// choice, measured on B300
#ifndef LBM_CLOSURE_TC
#define LBM_CLOSURE_TC 0
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
    ok = ok && isfinite(x[i]);
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
// (Pi = kappa_2/rho - I/3) and the density deviation
template <class T>
LBM_D void closure_features(const T (&K)[3][3][3], T drho, T omega_s, T (&raw)[NIN]) {
  const T a = K[2][0][0], b = K[0][2][0], c = K[0][0][2];
  const T p = K[1][1][0], q = K[1][0][1], r = K[0][1][1];
  const T s = T(-1.5) * omega_s;
  const T trP = a + b + c;
  const T i2P = a * b + b * c + c * a - p * p - q * q - r * r;
  const T detP = a * (b * c - r * r) - p * (p * c - r * q) + q * (p * r - b * q);
  const T t3 = trP * T(1.0 / 3.0);
  const T da = a - t3, db = b - t3, dc = c - t3;
  raw[0] = s * trP;
  raw[1] = s * s * i2P;
  raw[2] = s * s * s * detP;
  raw[3] = da * db + db * dc + dc * da - p * p - q * q - r * r;
  raw[4] = da * (db * dc - r * r) - p * (p * dc - r * q) + q * (p * r - db * q);
  raw[5] = sqrt_t(a * a + b * b + c * c + T(2) * (p * p + q * q + r * r));
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
constexpr int TC_BOFF_BYTES = ((NSMEM * 4 + 127) / 128) * 128;  // packed B after the floats
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
      ok = ok && isfinite(xin[i]);
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

// training forward: post-collision populations f* of every cell of a
// canonical snapshot (the pull layout of the next step)
__global__ void __launch_bounds__(128)
    k_closure_fwd(const float* __restrict__ snap, Geo g, Rates<float> keep,
                  const float* __restrict__ params, float* __restrict__ fstar) {
  __shared__ float sp[NSMEM];
  load_params(sp, params);
  const int64_t c = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (c >= g.N) return;
  float f[27];
  sfor<27>([&](auto I) { f[CI(I)] = snap[(int64_t)CI(I) * g.N + c]; });
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

// loss of one step and the adjoint seed: per cell y of the streamed state,
// r(y) = 2/N (u - u_target) / rho and u(y) (6 floats, SoA), plus per-block
// partial sums of |u - u_target|^2
constexpr int LOSS_THREADS = 256;
__global__ void __launch_bounds__(LOSS_THREADS)
    k_closure_loss(const float* __restrict__ fstar, const float* __restrict__ target, Geo g,
                   float* __restrict__ r6, double* __restrict__ part) {
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
      r6[(int64_t)d * g.N + c] = float(2.0 * invN * (u - ut) / rho);
      r6[(int64_t)(3 + d) * g.N + c] = float(u);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = LOSS_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0] * invN;
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

// training backward.  64 threads per block; every thread takes one cell
// per round, computes dL/domega through the tangents and the MLP backward,
// stages its activations and deltas in shared memory, then each thread
// accumulates the products of the parameters it owns over the round's 64
// cells.  One partial row of NPARAM doubles per block.
constexpr int BWD_THREADS = 64;
constexpr int BWD_PER_THREAD = (NPARAM + BWD_THREADS - 1) / BWD_THREADS;  // 23
__global__ void __launch_bounds__(BWD_THREADS)
    k_closure_bwd(const float* __restrict__ snap, const float* __restrict__ r6, Geo g,
                  Rates<float> keep, const float* __restrict__ params,
                  double* __restrict__ gpart) {
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
  const int64_t rounds = (g.N + (int64_t)gridDim.x * BWD_THREADS - 1) / ((int64_t)gridDim.x * BWD_THREADS);
  for (int64_t rd = 0; rd < rounds; ++rd) {
    const int64_t c = (rd * gridDim.x + blockIdx.x) * BWD_THREADS + tid;
    float xin[NIN], h1[NH], h2[NH], dz[NOUT], d1[NH], d2[NH];
    for (int i = 0; i < NIN; ++i) xin[i] = 0.f;
    for (int i = 0; i < NH; ++i) h1[i] = h2[i] = d1[i] = d2[i] = 0.f;
    for (int i = 0; i < NOUT; ++i) dz[i] = 0.f;
    if (c < g.N) {
      float f[27];
      sfor<27>([&](auto I) { f[CI(I)] = snap[(int64_t)CI(I) * g.N + c]; });
      CumState<float> s;
      cum_forward<float>(f, s);
      float raw[NIN], om[NOUT], dom[NOUT];
      closure_features<float>(s.Kn, s.drho, 1.0f - keep.om[0], raw);
      mlp_forward<float>(sp, raw, xin, h1, h2, om, dom);
      Rates<float> k = keep;
      for (int o = 0; o < NOUT; ++o) k.om[2 + o] = 1.0f - om[o];
      float Cs[3][3][3], post[27];
      cum_backward<float>(s, k, Cs, post);
      // adjoint of streaming and of the velocity: lambda_i = dL/df*_i(x)
      int x, y, z;
      cell_xyz(int(c), g, x, y, z);
      const Nbr n = neighbours(x, y, z, g);
      float lam[27];
      sfor<27>([&](auto I) {
        constexpr int i = CI(I);
        const int yc = cell_at(n, g, vel(D3Q27, i, 0), vel(D3Q27, i, 1), vel(D3Q27, i, 2));
        float l = 0.f;
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
    if (p < NPARAM) gpart[(int64_t)blockIdx.x * NPARAM + p] = acc[kk];
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
#if LBM_CLOSURE_TC
    k_closure_pull_tc<<<grid, 128, 0, a.stream>>>((const float*)a.src, (float*)a.dst, a.g, keep,
                                                   (const float*)closure, a.status);
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
  float* snaps;
  float* fstar;
  float* r6;
  double* lpart;
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
  for (int k = 0; k < NPARAM; ++k) hd[k] = bf16_bits_to_float(w->w[k]);
  for (int k = 0; k < NIN; ++k) {
    hd[NPARAM + k] = w->shift[k];
    hd[NPARAM + NIN + k] = w->scale[k];
  }
  // FP32: the float parameters, then the packed tensor-core B operands
  const size_t bytes = dbl ? lbm::NSMEM * sizeof(double)
                           : size_t(lbm::TC_BOFF_BYTES) + lbm::TC_BELEMS * sizeof(uint16_t);
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
  void* ptrs[] = {t->snaps, t->fstar, t->r6, t->lpart, t->gpart, t->grad, t->loss,
                  t->master, t->rounded, t->m1, t->m2};
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
  const size_t n = 27 * size_t(t->g.N);
  const float* snap = t->snaps + size_t(s) * n;
  const float* target = snap + n;
  const int blocks = int((t->g.N + 127) / 128);
  lbm::k_closure_fwd<<<blocks, 128, 0, t->stream>>>(snap, t->g, keep, t->rounded, t->fstar);
  lbm::k_closure_loss<<<t->lblocks, lbm::LOSS_THREADS, 0, t->stream>>>(t->fstar, target, t->g,
                                                                       t->r6, t->lpart);
  lbm::k_fold_sum<<<1, 32, 0, t->stream>>>(t->lpart, t->lblocks, 1, 1, t->loss);
  lbm::k_closure_bwd<<<t->gblocks, lbm::BWD_THREADS, 0, t->stream>>>(snap, t->r6, t->g, keep,
                                                                     t->rounded, t->gpart);
  lbm::k_fold_sum<<<(NPARAM + 127) / 128, 128, 0, t->stream>>>(t->gpart, t->gblocks, NPARAM,
                                                                NPARAM, t->grad);
  return cuda_err(cudaGetLastError());
}

int lbm_trainer_loss_grad(lbm_trainer* t, int s, double* loss, double* grad) {
  if (!t || s < 0 || s + 1 >= t->count) return LBM_ERR_INVALID;
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
  if (!t || s < 0 || s + 1 >= t->count || !(lr > 0)) return LBM_ERR_INVALID;
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
