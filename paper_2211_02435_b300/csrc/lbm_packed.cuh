// lbm_packed.cuh -- a packed pair of FP32 values for the two-cells-per-thread
// step kernels of the FP16/BF16 storage forms.  Blackwell executes
// add / multiply / fused multiply-add on float2 operands as one instruction
// (__fadd2_rn, __fmul2_rn, __ffma2_rn), so running the per-cell collision on
// P2 values halves its arithmetic instruction count per cell.
//
// A product is kept lazy (M2) so that `a * b + c` is emitted as one fused
// multiply-add, as the scalar compiler would contract it; each component is
// rounded exactly like an FP32 fused multiply-add.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

#define P2F __host__ __device__ __forceinline__

P2F float2 fadd2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
P2F float2 fmul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
P2F float2 ffma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(a, b, c);
#else
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

struct P2 {
  float2 v;
  P2() = default;
  P2F P2(float2 a) : v(a) {}
  P2F explicit P2(double s) : v(make_float2(float(s), float(s))) {}
  P2F explicit P2(float s) : v(make_float2(s, s)) {}
  P2F explicit P2(int s) : v(make_float2(float(s), float(s))) {}
};

struct M2 {  // lazy product a * b
  P2 a, b;
  P2F operator P2() const { return P2(fmul2(a.v, b.v)); }
};

P2F P2 neg(P2 x) { return P2(make_float2(-x.v.x, -x.v.y)); }
P2F P2 operator-(P2 x) { return neg(x); }
P2F M2 operator-(M2 m) { return M2{neg(m.a), m.b}; }

P2F P2 operator+(P2 a, P2 b) { return P2(fadd2(a.v, b.v)); }
P2F P2 operator-(P2 a, P2 b) { return P2(fadd2(a.v, neg(b).v)); }
P2F M2 operator*(P2 a, P2 b) { return M2{a, b}; }

P2F P2 operator+(M2 m, P2 c) { return P2(ffma2(m.a.v, m.b.v, c.v)); }
P2F P2 operator+(P2 c, M2 m) { return P2(ffma2(m.a.v, m.b.v, c.v)); }
P2F P2 operator-(M2 m, P2 c) { return P2(ffma2(m.a.v, m.b.v, neg(c).v)); }
P2F P2 operator-(P2 c, M2 m) { return P2(ffma2(neg(m.a).v, m.b.v, c.v)); }
P2F P2 operator+(M2 x, M2 y) { return x + P2(y); }
P2F P2 operator-(M2 x, M2 y) { return x - P2(y); }
P2F M2 operator*(M2 m, P2 b) { return M2{P2(m), b}; }
P2F M2 operator*(P2 a, M2 m) { return M2{a, P2(m)}; }
P2F M2 operator*(M2 x, M2 y) { return M2{P2(x), P2(y)}; }

P2F P2& operator+=(P2& a, P2 b) { return a = a + b; }
P2F P2& operator+=(P2& a, M2 b) { return a = a + b; }
P2F P2& operator-=(P2& a, P2 b) { return a = a - b; }
P2F P2& operator-=(P2& a, M2 b) { return a = a - b; }
P2F P2& operator*=(P2& a, P2 b) { return a = P2(a * b); }

P2F P2 rcp(P2 x) {
#ifdef __CUDA_ARCH__
  return P2(make_float2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)));
#else
  return P2(make_float2(1.0f / x.v.x, 1.0f / x.v.y));
#endif
}

// two cells' packed values of one population plane (x and x+1)
template <class S>
struct Pack;
// h * 2^-E as FP32 in one mixed-precision multiply-add (FP16 operands, FP32
// result: the product is exact); adding -0 keeps the sign of a zero, so the
// result equals the conversion followed by the power-of-two multiply bit
// for bit
template <int E>
P2F float h2f_scaled(__half h) {
#ifdef __CUDA_ARCH__
  static_assert(E >= 0 && E <= 14, "2^-E must be a normal FP16 number");
  float r;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;"
      : "=f"(r)
      : "h"(__half_as_ushort(h)), "h"((unsigned short)((15 - E) << 10)), "f"(-0.0f));
  return r;
#else
  return __half2float(h) / float(1u << E);
#endif
}

template <>
struct Pack<__half> {
  P2F static P2 load2(const __half* p) {
    return P2(__half22float2(*reinterpret_cast<const __half2*>(p)));
  }
  P2F static P2 load11(const __half* p0, const __half* p1) {
    return P2(make_float2(__half2float(*p0), __half2float(*p1)));
  }
  // the same values times 2^-E (the decode of the per-direction scale)
  template <int E>
  P2F static P2 load2s(const __half* p) {
    const __half2 h = *reinterpret_cast<const __half2*>(p);
    return P2(make_float2(h2f_scaled<E>(__low2half(h)), h2f_scaled<E>(__high2half(h))));
  }
  template <int E>
  P2F static P2 load11s(const __half* p0, const __half* p1) {
    return P2(make_float2(h2f_scaled<E>(*p0), h2f_scaled<E>(*p1)));
  }
  P2F static void store2(__half* p, P2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v);
  }
  P2F static void store11(__half* p0, __half* p1, P2 v) {
    *p0 = __float2half_rn(v.v.x);
    *p1 = __float2half_rn(v.v.y);
  }
};
template <>
struct Pack<__nv_bfloat16> {
  P2F static P2 load2(const __nv_bfloat16* p) {
    return P2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  P2F static P2 load11(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
    return P2(make_float2(__bfloat162float(*p0), __bfloat162float(*p1)));
  }
  // BF16 widens by a shift (not on the FMA pipe), so the scale stays a
  // separate packed multiply
  template <int E>
  P2F static P2 load2s(const __nv_bfloat16* p) {
    return load2(p) * P2(1.0f / float(1u << E));
  }
  template <int E>
  P2F static P2 load11s(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
    return load11(p0, p1) * P2(1.0f / float(1u << E));
  }
  P2F static void store2(__nv_bfloat16* p, P2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
  }
  P2F static void store11(__nv_bfloat16* p0, __nv_bfloat16* p1, P2 v) {
    *p0 = __float2bfloat16_rn(v.v.x);
    *p1 = __float2bfloat16_rn(v.v.y);
  }
};

}  // namespace lbm
