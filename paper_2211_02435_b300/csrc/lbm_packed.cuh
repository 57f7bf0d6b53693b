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

// four cells (x .. x+3) as two packed pairs; every operation is the P2
// operation on each pair, so each lane computes exactly what P2 (and the
// scalar FP32 path) computes
struct P4 {
  P2 l, h;
  P4() = default;
  P2F P4(P2 a, P2 b) : l(a), h(b) {}
  P2F explicit P4(double s) : l(s), h(s) {}
  P2F explicit P4(float s) : l(s), h(s) {}
  P2F explicit P4(int s) : l(s), h(s) {}
};
struct M4 {  // lazy product
  M2 l, h;
  P2F operator P4() const { return P4(P2(l), P2(h)); }
};
P2F P4 neg(P4 x) { return P4(neg(x.l), neg(x.h)); }
P2F P4 operator-(P4 x) { return neg(x); }
P2F M4 operator-(M4 m) { return M4{-m.l, -m.h}; }
P2F P4 operator+(P4 a, P4 b) { return P4(a.l + b.l, a.h + b.h); }
P2F P4 operator-(P4 a, P4 b) { return P4(a.l - b.l, a.h - b.h); }
P2F M4 operator*(P4 a, P4 b) { return M4{a.l * b.l, a.h * b.h}; }
P2F P4 operator+(M4 m, P4 c) { return P4(m.l + c.l, m.h + c.h); }
P2F P4 operator+(P4 c, M4 m) { return P4(c.l + m.l, c.h + m.h); }
P2F P4 operator-(M4 m, P4 c) { return P4(m.l - c.l, m.h - c.h); }
P2F P4 operator-(P4 c, M4 m) { return P4(c.l - m.l, c.h - m.h); }
P2F P4 operator+(M4 x, M4 y) { return P4(x.l + y.l, x.h + y.h); }
P2F P4 operator-(M4 x, M4 y) { return P4(x.l - y.l, x.h - y.h); }
P2F M4 operator*(M4 m, P4 b) { return M4{m.l * b.l, m.h * b.h}; }
P2F M4 operator*(P4 a, M4 m) { return M4{a.l * m.l, a.h * m.h}; }
P2F M4 operator*(M4 x, M4 y) { return M4{x.l * y.l, x.h * y.h}; }
P2F P4& operator+=(P4& a, P4 b) { return a = a + b; }
P2F P4& operator+=(P4& a, M4 b) { return a = a + b; }
P2F P4& operator-=(P4& a, P4 b) { return a = a - b; }
P2F P4& operator-=(P4& a, M4 b) { return a = a - b; }
P2F P4& operator*=(P4& a, P4 b) { return a = P4(a * b); }
P2F P4 rcp(P4 x) { return P4(rcp(x.l), rcp(x.h)); }

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

// the same for BF16: b * 2^-E in one mixed-precision multiply-add (BF16
// operands, exact product); equal, bit for bit, to the widening followed by
// the power-of-two multiply, in one FMA-pipe instruction and no shifts
template <int E>
P2F float b2f_scaled(__nv_bfloat16 b) {
#ifdef __CUDA_ARCH__
  static_assert(E >= 0 && E <= 126, "2^-E must be a normal BF16 number");
  float r;
  asm("fma.rn.f32.bf16 %0, %1, %2, %3;"
      : "=f"(r)
      : "h"(__bfloat16_as_ushort(b)), "h"((unsigned short)((127 - E) << 7)), "f"(-0.0f));
  return r;
#else
  return __bfloat162float(b) / float(1u << E);
#endif
}

template <>
struct Pack<__half> {
  // four cells (x .. x+3, Nx % 4 == 0): the aligned quad at p, times 2^-E
  template <int E>
  P2F static P4 load4s(const __half* p) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __half2 a = *reinterpret_cast<const __half2*>(&w.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&w.y);
    return P4(P2(make_float2(h2f_scaled<E>(__low2half(a)), h2f_scaled<E>(__high2half(a)))),
              P2(make_float2(h2f_scaled<E>(__low2half(b)), h2f_scaled<E>(__high2half(b)))));
  }
  // (e, q0, q1, q2): the element at pe and the first three of the quad at p
  template <int E>
  P2F static P4 load1_3s(const __half* pe, const __half* p) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __half2 a = *reinterpret_cast<const __half2*>(&w.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&w.y);
    return P4(P2(make_float2(h2f_scaled<E>(*pe), h2f_scaled<E>(__low2half(a)))),
              P2(make_float2(h2f_scaled<E>(__high2half(a)), h2f_scaled<E>(__low2half(b)))));
  }
  // (q1, q2, q3, e): the last three of the quad at p and the element at pe
  template <int E>
  P2F static P4 load3_1s(const __half* p, const __half* pe) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __half2 a = *reinterpret_cast<const __half2*>(&w.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&w.y);
    return P4(P2(make_float2(h2f_scaled<E>(__high2half(a)), h2f_scaled<E>(__low2half(b)))),
              P2(make_float2(h2f_scaled<E>(__high2half(b)), h2f_scaled<E>(*pe))));
  }
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
  // four cells (x .. x+3, Nx % 4 == 0): the aligned quad at p, times 2^-E
  template <int E>
  P2F static P4 load4s(const __nv_bfloat16* p) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
    return P4(P2(make_float2(b2f_scaled<E>(__low2bfloat16(a)), b2f_scaled<E>(__high2bfloat16(a)))),
              P2(make_float2(b2f_scaled<E>(__low2bfloat16(b)), b2f_scaled<E>(__high2bfloat16(b)))));
  }
  // (e, q0, q1, q2): the element at pe and the first three of the quad at p
  template <int E>
  P2F static P4 load1_3s(const __nv_bfloat16* pe, const __nv_bfloat16* p) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
    return P4(P2(make_float2(b2f_scaled<E>(*pe), b2f_scaled<E>(__low2bfloat16(a)))),
              P2(make_float2(b2f_scaled<E>(__high2bfloat16(a)), b2f_scaled<E>(__low2bfloat16(b)))));
  }
  // (q1, q2, q3, e): the last three of the quad at p and the element at pe
  template <int E>
  P2F static P4 load3_1s(const __nv_bfloat16* p, const __nv_bfloat16* pe) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
    return P4(P2(make_float2(b2f_scaled<E>(__high2bfloat16(a)), b2f_scaled<E>(__low2bfloat16(b)))),
              P2(make_float2(b2f_scaled<E>(__high2bfloat16(b)), b2f_scaled<E>(*pe))));
  }
  // the same values times 2^-E (the decode of the per-direction scale)
  template <int E>
  P2F static P2 load2s(const __nv_bfloat16* p) {
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(p);
    return P2(make_float2(b2f_scaled<E>(__low2bfloat16(h)), b2f_scaled<E>(__high2bfloat16(h))));
  }
  template <int E>
  P2F static P2 load11s(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
    return P2(make_float2(b2f_scaled<E>(*p0), b2f_scaled<E>(*p1)));
  }
  P2F static void store2(__nv_bfloat16* p, P2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
  }
  P2F static void store11(__nv_bfloat16* p0, __nv_bfloat16* p1, P2 v) {
    *p0 = __float2bfloat16_rn(v.v.x);
    *p1 = __float2bfloat16_rn(v.v.y);
  }
};

// four cells' stores (the same rounding as store2 / store11): the aligned
// quad at p; and the two shifted forms, whose four elements straddle a quad
// boundary: one element apart (at pe, possibly wrapped), an aligned pair and
// one more element
template <class S>
P2F void store4(S* p, P4 v) {
  uint2 w;
  Pack<S>::store2(reinterpret_cast<S*>(&w.x), v.l);
  Pack<S>::store2(reinterpret_cast<S*>(&w.y), v.h);
  *reinterpret_cast<uint2*>(p) = w;
}
// (v0 -> pe, v1 v2 -> p[0..1], v3 -> p[2])
template <class S>
P2F void store1_3(S* pe, S* p, P4 v) {
  Pack<S>::store11(pe, p + 2, P2(make_float2(v.l.v.x, v.h.v.y)));
  Pack<S>::store2(p, P2(make_float2(v.l.v.y, v.h.v.x)));
}
// (v0 -> p[1], v1 v2 -> p[2..3], v3 -> pe)
template <class S>
P2F void store3_1(S* p, S* pe, P4 v) {
  Pack<S>::store11(p + 1, pe, P2(make_float2(v.l.v.x, v.h.v.y)));
  Pack<S>::store2(p + 2, P2(make_float2(v.l.v.y, v.h.v.x)));
}

}  // namespace lbm
