// lbm_kernels.cuh -- CUDA kernels of the fused stream + collide step and
// its read-out / set-up kernels, templated over stencil, storage type,
// collision space and streaming pattern.  Included by lbm_inst.cu, which
// instantiates the launchers declared in lbm_internal.h.
//
// Data layout in HBM: one structure-of-arrays buffer per population set,
// buf[i * N + c] with c = (z * Ny + y) * Nx + x (x fastest), so a warp of
// 32 consecutive x reads 32 consecutive elements of each population plane.
// One thread updates one cell; a block covers LBM_BX consecutive x of one
// (y, z) row (LBM_PULL_BX for the pull step kernel); the grid is
// (ceil(Nx / block), Ny, Nz).
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_packed.cuh"
#include "lbm_staged.cuh"

namespace lbm {

#ifndef LBM_BX
#define LBM_BX 128
#endif
// block of the scalar pull step kernel k_pull: measured on B300 at 512^3
// (D3Q27 cumulant FP32) 31.58 GLUPS with 256 threads against 31.11 with 128
// and 31.17 with 64; the other kernels keep LBM_BX (the in-place patterns
// split between the two sizes, the packed FP16 / BF16 kernel lost 1.4 %)
#ifndef LBM_PULL_BX
#define LBM_PULL_BX 256
#endif
// minimum resident CTAs per SM asked of the packed FP16 / BF16 step kernel
// (a compile-time tuning knob; 0 leaves the register budget to the compiler,
// which measured fastest on B300: 7 -> -1 %, 8 -> -5 %, 1 -> -8 %)
#ifndef LBM_PULL2_MINB
#define LBM_PULL2_MINB 0
#endif
#if LBM_PULL2_MINB > 0
#define LBM_PULL2_BOUNDS __launch_bounds__(LBM_BX, LBM_PULL2_MINB)
#else
#define LBM_PULL2_BOUNDS __launch_bounds__(LBM_BX)
#endif
// the same for the four-cells-per-thread kernels (k_pull4, k_inplace4):
// left to the compiler they take 130 .. 164 registers, three CTAs per SM;
// four CTAs (128 registers, at most 36 bytes of spills) measured at 512^3
// FP16 (fraction of the copy bandwidth, three CTAs -> four): pull 0.906 ->
// 1.014, AA 0.872 -> 0.907, Esoteric Twist 0.870 -> 1.010, Esoteric Pull
// 0.844 -> 0.943, Esoteric Push 0.892 -> 0.913; five CTAs (96 registers,
// 380 .. 448 bytes of spills) fell to 0.61 .. 0.71.  The general-rate
// instances (every forward transform kept) need 160 .. 250 registers; at
// four CTAs they spill up to 480 bytes and run better at three (fraction of
// the copy bandwidth, FP16 D3Q27, four -> three CTAs): TRT 0.789 -> 0.866,
// raw moments 0.828 -> 0.883, cumulants 0.577 -> 0.685, central moments
// 0.825 -> 0.823; SRT (104 bytes of spills) keeps four, 0.944 -> 0.909.
#ifndef LBM_QUAD_MINB
#define LBM_QUAD_MINB 4
#endif
#ifndef LBM_QUAD_MINB_GENERAL
#define LBM_QUAD_MINB_GENERAL 3
#endif
#define LBM_QUAD_BOUNDS \
  __launch_bounds__(LBM_BX, (REG || SPACE == SP_SRT) ? LBM_QUAD_MINB : LBM_QUAD_MINB_GENERAL)

// how a kernel reads the canonical populations f(n) of a cell; the in-place
// family below takes an even and an odd value per pattern (3 + 2 k + parity)
enum {
  G_PULL = 0, G_LOCAL = 1, G_AAODD = 2, G_ET_EVEN = 3, G_ET_ODD = 4,
  G_EPULL_EVEN = 5, G_EPULL_ODD = 6, G_EPUSH_EVEN = 7, G_EPUSH_ODD = 8
};

// The esoteric in-place family (Sec. 4.3).  Every opposite pair (p, pbar),
// p the member whose first nonzero component is +1 (odd index), owns the two
// elements (x + a_p, slot p) and (x + a_p + xi_p, slot pbar) of cell x:
//   Esoteric Twist a_p = max(-xi_p, 0) per component (positive neighbours),
//   Esoteric Pull  a_p = 0  (p local, pbar pulled from x - xi_pbar),
//   Esoteric Push  a_p = -xi_p (pbar local, p pulled from x - xi_p).
// Population i of cell x is held at node x + r_i (slot i at even times, slot
// ibar at odd times); f*_i goes to node x + w_i, slot ibar at even steps and
// slot i at odd ones, which is where population i of cell x + xi_i is read
// at the next time.  A cell writes exactly the elements it read, so the
// update is race-free in place.
enum { IP_ET = 0, IP_EPULL = 1, IP_EPUSH = 2 };
LBM_HD constexpr int ip_kind(int mode) { return (mode - 3) / 2; }
LBM_HD constexpr bool ip_odd(int mode) { return mode >= 3 && ((mode - 3) & 1); }
LBM_HD constexpr int ip_alpha(int kind, int xi) {
  return kind == IP_ET ? (xi < 0 ? 1 : 0) : (kind == IP_EPULL ? 0 : -xi);
}
// component d of the read offset r_i and the write offset w_i
template <int ST, int KIND, int i, int d>
LBM_HD constexpr int ip_read_off() {
  constexpr int xi = vel(ST, i, d);
  return i == 0 ? 0 : ((i & 1) ? ip_alpha(KIND, xi) : ip_alpha(KIND, -xi) - xi);
}
template <int ST, int KIND, int i, int d>
LBM_HD constexpr int ip_write_off() {
  constexpr int xi = vel(ST, i, d);
  return i == 0 ? 0 : ((i & 1) ? ip_alpha(KIND, xi) + xi : ip_alpha(KIND, -xi));
}

// runtime gather mode -> compile-time constant for go(integral_constant)
template <class F>
void with_gather_mode(int gm, F&& go) {
  switch (gm) {
    case G_PULL: go(std::integral_constant<int, G_PULL>{}); break;
    case G_LOCAL: go(std::integral_constant<int, G_LOCAL>{}); break;
    case G_AAODD: go(std::integral_constant<int, G_AAODD>{}); break;
    case G_ET_EVEN: go(std::integral_constant<int, G_ET_EVEN>{}); break;
    case G_ET_ODD: go(std::integral_constant<int, G_ET_ODD>{}); break;
    case G_EPULL_EVEN: go(std::integral_constant<int, G_EPULL_EVEN>{}); break;
    case G_EPULL_ODD: go(std::integral_constant<int, G_EPULL_ODD>{}); break;
    case G_EPUSH_EVEN: go(std::integral_constant<int, G_EPUSH_EVEN>{}); break;
    default: go(std::integral_constant<int, G_EPUSH_ODD>{}); break;
  }
}

// absolute FP64 storage element (LBM_STORE_F64_ABSOLUTE): holds f_i itself
struct AbsF64 {
  double v;
};

// storage element <-> zero-centered population i (every read-out and set-up
// kernel works on df; absolute storage adds / removes the weight w_i)
template <int ST, int i, class S, class T>
LBM_D T dec_pop(S v) {
  if constexpr (std::is_same<S, AbsF64>::value) return T(v.v - weight(ST, i));
  else return Codec<S>::template dec<T>(v, scale_exp(ST, i));
}
template <int ST, int i, class S, class T>
LBM_D S enc_pop(T f) {
  if constexpr (std::is_same<S, AbsF64>::value) return AbsF64{double(f) + weight(ST, i)};
  else return Codec<S>::template enc<T>(f, scale_exp(ST, i));
}

// arithmetic form of the step kernel: deviations (default), Eq. 2.6 from
// zero-centered storage, Eq. 2.4 on absolute storage, deviations with the
// discrete second-order equilibrium (q_eq = T(f_eq), Sec. 2.4)
enum { FORM_DEV = 0, FORM_ABS_EQ = 1, FORM_ABS_STORE = 2, FORM_DISC = 3 };

// body force of a step: the uniform part F plus, for FORCE_FIELD, the cell's
// entry of a per-cell field field[d * N + c] in the compute type
template <class T>
struct ForceArg {
  T F[3];
  const T* field;
};
template <int ST, int FORCE, class T>
LBM_D void cell_force(const ForceArg<T>& fa, const Geo& g, int c, T (&Fc)[3]) {
  for (int d = 0; d < 3; ++d) {
    Fc[d] = d < dim_of(ST) ? fa.F[d] : T(0);
    if constexpr (FORCE == FORCE_FIELD || FORCE == FORCE_FIELD_HE)
      if (d < dim_of(ST)) Fc[d] += fa.field[(int64_t)d * g.N + c];
  }
}

struct Nbr {
  int x[3], y[3], z[3];  // coordinate of offset -1, 0, +1 (periodic)
};

LBM_D Nbr neighbours(int x, int y, int z, const Geo& g) {
  Nbr n;
  n.x[0] = x == 0 ? g.nx - 1 : x - 1;
  n.x[1] = x;
  n.x[2] = x + 1 == g.nx ? 0 : x + 1;
  n.y[0] = y == 0 ? g.ny - 1 : y - 1;
  n.y[1] = y;
  n.y[2] = y + 1 == g.ny ? 0 : y + 1;
  n.z[0] = z == 0 ? g.nz - 1 : z - 1;
  n.z[1] = z;
  n.z[2] = z + 1 == g.nz ? 0 : z + 1;
  return n;
}

// cell index of the neighbour at offset (ox, oy, oz) in {-1, 0, 1}
LBM_D int cell_at(const Nbr& n, const Geo& g, int ox, int oy, int oz) {
  return (n.z[oz + 1] * g.ny + n.y[oy + 1]) * g.nx + n.x[ox + 1];
}

// Gather the canonical pre-collision populations f(n) of one cell.
//   G_PULL : f_i(x) = buf[i][x - xi_i]       (pull buffer after a step)
//   G_LOCAL: f_i(x) = buf[i][x]              (AA, even parity)
//   G_AAODD: f_i(x) = buf[ibar][x - xi_i]    (AA, odd parity)
//   esoteric: f_i(x) = buf[i or ibar][x + r_i]  (even / odd parity)
template <int ST, class S, class T, int MODE>
LBM_D void load_pops(const S* buf, const Geo& g, const Nbr& n, int c, T (&f)[q_of(ST)]) {
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
    int src_c = c;
    int slot = i;
    if constexpr (MODE == G_PULL || MODE == G_AAODD) src_c = cell_at(n, g, -cx, -cy, -cz);
    if constexpr (MODE >= G_ET_EVEN) {
      constexpr int K = ip_kind(MODE);
      src_c = cell_at(n, g, ip_read_off<ST, K, i, 0>(), ip_read_off<ST, K, i, 1>(),
                      ip_read_off<ST, K, i, 2>());
    }
    if constexpr (MODE == G_AAODD || ip_odd(MODE)) slot = opp(i);
    const S v = buf[(int64_t)slot * g.N + src_c];
    f[i] = dec_pop<ST, i, S, T>(v);
  });
}

// ------------------------------------------------------------ step kernels
// Per-direction plane pointers of the pull kernel.  src[i] points at plane i
// of the source buffer already shifted by the interior stencil offset
// -(xi_z*Ny*Nx + xi_y*Nx + xi_x), so the gather of cell c reads
// src[i][c + wrap_i] with wrap_i nonzero only on the periodic boundary:
// one integer add and one wide address computation per load.
template <class S>
struct PullPtrs {
  const S* src[27];
  S* dst[27];
};

// pull: read f_i from x - xi_i of src, collide, write f*_i at x of dst
template <int ST, class S, class T, int SPACE, bool REG, int FORM = FORM_DEV, int FORCE = FORCE_NONE>
__global__ void __launch_bounds__(LBM_PULL_BX) k_pull(const __grid_constant__ PullPtrs<S> P, Geo g,
                                                      Rates<T> keep, ForceArg<T> fa = {},
                                                      int z0 = 0) {
  const int x = blockIdx.x * LBM_PULL_BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = z0 + int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  // wrap corrections for a read at x - xi (xi = +1 reads x-1, -1 reads x+1)
  const int wxp = x == 0 ? g.nx : 0, wxm = x == g.nx - 1 ? -g.nx : 0;
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  T f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
    const int wyz = (cy > 0 ? wyp : (cy < 0 ? wym : 0)) + (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
    const int wx = cx > 0 ? wxp : (cx < 0 ? wxm : 0);
    const S v = P.src[i][c + wx + wyz];
    if constexpr (FORM == FORM_ABS_STORE) f[i] = T(v.v);
    else f[i] = dec_pop<ST, i, S, T>(v);
  });
  if constexpr (FORM == FORM_DEV && FORCE != FORCE_NONE) {
    T Fc[3];
    cell_force<ST, FORCE>(fa, g, c, Fc);
    collide<ST, T, SPACE, REG, false, true, (FORCE >= FORCE_UNIFORM_HE)>(f, keep, Fc);
  } else if constexpr (FORM == FORM_DEV) {
    collide<ST, T, SPACE, REG>(f, keep);
  } else if constexpr (FORM == FORM_DISC) {
    collide<ST, T, SPACE, REG, false, false, false, true>(f, keep);
  } else {
    collide_abs<ST, T, SPACE, REG, FORM == FORM_ABS_EQ>(f, keep);
  }
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    if constexpr (FORM == FORM_ABS_STORE) P.dst[i][c] = S{double(f[i])};
    else P.dst[i][c] = enc_pop<ST, i, S, T>(f[i]);
  });
}

// Shallow-water step (D2Q9, absolute FP64 storage, pull): the absolute
// collision with the method's shallow-water equilibrium (Sec. 5.2).
template <int ST, int SPACE>
__global__ void __launch_bounds__(LBM_BX) k_pull_swe(const __grid_constant__ PullPtrs<AbsF64> P,
                                                     Geo g, Rates<double> keep, double grav) {
  const int x = blockIdx.x * LBM_BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  const int wxp = x == 0 ? g.nx : 0, wxm = x == g.nx - 1 ? -g.nx : 0;
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  double f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1);
    const int wy = cy > 0 ? wyp : (cy < 0 ? wym : 0);
    const int wx = cx > 0 ? wxp : (cx < 0 ? wxm : 0);
    f[i] = P.src[i][c + wx + wy].v;
  });
  collide_abs<ST, double, SPACE, false, false, true>(f, keep, grav);
  sfor<q_of(ST)>([&](auto I) { P.dst[CI(I)][c] = AbsF64{f[CI(I)]}; });
}

// Set-up of a shallow-water context from depth and velocity: the method's
// equilibrium written upstream (pull layout) as absolute FP64 populations.
template <int ST, int SPACE>
__global__ void __launch_bounds__(LBM_BX) k_scatter_swe(AbsF64* buf, Geo g, const double* h,
                                                        const double* u, double grav) {
  const int x = blockIdx.x * LBM_BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const Nbr n = neighbours(x, y, z, g);
  const int c = (z * g.ny + y) * g.nx + x;
  const double uu[3] = {u[c], u[g.N + c], 0.0};
  double f[q_of(ST)];
  swe_feq<ST, double, SPACE>(h ? h[c] : 1.0, uu, grav, f);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    const int dc = cell_at(n, g, -vel(ST, i, 0), -vel(ST, i, 1), -vel(ST, i, 2));
    buf[(int64_t)i * g.N + dc] = AbsF64{f[i]};
  });
}

// Two cells per thread (x even, x + 1) with the collision on packed FP32
// pairs, for FP16 / BF16 delta storage and even Nx.  Directions with
// xi_x = 0 read both cells with one aligned 2-element load; the others read
// the two cells separately (their x wrap differs at the row ends).  Stores
// are aligned 2-element stores.  The plane base of each direction is formed
// in the kernel from the two buffer pointers, the plane size and the
// compile-time offsets: warp-uniform values, which the compiler keeps on the
// uniform datapath (an earlier form passed 54 pre-shifted plane pointers as
// parameters, one constant-bank load and 64-bit add each: 50.7 -> 52.3 GLUPS
// at 512^3).
template <int ST, class S, int SPACE, bool REG>
__global__ void LBM_PULL2_BOUNDS k_pull2(const S* __restrict__ src, S* __restrict__ dst, Geo g,
                                         Rates<P2> keep, int z0 = 0) {
  const int x = 2 * (blockIdx.x * LBM_BX + threadIdx.x);
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = z0 + int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  const int wxp0 = x == 0 ? g.nx : 0;           // cell x reading x - 1
  const int wxm1 = x + 2 == g.nx ? -g.nx : 0;   // cell x + 1 reading x + 2
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  P2 f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
    // plane i shifted by the interior y / z offset of the gather
    const S* pl = src + (int64_t(i) * g.N - (int64_t(cz) * nxy + int64_t(cy) * g.nx));
    const int off = c + (cy > 0 ? wyp : (cy < 0 ? wym : 0)) + (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
    constexpr int E = scale_exp(ST, i);
    if constexpr (cx == 0) f[i] = Pack<S>::template load2s<E>(pl + off);
    else if constexpr (cx > 0) f[i] = Pack<S>::template load11s<E>(pl + (off - 1 + wxp0), pl + off);
    else f[i] = Pack<S>::template load11s<E>(pl + (off + 1), pl + (off + 2 + wxm1));
  });
  // the backward transform leaves population i multiplied by 2^|xi_i|^2;
  // the storage scale 2^s_i absorbs it exactly
  collide<ST, P2, SPACE, REG, true>(f, keep);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                      vel(ST, i, 2) * vel(ST, i, 2);
    Pack<S>::store2(dst + (int64_t(i) * g.N + c), f[i] * P2(float(1u << (scale_exp(ST, i) - k))));
  });
}

// Four cells per thread (x = 4k .. 4k + 3) for FP16 / BF16 delta storage
// when Nx % 4 == 0: the arithmetic of k_pull2 on two packed pairs per
// population (every lane computes what k_pull2 computes, so the states are
// bitwise equal).  xi_x = 0 planes: one aligned 8-byte load; xi_x = +-1: the
// aligned quad and the one element beyond it.  Half the loads, stores and
// address arithmetic per cell of k_pull2: 52.6 -> 54.6 GLUPS at 512^3 FP16,
// and 60.9 with four CTAs per SM (LBM_QUAD_MINB).
template <int ST, class S, int SPACE, bool REG>
__global__ void LBM_QUAD_BOUNDS k_pull4(const S* __restrict__ src, S* __restrict__ dst, Geo g,
                                         Rates<P4> keep) {
  const int x = 4 * (blockIdx.x * LBM_BX + threadIdx.x);
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  const int wxp0 = x == 0 ? g.nx : 0;           // cell x reading x - 1
  const int wxm3 = x + 4 == g.nx ? -g.nx : 0;   // cell x + 3 reading x + 4
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  P4 f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = dim_of(ST) == 3 ? vel(ST, i, 2) : 0;
    const S* pl = src + (int64_t(i) * g.N - (int64_t(cz) * nxy + int64_t(cy) * g.nx));
    const int off = c + (cy > 0 ? wyp : (cy < 0 ? wym : 0)) + (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
    constexpr int E = scale_exp(ST, i);
    if constexpr (cx == 0) f[i] = Pack<S>::template load4s<E>(pl + off);
    else if constexpr (cx > 0) f[i] = Pack<S>::template load1_3s<E>(pl + (off - 1 + wxp0), pl + off);
    else f[i] = Pack<S>::template load3_1s<E>(pl + off, pl + (off + 4 + wxm3));
  });
  // the backward transform leaves population i multiplied by 2^|xi_i|^2;
  // the storage scale 2^s_i absorbs it exactly
  collide<ST, P4, SPACE, REG, true>(f, keep);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                      vel(ST, i, 2) * vel(ST, i, 2);
    store4<S>(dst + (int64_t(i) * g.N + c), f[i] * P4(float(1u << (scale_exp(ST, i) - k))));
  });
}

// In-place streaming on one buffer (Sec. 4.3), every pattern through one
// kernel with per-direction plane pointers (as the pull kernel): population
// i is read from slot rd_i at node x + r_i and f*_i written to slot wr_i at
// node x + w_i, with the offsets r_i, w_i in {-1, 0, 1}^3 baked into the
// pointers and a wrap correction only on the periodic boundary.
//   AA, even: r = w = 0, read slot i, write slot ibar (the own cell).
//   AA, odd:  r = -xi_i, read slot ibar; w = +xi_i, write slot i.
//   Esoteric Twist / Pull / Push: r_i, w_i of the esoteric family above;
//     even steps read slot i and write slot ibar, odd steps read slot ibar
//     and write slot i.  For the Twist r_i = max(-xi_i, 0) and
//     w_i = max(xi_i, 0) per component: a cell touches itself and its
//     positive neighbours only.
// Each cell reads and writes the same set of elements in every variant.
template <class S>
struct InPlacePtrs {
  const S* rd[27];
  S* wr[27];
};

// the per-direction offsets and slots of an in-place variant
template <int ST, int MODE, int i>
struct InPlaceMap {
  static constexpr int b = opp(i);
  static constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = vel(ST, i, 2);
  static constexpr bool ESO = MODE >= MODE_ET_EVEN;
  static constexpr int K = ESO ? ip_kind(MODE) : 0;
  static constexpr bool ODD = MODE == MODE_AA_ODD || ip_odd(MODE);
  static constexpr int aa = MODE == MODE_AA_ODD ? 1 : 0;
  static constexpr int rx = ESO ? ip_read_off<ST, K, i, 0>() : -aa * cx;
  static constexpr int ry = ESO ? ip_read_off<ST, K, i, 1>() : -aa * cy;
  static constexpr int rz = ESO ? ip_read_off<ST, K, i, 2>() : -aa * cz;
  static constexpr int wx = ESO ? ip_write_off<ST, K, i, 0>() : aa * cx;
  static constexpr int wy = ESO ? ip_write_off<ST, K, i, 1>() : aa * cy;
  static constexpr int wz = ESO ? ip_write_off<ST, K, i, 2>() : aa * cz;
  static constexpr int rslot = ODD ? b : i;
  static constexpr int wslot = ODD ? i : b;
};

// Block traversal order of the in-place kernels: bit m of the mask runs the
// blocks of mode m in reverse (last row first).  Every cell still updates
// once; only the order in which the rows reach memory changes.  Measured on
// B300 (D3Q27 cumulant FP32, 512^3, MLUPS forward -> both parities
// reversed): Esoteric Pull 27,248 -> 29,994 (its non-local elements lie at
// +xi_p, ahead of a forward sweep), Esoteric Push 30,467 -> 29,629, AA
// 30,321 -> 29,042, Esoteric Twist unchanged; so only the Esoteric Pull
// modes (5, 6) run in reverse.
#ifndef LBM_INPLACE_REV_MASK
#define LBM_INPLACE_REV_MASK ((1 << MODE_EPULL_EVEN) | (1 << MODE_EPULL_ODD))
#endif

// Block size of the in-place kernel per mode: 256 threads for Esoteric Twist
// and Pull, 128 for AA and Esoteric Push (measured at 512^3, MLUPS with 128
// -> 256 threads: Twist 30,297 -> 30,866, Pull 29,850 -> 30,549, AA
// 30,273 -> 29,946, Push 30,332 -> 29,228).
LBM_HD constexpr int inplace_bx(int mode) {
  return (mode == MODE_ET_EVEN || mode == MODE_ET_ODD || mode == MODE_EPULL_EVEN ||
          mode == MODE_EPULL_ODD)
             ? 256
             : LBM_BX;
}

template <int ST, class S, class T, int SPACE, bool REG, int MODE, int FORCE = FORCE_NONE>
__global__ void __launch_bounds__(inplace_bx(MODE)) k_inplace(const __grid_constant__ InPlacePtrs<S> P,
                                                              Geo g, Rates<T> keep,
                                                              ForceArg<T> fa = {}) {
  constexpr bool REV = (LBM_INPLACE_REV_MASK >> MODE) & 1;
  constexpr int BX = inplace_bx(MODE);
  const int bx = REV ? int(gridDim.x) - 1 - int(blockIdx.x) : int(blockIdx.x);
  const int x = bx * BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = REV ? g.ny - 1 - int(blockIdx.y) : int(blockIdx.y);
  const int z = REV ? g.nz - 1 - int(blockIdx.z) : int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  // wrap corrections for an offset of -1 (p) and +1 (m) per axis
  const int wxp = x == 0 ? g.nx : 0, wxm = x == g.nx - 1 ? -g.nx : 0;
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  auto wrap = [&](int ox, int oy, int oz) {
    return (ox < 0 ? wxp : (ox > 0 ? wxm : 0)) + (oy < 0 ? wyp : (oy > 0 ? wym : 0)) +
           (oz < 0 ? wzp : (oz > 0 ? wzm : 0));
  };
  T f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    f[i] = dec_pop<ST, i, S, T>(P.rd[i][c + wrap(Mp::rx, Mp::ry, Mp::rz)]);
  });
  if constexpr (FORCE != FORCE_NONE) {
    T Fc[3];
    cell_force<ST, FORCE>(fa, g, c, Fc);
    collide<ST, T, SPACE, REG, false, true, (FORCE >= FORCE_UNIFORM_HE)>(f, keep, Fc);
  } else {
    collide<ST, T, SPACE, REG>(f, keep);
  }
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    P.wr[i][c + wrap(Mp::wx, Mp::wy, Mp::wz)] = enc_pop<ST, i, S, T>(f[i]);
  });
}

// host: the pointer table of an in-place variant on buffer buf
template <int ST, int MODE, class S>
InPlacePtrs<S> inplace_ptrs(S* buf, const Geo& g) {
  InPlacePtrs<S> P;
  const int64_t nx = g.nx, nxy = int64_t(g.nx) * g.ny;
  for (int i = 0; i < 27; ++i) P.rd[i] = nullptr, P.wr[i] = nullptr;
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    P.rd[i] = buf + (int64_t(Mp::rslot) * g.N + Mp::rz * nxy + Mp::ry * nx + Mp::rx);
    P.wr[i] = buf + (int64_t(Mp::wslot) * g.N + Mp::wz * nxy + Mp::wy * nx + Mp::wx);
  });
  return P;
}

template <int ST, class S, class T, int SPACE, bool REG, int FORCE = FORCE_NONE>
void launch_inplace(const StepArgs& a, const Rates<T>& keep, const dim3& grid,
                    const ForceArg<T>& fa = {}) {
  S* buf = (S*)a.dst;
  (void)grid;
  auto go = [&](auto mode_tag) {
    constexpr int MODE = decltype(mode_tag)::value;
    constexpr int BX = inplace_bx(MODE);
    const dim3 igrid((a.g.nx + BX - 1) / BX, a.g.ny, a.g.nz);
    k_inplace<ST, S, T, SPACE, REG, MODE, FORCE>
        <<<igrid, BX, 0, a.stream>>>(inplace_ptrs<ST, MODE>(buf, a.g), a.g, keep, fa);
  };
  switch (a.mode) {
    case MODE_AA_EVEN: go(std::integral_constant<int, MODE_AA_EVEN>{}); break;
    case MODE_AA_ODD: go(std::integral_constant<int, MODE_AA_ODD>{}); break;
    case MODE_ET_EVEN: go(std::integral_constant<int, MODE_ET_EVEN>{}); break;
    case MODE_ET_ODD: go(std::integral_constant<int, MODE_ET_ODD>{}); break;
    case MODE_EPULL_EVEN: go(std::integral_constant<int, MODE_EPULL_EVEN>{}); break;
    case MODE_EPULL_ODD: go(std::integral_constant<int, MODE_EPULL_ODD>{}); break;
    case MODE_EPUSH_EVEN: go(std::integral_constant<int, MODE_EPUSH_EVEN>{}); break;
    default: go(std::integral_constant<int, MODE_EPUSH_ODD>{}); break;
  }
}

// In-place step for FP16 / BF16 delta storage with even Nx: two cells (x,
// x + 1) per thread on packed FP32 pairs, the arithmetic of k_pull2 over the
// addressing of k_inplace.  An element offset of 0 along x keeps the pair's
// access one aligned 4-byte access; -1 or +1 splits it into two 2-byte
// accesses, of which the one at the row's end wraps.
// Block order of the packed in-place kernel (bit m: mode m in reverse).
// Measured at 512^3 FP16 with the Esoteric Pull modes reversed as in
// k_inplace: 0.803 of the copy bandwidth, forward 0.810 (the other patterns
// unchanged), so every mode runs forward here.
#ifndef LBM_INPLACE2_REV_MASK
#define LBM_INPLACE2_REV_MASK 0
#endif

template <int ST, class S, int SPACE, bool REG, int MODE>
__global__ void LBM_PULL2_BOUNDS k_inplace2(const __grid_constant__ InPlacePtrs<S> P, Geo g,
                                            Rates<P2> keep) {
  constexpr bool REV = (LBM_INPLACE2_REV_MASK >> MODE) & 1;
  const int bx = REV ? int(gridDim.x) - 1 - int(blockIdx.x) : int(blockIdx.x);
  const int x = 2 * (bx * LBM_BX + threadIdx.x);
  if (x >= g.nx) return;
  const int y = REV ? g.ny - 1 - int(blockIdx.y) : int(blockIdx.y);
  const int z = REV ? g.nz - 1 - int(blockIdx.z) : int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  const int wx0 = x == 0 ? g.nx : 0;           // cell x at offset -1
  const int wx1 = x + 2 == g.nx ? -g.nx : 0;   // cell x + 1 at offset +1
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  auto wyz = [&](int oy, int oz) {
    return (oy < 0 ? wyp : (oy > 0 ? wym : 0)) + (oz < 0 ? wzp : (oz > 0 ? wzm : 0));
  };
  // (plane pointers from the parameter table: forming the 2 q slot bases in
  // the kernel from one buffer pointer, as k_pull2 does, measured 14 %
  // slower here)
  P2 f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    const S* p = P.rd[i] + (c + wyz(Mp::ry, Mp::rz));
    constexpr int E = scale_exp(ST, i);
    if constexpr (Mp::rx == 0) f[i] = Pack<S>::template load2s<E>(p);
    else if constexpr (Mp::rx < 0) f[i] = Pack<S>::template load11s<E>(p + wx0, p + 1);
    else f[i] = Pack<S>::template load11s<E>(p, p + 1 + wx1);
  });
  // the backward transform leaves population i multiplied by 2^|xi_i|^2;
  // the storage scale 2^s_i absorbs it exactly
  collide<ST, P2, SPACE, REG, true>(f, keep);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                      vel(ST, i, 2) * vel(ST, i, 2);
    const P2 v = f[i] * P2(float(1u << (scale_exp(ST, i) - k)));
    S* p = P.wr[i] + (c + wyz(Mp::wy, Mp::wz));
    if constexpr (Mp::wx == 0) Pack<S>::store2(p, v);
    else if constexpr (Mp::wx < 0) Pack<S>::store11(p + wx0, p + 1, v);
    else Pack<S>::store11(p, p + 1 + wx1, v);
  });
}

// Block order of the four-cell in-place kernel (bit m: mode m in reverse).
// Measured at 512^3 FP16 (fraction of the copy bandwidth, forward ->
// reversed): AA 0.916 -> 0.927 with both parities reversed (0.925 even
// only, 0.919 odd only); Esoteric Push 0.937 -> 0.903 / 0.901 / 0.870 for
// its first / second / both parities, so only the AA modes run in reverse.
#ifndef LBM_INPLACE4_REV_MASK
#define LBM_INPLACE4_REV_MASK ((1 << MODE_AA_EVEN) | (1 << MODE_AA_ODD))
#endif

// Four cells per thread (Nx % 4 == 0): the arithmetic of k_inplace2 on two
// packed pairs per population, over the same pointer table.  A cell's x
// offset of 0 keeps the four cells' access one aligned 8-byte access; -1 or
// +1 splits it into the aligned quad (less one element) and the element
// beyond it, of which the one at the row's end wraps.  Each cell reads and
// writes its own set of elements, so grouping four of them per thread keeps
// the in-place update race-free (in either block order).
template <int ST, class S, int SPACE, bool REG, int MODE>
__global__ void LBM_QUAD_BOUNDS k_inplace4(const __grid_constant__ InPlacePtrs<S> P, Geo g,
                                            Rates<P4> keep) {
  constexpr bool REV = (LBM_INPLACE4_REV_MASK >> MODE) & 1;
  const int bx = REV ? int(gridDim.x) - 1 - int(blockIdx.x) : int(blockIdx.x);
  const int x = 4 * (bx * LBM_BX + threadIdx.x);
  if (x >= g.nx) return;
  const int y = REV ? g.ny - 1 - int(blockIdx.y) : int(blockIdx.y);
  const int z = REV ? g.nz - 1 - int(blockIdx.z) : int(blockIdx.z);
  const int c = (z * g.ny + y) * g.nx + x;
  const int nxy = g.nx * g.ny;
  const int wx0 = x == 0 ? g.nx : 0;           // cell x at offset -1
  const int wx3 = x + 4 == g.nx ? -g.nx : 0;   // cell x + 3 at offset +1
  const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
  const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
  auto wyz = [&](int oy, int oz) {
    return (oy < 0 ? wyp : (oy > 0 ? wym : 0)) + (oz < 0 ? wzp : (oz > 0 ? wzm : 0));
  };
  P4 f[q_of(ST)];
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    // p: the element cell x reads (its x offset included in the table)
    const S* p = P.rd[i] + (c + wyz(Mp::ry, Mp::rz));
    constexpr int E = scale_exp(ST, i);
    if constexpr (Mp::rx == 0) f[i] = Pack<S>::template load4s<E>(p);
    else if constexpr (Mp::rx < 0) f[i] = Pack<S>::template load1_3s<E>(p + wx0, p + 1);
    else f[i] = Pack<S>::template load3_1s<E>(p - 1, p + 3 + wx3);
  });
  collide<ST, P4, SPACE, REG, true>(f, keep);
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    using Mp = InPlaceMap<ST, MODE, i>;
    constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                      vel(ST, i, 2) * vel(ST, i, 2);
    const P4 v = f[i] * P4(float(1u << (scale_exp(ST, i) - k)));
    S* p = P.wr[i] + (c + wyz(Mp::wy, Mp::wz));
    if constexpr (Mp::wx == 0) store4<S>(p, v);
    else if constexpr (Mp::wx < 0) store1_3<S>(p + wx0, p + 1, v);
    else store3_1<S>(p - 1, p + 3 + wx3, v);
  });
}

template <int ST, class S, int SPACE, bool REG>
void launch_inplace2(const StepArgs& a, const Rates<P2>& keep) {
  S* buf = (S*)a.dst;
  const dim3 grid2((a.g.nx / 2 + LBM_BX - 1) / LBM_BX, a.g.ny, a.g.nz);
  // four cells per thread where Nx % 4 == 0, compiled for the D3Q27
  // regularised cumulant method only (for every method it took the compile
  // of one storage type from minutes to beyond 45 minutes)
  constexpr bool QUADS = ST == D3Q27 && SPACE == SP_CUMULANT && REG;
  Rates<P4> k4;
  for (int k = 0; k < 6; ++k) k4.om[k] = P4(keep.om[k], keep.om[k]);
  auto go = [&](auto mode_tag) {
    constexpr int MODE = decltype(mode_tag)::value;
    if constexpr (QUADS) {
      if (a.g.nx % 4 == 0) {
        const dim3 grid4((a.g.nx / 4 + LBM_BX - 1) / LBM_BX, a.g.ny, a.g.nz);
        k_inplace4<ST, S, SPACE, REG, MODE>
            <<<grid4, LBM_BX, 0, a.stream>>>(inplace_ptrs<ST, MODE>(buf, a.g), a.g, k4);
        return;
      }
    }
    k_inplace2<ST, S, SPACE, REG, MODE>
        <<<grid2, LBM_BX, 0, a.stream>>>(inplace_ptrs<ST, MODE>(buf, a.g), a.g, keep);
  };
  switch (a.mode) {
    case MODE_AA_EVEN: go(std::integral_constant<int, MODE_AA_EVEN>{}); break;
    case MODE_AA_ODD: go(std::integral_constant<int, MODE_AA_ODD>{}); break;
    case MODE_ET_EVEN: go(std::integral_constant<int, MODE_ET_EVEN>{}); break;
    case MODE_ET_ODD: go(std::integral_constant<int, MODE_ET_ODD>{}); break;
    case MODE_EPULL_EVEN: go(std::integral_constant<int, MODE_EPULL_EVEN>{}); break;
    case MODE_EPULL_ODD: go(std::integral_constant<int, MODE_EPULL_ODD>{}); break;
    case MODE_EPUSH_EVEN: go(std::integral_constant<int, MODE_EPUSH_EVEN>{}); break;
    default: go(std::integral_constant<int, MODE_EPUSH_ODD>{}); break;
  }
}

// ------------------------------------------------------ read-out kernels
// canonical populations -> FP64 SoA df[i * N + c] and / or macroscopic
// Slab of a read-out / set-up launch: block (bx, by, bz) covers row
// (y0 + by, z0 + bz); the staged arrays hold component k of cell c at
// k * stride + (c - c0).
struct Slab {
  int y0, z0;
  int64_t c0, stride;
};

template <int ST, class S, class T, int MODE>
__global__ void __launch_bounds__(LBM_BX) k_gather(const S* buf, Geo g, double* df, double* rho,
                                                   double* u, Slab sl, ForceArg<T> fa = {}) {
  const int x = blockIdx.x * LBM_BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = sl.y0 + blockIdx.y, z = sl.z0 + blockIdx.z;
  const Nbr n = neighbours(x, y, z, g);
  const int c = (z * g.ny + y) * g.nx + x;
  const int64_t s = c - sl.c0;  // index in the staged arrays
  T f[q_of(ST)];
  load_pops<ST, S, T, MODE>(buf, g, n, c, f);
  if (df) {
    sfor<q_of(ST)>([&](auto I) { df[(int64_t)CI(I) * sl.stride + s] = double(f[CI(I)]); });
  }
  if (rho || u) {
    double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      const double v = double(f[i]);
      dr += v;
      if constexpr (vel(ST, i, 0) != 0) j[0] += vel(ST, i, 0) * v;
      if constexpr (vel(ST, i, 1) != 0) j[1] += vel(ST, i, 1) * v;
      if constexpr (vel(ST, i, 2) != 0) j[2] += vel(ST, i, 2) * v;
    });
    const double r = 1.0 + dr;
    if (rho) rho[s] = r;
    if (u) {
      // under a body force the fluid velocity is (j + F/2) / rho
      for (int d = 0; d < dim_of(ST); ++d) {
        double Fd = double(fa.F[d]);
        if (fa.field) Fd += double(fa.field[(int64_t)d * g.N + c]);
        u[(int64_t)d * sl.stride + s] = (j[d] + 0.5 * Fd) / r;
      }
    }
  }
}

// write canonical populations (FP64 SoA df, or the method's equilibrium of
// rho / u when df is NULL) into the storage so that the next gather returns
// them: pull -> buf[i][x - xi_i] (moved back upstream, where the pull
// gather of cell x looks), AA -> buf[i][x] (even parity).
template <int ST, class S, class T, int SPACE, int LAYOUT, bool DISC = false>
__global__ void __launch_bounds__(LBM_BX) k_scatter(S* buf, Geo g, const double* df,
                                                    const double* rho, const double* u, Slab sl) {
  const int x = blockIdx.x * LBM_BX + threadIdx.x;
  if (x >= g.nx) return;
  const int y = sl.y0 + blockIdx.y, z = sl.z0 + blockIdx.z;
  const Nbr n = neighbours(x, y, z, g);
  const int c = (z * g.ny + y) * g.nx + x;
  const int64_t s = c - sl.c0;  // index in the staged arrays
  T f[q_of(ST)];
  if (df) {
    sfor<q_of(ST)>([&](auto I) { f[CI(I)] = T(df[(int64_t)CI(I) * sl.stride + s]); });
  } else {
    const T dr = rho ? T(rho[s] - 1.0) : T(0);
    T uu[3] = {T(0), T(0), T(0)};
    for (int d = 0; d < dim_of(ST); ++d) uu[d] = T(u[(int64_t)d * sl.stride + s]);
    if constexpr (DISC) disc_feq<ST, T>(dr, T(1) + dr, uu, f);
    else equilibrium<ST, T, SPACE>(dr, uu, f);
  }
  sfor<q_of(ST)>([&](auto I) {
    constexpr int i = CI(I);
    int dc = c;
    if constexpr (LAYOUT == G_PULL) dc = cell_at(n, g, -vel(ST, i, 0), -vel(ST, i, 1), -vel(ST, i, 2));
    if constexpr (LAYOUT >= G_ET_EVEN) {
      constexpr int K = ip_kind(LAYOUT);
      dc = cell_at(n, g, ip_read_off<ST, K, i, 0>(), ip_read_off<ST, K, i, 1>(),
                   ip_read_off<ST, K, i, 2>());
    }
    buf[(int64_t)i * g.N + dc] = enc_pop<ST, i, S, T>(f[i]);
  });
}

// FP64 invariant partial sums, one row of 8 per block (fixed cell order):
// sum(rho-1), sum(rho u_x), sum(rho u_y), sum(rho u_z), sum(rho|u|^2/2),
// max|u|, #non-finite cells, #cells.
constexpr int INV_THREADS = 256;
template <int ST, class S, class T, int MODE>
__global__ void __launch_bounds__(INV_THREADS) k_invariants(const S* buf, Geo g, double* part) {
  __shared__ double sh[INV_THREADS][8];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * INV_THREADS;
  for (int64_t c = (int64_t)blockIdx.x * INV_THREADS + threadIdx.x; c < g.N; c += stride) {
    const int x = int(c % g.nx), y = int((c / g.nx) % g.ny), z = int(c / ((int64_t)g.nx * g.ny));
    const Nbr n = neighbours(x, y, z, g);
    T f[q_of(ST)];
    load_pops<ST, S, T, MODE>(buf, g, n, int(c), f);
    double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
    bool finite = true;
    sfor<q_of(ST)>([&](auto I) {
      constexpr int i = CI(I);
      const double v = double(f[i]);
      finite = finite && isfinite(v);
      dr += v;
      if constexpr (vel(ST, i, 0) != 0) j[0] += vel(ST, i, 0) * v;
      if constexpr (vel(ST, i, 1) != 0) j[1] += vel(ST, i, 1) * v;
      if constexpr (vel(ST, i, 2) != 0) j[2] += vel(ST, i, 2) * v;
    });
    if (!finite) {
      acc[6] += 1.0;
    } else {
      const double r = 1.0 + dr;
      const double u0 = j[0] / r, u1 = j[1] / r, u2 = j[2] / r;
      const double uu = u0 * u0 + u1 * u1 + u2 * u2;
      acc[0] += dr;
      acc[1] += j[0];
      acc[2] += j[1];
      acc[3] += j[2];
      acc[4] += 0.5 * r * uu;
      acc[5] = fmax(acc[5], sqrt(uu));
    }
    acc[7] += 1.0;
  }
  for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = INV_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 8; ++k)
        sh[threadIdx.x][k] = k == 5 ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                    : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[(int64_t)blockIdx.x * 8 + threadIdx.x] = sh[0][threadIdx.x];
}

// ------------------------------------------------------ batched ensemble
// Persistent pull kernel over many instances: block b handles tiles b,
// b + gridDim.x, ... of the tile list; a tile is threads * cpt consecutive
// cells of one instance (cell index c -> x, y, z by division).
constexpr int BATCH_MAX_THREADS = 256;

LBM_D void cell_xyz(int c, const Geo& g, int& x, int& y, int& z) {
  const int yz = c / g.nx;
  x = c - yz * g.nx;
  z = yz / g.ny;
  y = yz - z * g.ny;
}

// q = a / d and a - q d for 0 <= a < 2^24 and d >= 1, from the float
// reciprocal rd = fl(1/d): a is exact in FP32 and the rounded product is
// within (a/d) 2^-23 < 1 of a/d, so one correction step gives the quotient
LBM_D int fast_divmod(int a, int d, float rd, int& r) {
  int q = int(float(a) * rd);
  r = a - q * d;
  if (r < 0) r += d, --q;
  else if (r >= d) r -= d, ++q;
  return q;
}

template <int ST, class S, class T, int SPACE, bool REG>
__global__ void __launch_bounds__(BATCH_MAX_THREADS)
    k_batch_pull(const S* __restrict__ src, S* __restrict__ dst, const BInst* __restrict__ inst,
                 const int2* __restrict__ tiles, int ntiles, int cpt, Rates<T> keep) {
  // the next tile's descriptors are loaded while the current one runs; two
  // cells are in flight per thread (the gathers of the next cell are issued
  // before the collision and stores of the current one), and a gather is
  // src_i[c - xi_i] with the periodic wrap as a correction, as in k_pull:
  // 0.94 -> 0.96 of the copy bandwidth at 4096 D3Q19 domains
  int t = blockIdx.x;
  int2 tl = t < ntiles ? tiles[t] : make_int2(0, 0);
  BInst I = inst[t < ntiles ? tl.x : 0];
  for (; t < ntiles; t += gridDim.x) {
    const int tn = t + gridDim.x;
    const int2 tln = tn < ntiles ? tiles[tn] : tl;
    const BInst In = inst[tln.x];
    const Geo g{I.nx, I.ny, I.nz, (int64_t)I.N};
    Rates<T> k = keep;
    k.om[0] = T(I.keep_shear);
    const S* s = src + I.off;
    S* d = dst + I.off;
    auto gather = [&](int c, T (&f)[q_of(ST)]) {
      int x, y, z;
      if (I.N < (1 << 24)) {  // float quotient within one of the true one
        const int yz = fast_divmod(c, I.nx, I.rnx, x);
        z = fast_divmod(yz, I.ny, I.rny, y);
      } else {
        cell_xyz(c, g, x, y, z);
      }
      // pull gather src_i[c - xi_i] with the periodic wrap as a correction
      // (the offsets are the instance's, uniform over the tile)
      const int nxy = g.nx * g.ny;
      const int wxp = x == 0 ? g.nx : 0, wxm = x == g.nx - 1 ? -g.nx : 0;
      const int wyp = y == 0 ? nxy : 0, wym = y == g.ny - 1 ? -nxy : 0;
      const int wzp = z == 0 ? int(g.N) : 0, wzm = z == g.nz - 1 ? -int(g.N) : 0;
      sfor<q_of(ST)>([&](auto I_) {
        constexpr int i = CI(I_);
        constexpr int cx = vel(ST, i, 0), cy = vel(ST, i, 1), cz = dim_of(ST) == 3 ? vel(ST, i, 2) : 0;
        const S* pl = s + (int64_t(i) * g.N - (int64_t(cz) * nxy + int64_t(cy) * g.nx + cx));
        const int w = (cx > 0 ? wxp : (cx < 0 ? wxm : 0)) + (cy > 0 ? wyp : (cy < 0 ? wym : 0)) +
                      (cz > 0 ? wzp : (cz < 0 ? wzm : 0));
        f[i] = dec_pop<ST, i, S, T>(pl[c + w]);
      });
    };
    auto finish = [&](int c, T (&f)[q_of(ST)]) {
      collide<ST, T, SPACE, REG>(f, k);
      sfor<q_of(ST)>([&](auto I_) {
        constexpr int i = CI(I_);
        d[(int64_t)i * g.N + c] = enc_pop<ST, i, S, T>(f[i]);
      });
    };
    const int B = (int)blockDim.x;
    int c = tl.y + (int)threadIdx.x;
    T fa[q_of(ST)], fb[q_of(ST)];
    if (cpt > 0 && c < I.N) {
      gather(c, fa);
      for (int j = 0;; j += 2) {
        const bool b1 = j + 1 < cpt && c + B < I.N;
        if (b1) gather(c + B, fb);
        finish(c, fa);
        if (!b1) break;
        const bool b2 = j + 2 < cpt && c + 2 * B < I.N;
        if (b2) gather(c + 2 * B, fa);
        finish(c + B, fb);
        if (!b2) break;
        c += 2 * B;
      }
    }
    tl = tln;
    I = In;
  }
}

// Taylor-Green set-up of every instance (Eq. 5.1 at t = 0, z-invariant,
// wavenumber 2 pi / N per axis): the method's equilibrium, written upstream
// for the pull gather.
template <int ST, class S, class T, int SPACE>
__global__ void __launch_bounds__(BATCH_MAX_THREADS)
    k_batch_tgv(S* __restrict__ buf, const BInst* __restrict__ inst, const int2* __restrict__ tiles,
                int ntiles, int cpt, const double* __restrict__ u0) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const BInst I = inst[tl.x];
    const Geo g{I.nx, I.ny, I.nz, (int64_t)I.N};
    const double a = u0[tl.x];
    const double kx = 2.0 * 3.14159265358979323846 / I.nx;
    const double ky = 2.0 * 3.14159265358979323846 / I.ny;
    S* b = buf + I.off;
    for (int j = 0; j < cpt; ++j) {
      const int c = tl.y + j * (int)blockDim.x + (int)threadIdx.x;
      if (c >= I.N) break;
      int x, y, z;
      cell_xyz(c, g, x, y, z);
      const Nbr n = neighbours(x, y, z, g);
      double sx, cx, sy, cy;
      sincos(kx * x, &sx, &cx);
      sincos(ky * y, &sy, &cy);
      const double rho = 1.0 - 0.75 * a * a * (cos(2.0 * kx * x) + cos(2.0 * ky * y));
      T uu[3] = {T(a * cx * sy), T(-a * sx * cy), T(0)};
      T f[q_of(ST)];
      equilibrium<ST, T, SPACE>(T(rho - 1.0), uu, f);
      sfor<q_of(ST)>([&](auto I_) {
        constexpr int i = CI(I_);
        const int dc = cell_at(n, g, -vel(ST, i, 0), -vel(ST, i, 1), -vel(ST, i, 2));
        b[(int64_t)i * g.N + dc] = enc_pop<ST, i, S, T>(f[i]);
      });
    }
  }
}

// --------------------------------------------------------------- launchers
inline dim3 step_grid(const Geo& g) { return dim3((g.nx + LBM_BX - 1) / LBM_BX, g.ny, g.nz); }
inline dim3 pull_grid(const Geo& g, int nzc = 0) {
  return dim3((g.nx + LBM_PULL_BX - 1) / LBM_PULL_BX, g.ny, nzc > 0 ? nzc : g.nz);
}

// forced steps (FP32 / FP64 storage, deviation arithmetic)
template <int ST, class S, class T, int SPACE, bool REG>
void launch_forced(const StepArgs& a, const Rates<T>& keep, const dim3& grid) {
  ForceArg<T> fa;
  for (int d = 0; d < 3; ++d) fa.F[d] = T(a.force[d]);
  fa.field = (const T*)a.force_field;
  auto go = [&](auto force_tag) {
    constexpr int FC = decltype(force_tag)::value;
    if constexpr (FC >= FORCE_UNIFORM_HE && SPACE == SP_CUMULANT) {
      return;  // refused at lbm_set_force_model
    } else if (a.mode == MODE_PULL) {
      PullPtrs<S> P;
      const int64_t nx = a.g.nx, nxy = int64_t(a.g.nx) * a.g.ny;
      for (int i = 0; i < 27; ++i) {
        const int64_t delta =
            i < q_of(ST) ? -(vel(ST, i, 2) * nxy + vel(ST, i, 1) * nx + vel(ST, i, 0)) : 0;
        P.src[i] = i < q_of(ST) ? (const S*)a.src + (int64_t(i) * a.g.N + delta) : nullptr;
        P.dst[i] = i < q_of(ST) ? (S*)a.dst + int64_t(i) * a.g.N : nullptr;
      }
      k_pull<ST, S, T, SPACE, REG, FORM_DEV, FC><<<pull_grid(a.g), LBM_PULL_BX, 0, a.stream>>>(P, a.g, keep, fa);
    } else {
      launch_inplace<ST, S, T, SPACE, REG, FC>(a, keep, grid, fa);
    }
  };
  const bool field = a.force_mode == FORCE_FIELD;
  if (a.force_model == 1) {
    if (field) go(std::integral_constant<int, FORCE_FIELD_HE>{});
    else go(std::integral_constant<int, FORCE_UNIFORM_HE>{});
  } else {
    if (field) go(std::integral_constant<int, FORCE_FIELD>{});
    else go(std::integral_constant<int, FORCE_UNIFORM>{});
  }
}

template <int ST, class S, class T, int SPACE, bool REG>
void launch_step_typed(const StepArgs& a) {
  Rates<T> keep;
  for (int k = 0; k < 6; ++k) keep.om[k] = T(1.0 - a.rates[k]);
  const dim3 grid = step_grid(a.g);
  // forced steps: FP32 / FP64 storage; raw-moment spaces run the general
  // instance (the context clears REG for them), the others keep REG
  if constexpr ((std::is_same<S, float>::value || std::is_same<S, double>::value) &&
                !(REG && (SPACE == SP_RAW || SPACE == SP_RAW_W))) {
    if (a.force_mode != FORCE_NONE) {
      launch_forced<ST, S, T, SPACE, REG>(a, keep, grid);
      return;
    }
  }
  if (a.mode == MODE_PULL) {
    PullPtrs<S> P;
    const int64_t nx = a.g.nx, nxy = int64_t(a.g.nx) * a.g.ny;
    for (int i = 0; i < q_of(ST); ++i) {
      const int64_t delta = -(vel(ST, i, 2) * nxy + vel(ST, i, 1) * nx + vel(ST, i, 0));
      P.src[i] = (const S*)a.src + (int64_t(i) * a.g.N + delta);
      P.dst[i] = (S*)a.dst + int64_t(i) * a.g.N;
    }
    for (int i = q_of(ST); i < 27; ++i) P.src[i] = nullptr, P.dst[i] = nullptr;
    if constexpr (!std::is_same<S, AbsF64>::value) {
      if (a.variant == VARIANT_STAGED && a.form == FORM_DEV) {
        launch_staged<ST, S, T, SPACE, REG>(a);
        return;
      }
    }
    if constexpr (std::is_same<S, AbsF64>::value) {
      if constexpr (ST == D2Q9 && (SPACE == SP_CENTRAL || SPACE == SP_CUMULANT) && !REG) {
        if (a.swe_g > 0.0) {
          k_pull_swe<ST, SPACE><<<grid, LBM_BX, 0, a.stream>>>(P, a.g, keep, a.swe_g);
          return;
        }
      }
      // absolute forms serve SRT and the moment spaces (TRT is refused at create)
      if constexpr (SPACE != SP_TRT)
        k_pull<ST, S, T, SPACE, REG, FORM_ABS_STORE><<<pull_grid(a.g), LBM_PULL_BX, 0, a.stream>>>(P, a.g, keep);
      return;
    } else if constexpr (std::is_same<S, double>::value && SPACE != SP_TRT) {
      if (a.form == FORM_ABS_EQ) {
        k_pull<ST, S, T, SPACE, REG, FORM_ABS_EQ><<<pull_grid(a.g), LBM_PULL_BX, 0, a.stream>>>(P, a.g, keep);
        return;
      }
    }
    // a.nzc > 0: the slab of z-planes [a.z0, a.z0 + a.nzc) only
    if constexpr ((std::is_same<S, float>::value || std::is_same<S, double>::value) &&
                  !(REG && (SPACE == SP_CENTRAL || SPACE == SP_CUMULANT))) {
      if (a.form == FORM_DISC) {
        k_pull<ST, S, T, SPACE, REG, FORM_DISC><<<pull_grid(a.g, a.nzc), LBM_PULL_BX, 0, a.stream>>>(
            P, a.g, keep, ForceArg<T>{}, a.z0);
        return;
      }
    }
    constexpr bool half = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
    if constexpr (half) {
      if (a.g.nx % 2 == 0) {
        Rates<P2> k2;
        for (int k = 0; k < 6; ++k) k2.om[k] = P2(1.0 - a.rates[k]);
        const dim3 grid2((a.g.nx / 2 + LBM_BX - 1) / LBM_BX, a.g.ny, a.nzc > 0 ? a.nzc : a.g.nz);
        if (a.g.nx % 4 == 0 && a.z0 == 0 && (a.nzc == 0 || a.nzc == a.g.nz)) {
          Rates<P4> k4;
          for (int k = 0; k < 6; ++k) k4.om[k] = P4(1.0 - a.rates[k]);
          const dim3 grid4((a.g.nx / 4 + LBM_BX - 1) / LBM_BX, a.g.ny, a.g.nz);
          k_pull4<ST, S, SPACE, REG><<<grid4, LBM_BX, 0, a.stream>>>((const S*)a.src, (S*)a.dst,
                                                                    a.g, k4);
          return;
        }
        k_pull2<ST, S, SPACE, REG><<<grid2, LBM_BX, 0, a.stream>>>((const S*)a.src, (S*)a.dst,
                                                                  a.g, k2, a.z0);
        return;
      }
    }
    k_pull<ST, S, T, SPACE, REG><<<pull_grid(a.g, a.nzc), LBM_PULL_BX, 0, a.stream>>>(
        P, a.g, keep, ForceArg<T>{}, a.z0);
  }
  else {
    // FP16 / BF16 with even Nx: the packed two-cells-per-thread kernel
    if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) {
      if (a.g.nx % 2 == 0) {
        Rates<P2> k2;
        for (int k = 0; k < 6; ++k) k2.om[k] = P2(1.0 - a.rates[k]);
        launch_inplace2<ST, S, SPACE, REG>(a, k2);
        return;
      }
    }
    launch_inplace<ST, S, T, SPACE, REG>(a, keep, grid);
  }
}

template <int ST, class S, class T>
void launch_step_space(const StepArgs& a) {
  switch (a.space * 2 + (a.reg ? 1 : 0)) {
    case SP_SRT * 2:
    case SP_SRT * 2 + 1: launch_step_typed<ST, S, T, SP_SRT, false>(a); break;
    case SP_RAW * 2: launch_step_typed<ST, S, T, SP_RAW, false>(a); break;
    case SP_RAW * 2 + 1: launch_step_typed<ST, S, T, SP_RAW, true>(a); break;
    case SP_RAW_W * 2: launch_step_typed<ST, S, T, SP_RAW_W, false>(a); break;
    case SP_RAW_W * 2 + 1: launch_step_typed<ST, S, T, SP_RAW_W, true>(a); break;
    case SP_CENTRAL * 2: launch_step_typed<ST, S, T, SP_CENTRAL, false>(a); break;
    case SP_CENTRAL * 2 + 1: launch_step_typed<ST, S, T, SP_CENTRAL, true>(a); break;
    case SP_CUMULANT * 2: launch_step_typed<ST, S, T, SP_CUMULANT, false>(a); break;
    case SP_CUMULANT * 2 + 1: launch_step_typed<ST, S, T, SP_CUMULANT, true>(a); break;
    default: launch_step_typed<ST, S, T, SP_TRT, false>(a); break;
  }
}

template <int ST, class S, class T>
void launch_aux_typed(const AuxArgs& a) {
  const dim3 grid = step_grid(a.g);
  const dim3 sgrid((a.g.nx + LBM_BX - 1) / LBM_BX, a.nyc, a.nzc);  // the slab
  const Slab sl{a.y0, a.z0, a.c0, a.stride};
  const int gm = a.gather_mode;
  switch (a.op) {
    case AUX_GATHER: {
      ForceArg<T> fa;
      for (int d = 0; d < 3; ++d) fa.F[d] = T(a.force_mode != FORCE_NONE ? a.force[d] : 0.0);
      fa.field = a.force_mode == FORCE_FIELD ? (const T*)a.force_field : nullptr;
      with_gather_mode(gm, [&](auto mode) {
        k_gather<ST, S, T, decltype(mode)::value>
            <<<sgrid, LBM_BX, 0, a.stream>>>((const S*)a.buf, a.g, a.df, a.rho, a.u, sl, fa);
      });
      break;
    }
    case AUX_SCATTER: {
      if constexpr (ST == D2Q9 && std::is_same<S, AbsF64>::value) {
        if (a.swe_g > 0.0 && !a.df_in) {
          if (a.space == SP_CENTRAL)
            k_scatter_swe<ST, SP_CENTRAL><<<grid, LBM_BX, 0, a.stream>>>((AbsF64*)a.buf, a.g, a.rho_in, a.u_in, a.swe_g);
          else
            k_scatter_swe<ST, SP_CUMULANT><<<grid, LBM_BX, 0, a.stream>>>((AbsF64*)a.buf, a.g, a.rho_in, a.u_in, a.swe_g);
          break;
        }
      }
      const bool raw = a.space == SP_RAW || a.space == SP_SRT || a.space == SP_TRT ||
                       a.space == SP_RAW_W;
      auto go = [&](auto layout) {
        constexpr int LY = decltype(layout)::value;
        if (a.disc)
          k_scatter<ST, S, T, SP_RAW, LY, true><<<sgrid, LBM_BX, 0, a.stream>>>((S*)a.buf, a.g, a.df_in, a.rho_in, a.u_in, sl);
        else if (raw)
          k_scatter<ST, S, T, SP_RAW, LY><<<sgrid, LBM_BX, 0, a.stream>>>((S*)a.buf, a.g, a.df_in, a.rho_in, a.u_in, sl);
        else
          k_scatter<ST, S, T, SP_CENTRAL, LY><<<sgrid, LBM_BX, 0, a.stream>>>((S*)a.buf, a.g, a.df_in, a.rho_in, a.u_in, sl);
      };
      switch (gm) {  // scatter writes the even-parity layout of each pattern
        case G_PULL: go(std::integral_constant<int, G_PULL>{}); break;
        case G_ET_EVEN: go(std::integral_constant<int, G_ET_EVEN>{}); break;
        case G_EPULL_EVEN: go(std::integral_constant<int, G_EPULL_EVEN>{}); break;
        case G_EPUSH_EVEN: go(std::integral_constant<int, G_EPUSH_EVEN>{}); break;
        default: go(std::integral_constant<int, G_LOCAL>{}); break;
      }
      break;
    }
    case AUX_INVARIANTS:
      with_gather_mode(gm, [&](auto mode) {
        k_invariants<ST, S, T, decltype(mode)::value>
            <<<a.nparts, INV_THREADS, 0, a.stream>>>((const S*)a.buf, a.g, a.part);
      });
      break;
  }
}

template <int ST, class S, class T, int SPACE, bool REG>
void launch_batch_typed(const BatchArgs& a) {
  if (a.op == BATCH_TGV) {
    k_batch_tgv<ST, S, T, (SPACE == SP_RAW || SPACE == SP_SRT || SPACE == SP_TRT || SPACE == SP_RAW_W ? SP_RAW : SP_CENTRAL)>
        <<<a.grid, a.threads, 0, a.stream>>>((S*)a.dst, a.inst, a.tiles, a.ntiles, a.cpt, a.u0);
    return;
  }
  Rates<T> keep;
  for (int k = 0; k < 6; ++k) keep.om[k] = T(1.0 - a.rates[k]);
  k_batch_pull<ST, S, T, SPACE, REG><<<a.grid, a.threads, 0, a.stream>>>(
      (const S*)a.src, (S*)a.dst, a.inst, a.tiles, a.ntiles, a.cpt, keep);
}

template <int ST, class S, class T>
void launch_batch_space(const BatchArgs& a) {
  switch (a.space * 2 + (a.reg ? 1 : 0)) {
    case SP_SRT * 2:
    case SP_SRT * 2 + 1: launch_batch_typed<ST, S, T, SP_SRT, false>(a); break;
    case SP_RAW * 2: launch_batch_typed<ST, S, T, SP_RAW, false>(a); break;
    case SP_RAW * 2 + 1: launch_batch_typed<ST, S, T, SP_RAW, true>(a); break;
    case SP_RAW_W * 2: launch_batch_typed<ST, S, T, SP_RAW_W, false>(a); break;
    case SP_RAW_W * 2 + 1: launch_batch_typed<ST, S, T, SP_RAW_W, true>(a); break;
    case SP_CENTRAL * 2: launch_batch_typed<ST, S, T, SP_CENTRAL, false>(a); break;
    case SP_CENTRAL * 2 + 1: launch_batch_typed<ST, S, T, SP_CENTRAL, true>(a); break;
    case SP_CUMULANT * 2: launch_batch_typed<ST, S, T, SP_CUMULANT, false>(a); break;
    case SP_CUMULANT * 2 + 1: launch_batch_typed<ST, S, T, SP_CUMULANT, true>(a); break;
    default: launch_batch_typed<ST, S, T, SP_TRT, false>(a); break;
  }
}

}  // namespace lbm
