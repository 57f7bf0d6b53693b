// lbm_staged.cuh -- pull step with the gather staged through shared memory
// by the bulk-copy (TMA) engine.
//
// The pull gather of one x-row (y, z) of cells reads, for every direction
// i, one whole x-row of plane i: row (y - xi_iy, z - xi_iz), periodic.  A
// persistent CTA owns rows r = blockIdx.x + k * gridDim.x; for each it
// issues q one-dimensional bulk copies global -> shared (one per direction,
// the full row, so the x wrap is resolved by indexing in shared memory) that
// complete on one mbarrier, and keeps `stages` rows (up to the compile-time
// cap, as many as fit the shared-memory budget) in flight while it collides
// the current one.  The copies need no registers and no warps, so
// the bytes in flight per SM no longer depend on the occupancy of the
// (register-heavy) collision.  Stores go straight from registers to global
// memory, coalesced along x.
//
// Requirements (checked by the host before choosing this path): pull
// streaming, each row a multiple of 16 bytes (bulk-copy granularity; the
// plane bases are then 16-byte aligned too), and the stage buffers within the
// shared-memory budget below.  Every wait on an mbarrier is bounded; a wait
// that runs out sets *status, waits (bounded) for the CTA's copies still in
// flight and returns.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_packed.cuh"

namespace lbm {

namespace tma {

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// default limit of a device wait: 2^31 SM cycles (about 1 s)
constexpr long long kWaitLimit = 1ll << 31;
// wait for the phase with the given parity to complete; false once `limit`
// SM cycles have passed without completion (0: at the first unsuccessful
// test)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitLimit) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 >= limit) return false;
    __nanosleep(40);
  }
  return true;
}

}  // namespace tma

// Plane base pointers (unshifted) of the staged kernels.
template <class S>
struct RowPtrs {
  const S* src[27];
  S* dst[27];
};

constexpr int STG_NT = 256;  // threads per CTA

// The row pipeline: calls body(rows_of_stage, r) for every row r of this
// CTA, with rows_of_stage[i * nx + x] = plane i of row (y - xi_iy, z - xi_iz).
// `limit` bounds each wait for a row's copies; the drain after a timeout
// waits with the default limit, so every copy issued lands before the CTA
// exits.
template <int ST, class S, class Body>
__device__ __forceinline__ void staged_rows(const RowPtrs<S>& P, const Geo& g, int stages,
                                            int* status, long long limit, Body&& body) {
  constexpr int Q = q_of(ST);
  extern __shared__ __align__(128) unsigned char stg_raw[];
  __shared__ __align__(8) uint64_t bar[STG_MAX_STAGES];
  __shared__ int abort_all;
  S* const stage = reinterpret_cast<S*>(stg_raw);
  const int nx = g.nx;
  const int rows = g.ny * g.nz;
  const int G = gridDim.x;
  const int b = blockIdx.x;
  const int K = b < rows ? (rows - 1 - b) / G + 1 : 0;
  const uint32_t row_bytes = uint32_t(nx) * uint32_t(sizeof(S));
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) tma::mbar_init(&bar[s], 1);
    tma::fence_init();
    abort_all = 0;
  }
  __syncthreads();
  auto issue = [&](int s, int r) {
    const int y = r % g.ny, z = r / g.ny;
    tma::mbar_expect_tx(&bar[s], row_bytes * uint32_t(Q));
    sfor<Q>([&](auto I) {
      constexpr int i = CI(I);
      constexpr int cy = vel(ST, i, 1), cz = vel(ST, i, 2);
      int ys = y - cy, zs = z - cz;
      ys += ys < 0 ? g.ny : (ys >= g.ny ? -g.ny : 0);
      zs += zs < 0 ? g.nz : (zs >= g.nz ? -g.nz : 0);
      tma::bulk_g2s(stage + (int64_t(s) * Q + i) * nx, P.src[i] + (int64_t(zs) * g.ny + ys) * nx,
                    row_bytes, &bar[s]);
    });
  };
  if (threadIdx.x == 0)
    for (int s = 0; s < stages && s < K; ++s) issue(s, b + s * G);
  int k = 0;
  for (; k < K; ++k) {
    const int s = k % stages;
    const int r = b + k * G;
    if (!tma::mbar_wait(&bar[s], uint32_t(k / stages) & 1u, limit)) abort_all = 1;
    __syncthreads();
    if (abort_all) break;
    body(static_cast<const S*>(stage + int64_t(s) * Q * nx), r);
    __syncthreads();  // every thread is done reading stage s
    if (threadIdx.x == 0 && k + stages < K) issue(s, r + stages * G);
  }
  if (abort_all && threadIdx.x == 0) {
    atomicExch(status, 1);
    // rows k .. k + stages - 1 were issued: let them land before exit
    for (int j = k; j < K && j < k + stages; ++j)
      tma::mbar_wait(&bar[j % stages], uint32_t(j / stages) & 1u);
  }
}

// Two cells per thread on packed FP32 pairs (FP16 / BF16 delta storage); the
// same per-cell arithmetic as k_pull2, so the results are bitwise equal.
template <int ST, class S, int SPACE, bool REG>
__global__ void __launch_bounds__(STG_NT, 3) k_pull2_staged(const __grid_constant__ RowPtrs<S> P,
                                                          Geo g, Rates<P2> keep, int stages,
                                                          int* status, long long limit) {
  constexpr int Q = q_of(ST);
  staged_rows<ST, S>(P, g, stages, status, limit, [&](const S* row, int r) {
    const int nx = g.nx;
    const int cbase = r * nx;
#pragma unroll 1
    for (int x = 2 * int(threadIdx.x); x < nx; x += 2 * STG_NT) {
      const int xm = x == 0 ? nx - 1 : x - 1;
      const int xp2 = x + 2 == nx ? 0 : x + 2;
      P2 f[Q];
      sfor<Q>([&](auto I) {
        constexpr int i = CI(I);
        constexpr int cx = vel(ST, i, 0);
        const S* rw = row + i * nx;
        constexpr int E = scale_exp(ST, i);
        if constexpr (cx == 0) f[i] = Pack<S>::template load2s<E>(rw + x);
        else if constexpr (cx > 0) f[i] = Pack<S>::template load11s<E>(rw + xm, rw + x);
        else f[i] = Pack<S>::template load11s<E>(rw + x + 1, rw + xp2);
      });
      collide<ST, P2, SPACE, REG, true>(f, keep);
      sfor<Q>([&](auto I) {
        constexpr int i = CI(I);
        constexpr int k = vel(ST, i, 0) * vel(ST, i, 0) + vel(ST, i, 1) * vel(ST, i, 1) +
                          vel(ST, i, 2) * vel(ST, i, 2);
        Pack<S>::store2(P.dst[i] + cbase + x, f[i] * P2(float(1u << (scale_exp(ST, i) - k))));
      });
    }
  });
}

// One cell per thread (FP32 / FP64 storage, deviation arithmetic); the same
// per-cell arithmetic as k_pull.
template <int ST, class S, class T, int SPACE, bool REG>
__global__ void __launch_bounds__(STG_NT, 2) k_pull_staged(const __grid_constant__ RowPtrs<S> P,
                                                         Geo g, Rates<T> keep, int stages,
                                                         int* status, long long limit) {
  constexpr int Q = q_of(ST);
  staged_rows<ST, S>(P, g, stages, status, limit, [&](const S* row, int r) {
    const int nx = g.nx;
    const int cbase = r * nx;
#pragma unroll 1
    for (int x = int(threadIdx.x); x < nx; x += STG_NT) {
      const int xm = x == 0 ? nx - 1 : x - 1;
      const int xp = x + 1 == nx ? 0 : x + 1;
      T f[Q];
      sfor<Q>([&](auto I) {
        constexpr int i = CI(I);
        constexpr int cx = vel(ST, i, 0);
        const int xs = cx > 0 ? xm : (cx < 0 ? xp : x);
        f[i] = Codec<S>::template dec<T>(row[i * nx + xs], scale_exp(ST, i));
      });
      collide<ST, T, SPACE, REG>(f, keep);
      sfor<Q>([&](auto I) {
        constexpr int i = CI(I);
        P.dst[i][cbase + x] = Codec<S>::template enc<T>(f[i], scale_exp(ST, i));
      });
    }
  });
}

// Persistent grid of the staged kernels: every CTA that fits on the device.
template <class K>
int staged_grid(K kernel, int smem, int rows) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  static int last_smem = -1, occ = 1;
  if (smem != last_smem) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, STG_NT, smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
    last_smem = smem;
  }
  const int64_t grid = int64_t(sms) * occ;
  return int(grid < rows ? grid : rows);
}

template <int ST, class S, class T, int SPACE, bool REG>
void launch_staged(const StepArgs& a) {
  constexpr int Q = q_of(ST);
  RowPtrs<S> P;
  for (int i = 0; i < 27; ++i) {
    P.src[i] = i < Q ? (const S*)a.src + int64_t(i) * a.g.N : nullptr;
    P.dst[i] = i < Q ? (S*)a.dst + int64_t(i) * a.g.N : nullptr;
  }
  const int stages = staged_stages(Q, a.g.nx, sizeof(S));
  const int smem = int(staged_smem_bytes(Q, a.g.nx, sizeof(S)));
  const int rows = a.g.ny * a.g.nz;
  constexpr bool half = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
  if constexpr (half) {
    auto kern = k_pull2_staged<ST, S, SPACE, REG>;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_MAX_SMEM);
      attr = true;
    }
    Rates<P2> k2;
    for (int k = 0; k < 6; ++k) k2.om[k] = P2(1.0 - a.rates[k]);
    kern<<<staged_grid(kern, smem, rows), STG_NT, smem, a.stream>>>(P, a.g, k2, stages, a.status,
                                                                    a.wait_limit);
  } else {
    auto kern = k_pull_staged<ST, S, T, SPACE, REG>;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, STG_MAX_SMEM);
      attr = true;
    }
    Rates<T> keep;
    for (int k = 0; k < 6; ++k) keep.om[k] = T(1.0 - a.rates[k]);
    kern<<<staged_grid(kern, smem, rows), STG_NT, smem, a.stream>>>(P, a.g, keep, stages,
                                                                    a.status, a.wait_limit);
  }
}

}  // namespace lbm
