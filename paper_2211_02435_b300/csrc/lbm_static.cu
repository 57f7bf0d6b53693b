// lbm_static.cu -- lbm_invariants_noalloc: the FP64 invariant reduction of
// a caller-owned population field with its scratch in a fixed, file-scope
// device array instead of memory obtained from cudaMalloc.
//
// Why: some callers must not allocate device memory at all -- code that runs
// inside a framework that owns the whole device pool, real-time loops where
// an allocation could block or fail mid-run, or hosts that hand this library
// a buffer and nothing else.  They still pass their inputs (the populations)
// and their outputs (8 doubles); the partial sums live in g_inv_scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int kRows = LBM_STATIC_SCRATCH_ROWS;  // partial-sum rows, one per block
constexpr int kMaxDevices = 64;

// Shared by every call on a device; kept until the process exits.  The
// reduction writes every row it later reads, so nothing needs clearing.
static __device__ __align__(256) double g_inv_scratch[kRows * 8 + 8];

// Device address of g_inv_scratch per device.  In host code the symbol name
// is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_inv_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LBM_OK;
}

template <int ST, class S, class T>
void launch_local(const void* df, const lbm::Geo& g, double* part, int rows, cudaStream_t s) {
  lbm::k_invariants<ST, S, T, lbm::G_LOCAL><<<rows, lbm::INV_THREADS, 0, s>>>((const S*)df, g, part);
}

template <int ST>
void launch_stencil(int storage, const void* df, const lbm::Geo& g, double* part, int rows,
                    cudaStream_t s) {
  switch (storage) {
    case LBM_STORE_F64: launch_local<ST, double, double>(df, g, part, rows, s); break;
    case LBM_STORE_F32: launch_local<ST, float, float>(df, g, part, rows, s); break;
    case LBM_STORE_F16_DELTA: launch_local<ST, __half, float>(df, g, part, rows, s); break;
    default: launch_local<ST, __nv_bfloat16, float>(df, g, part, rows, s); break;
  }
}

}  // namespace

extern "C" int lbm_invariants_noalloc(int stencil, int storage, const void* df,
                                      const int64_t dims[3], double out[8], int on_device,
                                      void* stream) {
  if (stencil < 0 || stencil > 2 || storage < 0 || storage > 3 || !df || !dims || !out)
    return LBM_ERR_INVALID;
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (stencil == LBM_D2Q9 && dims[2] != 1))
    return LBM_ERR_INVALID;
  // more cells than one call serves; every extent is bounded before any
  // product is formed (Nx * Ny < 2^62 then fits), and Nz is compared by
  // division, so no size wraps around int64
  constexpr int64_t kLim = LBM_STATIC_MAX_CELLS;
  if (dims[0] > kLim || dims[1] > kLim || dims[2] > kLim) return LBM_ERR_INVALID;
  const int64_t nxy = dims[0] * dims[1];
  if (nxy > kLim || dims[2] > kLim / nxy) return LBM_ERR_INVALID;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != LBM_OK) return rc;
  lbm::Geo g;
  g.nx = int(dims[0]);
  g.ny = int(dims[1]);
  g.nz = int(dims[2]);
  g.N = dims[0] * dims[1] * dims[2];
  const int64_t blocks = (g.N + lbm::INV_THREADS - 1) / lbm::INV_THREADS;
  const int rows = int(blocks < kRows ? blocks : kRows);
  cudaStream_t s = (cudaStream_t)stream;
  if (stencil == LBM_D2Q9) launch_stencil<lbm::D2Q9>(storage, df, g, scratch, rows, s);
  else if (stencil == LBM_D3Q19) launch_stencil<lbm::D3Q19>(storage, df, g, scratch, rows, s);
  else launch_stencil<lbm::D3Q27>(storage, df, g, scratch, rows, s);
  double* result = on_device ? out : scratch + size_t(kRows) * 8;
  lbm::launch_invariants_fold(scratch, rows, result, s);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  if (on_device) return LBM_OK;
  rc = cudaMemcpyAsync(out, result, 8 * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess
           ? LBM_OK
           : LBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = LBM_ERR_CUDA;
  if (rc == LBM_OK && out[6] > 0) rc = LBM_ERR_DIVERGED;
  return rc;
}
