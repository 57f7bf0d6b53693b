// lbm_api.cu -- C ABI (include/lbm.h): context management, validation,
// buffer bookkeeping of the pull / AA streaming patterns and dispatch to
// the per-(stencil, storage) kernel instantiations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

using lbm::AuxArgs;
using lbm::Geo;
using lbm::StepArgs;

typedef void (*step_fn)(const StepArgs&);
typedef void (*aux_fn)(const AuxArgs&);

const step_fn kStep[3][5] = {
    {lbm::launch_step_0_0, lbm::launch_step_0_1, lbm::launch_step_0_2, lbm::launch_step_0_3,
     lbm::launch_step_0_4},
    {lbm::launch_step_1_0, lbm::launch_step_1_1, lbm::launch_step_1_2, lbm::launch_step_1_3,
     lbm::launch_step_1_4},
    {lbm::launch_step_2_0, lbm::launch_step_2_1, lbm::launch_step_2_2, lbm::launch_step_2_3,
     lbm::launch_step_2_4}};
const aux_fn kAux[3][5] = {
    {lbm::launch_aux_0_0, lbm::launch_aux_0_1, lbm::launch_aux_0_2, lbm::launch_aux_0_3,
     lbm::launch_aux_0_4},
    {lbm::launch_aux_1_0, lbm::launch_aux_1_1, lbm::launch_aux_1_2, lbm::launch_aux_1_3,
     lbm::launch_aux_1_4},
    {lbm::launch_aux_2_0, lbm::launch_aux_2_1, lbm::launch_aux_2_2, lbm::launch_aux_2_3,
     lbm::launch_aux_2_4}};

constexpr int G_PULL = 0, G_LOCAL = 1, G_AAODD = 2;
// esoteric pattern k (Twist 0, Pull 1, Push 2) at parity p: 3 + 2 k + p,
// equal to the step modes MODE_ET_EVEN .. MODE_EPUSH_ODD
constexpr int G_ESO_BASE = 3;
static_assert(lbm::MODE_ET_EVEN == G_ESO_BASE && lbm::MODE_EPULL_EVEN == G_ESO_BASE + 2 &&
                  lbm::MODE_EPUSH_ODD == G_ESO_BASE + 5,
              "esoteric gather and step modes share their numbering");
bool esoteric(int streaming) {
  return streaming == LBM_ESOTERIC_TWIST || streaming == LBM_ESOTERIC_PULL ||
         streaming == LBM_ESOTERIC_PUSH;
}
int eso_mode(int streaming, int parity) {
  return G_ESO_BASE + 2 * (streaming - LBM_ESOTERIC_TWIST) + parity;
}
constexpr uint64_t kStateMagic = 0x4c424d3253544154ull;  // "LBM2STAT"

int q_of(int st) { return st == LBM_D2Q9 ? 9 : (st == LBM_D3Q19 ? 19 : 27); }
int elem_bytes(int storage) {
  return (storage == LBM_STORE_F64 || storage == LBM_STORE_F64_ABSOLUTE)
             ? 8
             : (storage == LBM_STORE_F32 ? 4 : 2);
}

struct StateHeader {
  uint64_t magic;
  int32_t stencil, space, equilibrium, storage, streaming, parity;
  int64_t dims[3];
  int64_t t;
  int64_t payload;
};

}  // namespace



namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

int gather_mode(const lbm_ctx* c) {
  if (c->p.streaming == LBM_PULL) return G_PULL;
  if (esoteric(c->p.streaming)) return eso_mode(c->p.streaming, c->parity);
  return c->parity ? G_AAODD : G_LOCAL;
}
void* state_buf(const lbm_ctx* c) {
  return c->p.streaming == LBM_PULL ? c->buf[c->cur] : c->buf[0];
}

void set_effective_rates(lbm_ctx* c, const double* r) {
  for (int k = 0; k < 6; ++k) c->rates[k] = c->p.space == LBM_SPACE_POPULATIONS ? r[0] : r[k];
  c->space = c->p.space;  // POPULATIONS / TRT: population-space kernels
  c->reg = c->p.space != LBM_SPACE_POPULATIONS && c->p.space != LBM_SPACE_TRT;
  for (int k = 1; k < 6; ++k)
    if (c->rates[k] != 1.0) c->reg = 0;
}

int valid_rates(const double* r) {
  for (int k = 0; k < 6; ++k)
    if (!(r[k] > 0.0 && r[k] <= 2.0)) return 0;
  return 1;
}

AuxArgs aux_base(const lbm_ctx* c, int op) {
  AuxArgs a;
  std::memset(&a, 0, sizeof(a));
  a.op = op;
  a.buf = state_buf(c);
  a.g = c->g;
  a.storage = c->p.storage;
  a.space = c->space;
  a.gather_mode = gather_mode(c);
  a.force_mode = c->force_mode;
  for (int d = 0; d < 3; ++d) a.force[d] = c->force[d];
  a.force_field = c->force_field;
  a.swe_g = c->swe_g;
  a.disc = c->p.equilibrium == LBM_EQ_DISCRETE2;
  a.stream = c->stream;
  lbm::whole_slab(a);
  return a;
}

// Copy a host array to a temporary device buffer (or pass a device pointer
// through).  The caller frees *tmp after synchronising the stream.
int stage_in(const lbm_ctx* c, const double* p, size_t n, int on_device, const double** dev,
             double** tmp) {
  *tmp = nullptr;
  if (!p || on_device) {
    *dev = p;
    return LBM_OK;
  }
  if (cudaMalloc((void**)tmp, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *tmp = nullptr;
    return LBM_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(*tmp, p, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  *dev = *tmp;
  return cuda_err(e);
}

}  // namespace

namespace lbm {

__global__ void __launch_bounds__(256) k_invariants_fold(const double* part, int nparts,
                                                        double* out) {
  __shared__ double sh[256][8];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = threadIdx.x; r < nparts; r += 256)
    for (int k = 0; k < 8; ++k)
      acc[k] = k == 5 ? fmax(acc[k], part[(int64_t)r * 8 + k]) : acc[k] + part[(int64_t)r * 8 + k];
  for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 8; ++k)
        sh[threadIdx.x][k] = k == 5 ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                    : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
    __syncthreads();
  }
  if (threadIdx.x < 8) out[threadIdx.x] = sh[0][threadIdx.x];
}

void launch_invariants_fold(const double* part, int nparts, double* out, cudaStream_t s) {
  k_invariants_fold<<<1, 256, 0, s>>>(part, nparts, out);
}

void dispatch_step(int stencil, int storage, const StepArgs& a) { kStep[stencil][storage](a); }
void dispatch_aux(int stencil, int storage, const AuxArgs& a) { kAux[stencil][storage](a); }

typedef void (*batch_fn)(const BatchArgs&);
static const batch_fn kBatch[3][5] = {
    {launch_batch_0_0, launch_batch_0_1, launch_batch_0_2, launch_batch_0_3, launch_batch_0_4},
    {launch_batch_1_0, launch_batch_1_1, launch_batch_1_2, launch_batch_1_3, launch_batch_1_4},
    {launch_batch_2_0, launch_batch_2_1, launch_batch_2_2, launch_batch_2_3, launch_batch_2_4}};
void dispatch_batch(int stencil, int storage, const BatchArgs& a) { kBatch[stencil][storage](a); }

}  // namespace lbm

extern "C" {

const char* lbm_error_string(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_INVALID: return "invalid argument";
    case LBM_ERR_UNSUPPORTED: return "unsupported";
    case LBM_ERR_INADMISSIBLE: return "inadmissible method combination";
    case LBM_ERR_OOM: return "device out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_DIVERGED: return "non-finite populations";
    case LBM_ERR_STATE_MISMATCH: return "state does not match this context";
    case LBM_ERR_TIMEOUT: return "a kernel's bounded wait ran out";
    default: return "unknown error";
  }
}

int lbm_create(lbm_ctx** out, const lbm_params* p) {
  if (!out || !p) return LBM_ERR_INVALID;
  *out = nullptr;
  if (p->stencil < 0 || p->stencil > 2 || p->space < 0 || p->space > 5 || p->storage < 0 ||
      p->storage > 4 || p->streaming < 0 || p->streaming > 4 ||
      (p->equilibrium != LBM_EQ_DELTA && p->equilibrium != LBM_EQ_ABSOLUTE &&
       p->equilibrium != LBM_EQ_DISCRETE2) ||
      (p->arithmetic != LBM_ARITH_DEVIATION && p->arithmetic != LBM_ARITH_AS_WRITTEN))
    return LBM_ERR_INVALID;
  // Sec. 3: no zero-centered cumulants; delta-equilibria need zero-centered storage
  if (p->space == LBM_SPACE_CUMULANT && p->equilibrium == LBM_EQ_DELTA)
    return LBM_ERR_INADMISSIBLE;
  if (p->storage == LBM_STORE_F64_ABSOLUTE && p->equilibrium == LBM_EQ_DELTA)
    return LBM_ERR_INADMISSIBLE;
  // the discrete equilibrium: FP64 / FP32 deviations, pull streaming
  if (p->equilibrium == LBM_EQ_DISCRETE2 &&
      ((p->storage != LBM_STORE_F64 && p->storage != LBM_STORE_F32) ||
       p->streaming != LBM_PULL || p->arithmetic != LBM_ARITH_DEVIATION))
    return LBM_ERR_UNSUPPORTED;
  if ((p->storage == LBM_STORE_F64_ABSOLUTE || p->arithmetic == LBM_ARITH_AS_WRITTEN) &&
      (p->streaming != LBM_PULL || p->space == LBM_SPACE_TRT ||
       (p->storage != LBM_STORE_F64 && p->storage != LBM_STORE_F64_ABSOLUTE)))
    return LBM_ERR_UNSUPPORTED;
  if (p->boundary != LBM_PERIODIC) return LBM_ERR_UNSUPPORTED;
  for (int k = 0; k < 3; ++k)
    if (p->dims[k] < 1) return LBM_ERR_INVALID;
  if (p->stencil == LBM_D2Q9 && p->dims[2] != 1) return LBM_ERR_INVALID;
  if (p->dims[1] > 65535 || p->dims[2] > 65535) return LBM_ERR_INVALID;
  if (p->dims[0] >= (int64_t(1) << 31) || p->dims[1] * p->dims[0] >= (int64_t(1) << 31))
    return LBM_ERR_INVALID;
  if (!lbm::index_fits(p->dims[0], p->dims[1], p->dims[2], p->stencil == LBM_D2Q9 ? 2 : 3))
    return LBM_ERR_INVALID;
  const int64_t N = p->dims[0] * p->dims[1] * p->dims[2];
  if (!valid_rates(p->rates)) return LBM_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }

  lbm_ctx* c = new (std::nothrow) lbm_ctx;
  if (!c) return LBM_ERR_OOM;
  std::memset(c, 0, sizeof(*c));
  c->p = *p;
  c->q = q_of(p->stencil);
  c->d = p->stencil == LBM_D2Q9 ? 2 : 3;
  c->g.nx = int(p->dims[0]);
  c->g.ny = int(p->dims[1]);
  c->g.nz = int(p->dims[2]);
  c->g.N = N;
  c->eb = elem_bytes(p->storage);
  c->stream = (cudaStream_t)p->stream;
  c->wait_limit = LBM_WAIT_LIMIT_DEFAULT;
  set_effective_rates(c, p->rates);
  const size_t bytes = size_t(c->q) * size_t(N) * size_t(c->eb);
  const int nbuf = p->streaming == LBM_PULL ? 2 : 1;
  for (int b = 0; b < nbuf; ++b) {
    if (cudaMalloc(&c->buf[b], bytes) != cudaSuccess) {
      cudaGetLastError();
      c->buf[b] = nullptr;
      lbm_destroy(c);
      return LBM_ERR_OOM;
    }
    if (cudaMemsetAsync(c->buf[b], 0, bytes, c->stream) != cudaSuccess) {
      lbm_destroy(c);
      return LBM_ERR_CUDA;
    }
  }
  const int64_t np = (N + 255) / 256;
  c->nparts = int(np < 148 * 8 ? np : 148 * 8);
  // invariants scratch (nparts rows + 8 results) and one status word
  if (cudaMalloc((void**)&c->part, sizeof(double) * (size_t(c->nparts) * 8 + 9)) != cudaSuccess) {
    cudaGetLastError();
    c->part = nullptr;
    lbm_destroy(c);
    return LBM_ERR_OOM;
  }
  c->status = reinterpret_cast<int*>(c->part + size_t(c->nparts) * 8 + 8);
  if (cudaMemsetAsync(c->status, 0, sizeof(int), c->stream) != cudaSuccess) {
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->io_stream) {
    cudaStreamSynchronize(c->io_stream);
    cudaStreamDestroy(c->io_stream);
    for (int b = 0; b < 2; ++b) {
      cudaEventDestroy(c->io_ready[b]);
      cudaEventDestroy(c->io_done[b]);
    }
  }
  for (int b = 0; b < 2; ++b) {
    if (c->io_buf[b]) cudaFree(c->io_buf[b]);
    if (c->buf[b]) cudaFree(c->buf[b]);
  }
  if (c->run_buf) cudaFree(c->run_buf);
  if (c->part) cudaFree(c->part);
  if (c->closure) lbm::free_closure(c->closure);
  if (c->force_field) cudaFree(c->force_field);
  delete c;
}

// ------------------------------------------------------------ body force
namespace {

__global__ void k_f64_to_f32(const double* in, float* out, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = float(in[k]);
}

bool force_served(const lbm_ctx* c) {
  return (c->p.storage == LBM_STORE_F64 || c->p.storage == LBM_STORE_F32) &&
         c->p.arithmetic == LBM_ARITH_DEVIATION && !c->closure && !(c->swe_g > 0.0) &&
         c->p.equilibrium != LBM_EQ_DISCRETE2;
}

void update_force_mode(lbm_ctx* c) {
  const bool uni = c->force[0] != 0.0 || c->force[1] != 0.0 || c->force[2] != 0.0;
  c->force_mode = c->force_field ? lbm::FORCE_FIELD : (uni ? lbm::FORCE_UNIFORM : lbm::FORCE_NONE);
}

}  // namespace

int lbm_set_force_model(lbm_ctx* c, int model) {
  if (!c || (model != LBM_FORCE_GUO && model != LBM_FORCE_HE)) return LBM_ERR_INVALID;
  if (model == LBM_FORCE_HE && c->p.space == LBM_SPACE_CUMULANT) return LBM_ERR_UNSUPPORTED;
  c->force_model = model;
  return LBM_OK;
}

int lbm_set_force(lbm_ctx* c, const double* F) {
  if (!c) return LBM_ERR_INVALID;
  if (F) {
    for (int d = 0; d < c->d; ++d)
      if (!std::isfinite(F[d])) return LBM_ERR_INVALID;
    if (!force_served(c)) return LBM_ERR_UNSUPPORTED;
  }
  for (int d = 0; d < 3; ++d) c->force[d] = (F && d < c->d) ? F[d] : 0.0;
  update_force_mode(c);
  return LBM_OK;
}

int lbm_set_force_field(lbm_ctx* c, const double* F, int on_device) {
  if (!c) return LBM_ERR_INVALID;
  if (!F) {
    if (c->force_field) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->force_field);
      c->force_field = nullptr;
    }
    update_force_mode(c);
    return LBM_OK;
  }
  if (!force_served(c)) return LBM_ERR_UNSUPPORTED;
  const int64_t n = int64_t(c->d) * c->g.N;
  const size_t eb = c->p.storage == LBM_STORE_F64 ? sizeof(double) : sizeof(float);
  void* dev = nullptr;
  if (cudaMalloc(&dev, size_t(n) * eb) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  int rc = LBM_OK;
  if (eb == sizeof(double)) {
    rc = cuda_err(cudaMemcpyAsync(dev, F, size_t(n) * eb,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream));
  } else if (on_device) {
    k_f64_to_f32<<<unsigned((n + 255) / 256), 256, 0, c->stream>>>(F, (float*)dev, n);
    rc = cuda_err(cudaGetLastError());
  } else {
    float* h = new (std::nothrow) float[size_t(n)];
    if (!h) rc = LBM_ERR_OOM;
    else {
      for (int64_t k = 0; k < n; ++k) h[k] = float(F[k]);
      rc = cuda_err(cudaMemcpyAsync(dev, h, size_t(n) * eb, cudaMemcpyHostToDevice, c->stream));
      if (cudaStreamSynchronize(c->stream) != cudaSuccess && rc == LBM_OK) rc = LBM_ERR_CUDA;
      delete[] h;
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess && rc == LBM_OK) rc = LBM_ERR_CUDA;
  if (rc != LBM_OK) {
    cudaFree(dev);
    return rc;
  }
  if (c->force_field) cudaFree(c->force_field);
  c->force_field = dev;
  update_force_mode(c);
  return LBM_OK;
}

int lbm_set_shallow_water(lbm_ctx* c, double g) {
  if (!c || !(g >= 0.0) || !std::isfinite(g)) return LBM_ERR_INVALID;
  if (g > 0.0 &&
      (c->p.stencil != LBM_D2Q9 || c->p.storage != LBM_STORE_F64_ABSOLUTE ||
       c->p.equilibrium != LBM_EQ_ABSOLUTE || c->p.streaming != LBM_PULL ||
       (c->p.space != LBM_SPACE_CENTRAL && c->p.space != LBM_SPACE_CUMULANT) || c->force_mode))
    return LBM_ERR_UNSUPPORTED;
  c->swe_g = g;
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
  if (!c) return LBM_ERR_INVALID;
  c->stream = (cudaStream_t)stream;
  c->p.stream = stream;
  return LBM_OK;
}

int lbm_set_rates(lbm_ctx* c, const double rates[6]) {
  if (!c || !rates || !valid_rates(rates)) return LBM_ERR_INVALID;
  for (int k = 0; k < 6; ++k) c->p.rates[k] = rates[k];
  set_effective_rates(c, rates);
  return LBM_OK;
}

int lbm_get_time(const lbm_ctx* c, int64_t* step, int* parity) {
  if (!c) return LBM_ERR_INVALID;
  if (step) *step = c->t;
  if (parity) *parity = c->parity;
  return LBM_OK;
}

static int scatter_layout(const lbm_ctx* c) {
  return c->p.streaming == LBM_PULL
             ? G_PULL
             : (esoteric(c->p.streaming) ? eso_mode(c->p.streaming, 0) : G_LOCAL);
}

static int scatter(lbm_ctx* c, const double* df, const double* rho, const double* u) {
  if (c->p.streaming != LBM_PULL) c->parity = 0;
  AuxArgs a = aux_base(c, lbm::AUX_SCATTER);
  a.gather_mode = scatter_layout(c);
  a.df_in = df;
  a.rho_in = rho;
  a.u_in = u;
  kAux[c->p.stencil][c->p.storage](a);
  return cuda_err(cudaGetLastError());
}

// NVTX range over a host entry point (visible in Nsight timelines)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static int read_status(lbm_ctx* c);

// ------------------------------------------------ host transfers in slabs
// Host arrays are moved slab by slab: a slab is a run of z-planes (of y-rows
// when Nz = 1) whose ncomp components sit in one of two device staging
// buffers (component k at k * cells + (c - c0)).  The copies of slab k run
// on the context's copy stream while the set-up / read-out kernel of slab
// k - 1 runs on its stream, so the host link and the kernels overlap; events
// keep a staging buffer from being refilled before its kernel (set-up) or
// its copy (read-out) is done.
namespace {

constexpr size_t IO_SLAB_BYTES = size_t(64) << 20;  // per staging buffer

struct SlabPlan {
  bool planes;  // slabs of z-planes (else of y-rows)
  int64_t unit_cells;
  int nunits, per;  // units in the lattice / in a full slab
};

// false: move the arrays whole (small lattices, or one plane beyond the
// staging size)
bool slab_plan(const lbm_ctx* c, int ncomp, SlabPlan* sp) {
  sp->planes = c->g.nz > 1;
  sp->unit_cells = sp->planes ? int64_t(c->g.nx) * c->g.ny : c->g.nx;
  sp->nunits = sp->planes ? c->g.nz : c->g.ny;
  const size_t unit_bytes = size_t(sp->unit_cells) * ncomp * sizeof(double);
  if (size_t(c->g.N) * ncomp * sizeof(double) < 4 * IO_SLAB_BYTES) return false;
  if (unit_bytes > IO_SLAB_BYTES) return false;
  sp->per = int(IO_SLAB_BYTES / unit_bytes);
  return true;
}

// create the copy stream and events once, grow the staging buffers
int io_ready(lbm_ctx* c, size_t doubles) {
  if (!c->io_stream) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 4 && ok; ++k)
      ok = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      for (int k = 0; k < 4; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
      if (s) cudaStreamDestroy(s);
      return LBM_ERR_CUDA;
    }
    c->io_stream = s;
    c->io_ready[0] = ev[0];
    c->io_ready[1] = ev[1];
    c->io_done[0] = ev[2];
    c->io_done[1] = ev[3];
  }
  if (c->io_cap < doubles) {
    for (int b = 0; b < 2; ++b) {
      if (c->io_buf[b]) cudaFree(c->io_buf[b]);
      c->io_buf[b] = nullptr;
    }
    c->io_cap = 0;
    for (int b = 0; b < 2; ++b) {
      if (cudaMalloc((void**)&c->io_buf[b], doubles * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < 2; ++k) {
          if (c->io_buf[k]) cudaFree(c->io_buf[k]);
          c->io_buf[k] = nullptr;
        }
        return LBM_ERR_OOM;
      }
    }
    c->io_cap = doubles;
  }
  return LBM_OK;
}

void set_slab(AuxArgs& a, const SlabPlan& sp, int u0, int nu, int64_t cells) {
  if (sp.planes) {
    a.z0 = u0;
    a.nzc = nu;
  } else {
    a.y0 = u0;
    a.nyc = nu;
  }
  a.c0 = int64_t(u0) * sp.unit_cells;
  a.stride = cells;
}

// host -> device: comps[k] is the host array of component k (N doubles) or
// NULL; df_mode: the q components are populations, else (rho, u_0..u_d-1)
int scatter_slabs(lbm_ctx* c, const SlabPlan& sp, const double* const* comps, int ncomp,
                  bool df_mode) {
  const int64_t cap = sp.unit_cells * sp.per;
  int rc = io_ready(c, size_t(cap) * ncomp);
  if (rc != LBM_OK) return rc;
  if (c->p.streaming != LBM_PULL) c->parity = 0;
  bool ok = true;
  // the copies start after the work already queued on the context's stream
  // (a staging buffer may still be read by an earlier call's kernel)
  ok = ok && cudaEventRecord(c->io_done[0], c->stream) == cudaSuccess;
  ok = ok && cudaStreamWaitEvent(c->io_stream, c->io_done[0], 0) == cudaSuccess;
  for (int k = 0, u0 = 0; ok && u0 < sp.nunits; ++k, u0 += sp.per) {
    const int nu = sp.per < sp.nunits - u0 ? sp.per : sp.nunits - u0;
    const int64_t c0 = int64_t(u0) * sp.unit_cells, cells = int64_t(nu) * sp.unit_cells;
    const int b = k & 1;
    double* sb = c->io_buf[b];
    if (k >= 2) ok = ok && cudaStreamWaitEvent(c->io_stream, c->io_done[b], 0) == cudaSuccess;
    for (int j = 0; j < ncomp && ok; ++j)
      if (comps[j])
        ok = cudaMemcpyAsync(sb + j * cells, comps[j] + c0, size_t(cells) * sizeof(double),
                             cudaMemcpyHostToDevice, c->io_stream) == cudaSuccess;
    ok = ok && cudaEventRecord(c->io_ready[b], c->io_stream) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(c->stream, c->io_ready[b], 0) == cudaSuccess;
    if (!ok) break;
    AuxArgs a = aux_base(c, lbm::AUX_SCATTER);
    a.gather_mode = scatter_layout(c);
    set_slab(a, sp, u0, nu, cells);
    if (df_mode) {
      a.df_in = sb;
    } else {
      a.rho_in = comps[0] ? sb : nullptr;
      a.u_in = sb + cells;
    }
    kAux[c->p.stencil][c->p.storage](a);
    ok = cudaGetLastError() == cudaSuccess;
    ok = ok && cudaEventRecord(c->io_done[b], c->stream) == cudaSuccess;
  }
  if (cudaStreamSynchronize(c->io_stream) != cudaSuccess) ok = false;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) ok = false;
  return ok ? LBM_OK : LBM_ERR_CUDA;
}

// device -> host: outs[k] is the host array of component k or NULL
int gather_slabs(lbm_ctx* c, const SlabPlan& sp, double* const* outs, int ncomp, bool df_mode) {
  const int64_t cap = sp.unit_cells * sp.per;
  int rc = io_ready(c, size_t(cap) * ncomp);
  if (rc != LBM_OK) return rc;
  bool ok = true;
  for (int k = 0, u0 = 0; ok && u0 < sp.nunits; ++k, u0 += sp.per) {
    const int nu = sp.per < sp.nunits - u0 ? sp.per : sp.nunits - u0;
    const int64_t c0 = int64_t(u0) * sp.unit_cells, cells = int64_t(nu) * sp.unit_cells;
    const int b = k & 1;
    double* sb = c->io_buf[b];
    if (k >= 2) ok = cudaStreamWaitEvent(c->stream, c->io_done[b], 0) == cudaSuccess;
    if (!ok) break;
    AuxArgs a = aux_base(c, lbm::AUX_GATHER);
    set_slab(a, sp, u0, nu, cells);
    if (df_mode) {
      a.df = sb;
    } else {
      a.rho = outs[0] ? sb : nullptr;
      a.u = outs[1] ? sb + cells : nullptr;
    }
    kAux[c->p.stencil][c->p.storage](a);
    ok = cudaGetLastError() == cudaSuccess;
    ok = ok && cudaEventRecord(c->io_ready[b], c->stream) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(c->io_stream, c->io_ready[b], 0) == cudaSuccess;
    for (int j = 0; j < ncomp && ok; ++j)
      if (outs[j])
        ok = cudaMemcpyAsync(outs[j] + c0, sb + j * cells, size_t(cells) * sizeof(double),
                             cudaMemcpyDeviceToHost, c->io_stream) == cudaSuccess;
    ok = ok && cudaEventRecord(c->io_done[b], c->io_stream) == cudaSuccess;
  }
  if (cudaStreamSynchronize(c->io_stream) != cudaSuccess) ok = false;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) ok = false;
  if (!ok) return LBM_ERR_CUDA;
  return read_status(c);
}

}  // namespace

int lbm_init_velocity(lbm_ctx* c, const double* rho, const double* u, int on_device) {
  if (!c || !u) return LBM_ERR_INVALID;
  NvtxRange range("lbm_init_velocity");
  const size_t N = size_t(c->g.N);
  SlabPlan sp;
  if (!on_device && c->swe_g == 0.0 && slab_plan(c, 1 + c->d, &sp)) {
    const double* comps[4] = {rho, u, u + N, c->d > 2 ? u + 2 * N : nullptr};
    c->t = 0;
    return scatter_slabs(c, sp, comps, 1 + c->d, false);
  }
  const double *drho = nullptr, *du = nullptr;
  double *trho = nullptr, *tu = nullptr;
  int rc = stage_in(c, rho, N, on_device, &drho, &trho);
  if (rc == LBM_OK) rc = stage_in(c, u, N * c->d, on_device, &du, &tu);
  if (rc == LBM_OK) {
    c->t = 0;
    rc = scatter(c, nullptr, drho, du);
  }
  if (trho || tu) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (trho) cudaFree(trho);
    if (tu) cudaFree(tu);
  }
  return rc;
}

int lbm_set_populations(lbm_ctx* c, const double* df, int on_device) {
  if (!c || !df) return LBM_ERR_INVALID;
  SlabPlan sp;
  if (!on_device && slab_plan(c, c->q, &sp)) {
    const double* comps[27];
    for (int i = 0; i < c->q; ++i) comps[i] = df + size_t(i) * size_t(c->g.N);
    return scatter_slabs(c, sp, comps, c->q, true);
  }
  const double* ddf = nullptr;
  double* tmp = nullptr;
  int rc = stage_in(c, df, size_t(c->g.N) * c->q, on_device, &ddf, &tmp);
  if (rc == LBM_OK) rc = scatter(c, ddf, nullptr, nullptr);
  if (tmp) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    cudaFree(tmp);
  }
  return rc;
}

// Can this context run the shared-memory staged pull kernel?
static bool staged_ok(const lbm_ctx* c) {
  const int64_t row = int64_t(c->g.nx) * c->eb;
  return c->p.streaming == LBM_PULL && c->p.storage != LBM_STORE_F64_ABSOLUTE &&
         c->p.arithmetic == LBM_ARITH_DEVIATION && !c->force_mode && row % 16 == 0 &&
         c->p.equilibrium != LBM_EQ_DISCRETE2 &&
         lbm::staged_stages(c->q, c->g.nx, c->eb) >= lbm::STG_MIN_STAGES;
}

// LBM_STEP_AUTO: measured on B300 (see the profiles of the staged kernel)
static bool use_staged(const lbm_ctx* c) {
  if (c->kernel == LBM_STEP_STAGED) return true;
  if (c->kernel == LBM_STEP_DIRECT || c->closure) return false;
  return false;
}

int lbm_set_divergence_check(lbm_ctx* c, int64_t every) {
  if (!c || every < 0) return LBM_ERR_INVALID;
  c->watch = every;
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* c, int64_t cycles) {
  if (!c || cycles < 0) return LBM_ERR_INVALID;
  c->wait_limit = cycles;
  return LBM_OK;
}

int lbm_set_step_kernel(lbm_ctx* c, int kernel) {
  if (!c || kernel < LBM_STEP_AUTO || kernel > LBM_STEP_STAGED) return LBM_ERR_INVALID;
  if (kernel == LBM_STEP_STAGED && !staged_ok(c)) return LBM_ERR_UNSUPPORTED;
  c->kernel = kernel;
  return LBM_OK;
}

// Nonzero status word: a staged kernel's bounded wait ran out (synchronises).
// The word is cleared once reported, so the context is usable again.
static int read_status(lbm_ctx* c) {
  int st = 0;
  if (cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (!st) return LBM_OK;
  if (cudaMemsetAsync(c->status, 0, sizeof(int), c->stream) != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_ERR_TIMEOUT;
}

// the step launch arguments of a context (every slab / the whole lattice)
static StepArgs step_args(const lbm_ctx* c) {
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = c->g;
  for (int k = 0; k < 6; ++k) a.rates[k] = c->rates[k];
  a.space = c->space;
  a.reg = c->reg;
  a.storage = c->p.storage;
  a.form = (c->p.arithmetic == LBM_ARITH_AS_WRITTEN && c->p.equilibrium == LBM_EQ_ABSOLUTE) ? 1 : 0;
  if (c->p.equilibrium == LBM_EQ_DISCRETE2) {
    a.form = 3;  // FORM_DISC
    // central moments / cumulants: the general instance (nonzero equilibria
    // of order >= 3)
    if (c->space == LBM_SPACE_CENTRAL || c->space == LBM_SPACE_CUMULANT) a.reg = 0;
  }
  a.variant = use_staged(c) ? lbm::VARIANT_STAGED : lbm::VARIANT_DIRECT;
  a.status = c->status;
  a.wait_limit = c->wait_limit;
  a.force_mode = c->force_mode;
  a.force_model = c->force_model;
  for (int d = 0; d < 3; ++d) a.force[d] = c->force[d];
  a.force_field = c->force_field;
  // forced raw-moment collisions use the general instance (the source needs
  // every orthogonal row)
  if (c->force_mode && (c->space == LBM_SPACE_RAW || c->space == LBM_SPACE_RAW_WEIGHTED))
    a.reg = 0;
  a.swe_g = c->swe_g;
  if (c->swe_g > 0.0) a.reg = 0;  // shallow water: the general instantiation
  a.stream = c->stream;
  return a;
}

int lbm_step(lbm_ctx* c, int64_t n) {
  if (!c || n < 0) return LBM_ERR_INVALID;
  NvtxRange range("lbm_step");
  StepArgs a = step_args(c);
  const step_fn fn = kStep[c->p.stencil][c->p.storage];
  for (int64_t s = 0; s < n; ++s) {
    if (c->p.streaming == LBM_PULL) {
      a.mode = lbm::MODE_PULL;
      a.src = c->buf[c->cur];
      a.dst = c->buf[1 - c->cur];
      if (c->closure)
        lbm::launch_closure_step(a, c->closure);
      else
        fn(a);
      c->cur = 1 - c->cur;
    } else {
      if (esoteric(c->p.streaming))
        a.mode = eso_mode(c->p.streaming, c->parity);
      else
        a.mode = c->parity ? lbm::MODE_AA_ODD : lbm::MODE_AA_EVEN;
      a.src = c->buf[0];
      a.dst = c->buf[0];
      fn(a);
      c->parity ^= 1;
    }
    c->t++;
    if (c->watch > 0 && c->t % c->watch == 0) {
      double inv[8];
      const int rc = lbm_invariants(c, inv);  // LBM_ERR_DIVERGED on a non-finite cell
      if (rc != LBM_OK) return rc;
    }
  }
  return cuda_err(cudaGetLastError());
}

static int gather(lbm_ctx* c, double* df, double* rho, double* u, int on_device) {
  NvtxRange range(df ? "lbm_get_populations" : "lbm_macroscopic");
  const size_t N = size_t(c->g.N);
  SlabPlan sp;
  if (!on_device && df && slab_plan(c, c->q, &sp)) {
    double* outs[27];
    for (int i = 0; i < c->q; ++i) outs[i] = df + size_t(i) * N;
    return gather_slabs(c, sp, outs, c->q, true);
  }
  if (!on_device && !df && slab_plan(c, 1 + c->d, &sp)) {
    double* outs[4] = {rho, u, u ? u + N : nullptr, (u && c->d > 2) ? u + 2 * N : nullptr};
    return gather_slabs(c, sp, outs, 1 + c->d, false);
  }
  double *tdf = nullptr, *trho = nullptr, *tu = nullptr;
  int rc = LBM_OK;
  if (!on_device) {
    if (df && cudaMalloc((void**)&tdf, N * c->q * sizeof(double)) != cudaSuccess) rc = LBM_ERR_OOM;
    if (rho && cudaMalloc((void**)&trho, N * sizeof(double)) != cudaSuccess) rc = LBM_ERR_OOM;
    if (u && cudaMalloc((void**)&tu, N * c->d * sizeof(double)) != cudaSuccess) rc = LBM_ERR_OOM;
    if (rc != LBM_OK) cudaGetLastError();
  }
  if (rc == LBM_OK) {
    AuxArgs a = aux_base(c, lbm::AUX_GATHER);
    a.df = on_device ? df : tdf;
    a.rho = on_device ? rho : trho;
    a.u = on_device ? u : tu;
    kAux[c->p.stencil][c->p.storage](a);
    rc = cuda_err(cudaGetLastError());
  }
  if (rc == LBM_OK && !on_device) {
    if (df)
      rc = cuda_err(cudaMemcpyAsync(df, tdf, N * c->q * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
    if (rho && rc == LBM_OK)
      rc = cuda_err(
          cudaMemcpyAsync(rho, trho, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u && rc == LBM_OK)
      rc = cuda_err(
          cudaMemcpyAsync(u, tu, N * c->d * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  }
  if (rc == LBM_OK && !on_device) rc = read_status(c);
  if (tdf) cudaFree(tdf);
  if (trho) cudaFree(trho);
  if (tu) cudaFree(tu);
  return rc;
}

int lbm_macroscopic(lbm_ctx* c, double* rho, double* u, int on_device) {
  if (!c) return LBM_ERR_INVALID;
  if (!rho && !u) return LBM_OK;
  return gather(c, nullptr, rho, u, on_device);
}

int lbm_get_populations(lbm_ctx* c, double* df, int on_device) {
  if (!c || !df) return LBM_ERR_INVALID;
  return gather(c, df, nullptr, nullptr, on_device);
}

// ------------------------------------------- pipelined host job (run_host)
// Set-up from host fields, n pull steps and read-out to host as one job:
// the lattice is cut into S slabs of z-planes, and the copies in, the steps
// and the copies out of different slabs overlap as a wavefront.  Slab s may
// take step k + 1 once its neighbours s - 1 and s + 1 (periodic) have
// taken step k: step k + 1 reads their post-collision values of step k and
// overwrites the buffer their step k read.  Step 1 needs only the slab's
// own set-up (the pull layout stores a cell's initial populations where
// that cell's first gather reads them).  A slab is read out once it and
// both neighbours have taken all n steps.  The order is fixed on the host
// in advance (greedy: after each arriving slab, every step that has become
// possible); the context's stream runs it in order, and events tie it to
// one copy stream per direction with a ring of staging buffers each.
namespace {

constexpr int RUN_RING = 4;  // staging slots per direction when memory is short

bool run_pipelined_ok(const lbm_ctx* c) {
  return c->p.streaming == LBM_PULL && c->p.storage != LBM_STORE_F64_ABSOLUTE &&
         c->p.arithmetic == LBM_ARITH_DEVIATION && !c->force_mode && !c->closure &&
         c->swe_g == 0.0 && !use_staged(c) && c->g.nz >= 3;
}

}  // namespace

int lbm_run_host(lbm_ctx* c, const double* rho, const double* u, int64_t n, double* rho_out,
                 double* u_out, int slabs) {
  if (!c || !u || n < 0 || slabs < 0) return LBM_ERR_INVALID;
  NvtxRange range("lbm_run_host");
  const size_t N = size_t(c->g.N);
  const int nz = c->g.nz, d = c->d;
  const int64_t plane = int64_t(c->g.nx) * c->g.ny;
  // slab count: about 64 MB of (rho, u) per slab, at least 3
  int S = slabs;
  if (S == 0) {
    const size_t per = size_t(plane) * (1 + d) * sizeof(double);
    S = int((size_t(nz) * per + IO_SLAB_BYTES - 1) / IO_SLAB_BYTES);
  }
  if (S > nz) S = nz;
  if (!run_pipelined_ok(c) || S < 3 || c->watch > 0) {  // one job after the other
    int rc = lbm_init_velocity(c, rho, u, 0);
    if (rc == LBM_OK) rc = lbm_step(c, n);
    if (rc == LBM_OK && (rho_out || u_out)) rc = lbm_macroscopic(c, rho_out, u_out, 0);
    return rc;
  }
  std::vector<int> z0(S + 1);
  for (int k = 0; k <= S; ++k) z0[k] = int(int64_t(nz) * k / S);
  int maxp = 0;
  for (int k = 0; k < S; ++k) maxp = std::max(maxp, z0[k + 1] - z0[k]);
  const int64_t cap = int64_t(maxp) * plane;  // cells of the largest slab
  const int ncomp = 1 + d;
  // one staging slot per slab and direction when the device has room (no
  // copy or step ever waits for a slot), else a ring of RUN_RING slots
  size_t free_b = 0, total_b = 0;
  const size_t slot_b = size_t(cap) * ncomp * sizeof(double);
  int R = RUN_RING;
  if (c->run_cap >= 2 * size_t(S) * slot_b ||
      (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
       2 * size_t(S) * slot_b + c->run_cap + (size_t(1) << 30) < free_b))
    R = S;
  cudaGetLastError();
  std::vector<double*> ring_in(R, nullptr), ring_out(R, nullptr);
  // the slots live in one block kept by the context between calls
  const size_t need = 2 * size_t(R) * slot_b;
  if (c->run_cap < need) {
    if (c->run_buf) cudaFree(c->run_buf);
    c->run_buf = nullptr;
    c->run_cap = 0;
    if (cudaMalloc((void**)&c->run_buf, need) != cudaSuccess) {
      cudaGetLastError();
      c->run_buf = nullptr;
      return LBM_ERR_OOM;
    }
    c->run_cap = need;
  }
  for (int r = 0; r < R; ++r) {
    ring_in[r] = c->run_buf + size_t(r) * (slot_b / sizeof(double));
    ring_out[r] = c->run_buf + size_t(R + r) * (slot_b / sizeof(double));
  }
  cudaStream_t s_in = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> ev;
  auto new_event = [&]() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return (cudaEvent_t) nullptr;
    ev.push_back(e);
    return e;
  };
  int rc = LBM_OK;
  bool ok = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking) == cudaSuccess;
  std::vector<cudaEvent_t> arrived(S), in_free(R), out_ready(S), out_free(R);
  for (int k = 0; k < S && ok; ++k) ok = (arrived[k] = new_event()) && (out_ready[k] = new_event());
  for (int r = 0; r < R && ok; ++r) ok = (in_free[r] = new_event()) && (out_free[r] = new_event());
  cudaEvent_t start = ok ? new_event() : nullptr;
  ok = ok && start;
  if (!ok) {
    cudaGetLastError();
    rc = LBM_ERR_OOM;
  }
  std::vector<int64_t> step(S, -1);   // steps taken by slab (-1: not set up)
  std::vector<char> emitted(S, 0);    // read-out issued
  const int cur0 = c->cur;
  StepArgs sa = step_args(c);
  sa.mode = lbm::MODE_PULL;
  const step_fn fn = kStep[c->p.stencil][c->p.storage];
  int out_count = 0;
  auto slab_cells = [&](int k) { return int64_t(z0[k + 1] - z0[k]) * plane; };
  auto set_slab_aux = [&](AuxArgs& a, int k) {
    a.z0 = z0[k];
    a.nzc = z0[k + 1] - z0[k];
    a.c0 = int64_t(z0[k]) * plane;
    a.stride = slab_cells(k);
  };
  // read-out of slab k into slot out_count % R, then its copy
  auto emit = [&](int k) {
    const int r = out_count % R;
    const int64_t cells = slab_cells(k), c0 = int64_t(z0[k]) * plane;
    if (out_count >= R) ok = ok && cudaStreamWaitEvent(c->stream, out_free[r], 0) == cudaSuccess;
    AuxArgs a = aux_base(c, lbm::AUX_GATHER);
    a.buf = c->buf[(cur0 + n) % 2];
    a.gather_mode = G_PULL;
    set_slab_aux(a, k);
    a.rho = rho_out ? ring_out[r] : nullptr;
    a.u = u_out ? ring_out[r] + cells : nullptr;
    if (ok && (rho_out || u_out)) {
      kAux[c->p.stencil][c->p.storage](a);
      ok = cudaGetLastError() == cudaSuccess;
    }
    ok = ok && cudaEventRecord(out_ready[k], c->stream) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(s_out, out_ready[k], 0) == cudaSuccess;
    if (rho_out)
      ok = ok && cudaMemcpyAsync(rho_out + c0, ring_out[r], size_t(cells) * sizeof(double),
                                 cudaMemcpyDeviceToHost, s_out) == cudaSuccess;
    if (u_out)
      for (int j = 0; j < d; ++j)
        ok = ok && cudaMemcpyAsync(u_out + size_t(j) * N + c0, ring_out[r] + (1 + j) * cells,
                                   size_t(cells) * sizeof(double), cudaMemcpyDeviceToHost,
                                   s_out) == cudaSuccess;
    ok = ok && cudaEventRecord(out_free[r], s_out) == cudaSuccess;
    emitted[k] = 1;
    ++out_count;
  };
  // every step (and read-out) that has become possible, until none: the
  // slabs able to advance are found first, then each run of adjacent ones
  // at the same step goes as one launch over their z-planes (a neighbour
  // advancing in between only adds to what they may do)
  std::vector<char> elig(S, 0);
  auto advance = [&]() {
    bool any = true;
    while (any && ok) {
      any = false;
      for (int k = 0; k < S; ++k) {
        const int km = (k + S - 1) % S, kp = (k + 1) % S;
        const int64_t t = step[k];
        elig[k] = t >= 0 && t < n && (t == 0 || (step[km] >= t && step[kp] >= t));
      }
      for (int k = 0; k < S && ok;) {
        if (!elig[k]) {
          ++k;
          continue;
        }
        int e = k;
        while (e + 1 < S && elig[e + 1] && step[e + 1] == step[k]) ++e;
        const int64_t t = step[k];
        sa.src = c->buf[(cur0 + t) % 2];
        sa.dst = c->buf[(cur0 + t + 1) % 2];
        sa.z0 = z0[k];
        sa.nzc = z0[e + 1] - z0[k];
        fn(sa);
        ok = cudaGetLastError() == cudaSuccess;
        for (int j = k; j <= e; ++j) step[j] = t + 1;
        any = true;
        k = e + 1;
      }
      for (int k = 0; k < S && ok; ++k) {
        const int km = (k + S - 1) % S, kp = (k + 1) % S;
        if (!emitted[k] && step[k] == n && step[km] == n && step[kp] == n) {
          emit(k);
          any = true;
        }
      }
    }
  };
  // copy of slab k into slot k % R; a slot is refilled only after the
  // set-up of the slab before in it, whose event is recorded first (a wait
  // on an event not yet recorded would not wait)
  auto copy_in = [&](int k) {
    const int r = k % R;
    const int64_t cells = slab_cells(k), c0 = int64_t(z0[k]) * plane;
    if (k >= R) ok = ok && cudaStreamWaitEvent(s_in, in_free[r], 0) == cudaSuccess;
    if (rho)
      ok = ok && cudaMemcpyAsync(ring_in[r], rho + c0, size_t(cells) * sizeof(double),
                                 cudaMemcpyHostToDevice, s_in) == cudaSuccess;
    for (int j = 0; j < d; ++j)
      ok = ok && cudaMemcpyAsync(ring_in[r] + (1 + j) * cells, u + size_t(j) * N + c0,
                                 size_t(cells) * sizeof(double), cudaMemcpyHostToDevice,
                                 s_in) == cudaSuccess;
    ok = ok && cudaEventRecord(arrived[k], s_in) == cudaSuccess;
  };
  if (ok) {
    // the copies start after the work already queued on the context's stream
    ok = cudaEventRecord(start, c->stream) == cudaSuccess &&
         cudaStreamWaitEvent(s_in, start, 0) == cudaSuccess &&
         cudaStreamWaitEvent(s_out, start, 0) == cudaSuccess;
    for (int k = 0; k < S && k < R; ++k) copy_in(k);
    // the compute order: set up each arriving slab, then every step it enables
    for (int k = 0; k < S && ok; ++k) {
      const int r = k % R;
      ok = cudaStreamWaitEvent(c->stream, arrived[k], 0) == cudaSuccess;
      AuxArgs a = aux_base(c, lbm::AUX_SCATTER);
      a.buf = c->buf[cur0];
      a.gather_mode = G_PULL;
      set_slab_aux(a, k);
      a.rho_in = rho ? ring_in[r] : nullptr;
      a.u_in = ring_in[r] + slab_cells(k);
      if (ok) {
        kAux[c->p.stencil][c->p.storage](a);
        ok = cudaGetLastError() == cudaSuccess;
      }
      ok = ok && cudaEventRecord(in_free[r], c->stream) == cudaSuccess;
      if (k + R < S) copy_in(k + R);
      step[k] = 0;
      advance();
    }
    advance();
    for (int k = 0; k < S && ok; ++k)
      if (!emitted[k]) ok = false;  // the schedule always completes
  }
  if (s_in && cudaStreamSynchronize(s_in) != cudaSuccess) ok = false;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) ok = false;
  if (s_out && cudaStreamSynchronize(s_out) != cudaSuccess) ok = false;
  if (rc == LBM_OK && !ok) rc = LBM_ERR_CUDA;
  if (rc == LBM_OK) {
    c->t = n;
    c->cur = int((cur0 + n) % 2);
    rc = read_status(c);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (s_in) cudaStreamDestroy(s_in);
  if (s_out) cudaStreamDestroy(s_out);
  return rc;
}

int lbm_invariants(lbm_ctx* c, double out[8]) {
  if (!c || !out) return LBM_ERR_INVALID;
  AuxArgs a = aux_base(c, lbm::AUX_INVARIANTS);
  a.part = c->part;
  a.nparts = c->nparts;
  kAux[c->p.stencil][c->p.storage](a);
  lbm::launch_invariants_fold(c->part, c->nparts, c->part + size_t(c->nparts) * 8, c->stream);
  int rc = cuda_err(cudaGetLastError());
  if (rc == LBM_OK)
    rc = cuda_err(cudaMemcpyAsync(out, c->part + size_t(c->nparts) * 8, 8 * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  if (rc == LBM_OK) rc = read_status(c);
  if (rc == LBM_OK && out[6] > 0) rc = LBM_ERR_DIVERGED;
  return rc;
}

int64_t lbm_state_bytes(const lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID;
  return int64_t(sizeof(StateHeader)) + int64_t(c->q) * c->g.N * c->eb;
}

int lbm_get_state(lbm_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf || int64_t(bytes) < lbm_state_bytes(c)) return LBM_ERR_INVALID;
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.stencil = c->p.stencil;
  h.space = c->p.space;
  h.equilibrium = c->p.equilibrium;
  h.storage = c->p.storage;
  h.streaming = c->p.streaming;
  h.parity = c->parity;
  for (int k = 0; k < 3; ++k) h.dims[k] = c->p.dims[k];
  h.t = c->t;
  h.payload = int64_t(c->q) * c->g.N * c->eb;
  std::memcpy(buf, &h, sizeof(h));
  int rc = cuda_err(cudaMemcpyAsync((char*)buf + sizeof(h), state_buf(c), size_t(h.payload),
                                    cudaMemcpyDeviceToHost, c->stream));
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  if (rc == LBM_OK) rc = read_status(c);
  return rc;
}

int lbm_set_state(lbm_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf || bytes < sizeof(StateHeader)) return LBM_ERR_INVALID;
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.stencil != c->p.stencil || h.storage != c->p.storage ||
      h.streaming != c->p.streaming || h.dims[0] != c->p.dims[0] || h.dims[1] != c->p.dims[1] ||
      h.dims[2] != c->p.dims[2] || h.payload != int64_t(c->q) * c->g.N * c->eb ||
      int64_t(bytes) < lbm_state_bytes(c) || (h.parity != 0 && h.parity != 1))
    return LBM_ERR_STATE_MISMATCH;
  c->parity = h.parity;
  c->t = h.t;
  int rc = cuda_err(cudaMemcpyAsync(state_buf(c), (const char*)buf + sizeof(h), size_t(h.payload),
                                    cudaMemcpyHostToDevice, c->stream));
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  return rc;
}

}  // extern "C"
