// lbm_batch.cu -- C ABI of the batched ensemble (include/lbm_batch.h):
// instance table, tile list, persistent launches captured in CUDA graphs,
// and the launch-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_batch.h"
#include "lbm_internal.h"

using lbm::AuxArgs;
using lbm::BatchArgs;
using lbm::BInst;
using lbm::StepArgs;

struct lbm_batch {
  lbm_params p;
  int n, q, d, eb;
  int space, reg;
  double rates[6];
  std::vector<BInst> inst;
  std::vector<double> shear;
  BInst* dinst;
  int2* dtiles;
  int ntiles;
  int sms;
  lbm_batch_tuning tune;
  void* buf[2];
  int cur;
  int64_t t;
  int64_t cells;
  cudaStream_t stream;   // user stream (work and graph launches)
  cudaStream_t capture;  // private stream the graphs are captured on
  cudaGraphExec_t graph[2];  // two steps starting from buffer 0 / buffer 1
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }
int q_of(int st) { return st == LBM_D2Q9 ? 9 : (st == LBM_D3Q19 ? 19 : 27); }
int elem_bytes(int storage) {
  return storage == LBM_STORE_F64 ? 8 : (storage == LBM_STORE_F32 ? 4 : 2);
}  // absolute storage is rejected at create

void drop_graphs(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
}

int build_tiles(lbm_batch* b) {
  const int tile = b->tune.threads * b->tune.cells_per_thread;
  std::vector<int2> tiles;
  for (int k = 0; k < b->n; ++k)
    for (int s = 0; s < b->inst[k].N; s += tile) tiles.push_back(make_int2(k, s));
  if (b->dtiles) cudaFree(b->dtiles);
  b->dtiles = nullptr;
  b->ntiles = int(tiles.size());
  if (cudaMalloc((void**)&b->dtiles, sizeof(int2) * tiles.size()) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  drop_graphs(b);
  return cuda_err(cudaMemcpy(b->dtiles, tiles.data(), sizeof(int2) * tiles.size(),
                             cudaMemcpyHostToDevice));
}

BatchArgs batch_args(const lbm_batch* b, int op, cudaStream_t s) {
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.op = op;
  a.inst = b->dinst;
  a.tiles = b->dtiles;
  a.ntiles = b->ntiles;
  a.cpt = b->tune.cells_per_thread;
  a.threads = b->tune.threads;
  a.grid = b->tune.blocks_per_sm * b->sms;
  for (int k = 0; k < 6; ++k) a.rates[k] = b->rates[k];
  a.space = b->space;
  a.reg = b->reg;
  a.storage = b->p.storage;
  a.stream = s;
  return a;
}

// one step of every instance from buffer `from` on stream s
void enqueue_step(const lbm_batch* b, int from, cudaStream_t s) {
  const char* src = (const char*)b->buf[from];
  char* dst = (char*)b->buf[1 - from];
  if (!b->tune.per_instance) {
    BatchArgs a = batch_args(b, lbm::BATCH_STEP, s);
    a.src = src;
    a.dst = dst;
    lbm::dispatch_batch(b->p.stencil, b->p.storage, a);
    return;
  }
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int k = 0; k < 6; ++k) a.rates[k] = b->rates[k];
  a.space = b->space;
  a.reg = b->reg;
  a.storage = b->p.storage;
  a.mode = lbm::MODE_PULL;
  a.stream = s;
  for (int k = 0; k < b->n; ++k) {
    const BInst& I = b->inst[k];
    a.g.nx = I.nx;
    a.g.ny = I.ny;
    a.g.nz = I.nz;
    a.g.N = I.N;
    a.rates[0] = b->shear[k];
    a.src = src + I.off * b->eb;
    a.dst = dst + I.off * b->eb;
    lbm::dispatch_step(b->p.stencil, b->p.storage, a);
  }
}

int capture(lbm_batch* b, int from) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return LBM_ERR_CUDA;
  enqueue_step(b, from, b->capture);
  enqueue_step(b, 1 - from, b->capture);
  cudaError_t e = cudaStreamEndCapture(b->capture, &g);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  e = cudaGraphInstantiate(&b->graph[from], g, 0);
  cudaGraphDestroy(g);
  return cuda_err(e);
}

AuxArgs aux_of(const lbm_batch* b, int k, int op) {
  AuxArgs a;
  std::memset(&a, 0, sizeof(a));
  const BInst& I = b->inst[k];
  a.op = op;
  a.buf = (char*)b->buf[b->cur] + I.off * b->eb;
  a.g.nx = I.nx;
  a.g.ny = I.ny;
  a.g.nz = I.nz;
  a.g.N = I.N;
  a.storage = b->p.storage;
  a.space = b->space;
  a.gather_mode = 0;  // pull
  a.stream = b->stream;
  lbm::whole_slab(a);
  return a;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch** out, const lbm_params* p, int n, const int64_t* dims,
                     const double* shear_rates) {
  if (!out || !p || n < 1 || !dims) return LBM_ERR_INVALID;
  *out = nullptr;
  if (p->stencil < 0 || p->stencil > 2 || p->space < 0 || p->space > 5 || p->storage < 0 ||
      p->storage > 4 || (p->equilibrium != LBM_EQ_DELTA && p->equilibrium != LBM_EQ_ABSOLUTE &&
                         p->equilibrium != LBM_EQ_DISCRETE2))
    return LBM_ERR_INVALID;
  if (p->equilibrium == LBM_EQ_DISCRETE2) return LBM_ERR_UNSUPPORTED;
  if (p->space == LBM_SPACE_CUMULANT && p->equilibrium == LBM_EQ_DELTA)
    return LBM_ERR_INADMISSIBLE;
  if (p->boundary != LBM_PERIODIC || p->streaming != LBM_PULL ||
      p->storage == LBM_STORE_F64_ABSOLUTE || p->arithmetic != LBM_ARITH_DEVIATION)
    return LBM_ERR_UNSUPPORTED;
  for (int k = 0; k < 6; ++k)
    if (!(p->rates[k] > 0.0 && p->rates[k] <= 2.0)) return LBM_ERR_INVALID;
  if (p->space == LBM_SPACE_POPULATIONS && shear_rates) return LBM_ERR_INVALID;
  // every instance's box and shear rate, before any device work
  for (int k = 0; k < n; ++k) {
    const int64_t nx = dims[3 * k], ny = dims[3 * k + 1], nz = dims[3 * k + 2];
    const double om = shear_rates ? shear_rates[k] : p->rates[0];
    if (nx < 1 || ny < 1 || nz < 1 || nx >= (int64_t(1) << 31) || ny > 65535 || nz > 65535 ||
        !lbm::index_fits(nx, ny, nz, p->stencil == LBM_D2Q9 ? 2 : 3) ||
        (p->stencil == LBM_D2Q9 && nz != 1) ||
        !(om > 0.0 && om <= 2.0))
      return LBM_ERR_INVALID;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->p = *p;
  b->n = n;
  b->q = q_of(p->stencil);
  b->d = p->stencil == LBM_D2Q9 ? 2 : 3;
  b->eb = elem_bytes(p->storage);
  b->stream = (cudaStream_t)p->stream;
  b->space = p->space;
  for (int k = 0; k < 6; ++k) b->rates[k] = p->space == LBM_SPACE_POPULATIONS ? p->rates[0] : p->rates[k];
  b->reg = p->space != LBM_SPACE_POPULATIONS && p->space != LBM_SPACE_TRT;
  for (int k = 1; k < 6; ++k)
    if (b->rates[k] != 1.0) b->reg = 0;
  int64_t off = 0;
  b->inst.resize(n);
  b->shear.resize(n);
  for (int k = 0; k < n; ++k) {
    const int64_t nx = dims[3 * k], ny = dims[3 * k + 1], nz = dims[3 * k + 2];
    const double om = shear_rates ? shear_rates[k] : p->rates[0];
    BInst& I = b->inst[k];
    I.nx = int(nx);
    I.ny = int(ny);
    I.nz = int(nz);
    I.N = int(nx * ny * nz);
    I.off = off;
    I.keep_shear = 1.0 - om;
    I.rnx = 1.0f / float(nx);
    I.rny = 1.0f / float(ny);
    b->shear[k] = om;
    off += int64_t(b->q) * I.N;
    b->cells += I.N;
  }
  b->tune.threads = 128;
  b->tune.cells_per_thread = 4;
  b->tune.blocks_per_sm = 8;
  b->tune.per_instance = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t bytes = size_t(off) * size_t(b->eb);
  int rc = LBM_OK;
  for (int k = 0; k < 2 && rc == LBM_OK; ++k) {
    if (cudaMalloc(&b->buf[k], bytes) != cudaSuccess) {
      cudaGetLastError();
      b->buf[k] = nullptr;
      rc = LBM_ERR_OOM;
    } else if (cudaMemsetAsync(b->buf[k], 0, bytes, b->stream) != cudaSuccess) {
      rc = LBM_ERR_CUDA;
    }
  }
  if (rc == LBM_OK && cudaMalloc((void**)&b->dinst, sizeof(BInst) * n) != cudaSuccess) {
    cudaGetLastError();
    b->dinst = nullptr;
    rc = LBM_ERR_OOM;
  }
  if (rc == LBM_OK)
    rc = cuda_err(cudaMemcpy(b->dinst, b->inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice));
  if (rc == LBM_OK) rc = cuda_err(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  if (rc == LBM_OK) rc = build_tiles(b);
  if (rc != LBM_OK) {
    lbm_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  drop_graphs(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int k = 0; k < 2; ++k)
    if (b->buf[k]) cudaFree(b->buf[k]);
  if (b->dinst) cudaFree(b->dinst);
  if (b->dtiles) cudaFree(b->dtiles);
  delete b;
}

int64_t lbm_batch_cells(const lbm_batch* b) { return b ? b->cells : LBM_ERR_INVALID; }
int lbm_batch_size(const lbm_batch* b) { return b ? b->n : LBM_ERR_INVALID; }

int lbm_batch_get_time(const lbm_batch* b, int64_t* step) {
  if (!b || !step) return LBM_ERR_INVALID;
  *step = b->t;
  return LBM_OK;
}

int lbm_batch_set_tuning(lbm_batch* b, const lbm_batch_tuning* t) {
  if (!b || !t || t->threads < 32 || t->threads > 256 || t->threads % 32 ||
      t->cells_per_thread < 1 || t->cells_per_thread > 16 || t->blocks_per_sm < 1 ||
      t->blocks_per_sm > 32 || (t->per_instance != 0 && t->per_instance != 1))
    return LBM_ERR_INVALID;
  const bool shape = t->threads != b->tune.threads || t->cells_per_thread != b->tune.cells_per_thread;
  const bool any = shape || t->blocks_per_sm != b->tune.blocks_per_sm ||
                   t->per_instance != b->tune.per_instance;
  b->tune = *t;
  if (shape) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    return build_tiles(b);
  }
  if (any) drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_get_tuning(const lbm_batch* b, lbm_batch_tuning* t) {
  if (!b || !t) return LBM_ERR_INVALID;
  *t = b->tune;
  return LBM_OK;
}

int lbm_batch_init_velocity(lbm_batch* b, int k, const double* rho, const double* u,
                            int on_device) {
  if (!b || !u || k < 0 || k >= b->n) return LBM_ERR_INVALID;
  const size_t N = size_t(b->inst[k].N);
  double *trho = nullptr, *tu = nullptr;
  const double *drho = rho, *du = u;
  int rc = LBM_OK;
  if (!on_device) {
    if (rho && cudaMalloc((void**)&trho, N * sizeof(double)) != cudaSuccess) rc = LBM_ERR_OOM;
    if (rc == LBM_OK && cudaMalloc((void**)&tu, N * b->d * sizeof(double)) != cudaSuccess)
      rc = LBM_ERR_OOM;
    if (rc != LBM_OK) cudaGetLastError();
    if (rc == LBM_OK && rho)
      rc = cuda_err(cudaMemcpyAsync(trho, rho, N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    if (rc == LBM_OK)
      rc = cuda_err(cudaMemcpyAsync(tu, u, N * b->d * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    drho = rho ? trho : nullptr;
    du = tu;
  }
  if (rc == LBM_OK) {
    AuxArgs a = aux_of(b, k, lbm::AUX_SCATTER);
    a.rho_in = drho;
    a.u_in = du;
    lbm::dispatch_aux(b->p.stencil, b->p.storage, a);
    rc = cuda_err(cudaGetLastError());
    b->t = 0;
  }
  if (!on_device) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (trho) cudaFree(trho);
    if (tu) cudaFree(tu);
  }
  return rc;
}

int lbm_batch_init_tgv(lbm_batch* b, const double* u0) {
  if (!b || !u0) return LBM_ERR_INVALID;
  double* du0 = nullptr;
  if (cudaMalloc((void**)&du0, sizeof(double) * b->n) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  int rc = cuda_err(cudaMemcpyAsync(du0, u0, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream));
  if (rc == LBM_OK) {
    BatchArgs a = batch_args(b, lbm::BATCH_TGV, b->stream);
    a.dst = b->buf[b->cur];
    a.u0 = du0;
    lbm::dispatch_batch(b->p.stencil, b->p.storage, a);
    rc = cuda_err(cudaGetLastError());
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
  cudaFree(du0);
  b->t = 0;
  return rc;
}

int lbm_batch_step(lbm_batch* b, int64_t n) {
  if (!b || n < 0) return LBM_ERR_INVALID;
  while (n >= 2) {
    if (!b->graph[b->cur]) {
      int rc = capture(b, b->cur);
      if (rc != LBM_OK) return rc;
    }
    if (cudaGraphLaunch(b->graph[b->cur], b->stream) != cudaSuccess) return LBM_ERR_CUDA;
    n -= 2;
    b->t += 2;
  }
  if (n == 1) {
    enqueue_step(b, b->cur, b->stream);
    b->cur = 1 - b->cur;
    b->t += 1;
  }
  return cuda_err(cudaGetLastError());
}

int lbm_batch_get_populations(lbm_batch* b, int k, double* df, int on_device) {
  if (!b || !df || k < 0 || k >= b->n) return LBM_ERR_INVALID;
  const size_t n = size_t(b->inst[k].N) * b->q;
  double* t = nullptr;
  if (!on_device && cudaMalloc((void**)&t, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_OOM;
  }
  AuxArgs a = aux_of(b, k, lbm::AUX_GATHER);
  a.df = on_device ? df : t;
  lbm::dispatch_aux(b->p.stencil, b->p.storage, a);
  int rc = cuda_err(cudaGetLastError());
  if (!on_device) {
    if (rc == LBM_OK)
      rc = cuda_err(cudaMemcpyAsync(df, t, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    cudaFree(t);
  }
  return rc;
}

int lbm_batch_macroscopic(lbm_batch* b, int k, double* rho, double* u, int on_device) {
  if (!b || k < 0 || k >= b->n) return LBM_ERR_INVALID;
  if (!rho && !u) return LBM_OK;
  const size_t N = size_t(b->inst[k].N);
  double *tr = nullptr, *tu = nullptr;
  int rc = LBM_OK;
  if (!on_device) {
    if (rho && cudaMalloc((void**)&tr, N * sizeof(double)) != cudaSuccess) rc = LBM_ERR_OOM;
    if (u && rc == LBM_OK && cudaMalloc((void**)&tu, N * b->d * sizeof(double)) != cudaSuccess)
      rc = LBM_ERR_OOM;
    if (rc != LBM_OK) cudaGetLastError();
  }
  if (rc == LBM_OK) {
    AuxArgs a = aux_of(b, k, lbm::AUX_GATHER);
    a.rho = on_device ? rho : tr;
    a.u = on_device ? u : tu;
    lbm::dispatch_aux(b->p.stencil, b->p.storage, a);
    rc = cuda_err(cudaGetLastError());
  }
  if (!on_device) {
    if (rc == LBM_OK && rho)
      rc = cuda_err(cudaMemcpyAsync(rho, tr, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (rc == LBM_OK && u)
      rc = cuda_err(cudaMemcpyAsync(u, tu, N * b->d * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (tr) cudaFree(tr);
    if (tu) cudaFree(tu);
  }
  return rc;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_tuning* best, double* best_mlups) {
  if (!b || trial_steps < 1) return LBM_ERR_INVALID;
  static const int kThreads[] = {64, 128, 256};
  static const int kCpt[] = {1, 2, 4, 8};
  static const int kBps[] = {4, 6, 8, 10, 12, 16};
  constexpr int kFinalists = 4, kRepeats = 3;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LBM_ERR_CUDA;
  const int steps = 2 * ((trial_steps + 1) / 2);  // whole graph replays
  std::vector<std::pair<double, lbm_batch_tuning>> rated;
  lbm_batch_tuning win = b->tune;
  double win_rate = -1.0;
  int rc = LBM_OK;
  // one timed trial of `steps` steps of shape t (after a capturing warm-up)
  auto trial = [&](const lbm_batch_tuning& t, double& rate) -> int {
    int r;
    if ((r = lbm_batch_set_tuning(b, &t)) != LBM_OK) return r;
    if ((r = lbm_batch_step(b, 2)) != LBM_OK) return r;  // capture + warm
    cudaEventRecord(e0, b->stream);
    if ((r = lbm_batch_step(b, steps)) != LBM_OK) return r;
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return LBM_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    rate = double(b->cells) * steps / (ms * 1e-3) / 1e6;
    return LBM_OK;
  };
  // screen every shape once, then time the fastest few kRepeats times more
  // and keep the best median: a single short trial ranks shapes within a
  // few per cent of each other by noise
  for (int th : kThreads)
    for (int cpt : kCpt)
      for (int bps : kBps) {
        lbm_batch_tuning t = {th, cpt, bps, 0};
        double rate = 0.0;
        if ((rc = trial(t, rate)) != LBM_OK) goto done;
        rated.push_back({rate, t});
      }
  std::sort(rated.begin(), rated.end(),
            [](const std::pair<double, lbm_batch_tuning>& x,
               const std::pair<double, lbm_batch_tuning>& y) { return x.first > y.first; });
  for (int f = 0; f < kFinalists && f < int(rated.size()); ++f) {
    double r[kRepeats];
    for (int k = 0; k < kRepeats; ++k)
      if ((rc = trial(rated[f].second, r[k])) != LBM_OK) goto done;
    std::sort(r, r + kRepeats);
    if (r[kRepeats / 2] > win_rate) {
      win_rate = r[kRepeats / 2];
      win = rated[f].second;
    }
  }
  rc = lbm_batch_set_tuning(b, &win);
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == LBM_OK) {
    if (best) *best = win;
    if (best_mlups) *best_mlups = win_rate;
  }
  return rc;
}

}  // extern "C"
