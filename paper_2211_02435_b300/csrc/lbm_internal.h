// lbm_internal.h -- host-side launch interface between the C ABI
// (lbm_api.cu) and the per-(stencil, storage) kernel instantiations
// (lbm_inst.cu, compiled once per combination).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

struct Geo {
  int nx, ny, nz;
  int64_t N;  // nx * ny * nz (< 2^31, see index_fits)
};

// The step kernels index cells with 32-bit integers: a gather forms c + w
// with c < N and a periodic wrap correction w.  On a 3-D stencil the z wrap
// (+N) applies in plane 0, c < Nx*Ny, and the y wrap (+Nx*Ny) in row 0 of a
// plane, so c + w stays below N + Nx*Ny + 2*Nx; a 2-D stencil has no z wrap
// and stays below N + 2*Nx.  The packed FP16 / BF16 accesses reach a few
// elements further and the tiles of the persistent and batched kernels run
// up to 2048 cells past N.  A lattice is accepted when all of these stay
// below 2^31.  The caller has already checked 1 <= Nx < 2^31 and Ny, Nz <=
// 65535, so no product wraps.
inline bool index_fits(int64_t nx, int64_t ny, int64_t nz, int dim) {
  return nx * ny * nz + (dim == 3 ? nx * ny : 0) + 2 * nx + 4096 < (int64_t(1) << 31);
}

enum { STORE_F64 = 0, STORE_F32 = 1, STORE_F16 = 2, STORE_BF16 = 3, STORE_F64_ABS = 4 };
enum {
  MODE_PULL = 0, MODE_AA_EVEN = 1, MODE_AA_ODD = 2, MODE_ET_EVEN = 3, MODE_ET_ODD = 4,
  MODE_EPULL_EVEN = 5, MODE_EPULL_ODD = 6, MODE_EPUSH_EVEN = 7, MODE_EPUSH_ODD = 8
};
enum { VARIANT_DIRECT = 0, VARIANT_STAGED = 1 };
enum { FORCE_NONE = 0, FORCE_UNIFORM = 1, FORCE_FIELD = 2, FORCE_UNIFORM_HE = 3, FORCE_FIELD_HE = 4 };

// shared-memory staged pull kernel (lbm_staged.cuh); the stage cap is a
// compile-time tuning knob
#ifndef LBM_STG_MAX_STAGES
#define LBM_STG_MAX_STAGES 2  // measured on B300: more stages cost CTAs per SM
#endif
constexpr int STG_MIN_STAGES = 2, STG_MAX_STAGES = LBM_STG_MAX_STAGES;  // rows in flight per CTA
constexpr int STG_MAX_SMEM = 110 * 1024;               // stage bytes per CTA: two CTAs per SM
// as many stages as fit the budget (0 when not even two fit)
inline int staged_stages(int q, int nx, int elem) {
  const int64_t row = int64_t(q) * nx * elem;
  int s = int(STG_MAX_SMEM / row);
  if (s > STG_MAX_STAGES) s = STG_MAX_STAGES;
  return s < STG_MIN_STAGES ? 0 : s;
}
inline int64_t staged_smem_bytes(int q, int nx, int elem) {
  return int64_t(staged_stages(q, nx, elem)) * q * nx * elem;
}
enum { AUX_GATHER = 0, AUX_SCATTER = 1, AUX_INVARIANTS = 2 };

struct StepArgs {
  const void* src;  // pull source buffer
  void* dst;        // pull destination / AA in-place buffer
  Geo g;
  double rates[6];
  int space;  // SP_RAW / SP_CENTRAL / SP_CUMULANT
  int reg;    // bulk and orders >= 3 relaxed with rate 1 (compile-time)
  int storage;
  int mode;
  int form;     // FORM_DEV / FORM_ABS_EQ (Eq. 2.6 arithmetic, FP64 storage) / FORM_DISC
  int variant;  // VARIANT_DIRECT / VARIANT_STAGED (pull only)
  int* status;  // device word set by a kernel whose bounded wait ran out
  long long wait_limit;  // SM cycles a device wait may take (lbm_set_wait_limit)
  int force_mode;           // FORCE_NONE / FORCE_UNIFORM / FORCE_FIELD
  int force_model;          // 0 Guo, 1 He
  double force[3];          // uniform body force
  const void* force_field;  // per-cell force [D][N] in the compute type (FORCE_FIELD)
  double swe_g;             // > 0: shallow-water method with this gravity (D2Q9)
  // pull steps over a slab of z-planes [z0, z0 + nzc) only (nzc = 0: all)
  int z0, nzc;
  cudaStream_t stream;
};

struct AuxArgs {
  int op;
  void* buf;
  Geo g;
  int storage;
  int space;
  int gather_mode;  // G_* of lbm_kernels.cuh (scatter: G_PULL, G_LOCAL or an even esoteric layout)
  double* df;       // gather outputs (nullable)
  double* rho;
  double* u;
  const double* df_in;  // scatter inputs (df_in, or rho_in / u_in)
  const double* rho_in;
  const double* u_in;
  double* part;  // invariants partials [nparts][8]
  int nparts;
  int force_mode;           // gather: fluid velocity (j + F/2) / rho under a force
  double force[3];
  const void* force_field;
  double swe_g;  // scatter from (h, u): the shallow-water equilibrium
  int disc;      // scatter from (rho, u): the discrete second-order equilibrium
  // gather / scatter over a slab of the lattice (chunked host transfers):
  // z-planes [z0, z0 + nzc) and rows [y0, y0 + nyc); the staged arrays hold
  // the slab's cells only, component k of cell c at k * stride + (c - c0).
  // Whole lattice: y0 = z0 = 0, nyc = Ny, nzc = Nz, c0 = 0, stride = N.
  int y0, z0, nyc, nzc;
  int64_t c0, stride;
  cudaStream_t stream;
};

// the whole lattice as the slab of a read-out / set-up launch
inline void whole_slab(AuxArgs& a) {
  a.y0 = 0;
  a.z0 = 0;
  a.nyc = a.g.ny;
  a.nzc = a.g.nz;
  a.c0 = 0;
  a.stride = a.g.N;
}

// one pair of entry points per (stencil, storage) object file
#define LBM_DECL(ST, SO)                           \
  void launch_step_##ST##_##SO(const StepArgs& a); \
  void launch_aux_##ST##_##SO(const AuxArgs& a);
LBM_DECL(0, 0) LBM_DECL(0, 1) LBM_DECL(0, 2) LBM_DECL(0, 3) LBM_DECL(0, 4)
LBM_DECL(1, 0) LBM_DECL(1, 1) LBM_DECL(1, 2) LBM_DECL(1, 3) LBM_DECL(1, 4)
LBM_DECL(2, 0) LBM_DECL(2, 1) LBM_DECL(2, 2) LBM_DECL(2, 3) LBM_DECL(2, 4)
#undef LBM_DECL

// ----- batched ensemble (lbm_batch.cu)
struct BInst {
  int nx, ny, nz, N;  // box of the instance, N = nx * ny * nz
  int64_t off;        // element offset of its population block
  double keep_shear;  // 1 - shear rate of the instance
  float rnx, rny;     // 1 / nx, 1 / ny (cell index -> x, y, z without division)
};
enum { BATCH_STEP = 0, BATCH_TGV = 1 };
struct BatchArgs {
  int op;
  const void* src;  // BATCH_STEP: pull source buffer
  void* dst;        // BATCH_STEP: destination; BATCH_TGV: buffer to set up
  const BInst* inst;
  const int2* tiles;  // (instance, first cell) of each tile
  int ntiles;
  int cpt;      // cells per thread
  int threads;  // block size
  int grid;     // persistent grid size
  double rates[6];
  int space, reg, storage;
  const double* u0;  // BATCH_TGV: amplitude per instance (device)
  cudaStream_t stream;
};
#define LBM_BDECL(ST, SO) void launch_batch_##ST##_##SO(const BatchArgs& a);
LBM_BDECL(0, 0) LBM_BDECL(0, 1) LBM_BDECL(0, 2) LBM_BDECL(0, 3) LBM_BDECL(0, 4)
LBM_BDECL(1, 0) LBM_BDECL(1, 1) LBM_BDECL(1, 2) LBM_BDECL(1, 3) LBM_BDECL(1, 4)
LBM_BDECL(2, 0) LBM_BDECL(2, 1) LBM_BDECL(2, 2) LBM_BDECL(2, 3) LBM_BDECL(2, 4)
#undef LBM_BDECL

void launch_invariants_fold(const double* part, int nparts, double* out, cudaStream_t s);

// table dispatch to the (stencil, storage) instantiations (lbm_api.cu)
void dispatch_step(int stencil, int storage, const StepArgs& a);
void dispatch_aux(int stencil, int storage, const AuxArgs& a);
void dispatch_batch(int stencil, int storage, const BatchArgs& a);

// closure (lbm_closure.cu): fused learned-rate step of a context; frees
// the context's device closure parameters
void launch_closure_step(const StepArgs& a, const void* closure);
void free_closure(void* closure);

}  // namespace lbm

// single-domain context (shared by lbm_api.cu and lbm_closure.cu)
struct lbm_ctx {
  lbm_params p;
  int q, d;
  lbm::Geo g;
  int eb;
  void* buf[2];
  int cur;     // pull: buffer holding the newest post-collision state
  int parity;  // AA: number of completed steps mod 2
  int64_t t;
  cudaStream_t stream;
  double* part;  // invariants scratch: nparts rows of 8 doubles, then 8
  int nparts;
  int space;  // effective collision space (POPULATIONS -> RAW)
  double rates[6];
  int reg;
  void* closure;  // device closure parameters (lbm_closure.cu), NULL = off
  int* status;    // device word after the invariants scratch: nonzero = a bounded wait ran out
  int kernel;     // requested step kernel (LBM_STEP_*)
  long long wait_limit;  // SM cycles a device wait may take before it gives up
  int force_mode;     // lbm::FORCE_*
  int force_model;    // LBM_FORCE_GUO / LBM_FORCE_HE
  double force[3];    // uniform body force (zeros when unset)
  void* force_field;  // device [D][N] in the compute type, or NULL
  double swe_g;       // > 0: shallow-water method (lbm_set_shallow_water)
  // host transfers in slabs (created on first use): a copy stream, two
  // staging buffers and the events that order them against c->stream
  cudaStream_t io_stream;
  cudaEvent_t io_ready[2], io_done[2];
  double* io_buf[2];
  size_t io_cap;  // doubles per staging buffer
  // staging of lbm_run_host (kept between calls): bytes at run_buf
  double* run_buf;
  size_t run_cap;
  int64_t watch;  // divergence watch period of lbm_step (0: off)
};

