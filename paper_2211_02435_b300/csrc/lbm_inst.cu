// lbm_inst.cu -- instantiates the kernels of one (stencil, storage) pair.
// Compiled once per pair with -DLBM_ST=<0|1|2> -DLBM_STORE=<0..3> so the
// twelve heavy translation units build in parallel.
#include "lbm_kernels.cuh"

#ifndef LBM_ST
#error "LBM_ST must be defined"
#endif
#ifndef LBM_STORE
#error "LBM_STORE must be defined"
#endif

namespace lbm {

#if LBM_STORE == 0
using StoreT = double;
using CompT = double;
#elif LBM_STORE == 1
using StoreT = float;
using CompT = float;
#elif LBM_STORE == 2
using StoreT = __half;
using CompT = float;
#elif LBM_STORE == 3
using StoreT = __nv_bfloat16;
using CompT = float;
#else
using StoreT = AbsF64;
using CompT = double;
#endif

#define LBM_CAT(a, b, c) a##b##_##c
#define LBM_FN(pre, st, so) LBM_CAT(pre, st, so)

void LBM_FN(launch_step_, LBM_ST, LBM_STORE)(const StepArgs& a) {
  launch_step_space<LBM_ST, StoreT, CompT>(a);
}
void LBM_FN(launch_aux_, LBM_ST, LBM_STORE)(const AuxArgs& a) {
  launch_aux_typed<LBM_ST, StoreT, CompT>(a);
}
#if LBM_STORE == 4
// the batched ensemble does not serve absolute storage (rejected at create)
void LBM_FN(launch_batch_, LBM_ST, LBM_STORE)(const BatchArgs&) {}
#else
void LBM_FN(launch_batch_, LBM_ST, LBM_STORE)(const BatchArgs& a) {
  launch_batch_space<LBM_ST, StoreT, CompT>(a);
}
#endif

}  // namespace lbm
