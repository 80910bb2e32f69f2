// complex128 plans in double-float arithmetic (SDFT_PLAN_FP64_DF): the level
// kernels instantiated for the `dfloat` type; instances small enough for the
// register and warp paths run those in FP64.
#include "levels.cuh"

namespace sdft {

sdft_status launch_plan_df(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  if (plan.levels.empty() || warp_path(plan, batch)) return launch_plan_f64(plan, batch, in, out, st);
  return launch_plan<dfloat>(plan, batch, in, out, st);
}

sdft_status launch_plan_inv_df(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  if (plan.levels.empty()) return launch_plan_inv_f64(plan, batch, in, out, st);
  return launch_plan_inv<dfloat>(plan, batch, in, out, st);
}

}  // namespace sdft
