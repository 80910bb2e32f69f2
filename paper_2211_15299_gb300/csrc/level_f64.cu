// complex128 instantiation of the level launcher.
#include <cmath>

#include "levels.cuh"

namespace sdft {
sdft_status launch_plan_f64(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  return launch_plan<double>(plan, batch, in, out, st);
}
}  // namespace sdft
