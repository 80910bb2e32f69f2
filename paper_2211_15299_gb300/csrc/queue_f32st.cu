// float instantiation of the work-queue kernel with whole twiddle tables staged
// in shared memory (one CTA per SM, four stages per pass).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32_st(const QParams& prm, int grid, cudaStream_t st) {
  return launch_queue<float, 4, true>(prm, grid, st);
}
int queue_grid_f32_st() { return queue_grid<float, 4, true>(); }
}  // namespace sdft
