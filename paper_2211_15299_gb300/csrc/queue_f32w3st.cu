// float instantiation of the work-queue kernel with whole twiddle tables staged
// in shared memory and three stages per pass (one CTA of 512 compute threads
// per SM).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32_w3st(const QParams& prm, int grid, cudaStream_t st) {
  return launch_queue<float, 3, true>(prm, grid, st);
}
int queue_grid_f32_w3st() { return queue_grid<float, 3, true>(); }
}  // namespace sdft
