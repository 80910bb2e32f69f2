// float instantiation of the work-queue kernel with three stages per pass.
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32_w3(const QParams& prm, int grid, cudaStream_t st) {
  return launch_queue<float, 3, false>(prm, grid, st);
}
int queue_grid_f32_w3() { return queue_grid<float, 3, false>(); }
}  // namespace sdft
