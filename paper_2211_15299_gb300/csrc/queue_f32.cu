// float instantiation of the work-queue kernel launcher.
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32(const QParams& prm, int grid, cudaStream_t st) { return launch_queue<float>(prm, grid, st); }
int queue_grid_f32() { return queue_grid<float>(); }
}  // namespace sdft
