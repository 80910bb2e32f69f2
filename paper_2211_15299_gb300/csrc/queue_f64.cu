// double instantiation of the work-queue kernel launcher.
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f64(const QParams& prm, int grid, cudaStream_t st) { return launch_queue<double>(prm, grid, st); }
int queue_grid_f64() { return queue_grid<double>(); }
}  // namespace sdft
