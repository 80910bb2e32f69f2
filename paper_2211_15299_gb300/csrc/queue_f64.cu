// double instantiation of the work-queue kernel launcher (four stages per pass).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f64(const QParams& prm, int grid, int, cudaStream_t st) {
  return launch_queue<double, 4>(prm, grid, st);
}
int queue_grid_f64(int) { return queue_grid<double, 4>(); }
}  // namespace sdft
