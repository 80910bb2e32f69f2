// double instantiation of the work-queue kernel launcher (four stages per pass,
// tables through registers and L1).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f64(const QParams& prm, int grid, int, bool, cudaStream_t st) {
  return launch_queue<double, 4, false>(prm, grid, st);
}
int queue_grid_f64(int, bool) { return queue_grid<double, 4, false>(); }
}  // namespace sdft
