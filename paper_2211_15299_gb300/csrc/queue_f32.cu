// float instantiation of the work-queue kernel launcher (four stages per pass;
// three in queue_f32w3.cu).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32_w3(const QParams& prm, int grid, cudaStream_t st);
int queue_grid_f32_w3();

sdft_status launch_queue_f32(const QParams& prm, int grid, int w, cudaStream_t st) {
  return w == 3 ? launch_queue_f32_w3(prm, grid, st) : launch_queue<float, 4>(prm, grid, st);
}
int queue_grid_f32(int w) { return w == 3 ? queue_grid_f32_w3() : queue_grid<float, 4>(); }
}  // namespace sdft
