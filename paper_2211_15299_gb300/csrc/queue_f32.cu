// float instantiation of the work-queue kernel (four stages per pass, tables
// through registers and L1) and the dispatch to the other variants, each
// compiled in a unit of its own: queue_f32w3.cu (three stages per pass),
// queue_f32st.cu and queue_f32w3st.cu (whole tables staged in shared memory).
#include "queue.cuh"

namespace sdft {
sdft_status launch_queue_f32_w3(const QParams& prm, int grid, cudaStream_t st);
int queue_grid_f32_w3();
sdft_status launch_queue_f32_st(const QParams& prm, int grid, cudaStream_t st);
int queue_grid_f32_st();
sdft_status launch_queue_f32_w3st(const QParams& prm, int grid, cudaStream_t st);
int queue_grid_f32_w3st();

sdft_status launch_queue_f32(const QParams& prm, int grid, int w, bool staged, cudaStream_t st) {
  if (staged) return w == 3 ? launch_queue_f32_w3st(prm, grid, st) : launch_queue_f32_st(prm, grid, st);
  return w == 3 ? launch_queue_f32_w3(prm, grid, st) : launch_queue<float, 4, false>(prm, grid, st);
}
int queue_grid_f32(int w, bool staged) {
  if (staged) return w == 3 ? queue_grid_f32_w3st() : queue_grid_f32_st();
  return w == 3 ? queue_grid_f32_w3() : queue_grid<float, 4, false>();
}
}  // namespace sdft
