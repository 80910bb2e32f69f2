// complex64 level kernels with three stages per pass (2^3 values per thread,
// 512 threads per 2^12-value tile), compiled apart from the four-stage ones.
#include <cmath>

#include "levels.cuh"

namespace sdft {
sdft_status dispatch_first_f32w3(int phi, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                                 const LevelArgs<float>& a, cudaStream_t st) {
  return dispatch_first_w<float, 3>(phi, last, grid, src, dst, a, st);
}
sdft_status dispatch_later_f32w3(int q, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                                 const LevelArgs<float>& a, cudaStream_t st) {
  return dispatch_later_w<float, 3>(q, last, grid, src, dst, a, st);
}
}  // namespace sdft
