// Uneven batches (placeholder until the work-queue kernel lands).
#include "launch.hpp"

extern "C" {
sdft_status sdft_batch_create(const sdft_plan*, uint64_t, sdft_batch* out) {
  if (out) *out = nullptr;
  return SDFT_ERR_UNSUPPORTED;
}
sdft_status sdft_batch_info(sdft_batch, uint64_t*, uint64_t*) { return SDFT_ERR_UNSUPPORTED; }
sdft_status sdft_batch_execute(sdft_batch, const void*, void*, void*) { return SDFT_ERR_UNSUPPORTED; }
sdft_status sdft_batch_device_status(sdft_batch, int) { return SDFT_ERR_UNSUPPORTED; }
sdft_status sdft_batch_destroy(sdft_batch) { return SDFT_ERR_UNSUPPORTED; }
}
