// Host-side launch interfaces shared by the C ABI and the per-precision units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "plan.hpp"

namespace sdft {

// Record a CUDA error for sdft_last_cuda_error and map it to a status.
sdft_status cuda_fail(cudaError_t e);

// Encode a 4-D tiled tensor map over 32-bit words with the 128-byte swizzle.
// dims[0] is 32 (one 128-byte row); strides are byte strides of dims 1..3.
sdft_status encode_map(CUtensorMap* map, const void* base, const uint64_t dims[4],
                       const uint64_t strides[3], const uint32_t box[4]);

// Number of SMs of the current device (cached).
int sm_count();

// Make sure a kernel may use `bytes` of dynamic shared memory (once per device).
sdft_status ensure_smem(const void* fn, int bytes);

// Global bound on device-side waits (nanoseconds).
uint64_t wait_timeout_ns();

// Run every level of `plan` on `batch` packed instances (complex64 / complex128).
sdft_status launch_plan_f32(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
sdft_status launch_plan_f64(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
// complex128 plans with SDFT_PLAN_FP64_DF: double-float butterflies where the
// level kernels run (small instances take the FP64 paths).
sdft_status launch_plan_df(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
sdft_status launch_plan_inv_df(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
// Synthesis: samples from coefficients (the adjoint network scaled by 1/N).
sdft_status launch_plan_inv_f32(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
sdft_status launch_plan_inv_f64(const Plan& plan, uint64_t batch, const void* in, void* out, cudaStream_t st);

// Strided execution of a multi-level plan through the work-queue kernel, with
// the queue for this batch size built on first use and cached in the plan.
sdft_status run_strided_queue(sdft_plan_s* plan, uint64_t batch, const void* in, void* out, cudaStream_t st);
// Release the cached queues of a plan.
void free_strided_queues(Plan& p);
// Release the cached sdft_execute_batched batches whose plan list names the plan
// with this serial (the caller has synchronised before destroying the plan).
void forget_batched(uint64_t serial);
// Pin (never evict implicitly) or unpin the cached sdft_execute_batched list of
// these plans, building it if needed; report whether a list is cached.
sdft_status pin_batched(const sdft_plan* plans, uint64_t n, int pin);
void batched_cache_info(const sdft_plan* plans, uint64_t n, int* cached, int* pinned, uint64_t* n_lists);

// Autotuner choices (autotune.cpp): strategy (plans), item order and grid
// (batches), stages per pass, and the time measured for them.
struct Tuning {
  int strategy = 0;
  int schedule = 0;
  int grid = 0;
  int spp = 4;
  float ms = 0.f;
  int staged = 0;    // uneven batches: whole twiddle tables in shared memory
  int lag = 6;       // uneven batches: dependency distance (x grid list places)
};
std::string plan_tuning_key(sdft_prec prec, uint32_t s, uint64_t batch);
std::string batch_tuning_key(sdft_prec prec, uint64_t n, uint64_t total);
void tuning_store(const std::string& key, const Tuning& t);
bool tuning_lookup(const std::string& key, Tuning* out);

}  // namespace sdft
