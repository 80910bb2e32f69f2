// C ABI of the library: plans, execution, diagnostics (declared in include/sdft.h).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "launch.hpp"
#include "plan.hpp"

namespace sdft {

namespace {
thread_local int g_last_cuda_error = 0;
std::mutex g_mu;
std::set<std::pair<int, const void*>> g_smem_set;
// Filled once and read from any thread (the caller's, a server's worker and
// planners): atomics, so the first-use checks below are race-free.
std::atomic<int> g_sm_count[64];            // static storage: zero-initialised
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

#if SDFT_BOUNDS_CHECK
// Readers of the per-translation-unit violation counters of the debug build.
static std::vector<uint64_t (*)(int)>& violation_readers() {
  static std::vector<uint64_t (*)(int)> v;
  return v;
}
void register_violation_reader(uint64_t (*reader)(int clear)) { violation_readers().push_back(reader); }
#endif

sdft_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = int(e);
  return SDFT_ERR_CUDA;
}

uint64_t wait_timeout_ns() {
  static const uint64_t v = [] {
    const char* s = std::getenv("SDFT_WAIT_TIMEOUT_NS");
    const unsigned long long x = s ? std::strtoull(s, nullptr, 10) : 0ull;
    return x ? uint64_t(x) : uint64_t(2000000000ull);
  }();
  return v;
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int v = g_sm_count[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    g_sm_count[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

sdft_status ensure_smem(const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_smem_set.count({dev, fn})) return SDFT_OK;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_fail(e);
  g_smem_set.insert({dev, fn});
  return SDFT_OK;
}

sdft_status encode_map(CUtensorMap* map, const void* base, const uint64_t dims[4], const uint64_t strides[3],
                       const uint32_t box[4]) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = g_encode.load(std::memory_order_acquire);
  if (!encode) {
    std::lock_guard<std::mutex> lk(g_mu);
    encode = g_encode.load(std::memory_order_acquire);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cuda_fail(e);
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
      g_encode.store(encode, std::memory_order_release);
    }
  }
  cuuint64_t gdim[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t gstr[3] = {strides[0], strides[1], strides[2]};
  cuuint32_t bdim[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), gdim, gstr, bdim,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_last_cuda_error = int(r);
    return SDFT_ERR_CUDA;
  }
  return SDFT_OK;
}

// Check buffers: 16-byte aligned, and either identical (in place) or disjoint.
static sdft_status check_buffers(const void* in, const void* out, uint64_t bytes) {
  if (!in || !out) return SDFT_ERR_ARG;
  if (!aligned16(in) || !aligned16(out)) return SDFT_ERR_ARG;
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
  if (a != b && a < b + bytes && b < a + bytes) return SDFT_ERR_ARG;
  return SDFT_OK;
}

static sdft_status check_device(const Plan& p) {
  if (p.device < 0 || !p.d_status) return SDFT_ERR_NO_DEVICE;
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  return dev == p.device ? SDFT_OK : SDFT_ERR_ARG;
}

// d_user[b k + u] = d_canonical[b k + pos[u]]: reads within one instance (cached),
// coalesced writes.
template <class C>
__global__ void __launch_bounds__(256) k_user_order(const C* __restrict__ src, C* __restrict__ dst,
                                                    const uint32_t* __restrict__ pos, uint64_t k, uint64_t total) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t b = i / k, u = i - b * k;
    dst[i] = src[b * k + pos[u]];
  }
}

sdft_status launch_user_order(const Plan& p, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  const uint64_t total = batch * p.k;
  const uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 8ull * uint64_t(sm_count()));
  if (p.prec == SDFT_C64)
    k_user_order<float2><<<unsigned(blocks), 256, 0, st>>>(static_cast<const float2*>(in), static_cast<float2*>(out),
                                                            p.d_user_pos, p.k, total);
  else
    k_user_order<double2><<<unsigned(blocks), 256, 0, st>>>(static_cast<const double2*>(in),
                                                             static_cast<double2*>(out), p.d_user_pos, p.k, total);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

sdft_status run_strided(sdft_plan_s* h, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  const Plan& p = h->p;
  sdft_status s = check_device(p);
  if (s != SDFT_OK) return s;
  if (batch == 0) return SDFT_OK;
  const uint64_t eb = uint64_t(elem_bytes(p.prec));
  if (batch > (~0ull / eb) / p.k) return SDFT_ERR_ARG;
  s = check_buffers(in, out, batch * p.k * eb);
  if (s != SDFT_OK) return s;
  // Several levels: one launch per level (each a persistent kernel whose CTAs take
  // every G-th tile), or, with the queue strategy, one persistent launch over a
  // work queue that keeps each instance's intermediate in L2. The per-level
  // launches run at the speed of a copy of every level's tiles and were measured
  // faster at N = 2^30, k = 2^20, batch 64; the queue halves the DRAM traffic
  // there but its per-item work bounds it.
  if (p.levels.size() > 1 && p.strategy == SDFT_STRATEGY_QUEUE) return run_strided_queue(h, batch, in, out, st);
  if (p.prec == SDFT_C64) return launch_plan_f32(p, batch, in, out, st);
  return p.d_tw_df ? launch_plan_df(p, batch, in, out, st) : launch_plan_f64(p, batch, in, out, st);
}

// Synthesis of `batch` instances: samples from coefficients.
static sdft_status run_strided_inverse(sdft_plan_s* h, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  const Plan& p = h->p;
  sdft_status s = check_device(p);
  if (s != SDFT_OK) return s;
  if (batch == 0) return SDFT_OK;
  const uint64_t eb = uint64_t(elem_bytes(p.prec));
  if (batch > (~0ull / eb) / p.k) return SDFT_ERR_ARG;
  s = check_buffers(in, out, batch * p.k * eb);
  if (s != SDFT_OK) return s;
  if (p.prec == SDFT_C64) return launch_plan_inv_f32(p, batch, in, out, st);
  return p.d_tw_df ? launch_plan_inv_df(p, batch, in, out, st) : launch_plan_inv_f64(p, batch, in, out, st);
}

}  // namespace sdft

using sdft::Plan;

extern "C" {

sdft_status sdft_plan_create(uint32_t log2N, const uint64_t* J, uint64_t k, sdft_prec prec, uint32_t flags,
                             sdft_plan* out) {
  if (!out) return SDFT_ERR_ARG;
  *out = nullptr;
  if (flags & ~(SDFT_PLAN_HOST_ONLY | SDFT_PLAN_DEFER_DEVICE | SDFT_PLAN_FP64_DF | SDFT_PLAN_USER_ORDER))
    return SDFT_ERR_ARG;
  if ((flags & SDFT_PLAN_HOST_ONLY) && (flags & SDFT_PLAN_DEFER_DEVICE)) return SDFT_ERR_ARG;
  if ((flags & SDFT_PLAN_FP64_DF) && prec != SDFT_C128) return SDFT_ERR_ARG;
  sdft_plan_s* h = new (std::nothrow) sdft_plan_s();
  if (!h) return SDFT_ERR_NOMEM;
  sdft_status s;
  try {
    s = sdft::build_plan(log2N, J, k, prec, h->p);
  } catch (const std::bad_alloc&) {
    s = SDFT_ERR_NOMEM;
  }
  if (s != SDFT_OK) {
    delete h;
    return s;
  }
  Plan& p = h->p;
  {
    static std::atomic<uint64_t> next_serial{1};
    p.serial = next_serial.fetch_add(1);
  }
  if (!(flags & SDFT_PLAN_HOST_ONLY)) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      delete h;
      return sdft::cuda_fail(e);
    }
    const size_t eb = size_t(sdft::elem_bytes(prec));
    const size_t tw_bytes = size_t(p.tw_elems) * eb;
    std::vector<unsigned char> host;
    try {
      host.resize(tw_bytes);
    } catch (const std::bad_alloc&) {
      delete h;
      return SDFT_ERR_NOMEM;
    }
    if (prec == SDFT_C64)
      sdft::fill_device_tables<float>(p, reinterpret_cast<float*>(host.data()));
    else
      sdft::fill_device_tables<double>(p, reinterpret_cast<double*>(host.data()));
    if (!p.levels.empty()) {  // entries 1..15 of the level-0 table go into kernel parameters
      for (int i = 0; i < 30 && size_t(2 + i) < 2 * size_t(p.tw_elems); ++i)
        p.tw0[i] = prec == SDFT_C64 ? double(reinterpret_cast<const float*>(host.data())[2 + i])
                                    : reinterpret_cast<const double*>(host.data())[2 + i];
    }
    if (flags & SDFT_PLAN_DEFER_DEVICE) {     // keep the tables on the host for a server
      p.host_tables.swap(host);
      p.deferred = true;
      p.device = dev;
      *out = h;
      return SDFT_OK;
    }
    e = cudaMalloc(&p.d_status, 256);
    if (e == cudaSuccess) e = cudaMemset(p.d_status, 0, 256);
    if (e == cudaSuccess && tw_bytes) e = cudaMalloc(&p.d_tw, tw_bytes);
    if (e == cudaSuccess && tw_bytes) e = cudaMemcpy(p.d_tw, host.data(), tw_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tw_bytes && (flags & SDFT_PLAN_FP64_DF)) {
      // the same entries split into hi = RN(x), lo = RN(x - hi) pairs, laid out
      // (re_hi, im_hi, re_lo, im_lo): 16 bytes per entry, as complex128
      std::vector<float> df;
      try {
        df.resize(4 * size_t(p.tw_elems));
      } catch (const std::bad_alloc&) {
        e = cudaErrorMemoryAllocation;
      }
      const double* tw64 = reinterpret_cast<const double*>(host.data());
      for (size_t i = 0; e == cudaSuccess && i < size_t(p.tw_elems); ++i) {
        const double re = tw64[2 * i], im = tw64[2 * i + 1];
        const float rh = float(re), ih = float(im);
        df[4 * i] = rh;
        df[4 * i + 1] = ih;
        df[4 * i + 2] = float(re - double(rh));
        df[4 * i + 3] = float(im - double(ih));
      }
      if (e == cudaSuccess) e = cudaMalloc(&p.d_tw_df, tw_bytes);
      if (e == cudaSuccess) e = cudaMemcpy(p.d_tw_df, df.data(), tw_bytes, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && (flags & SDFT_PLAN_USER_ORDER)) {
      // canonical position of J[u]: bit q of the key is bit r_q of J[u]
      std::vector<uint32_t> pos;
      try {
        pos.resize(size_t(p.k));
      } catch (const std::bad_alloc&) {
        e = cudaErrorMemoryAllocation;
      }
      for (uint64_t u = 0; e == cudaSuccess && u < p.k; ++u) {
        uint64_t t = 0;
        for (uint32_t q = 0; q < p.s; ++q) t |= ((J[u] >> p.pivots[q]) & 1ull) << q;
        pos[size_t(u)] = uint32_t(t);
      }
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p.d_user_pos), sizeof(uint32_t) * p.k);
      if (e == cudaSuccess)
        e = cudaMemcpy(p.d_user_pos, pos.data(), sizeof(uint32_t) * p.k, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      if (p.d_user_pos) cudaFree(p.d_user_pos);
      if (p.d_tw_df) cudaFree(p.d_tw_df);
      if (p.d_tw) cudaFree(p.d_tw);
      if (p.d_status) cudaFree(p.d_status);
      delete h;
      return e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : sdft::cuda_fail(e);
    }
    p.device = dev;
    p.device_bytes = tw_bytes + 256 + (p.d_tw_df ? tw_bytes : 0) +
                     (p.d_user_pos ? sizeof(uint32_t) * p.k : 0);
  }
  *out = h;
  return SDFT_OK;
}

sdft_status sdft_plan_info(sdft_plan plan, uint32_t* log2N, uint32_t* log2k, sdft_prec* prec) {
  if (!plan) return SDFT_ERR_ARG;
  if (log2N) *log2N = plan->p.M;
  if (log2k) *log2k = plan->p.s;
  if (prec) *prec = plan->p.prec;
  return SDFT_OK;
}

sdft_status sdft_plan_pivots(sdft_plan plan, uint32_t* pivots) {
  if (!plan || (!pivots && plan->p.s)) return SDFT_ERR_ARG;
  for (uint32_t q = 0; q < plan->p.s; ++q) pivots[q] = plan->p.pivots[q];
  return SDFT_OK;
}

sdft_status sdft_plan_sample_indices(sdft_plan plan, uint64_t* I) {
  if (!plan || !I) return SDFT_ERR_ARG;
  std::memcpy(I, plan->p.I.data(), sizeof(uint64_t) * plan->p.k);
  return SDFT_OK;
}

sdft_status sdft_plan_support_order(sdft_plan plan, uint64_t* Jc) {
  if (!plan || !Jc) return SDFT_ERR_ARG;
  std::memcpy(Jc, plan->p.Jc.data(), sizeof(uint64_t) * plan->p.k);
  return SDFT_OK;
}

sdft_status sdft_plan_twiddles(sdft_plan plan, double* tw) {
  if (!plan || (!tw && plan->p.k > 1)) return SDFT_ERR_ARG;
  const Plan& p = plan->p;
  for (uint32_t m = 1; m <= p.s; ++m)
    for (uint64_t u = 0; u < (1ull << (m - 1)); ++u) {
      const uint64_t idx = (1ull << (m - 1)) - 1 + u;
      sdft::twiddle_f64(p, m, u, tw[2 * idx], tw[2 * idx + 1]);
    }
  return SDFT_OK;
}

sdft_status sdft_plan_device_bytes(sdft_plan plan, uint64_t* bytes) {
  if (!plan || !bytes) return SDFT_ERR_ARG;
  *bytes = plan->p.device_bytes;
  return SDFT_OK;
}

sdft_status sdft_execute(sdft_plan plan, const void* d_samples, void* d_coeffs, void* stream) {
  if (!plan) return SDFT_ERR_ARG;
  return sdft::run_strided(plan, 1, d_samples, d_coeffs, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_execute_strided(sdft_plan plan, uint64_t batch, const void* d_samples, void* d_coeffs,
                                 void* stream) {
  if (!plan) return SDFT_ERR_ARG;
  return sdft::run_strided(plan, batch, d_samples, d_coeffs, static_cast<cudaStream_t>(stream));
}

// Host-buffer batches: chunked copy-in, transform (or synthesis) and copy-out
// overlapped on the plan's two copy streams and the caller's stream.
static sdft_status run_host(sdft_plan plan, uint64_t batch, const void* h_in_buf, void* h_out_buf, void* d_in_buf,
                            void* d_out_buf, uint64_t chunk, void* stream, bool inverse) {
  const void* h_samples = h_in_buf;
  void* h_coeffs = h_out_buf;
  void* d_samples = d_in_buf;
  void* d_coeffs = d_out_buf;
  if (!plan || !h_samples || !h_coeffs) return SDFT_ERR_ARG;
  const sdft::Plan& p = plan->p;
  if (p.device < 0 || !p.d_status) return SDFT_ERR_NO_DEVICE;
  if (batch == 0) return SDFT_OK;
  const uint64_t inst_bytes = p.k * uint64_t(sdft::elem_bytes(p.prec));
  if (batch > ~0ull / inst_bytes) return SDFT_ERR_ARG;
  const uint64_t total = batch * inst_bytes;
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(h_samples), b = reinterpret_cast<uintptr_t>(h_coeffs);
    if (a != b && a < b + total && b < a + total) return SDFT_ERR_ARG;   // host buffers: identical or disjoint
  }
  {  // the device side too, before anything is enqueued
    sdft_status s0 = sdft::check_device(p);
    if (s0 == SDFT_OK) s0 = sdft::check_buffers(d_samples, d_coeffs, total);
    if (s0 != SDFT_OK) return s0;
  }
  // chunks of about 16 MiB, each a multiple of 16 bytes so that every chunk's
  // device offset keeps the 16-byte alignment of the buffers
  const uint64_t unit = inst_bytes >= 16 ? 1 : 16 / inst_bytes;
  if (chunk == 0) chunk = std::max<uint64_t>(1, (16ull << 20) / inst_bytes);
  chunk = (chunk + unit - 1) / unit * unit;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(plan->host_mu);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    if (!plan->host_st[i]) {
      cudaStream_t st = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      plan->host_st[i] = st;
    }
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    if (!plan->host_ev[i]) {
      cudaEvent_t ev = nullptr;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      plan->host_ev[i] = ev;
    }
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  cudaStream_t in_st = static_cast<cudaStream_t>(plan->host_st[0]);
  cudaStream_t out_st = static_cast<cudaStream_t>(plan->host_st[1]);
  cudaEvent_t ev_in = static_cast<cudaEvent_t>(plan->host_ev[0]);    // a chunk's samples are on the device
  cudaEvent_t ev_done = static_cast<cudaEvent_t>(plan->host_ev[1]);  // a chunk's coefficients are computed
  cudaEvent_t ev_mark = static_cast<cudaEvent_t>(plan->host_ev[2]);  // start and end of the call
  // the copies start after the work already on the caller's stream
  e = cudaEventRecord(ev_mark, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(in_st, ev_mark, 0);
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  const char* hi = static_cast<const char*>(h_samples);
  char* ho = static_cast<char*>(h_coeffs);
  char* di = static_cast<char*>(d_samples);
  char* dout = static_cast<char*>(d_coeffs);
  for (uint64_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint64_t nb = std::min(chunk, batch - b0);
    const uint64_t off = b0 * inst_bytes, bytes = nb * inst_bytes;
    e = cudaMemcpyAsync(di + off, hi + off, bytes, cudaMemcpyHostToDevice, in_st);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, in_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in, 0);
    if (e != cudaSuccess) return sdft::cuda_fail(e);
    const sdft_status s = inverse ? sdft::run_strided_inverse(plan, nb, di + off, dout + off, cs)
                                  : sdft::run_strided(plan, nb, di + off, dout + off, cs);
    if (s != SDFT_OK) return s;
    e = cudaEventRecord(ev_done, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(out_st, ev_done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ho + off, dout + off, bytes, cudaMemcpyDeviceToHost, out_st);
    if (e != cudaSuccess) return sdft::cuda_fail(e);
  }
  // the caller's stream continues once the last copy-out is done
  e = cudaEventRecord(ev_mark, out_st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_mark, 0);
  return e == cudaSuccess ? SDFT_OK : sdft::cuda_fail(e);
}

sdft_status sdft_execute_strided_host(sdft_plan plan, uint64_t batch, const void* h_samples, void* h_coeffs,
                                      void* d_samples, void* d_coeffs, uint64_t chunk, void* stream) {
  return run_host(plan, batch, h_samples, h_coeffs, d_samples, d_coeffs, chunk, stream, false);
}

sdft_status sdft_synthesize_strided_host(sdft_plan plan, uint64_t batch, const void* h_coeffs, void* h_samples,
                                         void* d_coeffs, void* d_samples, uint64_t chunk, void* stream) {
  return run_host(plan, batch, h_coeffs, h_samples, d_coeffs, d_samples, chunk, stream, true);
}

sdft_status sdft_plan_to_user_order(sdft_plan plan, uint64_t batch, const void* d_canonical, void* d_user,
                                    void* stream) {
  if (!plan || !d_canonical || !d_user) return SDFT_ERR_ARG;
  const sdft::Plan& p = plan->p;
  if (p.device < 0 || !p.d_status) return SDFT_ERR_NO_DEVICE;
  if (!p.d_user_pos) return SDFT_ERR_ARG;
  if (batch == 0) return SDFT_OK;
  const uint64_t eb = uint64_t(sdft::elem_bytes(p.prec));
  if (batch > (~0ull / eb) / p.k) return SDFT_ERR_ARG;
  const uint64_t bytes = batch * p.k * eb;
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_canonical), b = reinterpret_cast<uintptr_t>(d_user);
  if (a < b + bytes && b < a + bytes) return SDFT_ERR_ARG;
  return sdft::launch_user_order(p, batch, d_canonical, d_user, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_synthesize(sdft_plan plan, const void* d_coeffs, void* d_samples, void* stream) {
  if (!plan) return SDFT_ERR_ARG;
  return sdft::run_strided_inverse(plan, 1, d_coeffs, d_samples, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_synthesize_strided(sdft_plan plan, uint64_t batch, const void* d_coeffs, void* d_samples,
                                    void* stream) {
  if (!plan) return SDFT_ERR_ARG;
  return sdft::run_strided_inverse(plan, batch, d_coeffs, d_samples, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_plan_set_strategy(sdft_plan plan, sdft_strategy strategy) {
  if (!plan) return SDFT_ERR_ARG;
  if (strategy != SDFT_STRATEGY_LEVELS && strategy != SDFT_STRATEGY_QUEUE) return SDFT_ERR_ARG;
  plan->p.strategy = int(strategy);
  return SDFT_OK;
}

// Stages per pass of a plan's level kernels; a change drops the plan's cached
// work queues (their grid follows the kernel's occupancy), after the device
// has finished any work that uses them.
static sdft_status set_plan_spp(sdft::Plan& p, uint32_t spp) {
  if (spp != 4 && !(spp == 3 && p.prec == SDFT_C64)) return SDFT_ERR_ARG;
  if (p.spp == spp) return SDFT_OK;
  if (p.queues) {
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return sdft::cuda_fail(e);
    sdft::free_strided_queues(p);
  }
  p.spp = spp;
  return SDFT_OK;
}

sdft_status sdft_plan_set_stages_per_pass(sdft_plan plan, uint32_t stages_per_pass) {
  if (!plan) return SDFT_ERR_ARG;
  return set_plan_spp(plan->p, stages_per_pass);
}

sdft_status sdft_plan_get_stages_per_pass(sdft_plan plan, uint32_t* stages_per_pass) {
  if (!plan || !stages_per_pass) return SDFT_ERR_ARG;
  *stages_per_pass = plan->p.spp;
  return SDFT_OK;
}

sdft_status sdft_plan_apply_tuning(sdft_plan plan, uint64_t batch, int* found) {
  if (!plan) return SDFT_ERR_ARG;
  sdft::Tuning t;
  const bool hit = sdft::tuning_lookup(sdft::plan_tuning_key(plan->p.prec, plan->p.s, batch), &t);
  if (found) *found = hit ? 1 : 0;
  if (!hit) return SDFT_OK;
  if (t.strategy != SDFT_STRATEGY_LEVELS && t.strategy != SDFT_STRATEGY_QUEUE) return SDFT_ERR_ARG;
  sdft_status s = set_plan_spp(plan->p, uint32_t(t.spp));
  if (s != SDFT_OK) return s;
  plan->p.strategy = t.strategy;
  return SDFT_OK;
}

sdft_status sdft_plan_autotune(sdft_plan plan, uint64_t batch, const void* d_samples, void* d_coeffs,
                               void* stream, int reps, sdft_strategy* chosen, float* ms_levels,
                               float* ms_queue) {
  if (!plan || reps <= 0) return SDFT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  sdft::Plan& p = plan->p;
  const bool multi = p.levels.size() > 1;
  // strategy (one launch per level, or the work queue) x stages per pass (four;
  // three as well for complex64)
  struct Cand {
    int strategy;
    uint32_t spp;
    float ms;
  };
  std::vector<Cand> cands;
  for (int strat : {int(SDFT_STRATEGY_LEVELS), int(SDFT_STRATEGY_QUEUE)}) {
    if (strat == SDFT_STRATEGY_QUEUE && !multi) continue;
    for (uint32_t spp : {4u, 3u})
      if (spp == 4 || p.prec == SDFT_C64) cands.push_back(Cand{strat, spp, 0.f});
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  sdft_status s = SDFT_OK;
  const int saved = p.strategy;
  const uint32_t saved_spp = p.spp;
  for (Cand& c : cands) {
    p.strategy = c.strategy;
    s = set_plan_spp(p, c.spp);
    if (s != SDFT_OK) break;
    s = sdft::run_strided(plan, batch, d_samples, d_coeffs, st);    // warm-up (builds a queue if needed)
    if (s == SDFT_OK) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == SDFT_OK && e == cudaSuccess; ++r)
      s = sdft::run_strided(plan, batch, d_samples, d_coeffs, st);
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventElapsedTime(&c.ms, e0, e1);
    if (e != cudaSuccess && s == SDFT_OK) s = sdft::cuda_fail(e);
    if (s != SDFT_OK) break;
    c.ms /= float(reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SDFT_OK) {
    p.strategy = saved;
    set_plan_spp(p, saved_spp);
    return s;
  }
  const Cand* best = &cands[0];
  float best_lv = -1.f, best_q = -1.f;
  for (const Cand& c : cands) {
    if (c.ms < best->ms) best = &c;
    float& slot = c.strategy == SDFT_STRATEGY_LEVELS ? best_lv : best_q;
    if (slot < 0.f || c.ms < slot) slot = c.ms;
  }
  p.strategy = best->strategy;
  s = set_plan_spp(p, best->spp);
  if (s != SDFT_OK) return s;
  sdft::tuning_store(sdft::plan_tuning_key(p.prec, p.s, batch),
                     sdft::Tuning{best->strategy, 0, 0, int(best->spp), best->ms});
  if (chosen) *chosen = sdft_strategy(best->strategy);
  if (ms_levels) *ms_levels = best_lv;
  if (ms_queue) *ms_queue = best_q < 0.f ? 0.f : best_q;
  return SDFT_OK;
}

sdft_status sdft_plan_device_status(sdft_plan plan, int clear) {
  if (!plan) return SDFT_ERR_ARG;
  if (!plan->p.d_status) return SDFT_ERR_NO_DEVICE;
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, plan->p.d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(plan->p.d_status, 0, sizeof(int));
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  return sdft_status(v);
}

sdft_status sdft_plan_destroy(sdft_plan plan) {
  if (!plan) return SDFT_ERR_ARG;
  sdft::free_strided_queues(plan->p);
  sdft::forget_batched(plan->p.serial);
  for (void* st : plan->host_st)
    if (st) cudaStreamDestroy(static_cast<cudaStream_t>(st));
  for (void* ev : plan->host_ev)
    if (ev) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
  if (plan->p.d_tw) cudaFree(plan->p.d_tw);
  if (plan->p.d_tw_df) cudaFree(plan->p.d_tw_df);
  if (plan->p.d_user_pos) cudaFree(plan->p.d_user_pos);
  if (plan->p.d_status) cudaFree(plan->p.d_status);
  delete plan;
  return SDFT_OK;
}

const char* sdft_status_string(sdft_status s) {
  switch (s) {
    case SDFT_OK: return "ok";
    case SDFT_ERR_ARG: return "invalid argument";
    case SDFT_ERR_NOT_POW2: return "support size is not a power of two";
    case SDFT_ERR_RANGE: return "support element or log2N out of range";
    case SDFT_ERR_DUPLICATE: return "support has a repeated element";
    case SDFT_ERR_NOT_HOMOGENEOUS: return "support is not homogeneous";
    case SDFT_ERR_NOMEM: return "out of memory";
    case SDFT_ERR_BUDGET: return "memory budget exceeded";
    case SDFT_ERR_CUDA: return "CUDA error";
    case SDFT_ERR_TIMEOUT: return "device-side wait timed out";
    case SDFT_ERR_UNSUPPORTED: return "unsupported size or mode";
    case SDFT_ERR_NO_DEVICE: return "plan has no device tables";
    case SDFT_ERR_PRECISION: return "plans of different precision in one batch";
  }
  return "unknown status";
}

int sdft_last_cuda_error(void) { return sdft::g_last_cuda_error; }

int sdft_version(void) { return 100; }

sdft_status sdft_debug_bounds_violations(int* enabled, uint64_t* count, int clear) {
#if SDFT_BOUNDS_CHECK
  uint64_t total = 0;
  for (auto* r : sdft::violation_readers()) {
    const uint64_t v = r(clear);
    if (v == ~0ull) return SDFT_ERR_CUDA;
    total += v;
  }
  if (enabled) *enabled = 1;
  if (count) *count = total;
#else
  (void)clear;
  if (enabled) *enabled = 0;
  if (count) *count = 0;
#endif
  return SDFT_OK;
}

}  // extern "C"
