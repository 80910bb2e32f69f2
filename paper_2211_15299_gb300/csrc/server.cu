// Serving engine: continuous batching of transform requests.
//
// Requests (a plan and pinned host buffers) enter a FIFO. A worker thread
// admits them while the device-memory budget allows: every request gets one
// block of an arena allocated once (a buddy allocator hands out blocks aligned
// to their size, so one set of tensor maps over the arena addresses every
// block). Admitted requests form a micro-batch run on one of a few slots: on the
// slot's stream, the samples are copied in, one persistent work-queue launch
// transforms every request in place, the coefficients are copied out, and a host
// callback stamps the completion. Requests that arrive while slots are busy are
// admitted as soon as a slot and memory free up, and the launches of different
// slots overlap on the device (each slot's grid is its share of the co-resident
// CTAs, so in-flight launches never wait on each other). Requests that bring a
// support instead of a plan are planned by the server's own planner threads
// (a deferred plan: tables built in host memory, uploaded into the arena with
// the request) and enter the FIFO once planned; the plan is released when the
// request completes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "plan.hpp"
#include "queue.cuh"

namespace sdft {
namespace {

using Clock = std::chrono::steady_clock;

// Buddy allocator over [0, 2^top) in units of 2^min_order bytes.
class Buddy {
 public:
  void init(uint32_t min_order, uint32_t top_order) {
    min_ = min_order;
    top_ = top_order;
    free_.assign(top_order + 1, {});
    free_[top_order].push_back(0);
  }
  // Returns the offset of a free block of 2^order bytes, or ~0 if none.
  uint64_t alloc(uint32_t order) {
    order = std::max(order, min_);
    if (order > top_) return ~0ull;
    uint32_t o = order;
    while (o <= top_ && free_[o].empty()) ++o;
    if (o > top_) return ~0ull;
    uint64_t off = free_[o].back();
    free_[o].pop_back();
    while (o > order) {            // split, keep the low half
      --o;
      free_[o].push_back(off + (1ull << o));
    }
    used_ += 1ull << order;
    peak_ = std::max(peak_, used_);
    return off;
  }
  void release(uint64_t off, uint32_t order) {
    order = std::max(order, min_);
    used_ -= 1ull << order;
    while (order < top_) {         // merge with the buddy while it is free
      const uint64_t buddy = off ^ (1ull << order);
      auto& fl = free_[order];
      auto it = std::find(fl.begin(), fl.end(), buddy);
      if (it == fl.end()) break;
      *it = fl.back();
      fl.pop_back();
      off = std::min(off, buddy);
      ++order;
    }
    free_[order].push_back(off);
  }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }

 private:
  uint32_t min_ = 7, top_ = 7;
  std::vector<std::vector<uint64_t>> free_;
  uint64_t used_ = 0, peak_ = 0;
};

struct Req {
  uint64_t tag;
  const Plan* plan;
  const void* h_in;
  void* h_out;
  Clock::time_point t_submit;
  uint64_t off = 0;      // arena byte offset
  uint32_t order = 0;    // log2 block bytes
  const void* tw = nullptr;   // device twiddle tables used for this request
  uint64_t tw_off = 0;        // arena block of a deferred plan's tables
  uint32_t tw_order = 0;
  bool own_tw = false;
  sdft_plan own_plan = nullptr;   // planned by the server for this request
  bool inj_seen = false;          // counted by the fault injector already
};

struct PlanJob {
  uint64_t tag;
  uint32_t M;
  std::vector<uint64_t> J;
  const void* h_in;
  void* h_out;
  Clock::time_point t_submit;
};

struct Done {
  uint64_t tag;
  double latency;
  int32_t status;
};

struct Slot {
  cudaStream_t stream = nullptr;
  QItem* d_items = nullptr;
  QInst* d_insts = nullptr;
  uint32_t* d_counters = nullptr;
  QItem* h_items = nullptr;      // pinned staging
  QInst* h_insts = nullptr;
  size_t cap_items = 0, cap_insts = 0, cap_ctr = 0;
  std::vector<Req> reqs;
  std::atomic<bool> done{false};
  Clock::time_point t_done;
  bool busy = false;
  std::condition_variable* cv = nullptr;   // the server's, notified on completion
};

}  // namespace

struct Server {
  int device = -1;
  sdft_prec prec = SDFT_C64;
  uint64_t budget = 0;
  char* d_arena = nullptr;
  int* d_status = nullptr;
  Buddy buddy;
  std::vector<Slot*> slots;
  uint32_t max_batch = 0;
  int grid = 0;
  QParams maps;                  // tensor maps over the arena (filled once)
  uint32_t later_slot[64][64];   // (lo, hi) -> map slot
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> waiting;
  std::vector<Done> done;
  sdft_server_stats stats{};
  std::thread worker;
  bool stop = false;
  sdft_status worker_error = SDFT_OK;
  // planner pool for requests that bring their own support
  std::vector<std::thread> planners;
  std::deque<PlanJob> plan_jobs;
  std::condition_variable plan_cv;
  uint64_t planning = 0;         // jobs queued or being planned
  // host-side fault injection (sdft_server_inject): every inj_every-th request
  // reaching admission is dropped, failed or delayed
  uint32_t inj_mode = 0;
  uint64_t inj_every = 0, inj_delay_us = 0, inj_count = 0;
};

namespace {

void CUDART_CB on_slot_done(void* p) {   // host callback: no CUDA calls here
  Slot* s = static_cast<Slot*>(p);
  s->t_done = Clock::now();
  s->done.store(true, std::memory_order_release);
  s->cv->notify_one();
}

sdft_status init_maps(Server& S) {
  const uint32_t TB = tile_bits(S.prec), CB = row_bits(S.prec);
  const uint64_t es = uint64_t(elem_bytes(S.prec));
  std::memset(&S.maps, 0, sizeof(S.maps));
  std::memset(S.later_slot, 0xff, sizeof(S.later_slot));
  const uint64_t rows = S.budget / 128;
  for (uint32_t r = 0; r <= 8; ++r) {
    if (rows < (1ull << r)) continue;
    const uint64_t dims[4] = {32, rows, 1, 1};
    const uint64_t strides[3] = {128, rows * 128, rows * 128};
    const uint32_t box[4] = {32, 1u << r, 1, 1};
    sdft_status s = encode_map(&S.maps.maps[2 * r], S.d_arena, dims, strides, box);
    if (s == SDFT_OK) s = encode_map(&S.maps.maps[2 * r + 1], S.d_arena, dims, strides, box);
    if (s != SDFT_OK) return s;
    q_set_limits(S.maps, 2 * r, dims);
    q_set_limits(S.maps, 2 * r + 1, dims);
  }
  uint32_t slot = 18;
  const uint64_t elems = S.budget / es;
  for (uint32_t lo = TB; lo < SDFT_MAX_LOG2K; lo += TB - CB) {
    for (uint32_t hi = lo + 1; hi <= lo + (TB - CB) && hi <= SDFT_MAX_LOG2K; ++hi) {
      if ((elems >> hi) == 0) continue;        // no instance that large fits the arena
      if (slot >= uint32_t(kMaxMaps)) return SDFT_ERR_UNSUPPORTED;
      const uint32_t Q = hi - lo, lg = TB - CB - Q;
      const uint64_t dims[4] = {32, 1ull << (lo - CB), 1ull << Q, elems >> hi};
      const uint64_t strides[3] = {128, (1ull << lo) * es, (1ull << hi) * es};
      const uint32_t box[4] = {32, 1u << lg, 1u << Q, 1};
      sdft_status s = encode_map(&S.maps.maps[slot], S.d_arena, dims, strides, box);
      if (s != SDFT_OK) return s;
      q_set_limits(S.maps, slot, dims);
      S.later_slot[lo][hi] = slot++;
    }
  }
  return SDFT_OK;
}

// Item list for one micro-batch (instances in arrival order, one instance per
// level-0 tile, later levels held back by 4 x grid items as in batch.cu).
sdft_status build_items(Server& S, Slot& sl, size_t& n_items, uint32_t& n_ctr) {
  const uint32_t TB = tile_bits(S.prec), CB = row_bits(S.prec);
  const uint32_t NT = S.prec == SDFT_C64 ? 256 : 128;
  const uint64_t es = uint64_t(elem_bytes(S.prec));
  const uint64_t lag = 4ull * uint64_t(S.grid);
  const size_t n = sl.reqs.size();
  for (size_t i = 0; i < n; ++i) {
    const Plan& p = *sl.reqs[i].plan;
    QInst& q = sl.h_insts[i];
    q.tw = sl.reqs[i].tw;
    q.off = sl.reqs[i].off / es;
    q.s = p.s;
    q.pad = 0;
    q.scale = std::ldexp(1.0, int(p.M) - int(p.s));
  }
  n_items = 0;
  n_ctr = 0;
  struct Group {
    uint64_t ready;
    size_t inst, level;
    uint32_t dep, need;
  };
  std::deque<Group> pending;
  auto push = [&](const QItem& it) -> sdft_status {
    if (n_items >= sl.cap_items) return SDFT_ERR_UNSUPPORTED;
    sl.h_items[n_items++] = it;
    return SDFT_OK;
  };
  std::function<sdft_status(const Group&)> emit_group;
  auto drain_ready = [&]() -> sdft_status {
    while (!pending.empty() && pending.front().ready <= n_items) {
      Group g = pending.front();
      pending.pop_front();
      sdft_status s = emit_group(g);
      if (s != SDFT_OK) return s;
    }
    return SDFT_OK;
  };
  emit_group = [&](const Group& g) -> sdft_status {
    const Plan& p = *sl.reqs[g.inst].plan;
    const Level& L = p.levels[g.level];
    const uint32_t slot = S.later_slot[L.lo][L.hi];
    if (slot == 0xffffffffu) return SDFT_ERR_UNSUPPORTED;
    const bool more = g.level + 1 < p.levels.size();
    const uint32_t sig = more ? n_ctr++ : kNone;
    const uint64_t z0 = sl.h_insts[g.inst].off >> L.hi, zs = 1ull << (p.s - L.hi);
    uint32_t cnt = 0;
    for (uint64_t gb = 0; gb < L.n_gb; ++gb)
      for (uint64_t z = 0; z < zs; ++z) {
        QItem it{};
        it.variant = uint16_t(q_variant_later(int(L.hi - L.lo), L.last));
        it.map = uint16_t(slot);
        it.count = 1;
        it.inst = uint32_t(g.inst);
        it.dep = g.dep;
        it.need = g.need;
        it.sig = sig;
        it.c1 = int32_t(gb << L.lg);
        it.c3 = int32_t(z0 + z);
        it.tw = static_cast<const char*>(sl.reqs[g.inst].tw) + (L.tw_off + gb * L.tw_len) * es -
                (size_t(1) << L.plo) * es;
        it.scale = sl.h_insts[g.inst].scale;
        sdft_status s = push(it);
        if (s != SDFT_OK) return s;
        ++cnt;
      }
    if (more) pending.push_back(Group{n_items + lag, g.inst, g.level + 1, sig, cnt});
    return SDFT_OK;
  };
  auto emit = [&](const QItem& it) -> sdft_status {
    sdft_status s = push(it);
    return s != SDFT_OK ? s : drain_ready();
  };

  size_t i = 0;
  while (i < n) {
    const Plan& p = *sl.reqs[i].plan;
    if (p.s <= kSmallMax) {
      size_t cnt = 0;
      while (i + cnt < n && sl.reqs[i + cnt].plan->s <= kSmallMax && cnt < NT) ++cnt;
      QItem it{};
      it.variant = uint16_t(kVSmall);
      it.count = uint32_t(cnt);
      it.inst = uint32_t(i);
      it.dep = kNone;
      it.sig = kNone;
      sdft_status s = emit(it);
      if (s != SDFT_OK) return s;
      i += cnt;
      continue;
    }
    const uint64_t row0 = sl.h_insts[i].off >> CB;
    if (p.s <= TB) {
      QItem it{};
      it.variant = uint16_t(q_variant_first(int(p.s)));
      it.map = uint16_t(2 * (p.s - CB));
      it.count = 1;
      it.inst = uint32_t(i);
      it.dep = kNone;
      it.sig = kNone;
      it.c1 = int32_t(row0);
      it.tw = sl.h_insts[i].tw;
      it.scale = sl.h_insts[i].scale;
      sdft_status s = emit(it);
      if (s != SDFT_OK) return s;
    } else {
      const uint64_t chunks = 1ull << (p.s - TB);
      const uint32_t sig = n_ctr++;
      for (uint64_t ch = 0; ch < chunks; ++ch) {
        QItem it{};
        it.variant = uint16_t(kVFirstChunk);
        it.map = uint16_t(2 * (TB - CB));
        it.count = 1;
        it.inst = uint32_t(i);
        it.dep = kNone;
        it.sig = sig;
        it.c1 = int32_t(row0 + (ch << (TB - CB)));
        it.tw = sl.h_insts[i].tw;
        it.scale = sl.h_insts[i].scale;
        sdft_status s = emit(it);
        if (s != SDFT_OK) return s;
      }
      pending.push_back(Group{n_items + lag, i, 1, sig, uint32_t(chunks)});
    }
    ++i;
  }
  while (!pending.empty()) {
    QItem nop{};
    nop.variant = uint16_t(kVNop);
    nop.dep = kNone;
    nop.sig = kNone;
    sdft_status s = emit(nop);
    if (s != SDFT_OK) return s;
  }
  return n_ctr <= sl.cap_ctr ? SDFT_OK : SDFT_ERR_UNSUPPORTED;
}

sdft_status launch_slot(Server& S, Slot& sl) {
  const uint64_t es = uint64_t(elem_bytes(S.prec));
  size_t n_items = 0;
  uint32_t n_ctr = 0;
  sdft_status s = build_items(S, sl, n_items, n_ctr);
  if (s != SDFT_OK) return s;
  cudaError_t e = cudaSuccess;
  for (const Req& r : sl.reqs) {
    if (r.own_tw) {   // a deferred plan's tables go into the arena with its request
      e = cudaMemcpyAsync(S.d_arena + r.tw_off, r.plan->host_tables.data(), r.plan->host_tables.size(),
                          cudaMemcpyHostToDevice, sl.stream);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    e = cudaMemcpyAsync(S.d_arena + r.off, r.h_in, r.plan->k * es, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  e = cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(QItem) * n_items, cudaMemcpyHostToDevice, sl.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_insts, sl.h_insts, sizeof(QInst) * sl.reqs.size(), cudaMemcpyHostToDevice, sl.stream);
  if (e == cudaSuccess && n_ctr) e = cudaMemsetAsync(sl.d_counters, 0, sizeof(uint32_t) * n_ctr, sl.stream);
  if (e != cudaSuccess) return cuda_fail(e);
  QParams prm = S.maps;
  prm.a.items = sl.d_items;
  prm.a.n_items = n_items;
  prm.a.insts = sl.d_insts;
  prm.a.counters = sl.d_counters;
  prm.a.in = S.d_arena;
  prm.a.out = S.d_arena;
  prm.a.status = S.d_status;
  prm.a.timeout_ns = wait_timeout_ns();
  prm.a.need_bias = 0;
  prm.a.n_counters = n_ctr;
  prm.a.n_insts = sl.reqs.size();
  prm.a.total = S.budget / es;
  const int grid = int(std::min<uint64_t>(uint64_t(S.grid), n_items));
  s = S.prec == SDFT_C64 ? launch_queue_f32(prm, grid, 4, false, sl.stream)
                          : launch_queue_f64(prm, grid, 4, false, sl.stream);
  if (s != SDFT_OK) return s;
  for (const Req& r : sl.reqs) {
    e = cudaMemcpyAsync(r.h_out, S.d_arena + r.off, r.plan->k * es, cudaMemcpyDeviceToHost, sl.stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  sl.done.store(false, std::memory_order_relaxed);
  e = cudaLaunchHostFunc(sl.stream, on_slot_done, &sl);
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

uint32_t block_order(const Server& S, const Plan& p) {
  const uint64_t bytes = std::max<uint64_t>(p.k * uint64_t(elem_bytes(S.prec)), 128);
  return uint32_t(63 - __builtin_clzll(bytes));
}

void worker_loop(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progressed = false;
    // Reap finished slots. Finished fresh plans are destroyed after the lock is
    // released (freeing their host tables takes time the submitters should not
    // wait for).
    std::vector<sdft_plan> finished;
    for (Slot* sl : S->slots) {
      if (!sl->busy || !sl->done.load(std::memory_order_acquire)) continue;
      for (const Req& r : sl->reqs) {
        S->buddy.release(r.off, r.order);
        if (r.own_tw) S->buddy.release(r.tw_off, r.tw_order);
        const double lat = std::chrono::duration<double>(sl->t_done - r.t_submit).count();
        S->done.push_back(Done{r.tag, lat, int32_t(SDFT_OK)});
        ++S->stats.completed;
        S->stats.coeffs += r.plan->k;
        if (r.own_plan) finished.push_back(r.own_plan);   // host tables only: no device work
      }
      S->stats.inflight -= sl->reqs.size();
      sl->reqs.clear();
      sl->busy = false;
      progressed = true;
    }
    if (!finished.empty()) {
      lk.unlock();
      for (sdft_plan h : finished) sdft_plan_destroy(h);
      lk.lock();
    }
    if (S->stop && S->waiting.empty() && S->planning == 0) {
      bool idle = true;
      for (Slot* sl : S->slots) idle = idle && !sl->busy;
      if (idle) break;
    }
    // Admit a micro-batch into a free slot.
    Slot* free_slot = nullptr;
    for (Slot* sl : S->slots)
      if (!sl->busy) {
        free_slot = sl;
        break;
      }
    if (free_slot && !S->waiting.empty()) {
      std::vector<Req>& batch = free_slot->reqs;
      while (!S->waiting.empty() && batch.size() < S->max_batch) {
        if (S->inj_mode && S->inj_every && !S->waiting.front().inj_seen) {
          Req& fr = S->waiting.front();
          fr.inj_seen = true;
          if (++S->inj_count % S->inj_every == 0) {
            ++S->stats.injected;
            if (S->inj_mode == SDFT_INJECT_DROP || S->inj_mode == SDFT_INJECT_FAIL) {
              if (S->inj_mode == SDFT_INJECT_FAIL) {   // completes at once, as if its launch had failed
                S->done.push_back(Done{fr.tag, 0.0, int32_t(SDFT_ERR_CUDA)});
                ++S->stats.failed;
              }                                        // a dropped request never completes
              if (fr.own_plan) sdft_plan_destroy(fr.own_plan);
              S->waiting.pop_front();
              progressed = true;
              continue;
            }
            // delay: the worker holds this request back (only the worker pops
            // the queue, so it is still at the front afterwards)
            const uint64_t us = S->inj_delay_us;
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(us));
            lk.lock();
          }
        }
        Req r = S->waiting.front();
        r.order = block_order(*S, *r.plan);
        const uint64_t tw_bytes = r.plan->deferred ? std::max<uint64_t>(r.plan->host_tables.size(), 128) : 0;
        r.tw_order = tw_bytes ? uint32_t(64 - __builtin_clzll(tw_bytes - 1)) : 0;
        if ((1ull << r.order) + (tw_bytes ? (1ull << r.tw_order) : 0) > S->budget) {   // can never fit
          S->waiting.pop_front();
          S->done.push_back(Done{r.tag, 0.0, int32_t(SDFT_ERR_BUDGET)});
          ++S->stats.failed;
          if (r.own_plan) sdft_plan_destroy(r.own_plan);
          progressed = true;
          continue;
        }
        const uint64_t off = S->buddy.alloc(r.order);
        if (off == ~0ull) break;                        // wait for memory to free up
        if (tw_bytes) {
          const uint64_t toff = S->buddy.alloc(r.tw_order);
          if (toff == ~0ull) {
            S->buddy.release(off, r.order);
            break;
          }
          r.tw_off = toff;
          r.tw = S->d_arena + toff;
          r.own_tw = true;
        } else {
          r.tw = r.plan->d_tw;
        }
        r.off = off;
        S->waiting.pop_front();
        batch.push_back(r);
      }
      if (!batch.empty()) {
        free_slot->busy = true;
        S->stats.inflight += batch.size();
        S->stats.max_inflight = std::max(S->stats.max_inflight, S->stats.inflight);
        S->stats.arena_peak_bytes = S->buddy.peak();
        ++S->stats.micro_batches;
        lk.unlock();
        const sdft_status st = launch_slot(*S, *free_slot);
        lk.lock();
        if (st != SDFT_OK) {
          // The launch was refused: fail its requests (nothing of it runs).
          cudaStreamSynchronize(free_slot->stream);
          for (const Req& r : free_slot->reqs) {
            S->buddy.release(r.off, r.order);
            if (r.own_tw) S->buddy.release(r.tw_off, r.tw_order);
            S->done.push_back(Done{r.tag, 0.0, int32_t(st)});
            ++S->stats.failed;
            if (r.own_plan) sdft_plan_destroy(r.own_plan);
          }
          S->stats.inflight -= free_slot->reqs.size();
          free_slot->reqs.clear();
          free_slot->busy = false;
          S->worker_error = st;
        }
        progressed = true;
      }
    }
    if (!progressed) S->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

// Planner thread: plan queued supports (deferred plans), then queue the
// request for admission; a support that fails validation completes at once
// with its plan-creation status.
void planner_loop(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    while (!S->stop && S->plan_jobs.empty()) S->plan_cv.wait(lk);
    if (S->plan_jobs.empty()) break;     // stopping, nothing left to plan
    PlanJob job = std::move(S->plan_jobs.front());
    S->plan_jobs.pop_front();
    lk.unlock();
    sdft_plan h = nullptr;
    const sdft_status st = sdft_plan_create(job.M, job.J.data(), job.J.size(), S->prec, SDFT_PLAN_DEFER_DEVICE, &h);
    lk.lock();
    --S->planning;
    if (st != SDFT_OK) {
      const double lat = std::chrono::duration<double>(Clock::now() - job.t_submit).count();
      S->done.push_back(Done{job.tag, lat, int32_t(st)});
      ++S->stats.failed;
      continue;
    }
    Req r;
    r.tag = job.tag;
    r.plan = &h->p;
    r.h_in = job.h_in;
    r.h_out = job.h_out;
    r.t_submit = job.t_submit;
    r.own_plan = h;
    S->waiting.push_back(r);
    ++S->stats.planned;
    S->cv.notify_one();
  }
}

void free_server(Server* S) {
  for (Slot* sl : S->slots) {
    if (sl->stream) cudaStreamDestroy(sl->stream);
    if (sl->d_items) cudaFree(sl->d_items);
    if (sl->d_insts) cudaFree(sl->d_insts);
    if (sl->d_counters) cudaFree(sl->d_counters);
    if (sl->h_items) cudaFreeHost(sl->h_items);
    if (sl->h_insts) cudaFreeHost(sl->h_insts);
    delete sl;
  }
  S->slots.clear();
  if (S->d_arena) cudaFree(S->d_arena);
  if (S->d_status) cudaFree(S->d_status);
}

}  // namespace
}  // namespace sdft

struct sdft_server_s {
  sdft::Server s;
};

extern "C" {

sdft_status sdft_server_create(sdft_prec prec, uint64_t budget_bytes, uint32_t n_slots, uint32_t max_batch,
                               uint32_t n_planners, sdft_server* out) {
  using namespace sdft;
  if (!out) return SDFT_ERR_ARG;
  *out = nullptr;
  if ((prec != SDFT_C64 && prec != SDFT_C128) || n_slots == 0 || n_slots > 16 || max_batch == 0 ||
      budget_bytes < 4096 || n_planners > 64)
    return SDFT_ERR_ARG;
  sdft_server_s* h = new (std::nothrow) sdft_server_s();
  if (!h) return SDFT_ERR_NOMEM;
  Server& S = h->s;
  S.prec = prec;
  S.max_batch = max_batch;
  cudaError_t e = cudaGetDevice(&S.device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e);
  }
  // Arena: the largest power of two not above the budget.
  const uint32_t top = uint32_t(63 - __builtin_clzll(budget_bytes));
  S.budget = 1ull << top;
  S.buddy.init(7, top);
  const int total = prec == SDFT_C64 ? queue_grid_f32(4, false) : queue_grid_f64(4, false);
  S.grid = total / int(n_slots);      // in-flight launches together fit the co-resident CTAs
  sdft_status st = S.grid > 0 ? SDFT_OK : SDFT_ERR_CUDA;
  if (st == SDFT_OK) {
    e = cudaMalloc(&S.d_arena, S.budget);
    if (e == cudaSuccess) e = cudaMalloc(&S.d_status, 256);
    if (e == cudaSuccess) e = cudaMemset(S.d_status, 0, 256);
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : cuda_fail(e);
  }
  if (st == SDFT_OK) st = init_maps(S);
  // Items per slot: every request may add level-0 tiles, later-level tiles and the
  // lag padding once.
  const size_t cap_items = size_t(max_batch) * 160 + 4 * size_t(S.grid) + 64;
  for (uint32_t i = 0; i < n_slots && st == SDFT_OK; ++i) {
    Slot* sl = new (std::nothrow) Slot();
    if (!sl) {
      st = SDFT_ERR_NOMEM;
      break;
    }
    S.slots.push_back(sl);
    sl->cv = &S.cv;
    sl->cap_items = cap_items;
    sl->cap_insts = max_batch;
    sl->cap_ctr = size_t(max_batch) * 3;
    e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sl->d_items, sizeof(QItem) * sl->cap_items);
    if (e == cudaSuccess) e = cudaMalloc(&sl->d_insts, sizeof(QInst) * sl->cap_insts);
    if (e == cudaSuccess) e = cudaMalloc(&sl->d_counters, sizeof(uint32_t) * sl->cap_ctr);
    if (e == cudaSuccess) e = cudaMallocHost(&sl->h_items, sizeof(QItem) * sl->cap_items);
    if (e == cudaSuccess) e = cudaMallocHost(&sl->h_insts, sizeof(QInst) * sl->cap_insts);
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : cuda_fail(e);
  }
  if (st != SDFT_OK) {
    free_server(&S);
    delete h;
    return st;
  }
  S.stats.arena_bytes = S.budget;
  try {
    S.worker = std::thread(worker_loop, &S);
    for (uint32_t i = 0; i < n_planners; ++i) S.planners.emplace_back(planner_loop, &S);
  } catch (const std::system_error&) {   // no thread: stop the ones started, as destroy does
    {
      std::lock_guard<std::mutex> lk(S.mu);
      S.stop = true;
    }
    S.plan_cv.notify_all();
    for (std::thread& t : S.planners)
      if (t.joinable()) t.join();
    S.cv.notify_one();
    if (S.worker.joinable()) S.worker.join();
    free_server(&S);
    delete h;
    return SDFT_ERR_NOMEM;
  }
  *out = h;
  return SDFT_OK;
}

sdft_status sdft_server_submit(sdft_server srv, sdft_plan plan, const void* h_samples, void* h_coeffs,
                               uint64_t tag) {
  using namespace sdft;
  if (!srv || !plan || !h_samples || !h_coeffs) return SDFT_ERR_ARG;
  Server& S = srv->s;
  if (plan->p.device != S.device) return SDFT_ERR_NO_DEVICE;
  if (!plan->p.deferred && !plan->p.d_status) return SDFT_ERR_NO_DEVICE;
  if (plan->p.prec != S.prec) return SDFT_ERR_PRECISION;
  Req r;
  r.tag = tag;
  r.plan = &plan->p;
  r.h_in = h_samples;
  r.h_out = h_coeffs;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stop) return SDFT_ERR_ARG;
    S.waiting.push_back(r);
    ++S.stats.submitted;
  }
  S.cv.notify_one();
  return SDFT_OK;
}

sdft_status sdft_server_submit_support(sdft_server srv, uint32_t log2N, const uint64_t* J, uint64_t k,
                                       const void* h_samples, void* h_coeffs, uint64_t tag) {
  using namespace sdft;
  if (!srv || !J || !h_samples || !h_coeffs || k == 0 || k > (1ull << SDFT_MAX_LOG2K)) return SDFT_ERR_ARG;
  Server& S = srv->s;
  PlanJob job;
  job.tag = tag;
  job.M = log2N;
  job.h_in = h_samples;
  job.h_out = h_coeffs;
  job.t_submit = Clock::now();
  try {
    job.J.assign(J, J + k);
  } catch (const std::bad_alloc&) {
    return SDFT_ERR_NOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stop) return SDFT_ERR_ARG;
    if (S.planners.empty()) return SDFT_ERR_UNSUPPORTED;
    S.plan_jobs.push_back(std::move(job));
    ++S.planning;
    ++S.stats.submitted;
  }
  S.plan_cv.notify_one();
  return SDFT_OK;
}

sdft_status sdft_server_poll(sdft_server srv, uint64_t* tags, double* latency_s, int32_t* status, uint64_t cap,
                             uint64_t* n_out) {
  if (!srv || !n_out || (cap && (!tags || !latency_s || !status))) return SDFT_ERR_ARG;
  sdft::Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  const uint64_t n = std::min<uint64_t>(cap, S.done.size());
  for (uint64_t i = 0; i < n; ++i) {
    tags[i] = S.done[i].tag;
    latency_s[i] = S.done[i].latency;
    status[i] = S.done[i].status;
  }
  S.done.erase(S.done.begin(), S.done.begin() + long(n));
  *n_out = n;
  return S.worker_error;
}

sdft_status sdft_server_drain(sdft_server srv, uint64_t timeout_ms) {
  if (!srv) return SDFT_ERR_ARG;
  sdft::Server& S = srv->s;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(S.mu);
      if (S.waiting.empty() && S.stats.inflight == 0 && S.planning == 0) return S.worker_error;
    }
    if (timeout_ms && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return SDFT_ERR_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

sdft_status sdft_server_inject(sdft_server srv, uint32_t mode, uint64_t every, uint64_t delay_us) {
  if (!srv) return SDFT_ERR_ARG;
  if (mode > SDFT_INJECT_DELAY || (mode != SDFT_INJECT_OFF && every == 0)) return SDFT_ERR_ARG;
  if (delay_us > 10000000ull) return SDFT_ERR_ARG;
  sdft::Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  S.inj_mode = mode;
  S.inj_every = every;
  S.inj_delay_us = delay_us;
  S.inj_count = 0;
  return SDFT_OK;
}

sdft_status sdft_server_get_stats(sdft_server srv, sdft_server_stats* st) {
  if (!srv || !st) return SDFT_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->s.mu);
  *st = srv->s.stats;
  st->arena_peak_bytes = srv->s.buddy.peak();
  return SDFT_OK;
}

sdft_status sdft_server_device_status(sdft_server srv, int clear) {
  if (!srv) return SDFT_ERR_ARG;
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, srv->s.d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(srv->s.d_status, 0, sizeof(int));
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  return sdft_status(v);
}

sdft_status sdft_server_destroy(sdft_server srv) {
  if (!srv) return SDFT_ERR_ARG;
  sdft::Server& S = srv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.plan_cv.notify_all();
  for (std::thread& t : S.planners)
    if (t.joinable()) t.join();
  S.cv.notify_one();
  if (S.worker.joinable()) S.worker.join();
  cudaDeviceSynchronize();
  sdft::free_server(&S);
  delete srv;
  return SDFT_OK;
}

}  // extern "C"
