// Uneven batches: many instances with their own plans in one persistent,
// cooperatively launched work-queue kernel (queue.cuh).
//
// Packing: instances are laid out by decreasing k, so every offset is a
// multiple of its own k (a prefix sum of larger or equal powers of two). One
// 2-D tensor map per power-of-two box height then covers every level-0 tile of
// the packed buffers, and one 4-D map per (lo, hi) covers every later-level tile.
//
// Item list: level-0 tiles instance by instance (whole same-size instances
// grouped into power-of-two tiles); an instance's next-level tiles are held back
// until at least 4 G items (G = grid size) have been emitted after its previous
// level, then emitted together; no-op items pad the tail where fewer items
// remain. Consecutive items go to consecutive CTAs, so list order is roughly
// time order and the intermediate of a multi-level instance is read back from L2.
#include <algorithm>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "plan.hpp"
#include "queue.cuh"

namespace sdft {

struct BatchMap {
  bool first;          // level-0 2-D map (else later-level 4-D map)
  bool load;           // level 0: load map (box of 2^r rows on the samples) or store map (coefficients)
  uint32_t r;          // level 0: log2 rows of the box
  uint32_t lo, hi, lg; // later levels
};

// Grid size assumed when a batch is built from host-only plans (2 CTAs x 152 SMs).
constexpr int kHostOnlyGrid = 304;

// Distance, in list places per CTA, at which a dependent item follows the
// last item it waits on: at least 4 (the queue kernel's publication order,
// check_items); 6 by default, the fastest of 4, 6, 8 and 12 on the
// 10,000-instance uneven batch (0.4531, 0.4409, 0.4474 and 0.4641 ms): later
// items find their counters already published, and the intermediates they
// read are still in L2.
constexpr int kMinLag = 4, kDefaultLag = 6, kMaxLag = 64;

struct Batch {
  int device = -1;
  sdft_prec prec = SDFT_C64;
  uint64_t n = 0, total = 0;
  std::vector<uint64_t> offsets;     // user order, plus total
  std::vector<QItem> items;
  std::vector<BatchMap> maps;        // slot -> map description
  QItem* d_items = nullptr;
  QInst* d_insts = nullptr;
  uint32_t* d_counters = nullptr;
  uint64_t n_counters = 0;
  int* d_status = nullptr;
  int grid = 0;
  uint64_t timeout_ns = 0;           // 0: library default
  uint32_t need_bias = 0;            // diagnostics: added to every dependency target
  int* d_status_shared = nullptr;    // if set, report into this word instead of d_status
  std::vector<sdft_plan> plans;      // caller's order (the plans outlive the batch)
  int schedule = SDFT_SCHEDULE_AUTO; // item order (sdft_schedule)
  int grid_req = 0;                  // CTAs requested (0: every co-resident CTA)
  uint32_t* noalloc_counters = nullptr;  // device address of the library's fixed counter array
  int spp = 4;                       // stages per pass of the queue kernel (3 or 4; 3: complex64 only)
  bool staged = false;               // whole twiddle tables in shared memory (complex64 only)
  int lag = kDefaultLag;             // a dependent item sits at least lag x grid list places after its producers
};

}  // namespace sdft

struct sdft_batch_s {
  sdft::Batch b;
};

namespace sdft {
namespace {

void free_batch(Batch& b) {
  if (b.d_items) cudaFree(b.d_items);
  if (b.d_insts) cudaFree(b.d_insts);
  if (b.d_counters) cudaFree(b.d_counters);
  if (b.d_status) cudaFree(b.d_status);
  b.d_items = nullptr;
  b.d_insts = nullptr;
  b.d_counters = nullptr;
  b.d_status = nullptr;
}

int log2u(uint64_t x) { return 63 - __builtin_clzll(x); }

// Invariants of an item list: every dependency refers to a counter signalled
// only by items earlier in the list, reaches its target exactly, and its last
// producer sits at least 4 x grid positions back. A CTA publishes item j's
// counter at the end of item j+2 and before the dependency wait of item j+4,
// so then a CTA never waits on an item whose counter it has not yet
// published, and no two CTAs wait on each other.
sdft_status check_items(const Batch& B) {
  std::vector<uint64_t> sig_count(B.n_counters, 0), sig_last(B.n_counters, 0);
  const uint64_t lag = 4ull * uint64_t(B.grid);
  for (uint64_t p = 0; p < B.items.size(); ++p) {
    const QItem& it = B.items[p];
    if (it.dep != kNone) {
      if (it.dep >= B.n_counters) return SDFT_ERR_ARG;
      if (sig_count[it.dep] != it.need) return SDFT_ERR_ARG;     // all producers precede
      if (p < sig_last[it.dep] + lag) return SDFT_ERR_ARG;
    }
    if (it.sig != kNone) {
      if (it.sig >= B.n_counters) return SDFT_ERR_ARG;
      ++sig_count[it.sig];
      sig_last[it.sig] = p;
    }
  }
  return SDFT_OK;
}

}  // namespace

// Build the item list and device arrays of a batch (plans already validated).
static sdft_status build_batch(Batch& B, const sdft_plan* plans, uint64_t n) {
  const sdft_prec prec = plans[0]->p.prec;
  const uint32_t TB = tile_bits(prec), CB = row_bits(prec);
  const uint32_t NT = prec == SDFT_C64 ? 256 : 128;
  B.prec = prec;
  B.n = n;
  if (B.device >= 0) {
    B.grid = prec == SDFT_C64 ? queue_grid_f32(B.spp, B.staged) : queue_grid_f64(B.spp, B.staged);
    if (B.grid <= 0) return SDFT_ERR_CUDA;
    if (B.grid_req > 0 && B.grid_req < B.grid) B.grid = B.grid_req;
  } else {
    B.grid = kHostOnlyGrid;     // host-only batches: item list for inspection only
    if (B.grid_req > 0 && B.grid_req < B.grid) B.grid = B.grid_req;
  }

  // Pack by decreasing k (stable).
  std::vector<uint64_t> order(n);
  for (uint64_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](uint64_t a, uint64_t b) { return plans[a]->p.s > plans[b]->p.s; });
  B.offsets.assign(n + 1, 0);
  std::vector<QInst> insts(n);
  uint64_t off = 0;
  for (uint64_t q = 0; q < n; ++q) {
    const Plan& p = plans[order[q]]->p;
    B.offsets[order[q]] = off;
    insts[q].tw = p.d_tw;
    insts[q].off = off;
    insts[q].s = p.s;
    insts[q].pad = 0;
    insts[q].scale = std::ldexp(1.0, int(p.M) - int(p.s));
    off += p.k;
  }
  B.total = off;
  B.offsets[n] = off;

  // Map slots: level-0 load/store pairs at 2r, 2r+1 (r = 0..8); later levels after.
  B.maps.assign(18, BatchMap{});
  for (uint32_t r = 0; r <= 8; ++r) {
    B.maps[2 * r] = BatchMap{true, true, r, 0, 0, 0};
    B.maps[2 * r + 1] = BatchMap{true, false, r, 0, 0, 0};
  }
  std::map<std::pair<uint32_t, uint32_t>, uint32_t> later_slot;
  auto slot_for = [&](const Level& L) -> int {
    auto key = std::make_pair(L.lo, L.hi);
    auto it = later_slot.find(key);
    if (it != later_slot.end()) return int(it->second);
    if (B.maps.size() >= size_t(kMaxMaps)) return -1;
    const uint32_t slot = uint32_t(B.maps.size());
    B.maps.push_back(BatchMap{false, false, 0, L.lo, L.hi, L.lg});
    later_slot[key] = slot;
    return int(slot);
  };

  // Phase 1: units of work. A unit is one instance's levels (stage 0 = its
  // level-0 chunks, stage j = its level-j tiles, each stage waiting on the
  // previous one's counter), a tile of whole same-size instances, or a range of
  // k <= 16 instances. cost = coefficients touched.
  struct Unit {
    std::vector<std::vector<QItem>> stages;
    uint64_t cost = 0;
  };
  std::vector<Unit> units;
  uint32_t n_ctr = 0;
  const size_t es = size_t(elem_bytes(prec));
  auto later_stage = [&](uint64_t q, size_t level, uint32_t dep, uint32_t need, std::vector<QItem>& out,
                         uint32_t& sig_out) -> sdft_status {
    const Plan& p = plans[order[q]]->p;
    const Level& L = p.levels[level];
    const int slot = slot_for(L);
    if (slot < 0) return SDFT_ERR_UNSUPPORTED;
    const uint64_t zs = 1ull << (p.s - L.hi);       // z rows of this instance
    const uint64_t z0 = insts[q].off >> L.hi;
    if (z0 + zs > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
    const bool more = level + 1 < p.levels.size();
    sig_out = more ? n_ctr++ : kNone;
    for (uint64_t gb = 0; gb < L.n_gb; ++gb)
      for (uint64_t z = 0; z < zs; ++z) {
        QItem it{};
        it.variant = uint16_t(q_variant_later(int(L.hi - L.lo), L.last));
        it.map = uint16_t(slot);
        it.count = 1;
        it.inst = uint32_t(q);
        it.dep = dep;
        it.need = need;
        it.sig = sig_out;
        it.c1 = int32_t(gb << L.lg);
        it.c3 = int32_t(z0 + z);
        it.tw = static_cast<const char*>(p.d_tw) + (L.tw_off + gb * L.tw_len) * es - (size_t(1) << L.plo) * es;
        it.scale = insts[q].scale;
        out.push_back(it);
      }
    return SDFT_OK;
  };

  uint64_t q = 0;
  while (q < n) {
    const uint32_t s = insts[q].s;
    if (s <= kSmallMax) {                       // one thread per instance
      uint64_t cnt = 0, cost = 0;
      while (q + cnt < n && insts[q + cnt].s <= kSmallMax && cnt < NT) cost += 1ull << insts[q + cnt++].s;
      QItem it{};
      it.variant = uint16_t(kVSmall);
      it.count = uint32_t(cnt);
      it.inst = uint32_t(q);
      it.dep = kNone;
      it.sig = kNone;
      units.push_back(Unit{{{it}}, cost});
      q += cnt;
    } else if (s <= TB) {                       // whole instances per tile
      uint64_t run = 0;
      while (q + run < n && insts[q + run].s == s) ++run;
      const uint64_t G = 1ull << (TB - s);
      uint64_t left = run;
      while (left) {
        const uint64_t cnt = 1ull << log2u(std::min(G, left));
        const uint64_t rows = cnt << (s - CB);
        const uint64_t row0 = insts[q].off >> CB;
        if (row0 + rows > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
        QItem it{};
        it.variant = uint16_t(q_variant_first(int(s)));
        it.map = uint16_t(2 * log2u(rows));
        it.count = uint32_t(cnt);
        it.inst = uint32_t(q);
        it.dep = kNone;
        it.sig = kNone;
        it.c1 = int32_t(row0);
        it.c3 = 0;
        it.tw = insts[q].tw;
        it.scale = insts[q].scale;
        units.push_back(Unit{{{it}}, cnt << s});
        q += cnt;
        left -= cnt;
      }
    } else {                                    // 2^TB chunks, then later levels
      const Plan& p = plans[order[q]]->p;
      const uint64_t chunks = 1ull << (s - TB);
      const uint32_t sig = n_ctr++;
      const uint64_t row0 = insts[q].off >> CB;
      if (row0 + (chunks << (TB - CB)) > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
      Unit u;
      u.stages.emplace_back();
      for (uint64_t ch = 0; ch < chunks; ++ch) {
        QItem it{};
        it.variant = uint16_t(kVFirstChunk);
        it.map = uint16_t(2 * (TB - CB));
        it.count = 1;
        it.inst = uint32_t(q);
        it.dep = kNone;
        it.sig = sig;
        it.c1 = int32_t(row0 + (ch << (TB - CB)));
        it.c3 = 0;
        it.tw = insts[q].tw;
        it.scale = insts[q].scale;
        u.stages[0].push_back(it);
      }
      uint32_t dep = sig, need = uint32_t(chunks);
      for (size_t level = 1; level < p.levels.size(); ++level) {
        u.stages.emplace_back();
        uint32_t next = kNone;
        sdft_status st = later_stage(q, level, dep, need, u.stages.back(), next);
        if (st != SDFT_OK) return st;
        need = uint32_t(u.stages.back().size());
        dep = next;
      }
      for (const auto& st : u.stages) u.cost += uint64_t(st.size()) << TB;
      units.push_back(std::move(u));
      ++q;
    }
  }
  B.n_counters = n_ctr;

  // Phase 2: order the items. Every dependency must sit at least 4 x grid list
  // positions behind the item that waits on it (CTA c takes positions c, c + G,
  // ...; a CTA issues item j's load after publishing item j - 4's store); the
  // orders place it lag x grid positions behind (lag >= 4).
  QItem nop{};
  nop.variant = uint16_t(kVNop);
  nop.dep = kNone;
  nop.sig = kNone;
  std::vector<QItem>& items = B.items;
  items.clear();
  items.clear();
  const uint64_t G = uint64_t(B.grid);
  struct Pending {
    uint64_t ready;
    size_t unit, stage;
  };
  // Round robin by default (measured faster on the uneven workload once tile
  // loads moved to a producer warp); lanes on request. Both satisfy the invariant.
  const bool use_lanes = B.schedule == SDFT_SCHEDULE_LANES;
  if (use_lanes) {
    // Lanes: a unit runs entirely in one CTA (its tables stay in registers and
    // L1, its intermediate in L2); units go to the least-loaded lane, largest
    // first, and a unit's next stage starts lag lane positions after its last item.
    std::vector<size_t> by_cost(units.size());
    for (size_t u = 0; u < units.size(); ++u) by_cost[u] = u;
    std::stable_sort(by_cost.begin(), by_cost.end(),
                     [&](size_t a, size_t b) { return units[a].cost > units[b].cost; });
    std::vector<std::vector<size_t>> lane_units(G);
    std::vector<std::pair<uint64_t, uint64_t>> heap;   // (load, lane), min-heap
    for (uint64_t l = 0; l < G; ++l) heap.push_back({0, l});
    auto cmp = [](const std::pair<uint64_t, uint64_t>& a, const std::pair<uint64_t, uint64_t>& b) {
      return a > b;
    };
    for (size_t u : by_cost) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto& top = heap.back();
      lane_units[top.second].push_back(u);
      top.first += units[u].cost;
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
    std::vector<std::vector<QItem>> lanes(G);
    size_t longest = 0;
    for (uint64_t l = 0; l < G; ++l) {
      std::vector<QItem>& lane = lanes[l];
      std::deque<Pending> pend;
      std::function<void(const QItem&)> put = [&](const QItem& it) {
        lane.push_back(it);
        while (!pend.empty() && pend.front().ready <= lane.size()) {
          const Pending pd = pend.front();
          pend.pop_front();
          const auto& st = units[pd.unit].stages[pd.stage];
          for (const QItem& x : st) lane.push_back(x);
          if (pd.stage + 1 < units[pd.unit].stages.size())
            pend.push_back(Pending{lane.size() + uint64_t(B.lag) - 1, pd.unit, pd.stage + 1});
        }
      };
      for (size_t u : lane_units[l]) {
        for (const QItem& it : units[u].stages[0]) put(it);
        if (units[u].stages.size() > 1) pend.push_back(Pending{lane.size() + uint64_t(B.lag) - 1, u, 1});
      }
      while (!pend.empty()) put(nop);
      longest = std::max(longest, lane.size());
    }
    items.resize(longest * G, nop);
    for (uint64_t l = 0; l < G; ++l)
      for (size_t idx = 0; idx < lanes[l].size(); ++idx) items[idx * G + l] = lanes[l][idx];
    while (!items.empty() && items.back().variant == kVNop) items.pop_back();
  } else {
    // Round robin in unit order: a unit's next stage is held back until lag x
    // grid more items exist (consecutive items go to consecutive CTAs).
    const uint64_t lag = uint64_t(B.lag) * G;
    std::deque<Pending> pend;
    std::function<void(const QItem&)> put = [&](const QItem& it) {
      items.push_back(it);
      while (!pend.empty() && pend.front().ready <= items.size()) {
        const Pending pd = pend.front();
        pend.pop_front();
        for (const QItem& x : units[pd.unit].stages[pd.stage]) items.push_back(x);
        if (pd.stage + 1 < units[pd.unit].stages.size())
          pend.push_back(Pending{items.size() + lag, pd.unit, pd.stage + 1});
      }
    };
    for (size_t u = 0; u < units.size(); ++u) {
      for (const QItem& it : units[u].stages[0]) put(it);
      if (units[u].stages.size() > 1) pend.push_back(Pending{items.size() + lag, u, 1});
    }
    while (!pend.empty()) put(nop);
  }
  if (B.device < 0) return SDFT_OK;

  // Device arrays.
  cudaError_t e = cudaMalloc(&B.d_status, 256);
  if (e == cudaSuccess) e = cudaMemset(B.d_status, 0, 256);
  if (e == cudaSuccess) e = cudaMalloc(&B.d_items, sizeof(QItem) * std::max<size_t>(items.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc(&B.d_insts, sizeof(QInst) * std::max<uint64_t>(n, 1));
  if (e == cudaSuccess) e = cudaMalloc(&B.d_counters, sizeof(uint32_t) * std::max<uint64_t>(n_ctr, 1));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(B.d_items, items.data(), sizeof(QItem) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B.d_insts, insts.data(), sizeof(QInst) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : cuda_fail(e);
  return SDFT_OK;
}

// Encode the batch's tensor maps over (in, out) into the kernel parameters.
static sdft_status encode_batch_maps(const Batch& B, const void* in, void* out, QParams& prm) {
  const uint32_t CB = row_bits(B.prec);
  const uint64_t es = uint64_t(elem_bytes(B.prec));
  const uint64_t rows = B.total >> CB;
  for (size_t slot = 0; slot < B.maps.size(); ++slot) {
    const BatchMap& m = B.maps[slot];
    std::memset(&prm.maps[slot], 0, sizeof(CUtensorMap));
    if (m.first) {
      if (rows < (1ull << m.r)) continue;       // never used: no tile of that height fits
      const uint64_t dims[4] = {32, rows, 1, 1};
      const uint64_t strides[3] = {128, rows * 128, rows * 128};
      const uint32_t box[4] = {32, 1u << m.r, 1, 1};
      sdft_status s = encode_map(&prm.maps[slot], m.load ? in : out, dims, strides, box);
      if (s != SDFT_OK) return s;
      q_set_limits(prm, slot, dims);
    } else {
      const uint32_t Q = m.hi - m.lo;
      const uint64_t zs = B.total >> m.hi;
      const uint64_t dims[4] = {32, 1ull << (m.lo - CB), 1ull << Q, zs};
      const uint64_t strides[3] = {128, (1ull << m.lo) * es, (1ull << m.hi) * es};
      const uint32_t box[4] = {32, 1u << m.lg, 1u << Q, 1};
      sdft_status s = encode_map(&prm.maps[slot], out, dims, strides, box);
      if (s != SDFT_OK) return s;
      q_set_limits(prm, slot, dims);
    }
  }
  prm.a.n_counters = uint32_t(B.n_counters);
  prm.a.n_insts = B.n;
  prm.a.total = B.total;
  return SDFT_OK;
}

static sdft_status run_batch(Batch& B, const void* in, void* out, cudaStream_t st) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev != B.device) return SDFT_ERR_ARG;
  if (!in || !out) return SDFT_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return SDFT_ERR_ARG;
  const uint64_t bytes = B.total * uint64_t(elem_bytes(B.prec));
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
  if (a != b && a < b + bytes && b < a + bytes) return SDFT_ERR_ARG;
  if (B.items.empty()) return SDFT_OK;
  QParams prm;
  std::memset(&prm, 0, sizeof(prm));
  sdft_status s = encode_batch_maps(B, in, out, prm);
  if (s != SDFT_OK) return s;
  prm.a.items = B.d_items;
  prm.a.n_items = B.items.size();
  prm.a.insts = B.d_insts;
  prm.a.counters = B.d_counters;
  prm.a.in = in;
  prm.a.out = out;
  prm.a.status = B.d_status_shared ? B.d_status_shared : B.d_status;
  prm.a.timeout_ns = B.timeout_ns ? B.timeout_ns : wait_timeout_ns();
  prm.a.need_bias = B.need_bias;
  if (B.n_counters) {
    e = cudaMemsetAsync(B.d_counters, 0, sizeof(uint32_t) * B.n_counters, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const int grid = int(std::min<uint64_t>(uint64_t(B.grid), B.items.size()));
  return B.prec == SDFT_C64 ? launch_queue_f32(prm, grid, B.spp, B.staged, st)
                            : launch_queue_f64(prm, grid, B.spp, B.staged, st);
}

// ---- allocation-free execution ------------------------------------------------
// Dependency counters for sdft_batch_execute_noalloc live in this fixed array
// instead of the batch's own allocation. Every device that loads the library
// holds it (256 KiB) until the process exits; all calls share it.
constexpr uint64_t kNoAllocCounters = 65536;
static __device__ __align__(256) uint32_t g_noalloc_counters[kNoAllocCounters];

// Device address of the array on the current device (cudaGetSymbolAddress needs
// that device current). In host code the array's name is only a host-side
// stand-in, so kernels get this address. It is looked up when a batch is
// created (sdft_batch_create, which allocates anyway: with lazy module loading
// the first lookup on a device loads this file's module) and kept in the
// batch, so the execute call does no lookup; a batch does not outlive its
// device context, so the address cannot go stale under it.
static sdft_status noalloc_counters(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counters);
  if (e != cudaSuccess) return cuda_fail(e);
  *out = static_cast<uint32_t*>(p);
  return SDFT_OK;
}

static sdft_status run_batch_noalloc(const Batch& B, const void* in, void* out, cudaStream_t st) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev != B.device) return SDFT_ERR_ARG;
  if (!in || !out) return SDFT_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return SDFT_ERR_ARG;
  const uint64_t bytes = B.total * uint64_t(elem_bytes(B.prec));
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
  if (a != b && a < b + bytes && b < a + bytes) return SDFT_ERR_ARG;
  if (B.n_counters > kNoAllocCounters) return SDFT_ERR_UNSUPPORTED;
  if (B.items.empty()) return SDFT_OK;
  uint32_t* counters = B.noalloc_counters;
  if (!counters) return SDFT_ERR_NO_DEVICE;
  sdft_status s;
  QParams prm;
  std::memset(&prm, 0, sizeof(prm));
  s = encode_batch_maps(B, in, out, prm);
  if (s != SDFT_OK) return s;
  prm.a.items = B.d_items;
  prm.a.n_items = B.items.size();
  prm.a.insts = B.d_insts;
  prm.a.counters = counters;
  prm.a.in = in;
  prm.a.out = out;
  prm.a.status = B.d_status;
  prm.a.timeout_ns = B.timeout_ns ? B.timeout_ns : wait_timeout_ns();
  prm.a.need_bias = B.need_bias;
  if (B.n_counters) {   // the array keeps the previous call's counts
    e = cudaMemsetAsync(counters, 0, sizeof(uint32_t) * B.n_counters, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const int grid = int(std::min<uint64_t>(uint64_t(B.grid), B.items.size()));
  return B.prec == SDFT_C64 ? launch_queue_f32(prm, grid, B.spp, B.staged, st)
                            : launch_queue_f64(prm, grid, B.spp, B.staged, st);
}

// Cached queues of strided multi-level execution, keyed by batch size.
struct StridedQueues {
  std::mutex mu;
  std::vector<std::pair<uint64_t, Batch*>> entries;   // most recent last
};
constexpr size_t kStridedQueueCache = 4;

sdft_status run_strided_queue(sdft_plan_s* plan, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  Plan& p = plan->p;
  if (batch > 0xffffffffull) return SDFT_ERR_UNSUPPORTED;
  {
    static std::mutex create_mu;
    std::lock_guard<std::mutex> lk(create_mu);
    if (!p.queues) p.queues = new (std::nothrow) StridedQueues();
    if (!p.queues) return SDFT_ERR_NOMEM;
  }
  StridedQueues* q = static_cast<StridedQueues*>(p.queues);
  Batch* b = nullptr;
  // The lock covers the enqueue as well: another thread's eviction (below)
  // synchronises the device before freeing a queue, which only protects work
  // that has been enqueued already.
  std::lock_guard<std::mutex> lk(q->mu);
  {
    for (auto& e : q->entries)
      if (e.first == batch) b = e.second;
    if (!b) {
      b = new (std::nothrow) Batch();
      if (!b) return SDFT_ERR_NOMEM;
      b->device = p.device;
      b->spp = int(p.spp);
      sdft_status s;
      try {
        std::vector<sdft_plan> plans(batch, plan);
        s = build_batch(*b, plans.data(), batch);
      } catch (const std::bad_alloc&) {
        s = SDFT_ERR_NOMEM;
      }
      if (s != SDFT_OK) {
        free_batch(*b);
        delete b;
        return s;
      }
      b->d_status_shared = p.d_status;     // report into the plan's status word
      if (q->entries.size() >= kStridedQueueCache) {
        // The oldest queue may still be in use by work in flight: synchronise first.
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
          free_batch(*b);
          delete b;
          return cuda_fail(e);
        }
        free_batch(*q->entries.front().second);
        delete q->entries.front().second;
        q->entries.erase(q->entries.begin());
      }
      q->entries.push_back({batch, b});
    }
  }
  return run_batch(*b, in, out, st);
}

// ---- sdft_execute_batched: instances at the caller's offsets ----------------------
// The batch path wants its own packing (instances by decreasing k, so tiles never
// straddle instances); sdft_execute_batched takes any packing: a cached batch of
// the same plans runs between a gather into its layout and a scatter back, both
// one kernel over chunks of at most kRepackChunk values. The caller's offsets
// stay on the device (graph-capturable); a kernel checks each against its plan.
constexpr uint64_t kRepackChunk = 8192;
constexpr int kBadOffsets = 0x104;     // status: offsets[i+1] - offsets[i] differs from plan i's k
constexpr size_t kBatchedCache = 8;

struct RepackItem {
  uint32_t inst;       // instance, caller order
  uint32_t pad;
  uint64_t local;      // first value within the instance
  uint64_t count;      // values
};

template <class C>
__global__ void __launch_bounds__(256) k_repack(const C* __restrict__ src, C* __restrict__ dst,
                                                const uint64_t* __restrict__ user_off,
                                                const uint64_t* __restrict__ kk, const uint64_t* __restrict__ boff,
                                                const RepackItem* __restrict__ items, uint64_t n_items, int* status,
                                                int to_batch) {
  for (uint64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const RepackItem c = items[it];
    const uint64_t uo = user_off[c.inst], un = user_off[c.inst + 1];
    if (un - uo != kk[c.inst]) {       // the caller's offsets do not fit the plans
      if (threadIdx.x == 0) atomicCAS(status, 0, kBadOffsets);
      continue;
    }
    const uint64_t s0 = (to_batch ? uo : boff[c.inst]) + c.local;
    const uint64_t d0 = (to_batch ? boff[c.inst] : uo) + c.local;
    for (uint64_t e = threadIdx.x; e < c.count; e += blockDim.x) dst[d0 + e] = src[s0 + e];
  }
}

struct BatchedEntry {
  std::vector<uint64_t> serials;
  bool pinned = false;                 // never evicted implicitly (sdft_execute_batched_pin)
  Batch* b = nullptr;
  void* d_stage = nullptr;             // 2 x total values: samples, then coefficients
  uint64_t* d_k = nullptr;             // k per instance (caller order)
  uint64_t* d_boff = nullptr;          // the batch's offset per instance (caller order)
  RepackItem* d_items = nullptr;
  uint64_t n_items = 0;
};

// Bytes of one staging half: the batch's values rounded up to 256 bytes.
static uint64_t stage_bytes(uint64_t total, size_t es) { return (std::max<uint64_t>(total, 1) * es + 255) & ~255ull; }

static void free_batched(BatchedEntry& E) {
  if (E.b) {
    free_batch(*E.b);
    delete E.b;
  }
  if (E.d_stage) cudaFree(E.d_stage);
  if (E.d_k) cudaFree(E.d_k);
  if (E.d_boff) cudaFree(E.d_boff);
  if (E.d_items) cudaFree(E.d_items);
  E = BatchedEntry{};
}

static std::mutex g_batched_mu;
static std::vector<BatchedEntry> g_batched;   // most recent last

static sdft_status batched_entry(const sdft_plan* plans, uint64_t n, BatchedEntry** out) {
  std::vector<uint64_t> key(n);
  for (uint64_t i = 0; i < n; ++i) key[i] = plans[i]->p.serial;
  for (auto& E : g_batched)
    if (E.serials == key) {
      *out = &E;
      return SDFT_OK;
    }
  BatchedEntry E;
  E.serials = key;
  E.b = new (std::nothrow) Batch();
  if (!E.b) return SDFT_ERR_NOMEM;
  E.b->device = plans[0]->p.device;
  E.b->plans.assign(plans, plans + n);
  sdft_status s = build_batch(*E.b, plans, n);
  if (s != SDFT_OK) {
    free_batched(E);
    return s;
  }
  E.b->d_status_shared = plans[0]->p.d_status;    // report into the first plan's status word
  std::vector<uint64_t> kk(n), boff(n);
  std::vector<RepackItem> items;
  for (uint64_t i = 0; i < n; ++i) {
    kk[i] = plans[i]->p.k;
    boff[i] = E.b->offsets[i];
    for (uint64_t l = 0; l < kk[i]; l += kRepackChunk)
      items.push_back(RepackItem{uint32_t(i), 0, l, std::min(kRepackChunk, kk[i] - l)});
  }
  E.n_items = items.size();
  const size_t es = size_t(elem_bytes(plans[0]->p.prec));
  cudaError_t e = cudaMalloc(&E.d_stage, 2 * stage_bytes(E.b->total, es));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&E.d_k), sizeof(uint64_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&E.d_boff), sizeof(uint64_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&E.d_items), sizeof(RepackItem) * items.size());
  if (e == cudaSuccess) e = cudaMemcpy(E.d_k, kk.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(E.d_boff, boff.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(E.d_items, items.data(), sizeof(RepackItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_batched(E);
    return e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : cuda_fail(e);
  }
  // Keep at most kBatchedCache unpinned lists: evict the oldest unpinned one.
  // A CUDA graph captured on an evicted list would replay on freed memory, so
  // lists that graphs were captured on must be pinned.
  size_t unpinned = 0;
  for (const auto& x : g_batched) unpinned += x.pinned ? 0 : 1;
  if (unpinned >= kBatchedCache) {
    // the oldest entry may still be in use by work in flight: synchronise first
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      free_batched(E);
      return cuda_fail(e);
    }
    for (size_t i = 0; i < g_batched.size(); ++i)
      if (!g_batched[i].pinned) {
        free_batched(g_batched[i]);
        g_batched.erase(g_batched.begin() + i);
        break;
      }
  }
  g_batched.push_back(std::move(E));
  *out = &g_batched.back();
  return SDFT_OK;
}

sdft_status run_batched(const sdft_plan* plans, uint64_t n, const void* in, const uint64_t* d_offsets, void* out,
                        cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_batched_mu);
  BatchedEntry* E = nullptr;
  sdft_status s = batched_entry(plans, n, &E);
  if (s != SDFT_OK) return s;
  const size_t es = size_t(elem_bytes(E->b->prec));
  char* stage_in = static_cast<char*>(E->d_stage);
  char* stage_out = stage_in + stage_bytes(E->b->total, es);    // 256-byte aligned like the first half
  int* status = plans[0]->p.d_status;
  const unsigned grid = unsigned(std::min<uint64_t>(E->n_items, 4ull * uint64_t(sm_count())));
  if (E->b->prec == SDFT_C64)
    k_repack<float2><<<grid, 256, 0, st>>>(static_cast<const float2*>(in), reinterpret_cast<float2*>(stage_in),
                                           d_offsets, E->d_k, E->d_boff, E->d_items, E->n_items, status, 1);
  else
    k_repack<double2><<<grid, 256, 0, st>>>(static_cast<const double2*>(in), reinterpret_cast<double2*>(stage_in),
                                            d_offsets, E->d_k, E->d_boff, E->d_items, E->n_items, status, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  s = run_batch(*E->b, stage_in, stage_out, st);
  if (s != SDFT_OK) return s;
  if (E->b->prec == SDFT_C64)
    k_repack<float2><<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(stage_out), static_cast<float2*>(out),
                                           d_offsets, E->d_k, E->d_boff, E->d_items, E->n_items, status, 0);
  else
    k_repack<double2><<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(stage_out), static_cast<double2*>(out),
                                            d_offsets, E->d_k, E->d_boff, E->d_items, E->n_items, status, 0);
  e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

sdft_status pin_batched(const sdft_plan* plans, uint64_t n, int pin) {
  std::lock_guard<std::mutex> lk(g_batched_mu);
  if (!pin) {                          // unpin a cached list; nothing to build
    std::vector<uint64_t> key(n);
    for (uint64_t i = 0; i < n; ++i) key[i] = plans[i]->p.serial;
    for (auto& E : g_batched)
      if (E.serials == key) E.pinned = false;
    return SDFT_OK;
  }
  BatchedEntry* E = nullptr;
  sdft_status s = batched_entry(plans, n, &E);
  if (s != SDFT_OK) return s;
  E->pinned = true;
  return SDFT_OK;
}

void batched_cache_info(const sdft_plan* plans, uint64_t n, int* cached, int* pinned, uint64_t* n_lists) {
  std::lock_guard<std::mutex> lk(g_batched_mu);
  int c = 0, p = 0;
  if (plans && n) {
    std::vector<uint64_t> key(n);
    for (uint64_t i = 0; i < n; ++i) key[i] = plans[i]->p.serial;
    for (const auto& E : g_batched)
      if (E.serials == key) {
        c = 1;
        p = E.pinned ? 1 : 0;
      }
  }
  if (cached) *cached = c;
  if (pinned) *pinned = p;
  if (n_lists) *n_lists = g_batched.size();
}

void forget_batched(uint64_t serial) {
  std::lock_guard<std::mutex> lk(g_batched_mu);
  for (size_t i = 0; i < g_batched.size();) {
    const auto& v = g_batched[i].serials;
    if (std::find(v.begin(), v.end(), serial) != v.end()) {
      free_batched(g_batched[i]);
      g_batched.erase(g_batched.begin() + i);
    } else {
      ++i;
    }
  }
}

void free_strided_queues(Plan& p) {
  if (!p.queues) return;
  StridedQueues* q = static_cast<StridedQueues*>(p.queues);
  for (auto& e : q->entries) {
    free_batch(*e.second);
    delete e.second;
  }
  delete q;
  p.queues = nullptr;
}

}  // namespace sdft

extern "C" {

sdft_status sdft_batch_create(const sdft_plan* plans, uint64_t n, sdft_batch* out) {
  if (!out) return SDFT_ERR_ARG;
  *out = nullptr;
  if (!plans || n == 0 || n > 0xffffffffull) return SDFT_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    if (!plans[i]) return SDFT_ERR_ARG;
    if (plans[i]->p.deferred) return SDFT_ERR_NO_DEVICE;   // tables only reach the device via a server
  }
  // Either every plan is host-only (a batch for inspection) or all live on the current device.
  const bool host_only = plans[0]->p.device < 0;
  int dev = -1;
  if (!host_only) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sdft::cuda_fail(e);
  }
  for (uint64_t i = 0; i < n; ++i) {
    if ((plans[i]->p.device < 0) != host_only) return SDFT_ERR_NO_DEVICE;
    if (!host_only && plans[i]->p.device != dev) return SDFT_ERR_ARG;
    if (plans[i]->p.prec != plans[0]->p.prec) return SDFT_ERR_PRECISION;
  }
  sdft_batch_s* h = new (std::nothrow) sdft_batch_s();
  if (!h) return SDFT_ERR_NOMEM;
  h->b.device = dev;
  sdft_status s;
  try {
    h->b.plans.assign(plans, plans + n);
    s = sdft::build_batch(h->b, plans, n);
  } catch (const std::bad_alloc&) {
    s = SDFT_ERR_NOMEM;
  }
  // the allocation-free entry point's counter array: its address on this device
  if (s == SDFT_OK && !host_only) s = sdft::noalloc_counters(&h->b.noalloc_counters);
  if (s != SDFT_OK) {
    sdft::free_batch(h->b);
    delete h;
    return s;
  }
  *out = h;
  return SDFT_OK;
}

sdft_status sdft_batch_info(sdft_batch batch, uint64_t* total, uint64_t* offsets) {
  if (!batch) return SDFT_ERR_ARG;
  if (total) *total = batch->b.total;
  if (offsets) std::memcpy(offsets, batch->b.offsets.data(), sizeof(uint64_t) * (batch->b.n + 1));
  return SDFT_OK;
}

sdft_status sdft_batch_execute(sdft_batch batch, const void* d_samples, void* d_coeffs, void* stream) {
  if (!batch) return SDFT_ERR_ARG;
  if (batch->b.device < 0) return SDFT_ERR_NO_DEVICE;
  return sdft::run_batch(batch->b, d_samples, d_coeffs, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_batch_execute_noalloc(sdft_batch batch, const void* d_samples, void* d_coeffs, void* stream) {
  if (!batch) return SDFT_ERR_ARG;
  if (batch->b.device < 0) return SDFT_ERR_NO_DEVICE;
  return sdft::run_batch_noalloc(batch->b, d_samples, d_coeffs, static_cast<cudaStream_t>(stream));
}

sdft_status sdft_execute_batched(const sdft_plan* plans, uint64_t n, const void* d_samples,
                                 const uint64_t* d_offsets, void* d_coeffs, void* stream) {
  if (!plans || n == 0 || n > 0xffffffffull || !d_samples || !d_offsets || !d_coeffs) return SDFT_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_samples) | reinterpret_cast<uintptr_t>(d_coeffs)) & 15u) return SDFT_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    if (!plans[i]) return SDFT_ERR_ARG;
    if (plans[i]->p.deferred || plans[i]->p.device < 0) return SDFT_ERR_NO_DEVICE;
    if (plans[i]->p.prec != plans[0]->p.prec) return SDFT_ERR_PRECISION;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  for (uint64_t i = 0; i < n; ++i)
    if (plans[i]->p.device != dev) return SDFT_ERR_ARG;
  try {
    return sdft::run_batched(plans, n, d_samples, d_offsets, d_coeffs, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    return SDFT_ERR_NOMEM;
  }
}

// Argument checks shared by the calls that name a list of plans.
static sdft_status check_plan_list(const sdft_plan* plans, uint64_t n) {
  if (!plans || n == 0 || n > 0xffffffffull) return SDFT_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    if (!plans[i]) return SDFT_ERR_ARG;
    if (plans[i]->p.deferred || plans[i]->p.device < 0) return SDFT_ERR_NO_DEVICE;
    if (plans[i]->p.prec != plans[0]->p.prec) return SDFT_ERR_PRECISION;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  for (uint64_t i = 0; i < n; ++i)
    if (plans[i]->p.device != dev) return SDFT_ERR_ARG;
  return SDFT_OK;
}

sdft_status sdft_execute_batched_pin(const sdft_plan* plans, uint64_t n, int pin) {
  sdft_status s = check_plan_list(plans, n);
  if (s != SDFT_OK) return s;
  try {
    return sdft::pin_batched(plans, n, pin);
  } catch (const std::bad_alloc&) {
    return SDFT_ERR_NOMEM;
  }
}

sdft_status sdft_execute_batched_cache_info(const sdft_plan* plans, uint64_t n, int* cached, int* pinned,
                                            uint64_t* n_lists) {
  if ((plans == nullptr) != (n == 0)) return SDFT_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i)
    if (!plans[i]) return SDFT_ERR_ARG;
  try {
    sdft::batched_cache_info(plans, n, cached, pinned, n_lists);
  } catch (const std::bad_alloc&) {
    return SDFT_ERR_NOMEM;
  }
  return SDFT_OK;
}

sdft_status sdft_batch_device_status(sdft_batch batch, int clear) {
  if (!batch) return SDFT_ERR_ARG;
  if (batch->b.device < 0) return SDFT_ERR_NO_DEVICE;
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, batch->b.d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(batch->b.d_status, 0, sizeof(int));
  if (e != cudaSuccess) return sdft::cuda_fail(e);
  return sdft_status(v);
}

sdft_status sdft_batch_set_wait(sdft_batch batch, uint64_t timeout_ns, uint32_t need_bias) {
  if (!batch) return SDFT_ERR_ARG;
  batch->b.timeout_ns = timeout_ns;
  batch->b.need_bias = need_bias;
  return SDFT_OK;
}

sdft_status sdft_batch_stats(sdft_batch batch, uint64_t* n_items, uint64_t* n_counters, int* grid) {
  if (!batch) return SDFT_ERR_ARG;
  if (n_items) *n_items = batch->b.items.size();
  if (n_counters) *n_counters = batch->b.n_counters;
  if (grid) *grid = batch->b.grid;
  return sdft::check_items(batch->b);
}

// Rebuild the item list and device arrays with the batch's current schedule
// and grid settings (offsets and tensor maps do not change).
static sdft_status rebuild_batch(sdft::Batch& B) {
  sdft::free_batch(B);
  try {
    return sdft::build_batch(B, B.plans.data(), B.n);
  } catch (const std::bad_alloc&) {
    return SDFT_ERR_NOMEM;
  }
}

// Item order, CTAs and stages per pass together (one rebuild; the grid and so
// the item list depend on the kernel's occupancy).
static sdft_status set_config(sdft::Batch& B, int schedule, int grid, int spp, bool staged, int lag) {
  if (B.schedule == schedule && B.grid_req == grid && B.spp == spp && B.staged == staged && B.lag == lag &&
      B.d_items)
    return SDFT_OK;
  B.schedule = schedule;
  B.grid_req = grid;
  B.spp = spp;
  B.staged = staged;
  B.lag = lag;
  return rebuild_batch(B);
}

sdft_status sdft_batch_set_schedule(sdft_batch batch, sdft_schedule schedule, uint32_t grid) {
  if (!batch) return SDFT_ERR_ARG;
  if (schedule != SDFT_SCHEDULE_AUTO && schedule != SDFT_SCHEDULE_LANES && schedule != SDFT_SCHEDULE_ROUND_ROBIN)
    return SDFT_ERR_ARG;
  if (grid > (1u << 20)) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  return set_config(B, int(schedule), int(grid), B.spp, B.staged, B.lag);
}

sdft_status sdft_batch_autotune(sdft_batch batch, const void* d_samples, void* d_coeffs, void* stream, int reps,
                                sdft_schedule* chosen, uint32_t* chosen_grid, float* ms_best) {
  if (!batch || reps <= 0) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  if (B.device < 0) return SDFT_ERR_NO_DEVICE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  struct Cand {
    int schedule, grid, spp;
    bool staged;
    int lag;
  };
  // Stages per pass (four; three as well for complex64) x tables in registers
  // and L1 or staged whole in shared memory (complex64) x item order x CTAs:
  // every co-resident CTA, or half of them (fewer intermediates in flight,
  // more L1 per resident CTA) x dependency distance (4, 6 or 8 x grid).
  std::vector<Cand> cands;
  for (int spp : {4, 3})
    for (bool staged : {false, true}) {
      if ((spp == 3 || staged) && B.prec != SDFT_C64) continue;
      const int full = B.prec == SDFT_C64 ? sdft::queue_grid_f32(spp, staged) : sdft::queue_grid_f64(spp, staged);
      if (full <= 0) return SDFT_ERR_CUDA;
      for (int sched : {int(SDFT_SCHEDULE_LANES), int(SDFT_SCHEDULE_ROUND_ROBIN)})
        for (int g : {0, full / 2})
          for (int lag : {sdft::kDefaultLag, 4, 8}) cands.push_back(Cand{sched, g, spp, staged, lag});
    }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return sdft::cuda_fail(e);
  }
  sdft_status s = SDFT_OK;
  float best = -1.f;
  Cand pick = cands[0];
  for (const Cand& c : cands) {
    s = set_config(B, c.schedule, c.grid, c.spp, c.staged, c.lag);
    if (s != SDFT_OK) break;
    s = sdft::run_batch(B, d_samples, d_coeffs, st);     // warm-up
    if (s != SDFT_OK) break;
    e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == SDFT_OK && e == cudaSuccess; ++r) s = sdft::run_batch(B, d_samples, d_coeffs, st);
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (s == SDFT_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess && s == SDFT_OK) s = sdft::cuda_fail(e);
    if (s != SDFT_OK) break;
    ms /= float(reps);
    if (best < 0.f || ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != SDFT_OK) return s;
  s = set_config(B, pick.schedule, pick.grid, pick.spp, pick.staged, pick.lag);
  if (s != SDFT_OK) return s;
  sdft::Tuning tn{0, pick.schedule, pick.grid, pick.spp, best, pick.staged ? 1 : 0};
  tn.lag = pick.lag;
  sdft::tuning_store(sdft::batch_tuning_key(B.prec, B.n, B.total), tn);
  if (chosen) *chosen = sdft_schedule(pick.schedule);
  if (chosen_grid) *chosen_grid = uint32_t(B.grid);
  if (ms_best) *ms_best = best;
  return SDFT_OK;
}

sdft_status sdft_batch_set_stages_per_pass(sdft_batch batch, uint32_t stages_per_pass) {
  if (!batch) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  if (stages_per_pass != 4 && !(stages_per_pass == 3 && B.prec == SDFT_C64)) return SDFT_ERR_ARG;
  return set_config(B, B.schedule, B.grid_req, int(stages_per_pass), B.staged, B.lag);
}

sdft_status sdft_batch_set_table_staging(sdft_batch batch, int staged) {
  if (!batch) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  if (staged && B.prec != SDFT_C64) return SDFT_ERR_ARG;
  return set_config(B, B.schedule, B.grid_req, B.spp, staged != 0, B.lag);
}

sdft_status sdft_batch_set_lag(sdft_batch batch, uint32_t lag) {
  if (!batch || lag < uint32_t(sdft::kMinLag) || lag > uint32_t(sdft::kMaxLag)) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  return set_config(B, B.schedule, B.grid_req, B.spp, B.staged, int(lag));
}

sdft_status sdft_batch_get_lag(sdft_batch batch, uint32_t* lag) {
  if (!batch || !lag) return SDFT_ERR_ARG;
  *lag = uint32_t(batch->b.lag);
  return SDFT_OK;
}

sdft_status sdft_batch_get_table_staging(sdft_batch batch, int* staged) {
  if (!batch || !staged) return SDFT_ERR_ARG;
  *staged = batch->b.staged ? 1 : 0;
  return SDFT_OK;
}

sdft_status sdft_batch_get_stages_per_pass(sdft_batch batch, uint32_t* stages_per_pass) {
  if (!batch || !stages_per_pass) return SDFT_ERR_ARG;
  *stages_per_pass = uint32_t(batch->b.spp);
  return SDFT_OK;
}

sdft_status sdft_batch_apply_tuning(sdft_batch batch, int* found) {
  if (!batch) return SDFT_ERR_ARG;
  sdft::Batch& B = batch->b;
  sdft::Tuning t;
  const bool hit = sdft::tuning_lookup(sdft::batch_tuning_key(B.prec, B.n, B.total), &t);
  if (found) *found = hit ? 1 : 0;
  if (!hit) return SDFT_OK;
  if (t.spp != 4 && !(t.spp == 3 && B.prec == SDFT_C64)) return SDFT_ERR_ARG;
  if (t.staged != 0 && !(t.staged == 1 && B.prec == SDFT_C64)) return SDFT_ERR_ARG;
  if (t.schedule != SDFT_SCHEDULE_AUTO && t.schedule != SDFT_SCHEDULE_LANES && t.schedule != SDFT_SCHEDULE_ROUND_ROBIN)
    return SDFT_ERR_ARG;
  if (t.grid < 0 || t.grid > (1 << 20)) return SDFT_ERR_ARG;
  if (t.lag < sdft::kMinLag || t.lag > sdft::kMaxLag) return SDFT_ERR_ARG;
  return set_config(B, t.schedule, t.grid, t.spp, t.staged != 0, t.lag);
}

sdft_status sdft_batch_destroy(sdft_batch batch) {
  if (!batch) return SDFT_ERR_ARG;
  sdft::free_batch(batch->b);
  delete batch;
  return SDFT_OK;
}

}  // extern "C"
