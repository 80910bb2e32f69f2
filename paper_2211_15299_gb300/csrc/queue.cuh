// Persistent work-queue kernel: many instances with their own plans (uneven
// batches) and multi-level instances with L2-resident intermediates, in one
// launch.
//
// Items (host-built, see batch.cu) are processed round-robin: CTA c takes items
// c, c + G, c + 2G, ... in list order, on a cooperatively launched grid (all
// CTAs resident). Each CTA has NT compute threads and one producer warp: the
// producer loads tiles (TMA) after their dependencies are met, stores computed
// tiles and publishes counters; the compute threads only wait for tiles
// (full barriers) and hand buffers back (empty barriers). Item kinds:
//   * small range: up to NT instances with log2 k <= 4, one thread each;
//   * level-0 tile: 2^(TB - s) whole instances of size 2^s (s <= TB), or one
//     2^TB chunk of a larger instance (stage bits [0, min(s, TB)));
//   * later-level tile: one group block of one instance (stage bits [lo, hi)).
// A later-level item waits (bounded) until its instance's previous level has
// signalled every tile; the host places it at least 4 G items after those
// tiles, so the wait never targets an item of the same CTA that has not yet
// signalled, and the intermediate is still in L2 when it is read back.
#pragma once

#include "kernels.cuh"
#include "launch.hpp"

namespace sdft {

constexpr uint32_t kNone = 0xffffffffu;
// Tile buffers per CTA. Two leave the L1 room for the next item's table
// entries, which the compute warps prefetch there; the dependency distance of
// four items per CTA (see above) stays above the buffers plus one.
constexpr int kQBufs = 2;

struct QItem {            // 48 bytes
  uint16_t variant;       // kind and template variant, see q_variant_*
  uint16_t map;           // map slot (level 0: load slot, store slot = map + 1)
  uint32_t count;         // instances (level 0: tile's instances; small: range length)
  uint32_t inst;          // first instance
  uint32_t dep;           // counter to wait on, or kNone
  uint32_t need;          // value the counter must reach
  uint32_t sig;           // counter to increment once the item's store is complete, or kNone
  int32_t c1, c3;         // TMA coordinates of the tile
  const void* tw;         // twiddle table, absolute-indexed: level 0 the (first) instance's
                          // plan table, later levels the group block's table
  double scale;           // N/k of the (first) instance
};

struct QInst {            // 32 bytes
  const void* tw;         // level-0 table of the instance's plan, absolute-indexed
  uint64_t off;           // element offset in the packed buffers
  uint32_t s;             // log2 k
  uint32_t pad;
  double scale;           // N/k
};

constexpr int kMaxMaps = 40;

struct QArgs {
  const QItem* items;
  uint64_t n_items;
  const QInst* insts;
  uint32_t* counters;       // zeroed before every launch
  const void* in;           // packed samples (small items use plain loads)
  void* out;                // packed coefficients
  int* status;
  uint64_t timeout_ns;
  uint32_t need_bias;       // added to every dependency target (0; non-zero only to test timeouts)
  uint32_t n_counters;      // counters in `counters` (range checks)
  uint64_t n_insts;         // records in `insts` (range checks)
  uint64_t total;           // values in each packed buffer (range checks)
};

// Item records are copied by the producer into a shared-memory ring three items
// ahead of use (cp.async), so it never waits on a global load of a record.
constexpr int kMetaSlots = 6;
static_assert(sizeof(QItem) % 16 == 0, "items are copied in 16-byte pieces");
// Per tile buffer, a shared-memory copy of the table entries its first and
// middle passes read (copied by the producer with the tile, on its barrier):
// entries below 2^8 with four stages per pass, below 2^9 with three (the two
// middle passes of a 2^12-value tile).
// ST (staged tables): one CTA per SM, and each tile buffer's table copy holds
// the item's whole table (2^TB entries, 32 KiB), so every pass, the top one
// included, reads its twiddles from shared memory and no compute warp waits on
// a global load.
template <class R, int W, bool ST = false>
constexpr uint32_t q_tw_entries() { return ST ? (1u << KT<R>::TB) : (W == 3 ? 512u : 256u); }
template <class R, int W, bool ST = false>
constexpr uint32_t q_tw_bytes() { return q_tw_entries<R, W, ST>() * KT<R>::ES; }
constexpr uint32_t kQTwOff = kQBufs * kTileBytes + 64 + kMetaSlots * sizeof(QItem);
static_assert(kQTwOff % 16 == 0, "table copies need 16-byte alignment");
template <class R, int W, bool ST = false>
constexpr uint32_t q_smem() { return kQTwOff + kQBufs * q_tw_bytes<R, W, ST>() + 1024; }

// Entries [lo, hi) of an item's table staged in shared memory, for a tile
// whose stages are [PLO, TB): the first pass's entries (PLO = 0) and the
// memory-read passes', when they fit the copy; hi = 0: none.
constexpr int q_stage_hi(int TB, int W, int PLO, int cap) {
  if (cap >= (1 << TB)) return 1 << TB;            // staged tables: everything
  const int mlo = mid_pass_lo(TB, W, PLO, TB), mhi = mid_pass_hi(TB, W, PLO, TB);
  if (mlo >= mhi || (1 << mhi) > cap) return PLO == 0 ? (1 << W) : 0;
  return 1 << mhi;
}
constexpr int q_stage_lo(int TB, int W, int PLO, int cap) {
  if (cap >= (1 << TB)) return PLO == 0 ? 0 : (1 << PLO);
  return PLO == 0 ? 0 : (q_stage_hi(TB, W, PLO, cap) ? (1 << mid_pass_lo(TB, W, PLO, TB)) : 0);
}

// Kernel parameters: the arguments and the tensor maps over the packed buffers
// (maps in parameter space are baked into a captured CUDA graph).
struct QParams {
  CUtensorMap maps[kMaxMaps];
  int32_t lim1[kMaxMaps], lim3[kMaxMaps];   // tile origins of map m lie in [0, lim1[m]) x [0, lim3[m]) (range checks)
  QArgs a;
};
// Record the coordinate extents of map `slot` (dims as given to encode_map).
inline void q_set_limits(QParams& prm, size_t slot, const uint64_t dims[4]) {
  prm.lim1[slot] = int32_t(dims[1] > 0x7fffffffull ? 0x7fffffffull : dims[1]);
  prm.lim3[slot] = int32_t(dims[3] > 0x7fffffffull ? 0x7fffffffull : dims[3]);
}

// Variant ids.
constexpr int kVSmall = 0;
constexpr int kVNop = 0x7fff;     // padding item: no data, keeps dependency distances
constexpr int q_variant_first(int s) { return 1 + (s - 5); }        // level 0, 5 <= s <= TB
constexpr int kVFirstChunk = 15;                                       // level 0, s > TB
constexpr int q_variant_later(int Q, bool last) { return 16 + 2 * (Q - 1) + (last ? 1 : 0); }

// ---- one pass with per-instance twiddle tables ------------------------------------
// Elements of the tile with index T belong to instance (T >> SB) of the tile
// (SB >= TB: one instance). tab[g] is the absolute-indexed table of the g-th
// instance among the thread's elements (g = E >> SB), sc[g] its N/k.
template <class R, int W, int B, int SLO, int SHI, bool SCALE, bool FENCE, int SB>
__device__ __forceinline__ void tile_pass_q(char* buf, const typename KT<R>::C* const* tab, const R* sc,
                                            uint32_t tid) {
  using C = typename KT<R>::C;
  constexpr uint32_t LOWM = (1u << B) - 1u;
  constexpr int NE = 1 << W;
  const uint32_t F = (tid & LOWM) | ((tid >> B) << (B + W));
  const uint32_t rF = row_part<R>(F), xF = xor_part<R>(F);
  C v[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const uint32_t E = uint32_t(e) << B;
    v[e] = *reinterpret_cast<const C*>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)));
  }
#pragma unroll
  for (int m1 = SLO; m1 < SHI; ++m1) {
    const int q = m1 - B;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if ((e >> q) & 1) continue;
      const int eh = e | (1 << q);
      const int g = (SB >= 32) ? 0 : int((uint32_t(e) << B) >> SB);
      const C wt = __ldg(tab[g] + (1u << m1) + (F & LOWM) + (uint32_t(e & ((1 << q) - 1)) << B));
      if (SCALE && m1 == SHI - 1)
        bfly_scaled(v[e], v[eh], wt, sc[g]);
      else
        bfly(v[e], v[eh], wt);
    }
  }
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const uint32_t E = uint32_t(e) << B;
    *reinterpret_cast<C*>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E))) = v[e];
  }
  if constexpr (FENCE) ptx::fence_proxy_async_smem();
  ptx::named_bar_sync(1, tile_threads<R, W>());     // the compute threads only (not the producer warp)
}

template <class R, int W, int PLO, int PHI, bool LAST, int SB, int P = 0>
__device__ __forceinline__ void run_passes_q(char* buf, const QArgs& a, const QItem& it, uint32_t tid) {
  using C = typename KT<R>::C;
  constexpr int TB = KT<R>::TB;
  if constexpr (P < n_passes(TB, W, PLO, PHI)) {
    constexpr int B = pass_b(TB, W, PLO, PHI, P), SLO = pass_done(TB, W, PLO, PHI, P),
                  SHI = pass_shi(TB, W, PLO, PHI, P);
    constexpr bool FINAL = (SHI == PHI);
    constexpr int NG = (SB >= 32 || B + W <= SB) ? 1 : (1 << (B + W - SB));
    const C* tab[NG];
    R sc[NG];
    if constexpr (SB >= 32) {
      tab[0] = static_cast<const C*>(it.tw);
      sc[0] = R(it.scale);
    } else {
      const uint32_t F = (tid & ((1u << B) - 1u)) | ((tid >> B) << (B + W));
      const uint32_t g0 = (SB >= TB) ? 0u : (F >> SB);
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        // threads beyond the tile's instances compute on stale rows that are never stored
        const uint32_t gi = (g0 + uint32_t(g) < it.count) ? g0 + uint32_t(g) : 0u;
        const QInst* ins = a.insts + it.inst + gi;
        tab[g] = static_cast<const C*>(ins->tw);
        sc[g] = R(ins->scale);
      }
    }
    tile_pass_q<R, W, B, SLO, SHI, LAST && FINAL, FINAL, SB>(buf, tab, sc, tid);
    run_passes_q<R, W, PLO, PHI, LAST, SB, P + 1>(buf, a, it, tid);
  }
}

// Level 0 with 5 <= s <= TB: tiles of whole instances.
template <class R, int W, int S = 5>
__device__ __forceinline__ bool dispatch_first_q(int v, char* buf, const QArgs& a, const QItem& it, uint32_t tid) {
  if constexpr (S > KT<R>::TB) {
    return false;
  } else {
    if (v == q_variant_first(S)) {
      run_passes_q<R, W, 0, S, true, S>(buf, a, it, tid);
      return true;
    }
    return dispatch_first_q<R, W, S + 1>(v, buf, a, it, tid);
  }
}

// Small instances: one thread per instance, k <= 16 in registers.
template <class R, int S>
__device__ __forceinline__ void small_one(const typename KT<R>::C* __restrict__ in, typename KT<R>::C* __restrict__ out,
                                          const typename KT<R>::C* __restrict__ tw, R sc) {
  using C = typename KT<R>::C;
  constexpr int K = 1 << S;
  C v[K];
#pragma unroll
  for (int e = 0; e < K; ++e) v[e] = in[e];
#pragma unroll
  for (int m1 = 0; m1 < S; ++m1) {
#pragma unroll
    for (int e = 0; e < K; ++e) {
      if ((e >> m1) & 1) continue;
      const C w = __ldg(tw + (1u << m1) + (e & ((1 << m1) - 1)));
      if (m1 == S - 1)
        bfly_scaled(v[e], v[e | (1 << m1)], w, sc);
      else
        bfly(v[e], v[e | (1 << m1)], w);
    }
  }
  if constexpr (S == 0) {
    v[0].x *= sc;
    v[0].y *= sc;
  }
#pragma unroll
  for (int e = 0; e < K; ++e) out[e] = v[e];
}

template <class R>
__device__ __forceinline__ void run_small(const QArgs& a, const QItem& it, uint32_t tid) {
  using C = typename KT<R>::C;
  if (tid >= it.count) return;
  const QInst ins = a.insts[it.inst + tid];
  if (!in_bounds(ins.s <= kSmallMax && ins.off + (1ull << ins.s) <= a.total, a.status)) return;   // debug build
  const C* in = static_cast<const C*>(a.in) + ins.off;
  C* out = static_cast<C*>(a.out) + ins.off;
  const C* tw = static_cast<const C*>(ins.tw);
  const R sc = R(ins.scale);
  switch (ins.s) {
    case 0: small_one<R, 0>(in, out, tw, sc); break;
    case 1: small_one<R, 1>(in, out, tw, sc); break;
    case 2: small_one<R, 2>(in, out, tw, sc); break;
    case 3: small_one<R, 3>(in, out, tw, sc); break;
    default: small_one<R, 4>(in, out, tw, sc); break;
  }
}

// A single-table item (a 2^TB chunk, a one-instance tile, a later-level group
// block): the passes of k_level with the top pass's twiddles loaded into
// registers for this item (the previous item prefetched them into L1).
template <class R, int W, int PLO, int PHI, bool LAST, bool ST = false>
__device__ __forceinline__ void run_single(char* buf, const typename KT<R>::C* tab, R sc, uint32_t tid,
                                           uint32_t wsm) {
  using C = typename KT<R>::C;
  constexpr int TB = KT<R>::TB;
  constexpr int NREG = ST ? 0 : reg_twiddles(TB, W, PLO, PHI);
  constexpr int CAP = int(q_tw_entries<R, W, ST>());
  C wreg[NREG > 0 ? NREG : 1];
  if constexpr (!ST) load_reg_twiddles<R, W, PLO, PHI>(tab, tid, wreg);
  // staged entries (q_stage_lo/hi) come from shared memory at wsm; the rest from
  // global memory (pass 0 reads entry 2^m1 + u as w0[2^m1 - 1 + u]: w0 = tab + 1)
  constexpr bool MID = q_stage_hi(TB, W, PLO, CAP) > (1 << W) || (PLO > 0 && q_stage_hi(TB, W, PLO, CAP) > 0);
  constexpr bool P0 = PLO == 0;
  run_passes<R, W, PLO, PHI, LAST, 0, 0, MID, NoHook, 1, P0, ST>(buf, wreg, tab + 1, tab, tid, sc, wsm);
}

template <class R, int W, bool ST, int Q = 1>
__device__ __forceinline__ void dispatch_later_single(int v, char* buf, const typename KT<R>::C* tab, R sc,
                                                      uint32_t tid, uint32_t wsm) {
  constexpr int TB = KT<R>::TB, CB = KT<R>::CB;
  if constexpr (Q <= TB - CB) {
    if (v == q_variant_later(Q, true)) return run_single<R, W, TB - Q, TB, true, ST>(buf, tab, sc, tid, wsm);
    if (v == q_variant_later(Q, false)) return run_single<R, W, TB - Q, TB, false, ST>(buf, tab, sc, tid, wsm);
    dispatch_later_single<R, W, ST, Q + 1>(v, buf, tab, sc, tid, wsm);
  }
}

template <class R, int W, int Q = 1>
__device__ __forceinline__ void dispatch_later_prefetch(int v, const typename KT<R>::C* tab, uint32_t tid) {
  constexpr int TB = KT<R>::TB, CB = KT<R>::CB;
  if constexpr (Q <= TB - CB) {
    if (v == q_variant_later(Q, true) || v == q_variant_later(Q, false))
      return prefetch_twiddles<R, W, TB - Q, TB>(tab, tid);
    dispatch_later_prefetch<R, W, Q + 1>(v, tab, tid);
  }
}

// Shared-memory layout after the tile buffers: full[3] and empty[3] mbarriers,
// the abort flag, then the record ring.
constexpr uint32_t kQFull = 0, kQEmpty = 24, kQAbort = 48;
template <class R, int W>
constexpr uint32_t q_threads() { return tile_threads<R, W>() + 32; }   // compute threads + one producer warp

__device__ __forceinline__ bool q_is_tma(const QItem& it) { return it.variant != kVSmall && it.variant != kVNop; }

__device__ __forceinline__ const QItem& q_meta(char* smem, uint64_t j) {
  return reinterpret_cast<const QItem*>(smem + kQBufs * kTileBytes + 64)[j % kMetaSlots];
}

// Range checks of a work-item record (debug build): map slots, tile origins
// against the maps' extents, counters, instance records. A failing item is
// turned into a no-op by the producer (its tile is neither loaded nor stored).
template <class R>
__device__ __forceinline__ bool q_item_in_bounds(const QParams& prm, const QItem& it) {
  const QArgs& a = prm.a;
  if (it.variant == kVNop) return true;
  if (it.variant == kVSmall) return in_bounds(it.count >= 1 && uint64_t(it.inst) + it.count <= a.n_insts, a.status);
  const uint32_t ld = it.map, sv = it.variant < 16 ? uint32_t(it.map) + 1u : uint32_t(it.map);
  bool ok = it.tw != nullptr && ld < uint32_t(kMaxMaps) && sv < uint32_t(kMaxMaps);
  ok = ok && it.c1 >= 0 && it.c3 >= 0 && it.c1 < prm.lim1[ld] && it.c3 < prm.lim3[ld] && it.c1 < prm.lim1[sv] &&
       it.c3 < prm.lim3[sv];
  ok = ok && (it.dep == kNone || it.dep < a.n_counters) && (it.sig == kNone || it.sig < a.n_counters);
  ok = ok && uint64_t(it.inst) + (it.variant < 15 ? uint64_t(it.count) : 1u) <= a.n_insts;
  return in_bounds(ok, a.status);
}

// The producer warp's loop (lane 0). CTA c takes items c, c + G, ... Iteration
// j: (1) once item i = j - kQBufs is computed (empty[i % kQBufs]), store it
// from its buffer, commit one bulk group, and publish item i - 1's counter (its
// store complete); (2) load item j into the freed buffer (after its
// dependency, if any, is met) and announce it on full[j % kQBufs]; fetch record
// j + 3 (into the slot of item j - 3, stored already). A counter is published
// before the dependency wait of the item kQBufs + 1 places later in the same
// CTA; the host places items that wait on one another at least 4 x grid list
// positions apart, so every wait ends (all CTAs are resident).
template <class R, int W, bool ST>
__device__ __forceinline__ void q_producer(const QParams& prm, char* smem, uint64_t n) {
  const uint64_t c = blockIdx.x, G = gridDim.x;
  const uint32_t bars = ptx::smem_addr(smem + kQBufs * kTileBytes);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kQBufs * kTileBytes + kQAbort);
  const uint64_t tmo = prm.a.timeout_ns;
  auto fetch_record = [&](uint64_t j) {
    if (j < n) {
      const char* src = reinterpret_cast<const char*>(&prm.a.items[c + j * G]);
      const uint32_t dst = ptx::smem_addr(&q_meta(smem, j));
#pragma unroll
      for (uint32_t o = 0; o < sizeof(QItem); o += 16) ptx::cp_async_16(dst + o, src + o);
    }
    ptx::cp_async_commit();
  };
  for (uint64_t j = 0; j < 3; ++j) fetch_record(j);
  uint32_t pending_sig = kNone;       // counter of the last stored item, not yet published
  uint32_t inflight = 0;              // buffers with a load whose tile is not yet consumed
  uint32_t load_par = 0;              // bit q: phase parity of buffer q's last load
  const void* last_tab = nullptr;     // table of the last item whose tables were prefetched
  bool failed = false;
  uint64_t j = 0;
  for (; j < n + kQBufs; ++j) {
    const uint32_t b = uint32_t(j % kQBufs);
    if (j >= kQBufs) {
      const uint64_t i = j - kQBufs;
      if (!ptx::mbar_wait_bounded(bars + kQEmpty + 8 * b, uint32_t((i / kQBufs) & 1), tmo)) {
        failed = true;
        break;
      }
      inflight &= ~(1u << b);
      const QItem& it = q_meta(smem, i);
      const bool tma = q_is_tma(it);
      if (tma) {
        const uint32_t slot = (it.variant < 16) ? uint32_t(it.map) + 1u : uint32_t(it.map);
        // an intermediate (read back by a later level) stays in L2 ahead of streaming data
        const uint64_t pol = (it.sig != kNone) ? ptx::policy_evict_last() : ptx::policy_evict_first();
        ptx::tma_store_4d_hint(&prm.maps[slot], ptx::smem_addr(smem + b * kTileBytes), 0, it.c1, 0, it.c3, pol);
      }
      ptx::bulk_commit();
      if (pending_sig != kNone) {      // the previous store is complete: publish it
        ptx::bulk_wait<1>();
        ptx::fence_proxy_async_global();
        ptx::red_add_release_gpu(prm.a.counters + pending_sig, 1u);
      }
      pending_sig = tma ? it.sig : kNone;
      if (j < n) ptx::bulk_wait_read<0>();   // the buffer is refilled below
    }
    if (j < n) {
      ptx::cp_async_wait<2>();         // record j has landed
      if (!q_item_in_bounds<R>(prm, q_meta(smem, j)))      // debug build only
        const_cast<QItem&>(q_meta(smem, j)).variant = kVNop;
      const QItem& it = q_meta(smem, j);
      const uint32_t full = bars + kQFull + 8 * b;
      if (q_is_tma(it)) {
        if (it.dep != kNone) {
          const uint32_t* ctr = prm.a.counters + it.dep;
          const uint32_t need = it.need + prm.a.need_bias;
          if (ptx::ld_acquire_gpu(ctr) < need) {
            const uint64_t t0 = ptx::globaltimer();
            while (ptx::ld_acquire_gpu(ctr) < need) {
              if (ptx::globaltimer() - t0 > tmo) {
                failed = true;
                break;
              }
            }
          }
          if (failed) {
            // wake the compute warps at this item: they stop at the abort flag
            *abort_flag = 1;
            ptx::mbar_arrive(full);
            break;
          }
          ptx::fence_proxy_async_global();
        }
        const uint32_t bytes = (it.variant < 16) ? (128u << (it.map / 2)) : kTileBytes;
        // the table entries the first and middle passes read, copied with the tile
        constexpr int TBs = KT<R>::TB, CAP = int(q_tw_entries<R, W, ST>());
        int slo = 0, shi = 0;
        if (it.variant == kVFirstChunk || it.variant == q_variant_first(TBs)) {
          slo = q_stage_lo(TBs, W, 0, CAP);
          shi = q_stage_hi(TBs, W, 0, CAP);
        } else if (it.variant >= 16) {
          const int plo = TBs - ((it.variant - 16) / 2 + 1);
          slo = q_stage_lo(TBs, W, plo, CAP);
          shi = q_stage_hi(TBs, W, plo, CAP);
        }
        const uint32_t tw_bytes = shi > slo ? uint32_t(shi - slo) * KT<R>::ES : 0u;
        ptx::mbar_arrive_expect_tx(full, bytes + tw_bytes);
        // samples and intermediates are read once: first out of L2
        ptx::tma_load_4d_hint(ptx::smem_addr(smem + b * kTileBytes), &prm.maps[it.map], full, 0, it.c1, 0, it.c3,
                              ptx::policy_evict_first());
        if (tw_bytes)
          ptx::bulk_load(ptx::smem_addr(smem + kQTwOff + b * q_tw_bytes<R, W, ST>()) + uint32_t(slo) * KT<R>::ES,
                         static_cast<const char*>(it.tw) + size_t(slo) * KT<R>::ES, tw_bytes, full);
        inflight |= 1u << b;
        load_par = (load_par & ~(1u << b)) | (uint32_t((j / kQBufs) & 1) << b);
        // the item's tables into L2 while its tile is in flight (once per table
        // in a row of items: repeated bulk prefetches of the same lines queue in
        // front of the tile copies)
        constexpr int TB = KT<R>::TB;
        constexpr uint32_t ES = KT<R>::ES;
        if (it.variant >= 16) {
          if (it.tw != last_tab) {
            const uint32_t first = 1u << (TB - ((it.variant - 16) / 2 + 1));
            ptx::prefetch_l2(static_cast<const char*>(it.tw) + first * ES, ((1u << TB) - first) * ES);
          }
        } else if (it.variant == kVFirstChunk || it.variant == q_variant_first(TB)) {
          if (it.tw != last_tab) ptx::prefetch_l2(it.tw, (1u << TB) * ES);
        } else {
          const int ss = it.variant - 1 + 5;
          const uint32_t cnt = it.count < 16u ? it.count : 16u;
          const void* last = nullptr;
          for (uint32_t g = 0; g < cnt; ++g) {        // distinct tables only
            const void* tw = prm.a.insts[it.inst + g].tw;
            if (tw && tw != last) ptx::prefetch_l2(tw, (1u << ss) * ES);
            last = tw;
          }
        }
        last_tab = it.tw;
      } else {
        ptx::mbar_arrive(full);        // nothing to load: the phase completes at once
      }
      fetch_record(j + 3);             // into the slot of item j - 3, computed already
    }
  }
  ptx::cp_async_wait<0>();
  if (failed) {
    // let every issued load land before the CTA's shared memory is released
    for (int q = 0; q < kQBufs; ++q)
      if (inflight >> q & 1u) ptx::mbar_wait_bounded(bars + kQFull + 8 * q, (load_par >> q) & 1u, drain_bound(tmo));
    atomicExch(prm.a.status, int(SDFT_ERR_TIMEOUT));
  }
  ptx::bulk_wait<0>();
  if (!failed && pending_sig != kNone) {
    ptx::fence_proxy_async_global();
    ptx::red_add_release_gpu(prm.a.counters + pending_sig, 1u);
  }
}

template <class R, int W, bool ST>
__global__ void __launch_bounds__(q_threads<R, W>(), ST ? 1 : 2) k_queue(const __grid_constant__ QParams prm) {
  const QArgs& a = prm.a;
  extern __shared__ char smem_raw[];
  char* smem = align1024(smem_raw);
  const uint32_t bars = ptx::smem_addr(smem + kQBufs * kTileBytes);
  const uint32_t tid = threadIdx.x;
  constexpr uint32_t NT = tile_threads<R, W>();
  {
    const uint32_t used = uint32_t(smem - smem_raw) + kQTwOff + kQBufs * q_tw_bytes<R, W, ST>();
    int bad = 0;
    if (ptx::dynamic_smem_size() < used) bad = kBadSmem;
    else if (reinterpret_cast<uintptr_t>(&prm.maps[0]) & 63u) bad = kBadMap;
    else if (reinterpret_cast<uintptr_t>(a.items) & 15u) bad = kBadTable;
    if (bad) {
      if (tid == 0) atomicCAS(a.status, 0, bad);
      return;
    }
  }
  const uint64_t c = blockIdx.x, G = gridDim.x;
  const uint64_t n = (a.n_items > c) ? (a.n_items - c + G - 1) / G : 0;
  if (n == 0) return;
  if (tid == 0) {
    for (int b = 0; b < kQBufs; ++b) {
      ptx::mbar_init(bars + kQFull + 8 * b, 1);        // the producer's arrival (+ the tile's bytes)
      ptx::mbar_init(bars + kQEmpty + 8 * b, NT);      // every compute thread, once done with the buffer
    }
    *reinterpret_cast<volatile int*>(smem + kQBufs * kTileBytes + kQAbort) = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (tid >= NT) {                     // the producer warp
    if (tid == NT) q_producer<R, W, ST>(prm, smem, n);
    return;
  }
  using C = typename KT<R>::C;
  constexpr int TB = KT<R>::TB;
  const volatile int* abort_flag = reinterpret_cast<const volatile int*>(smem + kQBufs * kTileBytes + kQAbort);
  for (uint64_t j = 0; j < n; ++j) {
    const uint32_t b = uint32_t(j % kQBufs);
    const bool ok = ptx::mbar_wait_bounded(bars + kQFull + 8 * b, uint32_t((j / kQBufs) & 1), a.timeout_ns);
    if (ptx::named_bar_or(1, NT, !ok || *abort_flag != 0)) {
      if (tid == 0 && !ok) atomicExch(a.status, int(SDFT_ERR_TIMEOUT));
      break;
    }
    const QItem it = q_meta(smem, j);
    const int v = it.variant;
    const C* tab = static_cast<const C*>(it.tw);
    const R sc = R(it.scale);
    char* buf = smem + b * kTileBytes;
    const uint32_t wsm = ptx::smem_addr(smem + kQTwOff + b * q_tw_bytes<R, W, ST>());
    if (v == kVNop) {
      // nothing to do
    } else if (v == kVSmall) {
      run_small<R>(a, it, tid);
    } else if (v == kVFirstChunk) {
      run_single<R, W, 0, TB, false, ST>(buf, tab, sc, tid, wsm);
    } else if (v == q_variant_first(TB)) {
      run_single<R, W, 0, TB, true, ST>(buf, tab, sc, tid, wsm);
    } else if (v >= 16) {
      dispatch_later_single<R, W, ST>(v, buf, tab, sc, tid, wsm);
    } else {
      dispatch_first_q<R, W>(v, buf, a, it, tid);   // several instances per tile
    }
    ptx::mbar_arrive(bars + kQEmpty + 8 * b);   // after the final pass's proxy fence and barrier
    // the next item's register and L1 twiddles, if its tile has landed already
    // (staged tables need none)
    if (!ST && j + 1 < n) {
      const uint32_t nb = uint32_t((j + 1) % kQBufs);
      if (ptx::mbar_test_wait(bars + kQFull + 8 * nb, uint32_t(((j + 1) / kQBufs) & 1))) {
        const QItem& nx = q_meta(smem, j + 1);
        const int nv = nx.variant;
        const C* nt = static_cast<const C*>(nx.tw);
        if (nt && nt != tab) {
          if (nv == kVFirstChunk || nv == q_variant_first(TB)) prefetch_twiddles<R, W, 0, TB>(nt, tid);
          else if (nv >= 16 && nv != kVNop) dispatch_later_prefetch<R, W>(nv, nt, tid);
        }
      }
    }
  }
}

}  // namespace sdft

namespace sdft {

// Host launchers (queue_f32*.cu, queue_f64.cu). `w`: stages per pass (3 or 4
// for complex64, 4 for complex128); `staged`: whole tables in shared memory
// (complex64 only).
sdft_status launch_queue_f32(const QParams& prm, int grid, int w, bool staged, cudaStream_t st);
sdft_status launch_queue_f64(const QParams& prm, int grid, int w, bool staged, cudaStream_t st);
// Co-resident CTAs of the queue kernel on the current device (occupancy x SMs).
int queue_grid_f32(int w, bool staged);
int queue_grid_f64(int w, bool staged);

template <class R, int W, bool ST>
int queue_grid() {
  auto fn = k_queue<R, W, ST>;
  if (ensure_smem(reinterpret_cast<const void*>(fn), int(q_smem<R, W, ST>())) != SDFT_OK) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, q_threads<R, W>(), q_smem<R, W, ST>()) !=
      cudaSuccess)
    return 0;
  return per_sm * sm_count();
}

template <class R, int W, bool ST>
sdft_status launch_queue(const QParams& prm, int grid, cudaStream_t st) {
  auto fn = k_queue<R, W, ST>;
  sdft_status s = ensure_smem(reinterpret_cast<const void*>(fn), int(q_smem<R, W, ST>()));
  if (s != SDFT_OK) return s;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(q_threads<R, W>());
  cfg.dynamicSmemBytes = q_smem<R, W, ST>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident: dependency waits make progress
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, prm);
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

}  // namespace sdft
