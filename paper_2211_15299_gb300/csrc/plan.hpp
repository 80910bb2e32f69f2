// Internal plan representation shared by the host planner and the launchers.
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>

#include "sdft.h"

namespace sdft {

// Tile geometry per precision. A tile is 32 KiB of complex values held in
// shared memory as rows of 128 bytes: 2^kTileBits elements, 2^kRowBits per row.
template <int P> struct Geom;
template <> struct Geom<SDFT_C64> {
  static constexpr int kTileBits = 12;   // 4096 complex64
  static constexpr int kRowBits = 4;     // 16 complex64 per 128-byte row
  static constexpr int kElem = 8;
};
template <> struct Geom<SDFT_C128> {
  static constexpr int kTileBits = 11;   // 2048 complex128
  static constexpr int kRowBits = 3;     // 8 complex128 per 128-byte row
  static constexpr int kElem = 16;
};

inline int tile_bits(sdft_prec p) { return p == SDFT_C64 ? 12 : 11; }
inline int row_bits(sdft_prec p) { return p == SDFT_C64 ? 4 : 3; }
inline int elem_bytes(sdft_prec p) { return p == SDFT_C64 ? 8 : 16; }

// Instances with log2 k <= kSmallMax run in registers, one thread per instance.
constexpr uint32_t kSmallMax = 4;

// One butterfly level of the multi-level schedule. Level 0 runs stage bits
// [0, hi) on contiguous tiles; a later level runs stage bits [lo, hi) on tiles
// made of 2^lg column groups (one 128-byte row each) x 2^(hi-lo) rows spaced
// 2^lo elements apart. Inside a tile the stage bits become the virtual bits
// [plo, tile_bits) of a tile-local index.
struct Level {
  uint32_t lo = 0, hi = 0;      // stage bits of the instance index t
  uint32_t plo = 0;             // first virtual stage bit inside the tile
  uint32_t lg = 0;              // log2 column groups per tile (later levels)
  uint64_t n_gb = 1;            // number of distinct twiddle tables (group blocks)
  uint64_t tw_off = 0;          // element offset of the level's tables
  uint64_t tw_len = 0;          // elements per table
  bool last = false;            // contains the final stage (applies N/k)
};

struct Plan {
  uint32_t M = 0, s = 0;
  uint64_t k = 1;
  sdft_prec prec = SDFT_C64;
  std::vector<uint32_t> pivots;   // r_1 < ... < r_s
  std::vector<uint64_t> Jc;       // canonical order
  std::vector<uint64_t> I;        // sample order
  std::vector<Level> levels;      // empty when s <= kSmallMax (register path)
  uint32_t spp = 4;               // stages per pass of the level kernels (3 or 4; 3: complex64 forward only)
  uint64_t tw_elems = 0;          // complex entries in the device table buffer
  int device = -1;
  void* d_tw = nullptr;           // device twiddles (float2 or double2)
  void* d_tw_df = nullptr;        // the same table as double-float pairs (SDFT_PLAN_FP64_DF)
  uint32_t* d_user_pos = nullptr; // SDFT_PLAN_USER_ORDER: canonical position of J[u]
  int* d_status = nullptr;        // device status word
  uint64_t device_bytes = 0;
  double tw0[32] = {0};           // level-0 table entries 1..15 (rounded to prec), for kernel params
  void* queues = nullptr;         // cached work queues of strided multi-level execution (batch.cu)
  bool deferred = false;          // device tables not uploaded: host_tables holds them (serving)
  std::vector<unsigned char> host_tables;
  int strategy = SDFT_STRATEGY_LEVELS;
  uint64_t serial = 0;            // creation number, never reused (caches keyed by plans)
};

// Host-side planning (plan.cpp). Fills everything except the device fields.
sdft_status build_plan(uint32_t log2N, const uint64_t* J, uint64_t k, sdft_prec prec, Plan& p);

// FP64 twiddle of stage m (1-based) at position u < 2^(m-1), unscaled:
// exp(-2 pi i (Jc[u] mod 2^r_m) / 2^(r_m+1)).
void twiddle_f64(const Plan& p, uint32_t m, uint64_t u, double& re, double& im);

// Every level at which the congruence tree of an arbitrary set J splits (bit l
// of level_mask), from depth-first neighbours; SDFT_ERR_DUPLICATE /
// SDFT_ERR_RANGE for repeated or out-of-range elements.
sdft_status split_levels(uint32_t M, const uint64_t* J, uint64_t k, uint64_t& level_mask);

// Device-table layout (rounded to the plan's precision, final stage scaled by
// N/k) written into `out` as interleaved pairs of `T`.
template <class T> void fill_device_tables(const Plan& p, T* out);

}  // namespace sdft

// The opaque handle of the C ABI.
struct sdft_plan_s {
  sdft::Plan p;
  // sdft_execute_strided_host: copy-in / copy-out streams and three events,
  // created on first use (cudaStream_t / cudaEvent_t), and the lock that keeps
  // one call's chain of copies, launches and event records in order.
  std::mutex host_mu;
  void* host_st[2] = {nullptr, nullptr};
  void* host_ev[3] = {nullptr, nullptr, nullptr};
};
