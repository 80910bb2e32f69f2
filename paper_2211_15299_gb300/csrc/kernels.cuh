// Device kernels of the generalized radix-2 transform.
//
// Data flow (Corollary "block-structure", Algorithm 1 unrolled): with samples in
// sample order t and coefficients in canonical order, the transform is an
// in-place decimation-in-time network. Stage m (1..s) pairs positions t and
// t + 2^(m-1) inside every aligned block of 2^m and applies the butterfly
//   x[t] <- x[t] + w x[t + 2^(m-1)],   x[t + 2^(m-1)] <- x[t] - w x[t + 2^(m-1)]
// with w = tw_m[t mod 2^(m-1)] (Lemma "rec-hom-tree-split"). The final stage
// multiplies by N/k (eq. "hom-implies-spectral" with the 1/N of F^{-1} kept):
// its twiddles arrive pre-scaled and the other operand is scaled by an FMA.
//
// Tiles: 32 KiB of complex values staged by TMA into shared memory with the
// 128-byte swizzle (16-byte chunk index XOR row index mod 8). A thread owns 16
// elements whose tile index differs in 4 consecutive bits [B, B+4) and runs up
// to four stages on them in registers ("pass"); passes are separated by CTA
// barriers. With the swizzle every pass reads and writes shared memory without
// bank conflicts for complex64.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ptx.cuh"
#include "sdft.h"

namespace sdft {

template <class R> struct KT;
template <> struct KT<float> {
  using C = float2;
  static constexpr int ES = 8, CB = 4, TB = 12, NT = 256, SUB = 1;
};
template <> struct KT<double> {
  using C = double2;
  static constexpr int ES = 16, CB = 3, TB = 11, NT = 128, SUB = 0;
};

constexpr uint32_t kTileBytes = 32768;
constexpr uint32_t kLevelSmem = 3 * kTileBytes + 64 + 1024;   // 2 data tiles, twiddles, barriers, align

// ---- swizzled tile addressing -------------------------------------------------
// byte(T) = (T >> CB) * 128 + ((col_chunk(T) ^ (row(T) & 7)) << 4) + sub(T) * ES.
// For disjoint bit sets F (runtime) and E (constant) the offset of F|E splits
// into row_part(F) + row_part(E) + (xor_part(F) ^ xor_part(E)).
template <class R>
__host__ __device__ constexpr uint32_t row_part(uint32_t X) {
  return ((X >> KT<R>::CB) << 7) + (X & ((1u << KT<R>::SUB) - 1u)) * KT<R>::ES;
}
template <class R>
__host__ __device__ constexpr uint32_t xor_part(uint32_t X) {
  return (((X & ((1u << KT<R>::CB) - 1u)) >> KT<R>::SUB) ^ ((X >> KT<R>::CB) & 7u)) << 4;
}

// ---- butterflies -----------------------------------------------------------------
__device__ __forceinline__ void bfly(float2& a, float2& b, const float2 w) {
  const float tr = fmaf(-w.y, b.y, w.x * b.x);
  const float ti = fmaf(w.y, b.x, w.x * b.y);
  b.x = a.x - tr;
  b.y = a.y - ti;
  a.x = a.x + tr;
  a.y = a.y + ti;
}
__device__ __forceinline__ void bfly_scaled(float2& a, float2& b, const float2 w, const float sc) {
  const float tr = fmaf(-w.y, b.y, w.x * b.x);
  const float ti = fmaf(w.y, b.x, w.x * b.y);
  b.x = fmaf(a.x, sc, -tr);
  b.y = fmaf(a.y, sc, -ti);
  a.x = fmaf(a.x, sc, tr);
  a.y = fmaf(a.y, sc, ti);
}
__device__ __forceinline__ void bfly(double2& a, double2& b, const double2 w) {
  const double tr = fma(-w.y, b.y, w.x * b.x);
  const double ti = fma(w.y, b.x, w.x * b.y);
  b.x = a.x - tr;
  b.y = a.y - ti;
  a.x = a.x + tr;
  a.y = a.y + ti;
}
__device__ __forceinline__ void bfly_scaled(double2& a, double2& b, const double2 w, const double sc) {
  const double tr = fma(-w.y, b.y, w.x * b.x);
  const double ti = fma(w.y, b.x, w.x * b.y);
  b.x = fma(a.x, sc, -tr);
  b.y = fma(a.y, sc, -ti);
  a.x = fma(a.x, sc, tr);
  a.y = fma(a.y, sc, ti);
}

// ---- one pass: stages with stage bits [SLO, SHI) on 16 elements per thread --------
// The thread covers tile-index bits [B, B+4); its other bits come from tid.
// Twiddles live in shared memory indexed absolutely: stage bit m1, position u
// at entry 2^m1 + u.
template <class R, int B, int SLO, int SHI, bool SCALE, bool FENCE>
__device__ __forceinline__ void tile_pass(char* buf, const char* tws, uint32_t tid, R sc) {
  using C = typename KT<R>::C;
  static_assert(B >= 0 && B + 4 <= KT<R>::TB, "pass bits out of tile");
  static_assert(SLO >= B && SHI <= B + 4 && SLO < SHI, "stage bits out of pass");
  constexpr uint32_t LOWM = (1u << B) - 1u;
  const uint32_t F = (tid & LOWM) | ((tid >> B) << (B + 4));
  const uint32_t rF = row_part<R>(F), xF = xor_part<R>(F);
  C v[16];
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float4 t = *reinterpret_cast<const float4*>(buf + rF + (xF ^ (uint32_t(c) << 4)));
      v[2 * c] = make_float2(t.x, t.y);
      v[2 * c + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t E = uint32_t(e) << B;
      v[e] = *reinterpret_cast<const C*>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)));
    }
  }
  const char* twb = tws + (F & LOWM) * sizeof(C);
#pragma unroll
  for (int m1 = SLO; m1 < SHI; ++m1) {
    const int q = m1 - B;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if ((e >> q) & 1) continue;
      const int eh = e | (1 << q);
      const uint32_t uE = (uint32_t(e) << B) & ((1u << m1) - 1u);
      const C w = *reinterpret_cast<const C*>(twb + ((1u << m1) + uE) * sizeof(C));
      if (SCALE && m1 == SHI - 1)
        bfly_scaled(v[e], v[eh], w, sc);
      else
        bfly(v[e], v[eh], w);
    }
  }
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      *reinterpret_cast<float4*>(buf + rF + (xF ^ (uint32_t(c) << 4))) =
          make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
  } else {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t E = uint32_t(e) << B;
      *reinterpret_cast<C*>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E))) = v[e];
    }
  }
  if constexpr (FENCE) ptx::fence_proxy_async_smem();  // the tile leaves through TMA next
  __syncthreads();
}

// Stage bits [DONE, PHI) in passes of at most four; the pass covering them is
// the 4-bit window starting at DONE (or the top window of the tile).
template <class R, int PHI, bool LAST, int DONE>
__device__ __forceinline__ void run_passes(char* buf, const char* tws, uint32_t tid, R sc) {
  if constexpr (DONE < PHI) {
    constexpr int TB = KT<R>::TB;
    constexpr int B = (DONE + 4 <= TB) ? DONE : TB - 4;
    constexpr int SHI = (B + 4 < PHI) ? B + 4 : PHI;
    constexpr bool FINAL = (SHI == PHI);
    tile_pass<R, B, DONE, SHI, LAST && FINAL, FINAL>(buf, tws, tid, sc);
    run_passes<R, PHI, LAST, SHI>(buf, tws, tid, sc);
  }
}

// ---- persistent level kernel ----------------------------------------------------
// Tile i of a level: a = i / nB selects the twiddle table (a group block for
// later levels), b = i % nB; TMA coordinates {0, a*a_step1 + b*b_step1, 0, b*b_step3}.
struct LevelArgs {
  uint64_t n_tiles;
  uint64_t nB;
  int32_t a_step1, b_step1, b_step3;
  uint32_t tw_first;       // first absolute table entry present in a table
  const void* tw;          // tables of this level (device)
  uint64_t tw_len;         // entries per table
  uint64_t tw_stride;      // entries between consecutive tables (0: one shared table)
  double scale;            // N/k, used when LAST
  int* status;             // device status word
  uint64_t timeout_ns;     // bound on every mbarrier wait
};

__device__ __forceinline__ char* align1024(char* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t s = ptx::smem_addr(p);
  return reinterpret_cast<char*>(a + ((1024u - (s & 1023u)) & 1023u));
}

template <class R>
__device__ __forceinline__ void load_table(char* tws, const LevelArgs& args, uint64_t tab, uint32_t tid) {
  const uint4* src = reinterpret_cast<const uint4*>(static_cast<const char*>(args.tw) +
                                                    tab * args.tw_stride * sizeof(typename KT<R>::C));
  uint4* dst = reinterpret_cast<uint4*>(tws + uint64_t(args.tw_first) * sizeof(typename KT<R>::C));
  const uint32_t n16 = uint32_t(args.tw_len * sizeof(typename KT<R>::C) / 16);
  for (uint32_t j = tid; j < n16; j += KT<R>::NT) dst[j] = __ldg(src + j);
}

template <class R, int PLO, int PHI, bool LAST>
__global__ void __launch_bounds__(KT<R>::NT, 2)
    k_level(const __grid_constant__ CUtensorMap src, const __grid_constant__ CUtensorMap dst, const LevelArgs args) {
  extern __shared__ char smem_raw[];
  char* smem = align1024(smem_raw);
  char* tws = smem + 2 * kTileBytes;
  const uint32_t bar0 = ptx::smem_addr(smem + 3 * kTileBytes);
  const uint32_t tid = threadIdx.x;
  const uint64_t G = gridDim.x;
  const uint64_t t0 = args.n_tiles * blockIdx.x / G;
  const uint64_t t1 = args.n_tiles * (blockIdx.x + 1) / G;
  if (t0 >= t1) return;

  auto issue_load = [&](uint64_t i, uint32_t b) {
    const int64_t a = int64_t(i / args.nB), bb = int64_t(i % args.nB);
    const uint32_t bar = bar0 + 8 * b;
    ptx::mbar_arrive_expect_tx(bar, kTileBytes);
    ptx::tma_load_4d(ptx::smem_addr(smem + b * kTileBytes), &src, bar, 0,
                     int(a * args.a_step1 + bb * args.b_step1), 0, int(bb * args.b_step3));
  };

  if (tid == 0) {
    ptx::mbar_init(bar0, 1);
    ptx::mbar_init(bar0 + 8, 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&src);
    ptx::prefetch_tensormap(&dst);
    issue_load(t0, 0);
    if (t0 + 1 < t1) issue_load(t0 + 1, 1);
  }
  const R sc = R(args.scale);
  uint64_t cur_tab = ~0ull;
  bool aborted = false;
  uint64_t it = 0;
  for (uint64_t i = t0; i < t1; ++i, ++it) {
    const uint32_t b = uint32_t(it & 1);
    char* buf = smem + b * kTileBytes;
    const uint64_t tab = args.tw_stride ? i / args.nB : 0;
    if (tab != cur_tab) {
      load_table<R>(tws, args, tab, tid);
      cur_tab = tab;
    }
    const bool ok = ptx::mbar_wait_bounded(bar0 + 8 * b, uint32_t((it >> 1) & 1), args.timeout_ns);
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    run_passes<R, PHI, LAST, PLO>(buf, tws, tid, sc);
    if (tid == 0) {
      const int64_t a = int64_t(i / args.nB), bb = int64_t(i % args.nB);
      ptx::tma_store_4d(&dst, ptx::smem_addr(buf), 0, int(a * args.a_step1 + bb * args.b_step1), 0,
                        int(bb * args.b_step3));
      ptx::bulk_commit();
      if (i + 2 < t1) {
        ptx::bulk_wait_read<0>();
        issue_load(i + 2, b);
      }
    }
  }
  if (tid == 0) {
    if (aborted) {
      // Let copies already in flight land before the CTA's shared memory is released.
      // Pending loads: tile `it` (buffer it & 1) and tile it + 1 (the other buffer).
      for (uint64_t j = it; j < it + 2 && t0 + j < t1; ++j)
        ptx::mbar_wait_bounded(bar0 + 8 * uint32_t(j & 1), uint32_t((j >> 1) & 1), args.timeout_ns);
      atomicExch(args.status, int(SDFT_ERR_TIMEOUT));
    }
    ptx::bulk_wait<0>();
  }
}

// ---- register path for log2 k <= 4: one thread per instance ------------------------
template <class R, int S>
__global__ void __launch_bounds__(256) k_small(const typename KT<R>::C* __restrict__ in,
                                               typename KT<R>::C* __restrict__ out, uint64_t batch,
                                               const typename KT<R>::C* __restrict__ tw, R sc) {
  using C = typename KT<R>::C;
  constexpr int K = 1 << S;
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  C v[K];
#pragma unroll
  for (int e = 0; e < K; ++e) v[e] = in[i * K + e];
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
  for (int e = 0; e < K; ++e) out[i * K + e] = v[e];
}

}  // namespace sdft
