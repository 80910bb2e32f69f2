// Host launch of the level schedule for one plan and a packed batch, templated
// on the real type. Included once per precision (level_f32.cu, level_f64.cu).
#pragma once

#include "kernels.cuh"
#include "launch.hpp"

namespace sdft {

template <class R, int W, int PLO, int PHI, bool LAST, bool INV = false>
sdft_status launch_level(int grid, const CUtensorMap& src, const CUtensorMap& dst, const LevelArgs<R>& a,
                         cudaStream_t st) {
  auto fn = k_level<R, W, PLO, PHI, LAST, INV>;
  sdft_status s = ensure_smem(reinterpret_cast<const void*>(fn), int(kLevelSmem));
  if (s != SDFT_OK) return s;
  fn<<<grid, tile_threads<R, W>(), kLevelSmem, st>>>(src, dst, a);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

// Level 0: stage bits [0, PHI).
template <class R, int W, bool INV = false, int PHI = 5>
sdft_status dispatch_first_w(int phi, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                             const LevelArgs<R>& a, cudaStream_t st) {
  constexpr int TB = KT<R>::TB;
  if constexpr (PHI > TB) {
    return SDFT_ERR_UNSUPPORTED;
  } else {
    if (phi == PHI) {
      if constexpr (PHI == TB) {
        if (!last) return launch_level<R, W, 0, PHI, false, INV>(grid, src, dst, a, st);
      }
      if (!last) return SDFT_ERR_UNSUPPORTED;
      return launch_level<R, W, 0, PHI, true, INV>(grid, src, dst, a, st);
    }
    return dispatch_first_w<R, W, INV, PHI + 1>(phi, last, grid, src, dst, a, st);
  }
}

// Later levels: virtual stage bits [TB - Q, TB).
template <class R, int W, bool INV = false, int Q = 1>
sdft_status dispatch_later_w(int q, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                             const LevelArgs<R>& a, cudaStream_t st) {
  constexpr int TB = KT<R>::TB, CB = KT<R>::CB;
  if constexpr (Q > TB - CB) {
    return SDFT_ERR_UNSUPPORTED;
  } else {
    if (q == Q)
      return last ? launch_level<R, W, TB - Q, TB, true, INV>(grid, src, dst, a, st)
                  : launch_level<R, W, TB - Q, TB, false, INV>(grid, src, dst, a, st);
    return dispatch_later_w<R, W, INV, Q + 1>(q, last, grid, src, dst, a, st);
  }
}

// Stages per pass (W, 2^W values per thread): 4 everywhere; the forward
// complex64 level kernels also come with 3 (twice the threads per tile, one
// more pass), chosen per plan (sdft_plan_set_stages_per_pass, the autotuner).
// Those are compiled in a unit of their own (level_f32w3.cu).
template <class R, bool INV>
constexpr bool has_w3() { return std::is_same<R, float>::value && !INV; }
sdft_status dispatch_first_f32w3(int phi, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                                 const LevelArgs<float>& a, cudaStream_t st);
sdft_status dispatch_later_f32w3(int q, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                                 const LevelArgs<float>& a, cudaStream_t st);

template <class R, bool INV = false>
sdft_status dispatch_first(int w, int phi, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                           const LevelArgs<R>& a, cudaStream_t st) {
  if constexpr (has_w3<R, INV>()) {
    if (w == 3) return dispatch_first_f32w3(phi, last, grid, src, dst, a, st);
  }
  return dispatch_first_w<R, 4, INV>(phi, last, grid, src, dst, a, st);
}
template <class R, bool INV = false>
sdft_status dispatch_later(int w, int q, bool last, int grid, const CUtensorMap& src, const CUtensorMap& dst,
                           const LevelArgs<R>& a, cudaStream_t st) {
  if constexpr (has_w3<R, INV>()) {
    if (w == 3) return dispatch_later_f32w3(q, last, grid, src, dst, a, st);
  }
  return dispatch_later_w<R, 4, INV>(q, last, grid, src, dst, a, st);
}

template <class R, int S = 0>
sdft_status dispatch_small(int s, uint64_t batch, const void* in, void* out, const void* tw, double scale,
                           cudaStream_t st) {
  using C = typename KT<R>::C;
  if constexpr (S > int(kSmallMax)) {
    return SDFT_ERR_UNSUPPORTED;
  } else {
    if (s == S) {
      const uint64_t blocks = (batch + 255) / 256;
      if (blocks > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
      k_small<R, S><<<unsigned(blocks), 256, 0, st>>>(static_cast<const C*>(in), static_cast<C*>(out), batch,
                                                      static_cast<const C*>(tw), R(scale));
      const cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
    }
    return dispatch_small<R, S + 1>(s, batch, in, out, tw, scale, st);
  }
}

// A table entry built on the host (kernel parameters), and the device table
// the level kernels of a real type read.
template <class R> inline typename KT<R>::C host_c(double re, double im);
template <> inline float2 host_c<float>(double re, double im) { return make_float2(float(re), float(im)); }
template <> inline double2 host_c<double>(double re, double im) { return make_double2(re, im); }
template <> inline dfc host_c<dfloat>(double re, double im) {
  dfc r;
  r.hi = make_float2(float(re), float(im));
  r.lo = make_float2(float(re - double(r.hi.x)), float(im - double(r.hi.y)));
  return r;
}
template <class R> inline const void* level_table(const Plan& p) {
  return std::is_same<R, dfloat>::value ? p.d_tw_df : p.d_tw;
}

// Tensor maps and kernel arguments of level 0 (stage bits [0, min(s, TB)) on
// contiguous tiles of 2^TB elements) over the packed buffers (src, dst).
template <class R>
sdft_status level0_setup(const Plan& p, uint64_t batch, const void* src, void* dst, CUtensorMap& ms,
                         CUtensorMap& md, LevelArgs<R>& a) {
  using C = typename KT<R>::C;
  constexpr int TB = KT<R>::TB, CB = KT<R>::CB;
  const Level& L = p.levels[0];
  const uint64_t rows_per_tile = 1ull << (TB - CB);
  const uint64_t rows = (batch * p.k) >> CB;
  const uint64_t n_tiles = (rows + rows_per_tile - 1) / rows_per_tile;
  if (rows > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
  const uint64_t dims[4] = {32, rows, 1, 1};
  const uint64_t strides[3] = {128, rows * 128, rows * 128};
  const uint32_t box[4] = {32, uint32_t(rows_per_tile), 1, 1};
  sdft_status s = encode_map(&ms, src, dims, strides, box);
  if (s == SDFT_OK) s = encode_map(&md, dst, dims, strides, box);
  if (s != SDFT_OK) return s;
  a = LevelArgs<R>{};
  for (int i = 0; i < 15; ++i) a.tw0[i] = host_c<R>(p.tw0[2 * i], p.tw0[2 * i + 1]);
  a.n_tiles = n_tiles;
  a.nB = n_tiles;
  a.a_step1 = 0;
  a.b_step1 = int32_t(rows_per_tile);
  a.b_step3 = 0;
  a.tw_first = 0;
  a.tw = static_cast<const C*>(level_table<R>(p)) + L.tw_off;
  a.tw_len = L.tw_len;
  a.tw_stride = 0;
  a.scale = std::ldexp(1.0, int(p.M) - int(p.s));
  a.inv_n = std::ldexp(1.0, -int(p.M));
  a.status = p.d_status;
  a.timeout_ns = wait_timeout_ns();
  a.lim1 = int64_t(rows);
  a.lim3 = 1;
  a.tw_tables = 1;
  return SDFT_OK;
}

// Instances (row blocks) per chunk of a later level's tile walk: a CTA keeps a
// group block's twiddle table for this many consecutive tiles.
constexpr uint64_t kLaterChunk = 8;

// Tensor maps and kernel arguments of later level j (stage bits [lo, hi) on
// group blocks: 2^lg column groups x 2^Q rows spaced 2^lo elements apart).
template <class R>
sdft_status later_setup(const Plan& p, uint64_t batch, size_t j, const void* src, void* dst, CUtensorMap& ms,
                        CUtensorMap& md, LevelArgs<R>& a) {
  using C = typename KT<R>::C;
  constexpr int CB = KT<R>::CB, ES = KT<R>::ES;
  const Level& L = p.levels[j];
  const uint32_t Q = L.hi - L.lo;
  const uint64_t Z = batch << (p.s - L.hi);
  if (Z > 0x7fffffffull || (1ull << (L.lo - CB)) > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
  const uint64_t dims[4] = {32, 1ull << (L.lo - CB), 1ull << Q, Z};
  const uint64_t strides[3] = {128, (1ull << L.lo) * ES, (1ull << L.hi) * ES};
  const uint32_t box[4] = {32, 1u << L.lg, 1u << Q, 1};
  sdft_status s = encode_map(&ms, src, dims, strides, box);
  if (s == SDFT_OK) s = encode_map(&md, dst, dims, strides, box);
  if (s != SDFT_OK) return s;
  a = LevelArgs<R>{};
  for (int i = 0; i < 15; ++i) a.tw0[i] = host_c<R>(p.tw0[2 * i], p.tw0[2 * i + 1]);
  a.n_tiles = L.n_gb * Z;
  a.nB = Z;
  a.a_step1 = int32_t(1u << L.lg);
  a.b_step1 = 0;
  a.b_step3 = 1;
  a.tw_first = 1u << L.plo;
  a.tw = static_cast<const C*>(level_table<R>(p)) + L.tw_off;
  a.tw_len = L.tw_len;
  a.tw_stride = L.tw_len;
  a.scale = std::ldexp(1.0, int(p.M) - int(p.s));
  a.inv_n = std::ldexp(1.0, -int(p.M));
  a.status = p.d_status;
  a.timeout_ns = wait_timeout_ns();
  a.lim1 = int64_t(1) << (L.lo - CB);
  a.lim3 = int64_t(Z);
  a.tw_tables = L.n_gb;
  a.chunk = kLaterChunk;
  return SDFT_OK;
}

inline int level_grid(uint64_t n_tiles) {
  const uint64_t max_grid = 2ull * uint64_t(sm_count());
  return int(n_tiles < max_grid ? n_tiles : max_grid);
}

// Small batches of 2^5 <= k <= 2^10 (at most kWarpMaxElems values in all): one
// warp per instance (k_warp) instead of a TMA-fed tile.
constexpr uint64_t kWarpMaxElems = 1ull << 14;

template <class R, int S = 5>
sdft_status dispatch_warp(int s, uint64_t batch, const void* in, void* out, const void* tw, double scale,
                          cudaStream_t st) {
  using C = typename KT<R>::C;
  if constexpr (S > 10) {
    return SDFT_ERR_UNSUPPORTED;
  } else {
    if (s == S) {
      const uint64_t blocks = (batch * 32 + 127) / 128;
      k_warp<R, S><<<unsigned(blocks), 128, 0, st>>>(static_cast<const C*>(in), static_cast<C*>(out), batch,
                                                     static_cast<const C*>(tw), R(scale));
      const cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
    }
    return dispatch_warp<R, S + 1>(s, batch, in, out, tw, scale, st);
  }
}

// Small batches of 2^5 <= k <= 2^10 take the warp path.
inline bool warp_path(const Plan& p, uint64_t batch) {
  return p.levels.size() == 1 && p.s >= 5 && p.s <= 10 && batch * p.k <= kWarpMaxElems;
}

template <class R>
sdft_status launch_plan(const Plan& p, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  const double scale = std::ldexp(1.0, int(p.M) - int(p.s));
  if constexpr (std::is_same<R, dfloat>::value) {
    if (p.levels.empty()) return SDFT_ERR_UNSUPPORTED;     // the caller runs these in FP64
  } else {
    if (p.levels.empty()) return dispatch_small<R>(int(p.s), batch, in, out, p.d_tw, scale, st);
    if (warp_path(p, batch))
      return dispatch_warp<R>(int(p.s), batch, in, out,
                              static_cast<const typename KT<R>::C*>(p.d_tw) + p.levels[0].tw_off, scale, st);
  }
  // Level 0 on contiguous tiles.
  {
    CUtensorMap ms, md;
    LevelArgs<R> a;
    sdft_status s = level0_setup<R>(p, batch, in, out, ms, md, a);
    if (s != SDFT_OK) return s;
    s = dispatch_first<R>(int(p.spp), int(p.levels[0].hi), p.levels[0].last, level_grid(a.n_tiles), ms, md, a, st);
    if (s != SDFT_OK) return s;
  }
  // Later levels in place on the output.
  for (size_t j = 1; j < p.levels.size(); ++j) {
    const Level& L = p.levels[j];
    CUtensorMap m, m2;
    LevelArgs<R> a;
    sdft_status s = later_setup<R>(p, batch, j, out, out, m, m2, a);
    if (s != SDFT_OK) return s;
    s = dispatch_later<R>(int(p.spp), int(L.hi - L.lo), L.last, level_grid(a.n_tiles), m, m, a, st);
    if (s != SDFT_OK) return s;
  }
  return SDFT_OK;
}

template <class R, int S = 0>
sdft_status dispatch_small_inv(int s, uint64_t batch, const void* in, void* out, const void* tw, double sc_top,
                               double sc_fin, cudaStream_t st) {
  using C = typename KT<R>::C;
  if constexpr (S > int(kSmallMax)) {
    return SDFT_ERR_UNSUPPORTED;
  } else {
    if (s == S) {
      const uint64_t blocks = (batch + 255) / 256;
      if (blocks > 0x7fffffffull) return SDFT_ERR_UNSUPPORTED;
      k_small_inv<R, S><<<unsigned(blocks), 256, 0, st>>>(static_cast<const C*>(in), static_cast<C*>(out), batch,
                                                          static_cast<const C*>(tw), R(sc_top), R(sc_fin));
      const cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
    }
    return dispatch_small_inv<R, S + 1>(s, batch, in, out, tw, sc_top, sc_fin, st);
  }
}

// Synthesis (the adjoint network scaled by 1/N): the levels in reverse order,
// each running its passes in reverse. The first level applied reads `in`, the
// others work in place on `out`.
template <class R>
sdft_status launch_plan_inv(const Plan& p, uint64_t batch, const void* in, void* out, cudaStream_t st) {
  const double scale = std::ldexp(1.0, int(p.M) - int(p.s));
  const double inv_n = std::ldexp(1.0, -int(p.M));
  if constexpr (std::is_same<R, dfloat>::value) {
    if (p.levels.empty()) return SDFT_ERR_UNSUPPORTED;     // the caller runs these in FP64
  } else {
    if (p.levels.empty()) return dispatch_small_inv<R>(int(p.s), batch, in, out, p.d_tw, 1.0 / scale, inv_n, st);
  }
  // Later levels first (last one first), the first reading `in`, then level 0.
  const void* src_base = in;
  for (size_t j = p.levels.size() - 1; j >= 1; --j) {
    const Level& L = p.levels[j];
    CUtensorMap ms, md;
    LevelArgs<R> a;
    sdft_status s = later_setup<R>(p, batch, j, src_base, out, ms, md, a);
    if (s != SDFT_OK) return s;
    s = dispatch_later<R, true>(4, int(L.hi - L.lo), L.last, level_grid(a.n_tiles), ms, md, a, st);
    if (s != SDFT_OK) return s;
    src_base = out;
  }
  CUtensorMap ms, md;
  LevelArgs<R> a;
  sdft_status s = level0_setup<R>(p, batch, src_base, out, ms, md, a);
  if (s != SDFT_OK) return s;
  return dispatch_first<R, true>(4, int(p.levels[0].hi), p.levels[0].last, level_grid(a.n_tiles), ms, md, a, st);
}

}  // namespace sdft
