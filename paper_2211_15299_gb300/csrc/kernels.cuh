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
// 128-byte swizzle (16-byte chunk index XOR row index mod 8). A thread owns 2^W
// elements (W = 4 or 3) whose tile index differs in W consecutive bits [B, B+W)
// and runs up to W stages on them in registers ("pass"); passes are separated by
// CTA barriers. With the swizzle the address pattern of every pass maps each
// warp access onto the minimum number of shared-memory wavefronts for complex64
// (16-byte accesses in the first pass, 8-byte ones after). The extra wavefronts
// ncu still counts as bank conflicts on these accesses (about a fifth) are all
// of the arbitration type (l1tex__data_bank_conflicts_type_arbitration): the
// tile loads and stores of the TMA engine use the same banks at the same time.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include <type_traits>

#include "ptx.cuh"
#include "sdft.h"

// Debug build with range checks (compiled with -DSDFT_BOUNDS_CHECK=1, see
// build.py): every TMA tile coordinate, twiddle-table range and work-queue
// record is checked against the extent it must lie in before it is used. A
// violation adds one to a device counter, records kBadBounds in the status word
// and makes the access harmless (coordinate 0, entry range of table 0); no
// kernel traps. sdft_debug_bounds_violations reads (and clears) the counts.
#ifndef SDFT_BOUNDS_CHECK
#define SDFT_BOUNDS_CHECK 0
#endif

namespace sdft {

constexpr int kBadBounds = 0x105;     // status: a range check of the debug build failed

#if SDFT_BOUNDS_CHECK
// One counter per translation unit (a static device variable of this header);
// each registers a host reader of its own copy when the library loads.
static __device__ unsigned long long g_bounds_violations = 0;
void register_violation_reader(uint64_t (*reader)(int clear));
namespace {
inline uint64_t read_violations_here(int clear) {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_violations, sizeof(v)) != cudaSuccess) return ~0ull;
  if (clear) {
    const unsigned long long z = 0;
    cudaMemcpyToSymbol(g_bounds_violations, &z, sizeof(z));
  }
  return v;
}
struct ViolationReaderRegistration {
  ViolationReaderRegistration() { register_violation_reader(&read_violations_here); }
};
static ViolationReaderRegistration g_violation_reader_registration;
}  // namespace
#endif

// `ok` false: count a violation (debug build) and record it in `status`.
// Returns `ok` in the debug build and true otherwise (the check compiles away).
__device__ __forceinline__ bool in_bounds(bool ok, int* status) {
#if SDFT_BOUNDS_CHECK
  if (!ok) {
    atomicAdd(&g_bounds_violations, 1ull);
    if (status) atomicCAS(status, 0, kBadBounds);
  }
  return ok;
#else
  (void)ok;
  (void)status;
  return true;
#endif
}

template <class R> struct KT;
template <> struct KT<float> {
  using C = float2;
  static constexpr int ES = 8, CB = 4, TB = 12, NT = 256, SUB = 1;
};
template <> struct KT<double> {
  using C = double2;
  static constexpr int ES = 16, CB = 3, TB = 11, NT = 128, SUB = 0;
};

// Double-float arithmetic for complex128 data: a value is an unevaluated sum
// hi + lo of two FP32 numbers (48-bit significand, FP32 exponent range), so the
// butterflies run on the FP32 pipes. `dfloat` is the real-type tag (a scale
// factor, always a power of two) and `dfc` a complex value: hi = (re, im) high
// parts, lo = (re, im) low parts. Tiles and tables keep 16 bytes per value, as
// complex128 does.
struct dfloat {
  float v;
  __host__ __device__ constexpr dfloat(double x = 0.0) : v(float(x)) {}
};
__host__ __device__ inline dfloat operator*(dfloat a, dfloat b) { return dfloat(double(a.v) * double(b.v)); }
struct __align__(16) dfc {
  float2 hi, lo;
};
template <> struct KT<dfloat> {
  using C = dfc;
  static constexpr int ES = 16, CB = 3, TB = 11, NT = 128, SUB = 0;
};

constexpr uint32_t kTileBytes = 32768;

// Launch self-check failures recorded in the device status word (see sdft.h:
// values above 255 are launch-check codes, below are sdft_status values).
constexpr int kBadSmem = 0x101;   // less dynamic shared memory than the layout needs
constexpr int kBadMap = 0x102;    // tensor map parameter not 64-byte aligned
constexpr int kBadTable = 0x103;  // twiddle table not 16-byte aligned
// Bound on the wait for a CTA's own copies already in flight after a failed
// wait: an issued copy lands within microseconds on a working GPU, so this
// bound is generous and independent of the (possibly short) bound whose expiry
// caused the abort; the CTA only releases its shared memory once they landed.
constexpr uint64_t kDrainNs = 2000000000ull;
__host__ __device__ constexpr uint64_t drain_bound(uint64_t t) { return t > kDrainNs ? t : kDrainNs; }
// Tile buffers per level-kernel CTA. Two keep the level kernel at the speed of a
// copy-only variant of itself (TMA in and out, no passes) on the 2^12-point
// batches, and leave more of the SM's combined L1/shared storage to the L1 cache
// that serves the table reads of later levels.
constexpr int kLevelBufs = 2;
// Shared-memory copy of the middle pass's table region (entries [16, 256),
// absolute-indexed) for the level kernel.
constexpr uint32_t kMidTwBytes = 256 * 16;
constexpr uint32_t kLevelSmem = kLevelBufs * kTileBytes + 64 + kMidTwBytes + 1024;   // tiles, barriers, table, slack

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
// Three fused multiply-adds per output component pair: the first output
// a' = a + w b takes two chained FMAs per component (the twiddle product is
// never rounded on its own), the second is b' = 2a - a' (one FMA per component,
// 2a exact). Six FMA-pipe operations per butterfly instead of eight for a
// separate product and two sums; b' carries a''s rounding error, so both
// outputs stay within a few units in the last place of max(|a|, |w b|).
__device__ __forceinline__ void bfly(float2& a, float2& b, const float2 w) {
  float2 n;
  n.x = fmaf(w.x, b.x, fmaf(-w.y, b.y, a.x));
  n.y = fmaf(w.x, b.y, fmaf(w.y, b.x, a.y));
  b.x = fmaf(2.f, a.x, -n.x);
  b.y = fmaf(2.f, a.y, -n.y);
  a = n;
}
// The last stage: both outputs scaled by sc (a power of two: exact); the
// twiddles arrive pre-scaled, so only a is scaled here.
__device__ __forceinline__ void bfly_scaled(float2& a, float2& b, const float2 w, const float sc) {
  const float2 as = __fmul2_rn(a, make_float2(sc, sc));
  float2 n;
  n.x = fmaf(w.x, b.x, fmaf(-w.y, b.y, as.x));
  n.y = fmaf(w.x, b.y, fmaf(w.y, b.x, as.y));
  b.x = fmaf(2.f, as.x, -n.x);
  b.y = fmaf(2.f, as.y, -n.y);
  a = n;
}
__device__ __forceinline__ void bfly(double2& a, double2& b, const double2 w) {
  const double nx = fma(w.x, b.x, fma(-w.y, b.y, a.x));
  const double ny = fma(w.x, b.y, fma(w.y, b.x, a.y));
  b.x = fma(2.0, a.x, -nx);
  b.y = fma(2.0, a.y, -ny);
  a.x = nx;
  a.y = ny;
}
__device__ __forceinline__ void bfly_scaled(double2& a, double2& b, const double2 w, const double sc) {
  const double ax = a.x * sc, ay = a.y * sc;
  const double nx = fma(w.x, b.x, fma(-w.y, b.y, ax));
  const double ny = fma(w.x, b.y, fma(w.y, b.x, ay));
  b.x = fma(2.0, ax, -nx);
  b.y = fma(2.0, ay, -ny);
  a.x = nx;
  a.y = ny;
}

// Adjoint butterflies (synthesis): (a, b) -> (a + b, conj(w) (a - b)); the
// scaled form multiplies the first output by ga and the second by gb, both
// powers of two (exact).
__device__ __forceinline__ void ibfly(float2& a, float2& b, const float2 w) {
  const float2 d = __ffma2_rn(b, make_float2(-1.f, -1.f), a);   // a - b
  a = __fadd2_rn(a, b);
  b.x = fmaf(w.y, d.y, w.x * d.x);
  b.y = fmaf(-w.y, d.x, w.x * d.y);
}
__device__ __forceinline__ void ibfly_scaled(float2& a, float2& b, float2 w, const float ga, const float gb) {
  w.x *= gb;
  w.y *= gb;
  const float2 d = __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  a = __fmul2_rn(__fadd2_rn(a, b), make_float2(ga, ga));
  b.x = fmaf(w.y, d.y, w.x * d.x);
  b.y = fmaf(-w.y, d.x, w.x * d.y);
}
__device__ __forceinline__ void ibfly(double2& a, double2& b, const double2 w) {
  const double dx = a.x - b.x, dy = a.y - b.y;
  a.x = a.x + b.x;
  a.y = a.y + b.y;
  b.x = fma(w.y, dy, w.x * dx);
  b.y = fma(-w.y, dx, w.x * dy);
}
__device__ __forceinline__ void ibfly_scaled(double2& a, double2& b, double2 w, const double ga, const double gb) {
  w.x *= gb;
  w.y *= gb;
  const double dx = a.x - b.x, dy = a.y - b.y;
  a.x = (a.x + b.x) * ga;
  a.y = (a.y + b.y) * ga;
  b.x = fma(w.y, dy, w.x * dx);
  b.y = fma(-w.y, dx, w.x * dy);
}

// ---- double-float butterflies ---------------------------------------------------
// Knuth's TwoSum (s + e = a + b exactly), Dekker's FastTwoSum (|a| >= |b|) and the
// FMA form of Dekker's TwoProduct; sums and products of hi + lo pairs renormalised
// by FastTwoSum (the "sloppy" double-float addition, whose error is bounded by a
// small multiple of 2^-48 (|x| + |y|), the bound a normwise FFT analysis uses).
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {   // (hi, lo) + (hi, lo)
  const float2 s = df_two_sum(x.x, y.x);
  return df_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_re(const dfc& v) { return make_float2(v.hi.x, v.lo.x); }
__device__ __forceinline__ float2 df_im(const dfc& v) { return make_float2(v.hi.y, v.lo.y); }
__device__ __forceinline__ dfc df_make(float2 re, float2 im) {
  dfc r;
  r.hi = make_float2(re.x, im.x);
  r.lo = make_float2(re.y, im.y);
  return r;
}
__device__ __forceinline__ dfc df_scale(const dfc& v, float s) {   // s a power of two: exact
  dfc r;
  r.hi = make_float2(v.hi.x * s, v.hi.y * s);
  r.lo = make_float2(v.lo.x * s, v.lo.y * s);
  return r;
}
// Packed forms: the real and imaginary parts travel together as FP32x2 pairs
// (hi = (re, im), lo = (re, im)), so one packed instruction serves both; the
// same steps as above, lane by lane.
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ dfc dfc_add(const dfc& x, const dfc& y) {
  const float2 s = __fadd2_rn(x.hi, y.hi);                  // TwoSum on the high parts
  const float2 bb = p_sub(s, x.hi);
  float2 e = __fadd2_rn(p_sub(x.hi, p_sub(s, bb)), p_sub(y.hi, bb));
  e = __fadd2_rn(e, __fadd2_rn(x.lo, y.lo));
  dfc r;                                                    // FastTwoSum renormalisation
  r.hi = __fadd2_rn(s, e);
  r.lo = p_sub(e, p_sub(r.hi, s));
  return r;
}
__device__ __forceinline__ dfc dfc_flip(const dfc& x, float2 sgn) {   // lane signs (+-1): exact
  dfc r;
  r.hi = __fmul2_rn(x.hi, sgn);
  r.lo = __fmul2_rn(x.lo, sgn);
  return r;
}
// (xr, xr) * (y.re, y.im) for a double-float scalar xr = (xh, xl) and complex y
__device__ __forceinline__ dfc dfc_scalar_mul(float xh, float xl, const dfc& y) {
  const float2 xh2 = make_float2(xh, xh), xl2 = make_float2(xl, xl);
  const float2 p = __fmul2_rn(xh2, y.hi);
  float2 e = __ffma2_rn(xh2, y.hi, __fmul2_rn(p, make_float2(-1.f, -1.f)));   // TwoProduct error
  e = __ffma2_rn(xh2, y.lo, e);
  e = __ffma2_rn(xl2, y.hi, e);
  dfc r;
  r.hi = __fadd2_rn(p, e);
  r.lo = p_sub(e, p_sub(r.hi, p));
  return r;
}
__device__ __forceinline__ dfc dfc_swap(const dfc& y) {
  dfc r;
  r.hi = make_float2(y.hi.y, y.hi.x);
  r.lo = make_float2(y.lo.y, y.lo.x);
  return r;
}
// t = w b (complex); then (a, b) <- (a + t, a - t)
__device__ __forceinline__ void df_bfly_core(dfc& a, dfc& b, const dfc& w) {
  // w b = wr (br, bi) + wi (-bi, br)
  const dfc A = dfc_scalar_mul(w.hi.x, w.lo.x, b);
  const dfc B = dfc_flip(dfc_scalar_mul(w.hi.y, w.lo.y, dfc_swap(b)), make_float2(-1.f, 1.f));
  const dfc t = dfc_add(A, B);
  b = dfc_add(a, dfc_flip(t, make_float2(-1.f, -1.f)));
  a = dfc_add(a, t);
}
__device__ __forceinline__ void bfly(dfc& a, dfc& b, const dfc w) { df_bfly_core(a, b, w); }
__device__ __forceinline__ void bfly_scaled(dfc& a, dfc& b, const dfc w, const dfloat sc) {
  a = df_scale(a, sc.v);
  df_bfly_core(a, b, w);
}
// adjoint: (a, b) -> (ga (a + b), gb conj(w) (a - b)); conj(w) d = wr (dr, di) + wi (di, -dr)
__device__ __forceinline__ void df_ibfly_core(dfc& a, dfc& b, const dfc& w, float ga, float gb) {
  const dfc d = dfc_add(a, dfc_flip(b, make_float2(-1.f, -1.f)));
  a = df_scale(dfc_add(a, b), ga);
  const dfc A = dfc_scalar_mul(w.hi.x, w.lo.x, d);
  const dfc B = dfc_flip(dfc_scalar_mul(w.hi.y, w.lo.y, dfc_swap(d)), make_float2(1.f, -1.f));
  b = df_scale(dfc_add(A, B), gb);
}
__device__ __forceinline__ void ibfly(dfc& a, dfc& b, const dfc w) { df_ibfly_core(a, b, w, 1.f, 1.f); }
__device__ __forceinline__ void ibfly_scaled(dfc& a, dfc& b, dfc w, const dfloat ga, const dfloat gb) {
  df_ibfly_core(a, b, w, ga.v, gb.v);
}

// ---- double <-> double-float by bit operations --------------------------------------
// The conversions stay off the FP64 pipe (a few integer operations, one integer
// to FP32 conversion, two FP32 multiplies; the join adds in FP64 once).
// Split: hi = x with its significand cut to 24 bits (exact), lo = RN(x - hi)
// from the 29 dropped bits, an integer times 2^(e - 52). |x| < 2^-126 gives
// 0 + 0; |x| >= 2^128, infinities and NaN give a signed infinity.
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const uint32_t hw = uint32_t(b >> 32), lw = uint32_t(b);
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t e = (hw >> 20) & 0x7ffu;                       // biased exponent of x
  if (e < 897u) return make_float2(0.f, 0.f);
  if (e > 1150u) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const uint32_t frac23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const uint32_t pow_bits = (e - 896u) << 23;                    // 2^(e - 1023) as FP32
  const float hi = __uint_as_float(sign | pow_bits | frac23);
  const float rem = __uint2float_rn(lw & 0x1fffffffu);           // 29 bits, rounded to 24
  const float lo = __fmul_rn(__fmul_rn(rem, 2.220446049250313e-16f), __uint_as_float(pow_bits));   // 2^-52
  return make_float2(hi, sign ? -lo : lo);
}
// An FP32 value as FP64 (exact); zero and subnormals give 0, inf/NaN keep their kind.
__device__ __forceinline__ double df_f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e8 = (u >> 23) & 0xffu;
  const uint32_t sign = u & 0x80000000u;
  if (e8 == 0u) return __hiloint2double(int(sign), 0);
  const uint32_t e11 = (e8 == 0xffu) ? 0x7ffu : e8 + 896u;
  return __hiloint2double(int(sign | (e11 << 20) | ((u & 0x7fffffu) >> 3)), int((u & 0x7u) << 29));
}
__device__ __forceinline__ double df_join(float hi, float lo) { return __dadd_rn(df_f2d(hi), df_f2d(lo)); }

// ---- element and table access ------------------------------------------------------
// Tile elements: as stored, except that a double-float pass reads complex128
// values (RAW) when it is the first pass of the plan's first level (the samples
// as the caller gave them) and writes complex128 from the last pass of its last
// level; between levels the split values go through HBM as they are (16 bytes
// per value, as complex128).
template <class R, bool RAW>
__device__ __forceinline__ typename KT<R>::C load_elem(const char* p) {
  if constexpr (std::is_same<R, dfloat>::value && RAW) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    const float2 re = df_split(x.x), im = df_split(x.y);
    return df_make(re, im);
  } else {
    return *reinterpret_cast<const typename KT<R>::C*>(p);
  }
}
template <class R, bool RAW>
__device__ __forceinline__ void store_elem(char* p, const typename KT<R>::C& v) {
  if constexpr (std::is_same<R, dfloat>::value && RAW) {
    *reinterpret_cast<double2*>(p) = make_double2(df_join(v.hi.x, v.lo.x), df_join(v.hi.y, v.lo.y));
  } else {
    *reinterpret_cast<typename KT<R>::C*>(p) = v;
  }
}
// A table entry through the read-only path.
__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dfc ldg_c(const dfc* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  dfc r;
  r.hi = make_float2(t.x, t.y);
  r.lo = make_float2(t.z, t.w);
  return r;
}

// ---- pass schedule ------------------------------------------------------------------
// Stage bits [PLO, PHI) of a tile run in passes of W stage bits (2^W elements
// per thread). Pass p covers the W-bit window starting at the first stage bit
// not yet done (or the top window of the tile) and runs the stages of that
// window that are still pending.
constexpr int pass_done(int TB, int W, int PLO, int PHI, int p) {
  int d = PLO;
  for (int i = 0; i < p; ++i) {
    const int b = (d + W <= TB) ? d : TB - W;
    d = (b + W < PHI) ? b + W : PHI;
  }
  return d;
}
constexpr int pass_b(int TB, int W, int PLO, int PHI, int p) {
  const int d = pass_done(TB, W, PLO, PHI, p);
  return (d + W <= TB) ? d : TB - W;
}
constexpr int pass_shi(int TB, int W, int PLO, int PHI, int p) {
  const int b = pass_b(TB, W, PLO, PHI, p);
  return (b + W < PHI) ? b + W : PHI;
}
constexpr int n_passes(int TB, int W, int PLO, int PHI) {
  int p = 0;
  while (pass_done(TB, W, PLO, PHI, p) < PHI) ++p;
  return p;
}
// Distinct twiddles a thread needs in one pass: stage bit m1 uses 2^(m1-B).
constexpr int pass_ntw(int B, int SLO, int SHI) {
  int n = 0;
  for (int m1 = SLO; m1 < SHI; ++m1) n += 1 << (m1 - B);
  return n;
}
// Twiddle sources per pass: a B = 0 pass (the same 2^W - 1 entries for every
// thread) reads kernel parameters; the top pass (B = TB - W, the largest table
// region) holds its entries in registers across tiles; any other pass reads its
// table region through the L1 cache, or (level kernel) from a shared-memory
// copy made when the table changes.
enum TwSrc { kTwParam = 0, kTwReg = 1, kTwGlobal = 2, kTwShared = 3 };
constexpr int pass_src(int TB, int W, int B) { return B == 0 ? kTwParam : (B == TB - W ? kTwReg : kTwGlobal); }
constexpr int reg_twiddles(int TB, int W, int PLO, int PHI) {
  int n = 0;
  for (int p = 0; p < n_passes(TB, W, PLO, PHI); ++p) {
    const int b = pass_b(TB, W, PLO, PHI, p);
    if (pass_src(TB, W, b) == kTwReg) n += pass_ntw(b, pass_done(TB, W, PLO, PHI, p), pass_shi(TB, W, PLO, PHI, p));
  }
  return n;
}
// Threads per tile: one per 2^W elements.
template <class R, int W>
constexpr uint32_t tile_threads() { return 1u << (KT<R>::TB - W); }

// One complex value from shared memory (byte address).
template <class R>
__device__ __forceinline__ typename KT<R>::C ld_shared_c(uint32_t addr);
template <>
__device__ __forceinline__ float2 ld_shared_c<float>(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
template <>
__device__ __forceinline__ double2 ld_shared_c<double>(uint32_t addr) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
  return v;
}
template <>
__device__ __forceinline__ dfc ld_shared_c<dfloat>(uint32_t addr) {
  dfc v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.hi.x), "=f"(v.hi.y), "=f"(v.lo.x), "=f"(v.lo.y)
               : "r"(addr)
               : "memory");
  return v;
}

// Stage range [lo, hi) covered by the passes that read their twiddles from
// memory (neither kernel parameters nor registers): lo of the first, hi of the
// last; {0, 0} if there is none.
constexpr int mid_pass_lo(int TB, int W, int PLO, int PHI) {
  for (int p = 0; p < n_passes(TB, W, PLO, PHI); ++p)
    if (pass_src(TB, W, pass_b(TB, W, PLO, PHI, p)) == kTwGlobal) return pass_done(TB, W, PLO, PHI, p);
  return 0;
}
constexpr int mid_pass_hi(int TB, int W, int PLO, int PHI) {
  int hi = 0;
  for (int p = 0; p < n_passes(TB, W, PLO, PHI); ++p)
    if (pass_src(TB, W, pass_b(TB, W, PLO, PHI, p)) == kTwGlobal) hi = pass_shi(TB, W, PLO, PHI, p);
  return hi;
}

// ---- one pass: stages with stage bits [SLO, SHI) on 2^W elements per thread -------
// The thread covers tile-index bits [B, B+W); its other bits (F) come from tid.
// Stage bit m1 on the element pair (e, e | 2^q), q = m1 - B, uses the table
// entry 2^m1 + u with u = (F mod 2^B) + ((e mod 2^q) << B); `w` holds exactly
// those entries in order (m1 ascending, then e mod 2^q).
// SRC = kTwParam / kTwReg: `w` holds exactly the pass's entries in order
// (m1 ascending, then e mod 2^q). SRC = kTwGlobal: `w` is the absolute-indexed
// table in global memory. SRC = kTwShared: `wsm` is the shared-memory address of
// the absolute-indexed table region.
// BAR = 1: the pass ends with named barrier 1 over the NT compute threads
// instead of a CTA barrier (a kernel with a separate producer warp).
template <class R, int W, int B, int SLO, int SHI, bool SCALE, bool FENCE, int SRC, int BAR = 0, bool FIRST = false,
          bool RAWOUT = false>
__device__ __forceinline__ void tile_pass(char* buf, const typename KT<R>::C* w, uint32_t tid, R sc,
                                          uint32_t wsm = 0) {
  using C = typename KT<R>::C;
  static_assert(B >= 0 && B + W <= KT<R>::TB, "pass bits out of tile");
  static_assert(SLO >= B && SHI <= B + W && SLO < SHI, "stage bits out of pass");
  constexpr uint32_t LOWM = (1u << B) - 1u;
  constexpr int NE = 1 << W;
  const uint32_t F = (tid & LOWM) | ((tid >> B) << (B + W));
  const uint32_t rF = row_part<R>(F), xF = xor_part<R>(F);
  C v[NE];
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < NE / 2; ++c) {
      const float4 t = *reinterpret_cast<const float4*>(buf + rF + (xF ^ (uint32_t(c) << 4)));
      v[2 * c] = make_float2(t.x, t.y);
      v[2 * c + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const uint32_t E = uint32_t(e) << B;
      v[e] = load_elem<R, FIRST>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)));
    }
  }
#pragma unroll
  for (int m1 = SLO; m1 < SHI; ++m1) {
    const int q = m1 - B;
    const int off = pass_ntw(B, SLO, m1);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if ((e >> q) & 1) continue;
      const int eh = e | (1 << q);
      C wt;
      if constexpr (SRC == kTwGlobal)
        wt = ldg_c(w + (1u << m1) + (F & LOWM) + (uint32_t(e & ((1 << q) - 1)) << B));
      else if constexpr (SRC == kTwShared)
        wt = ld_shared_c<R>(wsm + ((1u << m1) + (F & LOWM) + (uint32_t(e & ((1 << q) - 1)) << B)) * KT<R>::ES);
      else
        wt = w[off + (e & ((1 << q) - 1))];
      if (SCALE && m1 == SHI - 1)
        bfly_scaled(v[e], v[eh], wt, sc);
      else
        bfly(v[e], v[eh], wt);
    }
  }
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < NE / 2; ++c)
      *reinterpret_cast<float4*>(buf + rF + (xF ^ (uint32_t(c) << 4))) =
          make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const uint32_t E = uint32_t(e) << B;
      store_elem<R, RAWOUT>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)), v[e]);
    }
  }
  if constexpr (FENCE) ptx::fence_proxy_async_smem();  // the tile leaves through TMA next
  if constexpr (BAR == 0)
    __syncthreads();
  else
    ptx::named_bar_sync(1, tile_threads<R, W>());
}

// Load the register twiddles of every B > 0 pass from a table indexed
// absolutely (entry 2^m1 + u), in the order tile_pass consumes them.
template <class R, int W, int PLO, int PHI, int P = 0, int ROFF = 0>
__device__ __forceinline__ void load_reg_twiddles(const typename KT<R>::C* __restrict__ tw, uint32_t tid,
                                                  typename KT<R>::C* wreg) {
  constexpr int TB = KT<R>::TB;
  if constexpr (P < n_passes(TB, W, PLO, PHI)) {
    constexpr int B = pass_b(TB, W, PLO, PHI, P), SLO = pass_done(TB, W, PLO, PHI, P),
                  SHI = pass_shi(TB, W, PLO, PHI, P);
    if constexpr (pass_src(TB, W, B) == kTwReg) {
      const typename KT<R>::C* base = tw + (tid & ((1u << B) - 1u));
#pragma unroll
      for (int m1 = SLO; m1 < SHI; ++m1)
#pragma unroll
        for (int v = 0; v < (1 << (m1 - B)); ++v)
          wreg[ROFF + pass_ntw(B, SLO, m1) + v] = ldg_c(base + (1u << m1) + (uint32_t(v) << B));
      load_reg_twiddles<R, W, PLO, PHI, P + 1, ROFF + pass_ntw(B, SLO, SHI)>(tw, tid, wreg);
    } else {
      load_reg_twiddles<R, W, PLO, PHI, P + 1, ROFF>(tw, tid, wreg);
    }
  }
}

// Prefetch into L1 the entries a thread will read in every pass that takes
// its twiddles from memory (register-held top pass and L1-read middle pass).
template <class R, int W, int PLO, int PHI, int P = 0>
__device__ __forceinline__ void prefetch_twiddles(const typename KT<R>::C* __restrict__ tw, uint32_t tid) {
  constexpr int TB = KT<R>::TB;
  if constexpr (P < n_passes(TB, W, PLO, PHI)) {
    constexpr int B = pass_b(TB, W, PLO, PHI, P), SLO = pass_done(TB, W, PLO, PHI, P),
                  SHI = pass_shi(TB, W, PLO, PHI, P);
    if constexpr (B > 0) {
      const typename KT<R>::C* base = tw + (tid & ((1u << B) - 1u));
#pragma unroll
      for (int m1 = SLO; m1 < SHI; ++m1)
#pragma unroll
        for (int v = 0; v < (1 << (m1 - B)); ++v) ptx::prefetch_l1(base + (1u << m1) + (uint32_t(v) << B));
    }
    prefetch_twiddles<R, W, PLO, PHI, P + 1>(tw, tid);
  }
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// MIDSM: the memory-read pass takes its twiddles from the shared-memory copy
// at `wsm` instead of global memory. `hook` runs after the first pass's
// barrier (the level kernel issues its next load there).
// P0SM: the first pass (B = 0) also reads the shared-memory copy at `wsm`.
// TOPSM: the register pass (top pass) reads the shared-memory copy at `wsm`
// too (a kernel that stages whole tables).
template <class R, int W, int PLO, int PHI, bool LAST, int P = 0, int ROFF = 0, bool MIDSM = false,
          class Hook = NoHook, int BAR = 0, bool P0SM = false, bool TOPSM = false>
__device__ __forceinline__ void run_passes(char* buf, const typename KT<R>::C* wreg, const typename KT<R>::C* w0,
                                           const typename KT<R>::C* __restrict__ twg, uint32_t tid, R sc,
                                           uint32_t wsm = 0, const Hook& hook = Hook()) {
  constexpr int TB = KT<R>::TB;
  if constexpr (P < n_passes(TB, W, PLO, PHI)) {
    constexpr int B = pass_b(TB, W, PLO, PHI, P), SLO = pass_done(TB, W, PLO, PHI, P),
                  SHI = pass_shi(TB, W, PLO, PHI, P);
    constexpr bool FINAL = (SHI == PHI);
    // double-float: values arrive as complex128 only in the plan's first level and
    // leave as complex128 only from its last; between levels they stay split
    constexpr bool RAWIN = P == 0 && PLO == 0, RAWOUT = FINAL && LAST;
    constexpr int SRC = pass_src(TB, W, B);
    if constexpr (SRC == kTwParam) {
      if constexpr (P0SM)
        tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, kTwShared, BAR, RAWIN, RAWOUT>(buf, twg, tid, sc, wsm);
      else
        tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, SRC, BAR, RAWIN, RAWOUT>(buf, w0, tid, sc);
    } else if constexpr (SRC == kTwGlobal) {
      if constexpr (MIDSM)
        tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, kTwShared, BAR, RAWIN, RAWOUT>(buf, twg, tid, sc, wsm);
      else
        tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, SRC, BAR, RAWIN, RAWOUT>(buf, twg, tid, sc);
    } else if constexpr (TOPSM) {
      tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, kTwShared, BAR, RAWIN, RAWOUT>(buf, twg, tid, sc, wsm);
    } else {
      tile_pass<R, W, B, SLO, SHI, LAST && FINAL, FINAL, SRC, BAR, RAWIN, RAWOUT>(buf, wreg + ROFF, tid, sc);
    }
    if constexpr (P == 0) hook();
    constexpr int RNEXT = (SRC == kTwReg) ? ROFF + pass_ntw(B, SLO, SHI) : ROFF;
    run_passes<R, W, PLO, PHI, LAST, P + 1, RNEXT, MIDSM, Hook, BAR, P0SM, TOPSM>(buf, wreg, w0, twg, tid, sc, wsm,
                                                                                 hook);
  }
}

// ---- adjoint passes (synthesis) ------------------------------------------------
// The same tiles, element ownership and twiddle entries as tile_pass, with the
// stages of the pass in descending order and the adjoint butterfly. TOPSC: the
// pass holds the plan's last stage, whose table entries carry the factor N/k;
// its second outputs are scaled by sc_top = k/N. FINSC: the pass holds stage 1,
// the last one applied; both its outputs are scaled by sc_fin = 1/N.
template <class R, int W, int B, int SLO, int SHI, bool TOPSC, bool FINSC, bool FENCE, int SRC, bool FIRST = false,
          bool RAWOUT = false>
__device__ __forceinline__ void tile_pass_inv(char* buf, const typename KT<R>::C* w, uint32_t tid, R sc_top,
                                              R sc_fin, uint32_t wsm = 0) {
  using C = typename KT<R>::C;
  static_assert(B >= 0 && B + W <= KT<R>::TB, "pass bits out of tile");
  static_assert(SLO >= B && SHI <= B + W && SLO < SHI, "stage bits out of pass");
  constexpr uint32_t LOWM = (1u << B) - 1u;
  constexpr int NE = 1 << W;
  const uint32_t F = (tid & LOWM) | ((tid >> B) << (B + W));
  const uint32_t rF = row_part<R>(F), xF = xor_part<R>(F);
  C v[NE];
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < NE / 2; ++c) {
      const float4 t = *reinterpret_cast<const float4*>(buf + rF + (xF ^ (uint32_t(c) << 4)));
      v[2 * c] = make_float2(t.x, t.y);
      v[2 * c + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const uint32_t E = uint32_t(e) << B;
      v[e] = load_elem<R, FIRST>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)));
    }
  }
#pragma unroll
  for (int m1 = SHI - 1; m1 >= SLO; --m1) {
    const int q = m1 - B;
    const int off = pass_ntw(B, SLO, m1);
    const bool top = TOPSC && m1 == SHI - 1, fin = FINSC && m1 == SLO;
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      if ((e >> q) & 1) continue;
      const int eh = e | (1 << q);
      C wt;
      if constexpr (SRC == kTwGlobal)
        wt = ldg_c(w + (1u << m1) + (F & LOWM) + (uint32_t(e & ((1 << q) - 1)) << B));
      else if constexpr (SRC == kTwShared)
        wt = ld_shared_c<R>(wsm + ((1u << m1) + (F & LOWM) + (uint32_t(e & ((1 << q) - 1)) << B)) * KT<R>::ES);
      else
        wt = w[off + (e & ((1 << q) - 1))];
      if (top || fin)
        ibfly_scaled(v[e], v[eh], wt, fin ? sc_fin : R(1), (top ? sc_top : R(1)) * (fin ? sc_fin : R(1)));
      else
        ibfly(v[e], v[eh], wt);
    }
  }
  if constexpr (B == 0 && KT<R>::ES == 8) {
#pragma unroll
    for (int c = 0; c < NE / 2; ++c)
      *reinterpret_cast<float4*>(buf + rF + (xF ^ (uint32_t(c) << 4))) =
          make_float4(v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y);
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const uint32_t E = uint32_t(e) << B;
      store_elem<R, RAWOUT>(buf + rF + row_part<R>(E) + (xF ^ xor_part<R>(E)), v[e]);
    }
  }
  if constexpr (FENCE) ptx::fence_proxy_async_smem();
  __syncthreads();
}

// Register-twiddle offset of pass P (entries of the earlier register passes).
constexpr int reg_off(int TB, int W, int PLO, int PHI, int P) {
  int n = 0;
  for (int p = 0; p < P; ++p) {
    const int b = pass_b(TB, W, PLO, PHI, p);
    if (pass_src(TB, W, b) == kTwReg) n += pass_ntw(b, pass_done(TB, W, PLO, PHI, p), pass_shi(TB, W, PLO, PHI, p));
  }
  return n;
}

// The passes of a tile in reverse order (P = n-1 .. 0). LAST: the level holds
// the plan's last stage; PLO == 0: the level holds stage 1. `hook` runs after
// the first pass applied.
template <class R, int W, int PLO, int PHI, bool LAST, bool MIDSM, int P, class Hook>
__device__ __forceinline__ void run_passes_inv(char* buf, const typename KT<R>::C* wreg,
                                               const typename KT<R>::C* w0,
                                               const typename KT<R>::C* __restrict__ twg, uint32_t tid, R sc_top,
                                               R sc_fin, uint32_t wsm, const Hook& hook) {
  constexpr int TB = KT<R>::TB;
  constexpr int NP = n_passes(TB, W, PLO, PHI);
  if constexpr (P >= 0) {
    constexpr int B = pass_b(TB, W, PLO, PHI, P), SLO = pass_done(TB, W, PLO, PHI, P),
                  SHI = pass_shi(TB, W, PLO, PHI, P);
    constexpr bool TOPSC = LAST && P == NP - 1, FINSC = PLO == 0 && P == 0, FENCE = P == 0;
    // double-float: complex128 in at the first level applied (the plan's last),
    // out at the last applied (level 0); split values between levels
    constexpr bool FIRST = P == NP - 1 && LAST, RAWOUT = P == 0 && PLO == 0;
    constexpr int SRC = pass_src(TB, W, B);
    if constexpr (SRC == kTwParam) {
      tile_pass_inv<R, W, B, SLO, SHI, TOPSC, FINSC, FENCE, SRC, FIRST, RAWOUT>(buf, w0, tid, sc_top, sc_fin);
    } else if constexpr (SRC == kTwGlobal) {
      if constexpr (MIDSM)
        tile_pass_inv<R, W, B, SLO, SHI, TOPSC, FINSC, FENCE, kTwShared, FIRST, RAWOUT>(buf, twg, tid, sc_top,
                                                                                    sc_fin, wsm);
      else
        tile_pass_inv<R, W, B, SLO, SHI, TOPSC, FINSC, FENCE, SRC, FIRST, RAWOUT>(buf, twg, tid, sc_top, sc_fin);
    } else {
      tile_pass_inv<R, W, B, SLO, SHI, TOPSC, FINSC, FENCE, SRC, FIRST, RAWOUT>(
          buf, wreg + reg_off(TB, W, PLO, PHI, P), tid, sc_top, sc_fin);
    }
    if constexpr (P == NP - 1) hook();
    run_passes_inv<R, W, PLO, PHI, LAST, MIDSM, P - 1, Hook>(buf, wreg, w0, twg, tid, sc_top, sc_fin, wsm, hook);
  }
}

// ---- persistent level kernel ----------------------------------------------------
// Tile i of a level: a = i / nB selects the twiddle table (a group block for
// later levels), b = i % nB; TMA coordinates {0, a*a_step1 + b*b_step1, 0, b*b_step3}.
template <class R>
struct LevelArgs {
  uint64_t n_tiles;
  uint64_t nB;
  int32_t a_step1, b_step1, b_step3;
  uint32_t tw_first;       // first absolute table entry present in a table
  const void* tw;          // tables of this level (device)
  uint64_t tw_len;         // entries per table
  uint64_t tw_stride;      // entries between consecutive tables (0: one shared table)
  double scale;            // N/k, used when LAST
  double inv_n;            // 1/N, used by the adjoint kernel
  int* status;             // device status word
  uint64_t timeout_ns;     // bound on every mbarrier wait
  int64_t lim1, lim3;      // tile origins lie in [0, lim1) x [0, lim3) (range checks)
  uint64_t tw_tables;      // tables in `tw` (range checks)
  uint64_t chunk;          // later levels: consecutive b per chunk of the tile walk (0: interleaved walk)
  typename KT<R>::C tw0[16];  // tw0[i] = level-0 table entry i + 1 (stage bits 0..3), i < 15
};

// Range checks of a level launch (debug build): the table entries the passes
// of stage bits [PLO, PHI) read, [max(1, 2^PLO), 2^PHI) absolute, lie in every
// table's [tw_first, tw_first + tw_len).
template <class R, int PLO, int PHI>
__device__ __forceinline__ bool level_tables_in_bounds(const LevelArgs<R>& a) {
  const uint64_t lo = PLO == 0 ? 1u : (1ull << PLO), hi = 1ull << PHI;
  return in_bounds(a.tw_first <= lo && hi <= a.tw_first + a.tw_len && a.tw_tables >= 1, a.status);
}
// A tile origin outside the tensor becomes (0, 0) (debug build).
template <class R>
__device__ __forceinline__ void level_coords_in_bounds(const LevelArgs<R>& a, int& c1, int& c3) {
  if (!in_bounds(c1 >= 0 && c1 < a.lim1 && c3 >= 0 && c3 < a.lim3, a.status)) c1 = c3 = 0;
}

// Pointer arithmetic on the shared-memory symbol itself (no round trip through
// an integer), so that accesses through the result stay shared-space loads and
// stores instead of generic ones.
__device__ __forceinline__ char* align1024(char* p) {
  const uint32_t s = ptx::smem_addr(p);
  return p + ((1024u - (s & 1023u)) & 1023u);
}

// Pipeline per CTA (kLevelBufs = 2 tile buffers): tile j waits on full[j % 2],
// runs its passes in place, and leaves through a TMA store issued by thread 0.
// After tile j's first pass, the buffer of tile j-1 is refilled with tile j+1
// once its store has finished reading shared memory, so the next tile's load is
// in flight behind the tile being computed.
// INV: the adjoint (synthesis) passes instead of the forward ones.
template <class R, int W, int PLO, int PHI, bool LAST, bool INV = false>
__global__ void __launch_bounds__(tile_threads<R, W>(), 2)
    k_level(const __grid_constant__ CUtensorMap src, const __grid_constant__ CUtensorMap dst,
            const __grid_constant__ LevelArgs<R> args) {
  using C = typename KT<R>::C;
  constexpr int NREG = reg_twiddles(KT<R>::TB, W, PLO, PHI);
  constexpr uint32_t NT = tile_threads<R, W>();
  extern __shared__ char smem_raw[];
  char* smem = align1024(smem_raw);
  const uint32_t bar0 = ptx::smem_addr(smem + kLevelBufs * kTileBytes);
  const uint32_t tid = threadIdx.x;
  // Self-check of the launch before any shared-memory or TMA access: enough
  // dynamic shared memory for the aligned layout, tensor maps 64-byte aligned,
  // twiddle tables 16-byte aligned. A failed check records a status and exits.
  {
    const uint32_t used = uint32_t(smem - smem_raw) + kLevelBufs * kTileBytes + 64 + kMidTwBytes;
    int bad = 0;
    if (ptx::dynamic_smem_size() < used) bad = kBadSmem;
    else if ((reinterpret_cast<uintptr_t>(&src) | reinterpret_cast<uintptr_t>(&dst)) & 63u) bad = kBadMap;
    else if (reinterpret_cast<uintptr_t>(args.tw) & 15u) bad = kBadTable;
    if (bad) {
      if (tid == 0) atomicCAS(args.status, 0, bad);
      return;
    }
    if (!level_tables_in_bounds<R, PLO, PHI>(args)) return;   // debug build only
  }
  // Tile i = a * nB + b (a: the table, b: the instance or row block). Two walks:
  //  * chunk == 0 (level 0, one table): CTA c takes tiles c, c + G, c + 2G, ...,
  //    so the tiles in flight at any moment are neighbours in memory;
  //  * chunk > 0 (later levels, one table per group block a): chunks of `chunk`
  //    consecutive b on one a, chunk q = bB * nA + a; CTA c takes chunks
  //    c, c + G, ... and their tiles in order. A CTA then reloads its group
  //    block's table once per chunk instead of once per tile, and the CTAs in
  //    flight cover whole rows of one instance block (all a for the same b).
  //    The instance blocks run last to first: the previous level wrote them
  //    first to last, so the first blocks read here are still in L2.
  const uint64_t G = gridDim.x;
  const uint64_t t0 = blockIdx.x;
  // the walk is fixed at compile time: level 0 (PLO = 0) interleaved, later
  // levels chunked (args.chunk > 0)
  const uint64_t CH = PLO > 0 ? args.chunk : 0;
  const uint64_t nA = args.n_tiles / args.nB;
  const uint64_t nBB = CH ? (args.nB + CH - 1) / CH : 0;
  if (CH ? t0 >= nA * nBB : t0 >= args.n_tiles) return;
  // chunked walk: instance block bB of the walk is block nBB - 1 - bB in memory
  auto block_len = [&](uint64_t bB) {
    if (bB >= nBB) return uint64_t(0);
    const uint64_t r = nBB - 1 - bB;
    return (r + 1) * CH <= args.nB ? CH : args.nB - r * CH;
  };
  uint64_t n = 0;
  if (CH) {
    for (uint64_t q = t0; q < nA * nBB; q += G) n += block_len(q / nA);
  } else {
    n = (args.n_tiles - t0 + G - 1) / G;
  }

  // The walk advanced incrementally (no 64-bit division per tile).
  struct Cursor {
    uint64_t a, b;
    uint64_t bB, t, len;   // chunked walk: chunk (a, bB), position t of len
  };
  auto cursor_at = [&](uint64_t i) {
    if (PLO > 0 && CH) {
      const uint64_t bB = i / nA;
      return Cursor{i % nA, (nBB - 1 - bB) * CH, bB, 0, block_len(bB)};
    }
    return Cursor{i / args.nB, i % args.nB, 0, 0, 0};
  };
  const uint64_t step_a = CH ? G % nA : G / args.nB, step_b = CH ? G / nA : G % args.nB;
  auto advance = [&](Cursor& c) {
    if (PLO > 0 && CH) {
      if (++c.t < c.len) {
        ++c.b;
        return;
      }
      c.a += step_a;
      c.bB += step_b;
      if (c.a >= nA) {
        c.a -= nA;
        ++c.bB;
      }
      c.t = 0;
      c.len = block_len(c.bB);
      c.b = c.len ? (nBB - 1 - c.bB) * CH : 0;
      return;
    }
    c.a += step_a;
    c.b += step_b;
    if (c.b >= args.nB) {
      c.b -= args.nB;
      ++c.a;
    }
  };
  auto coords = [&](const Cursor& c, int& c1, int& c3) {
    c1 = int(int64_t(c.a) * args.a_step1 + int64_t(c.b) * args.b_step1);
    c3 = int(int64_t(c.b) * args.b_step3);
  };
  Cursor load_cur = cursor_at(t0);     // thread 0: next tile to load
  uint32_t load_buf = 0;               // thread 0: its buffer (tiles load in order, buffers cycle)
  auto issue_load = [&]() {
    const uint32_t b = load_buf;
    load_buf = (load_buf + 1 == uint32_t(kLevelBufs)) ? 0u : load_buf + 1;
    const uint32_t bar = bar0 + 8 * b;
    int c1, c3;
    coords(load_cur, c1, c3);
    level_coords_in_bounds(args, c1, c3);
    advance(load_cur);
    ptx::mbar_arrive_expect_tx(bar, kTileBytes);
    // every tile is read once: first out of L2
    ptx::tma_load_4d_hint(ptx::smem_addr(smem + b * kTileBytes), &src, bar, 0, c1, 0, c3, ptx::policy_evict_first());
  };

  if (tid == 0) {
    for (int b = 0; b < kLevelBufs; ++b) ptx::mbar_init(bar0 + 8 * b, 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&src);
    ptx::prefetch_tensormap(&dst);
    for (uint64_t j = 0; j < n && j < uint64_t(kLevelBufs); ++j) issue_load();
  }
  __syncthreads();
  const R sc = R(args.scale);
  const C* tw = static_cast<const C*>(args.tw) - args.tw_first;
  C wreg[NREG > 0 ? NREG : 1];
  constexpr int MLO = mid_pass_lo(KT<R>::TB, W, PLO, PHI), MHI = mid_pass_hi(KT<R>::TB, W, PLO, PHI);
  // a middle pass whose region fits the shared copy reads it from there
  constexpr bool MIDSM = MLO < MHI && (1u << MHI) * sizeof(C) <= kMidTwBytes;
  C* midtw = reinterpret_cast<C*>(smem + kLevelBufs * kTileBytes + 64);
  const uint32_t midtw_addr = ptx::smem_addr(midtw);
  const C* twt = tw;
  uint64_t cur_tab = ~0ull;
  bool aborted = false;
  Cursor cur = cursor_at(t0);          // tile being computed
  uint32_t b = 0;                      // its buffer
  uint32_t phases = 0;                 // bit q: parity of buffer q's next completion
  uint64_t j = 0;
  for (; j < n; ++j, advance(cur), b = (b + 1 == uint32_t(kLevelBufs)) ? 0u : b + 1) {
    char* buf = smem + b * kTileBytes;
    uint64_t tab = args.tw_stride ? cur.a : 0;
    if (!in_bounds(tab < args.tw_tables, args.status)) tab = 0;
    if (tab != cur_tab) {  // uniform across the CTA; the previous tile's passes are done
      twt = tw + tab * args.tw_stride;
      load_reg_twiddles<R, W, PLO, PHI>(twt, tid, wreg);
      if constexpr (MIDSM) {   // the middle pass's entries into shared memory (barrier below)
        for (uint32_t e = (1u << MLO) + tid; e < (1u << MHI); e += NT) midtw[e] = twt[e];
      }
      cur_tab = tab;
    }
    const bool ok = ptx::mbar_wait_bounded(bar0 + 8 * b, (phases >> b) & 1u, args.timeout_ns);
    phases ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    // After the first pass: once the store of tile j-1 (the latest one issued)
    // has left its buffer, load tile j + kLevelBufs - 1 into it, two thirds of a
    // tile earlier than at the end of this tile.
    auto refill = [&]() {
      if (tid == 0 && j >= 1 && j + kLevelBufs - 1 < n) {
        ptx::bulk_wait_read<0>();
        issue_load();
      }
    };
    if constexpr (INV)
      run_passes_inv<R, W, PLO, PHI, LAST, MIDSM, n_passes(KT<R>::TB, W, PLO, PHI) - 1>(
          buf, wreg, args.tw0, twt, tid, R(1.0 / args.scale), R(args.inv_n), midtw_addr, refill);
    else
      run_passes<R, W, PLO, PHI, LAST, 0, 0, MIDSM>(buf, wreg, args.tw0, twt, tid, sc, midtw_addr, refill);
    if (tid == 0) {
      int c1, c3;
      coords(cur, c1, c3);
      level_coords_in_bounds(args, c1, c3);
      // the final output leaves L2 first; an intermediate stays for the next level
      if constexpr (LAST)
        ptx::tma_store_4d_hint(&dst, ptx::smem_addr(buf), 0, c1, 0, c3, ptx::policy_evict_first());
      else
        ptx::tma_store_4d(&dst, ptx::smem_addr(buf), 0, c1, 0, c3);
      ptx::bulk_commit();
    }
  }
  if (tid == 0) {
    if (aborted) {
      // Let loads already issued (tiles j .. max(j + kLevelBufs - 2, kLevelBufs - 1))
      // land before the CTA's shared memory is released.
      const uint64_t last = (j + kLevelBufs - 2 > uint64_t(kLevelBufs - 1)) ? j + kLevelBufs - 2
                                                                             : uint64_t(kLevelBufs - 1);
      for (uint64_t q = j; q <= last && q < n; ++q)
        ptx::mbar_wait_bounded(bar0 + 8 * uint32_t(q % kLevelBufs), uint32_t((q / kLevelBufs) & 1),
                               drain_bound(args.timeout_ns));
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

// ---- warp path for small batches of 2^5 <= k <= 2^10 (latency) -------------------------
// One warp per instance, plain coalesced loads and stores (no TMA, no shared
// memory): element t = 32 r + lane sits in lane `lane`, register r. Stage bits
// 0..4 pair lanes (shuffles), stage bits 5..S-1 pair registers; the table is
// level 0's, indexed absolutely (entry 2^m1 + u), and its last stage's entries
// carry N/k, as for the level kernel.
template <class R, int S>
__global__ void __launch_bounds__(128) k_warp(const typename KT<R>::C* __restrict__ in,
                                              typename KT<R>::C* __restrict__ out, uint64_t batch,
                                              const typename KT<R>::C* __restrict__ tw, R sc) {
  using C = typename KT<R>::C;
  static_assert(S >= 5 && S <= 10, "warp path: 2^5 <= k <= 2^10");
  constexpr int K = 1 << S, V = K / 32;
  const uint64_t inst = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  if (inst >= batch) return;   // whole warps leave together (blockDim is a multiple of 32)
  const C* src = in + inst * K + lane;
  C x[V];
#pragma unroll
  for (int r = 0; r < V; ++r) x[r] = src[32 * r];
#pragma unroll
  for (int m1 = 0; m1 < S; ++m1) {
    const bool last = m1 == S - 1;
    if (m1 < 5) {
      const C w = __ldg(tw + (1u << m1) + (lane & ((1u << m1) - 1u)));
      const bool hi = (lane >> m1) & 1u;
#pragma unroll
      for (int r = 0; r < V; ++r) {
        C o;
        o.x = __shfl_xor_sync(0xffffffffu, x[r].x, 1 << m1);
        o.y = __shfl_xor_sync(0xffffffffu, x[r].y, 1 << m1);
        C a = hi ? o : x[r], b = hi ? x[r] : o;
        if (last)
          bfly_scaled(a, b, w, sc);
        else
          bfly(a, b, w);
        x[r] = hi ? b : a;
      }
    } else {
      const int q = m1 - 5;
#pragma unroll
      for (int r = 0; r < V; ++r) {
        if ((r >> q) & 1) continue;
        const C w = __ldg(tw + (1u << m1) + lane + 32u * uint32_t(r & ((1 << q) - 1)));
        if (last)
          bfly_scaled(x[r], x[r | (1 << q)], w, sc);
        else
          bfly(x[r], x[r | (1 << q)], w);
      }
    }
  }
  C* dst = out + inst * K + lane;
#pragma unroll
  for (int r = 0; r < V; ++r) dst[32 * r] = x[r];
}

// Adjoint of k_small: stages S-1 .. 0; the last stage's entries carry N/k
// (undone by sc_top = k/N), the final stage scales by sc_fin = 1/N.
template <class R, int S>
__global__ void __launch_bounds__(256) k_small_inv(const typename KT<R>::C* __restrict__ in,
                                                   typename KT<R>::C* __restrict__ out, uint64_t batch,
                                                   const typename KT<R>::C* __restrict__ tw, R sc_top, R sc_fin) {
  using C = typename KT<R>::C;
  constexpr int K = 1 << S;
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  C v[K];
#pragma unroll
  for (int e = 0; e < K; ++e) v[e] = in[i * K + e];
#pragma unroll
  for (int m1 = S - 1; m1 >= 0; --m1) {
#pragma unroll
    for (int e = 0; e < K; ++e) {
      if ((e >> m1) & 1) continue;
      const C w = __ldg(tw + (1u << m1) + (e & ((1 << m1) - 1)));
      const bool top = m1 == S - 1, fin = m1 == 0;
      if (top || fin)
        ibfly_scaled(v[e], v[e | (1 << m1)], w, fin ? sc_fin : R(1), (top ? sc_top : R(1)) * (fin ? sc_fin : R(1)));
      else
        ibfly(v[e], v[e | (1 << m1)], w);
    }
  }
  if constexpr (S == 0) {
    v[0].x *= sc_fin;
    v[0].y *= sc_fin;
  }
#pragma unroll
  for (int e = 0; e < K; ++e) out[i * K + e] = v[e];
}

}  // namespace sdft
