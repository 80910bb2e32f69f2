// Host planner: validation, pivots, canonical order, sample set, twiddle tables.
//
// Pivots (Definition 8) are the levels where the congruence tree T(J) splits;
// two leaves meet at level l iff their difference is an odd multiple of 2^l
// (Remark "tree-2-adic"). J is homogeneous iff there are exactly log2 k such
// levels (Definition 9). A homogeneous J is recognised in O(k) from the path
// of its first element; anything else goes to a sort of the bit-reversed
// values, which finds every split between depth-first neighbours and names
// the error.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "plan.hpp"

namespace sdft {
namespace {

inline uint64_t bitrev64(uint64_t x) {
  x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
  x = ((x >> 2) & 0x3333333333333333ull) | ((x & 0x3333333333333333ull) << 2);
  x = ((x >> 4) & 0x0F0F0F0F0F0F0F0Full) | ((x & 0x0F0F0F0F0F0F0F0Full) << 4);
  x = ((x >> 8) & 0x00FF00FF00FF00FFull) | ((x & 0x00FF00FF00FF00FFull) << 8);
  x = ((x >> 16) & 0x0000FFFF0000FFFFull) | ((x & 0x0000FFFF0000FFFFull) << 16);
  return (x >> 32) | (x << 32);
}

inline int highest_bit(uint64_t x) { return 63 - __builtin_clzll(x); }

// LSD radix sort of `bits`-bit keys in 8-bit digits (stable; tmp is scratch).
void radix_sort(std::vector<uint64_t>& a, std::vector<uint64_t>& tmp, uint32_t bits) {
  const size_t n = a.size();
  tmp.resize(n);
  for (uint32_t shift = 0; shift < bits; shift += 8) {
    size_t count[257] = {0};
    for (size_t i = 0; i < n; ++i) ++count[((a[i] >> shift) & 255u) + 1];
    for (int d = 0; d < 256; ++d) count[d + 1] += count[d];
    for (size_t i = 0; i < n; ++i) tmp[count[(a[i] >> shift) & 255u]++] = a[i];
    a.swap(tmp);
  }
}

// Byte lookup tables for a bit gather: out(x) = sum_q bit_{src[q]}(x) << dst[q],
// evaluated as the OR of one table entry per byte of x.
struct BitGather {
  uint32_t nbytes = 0;
  std::vector<uint64_t> lut;   // nbytes x 256
  void build(const uint32_t* src, const uint32_t* dst, uint32_t n, uint32_t in_bits) {
    nbytes = (in_bits + 7) / 8;
    lut.assign(size_t(nbytes) * 256, 0);
    for (uint32_t q = 0; q < n; ++q) {
      const uint32_t byte = src[q] / 8, bit = src[q] % 8;
      for (uint32_t v = 0; v < 256; ++v)
        if (v >> bit & 1u) lut[size_t(byte) * 256 + v] |= 1ull << dst[q];
    }
  }
  uint64_t operator()(uint64_t x) const {
    uint64_t r = 0;
    for (uint32_t b = 0; b < nbytes; ++b) r |= lut[size_t(b) * 256 + ((x >> (8 * b)) & 255u)];
    return r;
  }
};

// cos(pi x), sin(pi x) for a dyadic x in [0, 1): fold into [0, 1/4] with exact
// reflections so quarter turns come out exact, then call the C library.
void cos_sin_pi(double x, double& c, double& s) {
  double sc = 1.0;                 // sign of the cosine after x -> 1 - x
  if (x > 0.5) { x = 1.0 - x; sc = -1.0; }
  double cc, ss;
  if (x > 0.25) {
    const double y = 0.5 - x;      // cos(pi x) = sin(pi y), sin(pi x) = cos(pi y)
    cc = std::sin(M_PI * y);
    ss = std::cos(M_PI * y);
  } else {
    cc = std::cos(M_PI * x);
    ss = std::sin(M_PI * x);
  }
  c = sc * cc;
  s = ss;
}

}  // namespace

void twiddle_f64(const Plan& p, uint32_t m, uint64_t u, double& re, double& im) {
  // Lemma "rec-hom-tree-split": omega_{r+1}^{j} with r = r_m and j = Jc[u]
  // (bit r of Jc[u] is 0 for u < 2^(m-1)); only j mod 2^r matters.
  const uint32_t r = p.pivots[m - 1];
  const uint64_t rho = (r >= 64) ? p.Jc[u] : (p.Jc[u] & ((r == 0) ? 0ull : ((1ull << r) - 1)));
  const double x = std::ldexp(static_cast<double>(rho), -static_cast<int>(r));  // rho / 2^r
  double c, s;
  cos_sin_pi(x, c, s);
  re = c;
  im = -s;
}

namespace {

// Canonical order: coefficient t is the element whose pivot bits spell t.
// False if two elements share a key (then J is not homogeneous or repeats).
bool canonical_order(const uint64_t* J, uint64_t k, uint32_t s, uint32_t M, const std::vector<uint32_t>& qbits,
                     Plan& p) {
  BitGather key_of;
  key_of.build(p.pivots.data(), qbits.data(), s, M);
  p.Jc.assign(k, ~0ull);
  for (uint64_t i = 0; i < k; ++i) {
    const uint64_t key = key_of(J[i]);
    if (p.Jc[key] != ~0ull) return false;
    p.Jc[key] = J[i];
  }
  return true;
}

// O(k) path for a homogeneous J. Every leaf of a homogeneous congruence tree
// leaves the path of J[0] at a pivot level, and at every pivot level some leaf
// does, so the pivots are the levels ctz(j xor J[0]) (Remark "tree-2-adic").
// The candidate set is then confirmed: in canonical order, elements t and
// t - 2^h (h the highest key bit of t) must first differ at bit r_{h+1}. By
// induction over the key bits every pair of elements then first differs at a
// pivot level, so the tree splits at exactly s levels (Definition 9). False
// on any failure; the sorting path then decides and names the error.
bool pivots_along_first_path(uint32_t M, const uint64_t* J, uint64_t k, uint32_t s,
                             const std::vector<uint32_t>& qbits, Plan& p) {
  uint64_t mask = 0;
  for (uint64_t i = 1; i < k; ++i) {
    const uint64_t x = J[i] ^ J[0];
    if (!x) return false;
    mask |= 1ull << __builtin_ctzll(x);
  }
  if (static_cast<uint32_t>(__builtin_popcountll(mask)) != s) return false;
  p.pivots.clear();
  for (uint32_t l = 0; l < M; ++l)
    if (mask >> l & 1) p.pivots.push_back(l);
  if (!canonical_order(J, k, s, M, qbits, p)) return false;
  // For each key bit h: t in [2^h, 2^(h+1)) against t - 2^h; "first differ at
  // bit r" is (x & (2^(r+1) - 1)) == 2^r, checked over whole runs without branches.
  for (uint32_t h = 0; h < s; ++h) {
    const uint64_t half = 1ull << h, want = 1ull << p.pivots[h], low = (want << 1) - 1;
    const uint64_t* hi = p.Jc.data() + half;
    const uint64_t* lo = p.Jc.data();
    uint64_t bad = 0;
    for (uint64_t t = 0; t < half; ++t) bad |= ((hi[t] ^ lo[t]) & low) ^ want;
    if (bad) return false;
  }
  return true;
}

// Reference path: sorting J by its bit-reversed value lists the leaves of the
// LSB-first tree in depth-first order, so every split shows up between two
// neighbours, at the lowest bit where they differ; J is homogeneous iff there
// are exactly s such levels.
sdft_status pivots_by_sorting(uint32_t M, const uint64_t* J, uint64_t k, uint32_t s,
                              const std::vector<uint32_t>& qbits, Plan& p) {
  std::vector<uint64_t> rev(k), tmp;
  for (uint64_t i = 0; i < k; ++i) rev[i] = M ? (bitrev64(J[i]) >> (64 - M)) : 0;
  radix_sort(rev, tmp, M);
  std::vector<uint64_t>().swap(tmp);
  uint64_t level_mask = 0;
  for (uint64_t i = 0; i + 1 < k; ++i) {
    const uint64_t x = rev[i] ^ rev[i + 1];
    if (x == 0) return SDFT_ERR_DUPLICATE;
    level_mask |= 1ull << (M - 1 - highest_bit(x));
  }
  std::vector<uint64_t>().swap(rev);
  if (static_cast<uint32_t>(__builtin_popcountll(level_mask)) != s) return SDFT_ERR_NOT_HOMOGENEOUS;
  p.pivots.clear();
  for (uint32_t l = 0; l < M; ++l)
    if (level_mask >> l & 1) p.pivots.push_back(l);
  if (!canonical_order(J, k, s, M, qbits, p)) return SDFT_ERR_NOT_HOMOGENEOUS;  // cannot happen once the count matched
  return SDFT_OK;
}

}  // namespace

sdft_status build_plan(uint32_t M, const uint64_t* J, uint64_t k, sdft_prec prec, Plan& p) {
  if (!J && k) return SDFT_ERR_ARG;
  if (prec != SDFT_C64 && prec != SDFT_C128) return SDFT_ERR_ARG;
  if (M > SDFT_MAX_LOG2N) return SDFT_ERR_RANGE;
  if (k == 0) return SDFT_ERR_ARG;
  if (k & (k - 1)) return SDFT_ERR_NOT_POW2;
  const uint32_t s = static_cast<uint32_t>(__builtin_ctzll(k));
  if (s > SDFT_MAX_LOG2K) return SDFT_ERR_UNSUPPORTED;
  const uint64_t N = 1ull << M;
  for (uint64_t i = 0; i < k; ++i)
    if (J[i] >= N) return SDFT_ERR_RANGE;
  if (s > M) return SDFT_ERR_DUPLICATE;  // more than N distinct values is impossible

  p.M = M;
  p.s = s;
  p.k = k;
  p.prec = prec;

  std::vector<uint32_t> qbits(s), ibits(s);
  for (uint32_t q = 0; q < s; ++q) qbits[q] = q;
  if (!pivots_along_first_path(M, J, k, s, qbits, p)) {
    const sdft_status st = pivots_by_sorting(M, J, k, s, qbits, p);
    if (st != SDFT_OK) return st;
  }
  for (uint32_t q = 0; q < s; ++q) ibits[q] = M - 1 - p.pivots[q];

  // Pivoted sampling pattern (Definition "r_sampling_pattern"), sample order t:
  // I[t] = sum_q bit_q(t) 2^(M-1-r_{q+1}), built by doubling: the indices with
  // key bit q set are those below 2^q with that bit added.
  p.I.resize(k);
  p.I[0] = 0;
  for (uint32_t q = 0; q < s; ++q) {
    const uint64_t half = 1ull << q, bit = 1ull << ibits[q];
    uint64_t* out = p.I.data() + half;
    const uint64_t* in = p.I.data();
    for (uint64_t t = 0; t < half; ++t) out[t] = in[t] | bit;
  }

  // Level schedule.
  p.levels.clear();
  p.tw_elems = 0;
  if (s <= kSmallMax) {
    p.tw_elems = s ? (1ull << s) : 0;
    return SDFT_OK;
  }
  const uint32_t TB = tile_bits(prec), CB = row_bits(prec);
  Level l0;
  l0.lo = 0;
  l0.hi = std::min<uint32_t>(s, TB);
  l0.plo = 0;
  l0.n_gb = 1;
  l0.tw_off = 0;
  l0.tw_len = 1ull << l0.hi;
  l0.last = (l0.hi == s);
  p.levels.push_back(l0);
  uint64_t off = l0.tw_len;
  uint32_t lo = l0.hi;
  while (lo < s) {
    Level L;
    L.lo = lo;
    L.hi = std::min<uint32_t>(s, lo + (TB - CB));
    const uint32_t Q = L.hi - L.lo;
    L.lg = TB - CB - Q;
    L.plo = TB - Q;
    L.n_gb = 1ull << (L.lo - CB - L.lg);
    L.tw_len = (1ull << TB) - (1ull << L.plo);
    L.tw_off = off;
    L.last = (L.hi == s);
    off += L.n_gb * L.tw_len;
    p.levels.push_back(L);
    lo = L.hi;
  }
  p.tw_elems = off;
  return SDFT_OK;
}

sdft_status split_levels(uint32_t M, const uint64_t* J, uint64_t k, uint64_t& level_mask) {
  level_mask = 0;
  if (!J || k == 0) return SDFT_ERR_ARG;
  if (M > SDFT_MAX_LOG2N) return SDFT_ERR_RANGE;
  const uint64_t N = 1ull << M;
  for (uint64_t i = 0; i < k; ++i)
    if (J[i] >= N) return SDFT_ERR_RANGE;
  std::vector<uint64_t> rev(k), tmp;
  for (uint64_t i = 0; i < k; ++i) rev[i] = M ? (bitrev64(J[i]) >> (64 - M)) : 0;
  radix_sort(rev, tmp, M);
  for (uint64_t i = 0; i + 1 < k; ++i) {
    const uint64_t x = rev[i] ^ rev[i + 1];
    if (x == 0) return SDFT_ERR_DUPLICATE;
    level_mask |= 1ull << (M - 1 - highest_bit(x));
  }
  return SDFT_OK;
}

template <class T>
void fill_device_tables(const Plan& p, T* out) {
  if (p.tw_elems == 0) return;
  std::memset(out, 0, sizeof(T) * 2 * p.tw_elems);
  const int final_scale = static_cast<int>(p.M) - static_cast<int>(p.s);  // N/k = 2^(M-s)
  const uint32_t CB = row_bits(p.prec);
  // Segments of consecutive entries: stage m, entries base + v for v < cnt,
  // twiddle index u = v (level 0 and the register path) or, for a later-level
  // group block gb, v = (hq << plo) | (gl << CB) | c -> u = (hq << lo) | ((gb << lg | gl) << CB) | c.
  struct Seg {
    uint64_t base, cnt, gb;
    uint32_t m;
    const Level* L;
  };
  std::vector<Seg> segs;
  if (p.levels.empty()) {                      // register path: entry 2^(m-1) + u for stage m
    for (uint32_t m = 1; m <= p.s; ++m) segs.push_back(Seg{1ull << (m - 1), 1ull << (m - 1), 0, m, nullptr});
  } else {
    const Level& l0 = p.levels[0];
    for (uint32_t m = 1; m <= l0.hi; ++m)
      segs.push_back(Seg{l0.tw_off + (1ull << (m - 1)), 1ull << (m - 1), 0, m, nullptr});
    for (size_t j = 1; j < p.levels.size(); ++j) {
      const Level& L = p.levels[j];
      for (uint64_t gb = 0; gb < L.n_gb; ++gb)
        for (uint32_t q = 0; q < L.hi - L.lo; ++q) {
          const uint64_t cnt = 1ull << (L.plo + q);
          segs.push_back(Seg{L.tw_off + gb * L.tw_len - (1ull << L.plo) + cnt, cnt, gb, L.lo + q + 1, &L});
        }
    }
  }
  auto put = [&](const Seg& g, uint64_t v) {
    uint64_t u = v;
    if (g.L) {
      const uint64_t c = v & ((1ull << CB) - 1);
      const uint64_t gl = (v >> CB) & ((1ull << g.L->lg) - 1);
      const uint64_t hq = v >> g.L->plo;
      u = (hq << g.L->lo) | (((g.gb << g.L->lg) | gl) << CB) | c;
    }
    double re, im;
    twiddle_f64(p, g.m, u, re, im);
    if (g.m == p.s) {
      re = std::ldexp(re, final_scale);
      im = std::ldexp(im, final_scale);
    }
    out[2 * (g.base + v)] = static_cast<T>(re);
    out[2 * (g.base + v) + 1] = static_cast<T>(im);
  };
  // Entries [lo, hi) of the concatenated segments.
  auto fill_range = [&](uint64_t lo, uint64_t hi) {
    uint64_t pos = 0;
    for (const Seg& g : segs) {
      const uint64_t a = std::max(lo, pos), b = std::min(hi, pos + g.cnt);
      for (uint64_t x = a; x < b; ++x) put(g, x - pos);
      pos += g.cnt;
      if (pos >= hi) break;
    }
  };
  uint64_t total = 0;
  for (const Seg& g : segs) total += g.cnt;
  // Large tables are split over a few threads (each entry is independent).
  unsigned nt = 1;
  if (total >= (1ull << 15)) nt = std::max(1u, std::min(8u, std::thread::hardware_concurrency()));
  if (nt == 1) {
    fill_range(0, total);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned i = 1; i < nt; ++i) {
    const uint64_t a = total * i / nt, b = total * (i + 1) / nt;
    try {
      th.emplace_back(fill_range, a, b);
    } catch (...) {                 // no thread available: do that share here
      fill_range(a, b);
    }
  }
  fill_range(0, total / nt);
  for (std::thread& t : th) t.join();
}

template void fill_device_tables<float>(const Plan&, float*);
template void fill_device_tables<double>(const Plan&, double*);

}  // namespace sdft
