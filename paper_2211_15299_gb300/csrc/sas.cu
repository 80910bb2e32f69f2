// Shift-and-Sample (Algorithm "shift-sample") for supports that are not
// homogeneous: the coefficients of an arbitrary J from mu* transforms of a
// homogeneous "virtual" support, one per shifted sample set, followed by a
// small Vandermonde solve per class.
//
// Planning (host). Pivots r are the first R split levels of T(J), so J is
// r-part-homogeneous (Definition "part-H-tree"); the classes of J modulo
// 2^rho, rho = r_max + 1, are indexed by their pivot bits (key t). Unless the
// caller fixes R, it is the one with the smallest operation count of Lemma
// "computation_shift_sample", 1.5 R 2^R mu* + 6 sum_v mu(v)^2, among those
// whose class systems are well conditioned for the arithmetic. The virtual
// support has one residue per key: a class's residue mod 2^rho where J
// occupies it, otherwise a residue that keeps the set homogeneous with pivots
// r. Per class, the inverse of V[a][u] = z_u^a (z_u = exp(2 pi i l_u / N),
// a < mu) is computed in FP64 and rounded once.
//
// Execution (device). Stage 1 runs the virtual plan over the mu* shifted
// sample sets of every instance (the strided path). Stage 2 (k_sas_decode)
// forms every coefficient as a row of its class's inverse times the class's
// mu values: coefficient u of class t = sum_a Winv_t[u][a] Y_a[t] (eq.
// "alg1_system"). With mu* = 1 stage 2 is a gather (complete isolation).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "launch.hpp"
#include "levels.cuh"
#include "plan.hpp"

namespace sdft {
namespace {

constexpr uint32_t kSasMaxMu = 64;     // largest class the decoder accepts
constexpr uint32_t kSasMaxR = 24;      // largest number of pivots

struct SasOut {          // per output coefficient (16 bytes)
  uint32_t t;            // class key: column of the stage-1 output
  uint16_t u, mu;        // position in the class, class size
  uint32_t woff;         // first entry of the class's inverse (row-major mu x mu)
  uint32_t pad;
};

struct Sas {
  uint32_t M = 0, R = 0, mu_star = 0, occupied = 0;
  uint64_t k = 0;
  sdft_prec prec = SDFT_C64;
  std::vector<uint32_t> pivots;
  std::vector<uint64_t> order;     // J in output order (by class key, then value)
  std::vector<uint64_t> samples;   // mu* x 2^R sample indices
  std::vector<SasOut> meta;        // per output coefficient
  std::vector<std::complex<double>> winv;
  double max_cond = 1.0;
  std::vector<uint64_t> virt;      // the virtual homogeneous support (key order)
  sdft_plan vplan = nullptr;       // its plan on the device
  int device = -1;
  SasOut* d_meta = nullptr;
  void* d_winv = nullptr;
  bool two_stage = false;          // SDFT_SAS_TWO_STAGE: stage 2 as its own launch always
  uint16_t* d_col = nullptr;       // one-launch path (mu* = 1): t_i per coefficient
  void* d_w1 = nullptr;            //   and its class's 1 x 1 inverse
  uint32_t* d_gather = nullptr;    // gathered path (mu* > 1): t_i | i << 16, grouped by u_i
  std::vector<uint32_t> goff;      //   entries of shift a: [goff[a], goff[a + 1])
};

// Class keys of J for pivots p[0..R-1]: bit q of the key is bit p[q] of j.
void class_keys(const uint64_t* J, uint64_t k, const std::vector<uint32_t>& p, uint32_t R,
                std::vector<uint64_t>& key) {
  key.assign(k, 0);
  for (uint64_t i = 0; i < k; ++i) {
    uint64_t t = 0;
    for (uint32_t q = 0; q < R; ++q) t |= ((J[i] >> p[q]) & 1ull) << q;
    key[i] = t;
  }
}

// Inverse of the mu x mu Vandermonde matrix V[a][u] = z_u^a by Gauss-Jordan
// elimination with partial pivoting (FP64); returns its 1-norm condition.
double vandermonde_inverse(uint32_t M, const uint64_t* l, uint32_t mu, std::complex<double>* out) {
  using cd = std::complex<double>;
  const uint64_t N = 1ull << M;
  std::vector<cd> a(size_t(mu) * mu), inv(size_t(mu) * mu, cd(0.0, 0.0));
  for (uint32_t r = 0; r < mu; ++r)
    for (uint32_t u = 0; u < mu; ++u) {
      const unsigned __int128 e = (unsigned __int128)(r) * l[u];
      const double x = std::ldexp(double(uint64_t(e % N)), -int(M));     // (a l_u mod N) / N
      a[size_t(r) * mu + u] = cd(std::cos(2.0 * M_PI * x), std::sin(2.0 * M_PI * x));
    }
  double norm_a = 0.0;
  for (uint32_t u = 0; u < mu; ++u) {
    double col = 0.0;
    for (uint32_t r = 0; r < mu; ++r) col += std::abs(a[size_t(r) * mu + u]);
    norm_a = std::max(norm_a, col);
  }
  for (uint32_t r = 0; r < mu; ++r) inv[size_t(r) * mu + r] = cd(1.0, 0.0);
  for (uint32_t c = 0; c < mu; ++c) {
    uint32_t piv = c;
    for (uint32_t r = c + 1; r < mu; ++r)
      if (std::abs(a[size_t(r) * mu + c]) > std::abs(a[size_t(piv) * mu + c])) piv = r;
    if (std::abs(a[size_t(piv) * mu + c]) == 0.0) return INFINITY;
    if (piv != c)
      for (uint32_t u = 0; u < mu; ++u) {
        std::swap(a[size_t(piv) * mu + u], a[size_t(c) * mu + u]);
        std::swap(inv[size_t(piv) * mu + u], inv[size_t(c) * mu + u]);
      }
    const cd d = a[size_t(c) * mu + c];
    for (uint32_t u = 0; u < mu; ++u) {
      a[size_t(c) * mu + u] /= d;
      inv[size_t(c) * mu + u] /= d;
    }
    for (uint32_t r = 0; r < mu; ++r) {
      if (r == c) continue;
      const cd f = a[size_t(r) * mu + c];
      if (f == cd(0.0, 0.0)) continue;
      for (uint32_t u = 0; u < mu; ++u) {
        a[size_t(r) * mu + u] -= f * a[size_t(c) * mu + u];
        inv[size_t(r) * mu + u] -= f * inv[size_t(c) * mu + u];
      }
    }
  }
  double norm_i = 0.0;
  for (uint32_t u = 0; u < mu; ++u) {
    double col = 0.0;
    for (uint32_t r = 0; r < mu; ++r) col += std::abs(inv[size_t(r) * mu + u]);
    norm_i = std::max(norm_i, col);
  }
  std::copy(inv.begin(), inv.end(), out);
  return norm_a * norm_i;
}

sdft_status build_sas(uint32_t M, const uint64_t* J, uint64_t k, sdft_prec prec, uint32_t R_req, Sas& S) {
  if (!J || k == 0) return SDFT_ERR_ARG;
  if (prec != SDFT_C64 && prec != SDFT_C128) return SDFT_ERR_ARG;
  if (k > (1ull << SDFT_MAX_LOG2K)) return SDFT_ERR_UNSUPPORTED;
  uint64_t mask = 0;
  sdft_status st = split_levels(M, J, k, mask);
  if (st != SDFT_OK) return st;
  std::vector<uint32_t> levels;
  for (uint32_t l = 0; l < M; ++l)
    if (mask >> l & 1) levels.push_back(l);
  const uint32_t L = uint32_t(levels.size());
  if (R_req > L || R_req > kSasMaxR) return SDFT_ERR_ARG;

  // Choose R: among R with mu* <= kSasMaxMu whose class systems are well
  // enough conditioned for the arithmetic (1-norm condition <= 32 for
  // complex64, 100 for complex128), the smallest operation count; if none is,
  // the best-conditioned one. A class solve multiplies the relative error of
  // the stage-1 values (about 2e-7 in complex64, 2e-15 in complex128) by at
  // most its condition, so under these caps the result stays within 1e-5
  // (complex64) and 1e-12 (complex128) of the exact coefficients.
  std::vector<uint64_t> key;
  auto counts = [&](uint32_t R, std::vector<uint32_t>& mu) {
    std::vector<uint32_t> p(levels.begin(), levels.begin() + R);
    class_keys(J, k, p, R, key);
    mu.assign(size_t(1) << R, 0);
    for (uint64_t i = 0; i < k; ++i) ++mu[key[i]];
  };
  // Largest condition number of the class systems for the current keys.
  auto worst_cond = [&](uint32_t R, const std::vector<uint32_t>& mu) {
    const uint64_t nk = 1ull << R;
    std::vector<uint64_t> first(nk + 1, 0), members(k);
    for (uint64_t t = 0; t < nk; ++t) first[t + 1] = first[t] + mu[t];
    std::vector<uint64_t> fill(first.begin(), first.end() - 1);
    for (uint64_t i = 0; i < k; ++i) members[fill[key[i]]++] = J[i];
    double worst = 1.0;
    std::vector<std::complex<double>> scratch;
    for (uint64_t t = 0; t < nk; ++t) {
      if (mu[t] < 2) continue;
      std::sort(members.begin() + first[t], members.begin() + first[t + 1]);
      scratch.resize(size_t(mu[t]) * mu[t]);
      worst = std::max(worst, vandermonde_inverse(M, &members[first[t]], mu[t], scratch.data()));
    }
    return worst;
  };
  const double cond_limit = prec == SDFT_C64 ? 32.0 : 100.0;
  uint32_t R = R_req;
  std::vector<uint32_t> mu;
  if (R_req == 0) {
    uint32_t lk = 0;
    while ((1ull << lk) < k) ++lk;                      // ceil(log2 k)
    const uint32_t lo = lk > 4 ? lk - 4 : 0, hi = std::min<uint32_t>({L, lk + 2, kSasMaxR});
    double best = -1.0, best_cond = INFINITY;
    uint32_t R_cond = 0;
    bool any = false;
    for (uint32_t c = std::min(lo, hi); c <= hi; ++c) {
      counts(c, mu);
      const uint32_t ms = *std::max_element(mu.begin(), mu.end());
      if (ms > kSasMaxMu) continue;
      const double cond = worst_cond(c, mu);
      if (!any || cond < best_cond) {
        best_cond = cond;
        R_cond = c;
      }
      any = true;
      if (cond > cond_limit) continue;
      double sq = 0.0;
      for (uint32_t m : mu) sq += double(m) * m;
      const double cost = 1.5 * c * double(1ull << c) * ms + 6.0 * sq;
      if (best < 0.0 || cost < best) {
        best = cost;
        R = c;
      }
    }
    if (!any) return SDFT_ERR_UNSUPPORTED;
    if (best < 0.0) R = R_cond;
  }
  counts(R, mu);
  S.M = M;
  S.R = R;
  S.k = k;
  S.prec = prec;
  S.pivots.assign(levels.begin(), levels.begin() + R);
  S.mu_star = *std::max_element(mu.begin(), mu.end());
  if (S.mu_star > kSasMaxMu) return SDFT_ERR_UNSUPPORTED;
  const uint64_t nk = 1ull << R;
  S.occupied = 0;
  for (uint32_t m : mu) S.occupied += (m > 0);

  // Output order: by class key, then by value.
  std::vector<uint64_t> first(nk + 1, 0);
  for (uint64_t t = 0; t < nk; ++t) first[t + 1] = first[t] + mu[t];
  S.order.assign(k, 0);
  {
    std::vector<uint64_t> fill(first.begin(), first.end() - 1);
    for (uint64_t i = 0; i < k; ++i) S.order[fill[key[i]]++] = J[i];
    for (uint64_t t = 0; t < nk; ++t) std::sort(S.order.begin() + first[t], S.order.begin() + first[t + 1]);
  }

  // Virtual support: a representative per key prefix (length q, prefix value)
  // finds, for an empty class, the longest prefix J occupies.
  const uint32_t rho = R ? S.pivots[R - 1] + 1 : 0;
  const uint64_t rmask = rho >= 64 ? ~0ull : ((1ull << rho) - 1);
  std::vector<std::vector<int64_t>> rep(R + 1);
  for (uint32_t q = 0; q <= R; ++q) rep[q].assign(size_t(1) << q, -1);
  for (uint64_t i = 0; i < k; ++i)
    for (uint32_t q = 0; q <= R; ++q) {
      int64_t& slot = rep[q][key[i] & ((1ull << q) - 1)];
      if (slot < 0) slot = int64_t(i);
    }
  std::vector<uint64_t> V(nk);
  for (uint64_t t = 0; t < nk; ++t) {
    int64_t who = rep[R][t];
    if (who >= 0) {
      V[t] = J[who] & rmask;
      continue;
    }
    uint32_t q0 = R;
    while (rep[q0][t & ((1ull << q0) - 1)] < 0) --q0;     // q0 = 0 always has a member
    const uint64_t base = J[rep[q0][t & ((1ull << q0) - 1)]] & ((1ull << S.pivots[q0]) - 1);
    uint64_t v = base;
    for (uint32_t q = q0; q < R; ++q) v |= ((t >> q) & 1ull) << S.pivots[q];
    V[t] = v;
  }

  // Shifted sample sets: row a is I_r + a (mod N), in the virtual plan's order.
  Plan vp;
  st = build_plan(M, V.data(), nk, prec, vp);
  if (st != SDFT_OK) return st;
  if (vp.pivots != S.pivots) return SDFT_ERR_NOT_HOMOGENEOUS;   // cannot happen by construction
  const uint64_t N = 1ull << M;
  S.samples.resize(size_t(S.mu_star) * nk);
  for (uint32_t a = 0; a < S.mu_star; ++a)
    for (uint64_t t = 0; t < nk; ++t) S.samples[size_t(a) * nk + t] = (vp.I[t] + a) & (N - 1);

  // Per-class inverses and per-output metadata.
  S.meta.resize(k);
  S.winv.clear();
  S.max_cond = 1.0;
  for (uint64_t t = 0; t < nk; ++t) {
    const uint32_t m = mu[t];
    if (!m) continue;
    if (S.winv.size() + size_t(m) * m > 0xffffffffull) return SDFT_ERR_UNSUPPORTED;
    const uint32_t woff = uint32_t(S.winv.size());
    S.winv.resize(S.winv.size() + size_t(m) * m);
    const double cond = vandermonde_inverse(M, &S.order[first[t]], m, &S.winv[woff]);
    if (!std::isfinite(cond)) return SDFT_ERR_UNSUPPORTED;
    S.max_cond = std::max(S.max_cond, cond);
    for (uint32_t u = 0; u < m; ++u) S.meta[first[t] + u] = SasOut{uint32_t(t), uint16_t(u), uint16_t(m), woff, 0};
  }

  S.virt.swap(V);
  return SDFT_OK;
}

// Stage 2: coefficient i of instance b = sum_a Winv_t[u][a] Y[b][a][t]. A
// thread takes coefficient i of kSasDecodeB instances b = blockIdx.y + q
// gridDim.y (q < kSasDecodeB): its class's inverse row is read once for all of
// them and their values are gathered together.
// GATHERED: the stage-1 values arrive in output order, G[b][i] = Y[b][u_i][t_i]
// (k per instance), so the mu values of coefficient i's class are
// G[b][i - u + a], a < mu: adjacent, read from consecutive addresses by
// consecutive threads. The sums are formed in the same order either way.
constexpr uint32_t kSasDecodeB = 8;
template <class R, bool GATHERED = false>
__global__ void __launch_bounds__(256) k_sas_decode(const typename KT<R>::C* __restrict__ y,
                                                    typename KT<R>::C* __restrict__ out,
                                                    const SasOut* __restrict__ meta,
                                                    const typename KT<R>::C* __restrict__ winv, uint64_t k,
                                                    uint64_t nk, uint32_t mu_star, uint64_t batch,
                                                    uint64_t winv_len, int* status) {
  using C = typename KT<R>::C;
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const SasOut m = meta[i];
  // debug build: the class column, its size and its inverse row in range
  if (!in_bounds(m.t < nk && m.mu >= 1 && m.mu <= mu_star && m.u < m.mu &&
                     uint64_t(m.woff) + uint64_t(m.u + 1) * m.mu <= winv_len, status))
    return;
  const C* wrow = winv + m.woff + uint32_t(m.u) * m.mu;
  for (uint64_t b0 = blockIdx.y; b0 < batch; b0 += uint64_t(gridDim.y) * kSasDecodeB) {
    R re[kSasDecodeB], im[kSasDecodeB];
#pragma unroll
    for (uint32_t q = 0; q < kSasDecodeB; ++q) re[q] = im[q] = R(0);
    for (uint32_t a = 0; a < m.mu; ++a) {
      const C w = wrow[a];
#pragma unroll
      for (uint32_t q = 0; q < kSasDecodeB; ++q) {
        const uint64_t b = b0 + uint64_t(q) * gridDim.y;
        if (b < batch) {
          const C v = GATHERED ? y[b * k + (i - m.u + a)] : y[(b * uint64_t(mu_star) + a) * nk + m.t];
          re[q] = fma(w.x, v.x, fma(-w.y, v.y, re[q]));
          im[q] = fma(w.x, v.y, fma(w.y, v.x, im[q]));
        }
      }
    }
#pragma unroll
    for (uint32_t q = 0; q < kSasDecodeB; ++q) {
      const uint64_t b = b0 + uint64_t(q) * gridDim.y;
      if (b < batch) {
        C o;
        o.x = re[q];
        o.y = im[q];
        out[b * k + i] = o;
      }
    }
  }
}

// Both stages in one launch for complete isolation (mu* = 1: every class holds
// one member, coefficient i = Winv_i Y[t_i]) when one to four virtual instances
// fill one tile (TB - 2 <= R <= TB) and k <= 2^TB: CTA c takes tiles c, c + G,
// ... (the level kernel's passes with the last stage scaled), keeps the
// per-coefficient pairs (t_i, Winv_i) in shared memory for the whole launch,
// and after the passes writes every coefficient straight from the tile. The
// stage-1 output never leaves the SM; the product is formed as in k_sas_decode,
// so both paths give the same bits. (With mu* > 1 the class solves need mu*
// tiles per instance and their inverse rows: they stay a launch of their own.)
// GATHER (mu* > 1, the same tile shapes, k <= 8192): the kernel runs stage 1
// over the batch x mu* shifted sample sets (row r: instance r / mu*, shift
// r mod mu*) and writes, from the row of shift a, only the values the class
// solves read: G[b][i] = Y[b][a][t_i] for every coefficient i whose place in
// its class is u_i = a. The workspace then holds k values per instance in output
// order instead of mu* x 2^R, and stage 2 (k_sas_decode, GATHERED) reads a
// class's mu values side by side.
template <class R>
struct SasFusedArgs {
  LevelArgs<R> a;                        // level 0 of the virtual plan over the tiles
  const uint16_t* col;                   // t_i: column of the stage-1 output
  const typename KT<R>::C* w;            // Winv_i (1 x 1 inverses)
  typename KT<R>::C* out;                // batch x k coefficients (GATHER: the batch x k workspace G)
  uint64_t k, rows;                      // coefficients per instance; rows (virtual instances): batch x mu*
  const uint32_t* gtab;                  // GATHER: t_i | i << 16, grouped by u_i
  uint32_t mu_star;
  uint32_t goff[kSasMaxMu + 1];          // GATHER: entries of shift a are [goff[a], goff[a + 1])
};

template <class R>
constexpr uint32_t sas_fused_smem() {
  return kLevelBufs * kTileBytes + 64 + kMidTwBytes +
         (1u << KT<R>::TB) * uint32_t(sizeof(typename KT<R>::C) + sizeof(uint16_t)) + 1024;
}

// PHI = R: a tile holds 2^(TB - R) consecutive rows (virtual instances) of
// 2^R values; row q of tile j is row j 2^(TB - R) + q of the batch (rows past
// the last are the zero fill of the tile's load and are skipped).
template <class R, bool GATHER, int PHI>
__global__ void __launch_bounds__(KT<R>::NT, 2)
    k_sas_fused(const __grid_constant__ CUtensorMap src, const __grid_constant__ SasFusedArgs<R> fa) {
  using C = typename KT<R>::C;
  constexpr int TB = KT<R>::TB;
  static_assert(PHI >= 5 && PHI <= TB, "one or more whole rows per tile");
  constexpr uint32_t RP = 1u << (TB - PHI);        // rows per tile
  constexpr uint32_t NT = KT<R>::NT;
  constexpr int NREG = reg_twiddles(TB, 4, 0, PHI);
  constexpr int MLO = mid_pass_lo(TB, 4, 0, PHI), MHI = mid_pass_hi(TB, 4, 0, PHI);
  constexpr bool MIDSM = MLO < MHI && (1u << MHI) * sizeof(C) <= kMidTwBytes;
  extern __shared__ char smem_raw[];
  char* smem = align1024(smem_raw);
  const uint32_t bar0 = ptx::smem_addr(smem + kLevelBufs * kTileBytes);
  const uint32_t tid = threadIdx.x;
  C* midtw = reinterpret_cast<C*>(smem + kLevelBufs * kTileBytes + 64);
  C* ws = reinterpret_cast<C*>(smem + kLevelBufs * kTileBytes + 64 + kMidTwBytes);
  uint16_t* cs = reinterpret_cast<uint16_t*>(ws + (1u << TB));
  uint32_t* gs = reinterpret_cast<uint32_t*>(ws);    // GATHER: the gather table (k <= 8192 entries)
  {
    const uint32_t used = uint32_t(smem - smem_raw) + sas_fused_smem<R>() - 1024;
    int bad = 0;
    if (ptx::dynamic_smem_size() < used) bad = kBadSmem;
    else if (reinterpret_cast<uintptr_t>(&src) & 63u) bad = kBadMap;
    else if (reinterpret_cast<uintptr_t>(fa.a.tw) & 15u) bad = kBadTable;
    if (bad) {
      if (tid == 0) atomicCAS(fa.a.status, 0, bad);
      return;
    }
  }
  const uint64_t G = gridDim.x;
  if (blockIdx.x >= fa.a.n_tiles) return;
  const uint64_t n = (fa.a.n_tiles - blockIdx.x + G - 1) / G;     // tiles of this CTA
  uint32_t load_buf = 0;
  auto issue_load = [&](uint64_t j) {
    const uint32_t b = load_buf;
    load_buf = (load_buf + 1 == uint32_t(kLevelBufs)) ? 0u : load_buf + 1;
    const uint32_t bar = bar0 + 8 * b;
    ptx::mbar_arrive_expect_tx(bar, kTileBytes);
    int row = int(int64_t(blockIdx.x + j * G) * fa.a.b_step1), c3 = 0;
    level_coords_in_bounds(fa.a, row, c3);
    ptx::tma_load_4d(ptx::smem_addr(smem + b * kTileBytes), &src, bar, 0, row, 0, c3);
  };
  if (tid == 0) {
    for (int b = 0; b < kLevelBufs; ++b) ptx::mbar_init(bar0 + 8 * b, 1);
    ptx::fence_mbar_init();
    ptx::prefetch_tensormap(&src);
    for (uint64_t j = 0; j < n && j < uint64_t(kLevelBufs); ++j) issue_load(j);
  }
  const C* tw = static_cast<const C*>(fa.a.tw);
  C wreg[NREG > 0 ? NREG : 1];
  load_reg_twiddles<R, 4, 0, PHI>(tw, tid, wreg);
  if constexpr (MIDSM) {
    for (uint32_t e = (1u << MLO) + tid; e < (1u << MHI); e += NT) midtw[e] = tw[e];
  }
  for (uint64_t i = tid; i < fa.k; i += NT) {   // the decode (gather) table, once per CTA
    if constexpr (GATHER) {
      gs[i] = fa.gtab[i];
    } else {
      ws[i] = fa.w[i];
      cs[i] = fa.col[i];
    }
  }
  __syncthreads();
  const uint32_t midtw_addr = ptx::smem_addr(midtw);
  const R sc = R(fa.a.scale);
  bool aborted = false;
  uint32_t b = 0, phases = 0;
  uint64_t j = 0;
  for (; j < n; ++j, b = (b + 1 == uint32_t(kLevelBufs)) ? 0u : b + 1) {
    char* buf = smem + b * kTileBytes;
    const bool ok = ptx::mbar_wait_bounded(bar0 + 8 * b, (phases >> b) & 1u, fa.a.timeout_ns);
    phases ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    // after the first pass every thread is done with tile j-1: its buffer takes tile j+1
    auto refill = [&]() {
      if (tid == 0 && j >= 1 && j + kLevelBufs - 1 < n) issue_load(j + kLevelBufs - 1);
    };
    run_passes<R, 4, 0, PHI, true, 0, 0, MIDSM>(buf, wreg, fa.a.tw0, tw, tid, sc, midtw_addr, refill);
#pragma unroll 1
    for (uint32_t q = 0; q < RP; ++q) {
      const uint64_t r = (blockIdx.x + j * G) * RP + q;
      if (r >= fa.rows) break;
      const uint32_t base = q << PHI;                 // the row's first value in the tile
      if constexpr (GATHER) {
        const uint32_t a = uint32_t(r % fa.mu_star);
        C* gb = fa.out + (r / fa.mu_star) * fa.k;
        for (uint32_t e = fa.goff[a] + tid; e < fa.goff[a + 1]; e += NT) {
          const uint32_t g = gs[e];
          const uint32_t t = g & 0xffffu, i = g >> 16;
          if (!in_bounds(t < (1u << PHI) && i < fa.k, fa.a.status)) continue;   // debug build
          gb[i] = *reinterpret_cast<const C*>(buf + row_part<R>(base + t) + xor_part<R>(base + t));
        }
      } else {
        C* ob = fa.out + r * fa.k;
        for (uint64_t i = tid; i < fa.k; i += NT) {
          const C w = ws[i];
          uint32_t t = cs[i];
          if (!in_bounds(t < (1u << PHI), fa.a.status)) t = 0;   // debug build
          const C v = *reinterpret_cast<const C*>(buf + row_part<R>(base + t) + xor_part<R>(base + t));
          C o;
          o.x = fma(w.x, v.x, fma(-w.y, v.y, R(0)));
          o.y = fma(w.x, v.y, fma(w.y, v.x, R(0)));
          ob[i] = o;
        }
      }
    }
  }
  if (tid == 0 && aborted) {
    const uint64_t last = (j + kLevelBufs - 2 > uint64_t(kLevelBufs - 1)) ? j + kLevelBufs - 2
                                                                           : uint64_t(kLevelBufs - 1);
    for (uint64_t q = j; q <= last && q < n; ++q)
      ptx::mbar_wait_bounded(bar0 + 8 * uint32_t(q % kLevelBufs), uint32_t((q / kLevelBufs) & 1),
                             drain_bound(fa.a.timeout_ns));
    atomicExch(fa.a.status, int(SDFT_ERR_TIMEOUT));
  }
}

// One launch of k_sas_fused over the batch: the coefficients (mu* = 1) or,
// with `gather`, the gathered stage-1 values G into d_out (mu* > 1).
template <class R>
sdft_status launch_sas_fused(const Sas& S, uint64_t batch, const void* d_samples, void* d_out, bool gather,
                             cudaStream_t st) {
  const Plan& vp = S.vplan->p;
  const uint64_t rows = batch * (gather ? S.mu_star : 1u);
  CUtensorMap ms, md;
  SasFusedArgs<R> fa{};
  sdft_status s = level0_setup<R>(vp, rows, d_samples, const_cast<void*>(d_samples), ms, md, fa.a);
  if (s != SDFT_OK) return s;
  fa.col = S.d_col;
  fa.w = static_cast<const typename KT<R>::C*>(S.d_w1);
  fa.out = static_cast<typename KT<R>::C*>(d_out);
  fa.k = S.k;
  fa.rows = rows;
  fa.gtab = S.d_gather;
  fa.mu_star = gather ? S.mu_star : 1u;
  if (gather)
    for (uint32_t a = 0; a <= S.mu_star; ++a) fa.goff[a] = S.goff[a];
  constexpr int TB = KT<R>::TB;
  const int d = int(TB) - int(S.R);                 // R in [TB - 2, TB] (sas_*_shape)
  auto fn = gather ? (d == 0 ? k_sas_fused<R, true, TB> : d == 1 ? k_sas_fused<R, true, TB - 1>
                                                                 : k_sas_fused<R, true, TB - 2>)
                   : (d == 0 ? k_sas_fused<R, false, TB> : d == 1 ? k_sas_fused<R, false, TB - 1>
                                                                  : k_sas_fused<R, false, TB - 2>);
  s = ensure_smem(reinterpret_cast<const void*>(fn), int(sas_fused_smem<R>()));
  if (s != SDFT_OK) return s;
  const uint64_t max_grid = 2ull * uint64_t(sm_count());
  const unsigned grid = unsigned(fa.a.n_tiles < max_grid ? fa.a.n_tiles : max_grid);
  fn<<<grid, KT<R>::NT, sas_fused_smem<R>(), st>>>(ms, fa);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

// Complete isolation, one to four virtual instances per tile (R in
// [TB - 2, TB]), at most a tile's worth of coefficients.
bool sas_tile_shape(const Sas& S) {
  const uint32_t TB = S.prec == SDFT_C64 ? KT<float>::TB : KT<double>::TB;
  return S.R <= TB && S.R + 2 >= TB && S.k <= (1ull << TB);
}
bool sas_fused_shape(const Sas& S) { return S.mu_star == 1 && sas_tile_shape(S); }
bool sas_fused_applies(const Sas& S) { return !S.two_stage && S.d_col && S.d_w1 && sas_fused_shape(S); }
// mu* > 1 with the same tile shape: stage 1 writes only the values stage 2 reads.
// The gather table (one 32-bit entry per coefficient) sits in the shared
// memory of the mu* = 1 table, 2^TB complex values: up to 8192 coefficients.
bool sas_gather_shape(const Sas& S) {
  const uint32_t TB = S.prec == SDFT_C64 ? KT<float>::TB : KT<double>::TB;
  const uint64_t cap = (uint64_t(1) << TB) * uint64_t(elem_bytes(S.prec)) / sizeof(uint32_t);
  return S.mu_star > 1 && S.mu_star <= kSasMaxMu && S.R <= TB && S.R + 2 >= TB && S.k <= cap;
}
bool sas_gather_applies(const Sas& S) { return !S.two_stage && S.d_gather && sas_gather_shape(S); }

void free_sas(Sas& S) {
  if (S.vplan) sdft_plan_destroy(S.vplan);
  if (S.d_meta) cudaFree(S.d_meta);
  if (S.d_winv) cudaFree(S.d_winv);
  if (S.d_col) cudaFree(S.d_col);
  if (S.d_w1) cudaFree(S.d_w1);
  if (S.d_gather) cudaFree(S.d_gather);
  S.d_gather = nullptr;
  S.d_col = nullptr;
  S.d_w1 = nullptr;
  S.vplan = nullptr;
  S.d_meta = nullptr;
  S.d_winv = nullptr;
}

}  // namespace
}  // namespace sdft

struct sdft_sas_s {
  sdft::Sas s;
};

extern "C" {

sdft_status sdft_sas_create(uint32_t log2N, const uint64_t* J, uint64_t k, sdft_prec prec, uint32_t R,
                            uint32_t flags, sdft_sas* out) {
  using namespace sdft;
  if (!out) return SDFT_ERR_ARG;
  *out = nullptr;
  if (flags & ~(SDFT_PLAN_HOST_ONLY | SDFT_SAS_TWO_STAGE)) return SDFT_ERR_ARG;
  sdft_sas_s* h = new (std::nothrow) sdft_sas_s();
  if (!h) return SDFT_ERR_NOMEM;
  Sas& S = h->s;
  S.two_stage = (flags & SDFT_SAS_TWO_STAGE) != 0;
  sdft_status st;
  try {
    st = build_sas(log2N, J, k, prec, R, S);
  } catch (const std::bad_alloc&) {
    st = SDFT_ERR_NOMEM;
  }
  if (st == SDFT_OK && !(flags & SDFT_PLAN_HOST_ONLY)) {
    st = sdft_plan_create(log2N, S.virt.data(), S.virt.size(), prec, 0, &S.vplan);
    cudaError_t e = cudaSuccess;
    if (st == SDFT_OK) e = cudaGetDevice(&S.device);
    const size_t eb = size_t(elem_bytes(prec));
    if (st == SDFT_OK && e == cudaSuccess) e = cudaMalloc(&S.d_meta, sizeof(SasOut) * S.meta.size());
    if (st == SDFT_OK && e == cudaSuccess) e = cudaMalloc(&S.d_winv, eb * std::max<size_t>(S.winv.size(), 1));
    if (st == SDFT_OK && e == cudaSuccess)
      e = cudaMemcpy(S.d_meta, S.meta.data(), sizeof(SasOut) * S.meta.size(), cudaMemcpyHostToDevice);
    if (st == SDFT_OK && e == cudaSuccess) {
      std::vector<double> w(2 * S.winv.size());
      for (size_t i = 0; i < S.winv.size(); ++i) {
        w[2 * i] = S.winv[i].real();
        w[2 * i + 1] = S.winv[i].imag();
      }
      if (prec == SDFT_C64) {
        std::vector<float> wf(w.begin(), w.end());      // FP64 inverse rounded once
        e = cudaMemcpy(S.d_winv, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice);
      } else {
        e = cudaMemcpy(S.d_winv, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
      }
    }
    // the one-launch path's table: t_i and the 1 x 1 inverse of coefficient i's class,
    // the same rounded values stage 2 reads
    if (st == SDFT_OK && e == cudaSuccess && sas_fused_shape(S)) {
      std::vector<uint16_t> col(S.k);
      std::vector<double> w1(2 * S.k);
      for (uint64_t i = 0; i < S.k; ++i) {
        col[i] = uint16_t(S.meta[i].t);
        w1[2 * i] = S.winv[S.meta[i].woff].real();
        w1[2 * i + 1] = S.winv[S.meta[i].woff].imag();
      }
      e = cudaMalloc(reinterpret_cast<void**>(&S.d_col), sizeof(uint16_t) * S.k);
      if (e == cudaSuccess) e = cudaMalloc(&S.d_w1, eb * S.k);
      if (e == cudaSuccess) e = cudaMemcpy(S.d_col, col.data(), sizeof(uint16_t) * S.k, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        if (prec == SDFT_C64) {
          std::vector<float> wf(w1.begin(), w1.end());
          e = cudaMemcpy(S.d_w1, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice);
        } else {
          e = cudaMemcpy(S.d_w1, w1.data(), sizeof(double) * w1.size(), cudaMemcpyHostToDevice);
        }
      }
    }
    // the gathered path's table: coefficient i (its column t_i) in the group of
    // the shift u_i, the place of i in its class
    if (st == SDFT_OK && e == cudaSuccess && sas_gather_shape(S)) {
      std::vector<uint32_t> g;
      g.reserve(S.k);
      S.goff.assign(S.mu_star + 1, 0);
      for (uint32_t a = 0; a < S.mu_star; ++a) {
        S.goff[a] = uint32_t(g.size());
        for (uint64_t i = 0; i < S.k; ++i)
          if (S.meta[i].u == a) g.push_back(S.meta[i].t | uint32_t(i) << 16);
      }
      S.goff[S.mu_star] = uint32_t(g.size());
      e = cudaMalloc(reinterpret_cast<void**>(&S.d_gather), sizeof(uint32_t) * g.size());
      if (e == cudaSuccess)
        e = cudaMemcpy(S.d_gather, g.data(), sizeof(uint32_t) * g.size(), cudaMemcpyHostToDevice);
    }
    if (st == SDFT_OK && e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? SDFT_ERR_NOMEM : cuda_fail(e);
  }
  if (st != SDFT_OK) {
    free_sas(S);
    delete h;
    return st;
  }
  *out = h;
  return SDFT_OK;
}

sdft_status sdft_sas_info(sdft_sas sas, uint32_t* R, uint32_t* mu_star, uint64_t* samples_per_instance,
                          uint32_t* occupied_classes, double* max_cond) {
  if (!sas) return SDFT_ERR_ARG;
  const sdft::Sas& S = sas->s;
  if (R) *R = S.R;
  if (mu_star) *mu_star = S.mu_star;
  if (samples_per_instance) *samples_per_instance = uint64_t(S.mu_star) << S.R;
  if (occupied_classes) *occupied_classes = S.occupied;
  if (max_cond) *max_cond = S.max_cond;
  return SDFT_OK;
}

sdft_status sdft_sas_pivots(sdft_sas sas, uint32_t* r) {
  if (!sas || (!r && sas->s.R)) return SDFT_ERR_ARG;
  std::copy(sas->s.pivots.begin(), sas->s.pivots.end(), r);
  return SDFT_OK;
}

sdft_status sdft_sas_sample_indices(sdft_sas sas, uint64_t* idx) {
  if (!sas || !idx) return SDFT_ERR_ARG;
  std::copy(sas->s.samples.begin(), sas->s.samples.end(), idx);
  return SDFT_OK;
}

sdft_status sdft_sas_support_order(sdft_sas sas, uint64_t* J) {
  if (!sas || !J) return SDFT_ERR_ARG;
  std::copy(sas->s.order.begin(), sas->s.order.end(), J);
  return SDFT_OK;
}

sdft_status sdft_sas_workspace_bytes(sdft_sas sas, uint64_t batch, uint64_t* bytes) {
  if (!sas || !bytes) return SDFT_ERR_ARG;
  const sdft::Sas& S = sas->s;
  *bytes = batch * (uint64_t(S.mu_star) << S.R) * uint64_t(sdft::elem_bytes(S.prec));
  return SDFT_OK;
}

sdft_status sdft_sas_execute(sdft_sas sas, uint64_t batch, const void* d_samples, void* d_work, void* d_coeffs,
                             void* stream) {
  using namespace sdft;
  if (!sas) return SDFT_ERR_ARG;
  Sas& S = sas->s;
  if (!S.vplan) return SDFT_ERR_NO_DEVICE;
  if (batch == 0) return SDFT_OK;
  if (!d_samples || !d_work || !d_coeffs) return SDFT_ERR_ARG;
  const uint64_t eb = uint64_t(elem_bytes(S.prec));
  const uint64_t nk = 1ull << S.R;
  const uint64_t wbytes = batch * S.mu_star * nk * eb, obytes = batch * S.k * eb;
  const uintptr_t w = reinterpret_cast<uintptr_t>(d_work), o = reinterpret_cast<uintptr_t>(d_coeffs);
  if (w < o + obytes && o < w + wbytes) return SDFT_ERR_ARG;     // the decoder reads work while writing coeffs
  if ((w | o) & 15u) return SDFT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sas_fused_applies(S)) {
    if (reinterpret_cast<uintptr_t>(d_samples) & 15u) return SDFT_ERR_ARG;
    const uintptr_t in = reinterpret_cast<uintptr_t>(d_samples);
    if (in < o + obytes && o < in + wbytes) return SDFT_ERR_ARG;   // samples are read while coeffs are written
    return S.prec == SDFT_C64 ? launch_sas_fused<float>(S, batch, d_samples, d_coeffs, false, st)
                              : launch_sas_fused<double>(S, batch, d_samples, d_coeffs, false, st);
  }
  // gathered stage 1 where the workspace is not the samples buffer (tiles of
  // later instances are still to be read when earlier ones are written)
  const uintptr_t in = reinterpret_cast<uintptr_t>(d_samples);
  const bool gather = sas_gather_applies(S) && !(in < w + wbytes && w < in + wbytes) && !(in & 15u);
  sdft_status s = SDFT_OK;
  if (gather)
    s = S.prec == SDFT_C64 ? launch_sas_fused<float>(S, batch, d_samples, d_work, true, st)
                           : launch_sas_fused<double>(S, batch, d_samples, d_work, true, st);
  else
    s = sdft_execute_strided(S.vplan, batch * S.mu_star, d_samples, d_work, stream);
  if (s != SDFT_OK) return s;
  const dim3 block(256);
  const uint64_t rows = (batch + kSasDecodeB - 1) / kSasDecodeB;
  const dim3 grid(unsigned((S.k + 255) / 256), unsigned(std::min<uint64_t>(rows, 65535)));
  auto decode = [&](auto* work, auto* coeffs, auto* winv) {
    using C = std::remove_const_t<std::remove_pointer_t<decltype(work)>>;
    using RR = decltype(C{}.x);
    if (gather)
      k_sas_decode<RR, true><<<grid, block, 0, st>>>(work, coeffs, S.d_meta, winv, S.k, nk, S.mu_star, batch,
                                                     S.winv.size(), S.vplan->p.d_status);
    else
      k_sas_decode<RR, false><<<grid, block, 0, st>>>(work, coeffs, S.d_meta, winv, S.k, nk, S.mu_star, batch,
                                                      S.winv.size(), S.vplan->p.d_status);
  };
  if (S.prec == SDFT_C64)
    decode(static_cast<const float2*>(d_work), static_cast<float2*>(d_coeffs), static_cast<const float2*>(S.d_winv));
  else
    decode(static_cast<const double2*>(d_work), static_cast<double2*>(d_coeffs),
           static_cast<const double2*>(S.d_winv));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

sdft_status sdft_sas_path(sdft_sas sas, uint32_t* launches, uint64_t* work_values) {
  using namespace sdft;
  if (!sas) return SDFT_ERR_ARG;
  const Sas& S = sas->s;
  uint32_t l = 2;
  uint64_t v = uint64_t(S.mu_star) << S.R;
  if (!S.two_stage && sas_fused_shape(S)) {
    l = 1;
    v = 0;
  } else if (!S.two_stage && sas_gather_shape(S)) {
    v = S.k;
  }
  if (launches) *launches = l;
  if (work_values) *work_values = v;
  return SDFT_OK;
}

sdft_status sdft_sas_destroy(sdft_sas sas) {
  if (!sas) return SDFT_ERR_ARG;
  sdft::free_sas(sas->s);
  delete sas;
  return SDFT_OK;
}

}  // extern "C"
