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
#include <vector>

#include "kernels.cuh"
#include "launch.hpp"
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
  // complex64, 1000 for complex128), the smallest operation count; if none is,
  // the best-conditioned one.
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
  const double cond_limit = prec == SDFT_C64 ? 32.0 : 1000.0;
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

// Stage 2: coefficient i of instance b = sum_a Winv_t[u][a] Y[b][a][t].
template <class R>
__global__ void __launch_bounds__(256) k_sas_decode(const typename KT<R>::C* __restrict__ y,
                                                    typename KT<R>::C* __restrict__ out,
                                                    const SasOut* __restrict__ meta,
                                                    const typename KT<R>::C* __restrict__ winv, uint64_t k,
                                                    uint64_t nk, uint32_t mu_star, uint64_t batch) {
  using C = typename KT<R>::C;
  const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const SasOut m = meta[i];
  for (uint64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const C* yb = y + b * uint64_t(mu_star) * nk + m.t;
    R re = 0, im = 0;
    for (uint32_t a = 0; a < m.mu; ++a) {
      const C w = winv[m.woff + uint32_t(m.u) * m.mu + a];
      const C v = yb[uint64_t(a) * nk];
      re = fma(w.x, v.x, fma(-w.y, v.y, re));
      im = fma(w.x, v.y, fma(w.y, v.x, im));
    }
    C o;
    o.x = re;
    o.y = im;
    out[b * k + i] = o;
  }
}

void free_sas(Sas& S) {
  if (S.vplan) sdft_plan_destroy(S.vplan);
  if (S.d_meta) cudaFree(S.d_meta);
  if (S.d_winv) cudaFree(S.d_winv);
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
  if (flags & ~SDFT_PLAN_HOST_ONLY) return SDFT_ERR_ARG;
  sdft_sas_s* h = new (std::nothrow) sdft_sas_s();
  if (!h) return SDFT_ERR_NOMEM;
  Sas& S = h->s;
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
  sdft_status s = sdft_execute_strided(S.vplan, batch * S.mu_star, d_samples, d_work, stream);
  if (s != SDFT_OK) return s;
  const dim3 block(256);
  const dim3 grid(unsigned((S.k + 255) / 256), unsigned(std::min<uint64_t>(batch, 65535)));
  if (S.prec == SDFT_C64)
    k_sas_decode<float><<<grid, block, 0, st>>>(static_cast<const float2*>(d_work), static_cast<float2*>(d_coeffs),
                                                S.d_meta, static_cast<const float2*>(S.d_winv), S.k, nk, S.mu_star,
                                                batch);
  else
    k_sas_decode<double><<<grid, block, 0, st>>>(static_cast<const double2*>(d_work),
                                                 static_cast<double2*>(d_coeffs), S.d_meta,
                                                 static_cast<const double2*>(S.d_winv), S.k, nk, S.mu_star, batch);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SDFT_OK : cuda_fail(e);
}

sdft_status sdft_sas_destroy(sdft_sas sas) {
  if (!sas) return SDFT_ERR_ARG;
  sdft::free_sas(sas->s);
  delete sas;
  return SDFT_OK;
}

}  // extern "C"
