// Cache of the autotuners' choices, keyed by what decides them: for a plan, its
// precision, log2 k and the batch size's power-of-two bucket (the positions of
// the pivots do not change the dataflow, only the twiddle values); for an
// uneven batch, its precision and the buckets of its instance count and total
// size. sdft_plan_autotune / sdft_batch_autotune store what they chose;
// sdft_plan_apply_tuning / sdft_batch_apply_tuning apply a stored choice
// without timing; sdft_autotune_cache_save / _load keep the cache in a JSON
// file between processes:
//   {"plan/c64/s20/b6": {"strategy": 1, "schedule": 0, "grid": 0, "stages_per_pass": 4,
//                        "table_staging": 0, "lag": 6, "ms": 0.35}, ...}
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "launch.hpp"

namespace sdft {

namespace {
std::mutex g_tuning_mu;
std::map<std::string, Tuning>& tunings() {
  static std::map<std::string, Tuning> m;
  return m;
}
uint32_t log2_floor(uint64_t x) {
  uint32_t r = 0;
  while (x >>= 1) ++r;
  return r;
}
const char* prec_name(sdft_prec p) { return p == SDFT_C64 ? "c64" : "c128"; }

// A minimal reader for the file format above: an object of objects whose
// values are numbers. Returns false on anything else.
struct Reader {
  const char* p;
  void ws() {
    while (*p && std::isspace(static_cast<unsigned char>(*p))) ++p;
  }
  bool lit(char c) {
    ws();
    if (*p != c) return false;
    ++p;
    return true;
  }
  bool str(std::string& out) {
    ws();
    if (*p != '"') return false;
    ++p;
    out.clear();
    while (*p && *p != '"') {
      if (*p == '\\') return false;       // keys of this cache never need escapes
      out.push_back(*p++);
    }
    if (*p != '"') return false;
    ++p;
    return true;
  }
  bool num(double& v) {
    ws();
    char* end = nullptr;
    v = std::strtod(p, &end);
    if (end == p) return false;
    p = end;
    return true;
  }
};
}  // namespace

std::string plan_tuning_key(sdft_prec prec, uint32_t s, uint64_t batch) {
  return std::string("plan/") + prec_name(prec) + "/s" + std::to_string(s) + "/b" +
         std::to_string(log2_floor(batch ? batch : 1));
}
std::string batch_tuning_key(sdft_prec prec, uint64_t n, uint64_t total) {
  return std::string("batch/") + prec_name(prec) + "/n" + std::to_string(log2_floor(n ? n : 1)) + "/t" +
         std::to_string(log2_floor(total ? total : 1));
}

void tuning_store(const std::string& key, const Tuning& t) {
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  tunings()[key] = t;
}
bool tuning_lookup(const std::string& key, Tuning* out) {
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  auto it = tunings().find(key);
  if (it == tunings().end()) return false;
  *out = it->second;
  return true;
}

}  // namespace sdft

extern "C" {

sdft_status sdft_autotune_cache_save(const char* path) {
  if (!path) return SDFT_ERR_ARG;
  std::string out = "{\n";
  {
    std::lock_guard<std::mutex> lk(sdft::g_tuning_mu);
    bool first = true;
    for (const auto& kv : sdft::tunings()) {
      const sdft::Tuning& t = kv.second;
      char buf[256];
      std::snprintf(buf, sizeof(buf),
                    "%s \"%s\": {\"strategy\": %d, \"schedule\": %d, \"grid\": %d, \"stages_per_pass\": %d, "
                    "\"table_staging\": %d, \"lag\": %d, \"ms\": %.6g}",
                    first ? "" : ",\n", kv.first.c_str(), t.strategy, t.schedule, t.grid, t.spp, t.staged, t.lag,
                    double(t.ms));
      out += buf;
      first = false;
    }
  }
  out += "\n}\n";
  FILE* f = std::fopen(path, "wb");
  if (!f) return SDFT_ERR_ARG;
  const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
  return (std::fclose(f) == 0 && ok) ? SDFT_OK : SDFT_ERR_ARG;
}

sdft_status sdft_autotune_cache_load(const char* path) {
  if (!path) return SDFT_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return SDFT_ERR_ARG;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  std::fclose(f);
  std::map<std::string, sdft::Tuning> got;
  sdft::Reader r{text.c_str()};
  if (!r.lit('{')) return SDFT_ERR_ARG;
  if (!r.lit('}')) {
    do {
      std::string key;
      if (!r.str(key) || !r.lit(':') || !r.lit('{')) return SDFT_ERR_ARG;
      sdft::Tuning t;
      if (!r.lit('}')) {
        do {
          std::string field;
          double v = 0.0;
          if (!r.str(field) || !r.lit(':') || !r.num(v)) return SDFT_ERR_ARG;
          if (field == "strategy") t.strategy = int(v);
          else if (field == "schedule") t.schedule = int(v);
          else if (field == "grid") t.grid = int(v);
          else if (field == "stages_per_pass") t.spp = int(v);
          else if (field == "table_staging") t.staged = int(v);
          else if (field == "lag") t.lag = int(v);
          else if (field == "ms") t.ms = float(v);
          else return SDFT_ERR_ARG;
        } while (r.lit(','));
        if (!r.lit('}')) return SDFT_ERR_ARG;
      }
      got[key] = t;
    } while (r.lit(','));
    if (!r.lit('}')) return SDFT_ERR_ARG;
  }
  r.ws();
  if (*r.p) return SDFT_ERR_ARG;
  std::lock_guard<std::mutex> lk(sdft::g_tuning_mu);
  for (auto& kv : got) sdft::tunings()[kv.first] = kv.second;
  return SDFT_OK;
}

sdft_status sdft_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(sdft::g_tuning_mu);
  sdft::tunings().clear();
  return SDFT_OK;
}

sdft_status sdft_autotune_cache_size(uint64_t* entries) {
  if (!entries) return SDFT_ERR_ARG;
  std::lock_guard<std::mutex> lk(sdft::g_tuning_mu);
  *entries = sdft::tunings().size();
  return SDFT_OK;
}

}  // extern "C"
