// rska_tune.cu -- host side of the multi-right-hand-side autotuner: the
// candidate schedules and the cache of measured choices (no device work here;
// rska_mrhs.cu times the candidates on the device).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "rska_internal.h"
#include "rska_mrhs_tmem.h"
#include "rska_tune.h"

namespace rska {

int tune_candidates(int64_t n_p, int64_t R_p, int64_t eta_p64, int num_sms, bool persistent_ok,
                    int32_t* out, int max) {
  int cnt = 0;
  auto add = [&](int32_t c) {
    if (cnt < max && out != nullptr) out[cnt] = c;
    ++cnt;
  };
  // staged: the first product's split over n (one wave, then fixed splits
  // that leave at least one 64-column block per CTA), with and without
  // programmatic dependent launches
  const int64_t kblocks = n_p / 64;
  const int splits[] = {0, 16, 32, 64};
  for (int ks : splits) {
    if (ks > 0 && ks > kblocks) continue;
    for (int pdl = 1; pdl >= 0; --pdl) add(tune_code(kFormStaged, ks, pdl, 0));
  }
  // persistent: the gather schedules (with the residual product, right
  // after the grid barrier, or after chunk k of the scaled residual, for
  // each of its eta_p64 / 64 chunks)
  if (persistent_ok && mrhs_tmem_fits(n_p, R_p, eta_p64, num_sms))
    for (int g = 0; g < 2 + eta_p64 / 64; ++g) add(tune_code(kFormPersistent, 0, 0, g));
  return cnt;
}

namespace {

struct Entry {
  int32_t code;
  double us;
};

std::mutex g_mu;
std::map<std::string, Entry> g_cache;
bool g_env_loaded = false;

// one line per entry: the key (no spaces), the code, microseconds per iteration
int load_locked(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return -1;
  char key[512];
  int code = 0;
  double us = 0.0;
  int n = 0;
  while (std::fscanf(f, "%511s %d %lf", key, &code, &us) == 3) {
    g_cache[key] = Entry{(int32_t)code, us};
    ++n;
  }
  std::fclose(f);
  return n;
}

void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* path = std::getenv("RSKA_TUNE_CACHE");
  if (path && *path) load_locked(path);
}

}  // namespace

bool tune_cache_get(const std::string& key, int32_t* code, double* us) {
  std::lock_guard<std::mutex> lock(g_mu);
  env_load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  if (code) *code = it->second.code;
  if (us) *us = it->second.us;
  return true;
}

void tune_cache_put(const std::string& key, int32_t code, double us) {
  std::lock_guard<std::mutex> lock(g_mu);
  env_load_locked();
  g_cache[key] = Entry{code, us};
  const char* path = std::getenv("RSKA_TUNE_CACHE");
  if (path && *path) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%s %d %.6f\n", key.c_str(), (int)code, us);
      std::fclose(f);
    }
  }
}

int tune_cache_save(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return -1;
  for (const auto& kv : g_cache) std::fprintf(f, "%s %d %.6f\n", kv.first.c_str(), (int)kv.second.code, kv.second.us);
  std::fclose(f);
  return (int)g_cache.size();
}

int tune_cache_load(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  return load_locked(path);
}

void tune_cache_clear() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
}

}  // namespace rska

extern "C" {

int rska_tune_candidates(int64_t n, int64_t R, int32_t eta, int32_t num_sms, int32_t* codes_out,
                         int32_t max, int32_t* count_out) {
  if (n < 1 || R < 1 || eta < 1 || eta > rska::kMaxEta || num_sms < 1 || max < 0 || !count_out ||
      (max > 0 && !codes_out))
    return RSKA_EINVAL;
  const int64_t n_p = (n + 255) / 256 * 256;
  const int64_t R_p = (R + 255) / 256 * 256;
  const int64_t eta_p64 = ((int64_t)eta + 63) / 64 * 64;
  *count_out = rska::tune_candidates(n_p, R_p, eta_p64, num_sms, true, codes_out, max);
  return RSKA_OK;
}

int rska_tune_cache(int32_t op, const char* key_or_path, int32_t* code, double* us) {
  switch (op) {
    case 0:
      if (!key_or_path) return RSKA_EINVAL;
      return rska::tune_cache_get(key_or_path, code, us) ? RSKA_OK : RSKA_EUNSUPPORTED;
    case 1: {
      if (!key_or_path || !code || !us || std::strchr(key_or_path, ' ') ||
          std::strlen(key_or_path) == 0 || std::strlen(key_or_path) > 500)
        return RSKA_EINVAL;
      rska::tune_cache_put(key_or_path, *code, *us);
      return RSKA_OK;
    }
    case 2:
      if (!key_or_path) return RSKA_EINVAL;
      return rska::tune_cache_save(key_or_path) >= 0 ? RSKA_OK : RSKA_EINVAL;
    case 3:
      if (!key_or_path) return RSKA_EINVAL;
      return rska::tune_cache_load(key_or_path) >= 0 ? RSKA_OK : RSKA_EINVAL;
    case 4:
      rska::tune_cache_clear();
      return RSKA_OK;
    default:
      return RSKA_EINVAL;
  }
}

}  // extern "C"
