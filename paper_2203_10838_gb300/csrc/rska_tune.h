// rska_tune.h -- the schedule autotuner of the multi-right-hand-side form:
// the candidate space, its encoding, and the cache of measured choices.
#pragma once

#include <cstdint>
#include <string>

namespace rska {

// A candidate schedule as one int32: bits 0-1 the form (1 staged kernels, 2
// persistent kernel); staged: bits 8-15 the split of the first product over n
// (0 = one wave), bit 16 programmatic dependent launches; persistent: bits
// 17-19 the gather schedule (0 with the residual product, 1 right after the
// grid barrier, 2 + k after chunk k of the scaled residual is formed).
constexpr int32_t kFormStaged = 1;
constexpr int32_t kFormPersistent = 2;

inline int32_t tune_code(int form, int ksplit, int pdl, int gsched) {
  return (int32_t)(form | (ksplit << 8) | (pdl << 16) | (gsched << 17));
}
inline int tune_form(int32_t c) { return c & 3; }
inline int tune_ksplit(int32_t c) { return (c >> 8) & 0xff; }
inline int tune_pdl(int32_t c) { return (c >> 16) & 1; }
inline int tune_gsched(int32_t c) { return (c >> 17) & 7; }

// Candidates for a problem with n_p (multiple of 256), R_p (multiple of
// 256), eta_p64 (eta rounded up to 64) on num_sms SMs; persistent_ok says
// whether the persistent form fits.  Writes at most max codes, returns the
// number of candidates.
int tune_candidates(int64_t n_p, int64_t R_p, int64_t eta_p64, int num_sms, bool persistent_ok,
                    int32_t* out, int max);

// Process-wide cache of measured choices, keyed by problem shape, options and
// device.  With the environment variable RSKA_TUNE_CACHE naming a file, the
// file is read at the first lookup and every new entry is appended to it.
bool tune_cache_get(const std::string& key, int32_t* code, double* us);
void tune_cache_put(const std::string& key, int32_t code, double us);
int tune_cache_save(const char* path);
int tune_cache_load(const char* path);
void tune_cache_clear();

}  // namespace rska
