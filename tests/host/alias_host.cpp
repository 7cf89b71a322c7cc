// Host build of the device alias construction (csrc/rska_alias.cuh) for a CPU
// test against the oracle: the CUDA qualifiers become empty, the FP64
// intrinsics plain IEEE operations (volatile, so nothing is contracted).
#include <cstdint>
#include <cstring>
#include <vector>
#define __device__
#define __forceinline__ inline
#define __host__
#define __shared__ static
struct dim3s { unsigned x; };
static dim3s blockDim{1}, threadIdx{0};
template <class T> T __shfl_up_sync(unsigned, T v, int) { return v; }
static void __syncthreads() {}
static inline double __dadd_rn(double a, double b) { volatile double r = a + b; return r; }
static inline double __dsub_rn(double a, double b) { volatile double r = a - b; return r; }
static inline double __dmul_rn(double a, double b) { volatile double r = a * b; return r; }
static inline double __ddiv_rn(double a, double b) { volatile double r = a / b; return r; }
static inline uint32_t __double2uint_rz(double a) { return (uint32_t)a; }
static inline long long __double_as_longlong(double a) { long long r; std::memcpy(&r, &a, 8); return r; }

#include "../../paper_2203_10838_gb300/csrc/rska_alias.cuh"

// the partition of vose_block (T threads, contiguous segments, stable
// compaction) mirrored on one thread, then the header's pairing loop and
// thresholds
static void block_like(double* q, int32_t* stk, int64_t m, uint32_t* thr, int32_t* alias, int T) {
  std::vector<int64_t> cs(T), before(T);
  for (int t = 0; t < T; ++t) {
    int64_t lo = m * t / T, hi = m * (t + 1) / T, c = 0;
    for (int64_t i = lo; i < hi; ++i) c += rska::vose_small(q[i]) ? 1 : 0;
    cs[t] = c;
  }
  int64_t run = 0;
  for (int t = 0; t < T; ++t) { before[t] = run; run += cs[t]; }
  const int64_t ns = run;
  for (int t = 0; t < T; ++t) {
    int64_t lo = m * t / T, hi = m * (t + 1) / T, b = before[t];
    for (int64_t i = lo; i < hi; ++i) {
      if (rska::vose_small(q[i])) stk[b++] = (int32_t)i; else stk[m - 1 - (i - b)] = (int32_t)i;
    }
  }
  rska::VoseRest r = rska::vose_pair<int32_t>(q, stk, m, ns, m - ns, alias);
  for (int64_t s = 0; s < r.sp; ++s) q[stk[s]] = -1.0;
  for (int64_t s = m - r.lp; s < m; ++s) q[stk[s]] = -1.0;
  if (r.hot >= 0) q[r.hot] = -1.0;
  for (int64_t i = 0; i < m; ++i) {
    if (q[i] < 0.0) { thr[i] = 4294967295u; alias[i] = (int32_t)i; } else thr[i] = rska::vose_threshold(q[i]);
  }
}

extern "C" void host_alias(const double* nu, int64_t m, uint32_t* thr, int32_t* alias, int mode) {
  std::vector<double> q(m);
  std::vector<int32_t> stk(m);
  double W = 0.0;
  for (int64_t i = 0; i < m; ++i) W = __dadd_rn(W, nu[i]);
  for (int64_t i = 0; i < m; ++i) q[i] = __ddiv_rn(__dmul_rn(nu[i], (double)m), W);
  if (mode == 0) rska::vose_sequential<int32_t>(q.data(), stk.data(), m, thr, alias);
  else block_like(q.data(), stk.data(), m, thr, alias, mode);
}
