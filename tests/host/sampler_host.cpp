// Host build of the device sampler (csrc/rska_device.cuh: Philox4x32-10 and
// the alias draw of the index contract) for a CPU test against the oracle.
// The CUDA qualifiers become empty and the integer intrinsics plain C++; the
// barrier helpers of the header are declared here only so that it parses
// (they are never called).
#include <cstdint>
#include <math.h>
#include <cstring>
#define __device__
#define __forceinline__ inline
#define __host__
#include <cuda_runtime.h>

static inline uint32_t __umulhi(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}
template <class T> static inline T __ldg(const T* p) { return *p; }
static inline void __threadfence() {}
static inline void __syncthreads() {}
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p;
  *p = o + v;
  return o;
}
static inline int atomicCAS(int* p, int cmp, int v) {
  const int o = *p;
  if (o == cmp) *p = v;
  return o;
}
static dim3 gridDim, threadIdx;

#include "../../paper_2203_10838_gb300/csrc/rska_device.cuh"

// indices of iterations k0 .. k0+K-1 (eta each, row-major) for one problem
extern "C" void host_sample(const uint32_t* thr, const int32_t* alias, uint32_t m, uint64_t seed,
                            uint32_t problem, int64_t k0, int64_t K, int32_t eta, int32_t* out) {
  const uint32_t npairs = (uint32_t)((eta + 1) / 2);
  for (int64_t kk = 0; kk < K; ++kk) {
    for (uint32_t q = 0; q < npairs; ++q) {
      int32_t i0, i1;
      rska::draw_pair(seed, k0 + kk, q, problem, thr, alias, m, &i0, &i1);
      out[kk * eta + 2 * q] = i0;
      if (2 * q + 1 < (uint32_t)eta) out[kk * eta + 2 * q + 1] = i1;
    }
  }
}

extern "C" void host_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  rska::U4 c{ctr[0], ctr[1], ctr[2], ctr[3]};
  const rska::U4 u = rska::philox4x32_10(c, key[0], key[1]);
  out[0] = u.x;
  out[1] = u.y;
  out[2] = u.z;
  out[3] = u.w;
}
