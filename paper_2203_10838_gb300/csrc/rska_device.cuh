// rska_device.cuh -- device helpers shared by the librska kernels: the
// Philox4x32-10 counter-based generator, the alias-table draw of the index
// contract, the soft-shrinkage operator S_lambda, and a bounded grid barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rska {

// Device status word values (mirrors the RSKA_E* codes of rska.h).
constexpr int kStatusOk = 0;
constexpr int kStatusZeroRow = 2;
constexpr int kStatusNonFinite = 3;
constexpr int kStatusTimeout = 6;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32
// -> 64 bit multiplications by fixed odd constants, xor of the high halves
// with the remaining counter words and the round key, with a Weyl increment of
// the key between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    U4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// One draw of the index contract: bucket c = (u_bucket * m) >> 32, kept if
// u_accept < thr[c], else alias[c].  Row p_i = nu_i / sum nu (Sec. 5, v1/v2).
__device__ __forceinline__ int32_t alias_draw(uint32_t u_bucket, uint32_t u_accept,
                                              const uint32_t* __restrict__ thr,
                                              const int32_t* __restrict__ alias, uint32_t m) {
  const uint32_t c = (uint32_t)(((uint64_t)u_bucket * (uint64_t)m) >> 32);
  const uint32_t t = __ldg(thr + c);
  return (u_accept < t) ? (int32_t)c : __ldg(alias + c);
}

// Slots 2q and 2q+1 of iteration k (Algorithm 1, "tau_k <- eta indices").
__device__ __forceinline__ void draw_pair(uint64_t seed, int64_t k, uint32_t q, uint32_t problem,
                                          const uint32_t* __restrict__ thr,
                                          const int32_t* __restrict__ alias, uint32_t m,
                                          int32_t* i_even, int32_t* i_odd) {
  U4 c;
  c.x = (uint32_t)(uint64_t)k;
  c.y = (uint32_t)((uint64_t)k >> 32);
  c.z = q;
  c.w = problem;
  const U4 u = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  *i_even = alias_draw(u.x, u.y, thr, alias, m);
  *i_odd = alias_draw(u.z, u.w, thr, alias, m);
}

// Soft shrinkage S_lambda(v) = max(|v| - lambda, 0) sign(v) (Sec. 1.1).
__device__ __forceinline__ float soft_shrink(float v, float lam) {
  const float mag = fabsf(v) - lam;
  return mag > 0.0f ? copysignf(mag, v) : 0.0f;
}

__device__ __forceinline__ float4 soft_shrink4(float4 v, float lam) {
  return make_float4(soft_shrink(v.x, lam), soft_shrink(v.y, lam), soft_shrink(v.z, lam),
                     soft_shrink(v.w, lam));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Limit of a wait for work this CTA has already issued (a TMA copy into its
// shared memory, an MMA reading it): such work always completes, and the CTA
// must not end before it has, so these waits use at least one second even
// when the watchdog limit of the other waits is set much shorter.
constexpr uint64_t kDrainLimitNs = 1000000000ull;

__device__ __forceinline__ uint64_t drain_limit(uint64_t limit_ns) {
  return limit_ns > kDrainLimitNs ? limit_ns : kDrainLimitNs;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a co-resident (cooperative) grid.  `counter` counts
// arrivals monotonically; barrier number `gen` (1, 2, ...) completes when it
// reaches gen * gridDim.x.  Every wait is bounded: after `limit_ns` (or when
// another CTA has already reported an error) the status word is set and the
// function returns false; the caller must then leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned long long* counter, unsigned long long gen,
                                             int* status, uint64_t limit_ns, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(counter, 1ull);
    const unsigned long long target = gen * (unsigned long long)gridDim.x;
    const uint64_t t0 = global_timer_ns();
    uint32_t spins = 0;
    while (ld_acquire_u64(counter) < target) {
      if (limit_ns == 0 || global_timer_ns() - t0 > limit_ns) {
        atomicCAS(status, kStatusOk, kStatusTimeout);
        ok = 0;
        break;
      }
      if ((++spins & 7u) == 0 && ld_relaxed_s32(status) != kStatusOk) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

}  // namespace rska
