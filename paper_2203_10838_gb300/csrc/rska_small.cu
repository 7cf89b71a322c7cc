// rska_small.cu -- one-CTA RSKA kernel for small systems (eq. rska,
// Algorithm 1 with w_i = t): n <= 1024, eta <= 256, and one iteration's rows
// fit in shared memory.
//
// On such a system an iteration reads a few tens of KB (1000 x 500 with
// eta = 10: 20 KB, resident in L2), so its time is the latency of the
// iteration's dependent steps.  The row-split kernel run on one CTA splits
// every row over all of its threads and pays a block-wide reduction for each
// pair of rows.  Here a row belongs to one warp:
//
//  - The producer warp copies all eta rows of iteration j (one bulk copy per
//    row; tau_j, b and 1/||a||^2 at tau_j from the pre-sampled arrays, read
//    two iterations ahead) into slot j mod D of a ring of D
//    iteration slots as soon as the consumers have released that slot, so
//    up to D iterations are in flight (D = 1 when only one fits: the rows
//    of the next iteration are then fetched after this one is done).
//  - Consumer warp w takes rows s = w, w + 15, ... of the iteration.  Its
//    lanes hold x = S_lambda(z) in registers (float4 columns lane + 32 i),
//    form <a_s, x> by shuffles and publish
//    c_s = (t/eta)(<a_s, x> - b_s)/||a_s||^2.
//  - After a barrier over the consumers, consumer thread u owns float4 column
//    u of z (registers): it subtracts sum_s c_s a_s (the rows read from the
//    slot, summed in draw order), applies x = S_lambda(z) and publishes x.
//    After a second barrier every warp reloads its copy of x, and the slot
//    goes back to the producer.
//
// Two barriers per iteration and none per row; no exchange through global
// memory and no grid barrier.  Given xhat, the launch runs the stopping test
// of rska_solve_until itself (relative error of x to xhat, FP64) every
// check_every iterations and after its last one, and ends at the first test
// that passes, so a run to a tolerance takes a few launches.  Every wait is
// bounded.
#include <cstdint>
#include <cuda_runtime.h>

#include "rska_device.cuh"
#include "rska_internal.h"
#include "rska_tc.cuh"

namespace rska {

namespace {

constexpr int kSmT = 512;         // threads: 15 consumer warps and one producer warp
constexpr int kSmC = kSmT - 32;   // consumer threads
constexpr int kSmCW = kSmC / 32;  // consumer warps
constexpr int kSmQ = kSmallMaxEta / 32;  // rows of an iteration per producer lane

__device__ __forceinline__ void sm_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(b)) : "memory");
}

// Non-blocking probe of an mbarrier phase (try_wait may suspend the thread
// for a while before it answers).
__device__ __forceinline__ bool sm_test_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tc::saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: false after limit_ns, or once *abort is
// set (when given).  The first poll does not block, so a zero limit expires
// at a phase that is not complete when the wait begins.
__device__ __forceinline__ bool sm_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns,
                                        const volatile int* abort) {
  if (sm_test_wait(b, parity)) return true;
  if (limit_ns == 0) return false;
  const uint64_t t0 = global_timer_ns();
  while (!tc::mb_try_wait(b, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
    if (abort != nullptr && *abort) return false;
  }
  return true;
}

// Barrier among the consumer warps (named barrier 1), plain and OR-reducing.
__device__ __forceinline__ void csync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kSmC) : "memory");
}

__device__ __forceinline__ int csync_or(int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "n"(kSmC)
      : "memory");
  return r;
}

// S_lambda(v) = v - clamp(v, -lambda, lambda)
__device__ __forceinline__ float4 sm_shrink(float4 v, float lam) {
  return make_float4(v.x - fminf(fmaxf(v.x, -lam), lam), v.y - fminf(fmaxf(v.y, -lam), lam),
                     v.z - fminf(fmaxf(v.z, -lam), lam), v.w - fminf(fmaxf(v.w, -lam), lam));
}

// the components of float4 column c at or past n set to zero
__device__ __forceinline__ float4 sm_tail(float4 v, int c, int64_t n) {
  const int64_t base = 4 * (int64_t)c;
  if (base + 0 >= n) v.x = 0.f;
  if (base + 1 >= n) v.y = 0.f;
  if (base + 2 >= n) v.z = 0.f;
  if (base + 3 >= n) v.w = 0.f;
  return v;
}

__device__ __forceinline__ void sm_fma4(float4& acc, float4 a, float4 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.y = fmaf(a.y, b.y, acc.y);
  acc.z = fmaf(a.z, b.z, acc.z);
  acc.w = fmaf(a.w, b.w, acc.w);
}

// Dynamic shared memory: the ring (slots x eta rows of n4 float4), x (n4
// float4), b and 1/||a||^2 of every ring row (slots x eta floats each) and
// the coefficients of the current iteration (eta floats).
template <int NZ>
__global__ void __launch_bounds__(kSmT, 1) rska_small_kernel(SolveArgs a, int slots) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kSmallMaxSlots];
  __shared__ __align__(8) uint64_t empty[kSmallMaxSlots];
  __shared__ volatile int s_abort;      // consumers -> producer: stop issuing
  __shared__ volatile int s_pdone;      // producer -> consumers: no more copies
  __shared__ volatile long long s_prod; // iterations whose copies were issued
  __shared__ double s_red[2 * kSmCW];   // per-warp sums of the stopping test (owner warps)

  if (a.stop != nullptr && ld_relaxed_s32(a.stop) != 0) return;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int eta = a.eta;
  const int n4 = (int)((a.n + 3) >> 2);
  const uint32_t rowbytes = (uint32_t)n4 * 16u;
  float4* ring = reinterpret_cast<float4*>(smem);
  float4* xs = ring + (size_t)slots * eta * n4;
  float* mb = reinterpret_cast<float*>(xs + n4);
  float* miv = mb + (size_t)slots * eta;
  float* cs = miv + (size_t)slots * eta;

  if (tid == 0) {
    for (int i = 0; i < slots; ++i) {
      tc::mb_init(&full[i], 1);
      tc::mb_init(&empty[i], 1);
    }
    s_abort = 0;
    s_pdone = 0;
    s_prod = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  // ------------------------------------------------------------ producer --
  if (warp == kSmCW) {
    // lane l holds the row index, b and 1/||a||^2 of rows l + 32 q of two
    // iterations (register sets 0 and 1), fetched two iterations ahead of
    // their issue so the loads' latency is not on the producer's path
    int32_t pr[2][kSmQ];
    float pb[2][kSmQ], piv[2][kSmQ];
    auto fetch = [&](int64_t j, int32_t (&r)[kSmQ], float (&bb)[kSmQ], float (&iv)[kSmQ]) {
#pragma unroll
      for (int q = 0; q < kSmQ; ++q) {
        const int s = lane + 32 * q;
        r[q] = 0;
        bb[q] = 0.f;
        iv[q] = 0.f;
        if (s < eta && j < a.K) {
          const int64_t o = j * a.tstride + s;
          r[q] = a.tidx[o];
          bb[q] = a.tb[o];
          iv[q] = a.tiv[o];
        }
      }
    };
    // issue iteration j's rows from one register set; false: stop
    auto issue = [&](int64_t j, const int32_t (&r)[kSmQ], const float (&bb)[kSmQ],
                     const float (&iv)[kSmQ]) -> bool {
      const int sl = (int)(j % slots);
      const int64_t use = j / slots;
      int bad = 0;
      if (lane == 0) {
        if (use > 0 && !sm_wait(&empty[sl], (uint32_t)((use - 1) & 1), a.limit_ns, &s_abort))
          bad = 1;
        if (s_abort) bad = 1;
      }
      if (__shfl_sync(0xffffffffu, bad, 0)) return false;
#pragma unroll
      for (int q = 0; q < kSmQ; ++q) {
        const int s = lane + 32 * q;
        if (s < eta) {
          mb[(size_t)sl * eta + s] = bb[q];
          miv[(size_t)sl * eta + s] = iv[q];
        }
      }
      // the metadata stores come before the arrival that carries the byte
      // count, and the count before any copy that could complete it
      __syncwarp();
      if (lane == 0) tc::mb_expect_tx(&full[sl], (uint32_t)eta * rowbytes);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kSmQ; ++q) {
        const int s = lane + 32 * q;
        if (s < eta)
          tc::bulk_load(ring + ((size_t)sl * eta + s) * n4, a.A + (int64_t)r[q] * a.lda,
                        rowbytes, &full[sl]);
      }
      if (lane == 0) s_prod = j + 1;
      return true;
    };
    fetch(0, pr[0], pb[0], piv[0]);
    fetch(1, pr[1], pb[1], piv[1]);
    for (int64_t j = 0; j < a.K; j += 2) {
      if (!issue(j, pr[0], pb[0], piv[0])) break;
      fetch(j + 2, pr[0], pb[0], piv[0]);
      if (j + 1 >= a.K) break;
      if (!issue(j + 1, pr[1], pb[1], piv[1])) break;
      fetch(j + 3, pr[1], pb[1], piv[1]);
    }
    __syncwarp();
    if (lane == 0) s_pdone = 1;
    return;
  }

  // ------------------------------------------------------------ consumers --
  const int64_t k0 = *a.kdev;
  const float lam = a.lambda;
  const float coef = a.coef;
  // NZ = ceil(n4 / 32): a lane's columns lane + 32 i with i < NZ - 1 are
  // inside the row; only the last may lie past it (last_ok false) or be the
  // partly valid float4 when 4 does not divide n (last_tail)
  const int lastc = lane + 32 * (NZ - 1);
  const bool last_ok = lastc < n4;
  const bool last_tail = (a.n & 3) != 0 && lastc == n4 - 1;
  const bool owner = tid < n4;  // this thread's float4 column of z: tid
  const bool own_tail = (a.n & 3) != 0 && tid == n4 - 1;
  const float4* zin = reinterpret_cast<const float4*>(a.z);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

  float4 xr[NZ];
#pragma unroll
  for (int i = 0; i < NZ; ++i) {
    const int c = lane + 32 * i;
    xr[i] = (i < NZ - 1 || last_ok) ? sm_tail(sm_shrink(zin[c], lam), c, a.n) : zero4;
  }
  float4 zo = owner ? zin[tid] : zero4;

  // early end (a wait that ran out, or the stopping test passed): stop the
  // producer and let every copy it issued land before the CTA may end
  auto bail = [&](int64_t cons) {
    if (tid == 0) {
      s_abort = 1;
      const uint64_t dl = drain_limit(a.limit_ns);
      const uint64_t t0 = global_timer_ns();
      while (!s_pdone && global_timer_ns() - t0 < dl) {
      }
      const long long issued = s_prod;
      for (long long g = cons; g < issued; ++g)
        sm_wait(&full[g % slots], (uint32_t)((g / slots) & 1), dl, nullptr);
    }
    csync();
  };

  // The stopping test: ||x - xhat|| / ||xhat|| in FP64 for the current x.
  // The warps that own columns reduce their sums by shuffles; thread 0 adds
  // the warps' sums in a fixed order, records the error and decides, and an
  // OR-reducing barrier hands the decision to every consumer (FP64 is slow
  // on this GPU, so no thread repeats the others' work).  Returns 1 to stop.
  const int own_warps = (n4 + 31) / 32;
  auto stop_test = [&](int64_t done) -> int {
    if (warp < own_warps) {
      double ee = 0.0, hh = 0.0;
      if (owner) {
        const float4 xo = sm_shrink(zo, lam);
        const float xv[4] = {xo.x, xo.y, xo.z, xo.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int64_t e = 4 * (int64_t)tid + c;
          if (e < a.n) {
            const double h = (double)__ldg(a.xhat + e);
            const double d = (double)xv[c] - h;
            ee = fma(d, d, ee);
            hh = fma(h, h, hh);
          }
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        ee += __shfl_xor_sync(0xffffffffu, ee, o);
        hh += __shfl_xor_sync(0xffffffffu, hh, o);
      }
      if (lane == 0) {
        s_red[2 * warp] = ee;
        s_red[2 * warp + 1] = hh;
      }
    }
    csync();
    int stop_now = 0;
    if (tid == 0) {
      double se = 0.0, sh = 0.0;
      for (int w = 0; w < own_warps; ++w) {
        se += s_red[2 * w];
        sh += s_red[2 * w + 1];
      }
      const double err = sqrt(se) / (sh > 0.0 ? sqrt(sh) : 1e-30);
      a.macc[2] = se;
      a.macc[3] = sh;
      a.macc[5] = err;
      if (a.stop != nullptr && a.tol >= 0.0 && err <= a.tol) {
        *const_cast<int*>(a.stop) = 1;
        if (a.k_stop != nullptr) *a.k_stop = k0 + done;
        stop_now = 1;
      }
    }
    return csync_or(stop_now);
  };

  int64_t kend = a.K;  // iterations run by this launch
  for (int64_t j = 0; j < a.K; ++j) {
    const int sl = (int)(j % slots);
    const uint32_t par = (uint32_t)((j / slots) & 1);
    const float4* slot = ring + (size_t)sl * eta * n4;
    // every lane polls, so its own observation of the phase orders its reads
    int tmo = sm_wait(&full[sl], par, a.limit_ns, nullptr) ? 0 : 1;
    if (!tmo) {
      for (int s = warp; s < eta; s += kSmCW) {
        const float4* rowp = slot + (size_t)s * n4;
        float4 acc = zero4;
#pragma unroll
        for (int i = 0; i < NZ - 1; ++i) sm_fma4(acc, rowp[lane + 32 * i], xr[i]);
        if (last_ok) {
          float4 v = rowp[lastc];
          if (last_tail) v = sm_tail(v, lastc, a.n);
          sm_fma4(acc, v, xr[NZ - 1]);
        }
        float d = (acc.x + acc.y) + (acc.z + acc.w);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) {
          const size_t m = (size_t)sl * eta + s;
          cs[s] = coef * ((d - mb[m]) * miv[m]);
        }
      }
    }
    if (csync_or(tmo)) {
      if (tid == 0) atomicCAS(a.status, kStatusOk, kStatusTimeout);
      bail(j);
      return;
    }
    // z -= sum_s c_s a_s for this thread's column, in draw order
    if (owner) {
      float4 dz = zero4;
#pragma unroll 4
      for (int s = 0; s < eta; ++s) {
        float4 v = slot[(size_t)s * n4 + tid];
        if (own_tail) v = sm_tail(v, tid, a.n);
        const float c = cs[s];
        dz.x = fmaf(c, v.x, dz.x);
        dz.y = fmaf(c, v.y, dz.y);
        dz.z = fmaf(c, v.z, dz.z);
        dz.w = fmaf(c, v.w, dz.w);
      }
      zo = make_float4(zo.x - dz.x, zo.y - dz.y, zo.z - dz.z, zo.w - dz.w);
      xs[tid] = sm_shrink(zo, lam);
    }
    csync();
    if (tid == 0) sm_arrive(&empty[sl]);  // every consumer is done with the slot
#pragma unroll
    for (int i = 0; i < NZ - 1; ++i) xr[i] = xs[lane + 32 * i];
    xr[NZ - 1] = last_ok ? xs[lastc] : zero4;
    // given xhat: the test every check_every iterations and after the last
    const int64_t done = j + 1;
    if (a.xhat != nullptr &&
        ((a.check_every > 0 && done % a.check_every == 0) || done == a.K)) {
      if (stop_test(done)) {
        kend = done;
        break;
      }
    }
  }
  if (kend < a.K) bail(kend);  // stopped early: the producer stops, its copies land

  const float4 xo = sm_shrink(zo, lam);
  if (owner) {
    reinterpret_cast<float4*>(a.z)[tid] = zo;
    reinterpret_cast<float4*>(a.x)[tid] = xo;
  }
  if (tid == 0) *a.kdev = k0 + kend;
}

template <int NZ>
cudaError_t launch_small_t(const SolveArgs& a, const SmallGeometry& g, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(rska_small_kernel<NZ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  rska_small_kernel<NZ><<<1, kSmT, g.smem, s>>>(a, g.slots);
  return cudaGetLastError();
}

}  // namespace

bool plan_small(int64_t n, int32_t eta, size_t smem_optin, SmallGeometry* g) {
  const int64_t n4 = (n + 3) / 4;
  if (n < 1 || n4 > 32 * kSmallMaxNZ || eta < 1 || eta > kSmallMaxEta) return false;
  // static shared memory (mbarriers, flags) and a margin stay out of the budget
  const size_t cap = smem_optin < (size_t)(227 << 10) ? smem_optin : (size_t)(227 << 10);
  const size_t budget = cap > 1024 ? cap - 1024 : 0;
  const size_t per_slot = (size_t)eta * (size_t)n4 * 16 + 2 * (size_t)eta * sizeof(float);
  const size_t fixed = (size_t)n4 * 16 + (size_t)eta * sizeof(float);
  if (budget < fixed + per_slot) return false;
  size_t slots = (budget - fixed) / per_slot;
  if (slots > (size_t)kSmallMaxSlots) slots = kSmallMaxSlots;
  g->slots = (int)slots;
  g->nz = (int)((n4 + 31) / 32);
  g->smem = fixed + slots * per_slot;
  return true;
}

cudaError_t launch_small(const SolveArgs& a, const SmallGeometry& g, cudaStream_t s) {
  if (a.tstride == 0) return cudaErrorInvalidValue;  // pre-sampled indices only
  if (a.xhat != nullptr && a.macc == nullptr) return cudaErrorInvalidValue;
  cudaError_t e = launch_presample(a, s);
  if (e != cudaSuccess) return e;
  switch (g.nz) {
    case 1: return launch_small_t<1>(a, g, s);
    case 2: return launch_small_t<2>(a, g, s);
    case 3: return launch_small_t<3>(a, g, s);
    case 4: return launch_small_t<4>(a, g, s);
    case 5: return launch_small_t<5>(a, g, s);
    case 6: return launch_small_t<6>(a, g, s);
    case 7: return launch_small_t<7>(a, g, s);
    case 8: return launch_small_t<8>(a, g, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rska
