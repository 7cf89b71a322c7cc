// rska_rows.cu -- row-split persistent RSKA kernel (eq. rska, Algorithm 1 with
// w_i = t) for n <= 4 * kSolveThreads * kRowsMaxZ.
//
// Work split.  Slot s of tau_k belongs to CTA s mod P, which reads the whole
// row a_{tau_k(s)} (n floats, one TMA bulk copy into a ring of shared-memory
// slots), forms <a_s, x_k> with a block reduction, the coefficient
// c_s = (t/eta)(<a_s, x_k> - b_s)/||a_s||^2, and adds c_s a_s into its partial
// update Delta_p (registers).  The only exchange per iteration is the sum of
// the P partial updates: each CTA adds Delta_p into a global accumulator with
// 16-byte vector reductions, passes one grid barrier, and reads the total
// back; every CTA keeps a full copy of z = x^* (tensor memory, which the
// kernel uses for nothing else, so all of shared memory is ring) and of
// x = S_lambda(z) (registers) and applies z -= Delta, x = S_lambda(z) itself.
// Rows are reduced two at a time; the grid is the fewest CTAs that keep the
// busiest CTA's number of such rounds.
//
// Warp roles.  Warps 0..14 consume rows (each thread owns float4 columns
// t + 480 r); warp 15 is the producer: it reads tau, b and 1/||a||^2 of the
// upcoming rows from the pre-sampled arrays and, for each row, waits for its
// ring slot to be released and issues the TMA copy at once.  A consumer warp
// releases a slot (empty mbarrier) the moment the row is in its registers, so
// the ring stays full, also while the consumers are in the exchange: HBM
// streams the next iteration's rows through the barrier.  Every device-side
// wait (full/empty mbarriers, grid barrier) is bounded.
#include <algorithm>

#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int NT = kSolveThreads;   // threads per CTA
constexpr int NC = NT - 32;          // consumer threads (warps 0..14)
constexpr int NCW = NC / 32;         // consumer warps
constexpr int G = 2;                 // rows reduced together
constexpr int SLOTS_MAX = 16;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void red_add_v4(float* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

// Arrival on the grid barrier: a release at GPU scope.  Issued by one thread
// after a barrier over the consumer warps, it orders their reductions before
// the count (the barrier makes them visible to this thread, and a release is
// cumulative).
__device__ __forceinline__ void red_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Barrier among the consumer warps only (named barrier 1).
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
}

__device__ __forceinline__ int consumer_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "n"(NC)
      : "memory");
  return r;
}

// S_lambda(v) as v - clamp(v, -lambda, lambda): the same value as
// soft_shrink (up to the sign of a zero) in three instructions
__device__ __forceinline__ float4 shrink4_clamp(float4 v, float lam) {
  return make_float4(v.x - fminf(fmaxf(v.x, -lam), lam), v.y - fminf(fmaxf(v.y, -lam), lam),
                     v.z - fminf(fmaxf(v.z, -lam), lam), v.w - fminf(fmaxf(v.w, -lam), lam));
}

// acc += a * b componentwise (four independent FMA chains)
__device__ __forceinline__ void fma4(float4& acc, float4 a, float4 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.y = fmaf(a.y, b.y, acc.y);
  acc.z = fmaf(a.z, b.z, acc.z);
  acc.w = fmaf(a.w, b.w, acc.w);
}

__device__ __forceinline__ float4 mask_tail(float4 v, int64_t gc, int64_t n) {
  const int64_t base = gc * 4;
  float4 r = v;
  if (base + 0 >= n) r.x = 0.f;
  if (base + 1 >= n) r.y = 0.f;
  if (base + 2 >= n) r.z = 0.f;
  if (base + 3 >= n) r.w = 0.f;
  return r;
}

// z in tensor memory.  Each consumer thread keeps its ZREG float4 columns in
// its warp's lane quarter (warp % 4), in the column block warp / 4; the
// loads and stores are warp-wide (every lane of the warp executes them).
constexpr uint32_t kZCols = 128;  // allocated columns (16 ZREG <= 96 used)

__device__ __forceinline__ void tm_st4(uint32_t taddr, float4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
               "r"(__float_as_uint(v.w))
               : "memory");
}

__device__ __forceinline__ void tm_ld4(uint32_t taddr, uint32_t (&u)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
               : "r"(taddr));
}

// The loaded registers are tied to the wait, so no use moves above it.
template <int ZREG>
__device__ __forceinline__ void tm_load_z(uint32_t tz, float4 (&z)[ZREG]) {
  uint32_t u[ZREG][4];
#pragma unroll
  for (int r = 0; r < ZREG; ++r) tm_ld4(tz + 4u * r, u[r]);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int r = 0; r < ZREG; ++r) {
    asm volatile("" : "+r"(u[r][0]), "+r"(u[r][1]), "+r"(u[r][2]), "+r"(u[r][3]));
    z[r] = make_float4(__uint_as_float(u[r][0]), __uint_as_float(u[r][1]),
                       __uint_as_float(u[r][2]), __uint_as_float(u[r][3]));
  }
}

template <int ZREG>
__device__ __forceinline__ void tm_store_z(uint32_t tz, const float4 (&z)[ZREG]) {
#pragma unroll
  for (int r = 0; r < ZREG; ++r) tm_st4(tz + 4u * r, z[r]);
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tm_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Bounded wait on an mbarrier phase: false after limit_ns, or once *abort is
// set (when abort is given).  The timer is read after every poll, so even a
// limit of a microsecond is enforced.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity, uint64_t limit_ns,
                                                  const volatile int* abort) {
  if (mbar_try_wait(b, parity)) return true;
  if (limit_ns == 0) return false;  // a zero limit expires at the first failed poll
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(b, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
    if (abort != nullptr && *abort) return false;
  }
  return true;
}

template <int ZREG>
__global__ void __launch_bounds__(NT, 1)
    rska_rows_kernel(SolveArgs a, int slots, int rowbytes_pad) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[SLOTS_MAX];
  __shared__ __align__(8) uint64_t empty[SLOTS_MAX];
  __shared__ __align__(16) float wpart[2][G][16];  // warp partials, entry 15 stays 0
  __shared__ float sb[SLOTS_MAX];
  __shared__ float siv[SLOTS_MAX];
  __shared__ int s_flag;
  __shared__ volatile int s_abort;        // consumers -> producer: stop issuing
  __shared__ volatile int s_pdone;        // producer -> consumers: no more copies
  __shared__ volatile long long s_prod;   // rows issued so far
  __shared__ uint32_t s_tmem;

  if (a.stop != nullptr && ld_relaxed_s32(a.stop) != 0) return;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int P = gridDim.x;
  const int p = blockIdx.x;
  const int eta = a.eta;
  const int64_t n4 = (a.n + 3) >> 2;
  const bool single = (P == 1);
  const int rpi = (p < eta) ? (eta - p + P - 1) / P : 0;  // rows of tau_k owned per iteration
  const uint32_t rowbytes = (uint32_t)(n4 * 16);
  const int64_t total_rows = (int64_t)rpi * a.K;

  unsigned char* ring = smem;  // slots x rowbytes_pad

  if (tid < 2 * G * 16) (&wpart[0][0][0])[tid] = 0.f;
  if (tid == 0) {
    for (int i = 0; i < slots; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCW);
    }
    s_abort = 0;
    s_pdone = 0;
    s_prod = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&s_tmem)),
                 "r"(kZCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();

  // ------------------------------------------------------------ producer --
  if (warp == NCW) {
    bool stop_now = false;
    int32_t row = 0;
    float bv = 0.f, ivv = 0.f;
    auto fetch_meta = [&](int64_t g0) {  // lane l: metadata of row g0 + l
      const int64_t gl = g0 + lane;
      row = 0;
      bv = 0.f;
      ivv = 0.f;
      if (gl < total_rows) {
        const int64_t jj = gl / rpi;
        const int q = (int)(gl - jj * rpi);
        const int64_t o = jj * a.tstride + p + (int64_t)P * q;
        row = a.tidx[o];
        bv = a.tb[o];
        ivv = a.tiv[o];
      }
    };
    fetch_meta(0);
    int pslot = 0;      // slot of the next row to issue (kept incrementally:
    int64_t puse = 0;   // no 64-bit division per row) and its use count
    for (int64_t g0 = 0; g0 < total_rows && !stop_now; g0 += 32) {
      const int32_t crow = row;
      const float cb = bv, civ = ivv;
      if (g0 + 32 < total_rows) fetch_meta(g0 + 32);  // next batch in flight meanwhile
      const int cnt = (int)((total_rows - g0 < 32) ? (total_rows - g0) : 32);
      for (int i = 0; i < cnt; ++i) {
        const int32_t r_i = __shfl_sync(0xffffffffu, crow, i);
        const float b_i = __shfl_sync(0xffffffffu, cb, i);
        const float iv_i = __shfl_sync(0xffffffffu, civ, i);
        int bad = 0;
        if (lane == 0) {
          const int64_t gi = g0 + i;
          const int sl = pslot;
          const int64_t use = puse;
          if (use > 0 && !mbar_wait_bounded(&empty[sl], (uint32_t)((use - 1) & 1), a.limit_ns,
                                            &s_abort))
            bad = 1;
          if (!bad && s_abort) bad = 1;
          if (!bad) {
            sb[sl] = b_i;
            siv[sl] = iv_i;
            mbar_expect_tx(&full[sl], rowbytes);
            tma_load_1d(ring + (size_t)sl * rowbytes_pad, a.A + (int64_t)r_i * a.lda, rowbytes,
                        &full[sl]);
            s_prod = gi + 1;
            if (++pslot == slots) {
              pslot = 0;
              ++puse;
            }
          }
        }
        if (__shfl_sync(0xffffffffu, bad, 0)) {
          stop_now = true;
          break;
        }
      }
    }
    __syncwarp();
    if (lane == 0) s_pdone = 1;
    return;
  }

  // ------------------------------------------------------------ consumers --
  const int64_t k0 = *a.kdev;
  const float lam = a.lambda;
  const float coef = a.coef;

  // column ownership: float4 columns t + NC*r; this thread's z in tensor
  // memory at lane 32 (warp % 4) + lane, columns 4 ZREG (warp / 4) + 4 r
  const uint32_t tz = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 4u * ZREG * (uint32_t)(warp >> 2);
  float4 xr[ZREG];
  float4 dl[ZREG];
  {
    float4 zi[ZREG];
#pragma unroll
    for (int r = 0; r < ZREG; ++r) {
      const int64_t col = tid + (int64_t)NC * r;
      float4 zv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (col < n4) zv = reinterpret_cast<const float4*>(a.z)[col];
      zi[r] = zv;
      xr[r] = (col < n4) ? mask_tail(soft_shrink4(zv, lam), col, a.n)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
      dl[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    tm_store_z<ZREG>(tz, zi);
  }
  // tensor memory is freed by warp 0 once every consumer is done with it
  auto free_z = [&]() {
    tm_fence_before();
    consumer_sync();
    if (warp == 0) {
      tm_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                   "r"(kZCols)
                   : "memory");
    }
  };

  int64_t cons = 0;  // rows consumed
  int cslot = 0;     // slot of row `cons` and the parity of its current use,
  uint32_t cpar = 0; // kept incrementally (no 64-bit division per row)
  int gcount = 0;    // groups consumed (selects the wpart buffer)
  // error exit: stop the producer, let every issued copy land, leave
  auto bail = [&]() {
    if (tid == 0) {
      s_abort = 1;
      const uint64_t t0 = global_timer_ns();
      // the producer stops within one of its own bounded waits; every copy
      // it issued lands before the CTA may end (drain limit, not the watchdog)
      const uint64_t dl = drain_limit(a.limit_ns);
      while (!s_pdone && global_timer_ns() - t0 < dl) {
      }
      const int64_t issued = s_prod;
      for (int64_t g = cons; g < issued; ++g) {
        const int sl = (int)(g % slots);
        mbar_wait_bounded(&full[sl], (uint32_t)((g / slots) & 1), dl, nullptr);
      }
    }
    consumer_sync();
    free_z();
  };

  // ZREG = ceil(n4 / NC), so this thread's columns t + NC r with r < ZREG - 1
  // are always inside the row; only the last one, t + NC (ZREG - 1), may lie
  // past it (last_ok false) or be the partly valid float4 when 4 does not
  // divide n (last_tail)
  const int64_t last_col = tid + (int64_t)NC * (ZREG - 1);
  const bool last_ok = last_col < n4;
  const bool last_tail = (a.n & 3) != 0 && last_col == n4 - 1;
  float4 av[G][ZREG];
  float bg[G], ivg[G];
  bool have_pre = false;
  // wait for rows cons .. cons+ng-1, copy this thread's columns to registers,
  // release their slots; returns 1 on a timeout
  auto load_group = [&](int ng) -> int {
    int tmo = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      bg[g] = 0.f;
      ivg[g] = 0.f;
      if (g < ng) {
        int sl = cslot + g;
        uint32_t par = cpar;
        if (sl >= slots) {  // g < G <= 2 slots
          sl -= slots;
          par ^= 1u;
        }
        // every lane polls (one warp-wide instruction), so each lane's own
        // observation of the completed phase orders its reads of the row
        if (!mbar_wait_bounded(&full[sl], par, a.limit_ns, nullptr)) tmo = 1;
        const float4* rowp = reinterpret_cast<const float4*>(ring + (size_t)sl * rowbytes_pad);
#pragma unroll
        for (int r = 0; r < ZREG - 1; ++r) av[g][r] = rowp[tid + NC * r];
        {
          float4 v = last_ok ? rowp[last_col] : make_float4(0.f, 0.f, 0.f, 0.f);
          if (last_tail) v = mask_tail(v, last_col, a.n);
          av[g][ZREG - 1] = v;
        }
        bg[g] = sb[sl];
        ivg[g] = siv[sl];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sl]);  // the row is in registers: free the slot
      } else {
#pragma unroll
        for (int r = 0; r < ZREG; ++r) av[g][r] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    return tmo;
  };

  for (int64_t j = 0; j < a.K; ++j) {
    // ---- this CTA's rows of tau_k: dots, coefficients, partial update ----
    for (int q0 = 0; q0 < rpi; q0 += G) {
      const int ng = min(G, rpi - q0);
      float pd[G];
      int tmo = 0;
      if (!(q0 == 0 && have_pre)) tmo = load_group(ng);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < ZREG; ++r) fma4(acc, av[g][r], xr[r]);
        pd[g] = (acc.x + acc.y) + (acc.z + acc.w);
      }
      // warp sums of the two rows in one butterfly: after the first exchange
      // lanes 0-15 hold row 0's partials and lanes 16-31 row 1's, then four
      // levels finish both; lanes 0 and 16 publish them
      static_assert(G == 2, "the warp reduction pairs two rows");
      float ws = (lane & 16) ? pd[1] : pd[0];
      ws += __shfl_xor_sync(0xffffffffu, (lane & 16) ? pd[0] : pd[1], 16);
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
      const int wp = gcount & 1;
      ++gcount;
      if ((lane & 15) == 0) wpart[wp][lane >> 4][warp] = ws;
      if (consumer_sync_or(tmo)) {
        if (tid == 0) atomicCAS(a.status, kStatusOk, kStatusTimeout);
        bail();
        return;
      }
      cons += ng;
      cslot += ng;
      while (cslot >= slots) {
        cslot -= slots;
        cpar ^= 1u;
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        // every thread sums the 15 warp partials (and a zero) from shared
        // memory in one fixed pairwise order: the same value in all threads
        const float4* wv = reinterpret_cast<const float4*>(&wpart[wp][g][0]);
        const float4 w0 = wv[0], w1 = wv[1], w2 = wv[2], w3 = wv[3];
        const float d = (((w0.x + w0.y) + (w0.z + w0.w)) + ((w1.x + w1.y) + (w1.z + w1.w))) +
                        (((w2.x + w2.y) + (w2.z + w2.w)) + ((w3.x + w3.y) + (w3.z + w3.w)));
        if (g < ng) {
          const float cval = coef * ((d - bg[g]) * ivg[g]);
#pragma unroll
          for (int r = 0; r < ZREG; ++r) {
            dl[r].x = fmaf(cval, av[g][r].x, dl[r].x);
            dl[r].y = fmaf(cval, av[g][r].y, dl[r].y);
            dl[r].z = fmaf(cval, av[g][r].z, dl[r].z);
            dl[r].w = fmaf(cval, av[g][r].w, dl[r].w);
          }
        }
      }
    }
    have_pre = false;

    // ---- exchange: Delta = sum_p Delta_p ----
    if (single) {
      float4 zc[ZREG];
      tm_load_z<ZREG>(tz, zc);
#pragma unroll
      for (int r = 0; r < ZREG; ++r) {
        const int64_t col = tid + (int64_t)NC * r;
        if (r < ZREG - 1 || last_ok) {
          float4 zv = zc[r];
          zv.x -= dl[r].x;
          zv.y -= dl[r].y;
          zv.z -= dl[r].z;
          zv.w -= dl[r].w;
          if (r == ZREG - 1 && last_tail) zv = mask_tail(zv, col, a.n);
          zc[r] = zv;
          xr[r] = shrink4_clamp(zv, lam);
        }
        dl[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      tm_store_z<ZREG>(tz, zc);
      continue;
    }
    const int buf = (int)(j % 3);
    float* dacc = a.racc + (size_t)buf * n4 * 4;
#pragma unroll
    for (int r = 0; r < ZREG; ++r) {
      const int64_t col = tid + (int64_t)NC * r;
      if (rpi > 0 && (r < ZREG - 1 || last_ok)) red_add_v4(dacc + col * 4, dl[r]);
      dl[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    {
      // every CTA clears its 1/P slice of the accumulator of iteration j + 1
      // (one CTA clearing all of it would arrive at the barrier last)
      float4* nxt = reinterpret_cast<float4*>(a.racc + (size_t)((j + 1) % 3) * n4 * 4);
      const int64_t chunk = (n4 + P - 1) / P;
      for (int64_t c = tid; c < chunk; c += NC) {
        const int64_t col = (int64_t)p * chunk + c;
        if (col < n4) nxt[col] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // grid barrier (bounded): arrive, pull the next iteration's first rows
    // into registers (freeing their slots for the producer), then wait
    consumer_sync();
    if (tid == 0) red_release_u64(a.bar, 1ull);
    int pre_tmo = 0;
    if (j + 1 < a.K && rpi > 0) {
      pre_tmo = load_group(min(G, rpi));
      have_pre = true;
    }
    if (tid == 0) {
      int ok = 1;
      const unsigned long long target = (unsigned long long)(j + 1) * (unsigned long long)P;
      const uint64_t t0 = global_timer_ns();
      uint32_t spins = 0;
      while (ld_acquire_u64(a.bar) < target) {
        // the clock and the status word every fourth poll (a zero limit
        // expires at the first failed poll)
        ++spins;
        if (a.limit_ns == 0 || ((spins & 3u) == 0 && global_timer_ns() - t0 > a.limit_ns)) {
          atomicCAS(a.status, kStatusOk, kStatusTimeout);
          ok = 0;
          break;
        }
        if ((spins & 7u) == 0 && ld_relaxed_s32(a.status) != kStatusOk) {
          ok = 0;
          break;
        }
      }
      // the acquire load that saw the count orders this CTA's reads of the
      // reduced update after every CTA's reductions (the consumer barrier
      // below passes that order on to the other threads)
      s_flag = ok;
    }
    if (consumer_sync_or(pre_tmo) || !s_flag) {
      if (tid == 0) atomicCAS(a.status, kStatusOk, kStatusTimeout);
      bail();
      return;
    }
    const float4* dtot = reinterpret_cast<const float4*>(dacc);
    float4 zc[ZREG];
    tm_load_z<ZREG>(tz, zc);
#pragma unroll
    for (int r = 0; r < ZREG; ++r) {
      const int64_t col = tid + (int64_t)NC * r;
      if (r < ZREG - 1 || last_ok) {
        const float4 d = __ldcg(dtot + col);
        float4 zv = zc[r];
        zv.x -= d.x;
        zv.y -= d.y;
        zv.z -= d.z;
        zv.w -= d.w;
        if (r == ZREG - 1 && last_tail) zv = mask_tail(zv, col, a.n);
        zc[r] = zv;
        xr[r] = shrink4_clamp(zv, lam);
      }
    }
    tm_store_z<ZREG>(tz, zc);
  }

  if (p == 0) {
    float4 zc[ZREG];
    tm_load_z<ZREG>(tz, zc);
    float4* zo = reinterpret_cast<float4*>(a.z);
    float4* xo = reinterpret_cast<float4*>(a.x);
#pragma unroll
    for (int r = 0; r < ZREG; ++r) {
      const int64_t col = tid + (int64_t)NC * r;
      if (col < n4) {
        zo[col] = zc[r];
        xo[col] = xr[r];
      }
    }
    if (tid == 0) *a.kdev = k0 + a.K;
  }
  free_z();
}

template <int ZREG>
cudaError_t launch_rows_t(const SolveArgs& a, const RowsGeometry& g, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(rska_rows_kernel<ZREG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  SolveArgs args = a;
  int slots = g.slots;
  int rbp = g.rowbytes_pad;
  void* params[] = {&args, &slots, &rbp};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (void*)rska_rows_kernel<ZREG>, params);
}

}  // namespace

bool plan_rows(int64_t n, int32_t eta, int num_sms, int grid_override, size_t smem_optin,
               RowsGeometry* g) {
  const int64_t n4 = (n + 3) / 4;
  const int64_t zreg = (n4 + NC - 1) / NC;
  if (zreg > kRowsMaxZ) return false;
  const int z = (int)std::max<int64_t>(1, zreg);
  // Small iterations (all of tau_k within ~128 KB) run on one CTA: no grid
  // barrier at all; otherwise one CTA per SM up to one row per CTA.
  const int64_t iter_bytes = (int64_t)eta * n4 * 16;
  int64_t P = grid_override > 0 ? grid_override
                                : (iter_bytes <= (128 << 10) ? 1 : std::min<int64_t>(num_sms, eta));
  P = std::max<int64_t>(1, std::min<int64_t>(P, num_sms));
  if (grid_override <= 0 && P > 1 && eta > P) {
    // rows are reduced G at a time, and the busiest CTA sets the number of
    // reduction rounds: the fewest CTAs that keep that number give every CTA
    // full groups, and the exchange sums fewer partial updates
    const int64_t rounds = ((eta + P - 1) / P + G - 1) / G;
    P = (eta + rounds * G - 1) / (rounds * G);
  }
  const int64_t rowbytes = n4 * 16;
  const int64_t rowbytes_pad = (rowbytes + 127) / 128 * 128;
  const size_t fixed = 2048;  // z lives in tensor memory
  if (fixed + 2 * rowbytes_pad > smem_optin) return false;
  int64_t slots = (int64_t)((smem_optin - fixed) / rowbytes_pad);
  slots = std::min<int64_t>(slots, SLOTS_MAX);
  if (slots < 2) return false;
  g->grid = (int)P;
  g->zreg = z;
  g->slots = (int)slots;
  g->rowbytes_pad = (int)rowbytes_pad;
  g->smem = (size_t)slots * rowbytes_pad;
  return true;
}

cudaError_t launch_rows(const SolveArgs& a, const RowsGeometry& g, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (a.tstride != 0) e = launch_presample(a, s);
  if (e != cudaSuccess) return e;
  const int64_t n4 = (a.n + 3) / 4;
  e = cudaMemsetAsync(a.racc, 0, sizeof(float) * 3 * (size_t)n4 * 4, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  switch (g.zreg) {
    case 1: return launch_rows_t<1>(a, g, s);
    case 2: return launch_rows_t<2>(a, g, s);
    case 3: return launch_rows_t<3>(a, g, s);
    case 4: return launch_rows_t<4>(a, g, s);
    case 5: return launch_rows_t<5>(a, g, s);
    default: return launch_rows_t<6>(a, g, s);
  }
}

}  // namespace rska
