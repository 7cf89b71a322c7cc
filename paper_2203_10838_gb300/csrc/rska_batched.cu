// rska_batched.cu -- many independent RSKA systems in one persistent launch
// (eq. rska, Algorithm 1 with w_i = t, run on every (A_p, b_p) with its own
// index stream), each stopping by itself at a relative residual
// ||A_p x - b_p|| / ||b_p|| <= tol (Algorithm 1, "until a stopping criterion
// is satisfied").
//
// One CTA owns one problem at a time and takes problems from a queue sorted
// by estimated work (largest first).  Warp 7 only draws: it fills a ring of
// the next rows of tau (Philox4x32-10 + alias table, 32 draws per warp step,
// counter word 3 = problem id) with their b_i and 1/||a_i||^2, up to 512 rows
// ahead of the last completed iteration, and sleeps when it is ahead.  Warps
// 0..6 consume rows whole: warp w takes rows s = w, w + 7, ... of every tau_k,
// streams each with 16-byte cp.async copies into its own ring of shared-memory
// slots (each lane copies and later reads back only its own columns, so no
// barrier guards the ring), computes the dot by shuffles and accumulates
// c_s a_s into its share of the update in registers.  At the end of an
// iteration the shares are added into one shared vector and every consumer
// thread applies z -= update, x = S_lambda(z) to a slice of the columns: two
// block barriers per iteration, none per row.  (A TMA bulk copy per row and a
// column split of every row over all warps were the earlier designs; their
// per-row copy latency and per-row instruction and barrier overhead is what
// this layout removes.)
//
// Stopping: every C_p iterations the CTA first looks at an unbiased estimate
// of ||A_p x - b_p||^2 built for free from the sampled residuals
// (sum of r_s^2 / (eta p_s) over the window, p_s = ||a_s||^2 / W_p); only when
// it is within (4 tol)^2 ||b_p||^2 does it run the exact check (one pass over
// A_p; dot products by compensated FP32 Dot2, sums in FP64 -- FP64 arithmetic
// is slow on this GPU).  After an exact check that does not stop the problem,
// the next 1, 3, 7, 15 (at most) passing windows are skipped, so a problem
// hovering just above tol does not pay a pass over A_p every window.  Every device-side wait is
// bounded.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "rska_alias.cuh"
#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int BT = 256;          // threads per CTA
constexpr int BC = BT - 32;      // consumer threads (warps 0..6)
constexpr int BCW = BC / 32;     // consumer warps
constexpr int BIR = 512;         // index ring entries (rows drawn ahead; a power of 2)
constexpr int BMAXNZ = 21;       // float4 columns per lane: n <= 32 * 21 * 4 = 2688
constexpr int BRS_MAX = 16;      // ring slots per warp
constexpr size_t BVEC = (size_t)BMAXNZ * 32 * 16;       // bytes of z, x or the update
constexpr size_t BRING_OFF = 3 * BVEC;                  // rows start after z, x, update
constexpr size_t BRING_WARP = 24 * 1024;                // row slots of one consumer warp
constexpr int BHOLDNZ = 16;      // rows up to this many float4 per lane stay in registers
constexpr size_t BEXT_OFF = BRING_OFF + BCW * BRING_WARP;  // two more update-share buffers
constexpr size_t BSMEM = BEXT_OFF + 2 * (size_t)BHOLDNZ * 32 * 16;  // dynamic shared memory per CTA
constexpr int BMAX_ETA = 448;    // rows of one iteration stay inside the index ring
static_assert(BRING_WARP / BVEC >= 2, "every warp holds two of the widest rows");
static_assert(BMAX_ETA + 32 <= BIR, "an iteration's rows fit the index ring");

struct BatchArgs {
  int32_t P;
  const int32_t* order;      // problems, largest first
  const float* A;
  const int64_t* a_off;      // element offset of A_p
  const int32_t* m;
  const int32_t* n;
  const int64_t* lda;
  const float* b;
  const int64_t* b_off;
  const int64_t* row_off;    // offset of problem p's rows in the per-row tables
  const float* inv_nu;
  const uint32_t* thr;
  const int32_t* alias;
  const double* W;           // sum of ||a_i||^2 per problem
  const double* bnorm2;      // ||b_p||^2
  const int64_t* x_off;      // offset of problem p in z / x (n rounded up to 4)
  const uint32_t* sid;       // index-stream id of problem p (counter word 3; default p)
  float* z;
  float* x;
  int64_t* iters;
  double* relres;
  float lambda;
  float coef;                // t / eta
  int32_t eta;
  uint64_t seed;
  int64_t max_iters;
  double tol;                // 0: run max_iters on every problem
  int64_t check_every;       // 0: ceil(m_p / eta)
  int* queue;
  int* status;
  uint64_t limit_ns;
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(BC) : "memory");
}

// Pair barriers between consumer warps w and w + 3 (w = 1..3; named barriers
// 2..4, 64 threads): the writer (w) arrives, the reader (w + 3) waits.
__device__ __forceinline__ void pair_arrive(int warp) {
  if (warp == 1) asm volatile("bar.arrive 2, 64;" ::: "memory");
  else if (warp == 2) asm volatile("bar.arrive 3, 64;" ::: "memory");
  else asm volatile("bar.arrive 4, 64;" ::: "memory");
}
__device__ __forceinline__ void pair_wait(int warp) {
  if (warp == 4) asm volatile("bar.sync 2, 64;" ::: "memory");
  else if (warp == 5) asm volatile("bar.sync 3, 64;" ::: "memory");
  else asm volatile("bar.sync 4, 64;" ::: "memory");
}

__device__ __forceinline__ int consumer_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "n"(BC)
      : "memory");
  return r;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
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

// ---------------------------------------------------------------------------
// Setup: FP64 row norms in the canonical order (one CTA per problem, one warp
// per row), then one thread per problem builds its alias table and sums W_p
// and ||b_p||^2.
// ---------------------------------------------------------------------------
__global__ void batch_norms_kernel(BatchArgs a, double* nu, float* inv_nu, int* pstat) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const int m = a.m[p], n = a.n[p];
    const float* Ap = a.A + a.a_off[p];
    const float* bp = a.b + a.b_off[p];
    const int64_t lda = a.lda[p];
    const int64_t ro = a.row_off[p];
    for (int i = warp; i < m; i += nw) {
      const float* row = Ap + (int64_t)i * lda;
      double acc = 0.0;
      bool finite = true;
      for (int j = lane; j < n; j += 32) {
        const float v = __ldg(row + j);
        finite = finite && isfinite(v);
        const double vd = (double)v;
        acc = __fma_rn(vd, vd, acc);
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      finite = __all_sync(0xffffffffu, finite);
      if (lane == 0) {
        const float bi = __ldg(bp + i);
        if (!finite || !isfinite(bi) || !isfinite(acc))
          atomicCAS(pstat + p, kStatusOk, kStatusNonFinite);
        else if (acc == 0.0)
          atomicCAS(pstat + p, kStatusOk, kStatusZeroRow);
        nu[ro + i] = acc;
        inv_nu[ro + i] = (acc > 0.0) ? (float)__ddiv_rn(1.0, acc) : 0.0f;
      }
    }
  }
}

__global__ void batch_alias_kernel(BatchArgs a, const double* nu, double* q, int32_t* stk,
                                   uint32_t* thr, int32_t* alias, double* W, double* bnorm2,
                                   const int* pstat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int m = a.m[p];
  const int64_t ro = a.row_off[p];
  const float* bp = a.b + a.b_off[p];
  double bb = 0.0;
  for (int i = 0; i < m; ++i) {
    const double bi = (double)bp[i];
    bb = __fma_rn(bi, bi, bb);
  }
  bnorm2[p] = bb;
  if (pstat[p] != kStatusOk) {
    W[p] = 0.0;
    return;
  }
  double w = 0.0;
  for (int i = 0; i < m; ++i) w = __dadd_rn(w, nu[ro + i]);
  W[p] = w;
  const double md = (double)m;
  for (int i = 0; i < m; ++i) q[ro + i] = __ddiv_rn(__dmul_rn(nu[ro + i], md), w);
  vose_sequential<int32_t>(q + ro, stk + ro, m, thr + ro, alias + ro);
}

// ---------------------------------------------------------------------------
// The persistent batched solver.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Wait until at most `pending` of this thread's most recent copy groups are
// still in flight (the instruction takes an immediate).
__device__ __forceinline__ void cp_async_wait_pending(int pending) {
  switch (pending) {
#define RSKA_WG(N) \
  case N:          \
    asm volatile("cp.async.wait_group " #N ";" ::: "memory"); \
    break;
    RSKA_WG(0) RSKA_WG(1) RSKA_WG(2) RSKA_WG(3) RSKA_WG(4) RSKA_WG(5) RSKA_WG(6) RSKA_WG(7)
    RSKA_WG(8) RSKA_WG(9) RSKA_WG(10) RSKA_WG(11) RSKA_WG(12) RSKA_WG(13) RSKA_WG(14)
    RSKA_WG(15) RSKA_WG(16) RSKA_WG(17) RSKA_WG(18) RSKA_WG(19) RSKA_WG(20) RSKA_WG(21)
    RSKA_WG(22) RSKA_WG(23) RSKA_WG(24) RSKA_WG(25) RSKA_WG(26) RSKA_WG(27) RSKA_WG(28)
    RSKA_WG(29) RSKA_WG(30)
#undef RSKA_WG
    default:
      asm volatile("cp.async.wait_all;" ::: "memory");
      break;
  }
}

// One step of Dot2 (Ogita, Rump and Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 26(6), 2005): the product a*b split exactly into
// h + r by a fused multiply-add (TwoProduct), h added to the running sum p by
// Knuth's TwoSum with the rounding error q, and q + r gathered in c.  p + c is
// the dot product as if computed in twice the working precision.
__device__ __forceinline__ void dot2_acc(float a, float b, float& p, float& c) {
  const float h = __fmul_rn(a, b);
  const float r = __fmaf_rn(a, b, -h);
  const float s = __fadd_rn(p, h);
  const float z = __fsub_rn(s, p);
  const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(s, z)), __fsub_rn(h, z));
  p = s;
  c = __fadd_rn(c, __fadd_rn(q, r));
}

// Shared state of the CTA's current problem.
struct BatchShared {
  int32_t idx[BIR];
  float b[BIR];
  float iv[BIR];
  float est[BCW];
  double dpart[BCW];
  int prob;
  volatile long long drawn;  // rows of the current problem drawn so far
  volatile long long used;   // rows whose iteration is complete (ring entries free)
  volatile int stop;         // the current problem is finished
  volatile int abort;
  int gate;
  int skip;                  // passing windows to skip before the next exact check
  int backoff;               // next value of skip after a failed exact check
  double relres;
};

// The consumer side for one problem with n4 <= 32 NZ: warp w takes rows
// s = w, w + 7, ... of every tau_k; lane l owns float4 columns l + 32 j of
// x (registers), of its share of the update (registers) and of every row it
// copies (shared-memory ring slots of its warp, filled by its own cp.async
// and read back only by itself, so the ring needs no barrier).  Per row: the
// warp's dot <a_s, x> by shuffles, c_s = (t/eta) (<a_s, x> - b_s)/||a_s||^2,
// update += c_s a_s.  Per iteration: the warps' updates are added into one
// shared vector, then z -= update, x = S_lambda(z) (two consumer barriers).
template <int NZ>
__device__ void consume_problem(const BatchArgs& a, BatchShared& S, unsigned char* smem, int p,
                                int64_t* iters_out, double* relres_out, bool* fail_out) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int eta = a.eta;
  const int m = a.m[p];
  const int n = a.n[p];
  const int n4 = (n + 3) >> 2;
  const int64_t lda = a.lda[p];
  const float* Ap = a.A + a.a_off[p];
  const float* bp = a.b + a.b_off[p];
  const int64_t C = a.check_every > 0 ? a.check_every : (m + eta - 1) / eta;
  const int64_t kmax = a.max_iters;
  const float lam = a.lambda;
  const float coef = a.coef;
  const float w_over_eta = (float)(a.W[p] / (double)eta);
  float4* zsh = reinterpret_cast<float4*>(smem);
  float4* xsh = zsh + BMAXNZ * 32;
  float4* dsh = xsh + BMAXNZ * 32;
  float4* ext = reinterpret_cast<float4*>(smem + BEXT_OFF);  // 2 x BHOLDNZ * 32 float4
  const uint32_t slot_bytes = (uint32_t)n4 * 16u;
  // up to 16 float4 per lane a problem runs the instantiation of its own
  // width, NZ = ceil(n4 / 32): only a lane's last column can lie past the row
  constexpr bool kExact = NZ <= 16;
  const int RS = min(BRS_MAX, (int)(BRING_WARP / slot_bytes));  // ring slots of this warp
  unsigned char* ring = smem + BRING_OFF + (size_t)warp * BRING_WARP;
  // rows of this warp per iteration
  const int cw = (eta > warp) ? (eta - warp + BCW - 1) / BCW : 0;
  const int64_t trows = (int64_t)cw * kmax;  // rows of this warp over all iterations

  float4 xr[NZ], dl[NZ];
#pragma unroll
  for (int j = 0; j < NZ; ++j) {
    xr[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    dl[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float est = 0.f;  // lane 0: this warp's share of the windowed residual estimate
  int64_t issued = 0;   // rows of this warp whose copies this lane has issued
  int64_t drawn = 0;    // cached S.drawn
  bool fail = false;
  // the next row to issue, kept incrementally (no 64-bit divisions per row):
  // its global sequence number, its position in the iteration and its slot
  int64_t e_iss = warp;
  int i_iss = 0;
  int slot_iss = 0;

  // copy the next row of this warp into its ring slot (one commit group);
  // with `block`, wait until the producer has drawn it
  auto issue_row = [&](bool block) -> int {
    const int64_t e = e_iss;
    if (e >= drawn) {
      drawn = S.drawn;
      if (e >= drawn) {
        if (!block) return 0;
        const uint64_t t0 = global_timer_ns();
        uint32_t spins = 0;
        while ((drawn = S.drawn) <= e) {
          if (S.abort) return -1;
          if ((++spins & 63u) == 0 && (a.limit_ns == 0 || global_timer_ns() - t0 > a.limit_ns)) return -1;
        }
      }
      __threadfence_block();
    }
    const int32_t row = S.idx[(int)e & (BIR - 1)];
    const float4* src = reinterpret_cast<const float4*>(Ap + (int64_t)row * lda);
    float4* dst = reinterpret_cast<float4*>(ring + (size_t)slot_iss * slot_bytes);
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
      const int col = lane + 32 * j;
      if (!kExact || j == NZ - 1) {
        if (col < n4) cp_async16(dst + col, src + col);
      } else {
        cp_async16(dst + col, src + col);
      }
    }
    cp_async_commit();
    ++issued;
    slot_iss = (slot_iss + 1 == RS) ? 0 : slot_iss + 1;
    if (++i_iss == cw) {
      i_iss = 0;
      e_iss += eta - BCW * (cw - 1);  // first row of this warp in the next iteration
    } else {
      e_iss += BCW;
    }
    return 1;
  };

  int64_t t = 0;  // rows of this warp consumed
  int slot_t = 0; // ring slot of row t
  int64_t k = 0;
  for (; k < kmax && !fail; ++k) {
    for (int i = 0; i < cw; ++i, ++t, slot_t = (slot_t + 1 == RS) ? 0 : slot_t + 1) {
      // row t must be in flight; keep up to RS rows in flight when drawn
      while (issued <= t) {
        if (issue_row(true) < 0) {
          fail = true;
          break;
        }
      }
      if (fail) break;
      while (issued < t + RS && issued < trows && issue_row(false) > 0) {
      }
      { const int64_t pend = issued - t - 1; cp_async_wait_pending(pend < 30 ? (int)pend : 30); }
      const int64_t e = k * eta + warp + BCW * i;
      const float4* rowp = reinterpret_cast<const float4*>(ring + (size_t)slot_t * slot_bytes);
      // four independent partial sums keep the FMA chain short; up to 16
      // float4 per lane the row stays in registers for the update (the widest
      // form reads it from the ring again: its registers hold x and the share)
      constexpr bool kHold = NZ <= BHOLDNZ;
      float4 rv[kHold ? NZ : 1];
      float dp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        const int col = lane + 32 * j;
        if constexpr (kHold) rv[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((kExact && j < NZ - 1) || col < n4) {
          float4 v = rowp[col];
          if ((!kExact || j == NZ - 1) && col == n4 - 1) v = mask_tail(v, col, n);
          if constexpr (kHold) rv[j] = v;
          dp[j & 3] = fmaf(v.x, xr[j].x, dp[j & 3]);
          dp[j & 3] = fmaf(v.y, xr[j].y, dp[j & 3]);
          dp[j & 3] = fmaf(v.z, xr[j].z, dp[j & 3]);
          dp[j & 3] = fmaf(v.w, xr[j].w, dp[j & 3]);
        }
      }
      float d = (dp[0] + dp[1]) + (dp[2] + dp[3]);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      const int ei = (int)e & (BIR - 1);
      const float iv = S.iv[ei];
      const float r = d - S.b[ei];
      if (lane == 0) est = fmaf(w_over_eta * r, r * iv, est);
      const float cval = coef * (r * iv);
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        const int col = lane + 32 * j;
        if ((kExact && j < NZ - 1) || col < n4) {
          float4 v;
          if constexpr (kHold) {
            v = rv[j];
          } else {
            v = rowp[col];
            if (col == n4 - 1) v = mask_tail(v, col, n);
          }
          dl[j].x = fmaf(cval, v.x, dl[j].x);
          dl[j].y = fmaf(cval, v.y, dl[j].y);
          dl[j].z = fmaf(cval, v.z, dl[j].z);
          dl[j].w = fmaf(cval, v.w, dl[j].w);
        }
      }
    }
    // every consumer thread reaches the barriers below whether it failed or not
    // ---- end of iteration k: update = sum of the warps' shares ----
    if constexpr (NZ <= BHOLDNZ) {
      // no shared-memory atomics: warps 0..3 store their shares into four
      // buffers (the update buffer, the x buffer -- rewritten by the update
      // below -- and two more); warps 4..6 then add theirs into buffers 1..3,
      // each after a pair barrier with that buffer's writer; the update loop
      // sums the four buffers in order
      float4* dst = (warp == 0) ? dsh : (warp == 1 || warp == 4) ? xsh
                    : (warp == 2 || warp == 5) ? ext : ext + BHOLDNZ * 32;
      if (warp >= 4) pair_wait(warp);
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        const int col = lane + 32 * j;
        if ((kExact && j < NZ - 1) || col < n4) {
          if (warp >= 4) {
            const float4 o = dst[col];
            dst[col] = make_float4(o.x + dl[j].x, o.y + dl[j].y, o.z + dl[j].z, o.w + dl[j].w);
          } else {
            dst[col] = dl[j];
          }
        }
        dl[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (warp >= 1 && warp <= 3) pair_arrive(warp);
    } else {
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        const int col = lane + 32 * j;
        if (col < n4) {
          float* dp = reinterpret_cast<float*>(dsh + col);
          atomicAdd(dp + 0, dl[j].x);
          atomicAdd(dp + 1, dl[j].y);
          atomicAdd(dp + 2, dl[j].z);
          atomicAdd(dp + 3, dl[j].w);
        }
        dl[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (consumer_sync_or(fail ? 1 : 0)) {
      fail = true;
      break;
    }
    if (tid == 0) S.used = (k + 1) * (int64_t)eta;
    for (int c4 = tid; c4 < n4; c4 += BC) {
      float4 zv = zsh[c4];
      float4 dv = dsh[c4];
      if constexpr (NZ <= BHOLDNZ) {
        const float4 d1 = xsh[c4], d2 = ext[c4], d3 = ext[BHOLDNZ * 32 + c4];
        dv = make_float4(((dv.x + d1.x) + d2.x) + d3.x, ((dv.y + d1.y) + d2.y) + d3.y,
                         ((dv.z + d1.z) + d2.z) + d3.z, ((dv.w + d1.w) + d2.w) + d3.w);
      }
      zv.x -= dv.x;
      zv.y -= dv.y;
      zv.z -= dv.z;
      zv.w -= dv.w;
      if (c4 == n4 - 1) zv = mask_tail(zv, c4, n);
      zsh[c4] = zv;
      xsh[c4] = soft_shrink4(zv, lam);
      dsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (lane == 0) S.est[warp] = est;
    consumer_sync();
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
      const int col = lane + 32 * j;
      xr[j] = ((kExact && j < NZ - 1) || col < n4) ? xsh[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool last = (k + 1 == kmax);
    if ((k + 1) % C != 0 && !last) continue;

    // ---- check point: gate on the estimate, then the exact residual ----
    if (tid == 0) {
      float tot = 0.f;
      for (int w = 0; w < BCW; ++w) tot += S.est[w];
      const float window = (float)((k + 1) % C == 0 ? C : (k + 1) % C);
      const double est_mean = (double)(tot / window);
      const double lim = 4.0 * a.tol;
      const bool open = a.tol > 0.0 && est_mean <= lim * lim * a.bnorm2[p];
      // after an exact check that did not stop the problem, skip the next
      // 1, 2, 4, .. 16 windows whose estimate passes (the estimate hovers
      // near the gate while the residual is just above tol)
      S.gate = last || (open && S.skip == 0);
      if (open && S.skip > 0) --S.skip;
    }
    est = 0.f;
    consumer_sync();
    if (S.gate) {
      // exact check: one warp per row; each lane's share of <a_i, x> by the
      // compensated dot product Dot2 (FP32, as accurate as twice the working
      // precision), the lanes' shares and r_i^2 summed in FP64
      double acc = 0.0;
      for (int i = warp; i < m; i += BCW) {
        const float4* row = reinterpret_cast<const float4*>(Ap + (int64_t)i * lda);
        float ph = 0.f, pl = 0.f;
        // 4 loads per lane in flight at a time
        for (int j0 = 0; j0 < NZ; j0 += 4) {
          float4 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c4 = lane + 32 * (j0 + u);
            const bool in = (j0 + u < NZ) && ((kExact && j0 + u < NZ - 1) || c4 < n4);
            v[u] = in ? __ldg(row + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
            if ((!kExact || j0 + u == NZ - 1) && c4 == n4 - 1) v[u] = mask_tail(v[u], c4, n);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c4 = lane + 32 * (j0 + u);
            if ((j0 + u < NZ) && ((kExact && j0 + u < NZ - 1) || c4 < n4)) {
              const float4 xv = xsh[c4];
              dot2_acc(v[u].x, xv.x, ph, pl);
              dot2_acc(v[u].y, xv.y, ph, pl);
              dot2_acc(v[u].z, xv.z, ph, pl);
              dot2_acc(v[u].w, xv.w, ph, pl);
            }
          }
        }
        double dd = (double)ph + (double)pl;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
        if (lane == 0) {
          const double ri = dd - (double)__ldg(bp + i);
          acc += ri * ri;
        }
      }
      if (lane == 0) S.dpart[warp] = acc;
      consumer_sync();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < BCW; ++w) tot += S.dpart[w];
        const double bb = a.bnorm2[p];
        S.relres = sqrt(tot) / (bb > 0.0 ? sqrt(bb) : 1e-30);
      }
      consumer_sync();
      if ((a.tol > 0.0 && S.relres <= a.tol) || last) {
        k += 1;
        break;
      }
      if (tid == 0) {
        S.skip = S.backoff;
        S.backoff = min(2 * S.backoff + 1, 15);
      }
    }
  }
  // drain this thread's prefetched rows before the ring is reused
  cp_async_wait_all();
  *iters_out = k;
  *relres_out = S.relres;
  *fail_out = fail;

}

__global__ void __launch_bounds__(BT, 1) rska_batched_kernel(BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ BatchShared S;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int eta = a.eta;
  if (tid == 0) S.abort = 0;
  __syncthreads();

  for (;;) {
    if (tid == 0) {
      const int qi = atomicAdd(a.queue, 1);
      S.prob = (qi < a.P && ld_relaxed_s32(a.status) == kStatusOk) ? a.order[qi] : -1;
      S.stop = 0;
      S.drawn = 0;
      S.used = 0;
      S.relres = -1.0;
      S.skip = 0;
      S.backoff = 1;
    }
    __syncthreads();
    const int p = S.prob;
    if (p < 0) break;
    const int m = a.m[p];
    const int n = a.n[p];
    const int n4 = (n + 3) >> 2;
    const float* bp = a.b + a.b_off[p];
    const int64_t ro = a.row_off[p];
    const int64_t kmax = a.max_iters;

    if (warp == BCW) {
      // ------------------------------------------------- index producer --
      // Draws rows e, e+1, ... of this problem's index stream (row e is draw
      // s = e mod eta of iteration e / eta) with b and 1/||a||^2 into the
      // index ring, up to BIR rows ahead of the last completed iteration.
      int64_t jj0 = 0;
      int s0 = 0;
      const int64_t total = kmax * (int64_t)eta;
      for (int64_t e = 0; e < total; e += 32) {
        if (lane == 0) {
          const uint64_t t0 = global_timer_ns();
          uint32_t spins = 0;
          while (e + 32 - S.used > BIR && !S.stop && !S.abort) {
            // far ahead: sleep rather than spin, a spinning warp steals the
            // shared-memory pipe from the consumers
            __nanosleep(500);
            if ((++spins & 15u) == 0 && (a.limit_ns == 0 || global_timer_ns() - t0 > a.limit_ns)) {
              atomicCAS(a.status, kStatusOk, kStatusTimeout);
              S.abort = 1;
            }
          }
        }
        __syncwarp();
        if (S.stop || S.abort) break;
        int s = s0 + lane;
        int64_t jj = jj0;
        while (s >= eta) {
          s -= eta;
          ++jj;
        }
        int32_t i0, i1;
        draw_pair(a.seed, jj, (uint32_t)(s >> 1), a.sid[p], a.thr + ro, a.alias + ro,
                  (uint32_t)m, &i0, &i1);
        const int32_t row = (s & 1) ? i1 : i0;
        const int slot = (int)(e + lane) & (BIR - 1);
        S.idx[slot] = row;
        S.b[slot] = __ldg(bp + row);
        S.iv[slot] = __ldg(a.inv_nu + ro + row);
        __syncwarp();
        __threadfence_block();
        if (lane == 0) S.drawn = e + 32;
        s0 += 32;
        while (s0 >= eta) {
          s0 -= eta;
          ++jj0;
        }
      }
    } else {
      // ------------------------------------------------------ consumers --
      float4* zsh = reinterpret_cast<float4*>(smem);
      float4* xsh = zsh + BMAXNZ * 32;
      float4* dsh = xsh + BMAXNZ * 32;
      for (int c4 = tid; c4 < n4; c4 += BC) {
        zsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        xsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        dsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      consumer_sync();
      const int nz = (n4 + 31) >> 5;
      int64_t iters = 0;
      double relres = -1.0;
      bool fail = false;
      // one instantiation per width: columns a lane does not own still cost
      // issue slots and lengthen the dot's chains
      switch (nz) {
        case 1: consume_problem<1>(a, S, smem, p, &iters, &relres, &fail); break;
        case 2: consume_problem<2>(a, S, smem, p, &iters, &relres, &fail); break;
        case 3: consume_problem<3>(a, S, smem, p, &iters, &relres, &fail); break;
        case 4: consume_problem<4>(a, S, smem, p, &iters, &relres, &fail); break;
        case 5: consume_problem<5>(a, S, smem, p, &iters, &relres, &fail); break;
        case 6: consume_problem<6>(a, S, smem, p, &iters, &relres, &fail); break;
        case 7: consume_problem<7>(a, S, smem, p, &iters, &relres, &fail); break;
        case 8: consume_problem<8>(a, S, smem, p, &iters, &relres, &fail); break;
        case 9: consume_problem<9>(a, S, smem, p, &iters, &relres, &fail); break;
        case 10: consume_problem<10>(a, S, smem, p, &iters, &relres, &fail); break;
        case 11: consume_problem<11>(a, S, smem, p, &iters, &relres, &fail); break;
        case 12: consume_problem<12>(a, S, smem, p, &iters, &relres, &fail); break;
        case 13: consume_problem<13>(a, S, smem, p, &iters, &relres, &fail); break;
        case 14: consume_problem<14>(a, S, smem, p, &iters, &relres, &fail); break;
        case 15: consume_problem<15>(a, S, smem, p, &iters, &relres, &fail); break;
        case 16: consume_problem<16>(a, S, smem, p, &iters, &relres, &fail); break;
        default: consume_problem<BMAXNZ>(a, S, smem, p, &iters, &relres, &fail); break;
      }
      // problem finished (or failed): publish results, release the producer
      if (tid == 0) {
        S.stop = 1;
        if (fail) {
          atomicCAS(a.status, kStatusOk, kStatusTimeout);
          S.abort = 1;
        }
        a.iters[p] = iters;
        a.relres[p] = relres;
      }
      float4* zo = reinterpret_cast<float4*>(a.z + a.x_off[p]);
      float4* xo = reinterpret_cast<float4*>(a.x + a.x_off[p]);
      for (int c4 = tid; c4 < n4; c4 += BC) {
        zo[c4] = zsh[c4];
        xo[c4] = xsh[c4];
      }
    }
    __syncthreads();
    if (S.abort) break;
  }
  cp_async_wait_all();
}

}  // namespace
}  // namespace rska

using rska::BatchArgs;

struct rska_batch {
  int32_t P = 0;
  int32_t eta = 1;
  float lambda = 0.f, t = 1.f;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t total_rows = 0, total_x = 0;
  int max_n4 = 0;
  std::vector<int64_t> h_x_off;
  // device
  const float* A = nullptr;
  const float* b = nullptr;
  int32_t* d_order = nullptr;
  int64_t* d_a_off = nullptr;
  int32_t* d_m = nullptr;
  int32_t* d_n = nullptr;
  int64_t* d_lda = nullptr;
  int64_t* d_b_off = nullptr;
  int64_t* d_row_off = nullptr;
  int64_t* d_x_off = nullptr;
  double* nu = nullptr;
  float* inv_nu = nullptr;
  uint32_t* thr = nullptr;
  int32_t* alias = nullptr;
  double* W = nullptr;
  double* bnorm2 = nullptr;
  float* z = nullptr;
  float* x = nullptr;
  int64_t* iters = nullptr;
  double* relres = nullptr;
  int* pstat = nullptr;
  int* queue = nullptr;
  int* status = nullptr;
  uint32_t* d_sid = nullptr;        // index-stream id per problem
  int sticky = RSKA_OK;
  uint64_t limit_ns = 2000000000ull;
};

namespace {

void batch_free(rska_batch* bt) {
  void* ptrs[] = {bt->d_order, bt->d_a_off, bt->d_m,   bt->d_n,     bt->d_lda,  bt->d_b_off,
                  bt->d_row_off, bt->d_x_off, bt->nu,  bt->inv_nu,  bt->thr,    bt->alias,
                  bt->W,       bt->bnorm2,  bt->z,     bt->x,       bt->iters,  bt->relres,
                  bt->pstat,   bt->queue,   bt->status, bt->d_sid};
  for (void* p : ptrs) cudaFree(p);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

BatchArgs make_args(rska_batch* bt) {
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.P = bt->P;
  a.order = bt->d_order;
  a.A = bt->A;
  a.a_off = bt->d_a_off;
  a.m = bt->d_m;
  a.n = bt->d_n;
  a.lda = bt->d_lda;
  a.b = bt->b;
  a.b_off = bt->d_b_off;
  a.row_off = bt->d_row_off;
  a.inv_nu = bt->inv_nu;
  a.thr = bt->thr;
  a.alias = bt->alias;
  a.W = bt->W;
  a.bnorm2 = bt->bnorm2;
  a.x_off = bt->d_x_off;
  a.sid = bt->d_sid;
  a.z = bt->z;
  a.x = bt->x;
  a.iters = bt->iters;
  a.relres = bt->relres;
  a.lambda = bt->lambda;
  a.coef = bt->t / (float)bt->eta;
  a.eta = bt->eta;
  a.seed = bt->seed;
  a.queue = bt->queue;
  a.status = bt->status;
  a.limit_ns = bt->limit_ns;
  return a;
}

}  // namespace

extern "C" {

int rska_batch_setup(rska_batch** out, int32_t P, const float* A, const int64_t* a_off,
                     const int64_t* m, const int64_t* n, const int64_t* lda, const float* b,
                     const int64_t* b_off, float lambda, int32_t eta, float t, uint64_t seed,
                     void* stream) {
  if (!out) return RSKA_EINVAL;
  *out = nullptr;
  if (P < 1 || !A || !b || !a_off || !m || !n || !lda || !b_off || eta < 1 ||
      eta > rska::kMaxEta || !(lambda >= 0.f) || !std::isfinite(lambda) || !(t > 0.f) ||
      !std::isfinite(t))
    return RSKA_EINVAL;
  if ((reinterpret_cast<uintptr_t>(A) % 16) != 0) return RSKA_EINVAL;
  if (eta > rska::BMAX_ETA) return RSKA_EUNSUPPORTED;
  std::vector<int32_t> hm(P), hn(P);
  std::vector<int64_t> row_off(P), x_off(P + 1);
  int64_t rows = 0, xs = 0;
  int max_n4 = 1;
  for (int32_t p = 0; p < P; ++p) {
    if (m[p] < 1 || n[p] < 1 || lda[p] < n[p] || (lda[p] % 4) != 0 || (a_off[p] % 4) != 0 ||
        a_off[p] < 0 || b_off[p] < 0 || m[p] > 0x7fffffff)
      return RSKA_EINVAL;
    const int64_t n4 = (n[p] + 3) / 4;
    if (n4 > (int64_t)32 * rska::BMAXNZ) return RSKA_EUNSUPPORTED;
    hm[p] = (int32_t)m[p];
    hn[p] = (int32_t)n[p];
    row_off[p] = rows;
    rows += m[p];
    x_off[p] = xs;
    xs += n4 * 4;
    max_n4 = std::max<int>(max_n4, (int)n4);
  }
  x_off[P] = xs;
  // largest estimated work first (iterations and bytes per iteration both grow with n)
  std::vector<int32_t> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t u, int32_t v) {
    const double wu = (double)hn[u] * hn[u] + (double)hm[u] * hn[u] / eta;
    const double wv = (double)hn[v] * hn[v] + (double)hm[v] * hn[v] / eta;
    return wu > wv;
  });

  rska_batch* bt = new (std::nothrow) rska_batch;
  if (!bt) return RSKA_ENOMEM;
  bt->P = P;
  bt->eta = eta;
  bt->lambda = lambda;
  bt->t = t;
  bt->seed = seed;
  bt->stream = static_cast<cudaStream_t>(stream);
  bt->A = A;
  bt->b = b;
  bt->total_rows = rows;
  bt->total_x = xs;
  bt->max_n4 = max_n4;
  bt->h_x_off = x_off;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, dev);
  double* q = nullptr;
  int32_t* stk = nullptr;
  if (e == cudaSuccess &&
      ((e = dalloc(&bt->d_order, P)) != cudaSuccess || (e = dalloc(&bt->d_a_off, P)) != cudaSuccess ||
       (e = dalloc(&bt->d_m, P)) != cudaSuccess || (e = dalloc(&bt->d_n, P)) != cudaSuccess ||
       (e = dalloc(&bt->d_lda, P)) != cudaSuccess || (e = dalloc(&bt->d_b_off, P)) != cudaSuccess ||
       (e = dalloc(&bt->d_row_off, P)) != cudaSuccess ||
       (e = dalloc(&bt->d_x_off, P + 1)) != cudaSuccess || (e = dalloc(&bt->nu, rows)) != cudaSuccess ||
       (e = dalloc(&bt->inv_nu, rows)) != cudaSuccess || (e = dalloc(&bt->thr, rows)) != cudaSuccess ||
       (e = dalloc(&bt->alias, rows)) != cudaSuccess || (e = dalloc(&bt->W, P)) != cudaSuccess ||
       (e = dalloc(&bt->bnorm2, P)) != cudaSuccess || (e = dalloc(&bt->z, xs)) != cudaSuccess ||
       (e = dalloc(&bt->x, xs)) != cudaSuccess || (e = dalloc(&bt->iters, P)) != cudaSuccess ||
       (e = dalloc(&bt->relres, P)) != cudaSuccess || (e = dalloc(&bt->pstat, P)) != cudaSuccess ||
       (e = dalloc(&bt->queue, 1)) != cudaSuccess || (e = dalloc(&bt->status, 1)) != cudaSuccess ||
       (e = dalloc(&bt->d_sid, P)) != cudaSuccess ||
       (e = dalloc(&q, rows)) != cudaSuccess || (e = dalloc(&stk, rows)) != cudaSuccess)) {
  }
  cudaStream_t s = bt->stream;
  std::vector<uint32_t> sid(P);
  std::iota(sid.begin(), sid.end(), 0u);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_sid, sid.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_order, order.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_a_off, a_off, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_m, hm.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_n, hn.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_lda, lda, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_b_off, b_off, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_row_off, row_off.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_x_off, x_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->pstat, 0, sizeof(int) * P, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->z, 0, sizeof(float) * xs, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->x, 0, sizeof(float) * xs, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->iters, 0, sizeof(int64_t) * P, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->relres, 0, sizeof(double) * P, s);
  if (e == cudaSuccess) {
    BatchArgs a = make_args(bt);
    const int nblk = std::min<int>(P, bt->num_sms * 8);
    rska::batch_norms_kernel<<<nblk, 256, 0, s>>>(a, bt->nu, bt->inv_nu, bt->pstat);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      rska::batch_alias_kernel<<<(P + 63) / 64, 64, 0, s>>>(a, bt->nu, q, stk, bt->thr, bt->alias,
                                                            bt->W, bt->bnorm2, bt->pstat);
      e = cudaGetLastError();
    }
  }
  std::vector<int> hst(P, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), bt->pstat, sizeof(int) * P, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(stk);
  if (e != cudaSuccess) {
    batch_free(bt);
    delete bt;
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  for (int32_t p = 0; p < P; ++p) {
    if (hst[p] != 0) {
      batch_free(bt);
      delete bt;
      return hst[p];
    }
  }
  *out = bt;
  return RSKA_OK;
}

int rska_batch_set_stream_ids(rska_batch* bt, const uint32_t* ids) {
  if (!bt || !ids) return RSKA_EINVAL;
  cudaError_t e = cudaMemcpyAsync(bt->d_sid, ids, sizeof(uint32_t) * bt->P, cudaMemcpyHostToDevice,
                                  bt->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_batch_solve(rska_batch* bt, int64_t max_iters, double tol, int64_t check_every) {
  if (!bt || max_iters < 1 || !(tol >= 0.0) || check_every < 0) return RSKA_EINVAL;
  if (bt->sticky) return bt->sticky;
  cudaStream_t s = bt->stream;
  BatchArgs a = make_args(bt);
  a.max_iters = max_iters;
  a.tol = tol;
  a.check_every = check_every;
  const size_t smem = rska::BSMEM;
  cudaError_t e = cudaFuncSetAttribute(rska::rska_batched_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->queue, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->z, 0, sizeof(float) * bt->total_x, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->x, 0, sizeof(float) * bt->total_x, s);
  int blocks_per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, rska::rska_batched_kernel,
                                                      rska::BT, smem);
  if (e == cudaSuccess) {
    const int grid = std::max(1, std::min<int>(bt->P, bt->num_sms * std::max(1, blocks_per_sm)));
    rska::rska_batched_kernel<<<grid, rska::BT, smem, s>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    bt->sticky = RSKA_ECUDA;
    return RSKA_ECUDA;
  }
  return RSKA_OK;
}

int rska_batch_results(rska_batch* bt, int64_t* iters, double* rel_res) {
  if (!bt) return RSKA_EINVAL;
  cudaStream_t s = bt->stream;
  int st = 0;
  cudaError_t e = cudaSuccess;
  if (iters) e = cudaMemcpyAsync(iters, bt->iters, sizeof(int64_t) * bt->P, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && rel_res)
    e = cudaMemcpyAsync(rel_res, bt->relres, sizeof(double) * bt->P, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, bt->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return RSKA_ECUDA;
  if (st != 0) bt->sticky = st;
  return st;
}

int rska_batch_get_x(rska_batch* bt, float* x_out, float* z_out) {
  if (!bt) return RSKA_EINVAL;
  cudaStream_t s = bt->stream;
  cudaError_t e = cudaSuccess;
  if (x_out) e = cudaMemcpyAsync(x_out, bt->x, sizeof(float) * bt->total_x, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && z_out)
    e = cudaMemcpyAsync(z_out, bt->z, sizeof(float) * bt->total_x, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_batch_offsets(rska_batch* bt, int64_t* x_off) {
  if (!bt || !x_off) return RSKA_EINVAL;
  std::memcpy(x_off, bt->h_x_off.data(), sizeof(int64_t) * (bt->P + 1));
  return RSKA_OK;
}

int rska_batch_get_tables(rska_batch* bt, double* nu_out, uint32_t* thr_out, int32_t* alias_out) {
  if (!bt) return RSKA_EINVAL;
  cudaStream_t s = bt->stream;
  const size_t R = (size_t)bt->total_rows;
  cudaError_t e = cudaSuccess;
  if (nu_out) e = cudaMemcpyAsync(nu_out, bt->nu, sizeof(double) * R, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && thr_out)
    e = cudaMemcpyAsync(thr_out, bt->thr, sizeof(uint32_t) * R, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && alias_out)
    e = cudaMemcpyAsync(alias_out, bt->alias, sizeof(int32_t) * R, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_batch_destroy(rska_batch* bt) {
  if (!bt) return RSKA_EINVAL;
  cudaStreamSynchronize(bt->stream);
  batch_free(bt);
  delete bt;
  return RSKA_OK;
}

}  // extern "C"
