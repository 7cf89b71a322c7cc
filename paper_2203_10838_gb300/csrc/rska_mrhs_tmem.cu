// rska_mrhs_tmem.cu -- the shared-A multi-right-hand-side RSKA iteration as
// one persistent tensor-core kernel whose iterate never leaves the chip.
//
// With X = S_lambda(Z) (one column per right-hand side), one step of eq.
// (rska) for every right-hand side at once is the matrix form of Sec. 3:
//
//   Res = A_tau X - B_tau                  (eta x R, contraction over n)
//   Z  -= (t/eta) A_tau^T D_tau^-2 Res     (n x R,   contraction over eta)
//
// Work split.  CTA (rs, cs) owns the 128 right-hand sides 128 rs .. + 127 and
// the 256 columns 256 cs .. + 255 of Z^T, held in tensor memory for the whole
// launch (FP32, lanes = right-hand sides, columns 0..255).  Per iteration:
//
//  1. Its slice of A_tau (eta_p rows x 256 columns, BF16) arrives by TMA in
//     four 64-column chunks from a dense copy of A_tau in global memory that
//     all CTAs gathered during the previous iteration.
//  2. Eight epilogue warps read Z^T from tensor memory, form X = S_lambda(Z)
//     and split it into BF16 high and low parts, 64 columns at a time, into a
//     two-slot ring in shared memory; one thread issues the tcgen05 MMAs
//     P^T (128 x eta_p, tensor-memory columns 256..) += X^T_chunk A_tau_chunk^T
//     (M 128, N eta_p, K 16; both operands K-major).
//  3. P^T is this CTA's share of the residual product; the epilogue adds it
//     with reductions (one 128-byte line per warp instruction) into a global
//     accumulator of the right-hand-side slice that starts at -b_tau (the
//     helper warps of each CTA of the slice write a block of rows of that
//     start value one iteration ahead), and every CTA passes one bounded grid
//     barrier.
//  4. The epilogue reads the residuals back, forms the scaled residual
//     -(t/eta) (A_tau x - b_tau) / ||a_tau||^2 for its right-hand sides,
//     splits it into high and low parts and streams it through the ring;
//     the MMA thread forms D^T (M 128, N 256, K 16) = sum R'^T_chunk
//     A_tau_chunk in the tensor-memory columns the residual product used,
//     with A_tau read column-major (the same shared-memory tile serves as
//     the K-major operand of step 2 and the MN-major operand here), and the
//     epilogue adds D^T to Z^T in FP32 (one rounding per iteration, as when
//     z -= d is applied outside the tensor core).
//
// Two helper warps gather the rows of tau_{k+1} into the other dense A_tau
// buffer with bulk copies (and stage tau_{k+1} and 1/||a||^2 at tau_{k+1})
// while iteration k computes, so the only per-iteration exchanges are the residual reduction
// and the grid barrier.  Every wait is bounded; on expiry the kernel records
// a timeout, lets its issued copies and MMAs finish, and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rska_device.cuh"
#include "rska_mrhs_tmem.h"
#include "rska_tc.cuh"

namespace rska {
namespace {

using namespace tc;

constexpr int kThreads = 384;      // warp 0 TMA, warp 1 MMA, warps 2-3 gather, warps 4-11 epilogue
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kSliceR = 128;       // right-hand sides per CTA (tensor-memory lanes)
constexpr int kSliceN = 256;       // columns of Z^T per CTA
constexpr uint32_t kRingSlot = 32768;  // one ring slot: high part (16 KB) + low part (16 KB)
constexpr uint32_t kStage = 16384;     // gather staging buffer: one row piece of 8192 BF16
constexpr uint32_t kTmemCols = 512;    // Z^T in columns 0..255, the residual product from 256
constexpr uint32_t kTmemRes = 256;
// Register split: the block is launched with kLaunchRegs per thread (the
// count ptxas gives under the launch bounds; the launch refuses a build with
// any other count, since the epilogue's increase would then wait for
// registers that nobody releases).  Warps 0-3 hand registers back and the
// two epilogue warpgroups take them: 4 x 32 x kLowRegs + 8 x 32 x kHighRegs
// is exactly the launch's total, and the epilogue runs without spills.
constexpr int kLaunchRegs = 168;
constexpr int kLowRegs = 88;
constexpr int kHighRegs = 208;
static_assert(128 * kLowRegs + 256 * kHighRegs == kThreads * kLaunchRegs,
              "the register split must add up to the launch's registers");

// kind::f16 instruction descriptor: D FP32, A and B BF16, M = 128, N = n;
// b_mn: B read MN-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (b_mn ? (1u << 16) : 0u) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory descriptor of an MN-major operand written by TMA with the
// 128-byte swizzle: 64-element MN blocks `lbo` bytes apart, rows (K) of 128
// bytes in 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t smem_addr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// Bounded wait that also gives up once another role has raised *abort
// (abort may be null: a drain of work already issued, which always ends).
__device__ __forceinline__ bool wait_phase(uint64_t* b, uint32_t parity, uint64_t limit_ns,
                                           const volatile int* abort) {
  if (mb_try_wait(b, parity)) return true;
  if (limit_ns == 0) return false;  // a zero limit expires at the first failed poll
  const uint64_t t0 = global_timer_ns();
  while (!mb_try_wait(b, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
    if (abort != nullptr && *abort) return false;
  }
  return true;
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Barrier over the eight epilogue warps (named barrier 1) that also ORs a
// flag across them.
__device__ __forceinline__ int epi_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(pred), "n"(kEpiThreads)
      : "memory");
  return r;
}

// 32 FP32 values into 32 consecutive tensor-memory columns of this warp's lanes.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31, %32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Two FP32 values as BF16 high parts (one packed conversion, round to nearest
// even) and the low parts of what remains: v = hi + lo + O(2^-17 |v|).
__device__ __forceinline__ void split2(float v0, float v1, uint32_t* hi, uint32_t* lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);
  const float h0 = __uint_as_float(hb << 16);           // the BF16 value of v0, exactly
  const float h1 = __uint_as_float(hb & 0xFFFF0000u);  // the BF16 value of v1
  const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - h0, v1 - h1);
  *hi = hb;
  *lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 32 FP32 values of one row (row `row` of a 128-row, 64-column K-major BF16
// operand, columns 32 half .. + 31) into the high part at `hi` and, when
// `two`, the low part at `lo` (128-byte swizzle as TMA would write it); eight
// values (one 16-byte piece of each part) at a time.
__device__ __forceinline__ void store_split_row(unsigned char* hi, unsigned char* lo, int row,
                                                int half, const float (&v)[32], bool two) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split2(v[8 * q + 2 * j], v[8 * q + 2 * j + 1], &hw[j], &lw[j]);
    const uint32_t off = sw128_off(row, 4 * half + q);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if (two) *reinterpret_cast<uint4*>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

struct alignas(8) Bars {
  uint64_t a[4];        // A_tau chunk c landed (TMA transaction count)
  uint64_t full[2];     // ring slot written by the eight epilogue warps
  uint64_t empty[2];    // ring slot read by the MMAs (tcgen05.commit)
  uint64_t res_done;    // residual-product MMAs of this iteration complete
  uint64_t upd_done;    // update MMAs of this iteration complete
  uint64_t passed;      // this CTA has passed grid barrier b (one phase per barrier)
  uint64_t gathered;    // both helper warps finished the next iteration's gather
  uint64_t fin;         // every MMA of this CTA complete (exit drain)
  uint64_t stage;       // gather staging buffer filled (bulk copy)
  uint64_t rchunk;      // the eight epilogue warps formed chunk kq of R' (one phase per iteration)
};

__global__ void __launch_bounds__(kThreads, 1)
    mrhs_tmem_kernel(const __grid_constant__ CUtensorMap mapG, MrhsTmemArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ Bars bars;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_flag;
  __shared__ float s_iv[3][256];

  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int eta_p = a.eta_p;
  const uint32_t chunk_bytes = (uint32_t)eta_p * 128u;  // one 64-column chunk of A_tau
  unsigned char* atile = smem;                            // 4 chunks
  unsigned char* ring = smem + 4 * (size_t)chunk_bytes;  // 2 slots of 32 KB
  unsigned char* stagebuf = ring + 2 * (size_t)kRingSlot;  // 16 KB

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int nCTA = gridDim.x;
  // consecutive CTAs take consecutive column slices of one right-hand-side slice
  const int rs = blockIdx.x / a.n_slices;
  const int cs = blockIdx.x % a.n_slices;
  const int rchunks = eta_p / 64;                        // scaled-residual chunks
  // gather schedules 2.. start the next gather once chunk kq of the scaled
  // residual is formed (its reads of the accumulator have landed)
  const int kq = a.gather_sched >= 2 ? min(a.gather_sched - 2, rchunks - 1) : -1;
  const int cnt = a.cnt;

  if (tid == 0) {
    for (int c = 0; c < 4; ++c) mb_init(&bars.a[c], 1);
    for (int s = 0; s < 2; ++s) {
      mb_init(&bars.full[s], kEpiWarps);
      mb_init(&bars.empty[s], 1);
    }
    mb_init(&bars.res_done, 1);
    mb_init(&bars.upd_done, 1);
    mb_init(&bars.passed, 1);
    mb_init(&bars.gathered, 2);
    mb_init(&bars.fin, 1);
    mb_init(&bars.stage, 1);
    mb_init(&bars.rchunk, kEpiWarps);
    s_abort = 0;
    s_flag = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto fail = [&]() {
    atomicCAS(a.status, kStatusOk, kStatusTimeout);
    s_abort = 1;
  };

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kLowRegs));
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kHighRegs));
  }
  if (warp == 0) {
    // ------------------------------------------------ TMA producer --------
    int issued = 0;  // iterations whose A_tau slice was requested
    if (lane == 0) {
      for (int i = 0; i < cnt; ++i) {
        // the tile is free once the previous iteration's update MMAs are done
        // (which also orders this after grid barrier i, so the dense copy
        // of A_tau(i) is complete); the first waits for the start barrier
        const bool ok = (i == 0) ? wait_phase(&bars.passed, 0u, a.limit_ns, &s_abort)
                                 : wait_phase(&bars.upd_done, (uint32_t)((i - 1) & 1), a.limit_ns,
                                              &s_abort);
        if (!ok) {
          if (!s_abort) fail();
          break;
        }
        for (int c = 0; c < 4; ++c) {
          mb_expect_tx(&bars.a[c], chunk_bytes);
          tma_load_2d(atile + (size_t)c * chunk_bytes, &mapG, cs * kSliceN + 64 * c,
                      (i & 1) * eta_p, &bars.a[c]);
        }
        issued = i + 1;
      }
      // the copies this CTA requested land before it may end
      if (issued > 0) {
        const uint64_t dl = drain_limit(a.limit_ns);
        for (int c = 0; c < 4; ++c) wait_phase(&bars.a[c], (uint32_t)((issued - 1) & 1), dl, nullptr);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer ----------
    if (lane == 0) {
      const uint32_t id_res = idesc_bf16(eta_p, false);
      const uint32_t id_upd = idesc_bf16(kSliceN, true);
      const uint32_t abase = saddr(atile);
      const uint32_t rbase = saddr(ring);
      uint32_t u = 0;  // ring uses
      bool ok = true;
      for (int i = 0; i < cnt && ok; ++i) {
        // residual product over this CTA's 256 columns, 64 at a time
        for (int c = 0; c < 4 && ok; ++c) {
          const uint32_t slot = u & 1;
          ok = wait_phase(&bars.a[c], (uint32_t)(i & 1), a.limit_ns, &s_abort) &&
               wait_phase(&bars.full[slot], (u >> 1) & 1, a.limit_ns, &s_abort);
          if (!ok) break;
          tc_fence_after();
          const uint32_t xs = rbase + slot * kRingSlot;
          const uint32_t bc = abase + (uint32_t)c * chunk_bytes;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t db = desc_sw128(bc) + (uint64_t)(2 * kk);
            mma_bf16(tmem + kTmemRes, desc_sw128(xs) + (uint64_t)(2 * kk), db, id_res,
                     (c > 0 || kk > 0) ? 1u : 0u);
            if (a.nsplit_x == 2)
              mma_bf16(tmem + kTmemRes, desc_sw128(xs + 16384) + (uint64_t)(2 * kk), db, id_res, 1u);
          }
          mma_commit(&bars.empty[slot]);
          ++u;
        }
        if (!ok) break;
        mma_commit(&bars.res_done);
        // update: D^T = R'^T A_tau (R' carries the minus sign) into the
        // columns the residual product has left (its readout precedes the
        // grid barrier), 64 rows of A_tau (the contraction index) at a time;
        // the epilogue adds D^T to Z^T in FP32
        for (int qq = 0; qq < rchunks && ok; ++qq) {
          const uint32_t slot = u & 1;
          ok = wait_phase(&bars.full[slot], (u >> 1) & 1, a.limit_ns, &s_abort);
          if (!ok) break;
          tc_fence_after();
          const uint32_t rsl = rbase + slot * kRingSlot;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t db =
                desc_mn_sw128(abase + (uint32_t)(64 * qq + 16 * kk) * 128u, chunk_bytes);
            mma_bf16(tmem + kTmemRes, desc_sw128(rsl) + (uint64_t)(2 * kk), db, id_upd,
                     (qq > 0 || kk > 0) ? 1u : 0u);
            if (a.nsplit_r == 2)
              mma_bf16(tmem + kTmemRes, desc_sw128(rsl + 16384) + (uint64_t)(2 * kk), db, id_upd,
                       1u);
          }
          mma_commit(&bars.empty[slot]);
          ++u;
        }
        if (!ok) break;
        mma_commit(&bars.upd_done);
      }
      if (!ok && !s_abort) fail();
      // every MMA issued by this thread completes before the tensor memory
      // and the shared-memory operands go away
      mma_commit(&bars.fin);
      wait_phase(&bars.fin, 0u, drain_limit(a.limit_ns), nullptr);
    }
  } else if (warp < 4) {
    // ------------------------------------------------ gather helpers ------
    // Warp 3 stages 1/||a||^2 at tau_i into s_iv [i % 3];
    // lane 0 of warp 2 copies this CTA's rows of A_tau(i) (rows s = blockIdx
    // mod grid) into the dense buffer i % 2 with bulk copies through a 16 KB
    // staging buffer (global -> shared -> global), columns < n only; the
    // rest of the buffer stays zero.
    const int64_t n8 = a.n >> 3;  // whole 16-byte pieces of a row
    uint32_t stage_uses = 0;
    bool gok = true;
    auto stage = [&](int i) {
      const int32_t* tau = a.idx + (int64_t)i * a.eta;
      if (warp == 3) {
        for (int s = lane; s < eta_p; s += 32) {
          int32_t r = 0;
          float iv = 0.f;
          if (s < a.eta) {
            r = __ldg(tau + s);
            iv = __ldg(a.inv_nu + r);
          }
          s_iv[i % 3][s] = iv;
        }
        // this CTA's block of rows of the residual accumulator i % 3 of its
        // right-hand-side slice starts at -b_tau(i) (rows beyond eta: zero);
        // its previous use (iteration i - 3) was read before every CTA passed
        // grid barrier i - 1, and grid barrier i precedes this stage
        // (blocks of four rows of tau; a lane writes the four rows of one
        // right-hand side as one 16-byte piece)
        const int quads = (eta_p / 4 + a.n_slices - 1) / a.n_slices;
        const int q_lo = cs * quads, q_hi = min(eta_p / 4, q_lo + quads);
        float* acc = a.Res + ((int64_t)(i % 3) * a.r_slices + rs) * eta_p * kSliceR;
        const float* bcol = a.Bt + (int64_t)rs * kSliceR;
        for (int x = lane; x < (q_hi - q_lo) * kSliceR; x += 32) {
          const int q = q_lo + x / kSliceR;
          const int r = x % kSliceR;
          float v4[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int s = 4 * q + j;
            v4[j] = (s < a.eta) ? -__ldg(bcol + (int64_t)__ldg(tau + s) * a.R_p + r) : 0.f;
          }
          *reinterpret_cast<float4*>(acc + ((int64_t)q * kSliceR + r) * 4) =
              make_float4(v4[0], v4[1], v4[2], v4[3]);
        }
      } else {
        __nv_bfloat16* G = a.G + (int64_t)(i & 1) * eta_p * a.n_p;
        for (int s = blockIdx.x; s < a.eta; s += nCTA) {
          const int32_t r = __ldg(tau + s);
          const __nv_bfloat16* src = a.A + (int64_t)r * a.lda;
          __nv_bfloat16* dst = G + (int64_t)s * a.n_p;
          for (int64_t v0 = 0; v0 < n8; v0 += kStage / 16) {
            const int64_t left = n8 - v0;
            const uint32_t bytes = (uint32_t)((left < (int64_t)(kStage / 16) ? left : (int64_t)(kStage / 16)) * 16);
            if (lane == 0 && gok) {
              mb_expect_tx(&bars.stage, bytes);
              bulk_load(stagebuf, src + 8 * v0, bytes, &bars.stage);
              gok = wait_phase(&bars.stage, stage_uses & 1u, drain_limit(a.limit_ns), nullptr);
              if (gok) {
                bulk_store(dst + 8 * v0, stagebuf, bytes);
                bulk_commit();
                bulk_wait_read();  // the staging buffer may be refilled
              }
            }
            ++stage_uses;
          }
          // the last n mod 8 columns, one element per lane
          for (int64_t e = n8 * 8 + lane; e < a.n; e += 32) dst[e] = src[e];
        }
        if (lane == 0) bulk_wait_all();  // this CTA's rows written to global memory
      }
      // generic- and async-proxy writes of this thread become visible to the
      // TMA reads that follow the grid barrier
      fence_proxy_async_global();
      __syncwarp();
      if (lane == 0) {
        if (!gok && !s_abort) fail();
        mb_arrive(&bars.gathered);
      }
    };
    stage(0);
    for (int i = 0; i + 1 < cnt; ++i) {
      // buffer (i + 1) % 2, tables (i + 1) % 3 and accumulator (i + 1) % 3
      // are free once grid barrier i has passed (every CTA has finished
      // iteration i - 1): schedule 1 starts the gather then; schedule 0 waits
      // for this CTA's update of iteration i - 1 (which follows that
      // barrier), so the gather runs with iteration i's residual product,
      // while the tensor pipe, not memory, is busy; schedules 2.. wait until
      // chunk kq of iteration i - 1's scaled residual is formed, so the
      // first reads of the reduced residual do not share the memory system
      // with the gather (the epilogue cannot complete the next phase of
      // rchunk before this gather ends: that phase follows grid barrier
      // i + 1, which waits for it)
      int ok = 1;
      if (lane == 0) {
        if (i == 0 || a.gather_sched == 1) {
          ok = wait_phase(&bars.passed, (uint32_t)(i & 1), a.limit_ns, &s_abort);
        } else if (a.gather_sched == 0) {
          ok = wait_phase(&bars.upd_done, (uint32_t)((i - 1) & 1), a.limit_ns, &s_abort);
        } else {
          ok = wait_phase(&bars.passed, (uint32_t)(i & 1), a.limit_ns, &s_abort) &&
               wait_phase(&bars.rchunk, (uint32_t)((i - 1) & 1), a.limit_ns, &s_abort);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      stage(i + 1);
    }
  } else {
    // ------------------------------------------------ epilogue ------------
    const int e = warp - 4;
    const int q = e & 3;          // tensor-memory lane quarter (warp % 4)
    const int half = e >> 2;      // column half
    const int row = 32 * q + lane;  // right-hand side within the slice
    const int64_t rhs = (int64_t)rs * kSliceR + row;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    float* zt = a.Zt + rhs * a.n_p + (int64_t)cs * kSliceN;
    int bad = 0;
    // Z^T of this slice into tensor memory (columns 128 half .. + 127)
    for (int j = 0; j < 4; ++j) {
      float v[32];
      const float4* src = reinterpret_cast<const float4*>(zt + 128 * half + 32 * j);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float4 z4 = src[t];
        v[4 * t] = z4.x;
        v[4 * t + 1] = z4.y;
        v[4 * t + 2] = z4.z;
        v[4 * t + 3] = z4.w;
      }
      tmem_st32(tl + (uint32_t)(128 * half + 32 * j), v);
    }
    tc_fence_before();
    uint32_t u = 0;  // ring uses
    const uint64_t lim = a.limit_ns;
    // grid barrier b: every CTA's reductions, clears and gathers before it
    // are visible to every CTA after it
    auto grid_sync = [&](int b, int need_gather) -> int {
      if (epi_sync_or(bad)) return 0;
      if (tid == 128) {
        int ok = 1;
        if (need_gather && !wait_phase(&bars.gathered, (uint32_t)(b & 1), lim, &s_abort)) ok = 0;
        if (ok) {
          fence_proxy_async_global();
          red_release_u64(a.bar, 1ull);
          const unsigned long long target = (unsigned long long)(b + 1) * (unsigned long long)nCTA;
          const uint64_t t0 = global_timer_ns();
          uint32_t spins = 0;
          while (ld_acquire_u64(a.bar) < target) {
            if (lim == 0 || global_timer_ns() - t0 > lim) {
              ok = 0;
              break;
            }
            if ((++spins & 7u) == 0 && (ld_relaxed_s32(a.status) != kStatusOk || s_abort)) {
              ok = 0;
              break;
            }
          }
        }
        if (!ok && !s_abort) fail();
        if (ok) mb_arrive(&bars.passed);
        s_flag = ok;
      }
      return epi_sync_or(0) ? 0 : s_flag;
    };
    int ok = grid_sync(0, 1);
    for (int i = 0; i < cnt && ok; ++i) {
      // ---- X = S_lambda(Z), split, into the ring: 4 chunks of 64 columns ----
      for (int c = 0; c < 4; ++c) {
        const uint32_t slot = u & 1;
        if (!bad && u >= 2) {
          int w = 1;
          if (lane == 0) w = wait_phase(&bars.empty[slot], ((u >> 1) - 1) & 1, lim, &s_abort);
          bad |= !__shfl_sync(0xffffffffu, w, 0);
        }
        if (!bad) {
          tc_fence_after();
          float v[32];
          tmem_ld32(tl + (uint32_t)(64 * c + 32 * half), v);
#pragma unroll
          for (int t = 0; t < 32; ++t) v[t] = soft_shrink(v[t], a.lambda);
          unsigned char* xs = ring + (size_t)slot * kRingSlot;
          store_split_row(xs, xs + 16384, row, half, v, a.nsplit_x == 2);
          fence_proxy_async_smem();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mb_arrive(&bars.full[slot]);
        }
        ++u;
      }
      // ---- the residual product P^T into the slice's global accumulator ----
      if (!bad) {
        int w = 1;
        if (lane == 0) w = wait_phase(&bars.res_done, (uint32_t)(i & 1), lim, &s_abort);
        bad |= !__shfl_sync(0xffffffffu, w, 0);
      }
      // residual accumulator of this iteration and slice, in blocks of four
      // rows of tau: element (s, r) at ((s / 4) * 128 + r) * 4 + s % 4, so a
      // thread's four consecutive s are one 16-byte piece and a warp's 32
      // right-hand sides one 512-byte run
      float* resb = a.Res + ((int64_t)(i % 3) * a.r_slices + rs) * eta_p * kSliceR + 4 * row;
      // The 32 CTAs of a slice add into the same lines; each starts at the
      // 32-column group given by its column slice, so at any moment about a
      // quarter of them target one line (reductions to one line serialize
      // in L2; the read-back below keeps one order, as reads of a line by
      // many SMs at once are served together).
      if (!bad) {
        tc_fence_after();
        for (int j = 0; j < 4; ++j) {
          const int col = 128 * half + 32 * ((j + cs) & 3);
          if (col >= eta_p) continue;
          float v[32];
          tmem_ld32(tl + kTmemRes + (uint32_t)col, v);
#pragma unroll
          for (int t = 0; t < 8; ++t)
            red_add_v4(resb + ((col >> 2) + t) * (4 * kSliceR), v[4 * t], v[4 * t + 1],
                       v[4 * t + 2], v[4 * t + 3]);
        }
        tc_fence_before();
      }
      // slots s of tau beyond eta carry 1/||a||^2 = 0 (their residual is zero)
      const float* siv = s_iv[i % 3];
      ok = grid_sync(i + 1, (i + 1 < cnt) ? 1 : 0);
      if (!ok) break;
      // ---- scaled residual R' = -(t/eta)(A_tau x - b_tau)/||a_tau||^2, split
      // (the accumulator started at -b_tau); the loads of chunk qq + 1 are in
      // flight while chunk qq is formed ----
      {
        for (int qq = 0; qq < rchunks; ++qq) {
          const uint32_t slot = u & 1;
          const int s0 = 64 * qq + 32 * half;
          float v[32];
          if (!bad) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              const float4 r4 = __ldcg(reinterpret_cast<const float4*>(
                  resb + ((s0 >> 2) + t) * (4 * kSliceR)));
              v[4 * t] = r4.x;
              v[4 * t + 1] = r4.y;
              v[4 * t + 2] = r4.z;
              v[4 * t + 3] = r4.w;
            }
          }
          if (!bad && u >= 2) {
            int w = 1;
            if (lane == 0) w = wait_phase(&bars.empty[slot], ((u >> 1) - 1) & 1, lim, &s_abort);
            bad |= !__shfl_sync(0xffffffffu, w, 0);
          }
          if (!bad) {
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = -a.coef * (v[t] * siv[s0 + t]);
            unsigned char* rsl = ring + (size_t)slot * kRingSlot;
            store_split_row(rsl, rsl + 16384, row, half, v, a.nsplit_r == 2);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              mb_arrive(&bars.full[slot]);
              if (qq == kq) mb_arrive(&bars.rchunk);
            }
          }
          ++u;
        }
      }
      // ---- Z^T += D^T (FP32, rounded once per iteration) ----
      if (!bad) {
        int w = 1;
        if (lane == 0) w = wait_phase(&bars.upd_done, (uint32_t)(i & 1), lim, &s_abort);
        bad |= !__shfl_sync(0xffffffffu, w, 0);
      }
      if (!bad) {
        tc_fence_after();
        // the columns this warp reads again for the next X (64 j + 32 half),
        // so no other warp's tensor-memory writes are involved
        for (int j = 0; j < 4; ++j) {
          const uint32_t col = (uint32_t)(64 * j + 32 * half);
          float z[32], d[32];
          tmem_ld32(tl + col, z);
          tmem_ld32(tl + kTmemRes + col, d);
#pragma unroll
          for (int t = 0; t < 32; ++t) z[t] += d[t];
          tmem_st32(tl + col, z);
        }
        tc_fence_before();
      }
      if (bad && !s_abort) fail();
    }
    if (epi_sync_or(bad)) ok = 0;
    if (ok) {
      // Z^T of this slice back to global memory for the next launch
      tc_fence_after();
      for (int j = 0; j < 4; ++j) {
        float v[32];
        tmem_ld32(tl + (uint32_t)(128 * half + 32 * j), v);
        float4* dst = reinterpret_cast<float4*>(zt + 128 * half + 32 * j);
#pragma unroll
        for (int t = 0; t < 8; ++t)
          dst[t] = make_float4(v[4 * t], v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
      }
    } else if (tid == 128 && !s_abort) {
      fail();
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

size_t mrhs_tmem_smem(int eta_p) {
  return 4u * (size_t)eta_p * 128u + 2u * kRingSlot + kStage + 1024u;
}

bool mrhs_tmem_fits(int64_t n_p, int64_t R_p, int64_t eta_p, int num_sms) {
  return eta_p >= 64 && eta_p <= 256 && (eta_p % 64) == 0 && (n_p % kSliceN) == 0 &&
         (R_p % kSliceR) == 0 && (n_p / kSliceN) * (R_p / kSliceR) <= num_sms;
}

cudaError_t launch_mrhs_tmem(const CUtensorMap& mapG, const MrhsTmemArgs& a, cudaStream_t s) {
  const size_t smem = mrhs_tmem_smem(a.eta_p);
  cudaFuncAttributes fa = {};
  cudaError_t e = cudaFuncGetAttributes(&fa, mrhs_tmem_kernel);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(mrhs_tmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_slices * a.r_slices));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the grid barrier needs it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mrhs_tmem_kernel, mapG, a);
}

}  // namespace rska
