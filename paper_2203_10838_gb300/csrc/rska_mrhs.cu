// rska_mrhs.cu -- shared-A multi-right-hand-side RSKA on the tensor cores.
//
// R systems A x_j = b_j share A (stored in BF16) and one index stream tau_k.
// With X = [x_1 .. x_R] = S_lambda(Z), one RSKA step (eq. rska, Algorithm 1
// with w_i = t, applied to every column at once) is two dense contractions:
//
//   Res  = A_tau X - B_tau                    (eta x R,  contraction over n)
//   Z   -= (t/eta) A_tau^T D_tau^-2 Res       (n x R,    contraction over eta)
//
// (the matrix form A^T M_k (A x - b) of the update, Sec. 3).  Both run as
// tcgen05 MMAs with BF16 operands and FP32 accumulation in tensor memory.
// Every operand is K-major: Z, X and B are held per right-hand side (row j of
// Z^T is z_j), tau's rows are gathered each iteration into A_tau (eta x n) and
// its transpose A_tau^T (n x eta), and the scaled residual is written
// transposed (R x eta).  The operand that is not exact in BF16 (X in the
// first product, the scaled residual in the second) is split into a BF16 high
// part and a BF16 low part (v = hi + lo + O(2^-17 |v|)); both parts are
// multiplied and accumulated into the same tensor-memory tile.
//
// Per iteration: gather -> residual GEMM (split over n, partial tiles added
// into Res by TMA bulk reduce-add) -> scale (Res - B_tau, times t/(eta nu_i),
// transposed, split, Res cleared) -> update GEMM (epilogue through shared
// memory and TMA: z -= d, x = S_lambda(z), x split into hi/lo for the next
// residual GEMM).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "rska_device.cuh"
#include "rska_internal.h"
#include "rska_mrhs_tmem.h"
#include "rska_tc.cuh"
#include "rska_tune.h"

namespace rska {
namespace {

constexpr int TM = 128;             // tile rows (tensor-memory lanes)
constexpr int TN = 256;             // tile columns (tensor-memory columns, FP32)
constexpr int TK = 64;              // k-block: one 128-byte swizzle atom of BF16
constexpr int GEMM_THREADS = 256;   // warp 0: TMA, warp 1: MMA, all 8 warps: epilogue
constexpr int GEMM_STAGES = 2;
constexpr uint32_t TILE_A_BYTES = TM * TK * 2;   // 16 KB
constexpr uint32_t TILE_B_BYTES = TN * TK * 2;   // 32 KB
constexpr size_t ZREG0 = 131072;                  // update: first half of the z tile (64 KB)

enum GemmMode { kResidual = 0, kUpdate = 1 };

using namespace tc;

// Instruction descriptor for kind::f16: D FP32, A and B BF16, both K-major,
// M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

struct GemmArgs {
  int nsplit;          // 1: the inexact operand as one BF16 term, 2: hi + lo
  int kb_total;        // k-blocks (of TK) in the contraction
  int kb_per_cta;      // k-blocks per CTA along grid.z (residual GEMM: split over n)
  float* out;          // residual GEMM: Res, rows of ld_out floats (added atomically)
  int64_t ld_out;
  float* zt;           // update GEMM: Z^T, X_hi^T, X_lo^T, rows of ldz
  __nv_bfloat16* xhi;
  __nv_bfloat16* xlo;
  int64_t ldz;
  float lambda;
  int* status;
  uint64_t limit_ns;
};

// One 128 x 256 output tile per CTA, D = sum_k A[m][k] B[n][k] over this CTA's
// k-blocks, accumulated in tensor memory.  kResidual: A = A_tau (mapA0), B =
// X^T hi (mapB0) and lo (mapB1); D is added into Res.  kUpdate: A = scaled
// residual^T hi (mapA0) and lo (mapA1), B = A_tau^T (mapB0); Z^T -= D, then
// x = S_lambda(z) split into X_hi^T / X_lo^T.
template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    mrhs_gemm_kernel(const __grid_constant__ CUtensorMap mapA0,
                     const __grid_constant__ CUtensorMap mapA1,
                     const __grid_constant__ CUtensorMap mapB0,
                     const __grid_constant__ CUtensorMap mapB1,
                     const __grid_constant__ CUtensorMap mapE0,
                     const __grid_constant__ CUtensorMap mapE1,
                     const __grid_constant__ CUtensorMap mapE2, GemmArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[GEMM_STAGES];
  __shared__ __align__(8) uint64_t empty[GEMM_STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ __align__(8) uint64_t zbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_issued, s_consumed;

  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool splitA = (MODE == kUpdate) && a.nsplit == 2;
  const bool splitB = (MODE == kResidual) && a.nsplit == 2;
  const uint32_t a_bytes = TILE_A_BYTES * (splitA ? 2u : 1u);
  const uint32_t b_bytes = TILE_B_BYTES * (splitB ? 2u : 1u);
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int m0 = blockIdx.x * TM;
  const int n0 = blockIdx.y * TN;
  const int kb0 = blockIdx.z * a.kb_per_cta;
  const int nkb = max(0, min(a.kb_total, kb0 + a.kb_per_cta) - kb0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < GEMM_STAGES; ++i) {
      mb_init(&full[i], 1);
      mb_init(&empty[i], 1);
    }
    mb_init(&done, 1);
    mb_init(&zbar[0], 1);
    mb_init(&zbar[1], 1);
    s_err = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&s_tmem)),
                 "r"((uint32_t)TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  // everything above touches only this CTA's own resources; with a
  // programmatic launch it overlaps the previous kernel's tail.  From here on
  // this kernel reads what earlier kernels wrote.
  pdl_wait();
  if (threadIdx.x == 0) pdl_launch_dependents();
  if (MODE == kUpdate && threadIdx.x == 64 && nkb > 0) {
    // the update's z tile does not depend on the products: its first half
    // goes to its own shared-memory region now, the second half to L2
    mb_expect_tx(&zbar[0], 65536u);
    for (int b = 0; b < 4; ++b)
      tma_load_2d(smem + ZREG0 + (size_t)b * 16384, &mapE0, n0 + 32 * b, m0, &zbar[0]);
    for (int b = 4; b < TN / 32; ++b) tma_prefetch_2d(&mapE0, n0 + 32 * b, m0);
  }
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int it = 0;
    for (; it < nkb; ++it) {
      const int st = it % GEMM_STAGES;
      const int use = it / GEMM_STAGES;
      if (use > 0 && !mb_wait(&empty[st], (uint32_t)((use - 1) & 1), a.limit_ns)) {
        s_err = 1;
        break;
      }
      unsigned char* base = smem + (size_t)st * stage_bytes;
      const int k = (kb0 + it) * TK;
      mb_expect_tx(&full[st], stage_bytes);
      tma_load_2d(base, &mapA0, k, m0, &full[st]);
      if (splitA) tma_load_2d(base + TILE_A_BYTES, &mapA1, k, m0, &full[st]);
      tma_load_2d(base + a_bytes, &mapB0, k, n0, &full[st]);
      if (splitB) tma_load_2d(base + a_bytes + TILE_B_BYTES, &mapB1, k, n0, &full[st]);
    }
    s_issued = it;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int it = 0;
    for (; it < nkb; ++it) {
      const int st = it % GEMM_STAGES;
      if (!mb_wait(&full[st], (uint32_t)((it / GEMM_STAGES) & 1), a.limit_ns)) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t abase = saddr(smem + (size_t)st * stage_bytes);
      const uint32_t bbase = abase + a_bytes;
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        // advancing K by 16 BF16 = 32 bytes inside the swizzle atom
        const uint64_t da = desc_sw128(abase) + (uint64_t)(2 * kk);
        const uint64_t db = desc_sw128(bbase) + (uint64_t)(2 * kk);
        mma_bf16(tmem, da, db, kIdesc, (it > 0 || kk > 0) ? 1u : 0u);
        if (splitA) mma_bf16(tmem, desc_sw128(abase + TILE_A_BYTES) + (uint64_t)(2 * kk), db, kIdesc, 1u);
        if (splitB) mma_bf16(tmem, da, desc_sw128(bbase + TILE_B_BYTES) + (uint64_t)(2 * kk), kIdesc, 1u);
      }
      mma_commit(&empty[st]);
    }
    s_consumed = it;
    mma_commit(&done);
  }

  // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile
  // row 32 (w % 4) + lane) for its column chunks; tiles go through the (now
  // free) stage buffers in TMA's 128-byte-swizzled layout ----
  const int quarter = warp & 3;
  const int half = warp >> 2;
  const int r = quarter * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
  if (!mb_wait(&done, 0u, a.limit_ns)) s_err = 1;
  tc_fence_after();
  __syncthreads();
  const bool ok = (s_err == 0) && nkb > 0;
  unsigned char* epi = smem;
  if (MODE == kResidual) {
    // 8 boxes of 128 rows x 32 FP32 columns, added into Res by TMA reduce-add
    if (ok) {
#pragma unroll 1
      for (int c = half * 4; c < half * 4 + 4; ++c) {
        float v[32];
        tmem_ld32(trow + (uint32_t)(c * 32), v);
        unsigned char* box = epi + (size_t)c * 16384;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<float4*>(box + sw128_off(r, j)) =
              make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
      for (int c = 0; c < TN / 32; ++c) tma_reduce_add_2d(&mapE0, epi + (size_t)c * 16384, n0 + 32 * c, m0);
      bulk_commit();
      bulk_wait_read();  // the grid's completion orders the global writes
    }
  } else {
    // four quarters of 64 columns.  The z boxes of quarters 0 and 1 (FP32,
    // 32 columns x 128 rows = 16 KB each) were loaded at kernel start into
    // ZREG0; those of quarters 2 and 3 go into the freed stage buffers
    // [0, 64 KB).  Each quarter updates its z in place and splits
    // x = S_lambda(z) into one BF16 hi and one BF16 lo box (16 KB each) staged
    // in buffer q % 2 of [64 KB, 128 KB); its TMA stores then drain while the
    // next quarter computes, and a buffer is reused only after the stores of
    // two quarters back have read it.
    unsigned char* xreg = epi + 65536;
    if (threadIdx.x == 0 && ok) {
      mb_expect_tx(&zbar[1], 65536u);
      for (int b = 0; b < 4; ++b)
        tma_load_2d(epi + (size_t)b * 16384, &mapE0, n0 + 128 + 32 * b, m0, &zbar[1]);
    }
#pragma unroll 1
    for (int q = 0; q < 4 && ok; ++q) {
      if (q >= 2) {
        if (threadIdx.x == 0) bulk_wait_read_all_but_one();  // quarter q - 2 has read buffer q % 2
        __syncthreads();
      }
      const int cbase = n0 + 64 * q;
      unsigned char* zq = (q < 2) ? smem + ZREG0 + (size_t)q * 32768 : epi + (size_t)(q - 2) * 32768;
      unsigned char* xq = xreg + (size_t)(q & 1) * 32768;
      const bool zok = mb_wait(&zbar[q >> 1], 0u, a.limit_ns);
      {
        const int c = half;  // this warp's 32-column chunk of the quarter
        float v[32];
        tmem_ld32(trow + (uint32_t)(64 * q + 32 * c), v);
        unsigned char* zb = zq + (size_t)c * 16384;
        uint32_t hw[16], lw[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4* zp = reinterpret_cast<float4*>(zb + sw128_off(r, j));
          float4 z = *zp;
          z.x -= v[4 * j];
          z.y -= v[4 * j + 1];
          z.z -= v[4 * j + 2];
          z.w -= v[4 * j + 3];
          *zp = z;
          __nv_bfloat16 h[4], l[4];
          split_bf16(soft_shrink(z.x, a.lambda), &h[0], &l[0]);
          split_bf16(soft_shrink(z.y, a.lambda), &h[1], &l[1]);
          split_bf16(soft_shrink(z.z, a.lambda), &h[2], &l[2]);
          split_bf16(soft_shrink(z.w, a.lambda), &h[3], &l[3]);
          hw[2 * j] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
          hw[2 * j + 1] = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
          lw[2 * j] = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
          lw[2 * j + 1] = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
        }
        // 32 BF16 = 4 chunks of 16 bytes at chunks 4 c .. 4 c + 3 of the
        // quarter's 64-column box
        unsigned char* hb = xq;
        unsigned char* lb = xq + 16384;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const uint32_t off = sw128_off(r, 4 * c + qq);
          *reinterpret_cast<uint4*>(hb + off) = make_uint4(hw[4 * qq], hw[4 * qq + 1], hw[4 * qq + 2], hw[4 * qq + 3]);
          *reinterpret_cast<uint4*>(lb + off) = make_uint4(lw[4 * qq], lw[4 * qq + 1], lw[4 * qq + 2], lw[4 * qq + 3]);
        }
      }
      if (!zok) s_err = 1;
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0 && s_err == 0) {
        for (int b = 0; b < 2; ++b) tma_store_2d(&mapE0, zq + (size_t)b * 16384, cbase + 32 * b, m0);
        tma_store_2d(&mapE1, xq, cbase, m0);
        tma_store_2d(&mapE2, xq + 16384, cbase, m0);
        bulk_commit();
      }
    }
    // every store has read its shared-memory source before the CTA ends
    if (threadIdx.x == 0 && ok) bulk_wait_read();
    __syncthreads();
  }
  if (threadIdx.x == 0 && (!ok || s_err) && nkb > 0) atomicCAS(a.status, kStatusOk, kStatusTimeout);
  // let every issued copy land and every issued MMA finish before the shared
  // and tensor memory go away (drain limit: these always complete, however
  // short the watchdog limit of the waits above)
  const uint64_t dl = drain_limit(a.limit_ns);
  if (MODE == kUpdate && threadIdx.x == 64 && nkb > 0) mb_wait(&zbar[0], 0u, dl);
  if (threadIdx.x == 0) {
    if (MODE == kUpdate && ok) mb_wait(&zbar[1], 0u, dl);
    for (int it = s_consumed; it < s_issued; ++it)
      mb_wait(&full[it % GEMM_STAGES], (uint32_t)((it / GEMM_STAGES) & 1), dl);
    mb_wait(&done, 0u, dl);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TN)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Setup and per-iteration helper kernels.
// ---------------------------------------------------------------------------

// ||a_i||^2 in FP64 from the BF16 values, in the same canonical order as the
// FP32 setup (lane L sums j = L mod 32 ascending with exact squares, then the
// 32 partials are folded with xor offsets 16, 8, 4, 2, 1).
__global__ void mrhs_row_norms_kernel(const __nv_bfloat16* __restrict__ A, int64_t m, int64_t n,
                                      int64_t lda, double* __restrict__ nu,
                                      float* __restrict__ inv_nu, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const __nv_bfloat16* row = A + i * lda;
    double p = 0.0;
    bool finite = true;
    for (int64_t j = lane; j < n; j += 32) {
      const float a = __bfloat162float(row[j]);
      finite = finite && isfinite(a);
      const double ad = (double)a;
      p = __fma_rn(ad, ad, p);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) p = __dadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      if (!finite || !isfinite(p))
        atomicCAS(status, kStatusOk, kStatusNonFinite);
      else if (p == 0.0)
        atomicCAS(status, kStatusOk, kStatusZeroRow);
      nu[i] = p;
      inv_nu[i] = (p > 0.0) ? (float)__ddiv_rn(1.0, p) : 0.0f;
    }
  }
}

// Bt[i][j] = B[j][i] (B: R rows of ldb, one right-hand side per row; Bt: m
// rows of ldbt); columns j >= R of Bt are zero.  Flags non-finite entries.
__global__ void mrhs_transpose_b_kernel(const float* __restrict__ B, int64_t R, int64_t m,
                                        int64_t ldb, float* __restrict__ Bt, int64_t ldbt,
                                        int* status) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;  // equation
  const int64_t j0 = (int64_t)blockIdx.y * 32;  // right-hand side
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  bool bad = false;
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + tx;
    float v = 0.f;
    if (j < R && i < m) {
      v = B[j * ldb + i];
      bad = bad || !isfinite(v);
    }
    tile[r][tx] = v;
  }
  if (bad) atomicCAS(status, kStatusOk, kStatusNonFinite);
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + tx;
    if (i < m && j < ldbt) Bt[i * ldbt + j] = tile[tx][r];
  }
}

// A_tau[s][i] = A[tau_s][i] and A_tau^T[i][s] for one 64 x 64 tile;
// s >= eta or i >= n give zeros.  256 threads.
__global__ void mrhs_gather_kernel(const __nv_bfloat16* __restrict__ A, int64_t n, int64_t lda,
                                   const int32_t* __restrict__ tau, int32_t eta,
                                   __nv_bfloat16* __restrict__ Atau, int64_t ld_atau,
                                   __nv_bfloat16* __restrict__ AtauT, int64_t ld_atauT) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int64_t s0 = (int64_t)blockIdx.x * 64;
  const int64_t i0 = (int64_t)blockIdx.y * 64;
  const int t = threadIdx.x;
#pragma unroll
  for (int rep = 0; rep < 2; ++rep) {
    const int e = t + 256 * rep;
    const int r = e >> 3, c8 = e & 7;
    const int64_t s = s0 + r, i = i0 + 8 * c8;
    union {
      uint4 u;
      __nv_bfloat16 h[8];
    } v;
    v.u = make_uint4(0u, 0u, 0u, 0u);
    if (s < eta) {
      const __nv_bfloat16* src = A + (int64_t)__ldg(tau + s) * lda + i;
      if (i + 8 <= n) {
        v.u = __ldg(reinterpret_cast<const uint4*>(src));
      } else {
        for (int q = 0; q < 8; ++q)
          if (i + q < n) v.h[q] = src[q];
      }
    }
    *reinterpret_cast<uint4*>(Atau + s * ld_atau + i) = v.u;
#pragma unroll
    for (int q = 0; q < 8; ++q) tile[r][8 * c8 + q] = v.h[q];
  }
  __syncthreads();
#pragma unroll
  for (int rep = 0; rep < 2; ++rep) {
    const int e = t + 256 * rep;
    const int r = e >> 3, c8 = e & 7;  // r: column i0 + r, c8: rows s0 + 8 c8 ..
    union {
      uint4 u;
      __nv_bfloat16 h[8];
    } v;
#pragma unroll
    for (int q = 0; q < 8; ++q) v.h[q] = tile[8 * c8 + q][r];
    *reinterpret_cast<uint4*>(AtauT + (i0 + r) * ld_atauT + s0 + 8 * c8) = v.u;
  }
}

// Scaled residual, transposed and split: for s < eta, j < R
//   v = (t/eta) (Res[s][j] - b_j[tau_s]) / ||a_{tau_s}||^2,  Rt{hi,lo}[j][s] = split(v)
// and zeros elsewhere; Res is cleared for the next residual GEMM.  32 x 8 threads
// per 32 x 32 tile.
__global__ void mrhs_scale_kernel(float* __restrict__ Res, int64_t ld_res,
                                  const float* __restrict__ Bt, int64_t ldbt,
                                  const float* __restrict__ inv_nu, const int32_t* __restrict__ tau,
                                  int32_t eta, int64_t R, float coef,
                                  __nv_bfloat16* __restrict__ Rhi, __nv_bfloat16* __restrict__ Rlo,
                                  int64_t ld_rt) {
  __shared__ float tile[32][33];
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int64_t j0 = (int64_t)blockIdx.y * 32;
  pdl_wait();
  if (threadIdx.x == 0 && threadIdx.y == 0) pdl_launch_dependents();
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int64_t s = s0 + r, j = j0 + tx;
    float* rp = Res + s * ld_res + j;
    float v = 0.f;
    if (s < eta && j < R) {
      const int32_t row = __ldg(tau + s);
      v = coef * ((*rp - __ldg(Bt + (int64_t)row * ldbt + j)) * __ldg(inv_nu + row));
    }
    *rp = 0.f;
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t j = j0 + r, s = s0 + tx;
    __nv_bfloat16 h, l;
    split_bf16(tile[tx][r], &h, &l);
    Rhi[j * ld_rt + s] = h;
    Rlo[j * ld_rt + s] = l;
  }
}

}  // namespace
}  // namespace rska

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
using rska::GemmArgs;

struct rska_mrhs {
  const __nv_bfloat16* A = nullptr;
  int64_t m = 0, n = 0, lda = 0, R = 0;
  float lambda = 0.f, t = 1.f;
  int32_t eta = 1;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t n_p = 0, eta_p = 0, R_p = 0;
  // owned device memory
  double* nu = nullptr;
  float* inv_nu = nullptr;
  uint32_t* thr = nullptr;
  int32_t* alias = nullptr;
  float* Bt = nullptr;               // m x R_p
  __nv_bfloat16* Atau[2] = {nullptr, nullptr};    // eta_p x n_p, double-buffered
  __nv_bfloat16* AtauT[2] = {nullptr, nullptr};   // n_p x eta_p
  __nv_bfloat16* Xhi = nullptr;      // R_p x n_p
  __nv_bfloat16* Xlo = nullptr;
  __nv_bfloat16* Rhi = nullptr;      // R_p x eta_p
  __nv_bfloat16* Rlo = nullptr;
  float* Zt = nullptr;               // R_p x n_p
  float* Res = nullptr;              // eta_p x R_p
  int32_t* idx = nullptr;            // tau for up to idx_cap iterations
  int64_t idx_cap = 0;
  int* status = nullptr;
  CUtensorMap mapAtau[2], mapX[2], mapR[2], mapAtauT[2];
  CUtensorMap mapRes, mapZ, mapXs[2];  // epilogue boxes: Res and Z (FP32), X hi/lo (BF16)
  // the gather of iteration k+1 runs on `side` while iteration k computes
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_gathered[2] = {nullptr, nullptr},
              ev_used[2] = {nullptr, nullptr};
  // options and state
  int nsplit = 2;
  int ksplit = 0;                    // residual GEMM CTAs along n (0: automatic)
  int use_graph = 1;
  int use_pdl = 1;                   // programmatic dependent launches on the main stream
  int64_t k_host = 0;
  int sticky = RSKA_OK;
  uint64_t limit_ns = 2000000000ull;
  cudaGraphExec_t graph = nullptr;   // one chunk of idx_cap iterations
  int graph_nsplit = -1, graph_ksplit = -1, graph_pdl = -1;
  uint64_t graph_limit_ns = 0;       // the wait limit baked into the graph's kernel arguments
  // persistent form (rska_mrhs_tmem.cu): Z^T in tensor memory for a launch
  int form_opt = 0;                  // 0 automatic, 1 staged kernels, 2 persistent
  int form = 1;                      // form of the next solve
  int nsplit_r = 0;                  // terms of the scaled residual (0: as nsplit)
  bool x_stale = false;              // X hi/lo (staged form state) lag behind Z
  int64_t eta_p64 = 0;               // eta rounded up to 64
  __nv_bfloat16* G = nullptr;        // 2 x eta_p64 x n_p dense A_tau copies
  float* Res3 = nullptr;             // 3 x R_p x eta_p64 residual accumulators
  unsigned long long* pbar = nullptr;
  int32_t* pidx = nullptr;           // tau of one persistent launch
  int64_t pidx_cap = 0;
  int gather_sched = 2;              // persistent form: gather with the residual product (0),
                                     // right after the grid barrier (1), or once chunk k of the
                                     // scaled residual is formed (2 + k); 2 is the fastest on the
                                     // 16384 x 8192, R = 512, eta = 256 problem
  // autotuner: the schedule in use comes from it while the options that
  // choose a schedule (1, 4, 5, 7) are left automatic
  bool pinned = false;               // a schedule option was set explicitly
  bool tuned = false;
  int32_t tuned_code = 0;
  double tuned_us = 0.0;
  CUtensorMap mapG;
};

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Row-major matrix (rows x cols, ld elements per row) in boxes of 128-byte
// rows (64 BF16 or 32 FP32 columns, 128-byte swizzle) by box_rows rows.
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_rows, bool fp32 = false) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const uint64_t esize = fp32 ? 4 : 2;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * esize};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t v, int64_t k) { return (v + k - 1) / k * k; }

void mrhs_free(rska_mrhs* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  cudaEvent_t evs[] = {h->ev_fork, h->ev_gathered[0], h->ev_gathered[1], h->ev_used[0],
                       h->ev_used[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  void* ptrs[] = {h->nu,       h->inv_nu,   h->thr, h->alias, h->Bt,  h->Atau[0], h->Atau[1],
                  h->AtauT[0], h->AtauT[1], h->Xhi, h->Xlo,   h->Rhi, h->Rlo,     h->Zt,
                  h->Res,      h->idx,      h->status, h->G,  h->Res3, h->pbar,   h->pidx};
  for (void* p : ptrs) cudaFree(p);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

size_t gemm_smem(int mode, int nsplit) {
  const size_t a = rska::TILE_A_BYTES * ((mode == rska::kUpdate && nsplit == 2) ? 2 : 1);
  const size_t b = rska::TILE_B_BYTES * ((mode == rska::kResidual && nsplit == 2) ? 2 : 1);
  // the epilogue reuses the stage buffers for 128 KB of output boxes; the
  // update also keeps the first half of its z tile in 64 KB of its own
  return std::max<size_t>(rska::GEMM_STAGES * (a + b), 131072) + (mode == rska::kUpdate ? 65536 : 0) +
         1024;
}

int residual_splits(const rska_mrhs* h, int* kb_per) {
  const int kb_total = (int)(h->n_p / rska::TK);
  const int tiles = (int)((h->eta_p / rska::TM) * (h->R_p / rska::TN));
  int S = h->ksplit > 0 ? h->ksplit : std::max(1, h->num_sms / std::max(1, tiles));
  S = std::min(S, kb_total);
  *kb_per = (kb_total + S - 1) / S;
  return (kb_total + *kb_per - 1) / *kb_per;
}

// The launches of iterations [0, cnt) of the current tau chunk on stream s.
// Iteration k uses A_tau buffer k % 2; its gather runs on the side stream as
// soon as iteration k-2 (the buffer's previous user) is done, overlapping
// iteration k-1's products.
cudaError_t enqueue_iterations(rska_mrhs* h, int64_t cnt, cudaStream_t s) {
  int kb_per = 1;
  const int S = residual_splits(h, &kb_per);
  GemmArgs g1;
  std::memset(&g1, 0, sizeof(g1));
  g1.nsplit = h->nsplit;
  g1.kb_total = (int)(h->n_p / rska::TK);
  g1.kb_per_cta = kb_per;
  g1.out = h->Res;
  g1.ld_out = h->R_p;
  g1.status = h->status;
  g1.limit_ns = h->limit_ns;
  GemmArgs g2 = g1;
  g2.kb_total = (int)(h->eta_p / rska::TK);
  g2.kb_per_cta = g2.kb_total;
  g2.out = nullptr;
  g2.zt = h->Zt;
  g2.xhi = h->Xhi;
  g2.xlo = h->Xlo;
  g2.ldz = h->n_p;
  g2.lambda = h->lambda;
  const size_t sm1 = gemm_smem(rska::kResidual, h->nsplit);
  const size_t sm2 = gemm_smem(rska::kUpdate, h->nsplit);
  const dim3 ggrid((unsigned)(h->eta_p / 64), (unsigned)(h->n_p / 64));
  const dim3 grid1((unsigned)(h->eta_p / rska::TM), (unsigned)(h->R_p / rska::TN), (unsigned)S);
  const dim3 sgrid((unsigned)(h->eta_p / 32), (unsigned)(h->R_p / 32));
  const dim3 grid2((unsigned)(h->R_p / rska::TM), (unsigned)(h->n_p / rska::TN), 1);
  const float coef = h->t / (float)h->eta;
  cudaStream_t side = h->side;
  // launch on s, as a programmatic dependent of the previous kernel when asked
  auto launch = [&](auto kernel, dim3 grid, dim3 block, size_t smem, bool programmatic,
                    auto... args) -> cudaError_t {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (programmatic && h->use_pdl) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
  };
  auto gather = [&](int64_t k) -> cudaError_t {
    const int b = (int)(k & 1);
    if (k >= 2) {
      cudaError_t e = cudaStreamWaitEvent(side, h->ev_used[b], 0);
      if (e != cudaSuccess) return e;
    }
    rska::mrhs_gather_kernel<<<ggrid, 256, 0, side>>>(h->A, h->n, h->lda, h->idx + k * h->eta,
                                                      h->eta, h->Atau[b], h->n_p, h->AtauT[b],
                                                      h->eta_p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_gathered[b], side);
    return e;
  };
  cudaError_t e = cudaEventRecord(h->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, h->ev_fork, 0);
  if (e == cudaSuccess && cnt > 0) e = gather(0);
  for (int64_t k = 0; k < cnt && e == cudaSuccess; ++k) {
    const int b = (int)(k & 1);
    const int32_t* tau = h->idx + k * h->eta;
    e = cudaStreamWaitEvent(s, h->ev_gathered[b], 0);
    if (e != cudaSuccess) break;
    // the first kernel after the event wait keeps an ordinary dependency
    e = launch(rska::mrhs_gemm_kernel<rska::kResidual>, grid1, dim3(rska::GEMM_THREADS), sm1,
               k > 0, h->mapAtau[b], h->mapAtau[b], h->mapX[0], h->mapX[1], h->mapRes, h->mapRes,
               h->mapRes, g1);
    if (e != cudaSuccess) break;
    if (k + 1 < cnt && (e = gather(k + 1)) != cudaSuccess) break;
    e = launch(rska::mrhs_scale_kernel, sgrid, dim3(32, 8), 0, true, h->Res, h->R_p, h->Bt,
               h->R_p, h->inv_nu, tau, h->eta, h->R, coef, h->Rhi, h->Rlo, h->eta_p);
    if (e != cudaSuccess) break;
    e = launch(rska::mrhs_gemm_kernel<rska::kUpdate>, grid2, dim3(rska::GEMM_THREADS), sm2, true,
               h->mapR[0], h->mapR[1], h->mapAtauT[b], h->mapAtauT[b], h->mapZ, h->mapXs[0],
               h->mapXs[1], g2);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_used[b], s);
  }
  return e;
}

__global__ void mrhs_out_kernel(const float* __restrict__ Zt, int64_t ldz, int64_t R, int64_t n,
                                float lambda, float* __restrict__ x, float* __restrict__ z) {
  const int64_t total = R * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const float v = Zt[j * ldz + i];
    if (z) z[e] = v;
    if (x) x[e] = rska::soft_shrink(v, lambda);
  }
}

// X hi/lo of the staged form from Z^T (after persistent launches, which keep
// no X in global memory): x = S_lambda(z) split into BF16 high and low parts.
__global__ void mrhs_x_from_z_kernel(const float* __restrict__ Zt, int64_t total, float lambda,
                                     __nv_bfloat16* __restrict__ xhi,
                                     __nv_bfloat16* __restrict__ xlo) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    __nv_bfloat16 hv, lv;
    rska::tc::split_bf16(rska::soft_shrink(Zt[e], lambda), &hv, &lv);
    xhi[e] = hv;
    xlo[e] = lv;
  }
}

// K iterations with the staged kernels (gather, residual product, scale,
// update product per iteration; 64-iteration chunks replayed as a graph).
cudaError_t solve_staged(rska_mrhs* h, int64_t K) {
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  if (h->x_stale && K > 0) {
    // the persistent form kept X in tensor memory only
    const int64_t total = h->R_p * h->n_p;
    mrhs_x_from_z_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(
        h->Zt, total, h->lambda, h->Xhi, h->Xlo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    h->x_stale = false;
  }
  for (int64_t done = 0; done < K && e == cudaSuccess;) {
    const int64_t cnt = std::min(h->idx_cap, K - done);
    e = rska::launch_indices(h->thr, h->alias, h->m, h->seed, 0, h->k_host + done, cnt, h->eta,
                             h->idx, s);
    if (e != cudaSuccess) break;
    if (cnt == h->idx_cap && h->use_graph) {
      if (!h->graph || h->graph_nsplit != h->nsplit || h->graph_ksplit != h->ksplit ||
          h->graph_pdl != h->use_pdl || h->graph_limit_ns != h->limit_ns) {
        if (h->graph) {
          cudaGraphExecDestroy(h->graph);
          h->graph = nullptr;
        }
        cudaStream_t cap = nullptr;
        cudaGraph_t g = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const cudaError_t e1 = enqueue_iterations(h, cnt, cap);
          e = cudaStreamEndCapture(cap, &g);
          if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) break;
        h->graph_nsplit = h->nsplit;
        h->graph_ksplit = h->ksplit;
        h->graph_pdl = h->use_pdl;
        h->graph_limit_ns = h->limit_ns;
      }
      e = cudaGraphLaunch(h->graph, s);
    } else {
      e = enqueue_iterations(h, cnt, s);
    }
    done += cnt;
  }
  return e;
}

// K iterations with the persistent kernel: per launch of up to pidx_cap
// iterations, the indices are drawn, the residual accumulators and the
// barrier counter cleared, and Z^T stays in tensor memory for the launch.
cudaError_t solve_tmem(rska_mrhs* h, int64_t K) {
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  rska::MrhsTmemArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = h->A;
  a.lda = h->lda;
  a.n = h->n;
  a.n_p = h->n_p;
  a.R_p = h->R_p;
  a.eta = h->eta;
  a.eta_p = (int32_t)h->eta_p64;
  a.n_slices = (int32_t)(h->n_p / 256);
  a.r_slices = (int32_t)(h->R_p / 128);
  a.idx = h->pidx;
  a.inv_nu = h->inv_nu;
  a.Bt = h->Bt;
  a.G = h->G;
  a.Zt = h->Zt;
  a.Res = h->Res3;
  a.bar = h->pbar;
  a.lambda = h->lambda;
  a.coef = h->t / (float)h->eta;
  a.nsplit_x = h->nsplit;
  a.nsplit_r = h->nsplit_r > 0 ? h->nsplit_r : h->nsplit;
  a.status = h->status;
  a.limit_ns = h->limit_ns;
  a.gather_sched = h->gather_sched;
  for (int64_t done = 0; done < K && e == cudaSuccess;) {
    const int64_t cnt = std::min(h->pidx_cap, K - done);
    e = rska::launch_indices(h->thr, h->alias, h->m, h->seed, 0, h->k_host + done, cnt, h->eta,
                             h->pidx, s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(h->Res3, 0, sizeof(float) * 3 * (size_t)h->R_p * h->eta_p64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->pbar, 0, sizeof(unsigned long long), s);
    a.cnt = (int32_t)cnt;
    if (e == cudaSuccess) e = rska::launch_mrhs_tmem(h->mapG, a, s);
    done += cnt;
  }
  if (K > 0) h->x_stale = true;
  return e;
}

int fail(rska_mrhs* h, cudaError_t e);

// solves of at least this many iterations choose the schedule automatically
constexpr int64_t kAutoTuneMinIters = 128;

// The autotuner's key: problem shape, precision options and device.
std::string tune_key(const rska_mrhs* h) {
  int dev = 0;
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    std::snprintf(prop.name, sizeof(prop.name), "unknown");
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  char buf[400];
  std::snprintf(buf, sizeof(buf), "mrhs:m=%lld:n=%lld:R=%lld:eta=%d:terms=%d/%d:%s:sms=%d",
                (long long)h->m, (long long)h->n, (long long)h->R, (int)h->eta, h->nsplit,
                h->nsplit_r > 0 ? h->nsplit_r : h->nsplit, name.c_str(), h->num_sms);
  return std::string(buf);
}

void apply_code(rska_mrhs* h, int32_t code) {
  if (rska::tune_form(code) == rska::kFormPersistent && h->G != nullptr) {
    h->form = 2;
    h->gather_sched = rska::tune_gsched(code);
  } else {
    h->form = 1;
    h->ksplit = rska::tune_ksplit(code);
    h->use_pdl = rska::tune_pdl(code);
  }
}

cudaError_t solve_current(rska_mrhs* h, int64_t K) {
  return (h->form == 2) ? solve_tmem(h, K) : solve_staged(h, K);
}

// Time every candidate schedule for `iters` iterations (after a warm-up that
// also builds any CUDA graph) from a saved copy of the iterate, put the state
// back, and keep the fastest.  The iterate and the iteration count are the
// same afterwards as before.
int tune_impl(rska_mrhs* h, int32_t iters, int32_t* code_out, double* us_out) {
  int32_t cands[32];
  const int nc = rska::tune_candidates(h->n_p, h->R_p, h->eta_p64, h->num_sms, h->G != nullptr,
                                       cands, 32);
  cudaStream_t s = h->stream;
  const size_t zbytes = sizeof(float) * (size_t)h->R_p * h->n_p;
  float* zsave = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaError_t e = cudaMalloc(&zsave, zbytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(zsave, h->Zt, zbytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  const int64_t k0 = h->k_host;
  const int save_form = h->form, save_ks = h->ksplit, save_pdl = h->use_pdl, save_g = h->gather_sched;
  const bool save_stale = h->x_stale;
  auto restore = [&]() -> cudaError_t {
    h->k_host = k0;
    h->x_stale = true;  // the staged form rebuilds X from Z
    return cudaMemcpyAsync(h->Zt, zsave, zbytes, cudaMemcpyDeviceToDevice, s);
  };
  int32_t best = 0;
  double best_us = 0.0;
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    apply_code(h, cands[c]);
    e = restore();
    if (e == cudaSuccess) e = solve_current(h, std::min<int64_t>(iters, 64));
    if (e == cudaSuccess) e = restore();
    if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
    if (e == cudaSuccess) e = solve_current(h, iters);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    if (st != 0) {
      h->sticky = st;
      break;
    }
    const double us = 1000.0 * ms / iters;
    if (best == 0 || us < best_us) {
      best = cands[c];
      best_us = us;
    }
  }
  // back to the state before tuning, with the fastest schedule (or the
  // previous one when nothing could be timed)
  h->form = save_form;
  h->ksplit = save_ks;
  h->use_pdl = save_pdl;
  h->gather_sched = save_g;
  if (e == cudaSuccess && zsave) {
    e = restore();
    h->x_stale = save_stale || best != 0;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (zsave) cudaFree(zsave);
  if (e != cudaSuccess) return fail(h, e);
  if (h->sticky) return h->sticky;
  if (best != 0) {
    apply_code(h, best);
    h->tuned = true;
    h->tuned_code = best;
    h->tuned_us = best_us;
    rska::tune_cache_put(tune_key(h), best, best_us);
  }
  if (code_out) *code_out = best;
  if (us_out) *us_out = best_us;
  return RSKA_OK;
}

int fail(rska_mrhs* h, cudaError_t e) {
  h->sticky = (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  return h->sticky;
}

}  // namespace

extern "C" {

int rska_mrhs_setup(rska_mrhs** out, const void* A, int64_t m, int64_t n, int64_t lda,
                    const float* B, int64_t R, int64_t ldb, float lambda, int32_t eta, float t,
                    uint64_t seed, void* stream) {
  if (!out) return RSKA_EINVAL;
  *out = nullptr;
  if (!A || !B || m < 1 || n < 1 || R < 1 || lda < n || (lda % 8) != 0 || ldb < m || eta < 1 ||
      eta > rska::kMaxEta || !(lambda >= 0.f) || !std::isfinite(lambda) || !(t > 0.f) ||
      !std::isfinite(t) || m > 0x7fffffff || (reinterpret_cast<uintptr_t>(A) % 16) != 0)
    return RSKA_EINVAL;
  rska_mrhs* h = new (std::nothrow) rska_mrhs;
  if (!h) return RSKA_ENOMEM;
  h->A = static_cast<const __nv_bfloat16*>(A);
  h->m = m;
  h->n = n;
  h->lda = lda;
  h->R = R;
  h->lambda = lambda;
  h->t = t;
  h->eta = eta;
  h->seed = seed;
  h->stream = static_cast<cudaStream_t>(stream);
  h->n_p = round_up(n, rska::TN);
  h->eta_p = round_up(eta, rska::TM);
  h->R_p = round_up(R, rska::TN);
  h->idx_cap = 64;
  h->eta_p64 = round_up(eta, 64);
  h->pidx_cap = 512;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t xs = (size_t)h->R_p * h->n_p;
  const size_t as = (size_t)h->eta_p * h->n_p;
  const size_t rs = (size_t)h->R_p * h->eta_p;
  double* q = nullptr;
  int32_t* stk = nullptr;
  if (e == cudaSuccess &&
      ((e = dalloc(&h->nu, m)) != cudaSuccess || (e = dalloc(&h->inv_nu, m)) != cudaSuccess ||
       (e = dalloc(&h->thr, m)) != cudaSuccess || (e = dalloc(&h->alias, m)) != cudaSuccess ||
       (e = dalloc(&h->Bt, (size_t)m * h->R_p)) != cudaSuccess ||
       (e = dalloc(&h->Atau[0], as)) != cudaSuccess || (e = dalloc(&h->Atau[1], as)) != cudaSuccess ||
       (e = dalloc(&h->AtauT[0], as)) != cudaSuccess ||
       (e = dalloc(&h->AtauT[1], as)) != cudaSuccess ||
       (e = dalloc(&h->Xhi, xs)) != cudaSuccess || (e = dalloc(&h->Xlo, xs)) != cudaSuccess ||
       (e = dalloc(&h->Rhi, rs)) != cudaSuccess || (e = dalloc(&h->Rlo, rs)) != cudaSuccess ||
       (e = dalloc(&h->Zt, xs)) != cudaSuccess || (e = dalloc(&h->Res, rs)) != cudaSuccess ||
       (e = dalloc(&h->idx, (size_t)h->idx_cap * eta)) != cudaSuccess ||
       (e = dalloc(&h->status, 1)) != cudaSuccess || (e = dalloc(&q, m)) != cudaSuccess ||
       (e = dalloc(&stk, m)) != cudaSuccess)) {
  }
  const bool tmem_ok =
      e == cudaSuccess && rska::mrhs_tmem_fits(h->n_p, h->R_p, h->eta_p64, h->num_sms);
  const size_t gs = (size_t)2 * h->eta_p64 * h->n_p;
  if (tmem_ok &&
      ((e = dalloc(&h->G, gs)) != cudaSuccess ||
       (e = dalloc(&h->Res3, (size_t)3 * h->R_p * h->eta_p64)) != cudaSuccess ||
       (e = dalloc(&h->pbar, 1)) != cudaSuccess ||
       (e = dalloc(&h->pidx, (size_t)h->pidx_cap * eta)) != cudaSuccess)) {
  }
  h->form = tmem_ok ? 2 : 1;
  cudaStream_t s = h->stream;
  if (e == cudaSuccess && tmem_ok) e = cudaMemsetAsync(h->G, 0, gs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), s);
  for (int b = 0; b < 2; ++b) {
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Atau[b], 0, as * 2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->AtauT[b], 0, as * 2, s);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  for (int b = 0; b < 2; ++b) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_gathered[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_used[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Xhi, 0, xs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Xlo, 0, xs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Rhi, 0, rs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Rlo, 0, rs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Zt, 0, xs * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Res, 0, rs * 4, s);
  if (e == cudaSuccess) {
    const int64_t blocks = std::min<int64_t>((m + 7) / 8, (int64_t)h->num_sms * 32);
    rska::mrhs_row_norms_kernel<<<(unsigned)blocks, 256, 0, s>>>(h->A, m, n, lda, h->nu,
                                                                 h->inv_nu, h->status);
    rska::mrhs_transpose_b_kernel<<<dim3((unsigned)((m + 31) / 32), (unsigned)(h->R_p / 32)),
                                    dim3(32, 8), 0, s>>>(B, R, m, ldb, h->Bt, h->R_p, h->status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = rska::launch_alias_build(h->nu, m, h->thr, h->alias, q, stk, h->status, s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(stk);
  int rc = RSKA_OK;
  if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  else if (st != 0) rc = st;
  if (rc == RSKA_OK &&
      !(make_map(&h->mapAtau[0], h->Atau[0], h->eta_p, h->n_p, h->n_p, rska::TM) &&
        make_map(&h->mapAtau[1], h->Atau[1], h->eta_p, h->n_p, h->n_p, rska::TM) &&
        make_map(&h->mapAtauT[0], h->AtauT[0], h->n_p, h->eta_p, h->eta_p, rska::TN) &&
        make_map(&h->mapAtauT[1], h->AtauT[1], h->n_p, h->eta_p, h->eta_p, rska::TN) &&
        make_map(&h->mapX[0], h->Xhi, h->R_p, h->n_p, h->n_p, rska::TN) &&
        make_map(&h->mapX[1], h->Xlo, h->R_p, h->n_p, h->n_p, rska::TN) &&
        make_map(&h->mapR[0], h->Rhi, h->R_p, h->eta_p, h->eta_p, rska::TM) &&
        make_map(&h->mapR[1], h->Rlo, h->R_p, h->eta_p, h->eta_p, rska::TM) &&
        make_map(&h->mapRes, h->Res, h->eta_p, h->R_p, h->R_p, rska::TM, true) &&
        make_map(&h->mapZ, h->Zt, h->R_p, h->n_p, h->n_p, rska::TM, true) &&
        make_map(&h->mapXs[0], h->Xhi, h->R_p, h->n_p, h->n_p, rska::TM) &&
        make_map(&h->mapXs[1], h->Xlo, h->R_p, h->n_p, h->n_p, rska::TM) &&
        (!tmem_ok || make_map(&h->mapG, h->G, 2 * h->eta_p64, h->n_p, h->n_p, (uint32_t)h->eta_p64))))
    rc = RSKA_ECUDA;
  if (rc == RSKA_OK &&
      (cudaFuncSetAttribute(rska::mrhs_gemm_kernel<rska::kResidual>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)gemm_smem(rska::kResidual, 2)) != cudaSuccess ||
       cudaFuncSetAttribute(rska::mrhs_gemm_kernel<rska::kUpdate>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)gemm_smem(rska::kUpdate, 2)) != cudaSuccess))
    rc = RSKA_ECUDA;
  if (rc != RSKA_OK) {
    mrhs_free(h);
    delete h;
    return rc;
  }
  *out = h;
  return RSKA_OK;
}

int rska_mrhs_set_option(rska_mrhs* h, int what, int64_t value) {
  if (!h) return RSKA_EINVAL;
  switch (what) {
    case 0:
      if (value != 1 && value != 2) return RSKA_EINVAL;
      h->nsplit = (int)value;
      return RSKA_OK;
    case 1:
      if (value < 0 || value > 4096) return RSKA_EINVAL;
      h->ksplit = (int)value;
      h->pinned = true;
      return RSKA_OK;
    case 2:
      if (value < 0) return RSKA_EINVAL;
      h->limit_ns = (uint64_t)value * 1000ull;
      return RSKA_OK;
    case 3:
      if (value != 0 && value != 1) return RSKA_EINVAL;
      h->use_graph = (int)value;
      return RSKA_OK;
    case 4:
      if (value != 0 && value != 1) return RSKA_EINVAL;
      h->use_pdl = (int)value;
      h->pinned = true;
      return RSKA_OK;
    case 5:
      if (value < 0 || value > 2) return RSKA_EINVAL;
      if (value == 2 && h->G == nullptr) return RSKA_EUNSUPPORTED;
      h->form_opt = (int)value;
      h->form = value == 1 ? 1 : (h->G != nullptr ? 2 : 1);
      h->pinned = value != 0;
      return RSKA_OK;
    case 6:
      if (value < 0 || value > 2) return RSKA_EINVAL;
      h->nsplit_r = (int)value;
      return RSKA_OK;
    case 7:
      if (value < 0 || value > 5) return RSKA_EINVAL;
      h->gather_sched = (int)value;
      h->pinned = true;
      return RSKA_OK;
    default:
      return RSKA_EINVAL;
  }
}

int rska_mrhs_query(rska_mrhs* h, int what, int64_t* value) {
  if (!h || !value) return RSKA_EINVAL;
  int kb_per = 1;
  switch (what) {
    case 0: *value = h->k_host; return RSKA_OK;
    case 1: *value = residual_splits(h, &kb_per); return RSKA_OK;
    case 2: *value = h->n_p; return RSKA_OK;
    case 3: *value = h->eta_p; return RSKA_OK;
    case 4: *value = h->R_p; return RSKA_OK;
    case 5: *value = h->nsplit; return RSKA_OK;
    case 6: *value = h->form; return RSKA_OK;
    case 7: *value = h->nsplit_r > 0 ? h->nsplit_r : h->nsplit; return RSKA_OK;
    case 8: *value = h->gather_sched; return RSKA_OK;
    case 9: *value = h->tuned ? h->tuned_code : 0; return RSKA_OK;
    case 10: *value = h->tuned ? (int64_t)(1000.0 * h->tuned_us) : 0; return RSKA_OK;
    case 11: *value = h->form == 2 ? 0 : h->ksplit; return RSKA_OK;
    case 12: *value = h->use_pdl; return RSKA_OK;
    default: return RSKA_EINVAL;
  }
}

int rska_mrhs_tune(rska_mrhs* h, int32_t iters, int32_t* code_out, double* us_out) {
  if (!h || iters < 1 || iters > 100000) return RSKA_EINVAL;
  if (h->sticky) return h->sticky;
  return tune_impl(h, iters, code_out, us_out);
}

int rska_mrhs_solve(rska_mrhs* h, int64_t K) {
  if (!h || K < 0) return RSKA_EINVAL;
  if (h->sticky) return h->sticky;
  if (!h->pinned && !h->tuned && K >= kAutoTuneMinIters) {
    // the first long solve picks the schedule: from the cache when this
    // shape was measured before on this device, else by timing the candidates
    int32_t code = 0;
    double us = 0.0;
    if (rska::tune_cache_get(tune_key(h), &code, &us)) {
      apply_code(h, code);
      h->tuned = true;
      h->tuned_code = code;
      h->tuned_us = us;
    } else {
      const int rc = tune_impl(h, 64, nullptr, nullptr);
      if (rc != RSKA_OK) return rc;
    }
  }
  const cudaError_t e = (h->form == 2) ? solve_tmem(h, K) : solve_staged(h, K);
  if (e != cudaSuccess) return fail(h, e);
  h->k_host += K;
  return RSKA_OK;
}

int rska_mrhs_get_x(rska_mrhs* h, float* x_out, float* z_out) {
  if (!h) return RSKA_EINVAL;
  cudaStream_t s = h->stream;
  const int64_t total = h->R * h->n;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  mrhs_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(h->Zt, h->n_p, h->R, h->n, h->lambda, x_out,
                                                   z_out);
  int st = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, e);
  if (st != 0) h->sticky = st;
  return st;
}

int rska_mrhs_get_indices(rska_mrhs* h, int64_t k0, int64_t K, int32_t* out) {
  if (!h || !out || k0 < 0 || K < 0) return RSKA_EINVAL;
  cudaError_t e = rska::launch_indices(h->thr, h->alias, h->m, h->seed, 0, k0, K, h->eta, out,
                                       h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_mrhs_get_tables(rska_mrhs* h, double* nu_out, uint32_t* thr_out, int32_t* alias_out) {
  if (!h) return RSKA_EINVAL;
  cudaStream_t s = h->stream;
  const size_t m = (size_t)h->m;
  cudaError_t e = cudaSuccess;
  if (nu_out) e = cudaMemcpyAsync(nu_out, h->nu, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && thr_out)
    e = cudaMemcpyAsync(thr_out, h->thr, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && alias_out)
    e = cudaMemcpyAsync(alias_out, h->alias, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_mrhs_reset(rska_mrhs* h) {
  if (!h) return RSKA_EINVAL;
  cudaStream_t s = h->stream;
  const size_t xs = (size_t)h->R_p * h->n_p;
  const size_t rs = (size_t)h->R_p * h->eta_p;
  cudaError_t e = cudaMemsetAsync(h->Zt, 0, xs * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Xhi, 0, xs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Xlo, 0, xs * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Res, 0, rs * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail(h, e);
  h->k_host = 0;
  h->x_stale = false;
  h->sticky = RSKA_OK;
  return RSKA_OK;
}

int rska_mrhs_destroy(rska_mrhs* h) {
  if (!h) return RSKA_EINVAL;
  cudaStreamSynchronize(h->stream);
  mrhs_free(h);
  delete h;
  return RSKA_OK;
}

}  // extern "C"
