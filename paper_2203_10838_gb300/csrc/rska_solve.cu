// rska_solve.cu -- the persistent single-system RSKA kernel (eq. rska,
// Algorithm 1 with w_i = t).
//
// Work split: the n columns (as float4 groups) are split into P contiguous
// slices, one per CTA, and every CTA keeps its slice of z = x^* and of
// x = S_lambda(z) in shared memory for the whole launch.  One iteration:
//   1. dot phase: each CTA reads its slice of the eta sampled rows (coalesced
//      128-bit loads), forms the partial dots <a_i, x> over its columns with
//      warp shuffles and adds them into a global accumulator (one float per
//      row of tau_k); rows that fit stay in shared memory for step 3;
//   2. the CTA draws tau_{k+1} (Philox + alias table) and fetches b_i and
//      1/||a_i||^2 for it, hiding those latencies before the barrier;
//   3. grid barrier; c_i = (t/eta)(<a_i, x> - b_i)/||a_i||^2 from the reduced
//      dots; the CTA applies z_j -= sum_i c_i a_ij to its slice and
//      re-thresholds x_j = S_lambda(z_j) (steps 5-6 of Algorithm 1).
// The only cross-CTA exchange is eta floats per iteration.  A single-CTA grid
// keeps the accumulator in shared memory and uses __syncthreads instead.
#include <algorithm>

#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int NT = kSolveThreads;
constexpr int NW = NT / 32;

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Zero the components of v that lie at or beyond column n (only the last
// float4 group of a row can hold such padding).
__device__ __forceinline__ float4 mask_tail(float4 v, int64_t gc, int64_t n) {
  const int64_t base = gc * 4;
  if (base + 4 <= n) return v;
  float4 r = v;
  if (base + 0 >= n) r.x = 0.f;
  if (base + 1 >= n) r.y = 0.f;
  if (base + 2 >= n) r.z = 0.f;
  if (base + 3 >= n) r.w = 0.f;
  return r;
}

// Draw tau_k into idx[0..eta) and gather b_i, 1/||a_i||^2 for it.
__device__ __forceinline__ void draw_iteration(const SolveArgs& a, int64_t k, int32_t* idx,
                                               float* bsel, float* ivsel) {
  const int npairs = (a.eta + 1) >> 1;
  for (int q = threadIdx.x; q < npairs; q += NT) {
    int32_t i0, i1;
    draw_pair(a.seed, k, (uint32_t)q, a.problem, a.thr, a.alias, (uint32_t)a.m, &i0, &i1);
    idx[2 * q] = i0;
    bsel[2 * q] = __ldg(a.b + i0);
    ivsel[2 * q] = __ldg(a.inv_nu + i0);
    if (2 * q + 1 < a.eta) {
      idx[2 * q + 1] = i1;
      bsel[2 * q + 1] = __ldg(a.b + i1);
      ivsel[2 * q + 1] = __ldg(a.inv_nu + i1);
    }
  }
}

template <int CPL>
__global__ void __launch_bounds__(NT, 1)
    rska_persistent_kernel(SolveArgs a, int w4max, int rows_res) {
  constexpr int U = (CPL >= 8) ? 1 : 8 / CPL;  // rows in flight per lane
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;

  if (a.stop != nullptr && ld_relaxed_s32(a.stop) != 0) return;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int P = gridDim.x;
  const int eta = a.eta;
  const int64_t n4 = (a.n + 3) >> 2;
  const int64_t cb = (int64_t)blockIdx.x * n4 / P;
  const int64_t ce = (int64_t)(blockIdx.x + 1) * n4 / P;
  const int w4 = (int)(ce - cb);
  const bool single = (P == 1);

  float4* tile = reinterpret_cast<float4*>(smem);               // rows_res x w4max
  float4* zs = tile + (size_t)rows_res * w4max;                 // w4max
  float4* xs = zs + w4max;                                      // w4max
  float4* red = xs + w4max;                                     // NT
  int32_t* idx = reinterpret_cast<int32_t*>(red + NT);          // 2 x eta
  float* bsel = reinterpret_cast<float*>(idx + 2 * eta);        // 2 x eta
  float* ivsel = bsel + 2 * eta;                                // 2 x eta
  float* cs = ivsel + 2 * eta;                                  // eta
  float* sacc = cs + eta;                                       // eta (single-CTA grid only)

  const int64_t k0 = *a.kdev;
  const float lam = a.lambda;
  const float4* zg = reinterpret_cast<const float4*>(a.z);
  for (int c = tid; c < w4; c += NT) {
    const float4 zv = zg[cb + c];
    zs[c] = zv;
    xs[c] = mask_tail(soft_shrink4(zv, lam), cb + c, a.n);
  }
  if (single)
    for (int s = tid; s < eta; s += NT) sacc[s] = 0.f;
  draw_iteration(a, k0, idx, bsel, ivsel);
  __syncthreads();

  // dot-phase lane layout: L lanes per row, RPW rows per warp
  int L = 32;
  if (w4 <= 16) {
    L = 1;
    while (L < w4) L <<= 1;
  }
  const int RPW = 32 / L;
  const int sub = lane / L;
  const int lc = lane % L;
  const int rstride = NW * RPW;
  // scatter-phase layout: RG row groups of w4 threads
  const int RG = NT / w4;
  const int rg = tid / w4;
  const int sc = tid - rg * w4;

  const float* Ab = a.A + cb * 4;

  for (int64_t j = 0; j < a.K; ++j) {
    const int cur = (int)(j & 1);
    const int buf = (int)(j % 3);
    const int32_t* I = idx + cur * eta;
    float* acc_rows = single ? sacc : (a.racc + (size_t)buf * eta);

    float4 xr[CPL];
    bool tail[CPL];
#pragma unroll
    for (int jj = 0; jj < CPL; ++jj) {
      const int c = lc + L * jj;
      xr[jj] = (c < w4) ? xs[c] : make_float4(0.f, 0.f, 0.f, 0.f);
      tail[jj] = (c < w4) && ((cb + c) * 4 + 4 > a.n);
    }

    // ---- dot phase: r_i = <a_i, x_k> over this CTA's columns ----
    for (int s0 = warp * RPW; s0 < eta; s0 += rstride * U) {
      float4 av[U][CPL];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + sub + u * rstride;
        const bool rv = s < eta;
        const float* rowp = Ab + (int64_t)(rv ? I[s] : 0) * a.lda;
#pragma unroll
        for (int jj = 0; jj < CPL; ++jj) {
          const int c = lc + L * jj;
          av[u][jj] = (rv && c < w4) ? __ldg(reinterpret_cast<const float4*>(rowp) + c)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int s = s0 + sub + u * rstride;
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < CPL; ++jj) {
          float4 v = av[u][jj];
          if (tail[jj]) v = mask_tail(v, cb + lc + L * jj, a.n);
          acc += dot4(v, xr[jj]);
          const int c = lc + L * jj;
          if (s < rows_res && c < w4) tile[(size_t)s * w4max + c] = v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1)
          if (o < L) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lc == 0 && s < eta) {
          if (single)
            atomicAdd(acc_rows + s, acc);
          else
            atomicAdd(acc_rows + s, acc);
        }
      }
    }

    // ---- draw tau_{k+1}; recycle an accumulator buffer ----
    if (j + 1 < a.K) draw_iteration(a, k0 + j + 1, idx + (cur ^ 1) * eta,
                                    bsel + (cur ^ 1) * eta, ivsel + (cur ^ 1) * eta);
    if (!single && blockIdx.x == 0) {
      float* nxt = a.racc + (size_t)((j + 1) % 3) * eta;
      for (int s = tid; s < eta; s += NT) nxt[s] = 0.f;
    }

    if (single) {
      __syncthreads();
    } else if (!grid_barrier(a.bar, (unsigned long long)(j + 1), a.status, a.limit_ns,
                             &s_flag)) {
      return;
    }

    // ---- coefficients c_i = (t/eta) (r_i - b_i) / ||a_i||^2 ----
    const float* Bs = bsel + cur * eta;
    const float* Vs = ivsel + cur * eta;
    for (int s = tid; s < eta; s += NT) {
      float r;
      if (single) {
        r = sacc[s];
        sacc[s] = 0.f;
      } else {
        r = __ldcg(acc_rows + s);
      }
      cs[s] = a.coef * ((r - Bs[s]) * Vs[s]);
    }
    __syncthreads();

    // ---- scatter: z_j -= sum_i c_i a_ij over this CTA's columns ----
    if (rg < RG) {
      float4 acc4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const bool tl = ((cb + sc) * 4 + 4 > a.n);
      for (int s = rg; s < eta; s += RG) {
        const float cval = cs[s];
        float4 v;
        if (s < rows_res) {
          v = tile[(size_t)s * w4max + sc];
        } else {
          v = __ldg(reinterpret_cast<const float4*>(Ab + (int64_t)I[s] * a.lda) + sc);
          if (tl) v = mask_tail(v, cb + sc, a.n);
        }
        acc4.x = fmaf(cval, v.x, acc4.x);
        acc4.y = fmaf(cval, v.y, acc4.y);
        acc4.z = fmaf(cval, v.z, acc4.z);
        acc4.w = fmaf(cval, v.w, acc4.w);
      }
      red[tid] = acc4;
    }
    __syncthreads();
    for (int c = tid; c < w4; c += NT) {
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int g = 0; g < RG; ++g) {
        const float4 v = red[g * w4 + c];
        sum.x += v.x;
        sum.y += v.y;
        sum.z += v.z;
        sum.w += v.w;
      }
      float4 zv = zs[c];
      zv.x -= sum.x;
      zv.y -= sum.y;
      zv.z -= sum.z;
      zv.w -= sum.w;
      zv = mask_tail(zv, cb + c, a.n);
      zs[c] = zv;
      xs[c] = soft_shrink4(zv, lam);
    }
    __syncthreads();
  }

  float4* zo = reinterpret_cast<float4*>(a.z);
  float4* xo = reinterpret_cast<float4*>(a.x);
  for (int c = tid; c < w4; c += NT) {
    zo[cb + c] = zs[c];
    xo[cb + c] = xs[c];
  }
  if (blockIdx.x == 0 && tid == 0) *a.kdev = k0 + a.K;
}

size_t fixed_smem(int w4max, int eta) {
  return (size_t)2 * w4max * 16 + (size_t)NT * 16 + (size_t)2 * eta * 12 + (size_t)eta * 4 +
         (size_t)eta * 4;
}

template <int CPL>
cudaError_t set_smem_attr(size_t smem) {
  return cudaFuncSetAttribute(rska_persistent_kernel<CPL>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

bool plan_solve(int64_t n, int32_t eta, int num_sms, int grid_override, size_t smem_optin,
                SolveGeometry* g) {
  const int64_t n4 = (n + 3) / 4;
  int64_t P;
  if (grid_override > 0) {
    P = grid_override;
  } else if (n4 <= 128) {
    P = 1;  // small systems: one CTA, no grid barrier
  } else {
    P = std::min<int64_t>(num_sms, (n4 + 7) / 8);
  }
  P = std::max<int64_t>(1, std::min<int64_t>(P, std::min<int64_t>(num_sms, n4)));
  const int64_t w4max = (n4 + P - 1) / P;
  int cpl = 1;
  if (w4max > 32) cpl = 2;
  if (w4max > 64) cpl = 4;
  if (w4max > 128) cpl = 8;
  if (w4max > 256) return false;
  const size_t fixed = fixed_smem((int)w4max, eta) + 1024;
  if (fixed > smem_optin) return false;
  int64_t rows = (int64_t)((smem_optin - fixed) / ((size_t)w4max * 16));
  rows = std::min<int64_t>(rows, eta);
  g->grid = (int)P;
  g->w4max = (int)w4max;
  g->cpl = cpl;
  g->rows_res = (int)rows;
  g->smem = fixed_smem((int)w4max, eta) + (size_t)rows * w4max * 16;
  return true;
}

cudaError_t launch_solve(const SolveArgs& a, const SolveGeometry& g, cudaStream_t s) {
  cudaError_t e;
  void* fn = nullptr;
  switch (g.cpl) {
    case 1: e = set_smem_attr<1>(g.smem); fn = (void*)rska_persistent_kernel<1>; break;
    case 2: e = set_smem_attr<2>(g.smem); fn = (void*)rska_persistent_kernel<2>; break;
    case 4: e = set_smem_attr<4>(g.smem); fn = (void*)rska_persistent_kernel<4>; break;
    default: e = set_smem_attr<8>(g.smem); fn = (void*)rska_persistent_kernel<8>; break;
  }
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.racc, 0, sizeof(float) * 3 * (size_t)a.eta, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  SolveArgs args = a;
  int w4max = g.w4max;
  int rows_res = g.rows_res;
  void* params[] = {&args, &w4max, &rows_res};
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
  return cudaLaunchKernelExC(&cfg, fn, params);
}

}  // namespace rska
