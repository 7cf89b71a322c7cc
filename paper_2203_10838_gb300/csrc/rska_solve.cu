// rska_solve.cu -- the persistent single-system RSKA kernel (eq. rska,
// Algorithm 1 with w_i = t) and its index pre-sampler.
//
// Work split.  The n columns, as float4 groups, are split into P contiguous
// slices, one per CTA; a CTA keeps its slice of z = x^* and x = S_lambda(z)
// in shared memory for the whole launch.  Inside a CTA, thread (rg, c) owns
// float4 column c of the slice and the rows s = rg + RG*i of tau_k
// (RG = threads / slice width), so consecutive threads touch consecutive
// 16-byte words of a row (coalesced) and every thread's rows stay with it for
// the whole iteration.
//
// One iteration k:
//   1. the CTA's slice of the eta sampled rows is fetched once from HBM: the
//      first row steps with cp.async into shared memory (one commit group per
//      batch of kDotBatch row steps, so the dots start while later batches are
//      in flight), the next ones into registers; anything beyond on-chip
//      capacity is streamed and fetched again in step 4;
//   2. each thread forms <a_s, x> over its float4 column for a batch of row
//      steps into a shared buffer; the batch's rows are then summed across the
//      slice by a few threads each (a shuffle finishes them) and one global
//      atomic per row adds the CTA's partial dot to a padded accumulator;
//   3. grid barrier (bounded wait);  c_s = (t/eta)(<a_s, x_k> - b_s)/||a_s||^2;
//   4. z_j -= sum_s c_s a_sj from the on-chip rows, reduced over the row
//      groups of each column, then x_j = S_lambda(z_j).  As each on-chip slot
//      is consumed it is refilled with the row of tau_{k+1}, so HBM streams
//      the next iteration while this one finishes.
// tau_{k}, b_{tau} and 1/||a_tau||^2 come from a pre-sampler kernel that draws
// the whole launch's indices in parallel; the persistent kernel copies them
// one iteration ahead, so no dependent gather sits on the critical path.  The
// only cross-CTA exchange is eta floats per iteration.  A one-CTA grid keeps
// the accumulator in shared memory and uses __syncthreads as the barrier.
#include <algorithm>

#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int NT = kSolveThreads;

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Zero the components of v at or beyond column n (only the last float4 group
// of a row can hold padding).
__device__ __forceinline__ float4 mask_tail(float4 v, int64_t gc, int64_t n) {
  const int64_t base = gc * 4;
  float4 r = v;
  if (base + 0 >= n) r.x = 0.f;
  if (base + 1 >= n) r.y = 0.f;
  if (base + 2 >= n) r.z = 0.f;
  if (base + 3 >= n) r.w = 0.f;
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_smem)),
               "l"(src_gmem)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float4 ldg_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// Pre-sampler: tau_k, b_{tau_k}, 1/||a_{tau_k}||^2 for k = k0 .. k0+K-1, with
// k0 read from the device iteration counter.  Row j of each output (stride
// eta4 = eta rounded up to 4) belongs to iteration k0 + j.
// ---------------------------------------------------------------------------
__global__ void presample_kernel(const uint32_t* __restrict__ thr, const int32_t* __restrict__ alias,
                                 uint32_t m, uint64_t seed, uint32_t problem,
                                 const int64_t* __restrict__ kdev, int64_t K, int32_t eta,
                                 int32_t eta4, const float* __restrict__ b,
                                 const float* __restrict__ inv_nu, int32_t* __restrict__ tidx,
                                 float* __restrict__ tb, float* __restrict__ tiv,
                                 const int* stop) {
  if (stop != nullptr && ld_relaxed_s32(stop) != 0) return;
  const int64_t k0 = *kdev;
  const int64_t npairs = (eta + 1) / 2;
  const int64_t total = K * npairs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / npairs;
    const uint32_t q = (uint32_t)(e - j * npairs);
    int32_t i0, i1;
    draw_pair(seed, k0 + j, q, problem, thr, alias, m, &i0, &i1);
    const int64_t o = j * eta4 + 2 * q;
    tidx[o] = i0;
    tb[o] = __ldg(b + i0);
    tiv[o] = __ldg(inv_nu + i0);
    if (2 * (int64_t)q + 1 < eta) {
      tidx[o + 1] = i1;
      tb[o + 1] = __ldg(b + i1);
      tiv[o + 1] = __ldg(inv_nu + i1);
    }
  }
}

// cp.async.wait_group with a run-time count of groups allowed to stay pending.
__device__ __forceinline__ void cp_async_wait_dyn(int pending) {
  switch (pending) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    case 7: cp_async_wait<7>(); break;
    case 8: cp_async_wait<8>(); break;
    case 9: cp_async_wait<9>(); break;
    default: cp_async_wait<10>(); break;
  }
}

template <int RREG>
__global__ void __launch_bounds__(NT, 1)
    rska_persistent_kernel(SolveArgs a, int w4max, int tile_cap) {
  constexpr int B = kDotBatch;  // row steps reduced together
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag;

  if (a.stop != nullptr && ld_relaxed_s32(a.stop) != 0) return;

  const int tid = threadIdx.x;
  const int P = gridDim.x;
  const int eta = a.eta;
  const int eta4 = (eta + 3) & ~3;
  const int64_t n4 = (a.n + 3) >> 2;
  const int64_t cb = (int64_t)blockIdx.x * n4 / P;
  const int64_t ce = (int64_t)(blockIdx.x + 1) * n4 / P;
  const int w4 = (int)(ce - cb);
  const bool single = (P == 1);

  // thread layout: RG row groups x w4 columns
  const int RG = NT / w4;
  const int NTa = RG * w4;
  const int rg = tid / w4;
  const int c = tid - rg * w4;
  const bool active = rg < RG;
  const int NI = (eta + RG - 1) / RG;        // row steps
  const int IS = tile_cap / NTa;             // row steps held in shared memory
  const int nIs = min(IS, NI);
  const int nbs = (nIs + B - 1) / B;         // shared-memory batches (one cp.async group each)
  const bool tailc = active && ((cb + c) * 4 + 4 > a.n);
  // batch reduction layout: Q threads per row
  int Q = 1;
  while (Q < 32 && 2 * Q * B * RG <= NT) Q <<= 1;

  float4* tile = reinterpret_cast<float4*>(smem);                  // tile_cap
  float4* zs = tile + tile_cap;                                    // w4max
  float4* xs = zs + w4max;                                         // w4max
  float* ptile = reinterpret_cast<float*>(xs + w4max);             // B x NT (aliased by red)
  float4* red = reinterpret_cast<float4*>(ptile);                  // NT (scatter phase)
  int32_t* sidx = reinterpret_cast<int32_t*>(ptile + (size_t)B * NT);  // 2 x eta4
  float* sb = reinterpret_cast<float*>(sidx + 2 * eta4);           // eta4
  float* siv = sb + eta4;                                          // eta4
  float* cs = siv + eta4;                                          // eta4
  float* sdot = cs + eta4;                                         // eta4

  const int64_t k0 = *a.kdev;
  const float lam = a.lambda;
  {
    const float4* zg = reinterpret_cast<const float4*>(a.z);
    for (int q = tid; q < w4; q += NT) {
      const float4 zv = zg[cb + q];
      zs[q] = zv;
      xs[q] = mask_tail(soft_shrink4(zv, lam), cb + q, a.n);
    }
    for (int q = tid; q < eta4 / 4; q += NT) cp_async16(sidx + 4 * q, a.tidx + 4 * q);
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncthreads();

  const float* Ab = a.A + cb * 4 + (active ? c : 0) * 4;
  const int64_t lda = a.lda;
  auto row_ptr = [&](const int32_t* I, int s) {
    return reinterpret_cast<const float4*>(Ab + (int64_t)I[s] * lda);
  };

  // fetch of the first iteration's rows (later iterations are fetched during
  // the previous iteration's update phase)
  float4 rv[RREG > 0 ? RREG : 1];
  for (int b = 0; b < nbs; ++b) {
    if (active) {
      const int iend = min(nIs, (b + 1) * B);
      for (int i = b * B; i < iend; ++i) {
        const int s = rg + RG * i;
        if (s < eta) cp_async16(tile + (size_t)i * NTa + tid, row_ptr(sidx, s));
      }
    }
    cp_async_commit();
  }
#pragma unroll
  for (int r = 0; r < RREG; ++r) {
    const int i = IS + r;
    const int s = rg + RG * i;
    rv[r] = (active && i < NI && s < eta) ? ldg_stream(row_ptr(sidx, s))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
  }

  for (int64_t j = 0; j < a.K; ++j) {
    const int cur = (int)(j & 1);
    const int32_t* I = sidx + cur * eta4;
    const int32_t* In = sidx + (cur ^ 1) * eta4;
    const bool more = (j + 1 < a.K);
    const float4 xc = active ? xs[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int buf = (int)(j % 3);
    float* racc = a.racc + (size_t)buf * eta * kAccStride;

    {  // b, 1/||a||^2 of this iteration; tau of the next one
      const int nq = eta4 / 4;
      const int32_t* gi = a.tidx + (j + 1) * eta4;
      const float* gb = a.tb + j * eta4;
      const float* gv = a.tiv + j * eta4;
      int32_t* nidx = sidx + (cur ^ 1) * eta4;
      for (int q = tid; q < 3 * nq; q += NT) {
        if (q < nq) {
          cp_async16(sb + 4 * q, gb + 4 * q);
        } else if (q < 2 * nq) {
          cp_async16(siv + 4 * (q - nq), gv + 4 * (q - nq));
        } else if (more) {
          cp_async16(nidx + 4 * (q - 2 * nq), gi + 4 * (q - 2 * nq));
        }
      }
      cp_async_commit();
    }

    // ---- partial dots: products to ptile, then a per-batch row reduction ----
    auto product = [&](int i, float4 v) -> float {
      const int s = rg + RG * i;
      if (!(active && i < NI && s < eta)) return 0.f;
      if (tailc) v = mask_tail(v, cb + c, a.n);
      return dot4(v, xc);
    };
    auto reduce_batch = [&](int ib) {
      __syncthreads();
      const int rows = B * RG;
      for (int t0 = 0; t0 < rows * Q; t0 += NT) {
        const int t = t0 + tid;
        const int rl = t / Q;
        const int part = t - rl * Q;
        float sum = 0.f;
        int s = eta;
        if (rl < rows) {
          const int u = rl / RG;
          const int g = rl - u * RG;
          s = g + RG * (ib + u);
          const float* pr = ptile + (size_t)u * NT + g * w4;
          for (int cc = part; cc < w4; cc += Q) sum += pr[cc];
        }
        for (int o = Q >> 1; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (part == 0 && rl < rows && ib + rl / RG < NI && s < eta) {
          if (single)
            sdot[s] = sum;
          else
            atomicAdd(racc + (size_t)s * kAccStride, sum);
        }
      }
      __syncthreads();
    };
    for (int b = 0; b < nbs; ++b) {
      cp_async_wait_dyn(nbs - b);  // this batch's group done; later ones + meta may pend
      const int iend = min(nIs, (b + 1) * B);
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int i = b * B + u;
        ptile[(size_t)u * NT + tid] = (i < iend) ? product(i, tile[(size_t)i * NTa + tid]) : 0.f;
      }
      reduce_batch(b * B);
    }
    if (nIs < NI) {
#pragma unroll
      for (int rb = 0; rb < RREG; rb += B) {
#pragma unroll
        for (int u = 0; u < B; ++u)
          ptile[(size_t)u * NT + tid] = (rb + u < RREG) ? product(IS + rb + u, rv[rb + u]) : 0.f;
        if (IS + rb < NI) reduce_batch(IS + rb);
      }
      for (int ib = IS + RREG; ib < NI; ib += B) {  // beyond on-chip capacity
        float4 sv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int i = ib + u;
          const int s = rg + RG * i;
          sv[u] = (active && i < NI && s < eta) ? __ldg(row_ptr(I, s))
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) ptile[(size_t)u * NT + tid] = product(ib + u, sv[u]);
        reduce_batch(ib);
      }
    }
    if (!single) {
      // every CTA clears its share of the accumulators of iteration j + 1
      float* nxt = a.racc + (size_t)((j + 1) % 3) * eta * kAccStride;
      for (int s = blockIdx.x + (int)gridDim.x * tid; s < eta; s += (int)gridDim.x * NT)
        nxt[(size_t)s * kAccStride] = 0.f;
    }
    cp_async_wait<0>();

    // ---- exchange and coefficients ----
    if (single) {
      __syncthreads();
    } else if (!grid_barrier(a.bar, (unsigned long long)(j + 1), a.status, a.limit_ns,
                             &s_flag)) {
      return;
    }
    for (int s = tid; s < eta; s += NT) {
      const float r = single ? sdot[s] : __ldcg(racc + (size_t)s * kAccStride);
      cs[s] = a.coef * ((r - sb[s]) * siv[s]);
    }
    __syncthreads();

    // ---- z_j -= sum_s c_s a_sj; refill each slot with the next iteration's row ----
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    auto upd = [&](int i, float4 v) {
      const int s = rg + RG * i;
      if (active && i < NI && s < eta) {
        if (tailc) v = mask_tail(v, cb + c, a.n);
        const float cv = cs[s];
        acc.x = fmaf(cv, v.x, acc.x);
        acc.y = fmaf(cv, v.y, acc.y);
        acc.z = fmaf(cv, v.z, acc.z);
        acc.w = fmaf(cv, v.w, acc.w);
      }
    };
    for (int b = 0; b < nbs; ++b) {
      const int iend = min(nIs, (b + 1) * B);
      for (int i = b * B; i < iend; ++i) {
        float4* slot = tile + (size_t)i * NTa + tid;
        upd(i, *slot);
        const int s = rg + RG * i;
        if (more && active && s < eta) cp_async16(slot, row_ptr(In, s));
      }
      cp_async_commit();
    }
#pragma unroll
    for (int r = 0; r < RREG; ++r) {
      const int i = IS + r;
      upd(i, rv[r]);
      const int s = rg + RG * i;
      if (more && active && i < NI && s < eta) rv[r] = ldg_stream(row_ptr(In, s));
    }
    for (int ib = IS + RREG; ib < NI; ib += B) {
      float4 sv[B];
#pragma unroll
      for (int u = 0; u < B; ++u) {
        const int i = ib + u;
        const int s = rg + RG * i;
        sv[u] = (active && i < NI && s < eta) ? __ldg(row_ptr(I, s))
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < B; ++u) upd(ib + u, sv[u]);
    }
    red[tid] = acc;
    __syncthreads();
    {
      // column sums over the RG row groups: 4 threads per float4 component
      const float* redf = reinterpret_cast<const float*>(red);
      float* zf = reinterpret_cast<float*>(zs);
      float* xf = reinterpret_cast<float*>(xs);
      const int ncomp = w4 * 4;
      for (int t0 = 0; t0 < ncomp * 4; t0 += NT) {
        const int t = t0 + tid;
        const int e = t >> 2;
        const int part = t & 3;
        float sum = 0.f;
        if (e < ncomp)
          for (int g = part; g < RG; g += 4) sum += redf[(size_t)g * w4 * 4 + e];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (part == 0 && e < ncomp) {
          const int64_t col = cb * 4 + e;
          const float zv = (col < a.n) ? zf[e] - sum : 0.f;
          zf[e] = zv;
          xf[e] = soft_shrink(zv, lam);
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  float4* zo = reinterpret_cast<float4*>(a.z);
  float4* xo = reinterpret_cast<float4*>(a.x);
  for (int q = tid; q < w4; q += NT) {
    zo[cb + q] = zs[q];
    xo[cb + q] = xs[q];
  }
  if (blockIdx.x == 0 && tid == 0) *a.kdev = k0 + a.K;
}

size_t fixed_smem(int w4max, int eta) {
  const size_t eta4 = (size_t)((eta + 3) & ~3);
  const size_t ptile = std::max<size_t>((size_t)kDotBatch * NT * 4, (size_t)NT * 16);
  return (size_t)2 * w4max * 16 + ptile + 2 * eta4 * 4 + 4 * eta4 * 4;
}

template <int RREG>
cudaError_t set_smem_attr(size_t smem) {
  return cudaFuncSetAttribute(rska_persistent_kernel<RREG>,
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
  if (w4max > kSolveThreads / 2) return false;
  const size_t fixed = fixed_smem((int)w4max, eta) + 1024;
  if (fixed + 16 * (size_t)kSolveThreads > smem_optin) return false;
  const int tile_cap = (int)((smem_optin - fixed) / 16);
  // row steps of the widest CTA beyond shared memory decide the register part
  const int64_t RGw = kSolveThreads / w4max;
  const int64_t NI = (eta + RGw - 1) / RGw;
  const int64_t IS = tile_cap / (RGw * w4max);
  g->grid = (int)P;
  g->w4max = (int)w4max;
  g->tile_cap = tile_cap;
  g->rreg = (NI > IS) ? kSolveRegRows : 0;
  g->rows_res = (int)std::min<int64_t>(eta, (IS + g->rreg) * RGw);
  g->smem = fixed_smem((int)w4max, eta) + (size_t)tile_cap * 16;
  return true;
}

cudaError_t launch_presample(const SolveArgs& a, cudaStream_t s) {
  const int64_t total = a.K * ((a.eta + 1) / 2);
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  presample_kernel<<<(unsigned)blocks, 256, 0, s>>>(
      a.thr, a.alias, (uint32_t)a.m, a.seed, a.problem, a.kdev, a.K, a.eta, (a.eta + 3) & ~3,
      a.b, a.inv_nu, const_cast<int32_t*>(a.tidx), const_cast<float*>(a.tb),
      const_cast<float*>(a.tiv), a.stop);
  return cudaGetLastError();
}

cudaError_t launch_solve(const SolveArgs& a, const SolveGeometry& g, cudaStream_t s) {
  cudaError_t e;
  void* fn = nullptr;
  if (g.rreg > 0) {
    e = set_smem_attr<kSolveRegRows>(g.smem);
    fn = (void*)rska_persistent_kernel<kSolveRegRows>;
  } else {
    e = set_smem_attr<0>(g.smem);
    fn = (void*)rska_persistent_kernel<0>;
  }
  if (e != cudaSuccess) return e;
  e = launch_presample(a, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.racc, 0, sizeof(float) * 3 * (size_t)a.eta * kAccStride, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  SolveArgs args = a;
  int w4max = g.w4max;
  int tile_cap = g.tile_cap;
  void* params[] = {&args, &w4max, &tile_cap};
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
