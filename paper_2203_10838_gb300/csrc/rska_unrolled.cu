// rska_unrolled.cu -- K unrolled iterations of eq. (rska) on P independent
// problems and their hand-written adjoint, for gradients of a loss of x_K
// with respect to b, lambda and t (the paper has no gradient; this
// differentiates the iteration as written, with the index sequence fixed by
// the index contract).
//
// Forward (one CTA per problem, thread t owns float4 columns t + 256 r):
//   z_0 = 0;  x_k = S_lambda(z_k);  r_s = <a_s, x_k> - b_s;
//   z_{k+1} = z_k - (t/eta) sum_s r_s / ||a_s||^2 a_s;
// z_k is saved every `ckpt` iterations.
// Backward, with g = dL/dz_{k+1} and mask_k = 1[|z_k| > lambda]:
//   u_s        = (t/eta) <a_s, g> / ||a_s||^2
//   dL/db_i   += u_s for every draw s of row i (duplicates add)
//   dL/dt     += -(1/eta) sum_s r_s / ||a_s||^2 <a_s, g>
//   xbar       = -sum_s u_s a_s
//   dL/dlambda += sum_j xbar_j (-sign(z_kj)) mask_kj
//   dL/dz_k    = g + mask_k xbar
// starting from dL/dz_K = mask_K dL/dx_K and dL/dlambda = sum_j dL/dx_Kj
// (-sign z_Kj) mask_Kj.  Each checkpoint segment is recomputed forward into a
// per-problem buffer and then swept backward; tau_k is re-drawn from Philox
// for every k, so no index sequence is stored.  Rows are read straight from
// HBM in batches of 8 per thread (two dots per row in the backward step).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "rska_alias.cuh"
#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int UT = 256;             // threads per CTA
constexpr int UW = UT / 32;         // warps
constexpr int UB = 8;               // rows per batch
constexpr int UMAXETA = 1024;

struct UnrolledArgs {
  int32_t P;
  const float* A;
  const int64_t* a_off;
  const int32_t* m;
  const int32_t* n;
  const int64_t* lda;
  const float* b;
  const int64_t* b_off;
  const int64_t* row_off;
  const float* inv_nu;
  const uint32_t* thr;
  const int32_t* alias;
  const int64_t* x_off;
  const float* lambda;       // per problem
  const float* t;            // per problem
  int32_t eta;
  uint64_t seed;
  int32_t K;
  int32_t ckpt;
  float* ckpts;              // per problem: (K/ckpt + 1) x x_stride floats
  float* segbuf;             // per problem: ckpt x x_stride floats
  int64_t x_stride;          // floats per stored iterate (max n rounded to 4)
  float* x_out;              // packed by x_off
  const float* gx;           // dL/dx_K, packed by x_off
  float* gb;                 // dL/db, packed by b_off
  float* glam;               // per problem
  float* gt;                 // per problem
  int32_t* tidx;             // row-form kernels: tau_k per problem and iteration, [P][K][eta]
  float* tiv;                // 1/||a||^2 at tau_k, same layout
  float* tb;                 // b at tau_k for the current b, same layout
};

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

__device__ __forceinline__ float neg_sign_mask(float z, float lam) {
  return fabsf(z) > lam ? (z > 0.f ? -1.f : 1.f) : 0.f;
}

struct ProbCtx {
  int m, n;
  int64_t n4, lda;
  const float* Ap;
  const float* bp;
  const float* inv_nu;
  const uint32_t* thr;
  const int32_t* alias;
  float lam, coef, t;
};

// Draw tau_k of problem p into shared arrays (index, b, 1/||a||^2).
__device__ void draw_iter(const UnrolledArgs& a, const ProbCtx& c, int p, int k, int32_t* sidx,
                          float* sb, float* siv) {
  const int npairs = (a.eta + 1) >> 1;
  for (int q = threadIdx.x; q < npairs; q += UT) {
    int32_t i0, i1;
    draw_pair(a.seed, k, (uint32_t)q, (uint32_t)p, c.thr, c.alias, (uint32_t)c.m, &i0, &i1);
    sidx[2 * q] = i0;
    sb[2 * q] = __ldg(c.bp + i0);
    siv[2 * q] = __ldg(c.inv_nu + i0);
    if (2 * q + 1 < a.eta) {
      sidx[2 * q + 1] = i1;
      sb[2 * q + 1] = __ldg(c.bp + i1);
      siv[2 * q + 1] = __ldg(c.inv_nu + i1);
    }
  }
}

// Block reduction of NV values per thread for UB rows: out[v][u] = sum over
// threads of val[v][u].  Uses red (UW x NV x UB floats); ends synchronized.
template <int NV>
__device__ __forceinline__ void block_sum_rows(float (&val)[NV][UB], float* red,
                                               float (&out)[NV][UB]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      float s = val[v][u];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[(warp * NV + v) * UB + u] = s;
    }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < UW; ++w) s += red[(w * NV + v) * UB + u];
      out[v][u] = s;
    }
  __syncthreads();
}

// One forward step z <- z - (t/eta) sum_s r_s/||a_s||^2 a_s with x = S(z).
template <int UZ>
__device__ void forward_step(const UnrolledArgs& a, const ProbCtx& c, const int32_t* sidx,
                             const float* sb, const float* siv, float4 (&z)[UZ], float* red) {
  const int tid = threadIdx.x;
  float4 x[UZ], dl[UZ];
#pragma unroll
  for (int r = 0; r < UZ; ++r) {
    x[r] = soft_shrink4(z[r], c.lam);
    dl[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int s0 = 0; s0 < a.eta; s0 += UB) {
    float4 av[UB][UZ];
    float pd[1][UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int s = s0 + u;
      pd[0][u] = 0.f;
      const float4* row =
          reinterpret_cast<const float4*>(c.Ap + (int64_t)(s < a.eta ? sidx[s] : 0) * c.lda);
#pragma unroll
      for (int r = 0; r < UZ; ++r) {
        const int64_t col = tid + (int64_t)UT * r;
        float4 v = (s < a.eta && col < c.n4) ? __ldg(row + col) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (col == c.n4 - 1) v = mask_tail(v, col, c.n);
        av[u][r] = v;
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u)
#pragma unroll
      for (int r = 0; r < UZ; ++r) pd[0][u] += dot4(av[u][r], x[r]);
    float tot[1][UB];
    block_sum_rows<1>(pd, red, tot);
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int s = s0 + u;
      if (s < a.eta) {
        const float cval = c.coef * ((tot[0][u] - sb[s]) * siv[s]);
#pragma unroll
        for (int r = 0; r < UZ; ++r) {
          dl[r].x = fmaf(cval, av[u][r].x, dl[r].x);
          dl[r].y = fmaf(cval, av[u][r].y, dl[r].y);
          dl[r].z = fmaf(cval, av[u][r].z, dl[r].z);
          dl[r].w = fmaf(cval, av[u][r].w, dl[r].w);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < UZ; ++r) {
    const int64_t col = tid + (int64_t)UT * r;
    if (col < c.n4) {
      float4 zv = z[r];
      zv.x -= dl[r].x;
      zv.y -= dl[r].y;
      zv.z -= dl[r].z;
      zv.w -= dl[r].w;
      z[r] = mask_tail(zv, col, c.n);
    }
  }
}

template <int UZ>
__device__ void store_iter(float* dst, const float4 (&z)[UZ], int64_t n4) {
#pragma unroll
  for (int r = 0; r < UZ; ++r) {
    const int64_t col = threadIdx.x + (int64_t)UT * r;
    if (col < n4) reinterpret_cast<float4*>(dst)[col] = z[r];
  }
}

template <int UZ>
__device__ void load_iter(const float* src, float4 (&z)[UZ], int64_t n4) {
#pragma unroll
  for (int r = 0; r < UZ; ++r) {
    const int64_t col = threadIdx.x + (int64_t)UT * r;
    z[r] = (col < n4) ? __ldcg(reinterpret_cast<const float4*>(src) + col)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ ProbCtx prob_ctx(const UnrolledArgs& a, int p) {
  ProbCtx c;
  c.m = a.m[p];
  c.n = a.n[p];
  c.n4 = (c.n + 3) >> 2;
  c.lda = a.lda[p];
  c.Ap = a.A + a.a_off[p];
  c.bp = a.b + a.b_off[p];
  c.inv_nu = a.inv_nu + a.row_off[p];
  c.thr = a.thr + a.row_off[p];
  c.alias = a.alias + a.row_off[p];
  c.lam = a.lambda[p];
  c.t = a.t[p];
  c.coef = c.t / (float)a.eta;
  return c;
}

template <int UZ>
__global__ void __launch_bounds__(UT, 1) unrolled_forward_kernel(UnrolledArgs a) {
  __shared__ int32_t sidx[UMAXETA];
  __shared__ float sb[UMAXETA];
  __shared__ float siv[UMAXETA];
  __shared__ float red[UW * 2 * UB];
  const int nck = a.K / a.ckpt;
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const ProbCtx c = prob_ctx(a, p);
    float* ck = a.ckpts + (size_t)p * (nck + 1) * a.x_stride;
    float4 z[UZ];
#pragma unroll
    for (int r = 0; r < UZ; ++r) z[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    store_iter<UZ>(ck, z, c.n4);
    for (int k = 0; k < a.K; ++k) {
      draw_iter(a, c, p, k, sidx, sb, siv);
      __syncthreads();
      forward_step<UZ>(a, c, sidx, sb, siv, z, red);
      if ((k + 1) % a.ckpt == 0) store_iter<UZ>(ck + (size_t)((k + 1) / a.ckpt) * a.x_stride, z, c.n4);
      __syncthreads();
    }
    float* xo = a.x_out + a.x_off[p];
#pragma unroll
    for (int r = 0; r < UZ; ++r) {
      const int64_t col = threadIdx.x + (int64_t)UT * r;
      if (col < c.n4) reinterpret_cast<float4*>(xo)[col] = soft_shrink4(z[r], c.lam);
    }
    __syncthreads();
  }
}

template <int UZ>
__global__ void __launch_bounds__(UT, 1) unrolled_backward_kernel(UnrolledArgs a) {
  __shared__ int32_t sidx[UMAXETA];
  __shared__ float sb[UMAXETA];
  __shared__ float siv[UMAXETA];
  __shared__ float red[UW * 2 * UB];
  __shared__ float sfin[2][UW];
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nck = a.K / a.ckpt;
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const ProbCtx c = prob_ctx(a, p);
    const float* ck = a.ckpts + (size_t)p * (nck + 1) * a.x_stride;
    float* seg = a.segbuf + (size_t)p * a.ckpt * a.x_stride;
    float* gbp = a.gb + a.b_off[p];
    const float* gxp = a.gx + a.x_off[p];
    float glam = 0.f, gt = 0.f;
    // g = dL/dz_K = mask_K * dL/dx_K
    float4 z[UZ], g[UZ];
    load_iter<UZ>(ck + (size_t)nck * a.x_stride, z, c.n4);
#pragma unroll
    for (int r = 0; r < UZ; ++r) {
      const int64_t col = tid + (int64_t)UT * r;
      float4 gxv = (col < c.n4) ? __ldg(reinterpret_cast<const float4*>(gxp) + col)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      if (col == c.n4 - 1) gxv = mask_tail(gxv, col, c.n);
      const float sx = neg_sign_mask(z[r].x, c.lam), sy = neg_sign_mask(z[r].y, c.lam);
      const float sz = neg_sign_mask(z[r].z, c.lam), sw = neg_sign_mask(z[r].w, c.lam);
      glam += gxv.x * sx + gxv.y * sy + gxv.z * sz + gxv.w * sw;
      g[r] = make_float4(sx != 0.f ? gxv.x : 0.f, sy != 0.f ? gxv.y : 0.f,
                         sz != 0.f ? gxv.z : 0.f, sw != 0.f ? gxv.w : 0.f);
    }
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
      const int k0 = sgi * a.ckpt;
      // recompute z_{k0} .. z_{k0+ckpt-1} into the segment buffer
      load_iter<UZ>(ck + (size_t)sgi * a.x_stride, z, c.n4);
      store_iter<UZ>(seg, z, c.n4);
      for (int j = 0; j + 1 < a.ckpt; ++j) {
        draw_iter(a, c, p, k0 + j, sidx, sb, siv);
        __syncthreads();
        forward_step<UZ>(a, c, sidx, sb, siv, z, red);
        store_iter<UZ>(seg + (size_t)(j + 1) * a.x_stride, z, c.n4);
        __syncthreads();
      }
      // reverse sweep over the segment
      for (int j = a.ckpt - 1; j >= 0; --j) {
        const int k = k0 + j;
        load_iter<UZ>(seg + (size_t)j * a.x_stride, z, c.n4);
        draw_iter(a, c, p, k, sidx, sb, siv);
        __syncthreads();
        float4 x[UZ], xb[UZ];
#pragma unroll
        for (int r = 0; r < UZ; ++r) {
          x[r] = soft_shrink4(z[r], c.lam);
          xb[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int s0 = 0; s0 < a.eta; s0 += UB) {
          float4 av[UB][UZ];
          float pd[2][UB];
#pragma unroll
          for (int u = 0; u < UB; ++u) {
            const int s = s0 + u;
            pd[0][u] = 0.f;
            pd[1][u] = 0.f;
            const float4* row = reinterpret_cast<const float4*>(
                c.Ap + (int64_t)(s < a.eta ? sidx[s] : 0) * c.lda);
#pragma unroll
            for (int r = 0; r < UZ; ++r) {
              const int64_t col = tid + (int64_t)UT * r;
              float4 v = (s < a.eta && col < c.n4) ? __ldg(row + col)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
              if (col == c.n4 - 1) v = mask_tail(v, col, c.n);
              av[u][r] = v;
            }
          }
#pragma unroll
          for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int r = 0; r < UZ; ++r) {
              pd[0][u] += dot4(av[u][r], x[r]);
              pd[1][u] += dot4(av[u][r], g[r]);
            }
          float tot[2][UB];
          block_sum_rows<2>(pd, red, tot);
#pragma unroll
          for (int u = 0; u < UB; ++u) {
            const int s = s0 + u;
            if (s < a.eta) {
              const float rs = tot[0][u] - sb[s];
              const float dg = tot[1][u];
              const float us = c.coef * dg * siv[s];
              if (tid == 0) {
                atomicAdd(gbp + sidx[s], us);
                gt -= rs * siv[s] * dg / (float)a.eta;
              }
#pragma unroll
              for (int r = 0; r < UZ; ++r) {
                xb[r].x = fmaf(-us, av[u][r].x, xb[r].x);
                xb[r].y = fmaf(-us, av[u][r].y, xb[r].y);
                xb[r].z = fmaf(-us, av[u][r].z, xb[r].z);
                xb[r].w = fmaf(-us, av[u][r].w, xb[r].w);
              }
            }
          }
        }
        // dL/dlambda and dL/dz_k
#pragma unroll
        for (int r = 0; r < UZ; ++r) {
          const int64_t col = tid + (int64_t)UT * r;
          if (col < c.n4) {
            const float4 xv = mask_tail(xb[r], col, c.n);
            const float sx = neg_sign_mask(z[r].x, c.lam), sy = neg_sign_mask(z[r].y, c.lam);
            const float sz = neg_sign_mask(z[r].z, c.lam), sw = neg_sign_mask(z[r].w, c.lam);
            glam += xv.x * sx + xv.y * sy + xv.z * sz + xv.w * sw;
            if (sx != 0.f) g[r].x += xv.x;
            if (sy != 0.f) g[r].y += xv.y;
            if (sz != 0.f) g[r].z += xv.z;
            if (sw != 0.f) g[r].w += xv.w;
          }
        }
        __syncthreads();
      }
    }
    // reduce dL/dlambda over the CTA; dL/dt lives in thread 0
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) glam += __shfl_xor_sync(0xffffffffu, glam, o);
    if (lane == 0) sfin[0][warp] = glam;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int w = 0; w < UW; ++w) s += sfin[0][w];
      a.glam[p] = s;
      a.gt[p] = gt;
    }
    __syncthreads();
  }
}

// tau_k of every problem and iteration (index contract, counter word 3 = p)
// and 1/||a||^2 at the drawn rows: drawn once at setup, replayed by the
// forward, the recomputation and the reverse sweep.
__global__ void unrolled_presample_kernel(UnrolledArgs a) {
  const int npairs = (a.eta + 1) >> 1;
  const int64_t per_p = (int64_t)a.K * npairs;
  const int64_t total = per_p * a.P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / per_p);
    const int64_t r = e - (int64_t)p * per_p;
    const int k = (int)(r / npairs);
    const int q = (int)(r - (int64_t)k * npairs);
    const int64_t ro = a.row_off[p];
    int32_t i0, i1;
    draw_pair(a.seed, k, (uint32_t)q, (uint32_t)p, a.thr + ro, a.alias + ro, (uint32_t)a.m[p], &i0,
              &i1);
    const int64_t base = ((int64_t)p * a.K + k) * a.eta;
    a.tidx[base + 2 * q] = i0;
    a.tiv[base + 2 * q] = a.inv_nu[ro + i0];
    if (2 * q + 1 < a.eta) {
      a.tidx[base + 2 * q + 1] = i1;
      a.tiv[base + 2 * q + 1] = a.inv_nu[ro + i1];
    }
  }
}

// b at tau_k for the b of this forward.
__global__ void unrolled_gather_b_kernel(UnrolledArgs a) {
  const int64_t per_p = (int64_t)a.K * a.eta;
  const int64_t total = per_p * a.P;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / per_p);
    a.tb[e] = a.b[a.b_off[p] + a.tidx[e]];
  }
}

__global__ void unrolled_norms_kernel(UnrolledArgs a, double* nu, float* inv_nu, int* pstat) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int p = blockIdx.x; p < a.P; p += gridDim.x) {
    const int m = a.m[p], n = a.n[p];
    const float* Ap = a.A + a.a_off[p];
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
        if (!finite || !isfinite(acc))
          atomicCAS(pstat + p, kStatusOk, kStatusNonFinite);
        else if (acc == 0.0)
          atomicCAS(pstat + p, kStatusOk, kStatusZeroRow);
        nu[ro + i] = acc;
        inv_nu[ro + i] = (acc > 0.0) ? (float)__ddiv_rn(1.0, acc) : 0.0f;
      }
    }
  }
}

__global__ void unrolled_alias_kernel(UnrolledArgs a, const double* nu, double* q, int32_t* stk,
                                      uint32_t* thr, int32_t* alias, const int* pstat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P || pstat[p] != kStatusOk) return;
  const int m = a.m[p];
  const int64_t ro = a.row_off[p];
  double w = 0.0;
  for (int i = 0; i < m; ++i) w = __dadd_rn(w, nu[ro + i]);
  const double md = (double)m;
  for (int i = 0; i < m; ++i) q[ro + i] = __ddiv_rn(__dmul_rn(nu[ro + i], md), w);
  vose_sequential<int32_t>(q + ro, stk + ro, m, thr + ro, alias + ro);
}

// ---------------------------------------------------------------------------
// Row form (n <= 1024, eta <= 256): every row is consumed whole by one warp.
// Warp w takes rows s = w, w + 8, ... of each tau_k; lane l owns float4
// columns l + 32 j of x (and g in the adjoint) and of its share of the update
// in registers, and streams its own columns of its rows into its warp's slot
// ring with 16-byte cp.async (it reads back only what it copied, so the ring
// needs no barrier).  The dots are warp shuffles; the warps' shares of the
// update meet in shared memory once per iteration (two barriers).  tau_k, b
// and 1/||a||^2 come from arrays filled once (tau) and per forward (b); the
// next iteration's entries are loaded during the current one.
// ---------------------------------------------------------------------------
constexpr int RW_ETA = 256;                              // largest eta of the row form
constexpr int RW_N4 = 256;                               // largest n/4 of the row form
constexpr size_t RW_VEC = (size_t)RW_N4 * 16;            // bytes of one vector
constexpr size_t RW_RING = 21 * 1024;                    // row slots of one warp
constexpr int RW_NVEC = 5 + (UW - 1);                    // z, x, two update buffers, g, and
                                                         // the update shares of warps 1..UW-1
constexpr size_t RW_SMEM = RW_NVEC * RW_VEC + UW * RW_RING;
constexpr int RW_RS_MAX = 8;

struct RowIdx {
  int32_t idx[2][RW_ETA];
  float b[2][RW_ETA];
  float iv[2][RW_ETA];
};

__device__ __forceinline__ void ucp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

__device__ __forceinline__ void ucp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void ucp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void ucp_wait_pending(int pending) {
  switch (pending) {
#define RSKA_UWG(N) \
  case N:           \
    asm volatile("cp.async.wait_group " #N ";" ::: "memory"); \
    break;
    RSKA_UWG(0) RSKA_UWG(1) RSKA_UWG(2) RSKA_UWG(3) RSKA_UWG(4) RSKA_UWG(5) RSKA_UWG(6)
    RSKA_UWG(7)
#undef RSKA_UWG
    default:
      asm volatile("cp.async.wait_all;" ::: "memory");
      break;
  }
}

// Barrier over the CTAs of the cluster (release/acquire: shared-memory writes
// before it are visible to the peer CTA after it); a CTA barrier when CL = 1.
template <int CL>
__device__ __forceinline__ void cl_sync() {
  if constexpr (CL == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
  }
}

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// The same shared-memory float4 in CTA `peer` of the cluster.
__device__ __forceinline__ float4 ld_peer(const float4* p, uint32_t peer) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(ra)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(peer));
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(ra)
               : "memory");
  return v;
}

// Entries (index, b, 1/||a||^2) of iteration k of problem p, one per thread.
__device__ __forceinline__ void fetch_entry(const UnrolledArgs& a, int p, int k, int32_t& idx,
                                            float& bv, float& iv) {
  const int s = threadIdx.x;
  if (s < a.eta) {
    const int64_t e = ((int64_t)p * a.K + k) * a.eta + s;
    idx = __ldg(a.tidx + e);
    bv = __ldg(a.tb + e);
    iv = __ldg(a.tiv + e);
  }
}

__device__ __forceinline__ void put_entry(const UnrolledArgs& a, RowIdx& I, int buf, int32_t idx,
                                          float bv, float iv) {
  const int s = threadIdx.x;
  if (s < a.eta) {
    I.idx[buf][s] = idx;
    I.b[buf][s] = bv;
    I.iv[buf][s] = iv;
  }
}

// The rows of one warp in processing order, streamed through its ring.
struct WarpRows {
  unsigned char* ring;
  uint32_t slot_bytes;
  int RS, cw, count;
  int s0, ss;                 // rows s0, s0 + ss, ... of every tau_k
  int iq, ii, islot, cslot;   // next row to issue (iteration position, row), slots
  int allowed;                // iterations whose entries are visible in I
  int64_t issued, t;          // rows issued / consumed by this lane

  template <int NZ>
  __device__ __forceinline__ bool issue(const ProbCtx& c, const RowIdx& I, int lane, int warp) {
    if (cw == 0 || iq >= count || iq > allowed) return false;
    const int32_t row = I.idx[iq & 1][s0 + ss * ii];
    const float4* src = reinterpret_cast<const float4*>(c.Ap + (int64_t)row * c.lda);
    float4* dst = reinterpret_cast<float4*>(ring + (size_t)islot * slot_bytes);
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
      const int col = lane + 32 * j;
      if (col < c.n4) ucp_async16(dst + col, src + col);
    }
    ucp_commit();
    ++issued;
    islot = (islot + 1 == RS) ? 0 : islot + 1;
    if (++ii == cw) {
      ii = 0;
      ++iq;
    }
    return true;
  }

  // make row t resident for this lane and return its slot
  template <int NZ>
  __device__ __forceinline__ const float4* next(const ProbCtx& c, const RowIdx& I, int lane,
                                                int warp) {
    while (issued <= t && issue<NZ>(c, I, lane, warp)) {
    }
    while (issued < t + RS && issue<NZ>(c, I, lane, warp)) {
    }
    const int64_t pend = issued - t - 1;
    ucp_wait_pending(pend < 7 ? (int)pend : 7);
    return reinterpret_cast<const float4*>(ring + (size_t)cslot * slot_bytes);
  }

  __device__ __forceinline__ void advance() {
    ++t;
    cslot = (cslot + 1 == RS) ? 0 : cslot + 1;
  }
};

// Warp w of cluster rank r takes rows s = r UW + w + (UW CL) i.
template <int NZ, int CL>
__device__ __forceinline__ WarpRows make_rows(const UnrolledArgs& a, const ProbCtx& c,
                                              unsigned char* ring, int count, int warp,
                                              int rank) {
  WarpRows w;
  w.ring = ring;
  w.slot_bytes = (uint32_t)c.n4 * 16u;
  w.RS = min(RW_RS_MAX, (int)(RW_RING / w.slot_bytes));
  w.s0 = rank * UW + warp;
  w.ss = UW * CL;
  w.cw = (a.eta > w.s0) ? (a.eta - w.s0 + w.ss - 1) / w.ss : 0;
  w.count = count;
  w.iq = w.ii = w.islot = w.cslot = 0;
  w.allowed = 0;
  w.issued = w.t = 0;
  return w;
}

// One lane's columns of a landed row, copied to registers (its ring slot may
// then be refilled).
template <int NZ>
__device__ __forceinline__ void load_row(const float4* rowp, float4 (&r)[NZ], int lane, int n4,
                                         int64_t n) {
  if (n4 == 32 * NZ && (n & 3) == 0) {  // every lane's every column inside the row (uniform)
#pragma unroll
    for (int j = 0; j < NZ; ++j) r[j] = rowp[lane + 32 * j];
    return;
  }
#pragma unroll
  for (int j = 0; j < NZ; ++j) {
    const int col = lane + 32 * j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col < n4) {
      v = rowp[col];
      if (col == n4 - 1) v = mask_tail(v, col, n);
    }
    r[j] = v;
  }
}

// The update of one step from the warps' shares, without shared-memory
// atomics: warp 0 stores its share into `dcur`, warps 1.. into their own
// buffers `wsh`; after a block barrier every thread sums its columns in warp
// order into `dcur`.  The caller's cluster barrier then publishes `dcur` to
// the peer CTA.
template <int NZ>
__device__ __forceinline__ void merge_shares(float4 (&dl)[NZ], float4* dcur, float4* wsh, int n4) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* dst = (warp == 0) ? dcur : wsh + (size_t)(warp - 1) * RW_N4;
#pragma unroll
  for (int j = 0; j < NZ; ++j) {
    const int col = lane + 32 * j;
    if (col < n4) dst[col] = dl[j];
    dl[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  for (int c4 = tid; c4 < n4; c4 += UT) {
    float4 s = dcur[c4];
#pragma unroll
    for (int w = 1; w < UW; ++w) {
      const float4 v = wsh[(size_t)(w - 1) * RW_N4 + c4];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    dcur[c4] = s;
  }
}

// `count` forward iterations k_begin .. k_begin+count-1 of problem p.  On
// entry zsh/xsh hold z and x = S(z), both update buffers (dsh, dsh + RW_N4)
// are zero and I buffer 0 holds the entries of iteration k_begin, all visible
// to every thread of the cluster.  With CL = 2 the two CTAs of a cluster take
// alternate blocks of 8 rows and add their update shares through
// distributed shared memory; both keep identical z and x.  After local step
// j, z is stored (when `store`) at store_base + ((j+1)/store_every) x_stride
// if store_every divides j+1.  On exit zsh/xsh hold the last iterate and the
// update buffer of the last step is not zero.
template <int NZ, int CL>
__device__ void forward_rows(const UnrolledArgs& a, const ProbCtx& c, int p, RowIdx& I,
                             float4* zsh, float4* xsh, float4* dsh, float4* wsh, unsigned char* ring,
                             int k_begin, int count, float* store_base, int store_every,
                             bool store, int rank) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n4 = (int)c.n4;
  WarpRows W = make_rows<NZ, CL>(a, c, ring, count, warp, rank);
  float4 xr[NZ], dl[NZ];
#pragma unroll
  for (int j = 0; j < NZ; ++j) {
    const int col = lane + 32 * j;
    xr[j] = (col < n4) ? xsh[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    dl[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  while (W.issued < W.RS && W.issue<NZ>(c, I, lane, warp)) {
  }
  // entries run one iteration ahead in registers: those of iteration q + 1
  // are published at the start of iteration q (their buffer held iteration
  // q - 1's, which every warp has left), so the rings stream iteration q + 1's
  // rows during the whole of iteration q
  int32_t nidx = 0;
  float nb = 0.f, niv = 0.f;
  if (1 < count) fetch_entry(a, p, k_begin + 1, nidx, nb, niv);
  for (int q = 0; q < count; ++q) {
    const int buf = q & 1;
    if (q + 1 < count) {
      put_entry(a, I, buf ^ 1, nidx, nb, niv);
      if (q + 2 < count) fetch_entry(a, p, k_begin + q + 2, nidx, nb, niv);
      __syncthreads();
      W.allowed = q + 1;
    }
    // rows in pairs: both are copied to registers as they land, then their
    // dots, reductions and updates interleave (two independent chains)
    for (int i = 0; i < W.cw; i += 2) {
      const bool two = (i + 1 < W.cw);
      float4 r0[NZ], r1[NZ];
      load_row<NZ>(W.next<NZ>(c, I, lane, warp), r0, lane, n4, c.n);
      W.advance();
      if (two) {
        load_row<NZ>(W.next<NZ>(c, I, lane, warp), r1, lane, n4, c.n);
        W.advance();
      } else {
#pragma unroll
        for (int j = 0; j < NZ; ++j) r1[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        p0[j & 3] = fmaf(r0[j].x, xr[j].x, p0[j & 3]);
        p1[j & 3] = fmaf(r1[j].x, xr[j].x, p1[j & 3]);
        p0[j & 3] = fmaf(r0[j].y, xr[j].y, p0[j & 3]);
        p1[j & 3] = fmaf(r1[j].y, xr[j].y, p1[j & 3]);
        p0[j & 3] = fmaf(r0[j].z, xr[j].z, p0[j & 3]);
        p1[j & 3] = fmaf(r1[j].z, xr[j].z, p1[j & 3]);
        p0[j & 3] = fmaf(r0[j].w, xr[j].w, p0[j & 3]);
        p1[j & 3] = fmaf(r1[j].w, xr[j].w, p1[j & 3]);
      }
      float d0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
      float d1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      }
      const int s0 = W.s0 + W.ss * i;
      const float cv0 = c.coef * ((d0 - I.b[buf][s0]) * I.iv[buf][s0]);
      float cv1 = 0.f;
      if (two) {
        const int s1 = s0 + W.ss;
        cv1 = c.coef * ((d1 - I.b[buf][s1]) * I.iv[buf][s1]);
      }
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        dl[j].x = fmaf(cv0, r0[j].x, dl[j].x);
        dl[j].y = fmaf(cv0, r0[j].y, dl[j].y);
        dl[j].z = fmaf(cv0, r0[j].z, dl[j].z);
        dl[j].w = fmaf(cv0, r0[j].w, dl[j].w);
      }
      if (two) {
#pragma unroll
        for (int j = 0; j < NZ; ++j) {
          dl[j].x = fmaf(cv1, r1[j].x, dl[j].x);
          dl[j].y = fmaf(cv1, r1[j].y, dl[j].y);
          dl[j].z = fmaf(cv1, r1[j].z, dl[j].z);
          dl[j].w = fmaf(cv1, r1[j].w, dl[j].w);
        }
      }
    }
    float4* dcur = dsh + (size_t)buf * RW_N4;   // this step's update buffer
    float4* dnext = dsh + (size_t)(buf ^ 1) * RW_N4;
    merge_shares<NZ>(dl, dcur, wsh, n4);
    cl_sync<CL>();
    while (W.issued < W.t + W.RS && W.issue<NZ>(c, I, lane, warp)) {
    }
    const bool st = store && ((q + 1) % store_every) == 0;
    float4* dst = reinterpret_cast<float4*>(store_base + (size_t)((q + 1) / store_every) * a.x_stride);
    for (int c4 = tid; c4 < n4; c4 += UT) {
      float4 zv = zsh[c4];
      float4 dv = dcur[c4];
      if constexpr (CL == 2) {
        const float4 pv = ld_peer(dcur + c4, (uint32_t)(rank ^ 1));
        dv.x += pv.x;
        dv.y += pv.y;
        dv.z += pv.z;
        dv.w += pv.w;
      }
      zv.x -= dv.x;
      zv.y -= dv.y;
      zv.z -= dv.z;
      zv.w -= dv.w;
      zv = mask_tail(zv, c4, c.n);
      zsh[c4] = zv;
      xsh[c4] = soft_shrink4(zv, c.lam);
      dnext[c4] = make_float4(0.f, 0.f, 0.f, 0.f);  // read by the peer one step ago
      if (st) dst[c4] = zv;
    }
    // only this CTA's warps must see the new z and x: the peer's reads of
    // this step's update buffer are ordered before its next overwrite (two
    // steps on) by the next step's cluster barrier
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
      const int col = lane + 32 * j;
      xr[j] = (col < n4) ? xsh[col] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // the peer has finished reading the last step's update buffer before the
  // caller reuses the shared memory
  cl_sync<CL>();
  ucp_wait_all();
}

template <int NZ, int CL>
__global__ void __launch_bounds__(UT, 1) unrolled_fwd_rows_kernel(UnrolledArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RowIdx I;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rank = (CL == 1) ? 0 : (int)cl_rank();
  float4* zsh = reinterpret_cast<float4*>(smem);
  float4* xsh = zsh + RW_N4;
  float4* dsh = xsh + RW_N4;  // two buffers
  float4* wsh = zsh + 5 * RW_N4;  // update shares of warps 1..UW-1
  unsigned char* ring = smem + RW_NVEC * RW_VEC + (size_t)warp * RW_RING;
  const int nck = a.K / a.ckpt;
  for (int p = blockIdx.x / CL; p < a.P; p += gridDim.x / CL) {
    const ProbCtx c = prob_ctx(a, p);
    const int n4 = (int)c.n4;
    float* ck = a.ckpts + (size_t)p * (nck + 1) * a.x_stride;
    for (int c4 = tid; c4 < n4; c4 += UT) {
      zsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      xsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      dsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      dsh[RW_N4 + c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rank == 0) reinterpret_cast<float4*>(ck)[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    {
      int32_t idx = 0;
      float bv = 0.f, iv = 0.f;
      fetch_entry(a, p, 0, idx, bv, iv);
      put_entry(a, I, 0, idx, bv, iv);
    }
    cl_sync<CL>();
    forward_rows<NZ, CL>(a, c, p, I, zsh, xsh, dsh, wsh, ring, 0, a.K, ck, a.ckpt, rank == 0, rank);
    if (rank == 0) {
      float4* xo = reinterpret_cast<float4*>(a.x_out + a.x_off[p]);
      for (int c4 = tid; c4 < n4; c4 += UT) xo[c4] = xsh[c4];
    }
    cl_sync<CL>();
  }
}

// Reverse sweep over one checkpoint segment: iterations k = k0+cnt-1 down to
// k0.  On entry zsh/xsh hold z_{k0+cnt-1} and its shrink, gsh holds
// g = dL/dz_{k0+cnt}, dsh is zero, I buffer 0 holds iteration k0+cnt-1's
// entries.  seg[j] holds z_{k0+j}.  On exit gsh holds dL/dz_{k0}.
template <int NZ, int CL>
__device__ void backward_rows(const UnrolledArgs& a, const ProbCtx& c, int p, RowIdx& I,
                              float4* zsh, float4* xsh, float4* dsh, float4* gsh, float4* wsh,
                              unsigned char* ring, int k0, int cnt, const float* seg, float* gbp,
                              float& glam, float& gt, int rank) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n4 = (int)c.n4;
  // lane 0 adds each row's share of dL/dt; a product with 1/eta keeps a
  // division out of the warp's path (exact when eta is a power of two)
  const float inv_eta = 1.0f / (float)a.eta;
  WarpRows W = make_rows<NZ, CL>(a, c, ring, cnt, warp, rank);
  while (W.issued < W.RS && W.issue<NZ>(c, I, lane, warp)) {
  }
  // entries one step ahead, published at the start of the step before (as in
  // forward_rows)
  int32_t nidx = 0;
  float nb = 0.f, niv = 0.f;
  if (1 < cnt) fetch_entry(a, p, k0 + cnt - 2, nidx, nb, niv);
  for (int q = 0; q < cnt; ++q) {
    const int k = k0 + cnt - 1 - q;
    const int buf = q & 1;
    if (q + 1 < cnt) {
      put_entry(a, I, buf ^ 1, nidx, nb, niv);
      if (q + 2 < cnt) fetch_entry(a, p, k - 2, nidx, nb, niv);
      __syncthreads();
      W.allowed = q + 1;
    }
    // z_{k-1}, which this thread stored during the recompute, is read now so
    // its L2 latency overlaps the rows (n/4 <= UT: column tid is the thread's
    // only one in the update loop below)
    float4 zpre = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q + 1 < cnt && tid < n4)
      zpre = __ldcg(reinterpret_cast<const float4*>(seg + (size_t)(k - 1 - k0) * a.x_stride) + tid);
    float4 xr[NZ], gr[NZ], xb[NZ];
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
      const int col = lane + 32 * j;
      xr[j] = (col < n4) ? xsh[col] : make_float4(0.f, 0.f, 0.f, 0.f);
      gr[j] = (col < n4) ? gsh[col] : make_float4(0.f, 0.f, 0.f, 0.f);
      xb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // rows in pairs, as in forward_rows
    for (int i = 0; i < W.cw; i += 2) {
      const bool two = (i + 1 < W.cw);
      float4 r0[NZ], r1[NZ];
      load_row<NZ>(W.next<NZ>(c, I, lane, warp), r0, lane, n4, c.n);
      W.advance();
      if (two) {
        load_row<NZ>(W.next<NZ>(c, I, lane, warp), r1, lane, n4, c.n);
        W.advance();
      } else {
#pragma unroll
        for (int j = 0; j < NZ; ++j) r1[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;  // <a, x>, <a, g> of the two rows
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        a1 += dot4(r0[j], xr[j]);
        b1 += dot4(r1[j], xr[j]);
        a2 += dot4(r0[j], gr[j]);
        b2 += dot4(r1[j], gr[j]);
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        b1 += __shfl_xor_sync(0xffffffffu, b1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
      }
      const int s0 = W.s0 + W.ss * i;
      const int s1 = s0 + W.ss;
      float u0, u1 = 0.f;
      {
        const float rs = a1 - I.b[buf][s0];
        const float ivs = I.iv[buf][s0];
        u0 = c.coef * a2 * ivs;
        if (lane == 0) {
          atomicAdd(gbp + I.idx[buf][s0], u0);
          gt -= rs * ivs * a2 * inv_eta;
        }
      }
      if (two) {
        const float rs = b1 - I.b[buf][s1];
        const float ivs = I.iv[buf][s1];
        u1 = c.coef * b2 * ivs;
        if (lane == 0) {
          atomicAdd(gbp + I.idx[buf][s1], u1);
          gt -= rs * ivs * b2 * inv_eta;
        }
      }
#pragma unroll
      for (int j = 0; j < NZ; ++j) {
        xb[j].x = fmaf(-u0, r0[j].x, xb[j].x);
        xb[j].y = fmaf(-u0, r0[j].y, xb[j].y);
        xb[j].z = fmaf(-u0, r0[j].z, xb[j].z);
        xb[j].w = fmaf(-u0, r0[j].w, xb[j].w);
      }
      if (two) {
#pragma unroll
        for (int j = 0; j < NZ; ++j) {
          xb[j].x = fmaf(-u1, r1[j].x, xb[j].x);
          xb[j].y = fmaf(-u1, r1[j].y, xb[j].y);
          xb[j].z = fmaf(-u1, r1[j].z, xb[j].z);
          xb[j].w = fmaf(-u1, r1[j].w, xb[j].w);
        }
      }
    }
    float4* dcur = dsh + (size_t)buf * RW_N4;
    float4* dnext = dsh + (size_t)(buf ^ 1) * RW_N4;
    merge_shares<NZ>(xb, dcur, wsh, n4);
    cl_sync<CL>();
    while (W.issued < W.t + W.RS && W.issue<NZ>(c, I, lane, warp)) {
    }
    // dL/dlambda and dL/dz_k = g + mask_k xbar; then z_{k-1} for the next step
    const float4* zprev = reinterpret_cast<const float4*>(seg + (size_t)(k - 1 - k0) * a.x_stride);
    for (int c4 = tid; c4 < n4; c4 += UT) {
      float4 dv = dcur[c4];
      if constexpr (CL == 2) {
        const float4 pv = ld_peer(dcur + c4, (uint32_t)(rank ^ 1));
        dv.x += pv.x;
        dv.y += pv.y;
        dv.z += pv.z;
        dv.w += pv.w;
      }
      const float4 xv = mask_tail(dv, c4, c.n);
      const float4 zv = zsh[c4];
      const float sx = neg_sign_mask(zv.x, c.lam), sy = neg_sign_mask(zv.y, c.lam);
      const float sz = neg_sign_mask(zv.z, c.lam), sw = neg_sign_mask(zv.w, c.lam);
      if (rank == 0) glam += xv.x * sx + xv.y * sy + xv.z * sz + xv.w * sw;
      float4 g = gsh[c4];
      if (sx != 0.f) g.x += xv.x;
      if (sy != 0.f) g.y += xv.y;
      if (sz != 0.f) g.z += xv.z;
      if (sw != 0.f) g.w += xv.w;
      gsh[c4] = g;
      dnext[c4] = make_float4(0.f, 0.f, 0.f, 0.f);  // read by the peer one step ago
      if (q + 1 < cnt) {
        const float4 zp = (c4 == tid) ? zpre : __ldcg(zprev + c4);
        zsh[c4] = zp;
        xsh[c4] = soft_shrink4(zp, c.lam);
      }
    }
    __syncthreads();  // as in forward_rows: the next step's cluster barrier orders the peer
  }
  cl_sync<CL>();  // the peer has finished reading the last step's update buffer
  ucp_wait_all();
}

template <int NZ, int CL>
__global__ void __launch_bounds__(UT, 1) unrolled_bwd_rows_kernel(UnrolledArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RowIdx I;
  __shared__ float sfin[2][UW];
  __shared__ float4 s_gt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = (CL == 1) ? 0 : (int)cl_rank();
  float4* zsh = reinterpret_cast<float4*>(smem);
  float4* xsh = zsh + RW_N4;
  float4* dsh = xsh + RW_N4;       // two buffers
  float4* gsh = dsh + 2 * RW_N4;
  float4* wsh = zsh + 5 * RW_N4;  // update shares of warps 1..UW-1
  unsigned char* ring = smem + RW_NVEC * RW_VEC + (size_t)warp * RW_RING;
  const int nck = a.K / a.ckpt;
  for (int p = blockIdx.x / CL; p < a.P; p += gridDim.x / CL) {
    const ProbCtx c = prob_ctx(a, p);
    const int n4 = (int)c.n4;
    const float* ck = a.ckpts + (size_t)p * (nck + 1) * a.x_stride;
    float* seg = a.segbuf + ((size_t)p * CL + rank) * a.ckpt * a.x_stride;  // this CTA's own
    float* gbp = a.gb + a.b_off[p];
    const float4* gxp = reinterpret_cast<const float4*>(a.gx + a.x_off[p]);
    float glam = 0.f, gt = 0.f;
    // g = dL/dz_K = mask_K dL/dx_K (both CTAs; dL/dlambda counted by rank 0)
    const float4* zK = reinterpret_cast<const float4*>(ck + (size_t)nck * a.x_stride);
    for (int c4 = tid; c4 < n4; c4 += UT) {
      const float4 zv = __ldcg(zK + c4);
      const float4 gxv = mask_tail(__ldg(gxp + c4), c4, c.n);
      const float sx = neg_sign_mask(zv.x, c.lam), sy = neg_sign_mask(zv.y, c.lam);
      const float sz = neg_sign_mask(zv.z, c.lam), sw = neg_sign_mask(zv.w, c.lam);
      if (rank == 0) glam += gxv.x * sx + gxv.y * sy + gxv.z * sz + gxv.w * sw;
      gsh[c4] = make_float4(sx != 0.f ? gxv.x : 0.f, sy != 0.f ? gxv.y : 0.f,
                            sz != 0.f ? gxv.z : 0.f, sw != 0.f ? gxv.w : 0.f);
    }
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
      const int k0 = sgi * a.ckpt;
      // recompute z_{k0} .. z_{k0+ckpt-1} into this CTA's segment buffer
      const float4* zk0 = reinterpret_cast<const float4*>(ck + (size_t)sgi * a.x_stride);
      for (int c4 = tid; c4 < n4; c4 += UT) {
        const float4 zv = __ldcg(zk0 + c4);
        zsh[c4] = zv;
        xsh[c4] = soft_shrink4(zv, c.lam);
        dsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        dsh[RW_N4 + c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(seg)[c4] = zv;
      }
      {
        int32_t idx = 0;
        float bv = 0.f, iv = 0.f;
        fetch_entry(a, p, k0, idx, bv, iv);
        put_entry(a, I, 0, idx, bv, iv);
      }
      cl_sync<CL>();
      forward_rows<NZ, CL>(a, c, p, I, zsh, xsh, dsh, wsh, ring, k0, a.ckpt - 1, seg, 1, true, rank);
      // reverse sweep (zsh/xsh hold z_{k0+ckpt-1})
      {
        int32_t idx = 0;
        float bv = 0.f, iv = 0.f;
        fetch_entry(a, p, k0 + a.ckpt - 1, idx, bv, iv);
        put_entry(a, I, 0, idx, bv, iv);
      }
      for (int c4 = tid; c4 < n4; c4 += UT) {
        dsh[c4] = make_float4(0.f, 0.f, 0.f, 0.f);
        dsh[RW_N4 + c4] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      cl_sync<CL>();
      backward_rows<NZ, CL>(a, c, p, I, zsh, xsh, dsh, gsh, wsh, ring, k0, a.ckpt, seg, gbp, glam, gt,
                            rank);
    }
    // reduce dL/dlambda over the CTA and dL/dt over the warps and the cluster
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) glam += __shfl_xor_sync(0xffffffffu, glam, o);
    if (lane == 0) {
      sfin[0][warp] = glam;
      sfin[1][warp] = gt;
    }
    __syncthreads();
    float sl = 0.f, st = 0.f;
    if (tid == 0) {
      for (int w = 0; w < UW; ++w) {
        sl += sfin[0][w];
        st += sfin[1][w];
      }
      s_gt = make_float4(st, 0.f, 0.f, 0.f);
    }
    cl_sync<CL>();
    if (tid == 0 && rank == 0) {
      if constexpr (CL == 2) st += ld_peer(&s_gt, 1u).x;
      a.glam[p] = sl;
      a.gt[p] = st;
    }
    cl_sync<CL>();
  }
}

}  // namespace
}  // namespace rska

using rska::UnrolledArgs;

struct rska_unrolled {
  int32_t P = 0, eta = 1, K = 0, ckpt = 1;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t rows = 0, x_total = 0, b_total = 0, x_stride = 4;
  int zreg = 1;                 // float4 columns per thread of the widest problem
  std::vector<int64_t> h_x_off;
  const float* A = nullptr;
  int64_t *a_off = nullptr, *lda = nullptr, *b_off = nullptr, *row_off = nullptr,
          *x_off = nullptr;
  int32_t *m = nullptr, *n = nullptr;
  double* nu = nullptr;
  float* inv_nu = nullptr;
  uint32_t* thr = nullptr;
  int32_t* alias = nullptr;
  float *ckpts = nullptr, *segbuf = nullptr;
  int row_nz = 0;               // row form: float4 columns per lane (0: column form)
  int row_cl = 1;               // row form: CTAs (a cluster) per problem
  int32_t* tidx = nullptr;      // row form: tau for every problem and iteration [P][K][eta]
  float *tiv = nullptr, *tb = nullptr;
  // inputs of the last forward, kept for the backward
  const float* b = nullptr;
  const float* lambda = nullptr;
  const float* t = nullptr;
  bool have_forward = false;
};

namespace {

void unrolled_free(rska_unrolled* u) {
  void* ptrs[] = {u->a_off, u->lda,    u->b_off, u->row_off, u->x_off,  u->m,   u->n,
                  u->nu,    u->inv_nu, u->thr,   u->alias,   u->ckpts,  u->segbuf,
                  u->tidx,  u->tiv,    u->tb};
  for (void* p : ptrs) cudaFree(p);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

UnrolledArgs uargs(rska_unrolled* u) {
  UnrolledArgs a;
  std::memset(&a, 0, sizeof(a));
  a.P = u->P;
  a.A = u->A;
  a.a_off = u->a_off;
  a.m = u->m;
  a.n = u->n;
  a.lda = u->lda;
  a.b = u->b;
  a.b_off = u->b_off;
  a.row_off = u->row_off;
  a.inv_nu = u->inv_nu;
  a.thr = u->thr;
  a.alias = u->alias;
  a.x_off = u->x_off;
  a.lambda = u->lambda;
  a.t = u->t;
  a.eta = u->eta;
  a.seed = u->seed;
  a.K = u->K;
  a.ckpt = u->ckpt;
  a.ckpts = u->ckpts;
  a.segbuf = u->segbuf;
  a.x_stride = u->x_stride;
  a.tidx = u->tidx;
  a.tiv = u->tiv;
  a.tb = u->tb;
  return a;
}

// CL CTAs (one cluster) per problem with the row form's shared memory.
template <typename K>
cudaError_t launch_rows(K kernel, rska_unrolled* u, const UnrolledArgs& a, size_t smem, int CL) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(u->P * CL));
  cfg.blockDim = dim3(rska::UT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = u->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kernel, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int CL>
cudaError_t launch_fwd_rows(rska_unrolled* u, const UnrolledArgs& a) {
  const size_t sm = rska::RW_SMEM;
  switch (u->row_nz) {
    case 1: return launch_rows(rska::unrolled_fwd_rows_kernel<1, CL>, u, a, sm, CL);
    case 2: return launch_rows(rska::unrolled_fwd_rows_kernel<2, CL>, u, a, sm, CL);
    case 4: return launch_rows(rska::unrolled_fwd_rows_kernel<4, CL>, u, a, sm, CL);
    default: return launch_rows(rska::unrolled_fwd_rows_kernel<8, CL>, u, a, sm, CL);
  }
}

template <int CL>
cudaError_t launch_bwd_rows(rska_unrolled* u, const UnrolledArgs& a) {
  const size_t sm = rska::RW_SMEM;
  switch (u->row_nz) {
    case 1: return launch_rows(rska::unrolled_bwd_rows_kernel<1, CL>, u, a, sm, CL);
    case 2: return launch_rows(rska::unrolled_bwd_rows_kernel<2, CL>, u, a, sm, CL);
    case 4: return launch_rows(rska::unrolled_bwd_rows_kernel<4, CL>, u, a, sm, CL);
    default: return launch_rows(rska::unrolled_bwd_rows_kernel<8, CL>, u, a, sm, CL);
  }
}

}  // namespace

extern "C" {

int rska_unrolled_setup(rska_unrolled** out, int32_t P, const float* A, const int64_t* a_off,
                        const int64_t* m, const int64_t* n, const int64_t* lda, const int64_t* b_off,
                        int32_t eta, uint64_t seed, int32_t K, int32_t ckpt_every, void* stream) {
  if (!out) return RSKA_EINVAL;
  *out = nullptr;
  if (P < 1 || !A || !a_off || !m || !n || !lda || !b_off || eta < 1 || eta > rska::UMAXETA ||
      K < 1 || ckpt_every < 1 || (K % ckpt_every) != 0 ||
      (reinterpret_cast<uintptr_t>(A) % 16) != 0)
    return RSKA_EINVAL;
  std::vector<int32_t> hm(P), hn(P);
  std::vector<int64_t> row_off(P), x_off(P + 1);
  int64_t rows = 0, xs = 0, bt = 0, maxn4 = 1;
  for (int32_t p = 0; p < P; ++p) {
    if (m[p] < 1 || n[p] < 1 || lda[p] < n[p] || (lda[p] % 4) != 0 || (a_off[p] % 4) != 0 ||
        a_off[p] < 0 || b_off[p] < 0)
      return RSKA_EINVAL;
    const int64_t n4 = (n[p] + 3) / 4;
    if (n4 > (int64_t)rska::UT * rska::kUnrolledMaxZ) return RSKA_EUNSUPPORTED;
    hm[p] = (int32_t)m[p];
    hn[p] = (int32_t)n[p];
    row_off[p] = rows;
    rows += m[p];
    x_off[p] = xs;
    xs += n4 * 4;
    maxn4 = std::max(maxn4, n4);
    bt = std::max(bt, b_off[p] + m[p]);
  }
  x_off[P] = xs;
  rska_unrolled* u = new (std::nothrow) rska_unrolled;
  if (!u) return RSKA_ENOMEM;
  u->P = P;
  u->eta = eta;
  u->K = K;
  u->ckpt = ckpt_every;
  u->seed = seed;
  u->stream = static_cast<cudaStream_t>(stream);
  u->A = A;
  u->rows = rows;
  u->x_total = xs;
  u->b_total = bt;
  u->x_stride = maxn4 * 4;
  {
    const int64_t zr = (maxn4 + rska::UT - 1) / rska::UT;
    u->zreg = zr <= 1 ? 1 : (zr <= 2 ? 2 : 4);
    // row form for n <= 1024 and eta <= 256: float4 columns per lane
    if (maxn4 <= rska::RW_N4 && eta <= rska::RW_ETA) {
      const int64_t nz = (maxn4 + 31) / 32;
      u->row_nz = nz <= 1 ? 1 : (nz <= 2 ? 2 : (nz <= 4 ? 4 : 8));
    }
  }
  u->h_x_off = x_off;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&u->num_sms, cudaDevAttrMultiProcessorCount, dev);
  // two CTAs per problem when the problems fill at most half of the SMs
  if (e == cudaSuccess && u->row_nz && 2 * (int64_t)P <= u->num_sms) u->row_cl = 2;
  const int64_t nck = K / ckpt_every;
  double* q = nullptr;
  int32_t* stk = nullptr;
  int* pstat = nullptr;
  if (e == cudaSuccess &&
      ((e = dalloc(&u->a_off, P)) != cudaSuccess || (e = dalloc(&u->lda, P)) != cudaSuccess ||
       (e = dalloc(&u->b_off, P)) != cudaSuccess || (e = dalloc(&u->row_off, P)) != cudaSuccess ||
       (e = dalloc(&u->x_off, P + 1)) != cudaSuccess || (e = dalloc(&u->m, P)) != cudaSuccess ||
       (e = dalloc(&u->n, P)) != cudaSuccess || (e = dalloc(&u->nu, rows)) != cudaSuccess ||
       (e = dalloc(&u->inv_nu, rows)) != cudaSuccess || (e = dalloc(&u->thr, rows)) != cudaSuccess ||
       (e = dalloc(&u->alias, rows)) != cudaSuccess ||
       (e = dalloc(&u->ckpts, (size_t)P * (nck + 1) * u->x_stride)) != cudaSuccess ||
       (e = dalloc(&u->segbuf, (size_t)P * u->row_cl * ckpt_every * u->x_stride)) != cudaSuccess ||
       (u->row_nz && ((e = dalloc(&u->tidx, (size_t)P * K * eta)) != cudaSuccess ||
                      (e = dalloc(&u->tiv, (size_t)P * K * eta)) != cudaSuccess ||
                      (e = dalloc(&u->tb, (size_t)P * K * eta)) != cudaSuccess)) ||
       (e = dalloc(&q, rows)) != cudaSuccess || (e = dalloc(&stk, rows)) != cudaSuccess ||
       (e = dalloc(&pstat, P)) != cudaSuccess)) {
  }
  cudaStream_t s = u->stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->a_off, a_off, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->lda, lda, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->b_off, b_off, sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->row_off, row_off.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->x_off, x_off.data(), sizeof(int64_t) * (P + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->m, hm.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u->n, hn.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(pstat, 0, sizeof(int) * P, s);
  if (e == cudaSuccess) {
    UnrolledArgs a = uargs(u);
    rska::unrolled_norms_kernel<<<std::min<int>(P, u->num_sms * 8), 256, 0, s>>>(a, u->nu, u->inv_nu,
                                                                                 pstat);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      rska::unrolled_alias_kernel<<<(P + 63) / 64, 64, 0, s>>>(a, u->nu, q, stk, u->thr, u->alias,
                                                               pstat);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && u->row_nz) {
      rska::unrolled_presample_kernel<<<u->num_sms * 8, 256, 0, s>>>(a);
      e = cudaGetLastError();
    }
  }
  std::vector<int> hst(P, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), pstat, sizeof(int) * P, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(q);
  cudaFree(stk);
  cudaFree(pstat);
  if (e != cudaSuccess) {
    unrolled_free(u);
    delete u;
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  for (int32_t p = 0; p < P; ++p)
    if (hst[p] != 0) {
      unrolled_free(u);
      delete u;
      return hst[p];
    }
  *out = u;
  return RSKA_OK;
}

int rska_unrolled_forward(rska_unrolled* u, const float* b, const float* lambda, const float* t,
                          float* x_out) {
  if (!u || !b || !lambda || !t || !x_out) return RSKA_EINVAL;
  u->b = b;
  u->lambda = lambda;
  u->t = t;
  UnrolledArgs a = uargs(u);
  a.x_out = x_out;
  cudaError_t e = cudaSuccess;
  if (u->row_nz) {
    rska::unrolled_gather_b_kernel<<<u->num_sms * 8, 256, 0, u->stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = (u->row_cl == 2) ? launch_fwd_rows<2>(u, a) : launch_fwd_rows<1>(u, a);
  } else {
    const int z = u->zreg;
    if (z == 1)
      rska::unrolled_forward_kernel<1><<<u->P, rska::UT, 0, u->stream>>>(a);
    else if (z == 2)
      rska::unrolled_forward_kernel<2><<<u->P, rska::UT, 0, u->stream>>>(a);
    else
      rska::unrolled_forward_kernel<4><<<u->P, rska::UT, 0, u->stream>>>(a);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return RSKA_ECUDA;
  u->have_forward = true;
  return RSKA_OK;
}

int rska_unrolled_backward(rska_unrolled* u, const float* gx, float* gb, float* glam, float* gt) {
  if (!u || !gx || !gb || !glam || !gt) return RSKA_EINVAL;
  if (!u->have_forward) return RSKA_EINVAL;
  UnrolledArgs a = uargs(u);
  a.gx = gx;
  a.gb = gb;
  a.glam = glam;
  a.gt = gt;
  cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(float) * u->b_total, u->stream);
  if (e == cudaSuccess && u->row_nz) {
    e = (u->row_cl == 2) ? launch_bwd_rows<2>(u, a) : launch_bwd_rows<1>(u, a);
    if (e == cudaSuccess) e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    const int z = u->zreg;
    if (z == 1)
      rska::unrolled_backward_kernel<1><<<u->P, rska::UT, 0, u->stream>>>(a);
    else if (z == 2)
      rska::unrolled_backward_kernel<2><<<u->P, rska::UT, 0, u->stream>>>(a);
    else
      rska::unrolled_backward_kernel<4><<<u->P, rska::UT, 0, u->stream>>>(a);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? RSKA_OK : RSKA_ECUDA;
}

int rska_unrolled_offsets(rska_unrolled* u, int64_t* x_off) {
  if (!u || !x_off) return RSKA_EINVAL;
  std::memcpy(x_off, u->h_x_off.data(), sizeof(int64_t) * (u->P + 1));
  return RSKA_OK;
}

int rska_unrolled_destroy(rska_unrolled* u) {
  if (!u) return RSKA_EINVAL;
  cudaStreamSynchronize(u->stream);
  unrolled_free(u);
  delete u;
  return RSKA_OK;
}

}  // extern "C"
