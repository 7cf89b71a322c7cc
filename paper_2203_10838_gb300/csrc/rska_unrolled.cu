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
  // inputs of the last forward, kept for the backward
  const float* b = nullptr;
  const float* lambda = nullptr;
  const float* t = nullptr;
  bool have_forward = false;
};

namespace {

void unrolled_free(rska_unrolled* u) {
  void* ptrs[] = {u->a_off, u->lda,   u->b_off, u->row_off, u->x_off,  u->m,     u->n,
                  u->nu,    u->inv_nu, u->thr,  u->alias,   u->ckpts, u->segbuf};
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
  return a;
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
  }
  u->h_x_off = x_off;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&u->num_sms, cudaDevAttrMultiProcessorCount, dev);
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
       (e = dalloc(&u->segbuf, (size_t)P * ckpt_every * u->x_stride)) != cudaSuccess ||
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
  const int z = u->zreg;
  if (z == 1)
    rska::unrolled_forward_kernel<1><<<u->P, rska::UT, 0, u->stream>>>(a);
  else if (z == 2)
    rska::unrolled_forward_kernel<2><<<u->P, rska::UT, 0, u->stream>>>(a);
  else
    rska::unrolled_forward_kernel<4><<<u->P, rska::UT, 0, u->stream>>>(a);
  cudaError_t e = cudaGetLastError();
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
  if (e == cudaSuccess) {
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
