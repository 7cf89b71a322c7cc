// rska_sigma.cu -- sigma_max(A)^2 by power iteration on A^T A, and the step
// alpha^*(eta) of Corollary 1 (uniform weights) that needs it.
//
// Each iteration: u = A v (one warp per row), rq = ||u||^2 (the Rayleigh
// quotient for ||v|| = 1, FP64), w = A^T u (row chunks per block, partial sums
// reduced over the chunks in a fixed order), v = w / ||w|| (FP64 norm).
// Products are FP32; norms and the quotient FP64.  Deterministic: no atomics.
#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

namespace {

constexpr int kSigThreads = 256;
constexpr int kSigChunks = 16;  // row chunks of the transposed product

// Start vector: splitmix64 of (seed, j) mapped to [-1, 1), then normalised on
// the host side of the first iteration.
__global__ void sig_init_kernel(float* v, int64_t n, uint64_t seed) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1);
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    v[j] = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

// u_i = <a_i, v>, one warp per row; lane partials folded by xor shuffles.
__global__ void sig_av_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                              const float* __restrict__ v, float* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const float* row = A + i * lda;
    float acc = 0.f;
    for (int64_t j = lane; j < n; j += 32) acc = fmaf(__ldg(row + j), __ldg(v + j), acc);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[i] = acc;
  }
}

// part[c][j] = sum_{i in chunk c} a_ij u_i: block (x, c) covers kSigThreads
// columns of chunk c.
__global__ void sig_atu_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                               const float* __restrict__ u, float* __restrict__ part) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const int64_t rows = (m + kSigChunks - 1) / kSigChunks;
  const int64_t i0 = (int64_t)c * rows;
  const int64_t i1 = (i0 + rows < m) ? i0 + rows : m;
  if (j >= n) return;
  float acc = 0.f;
  for (int64_t i = i0; i < i1; ++i) acc = fmaf(__ldg(A + i * lda + j), __ldg(u + i), acc);
  part[(size_t)c * n + j] = acc;
}

// w_j = sum_c part[c][j] in chunk order.
__global__ void sig_sum_kernel(const float* __restrict__ part, int64_t n, float* __restrict__ w) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < kSigChunks; ++c) s += part[(size_t)c * n + j];
    w[j] = s;
  }
}

// out = sum_j x_j^2 in FP64 by one block (fixed order: strided lanes, then a
// shared-memory tree).
__global__ void sig_norm2_kernel(const float* __restrict__ x, int64_t n, double* out) {
  __shared__ double red[kSigThreads];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double d = (double)x[j];
    s = __fma_rn(d, d, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// v = w / sqrt(*nrm2) (a zero vector stays zero)
__global__ void sig_scale_kernel(const float* __restrict__ w, int64_t n, const double* nrm2,
                                 float* __restrict__ v) {
  const double s = *nrm2;
  const float inv = (s > 0.0) ? (float)(1.0 / sqrt(s)) : 0.f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    v[j] = w[j] * inv;
}

// fro2 = sum_i nu_i (FP64, one block)
__global__ void sig_sum_nu_kernel(const double* __restrict__ nu, int64_t m, double* out) {
  __shared__ double red[kSigThreads];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = __dadd_rn(s, nu[i]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

unsigned grid_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t sigma_scratch_floats(int64_t m, int64_t n) {
  return (size_t)m + 3 * (size_t)n + (size_t)kSigChunks * (size_t)n;
}

cudaError_t launch_sigma_max2(const float* A, int64_t m, int64_t n, int64_t lda, const double* nu,
                              int32_t iters, uint64_t seed, float* scratch, double* d2,
                              double* rq_out, double* fro2_out, cudaStream_t s) {
  float* u = scratch;
  float* v = u + m;
  float* w = v + n;
  float* part = w + n;
  sig_init_kernel<<<grid_for(n, kSigThreads), kSigThreads, 0, s>>>(v, n, seed);
  sig_norm2_kernel<<<1, kSigThreads, 0, s>>>(v, n, d2 + 1);
  sig_scale_kernel<<<grid_for(n, kSigThreads), kSigThreads, 0, s>>>(v, n, d2 + 1, v);
  const dim3 tgrid((unsigned)((n + kSigThreads - 1) / kSigThreads), kSigChunks);
  for (int32_t it = 0; it < iters; ++it) {
    sig_av_kernel<<<grid_for(m * 32, kSigThreads), kSigThreads, 0, s>>>(A, m, n, lda, v, u);
    sig_norm2_kernel<<<1, kSigThreads, 0, s>>>(u, m, rq_out);
    sig_atu_kernel<<<tgrid, kSigThreads, 0, s>>>(A, m, n, lda, u, part);
    sig_sum_kernel<<<grid_for(n, kSigThreads), kSigThreads, 0, s>>>(part, n, w);
    sig_norm2_kernel<<<1, kSigThreads, 0, s>>>(w, n, d2 + 1);
    sig_scale_kernel<<<grid_for(n, kSigThreads), kSigThreads, 0, s>>>(w, n, d2 + 1, v);
  }
  sig_sum_nu_kernel<<<1, kSigThreads, 0, s>>>(nu, m, fro2_out);
  return cudaGetLastError();
}

}  // namespace rska
