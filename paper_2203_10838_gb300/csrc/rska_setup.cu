// rska_setup.cu -- one-time setup kernels: FP64 row norms ||a_i||^2
// (Definition 1, matrix D), the alias table for p_i = ||a_i||^2/||A||_F^2
// (Sec. 5, variants v1/v2), index retrieval, and state fill.
#include "rska_alias.cuh"
#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

// One warp per row.  Lane L sums a_ij^2 for j = L mod 32 in ascending j (the
// squares of FP32 values are exact in FP64), then the 32 partials are folded
// pairwise with xor offsets 16, 8, 4, 2, 1; the value lands in every lane.
// Flags a zero row (Algorithm 1 requires a_i != 0) and non-finite A or b.
__global__ void row_norms_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                 const float* __restrict__ b, double* __restrict__ nu,
                                 float* __restrict__ inv_nu, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const float* row = A + i * lda;
    double p = 0.0;
    bool finite = true;
    for (int64_t j = lane; j < n; j += 32) {
      const float a = __ldg(row + j);
      finite = finite && isfinite(a);
      const double ad = (double)a;
      p = __fma_rn(ad, ad, p);  // a*a is exact in FP64, so this equals p + a*a
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) p = __dadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      const float bi = __ldg(b + i);
      if (!finite || !isfinite(bi) || !isfinite(p)) {
        atomicCAS(status, kStatusOk, kStatusNonFinite);
      } else if (p == 0.0) {
        atomicCAS(status, kStatusOk, kStatusZeroRow);
      }
      nu[i] = p;
      inv_nu[i] = (p > 0.0) ? (float)__ddiv_rn(1.0, p) : 0.0f;
    }
  }
}

// One block builds the table: all threads stage nu, thread 0 sums W in
// ascending order, all threads form q_i = (nu_i m) / W, then the block runs
// the Vose construction (parallel partition and thresholds, the pairing loop
// on thread 0).  With use_smem the q and stack arrays live in shared memory
// (stack indices as uint16, so m <= 65536); otherwise in the global scratch.
__global__ void alias_build_kernel(const double* __restrict__ nu, int64_t m, uint32_t* thr,
                                   int32_t* alias, double* gq, int32_t* gstk, const int* status,
                                   int use_smem, const double* Wpre) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sW;
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = (*status != kStatusOk);
  __syncthreads();
  if (sbad) return;
  double* q = use_smem ? reinterpret_cast<double*>(smem) : gq;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) q[i] = nu[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double W = 0.0;
    if (Wpre != nullptr) {
      W = *Wpre;  // the same ascending sum, taken chunk by chunk while A arrived
    } else {
      for (int64_t i = 0; i < m; ++i) W = __dadd_rn(W, q[i]);
    }
    sW = W;
  }
  __syncthreads();
  const double W = sW;
  const double md = (double)m;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) q[i] = __ddiv_rn(__dmul_rn(q[i], md), W);
  __syncthreads();
  if (use_smem)
    vose_block<uint16_t>(q, reinterpret_cast<uint16_t*>(q + m), m, thr, alias);
  else
    vose_block<int32_t>(q, gstk, m, thr, alias);
}

__global__ void indices_kernel(const uint32_t* __restrict__ thr, const int32_t* __restrict__ alias,
                               uint32_t m, uint64_t seed, uint32_t problem, int64_t k0, int64_t K,
                               int32_t eta, int32_t* __restrict__ out) {
  const int64_t npairs = (eta + 1) / 2;
  const int64_t total = K * npairs;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kk = e / npairs;
    const uint32_t q = (uint32_t)(e % npairs);
    int32_t i0, i1;
    draw_pair(seed, k0 + kk, q, problem, thr, alias, m, &i0, &i1);
    int32_t* o = out + kk * eta;
    o[2 * q] = i0;
    if (2 * q + 1 < (uint32_t)eta) o[2 * q + 1] = i1;
  }
}

// z <- z_in (or 0), x <- S_lambda(z); entries n .. n_pad-1 are zero.
__global__ void fill_shrink_kernel(float* __restrict__ z, float* __restrict__ x,
                                   const float* __restrict__ z_in, int64_t n, int64_t n_pad,
                                   float lambda) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float v = (j < n && z_in != nullptr) ? z_in[j] : 0.0f;
    z[j] = v;
    x[j] = soft_shrink(v, lambda);
  }
}

cudaError_t launch_row_norms(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                             double* nu, float* inv_nu, int* status, cudaStream_t s) {
  const int threads = 256;
  int64_t blocks = (m + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  row_norms_kernel<<<(unsigned)blocks, threads, 0, s>>>(A, m, n, lda, b, nu, inv_nu, status);
  return cudaGetLastError();
}

// Row weights w_i of eq. (rska) (the diagonal of W; Sec. 5, variants v3 and
// v4).  scale_i = w_i / nu_i rounded once to FP32 (the factor the solver applies
// to row i's residual; w = NULL gives 1/nu_i, the uniform-weight value), and
// rho_i = nu_i / w_i in FP64 when the sampling is coupled to the weights (v4),
// else nu_i.  A weight that is not finite and positive sets *bad.
__global__ void weights_kernel(const double* __restrict__ nu, const float* __restrict__ w,
                               int64_t m, int couple, float* __restrict__ scale,
                               double* __restrict__ rho, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double p = nu[i];
    double wi = 1.0;
    if (w != nullptr) {
      const float wf = w[i];
      if (!(isfinite(wf) && wf > 0.f)) {
        atomicExch(bad, 1);
      }
      wi = (double)wf;
    }
    scale[i] = (float)__ddiv_rn(wi, p);
    rho[i] = (couple && w != nullptr) ? __ddiv_rn(p, wi) : p;
  }
}

// The index list of a full sweep (every row once, in order) with b at the
// rows and a per-row factor of 1: the linearized Bregman step as one
// iteration of the row-split kernel.
__global__ void full_sweep_kernel(const float* __restrict__ b, int64_t m, int32_t* __restrict__ idx,
                                  float* __restrict__ tb, float* __restrict__ tiv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    idx[i] = (int32_t)i;
    tb[i] = b[i];
    tiv[i] = 1.0f;
  }
}

cudaError_t launch_full_sweep(const float* b, int64_t m, int32_t* idx, float* tb, float* tiv,
                              cudaStream_t s) {
  int64_t blocks = (m + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  full_sweep_kernel<<<(unsigned)blocks, 256, 0, s>>>(b, m, idx, tb, tiv);
  return cudaGetLastError();
}

cudaError_t launch_weights(const double* nu, const float* w, int64_t m, int couple, float* scale,
                           double* rho, int* bad, cudaStream_t s) {
  int64_t blocks = (m + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(nu, w, m, couple, scale, rho, bad);
  return cudaGetLastError();
}

// W += nu[0] + nu[1] + ... in ascending order, one thread (the canonical
// sum of the alias construction, continued over consecutive row chunks)
__global__ void w_accumulate_kernel(const double* __restrict__ nu, int64_t rows, double* W) {
  double w = *W;
  for (int64_t i = 0; i < rows; ++i) w = __dadd_rn(w, nu[i]);
  *W = w;
}

cudaError_t launch_w_accumulate(const double* nu, int64_t rows, double* W, cudaStream_t s) {
  w_accumulate_kernel<<<1, 1, 0, s>>>(nu, rows, W);
  return cudaGetLastError();
}

cudaError_t launch_alias_build(const double* nu, int64_t m, uint32_t* thr, int32_t* alias,
                               double* q_scratch, int32_t* stack_scratch, int* status,
                               cudaStream_t s, const double* Wpre) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t need = (size_t)m * (sizeof(double) + sizeof(uint16_t));
  const int use_smem = (m <= 65536 && need + 64 <= (size_t)optin) ? 1 : 0;
  const size_t smem = use_smem ? need : 0;
  if (use_smem) {
    e = cudaFuncSetAttribute(alias_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  alias_build_kernel<<<1, 256, smem, s>>>(nu, m, thr, alias, q_scratch, stack_scratch, status,
                                          use_smem, Wpre);
  return cudaGetLastError();
}

cudaError_t launch_indices(const uint32_t* thr, const int32_t* alias, int64_t m, uint64_t seed,
                           uint32_t problem, int64_t k0, int64_t K, int32_t eta, int32_t* out,
                           cudaStream_t s) {
  const int64_t total = K * ((eta + 1) / 2);
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  indices_kernel<<<(unsigned)blocks, 256, 0, s>>>(thr, alias, (uint32_t)m, seed, problem, k0, K,
                                                   eta, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_shrink(float* z, float* x, const float* z_in, int64_t n, int64_t n_pad,
                               float lambda, cudaStream_t s) {
  int64_t blocks = (n_pad + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  fill_shrink_kernel<<<(unsigned)blocks, 256, 0, s>>>(z, x, z_in, n, n_pad, lambda);
  return cudaGetLastError();
}

}  // namespace rska
