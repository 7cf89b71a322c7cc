// rska_metrics.cu -- FP64 metrics of Sec. 5: relative residual
// ||A x - b|| / ||b|| and relative error ||x - xhat|| / ||xhat|| with
// x = S_lambda(z), plus the device-side stopping test used by
// rska_solve_until (Algorithm 1, "until a stopping criterion is satisfied").
#include "rska_device.cuh"
#include "rska_internal.h"

namespace rska {

// acc[0] = sum (Ax-b)_i^2, acc[1] = sum b_i^2, acc[2] = sum (x-xhat)_j^2,
// acc[3] = sum xhat_j^2; acc[4], acc[5] = the two ratios (finish kernel).
__global__ void metrics_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                               const float* __restrict__ b, const float* __restrict__ z,
                               float lambda, const float* __restrict__ xhat, double* acc,
                               const int* stop) {
  if (stop != nullptr && ld_relaxed_s32(stop) != 0) return;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double rr = 0.0, bb = 0.0, ee = 0.0, hh = 0.0;
  for (int64_t i = warp; i < m; i += nwarps) {
    const float* row = A + i * lda;
    double d = 0.0;
    for (int64_t j = lane; j < n; j += 32)
      d = fma((double)__ldg(row + j), (double)soft_shrink(__ldg(z + j), lambda), d);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) {
      const double bi = (double)__ldg(b + i);
      rr += (d - bi) * (d - bi);
      bb += bi * bi;
    }
  }
  if (xhat != nullptr) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
      const double xj = (double)soft_shrink(__ldg(z + j), lambda);
      const double hj = (double)__ldg(xhat + j);
      ee += (xj - hj) * (xj - hj);
      hh += hj * hj;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
    ee += __shfl_xor_sync(0xffffffffu, ee, o);
    hh += __shfl_xor_sync(0xffffffffu, hh, o);
  }
  __shared__ double part[4][32];
  if (lane == 0) {
    part[0][wib] = rr;
    part[1][wib] = bb;
    part[2][wib] = ee;
    part[3][wib] = hh;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[threadIdx.x][w];
    atomicAdd(acc + threadIdx.x, s);
  }
}

__global__ void metrics_finish_kernel(double* acc, int use_err, double tol, int* stop,
                                      int64_t* iters_at_stop, const int64_t* kdev) {
  if (stop != nullptr && *stop != 0) return;
  const double res = sqrt(acc[0]) / (acc[1] > 0.0 ? sqrt(acc[1]) : 1e-30);
  const double err = sqrt(acc[2]) / (acc[3] > 0.0 ? sqrt(acc[3]) : 1e-30);
  acc[4] = res;
  acc[5] = err;
  if (stop != nullptr && tol >= 0.0) {
    const double v = use_err ? err : res;
    if (v <= tol) {
      *stop = 1;
      if (iters_at_stop != nullptr) *iters_at_stop = *kdev;
    }
  }
}

cudaError_t launch_metrics(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                           const float* z, float lambda, const float* xhat, double* acc,
                           const int* stop, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  int64_t blocks = (m + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  metrics_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, m, n, lda, b, z, lambda, xhat, acc, stop);
  return cudaGetLastError();
}

cudaError_t launch_metrics_finish(double* acc, int use_err, double tol, int* stop,
                                  int64_t* iters_at_stop, const int64_t* kdev, cudaStream_t s) {
  metrics_finish_kernel<<<1, 1, 0, s>>>(acc, use_err, tol, stop, iters_at_stop, kdev);
  return cudaGetLastError();
}

}  // namespace rska
