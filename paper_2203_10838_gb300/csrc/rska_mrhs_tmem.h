// rska_mrhs_tmem.h -- launcher of the persistent multi-right-hand-side kernel
// (rska_mrhs_tmem.cu): the iterate Z^T stays in tensor memory for a whole
// launch of `cnt` iterations.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace rska {

struct MrhsTmemArgs {
  const __nv_bfloat16* A;  // m x lda (BF16), read only
  int64_t lda;
  int64_t n;               // columns of A in use
  int64_t n_p;             // n rounded up to 256 (row length of G and Zt)
  int64_t R_p;             // right-hand sides rounded up to 128 (row length of Bt)
  int32_t eta;
  int32_t eta_p;           // eta rounded up to 64, at most 256
  int32_t n_slices;        // n_p / 256
  int32_t r_slices;        // R_p / 128
  int32_t cnt;             // iterations of this launch
  int32_t gather_sched;    // when the helper warps gather the next iteration's rows:
                           // 0 with the residual product (after this CTA's previous
                           // update), 1 as soon as the grid barrier has passed
  const int32_t* idx;      // tau of the cnt iterations, iteration-major, eta each
  const float* inv_nu;     // 1 / ||a_i||^2 (FP32 of the FP64 norms)
  const float* Bt;         // m x R_p: Bt[i][j] = (b_j)_i
  __nv_bfloat16* G;        // 2 x eta_p x n_p: dense copies of A_tau (padding zero)
  float* Zt;               // R_p x n_p: Z^T, read at the start, written at the end
  float* Res;              // 3 x r_slices x eta_p x 128 residual accumulators (per iteration
                           // buffer and right-hand-side slice, blocks of four rows of tau:
                           // element (s, r) at ((s / 4) 128 + r) 4 + s % 4)
  unsigned long long* bar; // grid barrier counter (zero at launch)
  float lambda;
  float coef;              // t / eta
  int nsplit_x;            // terms of X: 2 = BF16 high + low, 1 = high only
  int nsplit_r;            // terms of the scaled residual
  int* status;
  uint64_t limit_ns;
};

// dynamic shared memory of one CTA
size_t mrhs_tmem_smem(int eta_p);
// whether a problem fits the persistent form (eta_p <= 256, one CTA per
// 128 x 256 slice of Z^T, every CTA resident at once)
bool mrhs_tmem_fits(int64_t n_p, int64_t R_p, int64_t eta_p, int num_sms);
// mapG: 2-D map over G (n_p columns, 2 eta_p rows, BF16), box 64 x eta_p,
// 128-byte swizzle
cudaError_t launch_mrhs_tmem(const CUtensorMap& mapG, const MrhsTmemArgs& a, cudaStream_t s);

}  // namespace rska
