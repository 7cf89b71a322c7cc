// rska_internal.h -- host-side context and kernel launchers of librska.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rska.h"

namespace rska {

constexpr int kSolveThreads = 512;      // threads per CTA of the persistent solver
constexpr int kMaxEta = 4096;           // largest batch size eta
constexpr int kSolveRegRows = 12;       // row steps a thread may hold in registers
constexpr int kDotBatch = 6;           // row steps whose partial dots are reduced together
constexpr int kAccStride = 32;          // floats between two rows' dot accumulators (128 B)
constexpr int64_t kPresampleDraws = 1 << 21;  // draws pre-sampled per launch (at most)
constexpr int kUnrolledMaxZ = 4;        // unrolled-gradient kernels: float4 columns per thread (n <= 4096)
constexpr int kBatchMaxZ = 3;           // batched kernel: float4 columns per consumer thread (n <= 2688)
constexpr int kRowsMaxZ = 6;            // row-split kernel: float4 columns per consumer thread (n <= 11520)
constexpr int kSmallMaxNZ = 8;          // one-CTA small-system kernel: float4 columns per lane (n <= 1024)
constexpr int kSmallMaxEta = 256;       // ... rows per iteration
constexpr int kSmallMaxSlots = 8;       // ... iterations in its shared-memory ring

// Launch geometry of the persistent single-system solver.
struct SolveGeometry {
  int grid = 0;          // CTAs (one per SM at most; all co-resident)
  int w4max = 0;         // float4 columns of the widest CTA
  int tile_cap = 0;      // float4 elements of the shared-memory row tile
  int rreg = 0;          // row steps held in registers (0 or kSolveRegRows)
  int rows_res = 0;      // rows of tau_k kept on chip by the widest CTA
  size_t smem = 0;       // dynamic shared memory per CTA
};

// Launch geometry of the row-split single-system solver.
struct RowsGeometry {
  int grid = 0;          // CTAs
  int zreg = 0;          // float4 columns per thread
  int slots = 0;         // shared-memory row slots of the TMA ring
  int rowbytes_pad = 0;  // bytes per slot
  size_t smem = 0;
};

// Launch geometry of the one-CTA small-system solver.
struct SmallGeometry {
  int slots = 0;         // iteration slots of the ring (1..kSmallMaxSlots)
  int nz = 0;            // float4 columns per lane (ceil(n4 / 32))
  size_t smem = 0;       // dynamic shared memory
};

struct SolveArgs {
  const float* A;
  int64_t lda;
  int64_t m, n;
  const float* b;
  const float* inv_nu;         // 1/||a_i||^2 in FP32 (from the FP64 norms)
  const uint32_t* thr;
  const int32_t* alias;
  float lambda;
  float coef;                  // t / eta
  int32_t eta;
  uint64_t seed;
  uint32_t problem;
  float* z;                    // x^*, n floats (padded to a multiple of 4)
  float* x;                    // S_lambda(z), n floats (padded)
  float* racc;                 // 3 * eta partial-dot accumulators
  unsigned long long* bar;     // grid barrier arrival counter
  int* status;
  int64_t* kdev;               // iteration counter
  const int* stop;             // nullable: skip the launch when *stop != 0
  const int32_t* tidx;         // pre-sampled tau (K rows of eta4)
  const float* tb;             // b at tau
  const float* tiv;            // 1/||a||^2 at tau
  int64_t tstride;             // entries of tidx/tb/tiv per iteration (eta rounded up to 4);
                               // 0: one fixed list for every iteration (row-split kernel
                               // only, no pre-sampling)
  int64_t K;
  uint64_t limit_ns;
  // one-CTA small-system kernel only: the stopping test of rska_solve_until
  // run inside the launch when xhat is given, every check_every iterations
  // (0: only after the last) and after the last (relative error of
  // x = S_lambda(z) to xhat in FP64 into macc[2], macc[3], macc[5]); at or
  // below tol it sets *stop and k_stop = the iteration count and the launch
  // ends there (the device iteration counter then counts the iterations run)
  const float* xhat = nullptr;
  double* macc = nullptr;
  int64_t* k_stop = nullptr;
  double tol = -1.0;
  int64_t check_every = 0;
};

struct Ctx {
  // problem (borrowed)
  const float* A = nullptr;
  const float* b = nullptr;
  int64_t m = 0, n = 0, lda = 0;
  float lambda = 0.f, t = 1.f;
  int32_t eta = 1;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  // owned device memory
  double* nu = nullptr;
  float* inv_nu = nullptr;
  uint32_t* thr = nullptr;
  int32_t* alias = nullptr;
  float* z = nullptr;
  float* x = nullptr;
  float* racc = nullptr;
  unsigned long long* bar = nullptr;
  int* status = nullptr;
  int64_t* kdev = nullptr;
  int* stop = nullptr;
  double* macc = nullptr;      // metric accumulators and results
  int32_t* tidx = nullptr;     // pre-sampled tau for one launch
  float* tb = nullptr;
  float* tiv = nullptr;
  int64_t chunk = 1;           // iterations per persistent launch (pre-sample capacity)
  void* scratch = nullptr;     // alias-build scratch (q, stack, W), kept for rska_load_host
  float* A_own = nullptr;      // device copies made by rska_setup_host (else null)
  float* b_own = nullptr;
  // host-buffer loads: the copy stream, one event per row chunk, and the
  // timing events of the last setup or load (start, norms done, table done)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t chunk_ev[16] = {};
  cudaEvent_t phase_ev[3] = {};
  double setup_us[4] = {0, 0, 0, 0};  // allocation, copy + norms + W, alias table, whole call
  // host mirrors
  int64_t k_host = 0;
  int sticky = RSKA_OK;
  int grid_override = 0;
  uint64_t limit_ns = 2000000000ull;
  SolveGeometry geom;
  RowsGeometry rgeom;
  SmallGeometry sgeom;
  int kernel_choice = 0;       // 0 automatic, 1 column-split, 2 row-split, 3 one-CTA small
  bool use_rows = false;
  bool use_small = false;
};

// launchers (return cudaError_t of the launch)
cudaError_t launch_row_norms(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                             double* nu, float* inv_nu, int* status, cudaStream_t s);
// sigma_max(A)^2 by `iters` power iterations (rq_out: the last Rayleigh
// quotient; fro2_out: sum of nu); scratch holds sigma_scratch_floats(m, n)
// floats, d2 two doubles.
size_t sigma_scratch_floats(int64_t m, int64_t n);
cudaError_t launch_sigma_max2(const float* A, int64_t m, int64_t n, int64_t lda, const double* nu,
                              int32_t iters, uint64_t seed, float* scratch, double* d2,
                              double* rq_out, double* fro2_out, cudaStream_t s);
cudaError_t launch_w_accumulate(const double* nu, int64_t rows, double* W, cudaStream_t s);
cudaError_t launch_full_sweep(const float* b, int64_t m, int32_t* idx, float* tb, float* tiv,
                              cudaStream_t s);
cudaError_t launch_weights(const double* nu, const float* w, int64_t m, int couple, float* scale,
                           double* rho, int* bad, cudaStream_t s);
cudaError_t launch_alias_build(const double* nu, int64_t m, uint32_t* thr, int32_t* alias,
                               double* q_scratch, int32_t* stack_scratch, int* status,
                               cudaStream_t s,
                               const double* Wpre = nullptr);
cudaError_t launch_indices(const uint32_t* thr, const int32_t* alias, int64_t m, uint64_t seed,
                           uint32_t problem, int64_t k0, int64_t K, int32_t eta, int32_t* out,
                           cudaStream_t s);
bool plan_solve(int64_t n, int32_t eta, int num_sms, int grid_override, size_t smem_optin,
                SolveGeometry* g);
cudaError_t launch_solve(const SolveArgs& a, const SolveGeometry& g, cudaStream_t s);
cudaError_t launch_presample(const SolveArgs& a, cudaStream_t s);
bool plan_rows(int64_t n, int32_t eta, int num_sms, int grid_override, size_t smem_optin,
               RowsGeometry* g);
cudaError_t launch_rows(const SolveArgs& a, const RowsGeometry& g, cudaStream_t s);
// The small-system kernel: n <= 1024, eta <= 256, one iteration of rows in
// shared memory at least; pre-sampled indices (tstride != 0) only.
bool plan_small(int64_t n, int32_t eta, size_t smem_optin, SmallGeometry* g);
cudaError_t launch_small(const SolveArgs& a, const SmallGeometry& g, cudaStream_t s);
cudaError_t launch_metrics(const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
                           const float* z, float lambda, const float* xhat, double* acc,
                           const int* stop, cudaStream_t s);
cudaError_t launch_metrics_finish(double* acc, int use_err, double tol, int* stop,
                                  int64_t* iters_at_stop, const int64_t* kdev, cudaStream_t s);
cudaError_t launch_fill_shrink(float* z, float* x, const float* z_in, int64_t n, int64_t n_pad,
                               float lambda, cudaStream_t s);

}  // namespace rska
