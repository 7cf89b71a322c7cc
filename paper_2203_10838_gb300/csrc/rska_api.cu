// rska_api.cu -- the C ABI of librska (declared in include/rska.h).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <new>

#include "rska_internal.h"

using rska::Ctx;

struct rska_ctx {
  Ctx c;
};

namespace {

int cuda_fail(Ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return RSKA_OK;
  if (c) c->sticky = RSKA_ECUDA;
  return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void free_all(Ctx* c) {
  cudaFree(c->nu);
  cudaFree(c->inv_nu);
  cudaFree(c->thr);
  cudaFree(c->alias);
  cudaFree(c->z);
  cudaFree(c->x);
  cudaFree(c->racc);
  cudaFree(c->A_own);
  cudaFree(c->b_own);
  c->A_own = c->b_own = nullptr;
  cudaFree(c->bar);
  cudaFree(c->status);
  cudaFree(c->kdev);
  cudaFree(c->stop);
  cudaFree(c->macc);
  cudaFree(c->scratch);
  for (cudaEvent_t& ev : c->chunk_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
  for (cudaEvent_t& ev : c->phase_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->copy_stream = nullptr;
  cudaFree(c->tidx);
  cudaFree(c->tb);
  cudaFree(c->tiv);
  c->tidx = nullptr;
  c->tb = c->tiv = nullptr;
  c->nu = nullptr;
  c->inv_nu = nullptr;
  c->thr = nullptr;
  c->alias = nullptr;
  c->z = c->x = c->racc = nullptr;
  c->bar = nullptr;
  c->status = nullptr;
  c->kdev = nullptr;
  c->stop = nullptr;
  c->macc = nullptr;
  c->scratch = nullptr;
}

int64_t n_padded(int64_t n) { return ((n + 3) / 4) * 4; }

// Read the device status word; map it to a return code and make it sticky.
int check_status(Ctx* c) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (st != 0) c->sticky = st;
  return st;
}

int plan(Ctx* c) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) return cuda_fail(c, e);
  const bool col_ok =
      rska::plan_solve(c->n, c->eta, c->num_sms, c->grid_override, (size_t)optin, &c->geom);
  const bool rows_ok =
      rska::plan_rows(c->n, c->eta, c->num_sms, c->grid_override, (size_t)optin, &c->rgeom);
  const bool small_ok = rska::plan_small(c->n, c->eta, (size_t)optin, &c->sgeom);
  c->use_small = false;
  if (c->kernel_choice == 1) {
    if (!col_ok) return RSKA_EUNSUPPORTED;
    c->use_rows = false;
  } else if (c->kernel_choice == 2) {
    if (!rows_ok) return RSKA_EUNSUPPORTED;
    c->use_rows = true;
  } else if (c->kernel_choice == 3) {
    if (!small_ok) return RSKA_EUNSUPPORTED;
    c->use_rows = false;
    c->use_small = true;
  } else {
    if (!col_ok && !rows_ok) return RSKA_EUNSUPPORTED;
    c->use_rows = rows_ok;
    // where the row-split plan is a single CTA, the one-CTA kernel that
    // gives each row to one warp is the faster form
    if (rows_ok && c->rgeom.grid == 1 && small_ok) {
      c->use_rows = false;
      c->use_small = true;
    }
  }
  return RSKA_OK;
}

cudaError_t launch_any(Ctx* c, const rska::SolveArgs& a) {
  if (c->use_small) return rska::launch_small(a, c->sgeom, c->stream);
  return c->use_rows ? rska::launch_rows(a, c->rgeom, c->stream)
                     : rska::launch_solve(a, c->geom, c->stream);
}

rska::SolveArgs solve_args(Ctx* c, int64_t K, const int* stop) {
  rska::SolveArgs a;
  a.A = c->A;
  a.lda = c->lda;
  a.m = c->m;
  a.n = c->n;
  a.b = c->b;
  a.inv_nu = c->inv_nu;
  a.thr = c->thr;
  a.alias = c->alias;
  a.lambda = c->lambda;
  a.coef = c->t / (float)c->eta;
  a.eta = c->eta;
  a.seed = c->seed;
  a.problem = 0;
  a.z = c->z;
  a.x = c->x;
  a.racc = c->racc;
  a.bar = c->bar;
  a.status = c->status;
  a.kdev = c->kdev;
  a.stop = stop;
  a.tidx = c->tidx;
  a.tb = c->tb;
  a.tiv = c->tiv;
  a.tstride = (c->eta + 3) / 4 * 4;
  a.K = K;
  a.limit_ns = c->limit_ns;
  return a;
}

}  // namespace

namespace {

constexpr int kLoadChunks = 16;  // row chunks of a host-buffer load

double host_us_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

// Row norms and the alias table of the context's problem (Definition 1,
// Sec. 5 v1/v2), z = 0, k = 0, status cleared.  With A_host set, A and b are
// first copied from host buffers into the context's own device copies: b,
// then A in row chunks on the copy stream, each chunk's norms and its part of
// W following on the context's stream as soon as it has landed.  Records the
// device time of the copy + norms + W phase and of the alias construction.
int load_impl(Ctx* c, const float* A_host, const float* b_host) {
  const int64_t m = c->m, n = c->n, lda = c->lda;
  const int64_t np = n_padded(n);
  cudaStream_t s = c->stream;
  double* q = static_cast<double*>(c->scratch);
  int32_t* stk = reinterpret_cast<int32_t*>(q + m);
  double* Wdev = reinterpret_cast<double*>(stk + m + (m & 1));  // 8-byte aligned past the stack
  cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->kdev, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stop, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->macc, 0, 8 * sizeof(double), s);
  if (e == cudaSuccess) e = rska::launch_fill_shrink(c->z, c->x, nullptr, n, np, c->lambda, s);
  if (A_host == nullptr) {
    if (e == cudaSuccess) e = cudaEventRecord(c->phase_ev[0], s);
    if (e == cudaSuccess)
      e = rska::launch_row_norms(c->A, m, n, lda, c->b, c->nu, c->inv_nu, c->status, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->phase_ev[1], s);
    if (e == cudaSuccess)
      e = rska::launch_alias_build(c->nu, m, c->thr, c->alias, q, stk, c->status, s);
  } else {
    cudaStream_t cs = c->copy_stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(Wdev, 0, sizeof(double), s);
    // the copy stream starts after the context's stream has reached this point
    // (a previous solve may still read the device copies)
    if (e == cudaSuccess) e = cudaEventRecord(c->phase_ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, c->phase_ev[0], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->b_own, b_host, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, cs);
    const int64_t rows = (m + kLoadChunks - 1) / kLoadChunks;
    for (int k = 0; k < kLoadChunks && e == cudaSuccess; ++k) {
      const int64_t r0 = (int64_t)k * rows;
      if (r0 >= m) break;
      const int64_t r = std::min<int64_t>(rows, m - r0);
      e = cudaMemcpyAsync(c->A_own + r0 * lda, A_host + r0 * lda,
                          sizeof(float) * (size_t)r * (size_t)lda, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess) e = cudaEventRecord(c->chunk_ev[k], cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->chunk_ev[k], 0);
      if (e == cudaSuccess)
        e = rska::launch_row_norms(c->A_own + r0 * lda, r, n, lda, c->b_own + r0, c->nu + r0,
                                   c->inv_nu + r0, c->status, s);
      if (e == cudaSuccess) e = rska::launch_w_accumulate(c->nu + r0, r, Wdev, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->phase_ev[1], s);
    if (e == cudaSuccess)
      e = rska::launch_alias_build(c->nu, m, c->thr, c->alias, q, stk, c->status, s, Wdev);
  }
  if (e == cudaSuccess) e = cudaEventRecord(c->phase_ev[2], s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && c->copy_stream) e = cudaStreamSynchronize(c->copy_stream);
  if (e != cudaSuccess) return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  float ms01 = 0.f, ms12 = 0.f;
  if (cudaEventElapsedTime(&ms01, c->phase_ev[0], c->phase_ev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&ms12, c->phase_ev[1], c->phase_ev[2]) == cudaSuccess) {
    c->setup_us[1] = 1000.0 * ms01;
    c->setup_us[2] = 1000.0 * ms12;
  }
  c->k_host = 0;
  c->sticky = RSKA_OK;
  return check_status(c);
}

}  // namespace

namespace {

// rska_setup and rska_setup_host: with A_host set, the library allocates the
// device copies of A and b and overlaps their host-to-device copy (row
// chunks on a second stream) with the row norms and the ascending sum of W
// over the chunks that have landed.
int setup_impl(rska_ctx** out, const float* A, const float* b, const float* A_host,
               const float* b_host, int64_t m, int64_t n, int64_t lda, float lambda,
               int32_t eta, float t, uint64_t seed, void* stream) {
  const auto t_call = std::chrono::steady_clock::now();
  rska_ctx* h = new (std::nothrow) rska_ctx;
  if (!h) return RSKA_ENOMEM;
  Ctx* c = &h->c;
  c->m = m;
  c->n = n;
  c->lda = lda;
  c->lambda = lambda;
  c->t = t;
  c->eta = eta;
  c->seed = seed;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete h;
    return RSKA_ECUDA;
  }
  int rc = plan(c);
  if (rc != RSKA_OK) {
    delete h;
    return rc;
  }
  const int64_t np = n_padded(n);
  const int64_t eta4 = (eta + 3) / 4 * 4;
  c->chunk = rska::kPresampleDraws / eta4;
  if (c->chunk < 1) c->chunk = 1;
  if ((e = dalloc(&c->nu, m)) != cudaSuccess || (e = dalloc(&c->inv_nu, m)) != cudaSuccess ||
      (e = dalloc(&c->thr, m)) != cudaSuccess || (e = dalloc(&c->alias, m)) != cudaSuccess ||
      (e = dalloc(&c->z, np)) != cudaSuccess || (e = dalloc(&c->x, np)) != cudaSuccess ||
      (e = dalloc(&c->racc, 3 * std::max<size_t>((size_t)eta * rska::kAccStride, (size_t)np))) !=
          cudaSuccess ||
      (e = dalloc(&c->bar, 1)) != cudaSuccess || (e = dalloc(&c->status, 1)) != cudaSuccess ||
      (e = dalloc(&c->kdev, 1)) != cudaSuccess || (e = dalloc(&c->stop, 1)) != cudaSuccess ||
      (e = dalloc(&c->macc, 8)) != cudaSuccess ||
      (e = dalloc(&c->tidx, (size_t)c->chunk * eta4)) != cudaSuccess ||
      (e = dalloc(&c->tb, (size_t)c->chunk * eta4)) != cudaSuccess ||
      (e = dalloc(&c->tiv, (size_t)c->chunk * eta4)) != cudaSuccess ||
      (e = cudaMalloc(&c->scratch, (size_t)m * (sizeof(double) + sizeof(int32_t)) + 16)) !=
          cudaSuccess ||
      (A_host != nullptr && ((e = dalloc(&c->A_own, (size_t)m * (size_t)lda)) != cudaSuccess ||
                             (e = dalloc(&c->b_own, m)) != cudaSuccess))) {
    free_all(c);
    delete h;
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  c->A = A_host ? c->A_own : A;
  c->b = A_host ? c->b_own : b;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->phase_ev[k]);
  if (A_host != nullptr) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < kLoadChunks && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&c->chunk_ev[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_all(c);
    delete h;
    return RSKA_ECUDA;
  }
  c->setup_us[0] = host_us_since(t_call);
  rc = load_impl(c, A_host, b_host);
  if (rc != RSKA_OK) {
    free_all(c);
    delete h;
    return rc;
  }
  c->setup_us[3] = host_us_since(t_call);
  *out = h;
  return RSKA_OK;
}

bool setup_args_ok(int64_t m, int64_t n, int64_t lda, int32_t eta, float lambda, float t) {
  return m >= 1 && n >= 1 && lda >= n && (lda % 4) == 0 && m <= 0x7fffffffLL && eta >= 1 &&
         eta <= rska::kMaxEta && lambda >= 0.f && std::isfinite(lambda) && t > 0.f &&
         std::isfinite(t);
}

}  // namespace

extern "C" {

const char* rska_strerror(int code) {
  switch (code) {
    case RSKA_OK: return "ok";
    case RSKA_EINVAL: return "invalid argument";
    case RSKA_EZEROROW: return "matrix has a zero row";
    case RSKA_ENONFINITE: return "matrix or right-hand side holds Inf or NaN";
    case RSKA_ENOMEM: return "device allocation failed";
    case RSKA_ECUDA: return "CUDA runtime error";
    case RSKA_ETIMEOUT: return "device-side wait timed out";
    case RSKA_EUNSUPPORTED: return "problem outside the library's limits";
    default: return "unknown error";
  }
}


int rska_setup(rska_ctx** out, const float* A, int64_t m, int64_t n, int64_t lda, const float* b,
               float lambda, int32_t eta, float t, uint64_t seed, void* stream) {
  if (out == nullptr) return RSKA_EINVAL;
  *out = nullptr;
  if (A == nullptr || b == nullptr || (reinterpret_cast<uintptr_t>(A) % 16) != 0 ||
      !setup_args_ok(m, n, lda, eta, lambda, t))
    return RSKA_EINVAL;
  return setup_impl(out, A, b, nullptr, nullptr, m, n, lda, lambda, eta, t, seed, stream);
}

int rska_setup_host(rska_ctx** out, const float* A_host, int64_t m, int64_t n, int64_t lda,
                    const float* b_host, float lambda, int32_t eta, float t, uint64_t seed,
                    void* stream) {
  if (out == nullptr) return RSKA_EINVAL;
  *out = nullptr;
  if (A_host == nullptr || b_host == nullptr || !setup_args_ok(m, n, lda, eta, lambda, t))
    return RSKA_EINVAL;
  return setup_impl(out, nullptr, nullptr, A_host, b_host, m, n, lda, lambda, eta, t, seed,
                    stream);
}

int rska_solve(rska_ctx* h, int64_t K) {
  if (!h || K < 0) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky) return c->sticky;
  for (int64_t done = 0; done < K; done += c->chunk) {
    const int64_t Kc = (K - done < c->chunk) ? (K - done) : c->chunk;
    rska::SolveArgs a = solve_args(c, Kc, nullptr);
    cudaError_t e = launch_any(c, a);
    if (e != cudaSuccess) return cuda_fail(c, e);
    c->k_host += Kc;
  }
  return RSKA_OK;
}

int rska_solve_until(rska_ctx* h, int64_t max_iters, int64_t check_every, double tol,
                     const float* xhat, int64_t* iters_out, double* metric_out) {
  if (!h || max_iters < 0 || check_every < 1) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky) return c->sticky;
  cudaStream_t s = c->stream;
  const int64_t k_start = c->k_host;
  cudaError_t e = cudaMemsetAsync(c->stop, 0, sizeof(int), s);
  int64_t* k_stop = reinterpret_cast<int64_t*>(c->macc + 6);
  if (e == cudaSuccess) e = cudaMemsetAsync(k_stop, 0xff, sizeof(int64_t), s);
  const int64_t step = (check_every < c->chunk) ? check_every : c->chunk;
  // The one-CTA small-system kernel runs the test against xhat itself every
  // `step` iterations and ends its launch at the first test that passes, so
  // one launch covers up to 16 checked chunks; otherwise each chunk is
  // followed by the metrics pass over A and the test.
  const bool fused = c->use_small && xhat != nullptr;
  const int64_t per_launch =
      fused ? step * std::max<int64_t>(1, std::min<int64_t>(16, c->chunk / step)) : step;
  // Enqueue chunk + check pairs in waves; between waves read the stop flag,
  // so a run that stops early does not pay for enqueueing the whole budget.
  int64_t done = 0;
  int64_t wave = 4;
  int stopped = 0;
  while (e == cudaSuccess && done < max_iters && !stopped) {
    for (int64_t w = 0; w < wave && done < max_iters && e == cudaSuccess; ++w) {
      const int64_t K = (max_iters - done < per_launch) ? (max_iters - done) : per_launch;
      rska::SolveArgs a = solve_args(c, K, c->stop);
      if (fused) {
        a.xhat = xhat;
        a.macc = c->macc;
        a.k_stop = k_stop;
        a.tol = tol;
        a.check_every = step;
      }
      e = launch_any(c, a);
      if (e == cudaSuccess && !fused)
        e = rska::launch_metrics(c->A, c->m, c->n, c->lda, c->b, c->z, c->lambda, xhat, c->macc,
                                 c->stop, s);
      if (e == cudaSuccess && !fused)
        e = rska::launch_metrics_finish(c->macc, xhat != nullptr, tol, c->stop, k_stop, c->kdev,
                                        s);
      done += K;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&stopped, c->stop, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (wave < 64) wave *= 2;
  }
  if (e != cudaSuccess) return cuda_fail(c, e);
  double res[2];
  int64_t kd = 0;
  e = cudaMemcpyAsync(res, c->macc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&kd, c->kdev, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e);
  int rc = check_status(c);
  c->k_host = kd;
  if (iters_out) *iters_out = kd - k_start;
  if (metric_out) *metric_out = xhat ? res[1] : res[0];
  return rc;
}

int rska_get_x(rska_ctx* h, float* x_out, float* z_out) {
  if (!h) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky) return c->sticky;
  cudaError_t e = cudaSuccess;
  if (x_out)
    e = cudaMemcpyAsync(x_out, c->x, sizeof(float) * c->n, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && z_out)
    e = cudaMemcpyAsync(z_out, c->z, sizeof(float) * c->n, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  return check_status(c);
}

int rska_set_state(rska_ctx* h, const float* z_in, int64_t k) {
  if (!h || k < 0) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky) return c->sticky;
  cudaError_t e = rska::launch_fill_shrink(c->z, c->x, z_in, c->n, n_padded(c->n), c->lambda,
                                           c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->kdev, &k, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->k_host = k;
  return RSKA_OK;
}

int rska_iteration(rska_ctx* h, int64_t* k_out) {
  if (!h || !k_out) return RSKA_EINVAL;
  *k_out = h->c.k_host;
  return RSKA_OK;
}

int rska_get_indices(rska_ctx* h, int64_t k0, int64_t K, int32_t* out) {
  if (!h || k0 < 0 || K < 0 || (K > 0 && !out)) return RSKA_EINVAL;
  Ctx* c = &h->c;
  cudaError_t e = rska::launch_indices(c->thr, c->alias, c->m, c->seed, 0, k0, K, c->eta, out,
                                       c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_fail(c, e);
}

int rska_get_tables(rska_ctx* h, double* nu_out, uint32_t* thr_out, int32_t* alias_out) {
  if (!h) return RSKA_EINVAL;
  Ctx* c = &h->c;
  cudaError_t e = cudaSuccess;
  if (nu_out)
    e = cudaMemcpyAsync(nu_out, c->nu, sizeof(double) * c->m, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && thr_out)
    e = cudaMemcpyAsync(thr_out, c->thr, sizeof(uint32_t) * c->m, cudaMemcpyDeviceToDevice,
                        c->stream);
  if (e == cudaSuccess && alias_out)
    e = cudaMemcpyAsync(alias_out, c->alias, sizeof(int32_t) * c->m, cudaMemcpyDeviceToDevice,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_fail(c, e);
}

int rska_metrics(rska_ctx* h, const float* xhat, double* rel_res, double* rel_err) {
  if (!h) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky) return c->sticky;
  cudaError_t e = rska::launch_metrics(c->A, c->m, c->n, c->lda, c->b, c->z, c->lambda, xhat,
                                       c->macc, nullptr, c->stream);
  if (e == cudaSuccess)
    e = rska::launch_metrics_finish(c->macc, 0, -1.0, nullptr, nullptr, c->kdev, c->stream);
  double res[2];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res, c->macc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (rel_res) *rel_res = res[0];
  if (rel_err && xhat) *rel_err = res[1];
  return check_status(c);
}

int rska_reset(rska_ctx* h) {
  if (!h) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky == RSKA_ECUDA) return RSKA_ECUDA;
  cudaStream_t s = c->stream;
  cudaError_t e = rska::launch_fill_shrink(c->z, c->x, nullptr, c->n, n_padded(c->n), c->lambda, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->kdev, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stop, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->k_host = 0;
  c->sticky = RSKA_OK;
  return RSKA_OK;
}

int rska_set_weights(rska_ctx* h, const float* w, int couple) {
  if (!h || (couple != 0 && couple != 1)) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky != RSKA_OK) return c->sticky;
  cudaStream_t s = c->stream;
  const int64_t m = c->m;
  // scratch: the new scales, rho, the alias build's q and stack, a flag
  float* scale = nullptr;
  double* rho = nullptr;
  double* q = nullptr;
  int32_t* stk = nullptr;
  int* bad = nullptr;
  cudaError_t e = dalloc(&scale, m);
  if (e == cudaSuccess) e = dalloc(&rho, m);
  if (e == cudaSuccess) e = dalloc(&q, m);
  if (e == cudaSuccess) e = dalloc(&stk, m);
  if (e == cudaSuccess) e = dalloc(&bad, 1);
  auto release = [&]() {
    cudaFree(scale);
    cudaFree(rho);
    cudaFree(q);
    cudaFree(stk);
    cudaFree(bad);
  };
  if (e != cudaSuccess) {
    release();
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  int hbad = 0;
  e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) e = rska::launch_weights(c->nu, w, m, couple, scale, rho, bad, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e);
  }
  if (hbad) {  // nothing has changed
    release();
    return RSKA_EINVAL;
  }
  e = cudaMemcpyAsync(c->inv_nu, scale, sizeof(float) * (size_t)m, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = rska::launch_alias_build(rho, m, c->thr, c->alias, q, stk, c->status, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e);
  return check_status(c);
}

int rska_sigma_max2(rska_ctx* h, int32_t iters, uint64_t seed, double* sigma2_out,
                    double* fro2_out, double* alpha_out) {
  if (!h || !sigma2_out || iters < 1 || iters > 100000) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky != RSKA_OK) return c->sticky;
  cudaStream_t s = c->stream;
  float* scratch = nullptr;
  double* d = nullptr;
  cudaError_t e = dalloc(&scratch, rska::sigma_scratch_floats(c->m, c->n));
  if (e == cudaSuccess) e = dalloc(&d, 4);
  if (e != cudaSuccess) {
    cudaFree(scratch);
    cudaFree(d);
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  double host[2] = {0.0, 0.0};
  e = rska::launch_sigma_max2(c->A, c->m, c->n, c->lda, c->nu, iters, seed, scratch, d, d + 2,
                              d + 3, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, d + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(c, e);
  const double sigma2 = host[0], fro2 = host[1];
  *sigma2_out = sigma2;
  if (fro2_out) *fro2_out = fro2;
  if (alpha_out) {
    const double eta = (double)c->eta;
    *alpha_out = (fro2 > 0.0) ? eta / (1.0 + (eta - 1.0) * sigma2 / fro2) : 0.0;
  }
  return RSKA_OK;
}

int rska_linearized_bregman(rska_ctx* h, int64_t K, double step) {
  if (!h || K < 0 || !(step > 0.0) || !(step < 3.0e38)) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->sticky != RSKA_OK) return c->sticky;
  if (K == 0) return RSKA_OK;
  if (c->m > INT32_MAX) return RSKA_EUNSUPPORTED;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) return cuda_fail(c, e);
  // every row once per iteration: eta = m
  rska::RowsGeometry rg;
  if (!rska::plan_rows(c->n, (int32_t)c->m, c->num_sms, c->grid_override, (size_t)optin, &rg))
    return RSKA_EUNSUPPORTED;
  const int64_t m4 = (c->m + 3) / 4 * 4;
  int32_t* idx = nullptr;
  float* tb = nullptr;
  float* tiv = nullptr;
  int64_t* kscratch = nullptr;
  e = dalloc(&idx, m4);
  if (e == cudaSuccess) e = dalloc(&tb, m4);
  if (e == cudaSuccess) e = dalloc(&tiv, m4);
  if (e == cudaSuccess) e = dalloc(&kscratch, 1);
  auto release = [&]() {
    cudaFree(idx);
    cudaFree(tb);
    cudaFree(tiv);
    cudaFree(kscratch);
  };
  if (e != cudaSuccess) {
    release();
    return (e == cudaErrorMemoryAllocation) ? RSKA_ENOMEM : RSKA_ECUDA;
  }
  cudaStream_t s = c->stream;
  rska::SolveArgs a = solve_args(c, K, nullptr);
  a.eta = (int32_t)c->m;
  a.coef = (float)step;
  a.tidx = idx;
  a.tb = tb;
  a.tiv = tiv;
  a.tstride = 0;
  a.kdev = kscratch;  // the index counter k of the RSKA iteration is not advanced
  e = cudaMemsetAsync(kscratch, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = rska::launch_full_sweep(c->b, c->m, idx, tb, tiv, s);
  if (e == cudaSuccess) e = rska::launch_rows(a, rg, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e);
  return check_status(c);
}

int rska_load_host(rska_ctx* h, const float* A_host, const float* b_host) {
  if (!h || !A_host || !b_host) return RSKA_EINVAL;
  Ctx* c = &h->c;
  if (c->A_own == nullptr) return RSKA_EINVAL;  // not created by rska_setup_host
  if (c->sticky == RSKA_ECUDA) return RSKA_ECUDA;
  const auto t_call = std::chrono::steady_clock::now();
  c->setup_us[0] = 0.0;
  const int rc = load_impl(c, A_host, b_host);
  c->setup_us[3] = host_us_since(t_call);
  return rc;
}

int rska_destroy(rska_ctx* h) {
  if (!h) return RSKA_EINVAL;
  cudaStreamSynchronize(h->c.stream);
  free_all(&h->c);
  delete h;
  return RSKA_OK;
}

int rska_query(rska_ctx* h, int what, int64_t* value_out) {
  if (!h || !value_out) return RSKA_EINVAL;
  const rska::SolveGeometry& g = h->c.geom;
  switch (what) {
    case 0: *value_out = h->c.use_small ? 1 : h->c.use_rows ? h->c.rgeom.grid : g.grid; return RSKA_OK;
    case 1: *value_out = rska::kSolveThreads; return RSKA_OK;
    case 2: *value_out = g.rows_res; return RSKA_OK;
    case 3: *value_out = g.w4max; return RSKA_OK;
    case 4:
      *value_out = (int64_t)(h->c.use_small ? h->c.sgeom.smem
                                            : h->c.use_rows ? h->c.rgeom.smem : g.smem);
      return RSKA_OK;
    case 5: *value_out = g.rreg; return RSKA_OK;
    case 6: *value_out = h->c.use_small ? 3 : h->c.use_rows ? 2 : 1; return RSKA_OK;
    case 7:
    case 8:
    case 9:
    case 10: *value_out = (int64_t)std::llround(h->c.setup_us[what - 7]); return RSKA_OK;
    default: return RSKA_EINVAL;
  }
}

int rska_set_option(rska_ctx* h, int what, int64_t value) {
  if (!h) return RSKA_EINVAL;
  Ctx* c = &h->c;
  switch (what) {
    case 0: {
      if (value < 0 || value > c->num_sms) return RSKA_EINVAL;
      const int old = c->grid_override;
      c->grid_override = (int)value;
      int rc = plan(c);
      if (rc != RSKA_OK) {
        c->grid_override = old;
        plan(c);
      }
      return rc;
    }
    case 1:
      if (value < 0) return RSKA_EINVAL;
      c->limit_ns = (uint64_t)value * 1000ull;
      return RSKA_OK;
    case 2: {
      if (value < 0 || value > 3) return RSKA_EINVAL;
      const int old = c->kernel_choice;
      c->kernel_choice = (int)value;
      int rc = plan(c);
      if (rc != RSKA_OK) {
        c->kernel_choice = old;
        plan(c);
      }
      return rc;
    }
    default:
      return RSKA_EINVAL;
  }
}

}  // extern "C"
