// rska_noalloc.cu -- rska_solve_noalloc: a one-shot RSKA solve that allocates
// no device memory.  Its working memory (row norms, alias table, pre-sampled
// indices, iterate, accumulators, counters) lives in one file-scope device
// array of fixed size; the caller passes only inputs and outputs.
//
// It serves callers that cannot allocate device memory while they run: code
// executing under an external memory budget or a custom allocator that forbids
// cudaMalloc, and code that must not synchronize the device the way
// cudaMalloc/cudaFree may.  The array below is reserved on every GPU that
// loads this library and stays reserved until the process exits.
#include <mutex>

#include "rska_internal.h"

namespace {

// Limits of the allocation-free path (checked on entry).
constexpr int64_t kNaMaxM = 65536;
constexpr int64_t kNaMaxN = 16384;
constexpr int32_t kNaMaxEta = 1024;
constexpr int64_t kNaDraws = 1 << 16;     // pre-sampled draws per launch
constexpr size_t kNaScratchBytes = 4u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Host-side cache of the array's device address, one per device.  In host code
// the name g_noalloc_scratch is only a host stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct NaLayout {
  size_t nu, inv_nu, thr, alias, z, x, racc, bar, status, kdev, tidx, tb, tiv, total;
  size_t alias_q, alias_stk;  // alias-build scratch overlaps the pre-sample buffers
  int64_t chunk;
};

NaLayout layout(int64_t m, int64_t n, int32_t eta) {
  NaLayout L;
  const int64_t n4 = (n + 3) / 4;
  const int64_t eta4 = (eta + 3) / 4 * 4;
  L.chunk = kNaDraws / eta4 > 0 ? kNaDraws / eta4 : 1;
  size_t off = 0;
  L.nu = off;      off = align256(off + sizeof(double) * m);
  L.inv_nu = off;  off = align256(off + sizeof(float) * m);
  L.thr = off;     off = align256(off + sizeof(uint32_t) * m);
  L.alias = off;   off = align256(off + sizeof(int32_t) * m);
  L.z = off;       off = align256(off + sizeof(float) * n4 * 4);
  L.x = off;       off = align256(off + sizeof(float) * n4 * 4);
  const size_t racc_floats =
      3 * ((size_t)eta * rska::kAccStride > (size_t)n4 * 4 ? (size_t)eta * rska::kAccStride
                                                            : (size_t)n4 * 4);
  L.racc = off;    off = align256(off + sizeof(float) * racc_floats);
  L.bar = off;     off = align256(off + sizeof(unsigned long long));
  L.status = off;  off = align256(off + sizeof(int));
  L.kdev = off;    off = align256(off + sizeof(int64_t));
  const size_t ps = off;
  L.tidx = off;    off = align256(off + sizeof(int32_t) * L.chunk * eta4);
  L.tb = off;      off = align256(off + sizeof(float) * L.chunk * eta4);
  L.tiv = off;     off = align256(off + sizeof(float) * L.chunk * eta4);
  L.alias_q = ps;
  L.alias_stk = align256(ps + sizeof(double) * m);
  const size_t alias_end = align256(L.alias_stk + sizeof(int32_t) * m);
  L.total = off > alias_end ? off : alias_end;
  return L;
}

// Device address of g_noalloc_scratch on the current device, looked up once
// per device with that device current.
int scratch_ptr(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RSKA_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_dev_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return RSKA_ECUDA;
    g_dev_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_dev_ptr[dev]);
  return RSKA_OK;
}

}  // namespace

extern "C" int rska_solve_noalloc(const float* A, int64_t m, int64_t n, int64_t lda,
                                  const float* b, float lambda, int32_t eta, float t,
                                  uint64_t seed, int64_t K, float* x_out, float* z_out,
                                  void* stream) {
  if (A == nullptr || b == nullptr || (x_out == nullptr && z_out == nullptr) || m < 1 || n < 1 ||
      lda < n || (lda % 4) != 0 || (reinterpret_cast<uintptr_t>(A) % 16) != 0 || eta < 1 ||
      !(lambda >= 0.f) || !(lambda < 3.0e38f) || !(t > 0.f) || !(t < 3.0e38f) || K < 0)
    return RSKA_EINVAL;
  if (m > kNaMaxM || n > kNaMaxN || eta > kNaMaxEta) return RSKA_EUNSUPPORTED;
  const NaLayout L = layout(m, n, eta);
  if (L.total > kNaScratchBytes) return RSKA_EUNSUPPORTED;

  unsigned char* base = nullptr;
  int rc = scratch_ptr(&base);
  if (rc != RSKA_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return RSKA_ECUDA;
  rska::RowsGeometry rg;
  rska::SolveGeometry cg;
  rska::SmallGeometry sg;
  const bool use_rows = rska::plan_rows(n, eta, sms, 0, (size_t)optin, &rg);
  if (!use_rows && !rska::plan_solve(n, eta, sms, 0, (size_t)optin, &cg)) return RSKA_EUNSUPPORTED;
  // the same automatic choice as a context: the one-CTA kernel where the
  // row-split plan is a single CTA
  const bool use_small = use_rows && rg.grid == 1 && rska::plan_small(n, eta, (size_t)optin, &sg);

  double* nu = reinterpret_cast<double*>(base + L.nu);
  float* inv_nu = reinterpret_cast<float*>(base + L.inv_nu);
  uint32_t* thr = reinterpret_cast<uint32_t*>(base + L.thr);
  int32_t* alias = reinterpret_cast<int32_t*>(base + L.alias);
  float* z = reinterpret_cast<float*>(base + L.z);
  float* x = reinterpret_cast<float*>(base + L.x);
  int* status = reinterpret_cast<int*>(base + L.status);
  int64_t* kdev = reinterpret_cast<int64_t*>(base + L.kdev);
  const int64_t np = (n + 3) / 4 * 4;

  // Every call starts from zeroed state: the array keeps the previous call's contents.
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(kdev, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = rska::launch_fill_shrink(z, x, nullptr, n, np, lambda, s);
  if (e == cudaSuccess) e = rska::launch_row_norms(A, m, n, lda, b, nu, inv_nu, status, s);
  if (e == cudaSuccess)
    e = rska::launch_alias_build(nu, m, thr, alias, reinterpret_cast<double*>(base + L.alias_q),
                                 reinterpret_cast<int32_t*>(base + L.alias_stk), status, s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return RSKA_ECUDA;
  if (st != 0) return st;

  rska::SolveArgs a{};  // every field zero or its default
  a.A = A;
  a.lda = lda;
  a.m = m;
  a.n = n;
  a.b = b;
  a.inv_nu = inv_nu;
  a.thr = thr;
  a.alias = alias;
  a.lambda = lambda;
  a.coef = t / (float)eta;
  a.eta = eta;
  a.seed = seed;
  a.problem = 0;
  a.z = z;
  a.x = x;
  a.racc = reinterpret_cast<float*>(base + L.racc);
  a.bar = reinterpret_cast<unsigned long long*>(base + L.bar);
  a.status = status;
  a.kdev = kdev;
  a.stop = nullptr;
  a.tidx = reinterpret_cast<int32_t*>(base + L.tidx);
  a.tb = reinterpret_cast<float*>(base + L.tb);
  a.tiv = reinterpret_cast<float*>(base + L.tiv);
  a.tstride = (eta + 3) / 4 * 4;
  a.limit_ns = 2000000000ull;
  for (int64_t done = 0; done < K && e == cudaSuccess; done += L.chunk) {
    a.K = (K - done < L.chunk) ? (K - done) : L.chunk;
    e = use_small ? rska::launch_small(a, sg, s)
        : use_rows  ? rska::launch_rows(a, rg, s)
                    : rska::launch_solve(a, cg, s);
  }
  if (e == cudaSuccess && x_out)
    e = cudaMemcpyAsync(x_out, x, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && z_out)
    e = cudaMemcpyAsync(z_out, z, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return RSKA_ECUDA;
  return st;
}
