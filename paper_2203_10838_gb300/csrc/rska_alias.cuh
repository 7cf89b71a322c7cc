// rska_alias.cuh -- sequential Walker/Vose alias-table construction in FP64
// (the canonical order of the index contract in include/rska.h), shared by
// the single-system and the batched setup kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rska {

// Sequential Vose construction in FP64 by one thread (the canonical order of
// the index contract), on q[i] = (nu_i m) / W already in place.  `stk` holds
// both LIFO stacks: "small" grows up from index 0, "large" grows down from
// index m-1; together they never hold more than m entries.
template <typename IdxT>
__device__ void vose_sequential(double* q, IdxT* stk, int64_t m, uint32_t* thr, int32_t* alias) {
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (q[i] < 1.0) {
      stk[ns++] = (IdxT)i;
    } else {
      stk[m - 1 - nl] = (IdxT)i;
      ++nl;
    }
  }
  // The element pushed by a step is popped again by the next step (from the
  // stack it went to), so it is also kept in registers: the next step takes
  // it from there instead of waiting for the shared-memory round trip.  The
  // stacks and q[] are still written, for pops that reach older entries.
  bool s_hot = false, l_hot = false;  // top of small / large cached?
  int64_t s_idx = 0, l_idx = 0;
  double s_q = 0.0, l_q = 0.0;
  while (ns > 0 && nl > 0) {
    int64_t l;
    double ql;
    --ns;
    if (s_hot) {
      l = s_idx;
      ql = s_q;
      s_hot = false;
    } else {
      l = stk[ns];
      ql = q[l];
    }
    --nl;
    int64_t g;
    double qg0;
    if (l_hot) {
      g = l_idx;
      qg0 = l_q;
      l_hot = false;
    } else {
      g = stk[m - 1 - nl];
      qg0 = q[g];
    }
    const double scaled = __dmul_rn(ql, 4294967296.0);
    uint32_t t;
    if (ql <= 0.0) {
      t = 0u;
    } else if (scaled >= 4294967295.0) {
      t = 4294967295u;
    } else {
      t = __double2uint_rz(scaled);
    }
    thr[l] = t;
    alias[l] = (int32_t)g;
    const double qg = __dsub_rn(__dadd_rn(qg0, ql), 1.0);
    q[g] = qg;
    if (qg < 1.0) {
      stk[ns++] = (IdxT)g;
      s_hot = true;
      s_idx = g;
      s_q = qg;
    } else {
      stk[m - 1 - nl] = (IdxT)g;
      ++nl;
      l_hot = true;
      l_idx = g;
      l_q = qg;
    }
  }
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t l = stk[s];
    thr[l] = 4294967295u;
    alias[l] = (int32_t)l;
  }
  for (int64_t s = 0; s < nl; ++s) {
    const int64_t g = stk[m - 1 - s];
    thr[g] = 4294967295u;
    alias[g] = (int32_t)g;
  }
}

}  // namespace rska
