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
  while (ns > 0 && nl > 0) {
    const int64_t l = stk[--ns];
    --nl;
    const int64_t g = stk[m - 1 - nl];
    const double ql = q[l];
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
    const double qg = __dsub_rn(__dadd_rn(q[g], ql), 1.0);
    q[g] = qg;
    if (qg < 1.0) {
      stk[ns++] = (IdxT)g;
    } else {
      stk[m - 1 - nl] = (IdxT)g;
      ++nl;
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
