// rska_alias.cuh -- Walker/Vose alias-table construction in FP64 (the
// canonical order of the index contract in include/rska.h), shared by the
// single-system, batched and unrolled setup kernels.
//
// The canonical table.  q_i = (nu_i m) / W.  The "small" list holds the i with
// q_i < 1 in ascending order, the "large" list those with q_i >= 1; both are
// LIFO stacks.  Each step pops l from small and g from large, sets
// alias[l] = g and thr[l] from q_l, replaces q_g by (q_g + q_l) - 1 (two FP64
// roundings) and pushes g back onto small (if q_g < 1) or large.  When one
// stack is empty every remaining entry gets thr = 2^32 - 1, alias = itself.
//
// How it is computed here (same table, fewer dependent operations per step).
// The element pushed by a step is always popped again by the next step, from
// the stack it went to, so the stacks never grow above their initial lists:
// every step pairs the element just pushed (the "hot" one, kept in registers)
// with the next unpopped entry of the other initial list.  The loop therefore
// only walks two read-only lists; it computes both possible sums each step so
// the choice of list waits for no comparison, decides "q < 1" with an integer
// compare of the bit pattern, and leaves thr to a pass after the loop (the
// final q of every element popped as small stays in q[]).  Stack layout:
// small list ascending at stk[0, NS), large list with its r-th element
// (ascending) at stk[m-1-r]; the next small is stk[sp-1], the next large
// stk[m-lp].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rska {

// q < 1 for q >= +0 (all q here are non-negative): the IEEE bit patterns of
// non-negative doubles order like the values.
__device__ __forceinline__ bool vose_small(double q) {
  return __double_as_longlong(q) < 0x3FF0000000000000LL;
}

// thr for a finished small entry with probability mass q in [0, 1).
__device__ __forceinline__ uint32_t vose_threshold(double q) {
  if (q <= 0.0) return 0u;
  const double scaled = __dmul_rn(q, 4294967296.0);
  if (scaled >= 4294967295.0) return 4294967295u;
  return __double2uint_rz(scaled);
}

struct VoseRest {
  int64_t sp;   // unpopped small entries: stk[0, sp)
  int64_t lp;   // unpopped large entries: stk[m-lp, m)
  int64_t hot;  // the element pushed by the last step (-1: no step taken)
};

// The pairing loop, one thread.  Writes alias[l] for every element popped as
// small and the running q of the hot element into q[]; returns what is left.
template <typename IdxT>
__device__ VoseRest vose_pair(double* q, const IdxT* stk, int64_t m, int64_t NS, int64_t NL,
                              int32_t* alias) {
  VoseRest r{NS, NL, -1};
  if (NS == 0 || NL == 0) return r;
  int64_t sp = NS, lp = NL;
  int64_t si = stk[sp - 1], li = stk[m - lp];
  double sq = q[si], lq = q[li];
  // first step: both entries come from the lists
  alias[si] = (int32_t)li;
  double hq = __dsub_rn(__dadd_rn(lq, sq), 1.0);
  int64_t hi = li;
  q[hi] = hq;
  --sp;
  --lp;
  if (sp > 0) {
    si = stk[sp - 1];
    sq = q[si];
  }
  if (lp > 0) {
    li = stk[m - lp];
    lq = q[li];
  }
  bool hs = vose_small(hq);
  while (hs ? (lp > 0) : (sp > 0)) {
    // hot small + next large (l = hot, g = li), or next small + hot large
    // (l = si, g = hot); addition commutes exactly, so either operand order
    // gives the canonical (q_g + q_l) - 1
    const double a = __dsub_rn(__dadd_rn(hq, lq), 1.0);
    const double b = __dsub_rn(__dadd_rn(hq, sq), 1.0);
    if (hs) {
      alias[hi] = (int32_t)li;
      hi = li;
      hq = a;
      --lp;
      if (lp > 0) {
        li = stk[m - lp];
        lq = q[li];
      }
    } else {
      alias[si] = (int32_t)hi;
      hq = b;
      --sp;
      if (sp > 0) {
        si = stk[sp - 1];
        sq = q[si];
      }
    }
    q[hi] = hq;
    hs = vose_small(hq);
  }
  r.sp = sp;
  r.lp = lp;
  r.hot = hi;
  return r;
}

// Whole table by one thread (one problem per thread in the batched and
// unrolled setups), on q[i] = (nu_i m) / W already in place.
template <typename IdxT>
__device__ void vose_sequential(double* q, IdxT* stk, int64_t m, uint32_t* thr, int32_t* alias) {
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (vose_small(q[i])) {
      stk[ns++] = (IdxT)i;
    } else {
      stk[m - 1 - nl] = (IdxT)i;
      ++nl;
    }
  }
  const VoseRest r = vose_pair<IdxT>(q, stk, m, ns, nl, alias);
  // leftovers are marked with q = -1, then every entry gets its threshold
  for (int64_t s = 0; s < r.sp; ++s) q[stk[s]] = -1.0;
  for (int64_t s = m - r.lp; s < m; ++s) q[stk[s]] = -1.0;
  if (r.hot >= 0) q[r.hot] = -1.0;
  for (int64_t i = 0; i < m; ++i) {
    const double qi = q[i];
    if (qi < 0.0) {
      thr[i] = 4294967295u;
      alias[i] = (int32_t)i;
    } else {
      thr[i] = vose_threshold(qi);
    }
  }
}

// Whole table by one block (all threads call it), on q[i] = (nu_i m) / W
// already in place and visible to the block.  The partition is a stable
// compaction over per-thread contiguous segments, the pairing loop runs on
// thread 0, leftovers and thresholds are set by all threads.
template <typename IdxT>
__device__ void vose_block(double* q, IdxT* stk, int64_t m, uint32_t* thr, int32_t* alias) {
  __shared__ int64_t s_cnt[32];
  __shared__ VoseRest s_rest;
  __shared__ int64_t s_ns;
  const int T = blockDim.x;
  const int t = threadIdx.x;
  const int lane = t & 31;
  const int wid = t >> 5;
  const int nw = (T + 31) >> 5;
  const int64_t lo = m * t / T, hi = m * (t + 1) / T;
  int64_t cs = 0;
  for (int64_t i = lo; i < hi; ++i) cs += vose_small(q[i]) ? 1 : 0;
  // exclusive scan of the per-thread counts: within warps, then over warps
  int64_t inc = cs;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31 || t == T - 1) s_cnt[wid] = inc;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int w = 0; w < nw; ++w) {
      const int64_t c = s_cnt[w];
      s_cnt[w] = run;
      run += c;
    }
    s_ns = run;
  }
  __syncthreads();
  int64_t before = s_cnt[wid] + inc - cs;  // smalls with index < lo
  for (int64_t i = lo; i < hi; ++i) {
    if (vose_small(q[i])) {
      stk[before++] = (IdxT)i;
    } else {
      stk[m - 1 - (i - before)] = (IdxT)i;  // i - before = larges with index < i
    }
  }
  __syncthreads();
  if (t == 0) s_rest = vose_pair<IdxT>(q, stk, m, s_ns, m - s_ns, alias);
  __syncthreads();
  const VoseRest r = s_rest;
  for (int64_t s = t; s < r.sp; s += T) q[stk[s]] = -1.0;
  for (int64_t s = m - r.lp + t; s < m; s += T) q[stk[s]] = -1.0;
  if (t == 0 && r.hot >= 0) q[r.hot] = -1.0;
  __syncthreads();
  for (int64_t i = t; i < m; i += T) {
    const double qi = q[i];
    if (qi < 0.0) {
      thr[i] = 4294967295u;
      alias[i] = (int32_t)i;
    } else {
      thr[i] = vose_threshold(qi);
    }
  }
}

}  // namespace rska
