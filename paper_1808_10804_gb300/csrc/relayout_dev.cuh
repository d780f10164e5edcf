// Device helpers of the relayout kernels (block <-> strided region copies).
#pragma once

#include "bst_internal.h"

namespace bst {

// Division by a runtime constant d >= 1 for numerators below 2^31 with one
// high multiply, an add and a shift (Granlund and Montgomery's round-up
// method): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l.
struct FastDiv {
  uint32_t d, m, l;
  __host__ __device__ void init(uint32_t dd) {
    d = dd;
    l = 0;
    while ((1u << l) < d) ++l;
    m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// Copy the elements [begin, end) of one task (row-major over its shape on
// the contiguous side) between blk and the strided side mat.  Each thread
// handles four elements per pass (indices first, then all loads, then all
// stores), so a warp keeps four loads in flight.
//   dir 0: mat[strided] = blk[contiguous]
//   dir 1: blk[contiguous] = alpha * mat[strided] + beta * blk (beta == 0: overwrite)
template <int kThreads>
__device__ __forceinline__ void relayout_range(const RelTask& t, int begin, int end, double* blk, double* mat,
                                               int dir, double alpha, double beta) {
  const int r = t.rank;
  FastDiv fd[kMaxRank];
  long long ms[kMaxRank];
#pragma unroll
  for (int i = 0; i < kMaxRank; ++i) {
    fd[i].init(i < r ? uint32_t(t.shape[i]) : 1u);
    ms[i] = i < r ? t.mstride[i] : 0;
  }
  constexpr int kU = 4;
  for (int e0 = begin + int(threadIdx.x); e0 < end; e0 += kU * kThreads) {
    long long mo[kU];
    bool ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = e0 + u * kThreads;
      ok[u] = e < end;
      uint32_t rem = uint32_t(ok[u] ? e : 0);
      long long o = t.mat_base;
#pragma unroll
      for (int i = kMaxRank - 1; i >= 0; --i) {
        if (i < r) {
          const uint32_t q = fd[i].div(rem);
          o += (long long)(rem - q * fd[i].d) * ms[i];
          rem = q;
        }
      }
      mo[u] = o;
    }
    double v[kU];
    if (dir == 0) {
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) v[u] = blk[t.blk_off + e0 + u * kThreads];
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) mat[mo[u]] = v[u];
    } else if (alpha == 1.0 && beta == 0.0) {
      // plain gather: no FP64 arithmetic (the FP64 pipe is narrow enough
      // that one multiply per element would cost about as much as its
      // 16 bytes of traffic)
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) v[u] = mat[mo[u]];
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) blk[t.blk_off + e0 + u * kThreads] = v[u];
    } else {
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) {
          v[u] = alpha * mat[mo[u]];
          if (beta != 0.0) v[u] += beta * blk[t.blk_off + e0 + u * kThreads];
        }
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (ok[u]) blk[t.blk_off + e0 + u * kThreads] = v[u];
    }
  }
}

}  // namespace bst
