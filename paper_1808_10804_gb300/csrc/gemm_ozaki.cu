// FP64-accurate grouped GEMM on the BF16 tensor cores (tcgen05, sm_103a).
//
// Every FP64 row of an operand gets a power-of-two scale 2^e with
// |x| < 2^e; the scaled row is written, with integer arithmetic on the IEEE
// bit pattern, as a signed-digit expansion
//     x / 2^e = 2^-8 (a0 + 2^-9 (a1 + 2^-9 (a2 + 2^-9 (a3 + 2^-9 a4))))
// with integer digits |a_i| <= 256, which BF16 holds exactly (44 bits kept).
// A product of two digits is an integer below 2^16 in magnitude, exact in
// FP32.  The GEMM sums the 15 digit products with i + j <= 4 by diagonal
// d = i + j (weight 2^-16-9d) in tensor memory:
//   * d = 0, 1, 2 are read out every 64 K (two pipeline stages), where their
//     FP32 sums are exact integers of magnitude <= 3 * 2^22 < 2^24, and
//     added into one 64-bit integer per output (K <= 10000 keeps it from
//     overflowing);
//   * d = 3, 4 carry weights <= 2^-27 of the leading term and accumulate in
//     FP32 over the whole K.
// The epilogue forms the result with 64-bit integer arithmetic and one
// conversion to FP64.  Relative error ~2^-40 against the row/column scales.
//
// Kernel: persistent, one CTA per SM walking the plan's 128 x 64 (or
// 128 x 32) output tiles; warp 0 drives TMA (64-byte swizzled K-major tiles,
// a ring of 3 stages for five slices, up to 6 for three), warp 1 issues
// tcgen05.mma from one thread (the 15 digit products of a 16-K step as 8
// products, each an A slice times a run of stacked B slices), warps 2..9
// drain tensor memory.  Every wait of the pipeline
// is bounded by the launch's spin limit: on expiry the kernel records
// BST_E_TIMEOUT in the context's error word and every role leaves its loop;
// before tensor memory is freed and the CTA exits, the TMA copies it has
// issued and the products it has issued are waited for (they always
// complete; those waits carry a separate, much larger bound).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "bst_internal.h"
#include "relayout_dev.cuh"

namespace bst {

namespace oz {

constexpr int kTM = 128;           // tile rows (M)
constexpr int kTK = 32;            // K per stage (64 bytes of BF16)
constexpr int kABytes = kTM * kTK * 2;   // 8 KB per slice
constexpr int kThreads = 320;            // 10 warps: TMA, MMA, 8 epilogue
constexpr long long kSpinLimit = 1ll << 28;   // default bound of a pipeline wait (tries)
constexpr long long kDrainLimit = 1ll << 30;  // bound of the waits for issued copies and products

// Shape of one instantiation: S digit slices per operand (5: the FP64-
// accurate split; 3: 26 bits, the cheaper arithmetic), output tiles of
// 128 x TN (TN = 64, or 32 for narrow problems: twice the tiles).
//   tensor memory: d0, d1, d2 side by side, double-buffered (buffer b at
//   columns 3 TN b), then for S = 5 the whole-K diagonals d3 and d4 (2 TN
//   more, from 6 TN); allocated as the next power of two.
template <int S, int TN>
struct Cfg {
  static_assert(S == 5 || S == 3, "digit slices");
  static_assert(TN == 64 || TN == 32, "tile width");
  static constexpr int kBBytes = TN * kTK * 2;
  static constexpr int kStageBytes = S * (kABytes + kBBytes);
  static constexpr int kStages = (196608 / kStageBytes) < 6 ? (196608 / kStageBytes) : 6;
  static constexpr int kColD3 = 6 * TN;
  static constexpr int kCols = 6 * TN + (S - 3) * TN;
  static constexpr int kTmemCols = kCols <= 256 ? 256 : 512;
  // C = T 2^(ea + eb - kShift): T = S0 2^27 + S1 2^18 + S2 2^9 + S3 + S4 2^-9
  // (S = 5) or S0 2^18 + S1 2^9 + S2 (S = 3)
  static constexpr int kShift = S == 5 ? 43 : 34;
  static constexpr int kTopBits = 9 * S - 1;  // bits of the scaled integer (44 or 26)
};

struct Prob {
  int32_t M, N, K, pad;
  int32_t arow, brow;  // first row of this problem in the split A / B buffers
  int64_t c_off, c_m, c_n;
  // output scatter (scatter != 0): element (m, n) of the problem goes to
  // C[bbase[bb_off + r ncc + c] + mi w + ni] with (r, mi) = rowtab[rt_off + m]
  // and (c, ni, w) = coltab[ct_off + n]: the canonical block (r, c) of the
  // output tensor, row-major [rows of config r x w], instead of a strided
  // sector matrix
  int32_t scatter, ncc;
  int64_t rt_off, ct_off, bb_off;
};

// Output scatter tables of a plan (device pointers; all null for a plain
// strided output) and the epilogue's C = alpha * A B + beta * C.
struct Scatter {
  const int2* rowtab;
  const int4* coltab;
  const long long* bbase;
  double alpha, beta;
};

struct Tile {
  int32_t prob, m0, n0, pad;
};

struct SplitTask {
  int32_t rows, K;
  int32_t row0, pad;  // first row in the split buffer
  int64_t base, s_r, s_k;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false (and raises the abort flag) on expiry or when
// another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                                          long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, int(BST_E_TIMEOUT));
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(1) << 16;                    // leading byte offset (unused with swizzle)
  d |= uint64_t((512 >> 4) & 0x3FFF) << 32;  // stride byte offset
  d |= uint64_t(1) << 46;                    // descriptor version
  d |= uint64_t(4) << 61;                    // SWIZZLE_64B
  return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, both K-major.
template <int TN>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(TN >> 3) << 17) | (uint32_t(kTM >> 4) << 24);
}

// D[128 x N] (+)= A[128 x 16] B[N x 16]^T; N a multiple of 16, at most 256
template <int N>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "tcgen05.mma kind::f16 with M = 128");
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(instr_desc<N>()), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// kHalf (32 or 16) consecutive columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[32]) { tmem_ld32(taddr, r); }
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[16]) { tmem_ld16(taddr, r); }

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 2^e as a double for e in [-1022, 1023] (built from the bit pattern)
__device__ __forceinline__ double pow2i(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

template <int S, int TN>
struct Smem {
  alignas(1024) uint8_t stage[Cfg<S, TN>::kStages][Cfg<S, TN>::kStageBytes];
  uint64_t full[Cfg<S, TN>::kStages], empty[Cfg<S, TN>::kStages];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t acc34_empty;  // the epilogue has read d3, d4 of the previous tile
  uint64_t mma_drain;    // abort path: every product issued so far has completed
  uint32_t tmem_base;
  int abort_flag;
};

// Persistent: CTA b processes tiles b, b + gridDim.x, ... in the plan's tile
// order.  Every tile has at least one K chunk (the plan writes K == 0
// problems separately): the epilogue of a tile always waits for that tile's
// products, so no role runs two mbarrier phases ahead of another.  The three roles walk the same sequence of K chunks, counted across
// tiles (stage ring and mbarrier phases continue from tile to tile), and the
// epilogue of one tile overlaps the copies and products of the next: d0..d2
// are double-buffered per pair of chunks, d3 and d4 are released as soon as
// the epilogue has folded them into its integer accumulators.
template <int S, int TN>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                      const Prob* __restrict__ probs, const Tile* __restrict__ tiles, int ntiles,
                      const int* __restrict__ expA, const int* __restrict__ expB, int rowsA, int rowsB,
                      double* __restrict__ C, const Scatter sc, int* err, long long spin) {
  using CF = Cfg<S, TN>;
  constexpr int kStages = CF::kStages;
  constexpr int kStageBytes = CF::kStageBytes;
  constexpr int kBBytes = CF::kBBytes;
  constexpr int kColD3 = CF::kColD3;
  extern __shared__ uint8_t smem_raw[];
  Smem<S, TN>& sm = *reinterpret_cast<Smem<S, TN>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.acc_full[b], 1);
      mbar_init(&sm.acc_empty[b], 256);
    }
    mbar_init(&sm.acc34_empty, 256);
    mbar_init(&sm.mma_drain, 1);
    sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(CF::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort_flag;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long g = 0;  // chunks issued so far (all tiles)
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const Tile t = tiles[ti];
        const Prob p = probs[t.prob];
        const int nk = (p.K + kTK - 1) / kTK;
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = int(g % kStages);
          if (g >= kStages && !mbar_wait(&sm.empty[s], int((g / kStages) - 1) & 1, abort_flag, err, spin)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sm.full[s], kStageBytes);
          uint8_t* base = sm.stage[s];
          const int k0 = c * kTK;
          for (int i = 0; i < S; ++i)
            tma_load_2d(base + i * kABytes, &mapA, k0, i * rowsA + p.arow + t.m0, &sm.full[s]);
          for (int j = 0; j < S; ++j)
            tma_load_2d(base + S * kABytes + j * kBBytes, &mapB, k0, j * rowsB + p.brow + t.n0, &sm.full[s]);
        }
      }
      // every copy issued has landed before the CTA may exit, whichever
      // role aborted and when (after a normal run these phases are already
      // complete: the products consumed them)
      for (long long c = (g > kStages ? g - kStages : 0); c < g; ++c) {
        const int s = int(c % kStages);
        for (long long i = 0; i < kDrainLimit && !mbar_try(&sm.full[s], int(c / kStages) & 1); ++i) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // d0..d2 are drained every pair of K chunks (64 K): their FP32 sums stay
    // exact integers below 2^24 (at most 3 * 64 products of magnitude
    // <= 2^16 per diagonal entry)
    if (lane == 0) {
      long long g = 0, pg = 0;  // chunks and chunk pairs consumed so far (all tiles)
      int tn = 0;               // tiles of this CTA so far
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, ++tn) {
        const Prob p = probs[tiles[ti].prob];
        const int nk = (p.K + kTK - 1) / kTK;
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = int(g % kStages);
          const long long pc = pg + (c >> 1);
          const int buf = int(pc & 1);
          const bool first = (c & 1) == 0;
          if (!mbar_wait(&sm.full[s], int(g / kStages) & 1, abort_flag, err, spin)) {
            ok = false;
            break;
          }
          if (first && pc >= 2 && !mbar_wait(&sm.acc_empty[buf], int((pc >> 1) - 1) & 1, abort_flag, err, spin)) {
            ok = false;
            break;
          }
          if (S == 5 && c == 0 && tn > 0 && !mbar_wait(&sm.acc34_empty, (tn - 1) & 1, abort_flag, err, spin)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sm.stage[s]);
          const uint32_t b0 = a0 + S * kABytes;
          // The slices of B are stacked in the stage (slice j: rows
          // j TN .. j TN + TN - 1), so B slices j .. j + n - 1 form one
          // operand of n TN rows; in tensor memory the diagonals of a
          // buffer lie side by side (d at buf 3 TN + d TN; d3, d4 at
          // kColD3).  A slice i times B slices j .. j + n - 1 thus adds into
          // diagonals i + j .. i + j + n - 1 with one product: 8 products
          // of width TN .. 3 TN per 16 K instead of 15 of width TN (S = 5),
          // 3 instead of 6 (S = 3), each reading its A slice once.
          const uint32_t cb = tmem + uint32_t(buf * 3 * TN);
          const uint32_t c3 = tmem + uint32_t(kColD3);
          for (int ks = 0; ks < kTK / 16; ++ks) {
            const uint32_t acc_b = (!first || ks > 0) ? 1u : 0u;  // first writer of d0..d2 in this pair
            const uint32_t acc_3 = (c > 0 || ks > 0) ? 1u : 0u;   // first writer of d3, d4 in this tile
            auto ad = [&](int i) { return smem_desc(a0 + i * kABytes + ks * 32); };
            auto bd = [&](int j) { return smem_desc(b0 + j * kBBytes + ks * 32); };
            mma_bf16<3 * TN>(cb, ad(0), bd(0), acc_b);           // d0 d1 d2 += A0 [B0 B1 B2]
            if constexpr (S == 5) mma_bf16<2 * TN>(c3, ad(0), bd(3), acc_3);  // d3 d4 += A0 [B3 B4]
            mma_bf16<2 * TN>(cb + TN, ad(1), bd(0), 1u);         // d1 d2 += A1 [B0 B1]
            if constexpr (S == 5) mma_bf16<2 * TN>(c3, ad(1), bd(2), 1u);     // d3 d4 += A1 [B2 B3]
            mma_bf16<TN>(cb + 2 * TN, ad(2), bd(0), 1u);         // d2 += A2 B0
            if constexpr (S == 5) {
              mma_bf16<2 * TN>(c3, ad(2), bd(1), 1u);            // d3 d4 += A2 [B1 B2]
              mma_bf16<2 * TN>(c3, ad(3), bd(0), 1u);            // d3 d4 += A3 [B0 B1]
              mma_bf16<TN>(c3 + TN, ad(4), bd(0), 1u);           // d4 += A4 B0
            }
          }
          mma_commit(&sm.empty[s]);
          if (!first || c == nk - 1) mma_commit(&sm.acc_full[buf]);
        }
        pg += (nk + 1) >> 1;
      }
      // every product issued has written tensor memory before it is freed,
      // whichever role aborted and when (the commit arrives once they have
      // all completed; with none issued, at once)
      mma_commit(&sm.mma_drain);
      for (long long i = 0; i < kDrainLimit && !mbar_try(&sm.mma_drain, 0); ++i) {
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9 ----------------
    // warp w may access tensor-memory lanes 32*(w%4)..+31; the two warps of a
    // lane quarter split the 64 columns
    constexpr int kHalf = TN / 2;
    const int q = warp & 3;
    const int c0 = ((warp - 2) >> 2) * kHalf;
    const int row = q * 32 + lane;
    const uint32_t lane_base = tmem + (uint32_t(q * 32) << 16);
    long long pg = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      const Tile t = tiles[ti];
      const Prob p = probs[t.prob];
      const int nk = (p.K + kTK - 1) / kTK;
      // T = sum over chunk pairs of (S0 2^18 + S1 2^9 + S2): exact in 64 bits
      long long T[kHalf];
#pragma unroll
      for (int j = 0; j < kHalf; ++j) T[j] = 0;
      const int npair = (nk + 1) >> 1;
      for (int pp = 0; pp < npair; ++pp) {
        const long long pc = pg + pp;
        const int buf = int(pc & 1);
        ok = mbar_wait(&sm.acc_full[buf], int(pc >> 1) & 1, abort_flag, err, spin);
        if (!ok) break;
        tc_fence_after();
        // exact FP32 integers below 2^24: one round-to-nearest conversion
        // each; 16 columns at a time (the 64-bit sums hold the registers)
#pragma unroll
        for (int h = 0; h < kHalf; h += 16) {
          uint32_t v[16];
          tmem_ld16(lane_base + buf * 3 * TN + 0 * TN + c0 + h, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) T[h + j] += (long long)__float2int_rn(__uint_as_float(v[j])) << 18;
          tmem_ld16(lane_base + buf * 3 * TN + 1 * TN + c0 + h, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) T[h + j] += (long long)__float2int_rn(__uint_as_float(v[j])) << 9;
          tmem_ld16(lane_base + buf * 3 * TN + 2 * TN + c0 + h, v);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) T[h + j] += __float2int_rn(__uint_as_float(v[j]));
        }
        tc_fence_before();
        mbar_arrive(&sm.acc_empty[buf]);
      }
      if (!ok) break;
      pg += npair;
      // S = 5: X = S0 2^27 + S1 2^18 + S2 2^9 + (S3 + S4 2^-9), folded into
      // T; then d3 and d4 are released to the next tile's products
      if constexpr (S == 5) {
#pragma unroll
        for (int h = 0; h < kHalf / 16; ++h) {
          uint32_t w3[16], w4[16];
          if (nk > 0) {
            tmem_ld16(lane_base + kColD3 + 0 * TN + c0 + h * 16, w3);
            tmem_ld16(lane_base + kColD3 + 1 * TN + c0 + h * 16, w4);
            tmem_wait_ld();
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) w3[j] = w4[j] = 0u;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float small = __uint_as_float(w3[j]) + __uint_as_float(w4[j]) * (1.0f / 512.0f);
            T[h * 16 + j] = (T[h * 16 + j] << 9) + __float2ll_rn(small);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&sm.acc34_empty);
      // C = X 2^(ea+eb-43)
      const int gm = t.m0 + row;
      const bool row_ok = gm < p.M;
      const int ea = row_ok ? expA[p.arow + gm] : 0;
      if (p.scatter) {
        // straight into the output tensor's canonical blocks: this row's
        // block row r and row mi inside it; the columns' block, column and
        // block width are the same for every lane (broadcast loads)
        const int2 ri = row_ok ? sc.rowtab[p.rt_off + gm] : make_int2(0, 0);
        const long long* bb = sc.bbase + p.bb_off + (long long)ri.x * p.ncc;
        const bool plain = sc.alpha == 1.0 && sc.beta == 0.0;
#pragma unroll
        for (int jj = 0; jj < kHalf; ++jj) {
          const int gn = t.n0 + c0 + jj;
          if (row_ok && gn < p.N) {
            const int4 ci = sc.coltab[p.ct_off + gn];
            const long long dst = bb[ci.x] + (long long)ri.y * ci.z + ci.y;
            const int e = ea + expB[p.brow + gn] - CF::kShift;
            const double v = (double)T[jj] * pow2i(e >> 1) * pow2i(e - (e >> 1));
            if (plain) C[dst] = v;
            else C[dst] = sc.beta == 0.0 ? sc.alpha * v : fma(sc.alpha, v, sc.beta * C[dst]);
          }
        }
      } else {
        double* crow = C + p.c_off + (long long)gm * p.c_m;
#pragma unroll
        for (int jj = 0; jj < kHalf; ++jj) {
          const int gn = t.n0 + c0 + jj;
          if (row_ok && gn < p.N) {
            const int e = ea + expB[p.brow + gn] - CF::kShift;
            crow[(long long)gn * p.c_n] = (double)T[jj] * pow2i(e >> 1) * pow2i(e - (e >> 1));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CF::kTmemCols));
  }
}

// The outputs of problems with no matched block pair (K == 0), written by
// the last CTAs of the split or pack launch (kZeroCtas per problem): beta * C
// through the scatter tables, or zeros into the sector matrices of a plain
// plan.
constexpr int kZeroCtas = 8;
struct ZeroJob {
  int nz;
  const Prob* probs;      // scatter form: problems listed by zidx
  const int* zidx;
  Scatter sc;
  const GemmProb* zp;     // plain form (probs == nullptr)
  double* C;
};

__device__ __forceinline__ void zero_part(const ZeroJob& z, int cta) {
  const int pi = cta / kZeroCtas, part = cta - pi * kZeroCtas;
  const long long stride = (long long)kZeroCtas * blockDim.x;
  if (z.probs) {
    const Prob p = z.probs[z.zidx[pi]];
    const long long n = (long long)p.M * p.N;
    for (long long e = part * (long long)blockDim.x + threadIdx.x; e < n; e += stride) {
      const int m = int(e / p.N), c = int(e - (long long)m * p.N);
      const int2 ri = z.sc.rowtab[p.rt_off + m];
      const int4 ci = z.sc.coltab[p.ct_off + c];
      const long long dst = z.sc.bbase[p.bb_off + (long long)ri.x * p.ncc + ci.x] + (long long)ri.y * ci.z + ci.y;
      z.C[dst] = z.sc.beta == 0.0 ? 0.0 : z.sc.beta * z.C[dst];
    }
  } else {
    const GemmProb p = z.zp[pi];
    const long long n = (long long)p.M * p.N;
    for (long long e = part * (long long)blockDim.x + threadIdx.x; e < n; e += stride) {
      const long long m = e / p.N, c = e - m * p.N;
      z.C[p.c_off + m * p.c_m + c * p.c_n] = 0.0;
    }
  }
}

// Split FP64 rows into S BF16 digit slices (integer arithmetic on the bit
// pattern).  One warp per row; digits for k in [K, roundup(K, 32)) are 0.
// One launch splits both operands: CTAs [0, ga) take the rows of A, the
// others those of B.  The task of a row is found by binary search over the
// tasks' first rows (ascending).
struct SplitJob {
  const SplitTask* tasks;
  int ntasks, rows_total;
  const double* X;
  __nv_bfloat16* S;
  int* ex;
};

template <int S>
__global__ void ozaki_split_kernel(SplitJob ja, SplitJob jb, int ga, int gab, int kpitch, ZeroJob zj) {
  if (int(blockIdx.x) >= gab) {
    zero_part(zj, int(blockIdx.x) - gab);
    return;
  }
  const bool is_a = int(blockIdx.x) < ga;
  const SplitJob& J = is_a ? ja : jb;
  const SplitTask* __restrict__ tasks = J.tasks;
  const int ntasks = J.ntasks, rows_total = J.rows_total;
  const double* __restrict__ X = J.X;
  __nv_bfloat16* __restrict__ Sd = J.S;
  int* __restrict__ ex = J.ex;
  const int warp_g = ((int(blockIdx.x) - (is_a ? 0 : ga)) * int(blockDim.x) + int(threadIdx.x)) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp_g >= rows_total || ntasks == 0) return;
  // locate (task, row): last task whose first row is <= warp_g
  int tlo = 0, thi = ntasks - 1;
  while (tlo < thi) {
    const int mid = (tlo + thi + 1) >> 1;
    if (tasks[mid].row0 <= warp_g) tlo = mid;
    else thi = mid - 1;
  }
  const int t = tlo;
  const int r = warp_g - tasks[t].row0;
  if (r < 0 || r >= tasks[t].rows) return;
  const SplitTask tk = tasks[t];
  const double* xr = X + tk.base + (long long)r * tk.s_r;
  unsigned long long mx = 0;
  for (int k = lane; k < tk.K; k += 32) {
    unsigned long long b = __double_as_longlong(xr[(long long)k * tk.s_k]) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  // |x| < 2^e for every entry of the row (e from the largest exponent field)
  const int emax = int(mx >> 52);
  const int e = emax - 1022;
  const int grow = tk.row0 + r;
  if (lane == 0) ex[grow] = e;
  const int kend = (tk.K + 31) & ~31;
  for (int k = lane; k < kend; k += 32) {
    long long Xi = 0;
    if (k < tk.K && mx != 0) {
      const unsigned long long b = __double_as_longlong(xr[(long long)k * tk.s_k]);
      const int E = int((b >> 52) & 0x7FF);
      if (E != 0) {  // subnormals of a row with a normal maximum are below 2^-44 of it
        const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
        // X = round(m * 2^(E - 1075 - e + 9 S - 1)), |X| < 2^(9 S - 1)
        const int sh = E - 1075 - e + 9 * S - 1;
        if (sh >= 0) {
          Xi = m << sh;
        } else if (sh > -64) {
          const int rs = -sh;
          Xi = (m + (1ll << (rs - 1))) >> rs;
        }
        if (b >> 63) Xi = -Xi;
      }
    }
    // signed digits: X = sum_i a_i 2^(9 (S - 1 - i)), |a_i| <= 256
    int dig[S];
#pragma unroll
    for (int i = S - 1; i >= 1; --i) {
      long long lo = ((Xi + 256) & 511) - 256;
      dig[i] = int(lo);
      Xi = (Xi - lo) >> 9;
    }
    dig[0] = int(Xi);
#pragma unroll
    for (int i = 0; i < S; ++i)
      Sd[((long long)i * rows_total + grow) * kpitch + k] = __int2bfloat16_rn(dig[i]);
  }
}

// Gather and split in one pass (the operand's sector matrix is never
// formed): one warp per row of a sector matrix reads the row's K elements
// straight from the operand tensor's canonical blocks, takes the row's
// exponent and writes its S digit slices.  A row of sector s and row
// configuration r meets one block per column configuration c (a segment
// [k0, k0 + w) of the row); inside block (r, c) the element of row mi and
// column kk sits at  off + sum_rowlegs idx * str + sum_collegs idx * str,
// the indices from mi and kk row-major over the legs in matrix order.
// One warp per row, lanes along k: the reads are coalesced when the operand
// block's innermost leg is a contracted leg (consecutive k are consecutive
// in memory); plans whose operands are not laid out so gather and split in
// two passes instead (ozaki_packable).
struct PackGroup {
  int32_t pw0;    // first warp of this group
  int32_t row0;   // its first row in the split buffer
  int32_t h, K;   // rows of this (sector, row configuration), columns
  int64_t seg0;   // its segments (one per column configuration), k0 ascending
  int32_t nseg, pad;
};

struct PackSeg {
  int64_t off;          // block offset in its tensor (elements)
  int32_t k0, w;        // columns [k0, k0 + w) of the row
  int32_t nr, nc;       // row legs, column legs
  int32_t src, pad;     // index of the tensor in the job's pointer table
  int32_t dim[kMaxRank];  // row legs then column legs, matrix order
  int32_t str[kMaxRank];  // their strides inside the block
  uint32_t fm[kMaxRank], fl[kMaxRank];  // FastDiv of dim
};

struct PackJob {
  const PackGroup* groups;
  const PackSeg* segs;
  int ngroups, nwarps;         // groups, warps
  int rows_total;              // rows of the split buffer (slice stride)
  const double* src;           // the operand tensor (tab == nullptr)
  const double* const* tab;    // per-segment tensors (batched contractions)
  __nv_bfloat16* S;
  int* ex;
};

__device__ __forceinline__ uint32_t fdiv(uint32_t n, uint32_t m, uint32_t l) { return (__umulhi(n, m) + n) >> l; }


template <int S>
__global__ void __launch_bounds__(256) pack_split_kernel(PackJob ja, PackJob jb, int ga, int gab, int kpitch,
                                                         ZeroJob zj) {
  if (int(blockIdx.x) >= gab) {
    zero_part(zj, int(blockIdx.x) - gab);
    return;
  }
  const bool is_a = int(blockIdx.x) < ga;
  const PackJob& J = is_a ? ja : jb;
  const int w = ((int(blockIdx.x) - (is_a ? 0 : ga)) * int(blockDim.x) + int(threadIdx.x)) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= J.nwarps || J.ngroups == 0) return;
  int lo = 0, hi = J.ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (J.groups[mid].pw0 <= w) lo = mid;
    else hi = mid - 1;
  }
  const PackGroup G = J.groups[lo];
  const PackSeg* segs = J.segs + G.seg0;
  const int mi = w - G.pw0;
  if (mi < 0 || mi >= G.h) return;
  const int grow = G.row0 + mi;
  // row-leg indices of mi (the row legs' extents are those of every
  // segment of the group)
  int ridx[kMaxRank];
  {
    const PackSeg& s0 = segs[0];
    uint32_t rem = uint32_t(mi);
#pragma unroll
    for (int j = kMaxRank - 1; j >= 0; --j) {
      ridx[j] = 0;
      if (j < s0.nr) {
        const uint32_t q = fdiv(rem, s0.fm[j], s0.fl[j]);
        ridx[j] = int(rem - q * uint32_t(s0.dim[j]));
        rem = q;
      }
    }
  }
  // element k of the row (k < K), walking the segments forward
  int si = 0;
  long long rp = 0;
  const double* base = nullptr;
  auto enter = [&](int i) {
    const PackSeg& sg = segs[i];
    long long o = sg.off;
#pragma unroll
    for (int j = 0; j < kMaxRank; ++j)
      if (j < sg.nr) o += (long long)ridx[j] * sg.str[j];
    rp = o;
    base = J.tab ? J.tab[sg.src] : J.src;
  };
  auto load = [&](int k) -> double {
    while (k >= segs[si].k0 + segs[si].w) {
      ++si;
      enter(si);
    }
    const PackSeg& sg = segs[si];
    uint32_t rem = uint32_t(k - sg.k0);
    long long o = rp;
#pragma unroll
    for (int j = kMaxRank - 1; j >= 0; --j) {
      if (j < sg.nc) {
        const int jj = sg.nr + j;
        const uint32_t q = fdiv(rem, sg.fm[jj], sg.fl[jj]);
        o += (long long)(rem - q * uint32_t(sg.dim[jj])) * sg.str[jj];
        rem = q;
      }
    }
    return base[o];
  };
  // the digits of x against the row exponent e (the same integer
  // arithmetic as ozaki_split_kernel<S>)
  auto digits = [&](double x, int e, int (&dig)[S]) {
    long long Xi = 0;
    const unsigned long long b = __double_as_longlong(x);
    const int E = int((b >> 52) & 0x7FF);
    if (E != 0) {
      const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
      const int sh = E - 1075 - e + 9 * S - 1;
      if (sh >= 0) {
        Xi = m << sh;
      } else if (sh > -64) {
        const int rs = -sh;
        Xi = (m + (1ll << (rs - 1))) >> rs;
      }
      if (b >> 63) Xi = -Xi;
    }
#pragma unroll
    for (int i = S - 1; i >= 1; --i) {
      const long long lo9 = ((Xi + 256) & 511) - 256;
      dig[i] = int(lo9);
      Xi = (Xi - lo9) >> 9;
    }
    dig[0] = int(Xi);
  };
  const int kend = (G.K + 31) & ~31;
  enter(0);
  unsigned long long mx = 0;
  for (int k = lane; k < G.K; k += 32) {
    const unsigned long long b = __double_as_longlong(load(k)) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  const int e = int(mx >> 52) - 1022;
  if (lane == 0) J.ex[grow] = e;
  si = 0;
  enter(0);
  for (int k = lane; k < kend; k += 32) {
    int dig[S];
    if (k < G.K && mx != 0) {
      digits(load(k), e, dig);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) dig[i] = 0;
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
      J.S[((long long)i * J.rows_total + grow) * kpitch + k] = __int2bfloat16_rn(dig[i]);
  }
}

}  // namespace oz

// ---------------------------------------------------------------------------------
// host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    BST_CUDA(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q));
    BST_REQUIRE(p && q == cudaDriverEntryPointSuccess, BST_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiledFn)p;
  }
  return fn;
}

static CUtensorMap make_map(void* base, int kpitch, int rows, int box_rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  cuuint64_t dims[2] = {cuuint64_t(kpitch), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(kpitch) * 2};
  cuuint32_t box[2] = {cuuint32_t(oz::kTK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  BST_REQUIRE(r == CUDA_SUCCESS, BST_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
  return m;
}

struct OzakiPlan {
  int S = 5, TN = 64;  // digit slices per operand, output tile width
  int nprobs = 0, ntiles = 0;
  int rowsA = 0, rowsB = 0, kpitch = 32;
  oz::Prob* d_probs = nullptr;
  oz::Tile* d_tiles = nullptr;
  oz::SplitTask *d_sa = nullptr, *d_sb = nullptr;
  int nsa = 0, nsb = 0;
  __nv_bfloat16 *SA = nullptr, *SB = nullptr;
  int *eA = nullptr, *eB = nullptr;
  CUtensorMap mapA, mapB;
  // every problem reads B as it reads A (a Gram matrix X^T X): with the same
  // pointer for both, B's split is skipped and its tiles come from A's
  // digits through mapBA
  bool ab_same = false;
  CUtensorMap mapBA;
  double flops = 0;
  double split_bytes = 0;  // FP64 read + S BF16 digits written per element, exponent per row
  // K == 0 problems (no matched block pair): written as zeros by a separate
  // launch, so every tile of the persistent GEMM has at least one K chunk
  // (its epilogue then always waits for products of that tile, which keeps
  // the CTA's mbarrier phases in step)
  GemmProb* d_zprobs = nullptr;
  int nzprobs = 0;
  // output scatter into canonical blocks (plans built by
  // ozaki_prepare_scatter): tables on the device, K == 0 problems listed
  // by index for the beta-only pass
  int2* d_rowtab = nullptr;
  int4* d_coltab = nullptr;
  long long* d_bbase = nullptr;
  int* d_zidx = nullptr;
  bool scatter = false;
  // packed operands (pack_split_kernel reads the tensors' blocks; no
  // sector matrices, no separate split)
  bool packed = false;
  oz::PackGroup *d_pgA = nullptr, *d_pgB = nullptr;
  oz::PackSeg *d_psA = nullptr, *d_psB = nullptr;
  int ngA = 0, ngB = 0, nrA = 0, nrB = 0;  // groups and warps of each operand
  ~OzakiPlan() {
    cudaFree(d_pgA);
    cudaFree(d_pgB);
    cudaFree(d_psA);
    cudaFree(d_psB);
    cudaFree(d_rowtab);
    cudaFree(d_coltab);
    cudaFree(d_bbase);
    cudaFree(d_zidx);
    cudaFree(d_probs);
    cudaFree(d_tiles);
    cudaFree(d_sa);
    cudaFree(d_sb);
    cudaFree(SA);
    cudaFree(SB);
    cudaFree(eA);
    cudaFree(eB);
    cudaFree(d_zprobs);
  }
};

template <int S, int TN>
static size_t smem_bytes() { return sizeof(oz::Smem<S, TN>) + 1024; }

template <int S, int TN>
static void set_kernel_attrs() {
  static bool done = false;
  if (done) return;
  BST_CUDA(cudaFuncSetAttribute(oz::ozaki_gemm_kernel<S, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem_bytes<S, TN>())));
  done = true;
}

// streaming multiprocessors of the current device (one persistent CTA each)
static int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return n > 0 ? n : 152;
}

struct PackTables {
  std::vector<oz::PackGroup> g;
  std::vector<oz::PackSeg> sg;
  int nwarps = 0;
};

// Appends the pack groups and segments of one operand of one contraction:
// v is the operand's sector-matrix view of layout L (rows: its open legs,
// columns: its contracted legs), probs the contraction's problems in GEMM
// order (their operand sectors at a_off / b_off), `row` the split-buffer
// row of the first problem (advanced by M or N per problem), `src` the
// operand's index in a pointer table (0 for a single contraction).
static void append_pack(PackTables& T, const Layout* L, const MatView& v, const std::vector<GemmProb>& probs,
                        bool b_side, int& row, int src) {
  std::map<int64_t, const MatSector*> by_off;
  for (auto& sec : v.secs)
    if (sec.rows > 0 && sec.cols > 0) by_off[sec.off] = &sec;
  const int r = L->rank;
  const int nr = int(v.rowlegs.size()), nc = int(v.collegs.size());
  BST_REQUIRE(nr + nc == r && r <= kMaxRank, BST_E_ARG, "pack: view does not cover the tensor");

  std::vector<int32_t> tup(r);
  for (auto& g : probs) {
    const int rows = b_side ? g.N : g.M;
    if (g.K > 0) {
      auto it = by_off.find(b_side ? g.b_off : g.a_off);
      BST_REQUIRE(it != by_off.end() && it->second->rows == rows && it->second->cols == g.K, BST_E_SHAPE,
                  "pack: problem does not match its operand sector");
      const MatSector& sec = *it->second;
      for (size_t rc = 0; rc < sec.rcfg.size(); ++rc) {
        const int64_t h = (rc + 1 < sec.rcfg.size() ? sec.roff[rc + 1] : sec.rows) - sec.roff[rc];
        oz::PackGroup pg{};
        pg.pw0 = T.nwarps;
        pg.row0 = int32_t(row + sec.roff[rc]);
        pg.h = int32_t(h);
        pg.K = g.K;
        pg.seg0 = int64_t(T.sg.size());
        pg.nseg = int32_t(sec.ccfg.size());
        int64_t kcov = 0;
        for (size_t cc = 0; cc < sec.ccfg.size(); ++cc) {
          for (int j = 0; j < nr; ++j) tup[v.rowlegs[j]] = sec.rcfg[rc][j];
          for (int j = 0; j < nc; ++j) tup[v.collegs[j]] = sec.ccfg[cc][j];
          const int64_t b = L->block_of(tup.data());
          BST_REQUIRE(b >= 0, BST_E_SHAPE, "pack: missing operand block");
          const int64_t* sh = &L->shape[b * r];
          std::vector<int64_t> bst(r, 1);
          for (int i = r - 2; i >= 0; --i) bst[i] = bst[i + 1] * sh[i + 1];
          oz::PackSeg sg{};
          sg.off = L->offset[b];
          sg.k0 = int32_t(sec.coff[cc]);
          sg.nr = nr;
          sg.nc = nc;
          sg.src = src;
          int64_t hh = 1, w = 1;
          for (int j = 0; j < nr + nc; ++j) {
            const int leg = j < nr ? v.rowlegs[j] : v.collegs[j - nr];
            sg.dim[j] = int32_t(sh[leg]);
            sg.str[j] = int32_t(bst[leg]);
            FastDiv f;
            f.init(uint32_t(sh[leg]));
            sg.fm[j] = f.m;
            sg.fl[j] = f.l;
            (j < nr ? hh : w) *= sh[leg];
          }
          sg.w = int32_t(w);
          BST_REQUIRE(hh == h && sg.k0 == kcov, BST_E_SHAPE, "pack: segment does not tile the row");
          kcov += w;
          T.sg.push_back(sg);
        }
        BST_REQUIRE(kcov == g.K, BST_E_SHAPE, "pack: segments do not cover K");
        T.g.push_back(pg);
        T.nwarps += int32_t(h);
      }
    }
    row += rows;
  }
}

// Tile schedule of a plan (the order in which CTAs pick up output tiles):
// 0 problem order, row tiles outer; 1 longest K first (the tiles that take
// longest start first, so the last wave is short); 2 problem order, column
// tiles outer (CTAs that run together share B slices in L2).
struct ScatterSpec {
  std::vector<int2> rowtab;
  std::vector<int4> coltab;
  std::vector<long long> bbase;
  std::vector<int64_t> rt_off, ct_off, bb_off;  // per problem
  std::vector<int32_t> ncc;                     // per problem
};

static OzakiPlan* build_plan(Ctx* ctx, const std::vector<GemmProb>& probs, int order = 0,
                             const ScatterSpec* sc = nullptr, int S = 5, int TN = 64) {
  BST_REQUIRE((S == 5 || S == 3) && (TN == 64 || TN == 32), BST_E_ARG, "Ozaki GEMM: unsupported shape");
  auto* P = new OzakiPlan();
  P->S = S;
  P->TN = TN;
  std::vector<oz::Prob> hp;
  std::vector<oz::Tile> ht;
  std::vector<oz::SplitTask> sa, sb;
  std::vector<GemmProb> zp;
  int maxk = 1;
  P->ab_same = !probs.empty();
  for (auto& g : probs) {
    BST_REQUIRE(g.K <= 10000, BST_E_UNSUPPORTED, "Ozaki GEMM: K above 10000");
    maxk = std::max(maxk, g.K);
    P->ab_same = P->ab_same && g.M == g.N && g.a_off == g.b_off && g.a_m == g.b_n && g.a_k == g.b_k;
  }
  P->kpitch = (maxk + oz::kTK - 1) / oz::kTK * oz::kTK;
  for (auto& g : probs) {
    oz::Prob q{};
    q.M = g.M;
    q.N = g.N;
    q.K = g.K;
    q.arow = P->rowsA;
    q.brow = P->rowsB;
    q.c_off = g.c_off;
    q.c_m = g.c_m;
    q.c_n = g.c_n;
    if (sc) {
      const size_t pi = hp.size();
      q.scatter = 1;
      q.ncc = sc->ncc[pi];
      q.rt_off = sc->rt_off[pi];
      q.ct_off = sc->ct_off[pi];
      q.bb_off = sc->bb_off[pi];
    }
    sa.push_back({g.M, g.K, P->rowsA, 0, g.a_off, g.a_m, g.a_k});
    sb.push_back({g.N, g.K, P->rowsB, 0, g.b_off, g.b_n, g.b_k});
    P->rowsA += g.M;
    P->rowsB += g.N;
    const int pi = int(hp.size());
    hp.push_back(q);
    if (g.K == 0) {
      zp.push_back(g);
    } else if (order == 2) {
      for (int n0 = 0; n0 < g.N; n0 += TN)
        for (int m0 = 0; m0 < g.M; m0 += oz::kTM) ht.push_back({pi, m0, n0, 0});
    } else {
      for (int m0 = 0; m0 < g.M; m0 += oz::kTM)
        for (int n0 = 0; n0 < g.N; n0 += TN) ht.push_back({pi, m0, n0, 0});
    }
    P->flops += 2.0 * double(g.M) * g.N * g.K;
    P->split_bytes += double(g.M + g.N) * g.K * (8.0 + 2.0 * S) + 4.0 * (g.M + g.N);
  }
  if (order == 1)
    std::stable_sort(ht.begin(), ht.end(),
                     [&](const oz::Tile& x, const oz::Tile& y) { return hp[x.prob].K > hp[y.prob].K; });
  P->nprobs = int(hp.size());
  P->ntiles = int(ht.size());
  P->nsa = int(sa.size());
  P->nsb = int(sb.size());
  BST_REQUIRE(int64_t(P->rowsA) * S < (1ll << 31) && int64_t(P->rowsB) * S < (1ll << 31),
              BST_E_UNSUPPORTED, "Ozaki GEMM: too many rows");
  auto up = [](auto** dst, const auto& v) {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    if (v.empty()) return;
    BST_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    BST_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  };
  up(&P->d_probs, hp);
  up(&P->d_tiles, ht);
  up(&P->d_zprobs, zp);
  P->nzprobs = int(zp.size());
  up(&P->d_sa, sa);
  up(&P->d_sb, sb);
  if (sc) {
    P->scatter = true;
    up(&P->d_rowtab, sc->rowtab);
    up(&P->d_coltab, sc->coltab);
    up(&P->d_bbase, sc->bbase);
    std::vector<int> zi;
    for (int i = 0; i < int(hp.size()); ++i)
      if (hp[i].K == 0) zi.push_back(i);
    up(&P->d_zidx, zi);
  }
  // split buffers: S slices x rows x kpitch BF16, with room for a full tile
  // past the end so TMA boxes of the last rows stay inside the allocation
  const int64_t ra = int64_t(S) * std::max(P->rowsA, 1) + oz::kTM;
  const int64_t rb = int64_t(S) * std::max(P->rowsB, 1) + std::max(TN, oz::kTM);
  BST_CUDA(cudaMalloc(&P->SA, sizeof(__nv_bfloat16) * ra * P->kpitch));
  BST_CUDA(cudaMalloc(&P->SB, sizeof(__nv_bfloat16) * rb * P->kpitch));
  BST_CUDA(cudaMemset(P->SA, 0, sizeof(__nv_bfloat16) * ra * P->kpitch));
  BST_CUDA(cudaMemset(P->SB, 0, sizeof(__nv_bfloat16) * rb * P->kpitch));
  BST_CUDA(cudaMalloc(&P->eA, sizeof(int) * std::max(P->rowsA, 1)));
  BST_CUDA(cudaMalloc(&P->eB, sizeof(int) * std::max(P->rowsB, 1)));
  P->mapA = make_map(P->SA, P->kpitch, int(ra), oz::kTM);
  P->mapB = make_map(P->SB, P->kpitch, int(rb), TN);
  if (P->ab_same) P->mapBA = make_map(P->SA, P->kpitch, int(ra), TN);
  return P;
}

// A, B: the operands' sector matrices, or for a packed plan the operand
// tensors themselves (tabA / tabB: per-segment tensor tables of a batch)
static void run_plan(Ctx* ctx, OzakiPlan* P, const double* A, const double* B, double* C, cudaStream_t s,
                     bool split_a = true, double alpha = 1.0, double beta = 0.0,
                     const double* const* tabA = nullptr, const double* const* tabB = nullptr,
                     const long long* bbase = nullptr) {
  const oz::Scatter sc{P->d_rowtab, P->d_coltab, bbase ? bbase : P->d_bbase, alpha, beta};
  const bool b_from_a = P->ab_same && A == B && split_a;
  if (P->packed) {
    // gather + split: FP64 read once per element (and once more from cache),
    // S digits written; the byte count is that of the split of gathered
    // rows without the FP64 row write and read of a separate gather.  The
    // K == 0 problems' outputs are written by the same launch.
    ProfScope ps(ctx, s, "pack_bf16", 0.0, P->split_bytes);
    const oz::PackJob ja{P->d_pgA, P->d_psA, P->ngA, P->nrA, P->rowsA, A, tabA, P->SA, P->eA};
    const oz::PackJob jb{P->d_pgB, P->d_psB, P->ngB, P->nrB, P->rowsB, B, tabB, P->SB, P->eB};
    const oz::ZeroJob zj{P->nzprobs, P->scatter ? P->d_probs : nullptr, P->d_zidx, sc, P->d_zprobs, C};
    const int ga = (P->nrA + 7) / 8, gb = (P->nrB + 7) / 8, gz = P->nzprobs * oz::kZeroCtas;
    if (ga + gb + gz > 0) {
      if (P->S == 5) oz::pack_split_kernel<5><<<ga + gb + gz, 256, 0, s>>>(ja, jb, ga, ga + gb, P->kpitch, zj);
      else oz::pack_split_kernel<3><<<ga + gb + gz, 256, 0, s>>>(ja, jb, ga, ga + gb, P->kpitch, zj);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    if (P->ntiles == 0) return;
  } else {
    // the split of both operands; the K == 0 problems' outputs are written
    // by the same launch
    ProfScope ps(ctx, s, "split_bf16", 0.0, b_from_a ? 0.5 * P->split_bytes : P->split_bytes);
    const int wa = (split_a && P->ntiles) ? P->rowsA : 0, wb = (b_from_a || !P->ntiles) ? 0 : P->rowsB;
    const int ga = (wa + 7) / 8, gb = (wb + 7) / 8;  // 8 rows (warps) per CTA
    const int gz = P->nzprobs * oz::kZeroCtas;
    const oz::ZeroJob zj{P->nzprobs, P->scatter ? P->d_probs : nullptr, P->d_zidx, sc, P->d_zprobs, C};
    if (ga + gb + gz > 0) {
      const oz::SplitJob ja{P->d_sa, P->nsa, P->rowsA, A, P->SA, P->eA};
      const oz::SplitJob jb{P->d_sb, P->nsb, P->rowsB, B, P->SB, P->eB};
      if (P->S == 5) oz::ozaki_split_kernel<5><<<ga + gb + gz, 256, 0, s>>>(ja, jb, ga, ga + gb, P->kpitch, zj);
      else oz::ozaki_split_kernel<3><<<ga + gb + gz, 256, 0, s>>>(ja, jb, ga, ga + gb, P->kpitch, zj);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    if (P->ntiles == 0) return;
  }
  ProfScope ps(ctx, s, "gemm_ozaki", P->flops, 0.0);
  const int grid = std::min(P->ntiles, num_sms());
  const long long spin = ctx->spin_limit > 0 ? ctx->spin_limit : oz::kSpinLimit;
  const CUtensorMap& mB = b_from_a ? P->mapBA : P->mapB;
  const int* eB = b_from_a ? P->eA : P->eB;
  auto launch = [&](auto kern, size_t smem) {
    kern<<<grid, oz::kThreads, smem, s>>>(P->mapA, mB, P->d_probs, P->d_tiles, P->ntiles, P->eA, eB, P->rowsA,
                                           P->rowsB, C, sc, ctx->d_err, spin);
  };
  if (P->S == 5 && P->TN == 64) {
    set_kernel_attrs<5, 64>();
    launch(oz::ozaki_gemm_kernel<5, 64>, smem_bytes<5, 64>());
  } else if (P->S == 5) {
    set_kernel_attrs<5, 32>();
    launch(oz::ozaki_gemm_kernel<5, 32>, smem_bytes<5, 32>());
  } else if (P->TN == 64) {
    set_kernel_attrs<3, 64>();
    launch(oz::ozaki_gemm_kernel<3, 64>, smem_bytes<3, 64>());
  } else {
    set_kernel_attrs<3, 32>();
    launch(oz::ozaki_gemm_kernel<3, 32>, smem_bytes<3, 32>());
  }
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

int ozaki_slices(bst_prec prec) { return prec == BST_BF16X3 ? 3 : 5; }

int ozaki_pick_tn(const std::vector<GemmProb>& probs) {
  int64_t tiles64 = 0;
  double cols = 0, cols64 = 0;
  for (auto& g : probs) {
    if (g.K == 0) continue;
    tiles64 += int64_t((g.M + oz::kTM - 1) / oz::kTM) * ((g.N + 63) / 64);
    cols += double(g.N);
    cols64 += double((g.N + 63) / 64 * 64);
  }
  if (tiles64 == 0) return 64;
  return (tiles64 < num_sms() || cols < 0.5 * cols64) ? 32 : 64;
}

// Plan whose epilogue writes every product element into the output
// tensor's canonical block (Sec. 2: the reduced pair products land in the
// output block of their output quantum numbers).  C's legs are A's open
// legs then B's, so the block of (row config r, column config c) is a
// row-major [rows of r x columns of c] matrix: element (m, n) of a sector
// goes to offset(r, c) + mi * width(c) + ni.
// Appends the scatter tables of one contraction's problems (block offsets
// relative to its own output; bsrc, when given, records the contraction
// index `src` of every entry of bbase).
static void append_scatter(ScatterSpec& sc, ContractPlan* p, std::vector<int32_t>* bsrc, int src) {
  const Layout* C = p->C;
  std::vector<int32_t> tup(C->rank);
  size_t pi = 0;
  for (auto& cs : p->vc.secs) {
    if (!(cs.rows > 0 && cs.cols > 0)) continue;
    BST_REQUIRE(pi < p->probs.size() && p->probs[pi].M == cs.rows && p->probs[pi].N == cs.cols, BST_E_SHAPE,
                "scatter plan: problem list does not follow the output sectors");
    sc.rt_off.push_back(int64_t(sc.rowtab.size()));
    sc.ct_off.push_back(int64_t(sc.coltab.size()));
    sc.bb_off.push_back(int64_t(sc.bbase.size()));
    sc.ncc.push_back(int32_t(cs.ccfg.size()));
    std::vector<int64_t> width(cs.ccfg.size());
    for (size_t c = 0; c < cs.ccfg.size(); ++c) {
      const int64_t w = (c + 1 < cs.ccfg.size() ? cs.coff[c + 1] : cs.cols) - cs.coff[c];
      width[c] = w;
      for (int64_t ni = 0; ni < w; ++ni) sc.coltab.push_back(make_int4(int(c), int(ni), int(w), 0));
    }
    for (size_t r = 0; r < cs.rcfg.size(); ++r) {
      const int64_t h = (r + 1 < cs.rcfg.size() ? cs.roff[r + 1] : cs.rows) - cs.roff[r];
      for (int64_t mi = 0; mi < h; ++mi) sc.rowtab.push_back(make_int2(int(r), int(mi)));
      for (size_t c = 0; c < cs.ccfg.size(); ++c) {
        size_t k = 0;
        for (int32_t x : cs.rcfg[r]) tup[k++] = x;
        for (int32_t x : cs.ccfg[c]) tup[k++] = x;
        const int64_t b = C->block_of(tup.data());
        BST_REQUIRE(b >= 0, BST_E_SHAPE, "scatter plan: missing output block");
        sc.bbase.push_back((long long)C->offset[b]);
        if (bsrc) bsrc->push_back(src);
      }
    }
    ++pi;
  }
  BST_REQUIRE(pi == p->probs.size(), BST_E_SHAPE, "scatter plan: problem count mismatch");
  BST_REQUIRE(sc.rowtab.size() < (size_t(1) << 31) && sc.coltab.size() < (size_t(1) << 31), BST_E_UNSUPPORTED,
              "scatter plan: too many rows");
}

static OzakiPlan* prepare_scatter(Ctx* ctx, ContractPlan* p, int S) {
  ScatterSpec sc;
  append_scatter(sc, p, nullptr, 0);
  return build_plan(ctx, p->probs, 0, &sc, S, ozaki_pick_tn(p->probs));
}

// Device tables of the packed operands of a contraction plan.
static void attach_pack(OzakiPlan* P, const PackTables& ta, const PackTables& tb) {
  auto up = [](auto** dst, const auto& v) {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    if (v.empty()) return;
    BST_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    BST_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  };
  up(&P->d_pgA, ta.g);
  up(&P->d_psA, ta.sg);
  up(&P->d_pgB, tb.g);
  up(&P->d_psB, tb.sg);
  P->ngA = int(ta.g.size());
  P->ngB = int(tb.g.size());
  P->nrA = ta.nwarps;
  P->nrB = tb.nwarps;
  P->packed = true;
  P->ab_same = false;
}

static void attach_pack(OzakiPlan* P, ContractPlan* p) {
  PackTables ta, tb;
  int ra = 0, rb = 0;
  append_pack(ta, p->A, p->va, p->probs, false, ra, 0);
  append_pack(tb, p->B, p->vb, p->probs, true, rb, 0);
  BST_REQUIRE(ra == P->rowsA && rb == P->rowsB, BST_E_SHAPE, "pack: row count mismatch");
  attach_pack(P, ta, tb);
}

// The pack kernel reads a row's K elements with its lanes: coalesced when
// the last contracted leg (in pair order) is the operand tensor's innermost
// leg.  Plans whose operands are laid out otherwise gather (block-contiguous
// reads) and split in two passes.
bool ozaki_packable(const ContractPlan* p) {
  return !p->va.collegs.empty() && p->va.collegs.back() == p->A->rank - 1 && !p->vb.collegs.empty() &&
         p->vb.collegs.back() == p->B->rank - 1;
}

// Operands of a plan that is not packed: the gathered sector matrices.
static void gather_operands(Ctx* ctx, ContractPlan* p, const double* a, const double* b, const double** Am,
                            const double** Bm, cudaStream_t s) {
  double* am = (double*)ctx->buf("contract.A", sizeof(double) * std::max<int64_t>(p->amat, 1), s);
  double* bm = (double*)ctx->buf("contract.B", sizeof(double) * std::max<int64_t>(p->bmat, 1), s);
  launch_relayout(ctx, p->ra, a, am, 0, 1.0, 0.0, s);
  launch_relayout(ctx, p->rb, b, bm, 0, 1.0, 0.0, s);
  *Am = am;
  *Bm = bm;
}

void run_gemm_ozaki_scatter(Ctx* ctx, ContractPlan* p, int S, const double* a, const double* b, double* c,
                            double alpha, double beta, cudaStream_t s) {
  OzakiPlan*& P = p->oz[S == 3 ? 1 : 0][1];
  if (!P) {
    P = prepare_scatter(ctx, p, S);
    if (ozaki_packable(p)) attach_pack(P, p);
  }
  if (!P->packed) gather_operands(ctx, p, a, b, &a, &b, s);
  run_plan(ctx, P, a, b, c, s, true, alpha, beta);
}

void run_gemm_ozaki(Ctx* ctx, ContractPlan* p, int S, const double* a, const double* b, double* Cmat,
                    cudaStream_t s, const double* Am, const double* Bm) {
  OzakiPlan*& P = p->oz[S == 3 ? 1 : 0][0];
  if (!P) {
    P = build_plan(ctx, p->probs, 0, nullptr, S, ozaki_pick_tn(p->probs));
    if (ozaki_packable(p)) attach_pack(P, p);
  }
  if (!P->packed) {
    if (Am && Bm) a = Am, b = Bm;
    else gather_operands(ctx, p, a, b, &a, &b, s);
  }
  run_plan(ctx, P, a, b, Cmat, s);
}

void ozaki_free(OzakiPlan* oz) { delete oz; }

// Batched contractions: one packed, scattering plan over the problems of
// every contraction (probs: their concatenation, in plan order).  The
// output blocks of contraction i are addressed relative to the first
// output's pointer: bbase_rel holds each entry's offset inside its own
// output and bbase_src its contraction, and ozaki_batch_bbase turns them
// into element offsets from c[0] for one set of output pointers.
OzakiPlan* ozaki_batch_plan(Ctx* ctx, const std::vector<ContractPlan*>& plans, const std::vector<GemmProb>& probs,
                            int order, int S, int TN, bool pack, std::vector<long long>* bbase_rel,
                            std::vector<int32_t>* bbase_src) {
  ScatterSpec sc;
  bbase_src->clear();
  PackTables ta, tb;
  int ra = 0, rb = 0;
  for (size_t i = 0; i < plans.size(); ++i) {
    append_scatter(sc, plans[i], bbase_src, int(i));
    if (pack) {
      append_pack(ta, plans[i]->A, plans[i]->va, plans[i]->probs, false, ra, int(i));
      append_pack(tb, plans[i]->B, plans[i]->vb, plans[i]->probs, true, rb, int(i));
    }
  }
  BST_REQUIRE(sc.rt_off.size() == probs.size(), BST_E_SHAPE, "batch plan: problem count mismatch");
  *bbase_rel = sc.bbase;
  OzakiPlan* P = build_plan(ctx, probs, order, &sc, S, TN == 0 ? ozaki_pick_tn(probs) : TN);
  if (pack) {
    BST_REQUIRE(ra == P->rowsA && rb == P->rowsB, BST_E_SHAPE, "batch plan: row count mismatch");
    attach_pack(P, ta, tb);
  }
  return P;
}

void ozaki_batch_bbase(const std::vector<long long>& rel, const std::vector<int32_t>& src,
                       const std::vector<double*>& c, std::vector<long long>* out) {
  std::vector<long long> delta(c.size());
  const uintptr_t c0 = uintptr_t(c[0]);
  for (size_t i = 0; i < c.size(); ++i) {
    const long long d = (long long)(uintptr_t(c[i]) - c0);
    BST_REQUIRE(d % (long long)sizeof(double) == 0, BST_E_ARG, "output pointers must be 8-byte aligned");
    delta[i] = d / (long long)sizeof(double);
  }
  out->resize(rel.size());
  for (size_t j = 0; j < rel.size(); ++j) (*out)[j] = rel[j] + delta[src[j]];
}

void run_ozaki_batch(Ctx* ctx, OzakiPlan* P, double* const* bases, int n, const double* Am, const double* Bm,
                     double* c0, const long long* bbase, double alpha, double beta, cudaStream_t s) {
  if (P->packed) run_plan(ctx, P, nullptr, nullptr, c0, s, true, alpha, beta, bases, bases + n, bbase);
  else run_plan(ctx, P, Am, Bm, c0, s, true, alpha, beta, nullptr, nullptr, bbase);
}

void run_gemm_ozaki_probs(Ctx* ctx, const std::string& tag, const std::vector<GemmProb>& probs, const double* A,
                          const double* B, double* C, cudaStream_t s, int order, bool split_a, int S, int TN) {
  if (TN == 0) TN = ozaki_pick_tn(probs);
  // plans live in the context (freed with it), keyed by caller tag, problem
  // list, tile schedule, digit count and tile width
  const std::string key = tag + "/" + std::to_string(probs_hash(probs)) + "/" + std::to_string(order) + "/" +
                          std::to_string(S) + "x" + std::to_string(TN);
  OzakiPlan* P;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->ozplans.find(key);
    P = it == ctx->ozplans.end() ? nullptr : it->second.get();
  }
  if (!P) {
    std::shared_ptr<OzakiPlan> np(build_plan(ctx, probs, order, nullptr, S, TN));
    P = np.get();
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->ozplans[key] = std::move(np);
  }
  run_plan(ctx, P, A, B, C, s, split_a);
}

}  // namespace bst
