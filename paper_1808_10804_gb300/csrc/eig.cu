// Small dense kernels for the projector's eigensolver.
//
// The projector needs the leading eigenpairs of the sector Gram matrices
// G = N^T N.  Large sectors are first reduced by subspace iteration (GEMMs
// on the tensor cores); the resulting b x b (b <= 160) symmetric problems
// are solved here:
//   * jacobi_eig_f32: cyclic two-sided Jacobi in FP32, one CTA per problem,
//     parallel round-robin pair ordering, eigenvalues sorted descending;
//   * oa_update: one step of the Ogita-Aishima refinement, which lifts the
//     FP32 eigenvectors to FP64 accuracy using only matrix products
//     (R = I - X^T X, S = X^T H X, X <- X (I + E));
//   * cholinv_f32: FP32 Cholesky factor M = L L^T and the inverse of L^T,
//     used to orthonormalise the subspace-iteration block (CholQR).
#include <cmath>

#include "bst_internal.h"

namespace bst {

constexpr int kEigMax = 160;
constexpr int kOaMax = 160;  // largest b of oa_update
constexpr int kGramMaxParts = 16;  // most K slices of a partial Gram matrix

struct SmallProb {
  int32_t b, pad;
  int64_t in_off;   // b x b FP64 input, row-major
  int64_t out_off;  // b x b FP64 output, row-major
  int64_t val_off;  // b FP64 values
};

// One CTA per problem.  A and V live in shared memory as FP32.
__global__ void __launch_bounds__(1024) jacobi_eig_f32(const SmallProb* __restrict__ probs, const double* __restrict__ in,
                                                      double* __restrict__ out, double* __restrict__ vals,
                                                      int max_sweeps, float tfloor, float junk) {
  extern __shared__ float sh[];
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b;
  const int bp = b + (b & 1);  // even number of indices for the pairing
  const int ld = bp + 1;
  float* A = sh;
  float* V = A + bp * ld;
  // per pair: cos, sin and the two indices (as int bits), read with one
  // 16-byte load (offset 2 bp (bp+1) floats: a multiple of 16 bytes)
  float4* prm = reinterpret_cast<float4*>(V + bp * ld);
  float* red = reinterpret_cast<float*>(prm + bp / 2);
  int* order = (int*)(red + 1024);
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* H = in + pr.in_off;
  // scale by the largest diagonal entry (in FP64) so FP32 cannot overflow;
  // every loop over the matrix is flat over all threads so the global loads
  // are issued together
  __shared__ double dmax[32];
  {
    double m = 0;
    for (int i = tid; i < b; i += nt) m = fmax(m, fabs(H[(long long)i * b + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) dmax[tid >> 5] = m;
  }
  __syncthreads();
  __shared__ double hscale;
  if (tid == 0) {
    double m = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) m = fmax(m, dmax[w]);
    hscale = m > 0 ? m : 1.0;
  }
  __syncthreads();
  const double inv = 1.0 / hscale;
  for (int q = tid; q < bp * bp; q += nt) {
    const int i = q / bp, j = q - i * bp;
    A[i * ld + j] = (i < b && j < b) ? float(H[(long long)i * b + j] * inv) : 0.0f;
    V[i * ld + j] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int npair = bp / 2;
  // diagonal floor of the rotation test: 1e-5 of the scale, or the
  // convergence floor when that is lower (a graded matrix whose small
  // entries are accurate: pairs are then rotated relative to their own size)
  const float kTau = fminf(1e-5f, fmaxf(tfloor, 1e-30f));
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test relative to the diagonal (keeps small eigenvalues
    // accurate) with a floor tfloor below which values are not resolved:
    // max_{i<j} a_ij^2 / (max(|a_ii|, tfloor) max(|a_jj|, tfloor)); with a
    // floor of 1 (the scale) the test is absolute.  A pair also counts as
    // converged once the rotation it still needs is below 1e-6 rad,
    // a_ij^2 <= 1e-12 (a_ii - a_jj)^2: FP32 rounding keeps a_ij near
    // 6e-8 max(|a_ii|, |a_jj|), which the relative test cannot pass for a
    // pair of very different sizes, and the FP64 refinement that follows
    // converges from such angles.  Pairs whose diagonal entries are both
    // below `junk` are left out (a cluster at the FP32 rounding level of
    // the input, where rotations only move noise); one thread per row
    float worst = 0.f;
    for (int i = tid; i < b; i += nt) {
      const float aii = A[i * ld + i];
      const float ai = fabsf(aii);
      const float di = fmaxf(ai, tfloor);
      for (int j = i + 1; j < b; ++j) {
        const float a = A[i * ld + j];
        const float ajj = A[j * ld + j];
        const float aj = fabsf(ajj);
        if (fmaxf(ai, aj) >= junk) {
          const float rel = a * a / (di * fmaxf(aj, tfloor));
          const float gap = aii - ajj;
          const float ang = 0.1f * (a * a) / fmaxf(gap * gap, 1e-37f);
          worst = fmaxf(worst, fminf(rel, ang));
        }
      }
    }
    red[tid] = worst;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] = fmaxf(red[tid], red[tid + w]);
      __syncthreads();
    }
    const float wmax = red[0];
    __syncthreads();
    if (wmax <= 1e-13f) break;
    for (int r = 0; r < bp - 1; ++r) {
      // round-robin pairing: index bp-1 fixed, the others rotate
      for (int k = tid; k < npair; k += nt) {
        int p, q;
        if (k == 0) {
          p = bp - 1;
          q = r;
        } else {
          p = r + k;
          if (p >= bp - 1) p -= bp - 1;
          q = r - k;
          if (q < 0) q += bp - 1;
        }
        if (p > q) {
          int x = p;
          p = q;
          q = x;
        }
        const float apq = A[p * ld + q];
        float c = 1.f, s = 0.f;
        const float dd = fmaxf(fabsf(A[p * ld + p]), kTau) * fmaxf(fabsf(A[q * ld + q]), kTau);
        if (fabsf(apq) > 1e-30f && apq * apq > 1e-15f * dd) {
          const float app = A[p * ld + p], aqq = A[q * ld + q];
          const float tau = (aqq - app) / (2.f * apq);
          const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        prm[k] = make_float4(c, s, __int_as_float(p), __int_as_float(q));
      }
      __syncthreads();
      // A <- J^T A J by 2 x 2 blocks: the block of pair a (rows p_a, q_a) and
      // pair b (columns p_b, q_b) becomes G_a^T X G_b (rows rotated first,
      // then columns).  A is symmetric, so one thread takes the block and its
      // mirror (a <= b): every entry is read and written once per round.
      // Blocks whose two rotations are both the identity are left alone.
      const int nblk = npair * (npair + 1) / 2;
      for (int t = tid; t < nblk; t += nt) {
        // t -> (a, bq) with a <= bq: t = bq (bq + 1) / 2 + a
        int bq = int((sqrtf(8.f * float(t) + 1.f) - 1.f) * 0.5f);
        while (bq * (bq + 1) / 2 > t) --bq;
        while ((bq + 1) * (bq + 2) / 2 <= t) ++bq;
        const int a = t - bq * (bq + 1) / 2;
        const float4 ra = prm[a], rb = prm[bq];
        if (ra.y == 0.f && rb.y == 0.f) continue;
        const int pa = __float_as_int(ra.z), qa = __float_as_int(ra.w);
        const int pb = __float_as_int(rb.z), qb = __float_as_int(rb.w);
        const float x00 = A[pa * ld + pb], x01 = A[pa * ld + qb];
        const float x10 = A[qa * ld + pb], x11 = A[qa * ld + qb];
        // rows: Y = G_a^T X
        const float y00 = ra.x * x00 - ra.y * x10, y01 = ra.x * x01 - ra.y * x11;
        const float y10 = ra.y * x00 + ra.x * x10, y11 = ra.y * x01 + ra.x * x11;
        // columns: X' = Y G_b
        const float z00 = rb.x * y00 - rb.y * y01, z01 = rb.y * y00 + rb.x * y01;
        const float z10 = rb.x * y10 - rb.y * y11, z11 = rb.y * y10 + rb.x * y11;
        A[pa * ld + pb] = z00;
        A[pa * ld + qb] = z01;
        A[qa * ld + pb] = z10;
        A[qa * ld + qb] = z11;
        if (a != bq) {
          A[pb * ld + pa] = z00;
          A[qb * ld + pa] = z01;
          A[pb * ld + qa] = z10;
          A[qb * ld + qa] = z11;
        }
      }
      // V <- V J: thread (row i, pair group g) applies the rotations
      // k = g, g + G, ... to row i
      const int G = nt / bp > 0 ? nt / bp : 1;
      const int irow = tid % bp, grp = tid / bp;
      if (grp < G) {
        for (int k = grp; k < npair; k += G) {
          const float4 pr = prm[k];
          const float c = pr.x, s = pr.y;
          if (s == 0.f) continue;
          const int p = __float_as_int(pr.z), q = __float_as_int(pr.w);
          const float vp = V[irow * ld + p], vq = V[irow * ld + q];
          V[irow * ld + p] = c * vp - s * vq;
          V[irow * ld + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
  // descending order of the eigenvalues (ties and NaN: lower index first;
  // NaN compares as -inf so the ranks stay a permutation)
  for (int i = tid; i < b; i += nt) {
    float ai = A[i * ld + i];
    if (ai != ai) ai = -INFINITY;
    int rank = 0;
    for (int j = 0; j < b; ++j) {
      float aj = A[j * ld + j];
      if (aj != aj) aj = -INFINITY;
      rank += (aj > ai) || (aj == ai && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  double* X = out + pr.out_off;
  for (int q = tid; q < b * b; q += nt) {
    const int i = q / b, jn = q - i * b;
    X[q] = double(V[i * ld + order[jn]]);
  }
  for (int jn = tid; jn < b; jn += nt) vals[pr.val_off + jn] = double(A[order[jn] * ld + order[jn]]) * hscale;
}

// Block Jacobi: the same problem, interface and tests as jacobi_eig_f32,
// with the indices in blocks of 16.  A sweep is nb - 1 rounds (nb blocks,
// round-robin pairing of blocks); in a round every block pair P = I u J is
// one 32 x 32 subproblem: a warp runs one cyclic sweep of 2 x 2 rotations
// on A[P, P] (in its own shared buffer), accumulating Q^T in registers
// (lane i holds row i), then all threads apply A[P, :] <- Q^T A[P, :],
// A[:, P] <- A[:, P] Q and V[:, P] <- V[:, P] Q.  Per sweep this moves
// the matrix through shared memory nb - 1 times instead of b - 1 (the
// scalar kernel's rounds are bound by those passes), at the same
// arithmetic.  bp = b rounded up to 32 (zero padding, decoupled).
constexpr int kBjThreads = 512;
// row stride of a pair's Q^T (16-byte rows for vector loads)
constexpr int kQt = 36;

__global__ void __launch_bounds__(kBjThreads) jacobi_block_f32(const SmallProb* __restrict__ probs,
                                                               const double* __restrict__ in,
                                                               double* __restrict__ out, double* __restrict__ vals,
                                                               int max_sweeps, float tfloor, float junk,
                                                               float tol, float skip_ang,
                                                               int* __restrict__ sweeps_used) {
  extern __shared__ float sh[];
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b;
  const int bp = (b + 31) & ~31;
  const int ld = bp + 1;
  const int nb = bp >> 4;       // blocks of 16 (even)
  const int npair = nb >> 1;    // <= 5
  float* A = sh;
  float* V = A + bp * ld;
  float* Sub = V + bp * ld;     // npair x 32 x kQt: subproblem (row stride 33), then Q^T (row stride kQt)
  float* red = Sub + npair * 32 * kQt;
  int* order = reinterpret_cast<int*>(red + kBjThreads);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  const double* H = in + pr.in_off;
  __shared__ double dmax[32];
  __shared__ int moved[8];  // per subproblem of a round: some rotation was applied
  {
    double m = 0;
    for (int i = tid; i < b; i += nt) m = fmax(m, fabs(H[(long long)i * b + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) dmax[warp] = m;
  }
  __syncthreads();
  __shared__ double hscale;
  if (tid == 0) {
    double m = 0;
    for (int w = 0; w < nt / 32; ++w) m = fmax(m, dmax[w]);
    hscale = m > 0 ? m : 1.0;
  }
  __syncthreads();
  const double inv = 1.0 / hscale;
  for (int q = tid; q < bp * bp; q += nt) {
    const int i = q / bp, j = q - i * bp;
    A[i * ld + j] = (i < b && j < b) ? float(H[(long long)i * b + j] * inv) : 0.0f;
    V[i * ld + j] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const float kTau = fminf(1e-5f, fmaxf(tfloor, 1e-30f));
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence: the scalar kernel's test (relative with floor, or the
    // remaining rotation below 1e-6 rad; pairs both below junk left out)
    float worst = 0.f;
    for (int i = tid; i < b; i += nt) {
      const float aii = A[i * ld + i];
      const float ai = fabsf(aii);
      const float di = fmaxf(ai, tfloor);
      for (int j = i + 1; j < b; ++j) {
        const float a = A[i * ld + j];
        const float ajj = A[j * ld + j];
        const float aj = fabsf(ajj);
        if (fmaxf(ai, aj) >= junk) {
          const float rel = a * a / (di * fmaxf(aj, tfloor));
          const float gap = aii - ajj;
          const float ang = 0.1f * (a * a) / fmaxf(gap * gap, 1e-37f);
          worst = fmaxf(worst, fminf(rel, ang));
        }
      }
    }
    red[tid] = worst;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] = fmaxf(red[tid], red[tid + w]);
      __syncthreads();
    }
    const float wmax = red[0];
    __syncthreads();
    if (wmax <= tol) break;
    for (int r = 0; r < nb - 1; ++r) {
      // ---- the subproblems: warp p < npair takes block pair p ----
      if (warp < npair) {
        int bi, bj;
        if (warp == 0) {
          bi = nb - 1;
          bj = r;
        } else {
          bi = r + warp;
          if (bi >= nb - 1) bi -= nb - 1;
          bj = r - warp;
          if (bj < 0) bj += nb - 1;
        }
        // index map of the pair: local 0..15 -> block bi, 16..31 -> block bj
        float* S = Sub + warp * 32 * kQt;
        const int gl = (lane < 16 ? bi * 16 + lane : bj * 16 + lane - 16);
        for (int k = 0; k < 32; ++k) {
          const int gk = (k < 16 ? bi * 16 + k : bj * 16 + k - 16);
          S[lane * 33 + k] = A[gl * ld + gk];
        }
        float qt[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) qt[k] = (k == lane) ? 1.f : 0.f;
        __syncwarp();
        // one cyclic sweep: 31 rounds of 16 disjoint rotations
        bool any_rot = false;
        for (int rr = 0; rr < 31; ++rr) {
          // lane's partner in round rr (index 31 fixed, others rotate)
          int mate;
          if (lane == 31) mate = rr;
          else if (lane == rr) mate = 31;
          else {
            mate = 2 * rr - lane;
            mate %= 31;
            if (mate < 0) mate += 31;
          }
          const int p = min(lane, mate), q = max(lane, mate);
          const float apq = S[p * 33 + q], app = S[p * 33 + p], aqq = S[q * 33 + q];
          float c = 1.f, sn = 0.f;
          const float dd = fmaxf(fabsf(app), kTau) * fmaxf(fabsf(aqq), kTau);
          // (skip_ang > 0: rotations whose angle test 0.1 a^2 / gap^2 is
          // below it are left out)
          const float gq = aqq - app;
          const bool rot = fabsf(apq) > 1e-30f && apq * apq > 1e-15f * dd &&
                           !(skip_ang > 0.f && 0.1f * (apq * apq) <= skip_ang * fmaxf(gq * gq, 1e-37f));
          if (rot) {
            const float tau = gq / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            sn = t * c;
          }
          // a step without any rotation leaves S and Q^T as they are
          if (!__any_sync(0xffffffffu, rot)) continue;
          any_rot = true;
          // row of this lane: S'[lane] = c S[lane] -/+ s S[mate], then the
          // columns likewise (S' is no longer symmetric); in halves of 16
          // (reads of a half before anyone writes it)
          const bool lo = lane == p;
#pragma unroll
          for (int h = 0; h < 32; h += 16) {
            float rl[16], rm[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              rl[k] = S[lane * 33 + h + k];
              rm[k] = S[mate * 33 + h + k];
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k) S[lane * 33 + h + k] = lo ? (c * rl[k] - sn * rm[k]) : (sn * rm[k] + c * rl[k]);
            __syncwarp();
          }
#pragma unroll
          for (int h = 0; h < 32; h += 16) {
            float rl[16], rm[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              rl[k] = S[(h + k) * 33 + lane];
              rm[k] = S[(h + k) * 33 + mate];
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k) S[(h + k) * 33 + lane] = lo ? (c * rl[k] - sn * rm[k]) : (sn * rm[k] + c * rl[k]);
            __syncwarp();
          }
          // Q^T rows: row lane of Q^T = column lane of Q
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float m = __shfl_sync(0xffffffffu, qt[k], mate);
            qt[k] = lo ? (c * qt[k] - sn * m) : (sn * m + c * qt[k]);
          }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 32; ++k) S[lane * kQt + k] = qt[k];
        if (lane == 0) moved[warp] = int(any_rot);
      }
      __syncthreads();
      // ---- A[P, :] <- Q^T A[P, :]: task (pair, column) ----
      for (int t = tid; t < npair * bp; t += nt) {
        const int pp = t / bp, col = t - pp * bp;
        int bi, bj;
        if (pp == 0) {
          bi = nb - 1;
          bj = r;
        } else {
          bi = r + pp;
          if (bi >= nb - 1) bi -= nb - 1;
          bj = r - pp;
          if (bj < 0) bj += nb - 1;
        }
        if (!moved[pp]) continue;  // Q = I: A[P, :] unchanged
        const float* QT = Sub + pp * 32 * kQt;
        float a[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) a[k] = A[(k < 16 ? bi * 16 + k : bj * 16 + k - 16) * ld + col];
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
          float acc0 = 0.f, acc1 = 0.f;
          const float4* q4 = reinterpret_cast<const float4*>(QT + i * kQt);
#pragma unroll
          for (int k = 0; k < 32; k += 4) {
            const float4 q = q4[k >> 2];
            acc0 = fmaf(q.x, a[k], acc0);
            acc1 = fmaf(q.y, a[k + 1], acc1);
            acc0 = fmaf(q.z, a[k + 2], acc0);
            acc1 = fmaf(q.w, a[k + 3], acc1);
          }
          A[(i < 16 ? bi * 16 + i : bj * 16 + i - 16) * ld + col] = acc0 + acc1;
        }
      }
      __syncthreads();
      // ---- A[:, P] <- A[:, P] Q and V[:, P] <- V[:, P] Q: task (matrix, pair, row) ----
      for (int t = tid; t < 2 * npair * bp; t += nt) {
        const int which = t / (npair * bp);
        const int rem = t - which * npair * bp;
        const int pp = rem / bp, row = rem - pp * bp;
        int bi, bj;
        if (pp == 0) {
          bi = nb - 1;
          bj = r;
        } else {
          bi = r + pp;
          if (bi >= nb - 1) bi -= nb - 1;
          bj = r - pp;
          if (bj < 0) bj += nb - 1;
        }
        if (!moved[pp]) continue;  // Q = I
        float* M = which ? V : A;
        const float* QT = Sub + pp * 32 * kQt;
        float a[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) a[k] = M[row * ld + (k < 16 ? bi * 16 + k : bj * 16 + k - 16)];
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
          float acc0 = 0.f, acc1 = 0.f;
          const float4* q4 = reinterpret_cast<const float4*>(QT + j * kQt);
#pragma unroll
          for (int k = 0; k < 32; k += 4) {
            const float4 q = q4[k >> 2];
            acc0 = fmaf(a[k], q.x, acc0);
            acc1 = fmaf(a[k + 1], q.y, acc1);
            acc0 = fmaf(a[k + 2], q.z, acc0);
            acc1 = fmaf(a[k + 3], q.w, acc1);
          }
          M[row * ld + (j < 16 ? bi * 16 + j : bj * 16 + j - 16)] = acc0 + acc1;
        }
      }
      __syncthreads();
    }
  }
  if (sweeps_used && tid == 0) sweeps_used[blockIdx.x] = sweep;  // sweeps run (max_sweeps: not converged)
  for (int i = tid; i < b; i += nt) {
    float ai = A[i * ld + i];
    if (ai != ai) ai = -INFINITY;
    int rank = 0;
    for (int j = 0; j < b; ++j) {
      float aj = A[j * ld + j];
      if (aj != aj) aj = -INFINITY;
      rank += (aj > ai) || (aj == ai && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  double* X = out + pr.out_off;
  for (int q = tid; q < b * b; q += nt) {
    const int i = q / b, jn = q - i * b;
    X[q] = double(V[i * ld + order[jn]]);
  }
  for (int jn = tid; jn < b; jn += nt) vals[pr.val_off + jn] = double(A[order[jn] * ld + order[jn]]) * hscale;
}

size_t jacobi_block_smem(int b) {
  const int bp = (b + 31) & ~31;
  const int npair = bp / 32;
  return sizeof(float) * (2 * bp * (bp + 1) + npair * 32 * kQt + kBjThreads) + sizeof(int) * bp;
}

size_t jacobi_smem(int b) {
  const int bp = b + (b & 1);
  return sizeof(float) * (2 * bp * (bp + 1) + bp + 1024) + sizeof(int) * (bp + bp);
}

// Ogita-Aishima step, elementwise part.  In: XtX (b x b), S = X^T H X.
// Out: E (b x b) and lam (b):  R = I - XtX, lam_i = S_ii / (1 - R_ii),
// E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) when the pair is separated,
// |lam_i - lam_j| > rel_delta * max(|lam_i|, |lam_j|) and
// > acc * sqrt(max|lam|) (sqrt|lam_i| + sqrt|lam_j|) (the rounding of S
// when it is formed as W^T W, W = N X), and not both below junk * max|lam|
// (values the FP32 stage cannot resolve), else R_ij / 2.
// Grid (problem, slice): every CTA forms the b values in shared memory
// (slice 0 also stores them) and then its slice of the b x b entries, so
// the FP64 divisions spread over the whole GPU.
__global__ void oa_update(const SmallProb* __restrict__ probs, const double* __restrict__ XtX,
                          const double* __restrict__ S, double* __restrict__ E, double* __restrict__ lam,
                          double rel_delta, double junk, double acc) {
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b;
  const double* xx = XtX + pr.in_off;
  const double* s = S + pr.in_off;
  double* e = E + pr.in_off;
  __shared__ double l[kOaMax];
  __shared__ double smax;
  __shared__ double wmax[32];
  double m = 0;
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    const double rii = 1.0 - xx[(long long)i * b + i];
    const double li = s[(long long)i * b + i] / (1.0 - rii);
    l[i] = li;
    if (blockIdx.y == 0) lam[pr.val_off + i] = li;
    m = fmax(m, fabs(li));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0;
    for (int w = 0; w < int(blockDim.x + 31) / 32; ++w) mm = fmax(mm, wmax[w]);
    smax = mm;
  }
  __syncthreads();
  const int bb = b * b, per = (bb + int(gridDim.y) - 1) / int(gridDim.y);
  const int q0 = int(blockIdx.y) * per, q1 = min(bb, q0 + per);
  for (int q = q0 + int(threadIdx.x); q < q1; q += blockDim.x) {
    const int i = q / b, j = q - i * b;
    const double rij = (i == j ? 1.0 : 0.0) - xx[q];
    const double delta = fmax(rel_delta * fmax(fabs(l[i]), fabs(l[j])),
                              acc * sqrt(smax) * (sqrt(fabs(l[i])) + sqrt(fabs(l[j])))) + 1e-300 * smax;
    const bool unresolved = fabs(l[i]) < junk * smax && fabs(l[j]) < junk * smax;
    double v;
    if (i == j || unresolved || fabs(l[i] - l[j]) <= delta) v = 0.5 * rij;
    else v = (s[q] + l[j] * rij) / (l[j] - l[i]);
    e[q] = v;
  }
}

// X <- X + XE (in place; XE computed by a GEMM)
__global__ void add_inplace(double* __restrict__ X, const double* __restrict__ XE, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[i] += XE[i];
}

// Conversions between FP64 and FP32 with a power-of-two scale, built from
// the IEEE-754 fields with integer operations: the FP64 pipe of this part
// is narrow (a few operations per clock per SM), so per-element FP64
// multiplies and conversions would dominate the small kernels' loads and
// stores.
// float(x * 2^e), rounded to nearest even; results below the FP32 normal
// range flush to zero and above it saturate to infinity.
__device__ __forceinline__ float f64_to_f32_scaled(double x, int e) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = unsigned(u >> 32) & 0x80000000u;
  const int ex = int((u >> 52) & 0x7ff);
  const unsigned long long mant = u & 0xfffffffffffffull;
  if (ex == 0) return __uint_as_float(sign);  // zero and FP64 subnormals
  if (ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u));
  int fe = ex - 1023 + e + 127;
  unsigned m = unsigned(mant >> 29);
  const unsigned rest = unsigned(mant & 0x1fffffffull);  // the 29 dropped bits
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ++m;
  if (m == 0x800000u) {
    m = 0;
    ++fe;
  }
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | (unsigned(fe) << 23) | m);
}

// double(f) * 2^e, exact; FP32 subnormals flush to zero.
__device__ __forceinline__ double f32_to_f64_scaled(float f, int e) {
  const unsigned v = __float_as_uint(f);
  const unsigned long long sign = static_cast<unsigned long long>(v & 0x80000000u) << 32;
  const int ex = int((v >> 23) & 0xff);
  const unsigned long long mant = static_cast<unsigned long long>(v & 0x7fffffu) << 29;
  if (ex == 0) return __longlong_as_double(static_cast<long long>(sign));
  if (ex == 0xff) return __longlong_as_double(static_cast<long long>(sign | 0x7ff0000000000000ull | mant));
  const int de = ex - 127 + 1023 + e;
  if (de <= 0) return __longlong_as_double(static_cast<long long>(sign));
  if (de >= 0x7ff) return __longlong_as_double(static_cast<long long>(sign | 0x7ff0000000000000ull));
  return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(de) << 52) | mant));
}

// x = r * 2^k with r in [1, 2) (x > 0 finite and normal)
__device__ __forceinline__ void split_pow2(double x, int* k, float* r) {
  const int ex = int((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff);
  *k = ex - 1023;
  *r = f64_to_f32_scaled(x, -*k);
}

// FP32 Cholesky factor M = L L^T (after scaling M to unit diagonal) and the
// inverse of L^T, for the CholQR steps of the subspace iteration; b <= 160,
// one CTA of 512 threads (16 warps) per problem.  Output Rinv (FP64, upper)
// with Y Rinv orthonormal when M = Y^T Y.
//
// The scaled matrix is padded with the identity to bp (a multiple of 32), so
// every panel is one full 32 x 32 block and no loop carries a bound check.
// Per panel P (rows and columns kb = 32 P .. kb + 31), three phases between
// barriers:
//   1. warp 0 factors the diagonal block D in registers (lane r holds row r;
//      pivots and column entries travel by warp shuffles) and, in the same
//      pivot loop with the same broadcast column entries, eliminates below
//      each pivot in the identity to form D^-1 (lane c holds column c);
//      meanwhile the other warps
//      form T = L[P, 0:P] Li[0:P, 0:P], the product block row P of the
//      inverse needs, stashed transposed in the (otherwise unused) upper
//      triangle of Li;
//   2. the rows below the panel get L[i, P] = A[i, P] D^-T, and the inverse
//      gets its block row Li[P, 0:P] = -D^-1 T;
//   3. the trailing lower triangle gets A -= L[:, P] L[:, P]^T, 8-row
//      quarters of 32 x 32 blocks per warp.
// Operands that a lane reuses across rows (a column of D^-1, a row of the
// panel) sit in registers; the shared row it meets them with is read by all
// lanes at one address (a broadcast).  Columns whose pivot falls below 1e-6
// (numerically dependent on earlier ones at FP32 level) are dropped: their
// row and column of the factor become those of the identity, and their row
// and column of Rinv are zero.
constexpr int kCholThreads = 512;
constexpr int kCholWarps = kCholThreads / 32;

// Input: either the FP64 matrix M at in + in_off (nparts == 0), or nparts
// FP32 partial sums of it, partial s at gin + in_off + s b^2, added in slice
// order (gram_f32_kernel's output).
__global__ void __launch_bounds__(kCholThreads) cholinv_f32(const SmallProb* __restrict__ probs,
                                                            const double* __restrict__ in, double* __restrict__ out,
                                                            int* err, const float* __restrict__ gin, int nparts) {
  extern __shared__ float sh[];
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b, bb = b * b;
  const int bp = (b + 31) & ~31, ld = bp + 1, nbp = bp >> 5;
  float* L = sh;                 // bp x ld: the matrix, overwritten by its factor (lower)
  float* Li = L + bp * ld;       // bp x ld: inverse of the factor (lower); T stash (upper)
  float* rsc = Li + bp * ld;     // bp row-scale mantissas
  int* ksc = reinterpret_cast<int*>(rsc + bp);  // bp row-scale exponents
  int* drop = ksc + bp;          // bp dropped-column flags
  const double* M = in + pr.in_off;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const float* G = nparts > 0 ? gin + pr.in_off : nullptr;
  __shared__ __align__(16) float colb[2][32];  // phase 1: a column of the diagonal block
  if (G) {
    // FP32 partial sums, added in slice order.  Every thread keeps the
    // loads of all slices of one 4-wide group in flight at once (the sums
    // are latency bound otherwise); with b and the offset multiples of 4
    // the groups are aligned 16-byte words of each partial.
    const int b4 = ((b & 3) || (pr.in_off & 3)) ? 0 : b >> 2;
    for (int q = tid; q < (b4 ? 0 : b * b); q += kCholThreads) {  // (b not a multiple of 4)
      const int i = q / b, j = q - i * b;
      float g = 0.f;
      for (int s = 0; s < nparts; ++s) g += G[(long long)s * bb + q];
      L[i * ld + j] = g;
    }
    for (int g4 = tid; g4 < b * b4; g4 += kCholThreads) {
      const int i = g4 / b4, j = (g4 - i * b4) << 2;
      const float4* src = reinterpret_cast<const float4*>(G + (long long)i * b + j);
      float4 part[kGramMaxParts];
#pragma unroll
      for (int s = 0; s < kGramMaxParts; ++s)
        part[s] = s < nparts ? __ldg(src + (long long)s * (bb >> 2)) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int s = 0; s < kGramMaxParts; ++s)
        if (s < nparts) {
          g.x += part[s].x;
          g.y += part[s].y;
          g.z += part[s].z;
          g.w += part[s].w;
        }
      float* row = L + i * ld + j;
      row[0] = g.x;
      row[1] = g.y;
      row[2] = g.z;
      row[3] = g.w;
    }
    // padding: identity
    for (int q = tid; q < bp * bp; q += kCholThreads) {
      const int i = q / bp, j = q - i * bp;
      if (i >= b || j >= b) L[i * ld + j] = (i == j) ? 1.f : 0.f;
      Li[i * ld + j] = 0.f;
    }
    __syncthreads();
    // unit-diagonal scaling: row i times 1 / sqrt(M_ii) = rsc[i] 2^ksc[i]
    for (int i = tid; i < bp; i += kCholThreads) {
      int k = 0;
      float r = 1.f;
      if (i < b) {
        const double d = double(L[i * ld + i]);
        if (d > 0) split_pow2(1.0 / sqrt(d), &k, &r);
      }
      ksc[i] = k;
      rsc[i] = r;
      drop[i] = 0;
    }
    __syncthreads();
    // (the power of two exactly, the mantissas as two FP32 products)
    for (int q = tid; q < b * b; q += kCholThreads) {
      const int i = q / b, j = q - i * b;
      // 2^e as two exact factors (|e| <= 256: each half a normal FP32 power)
      const int e = ksc[i] + ksc[j], e1 = e >> 1, e2 = e - e1;
      L[i * ld + j] = L[i * ld + j] * __int_as_float((e1 + 127) << 23) * __int_as_float((e2 + 127) << 23) *
                      (rsc[i] * rsc[j]);
    }
  } else {
  // unit-diagonal scaling: row i times 1 / sqrt(M_ii) = rsc[i] 2^ksc[i]
  for (int i = tid; i < bp; i += kCholThreads) {
    int k = 0;
    float r = 1.f;
    if (i < b) {
      const double d = M[(long long)i * b + i];
      if (d > 0) split_pow2(1.0 / sqrt(d), &k, &r);
    }
    ksc[i] = k;
    rsc[i] = r;
    drop[i] = 0;
  }
  __syncthreads();
  for (int q0 = tid; q0 < bp * bp; q0 += 4 * kCholThreads) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * kCholThreads;
      const int i = q / bp, j = q - i * bp;
      v[u] = (q < bp * bp && i < b && j < b) ? M[(long long)i * b + j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * kCholThreads;
      if (q < bp * bp) {
        const int i = q / bp, j = q - i * bp;
        float a;
        if (i < b && j < b) a = f64_to_f32_scaled(v[u], ksc[i] + ksc[j]) * (rsc[i] * rsc[j]);
        else a = (i == j) ? 1.f : 0.f;
        L[i * ld + j] = a;
        Li[i * ld + j] = 0.f;
      }
    }
  }
  }
  __syncthreads();
  for (int P = 0; P < nbp; ++P) {
    const int kb = P << 5;
    // ---- phase 1 ----
    if (warp == 0) {
      float row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = L[(kb + lane) * ld + kb + c];
      int mydrop = 0;
      // column `lane` of D^-1, eliminated along with the factorisation:
      // D x = e_lane, pivot by pivot (x_k /= D_kk, then x_j -= D_jk x_k)
      float x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        // column k of the partly reduced block (D_rk of every lane r) goes
        // through shared memory and comes back to every lane as 16-byte
        // broadcast loads; double-buffered, so one warp barrier a pivot
        float* cb = colb[k & 1];
        cb[lane] = row[k];
        __syncwarp();
        float col[32];
#pragma unroll
        for (int g = k >> 2; g < 8; ++g) {
          const float4 v = reinterpret_cast<const float4*>(cb)[g];
          col[4 * g] = v.x;
          col[4 * g + 1] = v.y;
          col[4 * g + 2] = v.z;
          col[4 * g + 3] = v.w;
        }
        const float dkk = col[k];
        const bool dk = !(dkk > 1e-6f);  // the same on every lane
        const float inv = dk ? 1.f : rsqrtf(dkk);  // 1 / D_kk
        // (selects, not branches: the lanes stay converged)
        const float rk = row[k];
        row[k] = lane == k ? (dk ? 1.f : dkk * inv) : (lane > k ? (dk ? 0.f : rk * inv) : rk);
        if (dk) {  // uniform
          mydrop = lane == k ? 1 : mydrop;
#pragma unroll
          for (int c = 0; c < k; ++c) row[c] = lane == k ? 0.f : row[c];
        }
        x[k] *= inv;
        if (!dk) {
          // D_rj -= L_rk L_jk and x_j -= L_jk x_k with L_jk = D_jk / D_kk
          const float a = row[k] * inv, bx = x[k] * inv;
#pragma unroll
          for (int j = k + 1; j < 32; ++j) {
            if (lane >= j) row[j] = fmaf(-a, col[j], row[j]);
            x[j] = fmaf(-bx, col[j], x[j]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) L[(kb + lane) * ld + kb + c] = (c <= lane) ? row[c] : 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) Li[(kb + i) * ld + kb + lane] = (i >= lane) ? x[i] : 0.f;
      drop[kb + lane] = mydrop;
    } else if (P > 0) {
      // T[r][j] = sum_{k >= j} L[kb + r][k] Li[k][j] for j < kb, stashed at
      // Li[j][kb + r]; items: (column block J, 8 rows)
      const int nitem = P * 4;
      for (int it = warp - 1; it < nitem; it += kCholWarps - 1) {
        const int J = it >> 2, r0 = (it & 3) * 8;
        const int j = (J << 5) + lane;
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = 0.f;
        for (int k = J << 5; k < kb; ++k) {
          const float li = Li[k * ld + j];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = fmaf(L[(kb + r0 + u) * ld + k], li, acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) Li[j * ld + kb + r0 + u] = acc[u];
      }
    }
    __syncthreads();
    // ---- phase 2 ----
    {
      // rows below the panel: L[i][kb + c] = sum_k A[i][kb + k] D^-1[c][k]
      float dinv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) dinv[k] = Li[(kb + lane) * ld + kb + k];
      const bool dropc = drop[kb + lane] != 0;
      // (rows in pairs, four partial sums each: short dependency chains)
      for (int i = kb + 32 + warp; i < bp; i += 2 * kCholWarps) {
        const int i2 = i + kCholWarps;
        const bool two = i2 < bp;
        float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          s0[k & 3] = fmaf(L[i * ld + kb + k], dinv[k], s0[k & 3]);
          if (two) s1[k & 3] = fmaf(L[i2 * ld + kb + k], dinv[k], s1[k & 3]);
        }
        __syncwarp();
        L[i * ld + kb + lane] = dropc ? 0.f : (s0[0] + s0[1]) + (s0[2] + s0[3]);
        if (two) L[i2 * ld + kb + lane] = dropc ? 0.f : (s1[0] + s1[1]) + (s1[2] + s1[3]);
      }
      // inverse block row: Li[kb + r][j] = -sum_k D^-1[r][k] T[k][j], j < kb;
      // items: (column block J, 8 rows)
      const int nitem = P * 4;
      for (int it = warp; it < nitem; it += kCholWarps) {
        const int J = it >> 2, r0 = (it & 3) * 8;
        const int j = (J << 5) + lane;
        float t[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) t[k] = Li[j * ld + kb + k];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          const int r = r0 + u;
          float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            s0[k & 3] = fmaf(Li[(kb + r) * ld + kb + k], t[k], s0[k & 3]);
            s1[k & 3] = fmaf(Li[(kb + r + 1) * ld + kb + k], t[k], s1[k & 3]);
          }
          Li[(kb + r) * ld + j] = drop[kb + r] ? 0.f : -((s0[0] + s0[1]) + (s0[2] + s0[3]));
          Li[(kb + r + 1) * ld + j] = drop[kb + r + 1] ? 0.f : -((s1[0] + s1[1]) + (s1[2] + s1[3]));
        }
      }
    }
    __syncthreads();
    // ---- phase 3: trailing update of the lower block triangle ----
    const int nr = nbp - P - 1;
    if (nr > 0) {
      const int nblk = nr * (nr + 1) / 2;
      for (int it = warp; it < 4 * nblk; it += kCholWarps) {
        // block (I, J), I >= J, of the trailing part; quarter h of its rows
        int blk = it >> 2, I = 0;
        while (blk > I) {
          blk -= I + 1;
          ++I;
        }
        const int J = blk, h = it & 3;
        const int jr = kb + 32 + (J << 5) + lane;  // this lane's column of A
        float lj[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) lj[c] = L[jr * ld + kb + c];
        const int i0 = kb + 32 + (I << 5) + h * 8;
        for (int i = i0; i < i0 + 8; i += 2) {
          float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            s0[c & 3] = fmaf(L[i * ld + kb + c], lj[c], s0[c & 3]);
            s1[c & 3] = fmaf(L[(i + 1) * ld + kb + c], lj[c], s1[c & 3]);
          }
          L[i * ld + jr] -= (s0[0] + s0[1]) + (s0[2] + s0[3]);
          L[(i + 1) * ld + jr] -= (s1[0] + s1[1]) + (s1[2] + s1[3]);
        }
      }
    }
    __syncthreads();
  }
  // Rinv = S L^-T with S the unit-diagonal scaling: Rinv[i][j] = dsc[i] Li[j][i]
  double* R = out + pr.out_off;
  if ((b & 1) || (pr.out_off & 1)) {
    for (int q = tid; q < bb; q += kCholThreads) {
      const int i = q / b, j = q - i * b;
      R[q] = (drop[i] || drop[j] || j < i) ? 0.0 : f32_to_f64_scaled(rsc[i] * Li[j * ld + i], ksc[i]);
    }
  } else {
    // two neighbouring entries of a row per thread, one 16-byte store;
    // entries below the diagonal are zero without a look at Li
    double2* R2 = reinterpret_cast<double2*>(R);
    for (int q2 = tid; q2 < (bb >> 1); q2 += kCholThreads) {
      const int q = q2 << 1;
      const int i = q / b, j = q - i * b;
      double2 v = make_double2(0.0, 0.0);
      if (j + 1 >= i && !drop[i]) {
        const float r = rsc[i];
        const int e = ksc[i];
        if (j >= i && !drop[j]) v.x = f32_to_f64_scaled(r * Li[j * ld + i], e);
        if (!drop[j + 1]) v.y = f32_to_f64_scaled(r * Li[(j + 1) * ld + i], e);
      }
      R2[q2] = v;
    }
  }
}

// Partial Gram matrices in FP32 for the CholQR steps (whose factor is FP32
// anyway): CTA (p, s) adds x_r^T x_r over the rows r of slice s of problem p
// (rows [s M / nparts, (s + 1) M / nparts) of the row-major FP64 block X at
// x_off, row stride ld) and writes the b x b sum to out[out_off + s b^2].
// 256 threads as 16 x 16: thread (ti, tj) owns entries (ti + 16u, tj + 16v),
// u, v < 10 (b <= 160); rows are staged in shared memory 32 at a time.
struct GramProb {
  int32_t M, b;
  int64_t x_off, ld, out_off;
};

constexpr int kGramRows = 32;

// U x U entries per thread (ti + 16 u, tj + 16 v, u, v < U): U = 8 covers
// b <= 128, U = 10 covers b <= 160; the smaller instance does 64 instead of
// 100 multiply-adds per row for the common b = 128.
template <int U>
__device__ __forceinline__ void gram_f32_body(const GramProb& p, int s, int nparts, const double* __restrict__ X,
                                              float* __restrict__ out, float (*xs)[kEigMax + 4]) {
  const int r0 = int((long long)p.M * s / nparts), r1 = int((long long)p.M * (s + 1) / nparts);
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  for (int e = threadIdx.x; e < kGramRows * (kEigMax + 4); e += 256) (&xs[0][0])[e] = 0.f;
  float acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.f;
  for (int rb = r0; rb < r1; rb += kGramRows) {
    const int nr = min(kGramRows, r1 - rb);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * p.b; e += 256) {
      const int r = e / p.b, c = e - r * p.b;
      xs[r][c] = float(X[p.x_off + (long long)(rb + r) * p.ld + c]);
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      float a[U], c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = xs[r][ti + 16 * u];
        c[u] = xs[r][tj + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fmaf(a[u], c[v], acc[u][v]);
    }
  }
  float* o = out + p.out_off + (long long)s * p.b * p.b;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int i = ti + 16 * u, j = tj + 16 * v;
      if (i < p.b && j < p.b) o[i * p.b + j] = acc[u][v];
    }
}

__global__ void __launch_bounds__(256) gram_f32_kernel(const GramProb* __restrict__ probs, int nparts,
                                                       const double* __restrict__ X, float* __restrict__ out) {
  __shared__ float xs[kGramRows][kEigMax + 4];
  const GramProb p = probs[blockIdx.x];
  if (p.b <= 128) gram_f32_body<8>(p, int(blockIdx.y), nparts, X, out, xs);
  else gram_f32_body<10>(p, int(blockIdx.y), nparts, X, out, xs);
}

size_t cholinv_smem(int b) {
  // L, Li (bp x (bp + 1) floats), rsc (bp floats), ksc and drop (bp ints each)
  const int bp = (b + 31) & ~31;
  return sizeof(float) * (2 * size_t(bp) * (bp + 1) + 3 * size_t(bp));
}

// out = alpha * I + beta * in (square blocks)
// (grid: problems x row slices; CTA (p, y) takes rows y, y + gridDim.y, ...)
__global__ void ident_combo(const SmallProb* __restrict__ probs, const double* __restrict__ in, double* __restrict__ out,
                            double alpha, double beta) {
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b;
  for (int i = blockIdx.y; i < b; i += gridDim.y)
    for (int j = threadIdx.x; j < b; j += blockDim.x) {
      const long long q = (long long)i * b + j;
      out[pr.out_off + q] = (i == j ? alpha : 0.0) + beta * in[pr.in_off + q];
    }
}

// Deterministic pseudo-random normal entries (counter-based hash + Box-Muller).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// One launch fills several ranges: range blockIdx.y is x[off, off + n) with
// its own seed (table: off, n, seed as 64-bit words).
__global__ void randn_fill(double* x, const long long* __restrict__ ranges) {
  const long long off = ranges[3 * blockIdx.y], n = ranges[3 * blockIdx.y + 1];
  const uint64_t seed = static_cast<uint64_t>(ranges[3 * blockIdx.y + 2]);
  x += off;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t a = mix64(seed * 0x9E3779B97F4A7C15ull + 2 * i + 1);
    const uint64_t c = mix64(a ^ 0xD1B54A32D192ED03ull);
    const double u1 = (double((a >> 11) + 1)) * (1.0 / 9007199254740992.0);
    const double u2 = double(c >> 11) * (1.0 / 9007199254740992.0);
    x[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

// Residual norms of Ritz pairs: res_j = ||Y[:,j] - lam_j V[:,j]|| / lam_max
struct ResProb {
  int32_t m, k;
  int64_t y_off, v_off, val_off, ld;
};

__global__ void ritz_residual(const ResProb* __restrict__ probs, const double* __restrict__ Y,
                              const double* __restrict__ V, const double* __restrict__ vals, double* __restrict__ res) {
  const ResProb pr = probs[blockIdx.x];
  const int j = blockIdx.y;
  if (j >= pr.k) return;
  __shared__ double sh[256];
  const double lam = vals[pr.val_off + j];
  double acc = 0;
  for (int i = threadIdx.x; i < pr.m; i += blockDim.x) {
    const double r = Y[pr.y_off + (long long)i * pr.ld + j] - lam * V[pr.v_off + (long long)i * pr.ld + j];
    acc += r * r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[pr.val_off + j] = sqrt(sh[0]);
}

}  // namespace bst
