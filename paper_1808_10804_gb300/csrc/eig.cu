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
  constexpr float kTau = 1e-5f;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test relative to the diagonal (keeps small eigenvalues
    // accurate) with a floor tfloor below which values are not resolved:
    // max_{i<j} a_ij^2 / (max(|a_ii|, tfloor) max(|a_jj|, tfloor)); with a
    // floor of 1 (the scale) the test is absolute.  Pairs whose diagonal
    // entries are both below `junk` are left out (a cluster at the FP32
    // rounding level of the input, where rotations only move noise); one
    // thread per row
    float worst = 0.f;
    for (int i = tid; i < b; i += nt) {
      const float ai = fabsf(A[i * ld + i]);
      const float di = fmaxf(ai, tfloor);
      for (int j = i + 1; j < b; ++j) {
        const float a = A[i * ld + j];
        const float aj = fabsf(A[j * ld + j]);
        if (fmaxf(ai, aj) >= junk) worst = fmaxf(worst, a * a / (di * fmaxf(aj, tfloor)));
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
      // rows: A <- J^T A; thread (column j, pair group g) applies the
      // rotations k = g, g + G, ... (disjoint rows, so no conflicts)
      const int G = nt / bp > 0 ? nt / bp : 1;
      const int jcol = tid % bp, grp = tid / bp;
      if (grp < G) {
        const int j = jcol;
        for (int k = grp; k < npair; k += G) {
          const float4 pr = prm[k];
          const float c = pr.x, s = pr.y;
          if (s == 0.f) continue;
          const int p = __float_as_int(pr.z), q = __float_as_int(pr.w);
          const float ap = A[p * ld + j], aq = A[q * ld + j];
          A[p * ld + j] = c * ap - s * aq;
          A[q * ld + j] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns: A <- A J, V <- V J; thread (row i, pair group g)
      if (grp < G) {
        const int i = jcol;
        for (int k = grp; k < npair; k += G) {
          const float4 pr = prm[k];
          const float c = pr.x, s = pr.y;
          if (s == 0.f) continue;
          const int p = __float_as_int(pr.z), q = __float_as_int(pr.w);
          const float ap = A[i * ld + p], aq = A[i * ld + q];
          A[i * ld + p] = c * ap - s * aq;
          A[i * ld + q] = s * ap + c * aq;
          const float vp = V[i * ld + p], vq = V[i * ld + q];
          V[i * ld + p] = c * vp - s * vq;
          V[i * ld + q] = s * vp + c * vq;
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

size_t jacobi_smem(int b) {
  const int bp = b + (b & 1);
  return sizeof(float) * (2 * bp * (bp + 1) + bp + 1024) + sizeof(int) * (bp + bp);
}

// Ogita-Aishima step, elementwise part.  In: XtX (b x b), S = X^T H X.
// Out: E (b x b) and lam (b):  R = I - XtX, lam_i = S_ii / (1 - R_ii),
// E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) when the pair is separated,
// |lam_i - lam_j| > rel_delta * max(|lam_i|, |lam_j|) and not both below
// junk * max|lam| (values the FP32 stage cannot resolve), else R_ij / 2.
// Grid (problem, slice): every CTA forms the b values in shared memory
// (slice 0 also stores them) and then its slice of the b x b entries, so
// the FP64 divisions spread over the whole GPU.
__global__ void oa_update(const SmallProb* __restrict__ probs, const double* __restrict__ XtX,
                          const double* __restrict__ S, double* __restrict__ E, double* __restrict__ lam,
                          double rel_delta, double junk) {
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
    const double delta = rel_delta * fmax(fabs(l[i]), fabs(l[j])) + 1e-300 * smax;
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

// FP32 Cholesky of M (b x b, FP64 in) and Rinv = (L^T)^-1 (upper, FP64 out).
// 512 threads; b <= 160.
__global__ void __launch_bounds__(512) cholinv_f32(const SmallProb* __restrict__ probs, const double* __restrict__ in,
                                                  double* __restrict__ out, int* err) {
  extern __shared__ float sh[];
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b, ld = b + 1, bb = b * b;
  float* L = sh;            // b x ld
  float* Li = L + b * ld;   // b x ld, inverse of L
  int* drop = reinterpret_cast<int*>(Li + b * ld + b);
  float* rsc = Li + b * ld;                                  // b row scales: mantissas
  int* ksc = reinterpret_cast<int*>(Li + b * ld + 2 * b);    // b row scales: exponents
  const double* M = in + pr.in_off;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  // scale by the diagonal so the factorisation sees unit diagonal: row i is
  // scaled by 1/sqrt(M_ii) = rsc[i] 2^ksc[i] (one FP64 square root and
  // division per row); the entries take the power of two exactly in the
  // conversion to FP32 and the mantissas as two FP32 products
  for (int i = tid; i < b; i += nt) {
    const double d = M[(long long)i * b + i];
    int k = 0;
    float r = 1.f;
    if (d > 0) split_pow2(1.0 / sqrt(d), &k, &r);
    ksc[i] = k;
    rsc[i] = r;
  }
  __syncthreads();
  // eight global loads in flight per thread
  for (int q0 = tid; q0 < bb; q0 += 8 * nt) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * nt;
      v[u] = q < bb ? M[q] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * nt;
      if (q < bb) {
        const int i = q / b, j = q - i * b;
        L[i * ld + j] = f64_to_f32_scaled(v[u], ksc[i] + ksc[j]) * (rsc[i] * rsc[j]);
        Li[i * ld + j] = 0.f;
      }
    }
  }
  __syncthreads();
  // Blocked right-looking factorisation with 32-wide panels.  Warp 0
  // factors the diagonal block D in registers (lane i holds row i, pivots
  // and column entries travel by warp shuffles) and forms D^-1 column by
  // lane (stored as the diagonal block of Li).  The panel below is then panel * D^-T, and
  // all threads update the trailing lower triangle.  Columns whose pivot
  // falls below 1e-6 (numerically dependent on earlier ones at FP32 level)
  // are dropped: their row and column of the factor become the identity
  // and their column of Rinv is zero.
  for (int kb = 0; kb < b; kb += 32) {
    const int w = min(32, b - kb);
    if (warp == 0) {
      float row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = (lane < w && c < w) ? L[(kb + lane) * ld + kb + c] : 0.f;
      int mydrop = 0;
      float myinv = 1.f;  // 1 / D[lane][lane]
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (k < w) {
          const float dkk = __shfl_sync(0xffffffffu, row[k], k);
          const bool dk = !(dkk > 1e-6f);  // the same on every lane
          const float inv = dk ? 1.f : rsqrtf(dkk);
          const bool me = lane == k;
          row[k] = me ? (dk ? 1.f : dkk * inv) : (lane > k ? (dk ? 0.f : row[k] * inv) : row[k]);
          mydrop = me ? int(dk) : mydrop;
          myinv = me ? inv : myinv;
          if (dk) {
            // row k of the factor becomes that of the identity
#pragma unroll
            for (int c = 0; c < k; ++c) row[c] = me ? 0.f : row[c];
          } else {
#pragma unroll
            for (int j = k + 1; j < 32; ++j) {
              const float ljk = __shfl_sync(0xffffffffu, row[k], j);
              row[j] = lane >= j ? fmaf(-row[k], ljk, row[j]) : row[j];
            }
          }
        }
      }
      // column `lane` of D^-1 by forward substitution, D[i][k] and
      // 1 / D[i][i] broadcast from lane i
      float col[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float acc = (i == lane) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) acc = fmaf(-__shfl_sync(0xffffffffu, row[k], i), col[k], acc);
        col[i] = acc * __shfl_sync(0xffffffffu, myinv, i);
      }
      if (lane < w) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c < w) L[(kb + lane) * ld + kb + c] = row[c];
        drop[kb + lane] = mydrop;
      }
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (i < w && lane < w) Li[(kb + i) * ld + kb + lane] = col[i];
    }
    __syncthreads();
    // dropped columns of this block: zero their rows left of the block too
    for (int c = 0; c < w; ++c)
      if (drop[kb + c])
        for (int j = tid; j < kb; j += nt) L[(kb + c) * ld + j] = 0.f;
    // panel: rows i >= kb+w, L[i][kb..kb+w) <- L[i][kb..] D^-T; four threads
    // per row, eight columns each; the row is read whole before any thread
    // of it writes
    const int m = b - kb - w;
    for (int base = 0; base < 4 * m; base += nt) {
      const int item = base + tid;
      const bool act = item < 4 * m;
      const int i = kb + w + (act ? item >> 2 : 0), g = item & 3;
      float y[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) y[c] = (act && c < w) ? L[i * ld + kb + c] : 0.f;
      __syncthreads();
      if (act) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = 8 * g + u;
          if (c < w) {
            // D^-1 is lower triangular (zeros above its diagonal); columns
            // past the block (y = 0 there) read a valid entry instead
            const float* dinv = Li + (kb + c) * ld + kb;
            float acc = 0.f;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) acc = fmaf(y[cc], dinv[cc < w ? cc : 0], acc);
            L[i * ld + kb + c] = drop[kb + c] ? 0.f : acc;
          }
        }
      }
    }
    __syncthreads();
    // trailing update: L[i][j] -= sum_c L[i][kb+c] L[j][kb+c], kb+w <= j <= i;
    // a thread takes columns jj and m-1-jj (m+1 rows together, so the
    // threads are balanced) and every P-th row of them
    if (m > 0) {
      const int half = (m + 1) / 2;
      const int P = nt / half > 0 ? nt / half : 1;
      const int pj = tid % half, ph = tid / half;
      if (ph < P) {
        for (int side = 0; side < 2; ++side) {
          const int jj = side == 0 ? pj : m - 1 - pj;
          if (side == 1 && jj == pj) break;  // odd m: the middle column once
          const int j = kb + w + jj;
          float lj[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) lj[c] = c < w ? L[j * ld + kb + c] : 0.f;
          for (int i = j + ph; i < b; i += P) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < 32; ++c) acc += L[i * ld + kb + (c < w ? c : 0)] * lj[c];
            L[i * ld + j] -= acc;
          }
        }
      }
    }
    __syncthreads();
  }
  // inverse of the lower factor by block rows (the diagonal blocks D^-1 are
  // in place): Li[I][J] = -D_I^-1 sum_{K=J}^{I-1} L[I][K] Li[K][J].  Thread
  // (warp ty, lane tx) owns rows ib+ty, ib+ty+16 and columns tx+32s, s < I.
  const int nb = (b + 31) / 32;
  for (int I = 1; I < nb; ++I) {
    const int ib = I * 32;
    const int r0 = min(ib + warp, b - 1), r1 = min(ib + warp + 16, b - 1);
    // T[i][j] = sum_{k < ib} L[i][k] Li[k][j], stashed in the (unused)
    // upper triangle of Li at [j][i]
    float acc[2][4];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[0][s] = acc[1][s] = 0.f;
    // k by 32-row segments: in segment g the column groups s <= g take part
    // (Li[k][j] is zero for k < j, and the rows above block s hold earlier
    // stashes)
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g < I) {
        for (int k = 32 * g; k < 32 * g + 32; ++k) {
          const float a0 = L[r0 * ld + k], a1 = L[r1 * ld + k];
#pragma unroll
          for (int s = 0; s <= g; ++s) {
            const float v = Li[k * ld + lane + 32 * s];
            acc[0][s] = fmaf(a0, v, acc[0][s]);
            acc[1][s] = fmaf(a1, v, acc[1][s]);
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < I) {
        const int j = lane + 32 * s;
        if (ib + warp < b) Li[j * ld + ib + warp] = acc[0][s];
        if (ib + warp + 16 < b) Li[j * ld + ib + warp + 16] = acc[1][s];
      }
    __syncthreads();
    // Li[i][j] = -sum_{k in block I} D_I^-1[i][k] T[k][j]
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[0][s] = acc[1][s] = 0.f;
    const int wi = min(32, b - ib);
    for (int kk = 0; kk < wi; ++kk) {
      const int k = ib + kk;
      const float a0 = Li[r0 * ld + k], a1 = Li[r1 * ld + k];
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (s < I) {
          const float v = Li[(lane + 32 * s) * ld + k];
          acc[0][s] = fmaf(a0, v, acc[0][s]);
          acc[1][s] = fmaf(a1, v, acc[1][s]);
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < I) {
        const int j = lane + 32 * s;
        if (ib + warp < b) Li[(ib + warp) * ld + j] = -acc[0][s];
        if (ib + warp + 16 < b) Li[(ib + warp + 16) * ld + j] = -acc[1][s];
      }
    __syncthreads();
  }
  // Rinv = D^-1/2-scaled (L^-1)^T:  M = D^1/2 L L^T D^1/2  =>  with
  // Q = Y Rinv and Rinv[i][j] = dsc[i] * Li[j][i] = (rsc[i] Li[j][i]) 2^ksc[i]
  double* R = out + pr.out_off;
  for (int q0 = tid; q0 < bb; q0 += 4 * nt) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * nt;
      if (q < bb) {
        const int i = q / b, j = q - i * b;
        R[q] = (drop[i] || drop[j] || j < i) ? 0.0 : f32_to_f64_scaled(rsc[i] * Li[j * ld + i], ksc[i]);
      }
    }
  }
}

size_t cholinv_smem(int b) {
  // L, Li (b x (b+1) floats), rsc (b floats), drop (b ints), ksc (b ints)
  return sizeof(float) * (2 * b * (b + 1) + 3 * b);
}

// out = alpha * I + beta * in (square blocks)
__global__ void ident_combo(const SmallProb* __restrict__ probs, const double* __restrict__ in, double* __restrict__ out,
                            double alpha, double beta) {
  const SmallProb pr = probs[blockIdx.x];
  const int b = pr.b;
  for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
    const int i = q / b, j = q % b;
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

__global__ void randn_fill(double* x, long long n, uint64_t seed) {
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
