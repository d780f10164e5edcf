// Plain FP64 grouped GEMM on the FP64 tensor path (DMMA, mma.sync m8n8k4).
//
// This is the "plain FP64 GPU path": every matched sector GEMM of a
// contraction in one launch, one 64x64 output tile per CTA, operands read
// through generic element strides so transposed views need no copy.
#include <algorithm>

#include "bst_internal.h"

namespace bst {

const int kF64TileM = 64;
const int kF64TileN = 64;
constexpr int kBK = 16;
constexpr int kPad = 2;

void DevGemm::upload(const std::vector<GemmProb>& p, int tm, int tn, int order) {
  free_all();
  nprobs = int(p.size());
  flops = 0;
  for (auto& x : p) flops += 2.0 * double(x.M) * x.N * x.K;
  std::vector<int32_t> tp, ti;
  for (int i = 0; i < nprobs; ++i) {
    int mt = (p[i].M + tm - 1) / tm, nt = (p[i].N + tn - 1) / tn;
    for (int t = 0; t < mt * nt; ++t) {
      tp.push_back(i);
      ti.push_back(t);
    }
  }
  ntiles = int(tp.size());
  std::vector<int64_t> wo(std::max(nprobs, 1), 0);
  wtot = 0;
  maxK = 0;
  for (int i = 0; i < nprobs; ++i) {
    wo[i] = wtot;
    wtot += int64_t(p[i].M) * p[i].N;
    maxK = std::max(maxK, p[i].K);
  }
  hw_off.assign(wo.begin(), wo.begin() + nprobs);
  if (order == 1) {
    std::vector<int> idx(ntiles);
    for (int i = 0; i < ntiles; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return p[tp[x]].K > p[tp[y]].K; });
    std::vector<int32_t> tp2(ntiles), ti2(ntiles);
    for (int i = 0; i < ntiles; ++i) {
      tp2[i] = tp[idx[i]];
      ti2[i] = ti[idx[i]];
    }
    tp.swap(tp2);
    ti.swap(ti2);
  }
  if (nprobs) {
    BST_CUDA(cudaMalloc(&probs, sizeof(GemmProb) * nprobs));
    BST_CUDA(cudaMemcpy(probs, p.data(), sizeof(GemmProb) * nprobs, cudaMemcpyHostToDevice));
  }
  if (nprobs) {
    BST_CUDA(cudaMalloc(&w_off, sizeof(int64_t) * nprobs));
    BST_CUDA(cudaMemcpy(w_off, wo.data(), sizeof(int64_t) * nprobs, cudaMemcpyHostToDevice));
  }
  if (ntiles) {
    BST_CUDA(cudaMalloc(&tile_prob, sizeof(int32_t) * ntiles));
    BST_CUDA(cudaMalloc(&tile_idx, sizeof(int32_t) * ntiles));
    BST_CUDA(cudaMemcpy(tile_prob, tp.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice));
    BST_CUDA(cudaMemcpy(tile_idx, ti.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice));
  }
}

void DevGemm::free_all() {
  if (probs) cudaFree(probs);
  if (tile_prob) cudaFree(tile_prob);
  if (tile_idx) cudaFree(tile_idx);
  if (w_off) cudaFree(w_off);
  w_off = nullptr;
  probs = nullptr;
  tile_prob = tile_idx = nullptr;
  ntiles = nprobs = 0;
}

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// One 64x64 output tile of problem p over the K range [kb, ke), written to
// out[m * om + n * on].  128 threads = 4 warps in a 2x2 arrangement, each warp
// a 32x32 sub-tile made of 4x4 DMMA tiles of 8x8.  The operand tiles are
// double-buffered in shared memory: the next K block's loads are in flight
// (in registers) while the current block is multiplied.
constexpr int kLd = (kF64TileM * kBK) / 128;  // elements of a 64 x 16 tile per thread
__device__ __forceinline__ void f64_tile(const GemmProb& p, int m0, int n0, int kb, int ke,
                                         const double* __restrict__ A, const double* __restrict__ B,
                                         double* __restrict__ out, long long om, long long on,
                                         double (*sA)[kBK][kF64TileM + kPad], double (*sB)[kBK][kF64TileN + kPad]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tg = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  const double* Ap = A + p.a_off;
  const double* Bp = B + p.b_off;
  double ra[kLd], rb[kLd];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < kLd; ++u) {
      const int e = tid + u * 128;
      const int m = e / kBK, k = e % kBK;
      const int gm = m0 + m, gn = n0 + m, gk = k0 + k;
      ra[u] = (gm < p.M && gk < ke) ? Ap[(long long)gm * p.a_m + (long long)gk * p.a_k] : 0.0;
      rb[u] = (gn < p.N && gk < ke) ? Bp[(long long)gn * p.b_n + (long long)gk * p.b_k] : 0.0;
    }
  };
  if (kb < ke) fetch(kb);
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += kBK, buf ^= 1) {
#pragma unroll
    for (int u = 0; u < kLd; ++u) {
      const int e = tid + u * 128;
      sA[buf][e % kBK][e / kBK] = ra[u];
      sB[buf][e % kBK][e / kBK] = rb[u];
    }
    __syncthreads();
    if (k0 + kBK < ke) fetch(k0 + kBK);
    // (k steps past the end of the range hold only zero padding)
    const int kn = min(kBK, ke - k0);
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      if (kk >= kn) break;
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = sA[buf][kk + tg][wm + i * 8 + g];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = sB[buf][kk + tg][wn + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + i * 8 + g;
        const int gn = n0 + wn + j * 8 + tg * 2 + h;
        if (gm < p.M && gn < p.N) out[(long long)gm * om + (long long)gn * on] = acc[i][j][h];
      }
}

__global__ void __launch_bounds__(128, 3) gemm_f64_kernel(const GemmProb* __restrict__ probs,
                                                       const int32_t* __restrict__ tile_prob,
                                                       const int32_t* __restrict__ tile_idx,
                                                       const double* __restrict__ A,
                                                       const double* __restrict__ B, double* __restrict__ C) {
  __shared__ double sA[2][kBK][kF64TileM + kPad];
  __shared__ double sB[2][kBK][kF64TileN + kPad];
  const GemmProb p = probs[tile_prob[blockIdx.x]];
  const int nt = (p.N + kF64TileN - 1) / kF64TileN;
  const int m0 = (tile_idx[blockIdx.x] / nt) * kF64TileM;
  const int n0 = (tile_idx[blockIdx.x] % nt) * kF64TileN;
  f64_tile(p, m0, n0, 0, p.K, A, B, C + p.c_off, p.c_m, p.c_n, sA, sB);
}

// Split-K: CTA (tile, s) computes the partial product over the s-th K slice
// (slices of a multiple of 16) into W[s][problem][m][n]; the reduction adds
// the slices in a fixed order (deterministic result).
__global__ void __launch_bounds__(128, 3) gemm_f64_splitk_kernel(const GemmProb* __restrict__ probs,
                                                              const int32_t* __restrict__ tile_prob,
                                                              const int32_t* __restrict__ tile_idx,
                                                              const double* __restrict__ A,
                                                              const double* __restrict__ B, double* __restrict__ W,
                                                              const int64_t* __restrict__ w_off, long long wtot,
                                                              int ksplit) {
  __shared__ double sA[2][kBK][kF64TileM + kPad];
  __shared__ double sB[2][kBK][kF64TileN + kPad];
  const int pi = tile_prob[blockIdx.x];
  const GemmProb p = probs[pi];
  const int nt = (p.N + kF64TileN - 1) / kF64TileN;
  const int m0 = (tile_idx[blockIdx.x] / nt) * kF64TileM;
  const int n0 = (tile_idx[blockIdx.x] % nt) * kF64TileN;
  const int kc = ((p.K + ksplit - 1) / ksplit + kBK - 1) / kBK * kBK;
  const int kb = min(p.K, int(blockIdx.y) * kc), ke = min(p.K, kb + kc);
  f64_tile(p, m0, n0, kb, ke, A, B, W + blockIdx.y * wtot + w_off[pi], p.N, 1, sA, sB);
}

__global__ void gemm_f64_reduce_kernel(const GemmProb* __restrict__ probs, const double* __restrict__ W,
                                       const int64_t* __restrict__ w_off, long long wtot, int ksplit,
                                       double* __restrict__ C) {
  const GemmProb p = probs[blockIdx.y];
  const long long n = (long long)p.M * p.N;
  const double* w = W + w_off[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < ksplit; ++s) v += w[s * wtot + e];
    const long long m = e / p.N, c = e - m * p.N;
    C[p.c_off + m * p.c_m + c * p.c_n] = v;
  }
}

DevGemm* get_dev_gemm(Ctx* ctx, const std::string& key, const std::vector<GemmProb>& probs) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->gplans.find(key);
  if (it != ctx->gplans.end()) return it->second.get();
  auto g = std::make_unique<DevGemm>();
  g->upload(probs, kF64TileM, kF64TileN);
  DevGemm* raw = g.get();
  ctx->gplans[key] = std::move(g);
  return raw;
}

void launch_gemm_f64_splitk(Ctx* ctx, const DevGemm& g, int ksplit, const double* A, const double* B, double* C,
                            cudaStream_t s, const char* ws) {
  if (g.ntiles == 0) return;
  if (ksplit <= 1) {
    launch_gemm_f64(ctx, g, A, B, C, s);
    return;
  }
  double* W = (double*)ctx->buf(ws, sizeof(double) * std::max<int64_t>(1, g.wtot * ksplit), s);
  ProfScope ps(ctx, s, "gemm_f64", g.flops, 0.0);
  gemm_f64_splitk_kernel<<<dim3(unsigned(g.ntiles), unsigned(ksplit)), 128, 0, s>>>(
      g.probs, g.tile_prob, g.tile_idx, A, B, W, g.w_off, g.wtot, ksplit);
  gemm_f64_reduce_kernel<<<dim3(64, unsigned(g.nprobs)), 256, 0, s>>>(g.probs, W, g.w_off, g.wtot, ksplit, C);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx, 2);
}

void launch_ksplit_reduce(Ctx* ctx, const DevGemm& g, const double* W, int ksplit, double* C, cudaStream_t s) {
  if (g.nprobs == 0) return;
  gemm_f64_reduce_kernel<<<dim3(64, unsigned(g.nprobs)), 256, 0, s>>>(g.probs, W, g.w_off, g.wtot, ksplit, C);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

void launch_gemm_f64(Ctx* ctx, const DevGemm& g, const double* A, const double* B, double* C, cudaStream_t s) {
  if (g.ntiles == 0) return;
  ProfScope ps(ctx, s, "gemm_f64", g.flops, 0.0);
  gemm_f64_kernel<<<g.ntiles, 128, 0, s>>>(g.probs, g.tile_prob, g.tile_idx, A, B, C);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

}  // namespace bst
