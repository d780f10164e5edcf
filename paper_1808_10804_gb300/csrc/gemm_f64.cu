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
  probs = nullptr;
  tile_prob = tile_idx = nullptr;
  ntiles = nprobs = 0;
}

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// 128 threads = 4 warps in a 2x2 arrangement, each warp a 32x32 sub-tile
// made of 4x4 DMMA tiles of 8x8.
__global__ void __launch_bounds__(128) gemm_f64_kernel(const GemmProb* __restrict__ probs,
                                                       const int32_t* __restrict__ tile_prob,
                                                       const int32_t* __restrict__ tile_idx,
                                                       const double* __restrict__ A,
                                                       const double* __restrict__ B, double* __restrict__ C) {
  __shared__ double sA[kBK][kF64TileM + kPad];
  __shared__ double sB[kBK][kF64TileN + kPad];
  const GemmProb p = probs[tile_prob[blockIdx.x]];
  const int nt = (p.N + kF64TileN - 1) / kF64TileN;
  const int m0 = (tile_idx[blockIdx.x] / nt) * kF64TileM;
  const int n0 = (tile_idx[blockIdx.x] % nt) * kF64TileN;
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
  for (int k0 = 0; k0 < p.K; k0 += kBK) {
#pragma unroll
    for (int e = tid; e < kF64TileM * kBK; e += 128) {
      const int m = e / kBK, k = e % kBK;
      const int gm = m0 + m, gk = k0 + k;
      sA[k][m] = (gm < p.M && gk < p.K) ? Ap[(long long)gm * p.a_m + (long long)gk * p.a_k] : 0.0;
      const int gn = n0 + m;
      sB[k][m] = (gn < p.N && gk < p.K) ? Bp[(long long)gn * p.b_n + (long long)gk * p.b_k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = sA[kk + tg][wm + i * 8 + g];
#pragma unroll
      for (int j = 0; j < 4; ++j) bf[j] = sB[kk + tg][wn + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], af[i], bf[j]);
    }
    __syncthreads();
  }
  double* Cp = C + p.c_off;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gm = m0 + wm + i * 8 + g;
        const int gn = n0 + wn + j * 8 + tg * 2 + h;
        if (gm < p.M && gn < p.N) Cp[(long long)gm * p.c_m + (long long)gn * p.c_n] = acc[i][j][h];
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

void launch_gemm_f64(Ctx* ctx, const DevGemm& g, const double* A, const double* B, double* C, cudaStream_t s) {
  if (g.ntiles == 0) return;
  ProfScope ps(ctx, s, "gemm_f64", g.flops, 0.0);
  gemm_f64_kernel<<<g.ntiles, 128, 0, s>>>(g.probs, g.tile_prob, g.tile_idx, A, B, C);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

}  // namespace bst
