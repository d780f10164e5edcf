// Relayout kernel (block permute / fuse / sector-matrix gather and scatter)
// and small helper kernels.
//
// Every relayout is a list of tasks; a task moves one contiguous block,
// row-major over its own leg order, to or from a strided region of another
// buffer.  The work is split into chunks of kChunk elements, one CTA per
// chunk, so uneven block sizes load-balance across the 152 SMs.
#include <algorithm>

#include "bst_internal.h"
#include "relayout_dev.cuh"

namespace bst {

ProfScope::ProfScope(Ctx* ctx, cudaStream_t st, const char* cls, double flops, double bytes) : c(ctx), s(st) {
  if (!c->prof) return;
  while (c->evpool.size() < c->evused + 2) {
    cudaEvent_t e;
    BST_CUDA(cudaEventCreate(&e));
    c->evpool.push_back(e);
  }
  ProfRec r{cls, c->evpool[c->evused], c->evpool[c->evused + 1], flops, bytes};
  c->evused += 2;
  BST_CUDA(cudaEventRecord(r.a, s));
  idx = long(c->recs.size());
  c->recs.push_back(r);
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(c->recs[idx].b, s);
}

constexpr int kChunk = 2048;
constexpr int kRelThreads = 256;

std::vector<int2> relayout_chunks(const std::vector<RelTask>& t) {
  std::vector<int2> ch;
  for (int i = 0; i < int(t.size()); ++i)
    for (int s = 0; s < t[i].n; s += kChunk) ch.push_back(make_int2(i, s));
  return ch;
}

void DevRelayout::upload(const std::vector<RelTask>& t) {
  free_all();
  ntasks = int(t.size());
  elems = 0;
  for (auto& x : t) elems += x.n;
  std::vector<int2> ch;
  for (int i = 0; i < ntasks; ++i)
    for (int s = 0; s < t[i].n; s += kChunk) ch.push_back(make_int2(i, s));
  nchunks = int(ch.size());
  if (ntasks) {
    BST_CUDA(cudaMalloc(&tasks, sizeof(RelTask) * ntasks));
    BST_CUDA(cudaMemcpy(tasks, t.data(), sizeof(RelTask) * ntasks, cudaMemcpyHostToDevice));
  }
  if (nchunks) {
    BST_CUDA(cudaMalloc(&chunks, sizeof(int2) * nchunks));
    BST_CUDA(cudaMemcpy(chunks, ch.data(), sizeof(int2) * nchunks, cudaMemcpyHostToDevice));
  }
}

void DevRelayout::free_all() {
  if (tasks) cudaFree(tasks);
  if (chunks) cudaFree(chunks);
  tasks = nullptr;
  chunks = nullptr;
  ntasks = nchunks = 0;
}

void* DevBuf::get(size_t need, cudaStream_t s) {
  if (need <= bytes) return p;
  if (p) {
    // the stream may still read the old buffer
    BST_CUDA(cudaStreamSynchronize(s));
    BST_CUDA(cudaFree(p));
    p = nullptr;
    bytes = 0;
  }
  size_t nb = std::max(need, size_t(256));
  if (cudaMalloc(&p, nb) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    throw Error(BST_E_OOM, "device workspace allocation failed");
  }
  bytes = nb;
  return p;
}

void DevBuf::free_all() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

// dir 0: mat[strided] = blk[contiguous]
// dir 1: blk[contiguous] = alpha * mat[strided] + beta * blk   (beta == 0: overwrite)
__global__ void __launch_bounds__(kRelThreads) relayout_kernel(const RelTask* __restrict__ tasks,
                                                               const int2* __restrict__ chunks,
                                                               double* blk, double* mat, int dir,
                                                               double alpha, double beta) {
  const int2 c = chunks[blockIdx.x];
  const RelTask& t = tasks[c.x];
  relayout_range<kRelThreads>(t, c.y, min(t.n, c.y + kChunk), blk, mat, dir, alpha, beta);
}

void launch_relayout(Ctx* ctx, const DevRelayout& r, const double* blk, double* mat, int dir, double alpha,
                     double beta, cudaStream_t s) {
  if (r.nchunks == 0) return;
  ProfScope ps(ctx, s, "relayout", 0.0, 16.0 * r.elems);
  relayout_kernel<<<r.nchunks, kRelThreads, 0, s>>>(r.tasks, r.chunks, const_cast<double*>(blk), mat, dir,
                                                     alpha, beta);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

__global__ void scale_kernel(double* x, long long n, const double* inv) {
  const double f = 1.0 / sqrt(*inv);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= f;
}

// x /= sqrt(*sumsq)
void launch_scale(Ctx* ctx, double* x, int64_t n, const double* dev_sumsq, cudaStream_t s) {
  if (n == 0) return;
  int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  scale_kernel<<<grid, 256, 0, s>>>(x, n, dev_sumsq);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

// Sum of squares in FP64: per-CTA partial sums, then one CTA adds them in a
// fixed order (deterministic result).
__global__ void sumsq_partial(const double* x, long long n, double* part) {
  __shared__ double sh[256];
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += x[i] * x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sumsq_final(const double* part, int np, double* out) {
  __shared__ double sh[256];
  double acc = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Weighted sum of squares sum_i w_i x_i^2 (per-CTA partials, then one CTA in
// a fixed order): the Frobenius norm of an SU(2) tensor from its reduced
// blocks, w = 2J+1 of the element's block.
__global__ void sumsq_w_partial(const double* x, const double* w, long long n, double* part) {
  __shared__ double sh[256];
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += w[i] * x[i] * x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

void launch_sumsq_w(Ctx* ctx, const double* x, const double* w, int64_t n, double* dev_out, cudaStream_t s) {
  int grid = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 304)));
  double* part = (double*)ctx->buf("sumsq.part", sizeof(double) * 304, s);
  sumsq_w_partial<<<grid, 256, 0, s>>>(x, w, n, part);
  sumsq_final<<<1, 256, 0, s>>>(part, grid, dev_out);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx, 2);
}

void launch_sumsq(Ctx* ctx, const double* x, int64_t n, double* dev_out, cudaStream_t s) {
  int grid = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 304)));
  double* part = (double*)ctx->buf("sumsq.part", sizeof(double) * 304, s);
  sumsq_partial<<<grid, 256, 0, s>>>(x, n, part);
  sumsq_final<<<1, 256, 0, s>>>(part, grid, dev_out);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx, 2);
}

__global__ void fill_kernel(double* x, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

void launch_fill(Ctx* ctx, double* x, int64_t n, double v, cudaStream_t s) {
  if (n == 0) return;
  int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  fill_kernel<<<grid, 256, 0, s>>>(x, n, v);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

}  // namespace bst
