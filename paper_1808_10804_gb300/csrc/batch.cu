// Batched contractions: many independent contractions (uneven sector sizes)
// in one launch per stage -- one gather of every A, one of every B, one
// grouped GEMM over the sector matrices of all of them, one scatter of every
// C.  The matched block pairs of all contractions form one task list, so the
// GPU is filled even when each contraction alone is small (Sec. 2: the
// block pairs are independent, "straightforward to parallelise over").
//
// The per-contraction plans are the cached single-contraction plans; the
// batch plan concatenates their sector matrices into three combined buffers
// and tags every relayout task with the index of its tensor, whose device
// address comes from a small pointer table.  Each distinct set of data
// pointers gets its own table, uploaded once and kept with the plan, so a
// repeated call uploads nothing and a captured CUDA graph of it stays valid
// while other pointer sets are used in between.
#include <algorithm>
#include <cstring>

#include "bst_internal.h"

namespace bst {

struct BatchTask {
  RelTask t;     // t.blk_off is relative to bases[src]
  int32_t src;
  int32_t pad;
};

struct BatchRel {
  BatchTask* tasks = nullptr;
  int2* chunks = nullptr;
  int nchunks = 0;
  double elems = 0;
};

struct BatchPlan {
  std::vector<ContractPlan*> plans;
  int64_t amat = 0, bmat = 0, cmat = 0;
  BatchRel ra, rb, rc;
  std::vector<GemmProb> probs;
  DevGemm g;
  // data pointers (a[0..n), b[0..n), c[0..n)) -> device copy of that table
  std::map<std::vector<const void*>, double**> tables;
  // the plan's own sector-matrix buffers: a captured graph of this batch
  // keeps valid addresses for as long as the plan (the context) lives
  double *Am = nullptr, *Bm = nullptr, *Cm = nullptr;
  ~BatchPlan() {
    cudaFree(Am);
    cudaFree(Bm);
    cudaFree(Cm);
    cudaFree(ra.tasks);
    cudaFree(ra.chunks);
    cudaFree(rb.tasks);
    cudaFree(rb.chunks);
    cudaFree(rc.tasks);
    cudaFree(rc.chunks);
    for (auto& kv : tables) cudaFree(kv.second);
    g.free_all();
  }
};

constexpr int kBatchChunk = 2048;
constexpr int kBatchThreads = 256;

// Same element mapping as relayout_kernel, with a per-task base pointer.
__global__ void __launch_bounds__(kBatchThreads) relayout_batch_kernel(const BatchTask* __restrict__ tasks,
                                                                       const int2* __restrict__ chunks,
                                                                       double* const* __restrict__ bases,
                                                                       double* mat, int dir, double alpha,
                                                                       double beta) {
  const int2 c = chunks[blockIdx.x];
  const BatchTask& bt = tasks[c.x];
  const RelTask& t = bt.t;
  double* blk = bases[bt.src];
  const int r = t.rank;
  int shape[kMaxRank];
  long long ms[kMaxRank];
#pragma unroll
  for (int i = 0; i < kMaxRank; ++i) {
    shape[i] = i < r ? t.shape[i] : 1;
    ms[i] = i < r ? t.mstride[i] : 0;
  }
  const int end = min(t.n, c.y + kBatchChunk);
  for (int e = c.y + threadIdx.x; e < end; e += kBatchThreads) {
    int rem = e;
    long long mo = t.mat_base;
#pragma unroll
    for (int i = kMaxRank - 1; i >= 0; --i) {
      if (i < r) {
        const int ii = rem % shape[i];
        rem /= shape[i];
        mo += ii * ms[i];
      }
    }
    const long long bo = t.blk_off + e;
    if (dir == 0) {
      mat[mo] = blk[bo];
    } else {
      double v = alpha * mat[mo];
      if (beta != 0.0) v += beta * blk[bo];
      blk[bo] = v;
    }
  }
}

static void upload_rel(BatchRel& r, const std::vector<BatchTask>& tasks) {
  std::vector<int2> ch;
  r.elems = 0;
  for (int i = 0; i < int(tasks.size()); ++i) {
    r.elems += tasks[i].t.n;
    for (int s = 0; s < tasks[i].t.n; s += kBatchChunk) ch.push_back(make_int2(i, s));
  }
  r.nchunks = int(ch.size());
  if (!tasks.empty()) {
    BST_CUDA(cudaMalloc(&r.tasks, sizeof(BatchTask) * tasks.size()));
    BST_CUDA(cudaMemcpy(r.tasks, tasks.data(), sizeof(BatchTask) * tasks.size(), cudaMemcpyHostToDevice));
  }
  if (!ch.empty()) {
    BST_CUDA(cudaMalloc(&r.chunks, sizeof(int2) * ch.size()));
    BST_CUDA(cudaMemcpy(r.chunks, ch.data(), sizeof(int2) * ch.size(), cudaMemcpyHostToDevice));
  }
}

static void launch_rel(Ctx* ctx, const BatchRel& r, double* const* bases, double* mat, int dir, double alpha,
                       double beta, cudaStream_t s) {
  if (r.nchunks == 0) return;
  ProfScope ps(ctx, s, "relayout", 0.0, 16.0 * r.elems);
  relayout_batch_kernel<<<r.nchunks, kBatchThreads, 0, s>>>(r.tasks, r.chunks, bases, mat, dir, alpha, beta);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

static BatchPlan* get_batch_plan(Ctx* ctx, const std::vector<Layout*>& A, const std::vector<Layout*>& B,
                                 const std::vector<int>& la, const std::vector<int>& lb) {
  std::vector<ContractPlan*> plans;
  std::string key = "batch/";
  for (size_t i = 0; i < A.size(); ++i) {
    ContractPlan* p = get_contract_plan(ctx, A[i], B[i], la, lb);
    plans.push_back(p);
    key += std::to_string(uintptr_t(p)) + ",";
  }
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->bplans.find(key);
    if (it != ctx->bplans.end()) return it->second.get();
  }
  auto bp = std::make_shared<BatchPlan>();
  bp->plans = plans;
  std::vector<BatchTask> ta, tb, tc;
  for (size_t i = 0; i < plans.size(); ++i) {
    ContractPlan* p = plans[i];
    for (auto t : p->va.tasks) {
      t.mat_base += bp->amat;
      ta.push_back({t, int32_t(i), 0});
    }
    for (auto t : p->vb.tasks) {
      t.mat_base += bp->bmat;
      tb.push_back({t, int32_t(i), 0});
    }
    for (auto t : p->vc.tasks) {
      t.mat_base += bp->cmat;
      tc.push_back({t, int32_t(i), 0});
    }
    for (auto g : p->probs) {
      g.a_off += bp->amat;
      g.b_off += bp->bmat;
      g.c_off += bp->cmat;
      bp->probs.push_back(g);
    }
    bp->amat += p->amat;
    bp->bmat += p->bmat;
    bp->cmat += p->cmat;
  }
  upload_rel(bp->ra, ta);
  upload_rel(bp->rb, tb);
  upload_rel(bp->rc, tc);
  bp->g.upload(bp->probs, kF64TileM, kF64TileN);
  BST_CUDA(cudaMalloc(&bp->Am, sizeof(double) * std::max<int64_t>(bp->amat, 1)));
  BST_CUDA(cudaMalloc(&bp->Bm, sizeof(double) * std::max<int64_t>(bp->bmat, 1)));
  BST_CUDA(cudaMalloc(&bp->Cm, sizeof(double) * std::max<int64_t>(bp->cmat, 1)));
  BatchPlan* raw = bp.get();
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->bplans[key] = std::move(bp);
  return raw;
}

void contract_batched(Ctx* ctx, const std::vector<Layout*>& A, const std::vector<const double*>& a,
                      const std::vector<Layout*>& B, const std::vector<const double*>& b, const std::vector<int>& la,
                      const std::vector<int>& lb, bst_prec prec, double alpha, double beta,
                      const std::vector<Layout*>& C, const std::vector<double*>& c, cudaStream_t s) {
  const size_t n = A.size();
  BST_REQUIRE(n >= 1 && B.size() == n && C.size() == n && a.size() == n && b.size() == n && c.size() == n,
              BST_E_ARG, "batch arrays must all have nbatch entries");
  BatchPlan* bp = get_batch_plan(ctx, A, B, la, lb);
  for (size_t i = 0; i < n; ++i) {
    BST_REQUIRE(bp->plans[i]->C == C[i], BST_E_SHAPE, "C[i] is not the layout of contraction i");
    BST_REQUIRE((A[i]->nnz == 0 || a[i]) && (B[i]->nnz == 0 || b[i]) && (C[i]->nnz == 0 || c[i]), BST_E_ARG,
                "data pointer is NULL");
  }
  std::vector<const void*> ptrs;
  for (size_t i = 0; i < n; ++i) ptrs.push_back(a[i]);
  for (size_t i = 0; i < n; ++i) ptrs.push_back(b[i]);
  for (size_t i = 0; i < n; ++i) ptrs.push_back(c[i]);
  double** bases = nullptr;
  auto it = bp->tables.find(ptrs);
  if (it != bp->tables.end()) {
    bases = it->second;
  } else {
    // first call with this pointer set: allocate and fill its table (not
    // capturable; later calls with the same pointers only launch)
    BST_CUDA(cudaMalloc(&bases, sizeof(void*) * ptrs.size()));
    BST_CUDA(cudaMemcpy(bases, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice));
    bp->tables[ptrs] = bases;
  }
  double *Am = bp->Am, *Bm = bp->Bm, *Cm = bp->Cm;
  launch_rel(ctx, bp->ra, bases, Am, 0, 1.0, 0.0, s);
  launch_rel(ctx, bp->rb, bases + n, Bm, 0, 1.0, 0.0, s);
  if (prec == BST_FP64) {
    launch_gemm_f64(ctx, bp->g, Am, Bm, Cm, s);
  } else {
    // the same grouped tensor-core GEMM as a single contraction, over the
    // problems of all contractions
    run_gemm_ozaki_probs(ctx, "batch/" + std::to_string(uintptr_t(bp)), bp->probs, Am, Bm, Cm, s);
  }
  launch_rel(ctx, bp->rc, bases + 2 * n, Cm, 1, alpha, beta, s);
}

}  // namespace bst
