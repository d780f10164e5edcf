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
#include "relayout_dev.cuh"

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
  int chunk = 2048;  // elements per CTA
  double elems = 0;
  std::vector<BatchTask> host;
  void free_all() {
    cudaFree(tasks);
    cudaFree(chunks);
    tasks = nullptr;
    chunks = nullptr;
  }
};

struct BatchPlan {
  std::vector<ContractPlan*> plans;
  int64_t amat = 0, bmat = 0, cmat = 0;
  BatchRel ra, rb, rc;
  std::vector<GemmProb> probs;
  DevGemm g;
  // schedule chosen by the autotuner (defaults until tuned)
  bool tuned_rel = false;
  // per arithmetic (BST_FP64, BST_OZAKI, BST_BF16X3): tile schedule and,
  // for the tensor-core GEMM, the output tile width (128 x 64 or 128 x 32)
  bool tuned[3] = {false, false, false};
  int order[3] = {0, 0, 0};
  int tn[3] = {0, 0, 0};
  // data pointers (a[0..n), b[0..n), c[0..n)) -> device copy of that table
  std::map<std::vector<const void*>, double**> tables;
  // the plan's own sector-matrix buffers: a captured graph of this batch
  // keeps valid addresses for as long as the plan (the context) lives
  double *Am = nullptr, *Bm = nullptr, *Cm = nullptr;
  ~BatchPlan() {
    cudaFree(Am);
    cudaFree(Bm);
    cudaFree(Cm);
    ra.free_all();
    rb.free_all();
    rc.free_all();
    for (auto& kv : tables) cudaFree(kv.second);
    g.free_all();
  }
};

constexpr int kBatchThreads = 256;
constexpr int kChunkChoices[] = {1024, 2048, 4096, 8192};

// Same element mapping as relayout_kernel, with a per-task base pointer.
__global__ void __launch_bounds__(kBatchThreads) relayout_batch_kernel(const BatchTask* __restrict__ tasks,
                                                                       const int2* __restrict__ chunks,
                                                                       double* const* __restrict__ bases,
                                                                       double* mat, int dir, double alpha,
                                                                       double beta, int chunk) {
  const int2 c = chunks[blockIdx.x];
  const BatchTask& bt = tasks[c.x];
  relayout_range<kBatchThreads>(bt.t, c.y, min(bt.t.n, c.y + chunk), bases[bt.src], mat, dir, alpha, beta);
}

// (Re)build the chunk table of a relayout for `chunk` elements per CTA.
static void upload_rel(BatchRel& r, int chunk) {
  r.free_all();
  r.chunk = chunk;
  std::vector<int2> ch;
  r.elems = 0;
  for (int i = 0; i < int(r.host.size()); ++i) {
    r.elems += r.host[i].t.n;
    for (int s = 0; s < r.host[i].t.n; s += chunk) ch.push_back(make_int2(i, s));
  }
  r.nchunks = int(ch.size());
  if (!r.host.empty()) {
    BST_CUDA(cudaMalloc(&r.tasks, sizeof(BatchTask) * r.host.size()));
    BST_CUDA(cudaMemcpy(r.tasks, r.host.data(), sizeof(BatchTask) * r.host.size(), cudaMemcpyHostToDevice));
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
  relayout_batch_kernel<<<r.nchunks, kBatchThreads, 0, s>>>(r.tasks, r.chunks, bases, mat, dir, alpha, beta,
                                                            r.chunk);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
}

// Median over `reps` timed runs of f (after one untimed run), in ms.
template <class F>
static float time_ms(cudaStream_t s, int reps, F&& f) {
  cudaEvent_t a, b;
  BST_CUDA(cudaEventCreate(&a));
  BST_CUDA(cudaEventCreate(&b));
  std::vector<float> t;
  f();
  for (int i = 0; i < reps; ++i) {
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Autotuner: on the first call of a plan (per arithmetic), time every
// candidate schedule on the call's own data and keep the fastest.  Only the
// plan's own buffers are written while tuning; the caller's outputs are not.
//   relayout: elements per CTA of the gathers and the scatter (1K..8K);
//   GEMM: tile schedule (problem order / longest K first / column tiles
//   outer for the tensor-core GEMM; problem order / longest K first for FP64)
//   and, for the tensor-core GEMM, the output tile shape (128 x 64, or
//   128 x 32: twice the tiles, half the padding of narrow sectors).
static void autotune(Ctx* ctx, BatchPlan* bp, double* const* bases, size_t n, bst_prec prec, const std::string& tag,
                     cudaStream_t s) {
  const bool prof = ctx->prof;
  ctx->prof = false;
  char line[256];
  if (!bp->tuned_rel) {
    float best = 1e30f;
    int bc = 2048;
    for (int c : kChunkChoices) {
      upload_rel(bp->ra, c);
      upload_rel(bp->rb, c);
      const float t = time_ms(s, 3, [&] {
        launch_rel(ctx, bp->ra, bases, bp->Am, 0, 1.0, 0.0, s);
        launch_rel(ctx, bp->rb, bases + n, bp->Bm, 0, 1.0, 0.0, s);
      });
      snprintf(line, sizeof(line), "batch %p relayout chunk %d: %.4f ms\n", (void*)bp, c, t);
      ctx->tune_log += line;
      if (t < best) best = t, bc = c;
    }
    upload_rel(bp->ra, bc);
    upload_rel(bp->rb, bc);
    upload_rel(bp->rc, bc);
    snprintf(line, sizeof(line), "batch %p relayout chunk chosen %d\n", (void*)bp, bc);
    ctx->tune_log += line;
    bp->tuned_rel = true;
  }
  const int pi = int(prec);
  if (!bp->tuned[pi]) {
    launch_rel(ctx, bp->ra, bases, bp->Am, 0, 1.0, 0.0, s);
    launch_rel(ctx, bp->rb, bases + n, bp->Bm, 0, 1.0, 0.0, s);
    const int norders = prec == BST_FP64 ? 2 : 3;
    const int S = ozaki_slices(prec);
    const char* kname = prec == BST_FP64 ? "gemm_f64" : "gemm_ozaki";
    float best = 1e30f;
    int bo = 0, btn = 64;
    for (int tn : {64, 32}) {
      if (prec == BST_FP64 && tn != 64) continue;
      for (int o = 0; o < norders; ++o) {
        float t;
        if (prec == BST_FP64) {
          bp->g.upload(bp->probs, kF64TileM, kF64TileN, o);
          t = time_ms(s, 3, [&] { launch_gemm_f64(ctx, bp->g, bp->Am, bp->Bm, bp->Cm, s); });
        } else {
          t = time_ms(s, 3, [&] {
            run_gemm_ozaki_probs(ctx, tag, bp->probs, bp->Am, bp->Bm, bp->Cm, s, o, true, S, tn);
          });
        }
        snprintf(line, sizeof(line), "batch %p %s tile 128x%d order %d: %.4f ms\n", (void*)bp, kname,
                 prec == BST_FP64 ? kF64TileN : tn, o, t);
        ctx->tune_log += line;
        if (t < best) best = t, bo = o, btn = tn;
      }
    }
    if (prec == BST_FP64) bp->g.upload(bp->probs, kF64TileM, kF64TileN, bo);
    bp->order[pi] = bo;
    bp->tn[pi] = btn;
    bp->tuned[pi] = true;
    snprintf(line, sizeof(line), "batch %p %s tile order chosen %d, tile 128x%d\n", (void*)bp, kname, bo,
             prec == BST_FP64 ? kF64TileN : btn);
    ctx->tune_log += line;
  }
  ctx->prof = prof;
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
  for (size_t i = 0; i < plans.size(); ++i) {
    ContractPlan* p = plans[i];
    for (auto t : p->va.tasks) {
      t.mat_base += bp->amat;
      bp->ra.host.push_back({t, int32_t(i), 0});
    }
    for (auto t : p->vb.tasks) {
      t.mat_base += bp->bmat;
      bp->rb.host.push_back({t, int32_t(i), 0});
    }
    for (auto t : p->vc.tasks) {
      t.mat_base += bp->cmat;
      bp->rc.host.push_back({t, int32_t(i), 0});
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
  upload_rel(bp->ra, 2048);
  upload_rel(bp->rb, 2048);
  upload_rel(bp->rc, 2048);
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
  const std::string tag = "batch/" + std::to_string(uintptr_t(bp));
  if (ctx->autotune) autotune(ctx, bp, bases, n, prec, tag, s);
  double *Am = bp->Am, *Bm = bp->Bm, *Cm = bp->Cm;
  ctx->work_flops += bp->g.flops;
  launch_rel(ctx, bp->ra, bases, Am, 0, 1.0, 0.0, s);
  launch_rel(ctx, bp->rb, bases + n, Bm, 0, 1.0, 0.0, s);
  if (prec == BST_FP64) {
    launch_gemm_f64(ctx, bp->g, Am, Bm, Cm, s);
  } else {
    // the same grouped tensor-core GEMM as a single contraction, over the
    // problems of all contractions
    run_gemm_ozaki_probs(ctx, tag, bp->probs, Am, Bm, Cm, s, bp->order[int(prec)], true, ozaki_slices(prec),
                         bp->tn[int(prec)]);
  }
  launch_rel(ctx, bp->rc, bases + 2 * n, Cm, 1, alpha, beta, s);
}

}  // namespace bst
