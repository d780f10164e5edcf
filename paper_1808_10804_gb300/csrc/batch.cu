// Batched contractions: many independent contractions (uneven sector sizes)
// in a few launches for all of them.  The matched block pairs of every
// contraction form one problem list, so the GPU is filled even when each
// contraction alone is small (Sec. 2: the block pairs of a contraction are
// independent of one another, and so are separate contractions).
//
// Tensor-core arithmetic: two launches.  One pack launch gathers the rows
// of every contraction's operand sector matrices straight from the operand
// tensors and splits them into digits (each segment carries the index of
// its tensor in a device pointer table); one GEMM launch over all problems
// writes every product into its contraction's output blocks (the scatter
// tables address each output relative to the first output's pointer).
// FP64: one gather per operand into combined sector-matrix buffers, one
// grouped DMMA GEMM, one scatter.
//
// The per-contraction plans are the cached single-contraction plans.  Each
// distinct set of data pointers gets its own pointer table (and output
// offsets), uploaded once and kept with the plan, so a repeated call
// uploads nothing and a captured CUDA graph of it stays valid while other
// pointer sets are used in between.
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
  // one gather of both operands (B's tasks point past A's matrices and at
  // the second half of the pointer table), the FP64 path's scatter
  BatchRel rab, rc;
  bool packed = false;  // every contraction ozaki_packable
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
  // and, once a tensor-core call has used it, the output block offsets
  // relative to c[0]
  struct PtrSet {
    double** bases = nullptr;
    long long* bbase = nullptr;
  };
  std::map<std::vector<const void*>, PtrSet> tables;
  // tensor-core plans by digit count, tile width and tile order, and the
  // scatter offsets they share (inside each output, and its contraction)
  std::map<std::string, OzakiPlan*> ozp;
  std::vector<long long> bb_rel;
  std::vector<int32_t> bb_src;
  // the plan's own sector-matrix buffers (Bm = Am + amat): a captured graph
  // of this batch keeps valid addresses for as long as the plan (the
  // context) lives
  double *Am = nullptr, *Bm = nullptr, *Cm = nullptr;
  ~BatchPlan() {
    cudaFree(Am);
    cudaFree(Cm);
    rab.free_all();
    rc.free_all();
    for (auto& kv : tables) {
      cudaFree(kv.second.bases);
      cudaFree(kv.second.bbase);
    }
    for (auto& kv : ozp) ozaki_free(kv.second);
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

static OzakiPlan* batch_oz(Ctx* ctx, BatchPlan* bp, int order, int S, int TN) {
  const std::string key = std::to_string(S) + "/" + std::to_string(TN) + "/" + std::to_string(order);
  auto it = bp->ozp.find(key);
  if (it != bp->ozp.end()) return it->second;
  OzakiPlan* P = ozaki_batch_plan(ctx, bp->plans, bp->probs, order, S, TN, bp->packed, &bp->bb_rel, &bp->bb_src);
  bp->ozp[key] = P;
  return P;
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
                     cudaStream_t s, const std::vector<Layout*>& C) {
  const bool prof = ctx->prof;
  ctx->prof = false;
  char line[256];
  if (!bp->tuned_rel && !(prec != BST_FP64 && bp->packed)) {
    float best = 1e30f;
    int bc = 2048;
    for (int c : kChunkChoices) {
      upload_rel(bp->rab, c);
      const float t = time_ms(s, 3, [&] {
        launch_rel(ctx, bp->rab, bases, bp->Am, 0, 1.0, 0.0, s);
      });
      snprintf(line, sizeof(line), "batch %p relayout chunk %d: %.4f ms\n", (void*)bp, c, t);
      ctx->tune_log += line;
      if (t < best) best = t, bc = c;
    }
    upload_rel(bp->rab, bc);
    upload_rel(bp->rc, bc);
    snprintf(line, sizeof(line), "batch %p relayout chunk chosen %d\n", (void*)bp, bc);
    ctx->tune_log += line;
    bp->tuned_rel = true;
  }
  const int pi = int(prec);
  if (!bp->tuned[pi]) {
    if (!(prec != BST_FP64 && bp->packed)) launch_rel(ctx, bp->rab, bases, bp->Am, 0, 1.0, 0.0, s);
    // the tensor-core candidates write every output through the scatter
    // epilogue: while tuning they write a scratch copy of the outputs
    double* scratch = nullptr;
    long long* sbb = nullptr;
    if (prec != BST_FP64) {
      batch_oz(ctx, bp, 0, ozaki_slices(prec), 64);  // the shared scatter offsets
      int64_t tot = 0;
      std::vector<int64_t> coff(n);
      for (size_t i = 0; i < n; ++i) coff[i] = tot, tot += C[i]->nnz;
      std::vector<long long> abs(bp->bb_rel.size());
      for (size_t j = 0; j < abs.size(); ++j) abs[j] = bp->bb_rel[j] + coff[bp->bb_src[j]];
      BST_CUDA(cudaMalloc(&scratch, sizeof(double) * std::max<int64_t>(tot, 1)));
      BST_CUDA(cudaMalloc(&sbb, sizeof(long long) * std::max<size_t>(abs.size(), 1)));
      BST_CUDA(cudaMemcpy(sbb, abs.data(), sizeof(long long) * abs.size(), cudaMemcpyHostToDevice));
    }
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
          OzakiPlan* P = batch_oz(ctx, bp, o, S, tn);
          t = time_ms(s, 3, [&] { run_ozaki_batch(ctx, P, bases, int(n), bp->Am, bp->Bm, scratch, sbb, 1.0, 0.0, s); });
        }
        snprintf(line, sizeof(line), "batch %p %s tile 128x%d order %d: %.4f ms\n", (void*)bp, kname,
                 prec == BST_FP64 ? kF64TileN : tn, o, t);
        ctx->tune_log += line;
        if (t < best) best = t, bo = o, btn = tn;
      }
    }
    if (prec == BST_FP64) bp->g.upload(bp->probs, kF64TileM, kF64TileN, bo);
    if (scratch) {
      BST_CUDA(cudaStreamSynchronize(s));
      cudaFree(scratch);
      cudaFree(sbb);
    }
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
  const int32_t n = int32_t(plans.size());
  std::vector<BatchTask> btasks;
  bp->packed = true;
  for (size_t i = 0; i < plans.size(); ++i) {
    ContractPlan* p = plans[i];
    bp->packed = bp->packed && ozaki_packable(p);
    for (auto t : p->va.tasks) {
      t.mat_base += bp->amat;
      bp->rab.host.push_back({t, int32_t(i), 0});
    }
    for (auto t : p->vb.tasks) {
      t.mat_base += bp->bmat;  // shifted past A's matrices below
      btasks.push_back({t, n + int32_t(i), 0});
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
  for (auto& t : btasks) {
    t.t.mat_base += bp->amat;
    bp->rab.host.push_back(t);
  }
  upload_rel(bp->rab, 2048);
  upload_rel(bp->rc, 2048);
  bp->g.upload(bp->probs, kF64TileM, kF64TileN);
  BST_CUDA(cudaMalloc(&bp->Am, sizeof(double) * std::max<int64_t>(bp->amat + bp->bmat, 1)));
  bp->Bm = bp->Am + bp->amat;
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
  auto it = bp->tables.find(ptrs);
  if (it == bp->tables.end()) {
    // first call with this pointer set: allocate and fill its table (not
    // capturable; later calls with the same pointers only launch)
    BatchPlan::PtrSet ps;
    BST_CUDA(cudaMalloc(&ps.bases, sizeof(void*) * ptrs.size()));
    BST_CUDA(cudaMemcpy(ps.bases, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice));
    it = bp->tables.emplace(ptrs, ps).first;
  }
  double** bases = it->second.bases;
  const std::string tag = "batch/" + std::to_string(uintptr_t(bp));
  if (ctx->autotune) autotune(ctx, bp, bases, n, prec, tag, s, C);
  ctx->work_flops += bp->g.flops;
  if (prec == BST_FP64) {
    launch_rel(ctx, bp->rab, bases, bp->Am, 0, 1.0, 0.0, s);
    launch_gemm_f64(ctx, bp->g, bp->Am, bp->Bm, bp->Cm, s);
    launch_rel(ctx, bp->rc, bases + 2 * n, bp->Cm, 1, alpha, beta, s);
    return;
  }
  // packed: one pack launch over every operand; else one gather of both
  // operands and one split; then one GEMM whose epilogue writes every
  // output block (alpha, beta applied there)
  if (!bp->packed) launch_rel(ctx, bp->rab, bases, bp->Am, 0, 1.0, 0.0, s);
  const int pi = int(prec);
  OzakiPlan* P = batch_oz(ctx, bp, bp->order[pi], ozaki_slices(prec), bp->tn[pi] ? bp->tn[pi] : ozaki_pick_tn(bp->probs));
  if (!it->second.bbase) {
    std::vector<long long> abs;
    ozaki_batch_bbase(bp->bb_rel, bp->bb_src, c, &abs);
    BST_CUDA(cudaMalloc(&it->second.bbase, sizeof(long long) * std::max<size_t>(abs.size(), 1)));
    BST_CUDA(cudaMemcpy(it->second.bbase, abs.data(), sizeof(long long) * abs.size(), cudaMemcpyHostToDevice));
  }
  run_ozaki_batch(ctx, P, bases, int(n), bp->Am, bp->Bm, c[0], it->second.bbase, alpha, beta, s);
}

}  // namespace bst
