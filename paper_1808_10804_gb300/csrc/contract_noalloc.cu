// bst_contract_noalloc: the FP64 block-sparse contraction without any device
// allocation.
//
// Some callers cannot call cudaMalloc: hosts whose device memory is owned
// and pre-sized by another runtime (a framework's caching allocator, a
// fixed-budget serving process), or code for which an allocation would
// synchronise the device at the wrong moment.  This entry point serves them:
// the caller passes inputs and the output, and every intermediate (the
// relayout task tables, the GEMM problem and tile tables and the three sector
// matrices) lives in one file-scope device array of kScratchBytes.  That array
// is part of the loaded module, so every GPU that loads the library holds it
// until the process exits.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "bst_internal.h"

namespace bst {

// 64 MiB of scratch per device.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The CUDA context current on this thread (driver entry point, looked up
// once through the runtime).
static CUcontext current_context() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  static GetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    BST_CUDA(cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q));
    BST_REQUIRE(p && q == cudaDriverEntryPointSuccess, BST_E_CUDA, "cuCtxGetCurrent unavailable");
    fn = (GetCurrentFn)p;
  }
  CUcontext c = nullptr;
  BST_REQUIRE(fn(&c) == CUDA_SUCCESS, BST_E_CUDA, "cuCtxGetCurrent failed");
  return c;
}

// Device address of the scratch array for the current device.  The host-side
// symbol is only a stand-in for the array: its address has to be looked up,
// with the device current, before a kernel may be given it.  Looked up once
// per device and CUDA context (the first call on a device does it; make that
// first call before any stream capture begins): a reset device or a
// recreated primary context reloads the module, so an address is never
// reused across contexts.
static void* noalloc_scratch_ptr(int device) {
  static std::mutex mu;
  static std::map<std::pair<int, CUcontext>, void*> ptr;
  const CUcontext cur = current_context();
  std::lock_guard<std::mutex> g(mu);
  auto it = ptr.find({device, cur});
  if (it != ptr.end()) return it->second;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  BST_REQUIRE(e == cudaSuccess && p != nullptr, BST_E_CUDA,
              std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") + cudaGetErrorString(e));
  ptr[{device, cur}] = p;
  return p;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

void contract_noalloc(Ctx* ctx, Layout* A, const double* a, Layout* B, const double* b, const std::vector<int>& la,
                      const std::vector<int>& lb, double alpha, double beta, Layout* C, double* c,
                      cudaStream_t s) {
  BST_REQUIRE(la.size() == lb.size(), BST_E_ARG, "leg pair lists differ in length");
  std::vector<bool> ua(A->rank, false), ub(B->rank, false);
  for (size_t i = 0; i < la.size(); ++i) {
    BST_REQUIRE(la[i] >= 0 && la[i] < A->rank && lb[i] >= 0 && lb[i] < B->rank, BST_E_ARG,
                "contracted leg index out of range");
    BST_REQUIRE(!ua[la[i]] && !ub[lb[i]], BST_E_ARG, "a leg is contracted twice");
    ua[la[i]] = ub[lb[i]] = true;
    const Leg &x = A->legs[la[i]], &y = B->legs[lb[i]];
    BST_REQUIRE(x.flow == -y.flow && x.same_space(y), BST_E_SYMMETRY,
                "contracted legs need opposite flows and identical sectors");
  }
  std::vector<int> oa, ob;
  std::vector<Leg> cl;
  for (int i = 0; i < A->rank; ++i)
    if (!ua[i]) { oa.push_back(i); cl.push_back(A->legs[i]); }
  for (int i = 0; i < B->rank; ++i)
    if (!ub[i]) { ob.push_back(i); cl.push_back(B->legs[i]); }
  BST_REQUIRE(int(cl.size()) == C->rank, BST_E_SHAPE, "C is not the layout of this contraction");
  for (int i = 0; i < C->rank; ++i)
    BST_REQUIRE(cl[i] == C->legs[i], BST_E_SHAPE, "C is not the layout of this contraction");

  // host plan (host memory only)
  MatView va = make_matview(A, oa, la), vb = make_matview(B, ob, lb);
  std::vector<int> crow, ccol;
  for (size_t i = 0; i < oa.size(); ++i) crow.push_back(int(i));
  for (size_t i = 0; i < ob.size(); ++i) ccol.push_back(int(oa.size() + i));
  MatView vc = make_matview(C, crow, ccol);
  std::vector<GemmProb> probs;
  for (auto& cs : vc.secs) {
    const MatSector* as = va.find(cs.key);
    const MatSector* bs = vb.find(cnorm(A->group, -cs.key));
    GemmProb g{};
    g.M = int32_t(cs.rows);
    g.N = int32_t(cs.cols);
    g.K = (as && bs) ? int32_t(as->cols) : 0;
    g.a_off = as ? as->off : 0;
    g.b_off = bs ? bs->off : 0;
    g.c_off = cs.off;
    g.a_m = g.K;
    g.a_k = 1;
    g.b_n = g.K;
    g.b_k = 1;
    g.c_m = cs.cols;
    g.c_n = 1;
    if (g.M > 0 && g.N > 0) probs.push_back(g);
  }
  std::vector<int32_t> tprob, tidx;
  for (int i = 0; i < int(probs.size()); ++i) {
    const int mt = (probs[i].M + kF64TileM - 1) / kF64TileM, nt = (probs[i].N + kF64TileN - 1) / kF64TileN;
    for (int t = 0; t < mt * nt; ++t) {
      tprob.push_back(i);
      tidx.push_back(t);
    }
  }
  const std::vector<RelTask>* tasks[3] = {&va.tasks, &vb.tasks, &vc.tasks};
  std::vector<int2> chunks[3];
  for (int r = 0; r < 3; ++r) chunks[r] = relayout_chunks(*tasks[r]);

  // scratch layout, each piece 256-byte aligned
  size_t off = 0;
  size_t o_task[3], o_chunk[3];
  for (int r = 0; r < 3; ++r) {
    o_task[r] = off;
    off = align256(off + sizeof(RelTask) * tasks[r]->size());
    o_chunk[r] = off;
    off = align256(off + sizeof(int2) * chunks[r].size());
  }
  const size_t o_prob = off;
  off = align256(off + sizeof(GemmProb) * probs.size());
  const size_t o_tprob = off;
  off = align256(off + sizeof(int32_t) * tprob.size());
  const size_t o_tidx = off;
  off = align256(off + sizeof(int32_t) * tidx.size());
  const size_t o_am = off;
  off = align256(off + sizeof(double) * size_t(va.total));
  const size_t o_bm = off;
  off = align256(off + sizeof(double) * size_t(vb.total));
  const size_t o_cm = off;
  off = align256(off + sizeof(double) * size_t(vc.total));
  BST_REQUIRE(off <= kNoAllocScratchBytes, BST_E_SHAPE,
              "bst_contract_noalloc: this contraction needs " + std::to_string(off) +
                  " bytes of scratch, above the fixed maximum of " + std::to_string(kNoAllocScratchBytes) +
                  " bytes (64 MiB); use bst_contract");
  BST_REQUIRE((A->nnz == 0 || a) && (B->nnz == 0 || b) && (C->nnz == 0 || c), BST_E_ARG, "data pointer is NULL");

  int dev = 0;
  BST_CUDA(cudaGetDevice(&dev));
  unsigned char* base = static_cast<unsigned char*>(noalloc_scratch_ptr(dev));
  auto put = [&](size_t o, const void* src, size_t n) {
    if (n) BST_CUDA(cudaMemcpyAsync(base + o, src, n, cudaMemcpyHostToDevice, s));
  };
  DevRelayout rel[3];
  for (int r = 0; r < 3; ++r) {
    put(o_task[r], tasks[r]->data(), sizeof(RelTask) * tasks[r]->size());
    put(o_chunk[r], chunks[r].data(), sizeof(int2) * chunks[r].size());
    rel[r].tasks = reinterpret_cast<RelTask*>(base + o_task[r]);
    rel[r].chunks = reinterpret_cast<int2*>(base + o_chunk[r]);
    rel[r].ntasks = int(tasks[r]->size());
    rel[r].nchunks = int(chunks[r].size());
    rel[r].elems = 0;
    for (auto& t : *tasks[r]) rel[r].elems += t.n;
  }
  put(o_prob, probs.data(), sizeof(GemmProb) * probs.size());
  put(o_tprob, tprob.data(), sizeof(int32_t) * tprob.size());
  put(o_tidx, tidx.data(), sizeof(int32_t) * tidx.size());
  DevGemm g;
  g.probs = reinterpret_cast<GemmProb*>(base + o_prob);
  g.tile_prob = reinterpret_cast<int32_t*>(base + o_tprob);
  g.tile_idx = reinterpret_cast<int32_t*>(base + o_tidx);
  g.ntiles = int(tprob.size());
  g.nprobs = int(probs.size());
  double* Am = reinterpret_cast<double*>(base + o_am);
  double* Bm = reinterpret_cast<double*>(base + o_bm);
  double* Cm = reinterpret_cast<double*>(base + o_cm);
  // every entry of the three sector-matrix buffers is written before it is
  // read (the relayouts cover every block, the GEMM every output sector,
  // K = 0 sectors included), so nothing left by an earlier call is used
  launch_relayout(ctx, rel[0], a, Am, 0, 1.0, 0.0, s);
  launch_relayout(ctx, rel[1], b, Bm, 0, 1.0, 0.0, s);
  launch_gemm_f64(ctx, g, Am, Bm, Cm, s);
  launch_relayout(ctx, rel[2], c, Cm, 1, alpha, beta, s);
  // the structs point into the static array; nothing to free
  for (auto& r : rel) r.tasks = nullptr, r.chunks = nullptr;
  g.probs = nullptr;
  g.tile_prob = g.tile_idx = nullptr;
}

}  // namespace bst
