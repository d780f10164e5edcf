// Internal declarations of the block-sparse symmetric tensor library.
// Nothing here crosses the C ABI (include/bst.h): C++ types, exceptions and
// containers stay inside the shared library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/bst.h"

namespace bst {

constexpr int kMaxRank = 8;

// Internal error: converted to a bst_status at the ABI boundary.
struct Error : std::runtime_error {
  bst_status code;
  Error(bst_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define BST_REQUIRE(cond, code, msg)                                   \
  do {                                                                 \
    if (!(cond)) throw ::bst::Error((code), (msg));                    \
  } while (0)

#define BST_CUDA(call)                                                           \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      throw ::bst::Error(BST_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Charges of the abelian groups: U(1) charges are integers, Z2 charges are
// parities.  cnorm maps a sum of (flow-signed) charges to its canonical
// representative: itself for U(1), its parity (0 or 1) for Z2.
inline int64_t cnorm(int group, int64_t q) {
  if (group == BST_Z2) return q & 1;  // two's complement: parity of negative sums too
  return q;
}
inline bool is_abelian(int group) { return group == BST_U1 || group == BST_Z2; }

// One leg: flow and sectors (Sec. 2).  `off` are sector offsets in the dense
// index of the leg.
struct Leg {
  int flow = 1;
  std::vector<int> q;
  std::vector<int64_t> d;
  std::vector<int64_t> off;
  int64_t dim = 0;
  void finish();
  bool same_space(const Leg& o) const { return q == o.q && d == o.d; }
  bool operator==(const Leg& o) const { return flow == o.flow && same_space(o); }
  Leg dual() const { Leg l = *this; l.flow = -flow; return l; }
  int find(int charge) const;  // sector index of a charge or -1
};

// Canonical block layout (immutable, interned per context).
struct Layout {
  std::atomic<int> refs{1};
  struct Ctx* ctx = nullptr;
  uint64_t id = 0;
  int group = BST_U1;
  int rank = 0;
  std::vector<Leg> legs;
  int64_t nblocks = 0, nnz = 0;
  std::vector<int32_t> sect;    // nblocks * rank sector indices
  std::vector<int64_t> offset;  // nblocks element offsets
  std::vector<int64_t> shape;   // nblocks * rank extents
  // SU(2): tree labels of every block (ntree per block: in-tree
  // intermediates, coupled J, out-tree intermediates; doubled spins)
  int ntree = 0;
  std::vector<int32_t> tree;
  std::unordered_map<uint64_t, int64_t> index;  // packed sector tuple -> (first) block
  std::string key;              // structural key used for interning

  int64_t block_of(const int32_t* s) const;
  static uint64_t pack(const int32_t* s, int r) {
    uint64_t k = 0;
    for (int i = 0; i < r; ++i) k = (k << 8) | uint64_t(uint8_t(s[i]));
    return k;
  }
};

// Element-wise relayout between a contiguous block (row-major over `shape`)
// and a strided region of another buffer.
struct RelTask {
  int64_t blk_off;     // element offset of the contiguous side
  int64_t mat_base;    // element offset of the strided side
  int32_t rank;
  int32_t n;           // number of elements
  int32_t shape[kMaxRank];
  int64_t mstride[kMaxRank];
};

// Sector-matrix view of a block tensor w.r.t. (row legs, col legs): one dense
// row-major matrix per conserved charge through the cut (key = sum over the
// col legs of flow*q).
struct MatSector {
  int64_t key = 0;
  int64_t rows = 0, cols = 0;
  int64_t off = 0;  // element offset in the matrix buffer
  std::vector<std::vector<int32_t>> rcfg, ccfg;  // sector tuples
  std::vector<int64_t> roff, coff;                // offsets of each config
  std::map<std::vector<int32_t>, int64_t> rmap, cmap;
};

struct MatView {
  std::vector<int> rowlegs, collegs;
  std::vector<MatSector> secs;
  std::map<int64_t, int> by_key;
  int64_t total = 0;
  std::vector<RelTask> tasks;  // one per tensor block with nonzero size
  const MatSector* find(int64_t key) const {
    auto it = by_key.find(key);
    return it == by_key.end() ? nullptr : &secs[it->second];
  }
};

// A relayout ready to launch: tasks and chunk table on the device.
struct DevRelayout {
  RelTask* tasks = nullptr;
  int2* chunks = nullptr;
  int nchunks = 0;
  int ntasks = 0;
  double elems = 0;
  void upload(const std::vector<RelTask>& t);
  void free_all();
};

// One GEMM of a grouped launch: C[m,n] = sum_k A[m,k] B[n,k] with generic
// element strides (a_m, a_k), (b_n, b_k), (c_m, c_n).
struct GemmProb {
  int32_t M, N, K, pad;
  int64_t a_off, b_off, c_off;
  int64_t a_m, a_k, b_n, b_k, c_m, c_n;
};

// 64-bit FNV-1a hash of a problem list (plan-cache key)
inline uint64_t probs_hash(const std::vector<GemmProb>& probs) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(probs.data());
  const size_t n = probs.size() * sizeof(GemmProb);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h ^ (uint64_t(probs.size()) << 1);
}

struct DevGemm {
  GemmProb* probs = nullptr;
  int32_t* tile_prob = nullptr;   // tile -> problem
  int32_t* tile_idx = nullptr;    // tile -> linear tile index inside its problem
  int ntiles = 0, nprobs = 0;
  double flops = 0;  // algorithmic 2*M*N*K summed over the problems
  int64_t* w_off = nullptr;  // per problem: offset of its M x N slice in a split-K workspace
  std::vector<int64_t> hw_off;  // the same offsets on the host
  int64_t wtot = 0;          // sum of M*N
  int maxK = 0;
  // order 0: problem order; 1: tiles of the longest-K problems first
  void upload(const std::vector<GemmProb>& p, int tm, int tn, int order = 0);
  void free_all();
};

struct OzakiPlan;  // mixed-precision GEMM plan (gemm_ozaki.cu)
struct BatchPlan;  // batched-contraction plan (batch.cu)
struct Su2Plan;    // SU(2) contraction plan (su2.cu)
struct Su2PermPlan;  // SU(2) permutation with recoupling (su2.cu)
struct ProjView;   // projector layout view (projector.cu)

// Contraction plan (cached per (A, B, pairs)).
struct ContractPlan {
  Layout *A = nullptr, *B = nullptr, *C = nullptr;
  MatView va, vb, vc;
  DevRelayout ra, rb, rc;      // A->Amat, B->Bmat, Cmat->C
  std::vector<GemmProb> probs; // per matched sector
  DevGemm g;
  // tensor-core GEMM plans by digit count and output form: [S == 3][scatter]
  // (scatter: the output written straight into C's blocks)
  OzakiPlan* oz[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int64_t amat = 0, bmat = 0, cmat = 0;  // matrix buffer sizes (elements)
  ~ContractPlan();
};

// Device buffer that only grows (the caller synchronises before growth).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void* get(size_t need, cudaStream_t s);
  void free_all();
};

// Optional per-kernel-class timing with CUDA events on the launching stream.
struct ProfRec {
  std::string cls;
  cudaEvent_t a, b;
  double flops, bytes;
};

struct Ctx {
  int device = 0;
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  std::mutex mu;
  uint64_t next_id = 1;
  std::map<std::string, Layout*> interned;  // structural key -> layout (one ref held)
  std::map<std::string, std::unique_ptr<ContractPlan>> cplans;
  std::map<std::string, std::unique_ptr<DevRelayout>> rplans;
  std::map<std::string, DevBuf> bufs;
  std::map<std::string, std::unique_ptr<DevGemm>> gplans;
  std::map<std::string, std::shared_ptr<BatchPlan>> bplans;  // deleter bound in batch.cu
  std::map<std::string, std::shared_ptr<OzakiPlan>> ozplans;  // deleter bound in gemm_ozaki.cu
  std::map<std::string, std::shared_ptr<Su2Plan>> su2plans;   // deleter bound in su2.cu
  std::map<std::string, std::shared_ptr<Su2PermPlan>> su2perm; // deleter bound in su2.cu
  std::map<std::string, std::shared_ptr<ProjView>> projviews; // deleter bound in projector.cu
  std::map<uint64_t, DevBuf> su2_weights;  // SU(2) layout id -> per-element 2J+1 (norms)
  int* d_err = nullptr;                     // device error word
  long long spin_limit = 0;                 // bound of a pipeline wait in tries (0: the default)
  std::atomic<int64_t> launches{0};
  // algorithmic work of the method's contractions issued so far: 2 M N K
  // over the matched block pairs of every contraction (U(1) sector GEMMs,
  // SU(2) pair products, batched contractions) and of the projector's
  // P = Rb V S^-1/2 and Pt = S^-1/2 U^T Rt^T products; the projector's own
  // iterations (subspace products, Rayleigh-Ritz, refinement) are not
  // counted.  Enumerated from the plans, FP64-equivalent whatever the
  // arithmetic.
  double work_flops = 0;
  void* cusolver = nullptr;
  int proj_method = 1;   // 0: cuSOLVER gesvd per sector, 1: subspace iteration + small eigensolver
  int proj_iters = 9;    // subspace iterations
  // Rayleigh-Ritz eigenproblems of the subspace iteration start from the
  // nearly diagonal matrix itself (one relative Jacobi pass)
  bool rr_near_diag = true;
  double* d_scratch_small = nullptr;
  bool autotune = true;      // time schedule candidates on the first batched call of a plan
  std::string tune_log;      // one line per tuning decision
  // second stream for work that overlaps the caller's stream inside one
  // call (the projector's direct sectors), with its fork and join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // projector: per sector structure, whether the last call found every
  // directly decomposed sector unable to reach the truncation (scheduling
  // hint only: such sectors are then deferred and, if still provably
  // below the cut, skipped)
  std::map<std::string, bool> direct_below_cut;
  // projector: per sector structure, whether the last mixed-precision call
  // needed more than one subspace round (its intermediate Rayleigh-Ritz
  // steps then run in the mixed arithmetic)
  std::map<std::string, bool> multi_round;
  ~Ctx();
  void* buf(const std::string& name, size_t bytes, cudaStream_t s) { return bufs[name].get(bytes, s); }
};

// layout.cpp
Layout* make_layout(Ctx* ctx, int group, const std::vector<Leg>& legs);  // new reference
void retain(Layout* l);
void release(Layout* l);
Leg fuse_legs(const std::vector<Leg>& legs, std::vector<std::vector<int32_t>>* tuples_per_sector = nullptr,
              int group = BST_U1);
std::vector<std::vector<int32_t>> enum_configs(const std::vector<const Leg*>& legs, int64_t target,
                                               int group = BST_U1);

// plan.cpp
MatView make_matview(const Layout* L, const std::vector<int>& rowlegs, const std::vector<int>& collegs,
                     bool build_tasks = true);
ContractPlan* get_contract_plan(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la,
                                const std::vector<int>& lb);
DevRelayout* get_permute_plan(Ctx* ctx, Layout* src, const std::vector<int>& perm, Layout** dst);
DevRelayout* get_fuse_plan(Ctx* ctx, Layout* src, const std::vector<int>& groups, Layout** dst);
void run_contract(Ctx* ctx, ContractPlan* p, const double* a, const double* b, bst_prec prec,
                  double alpha, double beta, double* c, cudaStream_t s, bool scatter = true,
                  double** cmat_out = nullptr);

// plan_dev.cu: the sector matching of a contraction on the device
void plan_relayouts_on_device(Ctx* ctx, ContractPlan* p, const std::vector<int>& oa, const std::vector<int>& la,
                              const std::vector<int>& ob, const std::vector<int>& lb, cudaStream_t s);
int64_t plan_check(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la, const std::vector<int>& lb,
                   cudaStream_t s);

// relayout.cu
std::vector<int2> relayout_chunks(const std::vector<RelTask>& t);  // chunk table of a task list
void launch_relayout(Ctx* ctx, const DevRelayout& r, const double* blk, double* mat, int dir,
                     double alpha, double beta, cudaStream_t s);

// gemm_f64.cu
DevGemm* get_dev_gemm(Ctx* ctx, const std::string& key, const std::vector<GemmProb>& probs);
void launch_gemm_f64(Ctx* ctx, const DevGemm& g, const double* A, const double* B, double* C,
                     cudaStream_t s);
// the same product with K split into ksplit slices reduced in a fixed order
// (more CTAs for small, deep products)
// C[prob] = sum over the ksplit slices of W (slice stride g.wtot, problem
// offsets g.w_off, each M x N row-major), in slice order, into C's strides
void launch_ksplit_reduce(Ctx* ctx, const DevGemm& g, const double* W, int ksplit, double* C, cudaStream_t s);
// ws names the context buffer that holds the K-slice partial products
void launch_gemm_f64_splitk(Ctx* ctx, const DevGemm& g, int ksplit, const double* A, const double* B, double* C,
                            cudaStream_t s, const char* ws = "gemm_f64.splitk");
extern const int kF64TileM, kF64TileN;

// gemm_ozaki.cu
// digit slices per operand of a tensor-core arithmetic (5 for BST_OZAKI,
// 3 for BST_BF16X3)
int ozaki_slices(bst_prec prec);
// output tile width for a problem list: 64, or 32 when 128 x 64 tiles
// would leave SMs idle or pad narrow problems by more than half
int ozaki_pick_tn(const std::vector<GemmProb>& probs);
// The contraction plan's operands a, b (tensor data) are read by the pack
// kernel, which gathers each sector-matrix row from the blocks and splits it
// into digits in one pass.
// plain variant: the epilogue writes the sector matrices Cmat
// (Am, Bm: the operands' sector matrices when the caller has gathered them)
void run_gemm_ozaki(Ctx* ctx, ContractPlan* p, int S, const double* a, const double* b, double* Cmat,
                    cudaStream_t s, const double* Am = nullptr, const double* Bm = nullptr);
// scatter variant: the epilogue writes c = alpha * A B + beta * c straight
// into the output tensor's canonical blocks (no sector matrix, no scatter
// launch)
void run_gemm_ozaki_scatter(Ctx* ctx, ContractPlan* p, int S, const double* a, const double* b, double* c,
                            double alpha, double beta, cudaStream_t s);
void ozaki_free(OzakiPlan* oz);
// batched contractions (batch.cu): one packed plan whose epilogue scatters
// into every contraction's output (see gemm_ozaki.cu)
// pack: operands gathered and split by the pack kernel (every plan
// ozaki_packable), else split from the gathered sector matrices
bool ozaki_packable(const ContractPlan* p);
OzakiPlan* ozaki_batch_plan(Ctx* ctx, const std::vector<ContractPlan*>& plans, const std::vector<GemmProb>& probs,
                            int order, int S, int TN, bool pack, std::vector<long long>* bbase_rel,
                            std::vector<int32_t>* bbase_src);
void ozaki_batch_bbase(const std::vector<long long>& rel, const std::vector<int32_t>& src,
                       const std::vector<double*>& c, std::vector<long long>* out);
// bases: device table a[0..n), b[0..n) (packed plans) or Am, Bm: the
// gathered sector matrices; c0 = c[0]; bbase from ozaki_batch_bbase
void run_ozaki_batch(Ctx* ctx, OzakiPlan* P, double* const* bases, int n, const double* Am, const double* Bm,
                     double* c0, const long long* bbase, double alpha, double beta, cudaStream_t s);
// generic Ozaki GEMM over a problem list (used by the projector)
// `order` selects the tile schedule (0 problem order, 1 longest K first,
// 2 column tiles outer); each schedule is its own cached plan
// split_a = false reuses the A digits of this plan's previous call (the
// caller guarantees that A has not changed since)
// S digit slices (5 or 3); TN the output tile width (0: ozaki_pick_tn)
void run_gemm_ozaki_probs(Ctx* ctx, const std::string& tag, const std::vector<GemmProb>& probs,
                          const double* A, const double* B, double* C, cudaStream_t s, int order = 0,
                          bool split_a = true, int S = 5, int TN = 0);

// projector.cu
struct ProjResult {
  Layout* P = nullptr;
  Layout* Pt = nullptr;
  Leg newleg;
  std::vector<double> svals;
  int64_t kept = 0;
  double smin_over_smax = 0, trunc_weight = 0;
};
ProjResult svd_projector(Ctx* ctx, Layout* Rt, const double* rt, Layout* Rb, const double* rb, int ncut,
                         int64_t chi, double rel_cutoff, int new_flow, bst_prec prec, double* p, double* pt,
                         cudaStream_t s);

// SU(2): projectors from the reduced SVD per coupled spin J, truncated by
// whole multiplets to total dimension chi_total; P and Pt land in context
// buffers (*p, *pt); the new leg is incoming on P
ProjResult su2_projector(Ctx* ctx, Layout* Rt, const double* rt, Layout* Rb, const double* rb, int ncut,
                         int64_t chi_total, double rel_cutoff, bst_prec prec, double** p, double** pt,
                         cudaStream_t s);

void sym_eig_batched(Ctx* ctx, int n, int batch, const double* H, double* X, double* lam, bst_prec prec,
                     cudaStream_t s);

// contract_noalloc.cu
void contract_noalloc(Ctx* ctx, Layout* A, const double* a, Layout* B, const double* b, const std::vector<int>& la,
                      const std::vector<int>& lb, double alpha, double beta, Layout* C, double* c, cudaStream_t s);

// batch.cu
void contract_batched(Ctx* ctx, const std::vector<Layout*>& A, const std::vector<const double*>& a,
                      const std::vector<Layout*>& B, const std::vector<const double*>& b, const std::vector<int>& la,
                      const std::vector<int>& lb, bst_prec prec, double alpha, double beta,
                      const std::vector<Layout*>& C, const std::vector<double*>& c, cudaStream_t s);

// su2.cu
double su2_cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM);  // doubled spins
int su2_ntree(const std::vector<Leg>& legs);
void su2_enum_blocks(const std::vector<Leg>& legs, std::vector<int32_t>& sect, std::vector<int32_t>& tree);
Layout* su2_contract_layout(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la, const std::vector<int>& lb);
// dst = src with legs permuted (dst leg j = src leg perm[j]), trees recoupled;
// returns the (interned) dst layout; src/dst may be null when nnz is 0
Layout* su2_permute(Ctx* ctx, Layout* S, const double* src, const std::vector<int>& perm, double* dst,
                    cudaStream_t s);
void su2_contract(Ctx* ctx, Layout* A, const double* a, Layout* B, const double* b, const std::vector<int>& la,
                  const std::vector<int>& lb, bst_prec prec, double alpha, double beta, Layout* C, double* c,
                  cudaStream_t s);
inline void require_prec(bst_prec prec) {
  BST_REQUIRE(prec == BST_FP64 || prec == BST_OZAKI || prec == BST_BF16X3, BST_E_ARG, "unknown precision mode");
}

inline void require_u1(const Layout* L) {
  if (!is_abelian(L->group))
    throw Error(BST_E_UNSUPPORTED, "this operation is implemented for U(1) and Z2 tensors only");
}

// ctm.cpp
// Unit cell Lx x Ly (sites and environments in row-major position order
// x + Lx y); abelian double layers (ctm.cpp)
void ctm_move_cell(Ctx* ctx, int dir, int Lx, int Ly, Layout* const* a, const double* const* ad, bst_env* envs,
                   int64_t chi, double cutoff, bst_prec prec, cudaStream_t s);
void ctm_move(Ctx* ctx, int dir, Layout* a, const double* ad, bst_env* env, int64_t chi, double rel_cutoff,
              bst_prec prec, bst_ctm_stats* stats, cudaStream_t s);

// ctm.cpp / observe.cu: observables and the CTM error procedure
Layout* bond_rdm(Ctx* ctx, int bond, Layout* site, const double* sd, bst_env* env, bst_prec prec, double** rho,
                 cudaStream_t s);
Layout* double_layer_open(Ctx* ctx, Layout* LA, const double* A, Layout* LR, const double* R, double* out,
                          cudaStream_t s);
double block_dot(Ctx* ctx, const double* x, const double* y, int64_t n, cudaStream_t s);
void ctm_converge(Ctx* ctx, Layout* a, const double* ad, Layout* site, const double* sd, Layout* HL,
                  const double* H, bst_env* env, int64_t chi0, int64_t chi_max, double tol, int32_t max_steps,
                  double rel_cutoff, bst_prec prec, bst_ctm_converge_stats* st, cudaStream_t s);

// misc kernels (relayout.cu)
void launch_scale(Ctx* ctx, double* x, int64_t n, const double* dev_scalar_inv, cudaStream_t s);
void launch_sumsq(Ctx* ctx, const double* x, int64_t n, double* dev_out, cudaStream_t s);
void launch_fill(Ctx* ctx, double* x, int64_t n, double v, cudaStream_t s);
void launch_sumsq_w(Ctx* ctx, const double* x, const double* w, int64_t n, double* dev_out, cudaStream_t s);

inline void count_launch(Ctx* ctx, int n = 1) { ctx->launches += n; }

// Times the launches issued during its lifetime when profiling is on.
struct ProfScope {
  Ctx* c;
  cudaStream_t s;
  long idx = -1;
  ProfScope(Ctx* ctx, cudaStream_t st, const char* cls, double flops, double bytes);
  ~ProfScope();
};

}  // namespace bst
