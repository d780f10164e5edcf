// Planner: sector-matrix views, contraction plans, permute/fuse plans.
//
// Contraction (Sec. 2): blocks of A and B are paired when their charges on
// the contracted legs are equal; the results are then reduced over equal
// output labels.  Grouping the pairs by the charge that flows through the
// cut (the paper's advice to collect all pairs of one output configuration
// before reducing, so the unreduced result never exists) turns every group
// into one dense matrix product: A viewed as [open configs x contracted
// configs] times B viewed as [contracted configs x open configs].  Every
// entry of such a sector matrix is an allowed entry of its tensor, so the
// grouped GEMM performs exactly the matched-block multiply-adds.
#include <algorithm>
#include <functional>
#include <numeric>
#include <sstream>

#include "bst_internal.h"

namespace bst {

MatView make_matview(const Layout* L, const std::vector<int>& rowlegs, const std::vector<int>& collegs,
                     bool build_tasks) {
  MatView v;
  v.rowlegs = rowlegs;
  v.collegs = collegs;
  std::vector<const Leg*> rl, cl;
  for (int i : rowlegs) rl.push_back(&L->legs[i]);
  for (int i : collegs) cl.push_back(&L->legs[i]);
  // keys present in the tensor's blocks
  std::map<int64_t, bool> keys;
  for (int64_t b = 0; b < L->nblocks; ++b) {
    int64_t k = 0;
    for (int i : collegs) k += int64_t(L->legs[i].flow) * L->legs[i].q[L->sect[b * L->rank + i]];
    keys[cnorm(L->group, k)] = true;
  }
  int64_t off = 0;
  for (auto& kv : keys) {
    MatSector s;
    s.key = kv.first;
    s.rcfg = enum_configs(rl, -s.key, L->group);
    s.ccfg = enum_configs(cl, s.key, L->group);
    for (auto& t : s.rcfg) {
      int64_t n = 1;
      for (size_t j = 0; j < t.size(); ++j) n *= rl[j]->d[t[j]];
      s.rmap[t] = s.rows;
      s.roff.push_back(s.rows);
      s.rows += n;
    }
    for (auto& t : s.ccfg) {
      int64_t n = 1;
      for (size_t j = 0; j < t.size(); ++j) n *= cl[j]->d[t[j]];
      s.cmap[t] = s.cols;
      s.coff.push_back(s.cols);
      s.cols += n;
    }
    s.off = off;
    off += s.rows * s.cols;
    v.by_key[s.key] = int(v.secs.size());
    v.secs.push_back(std::move(s));
  }
  v.total = off;
  if (!build_tasks) return v;
  const int r = L->rank;
  std::vector<int> rowpos(r, -1), colpos(r, -1);
  for (size_t j = 0; j < rowlegs.size(); ++j) rowpos[rowlegs[j]] = int(j);
  for (size_t j = 0; j < collegs.size(); ++j) colpos[collegs[j]] = int(j);
  for (int64_t b = 0; b < L->nblocks; ++b) {
    const int32_t* sb = &L->sect[b * r];
    const int64_t* sh = &L->shape[b * r];
    int64_t n = 1;
    for (int i = 0; i < r; ++i) n *= sh[i];
    if (n == 0) continue;
    int64_t k = 0;
    std::vector<int32_t> rt, ct;
    for (int i : collegs) k += int64_t(L->legs[i].flow) * L->legs[i].q[sb[i]];
    k = cnorm(L->group, k);
    for (int i : rowlegs) rt.push_back(sb[i]);
    for (int i : collegs) ct.push_back(sb[i]);
    const MatSector& s = v.secs[v.by_key.at(k)];
    int64_t ro = s.rmap.at(rt), co = s.cmap.at(ct);
    RelTask t{};
    t.blk_off = L->offset[b];
    t.mat_base = s.off + ro * s.cols + co;
    t.rank = r;
    t.n = int32_t(n);
    for (int i = 0; i < r; ++i) t.shape[i] = int32_t(sh[i]);
    // strides of every tensor leg inside the sector matrix
    for (int i = 0; i < r; ++i) {
      int64_t st = 1;
      if (rowpos[i] >= 0) {
        for (size_t j = rowpos[i] + 1; j < rowlegs.size(); ++j) st *= sh[rowlegs[j]];
        st *= s.cols;
      } else {
        for (size_t j = colpos[i] + 1; j < collegs.size(); ++j) st *= sh[collegs[j]];
      }
      t.mstride[i] = st;
    }
    v.tasks.push_back(t);
  }
  return v;
}

static std::string vec_key(const std::vector<int>& v) {
  std::ostringstream os;
  for (int x : v) os << x << ",";
  return os.str();
}

ContractPlan::~ContractPlan() {
  ra.free_all();
  rb.free_all();
  rc.free_all();
  g.free_all();
  for (auto& row : oz)
    for (OzakiPlan* q : row)
      if (q) ozaki_free(q);
  release(A);
  release(B);
  release(C);
}

static Layout* contract_out_layout(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la,
                                   const std::vector<int>& lb, std::vector<int>* oa, std::vector<int>* ob) {
  BST_REQUIRE(la.size() == lb.size(), BST_E_ARG, "leg pair lists differ in length");
  BST_REQUIRE(A->group == B->group, BST_E_ARG, "A and B belong to different symmetry groups");
  std::vector<bool> ua(A->rank, false), ub(B->rank, false);
  for (size_t i = 0; i < la.size(); ++i) {
    BST_REQUIRE(la[i] >= 0 && la[i] < A->rank && lb[i] >= 0 && lb[i] < B->rank, BST_E_ARG,
                "contracted leg index out of range");
    BST_REQUIRE(!ua[la[i]] && !ub[lb[i]], BST_E_ARG, "a leg is contracted twice");
    ua[la[i]] = ub[lb[i]] = true;
    const Leg &x = A->legs[la[i]], &y = B->legs[lb[i]];
    BST_REQUIRE(x.flow == -y.flow, BST_E_SYMMETRY, "contracted legs must have opposite flows");
    BST_REQUIRE(x.same_space(y), BST_E_SYMMETRY, "contracted legs must carry identical sectors");
  }
  std::vector<Leg> cl;
  for (int i = 0; i < A->rank; ++i)
    if (!ua[i]) { oa->push_back(i); cl.push_back(A->legs[i]); }
  for (int i = 0; i < B->rank; ++i)
    if (!ub[i]) { ob->push_back(i); cl.push_back(B->legs[i]); }
  BST_REQUIRE(!cl.empty(), BST_E_UNSUPPORTED, "full contraction to a scalar is not supported");
  return make_layout(ctx, A->group, cl);
}

ContractPlan* get_contract_plan(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la,
                                const std::vector<int>& lb) {
  std::string key = std::to_string(A->id) + "/" + std::to_string(B->id) + "/" + vec_key(la) + "/" + vec_key(lb);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->cplans.find(key);
    if (it != ctx->cplans.end()) return it->second.get();
  }
  auto p = std::make_unique<ContractPlan>();
  std::vector<int> oa, ob;
  p->C = contract_out_layout(ctx, A, B, la, lb, &oa, &ob);
  p->A = A;
  p->B = B;
  retain(A);
  retain(B);
  p->va = make_matview(A, oa, la);
  p->vb = make_matview(B, ob, lb);
  std::vector<int> crow, ccol;
  for (size_t i = 0; i < oa.size(); ++i) crow.push_back(int(i));
  for (size_t i = 0; i < ob.size(); ++i) ccol.push_back(int(oa.size() + i));
  p->vc = make_matview(p->C, crow, ccol);
  p->amat = p->va.total;
  p->bmat = p->vb.total;
  p->cmat = p->vc.total;
  // one GEMM per C sector: A sector key s pairs with B sector key -s
  for (auto& cs : p->vc.secs) {
    const MatSector* as = p->va.find(cs.key);
    const MatSector* bs = p->vb.find(cnorm(A->group, -cs.key));
    GemmProb g{};
    g.M = int32_t(cs.rows);
    g.N = int32_t(cs.cols);
    g.K = (as && bs) ? int32_t(as->cols) : 0;
    if (as) BST_REQUIRE(as->rows == cs.rows, BST_E_SHAPE, "planner: row mismatch");
    if (bs) BST_REQUIRE(bs->rows == cs.cols, BST_E_SHAPE, "planner: col mismatch");
    if (as && bs) BST_REQUIRE(as->cols == bs->cols, BST_E_SHAPE, "planner: K mismatch");
    g.a_off = as ? as->off : 0;
    g.b_off = bs ? bs->off : 0;
    g.c_off = cs.off;
    g.a_m = g.K;
    g.a_k = 1;
    g.b_n = g.K;
    g.b_k = 1;
    g.c_m = cs.cols;
    g.c_n = 1;
    if (g.M > 0 && g.N > 0) p->probs.push_back(g);
  }
  if (ctx->device >= 0) {  // host-only contexts plan without device tables
    // the relayout task lists (every block's place in its sector matrix)
    // are built by the device planner, which matches the same sectors
    plan_relayouts_on_device(ctx, p.get(), oa, la, ob, lb, 0);
    p->g.upload(p->probs, kF64TileM, kF64TileN);
  }
  ContractPlan* raw = p.get();
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->cplans[key] = std::move(p);
  return raw;
}

void run_contract(Ctx* ctx, ContractPlan* p, const double* a, const double* b, bst_prec prec, double alpha,
                  double beta, double* c, cudaStream_t s, bool scatter, double** cmat_out) {
  ctx->work_flops += p->g.flops;
  if (prec != BST_FP64 && scatter && !cmat_out) {
    // the tensor-core path reads A's and B's blocks directly (gather and
    // digit split in one kernel) and its epilogue writes C's blocks
    run_gemm_ozaki_scatter(ctx, p, ozaki_slices(prec), a, b, c, alpha, beta, s);
    return;
  }
  double* Cm = (double*)ctx->buf(cmat_out ? "contract.Ckeep" : "contract.C",
                                 sizeof(double) * std::max<int64_t>(p->cmat, 1), s);
  if (prec == BST_FP64) {
    double* Am = (double*)ctx->buf("contract.A", sizeof(double) * std::max<int64_t>(p->amat, 1), s);
    double* Bm = (double*)ctx->buf("contract.B", sizeof(double) * std::max<int64_t>(p->bmat, 1), s);
    launch_relayout(ctx, p->ra, a, Am, 0, 1.0, 0.0, s);
    launch_relayout(ctx, p->rb, b, Bm, 0, 1.0, 0.0, s);
    launch_gemm_f64(ctx, p->g, Am, Bm, Cm, s);
  } else {
    run_gemm_ozaki(ctx, p, ozaki_slices(prec), a, b, Cm, s);
  }
  if (scatter) launch_relayout(ctx, p->rc, c, Cm, 1, alpha, beta, s);
  if (cmat_out) *cmat_out = Cm;
}

// ---- permute -------------------------------------------------------------------

DevRelayout* get_permute_plan(Ctx* ctx, Layout* src, const std::vector<int>& perm, Layout** dst) {
  const int r = src->rank;
  BST_REQUIRE(int(perm.size()) == r, BST_E_ARG, "perm length must equal the rank");
  std::vector<bool> seen(r, false);
  for (int x : perm) {
    BST_REQUIRE(x >= 0 && x < r && !seen[x], BST_E_ARG, "perm is not a permutation");
    seen[x] = true;
  }
  std::vector<Leg> dl;
  for (int j = 0; j < r; ++j) dl.push_back(src->legs[perm[j]]);
  Layout* D = make_layout(ctx, src->group, dl);
  *dst = D;
  std::string key = "perm/" + std::to_string(src->id) + "/" + vec_key(perm);
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->rplans.find(key);
  if (it != ctx->rplans.end()) return it->second.get();
  std::vector<int> inv(r);
  for (int j = 0; j < r; ++j) inv[perm[j]] = j;
  std::vector<RelTask> tasks;
  std::vector<int32_t> ds(r);
  for (int64_t b = 0; b < src->nblocks; ++b) {
    const int32_t* sb = &src->sect[b * r];
    for (int j = 0; j < r; ++j) ds[j] = sb[perm[j]];
    int64_t db = D->block_of(ds.data());
    BST_REQUIRE(db >= 0, BST_E_SHAPE, "permute: missing destination block");
    const int64_t* dsh = &D->shape[db * r];
    RelTask t{};
    t.blk_off = src->offset[b];
    t.mat_base = D->offset[db];
    t.rank = r;
    int64_t n = 1;
    for (int i = 0; i < r; ++i) {
      t.shape[i] = int32_t(src->shape[b * r + i]);
      n *= t.shape[i];
      int64_t st = 1;
      for (int j = inv[i] + 1; j < r; ++j) st *= dsh[j];
      t.mstride[i] = st;
    }
    t.n = int32_t(n);
    if (n) tasks.push_back(t);
  }
  auto rp = std::make_unique<DevRelayout>();
  if (ctx->device >= 0) rp->upload(tasks);
  DevRelayout* raw = rp.get();
  ctx->rplans[key] = std::move(rp);
  return raw;
}

// ---- fuse ----------------------------------------------------------------------

DevRelayout* get_fuse_plan(Ctx* ctx, Layout* src, const std::vector<int>& groups, Layout** dst) {
  const int r = src->rank;
  int tot = 0;
  for (int g : groups) {
    BST_REQUIRE(g >= 1, BST_E_ARG, "group sizes must be positive");
    tot += g;
  }
  BST_REQUIRE(tot == r, BST_E_ARG, "group sizes must add up to the rank");
  const int ng = int(groups.size());
  std::vector<Leg> fl(ng);
  // per fused leg: map member tuple -> (fused sector, sub offset)
  std::vector<std::map<std::vector<int32_t>, std::pair<int, int64_t>>> sub(ng);
  int first = 0;
  for (int g = 0; g < ng; ++g) {
    std::vector<Leg> mem(src->legs.begin() + first, src->legs.begin() + first + groups[g]);
    std::vector<std::vector<int32_t>> tuples;
    fl[g] = fuse_legs(mem, &tuples, src->group);
    size_t ti = 0;
    for (size_t s = 0; s < fl[g].q.size(); ++s) {
      int64_t acc = 0;
      while (acc < fl[g].d[s]) {
        auto& t = tuples[ti++];
        int64_t n = 1;
        for (size_t j = 0; j < t.size(); ++j) n *= mem[j].d[t[j]];
        sub[g][t] = {int(s), acc};
        acc += n;
      }
    }
    first += groups[g];
  }
  Layout* D = make_layout(ctx, src->group, fl);
  *dst = D;
  std::string key = "fuse/" + std::to_string(src->id) + "/" + vec_key(groups);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->rplans.find(key);
  if (it != ctx->rplans.end()) return it->second.get();
  std::vector<RelTask> tasks;
  std::vector<int32_t> ds(ng);
  for (int64_t b = 0; b < src->nblocks; ++b) {
    const int32_t* sb = &src->sect[b * r];
    const int64_t* sh = &src->shape[b * r];
    std::vector<int64_t> subo(ng);
    first = 0;
    for (int g = 0; g < ng; ++g) {
      std::vector<int32_t> t(sb + first, sb + first + groups[g]);
      auto pr = sub[g].at(t);
      ds[g] = pr.first;
      subo[g] = pr.second;
      first += groups[g];
    }
    int64_t db = D->block_of(ds.data());
    BST_REQUIRE(db >= 0, BST_E_SHAPE, "fuse: missing destination block");
    const int64_t* dsh = &D->shape[db * ng];
    RelTask t{};
    t.blk_off = src->offset[b];
    t.rank = r;
    int64_t n = 1;
    int64_t base = D->offset[db];
    first = 0;
    for (int g = 0; g < ng; ++g) {
      int64_t gst = 1;  // stride of fused leg g in the destination block
      for (int j = g + 1; j < ng; ++j) gst *= dsh[j];
      base += subo[g] * gst;
      int64_t inner = 1;
      for (int m = groups[g] - 1; m >= 0; --m) {
        int i = first + m;
        t.mstride[i] = inner * gst;
        inner *= sh[i];
      }
      first += groups[g];
    }
    for (int i = 0; i < r; ++i) {
      t.shape[i] = int32_t(sh[i]);
      n *= sh[i];
    }
    t.mat_base = base;
    t.n = int32_t(n);
    if (n) tasks.push_back(t);
  }
  auto rp = std::make_unique<DevRelayout>();
  if (ctx->device >= 0) rp->upload(tasks);
  DevRelayout* raw = rp.get();
  ctx->rplans[key] = std::move(rp);
  return raw;
}

}  // namespace bst
