// The C ABI (include/bst.h): argument checks, error capture, handle casts.
// No C++ exception crosses this file's functions.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

#include "bst_internal.h"

using namespace bst;

static thread_local std::string g_err;

struct bst_ctx_s {};
struct bst_layout_s {};

static inline Ctx* C_(bst_ctx c) { return reinterpret_cast<Ctx*>(c); }
static inline Layout* L_(bst_layout l) { return reinterpret_cast<Layout*>(l); }
static inline bst_layout H_(Layout* l) { return reinterpret_cast<bst_layout>(l); }

template <class F>
static bst_status guarded(F&& f) {
  try {
    g_err.clear();
    f();
    return BST_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return BST_E_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return BST_E_ARG;
  } catch (...) {
    g_err = "unknown error";
    return BST_E_ARG;
  }
}

namespace bst {
Ctx::~Ctx() {
  if (side) {
    cudaStreamSynchronize(side);
    cudaStreamDestroy(side);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  projviews.clear();
  su2plans.clear();
  su2perm.clear();
  bplans.clear();
  ozplans.clear();
  cplans.clear();
  rplans.clear();
  for (auto& kv : gplans) kv.second->free_all();
  gplans.clear();
  for (auto& kv : bufs) kv.second.free_all();
  for (auto& kv : su2_weights) kv.second.free_all();
  for (auto& kv : interned) delete kv.second;
  for (auto e : evpool) cudaEventDestroy(e);
  if (d_err) cudaFree(d_err);
}
}  // namespace bst

static void set_dev(Ctx* c) {
  BST_REQUIRE(c->device >= 0, BST_E_ARG, "host-only context (device -1) cannot run device work");
  BST_CUDA(cudaSetDevice(c->device));
}

static std::vector<Leg> legs_from(int32_t rank, const bst_leg* legs) {
  BST_REQUIRE(legs != nullptr, BST_E_ARG, "legs is NULL");
  BST_REQUIRE(rank >= 1 && rank <= kMaxRank, BST_E_ARG, "rank must be 1..8");
  std::vector<Leg> out(rank);
  for (int i = 0; i < rank; ++i) {
    BST_REQUIRE(legs[i].nsect >= 1 && legs[i].charge && legs[i].deg, BST_E_ARG, "bad leg description");
    out[i].flow = legs[i].flow;
    out[i].q.assign(legs[i].charge, legs[i].charge + legs[i].nsect);
    out[i].d.assign(legs[i].deg, legs[i].deg + legs[i].nsect);
  }
  return out;
}

extern "C" {

bst_status bst_ctx_create(int device, size_t workspace_bytes, bst_ctx* out) {
  return guarded([&] {
    BST_REQUIRE(out != nullptr, BST_E_ARG, "out is NULL");
    if (device == -1) {  // host-only context: layouts and plans' host side, no compute
      auto* c = new Ctx();
      c->device = -1;
      *out = reinterpret_cast<bst_ctx>(c);
      return;
    }
    int n = 0;
    BST_CUDA(cudaGetDeviceCount(&n));
    BST_REQUIRE(device >= 0 && device < n, BST_E_ARG, "no such CUDA device");
    BST_CUDA(cudaSetDevice(device));
    auto* c = new Ctx();
    c->device = device;
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess) {
      delete c;
      throw Error(BST_E_OOM, "cannot allocate the device error word");
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    if (workspace_bytes) c->buf("contract.A", workspace_bytes, 0);
    *out = reinterpret_cast<bst_ctx>(c);
  });
}

bst_status bst_ctx_destroy(bst_ctx ctx) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    if (C_(ctx)->device >= 0) {
      set_dev(C_(ctx));
      cudaDeviceSynchronize();
    }
    delete C_(ctx);
  });
}

const char* bst_last_error(void) { return g_err.c_str(); }

bst_status bst_ctx_sync(bst_ctx ctx, bst_stream stream) {
  int code = 0;
  bst_status st = guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    Ctx* c = C_(ctx);
    set_dev(c);
    BST_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    BST_CUDA(cudaMemcpy(&code, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    BST_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
  });
  if (st != BST_OK) return st;
  if (code == BST_E_TIMEOUT) {
    g_err = "a bounded device wait expired";
    return BST_E_TIMEOUT;
  }
  if (code != 0) {
    g_err = "a kernel recorded a numeric error";
    return BST_E_NUMERIC;
  }
  return BST_OK;
}

int64_t bst_ctx_launch_count(bst_ctx ctx) { return ctx ? C_(ctx)->launches.load() : 0; }

double bst_ctx_work_flops(bst_ctx ctx) { return ctx ? C_(ctx)->work_flops : 0.0; }

bst_status bst_ctx_set_projector(bst_ctx ctx, int32_t method, int32_t iters) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    BST_REQUIRE(method == BST_PROJ_GESVD || method == BST_PROJ_SUBSPACE, BST_E_ARG, "unknown projector method");
    BST_REQUIRE(iters >= 1 && iters <= 200, BST_E_ARG, "iters must be 1..200");
    C_(ctx)->proj_method = method;
    C_(ctx)->proj_iters = iters;
  });
}

bst_status bst_ctx_set_wait_limit(bst_ctx ctx, int64_t tries) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    BST_REQUIRE(tries >= 0, BST_E_ARG, "tries must be >= 0");
    C_(ctx)->spin_limit = tries;
  });
}

bst_status bst_ctx_set_autotune(bst_ctx ctx, int32_t enable) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    C_(ctx)->autotune = enable != 0;
  });
}

bst_status bst_ctx_tuning_log(bst_ctx ctx, char* buf, size_t cap, size_t* len) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    const std::string& log = C_(ctx)->tune_log;
    if (len) *len = log.size();
    if (buf && cap > 0) {
      const size_t n = std::min(cap - 1, log.size());
      std::memcpy(buf, log.data(), n);
      buf[n] = 0;
    }
  });
}

bst_status bst_ctx_profile(bst_ctx ctx, int32_t enable) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    Ctx* c = C_(ctx);
    if (c->device >= 0) BST_CUDA(cudaDeviceSynchronize());
    c->prof = enable != 0;
    c->recs.clear();
    c->evused = 0;
  });
}

bst_status bst_ctx_profile_read(bst_ctx ctx, int32_t idx, char* cls, int32_t cls_len, int64_t* launches,
                                double* ms, double* flops, double* bytes) {
  return guarded([&] {
    BST_REQUIRE(ctx, BST_E_ARG, "ctx is NULL");
    Ctx* c = C_(ctx);
    std::vector<std::string> names;
    for (auto& r : c->recs)
      if (std::find(names.begin(), names.end(), r.cls) == names.end()) names.push_back(r.cls);
    BST_REQUIRE(idx >= 0 && idx < int32_t(names.size()), BST_E_ARG, "no such kernel class");
    int64_t n = 0;
    double t = 0, f = 0, b = 0;
    for (auto& r : c->recs) {
      if (r.cls != names[idx]) continue;
      float x = 0;
      BST_CUDA(cudaEventSynchronize(r.b));
      BST_CUDA(cudaEventElapsedTime(&x, r.a, r.b));
      ++n;
      t += x;
      f += r.flops;
      b += r.bytes;
    }
    if (cls && cls_len > 0) {
      std::strncpy(cls, names[idx].c_str(), size_t(cls_len) - 1);
      cls[cls_len - 1] = 0;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (flops) *flops = f;
    if (bytes) *bytes = b;
  });
}

bst_status bst_layout_create(bst_ctx ctx, bst_group group, int32_t rank, const bst_leg* legs, bst_layout* out) {
  return guarded([&] {
    BST_REQUIRE(ctx && out, BST_E_ARG, "null argument");
    *out = H_(make_layout(C_(ctx), int(group), legs_from(rank, legs)));
  });
}

bst_status bst_layout_retain(bst_layout l) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    retain(L_(l));
  });
}

bst_status bst_layout_release(bst_layout l) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    release(L_(l));
  });
}

bst_status bst_layout_info(bst_layout l, int32_t* rank, int64_t* nblocks, int64_t* nnz) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    if (rank) *rank = L_(l)->rank;
    if (nblocks) *nblocks = L_(l)->nblocks;
    if (nnz) *nnz = L_(l)->nnz;
  });
}

bst_status bst_layout_leg(bst_layout l, int32_t i, int32_t* flow, int32_t* nsect, int32_t* charges, int64_t* degs) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    Layout* L = L_(l);
    BST_REQUIRE(i >= 0 && i < L->rank, BST_E_ARG, "leg index out of range");
    const Leg& g = L->legs[i];
    if (flow) *flow = g.flow;
    if (nsect) *nsect = int32_t(g.q.size());
    if (charges) std::copy(g.q.begin(), g.q.end(), charges);
    if (degs) std::copy(g.d.begin(), g.d.end(), degs);
  });
}

bst_status bst_layout_block(bst_layout l, int64_t i, int32_t* sector_idx, int64_t* offset, int64_t* shape) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    Layout* L = L_(l);
    BST_REQUIRE(i >= 0 && i < L->nblocks, BST_E_ARG, "block index out of range");
    if (sector_idx) std::copy(&L->sect[i * L->rank], &L->sect[i * L->rank] + L->rank, sector_idx);
    if (offset) *offset = L->offset[i];
    if (shape) std::copy(&L->shape[i * L->rank], &L->shape[i * L->rank] + L->rank, shape);
  });
}

bst_status bst_layout_tree(bst_layout l, int64_t i, int32_t* ntree, int32_t* labels) {
  return guarded([&] {
    BST_REQUIRE(l, BST_E_ARG, "layout is NULL");
    Layout* L = L_(l);
    BST_REQUIRE(i >= 0 && i < L->nblocks, BST_E_ARG, "block index out of range");
    if (ntree) *ntree = L->ntree;
    if (labels && L->ntree) std::copy(&L->tree[i * L->ntree], &L->tree[i * L->ntree] + L->ntree, labels);
  });
}

bst_status bst_su2_cg(int32_t tj1, int32_t tm1, int32_t tj2, int32_t tm2, int32_t tJ, int32_t tM, double* out) {
  return guarded([&] {
    BST_REQUIRE(out, BST_E_ARG, "out is NULL");
    *out = su2_cg(tj1, tm1, tj2, tm2, tJ, tM);
  });
}

bst_status bst_layout_dual(bst_layout l, bst_layout* out) {
  return guarded([&] {
    BST_REQUIRE(l && out, BST_E_ARG, "null argument");
    Layout* L = L_(l);
    std::vector<Leg> legs;
    for (auto& g : L->legs) legs.push_back(g.dual());
    *out = H_(make_layout(L->ctx, L->group, legs));
  });
}

bst_status bst_permute(bst_ctx ctx, bst_layout src, const double* src_data, const int32_t* perm, bst_layout* dst,
                       double* dst_data, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && src && perm && dst, BST_E_ARG, "null argument");
    Ctx* c = C_(ctx);
    set_dev(c);
    Layout* S = L_(src);
    std::vector<int> p(perm, perm + S->rank);
    if (S->group == BST_SU2) {
      // trees recoupled to the permuted leg order
      BST_REQUIRE(S->nnz == 0 || (src_data && dst_data), BST_E_ARG, "data pointer is NULL");
      Layout* D = su2_permute(c, S, src_data, p, dst_data, (cudaStream_t)stream);
      retain(D);
      *dst = H_(D);
      return;
    }
    require_u1(S);
    Layout* D = nullptr;
    DevRelayout* rp = get_permute_plan(c, S, p, &D);
    if (S->nnz) {
      if (!src_data || !dst_data) {
        release(D);
        throw Error(BST_E_ARG, "data pointer is NULL");
      }
      launch_relayout(c, *rp, src_data, dst_data, 0, 1.0, 0.0, (cudaStream_t)stream);
    }
    *dst = H_(D);
  });
}

bst_status bst_fuse(bst_ctx ctx, bst_layout src, const double* src_data, int32_t ngroups, const int32_t* group_sizes,
                    bst_layout* dst, double* dst_data, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && src && group_sizes && dst && ngroups >= 1, BST_E_ARG, "bad argument");
    require_u1(L_(src));
    Ctx* c = C_(ctx);
    set_dev(c);
    std::vector<int> g(group_sizes, group_sizes + ngroups);
    Layout* D = nullptr;
    DevRelayout* rp = get_fuse_plan(c, L_(src), g, &D);
    if (L_(src)->nnz) {
      if (!src_data || !dst_data) {
        release(D);
        throw Error(BST_E_ARG, "data pointer is NULL");
      }
      launch_relayout(c, *rp, src_data, dst_data, 0, 1.0, 0.0, (cudaStream_t)stream);
    }
    *dst = H_(D);
  });
}

bst_status bst_plan_check(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs, const int32_t* legsA,
                          const int32_t* legsB, int64_t* mismatches) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && B && mismatches && npairs >= 0, BST_E_ARG, "bad argument");
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    Ctx* c = C_(ctx);
    set_dev(c);
    require_u1(L_(A));
    require_u1(L_(B));
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    *mismatches = plan_check(c, L_(A), L_(B), la, lb, 0);
  });
}

bst_status bst_contract_flops(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs, const int32_t* legsA,
                              const int32_t* legsB, double* flops) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && B && flops && npairs >= 0, BST_E_ARG, "bad argument");
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    require_u1(L_(A));
    require_u1(L_(B));
    ContractPlan* p = get_contract_plan(C_(ctx), L_(A), L_(B), la, lb);
    double f = 0;
    for (auto& g : p->probs) f += 2.0 * double(g.M) * g.N * g.K;
    *flops = f;
  });
}

bst_status bst_contract_layout(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs, const int32_t* legsA,
                               const int32_t* legsB, bst_layout* C) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && B && C && npairs >= 0, BST_E_ARG, "bad argument");
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    BST_REQUIRE(L_(A)->group == L_(B)->group, BST_E_ARG, "A and B belong to different symmetry groups");
    if (L_(A)->group == BST_SU2) {
      Layout* out = su2_contract_layout(C_(ctx), L_(A), L_(B), la, lb);
      retain(out);
      *C = H_(out);
      return;
    }
    ContractPlan* p = get_contract_plan(C_(ctx), L_(A), L_(B), la, lb);
    retain(p->C);
    *C = H_(p->C);
  });
}

bst_status bst_contract(bst_ctx ctx, bst_layout A, const double* a, bst_layout B, const double* b, int32_t npairs,
                        const int32_t* legsA, const int32_t* legsB, bst_prec prec, double alpha, double beta,
                        bst_layout C, double* c, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && B && C && npairs >= 0, BST_E_ARG, "bad argument");
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    require_prec(prec);
    Ctx* cx = C_(ctx);
    set_dev(cx);
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    BST_REQUIRE(L_(A)->group == L_(B)->group, BST_E_ARG, "A and B belong to different symmetry groups");
    if (L_(A)->group == BST_SU2) {
      su2_contract(cx, L_(A), a, L_(B), b, la, lb, prec, alpha, beta, L_(C), c, (cudaStream_t)stream);
      return;
    }
    ContractPlan* p = get_contract_plan(cx, L_(A), L_(B), la, lb);
    BST_REQUIRE(p->C == L_(C), BST_E_SHAPE, "C is not the layout of this contraction");
    BST_REQUIRE((L_(A)->nnz == 0 || a) && (L_(B)->nnz == 0 || b) && (p->C->nnz == 0 || c), BST_E_ARG,
                "data pointer is NULL");
    run_contract(cx, p, a, b, prec, alpha, beta, c, (cudaStream_t)stream);
  });
}

bst_status bst_contract_noalloc(bst_ctx ctx, bst_layout A, const double* a, bst_layout B, const double* b,
                                int32_t npairs, const int32_t* legsA, const int32_t* legsB, double alpha,
                                double beta, bst_layout C, double* c, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && B && C && npairs >= 0, BST_E_ARG, "bad argument");
    require_u1(L_(A));
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    contract_noalloc(C_(ctx), L_(A), a, L_(B), b, la, lb, alpha, beta, L_(C), c, (cudaStream_t)stream);
  });
}

bst_status bst_contract_batched(bst_ctx ctx, int32_t nbatch, const bst_layout* A, const double* const* a,
                                const bst_layout* B, const double* const* b, int32_t npairs, const int32_t* legsA,
                                const int32_t* legsB, bst_prec prec, double alpha, double beta, const bst_layout* C,
                                double* const* c, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && nbatch >= 1 && A && a && B && b && C && c && npairs >= 0, BST_E_ARG, "bad argument");
    BST_REQUIRE(npairs == 0 || (legsA && legsB), BST_E_ARG, "leg lists are NULL");
    require_prec(prec);
    Ctx* cx = C_(ctx);
    set_dev(cx);
    std::vector<Layout*> la_(nbatch), lb_(nbatch), lc_(nbatch);
    std::vector<const double*> pa(nbatch), pb(nbatch);
    std::vector<double*> pc(nbatch);
    for (int i = 0; i < nbatch; ++i) {
      BST_REQUIRE(A[i] && B[i] && C[i], BST_E_ARG, "layout handle is NULL");
      require_u1(L_(A[i]));
      require_u1(L_(B[i]));
      la_[i] = L_(A[i]);
      lb_[i] = L_(B[i]);
      lc_[i] = L_(C[i]);
      pa[i] = a[i];
      pb[i] = b[i];
      pc[i] = c[i];
    }
    std::vector<int> la(legsA, legsA + npairs), lb(legsB, legsB + npairs);
    contract_batched(cx, la_, pa, lb_, pb, la, lb, prec, alpha, beta, lc_, pc, (cudaStream_t)stream);
  });
}

bst_status bst_double_layer(bst_ctx ctx, bst_layout A, const double* A_data, bst_layout R, const double* R_data,
                            bst_layout* a_layout, double* a, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && a_layout, BST_E_ARG, "null argument");
    require_u1(L_(A));
    Ctx* c = C_(ctx);
    set_dev(c);
    cudaStream_t s = (cudaStream_t)stream;
    Layout* LA = L_(A);
    BST_REQUIRE(LA->rank == 5, BST_E_ARG, "site tensor must have rank 5 [p,l,u,r,d]");
    std::vector<Leg> dl;
    for (auto& g : LA->legs) dl.push_back(g.dual());
    Layout* LAd = make_layout(c, LA->group, dl);
    ContractPlan* p1 = get_contract_plan(c, LA, LAd, {0}, {0});  // [l,u,r,d,l~,u~,r~,d~]
    release(LAd);
    Layout* L2 = nullptr;
    DevRelayout* perm = get_permute_plan(c, p1->C, {0, 4, 1, 5, 2, 6, 3, 7}, &L2);
    Layout* L3 = nullptr;
    DevRelayout* fuse = get_fuse_plan(c, L2, {2, 2, 2, 2}, &L3);
    release(L2);
    Layout* out = L3;
    ContractPlan* p2 = nullptr;
    DevRelayout *rperm = nullptr, *rfuse = nullptr, *aperm = nullptr;
    Layout *Lr3 = nullptr, *La4 = nullptr;
    ContractPlan* pr = nullptr;
    if (R) {
      Layout* LR = L_(R);
      BST_REQUIRE(LR->rank == 3, BST_E_ARG, "remover must have rank 3 [r,l',s]");
      std::vector<Leg> rl;
      for (auto& g : LR->legs) rl.push_back(g.dual());
      Layout* LRd = make_layout(c, LR->group, rl);
      pr = get_contract_plan(c, LR, LRd, {2}, {2});  // [r,l',r~,l'~]
      release(LRd);
      Layout* Lr2 = nullptr;
      rperm = get_permute_plan(c, pr->C, {0, 2, 1, 3}, &Lr2);
      rfuse = get_fuse_plan(c, Lr2, {2, 2}, &Lr3);  // rho[k_r, k_l']
      release(Lr2);
      p2 = get_contract_plan(c, L3, Lr3, {2}, {0});  // [kl, ku, kd, kl']
      aperm = get_permute_plan(c, p2->C, {0, 1, 3, 2}, &La4);
      release(L3);
      release(Lr3);
      out = La4;
    }
    if (a) {
      BST_REQUIRE(*a_layout == H_(out), BST_E_SHAPE, "a_layout is not the double-layer layout");
      BST_REQUIRE(A_data && (!R || R_data), BST_E_ARG, "data pointer is NULL");
      double* t1 = (double*)c->buf("dl.AA", sizeof(double) * std::max<int64_t>(p1->C->nnz, 1), s);
      double* t2 = (double*)c->buf("dl.AAp", sizeof(double) * std::max<int64_t>(p1->C->nnz, 1), s);
      run_contract(c, p1, A_data, A_data, BST_FP64, 1.0, 0.0, t1, s);
      launch_relayout(c, *perm, t1, t2, 0, 1.0, 0.0, s);
      if (!R) {
        launch_relayout(c, *fuse, t2, a, 0, 1.0, 0.0, s);
      } else {
        double* t3 = (double*)c->buf("dl.a", sizeof(double) * std::max<int64_t>(p1->C->nnz, 1), s);
        launch_relayout(c, *fuse, t2, t3, 0, 1.0, 0.0, s);
        double* r1 = (double*)c->buf("dl.RR", sizeof(double) * std::max<int64_t>(pr->C->nnz, 1), s);
        double* r2 = (double*)c->buf("dl.RRp", sizeof(double) * std::max<int64_t>(pr->C->nnz, 1), s);
        double* r3 = (double*)c->buf("dl.rho", sizeof(double) * std::max<int64_t>(pr->C->nnz, 1), s);
        run_contract(c, pr, R_data, R_data, BST_FP64, 1.0, 0.0, r1, s);
        launch_relayout(c, *rperm, r1, r2, 0, 1.0, 0.0, s);
        launch_relayout(c, *rfuse, r2, r3, 0, 1.0, 0.0, s);
        double* t4 = (double*)c->buf("dl.a2", sizeof(double) * std::max<int64_t>(p2->C->nnz, 1), s);
        run_contract(c, p2, t3, r3, BST_FP64, 1.0, 0.0, t4, s);
        launch_relayout(c, *aperm, t4, a, 0, 1.0, 0.0, s);
      }
      release(out);
    } else {
      *a_layout = H_(out);
    }
  });
}

bst_status bst_svd_projector(bst_ctx ctx, bst_layout Rtop, const double* rtop, bst_layout Rbot, const double* rbot,
                             int32_t ncut, int64_t chi, double rel_cutoff, int32_t new_flow, bst_prec prec,
                             bst_layout* P, double* p, bst_layout* Pt, double* pt, double* svals, int64_t* kept,
                             bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && Rtop && Rbot && rtop && rbot && P && p && Pt && pt && kept, BST_E_ARG, "null argument");
    require_u1(L_(Rtop));
    Ctx* c = C_(ctx);
    set_dev(c);
    ProjResult r = svd_projector(c, L_(Rtop), rtop, L_(Rbot), rbot, ncut, chi, rel_cutoff, new_flow, prec, p, pt,
                                 (cudaStream_t)stream);
    BST_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *P = H_(r.P);
    *Pt = H_(r.Pt);
    *kept = r.kept;
    if (svals) std::copy(r.svals.begin(), r.svals.end(), svals);
  });
}

bst_status bst_sym_eig(bst_ctx ctx, int32_t n, int32_t batch, const double* H, double* X, double* lam,
                       bst_prec prec, bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && H && X && lam, BST_E_ARG, "null argument");
    Ctx* c = C_(ctx);
    set_dev(c);
    // the refinement's products need the FP64-accurate arithmetic
    sym_eig_batched(c, n, batch, H, X, lam, prec == BST_BF16X3 ? BST_OZAKI : prec, (cudaStream_t)stream);
  });
}

bst_status bst_ctm_move_cell(bst_ctx ctx, int32_t dir, int32_t Lx, int32_t Ly, const bst_layout* a_layouts,
                             const double* const* a, bst_env* envs, int64_t chi, double rel_cutoff, bst_prec prec,
                             bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && a_layouts && a && envs, BST_E_ARG, "null argument");
    BST_REQUIRE(Lx >= 1 && Ly >= 1 && int64_t(Lx) * Ly <= 64, BST_E_ARG, "cell must be 1..64 sites");
    BST_REQUIRE(chi >= 1, BST_E_ARG, "chi must be positive");
    Ctx* c = C_(ctx);
    set_dev(c);
    std::vector<Layout*> L(size_t(Lx) * Ly);
    for (size_t i = 0; i < L.size(); ++i) {
      BST_REQUIRE(a_layouts[i], BST_E_ARG, "site layout is NULL");
      L[i] = L_(a_layouts[i]);
    }
    ctm_move_cell(c, dir, Lx, Ly, L.data(), a, envs, chi, rel_cutoff, prec, (cudaStream_t)stream);
  });
}

bst_status bst_ctm_move(bst_ctx ctx, int32_t dir, bst_layout a_layout, const double* a, bst_env* env, int64_t chi,
                        double rel_cutoff, bst_prec prec, bst_ctm_stats* stats, bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && a_layout && a && env, BST_E_ARG, "null argument");
    BST_REQUIRE(chi >= 1, BST_E_ARG, "chi must be positive");
    Ctx* c = C_(ctx);
    set_dev(c);
    ctm_move(c, dir, L_(a_layout), a, env, chi, rel_cutoff, prec, stats, (cudaStream_t)stream);
  });
}

bst_status bst_double_layer_open(bst_ctx ctx, bst_layout A, const double* A_data, bst_layout R, const double* R_data,
                                 bst_layout* a_layout, double* a, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && A && a_layout, BST_E_ARG, "null argument");
    Ctx* c = C_(ctx);
    set_dev(c);
    Layout* out = double_layer_open(c, L_(A), A_data, R ? L_(R) : nullptr, R_data, a, (cudaStream_t)stream);
    if (a) {
      const bool same = *a_layout == H_(out);
      release(out);
      BST_REQUIRE(same, BST_E_SHAPE, "a_layout is not the open double-layer layout");
    } else {
      *a_layout = H_(out);
    }
  });
}

bst_status bst_ctm_bond_rdm(bst_ctx ctx, int32_t bond, bst_layout site, const double* site_data, bst_env* env,
                            bst_prec prec, bst_layout* rho_layout, double* rho, int64_t rho_cap, bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && site && site_data && env && rho_layout, BST_E_ARG, "null argument");
    Ctx* c = C_(ctx);
    set_dev(c);
    cudaStream_t s = (cudaStream_t)stream;
    double* r = nullptr;
    Layout* RL = bond_rdm(c, bond, L_(site), site_data, env, prec, &r, s);
    if (rho) {
      if (RL->nnz > rho_cap) {
        release(RL);
        throw Error(BST_E_SHAPE, "rho buffer capacity too small");
      }
      BST_CUDA(cudaMemcpyAsync(rho, r, sizeof(double) * RL->nnz, cudaMemcpyDeviceToDevice, s));
    }
    *rho_layout = H_(RL);
  });
}

bst_status bst_dot(bst_ctx ctx, bst_layout layout, const double* x, const double* y, double* out, bst_stream stream) {
  return guarded([&] {
    BST_REQUIRE(ctx && layout && out, BST_E_ARG, "null argument");
    BST_REQUIRE(L_(layout)->nnz == 0 || (x && y), BST_E_ARG, "data pointer is NULL");
    Ctx* c = C_(ctx);
    set_dev(c);
    *out = block_dot(c, x, y, L_(layout)->nnz, (cudaStream_t)stream);
  });
}

bst_status bst_ctm_converge(bst_ctx ctx, bst_layout a_layout, const double* a, bst_layout site, const double* site_data,
                            bst_layout H_layout, const double* H, bst_env* env, int64_t chi0, int64_t chi_max,
                            double tol, int32_t max_steps, double rel_cutoff, bst_prec prec,
                            bst_ctm_converge_stats* stats, bst_stream stream) {
  return guarded([&] {
    require_prec(prec);
    BST_REQUIRE(ctx && a_layout && a && site && site_data && H_layout && H && env && stats, BST_E_ARG,
                "null argument");
    Ctx* c = C_(ctx);
    set_dev(c);
    bst_ctm_converge_stats st;
    ctm_converge(c, L_(a_layout), a, L_(site), site_data, L_(H_layout), H, env, chi0, chi_max, tol, max_steps,
                 rel_cutoff, prec, &st, (cudaStream_t)stream);
    *stats = st;
  });
}

}  // extern "C"
