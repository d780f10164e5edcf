// SU(2)-symmetric tensors (Sec. 2): every block is a reduced dense tensor
// times a generalised CGC tensor (Eq. "tensor-cgc").
//
// Basis of a block (the paper fixes it for ranks 2 and 3 only; this is the
// reading used for every rank): the block is a map from its outgoing legs to
// its incoming legs through one coupled spin J,
//     c[m_in; m_out] = sum_M <in-tree m_in | J M> <out-tree m_out | J M>,
// where a tree couples its legs left to right with Condon-Shortley
// Clebsch-Gordan coefficients (no leg: the singlet, one leg: that leg).  Tree
// labels: the in-tree intermediates, J, the out-tree intermediates, all as
// doubled spins.  Blocks are ordered by per-leg sector index, then by tree
// labels.  ||c||^2 = 2J + 1 and blocks of one sector tuple are orthogonal.
//
// Contraction (Sec. 2, the block-pair formula and the reduction after it):
// every pair of blocks that agree on the contracted legs gives the reduced
// product m_A . m_B and the CGC product c_A . c_B; the latter is expanded in
// the output's canonical blocks with coefficients
//     X = <c_C, c_A . c_B> / (2 J_C + 1)
// ("X-symbols", computed here by contracting the CGC tensors explicitly), and
// the output block is the X-weighted sum of its pair products.  On the GPU:
//   1. gather A's blocks into one matrix per contracted sector tuple sK
//      (rows: every A block with that sK, columns: the contracted reduced
//      indices) and B's likewise;
//   2. one grouped GEMM (FP64 or the BF16-slice tensor-core GEMM) computes,
//      per sK, every pair product at once: P_sK = A_sK . B_sK^T;
//   3. the recoupling kernel reads each pair product once and adds it, with
//      its X-symbols, into all output blocks of that sector tuple
//      (r_k = sum X . P), writing C = alpha r + beta C.
// The coefficient tables are host plan-time work, cached with the plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <tuple>
#include <unordered_map>

#include "bst_internal.h"
#include "relayout_dev.cuh"

namespace bst {

// ---------------------------------------------------------------------------
// Clebsch-Gordan coefficients: Racah's closed formula in long double

static long double lfact(int n) {
  static long double tab[256];
  static bool init = false;
  if (!init) {
    tab[0] = 1.0L;
    for (int i = 1; i < 256; ++i) tab[i] = tab[i - 1] * (long double)i;
    init = true;
  }
  return tab[n];
}

static double cg_compute(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  if (tm1 + tm2 != tM) return 0.0;
  if (tJ < std::abs(tj1 - tj2) || tJ > tj1 + tj2 || ((tj1 + tj2 + tJ) & 1)) return 0.0;
  if (std::abs(tm1) > tj1 || std::abs(tm2) > tj2 || std::abs(tM) > tJ) return 0.0;
  if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
  auto F = [](int n2) { return lfact(n2 / 2); };
  const long double pre2 = (long double)(tJ + 1) * F(tJ + tj1 - tj2) * F(tJ - tj1 + tj2) * F(tj1 + tj2 - tJ) /
                           F(tj1 + tj2 + tJ + 2) * F(tJ + tM) * F(tJ - tM) * F(tj1 - tm1) * F(tj1 + tm1) *
                           F(tj2 - tm2) * F(tj2 + tm2);
  long double s = 0.0L;
  for (int k = 0; 2 * k <= tj1 + tj2 + tJ; ++k) {
    const int a[5] = {tj1 + tj2 - tJ - 2 * k, tj1 - tm1 - 2 * k, tj2 + tm2 - 2 * k, tJ - tj2 + tm1 + 2 * k,
                      tJ - tj1 - tm2 + 2 * k};
    bool ok = true;
    for (int x : a) ok = ok && x >= 0;
    if (!ok) continue;
    long double den = lfact(k);
    for (int x : a) den *= F(x);
    s += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  return double(s * sqrtl(pre2));
}

double su2_cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  BST_REQUIRE(tj1 >= 0 && tj2 >= 0 && tJ >= 0 && tj1 + tj2 + tJ < 400, BST_E_ARG, "spins out of range");
  static std::mutex mu;
  static std::unordered_map<uint64_t, double> cache;
  auto enc = [](int x) { return uint64_t(uint32_t(x + 512) & 1023u); };
  const uint64_t key = enc(tj1) | enc(tm1) << 10 | enc(tj2) << 20 | enc(tm2) << 30 | enc(tJ) << 40 | enc(tM) << 50;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const double v = cg_compute(tj1, tm1, tj2, tm2, tJ, tM);
  std::lock_guard<std::mutex> g(mu);
  cache[key] = v;
  return v;
}

// ---------------------------------------------------------------------------
// coupling trees and block enumeration

// Left-to-right coupling trees of spins tjs: (intermediates after legs
// 2..n-1, final spin).
static void couplings(const std::vector<int>& tjs, std::vector<std::pair<std::vector<int>, int>>& out) {
  out.clear();
  const int n = int(tjs.size());
  if (n == 0) {
    out.push_back({{}, 0});
    return;
  }
  if (n == 1) {
    out.push_back({{}, tjs[0]});
    return;
  }
  std::vector<int> inter;
  std::function<void(int, int)> rec = [&](int k, int i) {
    for (int kn = std::abs(k - tjs[i]); kn <= k + tjs[i]; kn += 2) {
      if (i == n - 1) {
        out.push_back({inter, kn});
      } else {
        inter.push_back(kn);
        rec(kn, i + 1);
        inter.pop_back();
      }
    }
  };
  rec(tjs[0], 1);
}

static void in_out(const std::vector<int>& flows, std::vector<int>& ins, std::vector<int>& outs) {
  ins.clear();
  outs.clear();
  for (int i = 0; i < int(flows.size()); ++i) (flows[i] == 1 ? ins : outs).push_back(i);
}

int su2_ntree(const std::vector<Leg>& legs) {
  int ni = 0, no = 0;
  for (auto& l : legs) (l.flow == 1 ? ni : no)++;
  return std::max(ni - 2, 0) + 1 + std::max(no - 2, 0);
}

void su2_enum_blocks(const std::vector<Leg>& legs, std::vector<int32_t>& sect, std::vector<int32_t>& tree) {
  const int r = int(legs.size());
  std::vector<int> flows(r), ins, outs;
  for (int i = 0; i < r; ++i) flows[i] = legs[i].flow;
  in_out(flows, ins, outs);
  std::vector<int32_t> cur(r, 0);
  std::vector<std::pair<std::vector<int>, int>> tin, tout;
  std::vector<int> sin, sout;
  while (true) {
    sin.clear();
    sout.clear();
    for (int i : ins) sin.push_back(legs[i].q[cur[i]]);
    for (int i : outs) sout.push_back(legs[i].q[cur[i]]);
    couplings(sin, tin);
    couplings(sout, tout);
    std::vector<std::vector<int32_t>> labels;
    for (auto& a : tin)
      for (auto& b : tout)
        if (a.second == b.second) {
          std::vector<int32_t> t(a.first.begin(), a.first.end());
          t.push_back(a.second);
          t.insert(t.end(), b.first.begin(), b.first.end());
          labels.push_back(t);
        }
    std::sort(labels.begin(), labels.end());
    for (auto& t : labels) {
      sect.insert(sect.end(), cur.begin(), cur.end());
      tree.insert(tree.end(), t.begin(), t.end());
    }
    int i = r - 1;
    while (i >= 0 && ++cur[i] == int(legs[i].q.size())) cur[i--] = 0;
    if (i < 0) break;
  }
}

// ---------------------------------------------------------------------------
// generalised CGC tensors

// V[m_1..m_n, M] = <tree(m_1..m_n) | J M>, row-major, m descending.
static std::vector<double> tree_vector(const std::vector<int>& tjs, const int32_t* inter, int tJ, int* mdim) {
  const int n = int(tjs.size());
  if (n == 0) {
    *mdim = 1;
    return {1.0};
  }
  int tk = tjs[0];
  std::vector<double> V((tk + 1) * (tk + 1), 0.0);
  for (int a = 0; a <= tk; ++a) V[a * (tk + 1) + a] = 1.0;
  int64_t lead = tk + 1;  // product of the m extents so far
  for (int i = 1; i < n; ++i) {
    const int tkn = i < n - 1 ? inter[i - 1] : tJ;
    const int tji = tjs[i];
    std::vector<double> W((tk + 1) * (tji + 1) * (tkn + 1));
    for (int a = 0; a <= tk; ++a)
      for (int b = 0; b <= tji; ++b)
        for (int c = 0; c <= tkn; ++c)
          W[(a * (tji + 1) + b) * (tkn + 1) + c] = su2_cg(tk, tk - 2 * a, tji, tji - 2 * b, tkn, tkn - 2 * c);
    std::vector<double> Vn(lead * (tji + 1) * (tkn + 1), 0.0);
    for (int64_t p = 0; p < lead; ++p)
      for (int a = 0; a <= tk; ++a) {
        const double v = V[p * (tk + 1) + a];
        if (v == 0.0) continue;
        for (int b = 0; b <= tji; ++b)
          for (int c = 0; c <= tkn; ++c) Vn[(p * (tji + 1) + b) * (tkn + 1) + c] += v * W[(a * (tji + 1) + b) * (tkn + 1) + c];
      }
    V.swap(Vn);
    lead *= tji + 1;
    tk = tkn;
  }
  *mdim = tJ + 1;
  return V;
}

// Dense CGC tensor of one block, row-major over the legs' m in leg order.
static std::vector<double> basis_tensor(const std::vector<int>& tj, const std::vector<int>& flows,
                                        const int32_t* labels) {
  std::vector<int> ins, outs;
  in_out(flows, ins, outs);
  const int ni = int(ins.size()), no = int(outs.size());
  const int nii = std::max(ni - 2, 0);
  const int tJ = labels[nii];
  std::vector<int> sin, sout;
  for (int i : ins) sin.push_back(tj[i]);
  for (int i : outs) sout.push_back(tj[i]);
  int mi = 0, mo = 0;
  std::vector<double> Vi = tree_vector(sin, labels, tJ, &mi);
  std::vector<double> Vo = tree_vector(sout, labels + nii + 1, tJ, &mo);
  const int64_t ni_m = int64_t(Vi.size()) / mi, no_m = int64_t(Vo.size()) / mo;
  // c in (ins..., outs...) order
  std::vector<double> cio(ni_m * no_m, 0.0);
  for (int64_t p = 0; p < ni_m; ++p)
    for (int64_t q = 0; q < no_m; ++q) {
      double s = 0.0;
      for (int M = 0; M < mi; ++M) s += Vi[p * mi + M] * Vo[q * mo + M];
      cio[p * no_m + q] = s;
    }
  // to leg order
  const int r = int(tj.size());
  std::vector<int> order = ins;
  order.insert(order.end(), outs.begin(), outs.end());
  std::vector<int64_t> ext(r), src_stride(r);
  for (int i = 0; i < r; ++i) ext[i] = tj[i] + 1;
  // strides of the (ins, outs) layout, indexed by leg
  int64_t st = 1;
  for (int k = r - 1; k >= 0; --k) {
    src_stride[order[k]] = st;
    st *= ext[order[k]];
  }
  std::vector<double> c(st);
  std::vector<int> idx(r, 0);
  for (int64_t e = 0; e < st; ++e) {
    int64_t so = 0;
    for (int i = 0; i < r; ++i) so += idx[i] * src_stride[i];
    c[e] = cio[so];
    for (int i = r - 1; i >= 0; --i) {
      if (++idx[i] < ext[i]) break;
      idx[i] = 0;
    }
  }
  return c;
}

// ---------------------------------------------------------------------------
// contraction plan

constexpr int kMaxTau = 8;      // output blocks of one sector tuple per recoupling group
constexpr int kRcThreads = 256;  // one output element per thread
constexpr int kRcStage = 64;     // contributions staged in shared memory at a time

struct RcGroup {
  int32_t M, N;
  int32_t ntau, ncontrib;
  int64_t contrib0;
  int64_t c_off[kMaxTau];
};

struct RcContrib {
  int64_t p_off;  // first element of the pair product in P
  int64_t ld;     // row stride of that product in P
};

struct Su2Plan {
  Layout *A = nullptr, *B = nullptr, *C = nullptr;
  DevRelayout ra, rb;
  std::vector<GemmProb> probs;
  DevGemm g;
  int64_t amat = 0, bmat = 0, pmat = 0;
  double* Am = nullptr;
  double* Bm = nullptr;
  double* P = nullptr;
  RcGroup* d_groups = nullptr;
  int2* d_chunks = nullptr;
  RcContrib* d_ct = nullptr;
  double* d_x = nullptr;
  int nchunks = 0;
  double rc_reads = 0;  // elements of P the recoupling reads
  ~Su2Plan() {
    ra.free_all();
    rb.free_all();
    g.free_all();
    cudaFree(Am);
    cudaFree(Bm);
    cudaFree(P);
    cudaFree(d_groups);
    cudaFree(d_chunks);
    cudaFree(d_ct);
    cudaFree(d_x);
    release(A);
    release(B);
    release(C);
  }
};

// One output element per thread: acc[t] = sum over the group's
// contributions i of X[i][t] P_i[m][col], for the NT output trees of the
// group.  NT is a compile-time bound (1, 2, 4 or 8 >= the group's tree
// count): this part's FP64 pipe does about two FMAs per clock per SM, so the
// kernel is bound by its multiply-adds and does only the ones it needs.
template <int NT>
__device__ __forceinline__ void recouple_body(const RcGroup& g, int ntau, int e, bool live, int m, int col,
                                              const RcContrib* __restrict__ ct, const double* __restrict__ X,
                                              const double* __restrict__ P, double* C, double alpha, double beta,
                                              RcContrib* sct, double* sx) {
  double acc[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) acc[t] = 0.0;
  for (int c0 = 0; c0 < g.ncontrib; c0 += kRcStage) {
    const int nc = min(kRcStage, g.ncontrib - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += kRcThreads) sct[i] = ct[g.contrib0 + c0 + i];
    for (int i = threadIdx.x; i < nc * NT; i += kRcThreads) {
      const int ci = i / NT, t = i - ci * NT;
      sx[i] = X[(g.contrib0 + c0 + ci) * kMaxTau + t];
    }
    __syncthreads();
    if (live) {
      for (int i = 0; i < nc; ++i) {
        const double p = P[sct[i].p_off + (long long)m * sct[i].ld + col];
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[t] = fma(sx[i * NT + t], p, acc[t]);
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (t < ntau) {
      double* out = C + g.c_off[t] + e;
      double v = alpha * acc[t];
      if (beta != 0.0) v += beta * *out;
      *out = v;
    }
  }
}

__global__ void __launch_bounds__(kRcThreads) recouple_kernel(const RcGroup* __restrict__ groups,
                                                              const int2* __restrict__ chunks,
                                                              const RcContrib* __restrict__ ct,
                                                              const double* __restrict__ X,
                                                              const double* __restrict__ P, double* C,
                                                              double alpha, double beta) {
  __shared__ RcContrib sct[kRcStage];
  __shared__ double sx[kRcStage * kMaxTau];
  const int2 ch = chunks[blockIdx.x];
  const RcGroup& g = groups[ch.x];
  const int n = g.M * g.N;
  const int e = ch.y + threadIdx.x;
  const bool live = e < n;
  const int m = live ? e / g.N : 0, col = live ? e - m * g.N : 0;
  const int ntau = g.ntau;  // the same for the whole CTA
  if (ntau <= 1) recouple_body<1>(g, ntau, e, live, m, col, ct, X, P, C, alpha, beta, sct, sx);
  else if (ntau <= 2) recouple_body<2>(g, ntau, e, live, m, col, ct, X, P, C, alpha, beta, sct, sx);
  else if (ntau <= 4) recouple_body<4>(g, ntau, e, live, m, col, ct, X, P, C, alpha, beta, sct, sx);
  else recouple_body<kMaxTau>(g, ntau, e, live, m, col, ct, X, P, C, alpha, beta, sct, sx);
}

namespace {

struct BlockRef {
  int64_t blk;            // block index in its layout
  std::vector<int32_t> so;  // open sector indices
  int64_t row0 = 0;       // first row in its sK matrix
  int64_t rows = 0;       // product of open reduced extents
};

struct SkGroup {
  std::vector<BlockRef> a, b;
  int64_t K = 1, M = 0, N = 0;
  int64_t aoff = 0, boff = 0, poff = 0;
};

// Non-zero entries of a CGC tensor split into (contracted m index, open m
// index, value) for the given contracted legs (in pair order).
struct SplitC {
  std::vector<int64_t> kc, oc;
  std::vector<double> v;
};

SplitC split_basis(const std::vector<double>& c, const std::vector<int>& tj, const std::vector<int>& cl,
                   const std::vector<int>& ol) {
  const int r = int(tj.size());
  std::vector<std::tuple<int64_t, int64_t, double>> nz;
  std::vector<int> idx(r, 0);
  for (size_t e = 0; e < c.size(); ++e) {
    if (c[e] != 0.0) {
      int64_t k = 0, o = 0;
      for (int i : cl) k = k * (tj[i] + 1) + idx[i];
      for (int i : ol) o = o * (tj[i] + 1) + idx[i];
      nz.emplace_back(k, o, c[e]);
    }
    for (int i = r - 1; i >= 0; --i) {
      if (++idx[i] <= tj[i]) break;
      idx[i] = 0;
    }
  }
  std::stable_sort(nz.begin(), nz.end(),
                   [](const auto& x, const auto& y) { return std::get<0>(x) < std::get<0>(y); });
  SplitC s;
  for (auto& t : nz) {
    s.kc.push_back(std::get<0>(t));
    s.oc.push_back(std::get<1>(t));
    s.v.push_back(std::get<2>(t));
  }
  return s;
}

std::vector<int> spins_of(const Layout* L, int64_t b) {
  std::vector<int> tj(L->rank);
  for (int i = 0; i < L->rank; ++i) tj[i] = L->legs[i].q[L->sect[b * L->rank + i]];
  return tj;
}

std::vector<int> flows_of(const Layout* L) {
  std::vector<int> f(L->rank);
  for (int i = 0; i < L->rank; ++i) f[i] = L->legs[i].flow;
  return f;
}

// relayout task of one block into its sK matrix: row index over the open
// legs (row-major), column index over the contracted legs (pair order)
RelTask gather_task(const Layout* L, int64_t b, const std::vector<int>& ol, const std::vector<int>& cl,
                    int64_t mat_base, int64_t K) {
  RelTask t{};
  t.blk_off = L->offset[b];
  t.mat_base = mat_base;
  t.rank = L->rank;
  int64_t n = 1;
  for (int i = 0; i < L->rank; ++i) {
    t.shape[i] = int32_t(L->shape[b * L->rank + i]);
    n *= t.shape[i];
  }
  t.n = int32_t(n);
  int64_t st = K;
  for (int j = int(ol.size()) - 1; j >= 0; --j) {
    t.mstride[ol[j]] = st;
    st *= L->shape[b * L->rank + ol[j]];
  }
  st = 1;
  for (int j = int(cl.size()) - 1; j >= 0; --j) {
    t.mstride[cl[j]] = st;
    st *= L->shape[b * L->rank + cl[j]];
  }
  return t;
}

}  // namespace

static Su2Plan* build_su2_plan(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la,
                               const std::vector<int>& lb) {
  auto plan = std::make_unique<Su2Plan>();
  Su2Plan* p = plan.get();
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
    if (!ua[i]) oa.push_back(i), cl.push_back(A->legs[i]);
  for (int i = 0; i < B->rank; ++i)
    if (!ub[i]) ob.push_back(i), cl.push_back(B->legs[i]);
  BST_REQUIRE(!cl.empty(), BST_E_ARG, "contraction over every leg (rank-0 result) is not supported");
  p->A = A;
  p->B = B;
  retain(A);
  retain(B);
  p->C = make_layout(ctx, BST_SU2, cl);
  Layout* C = p->C;

  // group blocks by contracted sector tuple (pair order)
  std::map<std::vector<int32_t>, SkGroup> groups;
  for (int64_t b = 0; b < A->nblocks; ++b) {
    std::vector<int32_t> sk, so;
    for (int i : la) sk.push_back(A->sect[b * A->rank + i]);
    for (int i : oa) so.push_back(A->sect[b * A->rank + i]);
    BlockRef r;
    r.blk = b;
    r.so = so;
    r.rows = 1;
    for (int i : oa) r.rows *= A->shape[b * A->rank + i];
    groups[sk].a.push_back(r);
  }
  for (int64_t b = 0; b < B->nblocks; ++b) {
    std::vector<int32_t> sk, so;
    for (int i : lb) sk.push_back(B->sect[b * B->rank + i]);
    for (int i : ob) so.push_back(B->sect[b * B->rank + i]);
    BlockRef r;
    r.blk = b;
    r.so = so;
    r.rows = 1;
    for (int i : ob) r.rows *= B->shape[b * B->rank + i];
    auto it = groups.find(sk);
    if (it != groups.end()) it->second.b.push_back(r);
  }
  std::vector<RelTask> ta, tb;
  for (auto it = groups.begin(); it != groups.end();) {
    SkGroup& g = it->second;
    if (g.a.empty() || g.b.empty()) {
      it = groups.erase(it);
      continue;
    }
    g.K = 1;
    for (size_t j = 0; j < la.size(); ++j) g.K *= A->legs[la[j]].d[it->first[j]];
    for (auto& r : g.a) r.row0 = g.M, g.M += r.rows;
    for (auto& r : g.b) r.row0 = g.N, g.N += r.rows;
    g.aoff = p->amat;
    g.boff = p->bmat;
    g.poff = p->pmat;
    p->amat += g.M * g.K;
    p->bmat += g.N * g.K;
    p->pmat += g.M * g.N;
    for (auto& r : g.a) ta.push_back(gather_task(A, r.blk, oa, la, g.aoff + r.row0 * g.K, g.K));
    for (auto& r : g.b) tb.push_back(gather_task(B, r.blk, ob, lb, g.boff + r.row0 * g.K, g.K));
    GemmProb q{};
    q.M = int32_t(g.M);
    q.N = int32_t(g.N);
    q.K = int32_t(g.K);
    q.a_off = g.aoff;
    q.b_off = g.boff;
    q.c_off = g.poff;
    q.a_m = g.K;
    q.a_k = 1;
    q.b_n = g.K;
    q.b_k = 1;
    q.c_m = g.N;
    q.c_n = 1;
    p->probs.push_back(q);
    ++it;
  }

  // X-symbols: for every output sector tuple, its blocks (trees) tau and the
  // contributing pairs (a, b) with the coefficients X[tau]
  const std::vector<int> fA = flows_of(A), fB = flows_of(B), fC = flows_of(C);
  std::unordered_map<int64_t, SplitC> cA, cB;
  auto getA = [&](int64_t b) -> const SplitC& {
    auto it = cA.find(b);
    if (it != cA.end()) return it->second;
    const std::vector<int> tj = spins_of(A, b);
    return cA[b] = split_basis(basis_tensor(tj, fA, &A->tree[b * A->ntree]), tj, la, oa);
  };
  auto getB = [&](int64_t b) -> const SplitC& {
    auto it = cB.find(b);
    if (it != cB.end()) return it->second;
    const std::vector<int> tj = spins_of(B, b);
    return cB[b] = split_basis(basis_tensor(tj, fB, &B->tree[b * B->ntree]), tj, lb, ob);
  };
  int nCi = 0;
  for (int f : fC) nCi += f == 1;
  const int jpos = std::max(nCi - 2, 0);

  std::vector<RcGroup> hg;
  std::vector<RcContrib> hc;
  std::vector<double> hx;
  std::vector<int2> hch;
  const int na = int(oa.size());
  std::vector<double> dense_kc;  // per contracted-m index: scratch
  for (int64_t b0 = 0; b0 < C->nblocks;) {
    int64_t b1 = b0;
    while (b1 < C->nblocks &&
           std::equal(&C->sect[b1 * C->rank], &C->sect[b1 * C->rank] + C->rank, &C->sect[b0 * C->rank]))
      ++b1;
    const std::vector<int32_t> sC(&C->sect[b0 * C->rank], &C->sect[b0 * C->rank] + C->rank);
    const std::vector<int32_t> soa(sC.begin(), sC.begin() + na), sob(sC.begin() + na, sC.end());
    const std::vector<int> tjC = spins_of(C, b0);
    int64_t M = 1, N = 1;
    for (int i = 0; i < na; ++i) M *= C->shape[b0 * C->rank + i];
    for (int i = na; i < C->rank; ++i) N *= C->shape[b0 * C->rank + i];
    int64_t nob_m = 1;
    for (int i = na; i < C->rank; ++i) nob_m *= tjC[i] + 1;
    for (int64_t t0 = b0; t0 < b1; t0 += kMaxTau) {
      const int ntau = int(std::min<int64_t>(kMaxTau, b1 - t0));
      std::vector<std::vector<double>> cC(ntau);
      std::vector<double> norm(ntau);
      for (int t = 0; t < ntau; ++t) {
        cC[t] = basis_tensor(tjC, fC, &C->tree[(t0 + t) * C->ntree]);
        norm[t] = 1.0 / double(C->tree[(t0 + t) * C->ntree + jpos] + 1);
      }
      RcGroup g{};
      g.M = int32_t(M);
      g.N = int32_t(N);
      g.ntau = ntau;
      g.contrib0 = int64_t(hc.size());
      for (int t = 0; t < ntau; ++t) g.c_off[t] = C->offset[t0 + t];
      for (auto& kv : groups) {
        const SkGroup& sg = kv.second;
        for (const BlockRef& ra : sg.a) {
          if (ra.so != soa) continue;
          const SplitC& sa = getA(ra.blk);
          for (const BlockRef& rb : sg.b) {
            if (rb.so != sob) continue;
            const SplitC& sb = getB(rb.blk);
            // S_t = sum c_A c_B c_C[t] over all m, contracted m equal
            // (both entry lists are sorted by contracted m: merge equal runs)
            double S[kMaxTau] = {0};
            size_t i = 0, j = 0;
            while (i < sa.v.size() && j < sb.v.size()) {
              if (sa.kc[i] < sb.kc[j]) {
                ++i;
              } else if (sb.kc[j] < sa.kc[i]) {
                ++j;
              } else {
                const int64_t k = sa.kc[i];
                size_t j1 = j;
                while (j1 < sb.v.size() && sb.kc[j1] == k) ++j1;
                for (; i < sa.v.size() && sa.kc[i] == k; ++i)
                  for (size_t jj = j; jj < j1; ++jj) {
                    const int64_t ci = sa.oc[i] * nob_m + sb.oc[jj];
                    const double w = sa.v[i] * sb.v[jj];
                    for (int t = 0; t < ntau; ++t) S[t] += w * cC[t][ci];
                  }
                j = j1;
              }
            }
            bool any = false;
            for (int t = 0; t < ntau; ++t) {
              S[t] *= norm[t];
              any = any || std::fabs(S[t]) > 1e-13;
            }
            if (!any) continue;
            hc.push_back({sg.poff + ra.row0 * sg.N + rb.row0, sg.N});
            for (int t = 0; t < kMaxTau; ++t) hx.push_back(t < ntau ? S[t] : 0.0);
            p->rc_reads += double(M) * N;
          }
        }
      }
      g.ncontrib = int32_t(int64_t(hc.size()) - g.contrib0);
      const int gi = int(hg.size());
      hg.push_back(g);
      for (int64_t s = 0; s < M * N; s += kRcThreads) hch.push_back(make_int2(gi, int(s)));
    }
    b0 = b1;
  }
  p->nchunks = int(hch.size());

  // device side (a host-only context keeps the host plan only)
  if (ctx->device < 0) return plan.release();
  p->ra.upload(ta);
  p->rb.upload(tb);
  p->g.upload(p->probs, kF64TileM, kF64TileN);
  auto up = [](auto** dst, const auto& v) {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    if (v.empty()) return;
    BST_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    BST_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  };
  up(&p->d_groups, hg);
  up(&p->d_chunks, hch);
  up(&p->d_ct, hc);
  up(&p->d_x, hx);
  BST_CUDA(cudaMalloc(&p->Am, sizeof(double) * std::max<int64_t>(p->amat, 1)));
  BST_CUDA(cudaMalloc(&p->Bm, sizeof(double) * std::max<int64_t>(p->bmat, 1)));
  BST_CUDA(cudaMalloc(&p->P, sizeof(double) * std::max<int64_t>(p->pmat, 1)));
  return plan.release();
}

static std::string su2_key(Layout* A, Layout* B, const std::vector<int>& la, const std::vector<int>& lb) {
  std::string k = "su2/" + std::to_string(A->id) + "/" + std::to_string(B->id) + "/";
  for (int x : la) k += std::to_string(x) + ",";
  k += "/";
  for (int x : lb) k += std::to_string(x) + ",";
  return k;
}

static Su2Plan* get_su2_plan(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la,
                             const std::vector<int>& lb) {
  BST_REQUIRE(A->group == BST_SU2 && B->group == BST_SU2, BST_E_ARG, "both tensors must be SU(2) tensors");
  BST_REQUIRE(la.size() == lb.size(), BST_E_ARG, "leg pair lists differ in length");
  const std::string key = su2_key(A, B, la, lb);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->su2plans.find(key);
    if (it != ctx->su2plans.end()) return it->second.get();
  }
  std::shared_ptr<Su2Plan> p(build_su2_plan(ctx, A, B, la, lb));
  Su2Plan* raw = p.get();
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->su2plans[key] = std::move(p);
  return raw;
}

Layout* su2_contract_layout(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la, const std::vector<int>& lb) {
  return get_su2_plan(ctx, A, B, la, lb)->C;
}

void su2_contract(Ctx* ctx, Layout* A, const double* a, Layout* B, const double* b, const std::vector<int>& la,
                  const std::vector<int>& lb, bst_prec prec, double alpha, double beta, Layout* C, double* c,
                  cudaStream_t s) {
  BST_REQUIRE(ctx->device >= 0, BST_E_ARG, "host-only context (device -1) cannot run device work");
  Su2Plan* p = get_su2_plan(ctx, A, B, la, lb);
  BST_REQUIRE(p->C == C, BST_E_SHAPE, "C is not the layout of this contraction");
  BST_REQUIRE((A->nnz == 0 || a) && (B->nnz == 0 || b) && (C->nnz == 0 || c), BST_E_ARG, "data pointer is NULL");
  if (C->nnz == 0) return;
  launch_relayout(ctx, p->ra, a, p->Am, 0, 1.0, 0.0, s);
  launch_relayout(ctx, p->rb, b, p->Bm, 0, 1.0, 0.0, s);
  ctx->work_flops += p->g.flops;
  if (!p->probs.empty()) {
    if (prec == BST_FP64) {
      launch_gemm_f64(ctx, p->g, p->Am, p->Bm, p->P, s);
    } else {
      run_gemm_ozaki_probs(ctx, "su2/" + std::to_string(uintptr_t(p)), p->probs, p->Am, p->Bm, p->P, s, 0, true,
                           ozaki_slices(prec));
    }
  }
  if (p->nchunks) {
    ProfScope ps(ctx, s, "recouple", 0.0, 8.0 * (p->rc_reads + double(C->nnz) * (beta != 0.0 ? 2 : 1)));
    recouple_kernel<<<p->nchunks, kRcThreads, 0, s>>>(p->d_groups, p->d_chunks, p->d_ct, p->d_x, p->P, c, alpha,
                                                      beta);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  }
}

// ---------------------------------------------------------------------------
// Permutation with recoupling.  A block of S with sector tuple s and tree t
// is m_t (x) c_t; permuting the legs gives m_t^P (x) c_t^P, and c_t^P is a
// combination of the permuted layout's basis tensors of the same tuple,
//     c_t^P = sum_t' R[t', t] c'_t',  R[t', t] = <c'_t', c_t^P> / (2 J' + 1)
// (the bases are orthogonal with ||c||^2 = 2J+1), so the permuted tensor's
// reduced block t' is sum_t R[t', t] m_t^P.  R comes from the dense CGC
// tensors at plan time; the kernel forms every output element as that sum
// over the source trees of its tuple, each read through the permutation.

struct Su2PermTask {
  int64_t out_off;
  int32_t rank, n;
  int32_t shape[kMaxRank];  // output block extents (permuted leg order)
  int64_t istr[kMaxRank];   // stride in the source block of each output leg
  int64_t term0;
  int32_t nterm, pad;
};

struct Su2PermTerm {
  int64_t in_off;
  double coef;
};

struct Su2PermPlan {
  Layout* dst = nullptr;
  Su2PermTask* tasks = nullptr;
  Su2PermTerm* terms = nullptr;
  int2* chunks = nullptr;
  int ntasks = 0, nchunks = 0;
  double elems = 0;
  ~Su2PermPlan() {
    cudaFree(tasks);
    cudaFree(terms);
    cudaFree(chunks);
    if (dst) release(dst);
  }
};

constexpr int kPermChunk = 1024;
constexpr int kPermThreads = 256;

__global__ void __launch_bounds__(kPermThreads) su2_permute_kernel(const Su2PermTask* __restrict__ tasks,
                                                                   const Su2PermTerm* __restrict__ terms,
                                                                   const int2* __restrict__ chunks,
                                                                   const double* __restrict__ src,
                                                                   double* __restrict__ dst) {
  const int2 c = chunks[blockIdx.x];
  const Su2PermTask& t = tasks[c.x];
  FastDiv fd[kMaxRank];
#pragma unroll
  for (int i = 0; i < kMaxRank; ++i) fd[i].init(i < t.rank ? uint32_t(t.shape[i]) : 1u);
  const int end = min(t.n, c.y + kPermChunk);
  for (int e = c.y + int(threadIdx.x); e < end; e += kPermThreads) {
    uint32_t rem = uint32_t(e);
    long long o = 0;
#pragma unroll
    for (int i = kMaxRank - 1; i >= 0; --i) {
      if (i < t.rank) {
        const uint32_t q = fd[i].div(rem);
        o += (long long)(rem - q * fd[i].d) * t.istr[i];
        rem = q;
      }
    }
    double v = 0.0;
    for (int k = 0; k < t.nterm; ++k) {
      const Su2PermTerm tm = terms[t.term0 + k];
      v = fma(tm.coef, src[tm.in_off + o], v);
    }
    dst[t.out_off + e] = v;
  }
}

static Su2PermPlan* build_su2_perm(Ctx* ctx, Layout* S, const std::vector<int>& perm) {
  const int r = S->rank;
  std::vector<Leg> dl(r);
  for (int j = 0; j < r; ++j) dl[j] = S->legs[perm[j]];
  auto* P = new Su2PermPlan();
  P->dst = make_layout(ctx, BST_SU2, dl);
  Layout* D = P->dst;
  const std::vector<int> fs = flows_of(S), fd = flows_of(D);
  // R per source sector tuple: R[t' * nsrc + t] over its trees
  std::map<std::vector<int32_t>, std::vector<double>> rcache;
  std::vector<Su2PermTask> tasks;
  std::vector<Su2PermTerm> terms;
  std::vector<int32_t> ts(r);
  for (int64_t b = 0; b < D->nblocks; ++b) {
    const int32_t* sd = &D->sect[b * r];
    for (int j = 0; j < r; ++j) ts[perm[j]] = sd[j];
    const int64_t b0 = S->block_of(ts.data());
    BST_REQUIRE(b0 >= 0, BST_E_SHAPE, "SU(2) permute: source sector tuple missing");
    int64_t nsrc = 0;
    while (b0 + nsrc < S->nblocks && std::equal(ts.begin(), ts.end(), &S->sect[(b0 + nsrc) * r])) ++nsrc;
    // the destination trees of this tuple: consecutive blocks
    int64_t d0 = b;
    while (d0 > 0 && std::equal(sd, sd + r, &D->sect[(d0 - 1) * r])) --d0;
    int64_t ndst = 0;
    while (d0 + ndst < D->nblocks && std::equal(sd, sd + r, &D->sect[(d0 + ndst) * r])) ++ndst;
    auto it = rcache.find(ts);
    if (it == rcache.end()) {
      const std::vector<int> tjs = spins_of(S, b0), tjd = spins_of(D, d0);
      std::vector<std::vector<double>> cs(nsrc), cd(ndst);
      std::vector<int64_t> ext(r), sstr(r);
      for (int i = 0; i < r; ++i) ext[i] = tjs[i] + 1;
      int64_t st = 1;
      for (int i = r - 1; i >= 0; --i) sstr[i] = st, st *= ext[i];
      for (int64_t t = 0; t < nsrc; ++t) {
        const std::vector<double> c = basis_tensor(tjs, fs, &S->tree[(b0 + t) * S->ntree]);
        // permuted: element m' (dst order) = c at m_{perm[j]} = m'_j
        std::vector<double> cp(c.size());
        std::vector<int> idx(r, 0);
        for (size_t e = 0; e < cp.size(); ++e) {
          int64_t so = 0;
          for (int j = 0; j < r; ++j) so += idx[j] * sstr[perm[j]];
          cp[e] = c[so];
          for (int j = r - 1; j >= 0; --j) {
            if (++idx[j] < int(ext[perm[j]])) break;
            idx[j] = 0;
          }
        }
        cs[t] = std::move(cp);
      }
      for (int64_t t = 0; t < ndst; ++t) cd[t] = basis_tensor(tjd, fd, &D->tree[(d0 + t) * D->ntree]);
      int nin = 0;
      for (int f : fd) nin += f == 1;
      const int jpos = std::max(nin - 2, 0);
      std::vector<double> R(size_t(ndst * nsrc), 0.0);
      for (int64_t u = 0; u < ndst; ++u) {
        const double w = double(D->tree[(d0 + u) * D->ntree + jpos] + 1);
        for (int64_t t = 0; t < nsrc; ++t) {
          double dot = 0.0;
          for (size_t e = 0; e < cd[u].size(); ++e) dot += cd[u][e] * cs[t][e];
          R[size_t(u * nsrc + t)] = dot / w;
        }
      }
      it = rcache.emplace(ts, std::move(R)).first;
    }
    const std::vector<double>& R = it->second;
    Su2PermTask tk{};
    tk.out_off = D->offset[b];
    tk.rank = r;
    int64_t n = 1;
    std::vector<int64_t> bstr(r);
    int64_t st = 1;
    for (int i = r - 1; i >= 0; --i) bstr[i] = st, st *= S->shape[b0 * r + i];
    for (int j = 0; j < r; ++j) {
      tk.shape[j] = int32_t(D->shape[b * r + j]);
      tk.istr[j] = bstr[perm[j]];
      n *= tk.shape[j];
    }
    tk.n = int32_t(n);
    tk.term0 = int64_t(terms.size());
    for (int64_t t = 0; t < nsrc; ++t) {
      const double c = R[size_t((b - d0) * nsrc + t)];
      if (std::fabs(c) > 1e-14) terms.push_back({S->offset[b0 + t], c});
    }
    tk.nterm = int32_t(int64_t(terms.size()) - tk.term0);
    if (n > 0) tasks.push_back(tk);
  }
  std::vector<int2> ch;
  for (int i = 0; i < int(tasks.size()); ++i) {
    P->elems += tasks[i].n;
    for (int e = 0; e < tasks[i].n; e += kPermChunk) ch.push_back(make_int2(i, e));
  }
  P->ntasks = int(tasks.size());
  P->nchunks = int(ch.size());
  auto up = [](auto** dst, const auto& v) {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    if (v.empty()) return;
    BST_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
    BST_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  };
  up(&P->tasks, tasks);
  up(&P->terms, terms);
  up(&P->chunks, ch);
  return P;
}

Layout* su2_permute(Ctx* ctx, Layout* S, const double* src, const std::vector<int>& perm, double* dst,
                    cudaStream_t s) {
  BST_REQUIRE(S->group == BST_SU2, BST_E_ARG, "su2_permute: not an SU(2) layout");
  BST_REQUIRE(int(perm.size()) == S->rank, BST_E_ARG, "perm must list every leg");
  std::vector<bool> seen(S->rank, false);
  for (int x : perm) {
    BST_REQUIRE(x >= 0 && x < S->rank && !seen[x], BST_E_ARG, "perm is not a permutation");
    seen[x] = true;
  }
  std::string key = "su2perm/" + std::to_string(S->id) + "/";
  for (int x : perm) key += std::to_string(x) + ",";
  Su2PermPlan* P = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->su2perm.find(key);
    if (it != ctx->su2perm.end()) P = it->second.get();
  }
  if (!P) {
    std::shared_ptr<Su2PermPlan> np(build_su2_perm(ctx, S, perm));
    P = np.get();
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->su2perm[key] = std::move(np);
  }
  if (P->nchunks > 0) {
    BST_REQUIRE(src && dst, BST_E_ARG, "data pointer is NULL");
    ProfScope ps(ctx, s, "relayout", 0.0, 16.0 * P->elems);
    su2_permute_kernel<<<P->nchunks, kPermThreads, 0, s>>>(P->tasks, P->terms, P->chunks, src, dst);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  }
  return P->dst;
}

}  // namespace bst
