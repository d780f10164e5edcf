// Sector matching on the device (Sec. 2: block pairs are matched by the
// charges on the contracted legs, then reduced by the output charges).
//
// For a layout and a split of its legs into row legs and column legs, one
// CTA builds what the host planner's make_matview builds:
//   * every configuration of the row legs (a tuple of sector indices, in
//     lexicographic order) with its charge sum_i flow_i q_i and its extent,
//     and its offset among the configurations of the same charge; the same
//     for the column legs;
//   * the sector keys (charge through the column legs) that some block
//     carries, ascending, with their row and column totals and the element
//     offset of each sector matrix;
//   * one relayout task per block: its place in its sector matrix and the
//     strides of its legs there;
//   * the chunk table of the relayout launch (kChunkElems elements per CTA).
// Charges are reduced by the group's rule (U(1): themselves; Z2: parity),
// and every charge sum lies in a range known from the legs, so tables are
// indexed by charge directly: no sort.  A second kernel matches the sectors
// of A, B and C into the grouped GEMM's problem list.
#include <algorithm>

#include "bst_internal.h"

namespace bst {

constexpr int kPlanThreads = 1024;
constexpr int kChunkElems = 2048;  // elements per relayout CTA (relayout.cu)

struct DevLegs {
  int rank, group;
  int flow[kMaxRank], nsect[kMaxRank], qoff[kMaxRank];
};

struct ViewSpec {
  int nrow, ncol;
  int rowlegs[kMaxRank], collegs[kMaxRank];
  long long trow, tcol;           // configurations of the row / column legs
  long long rlo, rn, clo, cn;     // charge range of row / column sums (lowest, count)
};

struct DevSector {
  long long key, rows, cols, off;
};

__device__ __forceinline__ long long dnorm(int group, long long q) { return group == BST_Z2 ? (q & 1) : q; }

// Sector index of configuration t over the listed legs (leg 0 most
// significant), its charge sum and extent.
__device__ void decode_cfg(const DevLegs& L, const int* __restrict__ q, const long long* __restrict__ d,
                           const int* legs, int nleg, long long t, long long* charge, long long* ext) {
  long long c = 0, e = 1;
  for (int j = nleg - 1; j >= 0; --j) {
    const int i = legs[j];
    const int ns = L.nsect[i];
    const int s = int(t % ns);
    t /= ns;
    c += (long long)L.flow[i] * q[L.qoff[i] + s];
    e *= d[L.qoff[i] + s];
  }
  *charge = dnorm(L.group, c);
  *ext = e;
}

// One CTA.  Scratch (global): per row configuration charge, extent and
// offset; the same per column configuration; per row / column charge value
// the total extent; per column charge value the sector index (-1: no block).
__global__ void __launch_bounds__(kPlanThreads) plan_view_kernel(
    const DevLegs L, const ViewSpec V, const int* __restrict__ q, const long long* __restrict__ d,
    const int* __restrict__ sect, const long long* __restrict__ boff, int nblocks, long long* rch, long long* rext,
    long long* roff, long long* cch, long long* cext, long long* coff, long long* rtot, long long* ctot, int* secidx,
    DevSector* secs, int* nsec_out, RelTask* tasks, int2* chunks, int* nchunks_out) {
  const int tid = threadIdx.x;
  __shared__ int nsec;
  __shared__ long long sec_sum;
  // configurations: charge and extent
  for (long long t = tid; t < V.trow; t += kPlanThreads) decode_cfg(L, q, d, V.rowlegs, V.nrow, t, &rch[t], &rext[t]);
  for (long long t = tid; t < V.tcol; t += kPlanThreads) decode_cfg(L, q, d, V.collegs, V.ncol, t, &cch[t], &cext[t]);
  for (long long c = tid; c < V.cn; c += kPlanThreads) secidx[c] = -1;
  __syncthreads();
  // offsets inside each charge: one thread per charge value walks the
  // configurations in lexicographic order
  for (long long c = tid; c < V.rn; c += kPlanThreads) {
    long long acc = 0;
    for (long long t = 0; t < V.trow; ++t)
      if (rch[t] - V.rlo == c) {
        roff[t] = acc;
        acc += rext[t];
      }
    rtot[c] = acc;
  }
  for (long long c = tid; c < V.cn; c += kPlanThreads) {
    long long acc = 0;
    for (long long t = 0; t < V.tcol; ++t)
      if (cch[t] - V.clo == c) {
        coff[t] = acc;
        acc += cext[t];
      }
    ctot[c] = acc;
  }
  // sector keys carried by some block (charge through the column legs)
  for (int b = tid; b < nblocks; b += kPlanThreads) {
    long long k = 0;
    for (int j = 0; j < V.ncol; ++j) {
      const int i = V.collegs[j];
      k += (long long)L.flow[i] * q[L.qoff[i] + sect[(long long)b * L.rank + i]];
    }
    secidx[dnorm(L.group, k) - V.clo] = 0;  // present
  }
  __syncthreads();
  // sectors in ascending key order, their sizes and matrix offsets
  if (tid == 0) {
    int n = 0;
    long long off = 0;
    for (long long c = 0; c < V.cn; ++c) {
      if (secidx[c] < 0) continue;
      const long long key = c + V.clo;
      const long long rc = dnorm(L.group, -key) - V.rlo;
      const long long rows = (rc >= 0 && rc < V.rn) ? rtot[rc] : 0;
      DevSector s{key, rows, ctot[c], off};
      secs[n] = s;
      secidx[c] = n++;
      off += rows * ctot[c];
    }
    nsec = n;
    sec_sum = off;
    *nsec_out = n;
  }
  __syncthreads();
  // one task per block
  for (int b = tid; b < nblocks; b += kPlanThreads) {
    const int* sb = sect + (long long)b * L.rank;
    long long tr = 0, tc = 0, k = 0;
    for (int j = 0; j < V.nrow; ++j) tr = tr * L.nsect[V.rowlegs[j]] + sb[V.rowlegs[j]];
    for (int j = 0; j < V.ncol; ++j) {
      const int i = V.collegs[j];
      tc = tc * L.nsect[i] + sb[i];
      k += (long long)L.flow[i] * q[L.qoff[i] + sb[i]];
    }
    const DevSector s = secs[secidx[dnorm(L.group, k) - V.clo]];
    RelTask t;
    for (int i = 0; i < kMaxRank; ++i) {
      t.shape[i] = 0;
      t.mstride[i] = 0;
    }
    t.blk_off = boff[b];
    t.mat_base = s.off + roff[tr] * s.cols + coff[tc];
    t.rank = L.rank;
    long long n = 1;
    for (int i = 0; i < L.rank; ++i) {
      t.shape[i] = int(d[L.qoff[i] + sb[i]]);
      n *= t.shape[i];
    }
    t.n = int(n);
    long long st = s.cols;
    for (int j = V.nrow - 1; j >= 0; --j) {
      t.mstride[V.rowlegs[j]] = st;
      st *= t.shape[V.rowlegs[j]];
    }
    st = 1;
    for (int j = V.ncol - 1; j >= 0; --j) {
      t.mstride[V.collegs[j]] = st;
      st *= t.shape[V.collegs[j]];
    }
    tasks[b] = t;
  }
  __syncthreads();
  // chunk table: blocks in order, kChunkElems elements per chunk
  if (tid == 0) {
    int nc = 0;
    for (int b = 0; b < nblocks; ++b)
      for (int e = 0; e < tasks[b].n; e += kChunkElems) chunks[nc++] = make_int2(b, e);
    *nchunks_out = nc;
  }
}

// Problem list of a contraction: one GEMM per sector of C; A's sector with
// the same key and B's with the opposite charge (Z2: the same parity).
__global__ void match_sectors_kernel(const DevSector* __restrict__ sa, int na, const DevSector* __restrict__ sb,
                                     int nb, const DevSector* __restrict__ sc, int nc, int group,
                                     GemmProb* __restrict__ probs, int* nprobs) {
  if (threadIdx.x != 0) return;
  int n = 0;
  for (int i = 0; i < nc; ++i) {
    const DevSector c = sc[i];
    const long long kb = dnorm(group, -c.key);
    int ia = -1, ib = -1;
    for (int j = 0; j < na; ++j)
      if (sa[j].key == c.key) ia = j;
    for (int j = 0; j < nb; ++j)
      if (sb[j].key == kb) ib = j;
    GemmProb g{};
    g.M = int(c.rows);
    g.N = int(c.cols);
    g.K = (ia >= 0 && ib >= 0) ? int(sa[ia].cols) : 0;
    g.a_off = ia >= 0 ? sa[ia].off : 0;
    g.b_off = ib >= 0 ? sb[ib].off : 0;
    g.c_off = c.off;
    g.a_m = g.K;
    g.a_k = 1;
    g.b_n = g.K;
    g.b_k = 1;
    g.c_m = c.cols;
    g.c_n = 1;
    if (g.M > 0 && g.N > 0) probs[n++] = g;
  }
  *nprobs = n;
}

namespace {

struct DevLayoutTables {
  int* q = nullptr;
  long long* d = nullptr;
  int* sect = nullptr;
  long long* off = nullptr;
  ~DevLayoutTables() {
    cudaFree(q);
    cudaFree(d);
    cudaFree(sect);
    cudaFree(off);
  }
};

template <class T>
T* upload_vec(const std::vector<T>& v) {
  T* p = nullptr;
  BST_CUDA(cudaMalloc(&p, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!v.empty()) BST_CUDA(cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return p;
}

// charge range of flow-signed sums over the listed legs
void charge_range(const Layout* L, const std::vector<int>& legs, long long* lo, long long* n) {
  if (L->group == BST_Z2) {
    *lo = 0;
    *n = 2;
    return;
  }
  long long a = 0, b = 0;
  for (int i : legs) {
    const long long x = (long long)L->legs[i].flow * L->legs[i].q.front();
    const long long y = (long long)L->legs[i].flow * L->legs[i].q.back();
    a += std::min(x, y);
    b += std::max(x, y);
  }
  *lo = a;
  *n = b - a + 1;
}

}  // namespace

// Device-built view of L for (rowlegs, collegs): relayout tasks and chunk
// table (in r, device-owned), sector table (device) and its size.
struct DevView {
  DevRelayout rel;
  DevSector* secs = nullptr;
  int nsec = 0;
  ~DevView() {
    rel.free_all();
    cudaFree(secs);
  }
};

static void build_view(Ctx* ctx, const Layout* L, const std::vector<int>& rowlegs, const std::vector<int>& collegs,
                       DevView* out, cudaStream_t s) {
  BST_REQUIRE(is_abelian(L->group), BST_E_UNSUPPORTED, "device planner: U(1) and Z2 layouts only");
  DevLegs dl{};
  dl.rank = L->rank;
  dl.group = L->group;
  std::vector<int> q;
  std::vector<long long> d;
  for (int i = 0; i < L->rank; ++i) {
    dl.flow[i] = L->legs[i].flow;
    dl.nsect[i] = int(L->legs[i].q.size());
    dl.qoff[i] = int(q.size());
    for (size_t k = 0; k < L->legs[i].q.size(); ++k) {
      q.push_back(L->legs[i].q[k]);
      d.push_back(L->legs[i].d[k]);
    }
  }
  ViewSpec v{};
  v.nrow = int(rowlegs.size());
  v.ncol = int(collegs.size());
  v.trow = v.tcol = 1;
  for (int j = 0; j < v.nrow; ++j) v.rowlegs[j] = rowlegs[j], v.trow *= dl.nsect[rowlegs[j]];
  for (int j = 0; j < v.ncol; ++j) v.collegs[j] = collegs[j], v.tcol *= dl.nsect[collegs[j]];
  charge_range(L, rowlegs, &v.rlo, &v.rn);
  charge_range(L, collegs, &v.clo, &v.cn);
  BST_REQUIRE(v.trow < (1ll << 24) && v.tcol < (1ll << 24) && v.rn < (1ll << 22) && v.cn < (1ll << 22),
              BST_E_UNSUPPORTED, "device planner: too many leg configurations");
  DevLayoutTables t;
  t.q = upload_vec(q);
  t.d = upload_vec(d);
  t.sect = upload_vec(L->sect);
  std::vector<long long> offs(L->offset.begin(), L->offset.end());
  t.off = upload_vec(offs);
  const long long nb = L->nblocks;
  long long nchunk_max = 0;
  for (int64_t b = 0; b < nb; ++b) {
    int64_t n = 1;
    for (int i = 0; i < L->rank; ++i) n *= L->shape[b * L->rank + i];
    nchunk_max += (n + kChunkElems - 1) / kChunkElems;
  }
  // scratch: 3 x trow + 3 x tcol + rn + cn long longs, cn ints
  const size_t nll = size_t(3 * v.trow + 3 * v.tcol + v.rn + v.cn);
  char* ws = (char*)ctx->buf("plan.dev.ws", sizeof(long long) * nll + sizeof(int) * (v.cn + 4), s);
  long long* p = reinterpret_cast<long long*>(ws);
  long long *rch = p, *rext = rch + v.trow, *roff = rext + v.trow;
  long long *cch = roff + v.trow, *cext = cch + v.tcol, *coff = cext + v.tcol;
  long long *rtot = coff + v.tcol, *ctot = rtot + v.rn;
  int* secidx = reinterpret_cast<int*>(ctot + v.cn);
  int* counts = secidx + v.cn;  // nsec, nchunks
  BST_CUDA(cudaMalloc(&out->secs, sizeof(DevSector) * std::max<long long>(v.cn, 1)));
  BST_CUDA(cudaMalloc(&out->rel.tasks, sizeof(RelTask) * std::max<long long>(nb, 1)));
  BST_CUDA(cudaMalloc(&out->rel.chunks, sizeof(int2) * std::max<long long>(nchunk_max, 1)));
  plan_view_kernel<<<1, kPlanThreads, 0, s>>>(dl, v, t.q, t.d, t.sect, t.off, int(nb), rch, rext, roff, cch, cext,
                                              coff, rtot, ctot, secidx, out->secs, counts, out->rel.tasks,
                                              out->rel.chunks, counts + 1);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
  int hc[2] = {0, 0};
  BST_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));  // the tables above are freed on return
  out->nsec = hc[0];
  out->rel.ntasks = int(nb);
  out->rel.nchunks = hc[1];
  double e = 0;
  for (int64_t b = 0; b < nb; ++b) {
    int64_t n = 1;
    for (int i = 0; i < L->rank; ++i) n *= L->shape[b * L->rank + i];
    e += double(n);
  }
  out->rel.elems = e;
}

// The relayout task lists of a contraction plan, built on the device: A and
// B into their sector matrices, C's sector matrix into C.
void plan_relayouts_on_device(Ctx* ctx, ContractPlan* p, const std::vector<int>& oa, const std::vector<int>& la,
                              const std::vector<int>& ob, const std::vector<int>& lb, cudaStream_t s) {
  std::vector<int> crow, ccol;
  for (size_t i = 0; i < oa.size(); ++i) crow.push_back(int(i));
  for (size_t i = 0; i < ob.size(); ++i) ccol.push_back(int(oa.size() + i));
  DevView va, vb, vc;
  build_view(ctx, p->A, oa, la, &va, s);
  build_view(ctx, p->B, ob, lb, &vb, s);
  build_view(ctx, p->C, crow, ccol, &vc, s);
  for (DevView* v : {&va, &vb, &vc}) BST_REQUIRE(v->rel.ntasks >= 0, BST_E_CUDA, "device planner failed");
  p->ra = va.rel;
  p->rb = vb.rel;
  p->rc = vc.rel;
  va.rel = vb.rel = vc.rel = DevRelayout{};  // ownership moved to the plan
}

// Self-check: the device-built tables of contract(A, B) against the host
// planner's, entry by entry.  Returns the number of entries that differ
// (tasks, chunks, sectors and problems of the three views).
int64_t plan_check(Ctx* ctx, Layout* A, Layout* B, const std::vector<int>& la, const std::vector<int>& lb,
                   cudaStream_t s) {
  ContractPlan* hp = get_contract_plan(ctx, A, B, la, lb);
  std::vector<int> oa, ob;
  std::vector<bool> ua(A->rank, false), ub(B->rank, false);
  for (int i : la) ua[i] = true;
  for (int i : lb) ub[i] = true;
  for (int i = 0; i < A->rank; ++i)
    if (!ua[i]) oa.push_back(i);
  for (int i = 0; i < B->rank; ++i)
    if (!ub[i]) ob.push_back(i);
  std::vector<int> crow, ccol;
  for (size_t i = 0; i < oa.size(); ++i) crow.push_back(int(i));
  for (size_t i = 0; i < ob.size(); ++i) ccol.push_back(int(oa.size() + i));
  const MatView* hv[3] = {&hp->va, &hp->vb, &hp->vc};
  DevView dv[3];
  build_view(ctx, A, oa, la, &dv[0], s);
  build_view(ctx, B, ob, lb, &dv[1], s);
  build_view(ctx, hp->C, crow, ccol, &dv[2], s);
  int64_t bad = 0;
  auto same_task = [](const RelTask& x, const RelTask& y) {
    if (x.blk_off != y.blk_off || x.mat_base != y.mat_base || x.rank != y.rank || x.n != y.n) return false;
    for (int i = 0; i < x.rank; ++i)
      if (x.shape[i] != y.shape[i] || x.mstride[i] != y.mstride[i]) return false;
    return true;
  };
  for (int v = 0; v < 3; ++v) {
    std::vector<RelTask> dt(dv[v].rel.ntasks);
    std::vector<int2> dc(dv[v].rel.nchunks);
    std::vector<DevSector> ds(dv[v].nsec);
    if (!dt.empty())
      BST_CUDA(cudaMemcpy(dt.data(), dv[v].rel.tasks, sizeof(RelTask) * dt.size(), cudaMemcpyDeviceToHost));
    if (!dc.empty())
      BST_CUDA(cudaMemcpy(dc.data(), dv[v].rel.chunks, sizeof(int2) * dc.size(), cudaMemcpyDeviceToHost));
    if (!ds.empty())
      BST_CUDA(cudaMemcpy(ds.data(), dv[v].secs, sizeof(DevSector) * ds.size(), cudaMemcpyDeviceToHost));
    const std::vector<RelTask>& ht = hv[v]->tasks;
    const std::vector<int2> hc = relayout_chunks(ht);
    bad += std::abs(int64_t(ht.size()) - int64_t(dt.size()));
    for (size_t i = 0; i < std::min(ht.size(), dt.size()); ++i) bad += !same_task(ht[i], dt[i]);
    bad += std::abs(int64_t(hc.size()) - int64_t(dc.size()));
    for (size_t i = 0; i < std::min(hc.size(), dc.size()); ++i) bad += hc[i].x != dc[i].x || hc[i].y != dc[i].y;
    const auto& hs = hv[v]->secs;
    bad += std::abs(int64_t(hs.size()) - int64_t(ds.size()));
    for (size_t i = 0; i < std::min(hs.size(), ds.size()); ++i)
      bad += hs[i].key != ds[i].key || hs[i].rows != ds[i].rows || hs[i].cols != ds[i].cols || hs[i].off != ds[i].off;
  }
  // problem list
  GemmProb* dp = nullptr;
  int* dn = nullptr;
  BST_CUDA(cudaMalloc(&dp, sizeof(GemmProb) * std::max(dv[2].nsec, 1)));
  BST_CUDA(cudaMalloc(&dn, sizeof(int)));
  match_sectors_kernel<<<1, 32, 0, s>>>(dv[0].secs, dv[0].nsec, dv[1].secs, dv[1].nsec, dv[2].secs, dv[2].nsec,
                                        A->group, dp, dn);
  BST_CUDA(cudaGetLastError());
  count_launch(ctx);
  int n = 0;
  BST_CUDA(cudaMemcpyAsync(&n, dn, sizeof(int), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  std::vector<GemmProb> gp(n);
  if (n) BST_CUDA(cudaMemcpy(gp.data(), dp, sizeof(GemmProb) * n, cudaMemcpyDeviceToHost));
  cudaFree(dp);
  cudaFree(dn);
  bad += std::abs(int64_t(n) - int64_t(hp->probs.size()));
  for (size_t i = 0; i < std::min(size_t(n), hp->probs.size()); ++i) {
    const GemmProb &x = gp[i], &y = hp->probs[i];
    bad += x.M != y.M || x.N != y.N || x.K != y.K || x.a_off != y.a_off || x.b_off != y.b_off ||
           x.c_off != y.c_off || x.a_m != y.a_m || x.a_k != y.a_k || x.b_n != y.b_n || x.b_k != y.b_k ||
           x.c_m != y.c_m || x.c_n != y.c_n;
  }
  return bad;
}

}  // namespace bst
