// SVD projectors of the CTMRG move (Sec. 3: the corner transfer matrix is
// truncated as in corboz14).
//
// N = Rtop^T Rbot over the left cut is block diagonal in the charge through
// the right cut.  Each sector is decomposed with an FP64 SVD on the GPU
// (cuSOLVER gesvd), the chi largest singular values over all sectors are
// kept (a host decision: one stream synchronisation), and
//     P  = Rbot V S^-1/2,      Pt = S^-1/2 U^T Rtop^T
// are formed per sector with the grouped GEMM, then scattered into their
// canonical block layouts.  The sign of every kept left singular vector is
// fixed by making its largest-magnitude entry positive (lowest index on
// ties); the right vector follows.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "bst_internal.h"

namespace bst {

void launch_transpose(const double* A, double* Y, int M, int N, cudaStream_t s);

#define BST_CUSOLVER(call)                                                                 \
  do {                                                                                     \
    cusolverStatus_t st_ = (call);                                                         \
    if (st_ != CUSOLVER_STATUS_SUCCESS)                                                    \
      throw ::bst::Error(BST_E_CUDA, std::string(#call) + " failed: " + std::to_string(int(st_))); \
  } while (0)

// Gauge and scale: for kept vector j, u_j = column j of the left factor
// (element i at U[i*us_i + j*us_j]); sign from the largest |u_j(i)| (lowest i
// on ties); writes Uo[i*m + j] = sign*u/sqrt(s_j) (row-major [m x k]) and
// Vo[i*k + j] = sign*v/sqrt(s_j) (row-major [n x k]).
__global__ void gauge_scale_kernel(const double* U, long long us_i, long long us_j, int m,
                                   const double* V, long long vs_i, long long vs_j, int n,
                                   const double* S, int k, double* Uo, double* Vo) {
  const int j = blockIdx.x;
  if (j >= k) return;
  __shared__ double sv[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double a = fabs(U[i * us_i + j * us_j]);
    if (a > best || (a == best && i < bi)) {
      best = a;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double a = sv[threadIdx.x + w];
      int ai = si[threadIdx.x + w];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && ai < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const double sgn = (U[(long long)si[0] * us_i + j * us_j] < 0) ? -1.0 : 1.0;
  const double f = sgn / sqrt(S[j]);
  for (int i = threadIdx.x; i < m; i += blockDim.x) Uo[(long long)i * k + j] = f * U[i * us_i + j * us_j];
  for (int i = threadIdx.x; i < n; i += blockDim.x) Vo[(long long)i * k + j] = f * V[i * vs_i + j * vs_j];
}

// Views and scatter plans of a projector layout, cached by layout.
struct ProjView {
  MatView mv;
  DevRelayout rel;
};

static ProjView* get_projview(Ctx* ctx, Layout* L, const std::vector<int>& rows, const std::vector<int>& cols) {
  static std::mutex mu;
  static std::map<std::string, std::unique_ptr<ProjView>> cache;  // keyed by ctx+layout
  std::string key = std::to_string((uintptr_t)ctx) + "/" + std::to_string(L->id);
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second.get();
  auto pv = std::make_unique<ProjView>();
  pv->mv = make_matview(L, rows, cols);
  pv->rel.upload(pv->mv.tasks);
  ProjView* raw = pv.get();
  cache[key] = std::move(pv);
  return raw;
}

ProjResult svd_projector(Ctx* ctx, Layout* Rt, const double* rt, Layout* Rb, const double* rb, int ncut,
                         int64_t chi, double rel_cutoff, int new_flow, bst_prec prec, double* p, double* pt,
                         cudaStream_t s) {
  BST_REQUIRE(ncut >= 1 && ncut < Rt->rank && ncut < Rb->rank, BST_E_ARG, "bad ncut");
  BST_REQUIRE(chi >= 1, BST_E_ARG, "chi must be positive");
  BST_REQUIRE(new_flow == 1 || new_flow == -1, BST_E_ARG, "new_flow must be +1 or -1");
  if (!ctx->cusolver) {
    cusolverDnHandle_t h;
    BST_CUSOLVER(cusolverDnCreate(&h));
    ctx->cusolver = h;
  }
  cusolverDnHandle_t h = (cusolverDnHandle_t)ctx->cusolver;
  BST_CUSOLVER(cusolverDnSetStream(h, s));

  std::vector<int> cut(ncut);
  std::iota(cut.begin(), cut.end(), 0);
  ContractPlan* pn = get_contract_plan(ctx, Rt, Rb, cut, cut);
  double* Nm = nullptr;
  // N = Rt^T Rb as sector matrices (rows: right cut of Rt, cols: right cut of Rb)
  run_contract(ctx, pn, rt, rb, prec, 1.0, 0.0, nullptr, s, /*scatter=*/false, &Nm);
  const double* Am = (const double*)ctx->bufs["contract.A"].p;  // Rt as [beta x alpha]
  const double* Bm = (const double*)ctx->bufs["contract.B"].p;  // Rb as [beta' x alpha']
  // copy A/B sector matrices: later GEMMs reuse the contract buffers
  double* At = (double*)ctx->buf("proj.A", sizeof(double) * std::max<int64_t>(pn->amat, 1), s);
  double* Bt = (double*)ctx->buf("proj.B", sizeof(double) * std::max<int64_t>(pn->bmat, 1), s);
  BST_CUDA(cudaMemcpyAsync(At, Am, sizeof(double) * pn->amat, cudaMemcpyDeviceToDevice, s));
  BST_CUDA(cudaMemcpyAsync(Bt, Bm, sizeof(double) * pn->bmat, cudaMemcpyDeviceToDevice, s));

  struct Sec {
    const MatSector* cs;
    const MatSector* as;
    const MatSector* bs;
    int M, N, mn;
    bool trans;  // decompose N^T (col-major view of the row-major matrix)
    int64_t s_off, u_off, v_off;
  };
  std::vector<Sec> secs;
  int64_t stot = 0, utot = 0, vtot = 0;
  int lwork = 0;
  for (auto& cs : pn->vc.secs) {
    const MatSector* as = pn->va.find(cs.key);
    const MatSector* bs = pn->vb.find(-cs.key);
    if (!as || !bs || as->cols == 0 || cs.rows == 0 || cs.cols == 0) continue;
    Sec x{&cs, as, bs, int(cs.rows), int(cs.cols), int(std::min(cs.rows, cs.cols)), cs.cols >= cs.rows, 0, 0, 0};
    x.s_off = stot;
    stot += x.mn;
    x.u_off = utot;
    utot += int64_t(std::max(x.M, x.N)) * x.mn;
    x.v_off = vtot;
    vtot += int64_t(x.mn) * x.mn;
    int m = x.trans ? x.N : x.M, n = x.trans ? x.M : x.N, lw = 0;
    BST_CUSOLVER(cusolverDnDgesvd_bufferSize(h, m, n, &lw));
    lwork = std::max(lwork, lw);
    secs.push_back(x);
  }
  BST_REQUIRE(!secs.empty(), BST_E_NUMERIC, "projector: no non-empty sector");
  double* dS = (double*)ctx->buf("proj.S", sizeof(double) * stot, s);
  double* dU = (double*)ctx->buf("proj.U", sizeof(double) * utot, s);
  double* dV = (double*)ctx->buf("proj.V", sizeof(double) * vtot, s);
  double* dW = (double*)ctx->buf("proj.work", sizeof(double) * std::max(lwork, 1), s);
  int maxmn = 1;
  for (auto& x : secs) maxmn = std::max(maxmn, x.mn);
  double* dR = (double*)ctx->buf("proj.rwork", sizeof(double) * maxmn, s);
  double* dX = (double*)ctx->buf("proj.X", sizeof(double) * std::max<int64_t>(pn->cmat, 1), s);
  int* dInfo = (int*)ctx->buf("proj.info", sizeof(int) * secs.size(), s);
  BST_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int) * secs.size(), s));
  {
  ProfScope ps_svd(ctx, s, "svd_cusolver", 0.0, 0.0);
  for (size_t i = 0; i < secs.size(); ++i) {
    Sec& x = secs[i];
    double* A = Nm + x.cs->off;
    if (x.trans) {
      // row-major N_s [M x N] is col-major X = N_s^T [N x M], N >= M
      BST_CUSOLVER(cusolverDnDgesvd(h, 'S', 'S', x.N, x.M, A, x.N, dS + x.s_off, dU + x.u_off, x.N,
                                    dV + x.v_off, x.mn, dW, lwork, dR, dInfo + i));
    } else {
      // need rows >= cols: transpose into col-major Y = N_s [M x N]
      double* Y = dX + x.cs->off;
      // transpose: Y[i + j*M] = A[i*N + j]
      launch_transpose(A, Y, x.M, x.N, s);
      count_launch(ctx);
      BST_CUSOLVER(cusolverDnDgesvd(h, 'S', 'S', x.M, x.N, Y, x.M, dS + x.s_off, dU + x.u_off, x.M,
                                    dV + x.v_off, x.mn, dW, lwork, dR, dInfo + i));
    }
    count_launch(ctx);
  }
  }
  std::vector<double> hS(stot);
  std::vector<int> hInfo(secs.size());
  BST_CUDA(cudaMemcpyAsync(hS.data(), dS, sizeof(double) * stot, cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaMemcpyAsync(hInfo.data(), dInfo, sizeof(int) * secs.size(), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  for (int v : hInfo) BST_REQUIRE(v == 0, BST_E_NUMERIC, "projector: gesvd did not converge");

  // global truncation: sigma descending, |q| ascending, q ascending
  struct Cand { double sv; int q; int sec; int j; };
  std::vector<Cand> cand;
  double smax = 0, ssum = 0;
  for (size_t i = 0; i < secs.size(); ++i)
    for (int j = 0; j < secs[i].mn; ++j) {
      double v = hS[secs[i].s_off + j];
      BST_REQUIRE(std::isfinite(v), BST_E_NUMERIC, "projector: non-finite singular value");
      cand.push_back({v, int(new_flow * secs[i].cs->key), int(i), j});
      smax = std::max(smax, v);
      ssum += v;
    }
  std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    if (a.sv != b.sv) return a.sv > b.sv;
    if (std::abs(a.q) != std::abs(b.q)) return std::abs(a.q) < std::abs(b.q);
    if (a.q != b.q) return a.q < b.q;
    return a.j < b.j;
  });
  std::vector<int> kcount(secs.size(), 0);
  int64_t kept = 0;
  double kept_sum = 0, kmin = smax;
  for (auto& c : cand) {
    if (kept >= chi) break;
    if (!(c.sv > rel_cutoff * smax) || c.sv <= 0) break;
    // singular values of one sector come sorted, so the kept ones of a
    // sector are its leading ones
    kcount[c.sec]++;
    kept++;
    kept_sum += c.sv;
    kmin = std::min(kmin, c.sv);
  }
  BST_REQUIRE(kept > 0, BST_E_NUMERIC, "projector: nothing above the cutoff");
  for (size_t i = 0; i < secs.size(); ++i)
    for (int j = 0; j < kcount[i]; ++j)
      BST_REQUIRE(hS[secs[i].s_off + j] >= hS[secs[i].s_off + kcount[i] - 1], BST_E_NUMERIC, "projector: unsorted");

  // new leg: ascending charge
  std::vector<std::pair<int, int>> order;  // (charge, sec)
  for (size_t i = 0; i < secs.size(); ++i)
    if (kcount[i] > 0) order.push_back({int(new_flow * secs[i].cs->key), int(i)});
  std::sort(order.begin(), order.end());
  Leg nl;
  nl.flow = new_flow;
  ProjResult res;
  for (auto& o : order) {
    nl.q.push_back(o.first);
    nl.d.push_back(kcount[o.second]);
    for (int j = 0; j < kcount[o.second]; ++j) res.svals.push_back(hS[secs[o.second].s_off + j]);
  }
  nl.finish();
  res.newleg = nl;
  res.kept = kept;
  res.smin_over_smax = kmin / smax;
  res.trunc_weight = ssum > 0 ? (ssum - kept_sum) / ssum : 0;
  std::vector<Leg> pl(Rb->legs.begin(), Rb->legs.begin() + ncut);
  pl.push_back(nl);
  std::vector<Leg> ptl{nl.dual()};
  ptl.insert(ptl.end(), Rt->legs.begin(), Rt->legs.begin() + ncut);
  res.P = make_layout(ctx, Rb->group, pl);
  res.Pt = make_layout(ctx, Rt->group, ptl);
  std::vector<int> prow(ncut), pcol{ncut}, ptrow{0}, ptcol(ncut);
  std::iota(prow.begin(), prow.end(), 0);
  std::iota(ptcol.begin(), ptcol.end(), 1);
  ProjView* vp = get_projview(ctx, res.P, prow, pcol);
  ProjView* vpt = get_projview(ctx, res.Pt, ptrow, ptcol);

  // gauge-fixed, S^-1/2-scaled factors, then P and Pt sector GEMMs
  int64_t us_tot = 0, vs_tot = 0;
  for (size_t i = 0; i < secs.size(); ++i) {
    us_tot += int64_t(secs[i].M) * kcount[i];
    vs_tot += int64_t(secs[i].N) * kcount[i];
  }
  double* Us = (double*)ctx->buf("proj.Us", sizeof(double) * std::max<int64_t>(us_tot, 1), s);
  double* Vs = (double*)ctx->buf("proj.Vs", sizeof(double) * std::max<int64_t>(vs_tot, 1), s);
  double* Pm = (double*)ctx->buf("proj.Pm", sizeof(double) * std::max<int64_t>(vp->mv.total, 1), s);
  double* Ptm = (double*)ctx->buf("proj.Ptm", sizeof(double) * std::max<int64_t>(vpt->mv.total, 1), s);
  BST_CUDA(cudaMemsetAsync(Pm, 0, sizeof(double) * std::max<int64_t>(vp->mv.total, 1), s));
  BST_CUDA(cudaMemsetAsync(Ptm, 0, sizeof(double) * std::max<int64_t>(vpt->mv.total, 1), s));
  std::vector<GemmProb> gp, gpt;
  int64_t uo = 0, vo = 0;
  for (size_t i = 0; i < secs.size(); ++i) {
    const Sec& x = secs[i];
    const int k = kcount[i];
    if (k == 0) continue;
    // left vectors of N_s (length M) and right vectors (length N)
    const double *Ul, *Vr;
    long long ui, uj, vi, vj;
    if (x.trans) {  // X = N_s^T = Ux S VTx: left(N_s) = rows of VTx, right(N_s) = cols of Ux
      Ul = dV + x.v_off; ui = x.mn; uj = 1;     // VTx[j + i*ldvt], ldvt = mn
      Vr = dU + x.u_off; vi = 1; vj = x.N;      // Ux[i + j*N]
    } else {        // Y = N_s = Uy S VTy
      Ul = dU + x.u_off; ui = 1; uj = x.M;
      Vr = dV + x.v_off; vi = x.mn; vj = 1;
    }
    gauge_scale_kernel<<<k, 256, 0, s>>>(Ul, ui, uj, x.M, Vr, vi, vj, x.N, dS + x.s_off, k, Us + uo, Vs + vo);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
    const int key = int(x.cs->key);
    const MatSector* ps = vp->mv.find(key);
    const MatSector* pts = vpt->mv.find(key);
    BST_REQUIRE(ps && pts && ps->cols == k && pts->rows == k, BST_E_SHAPE, "projector: view mismatch");
    BST_REQUIRE(ps->rows == x.bs->cols && pts->cols == x.as->cols, BST_E_SHAPE, "projector: cut mismatch");
    // P_s[a', j] = sum_b' Rb[a', b'] V~[b', j]  with Rb^T stored as Bmat [b' x a']
    GemmProb g{};
    g.M = int(ps->rows); g.N = k; g.K = x.N;
    g.a_off = x.bs->off; g.a_m = 1; g.a_k = x.bs->cols;
    g.b_off = vo; g.b_n = 1; g.b_k = k;
    g.c_off = ps->off; g.c_m = k; g.c_n = 1;
    gp.push_back(g);
    // Pt_s[j, a] = sum_b U~[b, j] Rt[a, b]  with Rt^T stored as Amat [b x a]
    GemmProb h2{};
    h2.M = k; h2.N = int(pts->cols); h2.K = x.M;
    h2.a_off = uo; h2.a_m = 1; h2.a_k = k;
    h2.b_off = x.as->off; h2.b_n = 1; h2.b_k = x.as->cols;
    h2.c_off = pts->off; h2.c_m = pts->cols; h2.c_n = 1;
    gpt.push_back(h2);
    uo += int64_t(x.M) * k;
    vo += int64_t(x.N) * k;
  }
  if (prec == BST_FP64) {
    std::string base = std::to_string((uintptr_t)pn) + "/" + std::to_string(res.P->id);
    launch_gemm_f64(ctx, *get_dev_gemm(ctx, "projP/" + base, gp), Bt, Vs, Pm, s);
    launch_gemm_f64(ctx, *get_dev_gemm(ctx, "projPt/" + base, gpt), Us, At, Ptm, s);
  } else {
    run_gemm_ozaki_probs(ctx, "projP", gp, Bt, Vs, Pm, s);
    run_gemm_ozaki_probs(ctx, "projPt", gpt, Us, At, Ptm, s);
  }
  launch_relayout(ctx, vp->rel, p, Pm, 1, 1.0, 0.0, s);
  launch_relayout(ctx, vpt->rel, pt, Ptm, 1, 1.0, 0.0, s);
  return res;
}

__global__ void transpose_kernel(const double* A, double* Y, int M, int N) {
  // Y[i + j*M] = A[i*N + j]
  __shared__ double t[32][33];
  int j = blockIdx.x * 32 + threadIdx.x, i0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8)
    if (i0 + r < M && j < N) t[r][threadIdx.x] = A[(long long)(i0 + r) * N + j];
  __syncthreads();
  int i = i0 + threadIdx.x, j0 = blockIdx.x * 32;
  for (int c = threadIdx.y; c < 32; c += 8)
    if (i < M && j0 + c < N) Y[i + (long long)(j0 + c) * M] = t[threadIdx.x][c];
}

void launch_transpose(const double* A, double* Y, int M, int N, cudaStream_t s) {
  dim3 grid((N + 31) / 32, (M + 31) / 32), tb(32, 8);
  transpose_kernel<<<grid, tb, 0, s>>>(A, Y, M, N);
}

}  // namespace bst
