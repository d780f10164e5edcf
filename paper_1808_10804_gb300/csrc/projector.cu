// SVD projectors of the CTMRG move (Sec. 3: the corner transfer matrix is
// truncated as in corboz14).
//
// N = Rtop^T Rbot over the left cut is block diagonal in the charge through
// the right cut.  The leading singular pairs of every sector come from a
// residual-controlled subspace iteration on N^T N with an FP64 Rayleigh-Ritz
// step (factors_subspace; sectors of dimension <= 160 are decomposed
// directly), or from cuSOLVER's FP64 gesvd (factors_gesvd, on request or as
// the fallback); the chi largest singular values over all sectors are kept
// (a host decision: one stream synchronisation), and
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

// Gauge and scale (U = N V when u_div_sigma, else the left vector): for kept vector j, u_j = column j of the left factor
// (element i at U[i*us_i + j*us_j]); sign from the largest |u_j(i)| (lowest i
// on ties); writes Uo[i*m + j] = sign*u/sqrt(s_j) (row-major [m x k]) and
// Vo[i*k + j] = sign*v/sqrt(s_j) (row-major [n x k]).
__global__ void gauge_scale_kernel(const double* U, long long us_i, long long us_j, int m,
                                   const double* V, long long vs_i, long long vs_j, int n,
                                   const double* S, int k, double* Uo, double* Vo, int u_div_sigma,
                                   double sscale) {
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
  const double f = sgn / sqrt(S[j] * sscale);
  const double fu = u_div_sigma ? f / S[j] : f;
  for (int i = threadIdx.x; i < m; i += blockDim.x) Uo[(long long)i * k + j] = fu * U[i * us_i + j * us_j];
  for (int i = threadIdx.x; i < n; i += blockDim.x) Vo[(long long)i * k + j] = f * V[i * vs_i + j * vs_j];
}

// out[r][j] = in[r][perm[j]] for a row-major block with c columns
__global__ void permute_cols(const double* in, double* out, int c, const int* perm) {
  const long long r = blockIdx.x;
  for (int j = threadIdx.x; j < c; j += blockDim.x) out[r * c + j] = in[r * c + perm[j]];
}

// Views and scatter plans of a projector layout, cached by layout.
struct ProjView {
  MatView mv;
  DevRelayout rel;
  ~ProjView() { rel.free_all(); }
};

// Sector-matrix view of a projector layout, cached in the context (freed
// with it) by layout id and row legs.
static ProjView* get_projview(Ctx* ctx, Layout* L, const std::vector<int>& rows, const std::vector<int>& cols) {
  std::string key = std::to_string(L->id) + "/" + std::to_string(rows.size());
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->projviews.find(key);
    if (it != ctx->projviews.end()) return it->second.get();
  }
  auto pv = std::make_shared<ProjView>();
  pv->mv = make_matview(L, rows, cols);
  pv->rel.upload(pv->mv.tasks);
  ProjView* raw = pv.get();
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->projviews[key] = std::move(pv);
  return raw;
}


// kernels of eig.cu
struct SmallProb {
  int32_t b, pad;
  int64_t in_off, out_off, val_off;
};
struct ResProb {
  int32_t m, k;
  int64_t y_off, v_off, val_off, ld;
};
__global__ void jacobi_eig_f32(const SmallProb*, const double*, double*, double*, int, float, float);
__global__ void jacobi_block_f32(const SmallProb*, const double*, double*, double*, int, float, float, float, float,
                                 int*);
size_t jacobi_block_smem(int b);
__global__ void oa_update(const SmallProb*, const double*, const double*, double*, double*, double, double, double);
__global__ void add_inplace(double*, const double*, long long);
__global__ void cholinv_f32(const SmallProb*, const double*, double*, int*, const float*, int);
struct GramProb {
  int32_t M, b;
  int64_t x_off, ld, out_off;
};
__global__ void gram_f32_kernel(const GramProb*, int, const double*, float*);
__global__ void ident_combo(const SmallProb*, const double*, double*, double, double);
__global__ void randn_fill(double*, const long long*);
__global__ void ritz_residual(const ResProb*, const double*, const double*, const double*, double*);
size_t jacobi_smem(int b);
size_t cholinv_smem(int b);
constexpr int kEigMax = 160;
constexpr int kGramMaxParts = 16;  // most K slices of a partial Gram matrix (cholinv_f32 holds them all)

static GemmProb gp(int M, int N, int K, int64_t ao, int64_t am, int64_t ak, int64_t bo, int64_t bn, int64_t bk,
                   int64_t co, int64_t cm, int64_t cn) {
  GemmProb g{};
  g.M = M; g.N = N; g.K = K;
  g.a_off = ao; g.a_m = am; g.a_k = ak;
  g.b_off = bo; g.b_n = bn; g.b_k = bk;
  g.c_off = co; g.c_m = cm; g.c_n = cn;
  return g;
}

static std::string probs_key(const std::vector<GemmProb>& probs) {
  return std::to_string(probs_hash(probs));
}

// FP64-accurate grouped GEMM in the requested arithmetic.
// Number of K slices for `tiles` output tiles: at least enough CTAs to put
// `per_sm` on every SM, at most `kmax` slices; among those the count with
// the shortest busiest SM, ceil(tiles * ks / SMs) CTAs of 1/ks of K each,
// fewer slices on ties.
static int k_slices(int64_t tiles, int kmax, int per_sm) {
  const int64_t sms = 152;
  if (tiles <= 0 || kmax <= 1) return 1;
  const int kmin = int(std::max<int64_t>(1, std::min<int64_t>(kmax, (sms * per_sm + tiles - 1) / tiles)));
  int best = kmin;
  double best_t = 1e300;
  for (int ks = kmin; ks <= kmax; ++ks) {
    const double t = double((tiles * ks + sms - 1) / sms) / ks;
    if (t < best_t - 1e-12) {
      best_t = t;
      best = ks;
    }
  }
  return best;
}

static void gemm_any(Ctx* ctx, const std::string& tag, bst_prec prec, const std::vector<GemmProb>& probs,
                     const double* A, const double* B, double* C, cudaStream_t s, bool same_a = false,
                     const char* ws = "gemm_f64.splitk") {
  if (probs.empty()) return;
  if (prec == BST_FP64) {
    // the projector's FP64 products are small and deep (b x b x K), and an
    // SM does only ~8 GFLOP/s of FP64 tensor work: split K (slices down to
    // 16 deep) until about two CTAs per SM are busy
    const DevGemm& g = *get_dev_gemm(ctx, tag + "/" + probs_key(probs), probs);
    int ksplit = 1;
    if (g.ntiles > 0 && g.ntiles < 304) ksplit = k_slices(g.ntiles, std::min(g.maxK / 16, 16), 2);
    launch_gemm_f64_splitk(ctx, g, ksplit, A, B, C, s, ws);
    return;
  }
  // Mixed: the tcgen05 kernel gives each 128 x 64 output tile to one CTA,
  // so a small, deep product (the b x b Gram of an M x b block, N Q) keeps
  // few SMs busy.  Split K (slices of a multiple of 32, at most 8) until
  // about one tile per SM is in flight: the slices are problems of their
  // own writing an M x N workspace slice, summed in slice order in FP64.
  int64_t tiles = 0;
  int maxK = 0;
  for (auto& p : probs) {
    tiles += int64_t((p.M + 127) / 128) * ((p.N + 63) / 64);
    maxK = std::max(maxK, p.K);
  }
  int ks = 1;
  if (tiles > 0 && tiles < 152) ks = k_slices(tiles, std::min(maxK / 96, 8), 1);
  if (ks <= 1) {
    run_gemm_ozaki_probs(ctx, tag, probs, A, B, C, s, 0, !same_a);
    return;
  }
  const DevGemm& g = *get_dev_gemm(ctx, tag + "/ksred/" + probs_key(probs), probs);
  std::vector<GemmProb> sp;
  for (int sl = 0; sl < ks; ++sl)
    for (size_t i = 0; i < probs.size(); ++i) {
      const GemmProb& p = probs[i];
      const int kc = ((p.K + ks - 1) / ks + 31) / 32 * 32;
      const int kb = std::min(p.K, sl * kc), ke = std::min(p.K, kb + kc);
      GemmProb q = p;
      q.K = ke - kb;
      q.a_off = p.a_off + int64_t(kb) * p.a_k;
      q.b_off = p.b_off + int64_t(kb) * p.b_k;
      q.c_off = int64_t(sl) * g.wtot + g.hw_off[i];
      q.c_m = p.N;
      q.c_n = 1;
      sp.push_back(q);
    }
  const std::string wsname = std::string(ws) + ".oz";
  double* W = (double*)ctx->buf(wsname, sizeof(double) * std::max<int64_t>(1, g.wtot * ks), s);
  run_gemm_ozaki_probs(ctx, tag + "/ks", sp, A, B, W, s, 0, !same_a);
  launch_ksplit_reduce(ctx, g, W, ks, C, s);
}

template <class T>
static T* upload_cached(Ctx* ctx, const std::string& name, const std::vector<T>& v, cudaStream_t s) {
  T* d = (T*)ctx->buf(name, sizeof(T) * std::max<size_t>(v.size(), 1), s);
  BST_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return d;
}

struct PSec;
static bool cut_unresolved(const PSec& x, const std::vector<double>& hSig, double kmin);

struct PSec {
  const MatSector *cs, *as, *bs;
  int M, N;        // N_s is M x N (rows: right cut of Rt, cols: right cut of Rb)
  int c;           // candidate singular values (descending)
  int64_t v_off;   // right vectors, row-major N x c
  int64_t s_off;   // offset into the host sigma list
  bool direct;     // eigen-decomposition of N^T N without subspace iteration
  int b;           // small problem size
  int64_t q_off, z_off, sm_off, val_off;
  int64_t kmax;    // most states the truncation can keep from this sector (0: chi)
  int64_t u_off;   // left vectors, row-major M x c, from the full SVD (-1: none)
};

// The small eigensolver of an iterated sector resolves its eigenvalues of
// N^T N below 1e-6 of its largest only to ~1e-9 of the largest (one
// unresolved cluster): singular values below sqrt(1e-5) of the sector's
// largest (a tenfold margin) cannot decide the truncation.  A direct
// sector's graded solve resolves eigenvalues down to ~1e-12 of its largest
// (margin: 1e-11).  True when the smallest kept value kmin falls in that
// range of a sector that has values above it: the candidates are then
// recomputed by the full FP64 SVD.
static bool cut_unresolved(const PSec& x, const std::vector<double>& hSig, double kmin) {
  if (x.c <= 0) return false;
  const double top = hSig[x.s_off];  // candidates are sorted descending
  return top > kmin && kmin * kmin < (x.direct ? 1e-11 : 1e-5) * top * top;
}

static void setup_attrs() {
  static bool done = false;
  if (done) return;
  BST_CUDA(cudaFuncSetAttribute(jacobi_eig_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(jacobi_smem(kEigMax))));
  BST_CUDA(cudaFuncSetAttribute(jacobi_block_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(jacobi_block_smem(kEigMax))));
  BST_CUDA(cudaFuncSetAttribute(cholinv_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cholinv_smem(kEigMax))));
  done = true;
}

// Symmetric eigenproblems (b <= 160) in FP64 accuracy.  An FP32 Jacobi
// pass diagonalises H to FP32 level (off-diagonals tested absolutely, in
// units of the largest diagonal entry; pairs of values both below 1e-5 of
// it left to the next pass); H is rotated into that basis in FP64
// (H1 = X1^T H X1, nearly diagonal) and a second FP32 Jacobi pass resolves
// it to high relative accuracy (tested relative to the diagonal, floor
// 1e-5); two Ogita-Aishima steps then bring the vectors and values to FP64
// accuracy.  Values below 1e-6 of the largest
// are treated as one unresolved cluster.  `pre` prefixes every workspace,
// plan and table name, so calls with different prefixes may run on
// different streams at the same time.
// near_diag: H is already close to diagonal (the Rayleigh-Ritz matrix of a
// block from orthogonal iteration: CholQR keeps the columns in the order of
// the singular values they converge to, so only close pairs still mix); the
// first, absolute Jacobi pass and the rotation into its basis are skipped
// and the relative pass starts from H itself.
// Graded solves (`gr` set): H_i = N_i^T N_i of a sector matrix N_i
// (M_i x b_i, row-major at noff_i of Nm).  An eigenvector of a small
// eigenvalue lambda computed from H itself carries the rounding of H,
// eps lambda_max, over the gap: with lambda = sigma^2 the singular vectors
// at the truncation of a fast-decaying spectrum lose about as many digits
// as sigma_1^2 / sigma^2 has.  Here only the first, absolute FP32 pass uses
// H; the matrices of the second pass and of the refinement are formed as
// W^T W with W = N X, whose entries are accurate to eps sigma_1 (sigma_i +
// sigma_j), i.e. relative to the singular values themselves (the accuracy
// of an SVD of N), and that pass rotates pairs relative to their own size.
struct Graded {
  const double* Nm;
  std::vector<int> M;
  std::vector<int64_t> noff;
};

static void small_eig(Ctx* ctx, bst_prec prec, const std::vector<SmallProb>& sp, const double* H, double* X, double* lam,
                      int64_t smtot, int64_t valtot, cudaStream_t s, const std::string& pre = "",
                      bool near_diag = false, const Graded* gr = nullptr, int* dsweeps = nullptr) {
  if (sp.empty()) return;
  setup_attrs();
  SmallProb* dsp = upload_cached(ctx, pre + "eig.sp", sp, s);
  int bmax = 0;
  for (auto& p : sp) bmax = std::max(bmax, p.b);
  // FP32 Jacobi stage: the block kernel (32 x 32 subproblems per round)
  // (dsweeps: the sweeps each problem ran, of the last Jacobi stage)
  // (tol: the stop test on min(relative, angle) of every pair; 1e-13 is
  // the FP32 floor)
  auto jacobi = [&](const SmallProb* pp, const double* in, double* o, double* l, int sweeps, float tf, float jk,
                    float tol = 1e-13f, float skip_ang = 0.f) {
    jacobi_block_f32<<<int(sp.size()), 512, jacobi_block_smem(bmax), s>>>(pp, in, o, l, sweeps, tf, jk, tol,
                                                                          skip_ang, dsweeps);
  };
  double* X1 = (double*)ctx->buf(pre + "eig.x1", sizeof(double) * smtot, s);
  double* H1 = (double*)ctx->buf(pre + "eig.h1", sizeof(double) * smtot, s);
  double* XtX = (double*)ctx->buf(pre + "eig.xtx", sizeof(double) * smtot, s);
  double* T = (double*)ctx->buf(pre + "eig.t", sizeof(double) * smtot, s);
  double* S = (double*)ctx->buf(pre + "eig.s", sizeof(double) * smtot, s);
  double* E = (double*)ctx->buf(pre + "eig.e", sizeof(double) * smtot, s);
  const std::string wsname = pre + "gemm_f64.splitk";
  const char* ws = wsname.c_str();
  std::vector<GemmProb> g_xtx, g_hx, g_s, g_xe;
  for (auto& p : sp) {
    const int b = p.b;
    const int64_t o = p.in_off;
    g_xtx.push_back(gp(b, b, b, o, 1, b, o, 1, b, o, b, 1));     // X^T X
    g_hx.push_back(gp(b, b, b, o, b, 1, o, 1, b, o, b, 1));      // H X
    g_s.push_back(gp(b, b, b, o, 1, b, o, 1, b, o, b, 1));       // X^T T
    g_xe.push_back(gp(b, b, b, o, b, 1, o, 1, b, o, b, 1));      // X E
  }
  // graded: W = N X and W^T W per problem
  std::vector<GemmProb> g_w, g_ww;
  double* Wg = nullptr;
  if (gr) {
    BST_REQUIRE(gr->M.size() == sp.size() && gr->noff.size() == sp.size(), BST_E_ARG, "graded solve tables");
    int64_t wtot = 0;
    for (size_t i = 0; i < sp.size(); ++i) {
      const int b = sp[i].b;
      const int64_t o = sp[i].in_off;
      g_w.push_back(gp(gr->M[i], b, b, gr->noff[i], b, 1, o, 1, b, wtot, b, 1));  // W = N X
      g_ww.push_back(gp(b, b, gr->M[i], wtot, 1, b, wtot, 1, b, o, b, 1));        // W^T W
      wtot += int64_t(gr->M[i]) * b;
    }
    Wg = (double*)ctx->buf(pre + "eig.w", sizeof(double) * std::max<int64_t>(wtot, 1), s);
  }
  // nominal work of one Jacobi launch at its sweep limit: per sweep b-1
  // rounds of b/2 rotations, each touching 2 rows and 2 columns of A and V
  double jac_flops = 0;
  for (auto& p : sp) jac_flops += 7.0 * double(p.b) * p.b * 18.0 * p.b / 2.0;
  if (gr && !near_diag) {
    {
      ProfScope ps(ctx, s, "jacobi_f32", jac_flops, 0.0);
      jacobi(dsp, H, X1, lam, 7, 1.0f, 1e-5f);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    gemm_any(ctx, pre + "oa.w", prec, g_w, gr->Nm, X1, Wg, s, false, ws);
    gemm_any(ctx, pre + "oa.ww", prec, g_ww, Wg, Wg, H1, s, false, ws);
    {
      ProfScope ps(ctx, s, "jacobi_f32", jac_flops, 0.0);
      // pairs below 1e-14 of the largest (beyond the accuracy of H1) are
      // left out of the convergence test
      jacobi(dsp, H1, T, lam, 10, 1e-20f, 1e-14f);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    gemm_any(ctx, pre + "oa.xe", prec, g_xe, X1, T, X, s, false, ws);  // X = X1 X2
  } else if (near_diag) {
    ProfScope ps(ctx, s, "jacobi_f32", jac_flops, 0.0);
    // values below 1e-6 of the largest are not resolved by this FP32 pass
    // (nor refined below): their pairs are left out of the convergence test.
    // The pass stops once every pair's remaining rotation is below ~3e-4
    // (or its off-diagonal below 1e-4 of the diagonals' geometric mean):
    // the three refinement steps below square the angles three times, from
    // there to far below FP64 rounding.  Rotations by less than ~3e-5 are
    // left to the refinement as well (sweeps after the first find most
    // pairs there, and skip their updates).
    jacobi(dsp, H, X, lam, 10, 1e-5f, 1e-6f, 1e-8f, 1e-10f);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  } else {
    {
      ProfScope ps(ctx, s, "jacobi_f32", jac_flops, 0.0);
      jacobi(dsp, H, X1, lam, 7, 1.0f, 1e-5f);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    gemm_any(ctx, pre + "oa.hx", prec, g_hx, H, X1, T, s, false, ws);
    gemm_any(ctx, pre + "oa.s", prec, g_s, X1, T, H1, s, false, ws);
    {
      ProfScope ps(ctx, s, "jacobi_f32", jac_flops, 0.0);
      jacobi(dsp, H1, T, lam, 7, 1e-5f, 0.f);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    gemm_any(ctx, pre + "oa.xe", prec, g_xe, X1, T, X, s, false, ws);  // X = X1 X2
  }
  // three refinement steps: quadratic from the FP32 stage's angles, which
  // for a pair of values closer than ~1e-6 relative are limited by FP32
  // rounding to ~1e-2 (two steps reach 1e-8 there, three the FP64 floor)
  // (not graded) X and T = H X side by side in one buffer XC, so that
  // X^T X and X^T T are one launch: X^T [X | T]
  std::vector<GemmProb> g_hx2, g_xs;
  double *XC = nullptr, *XS = nullptr;
  if (!gr) {
    for (auto& p : sp) {
      const int b = p.b;
      const int64_t o = p.in_off;
      g_hx2.push_back(gp(b, b, b, o, b, 1, o, 1, b, smtot + o, b, 1));         // T = H X
      g_xs.push_back(gp(b, b, b, o, 1, b, o, 1, b, o, b, 1));                  // X^T X
    }
    for (auto& p : sp) {
      const int b = p.b;
      const int64_t o = p.in_off;
      g_xs.push_back(gp(b, b, b, o, 1, b, smtot + o, 1, b, smtot + o, b, 1));  // X^T T
    }
    XC = (double*)ctx->buf(pre + "eig.xc", sizeof(double) * 2 * smtot, s);
    XS = (double*)ctx->buf(pre + "eig.xs", sizeof(double) * 2 * smtot, s);
    BST_CUDA(cudaMemcpyAsync(XC, X, sizeof(double) * smtot, cudaMemcpyDeviceToDevice, s));
  }
  for (int it = 0; it < 3; ++it) {
    const double* xtx = XtX;
    const double* sm = S;
    if (gr) {
      gemm_any(ctx, pre + "oa.xtx", prec, g_xtx, X, X, XtX, s, false, ws);
      // S = (N X)^T (N X): accurate relative to the singular values, so
      // every pair above eps sigma_1 is refined
      gemm_any(ctx, pre + "oa.w", prec, g_w, gr->Nm, X, Wg, s, false, ws);
      gemm_any(ctx, pre + "oa.ww", prec, g_ww, Wg, Wg, S, s, false, ws);
    } else {
      gemm_any(ctx, pre + "oa.hx2", prec, g_hx2, H, XC, XC, s, false, ws);
      gemm_any(ctx, pre + "oa.xs", prec, g_xs, XC, XC, XS, s, false, ws);
      xtx = XS;
      sm = XS + smtot;
    }
    // about two CTAs per SM over all problems
    const int slices = std::max(1, std::min(64, 304 / int(sp.size())));
    // graded: the FP32 passes resolve eigenvalues down to ~1e-12 of the
    // largest; S is accurate to ~eps sigma_1 (sigma_i + sigma_j)
    oa_update<<<dim3(unsigned(sp.size()), unsigned(slices)), 256, 0, s>>>(dsp, xtx, sm, E, lam, 1e-9,
                                                                          gr ? 1e-12 : 1e-6, gr ? 1e-13 : 0.0);
    double* Xi = gr ? X : XC;
    gemm_any(ctx, pre + "oa.xe", prec, g_xe, Xi, E, T, s, false, ws);
    add_inplace<<<std::max<int64_t>(1, std::min<int64_t>((smtot + 255) / 256, 1216)), 256, 0, s>>>(Xi, T, smtot);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx, 2);
  }
  if (!gr) BST_CUDA(cudaMemcpyAsync(X, XC, sizeof(double) * smtot, cudaMemcpyDeviceToDevice, s));
}

// Sum of squares of each listed block of x (one CTA per block, fixed order).
__global__ void block_sumsq(const double* __restrict__ x, const int64_t* __restrict__ off_n, double* __restrict__ out) {
  const int64_t off = off_n[2 * blockIdx.x], n = off_n[2 * blockIdx.x + 1];
  __shared__ double sh[256];
  double acc = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[off + i] * x[off + i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// Leading right singular vectors of every sector of N: subspace iteration on
// N^T N (block b) and a Rayleigh-Ritz step; small sectors directly.
// Fills dV (row-major N x c per sector) and hSig; returns false when a
// sector needs more candidates than the small eigensolver holds.
// `top_chi`: the truncation keeps exactly the chi largest values (U(1));
// only then can a sector be skipped by the bound below.
static bool factors_subspace(Ctx* ctx, double* Nm, std::vector<PSec>& secs, int64_t chi, bst_prec prec, int iters,
                             double*& dV, std::vector<double>& hSig, cudaStream_t s, bool top_chi = true) {
  // The iterations only have to converge the subspace, so they run in the
  // call's arithmetic; the Rayleigh-Ritz stage fixes the individual vectors,
  // whose error is amplified by 1/gap: its Gram, eigensolver and V = Q W
  // run in FP64 (N Q itself comes from the call's product, see below).
  const bst_prec rr = BST_FP64;
  int64_t vtot = 0, qtot = 0, ztot = 0, smtot = 0, valtot = 0;
  // Block of an iterated sector.  In mixed precision: the sector keeps at
  // most kmax vectors (chi; for SU(2) chi over the multiplet dimension);
  // half as many again (plus 16) set the convergence rate (sigma_{b+1} /
  // sigma_kept)^2 per iteration; multiples of 32, 64 to 160 (the Cholesky
  // and eigensolver costs grow as b^2 and b^3, the products as b).  In
  // FP64 the full 160: the wider guard band keeps the vectors at the
  // truncation edge at FP64 accuracy.
  auto block_of = [&](const PSec& x) {
    if (prec == BST_FP64) return kEigMax;
    const int64_t k = x.kmax > 0 ? std::min<int64_t>(x.kmax, chi) : chi;
    return int(std::min<int64_t>(kEigMax, std::max<int64_t>(64, (k + k / 2 + 16 + 31) / 32 * 32)));
  };
  for (auto& x : secs) {
    x.u_off = -1;
    x.direct = x.N <= kEigMax;
    x.b = x.direct ? x.N : block_of(x);
    x.c = x.b;
    x.v_off = vtot;
    vtot += int64_t(x.N) * x.c;
    x.q_off = qtot;
    qtot += x.direct ? 0 : int64_t(x.N) * x.b;
    x.z_off = ztot;
    ztot += x.direct ? 0 : int64_t(std::max(x.M, x.N)) * x.b;
    x.sm_off = smtot;
    smtot += int64_t(x.b) * x.b;
    x.val_off = valtot;
    valtot += x.b;
  }
  dV = (double*)ctx->buf("proj.V2", sizeof(double) * std::max<int64_t>(vtot, 1), s);
  double* Q = (double*)ctx->buf("proj.Q", sizeof(double) * std::max<int64_t>(qtot, 1), s);
  double* Y = (double*)ctx->buf("proj.Y", sizeof(double) * std::max<int64_t>(qtot, 1), s);
  double* Z = (double*)ctx->buf("proj.Z", sizeof(double) * std::max<int64_t>(ztot, 1), s);
  double* Z2 = (double*)ctx->buf("proj.Z2", sizeof(double) * std::max<int64_t>(ztot, 1), s);
  double* Msm = (double*)ctx->buf("proj.M", sizeof(double) * std::max<int64_t>(smtot, 1), s);
  double* Rinv = (double*)ctx->buf("proj.Rinv", sizeof(double) * std::max<int64_t>(smtot, 1), s);
  double* Xv = (double*)ctx->buf("proj.X2", sizeof(double) * std::max<int64_t>(smtot, 1), s);
  double* lam = (double*)ctx->buf("proj.lam", sizeof(double) * std::max<int64_t>(valtot, 1), s);
  // row-major blocks: Q, Y [N x b] at q_off; Z, Z2 [M x b] at z_off
  std::vector<GemmProb> g_z, g_gz, g_qz, g_y, g_gy, g_qy, g_h, g_v, g_direct, g_polish;
  std::vector<SmallProb> sp_it;
  for (auto& x : secs) {
    SmallProb sp{x.b, 0, x.sm_off, x.sm_off, x.val_off};
    const int64_t no = x.cs->off;
    if (x.direct) {
      g_direct.push_back(gp(x.N, x.N, x.M, no, 1, x.N, no, 1, x.N, x.sm_off, x.N, 1));  // N^T N
      continue;
    }
    sp_it.push_back(sp);
    const int b = x.b;
    g_z.push_back(gp(x.M, b, x.N, no, x.N, 1, x.q_off, 1, b, x.z_off, b, 1));          // Z = N Q
    g_gz.push_back(gp(b, b, x.M, x.z_off, 1, b, x.z_off, 1, b, x.sm_off, b, 1));       // Z^T Z
    g_qz.push_back(gp(x.M, b, b, x.z_off, b, 1, x.sm_off, 1, b, x.z_off, b, 1));       // Z2 = Z Rinv
    g_y.push_back(gp(x.N, b, x.M, no, 1, x.N, x.z_off, 1, b, x.q_off, b, 1));          // Y = N^T Z2
    g_gy.push_back(gp(b, b, x.N, x.q_off, 1, b, x.q_off, 1, b, x.sm_off, b, 1));       // Y^T Y
    g_qy.push_back(gp(x.N, b, b, x.q_off, b, 1, x.sm_off, 1, b, x.q_off, b, 1));       // Q = Y Rinv
    g_h.push_back(gp(b, b, x.M, x.z_off, 1, b, x.z_off, 1, b, x.sm_off, b, 1));        // H = Z^T Z
    g_v.push_back(gp(x.N, b, b, x.q_off, b, 1, x.sm_off, 1, b, x.v_off, b, 1));        // V = Q W
  }
  SmallProb* dsp_it = sp_it.empty() ? nullptr : upload_cached(ctx, "proj.spit", sp_it, s);
  setup_attrs();
  int bmax = 1;
  for (auto& x : secs) bmax = std::max(bmax, x.b);
  double chol_flops = 0;
  for (auto& x : sp_it) chol_flops += 2.0 * 2.0 * double(x.b) * x.b * x.b / 3.0;  // factor + inverse, FMA = 2
  // CholQR of a block X (rows of every iterated sector at its q_off or z_off,
  // row stride b): the Gram matrix only feeds the FP32 factor, so it is
  // formed in FP32 by K-sliced partial sums (gram_f32_kernel, all SMs),
  // which the Cholesky kernel adds in slice order while it loads
  std::vector<SmallProb> sp_g;
  std::vector<GramProb> gq, gz;
  int64_t gtot = 0;
  int nparts = 1;
  if (!sp_it.empty()) {
    nparts = int(std::max<int64_t>(1, std::min<int64_t>(kGramMaxParts, (152 + int64_t(sp_it.size()) - 1) / int64_t(sp_it.size()))));
    for (auto& x : secs) {
      if (x.direct) continue;
      sp_g.push_back(SmallProb{x.b, 0, gtot, x.sm_off, x.val_off});
      gq.push_back(GramProb{x.N, x.b, x.q_off, x.b, gtot});
      gz.push_back(GramProb{x.M, x.b, x.z_off, x.b, gtot});
      gtot += int64_t(nparts) * x.b * x.b;
    }
  }
  SmallProb* dsp_g = sp_g.empty() ? nullptr : upload_cached(ctx, "proj.spg", sp_g, s);
  GramProb* dgq = gq.empty() ? nullptr : upload_cached(ctx, "proj.gq", gq, s);
  GramProb* dgz = gz.empty() ? nullptr : upload_cached(ctx, "proj.gz", gz, s);
  float* Gp = (float*)ctx->buf("proj.gparts", sizeof(float) * std::max<int64_t>(gtot, 1), s);
  double gram_flops = 0;
  for (auto& x : secs)
    if (!x.direct) gram_flops += 2.0 * double(std::max(x.M, x.N)) * x.b * x.b;
  auto cholqr_factor = [&](const double* X, bool z_side, double* Rout) {
    {
      ProfScope ps(ctx, s, "gram_f32", gram_flops, 0.0);
      gram_f32_kernel<<<dim3(unsigned(sp_g.size()), unsigned(nparts)), 256, 0, s>>>(z_side ? dgz : dgq, nparts, X,
                                                                                   Gp);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
    }
    ProfScope ps(ctx, s, "cholinv_f32", chol_flops, 0.0);
    cholinv_f32<<<int(sp_g.size()), 512, cholinv_smem(bmax), s>>>(dsp_g, Msm, Rout, ctx->d_err, Gp, nparts);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  };
  // CholQR with an FP32 factor after each half step: the blocks N Q and
  // N^T Z carry the condition number sigma_1/sigma_b once, not squared
  // N is split into tensor-core digits once per projector call: its two
  // plans ("ss.z": N, "ss.y": N^T) keep their A digits between steps
  //
  // The basis only has to stay well conditioned, not orthonormal: the
  // iterates span the same subspace whatever basis they are written in.
  // Once the block has settled (from the fourth step of a round on, mixed
  // precision), N Q is mapped with the previous step's factor of the N Q
  // side instead of a fresh one: both are close to the same diagonal of
  // singular values, so Z Rinv_prev stays near orthonormal, and the fresh
  // CholQR of the N^T side keeps Q orthonormal.  The Rayleigh-Ritz stage
  // re-orthonormalises the block to FP64 (and the residual test decides).
  double* Rz = (double*)ctx->buf("proj.Rinvz", sizeof(double) * std::max<int64_t>(smtot, 1), s);
  const int fresh_z = prec == BST_FP64 ? 1 << 30 : 3;
  bool n_split = false;
  auto iterate = [&](int n) {
    for (int t = 0; t < n; ++t) {
      gemm_any(ctx, "ss.z", prec, g_z, Nm, Q, Z, s, n_split);
      if (t < fresh_z) cholqr_factor(Z, true, Rz);
      gemm_any(ctx, "ss.qz", prec, g_qz, Z, Rz, Z2, s);
      gemm_any(ctx, "ss.y", prec, g_y, Nm, Z2, Y, s, n_split);
      n_split = true;
      cholqr_factor(Y, false, Rinv);
      gemm_any(ctx, "ss.qy", prec, g_qy, Y, Rinv, Q, s);
    }
  };
  // second CholQR pass and two first-order polishes: orthonormal to FP64
  auto orthonormalise = [&]() {
    cholqr_factor(Q, false, Rinv);
    gemm_any(ctx, "ss.qy", prec, g_qy, Q, Rinv, Y, s);
    for (int r = 0; r < 2; ++r) {
      double* src = (r == 0) ? Y : Q;
      double* dst = (r == 0) ? Q : Y;
      gemm_any(ctx, "ss.gy", prec, g_gy, src, src, Msm, s);
      ident_combo<<<dim3(unsigned(sp_it.size()), 32), 128, 0, s>>>(dsp_it, Msm, Rinv, 1.5, -0.5);
      count_launch(ctx);
      gemm_any(ctx, "ss.qy", prec, g_qy, src, Rinv, dst, s);
    }
    std::swap(Q, Y);  // the polished block is in Y
  };
  if (!sp_it.empty()) {
    // deterministic random start (a seed per sector, one launch)
    std::vector<long long> rng;
    int64_t nmax = 0;
    for (auto& x : secs)
      if (!x.direct) {
        const int64_t n = int64_t(x.N) * x.b;
        rng.push_back(x.q_off);
        rng.push_back(n);
        rng.push_back(static_cast<long long>(0x5eed0000ull + uint64_t(x.cs->key + 4096)));
        nmax = std::max(nmax, n);
      }
    const long long* drng = upload_cached(ctx, "proj.randn", rng, s);
    randn_fill<<<dim3(unsigned(std::min<int64_t>((nmax + 255) / 256, 256)), unsigned(rng.size() / 3)), 256, 0, s>>>(
        Q, drng);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  }
  // Rounds of `iters` iterations, each closed by a Rayleigh-Ritz step.  A
  // round is accepted when every Ritz pair that the truncation would keep
  // (plus a few below it) has a residual ||N^T N v - lambda v|| at most
  // tol * lambda_max, or when the residual has stopped falling (less than
  // halved by a round) while within 100 tol: the floor that the iterations'
  // arithmetic sets (the mixed-precision products) has been reached.
  // Otherwise iteration resumes from the Ritz vectors; after max_total
  // iterations the caller falls back to the full SVD.
  const double tol = prec == BST_FP64 ? 3e-14 : 4e-12;
  double prev_worst = 0;
  const int max_total = std::max(iters, 480);
  std::vector<double> hl(valtot), hres(valtot);
  // sweeps of the Rayleigh-Ritz eigensolver per iterated sector (tuning log)
  std::vector<int> hsw(sp_it.size(), 0);
  int* dsw = sp_it.empty() ? nullptr : (int*)ctx->buf("proj.sweeps", sizeof(int) * sp_it.size(), s);
  double* res = (double*)ctx->buf("proj.res", sizeof(double) * std::max<int64_t>(valtot, 1), s);
  // The direct sectors (N^T N decomposed whole) do not depend on the
  // iterations: their Gram products and eigensolver run once, on the
  // context's second stream, while the subspace iterations of the large
  // sectors run on `s`; they write disjoint parts of Msm, Xv and lam and
  // use their own workspaces.  A dense start needs several more Jacobi
  // sweeps than the nearly diagonal Rayleigh-Ritz matrices, so they are
  // kept out of the per-round eigensolver launches.
  //
  // A direct sector whose Frobenius norm is below the chi-th largest Ritz
  // value of the iterated sectors cannot reach the truncation: Ritz values
  // are lower bounds of the singular values (interlacing), so at least chi
  // states lie above every singular value of that sector.  When the last
  // call with this sector structure found all direct sectors below the
  // cut, they are deferred to after the first Rayleigh-Ritz step and
  // skipped if the bound holds again (their candidates are zero and never
  // kept); otherwise they overlap on the second stream.
  std::vector<int> dir_idx;
  std::string dir_key = "chi" + std::to_string(chi);
  for (size_t i = 0; i < secs.size(); ++i) {
    dir_key += "," + std::to_string(secs[i].M) + "x" + std::to_string(secs[i].N);
    if (secs[i].direct) dir_idx.push_back(int(i));
  }
  const bool can_defer = top_chi && !dir_idx.empty() && !sp_it.empty();
  const bool defer = can_defer && ctx->direct_below_cut.count(dir_key) && ctx->direct_below_cut[dir_key];
  double* dfro = nullptr;
  std::vector<double> hfro(dir_idx.size(), 0.0);
  if (can_defer) {
    std::vector<int64_t> offn;
    for (int i : dir_idx) {
      offn.push_back(secs[i].cs->off);
      offn.push_back(int64_t(secs[i].M) * secs[i].N);
    }
    int64_t* doffn = upload_cached(ctx, "proj.fro.offn", offn, s);
    dfro = (double*)ctx->buf("proj.fro", sizeof(double) * dir_idx.size(), s);
    block_sumsq<<<int(dir_idx.size()), 256, 0, s>>>(Nm, doffn, dfro);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  }
  bool forked = false;
  if (!g_direct.empty() && !defer) {
    std::vector<SmallProb> sp_dir;
    Graded gdir{Nm, {}, {}};
    for (auto& x : secs)
      if (x.direct) {
        sp_dir.push_back(SmallProb{x.b, 0, x.sm_off, x.sm_off, x.val_off});
        gdir.M.push_back(x.M);
        gdir.noff.push_back(x.cs->off);
      }
    if (!ctx->side) {
      BST_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
      BST_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      BST_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    // (an earlier call that left by an error may still have side work in
    // flight on these buffers: the fork orders after it)
    BST_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    BST_CUDA(cudaEventRecord(ctx->ev_fork, s));
    BST_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    gemm_any(ctx, "side.ss.direct", rr, g_direct, Nm, Nm, Msm, ctx->side, false, "side.gemm_f64.splitk");
    small_eig(ctx, rr, sp_dir, Msm, Xv, lam, smtot, valtot, ctx->side, "side.", false, &gdir);
    BST_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    forked = true;
  }
  // Rounds that only decide whether to iterate on (and restart from Ritz
  // vectors) do not need FP64 vectors: when the last mixed-precision call
  // with this sector structure needed several rounds, Rayleigh-Ritz runs in
  // the call's arithmetic until the residual test passes, and one more
  // round without iterations (re-orthonormalised block, FP64 Rayleigh-Ritz)
  // gives the vectors and must pass the test again.
  const std::string rr_key = dir_key + "/rounds";
  bool mixed_rr = prec != BST_FP64 && ctx->multi_round.count(rr_key) && ctx->multi_round[rr_key];
  if (mixed_rr && ctx->tune_log.size() < (1u << 20))
    ctx->tune_log += "projector subspace: intermediate Rayleigh-Ritz rounds in mixed arithmetic\n";
  int total = 0, steps = iters;
  for (int round = 0;; ++round) {
    const bst_prec rrp = mixed_rr ? prec : rr;
    if (!sp_it.empty()) {
      iterate(steps);
      total += steps;
      orthonormalise();
      // Rayleigh-Ritz: H = (N Q)^T (N Q).  N Q comes from the iterations'
      // product (the call's arithmetic, N's digits already split): the
      // digit GEMM reproduces it to ~2^-40 of its row and column scales,
      // which moves the Ritz pairs far less than the residual tolerance;
      // Z^T Z, the eigensolver and V = Q W run in the Rayleigh-Ritz
      // arithmetic (FP64 for the final round)
      gemm_any(ctx, "ss.z", prec, g_z, Nm, Q, Z, s, n_split);
      gemm_any(ctx, "ss.h", rrp, g_h, Z, Z, Msm, s);
    }
    small_eig(ctx, rrp, sp_it, Msm, Xv, lam, smtot, valtot, s, "", ctx->rr_near_diag, nullptr, dsw);
    // V = Q W (iterative) or W (direct, once the second stream is joined)
    if (!g_v.empty()) gemm_any(ctx, "ss.v", rrp, g_v, Q, Xv, dV, s);
    if (forked) {
      BST_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
      forked = false;
      for (auto& x : secs)
        if (x.direct)
          BST_CUDA(cudaMemcpyAsync(dV + x.v_off, Xv + x.sm_off, sizeof(double) * int64_t(x.N) * x.N,
                                   cudaMemcpyDeviceToDevice, s));
    }
    BST_CUDA(cudaMemcpyAsync(hl.data(), lam, sizeof(double) * valtot, cudaMemcpyDeviceToHost, s));
    if (dsw) BST_CUDA(cudaMemcpyAsync(hsw.data(), dsw, sizeof(int) * hsw.size(), cudaMemcpyDeviceToHost, s));
    if (round == 0 && dfro)
      BST_CUDA(cudaMemcpyAsync(hfro.data(), dfro, sizeof(double) * hfro.size(), cudaMemcpyDeviceToHost, s));
    BST_CUDA(cudaStreamSynchronize(s));
    if (round == 0 && can_defer) {
      // chi-th largest Ritz value of the iterated sectors
      std::vector<double> rv;
      for (auto& x : secs)
        if (!x.direct)
          for (int j = 0; j < x.c; ++j) rv.push_back(hl[x.val_off + j]);
      double cut = 0;
      if (int64_t(rv.size()) >= chi && chi > 0) {
        std::nth_element(rv.begin(), rv.begin() + (chi - 1), rv.end(), std::greater<double>());
        cut = rv[chi - 1];
      }
      // the margin covers the rounding of both sides
      std::vector<char> below(dir_idx.size());
      bool all_below = true;
      for (size_t t = 0; t < dir_idx.size(); ++t) {
        below[t] = cut > 0 && hfro[t] < 0.99 * cut;
        all_below = all_below && below[t];
      }
      // the hints are per sector structure: keep the maps bounded over long
      // runs whose structure keeps changing
      if (ctx->direct_below_cut.size() >= 4096) ctx->direct_below_cut.clear();
      ctx->direct_below_cut[dir_key] = all_below;
      if (defer) {
        std::vector<GemmProb> g_rel;
        std::vector<SmallProb> sp_rel;
        Graded grel{Nm, {}, {}};
        for (size_t t = 0; t < dir_idx.size(); ++t) {
          const PSec& x = secs[dir_idx[t]];
          if (below[t]) {
            BST_CUDA(cudaMemsetAsync(lam + x.val_off, 0, sizeof(double) * x.c, s));
            BST_CUDA(cudaMemsetAsync(dV + x.v_off, 0, sizeof(double) * int64_t(x.N) * x.c, s));
            for (int j = 0; j < x.c; ++j) hl[x.val_off + j] = 0.0;
          } else {
            const int64_t no = x.cs->off;
            g_rel.push_back(gp(x.N, x.N, x.M, no, 1, x.N, no, 1, x.N, x.sm_off, x.N, 1));  // N^T N
            sp_rel.push_back(SmallProb{x.b, 0, x.sm_off, x.sm_off, x.val_off});
            grel.M.push_back(x.M);
            grel.noff.push_back(no);
          }
        }
        if (!sp_rel.empty()) {
          gemm_any(ctx, "ss.direct.late", rr, g_rel, Nm, Nm, Msm, s);
          small_eig(ctx, rr, sp_rel, Msm, Xv, lam, smtot, valtot, s, "late.", false, &grel);
          for (size_t t = 0; t < dir_idx.size(); ++t)
            if (!below[t]) {
              const PSec& x = secs[dir_idx[t]];
              BST_CUDA(cudaMemcpyAsync(dV + x.v_off, Xv + x.sm_off, sizeof(double) * int64_t(x.N) * x.N,
                                       cudaMemcpyDeviceToDevice, s));
            }
          BST_CUDA(cudaMemcpyAsync(hl.data(), lam, sizeof(double) * valtot, cudaMemcpyDeviceToHost, s));
          BST_CUDA(cudaStreamSynchronize(s));
        }
      }
    }
    if (sp_it.empty()) break;
    // the Ritz pairs the truncation would keep
    double lmax = 0;
    std::vector<std::pair<double, int>> all;
    for (size_t i = 0; i < secs.size(); ++i)
      for (int j = 0; j < secs[i].c; ++j) {
        const double v = hl[secs[i].val_off + j];
        lmax = std::max(lmax, v);
        all.push_back({v, int(i)});
      }
    std::stable_sort(all.begin(), all.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<int> kc(secs.size(), 0);
    for (size_t t = 0; t < all.size() && int64_t(t) < chi; ++t) kc[all[t].second]++;
    std::vector<GemmProb> g_ry, g_rg;
    std::vector<ResProb> rp;
    int kmax = 0;
    for (size_t i = 0; i < secs.size(); ++i) {
      const PSec& x = secs[i];
      if (x.direct || kc[i] == 0) continue;
      const int k = std::min(x.c, kc[i] + 4);
      kmax = std::max(kmax, k);
      const int64_t no = x.cs->off;
      // N V[:, :k] = (N Q) W[:, :k]: Z still holds the Rayleigh-Ritz product N Q
      g_ry.push_back(gp(x.M, k, x.b, x.z_off, x.b, 1, x.sm_off, 1, x.b, x.z_off, k, 1));  // -> Z2
      g_rg.push_back(gp(x.N, k, x.M, no, 1, x.N, x.z_off, 1, k, x.q_off, x.b, 1));         // N^T (N V) -> Y
      rp.push_back({x.N, k, x.q_off, x.v_off, x.val_off, x.b});
    }
    double worst = 0;
    if (!rp.empty()) {
      // the residual only decides convergence: the call's arithmetic
      // suffices (the mixed products' error, ~1e-13 of ||N||^2, is far
      // below the 4e-12 tolerance)
      gemm_any(ctx, "ss.ry", prec, g_ry, Z, Xv, Z2, s);
      gemm_any(ctx, "ss.rg", prec, g_rg, Nm, Z2, Y, s);
      ResProb* drp = upload_cached(ctx, "proj.rp", rp, s);
      BST_CUDA(cudaMemsetAsync(res, 0, sizeof(double) * valtot, s));
      ritz_residual<<<dim3(unsigned(rp.size()), unsigned(kmax)), 256, 0, s>>>(drp, Y, dV, lam, res);
      BST_CUDA(cudaGetLastError());
      count_launch(ctx);
      BST_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * valtot, cudaMemcpyDeviceToHost, s));
      BST_CUDA(cudaStreamSynchronize(s));
      for (auto& r : rp)
        for (int j = 0; j < r.k; ++j) worst = std::max(worst, hres[r.val_off + j]);
      worst = lmax > 0 ? worst / lmax : 0.0;
    }
    if (ctx->tune_log.size() < (1u << 20)) {
      char line[160];
      snprintf(line, sizeof(line), "projector subspace: %d iterations, max residual/lambda_max %.3e, blocks", total,
               worst);
      ctx->tune_log += line;
      for (auto& x : secs)
        if (!x.direct) ctx->tune_log += " " + std::to_string(x.b);
      ctx->tune_log += ", Jacobi sweeps";
      for (int v : hsw) ctx->tune_log += " " + std::to_string(v);
      ctx->tune_log += "\n";
    }
    const bool ok = worst <= tol || (round > 0 && worst > 0.5 * prev_worst && worst <= 100 * tol);
    if (ok && !mixed_rr) break;
    if (total >= max_total) {
      if (ctx->multi_round.size() >= 4096) ctx->multi_round.clear();
      ctx->multi_round[rr_key] = true;
      return false;
    }
    // length of the next round: from the second round on, extrapolate the
    // residual's geometric decay per step to half the tolerance (at least
    // `iters`, at most 6 * iters steps), so slowly converging sectors are
    // checked with few Rayleigh-Ritz rounds
    int next = iters;
    if (ok) {
      mixed_rr = false;  // converged under mixed Rayleigh-Ritz: the FP64 round
      next = 0;
    } else if (round > 0 && steps > 0 && worst > 0 && prev_worst > worst) {
      const double rho = std::pow(worst / prev_worst, 1.0 / steps);
      const double need = std::log(0.5 * tol / worst) / std::log(rho);
      if (std::isfinite(need)) next = int(std::min<double>(6.0 * iters, std::max<double>(iters, std::ceil(need))));
    }
    steps = next == 0 ? 0 : std::min(next, std::max(1, max_total - total));
    prev_worst = worst;
    // resume from the Ritz vectors
    for (auto& x : secs)
      if (!x.direct)
        BST_CUDA(cudaMemcpyAsync(Q + x.q_off, dV + x.v_off, sizeof(double) * int64_t(x.N) * x.b,
                                 cudaMemcpyDeviceToDevice, s));
  }
  if (prec != BST_FP64) {
    if (ctx->multi_round.size() >= 4096) ctx->multi_round.clear();
    ctx->multi_round[rr_key] = total > iters;
  }
  hSig.assign(valtot, 0.0);
  for (auto& x : secs) {
    x.s_off = x.val_off;
    for (int j = 0; j < x.c; ++j) hSig[x.val_off + j] = std::sqrt(std::max(hl[x.val_off + j], 0.0));
  }
  return true;
}

// Full FP64 SVD of every sector with cuSOLVER (gesvd); used for sectors the
// small eigensolver cannot hold.
static void factors_gesvd(Ctx* ctx, double* Nm, int64_t cmat, std::vector<PSec>& secs, double*& dV,
                          double*& dUl, std::vector<double>& hSig, cudaStream_t s) {
  if (!ctx->cusolver) {
    cusolverDnHandle_t h;
    BST_CUSOLVER(cusolverDnCreate(&h));
    ctx->cusolver = h;
  }
  cusolverDnHandle_t h = (cusolverDnHandle_t)ctx->cusolver;
  BST_CUSOLVER(cusolverDnSetStream(h, s));
  int64_t stot = 0, utot = 0, vtot = 0, vt2 = 0, ultot = 0;
  int lwork = 0, maxmn = 1;
  std::vector<int64_t> u_off(secs.size()), vt_off(secs.size());
  for (size_t i = 0; i < secs.size(); ++i) {
    auto& x = secs[i];
    const int mn = std::min(x.M, x.N);
    x.c = mn;
    x.s_off = stot;
    stot += mn;
    u_off[i] = utot;
    utot += int64_t(std::max(x.M, x.N)) * mn;
    vt_off[i] = vt2;
    vt2 += int64_t(mn) * mn;
    x.v_off = vtot;
    vtot += int64_t(x.N) * mn;
    x.u_off = ultot;
    ultot += int64_t(x.M) * mn;
    const bool trans = x.N >= x.M;
    int m = trans ? x.N : x.M, n = trans ? x.M : x.N, lw = 0;
    BST_CUSOLVER(cusolverDnDgesvd_bufferSize(h, m, n, &lw));
    lwork = std::max(lwork, lw);
    maxmn = std::max(maxmn, mn);
  }
  double* dS = (double*)ctx->buf("proj.S", sizeof(double) * std::max<int64_t>(stot, 1), s);
  double* dU = (double*)ctx->buf("proj.U", sizeof(double) * std::max<int64_t>(utot, 1), s);
  double* dVT = (double*)ctx->buf("proj.VT", sizeof(double) * std::max<int64_t>(vt2, 1), s);
  double* dW = (double*)ctx->buf("proj.work", sizeof(double) * std::max(lwork, 1), s);
  double* dR = (double*)ctx->buf("proj.rwork", sizeof(double) * maxmn, s);
  double* dX = (double*)ctx->buf("proj.X", sizeof(double) * std::max<int64_t>(cmat, 1), s);
  dV = (double*)ctx->buf("proj.V2", sizeof(double) * std::max<int64_t>(vtot, 1), s);
  dUl = (double*)ctx->buf("proj.Ul", sizeof(double) * std::max<int64_t>(ultot, 1), s);
  int* dInfo = (int*)ctx->buf("proj.info", sizeof(int) * secs.size(), s);
  BST_CUDA(cudaMemsetAsync(dInfo, 0, sizeof(int) * secs.size(), s));
  {
    ProfScope ps_svd(ctx, s, "svd_cusolver", 0.0, 0.0);
    for (size_t i = 0; i < secs.size(); ++i) {
      auto& x = secs[i];
      const int mn = x.c;
      double* Y = dX + x.cs->off;
      if (x.N >= x.M) {
        // row-major N_s [M x N] is col-major X = N_s^T [N x M]; X = Ux S VTx,
        // right vectors of N_s = columns of Ux
        BST_CUDA(cudaMemcpyAsync(Y, Nm + x.cs->off, sizeof(double) * int64_t(x.M) * x.N, cudaMemcpyDeviceToDevice, s));
        BST_CUSOLVER(cusolverDnDgesvd(h, 'S', 'S', x.N, x.M, Y, x.N, dS + x.s_off, dU + u_off[i], x.N,
                                      dVT + vt_off[i], mn, dW, lwork, dR, dInfo + i));
        // V (row-major N x mn) from col-major Ux (N x mn): V[r][j] = Ux[r + j N];
        // the left vectors of N_s are the rows of VTx: U[r][j] = VTx[j + r mn],
        // the same memory order as row-major M x mn
        launch_transpose(dU + u_off[i], dV + x.v_off, mn, x.N, s);
        BST_CUDA(cudaMemcpyAsync(dUl + x.u_off, dVT + vt_off[i], sizeof(double) * int64_t(x.M) * mn,
                                 cudaMemcpyDeviceToDevice, s));
      } else {
        // col-major Y = N_s [M x N]; Y = Uy S VTy, right vectors = rows of VTy
        launch_transpose(Nm + x.cs->off, Y, x.M, x.N, s);
        BST_CUSOLVER(cusolverDnDgesvd(h, 'S', 'S', x.M, x.N, Y, x.M, dS + x.s_off, dU + u_off[i], x.M,
                                      dVT + vt_off[i], mn, dW, lwork, dR, dInfo + i));
        // V[r][j] = VTy[j + r mn]: the same memory order; U (row-major
        // M x mn) from col-major Uy (M x mn)
        BST_CUDA(cudaMemcpyAsync(dV + x.v_off, dVT + vt_off[i], sizeof(double) * int64_t(x.N) * mn,
                                 cudaMemcpyDeviceToDevice, s));
        launch_transpose(dU + u_off[i], dUl + x.u_off, mn, x.M, s);
      }
      count_launch(ctx, 2);
    }
  }
  hSig.assign(stot, 0.0);
  std::vector<int> hInfo(secs.size());
  BST_CUDA(cudaMemcpyAsync(hSig.data(), dS, sizeof(double) * stot, cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaMemcpyAsync(hInfo.data(), dInfo, sizeof(int) * secs.size(), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  for (int v : hInfo) BST_REQUIRE(v == 0, BST_E_NUMERIC, "projector: gesvd did not converge");
}

// Batched symmetric eigendecomposition of `batch` n x n matrices (n <= 160),
// row-major, back to back; eigenvalues descending.
void sym_eig_batched(Ctx* ctx, int n, int batch, const double* H, double* X, double* lam, bst_prec prec,
                     cudaStream_t s) {
  BST_REQUIRE(n >= 1 && n <= kEigMax && batch >= 1, BST_E_ARG, "sym_eig: n must be 1..160");
  std::vector<SmallProb> sp;
  for (int i = 0; i < batch; ++i) sp.push_back({n, 0, int64_t(i) * n * n, int64_t(i) * n * n, int64_t(i) * n});
  small_eig(ctx, prec, sp, H, X, lam, int64_t(batch) * n * n, int64_t(batch) * n, s);
}

ProjResult svd_projector(Ctx* ctx, Layout* Rt, const double* rt, Layout* Rb, const double* rb, int ncut,
                         int64_t chi, double rel_cutoff, int new_flow, bst_prec prec, double* p, double* pt,
                         cudaStream_t s) {
  // the subspace iterations and eigensolver resolve singular values far
  // below the largest: the cheaper three-slice arithmetic does not reach
  // them, so the projector runs in the five-slice one
  if (prec == BST_BF16X3) prec = BST_OZAKI;
  BST_REQUIRE(ncut >= 1 && ncut < Rt->rank && ncut < Rb->rank, BST_E_ARG, "bad ncut");
  BST_REQUIRE(chi >= 1, BST_E_ARG, "chi must be positive");
  BST_REQUIRE(new_flow == 1 || new_flow == -1, BST_E_ARG, "new_flow must be +1 or -1");
  std::vector<int> cut(ncut);
  std::iota(cut.begin(), cut.end(), 0);
  ContractPlan* pn = get_contract_plan(ctx, Rt, Rb, cut, cut);
  // Rt and Rb as sector matrices (kept for P and Pt below), and
  // N = Rt^T Rb (rows: right cut of Rt, cols: right cut of Rb); the
  // tensor-core product reads Rt's and Rb's blocks itself
  double* At = (double*)ctx->buf("proj.A", sizeof(double) * std::max<int64_t>(pn->amat, 1), s);  // [beta x alpha]
  double* Bt = (double*)ctx->buf("proj.B", sizeof(double) * std::max<int64_t>(pn->bmat, 1), s);  // [beta' x alpha']
  launch_relayout(ctx, pn->ra, rt, At, 0, 1.0, 0.0, s);
  launch_relayout(ctx, pn->rb, rb, Bt, 0, 1.0, 0.0, s);
  double* Nm = (double*)ctx->buf("contract.Ckeep", sizeof(double) * std::max<int64_t>(pn->cmat, 1), s);
  ctx->work_flops += pn->g.flops;
  if (prec == BST_FP64) launch_gemm_f64(ctx, pn->g, At, Bt, Nm, s);
  else run_gemm_ozaki(ctx, pn, ozaki_slices(prec), rt, rb, Nm, s, At, Bt);

  std::vector<PSec> secs;
  for (auto& cs : pn->vc.secs) {
    const MatSector* as = pn->va.find(cs.key);
    const MatSector* bs = pn->vb.find(cnorm(Rt->group, -cs.key));
    if (!as || !bs || as->cols == 0 || cs.rows == 0 || cs.cols == 0) continue;
    PSec x{};
    x.cs = &cs;
    x.as = as;
    x.bs = bs;
    x.M = int(cs.rows);
    x.N = int(cs.cols);
    secs.push_back(x);
  }
  BST_REQUIRE(!secs.empty(), BST_E_NUMERIC, "projector: no non-empty sector");
  // normalise N (Frobenius) so every later stage, FP32 ones included, works
  // on O(1) numbers; singular values are scaled back below
  double* dss = (double*)ctx->buf("proj.nss", sizeof(double), s);
  launch_sumsq(ctx, Nm, pn->cmat, dss, s);
  launch_scale(ctx, Nm, pn->cmat, dss, s);
  double* dV = nullptr;
  double* dUl = nullptr;  // left vectors of the full SVD (gesvd path)
  std::vector<double> hSig;
  double nscale = 0;
  struct Cand { double sv; int q; int sec; int j; };
  std::vector<int> kcount;
  int64_t kept = 0;
  double kept_sum = 0, kmin = 0, smax = 0, ssum = 0;
  // The subspace method computes the leading candidates of every sector; if
  // the global truncation keeps states up to the edge of some sector's
  // iterated block (fewer than 16 guard vectors left), that sector may need
  // more candidates than were computed: the projector is redone with the
  // full FP64 SVD.
  bool use_subspace = ctx->proj_method == 1;
  bool from_subspace = false;  // the candidates come from factors_subspace
  for (int attempt = 0; attempt < 2; ++attempt) {
    bool done = false;
    if (use_subspace) {
      ProfScope ps(ctx, s, "proj_subspace", 0.0, 0.0);
      done = factors_subspace(ctx, Nm, secs, chi, prec, ctx->proj_iters, dV, hSig, s);
    }
    if (!done) factors_gesvd(ctx, Nm, pn->cmat, secs, dV, dUl, hSig, s);
    from_subspace = done;
    if (attempt == 0) {
      double nss = 0;
      BST_CUDA(cudaMemcpy(&nss, dss, sizeof(double), cudaMemcpyDeviceToHost));
      nscale = std::sqrt(nss);
      BST_REQUIRE(std::isfinite(nscale) && nscale > 0, BST_E_NUMERIC, "projector: N is zero or not finite");
    }
    // per sector descending order of the candidates (refinement may swap
    // values that agree to rounding); the vectors are permuted to match
    {
      std::vector<int> perm_all;
      std::vector<int64_t> ptask;
      bool any = false;
      for (auto& x : secs) {
        std::vector<int> ord(x.c);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return hSig[x.s_off + a] > hSig[x.s_off + b]; });
        for (int j = 0; j < x.c; ++j) any |= ord[j] != j;
        std::vector<double> tmp(x.c);
        for (int j = 0; j < x.c; ++j) tmp[j] = hSig[x.s_off + ord[j]];
        for (int j = 0; j < x.c; ++j) hSig[x.s_off + j] = tmp[j];
        perm_all.insert(perm_all.end(), ord.begin(), ord.end());
      }
      if (any) {
        int64_t vtot = 0, po = 0;
        for (auto& x : secs) vtot = std::max(vtot, x.v_off + int64_t(x.N) * x.c);
        double* tmpv = (double*)ctx->buf("proj.Vperm", sizeof(double) * std::max<int64_t>(vtot, 1), s);
        int* dperm = upload_cached(ctx, "proj.perm", perm_all, s);
        for (auto& x : secs) {
          permute_cols<<<x.N, 128, 0, s>>>(dV + x.v_off, tmpv + x.v_off, x.c, dperm + po);
          po += x.c;
        }
        BST_CUDA(cudaMemcpyAsync(dV, tmpv, sizeof(double) * vtot, cudaMemcpyDeviceToDevice, s));
        count_launch(ctx, int(secs.size()));
        if (!done) {
          // the full SVD's left vectors follow
          int64_t utot = 0;
          for (auto& x : secs) utot = std::max(utot, x.u_off + int64_t(x.M) * x.c);
          double* tmpu = (double*)ctx->buf("proj.Uperm", sizeof(double) * std::max<int64_t>(utot, 1), s);
          po = 0;
          for (auto& x : secs) {
            permute_cols<<<x.M, 128, 0, s>>>(dUl + x.u_off, tmpu + x.u_off, x.c, dperm + po);
            po += x.c;
          }
          BST_CUDA(cudaMemcpyAsync(dUl, tmpu, sizeof(double) * utot, cudaMemcpyDeviceToDevice, s));
          count_launch(ctx, int(secs.size()));
        }
        if (done) {
          // the Rayleigh-Ritz vectors W of the iterated sectors follow V
          // (V = Q W), so that N V = (N Q) W column by column below
          int64_t wtot = 0;
          for (auto& x : secs) wtot = std::max(wtot, x.sm_off + int64_t(x.b) * x.b);
          double* Xv = (double*)ctx->buf("proj.X2", sizeof(double), s);
          double* tmpw = (double*)ctx->buf("proj.Wperm", sizeof(double) * std::max<int64_t>(wtot, 1), s);
          po = 0;
          int nw = 0;
          for (auto& x : secs) {
            if (!x.direct) {
              permute_cols<<<x.b, 128, 0, s>>>(Xv + x.sm_off, tmpw + x.sm_off, x.c, dperm + po);
              BST_CUDA(cudaMemcpyAsync(Xv + x.sm_off, tmpw + x.sm_off, sizeof(double) * int64_t(x.b) * x.b,
                                       cudaMemcpyDeviceToDevice, s));
              ++nw;
            }
            po += x.c;
          }
          count_launch(ctx, nw);
        }
      }
    }

    // global truncation: sigma descending, |q| ascending, q ascending
    std::vector<Cand> cand;
    smax = 0;
    ssum = 0;
    for (size_t i = 0; i < secs.size(); ++i)
      for (int j = 0; j < secs[i].c; ++j) {
        const double v = hSig[secs[i].s_off + j];
        BST_REQUIRE(std::isfinite(v), BST_E_NUMERIC, "projector: non-finite singular value");
        cand.push_back({v, int(cnorm(Rt->group, new_flow * secs[i].cs->key)), int(i), j});
        smax = std::max(smax, v);
        ssum += v;
      }
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
      if (a.sv != b.sv) return a.sv > b.sv;
      if (std::abs(a.q) != std::abs(b.q)) return std::abs(a.q) < std::abs(b.q);
      if (a.q != b.q) return a.q < b.q;
      return a.j < b.j;
    });
    kcount.assign(secs.size(), 0);
    kept = 0;
    kept_sum = 0;
    kmin = smax;
    for (auto& c : cand) {
      if (kept >= chi) break;
      if (!(c.sv > rel_cutoff * smax) || c.sv <= 0) break;
      kcount[c.sec]++;
      kept++;
      kept_sum += c.sv;
      kmin = std::min(kmin, c.sv);
    }
    BST_REQUIRE(kept > 0, BST_E_NUMERIC, "projector: nothing above the cutoff");
    for (size_t i = 0; i < secs.size(); ++i)
      for (int j = 1; j < kcount[i]; ++j)
        BST_REQUIRE(hSig[secs[i].s_off + j] <= hSig[secs[i].s_off + j - 1], BST_E_NUMERIC, "projector: unsorted");
    bool edge = false;
    if (done)
      for (size_t i = 0; i < secs.size(); ++i)
        edge = edge || (!secs[i].direct && kcount[i] + 16 > secs[i].c) || cut_unresolved(secs[i], hSig, kmin);
    if (!edge) break;
    if (ctx->tune_log.size() < (1u << 20))
      ctx->tune_log += "projector: truncation outside the resolved candidates, full SVD\n";
    use_subspace = false;
  }

  std::vector<std::pair<int, int>> order;  // (charge, sec)
  for (size_t i = 0; i < secs.size(); ++i)
    if (kcount[i] > 0) order.push_back({int(cnorm(Rt->group, new_flow * secs[i].cs->key)), int(i)});
  std::sort(order.begin(), order.end());
  Leg nl;
  nl.flow = new_flow;
  ProjResult res;
  for (auto& o : order) {
    nl.q.push_back(o.first);
    nl.d.push_back(kcount[o.second]);
    for (int j = 0; j < kcount[o.second]; ++j) res.svals.push_back(hSig[secs[o.second].s_off + j] * nscale);
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

  // kept sigma on the device, left vectors U = N V / sigma, gauge, scale
  int64_t us_tot = 0, vs_tot = 0, sk_tot = 0;
  std::vector<int64_t> sk_off(secs.size()), ur_off(secs.size());
  for (size_t i = 0; i < secs.size(); ++i) {
    sk_off[i] = sk_tot;
    sk_tot += kcount[i];
    ur_off[i] = us_tot;
    us_tot += int64_t(secs[i].M) * kcount[i];
    vs_tot += int64_t(secs[i].N) * kcount[i];
  }
  std::vector<double> hsk(std::max<int64_t>(sk_tot, 1));
  for (size_t i = 0; i < secs.size(); ++i)
    for (int j = 0; j < kcount[i]; ++j) hsk[sk_off[i] + j] = hSig[secs[i].s_off + j];
  double* dSk = upload_cached(ctx, "proj.sk", hsk, s);
  double* Ur = (double*)ctx->buf("proj.Ur", sizeof(double) * std::max<int64_t>(us_tot, 1), s);
  double* Us = (double*)ctx->buf("proj.Us", sizeof(double) * std::max<int64_t>(us_tot, 1), s);
  double* Vs = (double*)ctx->buf("proj.Vs", sizeof(double) * std::max<int64_t>(vs_tot, 1), s);
  double* Pm = (double*)ctx->buf("proj.Pm", sizeof(double) * std::max<int64_t>(vp->mv.total, 1), s);
  double* Ptm = (double*)ctx->buf("proj.Ptm", sizeof(double) * std::max<int64_t>(vpt->mv.total, 1), s);
  BST_CUDA(cudaMemsetAsync(Pm, 0, sizeof(double) * std::max<int64_t>(vp->mv.total, 1), s));
  BST_CUDA(cudaMemsetAsync(Ptm, 0, sizeof(double) * std::max<int64_t>(vpt->mv.total, 1), s));
  std::vector<GemmProb> gu, guz, gpp, gpt;
  for (size_t i = 0; i < secs.size(); ++i) {
    const int k = kcount[i];
    if (k == 0) continue;
    const PSec& x = secs[i];
    // Ur = N V_k  ([M x k]; V row-major N x c), in FP64 (see
    // factors_subspace); for an iterated sector N V = (N Q) W with N Q the
    // final Rayleigh-Ritz product, still in its buffer: M x k x b in place
    // of M x k x N
    if (x.u_off >= 0) continue;  // the full SVD gave the left vectors
    if (from_subspace && !x.direct)
      guz.push_back(gp(x.M, k, x.b, x.z_off, x.b, 1, x.sm_off, 1, x.b, ur_off[i], k, 1));
    else
      gu.push_back(gp(x.M, k, x.N, x.cs->off, x.N, 1, x.v_off, 1, x.c, ur_off[i], k, 1));
  }
  gemm_any(ctx, "proj.u", BST_FP64, gu, Nm, dV, Ur, s);
  gemm_any(ctx, "proj.uz", BST_FP64, guz, (const double*)ctx->buf("proj.Z", sizeof(double), s),
           (const double*)ctx->buf("proj.X2", sizeof(double), s), Ur, s);
  int64_t uo = 0, vo = 0;
  for (size_t i = 0; i < secs.size(); ++i) {
    const PSec& x = secs[i];
    const int k = kcount[i];
    if (k == 0) continue;
    // left vectors: those of the full SVD (consistent with its right
    // vectors to the SVD's own backward error), else u = N v / sigma
    if (x.u_off >= 0)
      gauge_scale_kernel<<<k, 256, 0, s>>>(dUl + x.u_off, x.c, 1, x.M, dV + x.v_off, x.c, 1, x.N, dSk + sk_off[i],
                                           k, Us + uo, Vs + vo, 0, nscale);
    else
      gauge_scale_kernel<<<k, 256, 0, s>>>(Ur + ur_off[i], k, 1, x.M, dV + x.v_off, x.c, 1, x.N, dSk + sk_off[i],
                                           k, Us + uo, Vs + vo, 1, nscale);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
    const int key = int(x.cs->key);
    const MatSector* ps = vp->mv.find(key);
    const MatSector* pts = vpt->mv.find(key);
    BST_REQUIRE(ps && pts && ps->cols == k && pts->rows == k, BST_E_SHAPE, "projector: view mismatch");
    BST_REQUIRE(ps->rows == x.bs->cols && pts->cols == x.as->cols, BST_E_SHAPE, "projector: cut mismatch");
    // P_s[a', j] = sum_b' Rb[a', b'] V~[b', j], Rb^T stored as Bmat [b' x a']
    gpp.push_back(gp(int(ps->rows), k, x.N, x.bs->off, 1, x.bs->cols, vo, 1, k, ps->off, k, 1));
    // Pt_s[j, a] = sum_b U~[b, j] Rt[a, b], Rt^T stored as Amat [b x a]
    gpt.push_back(gp(k, int(pts->cols), x.M, uo, 1, k, x.as->off, 1, x.as->cols, pts->off, pts->cols, 1));
    uo += int64_t(x.M) * k;
    vo += int64_t(x.N) * k;
  }
  for (auto* v : {&gpp, &gpt})
    for (auto& g : *v) ctx->work_flops += 2.0 * double(g.M) * g.N * g.K;
  gemm_any(ctx, "proj.P", prec, gpp, Bt, Vs, Pm, s);
  gemm_any(ctx, "proj.Pt", prec, gpt, Us, At, Ptm, s);
  launch_relayout(ctx, vp->rel, p, Pm, 1, 1.0, 0.0, s);
  launch_relayout(ctx, vpt->rel, pt, Ptm, 1, 1.0, 0.0, s);
  return res;
}

// ---------------------------------------------------------------------------
// SU(2) projector
//
// N = Rt^T Rb over the left cut, computed by the SU(2) contraction, has its
// right-cut legs of Rt (beta) outgoing and those of Rb (beta') incoming, so
// its canonical blocks are already in matrix form: the CGC of a block is
// sum_M <beta'-tree|J M><beta-tree|J M>, and N is the direct sum over the
// coupled spin J of reduced matrices N_J (rows: beta sector tuples with their
// tree intermediates and reduced indices; columns: the same for beta') times
// a projector of rank 2J+1.  The singular values of N are those of the N_J,
// each 2J+1 times; the singular vectors are the reduced ones times the
// coupled states (Sec. 2: SU(2) blocks store reduced tensors only).
//   * per J: the same leading-pair solvers as U(1) (subspace iteration or
//     gesvd);
//   * truncation by whole multiplets: by descending sigma (ties: smaller J,
//     then index), a multiplet is kept while the kept total dimension
//     sum (2J+1) stays <= chi_total; one that would overflow is skipped, so no
//     multiplet is cut;
//   * V[beta'^dual..., new] and Ut[new^dual, beta^dual...] are SU(2) tensors
//     whose reduced blocks are the gauge-fixed V_J S^-1/2 and (U_J S^-1/2)^T
//     (their CGC tensors are exactly the coupled states above), and
//     P = Rb . V, Pt = Ut . Rt by the SU(2) contraction.
ProjResult su2_projector(Ctx* ctx, Layout* Rt, const double* rt, Layout* Rb, const double* rb, int ncut,
                         int64_t chi_total, double rel_cutoff, bst_prec prec, double** p_out, double** pt_out,
                         cudaStream_t s) {
  BST_REQUIRE(Rt->group == BST_SU2 && Rb->group == BST_SU2, BST_E_ARG, "SU(2) projector needs SU(2) tensors");
  if (prec == BST_BF16X3) prec = BST_OZAKI;  // as for U(1)
  BST_REQUIRE(ncut >= 1 && ncut < Rt->rank && ncut < Rb->rank, BST_E_ARG, "bad ncut");
  BST_REQUIRE(chi_total >= 1, BST_E_ARG, "chi must be positive");
  std::vector<int> cut(ncut);
  std::iota(cut.begin(), cut.end(), 0);
  Layout* LN = su2_contract_layout(ctx, Rt, Rb, cut, cut);
  const int nb = Rt->rank - ncut, nbp = Rb->rank - ncut;
  for (int i = 0; i < nb; ++i)
    BST_REQUIRE(LN->legs[i].flow == -1, BST_E_UNSUPPORTED, "SU(2) projector: Rt's right-cut legs must be outgoing");
  for (int i = 0; i < nbp; ++i)
    BST_REQUIRE(LN->legs[nb + i].flow == 1, BST_E_UNSUPPORTED,
                "SU(2) projector: Rb's right-cut legs must be incoming");
  double* Nd = (double*)ctx->buf("su2p.N", sizeof(double) * std::max<int64_t>(LN->nnz, 1), s);
  su2_contract(ctx, Rt, rt, Rb, rb, cut, cut, prec, 1.0, 0.0, LN, Nd, s);

  // matrix view of N per J; labels = [beta' intermediates, J, beta intermediates]
  const int nin_inter = std::max(nbp - 2, 0);
  std::map<int, std::map<std::vector<int32_t>, int64_t>> rows, cols;  // J -> config -> extent
  auto cfg_of = [&](int64_t b, bool row) {
    std::vector<int32_t> k;
    const int32_t* sc = &LN->sect[b * LN->rank];
    const int32_t* lb = &LN->tree[b * LN->ntree];
    if (row) {
      for (int i = 0; i < nb; ++i) k.push_back(sc[i]);
      for (int i = nin_inter + 1; i < LN->ntree; ++i) k.push_back(lb[i]);
    } else {
      for (int i = 0; i < nbp; ++i) k.push_back(sc[nb + i]);
      for (int i = 0; i < nin_inter; ++i) k.push_back(lb[i]);
    }
    return k;
  };
  auto extent = [&](int64_t b, int first, int n) {
    int64_t e = 1;
    for (int i = first; i < first + n; ++i) e *= LN->shape[b * LN->rank + i];
    return e;
  };
  for (int64_t b = 0; b < LN->nblocks; ++b) {
    const int J = LN->tree[b * LN->ntree + nin_inter];
    rows[J][cfg_of(b, true)] = extent(b, 0, nb);
    cols[J][cfg_of(b, false)] = extent(b, nb, nbp);
  }
  std::vector<MatSector> msec;
  std::map<int, std::map<std::vector<int32_t>, int64_t>> roff, coff;
  int64_t ntot = 0;
  for (auto& kv : rows) {
    MatSector m;
    m.key = kv.first;
    for (auto& r : kv.second) roff[kv.first][r.first] = m.rows, m.rows += r.second;
    for (auto& c : cols[kv.first]) coff[kv.first][c.first] = m.cols, m.cols += c.second;
    m.off = ntot;
    ntot += m.rows * m.cols;
    msec.push_back(std::move(m));
  }
  std::map<int, int> sec_of_J;
  for (size_t i = 0; i < msec.size(); ++i) sec_of_J[int(msec[i].key)] = int(i);
  const std::string rkey = "su2p/view/" + std::to_string(LN->id);
  DevRelayout* rel = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->rplans.find(rkey);
    if (it != ctx->rplans.end()) rel = it->second.get();
  }
  if (!rel) {
    std::vector<RelTask> tasks;
    for (int64_t b = 0; b < LN->nblocks; ++b) {
      const int J = LN->tree[b * LN->ntree + nin_inter];
      const MatSector& m = msec[sec_of_J[J]];
      RelTask t{};
      t.blk_off = LN->offset[b];
      t.mat_base = m.off + roff[J][cfg_of(b, true)] * m.cols + coff[J][cfg_of(b, false)];
      t.rank = LN->rank;
      int64_t n = 1;
      for (int i = 0; i < LN->rank; ++i) {
        t.shape[i] = int32_t(LN->shape[b * LN->rank + i]);
        n *= t.shape[i];
      }
      t.n = int32_t(n);
      int64_t st = m.cols;
      for (int i = nb - 1; i >= 0; --i) t.mstride[i] = st, st *= t.shape[i];
      st = 1;
      for (int i = nb + nbp - 1; i >= nb; --i) t.mstride[i] = st, st *= t.shape[i];
      if (n > 0) tasks.push_back(t);
    }
    auto r = std::make_unique<DevRelayout>();
    r->upload(tasks);
    rel = r.get();
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->rplans[rkey] = std::move(r);
  }
  double* Nm = (double*)ctx->buf("su2p.Nm", sizeof(double) * std::max<int64_t>(ntot, 1), s);
  launch_relayout(ctx, *rel, Nd, Nm, 0, 1.0, 0.0, s);
  double* dss = (double*)ctx->buf("proj.nss", sizeof(double), s);
  launch_sumsq(ctx, Nm, ntot, dss, s);
  launch_scale(ctx, Nm, ntot, dss, s);

  std::vector<PSec> secs;
  for (auto& m : msec) {
    if (m.rows == 0 || m.cols == 0) continue;
    PSec x{};
    x.cs = &m;
    x.M = int(m.rows);
    x.N = int(m.cols);
    x.kmax = std::max<int64_t>(1, chi_total / (int64_t(m.key) + 1));  // a multiplet of spin J counts 2J+1
    secs.push_back(x);
  }
  BST_REQUIRE(!secs.empty(), BST_E_NUMERIC, "projector: no non-empty sector");
  double* dV = nullptr;
  std::vector<double> hSig;
  double* dUl = nullptr;
  double nscale = 0, smax = 0, kmin = 0;
  std::vector<int> kcount;
  int64_t kept_dim = 0, kept = 0;
  bool use_subspace = ctx->proj_method == 1;
  for (int attempt = 0; attempt < 2; ++attempt) {
    bool done = false;
    if (use_subspace) {
      ProfScope ps(ctx, s, "proj_subspace", 0.0, 0.0);
      // whole multiplets are kept while they fit, so a value below the
      // chi-th largest may still be kept: no sector is skipped
      done = factors_subspace(ctx, Nm, secs, chi_total, prec, ctx->proj_iters, dV, hSig, s, false);
    }
    if (!done) factors_gesvd(ctx, Nm, ntot, secs, dV, dUl, hSig, s);
    if (attempt == 0) {
      double nss = 0;
      BST_CUDA(cudaMemcpy(&nss, dss, sizeof(double), cudaMemcpyDeviceToHost));
      nscale = std::sqrt(nss);
      BST_REQUIRE(std::isfinite(nscale) && nscale > 0, BST_E_NUMERIC, "projector: N is zero or not finite");
    }
    // candidates in descending order per sector (host sort; vectors follow)
    std::vector<int> perm_all;
    bool any = false;
    for (auto& x : secs) {
      std::vector<int> ord(x.c);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hSig[x.s_off + a] > hSig[x.s_off + b]; });
      std::vector<double> tmp(x.c);
      for (int j = 0; j < x.c; ++j) tmp[j] = hSig[x.s_off + ord[j]], any |= ord[j] != j;
      for (int j = 0; j < x.c; ++j) hSig[x.s_off + j] = tmp[j];
      perm_all.insert(perm_all.end(), ord.begin(), ord.end());
    }
    if (any) {
      int64_t vtot = 0, po = 0;
      for (auto& x : secs) vtot = std::max(vtot, x.v_off + int64_t(x.N) * x.c);
      double* tmpv = (double*)ctx->buf("proj.Vperm", sizeof(double) * std::max<int64_t>(vtot, 1), s);
      int* dperm = upload_cached(ctx, "proj.perm", perm_all, s);
      for (auto& x : secs) {
        permute_cols<<<x.N, 128, 0, s>>>(dV + x.v_off, tmpv + x.v_off, x.c, dperm + po);
        po += x.c;
      }
      BST_CUDA(cudaMemcpyAsync(dV, tmpv, sizeof(double) * vtot, cudaMemcpyDeviceToDevice, s));
      count_launch(ctx, int(secs.size()));
      if (!done) {
        int64_t utot = 0;
        for (auto& x : secs) utot = std::max(utot, x.u_off + int64_t(x.M) * x.c);
        double* tmpu = (double*)ctx->buf("proj.Uperm", sizeof(double) * std::max<int64_t>(utot, 1), s);
        po = 0;
        for (auto& x : secs) {
          permute_cols<<<x.M, 128, 0, s>>>(dUl + x.u_off, tmpu + x.u_off, x.c, dperm + po);
          po += x.c;
        }
        BST_CUDA(cudaMemcpyAsync(dUl, tmpu, sizeof(double) * utot, cudaMemcpyDeviceToDevice, s));
        count_launch(ctx, int(secs.size()));
      }
    }
    struct Cand { double sv; int tJ; int sec; int j; };
    std::vector<Cand> cand;
    smax = 0;
    for (size_t i = 0; i < secs.size(); ++i)
      for (int j = 0; j < secs[i].c; ++j) {
        const double v = hSig[secs[i].s_off + j];
        BST_REQUIRE(std::isfinite(v), BST_E_NUMERIC, "projector: non-finite singular value");
        cand.push_back({v, int(secs[i].cs->key), int(i), j});
        smax = std::max(smax, v);
      }
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
      if (a.sv != b.sv) return a.sv > b.sv;
      if (a.tJ != b.tJ) return a.tJ < b.tJ;
      return a.j < b.j;
    });
    kcount.assign(secs.size(), 0);
    kept_dim = kept = 0;
    kmin = smax;
    for (auto& c : cand) {
      if (!(c.sv > rel_cutoff * smax) || c.sv <= 0) break;
      if (c.j != kcount[c.sec]) continue;  // an earlier multiplet of this sector was skipped
      if (kept_dim + c.tJ + 1 > chi_total) continue;
      kcount[c.sec]++;
      kept++;
      kept_dim += c.tJ + 1;
      kmin = std::min(kmin, c.sv);
    }
    BST_REQUIRE(kept > 0, BST_E_NUMERIC, "projector: nothing kept");
    bool edge = false;
    if (done)
      for (size_t i = 0; i < secs.size(); ++i)
        edge = edge || (!secs[i].direct && kcount[i] + 16 > secs[i].c) || cut_unresolved(secs[i], hSig, kmin);
    if (!edge) break;
    use_subspace = false;
  }

  // new leg (incoming on P): sectors J with kept multiplets
  Leg nl;
  nl.flow = 1;
  ProjResult res;
  std::map<int, int> kJ;  // J -> sector index in secs
  for (size_t i = 0; i < secs.size(); ++i)
    if (kcount[i] > 0) kJ[int(secs[i].cs->key)] = int(i);
  for (auto& kv : kJ) {
    nl.q.push_back(kv.first);
    nl.d.push_back(kcount[kv.second]);
    for (int j = 0; j < kcount[kv.second]; ++j) res.svals.push_back(hSig[secs[kv.second].s_off + j] * nscale);
  }
  nl.finish();
  res.newleg = nl;
  res.kept = kept_dim;
  res.smin_over_smax = kmin / smax;

  // gauge-fixed, scaled vectors per sector: Us [M x k], Vs [N x k]
  int64_t us_tot = 0, vs_tot = 0, sk_tot = 0;
  std::vector<int64_t> sk_off(secs.size()), ur_off(secs.size()), vs_off(secs.size());
  for (size_t i = 0; i < secs.size(); ++i) {
    sk_off[i] = sk_tot;
    sk_tot += kcount[i];
    ur_off[i] = us_tot;
    us_tot += int64_t(secs[i].M) * kcount[i];
    vs_off[i] = vs_tot;
    vs_tot += int64_t(secs[i].N) * kcount[i];
  }
  std::vector<double> hsk(std::max<int64_t>(sk_tot, 1));
  for (size_t i = 0; i < secs.size(); ++i)
    for (int j = 0; j < kcount[i]; ++j) hsk[sk_off[i] + j] = hSig[secs[i].s_off + j];
  double* dSk = upload_cached(ctx, "proj.sk", hsk, s);
  double* Ur = (double*)ctx->buf("proj.Ur", sizeof(double) * std::max<int64_t>(us_tot, 1), s);
  double* Us = (double*)ctx->buf("proj.Us", sizeof(double) * std::max<int64_t>(us_tot, 1), s);
  double* Vs = (double*)ctx->buf("proj.Vs", sizeof(double) * std::max<int64_t>(vs_tot, 1), s);
  std::vector<GemmProb> gu;
  for (size_t i = 0; i < secs.size(); ++i) {
    const int k = kcount[i];
    if (k == 0) continue;
    const PSec& x = secs[i];
    if (x.u_off >= 0) continue;  // the full SVD gave the left vectors
    gu.push_back(gp(x.M, k, x.N, x.cs->off, x.N, 1, x.v_off, 1, x.c, ur_off[i], k, 1));
  }
  gemm_any(ctx, "proj.u", BST_FP64, gu, Nm, dV, Ur, s);
  for (size_t i = 0; i < secs.size(); ++i) {
    const PSec& x = secs[i];
    const int k = kcount[i];
    if (k == 0) continue;
    if (x.u_off >= 0)
      gauge_scale_kernel<<<k, 256, 0, s>>>(dUl + x.u_off, x.c, 1, x.M, dV + x.v_off, x.c, 1, x.N, dSk + sk_off[i],
                                           k, Us + ur_off[i], Vs + vs_off[i], 0, nscale);
    else
      gauge_scale_kernel<<<k, 256, 0, s>>>(Ur + ur_off[i], k, 1, x.M, dV + x.v_off, x.c, 1, x.N, dSk + sk_off[i],
                                           k, Us + ur_off[i], Vs + vs_off[i], 1, nscale);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx);
  }

  // V[beta'^dual..., new] and Ut[new^dual, beta^dual...]
  std::vector<Leg> vl, ul{nl.dual()};
  for (int i = 0; i < nbp; ++i) vl.push_back(LN->legs[nb + i].dual());
  vl.push_back(nl);
  for (int i = 0; i < nb; ++i) ul.push_back(LN->legs[i].dual());
  Layout* LV = make_layout(ctx, BST_SU2, vl);
  Layout* LU = make_layout(ctx, BST_SU2, ul);
  std::vector<RelTask> tv, tu;
  // V: labels [J, beta' out-tree intermediates]; block [beta' extents..., k]
  for (int64_t b = 0; b < LV->nblocks; ++b) {
    const int32_t* sc = &LV->sect[b * LV->rank];
    const int32_t* lb = &LV->tree[b * LV->ntree];
    const int J = nl.q[sc[nbp]];
    const int si = kJ.at(J);
    std::vector<int32_t> key(sc, sc + nbp);
    key.insert(key.end(), lb + 1, lb + LV->ntree);
    auto it = coff[J].find(key);
    BST_REQUIRE(it != coff[J].end(), BST_E_SHAPE, "SU(2) projector: V block without a column of N");
    const int k = kcount[si];
    RelTask t{};
    t.blk_off = LV->offset[b];
    t.mat_base = vs_off[si] + it->second * k;
    t.rank = LV->rank;
    int64_t n = 1;
    for (int i = 0; i < LV->rank; ++i) t.shape[i] = int32_t(LV->shape[b * LV->rank + i]), n *= t.shape[i];
    t.n = int32_t(n);
    t.mstride[nbp] = 1;
    int64_t st = k;
    for (int i = nbp - 1; i >= 0; --i) t.mstride[i] = st, st *= t.shape[i];
    tv.push_back(t);
  }
  // Ut: labels [beta in-tree intermediates, J]; block [k, beta extents...]
  for (int64_t b = 0; b < LU->nblocks; ++b) {
    const int32_t* sc = &LU->sect[b * LU->rank];
    const int32_t* lb = &LU->tree[b * LU->ntree];
    const int J = nl.q[sc[0]];
    const int si = kJ.at(J);
    std::vector<int32_t> key(sc + 1, sc + 1 + nb);
    key.insert(key.end(), lb, lb + LU->ntree - 1);
    auto it = roff[J].find(key);
    BST_REQUIRE(it != roff[J].end(), BST_E_SHAPE, "SU(2) projector: Ut block without a row of N");
    const int k = kcount[si];
    RelTask t{};
    t.blk_off = LU->offset[b];
    t.mat_base = ur_off[si] + it->second * k;
    t.rank = LU->rank;
    int64_t n = 1;
    for (int i = 0; i < LU->rank; ++i) t.shape[i] = int32_t(LU->shape[b * LU->rank + i]), n *= t.shape[i];
    t.n = int32_t(n);
    t.mstride[0] = 1;
    int64_t st = k;
    for (int i = nb; i >= 1; --i) t.mstride[i] = st, st *= t.shape[i];
    tu.push_back(t);
  }
  double* vd = (double*)ctx->buf("su2p.V", sizeof(double) * std::max<int64_t>(LV->nnz, 1), s);
  double* ud = (double*)ctx->buf("su2p.Ut", sizeof(double) * std::max<int64_t>(LU->nnz, 1), s);
  {
    auto& slotv = ctx->rplans["su2p/V/" + std::to_string(LV->id) + "/" + std::to_string(LN->id)];
    if (!slotv) {
      slotv = std::make_unique<DevRelayout>();
      slotv->upload(tv);
    }
    auto& slotu = ctx->rplans["su2p/U/" + std::to_string(LU->id) + "/" + std::to_string(LN->id)];
    if (!slotu) {
      slotu = std::make_unique<DevRelayout>();
      slotu->upload(tu);
    }
    launch_relayout(ctx, *slotv, vd, Vs, 1, 1.0, 0.0, s);
    launch_relayout(ctx, *slotu, ud, Us, 1, 1.0, 0.0, s);
  }
  std::vector<int> lbp(nbp), lvb(nbp), lub(nb), lrt(nb);
  for (int i = 0; i < nbp; ++i) lbp[i] = ncut + i, lvb[i] = i;
  for (int i = 0; i < nb; ++i) lub[i] = 1 + i, lrt[i] = ncut + i;
  res.P = su2_contract_layout(ctx, Rb, LV, lbp, lvb);
  res.Pt = su2_contract_layout(ctx, LU, Rt, lub, lrt);
  retain(res.P);
  retain(res.Pt);
  double* pd = (double*)ctx->buf("su2p.P", sizeof(double) * std::max<int64_t>(res.P->nnz, 1), s);
  double* ptd = (double*)ctx->buf("su2p.Pt", sizeof(double) * std::max<int64_t>(res.Pt->nnz, 1), s);
  su2_contract(ctx, Rb, rb, LV, vd, lbp, lvb, prec, 1.0, 0.0, res.P, pd, s);
  su2_contract(ctx, LU, ud, Rt, rt, lub, lrt, prec, 1.0, 0.0, res.Pt, ptd, s);
  release(LV);
  release(LU);
  *p_out = pd;
  *pt_out = ptd;
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
