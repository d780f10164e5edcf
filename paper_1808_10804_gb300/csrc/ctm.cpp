// Directional CTMRG moves on a one-site cell (Sec. 3 and Sec. 3.2).
//
// A LEFT move absorbs the site column into the left environment column:
//   Q1 = C1 T1 T4 a, Q2 = T1 C2 a T2, Q3 = a T2 T3 C3, Q4 = T4 a C4 T3
//   Rt = Q1 Q2 (top half), Rb = Q4 Q3 (bottom half)
//   projectors P, Pt from the SVD of Rt^T Rb (svd_projector)
//   C1' = (C1 T1) P,  T4' = (Pt T4 a) P,  C4' = Pt (C4 T3),  each normalised.
// Other directions rotate the network by quarter turns (a leg permutation of
// every tensor), run the LEFT move and rotate the renewed tensors back.
//
// Leg directions of the roles: C1[R,D] C2[L,D] C3[U,L] C4[U,R]
// T1[L,D,R] T2[U,L,D] T3[L,U,R] T4[U,R,D], a[L,U,R,D].
#include <algorithm>
#include <array>
#include <cstring>
#include <numeric>
#include <string>

#include "bst_internal.h"

namespace bst {

namespace {

enum Role { C1 = 0, C2, C3, C4, T1, T2, T3, T4, SITE, NROLE };
const char* kDirs[NROLE] = {"RD", "LD", "UL", "UR", "LDR", "ULD", "LUR", "URD", "LURD"};
// one counter-clockwise quarter turn: the tensor at role r moves to kRot[r]
const Role kRot[NROLE] = {C4, C1, C2, C3, T4, T1, T2, T3, SITE};

char rot_dir(char d) {  // direction a leg points to after the turn
  switch (d) {
    case 'U': return 'L';
    case 'L': return 'D';
    case 'D': return 'R';
    default: return 'U';  // 'R'
  }
}

struct Src {
  int role;               // role in the original frame
  std::vector<int> perm;  // rotated leg j = original leg perm[j]
};

// For k quarter turns: where every rotated role comes from.
std::vector<Src> rotation(int k) {
  std::vector<Src> cur(NROLE);
  for (int r = 0; r < NROLE; ++r) {
    cur[r].role = r;
    cur[r].perm.resize(strlen(kDirs[r]));
    std::iota(cur[r].perm.begin(), cur[r].perm.end(), 0);
  }
  for (int t = 0; t < k; ++t) {
    std::vector<Src> nxt(NROLE);
    for (int o = 0; o < NROLE; ++o) {
      const int n = kRot[o];
      const char* od = kDirs[o];
      const char* nd = kDirs[n];
      const int r = int(strlen(nd));
      nxt[n].role = cur[o].role;
      nxt[n].perm.resize(r);
      for (int j = 0; j < r; ++j) {
        int src = -1;
        for (int i = 0; i < r; ++i)
          if (rot_dir(od[i]) == nd[j]) src = i;
        nxt[n].perm[j] = cur[o].perm[src];
      }
    }
    cur = nxt;
  }
  return cur;
}

inline Layout* L_(bst_layout x) { return reinterpret_cast<Layout*>(x); }

bool is_identity(const std::vector<int>& p) {
  for (size_t i = 0; i < p.size(); ++i)
    if (p[i] != int(i)) return false;
  return true;
}

struct T {
  Layout* L;
  const double* d;
};

// c = a.legs(la) * b.legs(lb); result in a named context buffer
T contract(Ctx* ctx, const char* name, T a, T b, std::vector<int> la, std::vector<int> lb, bst_prec prec,
           cudaStream_t s) {
  if (a.L->group == BST_SU2) {
    Layout* C = su2_contract_layout(ctx, a.L, b.L, la, lb);
    double* out = (double*)ctx->buf(name, sizeof(double) * std::max<int64_t>(C->nnz, 1), s);
    su2_contract(ctx, a.L, a.d, b.L, b.d, la, lb, prec, 1.0, 0.0, C, out, s);
    return {C, out};
  }
  ContractPlan* p = get_contract_plan(ctx, a.L, b.L, la, lb);
  double* out = (double*)ctx->buf(name, sizeof(double) * std::max<int64_t>(p->C->nnz, 1), s);
  run_contract(ctx, p, a.d, b.d, prec, 1.0, 0.0, out, s);
  return {p->C, out};
}

// Divide by the Frobenius norm of the full tensor; for SU(2) that is
// sum over blocks of (2J+1) times the squared reduced block (||c||^2 = 2J+1,
// blocks orthogonal).
void normalise(Ctx* ctx, Layout* L, double* x, cudaStream_t s) {
  const int64_t n = L->nnz;
  double* ss = (double*)ctx->buf("ctm.sumsq", sizeof(double), s);
  if (L->group == BST_SU2) {
    DevBuf& wb = ctx->su2_weights[L->id];
    if (!wb.p) {
      int nin = 0;
      for (auto& l : L->legs) nin += l.flow == 1;
      const int jpos = std::max(nin - 2, 0);
      std::vector<double> w(std::max<int64_t>(n, 1), 1.0);
      for (int64_t b = 0; b < L->nblocks; ++b) {
        const int64_t e = b + 1 < L->nblocks ? L->offset[b + 1] : n;
        for (int64_t i = L->offset[b]; i < e; ++i) w[i] = double(L->tree[b * L->ntree + jpos] + 1);
      }
      wb.get(sizeof(double) * w.size(), s);
      BST_CUDA(cudaMemcpy(wb.p, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice));
    }
    launch_sumsq_w(ctx, x, (const double*)wb.p, n, ss, s);
  } else {
    launch_sumsq(ctx, x, n, ss, s);
  }
  launch_scale(ctx, x, n, ss, s);
}

// Contraction with the double layer a = sum_P A (x) A* over X's legs lx[0],
// lx[1] and a's legs la[0], la[1] (directions 0..3 = L, U, R, D); output legs
// [X's other legs, a's two other legs], as contract(X, a, lx, la) gives.
// With the double layer given (rank-4 site) this is that one contraction.
// With a single-layer site A[P, L, U, R, D] (rank 5) a is never formed: X's
// two legs are split into their (ket, bra) parts (the fused double-layer
// leg of direction x is fuse(A.x, A.x^dual), so X's leg is
// fuse(A.x^dual, A.x)), the ket parts are contracted with A, the bra parts
// and P with A* (the dual layout, same data), and the open ket/bra pairs are
// fused again.  Same result up to rounding, fewer FLOPs (Sec. 3.2 forms the
// rank-4 double layer; this is the single-layer variant of the same sum).
T absorb(Ctx* ctx, const std::string& name, T X, std::vector<int> lx, std::vector<int> la, T site,
         Layout* site_dual, bst_prec prec, cudaStream_t s) {
  if (site.L->rank == 4) return contract(ctx, name.c_str(), X, site, lx, la, prec, s);
  Layout* A = site.L;
  const int rx = X.L->rank;
  std::vector<Leg> ul;
  std::vector<int> groups;
  int kpos[2], bpos[2];
  for (int j = 0; j < rx; ++j) {
    const int w = j == lx[0] ? 0 : j == lx[1] ? 1 : -1;
    if (w >= 0) {
      const Leg& sl = A->legs[la[w] + 1];
      kpos[w] = int(ul.size());
      ul.push_back(sl.dual());
      bpos[w] = int(ul.size());
      ul.push_back(sl);
      groups.push_back(2);
    } else {
      ul.push_back(X.L->legs[j]);
      groups.push_back(1);
    }
  }
  Layout* XuL = make_layout(ctx, A->group, ul);
  Layout* fused = nullptr;
  DevRelayout* up = get_fuse_plan(ctx, XuL, groups, &fused);
  release(fused);
  BST_REQUIRE(fused == X.L, BST_E_SHAPE, "edge leg does not match the fused ket/bra legs of the site");
  double* xu = (double*)ctx->buf("sl.Xu", sizeof(double) * std::max<int64_t>(XuL->nnz, 1), s);
  launch_relayout(ctx, *up, xu, const_cast<double*>(X.d), 1, 1.0, 0.0, s);  // split: Xu <- X
  T Xu{XuL, xu};
  T Y = contract(ctx, "sl.Y", Xu, site, {kpos[0], kpos[1]}, {la[0] + 1, la[1] + 1}, prec, s);
  auto ypos = [&](int p) {
    int c = 0;
    for (int q = 0; q < p; ++q) c += (q != kpos[0] && q != kpos[1]);
    return c;
  };
  const int pP = int(ul.size()) - 2;  // A's P leg opens A's part of Y
  T Q = contract(ctx, "sl.Q", Y, T{site_dual, site.d}, {ypos(bpos[0]), ypos(bpos[1]), pP}, {la[0] + 1, la[1] + 1, 0},
                 prec, s);
  // Q = [X's other legs, ket d1, ket d2, bra d1, bra d2] -> pair up and fuse
  const int no = rx - 2;
  std::vector<int> perm;
  for (int i = 0; i < no; ++i) perm.push_back(i);
  for (int i : {no, no + 2, no + 1, no + 3}) perm.push_back(i);
  Layout* QpL = nullptr;
  DevRelayout* pp = get_permute_plan(ctx, Q.L, perm, &QpL);
  double* qp = (double*)ctx->buf("sl.Qp", sizeof(double) * std::max<int64_t>(QpL->nnz, 1), s);
  launch_relayout(ctx, *pp, Q.d, qp, 0, 1.0, 0.0, s);
  std::vector<int> g2(no, 1);
  g2.push_back(2);
  g2.push_back(2);
  Layout* OL = nullptr;
  DevRelayout* fp = get_fuse_plan(ctx, QpL, g2, &OL);
  double* out = (double*)ctx->buf(name, sizeof(double) * std::max<int64_t>(OL->nnz, 1), s);
  launch_relayout(ctx, *fp, qp, out, 0, 1.0, 0.0, s);
  // the intern table keeps the layouts alive
  release(QpL);
  release(OL);
  release(XuL);
  return {OL, out};
}

}  // namespace

static void left_move(Ctx* ctx, T* r, Layout* site_dual, int64_t chi, double cutoff, bst_prec prec, T out[3],
                      ProjResult* pres, cudaStream_t s) {
  T a = r[SITE];
  T X1 = contract(ctx, "ctm.X1", r[C1], r[T1], {0}, {0}, prec, s);        // [C1.D, T1.D, T1.R]
  T X2 = contract(ctx, "ctm.X2", X1, r[T4], {0}, {0}, prec, s);           // [T1.D, T1.R, T4.R, T4.D]
  T Q1 = absorb(ctx, "ctm.Q1", X2, {0, 2}, {1, 0}, a, site_dual, prec, s);         // [T1.R, T4.D, a.R, a.D]
  T Y1 = contract(ctx, "ctm.Y1", r[T1], r[C2], {2}, {0}, prec, s);        // [T1.L, T1.D, C2.D]
  T Y2 = contract(ctx, "ctm.Y2", Y1, r[T2], {2}, {0}, prec, s);           // [T1.L, T1.D, T2.L, T2.D]
  T Q2 = absorb(ctx, "ctm.Q2", Y2, {1, 2}, {1, 2}, a, site_dual, prec, s);         // [T1.L, T2.D, a.L, a.D]
  T Rt = contract(ctx, "ctm.Rt", Q1, Q2, {0, 2}, {0, 2}, prec, s);        // [T4.D, a.D | T2.D, a.D]
  T Z1 = contract(ctx, "ctm.Z1", r[T4], r[C4], {2}, {0}, prec, s);        // [T4.U, T4.R, C4.R]
  T Z2 = contract(ctx, "ctm.Z2", Z1, r[T3], {2}, {0}, prec, s);           // [T4.U, T4.R, T3.U, T3.R]
  T Q4 = absorb(ctx, "ctm.Q4", Z2, {1, 2}, {0, 3}, a, site_dual, prec, s);         // [T4.U, T3.R, a.U, a.R]
  T W1 = contract(ctx, "ctm.W1", r[T2], r[C3], {2}, {0}, prec, s);        // [T2.U, T2.L, C3.L]
  T W2 = contract(ctx, "ctm.W2", W1, r[T3], {2}, {2}, prec, s);           // [T2.U, T2.L, T3.L, T3.U]
  T Q3 = absorb(ctx, "ctm.Q3", W2, {1, 3}, {2, 3}, a, site_dual, prec, s);         // [T2.U, T3.L, a.L, a.U]
  T Rb = contract(ctx, "ctm.Rb", Q4, Q3, {1, 3}, {1, 2}, prec, s);        // [T4.U, a.U | T2.U, a.U]
  double *P = nullptr, *Pt = nullptr;
  if (a.L->group == BST_SU2) {
    // chi is the total dimension; the new leg is incoming on P
    *pres = su2_projector(ctx, Rt.L, Rt.d, Rb.L, Rb.d, 2, chi, cutoff, prec, &P, &Pt, s);
  } else {
    const int new_flow = r[C1].L->legs[1].flow;
    int64_t pcap = Rb.L->legs[0].dim * Rb.L->legs[1].dim * chi;
    int64_t ptcap = Rt.L->legs[0].dim * Rt.L->legs[1].dim * chi;
    P = (double*)ctx->buf("ctm.P", sizeof(double) * pcap, s);
    Pt = (double*)ctx->buf("ctm.Pt", sizeof(double) * ptcap, s);
    *pres = svd_projector(ctx, Rt.L, Rt.d, Rb.L, Rb.d, 2, chi, cutoff, new_flow, prec, P, Pt, s);
  }
  T tP{pres->P, P}, tPt{pres->Pt, Pt};
  // renormalise: C1' = X1 P, T4' = ((Pt T4) a) P, C4' = Pt (C4 T3)
  out[0] = contract(ctx, "ctm.C1n", X1, tP, {0, 1}, {0, 1}, prec, s);    // [T1.R, new]
  T W = contract(ctx, "ctm.W", tPt, r[T4], {1}, {0}, prec, s);             // [new^, a.D, T4.R, T4.D]
  T Z = absorb(ctx, "ctm.Z", W, {2, 1}, {0, 1}, a, site_dual, prec, s);             // [new^, T4.D, a.R, a.D]
  out[1] = contract(ctx, "ctm.T4n", Z, tP, {1, 3}, {0, 1}, prec, s);     // [new^, a.R, new]
  T Y = contract(ctx, "ctm.Y", r[C4], r[T3], {1}, {0}, prec, s);           // [C4.U, T3.U, T3.R]
  out[2] = contract(ctx, "ctm.C4n", tPt, Y, {1, 2}, {0, 1}, prec, s);    // [new^, T3.R]
  for (int i = 0; i < 3; ++i) normalise(ctx, out[i].L, const_cast<double*>(out[i].d), s);
}

// ---------------------------------------------------------------------------
// Unit cells (Sec. 3.1; Sec. 4.1 times a 2 x 2 cell).  An Lx x Ly cell (x
// right, y down) holds a site per position, each with its own environment.
// The LEFT move absorbs column by column: for column x, plaquette (x, y)
// (sites (x, y), (x+1, y), (x, y+1), (x+1, y+1)) gives the projectors of
// the cut between rows y and y+1; then every row y of column x is absorbed
// into the left environment of site (x+1, y): C1' = (C1 T1) P[y-1],
// T4' = Pt[y-1] (T4 a) P[y], C4' = Pt[y] (C4 T3).  Other directions turn
// the cell: the site at (x, y) moves to (y, -x mod Lx) and every tensor is
// rotated as in the one-site move.

// Projectors of the left cut of plaquette (ul, ur, ll, lr); P into pbuf,
// Pt into ptbuf (named context buffers), layouts in the result.
static ProjResult plaquette_projector(Ctx* ctx, T* ul, T* ur, T* ll, T* lr, int64_t chi, double cutoff, bst_prec prec,
                               const std::string& pname, double** P, double** Pt, cudaStream_t s) {
  // the one-site move's contraction sequence, each quarter from its own site
  T X1 = contract(ctx, "ctm.X1", ul[C1], ul[T1], {0}, {0}, prec, s);                  // [C1.D, T1.D, T1.R]
  T X2 = contract(ctx, "ctm.X2", X1, ul[T4], {0}, {0}, prec, s);                     // [T1.D, T1.R, T4.R, T4.D]
  T Q1 = absorb(ctx, "ctm.Q1", X2, {0, 2}, {1, 0}, ul[SITE], nullptr, prec, s);      // [T1.R, T4.D, a.R, a.D]
  T Y1 = contract(ctx, "ctm.Y1", ur[T1], ur[C2], {2}, {0}, prec, s);                  // [T1.L, T1.D, C2.D]
  T Y2 = contract(ctx, "ctm.Y2", Y1, ur[T2], {2}, {0}, prec, s);                     // [T1.L, T1.D, T2.L, T2.D]
  T Q2 = absorb(ctx, "ctm.Q2", Y2, {1, 2}, {1, 2}, ur[SITE], nullptr, prec, s);      // [T1.L, T2.D, a.L, a.D]
  T Rt = contract(ctx, "ctm.Rt", Q1, Q2, {0, 2}, {0, 2}, prec, s);                   // [T4.D, a.D | T2.D, a.D]
  T Z1 = contract(ctx, "ctm.Z1", ll[T4], ll[C4], {2}, {0}, prec, s);                  // [T4.U, T4.R, C4.R]
  T Z2 = contract(ctx, "ctm.Z2", Z1, ll[T3], {2}, {0}, prec, s);                     // [T4.U, T4.R, T3.U, T3.R]
  T Q4 = absorb(ctx, "ctm.Q4", Z2, {1, 2}, {0, 3}, ll[SITE], nullptr, prec, s);      // [T4.U, T3.R, a.U, a.R]
  T W1 = contract(ctx, "ctm.W1", lr[T2], lr[C3], {2}, {0}, prec, s);                  // [T2.U, T2.L, C3.L]
  T W2 = contract(ctx, "ctm.W2", W1, lr[T3], {2}, {2}, prec, s);                     // [T2.U, T2.L, T3.L, T3.U]
  T Q3 = absorb(ctx, "ctm.Q3", W2, {1, 3}, {2, 3}, lr[SITE], nullptr, prec, s);      // [T2.U, T3.L, a.L, a.U]
  T Rb = contract(ctx, "ctm.Rb", Q4, Q3, {1, 3}, {1, 2}, prec, s);                   // [T4.U, a.U | T2.U, a.U]
  const int new_flow = ll[C1].L->legs[1].flow;
  const int64_t pcap = Rb.L->legs[0].dim * Rb.L->legs[1].dim * chi;
  const int64_t ptcap = Rt.L->legs[0].dim * Rt.L->legs[1].dim * chi;
  *P = (double*)ctx->buf(pname + ".P", sizeof(double) * pcap, s);
  *Pt = (double*)ctx->buf(pname + ".Pt", sizeof(double) * ptcap, s);
  return svd_projector(ctx, Rt.L, Rt.d, Rb.L, Rb.d, 2, chi, cutoff, new_flow, prec, *P, *Pt, s);
}

// Column absorption of one site: C1' = (C1 T1) Pa, T4' = Pta (T4 a) Pb,
// C4' = Ptb (C4 T3), each normalised, into buffers named by `tag`.
static void renormalise_site(Ctx* ctx, T* r, T tPa, T tPta, T tPb, T tPtb, bst_prec prec, const std::string& tag, T out[3],
                      cudaStream_t s) {
  T X1 = contract(ctx, "ctm.X1", r[C1], r[T1], {0}, {0}, prec, s);                    // [C1.D, T1.D, T1.R]
  out[0] = contract(ctx, (tag + ".C1n").c_str(), X1, tPa, {0, 1}, {0, 1}, prec, s);   // [T1.R, new_a]
  T W = contract(ctx, "ctm.W", tPta, r[T4], {1}, {0}, prec, s);                        // [new_a^, a.D, T4.R, T4.D]
  T Z = absorb(ctx, "ctm.Z", W, {2, 1}, {0, 1}, r[SITE], nullptr, prec, s);           // [new_a^, T4.D, a.R, a.D]
  out[1] = contract(ctx, (tag + ".T4n").c_str(), Z, tPb, {1, 3}, {0, 1}, prec, s);     // [new_a^, a.R, new_b]
  T Y = contract(ctx, "ctm.Y", r[C4], r[T3], {1}, {0}, prec, s);                       // [C4.U, T3.U, T3.R]
  out[2] = contract(ctx, (tag + ".C4n").c_str(), tPtb, Y, {1, 2}, {0, 1}, prec, s);    // [new_b^, T3.R]
  for (int i = 0; i < 3; ++i) normalise(ctx, out[i].L, const_cast<double*>(out[i].d), s);
}

void ctm_move_cell(Ctx* ctx, int dir, int Lx, int Ly, Layout* const* a, const double* const* ad, bst_env* envs,
                   int64_t chi, double cutoff, bst_prec prec, cudaStream_t s) {
  BST_REQUIRE(dir >= 0 && dir <= 4, BST_E_ARG, "dir must be 0..4");
  BST_REQUIRE(Lx >= 1 && Ly >= 1 && Lx * Ly <= 64, BST_E_ARG, "cell must be 1..64 sites");
  const int nsite = Lx * Ly;
  for (int i = 0; i < nsite; ++i) {
    BST_REQUIRE(a[i] && ad[i], BST_E_ARG, "site is NULL");
    BST_REQUIRE(a[i]->rank == 4, BST_E_ARG, "cell sites must be double layers a[L,U,R,D]");
    BST_REQUIRE(a[i]->group != BST_SU2, BST_E_UNSUPPORTED, "unit cells: abelian groups only");
    for (int j = 0; j < 4; ++j) {
      bst_env* e = &envs[i];
      BST_REQUIRE(e->C[j] && e->T[j] && e->c[j] && e->t[j], BST_E_ARG, "env has a null entry");
      BST_REQUIRE(L_(e->C[j])->rank == 2 && L_(e->T[j])->rank == 3, BST_E_ARG, "env ranks must be 2 (C) and 3 (T)");
      BST_REQUIRE(L_(e->C[j])->group == a[i]->group && L_(e->T[j])->group == a[i]->group, BST_E_ARG,
                  "environment and site belong to different symmetry groups");
    }
  }
  std::vector<int> seq;
  if (dir == 4) seq = {0, 2, 1, 3};  // LEFT, RIGHT, UP, DOWN
  else seq = {dir};
  for (int d : seq) {
    const int k = d;  // quarter turns (LEFT 0, UP 1, RIGHT 2, DOWN 3)
    std::vector<Src> rot = rotation(k);
    // rotated cell: position of every original site after k turns
    int lx = Lx, ly = Ly;
    std::vector<int> px(nsite), py(nsite);
    for (int i = 0; i < nsite; ++i) px[i] = i % Lx, py[i] = i / Lx;
    for (int t = 0; t < k; ++t) {
      for (int i = 0; i < nsite; ++i) {
        const int x = px[i], y = py[i];
        px[i] = y;
        py[i] = ((-x) % lx + lx) % lx;
      }
      std::swap(lx, ly);
    }
    std::vector<int> at(nsite);  // rotated position -> original site index
    for (int i = 0; i < nsite; ++i) at[px[i] + lx * py[i]] = i;
    // the rotated tensors of every site (role n of rotated site j)
    std::vector<std::vector<T>> R(nsite, std::vector<T>(NROLE));
    for (int j = 0; j < nsite; ++j) {
      const int i = at[j];
      T orig[NROLE];
      for (int q = 0; q < 4; ++q) {
        orig[C1 + q] = {L_(envs[i].C[q]), envs[i].c[q]};
        orig[T1 + q] = {L_(envs[i].T[q]), envs[i].t[q]};
      }
      orig[SITE] = {a[i], ad[i]};
      for (int n = 0; n < NROLE; ++n) {
        const Src& src = rot[n];
        if (is_identity(src.perm)) {
          R[j][n] = orig[src.role];
        } else {
          Layout* dst = nullptr;
          DevRelayout* rp = get_permute_plan(ctx, orig[src.role].L, src.perm, &dst);
          const std::string nm = "cell.rot." + std::to_string(j) + "." + std::to_string(n);
          double* buf = (double*)ctx->buf(nm, sizeof(double) * std::max<int64_t>(dst->nnz, 1), s);
          launch_relayout(ctx, *rp, orig[src.role].d, buf, 0, 1.0, 0.0, s);
          release(dst);  // interned
          R[j][n] = {dst, buf};
        }
      }
    }
    // LEFT move of the rotated cell, column by column
    for (int x = 0; x < lx; ++x) {
      const int xr = (x + 1) % lx;
      std::vector<ProjResult> pr(ly);
      std::vector<double*> P(ly), Pt(ly);
      for (int y = 0; y < ly; ++y) {
        const int yd = (y + 1) % ly;
        pr[y] = plaquette_projector(ctx, R[x + lx * y].data(), R[xr + lx * y].data(), R[x + lx * yd].data(),
                                    R[xr + lx * yd].data(), chi, cutoff, prec, "cell.p" + std::to_string(y), &P[y],
                                    &Pt[y], s);
      }
      std::vector<std::array<T, 3>> out(ly);
      for (int y = 0; y < ly; ++y) {
        const int ya = (y - 1 + ly) % ly;
        T o[3];
        renormalise_site(ctx, R[x + lx * y].data(), {pr[ya].P, P[ya]}, {pr[ya].Pt, Pt[ya]}, {pr[y].P, P[y]},
                         {pr[y].Pt, Pt[y]}, prec, "cell.n" + std::to_string(xr + lx * y), o, s);
        out[y] = {o[0], o[1], o[2]};
      }
      for (int y = 0; y < ly; ++y) {
        R[xr + lx * y][C1] = out[y][0];
        R[xr + lx * y][T4] = out[y][1];
        R[xr + lx * y][C4] = out[y][2];
      }
      for (auto& q : pr) {
        release(q.P);
        release(q.Pt);
      }
    }
    // renewed C1, T4, C4 of every rotated site back to the original frame
    const int renewed[3] = {C1, T4, C4};
    for (int j = 0; j < nsite; ++j) {
      bst_env* env = &envs[at[j]];
      for (int q = 0; q < 3; ++q) {
        const Src& src = rot[renewed[q]];
        const T& o = R[j][renewed[q]];
        std::vector<int> inv(src.perm.size());
        for (size_t m = 0; m < src.perm.size(); ++m) inv[src.perm[m]] = int(m);
        double* dst;
        int64_t cap;
        bst_layout* slot;
        if (src.role < T1) {
          dst = env->c[src.role - C1];
          cap = env->c_cap[src.role - C1];
          slot = &env->C[src.role - C1];
        } else {
          dst = env->t[src.role - T1];
          cap = env->t_cap[src.role - T1];
          slot = &env->T[src.role - T1];
        }
        Layout* nl = nullptr;
        if (is_identity(inv)) {
          nl = o.L;
          retain(nl);
          BST_REQUIRE(nl->nnz <= cap, BST_E_SHAPE, "env buffer capacity too small for the renewed tensor");
          BST_CUDA(cudaMemcpyAsync(dst, o.d, sizeof(double) * nl->nnz, cudaMemcpyDeviceToDevice, s));
        } else {
          DevRelayout* rp = get_permute_plan(ctx, o.L, inv, &nl);
          BST_REQUIRE(nl->nnz <= cap, BST_E_SHAPE, "env buffer capacity too small for the renewed tensor");
          launch_relayout(ctx, *rp, o.d, dst, 0, 1.0, 0.0, s);
        }
        release(L_(*slot));
        *slot = reinterpret_cast<bst_layout>(nl);
      }
    }
  }
}

void ctm_move(Ctx* ctx, int dir, Layout* a, const double* ad, bst_env* env, int64_t chi, double cutoff,
              bst_prec prec, bst_ctm_stats* stats, cudaStream_t s) {
  BST_REQUIRE(dir >= 0 && dir <= 4, BST_E_ARG, "dir must be 0..4");
  BST_REQUIRE(a->rank == 4 || a->rank == 5, BST_E_ARG,
              "site tensor must be the double layer a[L,U,R,D] or a single-layer A[P,L,U,R,D]");
  for (int i = 0; i < 4; ++i) {
    BST_REQUIRE(env->C[i] && env->T[i] && env->c[i] && env->t[i], BST_E_ARG, "env has a null entry");
    BST_REQUIRE(L_(env->C[i])->rank == 2 && L_(env->T[i])->rank == 3, BST_E_ARG,
                "env ranks must be 2 (C) and 3 (T)");
  }
  if (a->group == BST_SU2) {
    // quarter turns permute legs, which for SU(2) blocks means recoupling
    // their trees: not implemented, so only the LEFT move runs
    BST_REQUIRE(dir == 0, BST_E_UNSUPPORTED, "SU(2): only the LEFT move (dir 0) is implemented");
    BST_REQUIRE(a->rank == 4, BST_E_UNSUPPORTED, "SU(2): the site must be the double layer a[L,U,R,D]");
  }
  for (int i = 0; i < 4; ++i)
    BST_REQUIRE(L_(env->C[i])->group == a->group && L_(env->T[i])->group == a->group, BST_E_ARG,
                "environment and site belong to different symmetry groups");
  if (stats) memset(stats, 0, sizeof(*stats));
  std::vector<int> seq;
  if (dir == 4) seq = {0, 2, 1, 3};  // LEFT, RIGHT, UP, DOWN
  else seq = {dir};
  int step = 0;
  for (int d : seq) {
    // rotation index: LEFT 0, UP 1, RIGHT 2, DOWN 3 quarter turns
    const int k = d;
    std::vector<Src> rot = rotation(k);
    T orig[NROLE];
    for (int i = 0; i < 4; ++i) {
      orig[C1 + i] = {L_(env->C[i]), env->c[i]};
      orig[T1 + i] = {L_(env->T[i]), env->t[i]};
    }
    orig[SITE] = {a, ad};
    T r[NROLE];
    for (int n = 0; n < NROLE; ++n) {
      const Src& src = rot[n];
      std::vector<int> perm = src.perm;
      if (n == SITE && a->rank == 5) {  // the P leg stays first
        perm.insert(perm.begin(), -1);
        for (auto& x : perm) ++x;
      }
      if (is_identity(perm)) {
        r[n] = orig[src.role];
      } else {
        Layout* dst = nullptr;
        DevRelayout* rp = get_permute_plan(ctx, orig[src.role].L, perm, &dst);
        std::string nm = "ctm.rot" + std::to_string(n);
        double* buf = (double*)ctx->buf(nm, sizeof(double) * std::max<int64_t>(dst->nnz, 1), s);
        launch_relayout(ctx, *rp, orig[src.role].d, buf, 0, 1.0, 0.0, s);
        release(dst);  // the intern table keeps the layout alive
        r[n] = {dst, buf};
      }
    }
    T out[3];
    ProjResult pr;
    Layout* site_dual = nullptr;
    if (a->rank == 5) {
      std::vector<Leg> dl;
      for (auto& l : r[SITE].L->legs) dl.push_back(l.dual());
      site_dual = make_layout(ctx, a->group, dl);
      release(site_dual);  // interned
    }
    left_move(ctx, r, site_dual, chi, cutoff, prec, out, &pr, s);
    // map renewed rotated roles C1, T4, C4 back to the original frame
    const int renewed[3] = {C1, T4, C4};
    for (int i = 0; i < 3; ++i) {
      const Src& src = rot[renewed[i]];
      std::vector<int> inv(src.perm.size());
      for (size_t j = 0; j < src.perm.size(); ++j) inv[src.perm[j]] = int(j);
      Layout* nl = nullptr;
      double* dst;
      int64_t cap;
      bst_layout* slot;
      if (src.role < T1) {
        dst = env->c[src.role - C1];
        cap = env->c_cap[src.role - C1];
        slot = &env->C[src.role - C1];
      } else {
        dst = env->t[src.role - T1];
        cap = env->t_cap[src.role - T1];
        slot = &env->T[src.role - T1];
      }
      if (is_identity(inv)) {
        nl = out[i].L;
        retain(nl);
        BST_REQUIRE(nl->nnz <= cap, BST_E_SHAPE, "env buffer capacity too small for the renewed tensor");
        BST_CUDA(cudaMemcpyAsync(dst, out[i].d, sizeof(double) * nl->nnz, cudaMemcpyDeviceToDevice, s));
      } else {
        DevRelayout* rp = get_permute_plan(ctx, out[i].L, inv, &nl);
        BST_REQUIRE(nl->nnz <= cap, BST_E_SHAPE, "env buffer capacity too small for the renewed tensor");
        launch_relayout(ctx, *rp, out[i].d, dst, 0, 1.0, 0.0, s);
      }
      release(L_(*slot));
      *slot = reinterpret_cast<bst_layout>(nl);
    }
    if (stats && step < 4) {
      stats->kept[step] = pr.kept;
      stats->smin_over_smax[step] = pr.smin_over_smax;
      stats->trunc_weight[step] = pr.trunc_weight;
    }
    release(pr.P);
    release(pr.Pt);
    ++step;
  }
}

// Two-site reduced density matrix of a bond of the one-site cell from its
// environment (the observable of Sec. 3's error procedure and Sec. 4.1's
// energies).  The horizontal bond (site i and its right neighbour j) is the
// 3 x 4 network C1 T1 T1 C2 / T4 a_i a_j T2 / C4 T3 T3 C3 with both sites
// open: site[L, U, R, D, p, p'] (the open double layer); the vertical bond
// (i above j) is the horizontal bond of the network turned by a quarter
// turn.  Left half: ((((C1 T1) T4) C4) T3) a_i -> [T1.R, T3.R, a.R, p, p'];
// right half: ((((T1 C2) T2) C3) T3) a_j -> [T1.L, T3.L, a.L, p, p']; their
// product over the three cut bonds is rho[p_i, p_i', p_j, p_j'].
Layout* bond_rdm(Ctx* ctx, int bond, Layout* site, const double* sd, bst_env* env, bst_prec prec, double** rho,
                 cudaStream_t s) {
  BST_REQUIRE(bond == 0 || bond == 1, BST_E_ARG, "bond must be 0 (horizontal) or 1 (vertical)");
  BST_REQUIRE(site->rank == 6, BST_E_ARG, "the open site must have legs [L, U, R, D, p, p']");
  require_u1(site);
  for (int i = 0; i < 4; ++i) {
    BST_REQUIRE(env->C[i] && env->T[i] && env->c[i] && env->t[i], BST_E_ARG, "env has a null entry");
    BST_REQUIRE(L_(env->C[i])->group == site->group && L_(env->T[i])->group == site->group, BST_E_ARG,
                "environment and site belong to different symmetry groups");
  }
  const int k = bond;  // quarter turns: the upper site of a vertical bond becomes the left one
  std::vector<Src> rot = rotation(k);
  T orig[NROLE], r[NROLE];
  for (int i = 0; i < 4; ++i) {
    orig[C1 + i] = {L_(env->C[i]), env->c[i]};
    orig[T1 + i] = {L_(env->T[i]), env->t[i]};
  }
  orig[SITE] = {site, sd};
  for (int n = 0; n < NROLE; ++n) {
    std::vector<int> perm = rot[n].perm;
    if (n == SITE) {
      perm.push_back(4);  // the physical legs stay last
      perm.push_back(5);
    }
    if (is_identity(perm)) {
      r[n] = orig[rot[n].role];
    } else {
      Layout* dst = nullptr;
      DevRelayout* rp = get_permute_plan(ctx, orig[rot[n].role].L, perm, &dst);
      std::string nm = "rdm.rot" + std::to_string(n);
      double* buf = (double*)ctx->buf(nm, sizeof(double) * std::max<int64_t>(dst->nnz, 1), s);
      launch_relayout(ctx, *rp, orig[rot[n].role].d, buf, 0, 1.0, 0.0, s);
      release(dst);  // interned
      r[n] = {dst, buf};
    }
  }
  T X1 = contract(ctx, "rdm.X1", r[C1], r[T1], {0}, {0}, prec, s);          // [C1.D, T1.D, T1.R]
  T X2 = contract(ctx, "rdm.X2", X1, r[T4], {0}, {0}, prec, s);             // [T1.D, T1.R, T4.R, T4.D]
  T X3 = contract(ctx, "rdm.X3", X2, r[C4], {3}, {0}, prec, s);             // [T1.D, T1.R, T4.R, C4.R]
  T X4 = contract(ctx, "rdm.X4", X3, r[T3], {3}, {0}, prec, s);             // [T1.D, T1.R, T4.R, T3.U, T3.R]
  T Li = contract(ctx, "rdm.Li", X4, r[SITE], {0, 2, 3}, {1, 0, 3}, prec, s);  // [T1.R, T3.R, a.R, p, p']
  T Y1 = contract(ctx, "rdm.Y1", r[T1], r[C2], {2}, {0}, prec, s);          // [T1.L, T1.D, C2.D]
  T Y2 = contract(ctx, "rdm.Y2", Y1, r[T2], {2}, {0}, prec, s);             // [T1.L, T1.D, T2.L, T2.D]
  T Y3 = contract(ctx, "rdm.Y3", Y2, r[C3], {3}, {0}, prec, s);             // [T1.L, T1.D, T2.L, C3.L]
  T Y4 = contract(ctx, "rdm.Y4", Y3, r[T3], {3}, {2}, prec, s);             // [T1.L, T1.D, T2.L, T3.L, T3.U]
  T Rj = contract(ctx, "rdm.Rj", Y4, r[SITE], {1, 2, 4}, {1, 2, 3}, prec, s);  // [T1.L, T3.L, a.L, p, p']
  T R = contract(ctx, "rdm.rho", Li, Rj, {0, 1, 2}, {0, 1, 2}, prec, s);     // [p_i, p_i', p_j, p_j']
  *rho = const_cast<double*>(R.d);
  retain(R.L);
  return R.L;
}

}  // namespace bst
