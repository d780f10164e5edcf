// Observables of a one-site CTMRG environment and the paper's CTM error
// procedure (Sec. 3, implementation details; Sec. 4.1's energies).
//
//   * open double layer: the site's ket and bra multiplied without the sum
//     over the physical index (Sec. 3.2 with the physical legs kept open),
//     virtual ket/bra legs fused pairwise, the remover's double layer (its
//     extra leg traced between ket and bra, Sec. 3.1) absorbed on the right
//     leg: [L, U, R, D, p, p'];
//   * block-sparse dot product (FP64, fixed summation order) for traces and
//     expectation values Tr(rho H) of two-site operators whose tensor has
//     the density matrix's layout (Sec. 3.1: charged single-site operators
//     combined into a two-site operator that conserves the charge);
//   * the error procedure: CTM steps at fixed chi until the observable
//     changes by less than a threshold or a step limit is reached, error =
//     largest change among the last three steps; chi doubled until two
//     fixed-chi results agree to the threshold or chi would exceed its
//     maximum; error = the larger of the step and chi errors.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bst_internal.h"

namespace bst {

// sum_i x_i y_i: per-CTA partial sums, then one CTA adds them in order
__global__ void dot_partial(const double* __restrict__ x, const double* __restrict__ y, long long n,
                            double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

double block_dot(Ctx* ctx, const double* x, const double* y, int64_t n, cudaStream_t s) {
  double* part = (double*)ctx->buf("dot.part", sizeof(double) * 305, s);
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 304)));
  if (n > 0) {
    dot_partial<<<grid, 256, 0, s>>>(x, y, n, part);
    dot_final<<<1, 256, 0, s>>>(part, grid, part + 304);
    BST_CUDA(cudaGetLastError());
    count_launch(ctx, 2);
  } else {
    BST_CUDA(cudaMemsetAsync(part + 304, 0, sizeof(double), s));
  }
  double h = 0;
  BST_CUDA(cudaMemcpyAsync(&h, part + 304, sizeof(double), cudaMemcpyDeviceToHost, s));
  BST_CUDA(cudaStreamSynchronize(s));
  return h;
}

// Open double layer [kl, ku, kr, kd, p, p'] of a site A[p, l, u, r, d]
// (remover R[r, l', s] absorbed on the right leg when R is given).  Every
// intermediate has at most eight legs: p is fused with l first
// (pl = fuse(p, l)); the outer product of A'[pl, u, r, d] with its conjugate
// is permuted and its virtual pairs fused, then (pl, pl~) are split back into
// p, l, p~, l~ (inverse fuse relayouts) and (l, l~) fused.  First call with
// out == nullptr for the layout (returned, new reference).
Layout* double_layer_open(Ctx* ctx, Layout* LA, const double* A, Layout* LR, const double* R, double* out,
                          cudaStream_t s) {
  require_u1(LA);
  BST_REQUIRE(LA->rank == 5, BST_E_ARG, "site tensor must have rank 5 [p,l,u,r,d]");
  const int g = LA->group;
  const Leg &p = LA->legs[0], &l = LA->legs[1];
  Layout* Lpl = nullptr;  // [pl, u, r, d]
  DevRelayout* f_pl = get_fuse_plan(ctx, LA, {2, 1, 1, 1}, &Lpl);
  std::vector<Leg> dl;
  for (auto& x : Lpl->legs) dl.push_back(x.dual());
  Layout* Lpld = make_layout(ctx, g, dl);
  ContractPlan* po = get_contract_plan(ctx, Lpl, Lpld, {}, {});  // [pl, u, r, d, pl~, u~, r~, d~]
  release(Lpld);
  Layout* L8 = nullptr;  // [pl, pl~, u, u~, r, r~, d, d~]
  DevRelayout* perm8 = get_permute_plan(ctx, po->C, {0, 4, 1, 5, 2, 6, 3, 7}, &L8);
  Layout* L5 = nullptr;  // [pl, pl~, ku, kr, kd]
  DevRelayout* fuse5 = get_fuse_plan(ctx, L8, {1, 1, 2, 2, 2}, &L5);
  // split pl: [p, l, pl~, ku, kr, kd] fuses to L5
  std::vector<Leg> l6 = {p, l};
  for (int i = 1; i < 5; ++i) l6.push_back(L5->legs[i]);
  Layout* L6 = make_layout(ctx, g, l6);
  Layout* chk = nullptr;
  DevRelayout* split1 = get_fuse_plan(ctx, L6, {2, 1, 1, 1, 1}, &chk);
  BST_REQUIRE(chk == L5, BST_E_SHAPE, "open double layer: (p, l) does not split back");
  release(chk);
  // split pl~: [p, l, p~, l~, ku, kr, kd] fuses to L6
  std::vector<Leg> l7 = {p, l, p.dual(), l.dual()};
  for (int i = 3; i < 6; ++i) l7.push_back(L6->legs[i]);
  Layout* L7 = make_layout(ctx, g, l7);
  DevRelayout* split2 = get_fuse_plan(ctx, L7, {1, 1, 2, 1, 1, 1}, &chk);
  BST_REQUIRE(chk == L6, BST_E_SHAPE, "open double layer: (p~, l~) does not split back");
  release(chk);
  Layout* L7p = nullptr;  // [l, l~, ku, kr, kd, p, p~]
  DevRelayout* perm7 = get_permute_plan(ctx, L7, {1, 3, 4, 5, 6, 0, 2}, &L7p);
  Layout* Lo = nullptr;  // [kl, ku, kr, kd, p, p~]
  DevRelayout* fuse6 = get_fuse_plan(ctx, L7p, {2, 1, 1, 1, 1, 1}, &Lo);
  Layout* result = Lo;
  ContractPlan *pr = nullptr, *p2 = nullptr;
  DevRelayout *rperm = nullptr, *rfuse = nullptr, *aperm = nullptr;
  if (LR) {
    require_u1(LR);
    BST_REQUIRE(LR->rank == 3, BST_E_ARG, "remover must have rank 3 [r,l',s]");
    std::vector<Leg> rl;
    for (auto& x : LR->legs) rl.push_back(x.dual());
    Layout* LRd = make_layout(ctx, g, rl);
    pr = get_contract_plan(ctx, LR, LRd, {2}, {2});  // [r, l', r~, l'~]
    release(LRd);
    Layout* Lr2 = nullptr;
    rperm = get_permute_plan(ctx, pr->C, {0, 2, 1, 3}, &Lr2);
    Layout* Lr3 = nullptr;  // rho_R[kr_in, kl_out]
    rfuse = get_fuse_plan(ctx, Lr2, {2, 2}, &Lr3);
    release(Lr2);
    p2 = get_contract_plan(ctx, Lo, Lr3, {2}, {0});  // [kl, ku, kd, p, p~, kl_out]
    release(Lr3);
    Layout* La = nullptr;
    aperm = get_permute_plan(ctx, p2->C, {0, 1, 5, 2, 3, 4}, &La);
    result = La;
  }
  if (out) {
    BST_REQUIRE(A && (!LR || R), BST_E_ARG, "data pointer is NULL");
    auto buf = [&](const char* n, int64_t e) { return (double*)ctx->buf(n, sizeof(double) * std::max<int64_t>(e, 1), s); };
    double* a1 = buf("odl.A1", LA->nnz);
    const int64_t big = std::max<int64_t>(po->C->nnz, p2 ? p2->C->nnz : 0);
    double* a2 = buf("odl.A2", big);
    double* a3 = buf("odl.A3", big);
    launch_relayout(ctx, *f_pl, A, a1, 0, 1.0, 0.0, s);              // A -> A'
    run_contract(ctx, po, a1, a1, BST_FP64, 1.0, 0.0, a2, s);          // A' (x) A'*
    launch_relayout(ctx, *perm8, a2, a3, 0, 1.0, 0.0, s);
    launch_relayout(ctx, *fuse5, a3, a2, 0, 1.0, 0.0, s);             // [pl, pl~, ku, kr, kd]
    launch_relayout(ctx, *split1, a3, a2, 1, 1.0, 0.0, s);            // [p, l, pl~, ku, kr, kd]
    launch_relayout(ctx, *split2, a2, a3, 1, 1.0, 0.0, s);            // [p, l, p~, l~, ku, kr, kd]
    launch_relayout(ctx, *perm7, a2, a3, 0, 1.0, 0.0, s);             // [l, l~, ku, kr, kd, p, p~]
    if (!LR) {
      launch_relayout(ctx, *fuse6, a3, out, 0, 1.0, 0.0, s);
    } else {
      launch_relayout(ctx, *fuse6, a3, a2, 0, 1.0, 0.0, s);           // [kl, ku, kr, kd, p, p~]
      double* r1 = buf("odl.R1", pr->C->nnz);
      double* r2 = buf("odl.R2", pr->C->nnz);
      run_contract(ctx, pr, R, R, BST_FP64, 1.0, 0.0, r1, s);
      launch_relayout(ctx, *rperm, r1, r2, 0, 1.0, 0.0, s);
      launch_relayout(ctx, *rfuse, r2, r1, 0, 1.0, 0.0, s);           // rho_R
      run_contract(ctx, p2, a2, r1, BST_FP64, 1.0, 0.0, a3, s);
      launch_relayout(ctx, *aperm, a3, out, 0, 1.0, 0.0, s);
    }
  }
  // the intern table keeps the intermediate layouts alive
  release(Lpl);
  release(L8);
  release(L5);
  release(L6);
  release(L7);
  release(L7p);
  if (LR) release(Lo);
  return result;
}

// Energy per site of the one-site cell for a two-site operator H given as
// a tensor with the density matrix's layout: sum over the horizontal and
// vertical bonds of Tr(rho H) / Tr(rho), the traces as block dot products.
double site_observable(Ctx* ctx, Layout* site, const double* sd, bst_env* env, const double* Hbuf,
                       const double* Ibuf, Layout* HL, bst_prec prec, cudaStream_t s) {
  double e = 0;
  for (int bond = 0; bond < 2; ++bond) {
    double* rho = nullptr;
    Layout* RL = bond_rdm(ctx, bond, site, sd, env, prec, &rho, s);
    BST_REQUIRE(RL == HL, BST_E_SHAPE, "operator layout differs from the density matrix's");
    release(RL);
    const double num = block_dot(ctx, rho, Hbuf, HL->nnz, s);
    const double den = block_dot(ctx, rho, Ibuf, HL->nnz, s);
    BST_REQUIRE(std::isfinite(num) && std::isfinite(den) && den != 0.0, BST_E_NUMERIC,
                "density matrix with zero or non-finite trace");
    e += num / den;
  }
  return e;
}

// The error procedure of Sec. 3 around full CTM moves (L, R, U, D).
void ctm_converge(Ctx* ctx, Layout* a, const double* ad, Layout* site, const double* sd, Layout* HL,
                  const double* H, bst_env* env, int64_t chi0, int64_t chi_max, double tol, int32_t max_steps,
                  double rel_cutoff, bst_prec prec, bst_ctm_converge_stats* st, cudaStream_t s) {
  BST_REQUIRE(chi0 >= 1 && chi_max >= chi0 && max_steps >= 1 && tol > 0, BST_E_ARG, "bad driver parameters");
  // identity with the density matrix's layout: delta_{p_i p_i'} delta_{p_j p_j'}
  std::vector<double> id(std::max<int64_t>(HL->nnz, 1), 0.0);
  for (int64_t b = 0; b < HL->nblocks; ++b) {
    const int32_t* sc = &HL->sect[b * 4];
    if (HL->legs[0].q[sc[0]] != HL->legs[1].q[sc[1]] || HL->legs[2].q[sc[2]] != HL->legs[3].q[sc[3]]) continue;
    const int64_t* sh = &HL->shape[b * 4];
    for (int64_t i = 0; i < sh[0]; ++i)
      for (int64_t j = 0; j < sh[2]; ++j)
        id[HL->offset[b] + ((i * sh[1] + i) * sh[2] + j) * sh[3] + j] = 1.0;
  }
  double* Ibuf = (double*)ctx->buf("conv.id", sizeof(double) * id.size(), s);
  BST_CUDA(cudaMemcpyAsync(Ibuf, id.data(), sizeof(double) * id.size(), cudaMemcpyHostToDevice, s));
  std::memset(st, 0, sizeof(*st));
  std::vector<double> results;
  double err_steps = 0;
  int64_t chi = chi0;
  for (;;) {
    std::vector<double> vals;
    for (int t = 0; t < max_steps; ++t) {
      ctm_move(ctx, 4, a, ad, env, chi, rel_cutoff, prec, nullptr, s);
      vals.push_back(site_observable(ctx, site, sd, env, H, Ibuf, HL, prec, s));
      ++st->steps_total;
      if (vals.size() >= 2 && std::fabs(vals.back() - vals[vals.size() - 2]) < tol) break;
    }
    err_steps = 0;
    const size_t n = vals.size(), from = n >= 3 ? n - 3 : 0;
    for (size_t i = from + 1; i < n; ++i) err_steps = std::max(err_steps, std::fabs(vals[i] - vals[i - 1]));
    results.push_back(vals.back());
    if (st->nchi < 8) {
      st->chi[st->nchi] = chi;
      st->value_at_chi[st->nchi] = vals.back();
      st->steps_at_chi[st->nchi] = int32_t(n);
    }
    ++st->nchi;
    const size_t r = results.size();
    if (r >= 2 && std::fabs(results[r - 1] - results[r - 2]) < tol) break;
    if (2 * chi > chi_max) break;
    chi *= 2;
  }
  const size_t r = results.size();
  st->value = results.back();
  st->error_steps = err_steps;
  st->error_chi = r >= 2 ? std::fabs(results[r - 1] - results[r - 2]) : 0.0;
  st->error = std::max(st->error_steps, st->error_chi);
  st->chi_final = chi;
}

}  // namespace bst
