/*
 * bst.h -- C ABI of the block-sparse symmetric tensor library (GB300, sm_103a).
 *
 * A symmetric tensor is a direct sum of dense reduced blocks, each labelled
 * by one conserved charge per leg (Sec. 2, Eqs. "tensor-blocks" and
 * "tensor-cgc").  Every leg has a direction (flow); a block is allowed iff
 * its charges satisfy the addition rule sum_i flow_i * q_i = 0, all other
 * blocks being identically zero (Sec. 2, worked example and the remark on
 * forbidden blocks; no global charge shift is allowed).  For U(1) the
 * generalised Clebsch-Gordan coefficient of a block is a single number and
 * the rule is enforced by hand (Sec. 2, text after Eq. "tensor-cgc").
 *
 * Conventions used by every call:
 *   - charges are integers: 2*Sz for U(1), doubled spins 2j for SU(2);
 *   - a leg's sectors are given with strictly ascending charges and
 *     positive reduced degeneracies (Sec. 2, "Reduced and Total
 *     Dimensions": the reduced dimension is the sum of the degeneracies);
 *   - canonical layout: blocks are the allowed sector tuples sorted
 *     lexicographically by per-leg sector index (leg 0 most significant);
 *     each block is dense row-major (leg 0 slowest); blocks are stored
 *     back to back, so a tensor's data is one array of nnz doubles;
 *   - all data pointers named `*_data` / `a`, `b`, `c`, ... are DEVICE
 *     pointers owned by the caller; the library never frees them;
 *   - layouts are immutable and reference counted; every call that returns
 *     a layout returns a new reference the caller must release;
 *   - compute calls are asynchronous and ordered on the given stream; the
 *     returned status covers argument, symmetry and planning errors and
 *     launch failures; device-side errors (bounded waits, non-finite
 *     values) are recorded in a device error word read by bst_ctx_sync;
 *   - no C++ exception and no abort crosses this interface; on error the
 *     output arguments are left untouched and bst_last_error() returns a
 *     message for the calling thread.
 */
#ifndef BST_H
#define BST_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BST_API __attribute__((visibility("default")))
#else
#define BST_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* bst_stream; /* a cudaStream_t; NULL = legacy default */

typedef enum {
  BST_OK = 0,
  BST_E_ARG = 1,          /* bad argument (null pointer, out-of-range index, ...) */
  BST_E_SYMMETRY = 2,     /* flows/charges do not match on contracted legs */
  BST_E_SHAPE = 3,        /* sizes/capacities inconsistent */
  BST_E_OOM = 4,          /* device or host allocation failed */
  BST_E_CUDA = 5,         /* CUDA runtime/library error */
  BST_E_TIMEOUT = 6,      /* a bounded device wait expired */
  BST_E_NUMERIC = 7,      /* non-finite value or failed decomposition */
  BST_E_UNSUPPORTED = 8   /* valid request the library does not implement */
} bst_status;

/* Symmetry group of a layout.
 *   BST_U1:  charges are integers (2 S_z); a block is one sector per leg with
 *            sum_i flow_i q_i = 0; its data is the dense block.
 *   BST_SU2: charges are doubled spins 2j >= 0; degeneracies count
 *            multiplets (reduced dimensions).  A block is one sector per leg
 *            plus a fusion tree, and stores only the reduced tensor; its
 *            full form is reduced (x) CGC tensor (Sec. 2, Eq. "tensor-cgc").
 *            The CGC tensor of a block maps its outgoing legs to its
 *            incoming legs through one coupled spin J:
 *              c[m_in; m_out] = sum_M <in-tree m_in|J M> <out-tree m_out|J M>,
 *            each tree coupling its legs left to right (leg order) with
 *            Condon-Shortley Clebsch-Gordan coefficients (no leg: J = 0; one
 *            leg: J = its spin).  Tree labels (bst_layout_tree): the in-tree
 *            intermediates, J, the out-tree intermediates, as doubled spins.
 *            Blocks are ordered by sector indices, then tree labels.
 *   BST_Z2:  charges are parities 0 or 1 (the paper's third symmetry, Sec. 4.1
 *            compares none, Z2, U(1) and SU(2)); a block is allowed iff
 *            sum_i q_i is even, a fused leg's charge is the parity of its
 *            members' sum, and the pairing of sectors through a cut matches
 *            equal parities.  Everything else is as for BST_U1: every
 *            operation that takes BST_U1 layouts takes BST_Z2 layouts. */
typedef enum { BST_U1 = 1, BST_SU2 = 2, BST_Z2 = 3 } bst_group;

/* Arithmetic of the block GEMMs.
 *   BST_FP64:   plain FP64 (DMMA) grouped GEMM;
 *   BST_OZAKI:  FP64 operands split into five integer-valued BF16 slices
 *               with a shared power-of-two scale per row; slice products run
 *               on the tcgen05 tensor cores with FP32 accumulation in tensor
 *               memory, exact over short K chunks, and are recombined with
 *               FP64 weights in the epilogue.  ~44 significant bits (the 15
 *               slice products of weight >= 2^-36 of the leading one);
 *   BST_BF16X3: the cheaper mode: three slices (26 bits of each operand)
 *               and their 6 products of weight >= 2^-18, accumulated
 *               exactly; relative error ~2^-25 of sum |a||b| (FP32 class)
 *               at 40% of BST_OZAKI's tensor-core work and 60% of its
 *               operand bytes.  The block contractions run in it; the
 *               projector's eigensolver and subspace iterations, which must
 *               resolve singular values far below the largest, run in
 *               BST_OZAKI.
 * Any other value: BST_E_ARG. */
typedef enum { BST_FP64 = 0, BST_OZAKI = 1, BST_BF16X3 = 2 } bst_prec;

typedef struct {
  int32_t flow;           /* +1 incoming, -1 outgoing */
  int32_t nsect;          /* number of sectors (>0) */
  const int32_t* charge;  /* nsect charges, strictly ascending */
  const int64_t* deg;     /* nsect reduced degeneracies, each > 0 */
} bst_leg;

typedef struct bst_ctx_s* bst_ctx;
typedef struct bst_layout_s* bst_layout;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `workspace_bytes` is the initial
 * size of the device workspace used for intermediates (0: grow on demand at
 * plan time; once a plan is cached its calls allocate nothing). */
BST_API bst_status bst_ctx_create(int device, size_t workspace_bytes, bst_ctx* out);
BST_API bst_status bst_ctx_destroy(bst_ctx ctx);
/* Thread-local message of the last failed call on this thread ("" if none). */
BST_API const char* bst_last_error(void);
/* Synchronise `stream`, then read and clear the device error word.
 * Returns BST_E_TIMEOUT / BST_E_NUMERIC if a kernel recorded one. */
BST_API bst_status bst_ctx_sync(bst_ctx ctx, bst_stream stream);
/* Number of kernels this context launched so far (all calls). */
BST_API int64_t bst_ctx_launch_count(bst_ctx ctx);
/* Algorithmic work issued so far by this context's contractions, in
 * FP64-equivalent flops: 2 M N K summed over the matched block pairs of
 * every contraction (Sec. 2: the block products a symmetric contraction
 * consists of; U(1) sector GEMMs, SU(2) reduced pair products, batched
 * contractions) and over the projector's P and Pt products, enumerated
 * from the cached plans whatever the arithmetic.  The projector's own
 * eigensolver work (subspace iterations, Rayleigh-Ritz, refinement) is not
 * counted.  0 for a NULL context. */
BST_API double bst_ctx_work_flops(bst_ctx ctx);
/* Eigensolver behind bst_svd_projector and bst_ctm_move.
 *   BST_PROJ_SUBSPACE (default): per sector of N, subspace iteration on
 *     N^T N with a block of b vectors (CholQR orthonormalisation; b = 160
 *     for BST_FP64, for BST_OZAKI k + k/2 + 16 rounded up to 32 in 64..160,
 *     k the most states the sector can hold: chi, or chi / (2J+1) for an
 *     SU(2) sector of spin J), in rounds (the first two of `iters` steps,
 *     later ones sized by the residual's observed decay), each closed by a
 *     Rayleigh-Ritz step in FP64 (FP32 Jacobi eigensolver refined by
 *     Ogita-Aishima steps); sectors of dimension <= 160 are decomposed
 *     directly.  A round is accepted when every Ritz pair the truncation
 *     keeps has a residual ||N^T N v - lambda v|| <= tol * lambda_max (tol
 *     3e-14 for BST_FP64, 4e-12 for BST_OZAKI, whose iterations run on the
 *     tensor cores), or when the residual has stopped falling within
 *     100 tol.  Falls back to BST_PROJ_GESVD after 480 steps, or when the
 *     truncation keeps states within 16 of a sector's block edge.
 *     The context remembers, per sector structure, what earlier calls found
 *     and schedules later ones by it; the kept states and the residual test
 *     are unaffected, the rounding of the result may differ from a first
 *     call's (same context and call sequence: same bits):
 *       - U(1): directly decomposed sectors all below the truncation cut
 *         last time (Frobenius norm under the chi-th largest Ritz value)
 *         are checked again after the first Rayleigh-Ritz step and then not
 *         decomposed (they hold no kept state);
 *       - BST_OZAKI: when the last call needed several rounds, the
 *         intermediate Rayleigh-Ritz steps run in the mixed arithmetic and
 *         one more round without iterations repeats it in FP64.
 *   BST_PROJ_GESVD: full FP64 SVD of every sector with cuSOLVER gesvd. */
typedef enum { BST_PROJ_GESVD = 0, BST_PROJ_SUBSPACE = 1 } bst_proj_method;
BST_API bst_status bst_ctx_set_projector(bst_ctx ctx, int32_t method, int32_t iters);
/* Bound of every wait inside the tensor-core GEMM's pipeline (a thread
 * polling an mbarrier for a copy, a product or a drained accumulator), in
 * polls; 0 restores the default (2^28).  When a wait runs out the kernel
 * records BST_E_TIMEOUT (returned by the next bst_ctx_sync), waits for the
 * copies and products it has already issued (they always complete), frees
 * its tensor memory and returns; the context stays usable.  A small bound
 * makes the waits of a normal launch run out (for testing that path). */
BST_API bst_status bst_ctx_set_wait_limit(bst_ctx ctx, int64_t tries);
/* Autotuner of bst_contract_batched (on by default).  When on, the first
 * call of a new batch (per arithmetic) times every candidate schedule on
 * the call's own data, keeps the fastest for all later calls and appends
 * one line per timing to the context's tuning log.  Candidates: elements
 * per CTA of the gather and scatter launches (1024, 2048, 4096, 8192) and
 * the GEMM tile schedule (problem order, longest K first, or - for the
 * tensor-core GEMM - column tiles outer).  The schedule does not change any
 * result bit.  Tuning writes only the plan's own buffers. */
BST_API bst_status bst_ctx_set_autotune(bst_ctx ctx, int32_t enable);
/* Copies the tuning log (NUL-terminated, truncated to cap bytes) into buf
 * and its full length into *len (either may be NULL). */
BST_API bst_status bst_ctx_tuning_log(bst_ctx ctx, char* buf, size_t cap, size_t* len);
/* Per-kernel-class timing: enable != 0 starts recording a CUDA event pair
 * around every launch of the library's kernels on its stream (and clears
 * earlier records); 0 stops.  Synchronises the device. */
BST_API bst_status bst_ctx_profile(bst_ctx ctx, int32_t enable);
/* Aggregate of kernel class idx (0-based, in first-launch order): its name
 * (NUL-terminated, at most cls_len bytes), launches, summed event time in
 * ms, summed algorithmic FLOPs and bytes.  BST_E_ARG past the last class.
 * Waits for the recorded events. */
BST_API bst_status bst_ctx_profile_read(bst_ctx ctx, int32_t idx, char* cls, int32_t cls_len,
                                        int64_t* launches, double* ms, double* flops, double* bytes);

/* ---- layouts -------------------------------------------------------------- */

/* Canonical block layout of a tensor with the given legs (Sec. 2, Eq.
 * "tensor-blocks").  BST_E_ARG for rank < 1 or > 8, unsorted charges or
 * non-positive degeneracies. */
BST_API bst_status bst_layout_create(bst_ctx ctx, bst_group group, int32_t rank,
                             const bst_leg* legs, bst_layout* out);
BST_API bst_status bst_layout_retain(bst_layout l);
BST_API bst_status bst_layout_release(bst_layout l);
/* rank, number of blocks and number of stored elements. */
BST_API bst_status bst_layout_info(bst_layout l, int32_t* rank, int64_t* nblocks, int64_t* nnz);
/* Leg i: flow and sector count; if `charges`/`degs` are non-NULL they
 * receive nsect entries each. */
BST_API bst_status bst_layout_leg(bst_layout l, int32_t i, int32_t* flow, int32_t* nsect,
                          int32_t* charges, int64_t* degs);
/* Block i in canonical order: per-leg sector indices (rank entries),
 * element offset into the data array, per-leg extents (rank entries). */
BST_API bst_status bst_layout_block(bst_layout l, int64_t i, int32_t* sector_idx,
                            int64_t* offset, int64_t* shape);
/* Tree labels of block i of an SU(2) layout: *ntree labels (doubled spins:
 * in-tree intermediates, the coupled J, out-tree intermediates) into
 * `labels` if non-NULL.  U(1) layouts report *ntree = 0. */
BST_API bst_status bst_layout_tree(bst_layout l, int64_t i, int32_t* ntree, int32_t* labels);
/* Clebsch-Gordan coefficient <j1 m1 j2 m2 | J M> with every argument doubled
 * (Condon-Shortley phases), as the library uses it for SU(2) blocks.  Host
 * only; 0 for forbidden arguments. */
BST_API bst_status bst_su2_cg(int32_t tj1, int32_t tm1, int32_t tj2, int32_t tm2, int32_t tJ, int32_t tM,
                              double* out);
/* The dual layout: every flow reversed, same blocks, same storage order
 * (the conjugate tensor of Sec. 3.2's double layer A*). */
BST_API bst_status bst_layout_dual(bst_layout l, bst_layout* out);

/* ---- tensor operations ----------------------------------------------------- */

/* dst = src with legs permuted: dst leg j is src leg perm[j].  Returns the
 * canonical layout of the permuted legs in *dst (new reference) and writes
 * nnz(src) doubles to dst_data (must not alias src_data).  SU(2): the trees
 * of the permuted legs are recoupled: reduced block t' of dst is
 * sum_t R[t', t] (block t of the same sector tuple, legs permuted) with
 * R[t', t] = <c'_t', c_t permuted> / (2J'+1) from the Clebsch-Gordan
 * tensors (Sec. 2, Eq. tensor-cgc), so the dense tensor is permuted
 * exactly. */
BST_API bst_status bst_permute(bst_ctx ctx, bst_layout src, const double* src_data,
                       const int32_t* perm, bst_layout* dst, double* dst_data,
                       bst_stream stream);

/* Merge consecutive legs (Sec. 3.2: merging legs).  group_sizes[g] legs of
 * src (in order) become output leg g; sum(group_sizes) == rank(src).  The
 * fused leg takes the flow of its first member; its charge is
 * flow_0 * sum_i flow_i q_i; its sectors ascend in charge; inside a sector
 * the member-sector tuples ascend lexicographically and the inner index of
 * a tuple is row-major over the member legs.  Writes nnz(src) doubles. */
BST_API bst_status bst_fuse(bst_ctx ctx, bst_layout src, const double* src_data,
                    int32_t ngroups, const int32_t* group_sizes,
                    bst_layout* dst, double* dst_data, bst_stream stream);

/* Output layout of contracting legsA[i] of A with legsB[i] of B (Sec. 2,
 * contraction of block pairs with equal charges on the contracted legs).
 * Output legs: A's open legs in order, then B's open legs.  Contracted
 * legs must have opposite flows and identical sector lists
 * (BST_E_SYMMETRY otherwise). */
BST_API bst_status bst_contract_layout(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs,
                               const int32_t* legsA, const int32_t* legsB,
                               bst_layout* C);

/* Algorithmic work of contract(A, B) over the given leg pairs, without
 * running it: 2 M K N summed over every pair of blocks of A and B that agree
 * on the contracted legs (Sec. 2's block-pair contraction), in *flops.
 * Plans on the host only, so a host-only context (device -1) may answer it
 * (used to balance a batch of contractions over GPUs before any device
 * work).  U(1) layouts (BST_E_UNSUPPORTED otherwise); errors as
 * bst_contract_layout. */
BST_API bst_status bst_contract_flops(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs,
                                      const int32_t* legsA, const int32_t* legsB, double* flops);

/* Self-check of the sector matching (Sec. 2: block pairs matched by the
 * charges on the contracted legs, results reduced by the output charges).
 * Contraction plans take their relayout task lists (every block's place in
 * its sector matrix, and the launch's chunk table) from a device planner:
 * one CTA per view enumerates the leg configurations with their charges and
 * extents, offsets them within each charge, keeps the sector keys some block
 * carries and writes one task per block; a second kernel matches the sectors
 * of A, B and C into the GEMM problem list.  This call builds those tables
 * on the device for contract(A, B) and compares them with the host
 * planner's, entry by entry: *mismatches receives the number of entries
 * that differ (0 when they are identical).  U(1) and Z2 layouts.
 * Synchronises the device. */
BST_API bst_status bst_plan_check(bst_ctx ctx, bst_layout A, bst_layout B, int32_t npairs, const int32_t* legsA,
                                  const int32_t* legsB, int64_t* mismatches);

/* c = alpha * contract(a, b) + beta * c, with C the layout from
 * bst_contract_layout.  Matched block pairs are grouped by the conserved
 * charge through the cut, so every group is one dense GEMM whose result is
 * already reduced (Sec. 2, grouping by output quantum numbers so the
 * unreduced result never exists).  `prec` selects the GEMM arithmetic.
 * beta == 0 ignores the previous contents of c (NaN-safe).
 * SU(2) tensors (both A and B BST_SU2): every pair of blocks that agree on
 * the contracted legs contributes m_A . m_B, expanded into the output's
 * canonical blocks with X = <c_C, c_A . c_B> / (2 J_C + 1) (Sec. 2: the CGC
 * of a pair product is the product of the CGCs, then parallel blocks are
 * reduced).  The pair products of one contracted sector tuple form one GEMM;
 * a recoupling launch adds them with their X into the output blocks.  The
 * other tensor operations below are U(1)-only (BST_E_UNSUPPORTED). */
BST_API bst_status bst_contract(bst_ctx ctx, bst_layout A, const double* a,
                        bst_layout B, const double* b,
                        int32_t npairs, const int32_t* legsA, const int32_t* legsB,
                        bst_prec prec, double alpha, double beta,
                        bst_layout C, double* c, bst_stream stream);

/* bst_contract for callers that cannot allocate device memory: a process
 * whose device memory is owned and pre-sized by another runtime (a
 * framework's caching allocator, a fixed-budget serving process), where a
 * cudaMalloc would fail or would synchronise the device at the wrong moment.
 * The paper has no counterpart: this is a packaging of the same contraction.
 *
 * Same arguments and result as bst_contract with prec = BST_FP64, but the
 * call allocates nothing: its intermediates (relayout and GEMM tables, the
 * three sector matrices) live in one static device array of 64 MiB that the
 * library module carries, which every GPU that loads the library holds until
 * the process exits.  Runs on the current CUDA device.  The first call on a
 * device (per CUDA context) looks up that array's device address; make that
 * first call before any stream capture begins.  A contraction whose tables
 * and sector matrices need more than 64 MiB fails with BST_E_SHAPE.  All
 * calls share the array, so calls that overlap on the GPU (different streams
 * without ordering between them) race.  The layouts may come from a host-only
 * context (bst_ctx_create with device -1), whose use allocates no device
 * memory at all; C must be the layout bst_contract_layout returns. */
BST_API bst_status bst_contract_noalloc(bst_ctx ctx, bst_layout A, const double* a, bst_layout B,
                                        const double* b, int32_t npairs, const int32_t* legsA,
                                        const int32_t* legsB, double alpha, double beta,
                                        bst_layout C, double* c, bst_stream stream);

/* A batch of independent contractions (Sec. 2: contracting two symmetric
 * tensors is a set of independent dense block products, so products from
 * many contractions can share one launch):
 *     c[i] = alpha * contract(a[i], b[i]) + beta * c[i],   i < nbatch,
 * every one over the same leg pairs (legsA, legsB), each exactly as
 * bst_contract would compute it.  A, a, B, b, C, c are HOST arrays of
 * nbatch entries: layouts (A[i], B[i] any structure; C[i] the layout
 * bst_contract_layout returns for A[i], B[i]) and device data pointers.
 * Whatever nbatch is, the tensor-core arithmetics (BST_OZAKI, BST_BF16X3)
 * take two launches when every operand's last contracted leg (in pair
 * order) is its innermost leg: one gathers every operand row of every
 * contraction from its blocks and splits it into digits, one grouped GEMM
 * writes every output block in its epilogue (alpha, beta applied there);
 * otherwise three: one gather of both operands' sector matrices, one split,
 * the GEMM.  BST_FP64 takes one gather, one grouped DMMA GEMM and one
 * scatter.  The first call with a given list of layouts builds and
 * caches the plan, and the first call with a given list of data pointers
 * uploads a pointer table (both allocate and synchronise); a repeated call
 * launches those kernels and nothing else, so it may be captured into a
 * CUDA graph and replayed.
 * The c[i] must not overlap one another or any input (they are written
 * concurrently), and must be 8-byte aligned.  Errors: BST_E_ARG (NULL entries, nbatch < 1),
 * BST_E_SYMMETRY (a leg pair does not match), BST_E_SHAPE (C[i] wrong). */
BST_API bst_status bst_contract_batched(bst_ctx ctx, int32_t nbatch, const bst_layout* A, const double* const* a,
                                        const bst_layout* B, const double* const* b, int32_t npairs,
                                        const int32_t* legsA, const int32_t* legsB, bst_prec prec, double alpha,
                                        double beta, const bst_layout* C, double* const* c, bst_stream stream);

/* Double layer of a site tensor A[p,l,u,r,d] (Sec. 3.2): a = sum_p A (x) A*,
 * ket and bra legs fused pairwise into rank-4 legs [l,u,r,d] (fused charge
 * q_ket - q_bra).  If R is non-NULL it is a remover R[r,l',s] (Sec. 3.1,
 * incoming r, outgoing l' and s); its double layer is absorbed on the right
 * leg so that the result's right leg carries l''s structure.
 * First call with a == NULL to get the output layout in *a_layout (new
 * reference); then call again with the same inputs, *a_layout set and a
 * device buffer a of nnz(*a_layout) doubles. */
BST_API bst_status bst_double_layer(bst_ctx ctx, bst_layout A, const double* A_data,
                            bst_layout R, const double* R_data,
                            bst_layout* a_layout, double* a, bst_stream stream);

/* SVD projectors of a CTMRG move (Sec. 3: the truncation the paper takes
 * from corboz14).  Rtop[alpha, beta] and Rbot[alpha', beta'] are the two
 * half systems; their first `ncut` legs are the left cut (alpha, alpha')
 * and the remaining legs the right cut (beta, beta').  With
 * N = Rtop^T Rbot (over the left cut) = U S V^T per conserved-charge sector,
 * the chi largest singular values over all sectors are kept (ties: smaller
 * |q| then smaller q, where q is the charge of the new leg; values below
 * rel_cutoff * sigma_max dropped), and
 *     P  = Rbot V S^-1/2    legs [alpha'..., new]   (new leg flow new_flow)
 *     Pt = S^-1/2 U^T Rtop^T legs [new^dual, alpha...]
 * with the sign of every kept left singular vector fixed by making its
 * largest-magnitude entry positive (lowest index on ties).  The new leg
 * lists sectors by ascending charge, singular values descending inside a
 * sector.  p and pt are device buffers of at least dim(alpha')*chi and
 * chi*dim(alpha) doubles; svals (HOST, chi doubles) receives the kept
 * singular values in new-leg order; *kept their count.  This call
 * synchronises the stream once (the global truncation is a host decision). */
BST_API bst_status bst_svd_projector(bst_ctx ctx, bst_layout Rtop, const double* rtop,
                             bst_layout Rbot, const double* rbot, int32_t ncut,
                             int64_t chi, double rel_cutoff, int32_t new_flow,
                             bst_prec prec,
                             bst_layout* P, double* p, bst_layout* Pt, double* pt,
                             double* svals, int64_t* kept, bst_stream stream);

/* Batched dense symmetric eigendecomposition used by the projector: batch
 * row-major n x n symmetric matrices H (device, back to back, n <= 160) ->
 * eigenvectors X (device, same layout, column j = eigenvector j) and
 * eigenvalues lam (device, n per matrix, descending).  Two FP32 Jacobi
 * passes followed by three Ogita-Aishima refinement steps whose matrix
 * products run in `prec`.  Accuracy: eigenvalues above 1e-6 lambda_max (and
 * their eigenvectors, where separated) reach FP64 accuracy (BST_FP64) or
 * ~1e-12 lambda_max (BST_OZAKI); eigenvalues below 1e-6 lambda_max form one
 * cluster the FP32 stage does not resolve and are accurate only to about
 * 1e-9 lambda_max in absolute terms, with their eigenvectors spanning that
 * cluster's subspace.  No counterpart in the paper (a building block of the
 * SVD it uses). */
BST_API bst_status bst_sym_eig(bst_ctx ctx, int32_t n, int32_t batch, const double* H, double* X,
                               double* lam, bst_prec prec, bst_stream stream);

/* One-site CTMRG environment: corners C1..C4 and edges T1..T4 (index 0..3).
 * Legs: C1[R,D] C2[L,D] C3[U,L] C4[U,R]  T1[L,D,R] T2[U,L,D] T3[L,U,R]
 * T4[U,R,D]; the site tensor is a[L,U,R,D].  c[i], t[i] are device buffers
 * with capacities c_cap[i], t_cap[i] (doubles); a move rewrites the buffers
 * of the tensors it renews in place and replaces their layouts (releasing
 * the old references). */
typedef struct {
  bst_layout C[4], T[4];
  double* c[4];
  double* t[4];
  int64_t c_cap[4], t_cap[4];
} bst_env;

typedef struct {
  int64_t kept[4];        /* kept states per directional move (L,R,U,D order of execution) */
  double smin_over_smax[4];
  /* sum of discarded sigma / sum of all computed sigma: every sigma of a
   * directly decomposed sector, the leading block of an iterated one; a
   * small sector whose Frobenius norm is below the cut holds no kept state
   * and is not decomposed (it adds nothing to either sum) */
  double trunc_weight[4];
} bst_ctm_stats;

/* CTMRG move on a one-site cell (Sec. 3 and Sec. 3.2): dir 0 = LEFT (renews
 * C1, T4, C4), 1 = UP (C1, T1, C2), 2 = RIGHT (C2, T2, C3), 3 = DOWN
 * (C3, T3, C4), 4 = the full move LEFT, RIGHT, UP, DOWN in sequence, each
 * on the updated environment.  Every directional move computes the four
 * enlarged corners, the half systems, the projectors (as
 * bst_svd_projector with rel_cutoff) and renormalises and normalises the
 * renewed tensors (Frobenius norm 1).  stats may be NULL.
 *
 * Site: either the double layer a[L,U,R,D] (rank 4), or a single-layer
 * site A[P,L,U,R,D] (rank 5, U(1) only) whose double layer
 * sum_P A (x) A* has the legs fuse(A.x, A.x^dual); then a is never formed:
 * every contraction with it runs as a contraction with A and one with A*
 * (the edges' site legs are split into ket and bra parts and fused back).
 *
 * SU(2) (site and environment BST_SU2): dir 0 only (the other directions
 * permute legs, which for SU(2) blocks needs tree recoupling:
 * BST_E_UNSUPPORTED); chi is the total dimension of the new bond, filled by
 * whole multiplets in descending singular value (one that would overflow
 * chi is skipped), stats->kept is that total dimension; the new bond is
 * incoming on C1' and T4' (outgoing on T4''s first leg and on C4'). */
BST_API bst_status bst_ctm_move(bst_ctx ctx, int32_t dir, bst_layout a_layout, const double* a,
                        bst_env* env, int64_t chi, double rel_cutoff, bst_prec prec,
                        bst_ctm_stats* stats, bst_stream stream);

/* CTMRG move of an Lx x Ly unit cell (Sec. 3.1's unit cells; Sec. 4.1 times
 * a 2 x 2 cell): site i = x + Lx y (x right, y down) has the double layer
 * a[i] (rank 4, layout a_layouts[i]; BST_U1 or BST_Z2) and its own
 * environment envs[i] (its C1..C4, T1..T4 around it).  The LEFT move
 * absorbs the cell column by column: for column x, the plaquette of sites
 * (x, y), (x+1, y), (x, y+1), (x+1, y+1) (positions periodic) gives the
 * projectors of the cut between rows y and y+1 (as bst_svd_projector); then
 * every site (x, y) is absorbed into the left environment of (x+1, y):
 * C1 <- (C1 T1) P_above, T4 <- P~_above (T4 a) P_below, C4 <- P~_below
 * (C4 T3), each normalised; later columns see the renewed tensors.  The
 * other directions turn the cell by quarter turns (the site at (x, y) goes
 * to (y, -x mod Lx)) and every tensor as in bst_ctm_move; dir 4 runs LEFT,
 * RIGHT, UP, DOWN.  A 1 x 1 cell is bst_ctm_move.  a_layouts, a and envs
 * are HOST arrays of Lx Ly entries; renewed tensors are written into the
 * envs' buffers (capacities as for bst_ctm_move) and their layouts
 * replaced.  Errors: BST_E_ARG (NULL entries, Lx Ly outside 1..64, a site
 * not of rank 4, mixed groups), BST_E_UNSUPPORTED (SU(2)), BST_E_SYMMETRY
 * (legs of neighbouring sites do not match), BST_E_SHAPE (capacity). */
BST_API bst_status bst_ctm_move_cell(bst_ctx ctx, int32_t dir, int32_t Lx, int32_t Ly, const bst_layout* a_layouts,
                                     const double* const* a, bst_env* envs, int64_t chi, double rel_cutoff,
                                     bst_prec prec, bst_stream stream);

/* ---- observables and the CTM error procedure ------------------------------ */

/* Open double layer of a site A[p,l,u,r,d] (Sec. 3.2 with the physical legs
 * kept open): ket and bra multiplied without the sum over p, virtual ket/bra
 * legs fused pairwise as in bst_double_layer, the remover R[r,l',s]
 * (Sec. 3.1; its extra leg traced between ket and bra) absorbed on the
 * right leg when R is non-NULL.  Legs [L, U, R, D, p, p'] (p the ket's
 * physical leg, p' the bra's, its dual).  Summing p = p' gives
 * bst_double_layer's tensor.  Two calls as for bst_double_layer: a == NULL
 * returns the layout in *a_layout (new reference); then a device buffer of
 * nnz(*a_layout) doubles.  U(1) and Z2. */
BST_API bst_status bst_double_layer_open(bst_ctx ctx, bst_layout A, const double* A_data, bst_layout R,
                                         const double* R_data, bst_layout* a_layout, double* a, bst_stream stream);

/* Two-site reduced density matrix of a bond of the one-site cell from its
 * environment (the observable of Sec. 3's error procedure and of Sec. 4.1's
 * energies): bond 0 = horizontal (the site and its right neighbour, the
 * 3 x 4 network C1 T1 T1 C2 / T4 a a T2 / C4 T3 T3 C3 with both sites
 * open), 1 = vertical (the site and the one below: the network turned by a
 * quarter turn).  site is the open double layer [L,U,R,D,p,p'].  Result
 * rho[p_i, p_i', p_j, p_j'] (not normalised; Tr rho is the closed network's
 * value) in *rho_layout (new reference); its nnz(*rho_layout) doubles are
 * copied to the device buffer rho if rho is non-NULL (capacity rho_cap
 * doubles, BST_E_SHAPE if too small).  The contractions run in prec. */
BST_API bst_status bst_ctm_bond_rdm(bst_ctx ctx, int32_t bond, bst_layout site, const double* site_data,
                                    bst_env* env, bst_prec prec, bst_layout* rho_layout, double* rho,
                                    int64_t rho_cap, bst_stream stream);

/* sum_i x_i y_i over the nnz(layout) stored elements of two tensors with the
 * same layout (for U(1) and Z2 the Frobenius inner product; Tr(rho H) when H
 * is the operator's tensor in rho's layout), in FP64 with a fixed summation
 * order, into *out (host).  Synchronises the stream. */
BST_API bst_status bst_dot(bst_ctx ctx, bst_layout layout, const double* x, const double* y, double* out,
                           bst_stream stream);

typedef struct {
  double value;          /* observable at the last chi */
  double error;          /* max(error_steps, error_chi) */
  double error_steps;    /* largest change among the last three steps at the last chi */
  double error_chi;      /* change between the last two fixed-chi results (0 with one chi) */
  int64_t chi_final;     /* chi of the last fixed-chi run */
  int32_t steps_total;   /* full CTM moves done */
  int32_t nchi;          /* fixed-chi runs done */
  int64_t chi[8];        /* per run (the first 8): chi, result and moves */
  double value_at_chi[8];
  int32_t steps_at_chi[8];
} bst_ctm_converge_stats;

/* The CTM error procedure of Sec. 3 (implementation details) on a one-site
 * cell: full moves (bst_ctm_move, dir 4) at fixed chi until the energy per
 * site changes by less than tol or max_steps moves are done (the paper:
 * 1e-8 and 15); the first error is the largest change among the last three
 * moves.  chi is then doubled and the procedure repeated until two
 * fixed-chi results differ by less than tol or doubling would exceed
 * chi_max (the paper: 128); the second error is the change between the last
 * two fixed-chi results; stats->error is the larger.  The energy per site is
 * the sum over the horizontal and vertical bonds of Tr(rho H) / Tr(rho)
 * (bst_ctm_bond_rdm, bst_dot), H a two-site operator given as a tensor with
 * rho's layout (H[p_i, p_i', p_j, p_j'] = <p_i p_j|h|p_i' p_j'>; for the
 * Heisenberg coupling S.S it conserves the charge, Sec. 3.1's charged
 * operators being combined on the bond).  a is the closed site (as for
 * bst_ctm_move), site the open one; env buffers need capacity for chi_max.
 * Synchronises the stream after every move (the stopping rule is a host
 * decision). */
BST_API bst_status bst_ctm_converge(bst_ctx ctx, bst_layout a_layout, const double* a, bst_layout site,
                                    const double* site_data, bst_layout H_layout, const double* H, bst_env* env,
                                    int64_t chi0, int64_t chi_max, double tol, int32_t max_steps,
                                    double rel_cutoff, bst_prec prec, bst_ctm_converge_stats* stats,
                                    bst_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* BST_H */
