/*
 * nsp.h — C ABI of a GB300 (sm_103a) implementation of the two-level Nyström–Schur
 * preconditioner M2 for sparse SPD systems in doubly bordered block diagonal (DBBD)
 * form (Al Daas, Rees & Scott, "Two-level Nyström–Schur preconditioner for sparse
 * symmetric positive definite matrices").
 *
 * Problem statement (§2.3, eq. (perm_A)): A is SPD and, after a symmetric permutation
 * given by a partition of its unknowns, has the form
 *
 *        [ A_I    A_IG ]      A_I = diag(A_1, ..., A_N) block diagonal (one block per
 *        [ A_GI   A_G  ]      subdomain), G = the interface (separator) Gamma.
 *
 * The library builds M2 = A_G^{-1} + Z Sigma Z^T (§4.3 eq. (left_prec_mat), Algorithm 2)
 * and solves S_Gamma w = f (§2.3 eq. (Sx=b)) with PCG preconditioned by M2, where
 * S_Gamma = A_G - A_GI A_I^{-1} A_IG (§2.3 eq. (schur_complement)).
 *
 * Conventions used by every entry point:
 *  - Orderings seen by callers. "Gamma order": interface unknowns (part[i] < 0) sorted by
 *    their index i in A. "Interior order": interior unknowns block by block (block 0
 *    first), each block sorted by index in A. Full-length vectors use A's own order.
 *  - Blocks of vectors are row-major: a block of s columns over m unknowns is m*s
 *    contiguous values, entry (i, j) at [i*s + j].
 *  - Device pointers are CUDA global-memory pointers on the current device; all device
 *    work is ordered on the handle's stream (nsp_params.stream, 0 = legacy default).
 *  - Entry points never abort. They return an nsp_status; after NSP_ERR_CUDA the handle
 *    should be destroyed. A NULL handle or pointer argument gives NSP_ERR_INVALID_ARG.
 *  - One handle must not be used concurrently from several host threads.
 */
#ifndef NSP_H
#define NSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NSP_OK = 0,
  NSP_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, malformed CSR, bad parameter      */
  NSP_ERR_NOT_DBBD = 2,      /* two different interior blocks are coupled in A           */
  NSP_ERR_NOT_SPD = 3,       /* non-positive pivot in a Cholesky factor (see failed_block) */
  NSP_ERR_BREAKDOWN = 4,     /* block CG lost every search direction / PCG p^T S p <= 0   */
  NSP_ERR_NOT_CONVERGED = 5, /* iteration cap reached; outputs still hold the last iterate */
  NSP_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (scheduler dependency)      */
  NSP_ERR_CUDA = 7,          /* a CUDA runtime error                                      */
  NSP_ERR_OOM = 8,           /* device allocation failed                                  */
  NSP_ERR_UNSUPPORTED = 9    /* valid request this build does not handle                  */
} nsp_status;

typedef enum { NSP_FP64 = 0, NSP_FP32 = 1 } nsp_precision;

/* Outer solve forms, both PCG preconditioned by M2 (§2.3, §4.3):
 *  NSP_OUTER_SCHUR : PCG on S_Gamma w = f, f = b_G - A_GI A_I^{-1} b_I, then
 *                    x_I = A_I^{-1}(b_I - A_IG w)  (block elimination, eq. (A_LDLT)).
 *  NSP_OUTER_FULL  : PCG on A x = b with the block-factorization preconditioner of §2.3
 *                    whose Schur-complement block is M2, from x0 = (A_I^{-1} b_I, 0). With
 *                    exact A_I^{-1} its iterates equal those of NSP_OUTER_SCHUR; with an
 *                    FP32 factor the operator A stays FP64, so the residual is exact.
 *  NSP_OUTER_AUTO  : FULL when the factor precision is FP32, SCHUR when it is FP64. */
typedef enum { NSP_OUTER_AUTO = 0, NSP_OUTER_SCHUR = 1, NSP_OUTER_FULL = 2 } nsp_outer_form;

/* Inner system of Algorithm 2 step 3:
 *  NSP_FORM_SGAMMA : block PCG on S_Gamma E = A_GI A_I^{-1} A_IG G preconditioned by A_G
 *                    (first level S1, §2.3 eq. (S1)), then Y = A_G E. By the SMW identity
 *                    (§4.1 eq. (S-1)) Y = A_GI S_I^{-1} A_IG G, the Y of Algorithm 2.
 *                    Block vectors of n_Gamma rows.
 *  NSP_FORM_SI     : the system as Algorithm 2 writes it: F = A_IG G (step 2), block PCG on
 *                    S_I X = F with S_I = A_I - A_IG A_G^{-1} A_GI (§4.1 eq. (SI))
 *                    preconditioned by A_I (§5 setup), Y = A_GI X (step 4). Block vectors
 *                    of n_interior rows; each iteration applies A_I^{-1} (preconditioner)
 *                    and A_G^{-1} (inside S_I). Same Y for exact solves; at a loose
 *                    tolerance the two forms stop at different iterates. Single handles
 *                    only (nsp_build_batched: NSP_ERR_UNSUPPORTED). */
typedef enum { NSP_FORM_SGAMMA = 0, NSP_FORM_SI = 1 } nsp_inner_form;

/* Preconditioner built from the Nyström factor (§4.3):
 *  NSP_VARIANT_M2      : M2 = A_G^{-1} + Z Sigma Z^T, Z = A_G^{-1} U (eq. (left_prec_mat),
 *                        Algorithm 2 step 12).
 *  NSP_VARIANT_M2_ADEF : M_{2A-DEF}, the adapted-deflation form that §4.3 defines like
 *                        eq. (deflation_comp_from_low_rank) / eq. (our_two_level_preconditioner)
 *                        for M2's approximation. Written without R_G (Z = A_G^{-1} U,
 *                        E = Z^T S_G Z, k x k):  M = (I - Z E^{-1} Z^T S_G) A_G^{-1} + Z E^{-1} Z^T.
 *                        The build adds one S_G apply on k columns and a k x k Cholesky
 *                        (columns of E whose pivot falls below drop_tol of their diagonal are
 *                        left out of the deflation space); each application costs the A_G
 *                        solve of M2 plus three length-n_G products with k columns. M is not
 *                        symmetric; the outer PCG uses it as is, as §5 does.
 *  NSP_VARIANT_M3      : M3 = A_G^{-1} + Zh Sigma Zh^T (§4.3 eq. (left_prec_mat2)): Nyström
 *                        (Algorithm 1) of S_I^{-1} ~ V Sigma V^T (eq.
 *                        (internal_term_lr_approximation_2)) from a sketch G_I of n_interior
 *                        x (k+p), X = S_I^{-1} G_I by the S_I block PCG (preconditioner A_I,
 *                        tolerance eps_inner, whatever inner_form says), Zh = A_G^{-1} A_GI V.
 *                        params.sketch, when given, is then n_interior x s row-major in
 *                        interior order (see nsp_factor_solve). q must be 0
 *                        (NSP_ERR_UNSUPPORTED otherwise); nsp_get_intermediate is refused.
 *  NSP_VARIANT_M3_ADEF : M_{3A-DEF}: the deflation of NSP_VARIANT_M2_ADEF on span(Zh).
 *  NSP_VARIANT_M1      : M1 = A_G^{-1} + Zb Sigma Zb^T (§4.1 eq. (prec1S)) with A_G = R^T R
 *                        the handle's own Cholesky factor of A_G (R = L^T P^T for its fill-
 *                        reducing order P, A_G's rows permuted by P factorized as L L^T):
 *                        Nyström (Algorithm 1) of R^{-T} A_GI S_I^{-1} A_IG R^{-1}
 *                        (eq. (lr_approximation_S-1_A-I)) from the sketch G: the block PCG of
 *                        steps 2-4 runs on the sketch R^{-1} G, the Nyström core on (G,
 *                        R^{-T} Y), and Zb = R^{-1} Ub. R^{-1} and R^{-T} are the backward and
 *                        the forward half of the A_G sweep. M1 depends on R, hence on the
 *                        ordering: two implementations with different orderings agree only
 *                        where the Nyström approximation is exact (then M1 = S_G^{-1}). q must
 *                        be 0 (NSP_ERR_UNSUPPORTED otherwise).
 * Single handles only: nsp_build_batched returns NSP_ERR_UNSUPPORTED for any but M2. */
typedef enum { NSP_VARIANT_M2 = 0, NSP_VARIANT_M2_ADEF = 1, NSP_VARIANT_M3 = 2,
               NSP_VARIANT_M3_ADEF = 3, NSP_VARIANT_M1 = 4 } nsp_variant;

/* Sparse matrix in CSR. Full symmetric pattern (both triangles) with sorted column
 * indices and no duplicates. rowptr has n+1 entries. Host pointers unless on_device. */
typedef struct {
  int64_t n;
  const int64_t *rowptr;
  const int32_t *col;
  const double *val;
  int32_t on_device;         /* 1: rowptr/col/val are device pointers (values read only) */
} nsp_csr;

/* DBBD partition (§2.3 eq. (perm_A)). part[i] in [0, nblocks) puts unknown i in interior
 * block part[i]; part[i] = -1 puts it on the interface Gamma. perm (optional, may be NULL)
 * lists interior unknowns in a fill-reducing elimination order: for each block, the
 * relative order of its unknowns in perm is the order in which the block is factorized.
 * perm has n_interior entries (every interior unknown once). Without perm, and always for
 * A_G, the library computes a nested-dissection order of the block's graph. Host memory. */
typedef struct {
  int32_t nblocks;
  const int32_t *part;
  const int64_t *perm;
} nsp_partition;

typedef struct {
  int32_t k;                 /* Nyström rank k > 0 (Algorithm 2 input)                    */
  int32_t p;                 /* oversampling p >= 0; sketch width s = k + p               */
  double eps_inner;          /* relative tolerance of the inner block PCG (paper: 0.1)    */
  double eps_trunc_rel;      /* Algorithm 2 step 7 threshold, relative to max eig(C)      */
  double drop_tol;           /* block-PCG column drop threshold (relative pivot)          */
  int32_t max_inner_it;      /* inner block-PCG iteration cap (e.g. 500)                  */
  uint64_t seed;             /* Gaussian sketch seed (Philox4x32-10 + Box-Muller)          */
  const double *sketch;      /* optional caller sketch G: n_Gamma x s row-major, Gamma
                                order (n_interior x s, interior order, for the M3
                                variants), host or device memory; NULL = draw from seed   */
  int32_t precision;         /* nsp_precision of the factors and the inner block PCG      */
  int32_t outer_form;        /* nsp_outer_form                                            */
  int32_t inner_form;        /* nsp_inner_form                                            */
  int32_t keep_intermediates;/* 1: keep E, Y, U of Algorithm 2 for nsp_get_intermediate  */
  void *stream;              /* cudaStream_t for all device work (NULL = default stream)  */
  int32_t variant;           /* nsp_variant (default NSP_VARIANT_M2); other values:
                                NSP_ERR_INVALID_ARG                                        */
  int32_t q;                 /* power iterations (§2.1 eq. (power)), 0 <= q <= 16, default 0:
                                G = B^q Omega with B = A_GI S_I^{-1} A_IG and Omega the drawn
                                or given sketch; each application of B is one inner block PCG
                                (steps 2-4) and the columns are orthonormalized after it by
                                Cholesky-QR (a column whose pivot falls below drop_tol of its
                                squared norm becomes zero). Batched handles: q = 0 only      */
  /* Recursive treatment of A_G (concluding section: the systems with A_G replaced by systems
   * with a much smaller matrix). gamma_levels = 0 (default): A_G is factorized directly.
   * gamma_levels = 1: A_G gets a DBBD split of its own (§2.3 eq. (perm_A) applied to A_G:
   * interior blocks C_i, a second-level interface G2) and every A_G^{-1} of the build and of
   * the preconditioner (the block-PCG preconditioner of step 3, Z = A_G^{-1} U of step 11, the
   * A_G^{-1} r of each M2 application, nsp_factor_solve(which = 1)) becomes the block
   * elimination of §2.3 eq. (A_LDLT) for that split whose Schur-complement solve is the M2 of
   * the split, M2' (Algorithm 2 on A_G, S_Gamma form, with gamma_k, gamma_p, gamma_eps_inner,
   * the sketch gamma_sketch or one drawn from seed + 1, and the handle's other parameters):
   *   y = C_I^{-1} b_I,  x_G2 = M2' (b_G2 - C_G2I y),  x_I = C_I^{-1} (b_I - C_IG2 x_G2).
   * Only the C_i and C_G2 are factorized. It equals A_G^{-1} when M2' = S_C^{-1} (the Schur
   * complement of C_I in A_G). Requires the M2 variant, the S_Gamma inner form and q = 0
   * (NSP_ERR_UNSUPPORTED otherwise; batched handles: gamma_levels = 0 only). The split is
   * fixed at nsp_build: nsp_rebuild refuses a change of gamma_levels and reads neither
   * gamma_part nor gamma_nblocks. nsp_get_factor refuses the A_G block of such a handle.   */
  int32_t gamma_levels;      /* 0 or 1                                                     */
  int32_t gamma_nblocks;     /* interior blocks of A_G's split (>= 1)                       */
  const int32_t *gamma_part; /* host, n_Gamma labels in the caller's Gamma order (increasing
                                index in A): [0, gamma_nblocks), or -1 for G2; no entry of
                                A_G may couple two different blocks (NSP_ERR_NOT_DBBD)     */
  int32_t gamma_k;           /* Nyström rank of M2' (> 0)                                  */
  int32_t gamma_p;           /* oversampling of M2' (>= 0), gamma_k + gamma_p <= n_G2, 256 */
  double gamma_eps_inner;    /* relative tolerance of M2''s block PCG                       */
  const double *gamma_sketch;/* optional sketch of M2', host, n_G2 x (gamma_k + gamma_p)
                                row-major, G2 unknowns in increasing index in A; NULL =
                                drawn from seed + 1                                         */
} nsp_params;

typedef struct {
  int64_t n, n_interior, n_gamma;
  int32_t nblocks;
  int64_t nnz_L_interior;    /* structural nonzeros of the interior Cholesky factors      */
  int64_t nnz_L_gamma;       /* structural nonzeros of the A_G Cholesky factor            */
  int64_t n_supernodes;
  int32_t it_inner;          /* block-PCG iterations (it_{S_I} of §5)                     */
  int32_t inner_active_cols; /* search-direction columns left at the last iteration      */
  int32_t rank;              /* Nyström rank min(r, k) (§2.1)                             */
  int32_t it_pcg;            /* outer PCG iterations of the last nsp_solve (it_PCG)      */
  double inner_residual;     /* max relative column residual at exit of the block PCG     */
  double final_residual;     /* ||b - A x|| / ||b|| of the last nsp_solve (FP64)          */
  double pcg_residual;       /* updated-residual ratio ||r|| / ||f|| at exit              */
  int32_t failed_block;      /* block id for NSP_ERR_NOT_SPD (nblocks = the A_G factor)   */
  double ms_analyze, ms_factor, ms_inner, ms_core, ms_solve;   /* host wall times (ms)     */
  int32_t it_power;          /* block-PCG iterations of the q power passes (it_inner is the
                                final pass's)                                              */
  /* Condition estimate of the preconditioned operator of the last nsp_solve (the kappa of
   * the CG error bound, §1 eq. (k-th_error_cg), and kappa_eff of §4.2): extreme eigenvalues
   * of the Lanczos tridiagonal formed from the outer PCG's coefficients (alpha_j step
   * lengths, beta_j direction ratios; CG and Lanczos share one Krylov basis), computed by
   * Sturm-sequence bisection. They are Ritz values of M2 S_Gamma (for NSP_OUTER_FULL the
   * same numbers: its iterates equal the Schur form's). 0 when no iteration ran; batched
   * handles leave them 0.                                                                  */
  double lambda_min_est, lambda_max_est, kappa_est;
  /* gamma_levels = 1: size of the second-level interface G2, block-PCG iterations and
   * Nyström rank of M2' at the last build (0 otherwise)                                    */
  int64_t n_gamma2;
  int32_t it_inner_gamma, rank_gamma;
} nsp_info;

typedef struct nsp_handle nsp_handle;

/* Defaults: k=16, p=10, eps_inner=0.1, eps_trunc_rel=1e-10, drop_tol=1e-12 (FP64) /
 * 1e-6 (FP32), max_inner_it=500, precision=NSP_FP32, AUTO outer form, seed=210112164,
 * gamma_levels=0 (gamma_k=16, gamma_p=8, gamma_eps_inner=0.1, no gamma_part/gamma_sketch). */
void nsp_default_params(nsp_params *prm);

/* Algorithm 2 end to end: analysis of A's pattern and the partition (host), numeric
 * Cholesky factorization of every A_i and of A_G on the device, sketch G (step 1), inner
 * block PCG (steps 2-4), Nyström core (steps 5-10), Z = A_G^{-1} U (step 11).
 * A is copied; the caller keeps ownership of all inputs. On success *out owns all device
 * memory of the preconditioner. Errors: INVALID_ARG, NOT_DBBD, NOT_SPD, BREAKDOWN, CUDA,
 * OOM, UNSUPPORTED; *out is NULL on error. The parameter checks that need no analysis of A
 * (k, p, k + p, precision, inner_form, variant, q; for batched handles also their
 * restrictions) run on the host before any device work. */
nsp_status nsp_build(const nsp_csr *A, const nsp_partition *P, const nsp_params *prm,
                     nsp_handle **out);

/* Many independent SPD systems in one handle (the paper builds M2 for one matrix; a batch
 * applies Algorithm 2 to each matrix on its own): A[0..count), P[0..count) host CSRs and
 * partitions (perm given for all or none), one parameter set for all (k + p <= 96, and
 * k + p <= n_Gamma of every matrix). The matrices are concatenated block-diagonally, so
 * one factorization launch per tree level and one persistent sweep launch per triangular
 * solve serve all of them, while every quantity of Algorithm 2 (s x s Grams, Cholesky-QR,
 * drop decisions, stopping test, Nyström core) and of the outer PCG (scalars, stopping
 * test) is computed per matrix; a matrix that has converged stops changing.
 * On a batched handle: vectors are the matrices' vectors stacked in matrix order (Gamma
 * vectors likewise: matrix 0's Gamma unknowns in its order, then matrix 1's, ...);
 * prm->sketch, if given, is the matrices' sketches stacked that way; nsp_rebuild takes the
 * concatenated value arrays; nsp_apply, nsp_schur_apply and nsp_factor_solve act on all
 * matrices at once; nsp_get_basis returns all k columns (rank = k) and count x k values of
 * Sigma (per matrix, zero beyond its rank, see nsp_solve_batched's infos for the ranks);
 * nsp_solve is refused (INVALID_ARG), use nsp_solve_batched. Errors as nsp_build. */
nsp_status nsp_build_batched(int32_t count, const nsp_csr *A, const nsp_partition *P,
                             const nsp_params *prm, nsp_handle **out);

/* Solve every system of a batched handle: b and x are the matrices' vectors stacked in
 * matrix order (sum of n doubles; host or device pointers, detected). Each matrix runs its
 * own outer PCG (full-space form with the block preconditioner, see nsp_outer_form) until
 * its own ||r|| / ||r0|| <= rtol; one launch of every kernel serves all matrices still
 * iterating. infos (may be NULL) receives count nsp_info records (it_inner, inner_residual,
 * rank, it_pcg, pcg_residual, final_residual of that matrix). NOT_CONVERGED if some matrix
 * reached maxit (x holds every matrix's last iterate). */
nsp_status nsp_solve_batched(const nsp_handle *h, const double *b, double *x, double rtol,
                             int32_t maxit, nsp_info *infos);

/* Repeat the numeric part of nsp_build (factorization + Algorithm 2) for new values of A
 * with the same pattern (val has nnz entries in the CSR order given to nsp_build; device
 * memory if on_device). prm may change k, p, tolerances, seed, sketch, variant, inner_form, q (not
 * precision). */
nsp_status nsp_rebuild(nsp_handle *h, const double *val, int32_t on_device,
                       const nsp_params *prm);

/* z = M2 r = A_G^{-1} r + Z Sigma Z^T r (Algorithm 2 step 12), or z = M_{2A-DEF} r when the
 * handle was built with NSP_VARIANT_M2_ADEF (see nsp_variant). r, z: n_Gamma doubles in
 * Gamma order, device pointers, may not alias. */
nsp_status nsp_apply(const nsp_handle *h, const double *r_gamma, double *z_gamma);

/* Solve A x = b (n doubles, A's order) to ||r|| / ||f|| <= rtol with the outer form of
 * the handle (see nsp_outer_form). b and x may be host or device pointers (detected);
 * host buffers are staged through device memory inside the call. info may be NULL.
 * NOT_CONVERGED after maxit iterations (x holds the last iterate). */
nsp_status nsp_solve(const nsp_handle *h, const double *b, double *x, double rtol,
                     int32_t maxit, nsp_info *info);

/* Y = S_Gamma X = A_G X - A_GI A_I^{-1} A_IG X (§2.3 eq. (schur_complement)) for an
 * n_Gamma x s block (Gamma order, row-major, 1 <= s <= 256), in the handle's precision:
 * X, Y are float* for NSP_FP32 handles and double* for NSP_FP64 handles. Device pointers,
 * may not alias. This is the operator applied inside the inner block PCG. The work is
 * enqueued on the handle's stream and the call returns without waiting: synchronize that
 * stream before reading Y. Only the first call with a new width s allocates. */
nsp_status nsp_schur_apply(const nsp_handle *h, const void *X, void *Y, int32_t s);

/* Same result as nsp_schur_apply, for callers that cannot allocate device memory (for
 * example code that runs while a CUDA stream is being captured into a graph, or under an
 * allocator that forbids cudaMalloc): this call allocates nothing. Its temporaries live in
 * one fixed device array of NSP_NOALLOC_SCRATCH_BYTES (16 MiB) that the library defines and
 * that every GPU using the library keeps until the process exits. The paper has no
 * counterpart; it is an interface convenience.
 *  - Limit: (2 n_Gamma + 3 n_interior + update rows of the interior factor) * s * element
 *    size, each part rounded up to 256 bytes, must fit in the array; otherwise
 *    NSP_ERR_INVALID_ARG and nothing runs.
 *  - The sweep plan for the width class (s = 1, or s > 1) must exist: s > 1 is ready after
 *    nsp_build; s = 1 after any nsp_solve, nsp_apply or s = 1 nsp_schur_apply on the handle
 *    (NSP_ERR_INVALID_ARG otherwise).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream capture.
 *  - All calls share the array, so calls whose work overlaps on the GPU (other streams or
 *    other handles) race; the array keeps the last call's contents (every temporary is fully
 *    written before it is read, nothing needs clearing).
 * Asynchronous on the handle's stream like nsp_schur_apply: it never runs the sweep
 * autotuner (a width the handle has not tuned yet uses the default sweep grid). */
#define NSP_NOALLOC_SCRATCH_BYTES (16u << 20)
nsp_status nsp_schur_apply_noalloc(const nsp_handle *h, const void *X, void *Y, int32_t s);

/* X = A_I^{-1} B (interior order, n_interior x s) or X = A_G^{-1} B (Gamma order,
 * n_Gamma x s) with the device Cholesky factors, in the handle's precision (see
 * nsp_schur_apply). which: 0 = interior blocks, 1 = A_G. Device pointers. Asynchronous on
 * the handle's stream like nsp_schur_apply. */
nsp_status nsp_factor_solve(const nsp_handle *h, int32_t which, const void *B, void *X,
                            int32_t s);

/* Copy Sigma (rank doubles, descending) and Z (n_Gamma x rank row-major, Gamma order) of
 * M2 to host memory; either pointer may be NULL. *rank receives the rank. */
nsp_status nsp_get_basis(const nsp_handle *h, double *Z, double *Sigma, int32_t *rank);

/* Copy an intermediate of the last build to host (needs keep_intermediates=1), all
 * n_Gamma x s row-major in Gamma order as doubles: which = 0: G (the sketch, step 1; after
 * q > 0 power iterations the final orthonormalized G), 1: E (block-PCG solution, S_Gamma
 * form only: NSP_ERR_INVALID_ARG for the S_I form), 2: Y (step 4), 3: U (step 10,
 * n_Gamma x rank). */
nsp_status nsp_get_intermediate(const nsp_handle *h, int32_t which, double *out);

/* ---- Learned sketch proposal --------------------------------------------------------
 * The paper draws the sketch G of Algorithm 2 step 1 at random; its angle bound (§4.2,
 * Proposition 4.1, eq. (tight_bound)) says the Nyström factor improves when range(G) is
 * closer to the dominant eigenvectors. These calls train and run a small network phi that
 * proposes G row by row from raw per-interface-node attributes a_i (d_raw doubles, the
 * first n_coord of them coordinates in (0, 1)):
 *   e_i = [sin(pi j a_ic), cos(pi j a_ic), c < n_coord, j = 1..n_freq] ++ a_i[n_coord:]
 *   h1 = tanh(e W1 + b1), h2 = tanh(h1 W2 + b2), g_i = h2 W3 + b3   (s_out columns)
 * Training minimises, for a target basis U (n x k, orthonormal columns),
 *   L = ||U - G (G^T G)^{-1} G^T U||_F^2 + mu ||G^T G / n - I||_F^2.
 * Parameters are one flat vector [W1, b1, W2, b2, W3, b3], weights row-major with the input
 * dimension first (nsp_net_num_params entries). Arrays of attributes (n x d_raw), targets
 * (n x k) and sketches (n x s_out) are row-major doubles, host or device (detected); the
 * parameter arrays of nsp_net_create / set / get are host memory. Work runs on the stream
 * given at creation. The paper has none of this; it is the learned-proposal extension. */
typedef struct {
  int32_t d_raw;       /* raw attributes per node                                        */
  int32_t n_coord;     /* leading attributes that are coordinates in (0, 1)              */
  int32_t n_freq;      /* Fourier frequencies per coordinate                             */
  int32_t hidden;      /* width of both tanh layers, 1..256                              */
  int32_t s_out;       /* sketch columns (k + p), 1..128                                 */
  int32_t precision;   /* training arithmetic: NSP_FP32 or NSP_FP64                      */
  double mu;           /* weight of the conditioning term, >= 0                          */
} nsp_net_shape;
typedef struct nsp_net nsp_net;

/* Number of parameters of a network of this shape (-1 if the shape is invalid). */
int64_t nsp_net_num_params(const nsp_net_shape *sh);
/* Create a network with parameters theta0; stream is a cudaStream_t (NULL: default). */
nsp_status nsp_net_create(const nsp_net_shape *sh, const double *theta0, void *stream,
                          nsp_net **out);
/* Replace the parameters; clears the gradient and the Adam state. */
nsp_status nsp_net_set_params(nsp_net *net, const double *theta);
/* Copy to host: what = 0 parameters, 1 accumulated gradient, 2 / 3 Adam first / second
 * moments (nsp_net_num_params doubles). */
nsp_status nsp_net_get(const nsp_net *net, int32_t what, double *out);
/* G = phi(attrs) in the training precision (n x s_out). Synchronous. */
nsp_status nsp_net_forward(const nsp_net *net, const double *attrs, int64_t n, double *G);
/* Add dL/dtheta for one (attrs, U) pair to the accumulated gradient; *loss (host, may be
 * NULL: no synchronization) receives L. Needs n >= s_out, 1 <= k <= 256. */
nsp_status nsp_net_loss_grad(nsp_net *net, const double *attrs, int64_t n, const double *U,
                             int32_t k, double *loss);
nsp_status nsp_net_zero_grad(nsp_net *net);
/* One Adam step (Kingma & Ba, bias-corrected) with the accumulated gradient, which is
 * then cleared. */
nsp_status nsp_net_adam_step(nsp_net *net, double lr, double beta1, double beta2, double eps);
/* Inference for nsp_build's sketch: phi(attrs) with the embedding and hidden layers in
 * BF16 weights and BF16-rounded activations (FP32 sums) and the output layer in FP32 (BF16
 * there loses the small singular directions of the ill-conditioned proposed block), then
 * orthonormalized by Cholesky-QR in FP64: G = phi L^{-T}, phi^T phi = L L^T. Algorithm 2 only
 * depends on range(G) (G -> G R leaves the Nyström factor unchanged), and the orthonormal
 * basis keeps the FP32 block PCG well conditioned. Written as doubles (n x s_out, Gamma
 * order). *full_rank (may be NULL) is 1 when the Cholesky keeps every pivot above 1e-12
 * times the largest diagonal entry; otherwise G is the raw output and callers fall back to
 * the Gaussian sketch. With full_rank NULL no check and no orthonormalization is done.
 * Synchronous. */
nsp_status nsp_net_sketch(nsp_net *net, const double *attrs, int64_t n, double *G,
                          int32_t *full_rank);
nsp_status nsp_net_destroy(nsp_net *net);

/* Dense lower Cholesky factor entries of one factor, for tests: block in [0, nblocks]
 * (nblocks = A_G). Writes the block's elimination order (n_b global indices of A) to
 * order and the factor L (n_b x n_b column-major, zeros above the diagonal and outside
 * the structure) to L, host memory. The library stores inv(L_JJ) and L_J2 inv(L_JJ) per
 * supernode; this call reconstructs L from them on the host. Use only for small blocks. */
nsp_status nsp_get_factor(const nsp_handle *h, int32_t block, int64_t *order, double *L,
                          int64_t n_b);

/* Host-only validation, DBBD check, orderings and symbolic analysis of A's pattern (no CUDA
 * call; A must be host memory). Fills n, n_interior, n_gamma, nblocks, nnz_L_interior,
 * nnz_L_gamma, n_supernodes and ms_analyze of info. Errors as nsp_build's analysis part. */
nsp_status nsp_analyze(const nsp_csr *A, const nsp_partition *P, nsp_info *info);

nsp_status nsp_get_info(const nsp_handle *h, nsp_info *info);
nsp_status nsp_destroy(nsp_handle *h);
/* Failure-detection check (no counterpart in the paper): runs one single-vector sweep of the
 * handle's interior factor with every dependency made unreachable (its epoch moved 2^20
 * launches ahead of the completion counters) and each wait bounded by max_spins polls
 * (about 1 us each). The waits must run out: the sweep sets its abort flag, every CTA skips
 * its remaining items, the kernel returns and records a device timeout. *observed receives
 * the status the sweep reported (NSP_ERR_TIMEOUT when the path works). The plan's counters
 * and the device status are reset afterwards, so the handle stays usable. No GPU fault, trap
 * or hang is involved. */
nsp_status nsp_check_timeout_path(const nsp_handle *h, int32_t max_spins, int32_t *observed);

/* Message of the last failed call made on the calling thread ("" if none); valid until
 * the next failing call on that thread. */
const char *nsp_last_error(void);
const char *nsp_status_string(nsp_status s);

/* Number of CUDA kernels this library has launched in the process so far (all handles).
 * Used to count the device launches of a timed region. */
int64_t nsp_kernel_launches(void);

/* ---- Dense products of the inner block PCG (standalone, for tests and measurements) -----
 * The block-CG iteration (§5.1: breakdown-free block PCG) needs, besides the S_Gamma block
 * apply, s x s inner products of n x s blocks and tall updates of such blocks. The handle
 * runs them internally with the kernels these two calls expose: FP32 data on the tcgen05
 * tensor cores, each operand split into two TF32 parts (three MMAs per product, FP32-level
 * accuracy, FP32 accumulation in tensor memory; Gram partials of row chunks added in FP64
 * in a fixed order). Row-major device arrays; s1, s2 in [1, 256]; work is a device buffer of
 * at least the queried size that the call uses as scratch (its last 8 bytes receive a
 * device status word: nonzero if a bounded wait of the kernel ran out, which never happens
 * on a working GPU). Asynchronous on `stream` (cudaStream_t, NULL = default stream).
 *   nsp_gram         : C (s1 x s2, doubles) = X^T Y, X n x s1, Y n x s2 (floats).
 *   nsp_gram_compensated : the same product as the Nyström core forms K = Y^T Y and C = G^T Y
 *                      (Algorithm 2 steps 5-6), where the Cholesky-QR needs more than FP32
 *                      sums: FP32 pipes with compensated dot products (exact products and
 *                      TwoSum error terms, Ogita-Rump-Oishi Dot2), accurate as if summed in
 *                      twice FP32 precision; partials of row chunks added in FP64. Same work
 *                      size query as nsp_gram.
 *   nsp_block_update : Out (n x s2) = scale * A M + beta * Cin, A n x s1 (floats), M s1 x s2
 *                      (doubles), Cin n x s2 or NULL (may alias Out).                       */
int64_t nsp_gram_work_bytes(int64_t n, int32_t s1, int32_t s2);
nsp_status nsp_gram(const float *X, const float *Y, int64_t n, int32_t s1, int32_t s2,
                    double *C, void *work, void *stream);
nsp_status nsp_gram_compensated(const float *X, const float *Y, int64_t n, int32_t s1,
                                int32_t s2, double *C, void *work, void *stream);
int64_t nsp_block_update_work_bytes(int32_t s1, int32_t s2);
nsp_status nsp_block_update(const float *A, const double *M, int64_t n, int32_t s1, int32_t s2,
                            float scale, const float *Cin, float beta, float *Out, void *work,
                            void *stream);

/* Philox4x32-10 (Salmon et al., SC'11) + Box-Muller normals, as used for the sketch:
 * out[i] for i in [0, count), stream defined by seed; out is a device pointer. */
nsp_status nsp_gaussian(uint64_t seed, int64_t count, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NSP_H */
