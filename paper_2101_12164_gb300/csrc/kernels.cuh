// Kernel launchers of the hot path. Every launcher enqueues on the given stream and
// never synchronizes. Blocks of vectors are row-major (entry (i, j) at [i*s + j]).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace nsp {

// Device view of a supernodal forest (see symbolic.h for the meaning of each array).
struct ForestDev {
  int32_t nsn = 0;
  int64_t n = 0;
  const int32_t *sn_first = nullptr, *sn_w = nullptr, *sn_m = nullptr, *sn_block = nullptr;
  const int64_t *sn_rowptr = nullptr, *sn_panel = nullptr, *sn_front = nullptr, *sn_upd = nullptr;
  const int32_t *rows = nullptr, *relmap = nullptr, *ch_ptr = nullptr, *ch_list = nullptr;
  const int64_t *gptr = nullptr, *gsrc = nullptr;
  const int64_t *asm_ptr = nullptr, *asm_dst = nullptr, *asm_src = nullptr;
};

// A (sub)matrix in CSR with int32 indices on the device.
template <typename T>
struct CsrDev {
  int32_t nrows = 0, ncols = 0;
  int64_t nnz = 0;
  const int32_t *rowptr = nullptr, *col = nullptr;
  const T *val = nullptr;
};

// Work list of one persistent solve (see k_solve.cu): nfwd forward items, then backward
// items. Item i is a tile of supernode item_a[i] starting at row/column item_b[i], or, when
// item_b[i] < 0, a group of -item_b[i] small supernodes group_sn[item_a[i] ...]. Counters
// grow across launches (unsigned, compared modulo 2^32); launch number `epoch` waits for
// epoch x (units per supernode). The epoch and the claim base live in device memory and are
// advanced by a one-thread kernel before every sweep, so that sweeps can be captured in a
// CUDA graph and replayed.
struct SweepPlan {
  int32_t nitems = 0, nfwd = 0, max_m = 0;
  int32_t vec_cols = 0;  // columns per backward tile in vector mode (set by the plan)
  int32_t blk_rows = 64; // rows / columns of a block tile (kSweepBlockRows or kSweepBlockRowsNarrow)
  bool vector = false;
  const int32_t *item_a = nullptr, *item_b = nullptr, *group_sn = nullptr;
  const int32_t *sn_parent = nullptr, *need_f = nullptr, *units_f = nullptr, *units_b = nullptr;
  uint32_t *cnt_f = nullptr, *self_f = nullptr, *done_b = nullptr;
  uint32_t *claim = nullptr, *abort_flag = nullptr, *epoch = nullptr, *claim_base = nullptr;
  // Block-resident schedule (k_rsweep.cu): block b owns heights [res_blk_ptr[b],
  // res_blk_ptr[b+1]); height L owns supernodes res_job[res_lvl_ptr[L] .. res_lvl_ptr[L+1]),
  // the first res_lvl_nwarp[L] of them warp-sized (largest first), the rest CTA-sized.
  int32_t res_nblocks = 0;
  const int32_t *res_blk_ptr = nullptr, *res_lvl_ptr = nullptr, *res_lvl_nwarp = nullptr,
                *res_job = nullptr;
  // Vector plans, shared-memory sweep (k_vsweep.cu): block b's rows [vs_row_off[b],
  // vs_row_off[b+1]); its heights [vs_lvl_ptr[b], vs_lvl_ptr[b+1]), height L's batches
  // [vs_bat_ptr[L], vs_bat_ptr[L+1]). Batch q (vs_bat[3q..3q+2]): {first item, end item,
  // front entries, forward units}, {backward columns, any K-split item, first position,
  // first forward unit}, {first backward column, 0, 0, 0}. Item i (vs_item[4i..4i+3]):
  // {front offset, partial-sum offset, K groups, update-row slot}, {first forward unit,
  // first backward column, m, w}, {first row in the block, sn_rowptr low, high, sn_panel low},
  // {sn_panel high, supernode, 0, 0} (offsets within the batch). Per front position (all
  // batches back to back): vs_pfvi forward v index (-1: none), vs_pbvi backward source (v
  // index of y_J; -2 - v index of x for a row below; -1: padding), vs_pitem item (relative),
  // vs_pptr / vs_psrc its gather sources as slots of the block's shared-memory update-row
  // pool. vs_uitem / vs_citem: the item of each forward unit / backward column. vs_elems =
  // the largest block's rows + pool, each rounded up to 4 (0: no shared-memory sweep);
  // vs_scratch = scratch entries per batch.
  const int64_t *vs_row_off = nullptr;
  const int32_t *vs_lvl_ptr = nullptr, *vs_bat_ptr = nullptr;
  const int4 *vs_bat = nullptr, *vs_item = nullptr;
  const int32_t *vs_pfvi = nullptr, *vs_pbvi = nullptr, *vs_pptr = nullptr, *vs_psrc = nullptr;
  const uint16_t *vs_pitem = nullptr, *vs_uitem = nullptr, *vs_citem = nullptr;
  int64_t vs_elems = 0;
  int32_t vs_scratch = 0;
  // Block plans, column-sliced sweep (k_bsweep.cu): the same height / batch structure, with
  // batch q (bs_bat[3q..3q+2]) = {first item, end item, front positions, forward units},
  // {backward units, 0, first position, first forward unit}, {first backward unit, first
  // gather source, gather sources, 0};
  // item i (bs_item[3i..3i+2]) = {front offset, first forward unit, first backward unit, m},
  // {w, first row, first update row, 0}, {sn_panel low, high, 0, 0}. Per front position:
  // bs_pfvi forward row of B (top rows; -1: none), bs_pbvi backward source (row of Y for top
  // rows; -2 - row of X below; -1: padding), bs_pptr / bs_psrc the gather sources (update
  // rows). bs_uitem / bs_citem: item of each forward / backward unit. bs_positions = the
  // largest batch's front positions (0: no plan).
  const int32_t *bs_lvl_ptr = nullptr, *bs_bat_ptr = nullptr;
  const int4 *bs_bat = nullptr, *bs_item = nullptr;
  const int32_t *bs_pfvi = nullptr, *bs_pbvi = nullptr, *bs_pptr = nullptr, *bs_psrc = nullptr;
  const uint16_t *bs_uitem = nullptr, *bs_citem = nullptr;
  int32_t bs_positions = 0;
};

// ---- numeric factorization (k_factor.cu) -----------------------------------------
// Multifrontal partial Cholesky of the supernodes level_sn[0..count) (one CTA each), then
// the panel [inv(L_JJ); L_J2 inv(L_JJ)] (column-major, leading dimension panel_ld(m)).
// A non-positive pivot records DEV_NOT_SPD with the supernode's block id.
template <typename T>
void launch_factor_level(const ForestDev &f, const int32_t *level_sn, int count,
                         const double *Aval, T *front, T *panel, DevStatus *st,
                         cudaStream_t stream, int mode);
// mode: 0 one CTA per front, 1 a cluster of factor_cluster_size() CTAs per front, 2 a cluster
// of 16 CTAs, one per SM, per front (where factor_big_clusters_available(), else mode 1)
template <typename T>
bool factor_big_clusters_available();
int factor_cluster_size();
constexpr int kBigFront = 192;   // fronts with m >= kBigFront use the cluster kernel

// ---- supernodal multi-RHS solves (k_solve.cu) ------------------------------------
// One persistent launch: X = A_b^{-1} B for every block of the forest (s columns). B, X in
// the forest's internal order; Y (n x s) and U (update rows x s) are workspaces. claim_base
// is the claim counter's value before the launch; returns the grid size used (the counter
// advances by nitems + grid).
// Returns the grid used: grid_req CTAs (rounded to the SM count, capped by occupancy) or,
// when grid_req <= 0, the occupancy maximum (at most 4 CTAs per SM).
// max_spins bounds every dependency wait (0: the default, a few seconds at most); a wait that
// runs out sets the plan's abort flag (every CTA then skips its remaining items) and records
// DEV_TIMEOUT.
template <typename T>
int launch_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *Y, T *U,
                 T *X, int s, DevStatus *st, cudaStream_t stream, int grid_req = 0,
                 int max_spins = 0);
// The same solve with one CTA per block of the forest and no cross-CTA dependency (the
// plan's block-resident schedule), both sweeps of a block in its CTA. Grid = blocks.
// half = 1: the forward sweep only, Y = L^{-1} B (with A_b = L L^T in the forest's order);
// half = 2: the backward sweep only, X = L^{-T} Y (Y is then read, not written).
template <typename T>
void launch_res_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *Y,
                      T *U, T *X, int s, DevStatus *st, cudaStream_t stream, int half = 0);
constexpr int kResW = 32, kResM = 128;   // block mode: supernodes a warp runs (w, m bounds)
// One right-hand side with each block's vectors (b, y, x in place, and its update rows) in
// shared memory, one CTA per block of the vector plan's block-resident schedule; B, X in the
// forest's internal order. vsm_sweep_fits: how many CTAs per SM (2, 1; 0: none) the largest
// block's shared memory allows; per_sm (1 or 2, at most that) selects the register budget.
// s > 1 (s a multiple of 4) with one CTA per (block, slice of kBsmCols columns), heights in
// batches, no dependency waits (k_bsweep.cu); Y, U workspaces as launch_sweep's.
constexpr int kBsmCols = 32;
constexpr int kBsmScratchBytes = 192 * 1024;   // fronts of a batch
constexpr int kBsmMaxItems = 128;              // supernodes per batch
constexpr int kBsmMaxSources = 2560;           // gather sources per batch
template <typename T>
bool bsm_sweep_fits(const SweepPlan &p, int s);
template <typename T>
void launch_bsm_sweep(const SweepPlan &p, const T *panel, const T *B, T *Y, T *U, T *X, int s,
                      cudaStream_t stream, int half = 0);
constexpr int kVsmKG = 8;          // forward K groups of a CTA-sized supernode
constexpr int kVsmScratch = 4096;  // default scratch entries per batch (fronts + partials)
template <typename T>
int vsm_sweep_fits(const SweepPlan &p);
template <typename T>
void launch_vsm_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *X,
                      int per_sm, cudaStream_t stream);
// rows of a forward tile in vector mode for elements of elem_bytes
int sweep_vector_rows(int elem_bytes);
constexpr int kSweepBlockRows = 64;   // rows (forward) / columns (backward) per block tile
constexpr int kSweepBlockRowsNarrow = 32;   // the same for single-tree forests (A_G): twice the
                                            // tiles per supernode along the tree's top chain
constexpr int kSweepVectorCols = 16;  // default columns per backward tile in vector mode
constexpr int kSmallM = 96, kSmallW = 32, kGroup = 8;
// item_b of a subtree item: kSubtreeTag - L, item_a = offset of its L-entry member list
// (supernodes by height, -1 between heights) in group_sn
constexpr int kSubtreeTag = -(1 << 20);
constexpr double kSubtreeArea = 65536.0;  // largest summed m x w panel area of a subtree item

// ---- BLAS-like kernels (k_blas.cu) ------------------------------------------------
// Y = alpha * A X + beta * C  (C may be nullptr; Y may alias C)
template <typename T>
void launch_spmm(const CsrDev<T> &A, const T *X, T *Y, int s, T alpha, const T *C, T beta,
                 cudaStream_t stream);
// out[i*s+j] = (To) in[perm[i]*s + j]   (perm == nullptr: identity)
template <typename Ti, typename To>
void launch_gather_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s,
                        cudaStream_t stream);
// out[perm[i]*s+j] = (To) in[i*s + j]
template <typename Ti, typename To>
void launch_scatter_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s,
                         cudaStream_t stream);
// out[e] = (T) Aval[src[e]]
template <typename T>
void launch_gather_values(const int64_t *src, int64_t count, const double *Aval, T *out,
                          cudaStream_t stream);
// C (s1 x s2, FP64, row-major) = X^T Y for X (n x s1), Y (n x s2). work: scratch doubles,
// at least gram_work_size(n, s1, s2). Deterministic. AccT = accumulation type.
template <typename T, typename AccT>
void launch_gram(const T *X, const T *Y, int64_t n, int s1, int s2, double *C,
                 double *work, cudaStream_t stream);
size_t gram_work_size(int64_t n, int s1, int s2);
// C[e] = sum over chunks c (in order) of work[c * entries + e]
void launch_gram_reduce(const double *work, int nchunks, int64_t entries, double *C,
                        cudaStream_t stream);
// Tensor-core forms (k_tc.cu, FP32 data, 3xTF32 on tcgen05, FP32 accumulation in TMEM):
// C = X^T Y with FP64 chunk partials (work >= tc_gram_chunks(n) * s1 * s2 doubles), and
// Out = scale * A M + beta * C (mt_work >= tc_update_work_floats(s1, s2) floats). s1, s2 <=
// 256. A bounded wait that runs out records DEV_TIMEOUT in st.
size_t tc_gram_chunks(int64_t n);
void launch_tc_gram(const float *X, const float *Y, int64_t n, int s1, int s2, double *C,
                    double *work, DevStatus *st, cudaStream_t stream);
size_t tc_update_work_floats(int s1, int s2);
void launch_tc_block_update(const float *A, const double *M, int64_t n, int s1, int s2,
                            float scale, const float *C, float beta, float *Out, float *mt_work,
                            DevStatus *st, cudaStream_t stream);
// Out (n x s2) = scale * A (n x s1) M (s1 x s2, FP64) + beta * C  (C may alias Out or be
// nullptr)
template <typename T>
void launch_block_update(const T *A, const double *M, int64_t n, int s1, int s2, T scale,
                         const T *C, T beta, T *Out, cudaStream_t stream);
// X[i*s + j] *= scale[j]
void launch_scale_cols(double *X, int64_t n, int s, const double *scale, bool take_sqrt,
                       cudaStream_t stream);
// t = Z^T r and z = beta z + Z t for Z (n x k, FP64 row-major); work >= gram_work_size(n,k,1)
void launch_gemv_t(const double *Z, int64_t n, int k, const double *r, double *t, double *work,
                   cudaStream_t stream);
void launch_gemv_n(const double *Z, int64_t n, int k, const double *t, double beta, double *z,
                   cudaStream_t stream);
// colsq[j] = sum_i X[i*s+j]^2 (FP64), deterministic; work >= gram_work_size(n, s, 1)
template <typename T>
void launch_col_sumsq(const T *X, int64_t n, int s, double *colsq, double *work,
                      cudaStream_t stream);
// Philox4x32-10 + Box-Muller: out[i] ~ N(0,1), i in [0, count)
template <typename T>
void launch_gaussian(uint64_t seed, int64_t count, T *out, cudaStream_t stream);
// FP64 vector helpers for the outer PCG: out[i] = a*x[i] + b*y[i] etc.
void launch_dot(const double *x, const double *y, int64_t n, double *result, double *work,
                cudaStream_t stream);
void launch_axpby(int64_t n, const double *a_ptr, double a_sign, const double *x, double b,
                  double *y, cudaStream_t stream);   // y = (a_sign * *a_ptr) x + b y
// Fused PCG vector steps (FP64): alpha = *rz / *pq, x += alpha p, r -= alpha q, *rr = r.r
// (alpha recorded in *alpha); and p = z + beta p with beta = *rz_new / *rz_old (recorded in
// *beta). Bit-identical to launch_pcg_scalars + launch_axpby + launch_dot.
void launch_pcg_step(int64_t n, const double *rz, const double *pq, double *alpha,
                     const double *p, const double *q, double *x, double *r, double *rr,
                     double *work, cudaStream_t stream);
void launch_pcg_direction(int64_t n, const double *rz_new, const double *rz_old, double *beta,
                          const double *z, double *p, cudaStream_t stream);
void launch_pcg_scalars(const double *rz_new, const double *rz_old, const double *pq,
                        double *alpha, double *beta, cudaStream_t stream);

// ---- small dense FP64 core on one CTA (k_core.cu) ---------------------------------
// Cholesky-QR with column drop: C (s x s) = W^T W; writes Rinv (s x s, zero outside the kept
// columns) such that W Rinv has orthonormal kept columns, mask[j] = kept, *nkept.
// batch > 1 factors `batch` independent s x s matrices stored consecutively (one CTA each).
void launch_chol_drop(const double *C, int s, double drop_tol, double *Rinv, int32_t *mask,
                      int32_t *nkept, double *gwork, cudaStream_t stream, int batch = 1);
// doubles of scratch per problem for launch_chol_drop / launch_spd_solve_masked
size_t core_work_size(int s);
// out (s x r) = sign * PtQ^{-1} Rhs on the kept rows/cols (mask), zero elsewhere (r <= s).
// Non-SPD PtQ -> DEV_BREAKDOWN.
void launch_spd_solve_masked(const double *PtQ, const double *Rhs, int s, int r,
                             const int32_t *mask, double sign, double *out, double *gwork,
                             DevStatus *st, cudaStream_t stream);
// max_j sqrt(colsq[j]) / bnorm[j] -> *ratio
void launch_max_ratio(const double *colsq, const double *bnorm, int s, double *ratio,
                      cudaStream_t stream, int batch = 1);
void launch_sqrt_vec(const double *in, int s, double *out, cudaStream_t stream);
// Nyström core (Algorithm 2 steps 5-10) on K = Y^T Y and C = G^T Y (s x s FP64):
// writes Mix (s x k, row-major) with U = Y Mix, Sigma (k), *rank. work >= nystrom_work(s).
// polish: finish the eigenvectors with an FP64 Jacobi sweep (needed when K and C carry FP64
// information; with FP32 inputs the FP32 Jacobi vectors, FP64-reorthonormalized, are as
// accurate as the data and the eigenvalues are FP64 Rayleigh quotients).
void launch_nystrom_core(const double *K, const double *C, int s, int k, double eps_rel,
                         double drop_tol, double *Mix, double *Sigma, int32_t *rank,
                         double *work, cudaStream_t stream, int batch = 1, int polish = 1);
size_t nystrom_work_size(int s);   // doubles of scratch per problem

// ---- segmented kernels for batches of matrices (k_batch.cu) ------------------------
// Chunks of rows [row0[c], row1[c]) of segment seg[c]; segment g owns chunks
// [seg_first[g], seg_first[g+1]) in row order.
struct SegChunks {
  int nchunk = 0, nseg = 0;
  const int64_t *row0 = nullptr, *row1 = nullptr;
  const int32_t *seg = nullptr, *seg_first = nullptr;
};
// C[g] (s1 x s2) = X[rows of g]^T Y[rows of g]; work >= nchunk * s1 * s2 doubles
template <typename T, typename AccT>
void launch_seg_gram(const T *X, const T *Y, int s1, int s2, const SegChunks &ch, double *C,
                     double *work, cudaStream_t st);
template <typename T>
void launch_seg_colsq(const T *X, int s, const SegChunks &ch, double *colsq, double *work,
                      cudaStream_t st);
void launch_seg_dot(const double *x, const double *y, const SegChunks &ch, double *out,
                    double *work, cudaStream_t st);
void launch_seg_axpby(const SegChunks &ch, const double *a, double sign, const double *x,
                      double b, double *y, cudaStream_t st);
void launch_seg_ratio(const double *num, const double *den, const int32_t *active, int nseg,
                      double *out, cudaStream_t st);
template <typename T>
void launch_seg_scale_sqrt(const T *Zt, int k, const double *Sigma, const SegChunks &ch,
                           double *Zs, cudaStream_t st);
template <typename T>
void launch_seg_block_update(const T *A, const double *M, int s1, int s2, T scale, const T *C,
                             T beta, T *Out, const SegChunks &ch, const int32_t *active,
                             cudaStream_t st);
// Per-matrix outer-PCG bookkeeping on the device: fn = sqrt(ff), active = fn > 0, its = 0;
// then after each step: for active matrices its += 1, rel = ||r|| / fn, active stays on while
// rel > rtol and its < maxit; any = 1 if some matrix is still active.
void launch_seg_pcg_init(const double *ff, int nseg, double *fn, int32_t *active, int32_t *its,
                         double *rel, cudaStream_t st);
void launch_seg_converge(const double *rr, const double *fn, double rtol, int maxit,
                         int32_t *active, int32_t *its, double *rel, int32_t *any, int nseg,
                         cudaStream_t st);
// inner block-PCG stopping rule of every matrix, optionally driving a CUDA graph loop
void launch_seg_inner_decide(const double *ratio, const int32_t *nkept, double eps, int nseg,
                             int32_t *active, int32_t *its, double *rat, int32_t *act,
                             int32_t *go, int32_t *passes, int maxit,
                             cudaGraphConditionalHandle h, int set_cond, cudaStream_t st);
// sets a CUDA graph loop's conditional from *flag (and counts the pass)
void launch_loop_condition(const int32_t *flag, int32_t *passes, cudaGraphConditionalHandle h,
                           cudaStream_t st);

}  // namespace nsp
