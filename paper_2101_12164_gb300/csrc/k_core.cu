// Small dense linear algebra on one CTA: the s x s steps of the breakdown-free block PCG
// (Cholesky-QR with column drop, alpha/beta solves) and the Nyström core of Algorithm 2
// steps 5-10 (Cholesky-QR of Y, EVD of C, T, EVD of T). s <= 256. Working sets live in
// shared memory when they fit (s <= 88), otherwise in a global scratch area, except the
// Cholesky factor of k_chol_drop and the two FP32 Jacobi matrices of the EVDs, which stay in
// shared memory up to s = 160.
//
// Symmetric EVD: cyclic Jacobi (rotation of pair (p, q) from Golub & Van Loan's 2x2
// symmetric Schur decomposition: tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c) with the round-robin ordering of disjoint
// pairs, first in FP32; the FP32 eigenvectors are then orthonormalized in FP64 (modified
// Gram-Schmidt) and B = V^T C V is formed in FP64, whose diagonal gives the eigenvalues as
// FP64 Rayleigh quotients. For FP64 handles (polish) an FP64 Jacobi sweep with the
// threshold |b_pq| > tol sqrt(|b_pp b_qq|) then refines the vectors to FP64 accuracy; FP32
// handles skip it: their K and C come from FP32 block-PCG data, whose rounding is far above
// the FP32 Jacobi's, and the measured Nyström factor matches the FP64 oracle's to 3e-4 at
// s = 160 (the same difference the FP32 inner solves alone produce).
#include <cfloat>

#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int CT = 512;            // threads of the single CTA
constexpr int SMEM_S = 88;         // largest s whose three s x s FP64 buffers fit in smem
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// Thresholded right-looking Cholesky of L (s x s, row-major, lower part): column j is kept
// when its pivot exceeds drop_tol * diag0[j] (diag0[j] > 0), otherwise zeroed and skipped.
__device__ void chol_threshold(double *L, const double *diag0, int s, double drop_tol,
                               int32_t *mask, int *nkept) {
  __shared__ int keep;
  const int tid = threadIdx.x;
  if (tid == 0) *nkept = 0;
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid == 0) {
      const double piv = L[j * s + j];
      const double d0 = diag0[j];
      keep = (d0 > 0.0 && piv > drop_tol * d0 && piv > 0.0) ? 1 : 0;
      mask[j] = keep;
      if (keep) {
        L[j * s + j] = sqrt(piv);
        *nkept += 1;
      }
    }
    __syncthreads();
    if (keep) {
      const double d = L[j * s + j];
      for (int i = j + 1 + tid; i < s; i += CT) L[i * s + j] /= d;
      __syncthreads();
      for (int r = j + 1 + (tid >> 5); r < s; r += CT / 32) {
        const double lrj = L[r * s + j];
        for (int c = j + 1 + (tid & 31); c <= r; c += 32) L[r * s + c] -= lrj * L[c * s + j];
      }
    } else {
      for (int i = j + tid; i < s; i += CT) L[i * s + j] = 0.0;
    }
    __syncthreads();
  }
}

// Solve L X = X (fwd) or L^T X = X (bwd) in place; L lower s x s (row-major), X s x r
// (row-major); rows with mask == 0 are set to zero. Right-looking substitution: step i
// subtracts row i's contribution x_i = X_i / L_ii from the rows still to be solved (one
// barrier per step, all (row, column) updates of a step in parallel), and a last pass
// scales every row by 1 / L_ii. identity_rhs: X = I on entry (forward: only the columns
// <= i of row i can be nonzero, so the updates of step i stop there).
__device__ void trsm_masked(const double *L, int s, const int32_t *mask, double *X, int r,
                            bool transpose, bool identity_rhs = false) {
  __shared__ double invd[256];
  const int tid = threadIdx.x;
  for (int i = tid; i < s; i += CT) invd[i] = mask[i] ? 1.0 / L[i * s + i] : 0.0;
  __syncthreads();
  // forward solve of X = I: row i is zero beyond column i, so step i touches columns <= i
  const bool lower_id = identity_rhs && !transpose;
  for (int step = 0; step < s; ++step) {
    const int i = transpose ? s - 1 - step : step;
    if (mask[i]) {
      const double inv = invd[i];
      const int t0 = transpose ? 0 : i + 1, t1 = transpose ? i : s;
      const int nc = lower_id ? min(r, i + 1) : r;
      const int n = (t1 - t0) * nc;
      for (int e = tid; e < n; e += CT) {
        const int t = t0 + e / nc, c = e % nc;
        if (mask[t]) {
          const double lti = transpose ? L[i * s + t] : L[t * s + i];
          X[t * r + c] -= lti * (X[i * r + c] * inv);
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < s * r; e += CT) {
    const int i = e / r;
    X[e] = mask[i] ? X[e] * invd[i] : 0.0;
  }
  __syncthreads();
}

// Cyclic Jacobi on symmetric A (s x s row-major, leading dimension ld for A and V); V
// accumulates (A_in = V A_out V^T). A rotation is applied when |a_pq| > tol sqrt(|a_pp a_qq|)
// and |a_pq| > floor_rel ||A||_F (below that the entry is at the rounding level of the
// matrix). Each round rotates disjoint pairs; a warp owns its pairs for the whole round: it
// forms each rotation from the pair's 2 x 2 block (which no other pair touches), applies it
// to the pair's two columns of A and V, and after a barrier to the pair's two rows of A.
// An odd ld keeps the column accesses free of shared-memory bank conflicts.
template <typename F>
__device__ void jacobi(F *A, F *V, int s, int ld, int max_sweeps, F tol, F floor_rel) {
  __shared__ F cs[128], sn[128];
  __shared__ int pp[128], qq[128];
  __shared__ int any;
  __shared__ F fro_sh;
  __shared__ float red[CT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {  // ||A||_F (rotations keep it): off-diagonal entries below floor_rel ||A||_F are final
    float acc = 0.0f;
    for (int e = tid; e < s * s; e += CT) {
      const float a = (float)A[(e / s) * ld + e % s];
      acc += a * a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      float t = 0.0f;
      for (int w = 0; w < CT / 32; ++w) t += red[w];
      fro_sh = (F)sqrtf(t);
    }
    __syncthreads();
  }
  const F floor_abs = floor_rel * fro_sh;
  const int se = s + (s & 1);
  const int npair = se / 2;
  // round-robin pairing in closed form: the ring that fixes position 0 and rotates the other
  // se - 1 positions by one per round holds, after t rounds, 1 + ((j - 1 - t) mod (se - 1))
  // at position j >= 1
  auto ring_at = [se](int j, int t) {
    return j == 0 ? 0 : 1 + (((j - 1 - t) % (se - 1)) + (se - 1)) % (se - 1);
  };
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) any = 0;
    __syncthreads();
    for (int round = 0; round < se - 1; ++round) {
      {
        // lane l forms the rotation of the warp's l-th pair (the pairs' chains overlap), then
        // the warp applies each rotation to its pair's two columns of A and V
        const int kl = warp + lane * (CT / 32);
        int pl = 0, ql = 0;
        F cl = F(1), sl = F(0);
        if (kl < npair) {
          pl = ring_at(kl, round);
          ql = ring_at(se - 1 - kl, round);
          if (pl > ql) { const int x = pl; pl = ql; ql = x; }
          if (ql < s) {
            const F apq = A[pl * ld + ql], app = A[pl * ld + pl], aqq = A[ql * ld + ql];
            if (fabs(apq) > floor_abs && fabs(apq) > tol * sqrt_(fabs(app * aqq))) {
              const F tau = (aqq - app) / (F(2) * apq);
              const F tt = (tau >= F(0) ? F(1) : F(-1)) / (fabs(tau) + sqrt_(F(1) + tau * tau));
              cl = F(1) / sqrt_(F(1) + tt * tt);
              sl = tt * cl;
            }
          }
          pp[kl] = pl;
          qq[kl] = ql;
          cs[kl] = cl;
          sn[kl] = sl;
          if (sl != F(0)) any = 1;
        }
        __syncwarp();
        for (int l = 0; warp + l * (CT / 32) < npair; ++l) {
          const int p = __shfl_sync(0xffffffffu, pl, l), q = __shfl_sync(0xffffffffu, ql, l);
          const F c = __shfl_sync(0xffffffffu, cl, l), sv = __shfl_sync(0xffffffffu, sl, l);
          if (sv == F(0)) continue;
          for (int i = lane; i < s; i += 32) {
            const F ap = A[i * ld + p], aq = A[i * ld + q];
            A[i * ld + p] = c * ap - sv * aq;
            A[i * ld + q] = sv * ap + c * aq;
            const F vp = V[i * ld + p], vq = V[i * ld + q];
            V[i * ld + p] = c * vp - sv * vq;
            V[i * ld + q] = sv * vp + c * vq;
          }
        }
      }
      __syncthreads();
      for (int k = warp; k < npair; k += CT / 32) {  // A <- J^T A
        const F sv = sn[k];
        if (sv == F(0)) continue;
        const int p = pp[k], q = qq[k];
        const F c = cs[k];
        for (int j = lane; j < s; j += 32) {
          const F ap = A[p * ld + j], aq = A[q * ld + j];
          A[p * ld + j] = c * ap - sv * aq;
          A[q * ld + j] = sv * ap + c * aq;
        }
      }
      __syncthreads();
    }
    if (!any) break;
    __syncthreads();
  }
}

// C = A B for s x s row-major operands (warps over rows, lanes over columns).
__device__ void gemm_nn(const double *A, const double *B, double *Cm, int s) {  // C = A B
  for (int i = threadIdx.x >> 5; i < s; i += CT / 32)
    for (int j = threadIdx.x & 31; j < s; j += 32) {
      double v = 0.0;
      for (int t = 0; t < s; ++t) v += A[i * s + t] * B[t * s + j];
      Cm[i * s + j] = v;
    }
  __syncthreads();
}

// Gram-Schmidt on the columns of V (s x s row-major, FP64): column j minus its projections
// on the previous (orthonormal) columns, coefficients taken against the original column j,
// then normalized. FP64 arithmetic is the scarce resource here (about two FMAs per clock per
// SM), so every product is formed once: a thread per coefficient (a dot over the rows), a
// thread per row for the projection, one warp for the norm. The work runs on a copy in W
// (s x s) whose row r is rotated by r positions, so that threads walking down a column hit
// distinct shared-memory banks.
__device__ void mgs_columns(double *V, int s, double *W) {
  __shared__ double coef[256], colw[256];
  __shared__ double inv_nrm;
  const int tid = threadIdx.x;
  auto at = [s](int r, int c) { return r * s + (c + r) % s; };
  for (int e = tid; e < s * s; e += CT) W[at(e / s, e % s)] = V[e];
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid < j) {  // rotated positions advance by one per row, wrapping at s
      double d = 0.0;
      int ki = tid, kj = j;
      for (int r = 0; r < s; ++r) {
        d += W[r * s + ki] * W[r * s + kj];
        ki = ki + 1 == s ? 0 : ki + 1;
        kj = kj + 1 == s ? 0 : kj + 1;
      }
      coef[tid] = d;
    }
    __syncthreads();
    if (tid < s) {
      const double *row = W + tid * s;
      double v = row[(j + tid) % s];
      int k = tid;
      for (int i = 0; i < j; ++i) {
        v -= coef[i] * row[k];
        k = k + 1 == s ? 0 : k + 1;
      }
      colw[tid] = v;
    }
    __syncthreads();
    if (tid < 32) {
      double sq = 0.0;
      for (int r = tid; r < s; r += 32) sq += colw[r] * colw[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
      if (tid == 0) inv_nrm = sq > 0.0 ? 1.0 / sqrt(sq) : 0.0;
    }
    __syncthreads();
    if (tid < s) W[at(tid, j)] = colw[tid] * inv_nrm;
    __syncthreads();
  }
  for (int e = tid; e < s * s; e += CT) V[e] = W[at(e / s, e % s)];
  __syncthreads();
}

// FP64-accurate EVD of the symmetric matrix held in Bm (s x s): on return the eigenvalues
// are on the diagonal of Bm and the eigenvectors in the columns of V. W1 is s x s scratch,
// also used for the two FP32 matrices of the first phase. All three may be shared memory.
// jac (may be null): shared memory for the two FP32 matrices of the first phase (2 s (s|1)
// floats), used when the s x s FP64 buffers themselves are in global memory.
__device__ void eig_sym(double *Bm, int s, double *V, double *W1, bool polish,
                        float *jac = nullptr) {
  const int tid = threadIdx.x;
  const size_t ss = (size_t)s * s;
  const int ld = s | 1;  // odd leading dimension of the FP32 phase (s x ld floats fit in s x s doubles)
  float *A32 = jac ? jac : reinterpret_cast<float *>(W1);
  float *V32 = jac ? jac + (size_t)s * ld : reinterpret_cast<float *>(V);
  for (size_t e = tid; e < ss; e += CT) {
    const int i = e / s, j = e % s;
    A32[i * ld + j] = (float)Bm[e];
    V32[i * ld + j] = i == j ? 1.0f : 0.0f;
  }
  __syncthreads();
  jacobi<float>(A32, V32, s, ld, 8, 1e-6f, 2e-7f);
  if (jac) {
    for (size_t e = tid; e < ss; e += CT) V[e] = (double)V32[(e / s) * ld + e % s];
  } else {
    float *T32 = A32;  // A32 is no longer needed: V32 moves there before V is widened in place
    for (size_t e = tid; e < ss; e += CT) {
      const int i = e / s, j = e % s;
      T32[i * ld + j] = V32[i * ld + j];
    }
    __syncthreads();
    for (size_t e = tid; e < ss; e += CT) V[e] = (double)T32[(e / s) * ld + e % s];
  }
  __syncthreads();
  mgs_columns(V, s, W1);
  // W1 = C V ; Bm = V^T W1 (symmetric: upper triangle computed, mirrored)
  gemm_nn(Bm, V, W1, s);
  for (int i = tid >> 5; i < s; i += CT / 32)
    for (int j = i + (tid & 31); j < s; j += 32) {
      double v = 0.0;
      for (int t = 0; t < s; ++t) v += V[t * s + i] * W1[t * s + j];
      Bm[i * s + j] = v;
      Bm[j * s + i] = v;
    }
  __syncthreads();
  if (polish) jacobi<double>(Bm, V, s, s, 1, 1e-13, 1e-15);
}

struct Scratch {
  double *b0, *b1, *b2;  // three s x s buffers (smem or global)
};

// use_smem: 1 = all three buffers in shared memory, 2 = only b0 (the factor being
// decomposed) in shared memory, 0 = all in global memory
__device__ Scratch scratch(double *smem, double *global, int s, int use_smem) {
  const size_t ss = (size_t)s * s;
  if (use_smem == 2) return Scratch{smem, global + ss, global + 2 * ss};
  double *base = use_smem ? smem : global;
  return Scratch{base, base + ss, base + 2 * ss};
}

// ---------------------------------------------------------------- block PCG kernels
// C = W^T W -> thresholded Cholesky-QR: Rinv (upper, zero for dropped), mask, nkept.
__global__ void __launch_bounds__(CT) k_chol_drop(const double *C, int s, double drop_tol,
                                                  double *Rinv, int32_t *mask, int32_t *nkept,
                                                  double *gwork, int use_smem) {
  extern __shared__ __align__(16) double dsm[];
  __shared__ int nk;
  __shared__ double diag0[256];
  __shared__ int32_t msk[256];
  const int tid = threadIdx.x;
  const size_t ss = (size_t)s * s;
  {  // batch: block b works on the b-th s x s problem
    const size_t b = blockIdx.x;
    C += b * ss;
    Rinv += b * ss;
    mask += b * s;
    nkept += b;
    gwork += b * 3 * ss;
  }
  const Scratch S = scratch(dsm, gwork, s, use_smem);
  for (size_t i = tid; i < ss; i += CT) {
    S.b0[i] = C[i];
    S.b1[i] = (i / s == i % s) ? 1.0 : 0.0;
  }
  for (int i = tid; i < s; i += CT) diag0[i] = C[i * s + i];
  __syncthreads();
  chol_threshold(S.b0, diag0, s, drop_tol, msk, &nk);
  trsm_masked(S.b0, s, msk, S.b1, s, false, true);  // b1 = L^{-1} (dropped rows zero)
  for (size_t i = tid; i < ss; i += CT) {
    const int r = i / s, c = i % s;
    Rinv[i] = msk[c] ? S.b1[c * s + r] : 0.0;  // R^{-1} = L^{-T}
  }
  for (int i = tid; i < s; i += CT) mask[i] = msk[i];
  if (tid == 0) *nkept = nk;
}

// out (s x r) = sign * A^{-1} Rhs on the kept index set of mask.
__global__ void __launch_bounds__(CT) k_spd_solve_masked(const double *A, const double *Rhs, int s,
                                                         int r, const int32_t *mask, double sign,
                                                         double *out, double *gwork, int use_smem,
                                                         DevStatus *st) {
  extern __shared__ __align__(16) double dsm[];
  __shared__ int32_t msk[256];
  __shared__ double diag0[256];
  __shared__ int nk;
  const Scratch S = scratch(dsm, gwork, s, use_smem);
  const int tid = threadIdx.x;
  for (int i = tid; i < s; i += CT) msk[i] = mask[i];
  __syncthreads();
  for (int i = tid; i < s * s; i += CT) {
    const int a = i / s, b = i % s;
    S.b0[i] = (msk[a] && msk[b]) ? A[i] : 0.0;
  }
  for (int i = tid; i < s; i += CT) diag0[i] = msk[i] ? A[i * s + i] : 0.0;
  for (int i = tid; i < s * r; i += CT) S.b1[i] = Rhs[i];
  __syncthreads();
  // plain Cholesky on the kept set: a dropped pivot here means P^T Q lost definiteness
  __shared__ int32_t kept2[256];
  chol_threshold(S.b0, diag0, s, 0.0, kept2, &nk);
  for (int i = tid; i < s; i += CT)
    if (msk[i] && !kept2[i]) dev_fail(st, DEV_BREAKDOWN, i);
  trsm_masked(S.b0, s, kept2, S.b1, r, false);
  trsm_masked(S.b0, s, kept2, S.b1, r, true);
  for (int i = tid; i < s * r; i += CT) out[i] = sign * S.b1[i];
}

__global__ void k_max_ratio(const double *colsq, const double *bnorm, int s, double *ratio) {
  __shared__ double red[256];
  colsq += (size_t)blockIdx.x * s;
  bnorm += (size_t)blockIdx.x * s;
  ratio += blockIdx.x;
  double m = 0.0;
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    const double b = bnorm[j] > 0.0 ? bnorm[j] : 1.0;
    m = fmax(m, sqrt(colsq[j]) / b);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *ratio = red[0];
}

__global__ void k_sqrt_vec(const double *in, int s, double *out) {
  for (int j = threadIdx.x; j < s; j += blockDim.x) out[j] = sqrt(in[j]);
}

// ---------------------------------------------------------------- Nyström core
// Algorithm 2 steps 5-10 from K = Y^T Y and C = G^T Y (s x s):
//  5. Y = QR by Cholesky-QR: K = L L^T on the kept columns S (threshold drop_tol),
//     R_full = L^{-1} K[S, :] (= R when nothing is dropped), Q = Y_S L^{-T};
//  6. C = (C + C^T)/2;  7. EVD C = V D V^T, keep d >= eps_rel max(d), d > 0 (r values);
//  8. T = R_full V1 D1^{-1} V1^T R_full^T;  9. EVD T = W E W^T, descending;
// 10. U = Q W(:, 1:k) = Y (L^{-T} W(:, 1:k)): Mix (s x k), Sigma(1:kk), kk = min(k, r, |S|);
//     columns and Sigma beyond kk are zero.
// Three s x s buffers b0, b1, b2 (shared memory when s <= SMEM_S); gw (global) keeps L^{-1}
// and R_full between phases (2 s x s) plus the fallback buffers (3 s x s).

__global__ void __launch_bounds__(CT) k_nystrom(const double *K, const double *C, int s, int k,
                                                double eps_rel, double drop_tol, double *Mix,
                                                double *Sigma, int32_t *rank, double *gw,
                                                int use_smem, int polish, int jac_smem) {
  extern __shared__ __align__(16) double dsm[];
  __shared__ int nk, r_keep;
  __shared__ int32_t msk[256], keepc[256], order[256];
  __shared__ double diag0[256], dvals[256], evals[256];
  const int tid = threadIdx.x;
  const size_t ss = (size_t)s * s;
  {  // batch: block b works on the b-th problem
    const size_t b = blockIdx.x;
    K += b * ss;
    C += b * ss;
    Mix += b * (size_t)s * k;
    Sigma += b * (size_t)k;
    rank += b;
    gw += b * (5 * ss + 64);
  }
  double *gLinv = gw, *gRf = gw + ss;
  const Scratch S = scratch(dsm, gw + 2 * ss, s, use_smem);

  // step 5: Cholesky-QR of Y through K: b0 = L, b1 = L^{-1}
  for (size_t i = tid; i < ss; i += CT) {
    S.b0[i] = K[i];
    S.b1[i] = (i / s == i % s) ? 1.0 : 0.0;
  }
  for (int i = tid; i < s; i += CT) diag0[i] = K[i * s + i];
  __syncthreads();
  chol_threshold(S.b0, diag0, s, drop_tol, msk, &nk);
  trsm_masked(S.b0, s, msk, S.b1, s, false, true);
  for (size_t i = tid; i < ss; i += CT) {
    gLinv[i] = S.b1[i];
    S.b2[i] = K[i];
  }
  __syncthreads();
  gemm_nn(S.b1, S.b2, S.b0, s);  // R_full = L^{-1} K (rows of dropped columns are zero)
  for (size_t i = tid; i < ss; i += CT) gRf[i] = S.b0[i];
  // step 6: symmetric C into b0
  __shared__ int c_ok;
  __shared__ double red2[CT / 32];
  for (size_t idx = tid; idx < ss; idx += CT) {
    const int i = idx / s, j = idx % s;
    S.b0[idx] = 0.5 * (C[i * s + j] + C[j * s + i]);
  }
  for (int i = tid; i < s; i += CT) diag0[i] = 0.5 * (C[i * s + i] + C[i * s + i]);
  __syncthreads();
  // steps 7-8 when C is provably well conditioned: with C = L_C L_C^T and
  // lambda_min(C) >= 1 / ||L_C^{-1}||_F^2 >= eps_rel trace(C) >= eps_rel lambda_max(C), the
  // eigenvalue threshold of step 7 keeps every eigenvalue, so V1 D1^{-1} V1^T = C^{-1} and
  // R V1 D1^{-1/2} may be replaced by R L_C^{-T} (same T = R C^{-1} R^T); no EVD of C.
  chol_threshold(S.b0, diag0, s, 0.0, keepc, &r_keep);
  for (size_t i = tid; i < ss; i += CT) S.b1[i] = (i / s == i % s) ? 1.0 : 0.0;
  __syncthreads();
  trsm_masked(S.b0, s, keepc, S.b1, s, false, true);  // b1 = L_C^{-1}
  {
    double a = 0.0;
    for (size_t i = tid; i < ss; i += CT) a += S.b1[i] * S.b1[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
    if ((tid & 31) == 0) red2[tid >> 5] = a;
    __syncthreads();
    if (tid == 0) {
      double fro2 = 0.0, tr = 0.0;
      for (int w = 0; w < CT / 32; ++w) fro2 += red2[w];
      for (int i = 0; i < s; ++i) tr += diag0[i];
      c_ok = r_keep == s && tr > 0.0 && 1.0 / fro2 >= eps_rel * tr;
    }
    __syncthreads();
  }
  if (c_ok) {
    // b0 = RV = R_full L_C^{-T} (L_C^{-1} transposed in place first, so that the product
    // reads rows of both operands)
    for (size_t i = tid; i < ss; i += CT) S.b2[i] = gRf[i];
    for (size_t e = tid; e < ss; e += CT) {
      const int i = e / s, j = e % s;
      if (i > j) {
        const double x = S.b1[e];
        S.b1[e] = S.b1[j * s + i];
        S.b1[j * s + i] = x;
      }
    }
    __syncthreads();
    for (int i = tid >> 5; i < s; i += CT / 32)
      for (int j = tid & 31; j < s; j += 32) {
        double v = 0.0;
        for (int t = 0; t <= j; ++t) v += S.b2[i * s + t] * S.b1[t * s + j];
        S.b0[i * s + j] = v;
      }
    __syncthreads();
  } else {
    // step 7: EVD of C: eigenvalues on b0's diagonal, V in b1
    for (size_t idx = tid; idx < ss; idx += CT) {
      const int i = idx / s, j = idx % s;
      S.b0[idx] = 0.5 * (C[i * s + j] + C[j * s + i]);
    }
    __syncthreads();
    eig_sym(S.b0, s, S.b1, S.b2, polish != 0, jac_smem ? reinterpret_cast<float *>(dsm) : nullptr);
    if (tid == 0) {
      double dmax = 0.0;
      for (int j = 0; j < s; ++j) dmax = fmax(dmax, S.b0[j * s + j]);
      int r = 0;
      for (int j = 0; j < s; ++j) {
        const double d = S.b0[j * s + j];
        dvals[j] = d;
        keepc[j] = (d > 0.0 && d >= eps_rel * dmax) ? 1 : 0;
        r += keepc[j];
      }
      r_keep = r;
    }
    __syncthreads();
    // step 8: b0 = RV = R_full V1 D1^{-1/2}; b2 = R_full
    for (size_t i = tid; i < ss; i += CT) S.b2[i] = gRf[i];
    __syncthreads();
    gemm_nn(S.b2, S.b1, S.b0, s);
    for (size_t idx = tid; idx < ss; idx += CT) {
      const int j = idx % s;
      S.b0[idx] = keepc[j] ? S.b0[idx] / sqrt(dvals[j]) : 0.0;
    }
    __syncthreads();
  }
  for (size_t e = tid; e < ss; e += CT) S.b2[(e % s) * s + e / s] = S.b0[e];  // b2 = RV^T
  __syncthreads();
  for (int i = tid >> 5; i < s; i += CT / 32)  // b1 = T = RV RV^T (symmetric)
    for (int j = i + (tid & 31); j < s; j += 32) {
      double v = 0.0;
      for (int t = 0; t < s; ++t) v += S.b0[i * s + t] * S.b2[t * s + j];
      S.b1[i * s + j] = v;
      S.b1[j * s + i] = v;
    }
  __syncthreads();
  for (size_t i = tid; i < ss; i += CT) S.b0[i] = S.b1[i];
  __syncthreads();
  // step 9: EVD of T: eigenvalues on b0's diagonal, W in b1
  eig_sym(S.b0, s, S.b1, S.b2, polish != 0, jac_smem ? reinterpret_cast<float *>(dsm) : nullptr);
  for (int j = tid; j < s; j += CT) {
    evals[j] = S.b0[j * s + j];
    order[j] = j;
  }
  __syncthreads();
  if (tid < s) {  // descending order by rank (ties by index); every write stays in [0, s)
    const double e = evals[tid];
    int rk = 0;
    for (int b = 0; b < s; ++b) {
      const double f = evals[b];
      rk += (f > e || (f == e && b < tid)) ? 1 : 0;
    }
    order[min(rk, s - 1)] = tid;
  }
  __syncthreads();
  if (tid == 0) {
    const int kk = min(k, min(r_keep, nk));
    *rank = kk;
    for (int j = 0; j < k; ++j) Sigma[j] = j < kk ? fmax(evals[order[j]], 0.0) : 0.0;
    r_keep = kk;
  }
  for (size_t i = tid; i < ss; i += CT) S.b2[i] = gLinv[i];
  __syncthreads();
  // step 10: Mix = L^{-T} W(:, order[0:kk])
  const int kk = r_keep;
  for (size_t idx = tid; idx < (size_t)s * k; idx += CT) {
    const int i = idx / k, j = idx % k;
    double v = 0.0;
    if (j < kk && msk[i]) {
      const int col = order[j];
      for (int t = i; t < s; ++t) v += S.b2[t * s + i] * S.b1[t * s + col];
    }
    Mix[idx] = v;
  }
}

size_t smem_for(int s) { return s <= SMEM_S ? 3 * (size_t)s * s * sizeof(double) : 0; }
// above SMEM_S: shared memory for one s x s FP64 factor (Cholesky kernels), or for the two
// FP32 Jacobi matrices (Nyström core), when it fits in 210 KiB
constexpr size_t kCoreSmemMax = 206 * 1024;
size_t smem_factor(int s) {
  const size_t b = (size_t)s * s * sizeof(double);
  return s > SMEM_S && b <= kCoreSmemMax ? b : 0;
}
size_t smem_jacobi(int s) {
  const size_t b = 2 * (size_t)s * (size_t)(s | 1) * sizeof(float);
  return s > SMEM_S && b <= kCoreSmemMax ? b : 0;
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  ensure_dyn_smem(kernel, bytes);
}

}  // namespace

size_t core_work_size(int s) { return 3 * (size_t)s * s + 64; }

void launch_chol_drop(const double *C, int s, double drop_tol, double *Rinv, int32_t *mask,
                      int32_t *nkept, double *gwork, cudaStream_t stream, int batch) {
  size_t sm = smem_for(s);
  int mode = sm > 0 ? 1 : 0;
  if (!sm && (sm = smem_factor(s)) > 0) mode = 2;
  set_smem(k_chol_drop, sm);
  k_chol_drop<<<batch, CT, sm, stream>>>(C, s, drop_tol, Rinv, mask, nkept, gwork, mode);
  NSP_LAUNCH_CHECK();
}

void launch_spd_solve_masked(const double *PtQ, const double *Rhs, int s, int r,
                             const int32_t *mask, double sign, double *out, double *gwork,
                             DevStatus *st, cudaStream_t stream) {
  const size_t sm = (s <= SMEM_S && r <= s) ? smem_for(s) : 0;
  set_smem(k_spd_solve_masked, sm);
  k_spd_solve_masked<<<1, CT, sm, stream>>>(PtQ, Rhs, s, r, mask, sign, out, gwork, sm > 0, st);
  NSP_LAUNCH_CHECK();
}

void launch_max_ratio(const double *colsq, const double *bnorm, int s, double *ratio,
                      cudaStream_t stream, int batch) {
  k_max_ratio<<<batch, 256, 0, stream>>>(colsq, bnorm, s, ratio);
  NSP_LAUNCH_CHECK();
}

void launch_sqrt_vec(const double *in, int s, double *out, cudaStream_t stream) {
  k_sqrt_vec<<<1, 256, 0, stream>>>(in, s, out);
  NSP_LAUNCH_CHECK();
}

size_t nystrom_work_size(int s) { return 5 * (size_t)s * s + 64; }

void launch_nystrom_core(const double *K, const double *C, int s, int k, double eps_rel,
                         double drop_tol, double *Mix, double *Sigma, int32_t *rank,
                         double *work, cudaStream_t stream, int batch, int polish) {
  size_t sm = smem_for(s);
  int jac = 0;
  if (!sm && (sm = smem_jacobi(s)) > 0) jac = 1;
  set_smem(k_nystrom, sm);
  k_nystrom<<<batch, CT, sm, stream>>>(K, C, s, k, eps_rel, drop_tol, Mix, Sigma, rank, work,
                                       jac ? 0 : (sm > 0), polish, jac);
  NSP_LAUNCH_CHECK();
}

}  // namespace nsp
