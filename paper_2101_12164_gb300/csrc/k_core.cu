// Small dense linear algebra on one CTA: the s x s steps of the breakdown-free block PCG
// (Cholesky-QR with column drop, alpha/beta solves) and the Nyström core of Algorithm 2
// steps 5-10 (Cholesky-QR of Y, EVD of C, T, EVD of T). s <= 256. Working sets live in
// shared memory when they fit (s <= 88), otherwise in a global scratch area.
//
// Symmetric EVD: cyclic Jacobi (rotation of pair (p, q) from Golub & Van Loan's 2x2
// symmetric Schur decomposition: tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c) with the round-robin ordering of disjoint
// pairs, first in FP32; the FP32 eigenvectors are then orthonormalized in FP64 (modified
// Gram-Schmidt), B = V^T C V is formed in FP64 and FP64 Jacobi sweeps with the threshold
// |b_pq| > tol sqrt(|b_pp b_qq|) finish the decomposition, so eigenvalues and vectors are
// FP64-accurate while most rotations run at FP32 speed.
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
// (row-major); rows with mask == 0 are set to zero. Eight lanes share each column.
__device__ void trsm_masked(const double *L, int s, const int32_t *mask, double *X, int r,
                            bool transpose, bool identity_rhs = false) {
  // lanes per column: enough groups to cover all r columns in one pass when possible
  const int lpc = r <= CT / 8 ? 8 : 4;
  const int lane8 = threadIdx.x % lpc, grp = threadIdx.x / lpc;
  for (int c0 = 0; c0 < r; c0 += CT / lpc) {
    const int c = c0 + grp;
    const bool act = c < r;
    for (int step = 0; step < s; ++step) {
      const int i = transpose ? s - 1 - step : step;
      double part = 0.0;
      // forward solve of an identity column c: rows i < c stay zero
      if (act && mask[i] && !(identity_rhs && !transpose && i < c)) {
        if (!transpose) {
          for (int t = (identity_rhs ? c : 0) + lane8; t < i; t += lpc)
            if (mask[t]) part += L[i * s + t] * X[t * r + c];
        } else {
          for (int t = i + 1 + lane8; t < s; t += lpc)
            if (mask[t]) part += L[t * s + i] * X[t * r + c];
        }
      }
      if (lpc == 8) part += __shfl_xor_sync(FULL, part, 4);
      part += __shfl_xor_sync(FULL, part, 2);
      part += __shfl_xor_sync(FULL, part, 1);
      if (lane8 == 0 && act) X[i * r + c] = mask[i] ? (X[i * r + c] - part) / L[i * s + i] : 0.0;
      __syncwarp();
    }
  }
  __syncthreads();
}

// Cyclic Jacobi on symmetric A (s x s row-major); V accumulates (A_in = V A_out V^T).
// A rotation is applied when |a_pq| > tol * sqrt(|a_pp a_qq|) and |a_pq| > floor_rel ||A||_F
// (below that the entry is at the rounding level of the matrix).
template <typename F>
__device__ void jacobi(F *A, F *V, int s, int max_sweeps, F tol, F floor_rel) {
  __shared__ F cs[128], sn[128];
  __shared__ int pp[128], qq[128];
  __shared__ int any;
  __shared__ F fro_sh;
  __shared__ float red[CT];
  const int tid = threadIdx.x;
  {  // ||A||_F (rotations keep it): off-diagonal entries below floor_rel ||A||_F are final
    float acc = 0.0f;
    for (int i = tid; i < s * s; i += CT) acc += (float)A[i] * (float)A[i];
    red[tid] = acc;
    __syncthreads();
    for (int h = CT / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) fro_sh = (F)sqrtf(red[0]);
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
      for (int k = tid; k < npair; k += CT) {
        int p = ring_at(k, round), q = ring_at(se - 1 - k, round);
        if (p > q) { const int x = p; p = q; q = x; }
        pp[k] = p;
        qq[k] = q;
        F c = F(1), sv = F(0);
        if (q < s) {
          const F apq = A[p * s + q], app = A[p * s + p], aqq = A[q * s + q];
          if (fabs(apq) > floor_abs && fabs(apq) > tol * sqrt_(fabs(app * aqq))) {
            const F tau = (aqq - app) / (F(2) * apq);
            const F tt = (tau >= F(0) ? F(1) : F(-1)) / (fabs(tau) + sqrt_(F(1) + tau * tau));
            c = F(1) / sqrt_(F(1) + tt * tt);
            sv = tt * c;
            any = 1;
          }
        }
        cs[k] = c;
        sn[k] = sv;
      }
      __syncthreads();
      const int lane = tid & 31, warp = tid >> 5;
      for (int k = warp; k < npair; k += CT / 32) {  // A <- A J, V <- V J
        const F sv = sn[k];
        if (sv == F(0)) continue;
        const int p = pp[k], q = qq[k];
        const F c = cs[k];
        for (int i = lane; i < s; i += 32) {
          const F ap = A[i * s + p], aq = A[i * s + q];
          A[i * s + p] = c * ap - sv * aq;
          A[i * s + q] = sv * ap + c * aq;
          const F vp = V[i * s + p], vq = V[i * s + q];
          V[i * s + p] = c * vp - sv * vq;
          V[i * s + q] = sv * vp + c * vq;
        }
      }
      __syncthreads();
      for (int k = warp; k < npair; k += CT / 32) {  // A <- J^T A
        const F sv = sn[k];
        if (sv == F(0)) continue;
        const int p = pp[k], q = qq[k];
        const F c = cs[k];
        for (int j = lane; j < s; j += 32) {
          const F ap = A[p * s + j], aq = A[q * s + j];
          A[p * s + j] = c * ap - sv * aq;
          A[q * s + j] = sv * ap + c * aq;
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

// Modified Gram-Schmidt on the columns of V (s x s row-major, FP64).
__device__ void mgs_columns(double *V, int s) {
  __shared__ double red[CT];
  __shared__ double coef[256];
  const int tid = threadIdx.x;
  for (int j = 0; j < s; ++j) {
    // coefficients against the previous columns, then subtract, then normalize
    for (int i = tid; i < j; i += CT) {
      double d = 0.0;
      for (int r = 0; r < s; ++r) d += V[r * s + i] * V[r * s + j];
      coef[i] = d;
    }
    __syncthreads();
    for (int r = tid; r < s; r += CT) {
      double v = V[r * s + j];
      for (int i = 0; i < j; ++i) v -= coef[i] * V[r * s + i];
      V[r * s + j] = v;
    }
    __syncthreads();
    double sq = 0.0;
    for (int r = tid; r < s; r += CT) sq += V[r * s + j] * V[r * s + j];
    red[tid] = sq;
    __syncthreads();
    for (int h = CT / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    const double nrm = sqrt(red[0]);
    for (int r = tid; r < s; r += CT) V[r * s + j] = nrm > 0.0 ? V[r * s + j] / nrm : 0.0;
    __syncthreads();
  }
}

// FP64-accurate EVD of the symmetric matrix held in Bm (s x s): on return the eigenvalues
// are on the diagonal of Bm and the eigenvectors in the columns of V. W1 is s x s scratch,
// also used for the two FP32 matrices of the first phase. All three may be shared memory.
__device__ void eig_sym(double *Bm, int s, double *V, double *W1, bool polish) {
  const int tid = threadIdx.x;
  const size_t ss = (size_t)s * s;
  float *A32 = reinterpret_cast<float *>(W1), *V32 = A32 + ss;
  for (size_t i = tid; i < ss; i += CT) {
    A32[i] = (float)Bm[i];
    V32[i] = (i / s == i % s) ? 1.0f : 0.0f;
  }
  __syncthreads();
  jacobi<float>(A32, V32, s, 8, 1e-6f, 2e-7f);
  for (size_t i = tid; i < ss; i += CT) V[i] = (double)V32[i];
  __syncthreads();
  mgs_columns(V, s);
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
  if (polish) jacobi<double>(Bm, V, s, 1, 1e-13, 1e-15);
}

struct Scratch {
  double *b0, *b1, *b2;  // three s x s buffers (smem or global)
};

__device__ Scratch scratch(double *smem, double *global, int s, bool use_smem) {
  const size_t ss = (size_t)s * s;
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
                                                int use_smem, int polish) {
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
  __shared__ double red2[CT];
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
    red2[tid] = a;
    __syncthreads();
    for (int h = CT / 2; h > 0; h >>= 1) {
      if (tid < h) red2[tid] += red2[tid + h];
      __syncthreads();
    }
    if (tid == 0) {
      double tr = 0.0;
      for (int i = 0; i < s; ++i) tr += diag0[i];
      c_ok = r_keep == s && tr > 0.0 && 1.0 / red2[0] >= eps_rel * tr;
    }
    __syncthreads();
  }
  if (c_ok) {
    // b0 = RV = R_full L_C^{-T}
    for (size_t i = tid; i < ss; i += CT) S.b2[i] = gRf[i];
    __syncthreads();
    for (int i = tid >> 5; i < s; i += CT / 32)
      for (int j = tid & 31; j < s; j += 32) {
        double v = 0.0;
        for (int t = 0; t <= j; ++t) v += S.b2[i * s + t] * S.b1[j * s + t];
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
    eig_sym(S.b0, s, S.b1, S.b2, polish != 0);
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
  for (int i = tid >> 5; i < s; i += CT / 32)  // b1 = T = RV RV^T (symmetric)
    for (int j = i + (tid & 31); j < s; j += 32) {
      double v = 0.0;
      for (int t = 0; t < s; ++t) v += S.b0[i * s + t] * S.b0[j * s + t];
      S.b1[i * s + j] = v;
      S.b1[j * s + i] = v;
    }
  __syncthreads();
  for (size_t i = tid; i < ss; i += CT) S.b0[i] = S.b1[i];
  __syncthreads();
  // step 9: EVD of T: eigenvalues on b0's diagonal, W in b1
  eig_sym(S.b0, s, S.b1, S.b2, polish != 0);
  if (tid == 0) {
    for (int j = 0; j < s; ++j) { evals[j] = S.b0[j * s + j]; order[j] = j; }
    for (int a = 0; a < s; ++a) {  // selection sort, descending
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (evals[order[b]] > evals[order[best]]) best = b;
      const int x = order[a]; order[a] = order[best]; order[best] = x;
    }
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

template <typename K>
void set_smem(K kernel, size_t bytes) {
  ensure_dyn_smem(kernel, bytes);
}

}  // namespace

size_t core_work_size(int s) { return 3 * (size_t)s * s + 64; }

void launch_chol_drop(const double *C, int s, double drop_tol, double *Rinv, int32_t *mask,
                      int32_t *nkept, double *gwork, cudaStream_t stream, int batch) {
  const size_t sm = smem_for(s);
  set_smem(k_chol_drop, sm);
  k_chol_drop<<<batch, CT, sm, stream>>>(C, s, drop_tol, Rinv, mask, nkept, gwork, sm > 0);
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
  const size_t sm = smem_for(s);
  set_smem(k_nystrom, sm);
  k_nystrom<<<batch, CT, sm, stream>>>(K, C, s, k, eps_rel, drop_tol, Mix, Sigma, rank, work,
                                       sm > 0, polish);
  NSP_LAUNCH_CHECK();
}

}  // namespace nsp
