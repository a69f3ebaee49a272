// Small dense FP64 linear algebra on one CTA: the s x s steps of the breakdown-free block
// PCG (Cholesky-QR with column drop, alpha/beta solves) and the Nyström core of
// Algorithm 2 steps 5-10 (Cholesky-QR of Y, EVD of C, T, EVD of T). s <= 256.
// Matrices live in a global scratch area (row-major, s x s), cached in L1/L2.
#include <cfloat>

#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int CT = 512;  // threads of the single CTA

// In-place thresholded right-looking Cholesky of L (s x s, row-major, lower part used):
// column j is kept when its pivot exceeds drop_tol * diag0[j] (and diag0[j] > 0), otherwise
// it is zeroed and skipped. mask[j] = kept.
__device__ void chol_threshold(double *L, const double *diag0, int s, double drop_tol,
                               int32_t *mask, int *nkept_sh) {
  const int tid = threadIdx.x;
  if (tid == 0) *nkept_sh = 0;
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    __shared__ int keep;
    if (tid == 0) {
      const double piv = L[j * s + j];
      const double d0 = diag0[j];
      keep = (d0 > 0.0 && piv > drop_tol * d0 && piv > 0.0) ? 1 : 0;
      mask[j] = keep;
      if (keep) {
        L[j * s + j] = sqrt(piv);
        *nkept_sh += 1;
      }
    }
    __syncthreads();
    if (keep) {
      const double d = L[j * s + j];
      for (int i = j + 1 + tid; i < s; i += CT) L[i * s + j] /= d;
      __syncthreads();
      const int rem = s - j - 1;
      for (int idx = tid; idx < rem * rem; idx += CT) {
        const int r = j + 1 + idx / rem, c = j + 1 + idx % rem;
        if (r >= c) L[r * s + c] -= L[r * s + j] * L[c * s + j];
      }
    } else {
      for (int i = j + tid; i < s; i += CT) L[i * s + j] = 0.0;
    }
    __syncthreads();
  }
}

// Linv (s x s row-major) = inverse of the kept part of lower L; zero rows/cols for dropped.
// One thread per column c: forward substitution L x = e_c over kept indices.
__device__ void lower_inverse(const double *L, const int32_t *mask, int s, double *Linv) {
  for (int c = threadIdx.x; c < s; c += CT) {
    for (int i = 0; i < s; ++i) {
      double v = 0.0;
      if (mask[i] && mask[c] && i >= c) {
        v = (i == c) ? 1.0 : 0.0;
        for (int t = c; t < i; ++t)
          if (mask[t]) v -= L[i * s + t] * Linv[t * s + c];
        v /= L[i * s + i];
      }
      Linv[i * s + c] = v;
    }
  }
  __syncthreads();
}

// Cholesky-QR with drop: Rinv[i][c] = Linv[c][i] (upper), so W Rinv has orthonormal kept cols.
__global__ void __launch_bounds__(CT) k_chol_drop(const double *C, int s, double drop_tol,
                                                  double *Rinv, int32_t *mask, int32_t *nkept,
                                                  double *work) {
  __shared__ int nk;
  double *L = work;              // s*s
  double *Linv = work + s * s;   // s*s
  double *diag0 = work + 2 * s * s;
  for (int i = threadIdx.x; i < s * s; i += CT) L[i] = C[i];
  for (int i = threadIdx.x; i < s; i += CT) diag0[i] = C[i * s + i];
  __syncthreads();
  chol_threshold(L, diag0, s, drop_tol, mask, &nk);
  lower_inverse(L, mask, s, Linv);
  for (int i = threadIdx.x; i < s * s; i += CT) {
    const int r = i / s, c = i % s;
    Rinv[i] = Linv[c * s + r];
  }
  if (threadIdx.x == 0) *nkept = nk;
}

// out (s x r) = sign * A^{-1} Rhs on the kept index set of mask (A s x s SPD there).
__global__ void __launch_bounds__(CT) k_spd_solve_masked(const double *A, const double *Rhs, int s,
                                                         int r, const int32_t *mask, double sign,
                                                         double *out, double *work, DevStatus *st) {
  double *L = work;
  const int tid = threadIdx.x;
  for (int i = tid; i < s * s; i += CT) {
    const int a = i / s, b = i % s;
    L[i] = (mask[a] && mask[b]) ? A[i] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (!mask[j]) continue;  // uniform across the CTA
    __shared__ double d;
    if (tid == 0) {
      double piv = L[j * s + j];
      if (!(piv > 0.0)) {
        dev_fail(st, DEV_BREAKDOWN, j);
        piv = 1.0;
      }
      d = sqrt(piv);
      L[j * s + j] = d;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < s; i += CT)
      if (mask[i]) L[i * s + j] /= d;
    __syncthreads();
    const int rem = s - j - 1;
    for (int idx = tid; idx < rem * rem; idx += CT) {
      const int a = j + 1 + idx / rem, b = j + 1 + idx % rem;
      if (a >= b && mask[a] && mask[b]) L[a * s + b] -= L[a * s + j] * L[b * s + j];
    }
    __syncthreads();
  }
  // one thread per right-hand side column: L y = rhs, L^T x = y
  for (int c = tid; c < r; c += CT) {
    for (int i = 0; i < s; ++i) {
      double v = 0.0;
      if (mask[i]) {
        v = Rhs[i * r + c];
        for (int t = 0; t < i; ++t)
          if (mask[t]) v -= L[i * s + t] * out[t * r + c];
        v /= L[i * s + i];
      }
      out[i * r + c] = v;
    }
    for (int i = s - 1; i >= 0; --i) {
      double v = 0.0;
      if (mask[i]) {
        v = out[i * r + c];
        for (int t = i + 1; t < s; ++t)
          if (mask[t]) v -= L[t * s + i] * out[t * r + c];
        v /= L[i * s + i];
      }
      out[i * r + c] = v;
    }
    for (int i = 0; i < s; ++i) out[i * r + c] *= sign;
  }
}

__global__ void k_max_ratio(const double *colsq, const double *bnorm, int s, double *ratio) {
  __shared__ double red[256];
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

// Cyclic Jacobi eigenvalue algorithm for a symmetric s x s matrix A (row-major, in place)
// with parallel (round-robin tournament) ordering of the disjoint rotation pairs; V
// accumulates the rotations (A_orig = V diag(A) V^T). Rotation of pair (p, q) per Golub &
// Van Loan's 2x2 symmetric Schur decomposition: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.
__device__ void jacobi_evd(double *A, double *V, int s, double *cs, double *sn, int *pp, int *qq,
                           int *ring) {
  const int tid = threadIdx.x;
  for (int i = tid; i < s * s; i += CT) V[i] = (i / s == i % s) ? 1.0 : 0.0;
  const int se = s + (s & 1);  // even player count; player s (if odd) is a bye
  const int npair = se / 2;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    __shared__ double off, tot;
    __shared__ double red[CT];
    double o = 0.0, t = 0.0;
    for (int i = tid; i < s * s; i += CT) {
      const double v = A[i] * A[i];
      t += v;
      if (i / s != i % s) o += v;
    }
    red[tid] = o;
    __syncthreads();
    for (int h = CT / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) off = red[0];
    __syncthreads();
    red[tid] = t;
    __syncthreads();
    for (int h = CT / 2; h > 0; h >>= 1) {
      if (tid < h) red[tid] += red[tid + h];
      __syncthreads();
    }
    if (tid == 0) tot = red[0];
    __syncthreads();
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int i = tid; i < se; i += CT) ring[i] = i;
    __syncthreads();
    for (int round = 0; round < se - 1; ++round) {
      // pairs of this round: (ring[i], ring[se-1-i])
      for (int k = tid; k < npair; k += CT) {
        int p = ring[k], q = ring[se - 1 - k];
        if (p > q) { const int x = p; p = q; q = x; }
        pp[k] = p;
        qq[k] = q;
        double c = 1.0, sv = 0.0;
        if (q < s) {
          const double apq = A[p * s + q];
          if (apq != 0.0) {
            const double tau = (A[q * s + q] - A[p * s + p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            sv = tt * c;
          }
        }
        cs[k] = c;
        sn[k] = sv;
      }
      __syncthreads();
      // A <- A J (columns p, q), V <- V J
      for (int idx = tid; idx < npair * s; idx += CT) {
        const int k = idx / s, i = idx % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[i * s + p], aq = A[i * s + q];
        A[i * s + p] = c * ap - sv * aq;
        A[i * s + q] = sv * ap + c * aq;
        const double vp = V[i * s + p], vq = V[i * s + q];
        V[i * s + p] = c * vp - sv * vq;
        V[i * s + q] = sv * vp + c * vq;
      }
      __syncthreads();
      // A <- J^T A (rows p, q)
      for (int idx = tid; idx < npair * s; idx += CT) {
        const int k = idx / s, j = idx % s;
        const int p = pp[k], q = qq[k];
        if (q >= s) continue;
        const double c = cs[k], sv = sn[k];
        const double ap = A[p * s + j], aq = A[q * s + j];
        A[p * s + j] = c * ap - sv * aq;
        A[q * s + j] = sv * ap + c * aq;
      }
      __syncthreads();
      // rotate the tournament ring (player 0 fixed)
      if (tid == 0) {
        const int last = ring[se - 1];
        for (int i = se - 1; i > 1; --i) ring[i] = ring[i - 1];
        ring[1] = last;
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

// Algorithm 2 steps 5-10 from K = Y^T Y and C = G^T Y (s x s):
//  5. Y = QR by Cholesky-QR: K = R^T R on the kept columns S (threshold drop_tol);
//     R_full = L^{-1} K[S, :] (|S| x s), equal to R when nothing is dropped.
//  6. C = (C + C^T)/2;  7. EVD C = V D V^T, keep d >= eps_rel max(d), d > 0 (r values);
//  8. T = R_full V1 D1^{-1} V1^T R_full^T;  9. EVD T = W E W^T, descending;
// 10. U = Q W(:, 1:k) = Y (R_SS^{-1} W(:, 1:k)): Mix = L^{-T} W_k (s x kk), Sigma = E(1:kk),
//     kk = min(k, r).
__global__ void __launch_bounds__(CT) k_nystrom(const double *K, const double *C, int s, int k,
                                                double eps_rel, double drop_tol, double *Mix,
                                                double *Sigma, int32_t *rank, double *work) {
  __shared__ int nk;
  __shared__ int r_keep;
  const int tid = threadIdx.x;
  const size_t ss = (size_t)s * s;
  double *L = work;            // Cholesky of K
  double *Linv = L + ss;
  double *Rf = Linv + ss;      // R_full (s x s, rows of dropped = 0)
  double *Cs = Rf + ss;        // symmetric C -> eigenvalues on diagonal
  double *V = Cs + ss;
  double *RV = V + ss;         // R_full V1 D1^{-1/2}
  double *T = RV + ss;
  double *W = T + ss;
  double *diag0 = W + ss;
  double *dvals = diag0 + s;
  double *evals = dvals + s;
  double *cs = evals + s;
  double *sn = cs + s;
  int32_t *mask = reinterpret_cast<int32_t *>(sn + s);
  int32_t *keepc = mask + s;
  int32_t *order = keepc + s;
  int *pp = order + s;
  int *qq = pp + s;
  int *ring = qq + s;

  // step 5: Cholesky-QR
  for (size_t i = tid; i < ss; i += CT) L[i] = K[i];
  for (int i = tid; i < s; i += CT) diag0[i] = K[i * s + i];
  __syncthreads();
  chol_threshold(L, diag0, s, drop_tol, mask, &nk);
  lower_inverse(L, mask, s, Linv);
  // R_full = Linv K
  for (size_t idx = tid; idx < ss; idx += CT) {
    const int i = idx / s, j = idx % s;
    double v = 0.0;
    if (mask[i])
      for (int t = 0; t <= i; ++t) v += Linv[i * s + t] * K[t * s + j];
    Rf[idx] = v;
  }
  // step 6: symmetrize C
  for (size_t idx = tid; idx < ss; idx += CT) {
    const int i = idx / s, j = idx % s;
    Cs[idx] = 0.5 * (C[i * s + j] + C[j * s + i]);
  }
  __syncthreads();
  // step 7: EVD of C
  jacobi_evd(Cs, V, s, cs, sn, pp, qq, ring);
  if (tid == 0) {
    double dmax = 0.0;
    for (int j = 0; j < s; ++j) dmax = fmax(dmax, Cs[j * s + j]);
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double d = Cs[j * s + j];
      dvals[j] = d;
      keepc[j] = (d > 0.0 && d >= eps_rel * dmax) ? 1 : 0;
      r += keepc[j];
    }
    r_keep = r;
  }
  __syncthreads();
  // step 8: RV = R_full V1 D1^{-1/2} (s x s, zero columns for dropped eigenvalues)
  for (size_t idx = tid; idx < ss; idx += CT) {
    const int i = idx / s, j = idx % s;
    double v = 0.0;
    if (keepc[j]) {
      for (int t = 0; t < s; ++t) v += Rf[i * s + t] * V[t * s + j];
      v /= sqrt(dvals[j]);
    }
    RV[idx] = v;
  }
  __syncthreads();
  for (size_t idx = tid; idx < ss; idx += CT) {
    const int i = idx / s, j = idx % s;
    double v = 0.0;
    for (int t = 0; t < s; ++t) v += RV[i * s + t] * RV[j * s + t];
    T[idx] = v;
  }
  __syncthreads();
  // step 9: EVD of T, order descending
  jacobi_evd(T, W, s, cs, sn, pp, qq, ring);
  if (tid == 0) {
    for (int j = 0; j < s; ++j) { evals[j] = T[j * s + j]; order[j] = j; }
    for (int a = 0; a < s; ++a) {  // selection sort, descending
      int best = a;
      for (int b = a + 1; b < s; ++b)
        if (evals[order[b]] > evals[order[best]]) best = b;
      const int x = order[a]; order[a] = order[best]; order[best] = x;
    }
    const int kk = min(k, min(r_keep, nk));
    *rank = kk;
    for (int j = 0; j < k; ++j) Sigma[j] = j < kk ? fmax(evals[order[j]], 0.0) : 0.0;
  }
  __syncthreads();
  // step 10: Mix = Linv^T W(:, order[0:kk])  (U = Y Mix = Q W_k)
  const int kk = min(k, min(r_keep, nk));
  for (size_t idx = tid; idx < (size_t)s * k; idx += CT) {
    const int i = idx / k, j = idx % k;
    double v = 0.0;
    if (j < kk && mask[i]) {
      const int col = order[j];
      for (int t = i; t < s; ++t) v += Linv[t * s + i] * W[t * s + col];
    }
    Mix[idx] = v;
  }
}

}  // namespace

void launch_chol_drop(const double *C, int s, double drop_tol, double *Rinv, int32_t *mask,
                      int32_t *nkept, cudaStream_t stream) {
  // the scratch follows Rinv: callers allocate 3*s*s + s doubles after Rinv (see engine)
  k_chol_drop<<<1, CT, 0, stream>>>(C, s, drop_tol, Rinv, mask, nkept, Rinv + (size_t)s * s);
  NSP_LAUNCH_CHECK();
}

void launch_spd_solve_masked(const double *PtQ, const double *Rhs, int s, int r,
                             const int32_t *mask, double sign, double *out, double *Lwork,
                             DevStatus *st, cudaStream_t stream) {
  k_spd_solve_masked<<<1, CT, 0, stream>>>(PtQ, Rhs, s, r, mask, sign, out, Lwork, st);
  NSP_LAUNCH_CHECK();
}

void launch_max_ratio(const double *colsq, const double *bnorm, int s, double *ratio,
                      cudaStream_t stream) {
  k_max_ratio<<<1, 256, 0, stream>>>(colsq, bnorm, s, ratio);
  NSP_LAUNCH_CHECK();
}

void launch_sqrt_vec(const double *in, int s, double *out, cudaStream_t stream) {
  k_sqrt_vec<<<1, 256, 0, stream>>>(in, s, out);
  NSP_LAUNCH_CHECK();
}

size_t nystrom_work_size(int s) { return 8 * (size_t)s * s + 16 * (size_t)s + 64; }

void launch_nystrom_core(const double *K, const double *C, int s, int k, double eps_rel,
                         double drop_tol, double *Mix, double *Sigma, int32_t *rank,
                         double *work, cudaStream_t stream) {
  k_nystrom<<<1, CT, 0, stream>>>(K, C, s, k, eps_rel, drop_tol, Mix, Sigma, rank, work);
  NSP_LAUNCH_CHECK();
}

}  // namespace nsp
