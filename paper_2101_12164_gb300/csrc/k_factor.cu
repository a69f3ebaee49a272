// Batched multifrontal Cholesky of the diagonal blocks A_1..A_N of A_I and of A_G
// ("factorized cheaply in parallel using a direct algorithm", §2.3), one CTA per supernode,
// all supernodes of one elimination-tree level of every block in one launch.
//
// Front of supernode J (m x m, column-major, lower triangle used):
//   F = A entries of J's columns + extend-add of the children's update matrices,
//   partial Cholesky of the first w columns: F = [L11 0; L21 I] [I 0; 0 U] [L11 0; L21 I]^T,
//   U (rows/cols w..m-1 of F) is J's update matrix for its parent.
// Stored panel (m x w, column-major): [inv(L11); L21 inv(L11)], so that both triangular
// sweeps of the solve become dense products (see k_solve.cu).
#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int FT = 256;  // threads per CTA
constexpr int NB = 32;   // column block of the blocked factorization
constexpr int TT = 64;   // output tile of the trailing update

__device__ __forceinline__ float fsqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double fsqrt_(double x) { return sqrt(x); }

template <typename T>
struct FactorSmem {
  T D[NB][NB + 1];
  T Lr[TT][NB + 1];
  T Lc[TT][NB + 1];
};

// Right-looking blocked partial Cholesky of the first w columns of F (m x m).
template <typename T>
__device__ void partial_cholesky(T *F, int m, int w, int32_t blk, DevStatus *st,
                                 FactorSmem<T> &sm) {
  const int tid = threadIdx.x;
  for (int kb = 0; kb < w; kb += NB) {
    const int nb = min(NB, w - kb);
    for (int i = tid; i < NB * NB; i += FT) {
      int r = i % NB, c = i / NB;
      sm.D[r][c] = (r < nb && c < nb && r >= c) ? F[(size_t)(kb + r) + (size_t)(kb + c) * m] : T(0);
    }
    __syncthreads();
    // unblocked Cholesky of the diagonal block
    for (int j = 0; j < nb; ++j) {
      if (tid == 0) {
        T d = sm.D[j][j];
        if (!(d > T(0))) {
          dev_fail(st, DEV_NOT_SPD, blk);
          d = T(1);
        }
        sm.D[j][j] = fsqrt_(d);
      }
      __syncthreads();
      const T djj = sm.D[j][j];
      for (int i = j + 1 + tid; i < nb; i += FT) sm.D[i][j] /= djj;
      __syncthreads();
      const int rem = nb - j - 1;
      for (int idx = tid; idx < rem * rem; idx += FT) {
        int r = j + 1 + idx % rem, c = j + 1 + idx / rem;
        if (r >= c) sm.D[r][c] -= sm.D[r][j] * sm.D[c][j];
      }
      __syncthreads();
    }
    for (int i = tid; i < nb * nb; i += FT) {
      int r = i % nb, c = i / nb;
      if (r >= c) F[(size_t)(kb + r) + (size_t)(kb + c) * m] = sm.D[r][c];
    }
    // rows below the diagonal block: L[r, kb:kb+nb] = F[r, kb:kb+nb] * Ld^{-T}
    for (int r = kb + nb + tid; r < m; r += FT) {
      T x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        x[j] = T(0);
        if (j < nb) {
          T v = F[(size_t)r + (size_t)(kb + j) * m];
#pragma unroll
          for (int t = 0; t < NB; ++t)
            if (t < j) v -= x[t] * sm.D[j][t];
          x[j] = v / sm.D[j][j];
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < nb) F[(size_t)r + (size_t)(kb + j) * m] = x[j];
    }
    __syncthreads();
    // trailing update of the lower triangle [kb+nb, m)^2 (panel columns and update matrix)
    const int c0 = kb + nb;
    const int rem = m - c0;
    if (rem > 0) {
      const int nt = (rem + TT - 1) / TT;
      const int ntiles = nt * (nt + 1) / 2;
      const int tx = tid % 16, ty = tid / 16;
      for (int tile = 0; tile < ntiles; ++tile) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        const int tj = tile - ti * (ti + 1) / 2;
        const int rb = c0 + ti * TT, cb = c0 + tj * TT;
        for (int i = tid; i < TT * NB; i += FT) {
          int rr = i % TT, t = i / TT;
          T a = T(0), b = T(0);
          if (t < nb) {
            if (rb + rr < m) a = F[(size_t)(rb + rr) + (size_t)(kb + t) * m];
            if (cb + rr < m) b = F[(size_t)(cb + rr) + (size_t)(kb + t) * m];
          }
          sm.Lr[rr][t] = a;
          sm.Lc[rr][t] = b;
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        for (int t = 0; t < nb; ++t) {
          T a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = sm.Lr[tx + 16 * i][t];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = sm.Lc[ty + 16 * j][t];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            int r = rb + tx + 16 * i, c = cb + ty + 16 * j;
            if (r < m && c < m && r >= c) F[(size_t)r + (size_t)c * m] -= acc[i][j];
          }
        __syncthreads();
      }
    }
  }
}

// X = [I; L21] * inv(L11) written to the panel (m x w, column-major): the top w x w part is
// inv(L11) (lower triangular), the bottom part L21 inv(L11). Solved from the right,
// column blocks from the last to the first: X L11 = [I; L21].
template <typename T>
__device__ void inverse_panel(const T *F, T *P, int m, int w, FactorSmem<T> &sm) {
  const int tid = threadIdx.x;
  for (int i = tid; i < w * w; i += FT) {
    int r = i % w, c = i / w;
    if (r < c) P[(size_t)r + (size_t)c * m] = T(0);
  }
  __syncthreads();
  const int nblk = (w + NB - 1) / NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int jb = bi * NB;
    const int nb = min(NB, w - jb);
    for (int i = tid; i < NB * NB; i += FT) {
      int r = i % NB, c = i / NB;
      sm.D[r][c] = (r < nb && c < nb && r >= c) ? F[(size_t)(jb + r) + (size_t)(jb + c) * m] : T(0);
    }
    __syncthreads();
    const int cbeg = jb + nb;  // already computed columns of X: [cbeg, w)
    for (int rbase = jb; rbase < m; rbase += FT) {
      const int r = rbase + tid;
      T tmp[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        T v = T(0);
        if (r < m && t < nb) v = (r < w) ? T(r == jb + t ? 1 : 0) : F[(size_t)r + (size_t)(jb + t) * m];
        tmp[t] = v;
      }
      // tmp -= X[r, cbeg:w) * L11[cbeg:w, jb:jb+nb), staged TT rows of L11 at a time
      for (int cc = cbeg; cc < w; cc += TT) {
        const int cn = min(TT, w - cc);
        __syncthreads();
        for (int i = tid; i < TT * NB; i += FT) {
          int rr = i % TT, t = i / TT;
          sm.Lr[rr][t] = (rr < cn && t < nb) ? F[(size_t)(cc + rr) + (size_t)(jb + t) * m] : T(0);
        }
        __syncthreads();
        if (r < m) {
          for (int q = 0; q < cn; ++q) {
            const T xv = P[(size_t)r + (size_t)(cc + q) * m];
#pragma unroll
            for (int t = 0; t < NB; ++t) tmp[t] -= xv * sm.Lr[q][t];
          }
        }
      }
      // x * Ld = tmp  ->  x[t] = (tmp[t] - sum_{u>t} x[u] Ld[u][t]) / Ld[t][t]
      if (r < m) {
        T x[NB];
#pragma unroll
        for (int t = NB - 1; t >= 0; --t) {
          x[t] = T(0);
          if (t < nb) {
            T v = tmp[t];
#pragma unroll
            for (int u = 0; u < NB; ++u)
              if (u > t && u < nb) v -= x[u] * sm.D[u][t];
            x[t] = v / sm.D[t][t];
          }
        }
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < nb) P[(size_t)r + (size_t)(jb + t) * m] = x[t];
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(FT) k_factor(ForestDev f, const int32_t *level_sn,
                                               const double *Aval, T *front, T *panel,
                                               DevStatus *st) {
  __shared__ FactorSmem<T> sm;
  const int J = level_sn[blockIdx.x];
  const int w = f.sn_w[J], m = f.sn_m[J];
  T *F = front + f.sn_front[J];
  const int tid = threadIdx.x;
  for (size_t i = tid; i < (size_t)m * m; i += FT) F[i] = T(0);
  __syncthreads();
  for (int64_t e = f.asm_ptr[J] + tid; e < f.asm_ptr[J + 1]; e += FT)
    F[f.asm_dst[e]] = (T)Aval[f.asm_src[e]];
  __syncthreads();
  for (int ci = f.ch_ptr[J]; ci < f.ch_ptr[J + 1]; ++ci) {
    const int C = f.ch_list[ci];
    const int wc = f.sn_w[C], mc = f.sn_m[C], mu = mc - wc;
    const T *FC = front + f.sn_front[C];
    const int32_t *rm = f.relmap + f.sn_upd[C];
    for (int idx = tid; idx < mu * mu; idx += FT) {
      const int a = idx % mu, b = idx / mu;
      if (a >= b) F[(size_t)rm[a] + (size_t)rm[b] * m] += FC[(size_t)(wc + a) + (size_t)(wc + b) * mc];
    }
    __syncthreads();
  }
  partial_cholesky<T>(F, m, w, f.sn_block[J], st, sm);
  __syncthreads();
  inverse_panel<T>(F, panel + f.sn_panel[J], m, w, sm);
}

}  // namespace

template <typename T>
void launch_factor_level(const ForestDev &f, const int32_t *level_sn, int count,
                         const double *Aval, T *front, T *panel, DevStatus *st,
                         cudaStream_t stream) {
  if (count <= 0) return;
  k_factor<T><<<count, FT, 0, stream>>>(f, level_sn, Aval, front, panel, st);
  NSP_LAUNCH_CHECK();
}

template void launch_factor_level<float>(const ForestDev &, const int32_t *, int, const double *,
                                         float *, float *, DevStatus *, cudaStream_t);
template void launch_factor_level<double>(const ForestDev &, const int32_t *, int, const double *,
                                          double *, double *, DevStatus *, cudaStream_t);

}  // namespace nsp
