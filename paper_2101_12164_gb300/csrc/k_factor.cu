// Batched multifrontal Cholesky of the diagonal blocks A_1..A_N of A_I and of A_G
// ("factorized cheaply in parallel using a direct algorithm", §2.3). All supernodes of one
// elimination-tree level of every block run in one launch: small fronts one CTA each, large
// fronts a thread-block cluster of NC CTAs each (cluster barriers between the phases of the
// blocked factorization; the inverse-panel phase needs none because every row tile of a
// front is always handled by the same CTA).
//
// Front of supernode J (m x m, column-major, lower triangle used):
//   F = A entries of J's columns + extend-add of the children's update matrices,
//   partial Cholesky of the first w columns: F = [L11 0; L21 I] [I 0; 0 U] [L11 0; L21 I]^T,
//   U (rows/cols w..m-1 of F) is J's update matrix for its parent.
// Stored panel (column-major, leading dimension m rounded up to 4, zero pad rows):
// X = [inv(L11); L21 inv(L11)] = [I; L21] inv(L11), so that both triangular sweeps of the
// solve become dense products (see k_solve.cu).
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace nsp {
namespace {

constexpr int FT = 256;  // threads per CTA
// resident CTAs per SM the register budget is sized for: the small FP32 fronts of the lower
// tree levels are latency bound and gain from more CTAs per SM; FP64 keeps one
template <typename T>
struct FactorOcc {
  static constexpr int value = sizeof(T) == 4 ? 3 : 1;
};
constexpr int NB = 32;   // column block of the blocked factorization
constexpr int TT = 64;   // output tile of the trailing update / row tile of the inverse

__device__ __forceinline__ float fsqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double fsqrt_(double x) { return sqrt(x); }

template <typename T>
struct FactorSmem {
  T D[NB][NB + 1];
  T Lr[TT][NB + 1];
  T Lc[TT][NB + 1];
};

template <int NC>
__device__ __forceinline__ void front_sync() {
  if constexpr (NC > 1) cg::this_cluster().sync();
  else __syncthreads();
}

template <int NC>
__device__ __forceinline__ int front_rank() {
  if constexpr (NC > 1) return (int)cg::this_cluster().block_rank();
  else return 0;
}

// unblocked Cholesky of the nb x nb diagonal block staged in D (every CTA of the front does
// it on its own copy; only rank 0 reports a bad pivot)
template <typename T>
__device__ void diag_block_cholesky(FactorSmem<T> &sm, int nb, int32_t blk, DevStatus *st,
                                    bool report) {
  const int tid = threadIdx.x;
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      T d = sm.D[j][j];
      if (!(d > T(0))) {
        if (report) dev_fail(st, DEV_NOT_SPD, blk);
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
      const int r = j + 1 + idx % rem, c = j + 1 + idx / rem;
      if (r >= c) sm.D[r][c] -= sm.D[r][j] * sm.D[c][j];
    }
    __syncthreads();
  }
}

// stage the lower triangle of the nb x nb diagonal block at (kb, kb) of F into D, all loads
// in flight before the shared-memory writes
template <typename T>
__device__ __forceinline__ void stage_diag(const T *F, int m, int kb, int nb, FactorSmem<T> &sm) {
  constexpr int NQ = NB * NB / FT;
  T v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * FT, r = i % NB, c = i / NB;
    v[q] = (r < nb && c < nb && r >= c) ? F[(size_t)(kb + r) + (size_t)(kb + c) * m] : T(0);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * FT;
    sm.D[i % NB][i / NB] = v[q];
  }
}

// Right-looking blocked partial Cholesky of the first w columns of F (m x m).
template <typename T, int NC>
__device__ void partial_cholesky(T *F, int m, int w, int32_t blk, DevStatus *st,
                                 FactorSmem<T> &sm) {
  const int tid = threadIdx.x;
  const int rank = front_rank<NC>();
  for (int kb = 0; kb < w; kb += NB) {
    const int nb = min(NB, w - kb);
    stage_diag(F, m, kb, nb, sm);
    __syncthreads();
    diag_block_cholesky(sm, nb, blk, st, rank == 0);
    // rows below the diagonal block: L[r, kb:kb+nb] = F[r, kb:kb+nb] Ld^{-T}
    for (int r = kb + nb + rank * FT + tid; r < m; r += NC * FT) {
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
    front_sync<NC>();
    // every CTA has read the diagonal block: rank 0 stores its factor
    if (rank == 0)
      for (int i = tid; i < nb * nb; i += FT) {
        const int r = i % nb, c = i / nb;
        if (r >= c) F[(size_t)(kb + r) + (size_t)(kb + c) * m] = sm.D[r][c];
      }
    // trailing update of the lower triangle [kb+nb, m)^2 (panel columns and update matrix)
    const int c0 = kb + nb;
    const int rem = m - c0;
    if (rem > 0) {
      const int nt = (rem + TT - 1) / TT;
      const int ntiles = nt * (nt + 1) / 2;
      const int tx = tid % 16, ty = tid / 16;
      for (int tile = rank; tile < ntiles; tile += NC) {
        int ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
        const int tj = tile - ti * (ti + 1) / 2;
        const int rb = c0 + ti * TT, cb = c0 + tj * TT;
        {
          constexpr int NQ = TT * NB / FT;  // every load of the two tiles in flight together
          T a[NQ], b[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int i = tid + q * FT, rr = i % TT, t = i / TT;
            a[q] = (t < nb && rb + rr < m) ? F[(size_t)(rb + rr) + (size_t)(kb + t) * m] : T(0);
            b[q] = (t < nb && cb + rr < m) ? F[(size_t)(cb + rr) + (size_t)(kb + t) * m] : T(0);
          }
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int i = tid + q * FT, rr = i % TT, t = i / TT;
            sm.Lr[rr][t] = a[q];
            sm.Lc[rr][t] = b[q];
          }
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
        // read-modify-write of the 16 entries: every read issued before the first write (the
        // compiler cannot reorder loads past stores into the same array by itself)
        T cur[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = rb + tx + 16 * i, c = cb + ty + 16 * j;
            cur[i][j] = (r < m && c < m && r >= c) ? F[(size_t)r + (size_t)c * m] : T(0);
          }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = rb + tx + 16 * i, c = cb + ty + 16 * j;
            if (r < m && c < m && r >= c) F[(size_t)r + (size_t)c * m] = cur[i][j] - acc[i][j];
          }
        __syncthreads();
      }
    }
    front_sync<NC>();
  }
}

// X = [I; L21] inv(L11) written to the panel P (leading dimension ld): solved from the right,
// X L11 = [I; L21], one 32-column block at a time from the last to the first. Row tiles of 64
// rows go to CTA (tile % NC); a tile's earlier columns were computed by the same CTA.
template <typename T, int NC>
__device__ void inverse_panel(const T *F, T *P, int m, int w, FactorSmem<T> &sm) {
  const int tid = threadIdx.x;
  const int rank = front_rank<NC>();
  const int ld = (m + 3) & ~3;
  const int ntile = (m + TT - 1) / TT;
  // zero the strict upper triangle of the top block and the pad rows (tiles of this CTA)
  for (int t = rank; t < ntile; t += NC)
    for (int i = tid; i < TT * w; i += FT) {
      const int r = t * TT + i % TT, c = i / TT;
      if ((r < w && r < c) || (r >= m && r < ld)) P[(size_t)r + (size_t)c * ld] = T(0);
    }
  __syncthreads();
  // thread layout of a 64 x 32 accumulator tile: 2 rows x 4 columns per thread
  const int tr = tid / 8, tc = tid % 8;  // rows tr + 32 q, columns tc + 8 p
  const int nblk = (w + NB - 1) / NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int jb = bi * NB;
    const int nb = min(NB, w - jb);
    __syncthreads();
    stage_diag(F, m, jb, nb, sm);
    __syncthreads();
    const int tfirst = jb / TT;  // rows < jb of these columns are zero (upper triangle)
    for (int t = tfirst; t < ntile; ++t) {
      if (t % NC != rank) continue;
      const int r0 = t * TT;
      T acc[2][4];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int r = r0 + tr + 32 * q, c = tc + 8 * p;
          T v = T(0);
          if (r < m && c < nb) v = (r < w) ? T(r == jb + c ? 1 : 0) : F[(size_t)r + (size_t)(jb + c) * m];
          acc[q][p] = v;
        }
      // acc -= X[rows, cc] L11[cc, jb block] for the already computed columns cc >= jb + nb
      for (int cc = jb + nb; cc < w; cc += NB) {
        const int cn = min(NB, w - cc);
        __syncthreads();
        {
          constexpr int NQ = TT * NB / FT, NQ2 = NB * NB / FT;
          T a[NQ], b[NQ2];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int i = tid + q * FT, rr = i % TT, k = i / TT, r = r0 + rr;
            a[q] = (k < cn && r < m) ? P[(size_t)r + (size_t)(cc + k) * ld] : T(0);
          }
#pragma unroll
          for (int q = 0; q < NQ2; ++q) {
            const int i = tid + q * FT, k = i % NB, c = i / NB;
            b[q] = (k < cn && c < nb) ? F[(size_t)(cc + k) + (size_t)(jb + c) * m] : T(0);
          }
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int i = tid + q * FT;
            sm.Lr[i % TT][i / TT] = a[q];
          }
#pragma unroll
          for (int q = 0; q < NQ2; ++q) {
            const int i = tid + q * FT;
            sm.Lc[i % NB][i / NB] = b[q];
          }
        }
        __syncthreads();
        for (int k = 0; k < cn; ++k) {
          T a[2], b[4];
#pragma unroll
          for (int q = 0; q < 2; ++q) a[q] = sm.Lr[tr + 32 * q][k];
#pragma unroll
          for (int p = 0; p < 4; ++p) b[p] = sm.Lc[k][tc + 8 * p];
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] -= a[q] * b[p];
        }
      }
      // x Ld = acc for each row: stage in Lr, one thread per row solves from the right
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) sm.Lr[tr + 32 * q][tc + 8 * p] = acc[q][p];
      __syncthreads();
      if (tid < TT && r0 + tid < m) {
        T x[NB];
#pragma unroll
        for (int c = NB - 1; c >= 0; --c) {
          x[c] = T(0);
          if (c < nb) {
            T v = sm.Lr[tid][c];
#pragma unroll
            for (int u = 0; u < NB; ++u)
              if (u > c && u < nb) v -= x[u] * sm.D[u][c];
            x[c] = v / sm.D[c][c];
          }
        }
        const int r = r0 + tid;
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nb && !(r < w && r < jb + c)) P[(size_t)r + (size_t)(jb + c) * ld] = x[c];
      }
      __syncthreads();
    }
  }
}

template <typename T, int NC>
__device__ void factor_front(const ForestDev &f, int J, const double *Aval, T *front, T *panel,
                             DevStatus *st, FactorSmem<T> &sm) {
  const int w = f.sn_w[J], m = f.sn_m[J];
  T *F = front + f.sn_front[J];
  const int tid = threadIdx.x;
  const int rank = front_rank<NC>();
  const int gt = rank * FT + tid;
  for (size_t i = gt; i < (size_t)m * m; i += NC * FT) F[i] = T(0);
  front_sync<NC>();
  {  // A's entries of J's columns, four per thread in flight
    const int64_t a0 = f.asm_ptr[J], a1 = f.asm_ptr[J + 1];
    for (int64_t e = a0 + gt; e < a1; e += 4 * NC * FT) {
      int64_t dst[4];
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t ee = e + (int64_t)u * NC * FT;
        dst[u] = ee < a1 ? f.asm_dst[ee] : -1;
        v[u] = ee < a1 ? Aval[f.asm_src[ee]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) F[dst[u]] = (T)v[u];
    }
  }
  for (int ci = f.ch_ptr[J]; ci < f.ch_ptr[J + 1]; ++ci) {
    front_sync<NC>();
    const int C = f.ch_list[ci];
    const int wc = f.sn_w[C], mc = f.sn_m[C], mu = mc - wc;
    const T *FC = front + f.sn_front[C];
    const int32_t *rm = f.relmap + f.sn_upd[C];
    for (int idx0 = gt; idx0 < mu * mu; idx0 += 4 * NC * FT) {  // four entries in flight
      int64_t dst[4];
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = idx0 + u * NC * FT;
        const int a = idx % mu, b = idx / mu;
        const bool on = idx < mu * mu && a >= b;
        dst[u] = on ? (int64_t)rm[a] + (int64_t)rm[b] * m : -1;
        v[u] = on ? FC[(size_t)(wc + a) + (size_t)(wc + b) * mc] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (dst[u] >= 0) F[dst[u]] += v[u];
    }
  }
  front_sync<NC>();
  partial_cholesky<T, NC>(F, m, w, f.sn_block[J], st, sm);
  inverse_panel<T, NC>(F, panel + f.sn_panel[J], m, w, sm);
}

template <typename T>
__global__ void __launch_bounds__(FT, FactorOcc<T>::value) k_factor(ForestDev f, const int32_t *level_sn,
                                               const double *Aval, T *front, T *panel,
                                               DevStatus *st) {
  __shared__ FactorSmem<T> sm;
  factor_front<T, 1>(f, level_sn[blockIdx.x], Aval, front, panel, st, sm);
}

constexpr int CLUSTER = 8;

template <typename T>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(FT, FactorOcc<T>::value)
    k_factor_cluster(ForestDev f, const int32_t *level_sn, const double *Aval, T *front,
                     T *panel, DevStatus *st) {
  __shared__ FactorSmem<T> sm;
  factor_front<T, CLUSTER>(f, level_sn[blockIdx.x / CLUSTER], Aval, front, panel, st, sm);
}

// Levels with few large fronts (the top of the A_G tree): clusters of 16 CTAs (a size the
// hardware allows only on request), with a dynamic shared-memory request that leaves room for
// one CTA per SM, so that each front gets twice the SMs of an 8-CTA cluster.
constexpr int CLUSTER_BIG = 16;
constexpr size_t kBigFrontPad = 120 * 1024;   // dynamic shared memory, unused: one CTA per SM

template <typename T>
__global__ void __launch_bounds__(FT, 1)
    k_factor_cluster16(ForestDev f, const int32_t *level_sn, const double *Aval, T *front,
                       T *panel, DevStatus *st) {
  __shared__ FactorSmem<T> sm;
  factor_front<T, CLUSTER_BIG>(f, level_sn[blockIdx.x / CLUSTER_BIG], Aval, front, panel, st, sm);
}

// whether a 16-CTA cluster of k_factor_cluster16 can be resident on this device
template <typename T>
bool big_clusters_ok() {
  static int ok = -1;
  if (ok >= 0) return ok == 1;
  ok = 0;
  if (cudaFuncSetAttribute(k_factor_cluster16<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess ||
      cudaFuncSetAttribute(k_factor_cluster16<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBigFrontPad) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CLUSTER_BIG, 1, 1);
  cfg.blockDim = dim3(FT, 1, 1);
  cfg.dynamicSmemBytes = kBigFrontPad;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = CLUSTER_BIG;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_factor_cluster16<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ok = clusters >= 1 ? 1 : 0;
  return ok == 1;
}

}  // namespace

int factor_cluster_size() { return CLUSTER; }

template <typename T>
bool factor_big_clusters_available() {
  return big_clusters_ok<T>();
}

template <typename T>
void launch_factor_level(const ForestDev &f, const int32_t *level_sn, int count,
                         const double *Aval, T *front, T *panel, DevStatus *st,
                         cudaStream_t stream, int mode) {
  if (count <= 0) return;
  if (mode == 2 && big_clusters_ok<T>()) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * CLUSTER_BIG, 1, 1);
    cfg.blockDim = dim3(FT, 1, 1);
    cfg.dynamicSmemBytes = kBigFrontPad;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = CLUSTER_BIG;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    NSP_CUDA(cudaLaunchKernelEx(&cfg, k_factor_cluster16<T>, f, level_sn, Aval, front, panel, st));
  } else if (mode >= 1) {
    k_factor_cluster<T><<<count * CLUSTER, FT, 0, stream>>>(f, level_sn, Aval, front, panel, st);
  } else {
    k_factor<T><<<count, FT, 0, stream>>>(f, level_sn, Aval, front, panel, st);
  }
  NSP_LAUNCH_CHECK();
}

template bool factor_big_clusters_available<float>();
template bool factor_big_clusters_available<double>();
template void launch_factor_level<float>(const ForestDev &, const int32_t *, int, const double *,
                                         float *, float *, DevStatus *, cudaStream_t, int);
template void launch_factor_level<double>(const ForestDev &, const int32_t *, int, const double *,
                                          double *, double *, DevStatus *, cudaStream_t, int);

}  // namespace nsp
