// Supernodal triangular solves with s right-hand sides: X = A_b^{-1} B for every block b
// of a forest at once (the A_I^{-1} inside S_Gamma, §2.3 eq. (schur_complement), and
// A_G^{-1}, the first-level preconditioner S1 of eq. (S1)).
//
// With the panel P_J = [inv(L11); L21 inv(L11)] of each supernode J:
//   forward  (L y = b):  y_J = P_top f_top,  u_J = f_bot - P_bot f_top,
//     f = b on J's columns plus the children's update rows u_C (extend-add gather);
//   backward (L^T x = y): x_J = P_top^T y_J - P_bot^T x[rows of J below its columns].
// Each work item is one tile of rows of one supernode; items of one tree level run in one
// launch. The tile is a dense (TM x K) * (K x s) product on CUDA cores, K staged in chunks
// of TK through shared memory.
#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int ST = 256;  // threads
constexpr int TK = 32;   // K chunk

template <int TC, int CM, int RM>
struct Cfg {
  static constexpr int TR = ST / TC;
  static constexpr int TM = TR * RM;
  static constexpr int NCP = TC * CM;
};

template <typename T, int TC, int CM, int RM>
__global__ void __launch_bounds__(ST) k_fwd(ForestDev f, const TileItem *items,
                                            const T *__restrict__ panel,
                                            const T *__restrict__ B, T *__restrict__ Y,
                                            T *__restrict__ U, int s) {
  using C = Cfg<TC, CM, RM>;
  constexpr int TM = C::TM, NCP = C::NCP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *As = reinterpret_cast<T *>(smem_raw);  // [TK][TM + 1]
  T *Bs = As + TK * (TM + 1);               // [TK][NCP]
  const TileItem it = items[blockIdx.x];
  const int J = it.sn, r0 = it.r0;
  const int w = f.sn_w[J], m = f.sn_m[J];
  const int first = f.sn_first[J];
  const int64_t rp = f.sn_rowptr[J];
  const T *P = panel + f.sn_panel[J];
  const int r1 = min(r0 + TM, m);
  const int kmax = (r1 <= w) ? r1 : w;  // inv(L11) is lower triangular
  const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
  T acc[RM][CM];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < kmax; k0 += TK) {
    for (int i = tid; i < TK * TM; i += ST) {
      const int r = i % TM, k = i / TM;
      T v = T(0);
      if (r0 + r < m && k0 + k < kmax) v = P[(size_t)(r0 + r) + (size_t)(k0 + k) * m];
      As[k * (TM + 1) + r] = v;
    }
    for (int i = tid; i < TK * NCP; i += ST) {
      const int c = i % NCP, k = i / NCP;
      const int kk = k0 + k;
      T v = T(0);
      if (kk < kmax && c < s) {
        if (B) v = B[(size_t)(first + kk) * s + c];
        for (int64_t e = f.gptr[rp + kk]; e < f.gptr[rp + kk + 1]; ++e)
          v += U[(size_t)f.gsrc[e] * s + c];
      }
      Bs[k * NCP + c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      T a[RM], b[CM];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = As[k * (TM + 1) + tr * RM + i];
#pragma unroll
      for (int j = 0; j < CM; ++j) b[j] = Bs[k * NCP + tc + TC * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CM; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  const int64_t upd = f.sn_upd[J];
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + tr * RM + i;
    if (r >= r1) continue;
    if (r < w) {
#pragma unroll
      for (int j = 0; j < CM; ++j) {
        const int c = tc + TC * j;
        if (c < s) Y[(size_t)(first + r) * s + c] = acc[i][j];
      }
    } else {
      const int64_t g0 = f.gptr[rp + r], g1 = f.gptr[rp + r + 1];
#pragma unroll
      for (int j = 0; j < CM; ++j) {
        const int c = tc + TC * j;
        if (c < s) {
          T v = -acc[i][j];
          for (int64_t e = g0; e < g1; ++e) v += U[(size_t)f.gsrc[e] * s + c];
          U[(size_t)(upd + r - w) * s + c] = v;
        }
      }
    }
  }
}

template <typename T, int TC, int CM, int RM>
__global__ void __launch_bounds__(ST) k_bwd(ForestDev f, const TileItem *items,
                                            const T *__restrict__ panel,
                                            const T *__restrict__ Y, T *__restrict__ X,
                                            int s) {
  using C = Cfg<TC, CM, RM>;
  constexpr int TM = C::TM, NCP = C::NCP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *As = reinterpret_cast<T *>(smem_raw);  // [TK][TM + 1]
  T *Bs = As + TK * (TM + 1);               // [TK][NCP]
  const TileItem it = items[blockIdx.x];
  const int J = it.sn, r0 = it.r0;
  const int w = f.sn_w[J], m = f.sn_m[J];
  const int first = f.sn_first[J];
  const int64_t rp = f.sn_rowptr[J];
  const T *P = panel + f.sn_panel[J];
  const int r1 = min(r0 + TM, w);
  const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
  T acc[RM][CM];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[i][j] = T(0);

  for (int k0 = r0; k0 < m; k0 += TK) {
    for (int i = tid; i < TK * TM; i += ST) {
      const int k = i % TK, r = i / TK;
      T v = T(0);
      if (r0 + r < r1 && k0 + k < m) v = P[(size_t)(k0 + k) + (size_t)(r0 + r) * m];
      As[k * (TM + 1) + r] = v;
    }
    for (int i = tid; i < TK * NCP; i += ST) {
      const int c = i % NCP, k = i / NCP;
      const int kk = k0 + k;
      T v = T(0);
      if (kk < m && c < s) {
        if (kk < w) v = Y[(size_t)(first + kk) * s + c];
        else v = -X[(size_t)f.rows[rp + kk] * s + c];
      }
      Bs[k * NCP + c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TK; ++k) {
      T a[RM], b[CM];
#pragma unroll
      for (int i = 0; i < RM; ++i) a[i] = As[k * (TM + 1) + tr * RM + i];
#pragma unroll
      for (int j = 0; j < CM; ++j) b[j] = Bs[k * NCP + tc + TC * j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CM; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + tr * RM + i;
    if (r >= r1) continue;
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      const int c = tc + TC * j;
      if (c < s) X[(size_t)(first + r) * s + c] = acc[i][j];
    }
  }
}

template <typename T, int TC, int CM, int RM>
size_t smem_bytes() {
  using C = Cfg<TC, CM, RM>;
  return sizeof(T) * (size_t)(TK * (C::TM + 1) + TK * C::NCP);
}

template <typename T, int TC, int CM, int RM>
void run_fwd(const ForestDev &f, const TileItem *items, int n, const T *panel, const T *B,
             T *Y, T *U, int s, cudaStream_t st) {
  const size_t sm = smem_bytes<T, TC, CM, RM>();
  static bool attr = false;
  if (!attr) {
    NSP_CUDA(cudaFuncSetAttribute(k_fwd<T, TC, CM, RM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  k_fwd<T, TC, CM, RM><<<n, ST, sm, st>>>(f, items, panel, B, Y, U, s);
  NSP_LAUNCH_CHECK();
}

template <typename T, int TC, int CM, int RM>
void run_bwd(const ForestDev &f, const TileItem *items, int n, const T *panel, const T *Y,
             T *X, int s, cudaStream_t st) {
  const size_t sm = smem_bytes<T, TC, CM, RM>();
  static bool attr = false;
  if (!attr) {
    NSP_CUDA(cudaFuncSetAttribute(k_bwd<T, TC, CM, RM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  k_bwd<T, TC, CM, RM><<<n, ST, sm, st>>>(f, items, panel, Y, X, s);
  NSP_LAUNCH_CHECK();
}

// Column configurations: s == 1 (vector), else 16 threads across columns with CM columns
// each and 4 rows per thread (64-row tiles).
#define NSP_SOLVE_DISPATCH(FN, ...)                                  \
  do {                                                               \
    if (s == 1) FN<T, 1, 1, 1>(__VA_ARGS__);                         \
    else if (s <= 16) FN<T, 16, 1, 4>(__VA_ARGS__);                  \
    else if (s <= 32) FN<T, 16, 2, 4>(__VA_ARGS__);                  \
    else if (s <= 48) FN<T, 16, 3, 4>(__VA_ARGS__);                  \
    else if (s <= 64) FN<T, 16, 4, 4>(__VA_ARGS__);                  \
    else if (s <= 80) FN<T, 16, 5, 4>(__VA_ARGS__);                  \
    else if (s <= 96) FN<T, 16, 6, 4>(__VA_ARGS__);                  \
    else if (s <= 128) FN<T, 16, 8, 4>(__VA_ARGS__);                 \
    else if (s <= 160) FN<T, 16, 10, 4>(__VA_ARGS__);                \
    else if (s <= 256) FN<T, 16, 16, 4>(__VA_ARGS__);                \
    else throw Error(NSP_ERR_UNSUPPORTED, "more than 256 right-hand sides"); \
  } while (0)

}  // namespace

int solve_tile_rows(int s) { return s == 1 ? ST : 64; }

template <typename T>
void launch_solve_fwd(const ForestDev &f, const TileItem *items, int nitems, int tm,
                      const T *panel, const T *B, T *Y, T *U, int s, cudaStream_t stream) {
  if (nitems <= 0) return;
  require(tm == solve_tile_rows(s), NSP_ERR_INVALID_ARG, "tile height mismatch");
  NSP_SOLVE_DISPATCH(run_fwd, f, items, nitems, panel, B, Y, U, s, stream);
}

template <typename T>
void launch_solve_bwd(const ForestDev &f, const TileItem *items, int nitems, int tm,
                      const T *panel, const T *Y, T *X, int s, cudaStream_t stream) {
  if (nitems <= 0) return;
  require(tm == solve_tile_rows(s), NSP_ERR_INVALID_ARG, "tile height mismatch");
  NSP_SOLVE_DISPATCH(run_bwd, f, items, nitems, panel, Y, X, s, stream);
}

template void launch_solve_fwd<float>(const ForestDev &, const TileItem *, int, int,
                                      const float *, const float *, float *, float *, int,
                                      cudaStream_t);
template void launch_solve_fwd<double>(const ForestDev &, const TileItem *, int, int,
                                       const double *, const double *, double *, double *,
                                       int, cudaStream_t);
template void launch_solve_bwd<float>(const ForestDev &, const TileItem *, int, int,
                                      const float *, const float *, float *, int,
                                      cudaStream_t);
template void launch_solve_bwd<double>(const ForestDev &, const TileItem *, int, int,
                                       const double *, const double *, double *, int,
                                       cudaStream_t);

}  // namespace nsp
