// BLAS-like kernels of the hot path: CSR x dense-block SpMM (A_IG, A_GI, A_G), row
// gathers/scatters between the caller's and the factor's orderings, block-CG Gram products
// X^T Y, tall-skinny block updates, column norms, the Philox sketch generator and the FP64
// vector kernels of the outer PCG.
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int BT = 256;

// ---------------------------------------------------------------- SpMM
// Y[i, :] = alpha * sum_e val[e] X[col[e], :] + beta * C[i, :]. A group of L lanes per row
// (L = power of two >= s, at most 32) walks the row's entries; lanes cover the s columns.
template <typename T>
__global__ void __launch_bounds__(BT) k_spmm(CsrDev<T> A, const T *__restrict__ X,
                                             T *Y, int s, int lanes, T alpha, const T *C,
                                             T beta) {
  const int rows_per_block = BT / lanes;
  const int lane = threadIdx.x % lanes;
  const int64_t i = (int64_t)blockIdx.x * rows_per_block + threadIdx.x / lanes;
  if (i >= A.nrows) return;
  const int e0 = A.rowptr[i], e1 = A.rowptr[i + 1];
  for (int c = lane; c < s; c += lanes) {
    T acc = T(0);
    for (int e = e0; e < e1; ++e) acc += A.val[e] * X[(size_t)A.col[e] * s + c];
    T out = alpha * acc;
    if (C) out += beta * C[(size_t)i * s + c];
    Y[(size_t)i * s + c] = out;
  }
}

template <typename Ti, typename To>
__global__ void k_gather_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrows * s) return;
  const int64_t i = idx / s;
  const int c = (int)(idx % s);
  const int64_t src = perm ? perm[i] : i;
  out[idx] = (To)in[(size_t)src * s + c];
}

template <typename Ti, typename To>
__global__ void k_scatter_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrows * s) return;
  const int64_t i = idx / s;
  const int c = (int)(idx % s);
  const int64_t dst = perm ? perm[i] : i;
  out[(size_t)dst * s + c] = (To)in[idx];
}

template <typename T>
__global__ void k_gather_values(const int64_t *src, int64_t count, const double *Aval, T *out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (T)Aval[src[e]];
}

// ---------------------------------------------------------------- Gram X^T Y
// Stage 1: CTA (chunk, ta, tb) sums rows [chunk*rpc, ...) for a (16 RT) x (16 RT) output
// tile (ta, tb); each thread owns RT x RT outputs; rows are staged GR at a time. Stage 2
// adds the chunk partials in chunk order (deterministic).
constexpr int GR = 16;

template <typename T, typename AccT, int RT>
__global__ void __launch_bounds__(BT) k_gram_partial(const T *__restrict__ X,
                                                     const T *__restrict__ Y, int64_t n,
                                                     int s1, int s2, int64_t rpc,
                                                     double *work) {
  constexpr int TS = 16 * RT;
  __shared__ T Xs[GR][TS];
  __shared__ T Ys[GR][TS];
  const int chunk = blockIdx.x;
  const int a0 = blockIdx.y * TS, b0 = blockIdx.z * TS;
  const int64_t i0 = (int64_t)chunk * rpc;
  const int64_t i1 = min(n, i0 + rpc);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  AccT acc[RT][RT];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[i][j] = AccT(0);
  static_assert((GR * TS) % BT == 0, "staging tile must split evenly over the threads");
  constexpr int NQ = GR * TS / BT;
  for (int64_t ib = i0; ib < i1; ib += GR) {
    T xv[NQ], yv[NQ];  // every load of the two tiles in flight before the shared stores
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = tid + u * BT, r = q / TS, c = q % TS;
      const int64_t row = ib + r;
      xv[u] = (row < i1 && a0 + c < s1) ? X[(size_t)row * s1 + a0 + c] : T(0);
      yv[u] = (row < i1 && b0 + c < s2) ? Y[(size_t)row * s2 + b0 + c] : T(0);
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = tid + u * BT;
      Xs[q / TS][q % TS] = xv[u];
      Ys[q / TS][q % TS] = yv[u];
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < GR; ++r) {
      AccT xa[RT], yb[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) xa[i] = (AccT)Xs[r][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RT; ++j) yb[j] = (AccT)Ys[r][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) acc[i][j] += xa[i] * yb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < s1 && b < s2) work[((size_t)chunk * s1 + a) * s2 + b] = (double)acc[i][j];
    }
}

// Gram of FP32 data with twice-working-precision accuracy on the FP32 pipes (the s x s Grams
// of the Nyström core, K = Y^T Y and C = G^T Y, whose Cholesky-QR needs more than FP32 sums):
// compensated dot products, Algorithm Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005). Each product x y = p + e exactly (p = fl(x y),
// e = fma(x, y, -p), Dekker / Veltkamp TwoProduct); the running sum s and the error term c
// follow Knuth's TwoSum: t = s + p, z = t - s, c += ((s - (t - z)) + (p - z)) + e, s = t. The
// chunk partial s + c is stored in FP64 and the chunks are added in FP64 in chunk order. The
// _rn intrinsics keep the compiler from contracting the products into the sums.
template <int RT>
__global__ void __launch_bounds__(BT) k_gram_dot2(const float *__restrict__ X,
                                                  const float *__restrict__ Y, int64_t n,
                                                  int s1, int s2, int64_t rpc, double *work) {
  constexpr int TS = 16 * RT;
  __shared__ float Xs[GR][TS];
  __shared__ float Ys[GR][TS];
  const int chunk = blockIdx.x;
  const int a0 = blockIdx.y * TS, b0 = blockIdx.z * TS;
  const int64_t i0 = (int64_t)chunk * rpc;
  const int64_t i1 = min(n, i0 + rpc);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float sh[RT][RT], sc[RT][RT];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) sh[i][j] = sc[i][j] = 0.f;
  constexpr int NQ = GR * TS / BT;
  for (int64_t ib = i0; ib < i1; ib += GR) {
    float xv[NQ], yv[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = tid + u * BT, r = q / TS, c = q % TS;
      const int64_t row = ib + r;
      xv[u] = (row < i1 && a0 + c < s1) ? X[(size_t)row * s1 + a0 + c] : 0.f;
      yv[u] = (row < i1 && b0 + c < s2) ? Y[(size_t)row * s2 + b0 + c] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = tid + u * BT;
      Xs[q / TS][q % TS] = xv[u];
      Ys[q / TS][q % TS] = yv[u];
    }
    __syncthreads();
#pragma unroll 2
    for (int r = 0; r < GR; ++r) {
      float xa[RT], yb[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) xa[i] = Xs[r][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RT; ++j) yb[j] = Ys[r][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < RT; ++j) {
          const float p = __fmul_rn(xa[i], yb[j]);
          const float e = __fmaf_rn(xa[i], yb[j], -p);
          const float t = __fadd_rn(sh[i][j], p);
          const float z = __fsub_rn(t, sh[i][j]);
          const float err = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));
          sc[i][j] = __fadd_rn(sc[i][j], __fadd_rn(err, e));
          sh[i][j] = t;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < s1 && b < s2)
        work[((size_t)chunk * s1 + a) * s2 + b] = (double)sh[i][j] + (double)sc[i][j];
    }
}

// C[e] = sum over chunks of work[chunk * entries + e]. A CTA of BT threads serves RE = 32
// consecutive entries with RL = BT / 32 lanes each: lane l sums the chunks l, l + RL, ... in
// increasing order (eight loads in flight), then lane 0 adds the RL lane sums in lane order,
// so the result is deterministic. Splitting the chunks over lanes puts RL times more CTAs
// and RL times fewer dependent load passes per thread on the reduction than one thread per
// entry (the s x s Gram reduction sums 304 partials per entry over 6,400 entries).
constexpr int RE = 32, RL = BT / RE;
__global__ void __launch_bounds__(BT) k_gram_reduce(const double *work, int nchunks,
                                                    int64_t entries, double *C) {
  __shared__ double red[RL][RE + 1];
  const int tx = threadIdx.x % RE, ty = threadIdx.x / RE;
  const int64_t e = (int64_t)blockIdx.x * RE + tx;
  double acc = 0.0;
  if (e < entries) {
    int c = ty;
    for (; c + 7 * RL < nchunks; c += 8 * RL) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = work[(size_t)(c + u * RL) * entries + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; c < nchunks; c += RL) acc += work[(size_t)c * entries + e];
  }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && e < entries) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < RL; ++q) t += red[q][tx];
    C[e] = t;
  }
}

inline int reduce_grid(int64_t entries) { return (int)((entries + RE - 1) / RE); }

int gram_rt(int s1, int s2) {
  const int smax = std::max(s1, s2);
  return smax <= 32 ? 2 : smax <= 64 ? 4 : smax <= 96 ? 6 : 8;
}

int gram_chunks(int64_t n, int s1, int s2) {
  const int ts = 16 * gram_rt(s1, s2);
  const int tiles = ceil_div(s1, ts) * ceil_div(s2, ts);
  int target = std::max(1, 2 * 152 / tiles);
  int maxc = (int)std::max<int64_t>(1, (n + 4 * GR - 1) / (4 * GR));
  return std::max(1, std::min(target, maxc));
}

// ---------------------------------------------------------------- FP64 GEMV with a tall Z
// t = Z^T r (Z n x k row-major): partials per row chunk, then an ordered sum.
// A CTA owns a chunk of rows; per 32-column group, lane ty of 8 takes rows i0+ty, i0+ty+8, ...
// with four rows (four loads of Z and r) in flight per loop pass into four running sums, added
// in a fixed order, so every partial is deterministic for a given n and chunk count.
__global__ void __launch_bounds__(BT) k_gemv_t_partial(const double *Z, int64_t n, int k,
                                                       const double *r, int64_t rpc,
                                                       double *work) {
  __shared__ double red[8][33];
  const int64_t i0 = (int64_t)blockIdx.x * rpc, i1 = min(n, i0 + rpc);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int c0 = 0; c0 < k; c0 += 32) {
    const int c = c0 + tx;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (c < k) {
      int64_t i = i0 + ty;
      for (; i + 24 < i1; i += 32) {
        const double z0 = Z[(size_t)i * k + c], z1 = Z[(size_t)(i + 8) * k + c];
        const double z2 = Z[(size_t)(i + 16) * k + c], z3 = Z[(size_t)(i + 24) * k + c];
        const double r0 = r[i], r1 = r[i + 8], r2 = r[i + 16], r3 = r[i + 24];
        a0 += z0 * r0;
        a1 += z1 * r1;
        a2 += z2 * r2;
        a3 += z3 * r3;
      }
      for (; i < i1; i += 8) a0 += Z[(size_t)i * k + c] * r[i];
    }
    red[ty][tx] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (ty == 0 && c < k) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += red[q][tx];
      work[(size_t)blockIdx.x * k + c] = t;
    }
    __syncthreads();
  }
}

// row chunks of the FP64 GEMV: about 64 rows each, at most four CTAs per SM of a 152-SM part
int64_t gemv_chunks(int64_t n) {
  return std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + 63) / 64));
}

// z[i] = beta z[i] + sum_j Z[i, j] t[j]: eight lanes per row (four rows per warp), each lane
// taking columns l, l + 8, ... so that the eight lanes of a row read it contiguously.
constexpr int GN = 8;
__global__ void __launch_bounds__(BT) k_gemv_n(const double *Z, int64_t n, int k,
                                               const double *t, double beta, double *z) {
  const int64_t i = ((int64_t)blockIdx.x * BT + threadIdx.x) / GN;
  const int l = threadIdx.x % GN;
  double acc = 0.0;
  if (i < n) {
#pragma unroll 4
    for (int j = l; j < k; j += GN) acc += Z[(size_t)i * k + j] * t[j];
  }
#pragma unroll
  for (int o = GN / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (l == 0 && i < n) z[i] = beta * z[i] + acc;
}

// ---------------------------------------------------------------- block update
// Out = A M + beta C, A n x s1 (T), M s1 x s2 (FP64), 32 rows per CTA, s1 in chunks of 32.
constexpr int UR = 32, UK = 32;

template <typename T>
__global__ void __launch_bounds__(BT) k_block_update(const T *__restrict__ A,
                                                     const double *__restrict__ M, int64_t n,
                                                     int s1, int s2, T scale, const T *C,
                                                     T beta, T *Out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *As = reinterpret_cast<T *>(smem_raw);  // [UR][UK + 1]
  T *Ms = As + UR * (UK + 1);               // [UK][s2]
  const int64_t i0 = (int64_t)blockIdx.x * UR;
  const int tid = threadIdx.x, tx = tid % 32, ty = tid / 32;  // 8 row groups x 32 lanes
  constexpr int MAXJ = 8;                                     // s2 <= 256
  T acc[4][MAXJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) acc[i][j] = T(0);
  for (int kc = 0; kc < s1; kc += UK) {
    {  // loads of the A tile in flight together, then the M rows four at a time
      constexpr int NQ = UR * UK / BT;
      T av[NQ];
#pragma unroll
      for (int u = 0; u < NQ; ++u) {
        const int q = tid + u * BT, r = q / UK, k = q % UK;
        av[u] = (i0 + r < n && kc + k < s1) ? A[(size_t)(i0 + r) * s1 + kc + k] : T(0);
      }
#pragma unroll
      for (int u = 0; u < NQ; ++u) {
        const int q = tid + u * BT;
        As[(q / UK) * (UK + 1) + q % UK] = av[u];
      }
    }
    for (int q0 = tid; q0 < UK * s2; q0 += 4 * BT) {
      T mv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * BT, k = q / s2, c = q % s2;
        mv[u] = (q < UK * s2 && kc + k < s1) ? (T)M[(size_t)(kc + k) * s2 + c] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q0 + u * BT < UK * s2) Ms[q0 + u * BT] = mv[u];
    }
    __syncthreads();
    for (int k = 0; k < UK; ++k) {
      T a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[(ty + 8 * i) * (UK + 1) + k];
#pragma unroll
      for (int j = 0; j < MAXJ; ++j) {
        const int c = tx + 32 * j;
        if (c < s2) {
          const T mv = Ms[k * s2 + c];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][j] += a[i] * mv;
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = i0 + ty + 8 * i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int c = tx + 32 * j;
      if (c < s2) {
        T v = scale * acc[i][j];
        if (C) v += beta * C[(size_t)row * s2 + c];
        Out[(size_t)row * s2 + c] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- column sums of squares
template <typename T>
__global__ void __launch_bounds__(BT) k_colsq_partial(const T *X, int64_t n, int s, int64_t rpc,
                                                      double *work) {
  __shared__ double red[8][33];
  const int64_t i0 = (int64_t)blockIdx.x * rpc, i1 = min(n, i0 + rpc);
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int c0 = 0; c0 < s; c0 += 32) {
    const int c = c0 + tx;
    double acc = 0.0;
    if (c < s)
      for (int64_t i = i0 + ty; i < i1; i += 8) {
        const double v = (double)X[(size_t)i * s + c];
        acc += v * v;
      }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && c < s) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += red[q][tx];
      work[(size_t)blockIdx.x * s + c] = t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// 10 rounds of (two 32x32->64 multiplies, xor with key and swapped halves), Weyl key bumps.
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                             uint32_t &c3, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
  c0 = n0; c1 = n1; c2 = n2; c3 = n3;
}

__device__ void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(c0, c1, c2, c3, k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  ctr[0] = c0; ctr[1] = c1; ctr[2] = c2; ctr[3] = c3;
}

// Element i: counter (i/2 low word, i/2 high word, 0, 0), key = seed; uniforms
// u1 = (x0 + 0.5) 2^-32, u2 = (x1 + 0.5) 2^-32; Box-Muller radius sqrt(-2 ln u1), angle
// 2 pi u2; even i takes the cosine, odd i the sine.
template <typename T>
__global__ void k_gaussian(uint64_t seed, int64_t count, T *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint64_t q = (uint64_t)i >> 1;
  uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), 0u, 0u};
  philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)ctr[0] + 0.5) * 2.3283064365386963e-10;
  const double u2 = ((double)ctr[1] + 0.5) * 2.3283064365386963e-10;
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 6.283185307179586 * u2;
  out[i] = (T)((i & 1) ? rad * sin(ang) : rad * cos(ang));
}

// ---------------------------------------------------------------- FP64 vectors
__global__ void __launch_bounds__(BT) k_dot_partial(const double *x, const double *y, int64_t n,
                                                    int64_t rpc, double *work) {
  __shared__ double red[BT];
  const int64_t i0 = (int64_t)blockIdx.x * rpc, i1 = min(n, i0 + rpc);
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) acc += x[i] * y[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = BT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) work[blockIdx.x] = red[0];
}

__global__ void k_sum(const double *work, int count, double *out) {
  __shared__ double red[BT];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += BT) acc += work[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = BT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_axpby(int64_t n, const double *a_ptr, double a_sign, const double *x,
                        double b, double *y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = a_sign * (a_ptr ? *a_ptr : 1.0);
  y[i] = a * x[i] + b * y[i];
}

__global__ void k_scale_cols(double *X, int64_t n, int s, const double *scale, int take_sqrt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * s) return;
  const double f = scale[idx % s];
  X[idx] *= take_sqrt ? sqrt(f) : f;
}

// One PCG step after q = A p: alpha = rz / pq (block 0 records it), x += alpha p,
// r -= alpha q, and this chunk's partial sum of r.r; the same chunks, per-thread order and
// tree as k_dot_partial, the same roundings as two k_axpby launches and a dot.
__global__ void __launch_bounds__(BT) k_pcg_step(int64_t n, int64_t rpc, const double *rz,
                                                 const double *pq, double *alpha_out,
                                                 const double *p, const double *q, double *x,
                                                 double *r, double *work) {
  __shared__ double red[BT];
  const double a = *rz / *pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) *alpha_out = a;
  const int64_t i0 = (int64_t)blockIdx.x * rpc, i1 = min(n, i0 + rpc);
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    acc += ri * ri;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = BT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) work[blockIdx.x] = red[0];
}

// p = z + beta p with beta = rz_new / rz_old (block 0 records it); the roundings of
// p = beta p followed by p = z + p
__global__ void k_pcg_direction(int64_t n, const double *rz_new, const double *rz_old,
                                double *beta_out, const double *z, double *p) {
  const double b = *rz_new / *rz_old;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *beta_out = b;
  if (i >= n) return;
  p[i] = __dadd_rn(z[i], __dmul_rn(b, p[i]));
}

__global__ void k_pcg_scalars(const double *rz_new, const double *rz_old, const double *pq,
                              double *alpha, double *beta) {
  if (threadIdx.x != 0) return;
  if (pq && alpha) *alpha = *rz_new / *pq;
  if (rz_old && beta) *beta = *rz_new / *rz_old;
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_spmm(const CsrDev<T> &A, const T *X, T *Y, int s, T alpha, const T *C, T beta,
                 cudaStream_t stream) {
  if (A.nrows <= 0 || s <= 0) return;
  int lanes = 1;
  while (lanes < s && lanes < 32) lanes <<= 1;
  const int rpb = BT / lanes;
  k_spmm<T><<<ceil_div(A.nrows, rpb), BT, 0, stream>>>(A, X, Y, s, lanes, alpha, C, beta);
  NSP_LAUNCH_CHECK();
}

template <typename Ti, typename To>
void launch_gather_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s,
                        cudaStream_t stream) {
  const int64_t tot = nrows * s;
  if (tot <= 0) return;
  k_gather_rows<Ti, To><<<ceil_div(tot, BT), BT, 0, stream>>>(perm, nrows, in, out, s);
  NSP_LAUNCH_CHECK();
}

template <typename Ti, typename To>
void launch_scatter_rows(const int64_t *perm, int64_t nrows, const Ti *in, To *out, int s,
                         cudaStream_t stream) {
  const int64_t tot = nrows * s;
  if (tot <= 0) return;
  k_scatter_rows<Ti, To><<<ceil_div(tot, BT), BT, 0, stream>>>(perm, nrows, in, out, s);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_gather_values(const int64_t *src, int64_t count, const double *Aval, T *out,
                          cudaStream_t stream) {
  if (count <= 0) return;
  k_gather_values<T><<<ceil_div(count, BT), BT, 0, stream>>>(src, count, Aval, out);
  NSP_LAUNCH_CHECK();
}

size_t gram_work_size(int64_t n, int s1, int s2) {
  const int ch = std::max<int>(gram_chunks(n, s1, s2), (int)tc_gram_chunks(n));
  const size_t g = (size_t)ch * s1 * s2;
  const int64_t cs = std::max(gemv_chunks(n),
                              std::max<int64_t>(1, std::min<int64_t>(2 * 152, (n + 255) / 256)));
  const size_t c = (size_t)cs * std::max(s1, s2);
  return std::max<size_t>(std::max(g, c), 4 * 152 + 8);
}

template <typename T, typename AccT, int RT>
void gram_rt_launch(const T *X, const T *Y, int64_t n, int s1, int s2, double *C, double *work,
                    cudaStream_t stream) {
  const int ch = gram_chunks(n, s1, s2);
  const int64_t rpc = std::max<int64_t>(GR, ((n + ch - 1) / ch + GR - 1) / GR * GR);
  dim3 grid(ch, ceil_div(s1, 16 * RT), ceil_div(s2, 16 * RT));
  k_gram_partial<T, AccT, RT><<<grid, BT, 0, stream>>>(X, Y, n, s1, s2, rpc, work);
  NSP_LAUNCH_CHECK();
  const int64_t ent = (int64_t)s1 * s2;
  k_gram_reduce<<<reduce_grid(ent), BT, 0, stream>>>(work, ch, ent, C);
  NSP_LAUNCH_CHECK();
}

template <typename T, typename AccT>
void launch_gram(const T *X, const T *Y, int64_t n, int s1, int s2, double *C, double *work,
                 cudaStream_t stream) {
  if (s1 <= 0 || s2 <= 0) return;
  if constexpr (std::is_same<T, float>::value && std::is_same<AccT, double>::value) {
    // FP32 data, FP64-class sums: compensated FP32 (same chunk count as the plain kernel, so
    // the same partials buffer serves)
    constexpr int RT = 4, TS = 16 * RT;
    const int ch = gram_chunks(n, s1, s2);
    const int64_t rpc = std::max<int64_t>(GR, ((n + ch - 1) / ch + GR - 1) / GR * GR);
    dim3 grid(ch, ceil_div(s1, TS), ceil_div(s2, TS));
    k_gram_dot2<RT><<<grid, BT, 0, stream>>>(X, Y, n, s1, s2, rpc, work);
    NSP_LAUNCH_CHECK();
    const int64_t ent = (int64_t)s1 * s2;
    k_gram_reduce<<<reduce_grid(ent), BT, 0, stream>>>(work, ch, ent, C);
    NSP_LAUNCH_CHECK();
    return;
  }
  switch (gram_rt(s1, s2)) {
    case 2: gram_rt_launch<T, AccT, 2>(X, Y, n, s1, s2, C, work, stream); break;
    case 4: gram_rt_launch<T, AccT, 4>(X, Y, n, s1, s2, C, work, stream); break;
    case 6: gram_rt_launch<T, AccT, 6>(X, Y, n, s1, s2, C, work, stream); break;
    default: gram_rt_launch<T, AccT, 8>(X, Y, n, s1, s2, C, work, stream); break;
  }
}

void launch_gram_reduce(const double *work, int nchunks, int64_t entries, double *C,
                        cudaStream_t stream) {
  if (entries <= 0) return;
  k_gram_reduce<<<reduce_grid(entries), BT, 0, stream>>>(work, nchunks, entries, C);
  NSP_LAUNCH_CHECK();
}

void launch_gemv_t(const double *Z, int64_t n, int k, const double *r, double *t, double *work,
                   cudaStream_t stream) {
  if (k <= 0) return;
  const int64_t cs = gemv_chunks(n);
  const int64_t rpc = (n + cs - 1) / cs;
  k_gemv_t_partial<<<(int)cs, BT, 0, stream>>>(Z, n, k, r, std::max<int64_t>(rpc, 1), work);
  NSP_LAUNCH_CHECK();
  k_gram_reduce<<<reduce_grid(k), BT, 0, stream>>>(work, (int)cs, k, t);
  NSP_LAUNCH_CHECK();
}

void launch_gemv_n(const double *Z, int64_t n, int k, const double *t, double beta, double *z,
                   cudaStream_t stream) {
  if (n <= 0 || k <= 0) return;
  k_gemv_n<<<ceil_div(n, BT / GN), BT, 0, stream>>>(Z, n, k, t, beta, z);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_block_update(const T *A, const double *M, int64_t n, int s1, int s2, T scale,
                         const T *C, T beta, T *Out, cudaStream_t stream) {
  if (n <= 0 || s2 <= 0) return;
  require(s2 <= 256, NSP_ERR_UNSUPPORTED, "block update with more than 256 columns");
  const size_t sm = sizeof(T) * (size_t)(UR * (UK + 1) + UK * s2);
  static bool attr = false;
  if (!attr) {
    NSP_CUDA(cudaFuncSetAttribute(k_block_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(T) * (UR * (UK + 1) + UK * 256))));
    attr = true;
  }
  k_block_update<T><<<ceil_div(n, UR), BT, sm, stream>>>(A, M, n, s1, s2, scale, C, beta, Out);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_col_sumsq(const T *X, int64_t n, int s, double *colsq, double *work,
                      cudaStream_t stream) {
  const int64_t cs = std::max<int64_t>(1, std::min<int64_t>(2 * 152, (n + 255) / 256));
  const int64_t rpc = (n + cs - 1) / cs;
  k_colsq_partial<T><<<(int)cs, BT, 0, stream>>>(X, n, s, std::max<int64_t>(rpc, 1), work);
  NSP_LAUNCH_CHECK();
  k_gram_reduce<<<reduce_grid(s), BT, 0, stream>>>(work, (int)cs, s, colsq);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_gaussian(uint64_t seed, int64_t count, T *out, cudaStream_t stream) {
  if (count <= 0) return;
  k_gaussian<T><<<ceil_div(count, BT), BT, 0, stream>>>(seed, count, out);
  NSP_LAUNCH_CHECK();
}

void launch_dot(const double *x, const double *y, int64_t n, double *result, double *work,
                cudaStream_t stream) {
  const int64_t cs = std::max<int64_t>(1, std::min<int64_t>(2 * 152, (n + 1023) / 1024));
  const int64_t rpc = (n + cs - 1) / cs;
  k_dot_partial<<<(int)cs, BT, 0, stream>>>(x, y, n, std::max<int64_t>(rpc, 1), work);
  NSP_LAUNCH_CHECK();
  k_sum<<<1, BT, 0, stream>>>(work, (int)cs, result);
  NSP_LAUNCH_CHECK();
}

void launch_axpby(int64_t n, const double *a_ptr, double a_sign, const double *x, double b,
                  double *y, cudaStream_t stream) {
  if (n <= 0) return;
  k_axpby<<<ceil_div(n, BT), BT, 0, stream>>>(n, a_ptr, a_sign, x, b, y);
  NSP_LAUNCH_CHECK();
}

void launch_scale_cols(double *X, int64_t n, int s, const double *scale, bool take_sqrt,
                       cudaStream_t stream) {
  if (n * s <= 0) return;
  k_scale_cols<<<ceil_div(n * s, BT), BT, 0, stream>>>(X, n, s, scale, take_sqrt ? 1 : 0);
  NSP_LAUNCH_CHECK();
}

void launch_pcg_step(int64_t n, const double *rz, const double *pq, double *alpha,
                     const double *p, const double *q, double *x, double *r, double *rr,
                     double *work, cudaStream_t stream) {
  const int64_t cs = std::max<int64_t>(1, std::min<int64_t>(2 * 152, (n + 1023) / 1024));
  const int64_t rpc = (n + cs - 1) / cs;
  k_pcg_step<<<(int)cs, BT, 0, stream>>>(n, std::max<int64_t>(rpc, 1), rz, pq, alpha, p, q, x,
                                          r, work);
  NSP_LAUNCH_CHECK();
  k_sum<<<1, BT, 0, stream>>>(work, (int)cs, rr);
  NSP_LAUNCH_CHECK();
}

void launch_pcg_direction(int64_t n, const double *rz_new, const double *rz_old, double *beta,
                          const double *z, double *p, cudaStream_t stream) {
  k_pcg_direction<<<ceil_div(std::max<int64_t>(n, 1), BT), BT, 0, stream>>>(n, rz_new, rz_old,
                                                                             beta, z, p);
  NSP_LAUNCH_CHECK();
}

void launch_pcg_scalars(const double *rz_new, const double *rz_old, const double *pq,
                        double *alpha, double *beta, cudaStream_t stream) {
  k_pcg_scalars<<<1, 32, 0, stream>>>(rz_new, rz_old, pq, alpha, beta);
  NSP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- instantiations
template void launch_spmm<float>(const CsrDev<float> &, const float *, float *, int, float,
                                 const float *, float, cudaStream_t);
template void launch_spmm<double>(const CsrDev<double> &, const double *, double *, int, double,
                                  const double *, double, cudaStream_t);
#define NSP_GS(Ti, To)                                                                        \
  template void launch_gather_rows<Ti, To>(const int64_t *, int64_t, const Ti *, To *, int,   \
                                           cudaStream_t);                                     \
  template void launch_scatter_rows<Ti, To>(const int64_t *, int64_t, const Ti *, To *, int,  \
                                            cudaStream_t);
NSP_GS(float, float)
NSP_GS(double, double)
NSP_GS(float, double)
NSP_GS(double, float)
template void launch_gather_values<float>(const int64_t *, int64_t, const double *, float *,
                                          cudaStream_t);
template void launch_gather_values<double>(const int64_t *, int64_t, const double *, double *,
                                           cudaStream_t);
template void launch_gram<float, float>(const float *, const float *, int64_t, int, int, double *,
                                        double *, cudaStream_t);
template void launch_gram<float, double>(const float *, const float *, int64_t, int, int, double *,
                                         double *, cudaStream_t);
template void launch_gram<double, double>(const double *, const double *, int64_t, int, int,
                                          double *, double *, cudaStream_t);
template void launch_block_update<float>(const float *, const double *, int64_t, int, int,
                                         float, const float *, float, float *, cudaStream_t);
template void launch_block_update<double>(const double *, const double *, int64_t, int, int,
                                          double, const double *, double, double *,
                                          cudaStream_t);
template void launch_col_sumsq<float>(const float *, int64_t, int, double *, double *, cudaStream_t);
template void launch_col_sumsq<double>(const double *, int64_t, int, double *, double *,
                                       cudaStream_t);
template void launch_gaussian<float>(uint64_t, int64_t, float *, cudaStream_t);
template void launch_gaussian<double>(uint64_t, int64_t, double *, cudaStream_t);

}  // namespace nsp
