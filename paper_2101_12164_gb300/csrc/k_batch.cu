// Segmented kernels for a batch of independent matrices solved in one handle: rows of a
// vector block belong to one matrix ("segment") each, and every s x s quantity, scalar and
// convergence flag is per segment. Work is cut into chunks of rows that never cross a
// segment boundary (host-built), so each reduction is a per-chunk partial followed by an
// ordered per-segment sum (deterministic).
#include <algorithm>

#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int BT = 256;
constexpr int GR = 16;

// ---------------------------------------------------------------- segmented Gram
template <typename T, typename AccT, int RT>
__global__ void __launch_bounds__(BT) k_seg_gram_partial(const T *__restrict__ X,
                                                         const T *__restrict__ Y, int s1, int s2,
                                                         SegChunks ch, double *work) {
  constexpr int TS = 16 * RT;
  __shared__ T Xs[GR][TS];
  __shared__ T Ys[GR][TS];
  const int c = blockIdx.x;
  const int64_t i0 = ch.row0[c], i1 = ch.row1[c];
  const int a0 = blockIdx.y * TS, b0 = blockIdx.z * TS;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  AccT acc[RT][RT];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[i][j] = AccT(0);
  constexpr int NQ = GR * TS / BT;
  for (int64_t ib = i0; ib < i1; ib += GR) {
    T xv[NQ], yv[NQ];  // every load of the two tiles in flight before the shared stores
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = tid + u * BT, r = q / TS, cc = q % TS;
      const int64_t row = ib + r;
      xv[u] = (row < i1 && a0 + cc < s1) ? X[(size_t)row * s1 + a0 + cc] : T(0);
      yv[u] = (row < i1 && b0 + cc < s2) ? Y[(size_t)row * s2 + b0 + cc] : T(0);
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
      if (a < s1 && b < s2) work[((size_t)c * s1 + a) * s2 + b] = (double)acc[i][j];
    }
}

// out[seg][e] = sum over the segment's chunks (in order) of work[chunk][e]
__global__ void k_seg_reduce(const double *work, SegChunks ch, int64_t entries, double *out) {
  const int seg = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  double acc = 0.0;
  const int c1 = ch.seg_first[seg + 1];
  int c = ch.seg_first[seg];
  for (; c + 8 <= c1; c += 8) {  // eight partials in flight, summed in chunk order
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = work[(size_t)(c + u) * entries + e];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  for (; c < c1; ++c) acc += work[(size_t)c * entries + e];
  out[(size_t)seg * entries + e] = acc;
}

// ---------------------------------------------------------------- segmented column sums
template <typename T>
__global__ void __launch_bounds__(BT) k_seg_colsq_partial(const T *X, int s, SegChunks ch,
                                                          double *work) {
  __shared__ double red[8][33];
  const int c = blockIdx.x;
  const int64_t i0 = ch.row0[c], i1 = ch.row1[c];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int c0 = 0; c0 < s; c0 += 32) {
    const int col = c0 + tx;
    double acc = 0.0;
    if (col < s)
      for (int64_t i = i0 + ty; i < i1; i += 8) {
        const double v = (double)X[(size_t)i * s + col];
        acc += v * v;
      }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && col < s) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += red[q][tx];
      work[(size_t)c * s + col] = t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- segmented dot / axpy
__global__ void __launch_bounds__(BT) k_seg_dot_partial(const double *x, const double *y,
                                                        SegChunks ch, double *work) {
  __shared__ double red[BT];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = ch.row0[c] + threadIdx.x; i < ch.row1[c]; i += BT) acc += x[i] * y[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = BT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) work[c] = red[0];
}

// y = (sign * a[seg]) x + b y, per chunk (a == nullptr: coefficient sign)
__global__ void k_seg_axpby(SegChunks ch, const double *a, double sign, const double *x, double b,
                            double *y) {
  const int c = blockIdx.x;
  const double coef = sign * (a ? a[ch.seg[c]] : 1.0);
  for (int64_t i = ch.row0[c] + threadIdx.x; i < ch.row1[c]; i += blockDim.x)
    y[i] = coef * x[i] + b * y[i];
}

// alpha[seg] = active ? num[seg] / den[seg] : 0
__global__ void k_seg_ratio(const double *num, const double *den, const int32_t *active, int nseg,
                            double *out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < nseg) out[g] = (active && !active[g]) ? 0.0 : num[g] / den[g];
}

// ---------------------------------------------------------------- segmented block update
// Out rows of chunk c = scale * A rows (n x s1) M[seg] (s1 x s2, FP64) + beta C rows.
// A segment whose active flag is 0 keeps Out = beta C (its M is treated as zero).
template <typename T>
__global__ void __launch_bounds__(BT) k_seg_block_update(const T *__restrict__ A,
                                                         const double *__restrict__ M, int s1,
                                                         int s2, T scale, const T *C, T beta,
                                                         T *Out, SegChunks ch,
                                                         const int32_t *active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ms = reinterpret_cast<T *>(smem_raw);  // [s1][s2]
  const int c = blockIdx.x;
  const int seg = ch.seg[c];
  const bool on = !active || active[seg];
  const double *Mg = M + (size_t)seg * s1 * s2;
  for (int q0 = threadIdx.x; q0 < s1 * s2; q0 += 8 * BT) {  // eight loads in flight
    double mv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * BT;
      mv[u] = (on && q < s1 * s2) ? Mg[q] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (q0 + u * BT < s1 * s2) Ms[q0 + u * BT] = (T)mv[u];
  }
  __syncthreads();
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int64_t i = ch.row0[c] + ty; i < ch.row1[c]; i += 8) {
    for (int col = tx; col < s2; col += 32) {
      T acc = T(0);
#pragma unroll 8
      for (int k = 0; k < s1; ++k) acc += A[(size_t)i * s1 + k] * Ms[k * s2 + col];
      T v = scale * acc;
      if (C) v += beta * C[(size_t)i * s2 + col];
      Out[(size_t)i * s2 + col] = v;
    }
  }
}

__global__ void k_seg_pcg_init(const double *ff, int nseg, double *fn, int32_t *active,
                               int32_t *its, double *rel) {
  for (int g = threadIdx.x; g < nseg; g += blockDim.x) {
    const double f = sqrt(fmax(ff[g], 0.0));
    fn[g] = f;
    active[g] = f > 0.0;
    its[g] = 0;
    rel[g] = f > 0.0 ? 1.0 : 0.0;
  }
}

__global__ void k_seg_converge(const double *rr, const double *fn, double rtol, int maxit,
                               int32_t *active, int32_t *its, double *rel, int32_t *any, int nseg) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < nseg; g += blockDim.x) {
    if (!active[g]) continue;
    const int it = its[g] + 1;
    its[g] = it;
    const double r = sqrt(fmax(rr[g], 0.0)) / fn[g];
    rel[g] = r;
    const int still = (r > rtol) && (it < maxit);
    active[g] = still;
    if (still) s_any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) *any = s_any;
}

// The per-matrix stopping rule of the inner block PCG after an iteration (one block): a
// matrix with no search direction left stops without counting the iteration; otherwise its
// count grows, its residual ratio and kept columns are recorded, and it stops once the ratio
// is at most eps. *passes counts the iterations of the whole batch; *go = (a matrix is still
// active and passes < maxit) is also written to the conditional of the CUDA graph loop that
// runs the iterations, when set_cond is 1.
__global__ void k_seg_inner_decide(const double *ratio, const int32_t *nkept, double eps,
                                   int nseg, int32_t *active, int32_t *its, double *rat,
                                   int32_t *act, int32_t *go, int32_t *passes, int maxit,
                                   cudaGraphConditionalHandle h, int set_cond) {
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < nseg; g += blockDim.x) {
    if (!active[g]) continue;
    if (nkept[g] == 0) {
      active[g] = 0;
      act[g] = 0;
      continue;
    }
    its[g] += 1;
    rat[g] = ratio[g];
    act[g] = nkept[g];
    if (!(ratio[g] > eps)) active[g] = 0;
    else s_any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int pcount = *passes + 1;
    *passes = pcount;
    const int more = s_any && pcount < maxit;
    *go = more;
    if (set_cond) cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

// the conditional of a CUDA graph loop from a flag the loop body computed; counts passes
__global__ void k_loop_condition(const int32_t *flag, int32_t *passes,
                                 cudaGraphConditionalHandle h) {
  *passes += 1;
  cudaGraphSetConditional(h, *flag != 0 ? 1u : 0u);
}

// Zs[i][j] = (double) Zt[i][j] * sqrt(Sigma[seg][j]) over chunks
template <typename T>
__global__ void k_seg_scale_sqrt(const T *Zt, int k, const double *Sigma, SegChunks ch, double *Zs) {
  const int c = blockIdx.x;
  const double *sg = Sigma + (size_t)ch.seg[c] * k;
  for (int64_t i = ch.row0[c]; i < ch.row1[c]; ++i)
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      Zs[(size_t)i * k + j] = (double)Zt[(size_t)i * k + j] * sqrt(fmax(sg[j], 0.0));
}

int seg_rt(int s) { return s <= 32 ? 2 : s <= 64 ? 4 : s <= 96 ? 6 : 8; }

template <typename T, typename AccT, int RT>
void seg_gram_rt(const T *X, const T *Y, int s1, int s2, const SegChunks &ch, double *C,
                 double *work, cudaStream_t st) {
  dim3 grid(ch.nchunk, ceil_div(s1, 16 * RT), ceil_div(s2, 16 * RT));
  k_seg_gram_partial<T, AccT, RT><<<grid, BT, 0, st>>>(X, Y, s1, s2, ch, work);
  NSP_LAUNCH_CHECK();
  const int64_t ent = (int64_t)s1 * s2;
  k_seg_reduce<<<dim3(ceil_div(ent, BT), ch.nseg), BT, 0, st>>>(work, ch, ent, C);
  NSP_LAUNCH_CHECK();
}

}  // namespace

template <typename T, typename AccT>
void launch_seg_gram(const T *X, const T *Y, int s1, int s2, const SegChunks &ch, double *C,
                     double *work, cudaStream_t st) {
  switch (seg_rt(std::max(s1, s2))) {
    case 2: seg_gram_rt<T, AccT, 2>(X, Y, s1, s2, ch, C, work, st); break;
    case 4: seg_gram_rt<T, AccT, 4>(X, Y, s1, s2, ch, C, work, st); break;
    case 6: seg_gram_rt<T, AccT, 6>(X, Y, s1, s2, ch, C, work, st); break;
    default: seg_gram_rt<T, AccT, 8>(X, Y, s1, s2, ch, C, work, st); break;
  }
}

template <typename T>
void launch_seg_colsq(const T *X, int s, const SegChunks &ch, double *colsq, double *work,
                      cudaStream_t st) {
  k_seg_colsq_partial<T><<<ch.nchunk, BT, 0, st>>>(X, s, ch, work);
  NSP_LAUNCH_CHECK();
  k_seg_reduce<<<dim3(ceil_div(s, BT), ch.nseg), BT, 0, st>>>(work, ch, s, colsq);
  NSP_LAUNCH_CHECK();
}

void launch_seg_dot(const double *x, const double *y, const SegChunks &ch, double *out,
                    double *work, cudaStream_t st) {
  k_seg_dot_partial<<<ch.nchunk, BT, 0, st>>>(x, y, ch, work);
  NSP_LAUNCH_CHECK();
  k_seg_reduce<<<dim3(1, ch.nseg), BT, 0, st>>>(work, ch, 1, out);
  NSP_LAUNCH_CHECK();
}

void launch_seg_axpby(const SegChunks &ch, const double *a, double sign, const double *x,
                      double b, double *y, cudaStream_t st) {
  k_seg_axpby<<<ch.nchunk, BT, 0, st>>>(ch, a, sign, x, b, y);
  NSP_LAUNCH_CHECK();
}

void launch_seg_ratio(const double *num, const double *den, const int32_t *active, int nseg,
                      double *out, cudaStream_t st) {
  k_seg_ratio<<<ceil_div(nseg, 128), 128, 0, st>>>(num, den, active, nseg, out);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_seg_block_update(const T *A, const double *M, int s1, int s2, T scale, const T *C,
                             T beta, T *Out, const SegChunks &ch, const int32_t *active,
                             cudaStream_t st) {
  const size_t sm = sizeof(T) * (size_t)s1 * s2;
  require(sm <= 200 * 1024, NSP_ERR_UNSUPPORTED, "segmented update: s too large");
  static bool attr = false;
  if (!attr) {
    NSP_CUDA(cudaFuncSetAttribute(k_seg_block_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    attr = true;
  }
  k_seg_block_update<T><<<ch.nchunk, BT, sm, st>>>(A, M, s1, s2, scale, C, beta, Out, ch, active);
  NSP_LAUNCH_CHECK();
}

void launch_seg_pcg_init(const double *ff, int nseg, double *fn, int32_t *active, int32_t *its,
                         double *rel, cudaStream_t st) {
  k_seg_pcg_init<<<1, 1024, 0, st>>>(ff, nseg, fn, active, its, rel);
  NSP_LAUNCH_CHECK();
}

void launch_seg_converge(const double *rr, const double *fn, double rtol, int maxit,
                         int32_t *active, int32_t *its, double *rel, int32_t *any, int nseg,
                         cudaStream_t st) {
  k_seg_converge<<<1, 1024, 0, st>>>(rr, fn, rtol, maxit, active, its, rel, any, nseg);
  NSP_LAUNCH_CHECK();
}

void launch_seg_inner_decide(const double *ratio, const int32_t *nkept, double eps, int nseg,
                             int32_t *active, int32_t *its, double *rat, int32_t *act,
                             int32_t *go, int32_t *passes, int maxit,
                             cudaGraphConditionalHandle h, int set_cond, cudaStream_t st) {
  k_seg_inner_decide<<<1, 1024, 0, st>>>(ratio, nkept, eps, nseg, active, its, rat, act, go,
                                         passes, maxit, h, set_cond);
  NSP_LAUNCH_CHECK();
}

void launch_loop_condition(const int32_t *flag, int32_t *passes, cudaGraphConditionalHandle h,
                           cudaStream_t st) {
  k_loop_condition<<<1, 1, 0, st>>>(flag, passes, h);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_seg_scale_sqrt(const T *Zt, int k, const double *Sigma, const SegChunks &ch,
                           double *Zs, cudaStream_t st) {
  k_seg_scale_sqrt<T><<<ch.nchunk, 128, 0, st>>>(Zt, k, Sigma, ch, Zs);
  NSP_LAUNCH_CHECK();
}
template void launch_seg_scale_sqrt<float>(const float *, int, const double *, const SegChunks &,
                                           double *, cudaStream_t);
template void launch_seg_scale_sqrt<double>(const double *, int, const double *, const SegChunks &,
                                            double *, cudaStream_t);

template void launch_seg_gram<float, float>(const float *, const float *, int, int,
                                            const SegChunks &, double *, double *, cudaStream_t);
template void launch_seg_gram<float, double>(const float *, const float *, int, int,
                                             const SegChunks &, double *, double *, cudaStream_t);
template void launch_seg_gram<double, double>(const double *, const double *, int, int,
                                              const SegChunks &, double *, double *, cudaStream_t);
template void launch_seg_colsq<float>(const float *, int, const SegChunks &, double *, double *,
                                      cudaStream_t);
template void launch_seg_colsq<double>(const double *, int, const SegChunks &, double *, double *,
                                       cudaStream_t);
template void launch_seg_block_update<float>(const float *, const double *, int, int, float,
                                             const float *, float, float *, const SegChunks &,
                                             const int32_t *, cudaStream_t);
template void launch_seg_block_update<double>(const double *, const double *, int, int, double,
                                              const double *, double, double *, const SegChunks &,
                                              const int32_t *, cudaStream_t);

}  // namespace nsp
