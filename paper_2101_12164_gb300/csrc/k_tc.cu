// Tall-skinny dense products of the inner block PCG on the tcgen05 tensor cores (FP32 data,
// 3xTF32 operands, FP32 accumulation in tensor memory):
//   Gram    C = X^T Y      (X n x s1, Y n x s2, s1, s2 <= 256): the block-CG inner products
//           P^T R, Q^T Z, W^T Z (block CG as in §5.1 of the paper, Ji & Li / O'Leary);
//   update  Out = scale * A M + beta * C   (A n x s1, M s1 x s2 FP64): X += P alpha,
//           R -= Q alpha, P = W L^-T, ... .
// Both are HBM-bound (arithmetic intensity s / 2 flops per byte of FP32): the tensor cores
// keep the arithmetic off the critical path where the FP32 SIMT pipes could not
// (2 n s^2 flops at 67 TFLOP/s take four times the HBM time of the operands at s = 160).
//
// Gram: one CTA per chunk of rows; stages of 16 rows of X and Y are split into TF32 hi/lo
// parts while being written to shared memory in the K-major tile layout (tc.cuh), double
// buffered against the MMAs of the previous stage; each CTA's 128 x N accumulators (two M
// tiles for s1 > 128) live in TMEM and are written as FP64 partials, which k_gram_reduce
// (k_blas.cu) adds in chunk order (deterministic).
// Update: each CTA takes 256-row tiles of A (two M tiles); the hi/lo split of M^T is prepared
// once per call in the same K-major layout (k_split_mt) and copied next to each A stage.
#include <algorithm>

#include "kernels.cuh"
#include "tc.cuh"

namespace nsp {
namespace {

constexpr int TT = 128;                 // threads per CTA (four warps read the 128 TMEM lanes)
constexpr int KS = 16;                  // K (rows of X, Y / columns of A) per stage
constexpr int SBO = (KS / 4) * 128;     // bytes between 8-row groups of a stage tile
constexpr int MAX_SPINS = 1 << 24;      // bound of every mbarrier wait

__host__ __device__ constexpr int pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int tmem_cols(int c) {
  int n = 32;
  while (n < c) n <<= 1;
  return n;
}

// stage tile bytes: R rows x KS columns of FP32
__host__ __device__ constexpr int tile_bytes(int R) { return (R / 8) * SBO; }

// Stage loads are issued one stage ahead into registers (they travel while the previous
// stage's MMAs run); a stage item is 4 consecutive rows (K) x 1 column (tile row) of a
// row-major matrix, stored split as one 16-byte group of the K-major layout.
__device__ __forceinline__ void load_item(const float *M, int64_t ld, int64_t row0,
                                          int64_t row_end, int col, int ncols, float (&v)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t row = row0 + j;
    v[j] = (row < row_end && col < ncols) ? __ldcg(&M[(size_t)row * ld + col]) : 0.f;
  }
}
__device__ __forceinline__ void store_item(const float (&v)[4], int r_tile, int g,
                                           unsigned char *hi, unsigned char *lo) {
  float4 h, l;
  tc::split_tf32(v[0], h.x, l.x);
  tc::split_tf32(v[1], h.y, l.y);
  tc::split_tf32(v[2], h.z, l.z);
  tc::split_tf32(v[3], h.w, l.w);
  const int off = tc::element_offset(r_tile, 4 * g, SBO);
  *reinterpret_cast<float4 *>(hi + off) = h;
  *reinterpret_cast<float4 *>(lo + off) = l;
}

// Three MMAs (hi hi, hi lo, lo hi) per K step of one stage into the accumulator at d.
__device__ __forceinline__ void mma_stage(uint32_t d, uint32_t ahi, uint32_t alo, uint32_t bhi,
                                          uint32_t blo, uint32_t idesc, bool first) {
#pragma unroll
  for (int ks = 0; ks < KS / 8; ++ks) {
    const uint32_t dk = ks * 2 * tc::kLbo;
    tc::mma_tf32(d, tc::smem_desc(ahi + dk, tc::kLbo, SBO), tc::smem_desc(bhi + dk, tc::kLbo, SBO),
                 idesc, !(first && ks == 0));
    tc::mma_tf32(d, tc::smem_desc(ahi + dk, tc::kLbo, SBO), tc::smem_desc(blo + dk, tc::kLbo, SBO),
                 idesc, true);
    tc::mma_tf32(d, tc::smem_desc(alo + dk, tc::kLbo, SBO), tc::smem_desc(bhi + dk, tc::kLbo, SBO),
                 idesc, true);
  }
}

// ---------------------------------------------------------------- Gram
template <int MT>
__global__ void __launch_bounds__(TT, 1)
    k_tc_gram(const float *__restrict__ X, const float *__restrict__ Y, int64_t n, int s1, int s2,
              int NP, int64_t rpc, double *work, DevStatus *st) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  constexpr int MP = 128 * MT;
  constexpr int AI = MP * (KS / 4) / TT;    // A items per thread
  constexpr int BI = 256 * (KS / 4) / TT;   // B items per thread (at most)
  const int ab = tile_bytes(MP), bb = tile_bytes(NP);
  const int stage = 2 * ab + 2 * bb;     // A hi, A lo, B hi, B lo
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = tmem_cols(MT * NP);
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int64_t i0 = (int64_t)blockIdx.x * rpc, i1 = min(n, i0 + rpc);
  const int64_t nrow = i1 > i0 ? i1 - i0 : 0;
  const int nst = (int)((nrow + KS - 1) / KS);
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  float av[AI][4], bv[BI][4];
  auto load_stage = [&](int it) {
    const int64_t r0 = i0 + (int64_t)it * KS;
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int q = tid + u * TT, a = q % MP, g = q / MP;
      load_item(X, s1, r0 + 4 * g, i1, a, s1, av[u]);
    }
#pragma unroll
    for (int u = 0; u < BI; ++u) {
      const int q = tid + u * TT, b = q % NP, g = q / NP;
      if (q < NP * (KS / 4)) load_item(Y, s2, r0 + 4 * g, i1, b, s2, bv[u]);
    }
  };
  bool ok = true;
  if (nst > 0) load_stage(0);
  for (int it = 0; it < nst; ++it) {
    const int buf = it & 1;
    unsigned char *sb = smem + buf * stage;
    if (it >= 2) {   // the MMAs of stage it - 2 read this buffer
      if (!tc::mbar_wait(&mbar[buf], ((it >> 1) - 1) & 1, MAX_SPINS)) ok = false;
    }
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int q = tid + u * TT;
      store_item(av[u], q % MP, q / MP, sb, sb + ab);
    }
#pragma unroll
    for (int u = 0; u < BI; ++u) {
      const int q = tid + u * TT;
      if (q < NP * (KS / 4)) store_item(bv[u], q % NP, q / NP, sb + 2 * ab, sb + 2 * ab + bb);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t base = tc::smem_u32(sb);
      for (int t = 0; t < MT; ++t) {
        const uint32_t ahi = base + t * (128 / 8) * SBO;
        mma_stage(tmem + t * NP, ahi, ahi + ab, base + 2 * ab, base + 2 * ab + bb, idesc, it == 0);
      }
      tc::commit(&mbar[buf]);
    }
    if (it + 1 < nst) load_stage(it + 1);
  }
  if (nst > 0) {   // every MMA done once the last stage's commit has arrived
    const int last = nst - 1;
    if (!tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, MAX_SPINS)) ok = false;
  }
  tc::fence_after();
  if (!ok && tid == 0) dev_fail(st, DEV_TIMEOUT, -3);
  // epilogue: lane = output row, eight columns per TMEM load
  for (int t = 0; t < MT; ++t) {
    const int a = t * 128 + 32 * warp + lane;
    for (int c0 = 0; c0 < NP; c0 += 8) {
      float v[8];
      if (nst > 0) {
        tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + t * NP + c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
      }
      if (a < s1) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < s2) work[((size_t)blockIdx.x * s1 + a) * s2 + c0 + j] = ok ? (double)v[j] : 0.0;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------- block update
// M^T split into TF32 hi / lo in the stage layout: for K chunk c (KS columns of A), rows
// = output columns (NP), [c][hi | lo][tile_bytes(NP)].
__global__ void k_split_mt(const double *__restrict__ M, int s1, int s2, int NP, float *out) {
  const int nch = (s1 + KS - 1) / KS;
  const int64_t total = (int64_t)nch * NP * KS;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int c = (int)(e / ((int64_t)NP * KS));
  const int rem = (int)(e % ((int64_t)NP * KS));
  const int col = rem / KS, k = rem % KS;   // output column, K index within the chunk
  const int kk = c * KS + k;
  const float x = (col < s2 && kk < s1) ? (float)M[(size_t)kk * s2 + col] : 0.f;
  float h, l;
  tc::split_tf32(x, h, l);
  unsigned char *base = reinterpret_cast<unsigned char *>(out) + (size_t)c * 2 * tile_bytes(NP);
  const int off = tc::element_offset(col, k, SBO);
  *reinterpret_cast<float *>(base + off) = h;
  *reinterpret_cast<float *>(base + tile_bytes(NP) + off) = l;
}

// Stages j = (tile, chunk) of this CTA's 256-row tiles, chunk-major inside a tile; the
// loads of stage j + 1 (A rows and the M^T chunk) are in flight during stage j.
__global__ void __launch_bounds__(TT, 1)
    k_tc_update(const float *__restrict__ A, const float *__restrict__ Mt, int64_t n, int s1,
                int s2, int NP, float scale, const float *C, float beta, float *Out,
                DevStatus *st) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tslot;
  constexpr int MT = 2, MP = 128 * MT;
  constexpr int AI = MP * (KS / 4) / TT;                 // A items (4 columns of a row) each
  constexpr int MI = 2 * tile_bytes(256) / 16 / TT;      // 16-byte M^T pieces each (at most)
  const int ab = tile_bytes(MP), bb = tile_bytes(NP);
  const int stage = 2 * ab + 2 * bb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = tmem_cols(MT * NP);
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tslot;
  const int nch = (s1 + KS - 1) / KS;
  const int64_t ntiles = (n + MP - 1) / MP;
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t nstage = my_tiles * nch;
  const uint32_t idesc = tc::idesc_tf32(128, NP);
  const int mi_count = 2 * bb / 16;
  float av[AI][4];
  float4 mv[MI];
  auto load_stage = [&](int64_t j) {
    const int64_t row0 = (blockIdx.x + (j / nch) * gridDim.x) * MP;
    const int c = (int)(j % nch);
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int q = tid + u * TT, r = q / (KS / 4), g = q % (KS / 4);
      const int64_t row = row0 + r;
      const int col0 = c * KS + 4 * g;
      if (row < n && (s1 & 3) == 0 && col0 + 3 < s1) {
        const float4 x = __ldcg(reinterpret_cast<const float4 *>(A + (size_t)row * s1 + col0));
        av[u][0] = x.x; av[u][1] = x.y; av[u][2] = x.z; av[u][3] = x.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = col0 + k;
          av[u][k] = (row < n && col < s1) ? __ldcg(&A[(size_t)row * s1 + col]) : 0.f;
        }
      }
    }
    const float4 *src = reinterpret_cast<const float4 *>(
        reinterpret_cast<const unsigned char *>(Mt) + (size_t)c * 2 * bb);
#pragma unroll
    for (int u = 0; u < MI; ++u) {
      const int q = tid + u * TT;
      if (q < mi_count) mv[u] = __ldg(src + q);
    }
  };
  bool ok = true;
  if (nstage > 0) load_stage(0);
  for (int64_t j = 0; j < nstage; ++j) {
    const int buf = (int)(j & 1);
    const int c = (int)(j % nch);
    const int64_t row0 = (blockIdx.x + (j / nch) * gridDim.x) * MP;
    unsigned char *sb = smem + buf * stage;
    if (j >= 2)
      if (!tc::mbar_wait(&mbar[buf], (uint32_t)(((j >> 1) - 1) & 1), MAX_SPINS)) ok = false;
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int q = tid + u * TT;
      store_item(av[u], q / (KS / 4), q % (KS / 4), sb, sb + ab);
    }
    {
      float4 *dst = reinterpret_cast<float4 *>(sb + 2 * ab);
#pragma unroll
      for (int u = 0; u < MI; ++u) {
        const int q = tid + u * TT;
        if (q < mi_count) dst[q] = mv[u];
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t base = tc::smem_u32(sb);
      for (int t = 0; t < MT; ++t) {
        const uint32_t ahi = base + t * (128 / 8) * SBO;
        mma_stage(tmem + t * NP, ahi, ahi + ab, base + 2 * ab, base + 2 * ab + bb, idesc, c == 0);
      }
      tc::commit(&mbar[buf]);
    }
    if (j + 1 < nstage) load_stage(j + 1);
    if (c == nch - 1) {   // the tile's accumulators are complete: epilogue
      if (!tc::mbar_wait(&mbar[buf], (uint32_t)((j >> 1) & 1), MAX_SPINS)) ok = false;
      tc::fence_after();
      // 32 columns per round: the C values (16-byte loads when rows are 16-byte aligned) are
      // requested before the two TMEM loads, and one wait covers both
      const bool vec = (s2 & 3) == 0;
      for (int t = 0; t < MT; ++t) {
        const int64_t row = row0 + t * 128 + 32 * warp + lane;
        const bool rok = row < n && ok;
        for (int c0 = 0; c0 < NP; c0 += 32) {
          float cv[32];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = c0 + 4 * q;
            if (C && rok && vec && col + 3 < s2) {
              const float4 x = __ldcg(reinterpret_cast<const float4 *>(C + (size_t)row * s2 + col));
              cv[4 * q] = x.x; cv[4 * q + 1] = x.y; cv[4 * q + 2] = x.z; cv[4 * q + 3] = x.w;
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                cv[4 * q + u] = (C && rok && col + u < s2) ? __ldcg(&C[(size_t)row * s2 + col + u]) : 0.f;
            }
          }
          uint32_t r0[16], r1[16];
          const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + t * NP + c0;
          tc::tmem_ld16_nowait(ta, r0);
          if (c0 + 16 < NP) tc::tmem_ld16_nowait(ta + 16, r1);
          tc::tmem_wait_ld();
          if (!rok) continue;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = c0 + 4 * q;
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int jj = 4 * q + u;
              const float acc = __uint_as_float(jj < 16 ? r0[jj] : r1[jj - 16]);
              o[u] = scale * acc + (C ? beta * cv[jj] : 0.f);
            }
            if (vec && col + 3 < s2) {
              *reinterpret_cast<float4 *>(Out + (size_t)row * s2 + col) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (col + u < s2) Out[(size_t)row * s2 + col + u] = o[u];
            }
          }
        }
      }
      // every thread's TMEM reads finish before the next tile's first MMA overwrites them
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
    }
  }
  if (!ok && tid == 0) dev_fail(st, DEV_TIMEOUT, -4);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    NSP_CUDA(cudaGetDevice(&dev));
    NSP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

template <typename K>
void set_smem_attr(K kernel, size_t bytes) {
  NSP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

size_t tc_gram_chunks(int64_t n) {
  return (size_t)std::max<int64_t>(1, std::min<int64_t>(num_sms(), (n + 4 * KS - 1) / (4 * KS)));
}

void launch_tc_gram(const float *X, const float *Y, int64_t n, int s1, int s2, double *C,
                    double *work, DevStatus *st, cudaStream_t stream) {
  if (s1 <= 0 || s2 <= 0) return;
  require(s1 <= 256 && s2 <= 256, NSP_ERR_UNSUPPORTED, "tensor-core Gram wider than 256");
  const int NP = pad16(s2);
  const int ch = (int)tc_gram_chunks(n);
  const int64_t rpc = std::max<int64_t>(KS, ((n + ch - 1) / ch + KS - 1) / KS * KS);
  if (s1 <= 128) {
    const size_t sm = 2 * (size_t)(2 * tile_bytes(128) + 2 * tile_bytes(NP));
    set_smem_attr(k_tc_gram<1>, sm);
    k_tc_gram<1><<<ch, TT, sm, stream>>>(X, Y, n, s1, s2, NP, rpc, work, st);
  } else {
    const size_t sm = 2 * (size_t)(2 * tile_bytes(256) + 2 * tile_bytes(NP));
    set_smem_attr(k_tc_gram<2>, sm);
    k_tc_gram<2><<<ch, TT, sm, stream>>>(X, Y, n, s1, s2, NP, rpc, work, st);
  }
  NSP_LAUNCH_CHECK();
  launch_gram_reduce(work, ch, (int64_t)s1 * s2, C, stream);
}

size_t tc_update_work_floats(int s1, int s2) {
  const int nch = (s1 + KS - 1) / KS;
  return (size_t)nch * 2 * pad16(std::max(s2, 1)) * KS;
}

void launch_tc_block_update(const float *A, const double *M, int64_t n, int s1, int s2,
                            float scale, const float *C, float beta, float *Out, float *mt_work,
                            DevStatus *st, cudaStream_t stream) {
  if (n <= 0 || s2 <= 0) return;
  require(s1 <= 256 && s2 <= 256, NSP_ERR_UNSUPPORTED, "tensor-core update wider than 256");
  const int NP = pad16(s2);
  const int64_t tot = (int64_t)tc_update_work_floats(s1, s2);
  k_split_mt<<<(int)((tot + 255) / 256), 256, 0, stream>>>(M, s1, s2, NP, mt_work);
  NSP_LAUNCH_CHECK();
  const size_t sm = 2 * (size_t)(2 * tile_bytes(256) + 2 * tile_bytes(NP));
  set_smem_attr(k_tc_update, sm);
  const int64_t ntiles = (n + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, num_sms()));
  k_tc_update<<<grid, TT, sm, stream>>>(A, mt_work, n, s1, s2, NP, scale, C, beta, Out, st);
  NSP_LAUNCH_CHECK();
}

}  // namespace nsp
