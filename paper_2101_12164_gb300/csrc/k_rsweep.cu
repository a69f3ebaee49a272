// Block-resident supernodal sweeps: X = A_b^{-1} B with one CTA per block b of a forest (the
// interior blocks A_1..A_N of §2.3 eq. (perm_A) are independent, "factorized cheaply in
// parallel"), both triangular sweeps of a block inside its CTA.
//
// Same arithmetic as the dependency-driven sweep of k_solve.cu (panels
// P_J = [inv(L11); L21 inv(L11)]; forward y_J = P_top f_top, u_J = f_bot - P_bot f_top;
// backward x_J = P_top^T y_J - P_bot^T x[rows below]), but scheduled by tree height inside
// the CTA: the supernodes of one height are independent, so they run concurrently and a
// barrier separates heights. No counters, flags or dependency waits cross CTAs. Per height:
//   small supernodes (block mode: w <= kResW, m <= kResM; vector mode: the warp limits of the
//   single-vector items) a warp each, the warps taking them in decreasing size order;
//   the others one at a time with every thread of the CTA, in the tiles of k_solve.cu.
// Block-mode warp items are the warp jobs of sweep_tiles.cuh (every dependent load chain of
// a supernode issued at once, panel chunks prefetched one ahead).
#include "sweep_tiles.cuh"

namespace nsp {
namespace {

// One CTA per block: forward heights upwards, then backward heights downwards.
// half: 0 both sweeps, 1 the forward sweep only (y = L^{-1} b into Y), 2 the backward sweep
// only (x = L^{-T} y from Y)
template <typename T, int TC, int CM, int RM, bool VECTOR>
__global__ void __launch_bounds__(ST, sizeof(T) == 8 ? 1 : 2)
    k_res_sweep(SweepCtx c, const T *__restrict__ panel, const T *B, T *Y, T *U, T *X, int half) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  constexpr int NW = ST / 32, CPL = WarpCpl<T>::value;
  T *wsm = sm + (size_t)(threadIdx.x >> 5) * wj_elems<T>();                  // this warp's
  int32_t *wim = reinterpret_cast<int32_t *>(sm + (size_t)NW * wj_elems<T>()) +
                 (threadIdx.x >> 5) * wj_ints();
  const SweepPlan &p = c.p;
  const int b = blockIdx.x;
  const int L0 = p.res_blk_ptr[b], L1 = p.res_blk_ptr[b + 1];
  const int wid = threadIdx.x >> 5;
  for (int L = L0; L < L1 && half != 2; ++L) {
    const int j0 = p.res_lvl_ptr[L], j1 = p.res_lvl_ptr[L + 1], jw = j0 + p.res_lvl_nwarp[L];
    for (int q = j0 + wid; q < jw; q += NW) {
      const int J = p.res_job[q];
      if constexpr (VECTOR) vec_fwd_small<T>(c, panel, B, Y, U, J);
      else warp_fwd_job<T, CPL>(c, panel, B, Y, U, J, wsm, wim);
    }
    __syncthreads();
    for (int q = jw; q < j1; ++q) {
      const int J = p.res_job[q], m = c.f.sn_m[J];
      if constexpr (VECTOR) {
        const int tm = kVecRG * Vec<T>::N;
        for (int r0 = 0; r0 < m; r0 += tm) {
          vec_fwd_tile<T>(c, panel, B, Y, U, J, r0, sm);
          __syncthreads();
        }
      } else {
        constexpr int TM = Cfg<TC, CM, RM>::TM;
        for (int r0 = 0; r0 < m; r0 += TM) {
          blk_fwd_tile<T, TC, CM, RM>(c, panel, B, Y, U, J, r0, sm);
          __syncthreads();
        }
      }
    }
  }
  for (int L = L1 - 1; L >= L0 && half != 1; --L) {
    const int j0 = p.res_lvl_ptr[L], j1 = p.res_lvl_ptr[L + 1], jw = j0 + p.res_lvl_nwarp[L];
    for (int q = j0 + wid; q < jw; q += NW) {
      const int J = p.res_job[q];
      if constexpr (VECTOR) vec_bwd_small<T>(c, panel, Y, X, J, sm + wid * 32 * 33);
      else warp_bwd_job<T, CPL>(c, panel, Y, X, J, wsm, wim);
    }
    __syncthreads();
    for (int q = jw; q < j1; ++q) {
      const int J = p.res_job[q], w = c.f.sn_w[J];
      if constexpr (VECTOR) {
        for (int c0 = 0; c0 < w; c0 += p.vec_cols) {
          vec_bwd_tile<T>(c, panel, Y, X, J, c0, sm);
          __syncthreads();
        }
      } else {
        constexpr int TM = Cfg<TC, CM, RM>::TM;
        for (int r0 = 0; r0 < w; r0 += TM) {
          blk_bwd_tile<T, TC, CM, RM>(c, panel, Y, X, J, r0, sm);
          __syncthreads();
        }
      }
    }
  }
}

template <typename T, int TC, int CM, int RM, bool VECTOR>
void run_res(const SweepCtx &c, int nblocks, size_t smem, const T *panel, const T *B, T *Y, T *U,
             T *X, int half, cudaStream_t st) {
  static size_t attr = 0;
  if (smem > attr) {
    ensure_dyn_smem(k_res_sweep<T, TC, CM, RM, VECTOR>, smem);
    attr = smem;
  }
  k_res_sweep<T, TC, CM, RM, VECTOR><<<nblocks, ST, smem, st>>>(c, panel, B, Y, U, X, half);
  NSP_LAUNCH_CHECK();
}

template <typename T, int TC, int CM, int RM>
size_t res_blk_smem() {
  using C = Cfg<TC, CM, RM>;
  const size_t tile = (size_t)(TK * (C::TM + 1) + TK * C::NCP);
  const size_t warps = (size_t)(ST / 32) * (sizeof(T) * wj_elems<T>() + 4 * wj_ints());
  return std::max(sizeof(T) * tile, warps);
}

}  // namespace

template <typename T>
void launch_res_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *Y,
                      T *U, T *X, int s, DevStatus *st, cudaStream_t stream, int half) {
  require(half >= 0 && half <= 2, NSP_ERR_INVALID_ARG, "block-resident sweep: bad half");
  require(p.res_nblocks > 0, NSP_ERR_INVALID_ARG, "block-resident sweep: no schedule");
  SweepCtx c{f, p, s, st, 0};
  if (s == 1) {
    require(p.vector, NSP_ERR_INVALID_ARG, "vector plan needed for one right-hand side");
    const size_t ldmax = (size_t)((p.max_m + 3) & ~3) + 8;
    const size_t smem = sizeof(T) * std::max<size_t>(
        ldmax + (size_t)(ST / kVecRG + 1) * kVecRG * (16 / sizeof(T)), 8 * 32 * 33);
    run_res<T, 1, 1, 1, true>(c, p.res_nblocks, smem, panel, B, Y, U, X, half, stream);
    return;
  }
  require(!p.vector, NSP_ERR_INVALID_ARG, "block plan needed for several right-hand sides");
#define NSP_RES(TC_, CM_, RM_) \
  run_res<T, TC_, CM_, RM_, false>(c, p.res_nblocks, res_blk_smem<T, TC_, CM_, RM_>(), panel, B, Y, U, X, half, stream)
  if (s <= 16) NSP_RES(16, 1, 4);
  else if (s <= 32) NSP_RES(16, 2, 4);
  else if (s <= 48) NSP_RES(16, 3, 4);
  else if (s <= 64) NSP_RES(16, 4, 4);
  else if (s <= 80) NSP_RES(16, 5, 4);
  else if (s <= 96) NSP_RES(16, 6, 4);
  else if (s <= 128) NSP_RES(16, 8, 4);
  else if (s <= 160) NSP_RES(16, 10, 4);
  else if (s <= 256) NSP_RES(16, 16, 4);
  else throw Error(NSP_ERR_UNSUPPORTED, "more than 256 right-hand sides");
#undef NSP_RES
}

template void launch_res_sweep<float>(const ForestDev &, const SweepPlan &, const float *,
                                      const float *, float *, float *, float *, int, DevStatus *,
                                      cudaStream_t, int);
template void launch_res_sweep<double>(const ForestDev &, const SweepPlan &, const double *,
                                       const double *, double *, double *, double *, int,
                                       DevStatus *, cudaStream_t, int);

}  // namespace nsp
