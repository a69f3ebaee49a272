// Supernodal triangular solves X = A_b^{-1} B for every block b of a forest at once, s right-
// hand sides (the A_I^{-1} inside S_Gamma, §2.3 eq. (schur_complement), and A_G^{-1}, the
// first-level preconditioner S1 of §2.3 eq. (S1)).
//
// With the panel P_J = [inv(L11); L21 inv(L11)] of each supernode J (see k_factor.cu):
//   forward  (L y = b):  y_J = P_top f_top,  u_J = f_bot - P_bot f_top,
//     f = b on J's columns plus the children's update rows u_C (extend-add gather);
//   backward (L^T x = y): x_J = P_top^T y_J - P_bot^T x[rows of J below its columns].
//
// One persistent launch runs a whole solve: CTAs claim work items in topological order
// (all forward items by tree level, then all backward items by reverse level) from an atomic
// counter and wait, with a bounded spin, on per-supernode completion counters:
//   forward item of J   : after every forward item of J's children;
//   backward item of J  : after every backward item of J's parent (after J's own forward
//                         items for a root).
// A CTA only waits for items claimed before its own, so the schedule cannot deadlock.
// Counters grow monotonically (unsigned, compared modulo 2^32); launch e waits for
// e x (units per supernode). The epoch e and the claim base are read from device memory,
// where k_sweep_begin advances them before every launch.
// Item kinds:
//   vector (s = 1): 16-byte vector loads of the panel, 8 warps split the K dimension
//                   (forward) or a warp per panel column, vec_cols columns a tile
//                   (backward); supernodes with m <= 96, w <= 32 are processed a warp
//                   each, up to 8 per item;
//   block (s > 1):  a register-blocked (TM x K) * (K x s) product per tile on CUDA cores.
#include "sweep_tiles.cuh"

namespace nsp {
namespace {

constexpr int MAX_SPINS = 1 << 22;  // default bound of a dependency wait (seconds at most)

// ---------------------------------------------------------------- synchronization
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *p >= target (modulo 2^32). Returns false (and sets the abort flag)
// on timeout or when another CTA has aborted.
__device__ bool wait_geq(const uint32_t *p, uint32_t target, uint32_t *abort_flag, DevStatus *st,
                         int32_t where, int max_spins) {
  int spins = 0;
  while ((int32_t)(ld_acquire(p) - target) < 0) {
    if (ld_relaxed(abort_flag)) return false;
    if (++spins > max_spins) {
      atomicExch(abort_flag, 1u);
      dev_fail(st, DEV_TIMEOUT, where);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Before every sweep: next epoch; items of this launch are numbered from the claim counter's
// current value (every earlier launch on the plan has finished, stream order).
__global__ void k_sweep_begin(SweepPlan p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *p.epoch += 1u;
    *p.claim_base = *p.claim;
  }
}
// ---------------------------------------------------------------- the persistent sweep
// item_b >= 0: tile of supernode item_a starting at row/column item_b;
// item_b < 0 : group of -item_b small supernodes group_sn[item_a ...] (vector mode only).
template <typename T, int TC, int CM, int RM, bool VECTOR>
__global__ void __launch_bounds__(ST, sizeof(T) == 8 ? 1 : VECTOR ? 4 : 2) k_sweep(SweepCtx c, const T *__restrict__ panel,
                                              const T *B, T *Y, T *U, T *X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  __shared__ int s_item, s_ok;
  __shared__ uint32_t s_epoch, s_base;
  const SweepPlan &p = c.p;
  if (threadIdx.x == 0) {
    s_epoch = *(volatile uint32_t *)p.epoch;
    s_base = *(volatile uint32_t *)p.claim_base;
  }
  __syncthreads();
  const uint32_t epoch = s_epoch;
  while (true) {
    if (threadIdx.x == 0) s_item = (int)(atomicAdd(p.claim, 1u) - s_base);
    __syncthreads();
    const int it = s_item;
    if (it >= p.nitems) break;
    const bool fwd = it < p.nfwd;
    const int a = p.item_a[it], b = p.item_b[it];
    const int sub_len = b <= kSubtreeTag ? kSubtreeTag - b : 0;  // subtree item: list length
    const int nmem = sub_len ? 1 : b < 0 ? -b : 1;
    // the supernode a member q of the item stands for in the dependency counters (a subtree
    // item: its head, the last entry of its member list)
    auto dep_sn = [&](int q) {
      return sub_len ? p.group_sn[a + sub_len - 1] : b < 0 ? p.group_sn[a + q] : a;
    };
    // dependencies: lane q of warp 0 waits for member q, so a group's waits overlap
    if (threadIdx.x < 32) {
      const int q = threadIdx.x;
      bool ok = ld_relaxed(p.abort_flag) == 0;
      if (q < nmem && ok) {
        const int J = dep_sn(q);
        if (fwd) {
          ok = wait_geq(&p.cnt_f[J], epoch * (uint32_t)p.need_f[J], p.abort_flag, c.st, J,
                        c.max_spins);
        } else {
          const int par = p.sn_parent[J];
          ok = par >= 0
                   ? wait_geq(&p.done_b[par], epoch * (uint32_t)p.units_b[par], p.abort_flag,
                              c.st, J, c.max_spins)
                   : wait_geq(&p.self_f[J], epoch * (uint32_t)p.units_f[J], p.abort_flag, c.st,
                              J, c.max_spins);
        }
      }
      ok = __all_sync(0xffffffffu, ok);
      if (q == 0) s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      if constexpr (VECTOR) {
        if (b < 0) {
          // a group (L members of one height) or a subtree (members by height, -1 between
          // heights): the members of one height a warp each, a barrier between heights
          const int32_t *lst = p.group_sn + a;
          const int L = sub_len ? sub_len : -b;
          const int wid = threadIdx.x >> 5;
          int q = fwd ? 0 : L - 1;
          while (fwd ? q < L : q >= 0) {
            int e = q;
            if (fwd) {
              while (e < L && lst[e] >= 0) ++e;
            } else {
              while (e >= 0 && lst[e] >= 0) --e;
            }
            const int lo = fwd ? q : e + 1, hi = fwd ? e : q + 1;  // members [lo, hi)
            for (int t = lo + wid; t < hi; t += ST / 32) {
              if (fwd) vec_fwd_small<T>(c, panel, B, Y, U, lst[t]);
              else vec_bwd_small<T>(c, panel, Y, X, lst[t], sm + wid * 32 * 33);
            }
            if (sub_len) __syncthreads();
            q = fwd ? e + 1 : e - 1;
          }
        } else {
          if (fwd) vec_fwd_tile<T>(c, panel, B, Y, U, a, b, sm);
          else vec_bwd_tile<T>(c, panel, Y, X, a, b, sm);
        }
      } else {
        // one tile (supernode a, first row / column b), or every tile of a subtree's members
        // (heights upwards forward, downwards backward; -1 separates heights and is a barrier
        // that makes one height's U / X rows visible to the next)
        constexpr int TM = Cfg<TC, CM, RM>::TM;
        int pos = sub_len ? (fwd ? 0 : sub_len - 1) : 0;
        int J = sub_len ? p.group_sn[a + pos] : a;
        int r0 = sub_len ? 0 : b;
        while (true) {
          if (J >= 0) {
            if (fwd) blk_fwd_tile<T, TC, CM, RM>(c, panel, B, Y, U, J, r0, sm);
            else blk_bwd_tile<T, TC, CM, RM>(c, panel, Y, X, J, r0, sm);
          } else {
            __syncthreads();
          }
          if (!sub_len) break;
          if (J >= 0 && r0 + TM < (fwd ? c.f.sn_m[J] : c.f.sn_w[J])) {
            r0 += TM;
            continue;
          }
          pos += fwd ? 1 : -1;
          if (pos < 0 || pos >= sub_len) break;
          J = p.group_sn[a + pos];
          r0 = 0;
        }
      }
    }
    // the barrier orders every thread's writes before thread 0's device-scope fence, which
    // publishes them before the completion counters move
    __syncthreads();
    if (threadIdx.x == 0 && s_ok) {
      __threadfence();
      for (int q = 0; q < nmem; ++q) {
        const int J = dep_sn(q);
        if (fwd) {
          atomicAdd(&p.self_f[J], 1u);
          const int par = p.sn_parent[J];
          if (par >= 0) atomicAdd(&p.cnt_f[par], 1u);
        } else {
          atomicAdd(&p.done_b[J], 1u);
        }
      }
    }
  }
}

template <typename T, int TC, int CM, int RM, bool VECTOR>
void run_sweep(const SweepCtx &c, int grid, size_t smem, const T *panel, const T *B, T *Y,
               T *U, T *X, cudaStream_t st) {
  static size_t attr = 0;
  if (smem > attr) {
    ensure_dyn_smem(k_sweep<T, TC, CM, RM, VECTOR>, smem);
    attr = smem;
  }
  k_sweep<T, TC, CM, RM, VECTOR><<<grid, ST, smem, st>>>(c, panel, B, Y, U, X);
  NSP_LAUNCH_CHECK();
}

template <typename T, int TC, int CM, int RM>
size_t blk_smem() {
  using C = Cfg<TC, CM, RM>;
  return sizeof(T) * (size_t)(TK * (C::TM + 1) + TK * C::NCP);
}

template <typename T, int TC, int CM, int RM, bool VECTOR>
int sweep_grid(size_t smem) {
  static int grid = 0;
  static size_t for_smem = 0;
  if (grid == 0 || for_smem != smem) {
    int dev = 0, sms = 0, per = 0;
    NSP_CUDA(cudaGetDevice(&dev));
    NSP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ensure_dyn_smem(k_sweep<T, TC, CM, RM, VECTOR>, smem);
    NSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<T, TC, CM, RM, VECTOR>,
                                                           ST, smem));
    grid = sms * std::max(1, std::min(per, 4));
    for_smem = smem;
  }
  return grid;
}

template <typename T, int TC, int CM, int RM, bool VECTOR>
void dispatch(SweepCtx c, size_t smem, const T *panel, const T *B, T *Y, T *U, T *X,
              cudaStream_t st, int *grid_out) {
  const int gmax = sweep_grid<T, TC, CM, RM, VECTOR>(smem);
  const int grid = *grid_out > 0 ? std::min(*grid_out, gmax) : gmax;
  *grid_out = grid;
  run_sweep<T, TC, CM, RM, VECTOR>(c, grid, smem, panel, B, Y, U, X, st);
}

}  // namespace

int sweep_vector_rows(int elem_bytes) { return kVecRG * (16 / elem_bytes); }

template <typename T>
int launch_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *Y, T *U,
                 T *X, int s, DevStatus *st, cudaStream_t stream, int grid_req, int max_spins) {
  SweepCtx c{f, p, s, st, max_spins > 0 ? max_spins : MAX_SPINS};
  int grid = grid_req;
  k_sweep_begin<<<1, 32, 0, stream>>>(p);
  NSP_LAUNCH_CHECK();
  if (s == 1) {
    require(p.vector, NSP_ERR_INVALID_ARG, "vector plan needed for one right-hand side");
    const size_t ldmax = (size_t)((p.max_m + 3) & ~3) + 8;
    const size_t smem = sizeof(T) * std::max<size_t>(
        ldmax + (size_t)(ST / kVecRG + 1) * kVecRG * (16 / sizeof(T)), 8 * 32 * 33);
    dispatch<T, 1, 1, 1, true>(c, smem, panel, B, Y, U, X, stream, &grid);
    return grid;
  }
  require(!p.vector, NSP_ERR_INVALID_ARG, "block plan needed for several right-hand sides");
#define NSP_BLK(TC_, CM_, RM_) \
  dispatch<T, TC_, CM_, RM_, false>(c, blk_smem<T, TC_, CM_, RM_>(), panel, B, Y, U, X, stream, &grid)
  if (p.blk_rows == kSweepBlockRowsNarrow) {   // 32-row tiles: 32 column threads x 8 row threads
    if (s <= 32) NSP_BLK(32, 1, 4);
    else if (s <= 64) NSP_BLK(32, 2, 4);
    else if (s <= 96) NSP_BLK(32, 3, 4);
    else if (s <= 128) NSP_BLK(32, 4, 4);
    else if (s <= 160) NSP_BLK(32, 5, 4);
    else if (s <= 256) NSP_BLK(32, 8, 4);
    else throw Error(NSP_ERR_UNSUPPORTED, "more than 256 right-hand sides");
    return grid;
  }
  require(p.blk_rows == kSweepBlockRows, NSP_ERR_INVALID_ARG, "sweep plan tile rows");
  if (s <= 16) NSP_BLK(16, 1, 4);
  else if (s <= 32) NSP_BLK(16, 2, 4);
  else if (s <= 48) NSP_BLK(16, 3, 4);
  else if (s <= 64) NSP_BLK(16, 4, 4);
  else if (s <= 80) NSP_BLK(16, 5, 4);
  else if (s <= 96) NSP_BLK(16, 6, 4);
  else if (s <= 128) NSP_BLK(16, 8, 4);
  else if (s <= 160) NSP_BLK(16, 10, 4);
  else if (s <= 256) NSP_BLK(16, 16, 4);
  else throw Error(NSP_ERR_UNSUPPORTED, "more than 256 right-hand sides");
#undef NSP_BLK
  return grid;
}

template int launch_sweep<float>(const ForestDev &, const SweepPlan &, const float *,
                                 const float *, float *, float *, float *, int, DevStatus *,
                                 cudaStream_t, int, int);
template int launch_sweep<double>(const ForestDev &, const SweepPlan &, const double *,
                                  const double *, double *, double *, double *, int, DevStatus *,
                                  cudaStream_t, int, int);

}  // namespace nsp
