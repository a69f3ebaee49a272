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
#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int ST = 256;      // threads per CTA
constexpr int TK = 64;       // K chunk of the block product
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

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static V load(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
  __device__ static float get(const V &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static V load(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
  __device__ static double get(const V &v, int i) { return i == 0 ? v.x : v.y; }
};

struct SweepCtx {
  ForestDev f;
  SweepPlan p;
  int s;
  DevStatus *st;
  int max_spins;
};

// f_top / f_bot entry k of supernode J (column b, s columns): B row + children's update rows
template <typename T>
__device__ __forceinline__ T front_rhs(const SweepCtx &c, const T *B, const T *U, int J, int k,
                                       int col, bool with_b) {
  const int64_t rp = c.f.sn_rowptr[J];
  T v = (with_b && B) ? B[(size_t)(c.f.sn_first[J] + k) * c.s + col] : T(0);
  for (int64_t e = c.f.gptr[rp + k]; e < c.f.gptr[rp + k + 1]; ++e)
    v += __ldcg(&U[(size_t)c.f.gsrc[e] * c.s + col]);
  return v;
}

// v[i] += the update rows landing on front position pos[i] of the supernode whose rows start
// at rp (pos[i] < 0: none), column col: the NR positions advance together so that their
// dependent index and value loads are in flight at the same time.
template <typename T, int NR>
__device__ __forceinline__ void gather_rows(const SweepCtx &c, const T *U, int64_t rp,
                                            const int (&pos)[NR], T (&v)[NR], int col) {
  int64_t e[NR], ee[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    e[i] = pos[i] >= 0 ? c.f.gptr[rp + pos[i]] : 0;
    ee[i] = pos[i] >= 0 ? c.f.gptr[rp + pos[i] + 1] : 0;
  }
  bool more = true;
  while (more) {
    int64_t src[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) src[i] = e[i] < ee[i] ? c.f.gsrc[e[i]] : -1;
    more = false;
#pragma unroll
    for (int i = 0; i < NR; ++i)
      if (src[i] >= 0) {
        v[i] += __ldcg(&U[(size_t)src[i] * c.s + col]);
        more |= ++e[i] < ee[i];
      }
  }
}

// ---------------------------------------------------------------- vector items (s = 1)
// Forward tile: kVecRG row groups of VN rows x ST / kVecRG K groups; each thread keeps 8
// vector loads in flight. Rows of the tile: kVecRG VN.
constexpr int kVecRG = 32;
template <typename T>
__device__ void vec_fwd_tile(const SweepCtx &c, const T *panel, const T *B, T *Y, T *U, int J,
                             int r0, T *sm) {
  using VT = Vec<T>;
  constexpr int VN = VT::N, TMV = kVecRG * VN, KG = ST / kVecRG;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const T *P = panel + c.f.sn_panel[J];
  const int r1 = min(r0 + TMV, m);
  const int kmax = (r1 <= w) ? r1 : w;
  T *fs = sm;                      // [kmax]
  T *red = sm + ((ld + 3) & ~3);   // [KG][TMV]
  T *gb = red + KG * TMV;          // [TMV] update-row gathers of the tile's rows
  const int tid = threadIdx.x;
  for (int kb = tid; kb < kmax; kb += 3 * ST) {  // three positions' gathers in flight
    int pos[3];
    T v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int k = kb + q * ST;
      pos[q] = k < kmax ? k : -1;
      v[q] = (k < kmax && B) ? B[first + k] : T(0);
    }
    gather_rows<T, 3>(c, U, c.f.sn_rowptr[J], pos, v, 0);
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (kb + q * ST < kmax) fs[kb + q * ST] = v[q];
  }
  if (kmax <= ST - TMV && tid >= ST - TMV) {  // otherwise idle threads gather concurrently
    const int i = tid - (ST - TMV), r = r0 + i;
    int pos[1] = {(r >= w && r < r1) ? r : -1};
    T v[1] = {T(0)};
    gather_rows<T, 1>(c, U, c.f.sn_rowptr[J], pos, v, 0);
    gb[i] = v[0];
  }
  __syncthreads();
  const int rg = tid % kVecRG, kg = tid / kVecRG;
  const int row = r0 + VN * rg;
  T acc[VN];
#pragma unroll
  for (int i = 0; i < VN; ++i) acc[i] = T(0);
  if (row < ld) {
    int k = kg;
    for (; k + 7 * KG < kmax; k += 8 * KG) {
      typename VT::V v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = VT::load(P + row + (size_t)(k + KG * u) * ld);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T f = fs[k + KG * u];
#pragma unroll
        for (int i = 0; i < VN; ++i) acc[i] += VT::get(v[u], i) * f;
      }
    }
    for (; k < kmax; k += KG) {
      typename VT::V v0 = VT::load(P + row + (size_t)k * ld);
      const T f0 = fs[k];
#pragma unroll
      for (int i = 0; i < VN; ++i) acc[i] += VT::get(v0, i) * f0;
    }
  }
#pragma unroll
  for (int i = 0; i < VN; ++i) red[kg * TMV + VN * rg + i] = acc[i];
  __syncthreads();
  if (tid < TMV) {
    const int r = r0 + tid;
    if (r < r1) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < KG; ++q) v += red[q * TMV + tid];
      if (r < w) {
        Y[first + r] = v;
      } else {
        const T g = kmax <= ST - TMV ? gb[tid] : front_rhs<T>(c, B, U, J, r, 0, false);
        U[c.f.sn_upd[J] + r - w] = g - v;
      }
    }
  }
}

// Backward tile: vec_cols consecutive panel columns, a warp per column in turn, over one
// gathered front vector; a lane keeps up to 4 vector loads of its column in flight.
template <typename T>
__device__ void vec_bwd_tile(const SweepCtx &c, const T *panel, const T *Y, T *X, int J, int c0,
                             T *sm) {
  using VT = Vec<T>;
  constexpr int VN = VT::N, STEP = 32 * VN;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J];
  const T *P = panel + c.f.sn_panel[J];
  const int kbeg = c0 & ~(VN - 1);
  T *g = sm;  // [ld]
  const int tid = threadIdx.x;
  for (int kb = kbeg + tid; kb < ld; kb += 3 * ST) {  // indices, then values, in flight
    int64_t row[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int k = kb + q * ST;
      row[q] = k < w ? (int64_t)(first + k) : k < m ? (int64_t)c.f.rows[rp + k] : -1;
    }
    T v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int k = kb + q * ST;
      v[q] = row[q] < 0 ? T(0) : k < w ? __ldcg(&Y[row[q]]) : -__ldcg(&X[row[q]]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (kb + q * ST < ld) g[kb + q * ST] = v[q];
  }
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5;
  const int c1 = min(c0 + c.p.vec_cols, w);
  for (int col = c0 + wid; col < c1; col += ST / 32) {  // the gathered g serves every column
    const T *Pc = P + (size_t)col * ld;
    const int ks = col & ~(VN - 1);
    T acc = T(0);
    int k = ks + VN * lane;
    for (; k + 3 * STEP < ld; k += 4 * STEP) {
      typename VT::V v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = VT::load(Pc + k + u * STEP);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int i = 0; i < VN; ++i) acc += VT::get(v[u], i) * g[k + u * STEP + i];
    }
    for (; k < ld; k += STEP) {
      typename VT::V v = VT::load(Pc + k);
#pragma unroll
      for (int i = 0; i < VN; ++i) acc += VT::get(v, i) * g[k + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) X[first + col] = acc;
  }
}

// a warp processes one small supernode (m <= 96, w <= 32)
template <typename T>
__device__ void vec_fwd_small(const SweepCtx &c, const T *panel, const T *B, T *Y, T *U, int J) {
  const int lane = threadIdx.x & 31;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const T *P = panel + c.f.sn_panel[J];
  // f_top entry of row lane (< w) and the update-row gathers of rows lane + 32 q (>= w)
  int pos[3];
  T gv[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int r = lane + 32 * q;
    pos[q] = r < m ? r : -1;
    gv[q] = (r < w && B) ? B[first + r] : T(0);
  }
  gather_rows<T, 3>(c, U, c.f.sn_rowptr[J], pos, gv, 0);
  const T fk = lane < w ? gv[0] : T(0);
  T acc[3] = {T(0), T(0), T(0)};
  for (int k0 = 0; k0 < w; k0 += 8) {  // 8 x 3 independent loads in flight per lane
    T v[3][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int r = lane + 32 * q;
        v[q][u] = (k0 + u < w && r < m) ? __ldg(&P[r + (size_t)(k0 + u) * ld]) : T(0);
      }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T f = __shfl_sync(0xffffffffu, fk, (k0 + u) & 31);
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[q] += v[q][u] * f;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int r = lane + 32 * q;
    if (r >= m) continue;
    if (r < w) Y[first + r] = acc[q];
    else U[c.f.sn_upd[J] + r - w] = gv[q] - acc[q];
  }
}

template <typename T>
__device__ void vec_bwd_small(const SweepCtx &c, const T *panel, const T *Y, T *X, int J,
                              T *tile /* [32][33] of this warp */) {
  const int lane = threadIdx.x & 31;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J];
  const T *P = panel + c.f.sn_panel[J];
  T acc = T(0);
  for (int kb = 0; kb < m; kb += 32) {
    const int k = kb + lane;
    T gk = T(0);
    if (k < w) gk = __ldcg(&Y[first + k]);
    else if (k < m) gk = -__ldcg(&X[c.f.rows[rp + k]]);
    for (int c0 = 0; c0 < w; c0 += 8) {  // 8 independent loads in flight per lane
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (k < m && c0 + u < w) ? __ldg(&P[k + (size_t)(c0 + u) * ld]) : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + u < w) tile[lane * 33 + c0 + u] = v[u];
    }
    __syncwarp();
    const int kn = min(32, m - kb);
    for (int kk = 0; kk < kn; ++kk) {
      const T gv = __shfl_sync(0xffffffffu, gk, kk);
      if (lane < w) acc += tile[kk * 33 + lane] * gv;
    }
    __syncwarp();
  }
  if (lane < w) X[first + lane] = acc;
}

// ---------------------------------------------------------------- block items (s > 1)
template <int TC, int CM, int RM>
struct Cfg {
  static constexpr int TR = ST / TC;
  static constexpr int TM = TR * RM;
  static constexpr int NCP = TC * CM;
};

// acc += As[0:kc, rows of this thread]^T Bs[0:kc, columns of this thread] (unrolled by 4:
// full unrolling of every chunk made the kernel too large for the instruction cache).
template <typename T, int TC, int CM, int RM>
__device__ __forceinline__ void mac_chunk(const T *As, const T *Bs, int tc, int tr, int kc,
                                          T (&acc)[RM][CM]) {
  using C = Cfg<TC, CM, RM>;
  constexpr int TM = C::TM, NCP = C::NCP;
  auto step = [&](int k) {
    T a[RM], b[CM];
#pragma unroll
    for (int i = 0; i < RM; ++i) a[i] = As[k * (TM + 1) + tr * RM + i];
#pragma unroll
    for (int j = 0; j < CM; ++j) b[j] = Bs[k * NCP + tc + TC * j];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < CM; ++j) acc[i][j] += a[i] * b[j];
  };
#pragma unroll 4
  for (int k = 0; k < kc; ++k) step(k);
}

// Staging of one K chunk. In-order issue stalls a thread at the first use of a load, so
// every staging step first issues all its independent loads into registers and only then
// writes shared memory: the panel tile (NA values per thread), and the right-hand-side rows
// of a warp (RB rows x CPW columns per lane; row indices, first gather sources, values in
// three waves). Sums are formed in the same order as one row at a time would.
template <typename T, int TM>
__device__ __forceinline__ void stage_panel_fwd(const T *P, int ld, int m, int r0, int k0, int kc,
                                                T *As) {
  constexpr int NA = (TK * TM + ST - 1) / ST;
  T av[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int i = threadIdx.x + q * ST, r = i % TM, k = i / TM;
    av[q] = (k < kc && r0 + r < m) ? __ldg(&P[(size_t)(r0 + r) + (size_t)(k0 + k) * ld]) : T(0);
  }
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int i = threadIdx.x + q * ST, r = i % TM, k = i / TM;
    if (k < kc) As[k * (TM + 1) + r] = av[q];
  }
}

template <typename T, int TM>
__device__ __forceinline__ void stage_panel_bwd(const T *P, int ld, int r0, int r1, int k0, int kc,
                                                T *As) {
  constexpr int NA = (TK * TM + ST - 1) / ST;
  T av[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int i = threadIdx.x + q * ST, k = i % TK, r = i / TK;
    av[q] = (k < kc && r0 + r < r1) ? __ldg(&P[(size_t)(k0 + k) + (size_t)(r0 + r) * ld]) : T(0);
  }
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int i = threadIdx.x + q * ST, k = i % TK, r = i / TK;
    if (k < kc) As[k * (TM + 1) + r] = av[q];
  }
}

// f rows k0 + [0, kc) of supernode J: b + the children's update rows landing there
template <typename T, int NCP>
__device__ __forceinline__ void stage_f(const SweepCtx &c, const T *B, const T *U, int64_t rp,
                                        int first, int k0, int kc, T *Bs) {
  constexpr int NW = ST / 32, CPW = (NCP + 31) / 32, RB = CPW >= 8 ? 2 : 24 / CPW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int s = c.s;
  for (int kb = wid; kb < kc; kb += NW * RB) {
    int32_t e0[RB], e1[RB];
    T v[RB][CPW];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int k = kb + q * NW;
      const bool on = k < kc;
      e0[q] = on ? (int32_t)c.f.gptr[rp + k0 + k] : 0;
      e1[q] = on ? (int32_t)c.f.gptr[rp + k0 + k + 1] : 0;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int col = lane + 32 * j;
        v[q][j] = (on && B && col < s) ? B[(size_t)(first + k0 + k) * s + col] : T(0);
      }
    }
    int64_t src[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) src[q] = e0[q] < e1[q] ? c.f.gsrc[e0[q]] : -1;
#pragma unroll
    for (int q = 0; q < RB; ++q)
      if (src[q] >= 0) {
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int col = lane + 32 * j;
          if (col < s) v[q][j] += __ldcg(&U[(size_t)src[q] * s + col]);
        }
      }
#pragma unroll
    for (int q = 0; q < RB; ++q)
      for (int e = e0[q] + 1; e < e1[q]; ++e) {
        const int64_t sr = c.f.gsrc[e];
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int col = lane + 32 * j;
          if (col < s) v[q][j] += __ldcg(&U[(size_t)sr * s + col]);
        }
      }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int k = kb + q * NW;
      if (k < kc) {
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int col = lane + 32 * j;
          if (col < NCP) Bs[k * NCP + col] = v[q][j];
        }
      }
    }
  }
}

// g rows k0 + [0, kc) of supernode J for the backward sweep: y of its own rows, -x below
template <typename T, int NCP>
__device__ __forceinline__ void stage_g(const SweepCtx &c, const T *Y, const T *X, int64_t rp,
                                        int first, int w, int k0, int kc, T *Bs) {
  constexpr int NW = ST / 32, CPW = (NCP + 31) / 32, RB = CPW >= 8 ? 2 : 24 / CPW;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int s = c.s;
  for (int kb = wid; kb < kc; kb += NW * RB) {
    int64_t row[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int k = kb + q * NW, kk = k0 + k;
      row[q] = k >= kc ? -1 : kk < w ? (int64_t)(first + kk) : (int64_t)c.f.rows[rp + kk];
    }
    T v[RB][CPW];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int kk = k0 + kb + q * NW;
      const T *src = kk < w ? Y : X;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int col = lane + 32 * j;
        v[q][j] = (row[q] >= 0 && col < s) ? __ldcg(&src[(size_t)row[q] * s + col]) : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const int k = kb + q * NW;
      if (k < kc) {
        const T sg = k0 + k < w ? T(1) : T(-1);
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int col = lane + 32 * j;
          if (col < NCP) Bs[k * NCP + col] = sg * v[q][j];
        }
      }
    }
  }
}

// Forward tile: rows [r0, r0 + TM) of supernode J, all s columns, K = panel columns.
template <typename T, int TC, int CM, int RM>
__device__ void blk_fwd_tile(const SweepCtx &c, const T *__restrict__ panel, const T *B, T *Y,
                             T *U, int J, int r0, T *sm) {
  using C = Cfg<TC, CM, RM>;
  constexpr int TM = C::TM, NCP = C::NCP;
  static_assert((TM & (TM - 1)) == 0, "tile rows must be a power of two");
  T *As = sm;                  // [TK][TM + 1]
  T *Bs = As + TK * (TM + 1);  // [TK][NCP]
  const int s = c.s;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J];
  const T *P = panel + c.f.sn_panel[J];
  const int r1 = min(r0 + TM, m);
  const int kmax = (r1 <= w) ? r1 : w;
  const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
  T acc[RM][CM];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < kmax; k0 += TK) {
    const int kc = min(TK, kmax - k0);
    stage_panel_fwd<T, TM>(P, ld, m, r0, k0, kc, As);
    stage_f<T, NCP>(c, B, U, rp, first, k0, kc, Bs);
    __syncthreads();
    if (r0 + tr * RM < r1) mac_chunk<T, TC, CM, RM>(As, Bs, tc, tr, kc, acc);
    __syncthreads();
  }
  // epilogue: y rows, or update rows u = f_bot - P_bot f_top (gathers of the thread's rows
  // issued together)
  const int64_t upd = c.f.sn_upd[J];
  int32_t e0[RM], e1[RM];
  int64_t src[RM];
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + tr * RM + i;
    const bool bot = r < r1 && r >= w;
    e0[i] = bot ? (int32_t)c.f.gptr[rp + r] : 0;
    e1[i] = bot ? (int32_t)c.f.gptr[rp + r + 1] : 0;
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) src[i] = e0[i] < e1[i] ? c.f.gsrc[e0[i]] : -1;
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + tr * RM + i;
    if (r >= r1) continue;
    if (r < w) {
#pragma unroll
      for (int j = 0; j < CM; ++j) {
        const int col = tc + TC * j;
        if (col < s) Y[(size_t)(first + r) * s + col] = acc[i][j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < CM; ++j) {
        const int col = tc + TC * j;
        if (col < s) {
          T v = src[i] >= 0 ? __ldcg(&U[(size_t)src[i] * s + col]) : T(0);
          for (int e = e0[i] + 1; e < e1[i]; ++e) v += __ldcg(&U[(size_t)c.f.gsrc[e] * s + col]);
          U[(size_t)(upd + r - w) * s + col] = v - acc[i][j];
        }
      }
    }
  }
}

// Backward tile: x rows [r0, r0 + TM) of supernode J (rows of its own columns), all s
// columns, K over the m front positions.
template <typename T, int TC, int CM, int RM>
__device__ void blk_bwd_tile(const SweepCtx &c, const T *__restrict__ panel, const T *Y, T *X,
                             int J, int r0, T *sm) {
  using C = Cfg<TC, CM, RM>;
  constexpr int TM = C::TM, NCP = C::NCP;
  T *As = sm;
  T *Bs = As + TK * (TM + 1);
  const int s = c.s;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J];
  const T *P = panel + c.f.sn_panel[J];
  const int r1 = min(r0 + TM, w);
  const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
  T acc[RM][CM];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < CM; ++j) acc[i][j] = T(0);
  for (int k0 = r0; k0 < m; k0 += TK) {
    const int kc = min(TK, m - k0);
    stage_panel_bwd<T, TM>(P, ld, r0, r1, k0, kc, As);
    stage_g<T, NCP>(c, Y, X, rp, first, w, k0, kc, Bs);
    __syncthreads();
    if (r0 + tr * RM < r1) mac_chunk<T, TC, CM, RM>(As, Bs, tc, tr, kc, acc);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int r = r0 + tr * RM + i;
    if (r >= r1) continue;
#pragma unroll
    for (int j = 0; j < CM; ++j) {
      const int col = tc + TC * j;
      if (col < s) X[(size_t)(first + r) * s + col] = acc[i][j];
    }
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
