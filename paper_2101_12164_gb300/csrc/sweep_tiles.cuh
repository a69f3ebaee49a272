// Device building blocks of the supernodal triangular sweeps, shared by the two sweep
// schedulers (k_solve.cu: dependency-driven persistent sweep over a whole forest;
// k_rsweep.cu: one CTA per block of the forest). See k_solve.cu for the panel layout and the
// forward / backward formulas.
#pragma once
#include "kernels.cuh"

namespace nsp {
namespace {

constexpr int ST = 256;      // threads per CTA
constexpr int TK = 64;       // K chunk of the block product

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

}  // namespace
}  // namespace nsp

namespace nsp {
namespace {

// ---------------------------------------------------------------- warp jobs (s > 1)
// One small supernode (w <= kResW, m <= kResM) by one warp, all s columns in passes of
// 32 CPL (lanes own CPL columns each). Every dependent load chain is issued for all rows at
// once: the gather indices of the m front rows (two rounds), then the f_top rows (one
// round), then row chunks of 8 whose panel values are prefetched into registers one chunk
// ahead and whose update-row sources are loaded before the chunk's products.
// Per-warp shared memory: wj_elems<T>() elements of T followed by wj_ints() int32.
template <typename T>
struct WarpCpl {
  static constexpr int value = 2;
};
constexpr int kWjRG = 8;     // panel rows per chunk (forward) / front rows per chunk (backward)
constexpr int kWjIG = 16;    // own rows per group (backward)
template <typename T>
__host__ __device__ constexpr int wj_elems() {
  return kResW * 32 * WarpCpl<T>::value + 2 * kResW * kWjRG;
}
__host__ __device__ constexpr int wj_ints() { return 3 * kResM; }

// eight consecutive values from global memory (read-only path) / from shared memory, with
// 16-byte loads (p 16-byte aligned)
template <typename T>
__device__ __forceinline__ void vec_load8(const T *p, T (&v)[kWjRG]) {
  using VT = Vec<T>;
#pragma unroll
  for (int q = 0; q < kWjRG / VT::N; ++q) {
    const typename VT::V x = VT::load(p + VT::N * q);
#pragma unroll
    for (int i = 0; i < VT::N; ++i) v[VT::N * q + i] = VT::get(x, i);
  }
}
template <typename T>
__device__ __forceinline__ void smem_load8(const T *p, T (&v)[kWjRG]) {
  using VT = Vec<T>;
#pragma unroll
  for (int q = 0; q < kWjRG / VT::N; ++q) {
    const typename VT::V x = reinterpret_cast<const typename VT::V *>(p)[q];
#pragma unroll
    for (int i = 0; i < VT::N; ++i) v[VT::N * q + i] = VT::get(x, i);
  }
}

template <typename T, int CPL>
__device__ void warp_fwd_job(const SweepCtx &c, const T *__restrict__ panel, const T *B, T *Y,
                             T *U, int J, T *ws, int32_t *wi) {
  constexpr int CW = 32 * CPL, RG = kWjRG, NQ = kResM / 32;
  T *fs = ws;                      // [kResW][CW]  f_top of this pass
  T *pan = ws + kResW * CW;        // [2][kResW][RG] panel chunks, 8 rows per panel column
  int32_t *me0 = wi, *me1 = wi + kResM, *msrc = wi + 2 * kResM;
  const int lane = threadIdx.x & 31, s = c.s;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J], upd = c.f.sn_upd[J];
  const T *P = panel + c.f.sn_panel[J];
  {  // gather lists of every front row: [e0, e1) into gsrc, first source
    int32_t e0[NQ], e1[NQ], s0[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      e0[q] = i < m ? (int32_t)c.f.gptr[rp + i] : 0;
      e1[q] = i < m ? (int32_t)c.f.gptr[rp + i + 1] : 0;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) s0[q] = e0[q] < e1[q] ? (int32_t)c.f.gsrc[e0[q]] : -1;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      if (i < m) {
        me0[i] = e0[q];
        me1[i] = e1[q];
        msrc[i] = s0[q];
      }
    }
  }
  __syncwarp();
  for (int c0 = 0; c0 < s; c0 += CW) {
    for (int k0 = 0; k0 < w; k0 += 8) {   // f_top rows, 8 rows' loads in flight
      T v[8][CPL];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        const int src = k < w ? msrc[k] : -1;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int col = c0 + lane + 32 * j;
          const bool on = k < w && col < s;
          v[q][j] = (on && B) ? B[(size_t)(first + k) * s + col] : T(0);
          if (on && src >= 0) v[q][j] += __ldcg(&U[(size_t)src * s + col]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        if (k >= w) break;
        for (int e = me0[k] + 1; e < me1[k]; ++e) {   // further children on this row
          const int64_t sr = c.f.gsrc[e];
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            const int col = c0 + lane + 32 * j;
            if (col < s) v[q][j] += __ldcg(&U[(size_t)sr * s + col]);
          }
        }
#pragma unroll
        for (int j = 0; j < CPL; ++j) fs[k * CW + lane + 32 * j] = v[q][j];
      }
    }
    // panel chunk r0: lane k holds rows r0..r0+7 of panel column k
    auto load_chunk = [&](int r0, T (&pv)[RG]) {
      if (lane < w) {
        const T *src = P + r0 + (size_t)lane * ld;
        if (r0 + RG <= ld) {
          vec_load8<T>(src, pv);
        } else {
#pragma unroll
          for (int i = 0; i < RG; ++i) pv[i] = r0 + i < ld ? __ldg(src + i) : T(0);
        }
      }
    };
    T pv[RG];
#pragma unroll
    for (int i = 0; i < RG; ++i) pv[i] = T(0);
    load_chunk(0, pv);
    __syncwarp();
    for (int r0 = 0, buf = 0; r0 < m; r0 += RG, buf ^= 1) {
      T *pb = pan + buf * kResW * RG;
      if (lane < w) {
#pragma unroll
        for (int i = 0; i < RG; ++i) pb[lane * RG + i] = pv[i];
      }
      __syncwarp();
      if (r0 + RG < m) load_chunk(r0 + RG, pv);   // next chunk in flight during the products
      T g[RG][CPL];
#pragma unroll
      for (int i = 0; i < RG; ++i) {
        const int r = r0 + i;
        const int src = (r >= w && r < m) ? msrc[r] : -1;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int col = c0 + lane + 32 * j;
          g[i][j] = (src >= 0 && col < s) ? __ldcg(&U[(size_t)src * s + col]) : T(0);
        }
      }
      T acc[RG][CPL];
#pragma unroll
      for (int i = 0; i < RG; ++i)
#pragma unroll
        for (int j = 0; j < CPL; ++j) acc[i][j] = T(0);
#pragma unroll 4
      for (int k = 0; k < w; ++k) {
        T p[RG];
        smem_load8<T>(pb + k * RG, p);
        T f[CPL];
#pragma unroll
        for (int j = 0; j < CPL; ++j) f[j] = fs[k * CW + lane + 32 * j];
#pragma unroll
        for (int i = 0; i < RG; ++i)
#pragma unroll
          for (int j = 0; j < CPL; ++j) acc[i][j] += p[i] * f[j];
      }
#pragma unroll
      for (int i = 0; i < RG; ++i) {
        const int r = r0 + i;
        if (r >= m) break;
        if (r >= w)
          for (int e = me0[r] + 1; e < me1[r]; ++e) {   // further children on this row
            const int64_t sr = c.f.gsrc[e];
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
              const int col = c0 + lane + 32 * j;
              if (col < s) g[i][j] += __ldcg(&U[(size_t)sr * s + col]);
            }
          }
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int col = c0 + lane + 32 * j;
          if (col >= s) continue;
          if (r < w) Y[(size_t)(first + r) * s + col] = acc[i][j];
          else U[(size_t)(upd + r - w) * s + col] = g[i][j] - acc[i][j];
        }
      }
    }
    __syncwarp();
  }
}

// Backward step of one small supernode by one warp: x_J = P^T g over the m front rows,
// g = y (own rows) or -x (rows below). Own rows in groups of 16; front rows in chunks of 8,
// the next chunk's g rows and panel values loaded into registers during the current chunk's
// products.
template <typename T, int CPL>
__device__ void warp_bwd_job(const SweepCtx &c, const T *__restrict__ panel, const T *Y, T *X,
                             int J, T *ws, int32_t *wi) {
  constexpr int CW = 32 * CPL, KC = kWjRG, IG = kWjIG, NQ = kResM / 32;
  T *pan = ws;                     // [2][KC][IG]
  int32_t *mrow = wi;              // front row -> global row (rows below the own columns)
  const int lane = threadIdx.x & 31, s = c.s;
  const int w = c.f.sn_w[J], m = c.f.sn_m[J], ld = (m + 3) & ~3;
  const int first = c.f.sn_first[J];
  const int64_t rp = c.f.sn_rowptr[J];
  const T *P = panel + c.f.sn_panel[J];
  {
    int32_t r[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int k = lane + 32 * q;
      r[q] = k < w ? first + k : k < m ? c.f.rows[rp + k] : -1;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (lane + 32 * q < m) mrow[lane + 32 * q] = r[q];
  }
  __syncwarp();
  const int li = lane & (IG - 1), lh = lane / IG;   // panel staging: own row li, k half lh
  for (int c0 = 0; c0 < s; c0 += CW) {
    for (int i0 = 0; i0 < w; i0 += IG) {
      auto load_chunk = [&](int k0, T (&pv)[KC / 2], T (&gv)[KC][CPL]) {
        const int i = i0 + li, kb = k0 + (KC / 2) * lh;
        if (i < w) {
          const T *src = P + kb + (size_t)i * ld;
          if (kb + KC / 2 <= ld) {
            using VT = Vec<T>;
#pragma unroll
            for (int q = 0; q < KC / 2 / VT::N; ++q) {
              const typename VT::V x = VT::load(src + VT::N * q);
#pragma unroll
              for (int t = 0; t < VT::N; ++t) pv[VT::N * q + t] = VT::get(x, t);
            }
          } else {
#pragma unroll
            for (int t = 0; t < KC / 2; ++t) pv[t] = kb + t < ld ? __ldg(src + t) : T(0);
          }
        } else {
#pragma unroll
          for (int t = 0; t < KC / 2; ++t) pv[t] = T(0);
        }
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          const int k = k0 + q;
          const int row = k < m ? mrow[k] : -1;
          const T *gsrc = k < w ? Y : X;
          const T sg = k < w ? T(1) : T(-1);
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            const int col = c0 + lane + 32 * j;
            gv[q][j] = (row >= 0 && col < s) ? sg * __ldcg(&gsrc[(size_t)row * s + col]) : T(0);
          }
        }
      };
      T pv[KC / 2], gv[KC][CPL];
      load_chunk(0, pv, gv);
      T acc[IG][CPL];
#pragma unroll
      for (int i = 0; i < IG; ++i)
#pragma unroll
        for (int j = 0; j < CPL; ++j) acc[i][j] = T(0);
      for (int k0 = 0, buf = 0; k0 < m; k0 += KC, buf ^= 1) {
        T *pb = pan + buf * KC * IG;
#pragma unroll
        for (int t = 0; t < KC / 2; ++t) pb[((KC / 2) * lh + t) * IG + li] = pv[t];
        T gc[KC][CPL];
#pragma unroll
        for (int q = 0; q < KC; ++q)
#pragma unroll
          for (int j = 0; j < CPL; ++j) gc[q][j] = gv[q][j];
        __syncwarp();
        if (k0 + KC < m) load_chunk(k0 + KC, pv, gv);
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          T p[IG];
#pragma unroll
          for (int t = 0; t < IG / kWjRG; ++t) {
            T h[kWjRG];
            smem_load8<T>(pb + q * IG + kWjRG * t, h);
#pragma unroll
            for (int u = 0; u < kWjRG; ++u) p[kWjRG * t + u] = h[u];
          }
#pragma unroll
          for (int i = 0; i < IG; ++i)
#pragma unroll
            for (int j = 0; j < CPL; ++j) acc[i][j] += p[i] * gc[q][j];
        }
      }
#pragma unroll
      for (int i = 0; i < IG; ++i) {
        if (i0 + i >= w) break;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int col = c0 + lane + 32 * j;
          if (col < s) X[(size_t)(first + i0 + i) * s + col] = acc[i][j];
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace
}  // namespace nsp
