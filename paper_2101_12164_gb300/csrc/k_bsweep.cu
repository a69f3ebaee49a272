// Multi-right-hand-side supernodal sweeps X = A_b^{-1} B (s > 1) by blocks and column slices:
// one CTA per (block b, slice of kBsmCols columns) of a forest, no dependency waits. The
// interior blocks A_1..A_N of §2.3 eq. (perm_A) are independent and so are the columns of B,
// so a CTA runs both triangular sweeps of its block on its columns alone, tree height by tree
// height, with a barrier between heights. Same formulas as k_solve.cu (panels P_J = [inv(L11);
// L21 inv(L11)]; forward y_J = P_top f_top, u_J = f_bot - P_bot f_top with f = b + the
// children's update rows; backward x_J = P_top^T y_J - P_bot^T x[rows below]); the update rows
// U, the intermediate Y and X stay in global memory (n x s and update rows x s, row-major).
//
// The plan cuts every height of every block into batches whose fronts fit the shared-memory
// scratch (front positions x kBsmCols); a batch runs as flat loops over all of its supernodes:
//   forward:  (A) every front f (positions x slice columns) gathered into scratch from B and
//             the children's update rows, from precomputed per-position source lists;
//             (B) one unit per (4-row group, 8-column group) of each panel: the product with
//             f_top from scratch, written to Y (rows < w) or U (f_bot - product);
//   backward: (A) g = [y_J; -x(rows below)] for every supernode into scratch;
//             (B) one unit per (4 panel columns, 8 slice columns): P[:, cols]^T g, to X.
// half = 1 runs the forward sweep alone (Y = L^{-1} B), half = 2 the backward sweep alone
// (X = L^{-T} Y). Every K loop sums sequentially; the columns of a slice never meet another CTA's, the rows
// of a block never another block's, and a CTA reads its own global writes of an earlier
// height only after a barrier.
#include "sweep_tiles.cuh"

namespace nsp {
namespace {

constexpr int BT = 512;                 // threads per CTA
constexpr int BCS = kBsmCols;           // columns per slice (32)
constexpr int BCQ = BCS / 4;            // column quads per position

// item record: {front offset, first forward unit, first backward unit, m},
//              {w, first row, first update row, 0}, {sn_panel low, high, 0, 0}
struct BsItem {
  int fo, uf, ub, m, w, first, upd;
  int64_t po;
  __device__ void load(const int4 *items, int i) {   // the batch's shared-memory copy
    const int4 a = items[3 * i], b = items[3 * i + 1], c = items[3 * i + 2];
    fo = a.x; uf = a.y; ub = a.z; m = a.w;
    w = b.x; first = b.y; upd = b.z;
    po = (int64_t)(uint32_t)c.x | ((int64_t)c.y << 32);
  }
};

// Shared-memory copies of a batch's plan data (item records, per-position data, unit items,
// gather sources), staged once at the start of the batch in one round of loads.
constexpr int kMetaPos = 1536 + 16;                       // positions (+1), padded
constexpr int kMetaUnits = 1536 + 3 * kBsmMaxItems + 16;  // forward or backward units
struct BsMeta {
  int4 *items;       // 3 x kBsmMaxItems
  int32_t *pptr;     // kMetaPos: gather-source offsets, relative to the batch's first source
  int32_t *pvi;      // kMetaPos: B / Y / X rows
  uint16_t *uit;     // kMetaUnits: item (relative) of each unit
  int32_t *psrc;     // kBsmMaxSources
};
constexpr size_t kMetaBytes =
    16 * 3 * kBsmMaxItems + 4 * 2 * kMetaPos + 2 * kMetaUnits + 4 * kBsmMaxSources;
static_assert(kMetaPos > kBsmScratchBytes / (kBsmCols * 4), "a batch's positions (+1) fit");
static_assert(kMetaUnits >= kBsmScratchBytes / (kBsmCols * 4), "a batch's units fit");
static_assert(kBsmScratchBytes + 16 + kMetaBytes <= 227 * 1024, "fronts + plan data fit");
__device__ __forceinline__ BsMeta meta_at(unsigned char *base) {
  BsMeta M;
  M.items = reinterpret_cast<int4 *>(base);
  M.pptr = reinterpret_cast<int32_t *>(M.items + 3 * kBsmMaxItems);
  M.pvi = M.pptr + kMetaPos;
  M.psrc = M.pvi + kMetaPos;
  M.uit = reinterpret_cast<uint16_t *>(M.psrc + kBsmMaxSources);
  return M;
}

// every load of the staging issued before any shared-memory store
__device__ __forceinline__ void bs_stage_meta(const BsMeta &M, const int4 *items, int i0, int ni,
                                              const int32_t *pptr, const int32_t *pvi, int pb,
                                              int nf, const uint16_t *uit, int ubase, int nu,
                                              const int32_t *psrc, int sb, int nsrc) {
  const int tid = threadIdx.x;
  constexpr int KP = (kMetaPos + BT - 1) / BT, KU = (kMetaUnits + BT - 1) / BT,
                KS = (kBsmMaxSources + BT - 1) / BT;
  static_assert(3 * kBsmMaxItems <= BT, "one item word per thread");
  const int4 it = tid < 3 * ni ? __ldg(&items[3 * i0 + tid]) : make_int4(0, 0, 0, 0);
  int32_t vp[KP], vv[KP], vs[KS];
  uint16_t vu[KU];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int j = tid + k * BT;
    vp[k] = (pptr && j <= nf) ? __ldg(&pptr[pb + j]) : 0;
    vv[k] = j < nf ? __ldg(&pvi[pb + j]) : 0;
  }
#pragma unroll
  for (int k = 0; k < KU; ++k) {
    const int j = tid + k * BT;
    vu[k] = j < nu ? __ldg(&uit[ubase + j]) : (uint16_t)0;
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int j = tid + k * BT;
    vs[k] = j < nsrc ? __ldg(&psrc[sb + j]) : 0;
  }
  if (tid < 3 * ni) M.items[tid] = it;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int j = tid + k * BT;
    if (pptr && j <= nf) M.pptr[j] = vp[k] - sb;
    if (j < nf) M.pvi[j] = vv[k];
  }
#pragma unroll
  for (int k = 0; k < KU; ++k) {
    const int j = tid + k * BT;
    if (j < nu) M.uit[j] = vu[k];
  }
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const int j = tid + k * BT;
    if (j < nsrc) M.psrc[j] = vs[k];
  }
  __syncthreads();
}

template <typename T>
struct V4;
template <>
struct V4<float> {
  float a[4];
  __device__ void ld(const float *p) {       // global, read-only path
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
  __device__ void ldcg(const float *p) {     // global, written earlier by this launch
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
  __device__ void lds(const float *p) {      // shared
    const float4 t = *reinterpret_cast<const float4 *>(p);
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
  __device__ void st(float *p) const {
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
  }
};
template <>
struct V4<double> {
  double a[4];
  __device__ void ld(const double *p) {
    const double2 t0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 t1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
  }
  __device__ void ldcg(const double *p) {
    const double2 t0 = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 t1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
  }
  __device__ void lds(const double *p) {
    const double2 t0 = *reinterpret_cast<const double2 *>(p);
    const double2 t1 = *(reinterpret_cast<const double2 *>(p) + 1);
    a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
  }
  __device__ void st(double *p) const {
    reinterpret_cast<double2 *>(p)[0] = make_double2(a[0], a[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(a[2], a[3]);
  }
};

constexpr int BNR = 8;   // position quads per thread in flight in the gathers

template <typename T>
__device__ void bs_forward(const SweepPlan &p, const T *panel, const T *B, T *Y, T *U, int s,
                           int c0, int ncq, T *fs, const BsMeta &M, int q) {
  const int4 B0 = __ldg(&p.bs_bat[3 * q]), B1 = __ldg(&p.bs_bat[3 * q + 1]),
             B2 = __ldg(&p.bs_bat[3 * q + 2]);
  const int i0 = B0.x, nf = B0.z, nu = B0.w, pb = B1.z, ubase = B1.w;
  const int tid = threadIdx.x;
  bs_stage_meta(M, p.bs_item, i0, B0.y - i0, p.bs_pptr, p.bs_pfvi, pb, nf, p.bs_uitem, ubase, nu,
                p.bs_psrc, B2.y, B2.z);
  // (A) fronts: flat over (position, column quad), BNR in flight per thread
  const int nt = nf * BCQ;
  for (int t0 = tid; t0 < nt; t0 += BNR * BT) {
    int32_t e[BNR], ee[BNR];
    V4<T> val[BNR];
#pragma unroll
    for (int h = 0; h < BNR; ++h) {
      const int t = t0 + h * BT, pp = t / BCQ, cq = t - pp * BCQ;
      e[h] = ee[h] = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) val[h].a[i] = T(0);
      if (t < nt && cq < ncq) {
        e[h] = M.pptr[pp];
        ee[h] = M.pptr[pp + 1];
        const int row = M.pvi[pp];
        if (row >= 0) val[h].ld(B + (size_t)row * s + c0 + 4 * cq);
      }
    }
    bool more = true;
    while (more) {
      int32_t src[BNR];
#pragma unroll
      for (int h = 0; h < BNR; ++h) src[h] = e[h] < ee[h] ? M.psrc[e[h]] : -1;
      more = false;
#pragma unroll
      for (int h = 0; h < BNR; ++h)
        if (src[h] >= 0) {
          const int t = t0 + h * BT, cq = t - (t / BCQ) * BCQ;
          V4<T> u;
          u.ldcg(U + (size_t)src[h] * s + c0 + 4 * cq);
#pragma unroll
          for (int i = 0; i < 4; ++i) val[h].a[i] += u.a[i];
          more |= ++e[h] < ee[h];
        }
    }
#pragma unroll
    for (int h = 0; h < BNR; ++h) {
      const int t = t0 + h * BT;
      if (t < nt) val[h].st(fs + (size_t)t * 4);
    }
  }
  __syncthreads();
  // (B) products: unit = (item, 4-row group, 8-column group); the 4 column groups of a row
  // group are consecutive units
  for (int u = tid; u < nu; u += BT) {
    BsItem I;
    I.load(M.items, M.uit[u]);
    const int lu = u - I.uf, rg = lu >> 2, cg = lu & 3;
    if (2 * cg >= ncq) continue;   // beyond the slice's last column
    const int w = I.w, m = I.m, ld = (m + 3) & ~3, row = 4 * rg;
    const int kmax = min(w, row + 4);
    const T *P = panel + I.po + row;
    const T *F = fs + (size_t)I.fo * BCS + 8 * cg;
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    int k = 0;
    if constexpr (sizeof(T) == 4) {
      // eight panel rows of K in flight as a ring: each is reloaded for the next chunk of
      // eight as soon as its products are issued, so the loads overlap the FMAs
      const int kfull = kmax & ~7;
      V4<T> pv[8];
      if (kfull > 0) {
#pragma unroll
        for (int t = 0; t < 8; ++t) pv[t].ld(P + (size_t)t * ld);
      }
      for (; k < kfull; k += 8) {
        const bool more = k + 8 < kfull;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          V4<T> f0, f1;
          f0.lds(F + (size_t)(k + t) * BCS);
          f1.lds(F + (size_t)(k + t) * BCS + 4);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              acc[i][j] += pv[t].a[i] * f0.a[j];
              acc[i][4 + j] += pv[t].a[i] * f1.a[j];
            }
          if (more) pv[t].ld(P + (size_t)(k + 8 + t) * ld);
        }
      }
    } else {   // FP64: the ring needs more registers than 128 (spills); chunks of eight
      for (; k + 7 < kmax; k += 8) {
        V4<T> pv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) pv[t].ld(P + (size_t)(k + t) * ld);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          V4<T> f0, f1;
          f0.lds(F + (size_t)(k + t) * BCS);
          f1.lds(F + (size_t)(k + t) * BCS + 4);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              acc[i][j] += pv[t].a[i] * f0.a[j];
              acc[i][4 + j] += pv[t].a[i] * f1.a[j];
            }
        }
      }
    }
    for (; k < kmax; ++k) {
      V4<T> pk, f0, f1;
      pk.ld(P + (size_t)k * ld);
      f0.lds(F + (size_t)k * BCS);
      f1.lds(F + (size_t)k * BCS + 4);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] += pk.a[i] * f0.a[j];
          acc[i][4 + j] += pk.a[i] * f1.a[j];
        }
    }
    const bool two = 2 * cg + 1 < ncq;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = row + i;
      if (r >= m) break;
      V4<T> o0, o1;
      if (r < w) {
#pragma unroll
        for (int j = 0; j < 4; ++j) { o0.a[j] = acc[i][j]; o1.a[j] = acc[i][4 + j]; }
        T *dst = Y + (size_t)(I.first + r) * s + c0 + 8 * cg;
        o0.st(dst);
        if (two) o1.st(dst + 4);
      } else {
        V4<T> f0, f1;
        f0.lds(F + (size_t)r * BCS);
        f1.lds(F + (size_t)r * BCS + 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          o0.a[j] = f0.a[j] - acc[i][j];
          o1.a[j] = f1.a[j] - acc[i][4 + j];
        }
        T *dst = U + (size_t)(I.upd + r - w) * s + c0 + 8 * cg;
        o0.st(dst);
        if (two) o1.st(dst + 4);
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void bs_backward(const SweepPlan &p, const T *panel, const T *Y, T *X, int s, int c0,
                            int ncq, T *gs, const BsMeta &M, int q) {
  const int4 B0 = __ldg(&p.bs_bat[3 * q]), B1 = __ldg(&p.bs_bat[3 * q + 1]),
             B2 = __ldg(&p.bs_bat[3 * q + 2]);
  const int i0 = B0.x, nf = B0.z, nc = B1.x, pb = B1.z, cbase = B2.x;
  const int tid = threadIdx.x;
  bs_stage_meta(M, p.bs_item, i0, B0.y - i0, nullptr, p.bs_pbvi, pb, nf, p.bs_citem, cbase, nc,
                p.bs_psrc, 0, 0);
  // (A) g = [y_J; -x(rows below); 0 padding], flat over (position, column quad)
  const int nt = nf * BCQ;
  for (int t0 = tid; t0 < nt; t0 += BNR * BT) {
    V4<T> val[BNR];
#pragma unroll
    for (int h = 0; h < BNR; ++h) {
      const int t = t0 + h * BT, pp = t / BCQ, cq = t - pp * BCQ;
#pragma unroll
      for (int i = 0; i < 4; ++i) val[h].a[i] = T(0);
      if (t < nt && cq < ncq) {
        const int vi = M.pvi[pp];
        if (vi >= 0) {
          val[h].ldcg(Y + (size_t)vi * s + c0 + 4 * cq);
        } else if (vi < -1) {
          val[h].ldcg(X + (size_t)(-2 - vi) * s + c0 + 4 * cq);
#pragma unroll
          for (int i = 0; i < 4; ++i) val[h].a[i] = -val[h].a[i];
        }
      }
    }
#pragma unroll
    for (int h = 0; h < BNR; ++h) {
      const int t = t0 + h * BT;
      if (t < nt) val[h].st(gs + (size_t)t * 4);
    }
  }
  __syncthreads();
  // (B) unit = (item, 4 panel columns, 8 slice columns): x[cols] = P[:, cols]^T g
  for (int u = tid; u < nc; u += BT) {
    BsItem I;
    I.load(M.items, M.uit[u]);
    const int lu = u - I.ub, qg = lu >> 2, cg = lu & 3;
    if (2 * cg >= ncq) continue;
    const int w = I.w, ld = (I.m + 3) & ~3, col = 4 * qg;
    const int ncol = min(4, w - col);
    const T *Pc = panel + I.po + (size_t)col * ld;
    const T *G = gs + (size_t)I.fo * BCS + 8 * cg;
    T acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    if constexpr (sizeof(T) == 4) {
      // P_top is lower triangular: rows >= col. Eight rows of the four columns in flight as a
      // ring of two quads per column: a quad is reloaded for the next chunk of eight rows as
      // soon as its products are issued
      V4<T> pc[8];
      {
        const bool hi = col + 4 < ld;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < ncol) {
            pc[i].ld(Pc + (size_t)i * ld + col);
            if (hi) pc[4 + i].ld(Pc + (size_t)i * ld + col + 4);
          }
      }
      for (int k = col; k < ld; k += 8) {
        const bool hi = k + 4 < ld, more = k + 8 < ld, more_hi = k + 12 < ld;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !hi) break;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            V4<T> g0, g1;
            g0.lds(G + (size_t)(k + 4 * h + t) * BCS);
            g1.lds(G + (size_t)(k + 4 * h + t) * BCS + 4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (i < ncol)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  const T pk = pc[4 * h + i].a[t];
                  acc[i][j] += pk * g0.a[j];
                  acc[i][4 + j] += pk * g1.a[j];
                }
          }
          if (h == 0 ? more : more_hi) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (i < ncol) pc[4 * h + i].ld(Pc + (size_t)i * ld + k + 8 + 4 * h);
          }
        }
      }
    } else {   // FP64: chunks of eight rows (the ring spills at 128 registers)
      for (int k = col; k < ld; k += 8) {
        const bool hi = k + 4 < ld;
        V4<T> pc[8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < ncol) {
            pc[i].ld(Pc + (size_t)i * ld + k);
            if (hi) pc[4 + i].ld(Pc + (size_t)i * ld + k + 4);
          }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (t >= 4 && !hi) break;
          V4<T> g0, g1;
          g0.lds(G + (size_t)(k + t) * BCS);
          g1.lds(G + (size_t)(k + t) * BCS + 4);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (i < ncol)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const T pk = pc[(t >> 2) * 4 + i].a[t & 3];
                acc[i][j] += pk * g0.a[j];
                acc[i][4 + j] += pk * g1.a[j];
              }
        }
      }
    }
    const bool two = 2 * cg + 1 < ncq;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= ncol) break;
      V4<T> o0, o1;
#pragma unroll
      for (int j = 0; j < 4; ++j) { o0.a[j] = acc[i][j]; o1.a[j] = acc[i][4 + j]; }
      T *dst = X + (size_t)(I.first + col + i) * s + c0 + 8 * cg;
      o0.st(dst);
      if (two) o1.st(dst + 4);
    }
  }
  __syncthreads();
}

// CTA = (block, column slice); shared memory: the batch scratch (positions x kBsmCols), then
// the batch's plan data (BsMeta)
template <typename T>
__global__ void __launch_bounds__(BT, 1)
    k_bsm_sweep(SweepPlan p, const T *__restrict__ panel, const T *B, T *Y, T *U, T *X, int s,
                int nslices, int half) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *scr = reinterpret_cast<T *>(smem_raw);
  const BsMeta M = meta_at(smem_raw + (((size_t)p.bs_positions * BCS * sizeof(T) + 15) & ~(size_t)15));
  const int b = blockIdx.x / nslices, sl = blockIdx.x - b * nslices;
  const int c0 = sl * BCS, ncq = min(BCS, s - c0) / 4;
  const int L0 = p.bs_lvl_ptr[b], L1 = p.bs_lvl_ptr[b + 1];
  for (int L = L0; L < L1 && half != 2; ++L)
    for (int q = p.bs_bat_ptr[L]; q < p.bs_bat_ptr[L + 1]; ++q)
      bs_forward<T>(p, panel, B, Y, U, s, c0, ncq, scr, M, q);
  for (int L = L1 - 1; L >= L0 && half != 1; --L)
    for (int q = p.bs_bat_ptr[L]; q < p.bs_bat_ptr[L + 1]; ++q)
      bs_backward<T>(p, panel, Y, X, s, c0, ncq, scr, M, q);
}

}  // namespace

template <typename T>
bool bsm_sweep_fits(const SweepPlan &p, int s) {
  return p.bs_item && !p.vector && s > 1 && s % 4 == 0 && p.bs_positions > 0 &&
         (size_t)p.bs_positions * BCS * sizeof(T) <= (size_t)kBsmScratchBytes;
}

template <typename T>
void launch_bsm_sweep(const SweepPlan &p, const T *panel, const T *B, T *Y, T *U, T *X, int s,
                      cudaStream_t stream, int half) {
  require(bsm_sweep_fits<T>(p, s), NSP_ERR_INVALID_ARG,
          "column-sliced block sweep: no plan for this width");
  require(half >= 0 && half <= 2, NSP_ERR_INVALID_ARG, "column-sliced block sweep: bad half");
  const int nslices = (s + BCS - 1) / BCS;
  const size_t smem = (((size_t)p.bs_positions * BCS * sizeof(T) + 15) & ~(size_t)15) + kMetaBytes;
  static size_t attr = 0;
  if (smem > attr) {
    ensure_dyn_smem(k_bsm_sweep<T>, smem);
    attr = smem;
  }
  k_bsm_sweep<T><<<p.res_nblocks * nslices, BT, smem, stream>>>(p, panel, B, Y, U, X, s, nslices,
                                                                  half);
  NSP_LAUNCH_CHECK();
}

template bool bsm_sweep_fits<float>(const SweepPlan &, int);
template bool bsm_sweep_fits<double>(const SweepPlan &, int);
template void launch_bsm_sweep<float>(const SweepPlan &, const float *, const float *, float *,
                                      float *, float *, int, cudaStream_t, int);
template void launch_bsm_sweep<double>(const SweepPlan &, const double *, const double *,
                                       double *, double *, double *, int, cudaStream_t, int);

}  // namespace nsp
