// Single-vector supernodal sweeps x = A_b^{-1} b with each block's vectors in shared memory:
// one CTA per block b of a forest (the interior blocks A_1..A_N of §2.3 eq. (perm_A) are
// independent), the block's right-hand side, its intermediate y and its solution x in one
// shared-memory vector v (n_b entries, overwritten in place), and the update rows of its
// supernodes in a shared-memory pool (a supernode's rows hold a slot from its height to its
// parent's). Only the panels and the index metadata come from global memory; b is read and x
// written once, coalesced.
//
// Same formulas as k_solve.cu (panels P_J = [inv(L11); L21 inv(L11)]; forward y_J = P_top
// f_top, u_J = f_bot - P_bot f_top with f = b + the children's update rows; backward x_J =
// P_top^T y_J - P_bot^T x[rows below]). The supernodes of one tree height are independent;
// the plan cuts each height of each block into batches whose fronts fit a scratch area, and
// every batch runs as flat parallel loops over all of its supernodes at once (the plan gives
// every front position its gather sources and v index, and every unit its item record, which
// carries the supernode's sizes and offsets):
//   forward:  (A) gather every front f of the batch into scratch; (B) one unit per (K group,
//             4-row group) of each panel, the product with f, written to v (rows < w) or U
//             (update rows), or, for K-split supernodes, to partial sums after the fronts;
//             (C) the partial sums added in group order and written;
//   backward: (A) g = [y_J; -x(rows below)] for every supernode of the batch; (B) one thread
//             per panel column, x_J[col] = P[:, col]^T g, written in place of y_J.
// A barrier separates the phases; no dependency waits, no global intermediates. Forward
// products with one K group sum K sequentially (as the small single-vector items of
// k_solve.cu), the others in interleaved groups added in group order; backward columns sum
// sequentially over the front.
#include "sweep_tiles.cuh"

namespace nsp {
namespace {

constexpr int VT = 512;            // threads per CTA

// one item record: what a forward unit or backward column needs about its supernode
struct VsItem {
  int fo, ro, kg, us;      // front offset, partial-sum offset, K groups, update-row slot
  int uf, ub, m, w;        // first forward unit, first backward column, rows, columns
  int fl;                  // first row in the block
  int64_t po;              // sn_panel
  __device__ void load(const int4 *items, int i) {
    const int4 a = __ldg(&items[4 * i]), b = __ldg(&items[4 * i + 1]),
               c = __ldg(&items[4 * i + 2]), d = __ldg(&items[4 * i + 3]);
    fo = a.x; ro = a.y; kg = a.z; us = a.w;
    uf = b.x; ub = b.y; m = b.z; w = b.w;
    fl = c.x;
    po = (int64_t)(uint32_t)c.w | ((int64_t)d.x << 32);
  }
};

// four consecutive panel rows at column k (row a multiple of 4, ld a multiple of 4)
template <typename T>
struct Quad;
template <>
struct Quad<float> {
  float a[4];
  __device__ void load(const float *p) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
};
template <>
struct Quad<double> {
  double a[4];
  __device__ void load(const double *p) {
    const double2 t0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 t1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
  }
};

constexpr int VNR = 4;   // front positions per thread in flight (phase A of the forward)

template <typename T>
__device__ void vs_forward(const SweepPlan &p, const T *panel, T *v, T *Us, T *scr, int q) {
  const int4 B0 = __ldg(&p.vs_bat[3 * q]), B1 = __ldg(&p.vs_bat[3 * q + 1]);
  const int i0 = B0.x, nf = B0.z, nu = B0.w, pb = B1.z, ubase = B1.w;
  const int4 *items = p.vs_item;
  T *fs = scr, *red = scr + nf;
  const int tid = threadIdx.x;
  // (A) fronts f = b (top rows) + the children's update rows, VNR positions in flight
  for (int p0 = tid; p0 < nf; p0 += VNR * VT) {
    int32_t e[VNR], ee[VNR];
    T val[VNR];
#pragma unroll
    for (int h = 0; h < VNR; ++h) {
      const int pp = p0 + h * VT;
      e[h] = ee[h] = 0;
      val[h] = T(0);
      if (pp < nf) {
        e[h] = __ldg(&p.vs_pptr[pb + pp]);
        ee[h] = __ldg(&p.vs_pptr[pb + pp + 1]);
        const int vi = __ldg(&p.vs_pfvi[pb + pp]);
        if (vi >= 0) val[h] = v[vi];
      }
    }
    bool more = true;
    while (more) {
      int32_t src[VNR];
#pragma unroll
      for (int h = 0; h < VNR; ++h) src[h] = e[h] < ee[h] ? __ldg(&p.vs_psrc[e[h]]) : -1;
      more = false;
#pragma unroll
      for (int h = 0; h < VNR; ++h)
        if (src[h] >= 0) {
          val[h] += Us[src[h]];
          more |= ++e[h] < ee[h];
        }
    }
#pragma unroll
    for (int h = 0; h < VNR; ++h)
      if (p0 + h * VT < nf) fs[p0 + h * VT] = val[h];
  }
  __syncthreads();
  // (B) products; the next unit's record is fetched while this unit's panel loads are in
  // flight
  {
    int u = tid;
    VsItem I;
    if (u < nu) I.load(items, i0 + __ldg(&p.vs_uitem[ubase + u]));
    while (u < nu) {
      const int un = u + VT;
      VsItem In;
      if (un < nu) In.load(items, i0 + __ldg(&p.vs_uitem[ubase + un]));
      const int kg = I.kg, lu = u - I.uf, w = I.w, m = I.m, ld = (m + 3) & ~3, nrg = ld >> 2;
      const int g = lu / nrg, row = 4 * (lu - g * nrg);
      const int kmax = min(w, row + 4);
      const T *P = panel + I.po + row;
      const T *F = fs + I.fo;
      T acc[4] = {T(0), T(0), T(0), T(0)};
      int k = g;
      for (; k + 7 * kg < kmax; k += 8 * kg) {
        Quad<T> pv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) pv[t].load(P + (size_t)(k + kg * t) * ld);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const T fk = F[k + kg * t];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] += pv[t].a[i] * fk;
        }
      }
      for (; k < kmax; k += kg) {
        Quad<T> p0;
        p0.load(P + (size_t)k * ld);
        const T fk = F[k];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += p0.a[i] * fk;
      }
      if (kg == 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = row + i;
          if (r >= m) break;
          if (r < w) v[I.fl + r] = acc[i];
          else Us[I.us + r - w] = F[r] - acc[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) red[I.ro + g * ld + row + i] = acc[i];
      }
      I = In;
      u = un;
    }
  }
  __syncthreads();
  if (!B1.y) return;
  // (C) K-split partial sums, in group order
  for (int pp = tid; pp < nf; pp += VT) {
    VsItem I;
    I.load(items, i0 + __ldg(&p.vs_pitem[pb + pp]));
    const int k = pp - I.fo, ld = (I.m + 3) & ~3;
    if (I.kg == 1 || k >= I.m) continue;
    T s = T(0);
    for (int g = 0; g < I.kg; ++g) s += red[I.ro + g * ld + k];
    if (k < I.w) v[I.fl + k] = s;
    else Us[I.us + k - I.w] = fs[pp] - s;
  }
  __syncthreads();
}

template <typename T>
__device__ void vs_backward(const SweepPlan &p, const T *panel, T *v, T *scr, int q) {
  const int4 B0 = __ldg(&p.vs_bat[3 * q]), B1 = __ldg(&p.vs_bat[3 * q + 1]),
             B2 = __ldg(&p.vs_bat[3 * q + 2]);
  const int i0 = B0.x, nf = B0.z, nc = B1.x, pb = B1.z, cbase = B2.x;
  const int4 *items = p.vs_item;
  T *gs = scr;
  const int tid = threadIdx.x;
  // (A) g = [y_J; -x(rows below); 0 padding]
  for (int pp = tid; pp < nf; pp += VT) {
    const int vi = __ldg(&p.vs_pbvi[pb + pp]);
    gs[pp] = vi >= 0 ? v[vi] : vi < -1 ? -v[-2 - vi] : T(0);
  }
  __syncthreads();
  // (B) a thread per column, sequential over the front from the diagonal's 4-row group
  {
    int u = tid;
    VsItem I;
    if (u < nc) I.load(items, i0 + __ldg(&p.vs_citem[cbase + u]));
    while (u < nc) {
      const int un = u + VT;
      VsItem In;
      if (un < nc) In.load(items, i0 + __ldg(&p.vs_citem[cbase + un]));
      const int col = u - I.ub, ld = (I.m + 3) & ~3;
      const T *Pc = panel + I.po + (size_t)col * ld;
      const T *G = gs + I.fo;
      T acc = T(0);
      int k = col & ~3;
      for (; k + 28 < ld; k += 32) {
        Quad<T> pv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) pv[t].load(Pc + k + 4 * t);
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc += pv[t].a[i] * G[k + 4 * t + i];
      }
      for (; k < ld; k += 4) {
        Quad<T> p0;
        p0.load(Pc + k);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc += p0.a[i] * G[k + i];
      }
      v[I.fl + col] = acc;
      I = In;
      u = un;
    }
  }
  __syncthreads();
}

// Shared memory: [scratch: vs_scratch entries] [v: n_b, rounded to 4] [update-row pool]
template <typename T, int MINB>
__global__ void __launch_bounds__(VT, MINB)
    k_vsm_sweep(ForestDev f, SweepPlan p, const T *__restrict__ panel, const T *B, T *X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *scr = reinterpret_cast<T *>(smem_raw);
  const int b = blockIdx.x;
  const int64_t r0 = p.vs_row_off[b], nb = p.vs_row_off[b + 1] - r0;
  T *v = scr + p.vs_scratch;
  T *Us = v + ((nb + 3) & ~int64_t(3));
  const int tid = threadIdx.x;
  for (int64_t i = tid; i < nb; i += VT) v[i] = B ? B[r0 + i] : T(0);
  __syncthreads();
  const int L0 = p.vs_lvl_ptr[b], L1 = p.vs_lvl_ptr[b + 1];
  for (int L = L0; L < L1; ++L)
    for (int q = p.vs_bat_ptr[L]; q < p.vs_bat_ptr[L + 1]; ++q)
      vs_forward<T>(p, panel, v, Us, scr, q);
  for (int L = L1 - 1; L >= L0; --L)
    for (int q = p.vs_bat_ptr[L]; q < p.vs_bat_ptr[L + 1]; ++q)
      vs_backward<T>(p, panel, v, scr, q);
  for (int64_t i = tid; i < nb; i += VT) X[r0 + i] = v[i];
}

}  // namespace

template <typename T>
size_t vsm_sweep_smem(const SweepPlan &p) {
  if (!p.vs_item || p.vs_elems <= 0) return 0;
  return sizeof(T) * (size_t)((int64_t)p.vs_scratch + p.vs_elems);
}

// largest number of CTAs per SM (1 or 2) whose shared memory fits; 0: none
template <typename T>
int vsm_sweep_fits(const SweepPlan &p) {
  const size_t bytes = vsm_sweep_smem<T>(p);
  if (bytes == 0 || !p.vector || p.res_nblocks <= 0) return 0;
  int dev = 0, optin = 0, per_sm = 0;
  NSP_CUDA(cudaGetDevice(&dev));
  NSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  NSP_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  if (bytes > (size_t)optin) return 0;
  return 2 * (bytes + 1024) <= (size_t)per_sm ? 2 : 1;
}

template <typename T, int MINB>
void run_vsm(const ForestDev &f, const SweepPlan &p, size_t smem, const T *panel, const T *B,
             T *X, cudaStream_t stream) {
  static size_t attr = 0;
  if (smem > attr) {
    ensure_dyn_smem(k_vsm_sweep<T, MINB>, smem);
    attr = smem;
  }
  k_vsm_sweep<T, MINB><<<p.res_nblocks, VT, smem, stream>>>(f, p, panel, B, X);
  NSP_LAUNCH_CHECK();
}

template <typename T>
void launch_vsm_sweep(const ForestDev &f, const SweepPlan &p, const T *panel, const T *B, T *X,
                      int per_sm, cudaStream_t stream) {
  const int fits = vsm_sweep_fits<T>(p);
  require(fits >= 1 && per_sm >= 1 && per_sm <= fits, NSP_ERR_INVALID_ARG,
          "shared-memory single-vector sweep: the block vectors do not fit");
  const size_t smem = vsm_sweep_smem<T>(p);
  if (per_sm == 2) run_vsm<T, 2>(f, p, smem, panel, B, X, stream);
  else run_vsm<T, 1>(f, p, smem, panel, B, X, stream);
}

template int vsm_sweep_fits<float>(const SweepPlan &);
template int vsm_sweep_fits<double>(const SweepPlan &);
template void launch_vsm_sweep<float>(const ForestDev &, const SweepPlan &, const float *,
                                      const float *, float *, int, cudaStream_t);
template void launch_vsm_sweep<double>(const ForestDev &, const SweepPlan &, const double *,
                                       const double *, double *, int, cudaStream_t);

}  // namespace nsp
