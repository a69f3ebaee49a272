// Host runtime of the Nyström–Schur preconditioner and the C ABI of include/nsp.h.
//
// nsp_build = validation + DBBD extraction (§2.3 eq. (perm_A)) + symbolic analysis (host)
//           + numeric factorization of A_1..A_N and A_G (device)
//           + Algorithm 2: sketch G (step 1), inner block PCG (steps 2-4), Nyström core
//             (steps 5-10), Z = A_G^{-1} U (step 11)             (device)
// nsp_solve = outer PCG preconditioned by M2 (§2.3 eq. (Sx=b), §4.3 eq. (left_prec_mat)).
//
// Device vectors use the factor ("internal") orderings: interior unknowns by block, each
// block in its postordered elimination order; interface unknowns in A_G's elimination order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "symbolic.h"

namespace nsp {

static std::atomic<int64_t> g_launches{0};
int64_t count_launch() { return g_launches.fetch_add(1, std::memory_order_relaxed) + 1; }
int64_t launches_counted() { return g_launches.load(); }
// Launches recorded into a CUDA graph run at its replays: the capture removes them from the
// count and each replay adds them back.
void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// ------------------------------------------------------------------ host analysis
struct HostSub {                     // a sub-matrix of A in internal numbering
  int32_t nrows = 0, ncols = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<int64_t> src;          // index into A's values
};

struct Analysis {
  int64_t n = 0, nnz = 0, nI = 0, nG = 0;
  int32_t nblocks = 0;
  std::vector<int64_t> rowptr;       // copy of A's pattern
  std::vector<int32_t> col;
  Forest FI, FG;
  std::vector<int64_t> i2g_I, i2g_G; // internal -> index in A
  std::vector<int64_t> i2u_I, i2u_G; // internal -> caller interior / Gamma order
  HostSub A_I, A_IG, A_GI, A_G;
  double ms = 0;
};

static void validate_csr(const nsp_csr *A) {
  require(A && A->n > 0 && A->rowptr && A->col && A->val, NSP_ERR_INVALID_ARG, "CSR: null or empty");
  require(A->n < (int64_t(1) << 31) - 1, NSP_ERR_UNSUPPORTED, "CSR: n too large");
}

// Leaf size of the library's nested dissection (NSP_ND_LEAF, default 64).
static int nd_leaf() {
  const char *e = std::getenv("NSP_ND_LEAF");
  const int v = e ? std::atoi(e) : 64;
  return v >= 8 ? v : 64;
}

// Largest subtree (supernodes) a sweep runs as one item (NSP_SUBTREE, default 32; <= 1: off).
static int subtree_max() {
  const char *e = std::getenv("NSP_SUBTREE");
  return e ? std::atoi(e) : 32;
}

// Largest front (rows) of a subtree member (NSP_SUBTREE_M, default 128).
static int subtree_m() {
  const char *e = std::getenv("NSP_SUBTREE_M");
  return e ? std::atoi(e) : 128;
}

// Columns per backward tile of a single-vector sweep (NSP_VEC_COLS, default 16).
static int vec_cols() {
  const char *e = std::getenv("NSP_VEC_COLS");
  const int v = e ? std::atoi(e) : kSweepVectorCols;
  return v >= 1 ? v : kSweepVectorCols;
}

// Block tiles of 32 rows instead of 64 in the dependency-driven sweeps of single-tree forests
// (A_G), whose top supernodes form a long chain: twice the tiles work on each of them at once
// (128^3, s = 160: 5.67 -> 4.45 ms per A_G sweep; 16-row tiles 4.62 ms). NSP_GTILE=64
// restores 64 (measurements).
static int narrow_tiles() {
  const char *e = std::getenv("NSP_GTILE");
  return e && std::atoi(e) == 64 ? kSweepBlockRows : kSweepBlockRowsNarrow;
}

// K steps per forward K group of the single-vector shared-memory sweep (NSP_VSM_KDIV,
// default 48; measurements)
static int vsm_kdiv() {
  const char *e = std::getenv("NSP_VSM_KDIV");
  const int v = e ? std::atoi(e) : 48;
  return v >= 8 ? v : 48;
}

static int relax_level() {
  const char *e = std::getenv("NSP_RELAX");
  return e ? std::atoi(e) : 2;
}

static void analyze(const nsp_csr *A, const int64_t *rowptr, const int32_t *col,
                    const nsp_partition *P, Analysis &an) {
  auto t0 = Clock::now();
  const int64_t n = A->n;
  an.n = n;
  require(rowptr[0] == 0, NSP_ERR_INVALID_ARG, "CSR: rowptr[0] != 0");
  for (int64_t i = 0; i < n; ++i) require(rowptr[i + 1] >= rowptr[i], NSP_ERR_INVALID_ARG, "CSR: rowptr not monotone");
  an.nnz = rowptr[n];
  require(an.nnz < (int64_t(1) << 31) - 1, NSP_ERR_UNSUPPORTED, "CSR: too many nonzeros");
  an.rowptr.assign(rowptr, rowptr + n + 1);
  an.col.assign(col, col + an.nnz);
  const int64_t vchunk = 16384, nvch = (n + vchunk - 1) / vchunk;
  parallel_for(nvch, [&](int64_t c) {
    for (int64_t i = c * vchunk; i < std::min(n, (c + 1) * vchunk); ++i) {
      bool diag = false;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        require(col[e] >= 0 && col[e] < n, NSP_ERR_INVALID_ARG, "CSR: column out of range");
        if (e > rowptr[i]) require(col[e] > col[e - 1], NSP_ERR_INVALID_ARG, "CSR: columns not sorted/unique");
        diag |= col[e] == i;
      }
      require(diag, NSP_ERR_INVALID_ARG, "CSR: missing diagonal entry");
    }
  });
  // symmetric pattern
  parallel_for(nvch, [&](int64_t c) {
    for (int64_t i = c * vchunk; i < std::min(n, (c + 1) * vchunk); ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t j = col[e];
        const int32_t *b = col + rowptr[j], *en = col + rowptr[j + 1];
        require(std::binary_search(b, en, (int32_t)i), NSP_ERR_INVALID_ARG, "CSR: pattern not symmetric");
      }
  });
  // partition
  require(P && P->part && P->nblocks >= 1, NSP_ERR_INVALID_ARG, "partition: null");
  const int32_t nb = P->nblocks;
  an.nblocks = nb;
  const int32_t *part = P->part;
  std::vector<std::vector<int64_t>> nodes(nb);
  std::vector<int64_t> gam;
  for (int64_t i = 0; i < n; ++i) {
    require(part[i] >= -1 && part[i] < nb, NSP_ERR_INVALID_ARG, "partition: part out of range");
    if (part[i] < 0) gam.push_back(i);
    else nodes[part[i]].push_back(i);
  }
  for (int64_t i = 0; i < n; ++i)
    if (part[i] >= 0)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t pj = part[col[e]];
        require(pj < 0 || pj == part[i], NSP_ERR_NOT_DBBD, "interior blocks are coupled");
      }
  an.nG = (int64_t)gam.size();
  an.nI = n - an.nG;
  require(an.nG > 0, NSP_ERR_INVALID_ARG, "partition: empty interface");
  require(an.nI > 0, NSP_ERR_INVALID_ARG, "partition: no interior unknowns");
  // caller order of interior / interface unknowns
  std::vector<int64_t> g2u(n, -1);
  {
    int64_t u = 0;
    for (int32_t b = 0; b < nb; ++b) for (int64_t g : nodes[b]) g2u[g] = u++;
    for (int64_t t = 0; t < an.nG; ++t) g2u[gam[t]] = t;
  }
  // initial (elimination) order of each block
  std::vector<std::vector<int64_t>> init(nb);
  if (P->perm) {
    std::vector<char> seen(n, 0);
    for (int64_t q = 0; q < an.nI; ++q) {
      const int64_t g = P->perm[q];
      require(g >= 0 && g < n && part[g] >= 0 && !seen[g], NSP_ERR_INVALID_ARG, "partition: perm is not a permutation of the interior unknowns");
      seen[g] = 1;
      init[part[g]].push_back(g);
    }
  }
  std::vector<int64_t> g2l(n, -1);
  auto graph_of = [&](const std::vector<int64_t> &vs, int32_t label) {
    Graph gr;
    gr.n = (int32_t)vs.size();
    gr.ptr.assign(gr.n + 1, 0);
    for (int32_t l = 0; l < gr.n; ++l) g2l[vs[l]] = l;
    for (int32_t l = 0; l < gr.n; ++l) {
      const int64_t g = vs[l];
      for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e)
        if (col[e] != g && part[col[e]] == label) gr.adj.push_back((int32_t)g2l[col[e]]);
      gr.ptr[l + 1] = (int64_t)gr.adj.size();
    }
    return gr;
  };
  // orderings: every interior block and the interface, in parallel (task 0 = the interface;
  // graph_of writes g2l only at the task's own, disjoint, unknowns)
  std::vector<int64_t> ginit;
  parallel_for(nb + 1, [&](int64_t t) {
    if (t == 0) {   // the interface graph is the largest: started first
      Graph gr = graph_of(gam, -1);
      std::vector<int32_t> ord = nested_dissection(gr, nd_leaf());
      ginit.resize(ord.size());
      for (size_t q = 0; q < ord.size(); ++q) ginit[q] = gam[ord[q]];
      return;
    }
    const int32_t b = (int32_t)t - 1;
    if (!P->perm && !nodes[b].empty()) {
      Graph gr = graph_of(nodes[b], b);
      std::vector<int32_t> ord = nested_dissection(gr, nd_leaf());
      init[b].resize(ord.size());
      for (size_t q = 0; q < ord.size(); ++q) init[b][q] = nodes[b][ord[q]];
    }
  });
  // lower-triangle patterns in the initial orders
  auto pattern = [&](const std::vector<int64_t> &ord, int32_t label) {
    BlockPattern bp;
    bp.n = (int32_t)ord.size();
    for (int32_t l = 0; l < bp.n; ++l) g2l[ord[l]] = l;
    bp.colptr.assign(bp.n + 1, 0);
    for (int32_t j = 0; j < bp.n; ++j) {
      const int64_t g = ord[j];
      for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
        const int32_t c = col[e];
        if (part[c] != label) continue;
        const int64_t i = g2l[c];
        if (i >= j) { bp.rowidx.push_back((int32_t)i); bp.src.push_back(e); }
      }
      bp.colptr[j + 1] = (int64_t)bp.rowidx.size();
    }
    return bp;
  };
  {
    std::vector<BlockPattern> pats(nb);
    parallel_for(nb, [&](int64_t b) { pats[b] = pattern(init[b], (int32_t)b); });
    analyze_forest(pats, relax_level(), an.FI);
  }
  {
    std::vector<BlockPattern> pats(1);
    pats[0] = pattern(ginit, -1);
    analyze_forest(pats, relax_level(), an.FG);
  }
  // internal numbering
  an.i2g_I.resize(an.nI);
  an.i2u_I.resize(an.nI);
  std::vector<int64_t> g2int(n, -1);
  for (int32_t b = 0; b < nb; ++b) {
    const int64_t off = an.FI.block_off[b];
    for (int64_t t = off; t < an.FI.block_off[b + 1]; ++t) {
      const int64_t g = init[b][an.FI.order[t]];
      an.i2g_I[t] = g;
      an.i2u_I[t] = g2u[g];
      g2int[g] = t;
    }
  }
  an.i2g_G.resize(an.nG);
  an.i2u_G.resize(an.nG);
  for (int64_t t = 0; t < an.nG; ++t) {
    const int64_t g = ginit[an.FG.order[t]];
    an.i2g_G[t] = g;
    an.i2u_G[t] = g2u[g];
    g2int[g] = t;
  }
  // rows of A restricted to interior or interface columns: counts, then the entries, both
  // in parallel over row chunks
  auto sub = [&](const std::vector<int64_t> &rows_g, bool cols_gamma, int32_t ncols) {
    HostSub h;
    h.nrows = (int32_t)rows_g.size();
    h.ncols = ncols;
    h.rowptr.assign(h.nrows + 1, 0);
    const int64_t chunk = 4096, nch = (h.nrows + chunk - 1) / chunk;
    parallel_for(nch, [&](int64_t c) {
      for (int64_t r = c * chunk; r < std::min<int64_t>(h.nrows, (c + 1) * chunk); ++r) {
        const int64_t g = rows_g[r];
        int32_t cnt = 0;
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) cnt += (part[col[e]] < 0) == cols_gamma;
        h.rowptr[r + 1] = cnt;
      }
    });
    for (int32_t r = 0; r < h.nrows; ++r) h.rowptr[r + 1] += h.rowptr[r];
    h.col.resize(h.rowptr[h.nrows]);
    h.src.resize(h.rowptr[h.nrows]);
    parallel_for(nch, [&](int64_t c) {
      for (int64_t r = c * chunk; r < std::min<int64_t>(h.nrows, (c + 1) * chunk); ++r) {
        const int64_t g = rows_g[r];
        int64_t q = h.rowptr[r];
        for (int64_t e = rowptr[g]; e < rowptr[g + 1]; ++e) {
          if ((part[col[e]] < 0) != cols_gamma) continue;
          h.col[q] = (int32_t)g2int[col[e]];
          h.src[q] = e;
          ++q;
        }
      }
    });
    return h;
  };
  an.A_I = sub(an.i2g_I, false, (int32_t)an.nI);
  an.A_IG = sub(an.i2g_I, true, (int32_t)an.nG);
  an.A_GI = sub(an.i2g_G, false, (int32_t)an.nI);
  an.A_G = sub(an.i2g_G, true, (int32_t)an.nG);
  an.ms = ms_since(t0);
}

// Extreme eigenvalues of the Lanczos tridiagonal of a PCG run (Saad, Iterative Methods for
// Sparse Linear Systems, §6.7.3): diagonal 1/a_0, 1/a_j + b_{j-1}/a_{j-1}; off-diagonal
// sqrt(b_{j-1})/a_{j-1}. Bisection on the Sturm count (number of eigenvalues below x, the
// negative pivots of T - x I; Golub & Van Loan §8.4), inside the Gershgorin interval.
static void lanczos_extremes(const std::vector<double> &a, const std::vector<double> &b,
                             double *lmin, double *lmax) {
  *lmin = *lmax = 0.0;
  const int m = (int)a.size();
  if (m == 0) return;
  std::vector<double> d(m), e2(m, 0.0), e(m, 0.0);
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / a[j] + (j > 0 ? b[j - 1] / a[j - 1] : 0.0);
    if (j > 0) {
      e[j] = std::sqrt(std::max(b[j - 1], 0.0)) / a[j - 1];
      e2[j] = e[j] * e[j];
    }
  }
  double lo = d[0], hi = d[0];
  for (int j = 0; j < m; ++j) {
    const double r = (j > 0 ? std::fabs(e[j]) : 0.0) + (j + 1 < m ? std::fabs(e[j + 1]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  auto below = [&](double x) {           // eigenvalues < x
    int c = 0;
    double q = 1.0;
    for (int j = 0; j < m; ++j) {
      q = d[j] - x - (j > 0 ? e2[j] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++c;
    }
    return c;
  };
  auto kth = [&](int k) {                // k-th smallest (0-based)
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
      const double mid = 0.5 * (l + h);
      if (below(mid) > k) h = mid;
      else l = mid;
    }
    return 0.5 * (l + h);
  };
  *lmin = kth(0);
  *lmax = kth(m - 1);
}

// ------------------------------------------------------------------ device containers
template <typename T>
struct DevCsr {
  int32_t nrows = 0, ncols = 0;
  int64_t nnz = 0;
  DBuf<int32_t> rowptr, col;
  DBuf<int64_t> src;
  DBuf<double> v64;
  DBuf<T> vT;
  void upload(const HostSub &h, cudaStream_t st) {
    nrows = h.nrows;
    ncols = h.ncols;
    nnz = (int64_t)h.col.size();
    rowptr.upload(h.rowptr, st);
    col.upload(h.col, st);
    src.upload(h.src, st);
    v64.alloc(nnz);
    vT.alloc(nnz);
  }
  void refresh(const double *Aval, cudaStream_t st) {
    launch_gather_values<double>(src.p, nnz, Aval, v64.p, st);
    launch_gather_values<T>(src.p, nnz, Aval, vT.p, st);
  }
  CsrDev<double> d64() const { return CsrDev<double>{nrows, ncols, nnz, rowptr.p, col.p, v64.p}; }
  CsrDev<T> dT() const { return CsrDev<T>{nrows, ncols, nnz, rowptr.p, col.p, vT.p}; }
};

struct ForestData {
  Forest h;
  DBuf<int32_t> sn_first, sn_w, sn_m, sn_block, rows, relmap, ch_ptr, ch_list, level_sn;
  std::vector<int32_t> level_small;   // per level: number of fronts below kBigFront rows
  DBuf<int64_t> sn_rowptr, sn_panel, sn_front, sn_upd, gptr, gsrc, asm_ptr, asm_dst, asm_src;
  ForestDev dev;
  struct Plan {
    SweepPlan d;
    DBuf<int32_t> item_a, item_b, group_sn, sn_parent, need_f, units_f, units_b;
    DBuf<uint32_t> counters;  // cnt_f, self_f, done_b (nsn each), claim, abort, epoch, base
    DBuf<int32_t> res_blk_ptr, res_lvl_ptr, res_lvl_nwarp, res_job;   // block-resident schedule
    DBuf<int64_t> vs_row_off;                                        // vector plans
    DBuf<int32_t> vs_lvl_ptr, vs_bat_ptr, vs_pfvi, vs_pbvi, vs_pptr, vs_psrc;
    DBuf<uint16_t> vs_pitem, vs_uitem, vs_citem;
    DBuf<int32_t> bs_lvl_ptr, bs_bat_ptr, bs_pfvi, bs_pbvi, bs_pptr, bs_psrc;   // block plans
    DBuf<int4> bs_bat, bs_item;
    DBuf<uint16_t> bs_uitem, bs_citem;
    DBuf<int4> vs_bat, vs_item;
    int32_t maxneed = 1;
    // right-hand-side count -> persistent grid of the dependency-driven sweep, or
    // kResidentGrid for the block-resident sweep (autotuner)
    std::map<int, int> tuned_grid;
  };
  std::unique_ptr<Plan> plans[2];  // 0: block (s > 1), 1: vector (s = 1)
  int vec_rows = 128;
  int elem_bytes = 4;   // element size of the handle (shared-memory sweep budget)
  // rows (forward) / columns (backward) of a block tile of the dependency-driven sweep
  int blk_rows = kSweepBlockRows;

  Plan &plan(bool vector, cudaStream_t st) {
    auto &pp = plans[vector ? 1 : 0];
    if (pp) return *pp;
    pp = std::make_unique<Plan>();
    Plan &P = *pp;
    const int nsn = h.nsn;
    const int tf = vector ? vec_rows : blk_rows;
    const int tb = vector ? vec_cols() : blk_rows;
    std::vector<int32_t> ia, ib, gs, uf(nsn, 0), ub(nsn, 0), need(nsn, 0);
    auto small = [&](int J) { return vector && h.sn_m[J] <= kSmallM && h.sn_w[J] <= kSmallW; };
    // Subtrees of small supernodes run as one item each (one CTA, no dependency wait inside):
    // J heads one when its whole subtree is at most subtree_max() supernodes of bounded size
    // and panel area, numbered contiguously below J (postorder).
    std::vector<char> in_sub(nsn, 0);
    std::vector<int32_t> sub_first(nsn), sub_cnt(nsn, 1), sub_off(nsn, -1), sub_len_of(nsn, 0);
    {
      const int smax = subtree_max();
      std::vector<char> ok(nsn);
      std::vector<double> area(nsn);
      bool post = true;
      for (int J = 0; J < nsn; ++J) {
        const int m = h.sn_m[J], w = h.sn_w[J];
        ok[J] = m <= subtree_m() && 2 * w <= subtree_m();
        area[J] = (double)m * w;
        sub_first[J] = J;
        if (h.sn_parent[J] >= 0 && h.sn_parent[J] <= J) post = false;
      }
      // block mode only: in vector mode a small supernode is a warp's work, and running a
      // subtree's heights one after another in one CTA lengthened the single-vector sweep
      for (int J = 0; J < nsn && post && smax > 1 && !vector; ++J) {
        in_sub[J] = ok[J] && sub_cnt[J] <= smax && area[J] <= kSubtreeArea && J - sub_first[J] + 1 == sub_cnt[J];
        const int par = h.sn_parent[J];
        if (par < 0) continue;
        sub_first[par] = std::min(sub_first[par], sub_first[J]);
        sub_cnt[par] += sub_cnt[J];
        area[par] += area[J];
        ok[par] = ok[par] && ok[J];
      }
    }
    // member list of the subtree headed by R in group_sn: members by height, -1 between heights
    auto emit_subtree = [&](int R) {
      if (sub_off[R] < 0) {
        std::vector<std::pair<int, int>> mem;
        for (int J = sub_first[R]; J <= R; ++J) mem.push_back({h.sn_level[J], J});
        std::stable_sort(mem.begin(), mem.end());
        sub_off[R] = (int32_t)gs.size();
        for (size_t q = 0; q < mem.size(); ++q) {
          if (q > 0 && mem[q].first != mem[q - 1].first) gs.push_back(-1);
          gs.push_back(mem[q].second);
        }
        sub_len_of[R] = (int32_t)gs.size() - sub_off[R];
      }
      ia.push_back(sub_off[R]);
      ib.push_back(kSubtreeTag - sub_len_of[R]);
    };
    auto emit_level = [&](int l, bool fwd) {
      std::vector<int32_t> grp;
      auto flush = [&]() {
        if (grp.empty()) return;
        ia.push_back((int32_t)gs.size());
        ib.push_back(-(int32_t)grp.size());
        for (int J : grp) { gs.push_back(J); (fwd ? uf : ub)[J] = 1; }
        grp.clear();
      };
      for (int q = h.level_ptr[l]; q < h.level_ptr[l + 1]; ++q) {
        const int J = h.level_sn[q];
        if (in_sub[J]) {
          const int par = h.sn_parent[J];
          if (par >= 0 && in_sub[par]) continue;  // runs inside its head's item
          if (sub_cnt[J] > 1) {                   // the whole subtree in one item
            emit_subtree(J);
            (fwd ? uf : ub)[J] = 1;
            continue;
          }
        }
        if (small(J)) {
          grp.push_back(J);
          if ((int)grp.size() == kGroup) flush();
          continue;
        }
        const int extent = fwd ? h.sn_m[J] : h.sn_w[J];
        const int tile = fwd ? tf : tb;
        for (int r0 = 0; r0 < extent; r0 += tile) { ia.push_back(J); ib.push_back(r0); }
        (fwd ? uf : ub)[J] = (extent + tile - 1) / tile;
      }
      flush();
    };
    for (int l = 0; l < h.nlevels; ++l) emit_level(l, true);
    const int nfwd = (int)ia.size();
    for (int l = h.nlevels - 1; l >= 0; --l) emit_level(l, false);
    for (int J = 0; J < nsn; ++J)
      if (h.sn_parent[J] >= 0) need[h.sn_parent[J]] += uf[J];
    for (int J = 0; J < nsn; ++J) P.maxneed = std::max({P.maxneed, need[J], uf[J], ub[J]});
    if (gs.empty()) gs.push_back(0);
    P.item_a.upload(ia, st);
    P.item_b.upload(ib, st);
    P.group_sn.upload(gs, st);
    P.sn_parent.upload(h.sn_parent, st);
    P.need_f.upload(need, st);
    P.units_f.upload(uf, st);
    P.units_b.upload(ub, st);
    P.counters.alloc(3 * (size_t)nsn + 4);
    NSP_CUDA(cudaMemsetAsync(P.counters.p, 0, P.counters.bytes(), st));
    int mm = 0;
    for (int J = 0; J < nsn; ++J) mm = std::max(mm, h.sn_m[J]);
    P.d.nitems = (int32_t)ia.size();
    P.d.nfwd = nfwd;
    P.d.max_m = mm;
    P.d.vec_cols = tb;
    P.d.blk_rows = vector ? kSweepBlockRows : blk_rows;
    P.d.vector = vector;
    P.d.item_a = P.item_a.p;
    P.d.item_b = P.item_b.p;
    P.d.group_sn = P.group_sn.p;
    P.d.sn_parent = P.sn_parent.p;
    P.d.need_f = P.need_f.p;
    P.d.units_f = P.units_f.p;
    P.d.units_b = P.units_b.p;
    P.d.cnt_f = P.counters.p;
    P.d.self_f = P.counters.p + nsn;
    P.d.done_b = P.counters.p + 2 * (size_t)nsn;
    P.d.claim = P.counters.p + 3 * (size_t)nsn;
    P.d.abort_flag = P.counters.p + 3 * (size_t)nsn + 1;
    P.d.epoch = P.counters.p + 3 * (size_t)nsn + 2;
    P.d.claim_base = P.counters.p + 3 * (size_t)nsn + 3;
    // block-resident schedule: per block, its supernodes by height; warp-sized ones first,
    // largest first, so that the warps' shares of a height are balanced
    {
      const int nb = h.nblocks;
      std::vector<std::vector<std::vector<int32_t>>> bl(nb);
      for (int J = 0; J < nsn; ++J) {
        auto &v = bl[h.sn_block[J]];
        const int l = h.sn_level[J];
        if ((int)v.size() <= l) v.resize(l + 1);
        v[l].push_back(J);
      }
      auto warp_sized = [&](int J) {
        return vector ? (h.sn_m[J] <= kSmallM && h.sn_w[J] <= kSmallW)
                      : (h.sn_w[J] <= kResW && h.sn_m[J] <= kResM);
      };
      std::vector<int32_t> bptr(nb + 1, 0), lptr(1, 0), lnw, job;
      for (int b = 0; b < nb; ++b) {
        for (auto &lev : bl[b]) {
          if (lev.empty()) continue;
          std::vector<int32_t> wv, cv;
          for (int J : lev) (warp_sized(J) ? wv : cv).push_back(J);
          std::stable_sort(wv.begin(), wv.end(), [&](int a, int c) {
            return (int64_t)h.sn_m[a] * h.sn_w[a] > (int64_t)h.sn_m[c] * h.sn_w[c];
          });
          job.insert(job.end(), wv.begin(), wv.end());
          job.insert(job.end(), cv.begin(), cv.end());
          lnw.push_back((int32_t)wv.size());
          lptr.push_back((int32_t)job.size());
        }
        bptr[b + 1] = (int32_t)lnw.size();
      }
      if (job.empty()) job.push_back(0);
      if (lnw.empty()) lnw.push_back(0);
      P.res_blk_ptr.upload(bptr, st);
      P.res_lvl_ptr.upload(lptr, st);
      P.res_lvl_nwarp.upload(lnw, st);
      P.res_job.upload(job, st);
      P.d.res_nblocks = nb;
      P.d.res_blk_ptr = P.res_blk_ptr.p;
      P.d.res_lvl_ptr = P.res_lvl_ptr.p;
      P.d.res_lvl_nwarp = P.res_lvl_nwarp.p;
      P.d.res_job = P.res_job.p;
      // shared-memory single-vector sweep: per-block row and update-row ranges (every index a
      // block's supernodes touch must stay inside them) and, per height, batches of
      // supernodes whose fronts and K-split partial sums fit the scratch
      if (vector && nb > 0) build_vsm(P, bl, st);
      if (!vector && nb > 0) build_bsm(P, bl, st);
    }
    return P;
  }

  // Batches of the column-sliced block sweep (k_bsweep.cu) from the per-block, per-height
  // supernode lists bl: each batch's fronts (positions x kBsmCols elements of elem_bytes)
  // fit kBsmScratchBytes. Per front position the B row (forward, top rows), the Y / X source
  // (backward) and the gather sources (update rows); forward units (4-row group, 8-column
  // group), backward units (4 panel columns, 8-column group).
  void build_bsm(Plan &P, const std::vector<std::vector<std::vector<int32_t>>> &bl,
                 cudaStream_t st) {
    const int nb = h.nblocks;
    const int maxpos = kBsmScratchBytes / (kBsmCols * elem_bytes);
    if (h.n >= INT32_MAX - 2 || h.upd_rows >= INT32_MAX || (int64_t)h.gsrc.size() >= INT32_MAX)
      return;
    for (int J = 0; J < h.nsn; ++J)
      if ((int)panel_ld(h.sn_m[J]) > maxpos) return;
    std::vector<int32_t> lvl(1, 0), bptr(1, 0), pfvi, pbvi, pptr(1, 0), psrc;
    std::vector<uint16_t> uitem, citem;
    std::vector<int4> bat, item;
    int positions = 0;
    for (int b = 0; b < nb; ++b) {
      for (const auto &lev : bl[b]) {
        if (lev.empty()) continue;
        std::vector<int32_t> cur;
        int nf = 0;
        int64_t nsrc = 0;
        auto close = [&]() {
          if (cur.empty()) return;
          const int i0 = (int)item.size() / 3;
          const int pos_base = (int)pfvi.size(), unit_base = (int)uitem.size(),
                    col_base = (int)citem.size();
          int fo = 0, uf = 0, ub = 0;
          for (size_t t = 0; t < cur.size(); ++t) {
            const int J = cur[t], m = h.sn_m[J], w = h.sn_w[J], ld = (int)panel_ld(m);
            const int64_t rp = h.sn_rowptr[J], po = h.sn_panel[J];
            const int first = (int)h.sn_first[J], upd = (int)h.sn_upd[J];
            item.push_back(int4{fo, uf, ub, m});
            item.push_back(int4{w, first, upd, 0});
            item.push_back(int4{(int)(po & 0xffffffff), (int)(po >> 32), 0, 0});
            for (int k = 0; k < ld; ++k) {
              pfvi.push_back(k < w ? first + k : -1);
              pbvi.push_back(k < w ? first + k : k < m ? -2 - h.rows[rp + k] : -1);
              if (k < m)
                for (int64_t e = h.gptr[rp + k]; e < h.gptr[rp + k + 1]; ++e)
                  psrc.push_back((int32_t)h.gsrc[e]);
              pptr.push_back((int32_t)psrc.size());
            }
            const int nuf = (ld / 4) * 4, nub = ((w + 3) / 4) * 4;
            for (int q = 0; q < nuf; ++q) uitem.push_back((uint16_t)t);
            for (int q = 0; q < nub; ++q) citem.push_back((uint16_t)t);
            fo += ld;
            uf += nuf;
            ub += nub;
          }
          positions = std::max(positions, fo);
          const int sb = pptr[pos_base];
          bat.push_back(int4{i0, i0 + (int)cur.size(), fo, uf});
          bat.push_back(int4{ub, 0, pos_base, unit_base});
          bat.push_back(int4{col_base, sb, (int)psrc.size() - sb, 0});
          cur.clear();
          nf = 0;
          nsrc = 0;
        };
        // a batch's plan data is staged in shared memory: at most kBsmMaxItems supernodes
        // and kBsmMaxSources gather sources per batch
        for (int J : lev) {
          const int ld = (int)panel_ld(h.sn_m[J]);
          const int64_t rp = h.sn_rowptr[J];
          const int64_t js = h.gptr[rp + h.sn_m[J]] - h.gptr[rp];
          if (js > kBsmMaxSources) return;
          if (nf + ld > maxpos || (int)cur.size() >= kBsmMaxItems || nsrc + js > kBsmMaxSources)
            close();
          cur.push_back(J);
          nf += ld;
          nsrc += js;
        }
        close();
        bptr.push_back((int)bat.size() / 3);
      }
      lvl.push_back((int)bptr.size() - 1);
    }
    if (item.empty() || pfvi.size() >= (size_t)INT32_MAX || psrc.size() >= (size_t)INT32_MAX) return;
    if (psrc.empty()) psrc.push_back(0);
    P.bs_lvl_ptr.upload(lvl, st);
    P.bs_bat_ptr.upload(bptr, st);
    P.bs_bat.upload(bat, st);
    P.bs_item.upload(item, st);
    P.bs_pfvi.upload(pfvi, st);
    P.bs_pbvi.upload(pbvi, st);
    P.bs_pptr.upload(pptr, st);
    P.bs_psrc.upload(psrc, st);
    P.bs_uitem.upload(uitem, st);
    P.bs_citem.upload(citem, st);
    P.d.bs_lvl_ptr = P.bs_lvl_ptr.p;
    P.d.bs_bat_ptr = P.bs_bat_ptr.p;
    P.d.bs_bat = P.bs_bat.p;
    P.d.bs_item = P.bs_item.p;
    P.d.bs_pfvi = P.bs_pfvi.p;
    P.d.bs_pbvi = P.bs_pbvi.p;
    P.d.bs_pptr = P.bs_pptr.p;
    P.d.bs_psrc = P.bs_psrc.p;
    P.d.bs_uitem = P.bs_uitem.p;
    P.d.bs_citem = P.bs_citem.p;
    P.d.bs_positions = positions;
  }

  // Batches of the shared-memory single-vector sweep (k_vsweep.cu) from the per-block,
  // per-height supernode lists bl, for elements of elem_bytes. Each block's update rows live
  // in a shared-memory pool: supernode J's rows occupy a slot from its height to its
  // parent's height (inclusive), allocated first-fit in height order, so the pool holds the
  // largest live set rather than every update row. Forward units: (K group, 4-row group)
  // pairs, K split into ceil(w / 48) groups (at most kVsmKG); backward units: columns. The
  // scratch of a batch (fronts, then the K groups' partial sums) takes what shared memory
  // leaves, two CTAs per SM where that leaves at least kVsmScratch entries.
  void build_vsm(Plan &P, const std::vector<std::vector<std::vector<int32_t>>> &bl,
                 cudaStream_t st) {
    const int nb = h.nblocks, nsn = h.nsn;
    const int64_t eb = elem_bytes;
    std::vector<int64_t> roff(nb + 1);
    for (int b = 0; b <= nb; ++b) roff[b] = h.block_off[b];
    // owner of every update row, and the containment checks
    std::vector<int32_t> owner(h.upd_rows > 0 ? h.upd_rows : 1, -1);
    for (int J = 0; J < nsn; ++J)
      for (int64_t i = 0; i < h.sn_m[J] - h.sn_w[J]; ++i) owner[h.sn_upd[J] + i] = J;
    bool ok = true;
    int ldmax = 4;
    for (int J = 0; J < nsn && ok; ++J) {
      const int b = h.sn_block[J];
      const int64_t rp = h.sn_rowptr[J];
      ldmax = std::max(ldmax, (int)panel_ld(h.sn_m[J]));
      if (h.sn_first[J] < roff[b] || h.sn_first[J] + h.sn_w[J] > roff[b + 1]) ok = false;
      for (int k = 0; k < h.sn_m[J] && ok; ++k) {
        if (k >= h.sn_w[J] && (h.rows[rp + k] < roff[b] || h.rows[rp + k] >= roff[b + 1]))
          ok = false;
        for (int64_t e = h.gptr[rp + k]; e < h.gptr[rp + k + 1]; ++e) {
          const int64_t g = h.gsrc[e];
          if (g < 0 || g >= h.upd_rows || owner[g] < 0 || h.sn_block[owner[g]] != b ||
              h.sn_parent[owner[g]] != J)
            ok = false;
        }
      }
    }
    if (!ok) return;
    // update-row slots per block: live from height(J) to height(parent(J))
    std::vector<int32_t> uslot(nsn, 0);
    std::vector<int64_t> pool(nb, 0);
    for (int b = 0; b < nb; ++b) {
      std::vector<std::pair<int32_t, int32_t>> fr;   // free intervals [start, end), sorted
      int32_t top = 0;
      std::vector<std::vector<int32_t>> release(bl[b].size() + 1);
      for (size_t l = 0; l < bl[b].size(); ++l) {
        for (int J : bl[b][l]) {
          const int32_t sz = h.sn_m[J] - h.sn_w[J];
          const int par = h.sn_parent[J];
          if (sz <= 0 || par < 0) continue;
          int32_t at = -1;
          for (auto &iv : fr)
            if (iv.second - iv.first >= sz) {
              at = iv.first;
              iv.first += sz;
              break;
            }
          if (at < 0) {
            at = top;
            top += sz;
          }
          uslot[J] = at;
          release[std::min<size_t>(h.sn_level[par], bl[b].size())].push_back(J);
        }
        // slots whose last reader is this height become free for the next height
        for (int J : release[l]) {
          fr.push_back({uslot[J], uslot[J] + h.sn_m[J] - h.sn_w[J]});
        }
        std::sort(fr.begin(), fr.end());
        std::vector<std::pair<int32_t, int32_t>> merged;
        for (auto &iv : fr) {
          if (iv.first >= iv.second) continue;
          if (!merged.empty() && merged.back().second == iv.first) merged.back().second = iv.second;
          else merged.push_back(iv);
        }
        fr.swap(merged);
      }
      pool[b] = top;
    }
    int64_t vu = 0;
    for (int b = 0; b < nb; ++b)
      vu = std::max(vu, ((roff[b + 1] - roff[b] + 3) & ~int64_t(3)) + ((pool[b] + 3) & ~int64_t(3)));
    const int kdiv = vsm_kdiv();
    auto kg_of = [&](int J) {
      return std::min(kVsmKG, std::max(1, (h.sn_w[J] + kdiv - 1) / kdiv));
    };
    int need_max = 4;
    for (int J = 0; J < nsn; ++J) {
      const int ld = (int)panel_ld(h.sn_m[J]), kg = kg_of(J);
      need_max = std::max(need_max, ld + (kg > 1 ? kg * ld : 0));
    }
    int dev = 0, optin = 0, per_sm = 0;
    NSP_CUDA(cudaGetDevice(&dev));
    NSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    NSP_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int64_t two = ((int64_t)(per_sm / 2 - 1024) / eb - vu) & ~int64_t(3);
    const int64_t one = ((int64_t)optin / eb - vu) & ~int64_t(3);
    int64_t scr;
    if (two >= std::max<int64_t>(need_max, kVsmScratch)) scr = two;
    else if (one >= need_max) scr = std::min<int64_t>(one, 8 * (int64_t)kVsmScratch);
    else return;
    scr = std::min<int64_t>(scr, 1 << 20);
    // flat per-batch arrays: per front position (fronts of a batch back to back, ld entries
    // each) the forward v index (top rows, else -1), the backward source (v index of y_J, or
    // -2 - v index of x for a row below, or -1 for padding), the item (relative to the
    // batch's first) and the gather sources (pool slots, by position); per forward unit and
    // per backward column the item
    std::vector<int32_t> lvl(1, 0), bptr(1, 0), pfvi, pbvi, pptr(1, 0), psrc;
    std::vector<uint16_t> pitem, uitem, citem;
    std::vector<int4> bat, item;
    for (int b = 0; b < nb; ++b) {
      for (const auto &lev : bl[b]) {
        if (lev.empty()) continue;
        std::vector<int32_t> cur;
        int64_t nf = 0, red = 0;
        auto close = [&]() {
          if (cur.empty()) return;
          const int i0 = (int)item.size() / 4;
          const int pos_base = (int)pfvi.size(), unit_base = (int)uitem.size(),
                    col_base = (int)citem.size();
          int fo = 0, ro = 0, uf = 0, ub = 0, any_red = 0;
          for (size_t t = 0; t < cur.size(); ++t) {
            const int J = cur[t], m = h.sn_m[J], w = h.sn_w[J], ld = (int)panel_ld(m);
            const int kg = kg_of(J);
            const int64_t rp = h.sn_rowptr[J], po = h.sn_panel[J];
            const int fl = (int)(h.sn_first[J] - roff[b]);
            item.push_back(int4{fo, kg > 1 ? ro : -1, kg, uslot[J]});
            item.push_back(int4{uf, ub, m, w});
            item.push_back(int4{fl, (int)(rp & 0xffffffff), (int)(rp >> 32), (int)(po & 0xffffffff)});
            item.push_back(int4{(int)(po >> 32), J, 0, 0});
            for (int k = 0; k < ld; ++k) {
              pfvi.push_back(k < w ? fl + k : -1);
              pbvi.push_back(k < w ? fl + k : k < m ? -2 - (int32_t)(h.rows[rp + k] - roff[b]) : -1);
              pitem.push_back((uint16_t)t);
              if (k < m)
                for (int64_t e = h.gptr[rp + k]; e < h.gptr[rp + k + 1]; ++e) {
                  const int64_t g = h.gsrc[e];
                  const int C = owner[g];
                  psrc.push_back(uslot[C] + (int32_t)(g - h.sn_upd[C]));
                }
              pptr.push_back((int32_t)psrc.size());
            }
            for (int q = 0; q < kg * (ld / 4); ++q) uitem.push_back((uint16_t)t);
            for (int q = 0; q < w; ++q) citem.push_back((uint16_t)t);
            fo += ld;
            if (kg > 1) { ro += kg * ld; any_red = 1; }
            uf += kg * (ld / 4);
            ub += w;
          }
          bat.push_back(int4{i0, i0 + (int)cur.size(), fo, uf});
          bat.push_back(int4{ub, any_red, pos_base, unit_base});
          bat.push_back(int4{col_base, 0, 0, 0});
          cur.clear();
          nf = 0;
          red = 0;
        };
        for (int J : lev) {
          const int ld = (int)panel_ld(h.sn_m[J]), kg = kg_of(J);
          const int need = ld + (kg > 1 ? kg * ld : 0);
          if (nf + red + need > scr || cur.size() >= 65535) close();
          cur.push_back(J);
          nf += ld;
          if (kg > 1) red += (int64_t)kg * ld;
        }
        close();
        bptr.push_back((int)bat.size() / 3);
      }
      lvl.push_back((int)bptr.size() - 1);
    }
    if (item.empty() || psrc.size() >= (size_t)INT32_MAX || pfvi.size() >= (size_t)INT32_MAX) return;
    if (psrc.empty()) psrc.push_back(0);
    P.vs_row_off.upload(roff, st);
    P.vs_lvl_ptr.upload(lvl, st);
    P.vs_bat_ptr.upload(bptr, st);
    P.vs_bat.upload(bat, st);
    P.vs_item.upload(item, st);
    P.vs_pfvi.upload(pfvi, st);
    P.vs_pbvi.upload(pbvi, st);
    P.vs_pptr.upload(pptr, st);
    P.vs_psrc.upload(psrc, st);
    P.vs_pitem.upload(pitem, st);
    P.vs_uitem.upload(uitem, st);
    P.vs_citem.upload(citem, st);
    P.d.vs_row_off = P.vs_row_off.p;
    P.d.vs_lvl_ptr = P.vs_lvl_ptr.p;
    P.d.vs_bat_ptr = P.vs_bat_ptr.p;
    P.d.vs_bat = P.vs_bat.p;
    P.d.vs_item = P.vs_item.p;
    P.d.vs_pfvi = P.vs_pfvi.p;
    P.d.vs_pbvi = P.vs_pbvi.p;
    P.d.vs_pptr = P.vs_pptr.p;
    P.d.vs_psrc = P.vs_psrc.p;
    P.d.vs_pitem = P.vs_pitem.p;
    P.d.vs_uitem = P.vs_uitem.p;
    P.d.vs_citem = P.vs_citem.p;
    P.d.vs_elems = vu;
    P.d.vs_scratch = (int32_t)scr;
  }

  void upload(cudaStream_t st) {
    // within each level, fronts with m < kBigFront first (one CTA each), then the big ones
    level_small.assign(h.nlevels, 0);
    for (int l = 0; l < h.nlevels; ++l) {
      auto b = h.level_sn.begin() + h.level_ptr[l], e = h.level_sn.begin() + h.level_ptr[l + 1];
      auto mid = std::stable_partition(b, e, [&](int J) { return h.sn_m[J] < kBigFront; });
      level_small[l] = (int32_t)(mid - b);
    }
    sn_first.upload(h.sn_first, st);
    sn_w.upload(h.sn_w, st);
    sn_m.upload(h.sn_m, st);
    sn_block.upload(h.sn_block, st);
    rows.upload(h.rows, st);
    relmap.upload(h.relmap, st);
    ch_ptr.upload(h.ch_ptr, st);
    ch_list.upload(h.ch_list, st);
    level_sn.upload(h.level_sn, st);
    sn_rowptr.upload(h.sn_rowptr, st);
    sn_panel.upload(h.sn_panel, st);
    sn_front.upload(h.sn_front, st);
    sn_upd.upload(h.sn_upd, st);
    gptr.upload(h.gptr, st);
    gsrc.upload(h.gsrc, st);
    asm_ptr.upload(h.asm_ptr, st);
    asm_dst.upload(h.asm_dst, st);
    asm_src.upload(h.asm_src, st);
    dev.nsn = h.nsn;
    dev.n = h.n;
    dev.sn_first = sn_first.p;
    dev.sn_w = sn_w.p;
    dev.sn_m = sn_m.p;
    dev.sn_block = sn_block.p;
    dev.sn_rowptr = sn_rowptr.p;
    dev.sn_panel = sn_panel.p;
    dev.sn_front = sn_front.p;
    dev.sn_upd = sn_upd.p;
    dev.rows = rows.p;
    dev.relmap = relmap.p;
    dev.ch_ptr = ch_ptr.p;
    dev.ch_list = ch_list.p;
    dev.gptr = gptr.p;
    dev.gsrc = gsrc.p;
    dev.asm_ptr = asm_ptr.p;
    dev.asm_dst = asm_dst.p;
    dev.asm_src = asm_src.p;
  }

};

// ------------------------------------------------------------------ engine
struct EngineBase {
  virtual ~EngineBase() = default;
  virtual void factorize(const double *val, bool on_device) = 0;
  virtual void construct(const nsp_params &prm) = 0;
  virtual void apply_m2(const double *r, double *z) = 0;
  virtual void solve(const double *b, double *x, double rtol, int maxit, int form) = 0;
  virtual void schur_apply_user(const void *X, void *Y, int s) = 0;
  virtual void setup_batch(const std::vector<int64_t> &mat_off) = 0;
  virtual void construct_batched(const nsp_params &prm) = 0;
  virtual void solve_batched(const double *b, double *x, double rtol, int maxit) = 0;
  std::vector<nsp_info> binfo;     // per matrix of a batched handle
  virtual size_t schur_noalloc_bytes(int s) const = 0;
  virtual nsp_status timeout_selftest(int max_spins) = 0;
  virtual void schur_apply_noalloc(const void *X, void *Y, int s, unsigned char *scratch) = 0;
  virtual void factor_solve_user(int which, const void *B, void *X, int s) = 0;
  virtual void attach_gamma(const nsp_params &prm) = 0;
  virtual void get_basis(double *Z, double *Sigma, int32_t *rank) = 0;
  virtual void get_intermediate(int which, double *out) = 0;
  virtual void get_factor(int block, int64_t *order, double *L, int64_t nb) = 0;
  nsp_info info{};
  cudaStream_t st = nullptr;
  int precision = NSP_FP32;
  DBuf<double> stage_b, stage_x;   // device staging of host vectors in nsp_solve
};

template <typename T>
struct Engine : EngineBase {
  Analysis an;
  ForestData FI, FG;
  DevCsr<T> A_I, A_IG, A_GI, A_G;
  DBuf<int32_t> full_rowptr, full_col;   // A in caller order (FP64 residual)
  DBuf<int64_t> i2g_I, i2g_G, i2u_I, i2u_G;
  DBuf<double> Aval;
  DBuf<T> panelI, panelG, front, frontG;   // fronts of the interior and the A_G factors
  DBuf<DevStatus> dstat, dstatG;   // device status words (dstatG: the A_G factorization)
  // the A_G factorization runs on its own stream beside the interior one (factorize)
  cudaStream_t fstream = nullptr;
  cudaEvent_t fev[2] = {nullptr, nullptr};
  DevStatus *hstat = nullptr;            // pinned
  double *hscal = nullptr;               // pinned scalars
  int32_t *hint = nullptr;               // pinned ints
  // solve workspaces (sized for s_ws columns)
  int s_ws = 0;
  DBuf<T> Bv, Yw, Xw, Uw, YwG, UwG;
  // Algorithm 2 state
  int s = 0, k = 0, rank = 0;
  DBuf<T> G, Fh, E, R, P, Q, Z, W, Y, U, Zt;
  DBuf<double> gram_work, PtQ, PtR, QtZ, Cg, alpha, beta, Rinv, Lwork, colsq, bnorm, ratio;
  DBuf<double> K, Cn, Mix, Sigma, nys_work, Zs;
  DBuf<int32_t> mask, nkept, drank;
  DBuf<double> g64, ri_buf, zi_buf;
  // The sketch into g64: the caller's, or `count` Gaussian values drawn from prm.seed, unless
  // g64 already holds that very draw (a rebuild with the same seed draws the same sketch).
  uint64_t g64_seed = 0;
  size_t g64_count = 0;   // Gaussian values of g64_seed held in g64 (0: none)
  void draw_sketch(const nsp_params &prm, size_t count) {
    const size_t cap = g64.n;
    g64.ensure(count);
    if (g64.n != cap) g64_count = 0;   // reallocated: nothing held
    if (prm.sketch) {
      NSP_CUDA(cudaMemcpyAsync(g64.p, prm.sketch, count * sizeof(double), cudaMemcpyDefault, st));
      g64_count = 0;
      return;
    }
    if (g64_count == count && g64_seed == prm.seed) return;
    launch_gaussian<double>(prm.seed, (int64_t)count, g64.p, st);
    g64_seed = prm.seed;
    g64_count = count;
  }
  bool keep = false;
  // outer PCG vectors (FP64)
  DBuf<double> vb, vx, vr, vz, vp, vq, vt, vu, vf, dwork, dscal;
  DBuf<T> sT, sT2;

  Engine(const nsp_csr *A, const int64_t *rowptr, const int32_t *col, const nsp_partition *P,
         cudaStream_t stream) {
    st = stream;
    precision = std::is_same<T, double>::value ? NSP_FP64 : NSP_FP32;
    analyze(A, rowptr, col, P, an);
    FI.h = std::move(an.FI);
    FG.h = std::move(an.FG);
    FI.upload(st);
    FG.upload(st);
    A_I.upload(an.A_I, st);
    A_IG.upload(an.A_IG, st);
    A_GI.upload(an.A_GI, st);
    A_G.upload(an.A_G, st);
    {
      std::vector<int32_t> rp(an.n + 1);
      for (int64_t i = 0; i <= an.n; ++i) rp[i] = (int32_t)an.rowptr[i];
      full_rowptr.upload(rp, st);
      full_col.upload(an.col, st);
    }
    i2g_I.upload(an.i2g_I, st);
    i2g_G.upload(an.i2g_G, st);
    i2u_I.upload(an.i2u_I, st);
    i2u_G.upload(an.i2u_G, st);
    Aval.alloc(an.nnz);
    panelI.alloc(FI.h.panel_size);
    panelG.alloc(FG.h.panel_size);
    front.alloc(std::max<int64_t>(FI.h.front_size, 1));
    frontG.alloc(std::max<int64_t>(FG.h.front_size, 1));
    dstat.alloc(1);
    dstatG.alloc(1);
    NSP_CUDA(cudaMallocHost(&hstat, sizeof(DevStatus)));
    NSP_CUDA(cudaMallocHost(&hscal, 16 * sizeof(double)));
    NSP_CUDA(cudaMallocHost(&hint, 16 * sizeof(int32_t)));
    dscal.alloc(16);
    info.n = an.n;
    info.n_interior = an.nI;
    info.n_gamma = an.nG;
    info.nblocks = an.nblocks;
    info.nnz_L_interior = FI.h.nnz_L;
    info.nnz_L_gamma = FG.h.nnz_L;
    info.n_supernodes = FI.h.nsn + FG.h.nsn;
    info.ms_analyze = an.ms;
    info.failed_block = -1;
  }
  ~Engine() override {
    if (fstream) cudaStreamSynchronize(fstream);   // no kernel may outlive the buffers
    if (gstream) cudaStreamDestroy(gstream);
    if (fstream) cudaStreamDestroy(fstream);
    for (cudaEvent_t e : fev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : gev)
      if (e) cudaEventDestroy(e);
    if (h_any) cudaFreeHost(h_any);
    if (hstat) cudaFreeHost(hstat);
    if (hscal) cudaFreeHost(hscal);
    if (hint) cudaFreeHost(hint);
  }

  void sync() { NSP_CUDA(cudaStreamSynchronize(st)); }

  void check_status() {
    NSP_CUDA(cudaMemcpyAsync(hstat, dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    sync();
    if (hstat->code == DEV_NOT_SPD) {
      info.failed_block = hstat->aux < 0 ? an.nblocks : hstat->aux;
      throw Error(NSP_ERR_NOT_SPD, "non-positive pivot in a Cholesky factor");
    }
    if (hstat->code == DEV_BREAKDOWN) throw Error(NSP_ERR_BREAKDOWN, "block PCG breakdown");
    if (hstat->code == DEV_TIMEOUT) throw Error(NSP_ERR_TIMEOUT, "a device wait timed out");
    if (hstat->code != DEV_OK) throw Error(NSP_ERR_CUDA, "device error");
  }

  void ensure_ws(int sc) {
    if (sc <= s_ws) return;
    s_ws = sc;
    Bv.alloc((size_t)an.nI * sc);
    Yw.alloc((size_t)an.nI * sc);
    Xw.alloc((size_t)an.nI * sc);
    Uw.alloc((size_t)std::max<int64_t>(FI.h.upd_rows, 1) * sc);
    YwG.alloc((size_t)an.nG * sc);
    UwG.alloc((size_t)std::max<int64_t>(FG.h.upd_rows, 1) * sc);
  }

  // ---- numeric factorization of every A_b and of A_G (§2.3)
  void factorize(const double *val, bool on_device) override {
    auto t0 = Clock::now();
    NSP_CUDA(cudaMemcpyAsync(Aval.p, val, an.nnz * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    A_I.refresh(Aval.p, st);
    A_IG.refresh(Aval.p, st);
    A_GI.refresh(Aval.p, st);
    A_G.refresh(Aval.p, st);
    NSP_CUDA(cudaMemsetAsync(dstat.p, 0, sizeof(DevStatus), st));
    NSP_CUDA(cudaMemsetAsync(dstatG.p, 0, sizeof(DevStatus), st));
    // The interior and the A_G factors are independent: A_G's (one tree whose top levels hold
    // one or two large fronts each, so few CTAs are busy) runs on a second stream beside the
    // interior one, each with its own fronts and status word, joined before the checks.
    if (!fstream) {   // high priority: A_G's chain of large fronts is the critical path
      int lo = 0, hi = 0;
      NSP_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      NSP_CUDA(cudaStreamCreateWithPriority(&fstream, cudaStreamNonBlocking, hi));
      NSP_CUDA(cudaEventCreateWithFlags(&fev[0], cudaEventDisableTiming));
      NSP_CUDA(cudaEventCreateWithFlags(&fev[1], cudaEventDisableTiming));
    }
    if (gnest) {   // recursive A_G: the nested handle factorizes A_G's blocks and G2 block
      factor_forest(FI, panelI.p, front.p, dstat.p, st);
      check_factor_status(dstat.p, -1);
      launch_gather_values<double>(gnest_src.p, (int64_t)gnest_src.n, Aval.p, gnest_val.p, st);
      try {
        gnest->factorize(gnest_val.p, true);
      } catch (const Error &e) {   // a failed nested block reports the A_G block
        info.failed_block = an.nblocks;
        throw;
      }
      info.ms_factor = ms_since(t0);
      return;
    }
    NSP_CUDA(cudaEventRecord(fev[0], st));
    NSP_CUDA(cudaStreamWaitEvent(fstream, fev[0], 0));
    factor_forest(FG, panelG.p, frontG.p, dstatG.p, fstream);
    factor_forest(FI, panelI.p, front.p, dstat.p, st);
    NSP_CUDA(cudaEventRecord(fev[1], fstream));
    check_factor_status(dstat.p, -1);
    // the A_G factor is joined where it is first needed (join_fg), so that the work of the
    // build that needs only the interior factor overlaps its last fronts
    fg_pending = true;
    info.ms_factor = ms_since(t0);
  }

  // Orders the handle's stream after the A_G factorization and checks its status (a failure
  // in the A_G factor reports block nblocks). Called before every use of the A_G factor and
  // at the end of a build.
  // NSP_BIGCLUSTER=0 keeps 8-CTA clusters for every large front; =n uses 16-CTA clusters on
  // levels with at most n large fronts (measurements; default kFewFronts)
  static constexpr int kFewFronts = 4;
  static int few_fronts() {
    const char *e = std::getenv("NSP_BIGCLUSTER");
    return e ? std::max(0, std::atoi(e)) : kFewFronts;
  }
  static bool big_fronts_enabled() { return few_fronts() > 0; }
  bool fg_pending = false;
  void join_fg() {
    if (!fg_pending) return;
    fg_pending = false;
    NSP_CUDA(cudaStreamWaitEvent(st, fev[1], 0));
    check_factor_status(dstatG.p, an.nblocks);
  }

  void factor_forest(ForestData &F, T *panel, T *fronts, DevStatus *status, cudaStream_t s) {
    for (int l = 0; l < F.h.nlevels; ++l) {
      const int c0 = F.h.level_ptr[l], c1 = F.h.level_ptr[l + 1], ns = F.level_small[l];
      // fronts below kBigFront rows one CTA each; larger ones a cluster each, of 16 CTAs
      // where the level holds at most kFewFronts of them (the top of a single tree)
      const int nbig = c1 - c0 - ns;
      launch_factor_level<T>(F.dev, F.level_sn.p + c0, ns, Aval.p, fronts, panel, status, s, 0);
      launch_factor_level<T>(F.dev, F.level_sn.p + c0 + ns, nbig, Aval.p, fronts, panel, status,
                             s, nbig <= few_fronts() ? 2 : 1);
    }
  }

  void check_factor_status(const DevStatus *status, int block_override) {
    NSP_CUDA(cudaMemcpyAsync(hstat, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    sync();
    if (hstat->code == DEV_NOT_SPD) {
      info.failed_block = block_override >= 0 ? block_override : hstat->aux;
      throw Error(NSP_ERR_NOT_SPD, "non-positive pivot in a Cholesky factor");
    }
    if (hstat->code != DEV_OK) throw Error(NSP_ERR_CUDA, "device error in factorization");
  }

  // ---- X = A_b^{-1} B over a forest (internal order, s columns): one persistent launch
  // tune = false (the allocation-free apply): no autotuning when no grid is cached yet, the
  // default grid instead, so that the call never synchronizes
  void solve_forest(ForestData &F, const T *panel, const T *B, T *Ywk, T *Uwk, T *X, int sc,
                    bool tune = true) {
    F.vec_rows = sweep_vector_rows((int)sizeof(T));
    F.elem_bytes = (int)sizeof(T);
    F.blk_rows = F.h.nblocks == 1 ? narrow_tiles() : kSweepBlockRows;
    auto &P = F.plan(sc == 1, st);
    int grid = 0;
    auto it = P.tuned_grid.find(sc);
    if (const int forced = forced_scheduler(); forced != 0) {
      grid = forced > 0 ? 0 : forced == -2 ? (sc == 1 ? kVsmGrid - 1 : kBsmGrid) : kResidentGrid;
    } else if (it != P.tuned_grid.end()) {
      grid = it->second;
    } else if (tune && autotune_enabled() && !capturing()) {
      grid = tune_sweep(F, P, panel, B, Ywk, Uwk, X, sc);
      P.tuned_grid[sc] = grid;
    }
    if (grid == kBsmGrid && !(sc > 1 && bsm_sweep_fits<T>(P.d, sc))) grid = kResidentGrid;
    if (grid == kBsmGrid) {
      launch_bsm_sweep<T>(P.d, panel, B, Ywk, Uwk, X, sc, st);
      return;
    }
    if (grid <= kVsmGrid) {   // kVsmGrid - 1 + c: c CTAs per SM
      const int fits = sc == 1 ? vsm_sweep_fits<T>(P.d) : 0;
      grid = fits == 0 ? kResidentGrid : std::max(grid, kVsmGrid - fits + 1);
    }
    if (grid == kResidentGrid && F.h.nblocks < 2) grid = 0;
    if (grid <= kVsmGrid)
      launch_vsm_sweep<T>(F.dev, P.d, panel, B, X, kVsmGrid - grid + 1, st);
    else if (grid == kResidentGrid)
      launch_res_sweep<T>(F.dev, P.d, panel, B, Ywk, Uwk, X, sc, dstat.p, st);
    else
      launch_sweep<T>(F.dev, P.d, panel, B, Ywk, Uwk, X, sc, dstat.p, st, grid);
  }
  // grid codes besides persistent grid sizes: the block-resident sweep, the shared-memory
  // single-vector sweep with one (kVsmGrid) or two (kVsmGrid - 1) CTAs per SM, and the
  // column-sliced block sweep (kBsmGrid)
  static constexpr int kResidentGrid = -1, kVsmGrid = -2, kBsmGrid = -4;
  // NSP_SWEEP=resident / global / smem forces one scheduler (measurements; smem: for one
  // right-hand side the shared-memory single-vector sweep where it fits, with as many CTAs per
  // SM as fit, for several the column-sliced block sweep where it has a plan, else
  // resident); unset: the autotuner
  static int forced_scheduler() {
    const char *e = std::getenv("NSP_SWEEP");
    if (!e) return 0;
    if (e[0] == 'r') return -1;
    if (e[0] == 's') return -2;
    if (e[0] == 'g') return 1;
    return 0;
  }

  // Autotuner of the persistent sweep: the grid (CTAs resident per SM, 1 to the occupancy
  // limit) is timed on the handle's own forest and right-hand-side count with CUDA events,
  // once per (forest, s); the fastest is kept. Every candidate computes the same result.
  static bool autotune_enabled() {
    const char *e = std::getenv("NSP_AUTOTUNE");
    return !(e && e[0] == '0');
  }
  bool capturing() {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NSP_CUDA(cudaStreamIsCapturing(st, &cs));
    return cs != cudaStreamCaptureStatusNone;
  }
  std::vector<std::pair<int, float>> tune_log;
  int tune_sweep(ForestData &F, ForestData::Plan &P, const T *panel, const T *B, T *Ywk, T *Uwk,
                 T *X, int sc) {
    int dev = 0, sms = 0;
    NSP_CUDA(cudaGetDevice(&dev));
    NSP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int gmax = launch_sweep<T>(F.dev, P.d, panel, B, Ywk, Uwk, X, sc, dstat.p, st, 0);
    cudaEvent_t e0, e1;
    NSP_CUDA(cudaEventCreate(&e0));
    NSP_CUDA(cudaEventCreate(&e1));
    // a candidate's time: one untimed launch first (a kernel's first launch also loads its
    // module and sets its shared-memory limit), then the fastest of three timed launches
    auto time_of = [&](auto &&launch) {
      launch();
      float best_rep = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        NSP_CUDA(cudaEventRecord(e0, st));
        launch();
        NSP_CUDA(cudaEventRecord(e1, st));
        NSP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        NSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best_rep = std::min(best_rep, ms);
      }
      return best_rep;
    };
    int best = gmax;
    float best_ms = 1e30f;
    auto consider = [&](int grid, float ms) {
      tune_log.push_back({grid, ms});
      if (ms < best_ms) {
        best_ms = ms;
        best = grid;
      }
    };
    if (F.h.nblocks >= 2)   // the block-resident sweep is a candidate for forests of blocks
      consider(kResidentGrid, time_of([&] {
                 launch_res_sweep<T>(F.dev, P.d, panel, B, Ywk, Uwk, X, sc, dstat.p, st);
               }));
    if (sc > 1 && F.h.nblocks >= 2 && bsm_sweep_fits<T>(P.d, sc))
      consider(kBsmGrid, time_of([&] {
                 launch_bsm_sweep<T>(P.d, panel, B, Ywk, Uwk, X, sc, st);
               }));
    const int vfits = (sc == 1 && F.h.nblocks >= 2) ? vsm_sweep_fits<T>(P.d) : 0;
    for (int per_sm = 1; per_sm <= vfits; ++per_sm)
      consider(kVsmGrid - per_sm + 1, time_of([&] {
                 launch_vsm_sweep<T>(F.dev, P.d, panel, B, X, per_sm, st);
               }));
    for (int g = sms; g <= gmax; g += sms)
      consider(g, time_of([&] {
                 launch_sweep<T>(F.dev, P.d, panel, B, Ywk, Uwk, X, sc, dstat.p, st, g);
               }));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
  }
  void solve_I(const T *B, T *X, int sc) {
    ensure_ws(sc);
    solve_forest(FI, panelI.p, B, Yw.p, Uw.p, X, sc);
  }
  void solve_G(const T *B, T *X, int sc) {
    if (gnest) {
      gnest->nested_inverse(B, X, sc);
      return;
    }
    join_fg();
    ensure_ws(sc);
    solve_forest(FG, panelG.p, B, YwG.p, UwG.p, X, sc);
  }

  // ---- Recursive treatment of A_G (concluding section: systems with A_G replaced by systems
  // with a much smaller matrix). The nested handle gnest is an Engine on A_G itself, rows and
  // columns in this handle's internal Gamma order, split by the caller's gamma_part into
  // interior blocks C_i and a second-level interface G2; its Algorithm 2 gives M2' for the
  // Schur complement S_C = C_G2 - C_G2I C_I^{-1} C_IG2, and A_G^{-1} is replaced by the block
  // elimination of §2.3 eq. (A_LDLT) with M2' as the Schur solve (nested_inverse).
  std::unique_ptr<Engine<T>> gnest;
  DBuf<int64_t> gnest_src;             // nested CSR entry -> index into A's values
  DBuf<double> gnest_val;              // nested CSR values
  std::vector<int64_t> gnest_row;      // caller sketch row j (G2 in increasing index) -> row
  std::vector<double> gnest_sketch;    // the caller's nested sketch in the nested order
  void attach_gamma(const nsp_params &prm) override {
    const HostSub &S = an.A_G;         // rows: internal Gamma order; columns: the same order
    std::vector<int64_t> rp(an.nG + 1, 0), src;
    std::vector<int32_t> col;
    src.reserve(S.col.size());
    col.reserve(S.col.size());
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int32_t r = 0; r < S.nrows; ++r) {
      row.clear();
      for (int32_t q = S.rowptr[r]; q < S.rowptr[r + 1]; ++q) row.push_back({S.col[q], S.src[q]});
      std::sort(row.begin(), row.end());
      for (const auto &e : row) {
        col.push_back(e.first);
        src.push_back(e.second);
      }
      rp[r + 1] = (int64_t)col.size();
    }
    // labels in the nested order (internal Gamma index t <- caller Gamma index i2u_G[t])
    std::vector<int32_t> part2(an.nG);
    for (int64_t t = 0; t < an.nG; ++t) part2[t] = prm.gamma_part[an.i2u_G[t]];
    static const double unused_value = 0.0;   // the nested analysis reads the pattern only
    nsp_csr c{an.nG, rp.data(), col.data(), &unused_value, 0};
    nsp_partition P2{prm.gamma_nblocks, part2.data(), nullptr};
    gnest.reset(new Engine<T>(&c, rp.data(), col.data(), &P2, st));
    gnest_src.upload(src, st);
    gnest_val.alloc(src.size());
    // the nested caller order of G2 is increasing t; the caller's is increasing index in A
    std::vector<int64_t> u2t(an.nG), pos(an.nG, -1);
    for (int64_t t = 0; t < an.nG; ++t) u2t[an.i2u_G[t]] = t;
    int64_t q = 0;
    for (int64_t t = 0; t < an.nG; ++t)
      if (part2[t] < 0) pos[t] = q++;
    gnest_row.clear();
    for (int64_t u = 0; u < an.nG; ++u)
      if (prm.gamma_part[u] < 0) gnest_row.push_back(pos[u2t[u]]);
    // the full A_G factor is not needed: its panels and fronts are released
    panelG.release();
    frontG.release();
    info.nnz_L_gamma = gnest->FI.h.nnz_L + gnest->FG.h.nnz_L;
    info.n_gamma2 = gnest->an.nG;
    NSP_CUDA(cudaStreamSynchronize(st));   // the uploads read host vectors of this scope
  }
  // M2' of the nested handle (Algorithm 2 on A_G's split) with the handle's parameters
  void construct_gamma(const nsp_params &prm) {
    nsp_params p2 = prm;
    p2.k = prm.gamma_k;
    p2.p = prm.gamma_p;
    p2.eps_inner = prm.gamma_eps_inner;
    p2.seed = prm.seed + 1;
    p2.sketch = nullptr;
    p2.keep_intermediates = 0;
    p2.gamma_levels = 0;
    p2.gamma_sketch = nullptr;
    const int s2 = prm.gamma_k + prm.gamma_p;
    require(s2 <= gnest->an.nG, NSP_ERR_INVALID_ARG, "gamma_k + gamma_p exceeds the size of G2");
    if (prm.gamma_sketch) {
      gnest_sketch.assign((size_t)gnest->an.nG * s2, 0.0);
      for (size_t j = 0; j < gnest_row.size(); ++j)
        std::memcpy(&gnest_sketch[(size_t)gnest_row[j] * s2], prm.gamma_sketch + j * s2,
                    s2 * sizeof(double));
      p2.sketch = gnest_sketch.data();
    }
    gnest->construct(p2);
    gnest->prepare_nested();
    info.it_inner_gamma = gnest->info.it_inner;
    info.rank_gamma = gnest->rank;
  }
  // (on the nested handle) Zsig = Zt Sigma, the low-rank term of M2' in the handle precision
  DBuf<T> nz_sig, nz_bI, nz_bG, nz_y, nz_r, nz_z;
  DBuf<double> nz_dg, nz_c;
  void prepare_nested() {
    if (rank <= 0) return;
    std::vector<double> sig(k), dg((size_t)k * k, 0.0);
    NSP_CUDA(cudaMemcpyAsync(sig.data(), Sigma.p, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    for (int j = 0; j < k; ++j) dg[(size_t)j * k + j] = sig[j];
    nz_dg.upload(dg, st);
    nz_sig.ensure((size_t)an.nG * k);
    block_update(Zt.p, nz_dg.p, an.nG, k, k, T(1), nullptr, T(0), nz_sig.p);
    sync();
  }
  // (on the nested handle) X = A_G~^{-1} B, B and X in this handle's caller order (= the
  // outer handle's internal Gamma order), sc columns:
  //   y = C_I^{-1} b_I, r = b_G2 - C_G2I y, x_G2 = C_G2^{-1} r + Zt Sigma Zt^T r,
  //   x_I = C_I^{-1} (b_I - C_IG2 x_G2)
  void nested_inverse(const T *B, T *X, int sc) {
    const size_t ni = (size_t)an.nI * sc, ng = (size_t)an.nG * sc;
    nz_bI.ensure(ni);
    nz_y.ensure(ni);
    nz_bG.ensure(ng);
    nz_r.ensure(ng);
    nz_z.ensure(ng);
    launch_gather_rows<T, T>(i2g_I.p, an.nI, B, nz_bI.p, sc, st);
    launch_gather_rows<T, T>(i2g_G.p, an.nG, B, nz_bG.p, sc, st);
    solve_I(nz_bI.p, nz_y.p, sc);
    launch_spmm<T>(A_GI.dT(), nz_y.p, nz_r.p, sc, T(-1), nz_bG.p, T(1), st);
    solve_G(nz_r.p, nz_z.p, sc);
    if (rank > 0) {
      nz_c.ensure((size_t)k * sc);
      gram_n(Zt.p, nz_r.p, an.nG, k, sc, nz_c.p);                      // Zt^T r
      block_update(nz_sig.p, nz_c.p, an.nG, k, sc, T(1), nz_z.p, T(1), nz_z.p);
    }
    launch_spmm<T>(A_IG.dT(), nz_z.p, nz_bI.p, sc, T(-1), nz_bI.p, T(1), st);
    solve_I(nz_bI.p, nz_y.p, sc);
    launch_scatter_rows<T, T>(i2g_I.p, an.nI, nz_y.p, X, sc, st);
    launch_scatter_rows<T, T>(i2g_G.p, an.nG, nz_z.p, X, sc, st);
  }

  // ---- S_Gamma X (with_AG) or A_GI A_I^{-1} A_IG X (internal Gamma order)
  void schur_apply(const T *X, T *Yo, int sc, bool with_AG) {
    ensure_ws(sc);
    launch_spmm<T>(A_IG.dT(), X, Bv.p, sc, T(1), nullptr, T(0), st);
    solve_forest(FI, panelI.p, Bv.p, Yw.p, Uw.p, Xw.p, sc);
    if (with_AG) {
      launch_spmm<T>(A_G.dT(), X, Yo, sc, T(1), nullptr, T(0), st);
      launch_spmm<T>(A_GI.dT(), Xw.p, Yo, sc, T(-1), Yo, T(1), st);
    } else {
      launch_spmm<T>(A_GI.dT(), Xw.p, Yo, sc, T(1), nullptr, T(0), st);
    }
  }

  // ---- S_I V = A_I V - A_IG A_G^{-1} A_GI V (§4.1 eq. (SI)), interior order, sc columns
  int inner_form = NSP_FORM_SGAMMA;
  DBuf<T> siA, siB;
  // Half sweeps of the A_G factor in the internal interface order (where A_G = L L^T):
  // half = 1: O = L^{-1} V (R^{-T} in the caller's order), half = 2: O = L^{-T} V (R^{-1}).
  // The column-sliced sweep where it has a plan for this width, else the block-resident one.
  DBuf<T> G1;
  void half_G(int half, const T *V, T *O, int sc) {
    require(!gnest, NSP_ERR_UNSUPPORTED, "half sweeps need the A_G factor (gamma_levels = 0)");
    join_fg();
    FG.vec_rows = sweep_vector_rows((int)sizeof(T));
    FG.elem_bytes = (int)sizeof(T);
    auto &P = FG.plan(sc == 1, st);
    ensure_ws(sc);
    if (sc > 1 && bsm_sweep_fits<T>(P.d, sc)) {
      if (half == 1) launch_bsm_sweep<T>(P.d, panelG.p, V, O, UwG.p, nullptr, sc, st, 1);
      else launch_bsm_sweep<T>(P.d, panelG.p, nullptr, const_cast<T *>(V), UwG.p, O, sc, st, 2);
    } else {
      if (half == 1)
        launch_res_sweep<T>(FG.dev, P.d, panelG.p, V, O, UwG.p, nullptr, sc, dstat.p, st, 1);
      else
        launch_res_sweep<T>(FG.dev, P.d, panelG.p, nullptr, const_cast<T *>(V), UwG.p, O, sc,
                            dstat.p, st, 2);
    }
  }

  void apply_SI(const T *V, T *O, int sc) {
    launch_spmm<T>(A_GI.dT(), V, siA.p, sc, T(1), nullptr, T(0), st);
    solve_G(siA.p, siB.p, sc);
    launch_spmm<T>(A_I.dT(), V, O, sc, T(1), nullptr, T(0), st);
    launch_spmm<T>(A_IG.dT(), siB.p, O, sc, T(-1), O, T(1), st);
  }

  // ---- S_Gamma X with caller-order X, Y and every temporary carved from `scratch`
  // (no allocation). The sweep plan of the needed kind must already exist.
  static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
  size_t schur_noalloc_bytes(int sc) const override {
    const size_t e = sizeof(T) * (size_t)sc;
    return 2 * align256(an.nG * e) + 3 * align256(an.nI * e) +
           align256(std::max<int64_t>(FI.h.upd_rows, 1) * e);
  }
  void schur_apply_noalloc(const void *X, void *Yv, int sc, unsigned char *scratch) override {
    require(FI.plans[sc == 1 ? 1 : 0] != nullptr, NSP_ERR_INVALID_ARG,
            "no sweep plan for this width yet: run nsp_schur_apply once with the same s");
    const size_t e = sizeof(T) * (size_t)sc;
    unsigned char *q = scratch;
    auto take = [&](size_t bytes) { T *p = reinterpret_cast<T *>(q); q += align256(bytes); return p; };
    T *xi = take(an.nG * e), *yi = take(an.nG * e);
    T *b = take(an.nI * e), *yw = take(an.nI * e), *xw = take(an.nI * e);
    T *uw = take(std::max<int64_t>(FI.h.upd_rows, 1) * e);
    launch_gather_rows<T, T>(i2u_G.p, an.nG, (const T *)X, xi, sc, st);
    launch_spmm<T>(A_IG.dT(), xi, b, sc, T(1), nullptr, T(0), st);
    solve_forest(FI, panelI.p, b, yw, uw, xw, sc, false);
    launch_spmm<T>(A_G.dT(), xi, yi, sc, T(1), nullptr, T(0), st);
    launch_spmm<T>(A_GI.dT(), xw, yi, sc, T(-1), yi, T(1), st);
    launch_scatter_rows<T, T>(i2u_G.p, an.nG, yi, (T *)Yv, sc, st);
  }

  void gram(const T *X, const T *Yv, int s1, int s2, double *C) { gram_n(X, Yv, an.nG, s1, s2, C); }
  // X^T Y (n rows): FP32 on the tensor cores (3xTF32), FP64 on the SIMT pipes
  // every Gram sizes the chunk partials for its own (n, s1, s2): the SIMT kernel splits the
  // rows into more chunks when the output is a single tile
  void gram_n(const T *X, const T *Yv, int64_t n, int s1, int s2, double *C) {
    gram_work.ensure(gram_work_size(n, s1, s2));
    if constexpr (std::is_same<T, float>::value) {
      if (tc_enabled()) {
        launch_tc_gram(X, Yv, n, s1, s2, C, gram_work.p, dstat.p, st);
        return;
      }
    }
    launch_gram<T, T>(X, Yv, n, s1, s2, C, gram_work.p, st);
  }
  // Out = scale A M + beta C (A n x s1, M s1 x s2 FP64)
  DBuf<float> tc_mt;
  void block_update(const T *A, const double *M, int64_t n, int s1, int s2, T scale, const T *C,
                    T beta, T *Out) {
    if constexpr (std::is_same<T, float>::value) {
      if (tc_enabled()) {
        tc_mt.ensure(tc_update_work_floats(256, 256));
        launch_tc_block_update(A, M, n, s1, s2, scale, C, beta, Out, tc_mt.p, dstat.p, st);
        return;
      }
    }
    launch_block_update<T>(A, M, n, s1, s2, scale, C, beta, Out, st);
  }
  // NSP_TC=0 keeps the FP32 Grams and block updates on the SIMT pipes (measurements)
  static bool tc_enabled() {
    const char *e = std::getenv("NSP_TC");
    return !(e && e[0] == '0');
  }
  void gram_acc64(const T *X, const T *Yv, int s1, int s2, double *C) {
    gram_acc64_n(X, Yv, an.nG, s1, s2, C);
  }
  void gram_acc64_n(const T *X, const T *Yv, int64_t n, int s1, int s2, double *C) {
    gram_work.ensure(gram_work_size(n, s1, s2));
    launch_gram<T, double>(X, Yv, n, s1, s2, C, gram_work.p, st);
  }

  // ---- Algorithm 2
  void construct(const nsp_params &prm) override {
    auto t0 = Clock::now();
    require(prm.k > 0 && prm.p >= 0, NSP_ERR_INVALID_ARG, "k > 0 and p >= 0 required");
    s = prm.k + prm.p;
    k = prm.k;
    require(s <= 256, NSP_ERR_UNSUPPORTED, "k + p > 256");
    require(s <= an.nG, NSP_ERR_INVALID_ARG, "k + p exceeds the interface size");
    require(prm.inner_form == NSP_FORM_SGAMMA || prm.inner_form == NSP_FORM_SI,
            NSP_ERR_INVALID_ARG, "unknown inner form");
    require(prm.variant >= NSP_VARIANT_M2 && prm.variant <= NSP_VARIANT_M1,
            NSP_ERR_INVALID_ARG, "unknown preconditioner variant");
    variant = prm.variant;
    require(prm.q >= 0 && prm.q <= 16, NSP_ERR_INVALID_ARG, "power iterations q in [0, 16]");
    // M3 (§4.3): Nyström of S_I^{-1} from an n_interior x s sketch, always by the S_I
    // block PCG (S_I X = G_I, preconditioner A_I), without power iterations
    m3 = variant == NSP_VARIANT_M3 || variant == NSP_VARIANT_M3_ADEF;
    require(!m3 || prm.q == 0, NSP_ERR_UNSUPPORTED, "M3 takes no power iterations");
    // M1 (§4.1): the same steps on the sketch R^{-1} G, the Nyström core on (G, R^{-T} Y) and
    // Zb = R^{-1} Ub, with A_G = R^T R the handle's own factor
    const bool m1 = variant == NSP_VARIANT_M1;
    require(!m1 || prm.q == 0, NSP_ERR_UNSUPPORTED, "M1 takes no power iterations");
    keep = prm.keep_intermediates != 0;
    if (gnest) construct_gamma(prm);
    ensure_ws(s);
    const size_t ns = (size_t)an.nG * s;
    // block-PCG vector length: n_Gamma (S_Gamma form) or n_interior (S_I form)
    const bool si = m3 || prm.inner_form == NSP_FORM_SI;
    inner_form = si ? NSP_FORM_SI : NSP_FORM_SGAMMA;
    const int64_t nv = si ? an.nI : an.nG;
    const size_t nvs = (size_t)std::max<int64_t>(nv, 1) * s;
    for (DBuf<T> *b : {&G, &Y}) b->ensure(ns);
    for (DBuf<T> *b : {&Fh, &E, &R, &P, &Q, &Z, &W}) b->ensure(std::max(ns, nvs));
    if (si) {
      siA.ensure(ns);
      siB.ensure(ns);
    }
    const int64_t nmax = std::max(an.nG, nv);
    gram_work.ensure(std::max(gram_work_size(nmax, s, s), gram_work_size(nmax, s, 1)));
    for (DBuf<double> *b : {&PtQ, &PtR, &QtZ, &Cg, &alpha, &beta, &K, &Cn})
      b->ensure((size_t)s * s);
    Rinv.ensure((size_t)s * s);
    Lwork.ensure(core_work_size(s));
    colsq.ensure(s);
    bnorm.ensure(s);
    ratio.ensure(1);
    Mix.ensure((size_t)s * k);
    Sigma.ensure(k);
    nys_work.ensure(nystrom_work_size(s));
    mask.ensure(s);
    nkept.ensure(1);
    drank.ensure(1);
    NSP_CUDA(cudaMemsetAsync(dstat.p, 0, sizeof(DevStatus), st));

    // step 1: sketch G (caller order), moved to the internal order; for M3 the sketch G_I
    // (n_interior x s, interior order) goes straight into the block-PCG right-hand side Fh
    if (m3) {
      const size_t nis = (size_t)an.nI * s;
      draw_sketch(prm, nis);
      launch_gather_rows<double, T>(i2u_I.p, an.nI, g64.p, Fh.p, s, st);
      sync();
    } else {
      draw_sketch(prm, ns);
      launch_gather_rows<double, T>(i2u_G.p, an.nG, g64.p, G.p, s, st);
      if (m1) {   // keep G for the core; the block PCG runs on R^{-1} G
        G1.ensure(ns);
        NSP_CUDA(cudaMemcpyAsync(G1.p, G.p, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
        half_G(2, G1.p, G.p, s);
      }
      sync();
    }
    // q-power iteration (§2.1 eq. (power)): passes 0..q-1 apply B = A_GI S_I^{-1} A_IG to G
    // by steps 2-4 and replace G by an orthonormal basis of B G (thresholded Cholesky-QR,
    // dropped columns become zero columns); pass q gives the Y of step 4 for the final G.
    int it_power = 0, it = 0, active = s;
    double rat = 1.0;
    for (int pass = 0; pass <= prm.q; ++pass) {
      if (pass > 0) {
        it_power += it;
        gram_acc64(Y.p, Y.p, s, s, K.p);
        launch_chol_drop(K.p, s, prm.drop_tol, Rinv.p, mask.p, nkept.p, Lwork.p, st);
        block_update(Y.p, Rinv.p, an.nG, s, s, T(1), nullptr, T(0), G.p);
      }
      // steps 2-3: block PCG on S_Gamma E = A_GI A_I^{-1} A_IG G, preconditioner A_G^{-1}
      // (S_Gamma form), or on S_I X = F = A_IG G, preconditioner A_I^{-1} (S_I form, the
      // system of Algorithm 2 step 3 as the paper writes it, §5 setup)
      // (M3: Fh already holds G_I; X = S_I^{-1} G_I is Algorithm 1 step 2 for B = S_I^{-1})
      if (!m3 && si)
        launch_spmm<T>(A_IG.dT(), G.p, Fh.p, s, T(1), nullptr, T(0), st);   // step 2
      else if (!m3)
        schur_apply(G.p, Fh.p, s, false);
      launch_col_sumsq<T>(Fh.p, nv, s, colsq.p, gram_work.p, st);
      launch_sqrt_vec(colsq.p, s, bnorm.p, st);
      // Breakdown-free block PCG (the paper's inner solver, §5.1) with search directions kept
      // operator-orthonormal: W spans the new directions, Qw = S W, C = W^T Qw = L L^T
      // (columns whose pivot falls below drop_tol are dropped), P = W L^{-T}, Q = Qw L^{-T}, so
      // that P^T Q = I and alpha = P^T R, beta = -Q^T Z need no s x s solve. The block Krylov
      // space, hence every iterate E, is the one of the 2-norm-orthonormal form.
      NSP_CUDA(cudaMemsetAsync(E.p, 0, nvs * sizeof(T), st));
      NSP_CUDA(cudaMemcpyAsync(R.p, Fh.p, nvs * sizeof(T), cudaMemcpyDeviceToDevice, st));
      if (si) solve_I(R.p, W.p, s);         // W = Z0 = A_I^{-1} R0
      else solve_G(R.p, W.p, s);            // W = Z0 = A_G^{-1} R0
      it = 0;
      rat = 1.0;
      active = s;
      while (it < prm.max_inner_it) {
        if (si) apply_SI(W.p, Z.p, s);      // Z holds Qw = S_I W
        else schur_apply(W.p, Z.p, s, true);  // Z holds Qw = S_Gamma W
        gram_n(W.p, Z.p, nv, s, s, Cg.p);
        launch_chol_drop(Cg.p, s, prm.drop_tol, Rinv.p, mask.p, nkept.p, Lwork.p, st);
        block_update(W.p, Rinv.p, nv, s, s, T(1), nullptr, T(0), P.p);
        block_update(Z.p, Rinv.p, nv, s, s, T(1), nullptr, T(0), Q.p);
        gram_n(P.p, R.p, nv, s, s, alpha.p);   // alpha = P^T R
        block_update(P.p, alpha.p, nv, s, s, T(1), E.p, T(1), E.p);
        block_update(Q.p, alpha.p, nv, s, s, T(-1), R.p, T(1), R.p);
        ++it;
        launch_col_sumsq<T>(R.p, nv, s, colsq.p, gram_work.p, st);
        launch_max_ratio(colsq.p, bnorm.p, s, ratio.p, st);
        NSP_CUDA(cudaMemcpyAsync(hscal, ratio.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        NSP_CUDA(cudaMemcpyAsync(hint, nkept.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        sync();
        rat = hscal[0];
        active = hint[0];
        if (active == 0) {  // no search direction left: the last pass changed nothing
          --it;
          break;
        }
        if (!(rat > prm.eps_inner)) break;
        if (si) solve_I(R.p, Z.p, s);       // Z = A_I^{-1} R
        else solve_G(R.p, Z.p, s);          // Z = A_G^{-1} R
        gram_n(Q.p, Z.p, nv, s, s, beta.p);    // Q^T Z
        block_update(P.p, beta.p, nv, s, s, T(-1), Z.p, T(1), W.p);  // W = Z - P Q^T Z
      }
      check_status();
      // step 4: Y = A_GI X (S_I form) or Y = A_G E (S_Gamma form; = A_GI S_I^{-1} A_IG G);
      // M3 uses X itself (E, n_interior x s) as the Y of its Nyström step
      if (m3 || si)
        launch_spmm<T>(A_GI.dT(), E.p, Y.p, s, T(1), nullptr, T(0), st);
      else
        launch_spmm<T>(A_G.dT(), E.p, Y.p, s, T(1), nullptr, T(0), st);
    }
    info.it_inner = it;
    info.it_power = it_power;
    info.inner_residual = rat;
    info.inner_active_cols = active;
    info.ms_inner = ms_since(t0);
    auto t1 = Clock::now();
    // M1: F = R^{-T} Y takes the place of Y from here on (into Y, through W)
    if (m1) {
      half_G(1, Y.p, W.p, s);
      NSP_CUDA(cudaMemcpyAsync(Y.p, W.p, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }
    // steps 5-10 (M3: on G_I and X = S_I^{-1} G_I, n_interior rows; M1: on G and F)
    {
      const T *Ys = m3 ? E.p : Y.p, *Gs = m3 ? Fh.p : m1 ? G1.p : G.p;
      const int64_t ny = m3 ? an.nI : an.nG;
      gram_acc64_n(Ys, Ys, ny, s, s, K.p);
      gram_acc64_n(Gs, Ys, ny, s, s, Cn.p);
    }
    launch_nystrom_core(K.p, Cn.p, s, k, prm.eps_trunc_rel, 1e-14, Mix.p, Sigma.p, drank.p,
                        nys_work.p, st, 1, std::is_same<T, double>::value ? 1 : 0);
    NSP_CUDA(cudaMemcpyAsync(hint, drank.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    sync();
    rank = hint[0];
    info.rank = rank;
    U.ensure((size_t)an.nG * k);
    Zt.ensure((size_t)an.nG * k);
    Zs.ensure((size_t)an.nG * k);
    if (rank > 0) {
      if (m3) {
        // V = X Mix (n_interior x k), then U = A_GI V so that Zt = A_G^{-1} A_GI V = Zh
        block_update(E.p, Mix.p, an.nI, s, k, T(1), nullptr, T(0), W.p);
        launch_spmm<T>(A_GI.dT(), W.p, U.p, k, T(1), nullptr, T(0), st);
      } else {
        // U = Y Mix (columns beyond the rank are zero, Sigma there is zero)
        block_update(Y.p, Mix.p, an.nG, s, k, T(1), nullptr, T(0), U.p);
      }
      // step 11: Z = A_G^{-1} U (M1: Zb = R^{-1} Ub); the low-rank term kept as
      // Zs = Z Sigma^{1/2} in FP64
      if (m1) half_G(2, U.p, Zt.p, k);
      else solve_G(U.p, Zt.p, k);
      launch_gather_rows<T, double>(nullptr, an.nG, Zt.p, Zs.p, k, st);
      launch_scale_cols(Zs.p, an.nG, k, Sigma.p, true, st);
      if (variant == NSP_VARIANT_M2_ADEF || variant == NSP_VARIANT_M3_ADEF)
        build_adef(prm.drop_tol);
      sync();
    }
    join_fg();
    info.ms_core = ms_since(t1);
  }

  // ---- M_{2A-DEF} (§4.3): M = (I - Q S_G) A_G^{-1} + Q with Q = Zk E^{-1} Zk^T,
  // Zk = A_G^{-1} U and E = Zk^T S_G Zk. With E = L L^T (columns whose pivot falls below
  // drop_tol of their diagonal are dropped), Zd = Zk L^{-T} gives Q = Zd Zd^T, and
  // Wd = S_G Zd turns the S_G A_G^{-1} r of every application into Wd^T (A_G^{-1} r):
  // one S_G apply on k columns here, none per application.
  int variant = NSP_VARIANT_M2;
  bool m3 = false;
  DBuf<T> adefS;
  DBuf<double> Zd, Wd, adefT, Ead, Rad;
  DBuf<int32_t> adef_mask, adef_nk;
  void build_adef(double drop_tol) {
    const size_t nk = (size_t)an.nG * k;
    adefS.ensure(nk);
    for (DBuf<double> *b : {&Zd, &Wd, &adefT}) b->ensure(nk);
    Ead.ensure((size_t)k * k);
    Rad.ensure((size_t)k * k);
    adef_mask.ensure(k);
    adef_nk.ensure(1);
    schur_apply(Zt.p, adefS.p, k, true);                     // S_G Zk (handle precision)
    gram_acc64(Zt.p, adefS.p, k, k, Ead.p);                  // E = Zk^T S_G Zk
    launch_chol_drop(Ead.p, k, drop_tol, Rad.p, adef_mask.p, adef_nk.p, Lwork.p, st);
    launch_gather_rows<T, double>(nullptr, an.nG, Zt.p, adefT.p, k, st);
    launch_block_update<double>(adefT.p, Rad.p, an.nG, k, k, 1.0, nullptr, 0.0, Zd.p, st);
    launch_gather_rows<T, double>(nullptr, an.nG, adefS.p, adefT.p, k, st);
    launch_block_update<double>(adefT.p, Rad.p, an.nG, k, k, 1.0, nullptr, 0.0, Wd.p, st);
  }

  // ---- M2 r = A_G^{-1} r + Z Sigma Z^T r (internal order, FP64 in/out)
  DBuf<double> zt_vec;
  void m2_apply_internal(const double *r, double *z) {
    if (nseg > 1) {
      m2_batched(r, z);
      return;
    }
    if (std::is_same<T, double>::value) {
      solve_G(reinterpret_cast<const T *>(r), reinterpret_cast<T *>(z), 1);
    } else {
      sT.ensure(an.nG);
      sT2.ensure(an.nG);
      launch_gather_rows<double, T>(nullptr, an.nG, r, sT.p, 1, st);
      solve_G(sT.p, sT2.p, 1);
      launch_gather_rows<T, double>(nullptr, an.nG, sT2.p, z, 1, st);
    }
    if (rank > 0 && (variant == NSP_VARIANT_M2_ADEF || variant == NSP_VARIANT_M3_ADEF)) {
      // z = y + Zd (Zd^T r - Wd^T y) with y = A_G^{-1} r already in z
      zt_vec.ensure(2 * (size_t)k);
      launch_gemv_t(Zd.p, an.nG, k, r, zt_vec.p, dwork.p, st);
      launch_gemv_t(Wd.p, an.nG, k, z, zt_vec.p + k, dwork.p, st);
      launch_axpby(k, nullptr, -1.0, zt_vec.p + k, 1.0, zt_vec.p, st);
      launch_gemv_n(Zd.p, an.nG, k, zt_vec.p, 1.0, z, st);
    } else if (rank > 0) {
      zt_vec.ensure(k);
      launch_gemv_t(Zs.p, an.nG, k, r, zt_vec.p, dwork.p, st);
      launch_gemv_n(Zs.p, an.nG, k, zt_vec.p, 1.0, z, st);
    }
  }

  // interior solve on FP64 vectors with the T factor
  void solve_I64(const double *b, double *x) {
    if (std::is_same<T, double>::value) {
      solve_I(reinterpret_cast<const T *>(b), reinterpret_cast<T *>(x), 1);
    } else {
      sT.ensure(std::max(an.nI, an.nG));
      sT2.ensure(std::max(an.nI, an.nG));
      launch_gather_rows<double, T>(nullptr, an.nI, b, sT.p, 1, st);
      solve_I(sT.p, sT2.p, 1);
      launch_gather_rows<T, double>(nullptr, an.nI, sT2.p, x, 1, st);
    }
  }

  void schur64(const double *p, double *q) {
    if (std::is_same<T, double>::value) {
      schur_apply(reinterpret_cast<const T *>(p), reinterpret_cast<T *>(q), 1, true);
    } else {
      sT.ensure(std::max(an.nI, an.nG));
      sT2.ensure(std::max(an.nI, an.nG));
      launch_gather_rows<double, T>(nullptr, an.nG, p, sT.p, 1, st);
      schur_apply(sT.p, sT2.p, 1, true);
      launch_gather_rows<T, double>(nullptr, an.nG, sT2.p, q, 1, st);
    }
  }

  void apply_m2(const double *r, double *z) override {
    dwork.ensure(gram_work_size(std::max(an.n, an.nG), 256, 1));
    ri_buf.ensure(an.nG);
    zi_buf.ensure(an.nG);
    launch_gather_rows<double, double>(i2u_G.p, an.nG, r, ri_buf.p, 1, st);
    m2_apply_internal(ri_buf.p, zi_buf.p);
    launch_scatter_rows<double, double>(i2u_G.p, an.nG, zi_buf.p, z, 1, st);
    sync();
  }

  // ---- PCG (textbook; FP64 recurrences, scalars kept on the device)
  std::vector<double> lanczos_alpha, lanczos_beta;   // coefficients of the last outer PCG

  template <typename Aop, typename Mop>
  int pcg(int64_t n, Aop &&A, Mop &&M, const double *f, double *x, double rtol, int maxit,
          double *rel_out) {
    vr.ensure(n); vz.ensure(n); vp.ensure(n); vq.ensure(n);
    dwork.ensure(gram_work_size(std::max(an.n, an.nG), 256, 1));
    double *d_rz = dscal.p, *d_pq = dscal.p + 1, *d_alpha = dscal.p + 2, *d_beta = dscal.p + 3,
           *d_rr = dscal.p + 4, *d_rznew = dscal.p + 5, *d_ff = dscal.p + 6;
    NSP_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    NSP_CUDA(cudaMemcpyAsync(vr.p, f, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_dot(f, f, n, d_ff, dwork.p, st);
    NSP_CUDA(cudaMemcpyAsync(hscal, d_ff, sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    const double fn = std::sqrt(hscal[0]);
    *rel_out = 0.0;
    lanczos_alpha.clear();
    lanczos_beta.clear();
    if (fn == 0.0) return 0;
    M(vr.p, vz.p);
    NSP_CUDA(cudaMemcpyAsync(vp.p, vz.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_dot(vr.p, vz.p, n, d_rz, dwork.p, st);
    int it = 0;
    double rel = 1.0;
    // r^T z of the current and of the next direction: the two slots swap roles each
    // iteration (no copy)
    double *rz_cur = d_rz, *rz_next = d_rznew;
    while (it < maxit) {
      A(vp.p, vq.p);
      launch_dot(vp.p, vq.p, n, d_pq, dwork.p, st);
      // alpha = r^T z / p^T q, x += alpha p, r -= alpha q, r^T r: one fused pass
      launch_pcg_step(n, rz_cur, d_pq, d_alpha, vp.p, vq.p, x, vr.p, d_rr, dwork.p, st);
      ++it;
      // alpha_j, beta_{j-1} (the ratio that formed this direction) and r^T r in one copy
      NSP_CUDA(cudaMemcpyAsync(hscal + 2, d_alpha, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
      sync();
      lanczos_alpha.push_back(hscal[2]);
      if (it >= 2) lanczos_beta.push_back(hscal[3]);
      rel = std::sqrt(std::max(hscal[4], 0.0)) / fn;
      if (!(rel > rtol)) break;
      M(vr.p, vz.p);
      launch_dot(vr.p, vz.p, n, rz_next, dwork.p, st);
      launch_pcg_direction(n, rz_next, rz_cur, d_beta, vz.p, vp.p, st);   // p = z + beta p
      std::swap(rz_cur, rz_next);
    }
    *rel_out = rel;
    return it;
  }

  void solve(const double *b_user, double *x_user, double rtol, int maxit, int form) override {
    auto t0 = Clock::now();
    const int64_t n = an.n, nI = an.nI, nG = an.nG;
    vb.ensure(n); vx.ensure(n); vt.ensure(n); vu.ensure(n); vf.ensure(n);
    dwork.ensure(gram_work_size(std::max(an.n, an.nG), 256, 1));
    ensure_ws(1);
    if (form == NSP_OUTER_AUTO) form = std::is_same<T, double>::value ? NSP_OUTER_SCHUR : NSP_OUTER_FULL;
    // internal layout of full vectors: [interior (FI order); interface (FG order)]
    double *bI = vb.p, *bG = vb.p + nI;
    launch_gather_rows<double, double>(i2g_I.p, nI, b_user, bI, 1, st);
    launch_gather_rows<double, double>(i2g_G.p, nG, b_user, bG, 1, st);
    double rel = 0.0;
    int it = 0;
    if (form == NSP_OUTER_SCHUR) {
      // f = b_G - A_GI A_I^{-1} b_I
      solve_I64(bI, vt.p);
      launch_spmm<double>(A_GI.d64(), vt.p, vf.p, 1, -1.0, bG, 1.0, st);
      double *w = vx.p + nI;
      it = pcg(nG, [&](const double *p, double *q) { schur64(p, q); },
               [&](const double *r, double *z) { m2_apply_internal(r, z); }, vf.p, w, rtol,
               maxit, &rel);
      // x_I = A_I^{-1}(b_I - A_IG w)
      launch_spmm<double>(A_IG.d64(), w, vt.p, 1, -1.0, bI, 1.0, st);
      solve_I64(vt.p, vx.p);
    } else {
      // x0 = (A_I^{-1} b_I, 0); r0 = b - A x0; PCG on A d = r0 with the block preconditioner
      double *x0 = vu.p;
      solve_I64(bI, x0);
      NSP_CUDA(cudaMemsetAsync(x0 + nI, 0, nG * sizeof(double), st));
      auto Aop = [&](const double *v, double *o) {
        launch_spmm<double>(A_I.d64(), v, o, 1, 1.0, nullptr, 0.0, st);
        launch_spmm<double>(A_IG.d64(), v + nI, o, 1, 1.0, o, 1.0, st);
        launch_spmm<double>(A_GI.d64(), v, o + nI, 1, 1.0, nullptr, 0.0, st);
        launch_spmm<double>(A_G.d64(), v + nI, o + nI, 1, 1.0, o + nI, 1.0, st);
      };
      Aop(x0, vf.p);
      launch_axpby(n, nullptr, 1.0, vb.p, -1.0, vf.p, st);   // r0 = b - A x0
      pfull_t.ensure(n);
      auto Mop = [&](const double *r, double *z) {
        double *t = pfull_t.p;            // t_I = A_I^{-1} r_I, t_G = r_G - A_GI t_I
        solve_I64(r, t);
        launch_spmm<double>(A_GI.d64(), t, t + nI, 1, -1.0, r + nI, 1.0, st);
        m2_apply_internal(t + nI, z + nI);
        launch_spmm<double>(A_IG.d64(), z + nI, t, 1, -1.0, r, 1.0, st);   // r_I - A_IG z_G
        solve_I64(t, z);
      };
      it = pcg(n, Aop, Mop, vf.p, vx.p, rtol, maxit, &rel);
      launch_axpby(n, nullptr, 1.0, x0, 1.0, vx.p, st);     // x = x0 + d
    }
    // back to the caller's order; true residual ||b - A x|| / ||b|| in FP64
    launch_scatter_rows<double, double>(i2g_I.p, nI, vx.p, x_user, 1, st);
    launch_scatter_rows<double, double>(i2g_G.p, nG, vx.p + nI, x_user, 1, st);
    CsrDev<double> Af{(int32_t)n, (int32_t)n, an.nnz, full_rowptr.p, full_col.p, Aval.p};
    launch_spmm<double>(Af, x_user, vt.p, 1, -1.0, b_user, 1.0, st);
    launch_dot(vt.p, vt.p, n, dscal.p + 8, dwork.p, st);
    launch_dot(b_user, b_user, n, dscal.p + 9, dwork.p, st);
    NSP_CUDA(cudaMemcpyAsync(hscal + 8, dscal.p + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    check_status();
    info.it_pcg = it;
    info.pcg_residual = rel;
    lanczos_extremes(lanczos_alpha, lanczos_beta, &info.lambda_min_est, &info.lambda_max_est);
    info.kappa_est = info.lambda_min_est > 0 ? info.lambda_max_est / info.lambda_min_est : 0.0;
    info.final_residual = hscal[9] > 0 ? std::sqrt(hscal[8] / hscal[9]) : 0.0;
    info.ms_solve = ms_since(t0);
    if (rel > rtol) throw Error(NSP_ERR_NOT_CONVERGED, "outer PCG did not converge");
  }
  DBuf<double> pfull_t;

  // ==== batches of independent matrices (one block-diagonal problem, per-matrix algebra)
  struct Chunks {
    SegChunks d;
    DBuf<int64_t> row0, row1;
    DBuf<int32_t> seg, seg_first;
    void build(const std::vector<std::vector<std::pair<int64_t, int64_t>>> &ranges, int64_t len,
               cudaStream_t st) {
      std::vector<int64_t> a, b;
      std::vector<int32_t> sg, first(ranges.size() + 1, 0);
      for (size_t g = 0; g < ranges.size(); ++g) {
        first[g] = (int32_t)a.size();
        for (auto rg : ranges[g])
          for (int64_t r = rg.first; r < rg.second; r += len) {
            a.push_back(r);
            b.push_back(std::min(rg.second, r + len));
            sg.push_back((int32_t)g);
          }
      }
      first[ranges.size()] = (int32_t)a.size();
      row0.upload(a, st);
      row1.upload(b, st);
      seg.upload(sg, st);
      seg_first.upload(first, st);
      d = SegChunks{(int)a.size(), (int)ranges.size(), row0.p, row1.p, seg.p, seg_first.p};
    }
  };
  int nseg = 1;
  std::vector<int64_t> bmat_off;          // caller-order offsets of the matrices (nseg + 1)
  Chunks chG, chF, chU;                   // Gamma rows, internal full rows, caller rows
  DBuf<double> bwork, bscal, bK, bC, bSig;
  DBuf<int32_t> bactive;
  DBuf<int32_t> bits_in, bact_in, bgo, bpass;   // inner block-PCG bookkeeping of a batch
  DBuf<double> brat_in;
  std::vector<int64_t> seg_nG;            // interface size of every matrix

  void setup_batch(const std::vector<int64_t> &mat_off) override {
    nseg = (int)mat_off.size() - 1;
    bmat_off = mat_off;
    auto mat_of = [&](int64_t g) {
      return (int)(std::upper_bound(mat_off.begin(), mat_off.end(), g) - mat_off.begin()) - 1;
    };
    std::vector<std::vector<std::pair<int64_t, int64_t>>> rG(nseg), rF(nseg), rU(nseg);
    auto ranges = [&](const std::vector<int64_t> &i2g, int64_t base,
                      std::vector<std::vector<std::pair<int64_t, int64_t>>> &out) {
      // maximal runs of one matrix in the internal order (a matrix may own several runs)
      int64_t t = 0, n = (int64_t)i2g.size();
      while (t < n) {
        const int g = mat_of(i2g[t]);
        int64_t e = t;
        while (e < n && mat_of(i2g[e]) == g) ++e;
        out[g].push_back({base + t, base + e});
        t = e;
      }
    };
    ranges(an.i2g_G, 0, rG);
    ranges(an.i2g_I, 0, rF);
    ranges(an.i2g_G, an.nI, rF);
    for (int g = 0; g < nseg; ++g) rU[g].push_back({mat_off[g], mat_off[g + 1]});
    seg_nG.assign(nseg, 0);
    for (int g = 0; g < nseg; ++g)
      for (auto rg : rG[g]) seg_nG[g] += rg.second - rg.first;
    chG.build(rG, 1024, st);
    chF.build(rF, 2048, st);
    chU.build(rU, 2048, st);
    binfo.assign(nseg, info);
  }

  void construct_batched(const nsp_params &prm) override {
    require(prm.variant == NSP_VARIANT_M2, NSP_ERR_UNSUPPORTED,
            "batched handles build M2 only");
    require(prm.q == 0, NSP_ERR_UNSUPPORTED, "batched handles take no power iterations");
    auto t0 = Clock::now();
    require(prm.k > 0 && prm.p >= 0, NSP_ERR_INVALID_ARG, "k > 0 and p >= 0 required");
    s = prm.k + prm.p;
    k = prm.k;
    require(s <= 96, NSP_ERR_UNSUPPORTED, "batched handles support k + p <= 96");
    for (int64_t ng : seg_nG)
      require(s <= ng, NSP_ERR_INVALID_ARG, "k + p exceeds the interface size of a matrix");
    require(prm.inner_form == NSP_FORM_SGAMMA, NSP_ERR_UNSUPPORTED, "inner form");
    keep = prm.keep_intermediates != 0;
    ensure_ws(s);
    const size_t ns = (size_t)an.nG * s, ss = (size_t)s * s;
    for (DBuf<T> *b : {&G, &Fh, &E, &R, &P, &Q, &Z, &W, &Y}) b->ensure(ns);
    const int nch = std::max({chG.d.nchunk, chF.d.nchunk, chU.d.nchunk});
    bwork.ensure((size_t)nch * std::max<size_t>(ss, (size_t)s * k) + 64);
    for (DBuf<double> *b : {&Cg, &alpha, &beta, &Rinv, &bK, &bC}) b->ensure(nseg * ss);
    Lwork.ensure(nseg * core_work_size(s));
    nys_work.ensure(nseg * nystrom_work_size(s));
    colsq.ensure((size_t)nseg * s);
    bnorm.ensure((size_t)nseg * s);
    ratio.ensure(nseg);
    Mix.ensure((size_t)nseg * s * k);
    bSig.ensure((size_t)nseg * k);
    mask.ensure((size_t)nseg * s);
    nkept.ensure(nseg);
    drank.ensure(nseg);
    bactive.ensure(nseg);
    bscal.ensure(16 * (size_t)nseg);
    NSP_CUDA(cudaMemsetAsync(dstat.p, 0, sizeof(DevStatus), st));
    draw_sketch(prm, ns);
    launch_gather_rows<double, T>(i2u_G.p, an.nG, g64.p, G.p, s, st);
    // block PCG for every matrix at once (per-matrix scalars, one sweep per operator)
    schur_apply(G.p, Fh.p, s, false);
    launch_seg_colsq<T>(Fh.p, s, chG.d, colsq.p, bwork.p, st);
    launch_sqrt_vec(colsq.p, nseg * s, bnorm.p, st);
    NSP_CUDA(cudaMemsetAsync(E.p, 0, ns * sizeof(T), st));
    NSP_CUDA(cudaMemcpyAsync(R.p, Fh.p, ns * sizeof(T), cudaMemcpyDeviceToDevice, st));
    solve_G(R.p, W.p, s);
    // Per-matrix bookkeeping on the device (k_seg_inner_decide, which also masks the matrices
    // that stopped): the first iteration runs eagerly, so that every plan and workspace of the
    // loop exists, the others as a device-driven CUDA graph loop with no host decision.
    bits_in.ensure(nseg);
    brat_in.ensure(nseg);
    bact_in.ensure(nseg);
    bgo.ensure(1);
    bpass.ensure(2);
    std::vector<int32_t> its(nseg, 0), act_cols(nseg, s), ones(nseg, 1);
    std::vector<double> rat(nseg, 1.0);
    NSP_CUDA(cudaMemcpyAsync(bactive.p, ones.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NSP_CUDA(cudaMemcpyAsync(bits_in.p, its.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NSP_CUDA(cudaMemcpyAsync(bact_in.p, act_cols.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    NSP_CUDA(cudaMemcpyAsync(brat_in.p, rat.data(), nseg * sizeof(double), cudaMemcpyHostToDevice, st));
    NSP_CUDA(cudaMemsetAsync(bpass.p, 0, 2 * sizeof(int32_t), st));
    // Q = S W, P and Q made S-orthonormal, E += P alpha, R -= Q alpha, then the stopping rule
    auto first_half = [&](cudaGraphConditionalHandle h, int set_cond) {
      schur_apply(W.p, Z.p, s, true);
      launch_seg_gram<T, T>(W.p, Z.p, s, s, chG.d, Cg.p, bwork.p, st);
      launch_chol_drop(Cg.p, s, prm.drop_tol, Rinv.p, mask.p, nkept.p, Lwork.p, st, nseg);
      launch_seg_block_update<T>(W.p, Rinv.p, s, s, T(1), nullptr, T(0), P.p, chG.d, bactive.p, st);
      launch_seg_block_update<T>(Z.p, Rinv.p, s, s, T(1), nullptr, T(0), Q.p, chG.d, bactive.p, st);
      launch_seg_gram<T, T>(P.p, R.p, s, s, chG.d, alpha.p, bwork.p, st);
      launch_seg_block_update<T>(P.p, alpha.p, s, s, T(1), E.p, T(1), E.p, chG.d, bactive.p, st);
      launch_seg_block_update<T>(Q.p, alpha.p, s, s, T(-1), R.p, T(1), R.p, chG.d, bactive.p, st);
      launch_seg_colsq<T>(R.p, s, chG.d, colsq.p, bwork.p, st);
      launch_max_ratio(colsq.p, bnorm.p, s, ratio.p, st, nseg);
      launch_seg_inner_decide(ratio.p, nkept.p, prm.eps_inner, nseg, bactive.p, bits_in.p,
                              brat_in.p, bact_in.p, bgo.p, bpass.p, prm.max_inner_it, h,
                              set_cond, st);
    };
    // the next directions W = A_G^{-1} R - P Q^T A_G^{-1} R of the matrices still active
    auto second_half = [&]() {
      solve_G(R.p, Z.p, s);
      launch_seg_gram<T, T>(Q.p, Z.p, s, s, chG.d, beta.p, bwork.p, st);
      launch_seg_block_update<T>(P.p, beta.p, s, s, T(-1), Z.p, T(1), W.p, chG.d, bactive.p, st);
    };
    if (prm.max_inner_it > 0) {
      first_half(cudaGraphConditionalHandle(0), 0);
      NSP_CUDA(cudaMemcpyAsync(hint, bgo.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      sync();
      if (hint[0]) {
        device_while(
            [&](cudaGraphConditionalHandle h) {
              second_half();
              first_half(h, 1);
            },
            bpass.p);
      }
    }
    NSP_CUDA(cudaMemcpyAsync(its.data(), bits_in.p, nseg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaMemcpyAsync(act_cols.data(), bact_in.p, nseg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaMemcpyAsync(rat.data(), brat_in.p, nseg * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    check_status();
    auto t1 = Clock::now();
    launch_spmm<T>(A_G.dT(), E.p, Y.p, s, T(1), nullptr, T(0), st);
    launch_seg_gram<T, double>(Y.p, Y.p, s, s, chG.d, bK.p, bwork.p, st);
    launch_seg_gram<T, double>(G.p, Y.p, s, s, chG.d, bC.p, bwork.p, st);
    launch_nystrom_core(bK.p, bC.p, s, k, prm.eps_trunc_rel, 1e-14, Mix.p, bSig.p, drank.p,
                        nys_work.p, st, nseg, std::is_same<T, double>::value ? 1 : 0);
    U.ensure((size_t)an.nG * k);
    Zt.ensure((size_t)an.nG * k);
    Zs.ensure((size_t)an.nG * k);
    launch_seg_block_update<T>(Y.p, Mix.p, s, k, T(1), nullptr, T(0), U.p, chG.d, nullptr, st);
    solve_G(U.p, Zt.p, k);
    launch_seg_scale_sqrt<T>(Zt.p, k, bSig.p, chG.d, Zs.p, st);
    std::vector<int32_t> rk(nseg);
    NSP_CUDA(cudaMemcpyAsync(rk.data(), drank.p, nseg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    sync();
    const double ms_in = std::chrono::duration<double, std::milli>(t1 - t0).count();
    rank = 0;
    for (int g = 0; g < nseg; ++g) {
      binfo[g] = info;
      binfo[g].it_inner = its[g];
      binfo[g].inner_residual = rat[g];
      binfo[g].inner_active_cols = act_cols[g];
      binfo[g].rank = rk[g];
      binfo[g].ms_inner = ms_in;
      binfo[g].ms_core = ms_since(t1);
      rank = std::max(rank, rk[g]);
    }
    join_fg();
    info.ms_inner = ms_in;
    info.ms_core = ms_since(t1);
  }

  // M2 of every matrix on the interface part of a full internal vector (FP64)
  DBuf<double> bt;
  void m2_batched(const double *rG, double *zG) {
    if (std::is_same<T, double>::value) {
      solve_G(reinterpret_cast<const T *>(rG), reinterpret_cast<T *>(zG), 1);
    } else {
      sT.ensure(std::max(an.nI, an.nG));
      sT2.ensure(std::max(an.nI, an.nG));
      launch_gather_rows<double, T>(nullptr, an.nG, rG, sT.p, 1, st);
      solve_G(sT.p, sT2.p, 1);
      launch_gather_rows<T, double>(nullptr, an.nG, sT2.p, zG, 1, st);
    }
    bt.ensure((size_t)nseg * k);
    launch_seg_gram<double, double>(Zs.p, rG, k, 1, chG.d, bt.p, bwork.p, st);
    launch_seg_block_update<double>(Zs.p, bt.p, k, 1, 1.0, zG, 1.0, zG, chG.d, nullptr, st);
  }

  // Outer PCG of every matrix at once. The per-matrix bookkeeping (step counts, stopping
  // test, masks) lives on the device, so an iteration is a fixed sequence of launches with no
  // host decision; matrices that stop early are masked (alpha = 0).
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  DBuf<double> bfn, brel;
  DBuf<int32_t> bits, bany;
  int32_t *h_any = nullptr;

  // ---- Device-driven loops (CUDA graph conditional nodes): body(h) is captured once into
  // the body graph of a WHILE node whose conditional h the body's last kernel sets, so the
  // passes run back to back with no host decision; the body runs at least once. Captured and
  // launched on the engine's own non-blocking stream (the caller's may be the legacy default
  // stream, which cannot be captured), ordered after the handle's stream by events. Every
  // workspace, sweep plan and tuned grid the body uses must already exist (an eager pass
  // first), and the body must end every pass count at a bound (its kernels decide). `passes`
  // is a device counter the body increments once per pass: the launches of every pass are
  // added to the launch counter from it.
  template <class Body>
  void device_while(Body &&body, int32_t *passes) {
    if (!gstream) {
      NSP_CUDA(cudaStreamCreateWithFlags(&gstream, cudaStreamNonBlocking));
      NSP_CUDA(cudaEventCreateWithFlags(&gev[0], cudaEventDisableTiming));
      NSP_CUDA(cudaEventCreateWithFlags(&gev[1], cudaEventDisableTiming));
    }
    NSP_CUDA(cudaMemcpyAsync(hint + 9, passes, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    sync();
    const int32_t p0 = hint[9];
    cudaStream_t main_st = st;
    NSP_CUDA(cudaEventRecord(gev[0], main_st));
    NSP_CUDA(cudaStreamWaitEvent(gstream, gev[0], 0));
    struct Scope {   // restores the handle's stream and frees the graph on every exit
      cudaStream_t &ref, saved;
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      ~Scope() {
        ref = saved;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
      }
    } sc{st, main_st};
    st = gstream;
    NSP_CUDA(cudaGraphCreate(&sc.graph, 0));
    cudaGraphConditionalHandle h = 0;
    NSP_CUDA(cudaGraphConditionalHandleCreate(&h, sc.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    NSP_CUDA(cudaGraphAddNode(&node, sc.graph, nullptr, nullptr, 0, &np));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    const int64_t l0 = launches_counted();
    NSP_CUDA(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    try {
      body(h);
    } catch (...) {
      cudaGraph_t unused = nullptr;
      cudaStreamEndCapture(st, &unused);
      throw;
    }
    NSP_CUDA(cudaStreamEndCapture(st, &bodyg));
    const int64_t per_pass = launches_counted() - l0;
    add_launches(-per_pass);   // counted when they run
    NSP_CUDA(cudaGraphInstantiate(&sc.exec, sc.graph, 0));
    NSP_CUDA(cudaGraphLaunch(sc.exec, st));
    NSP_CUDA(cudaMemcpyAsync(hint + 8, passes, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaStreamSynchronize(st));
    add_launches(per_pass * (int64_t)(hint[8] - p0));
    NSP_CUDA(cudaEventRecord(gev[1], gstream));
    NSP_CUDA(cudaStreamWaitEvent(main_st, gev[1], 0));
  }

  void pcg_batched_iteration(double rtol, int maxit) {
    const int64_t n = an.n, nI = an.nI;
    double *sc = bscal.p;
    double *d_rz = sc, *d_pq = sc + nseg, *d_al = sc + 2 * nseg, *d_be = sc + 3 * nseg,
           *d_rr = sc + 4 * nseg, *d_rzn = sc + 5 * nseg;
    // q = A p
    launch_spmm<double>(A_I.d64(), vp.p, vq.p, 1, 1.0, nullptr, 0.0, st);
    launch_spmm<double>(A_IG.d64(), vp.p + nI, vq.p, 1, 1.0, vq.p, 1.0, st);
    launch_spmm<double>(A_GI.d64(), vp.p, vq.p + nI, 1, 1.0, nullptr, 0.0, st);
    launch_spmm<double>(A_G.d64(), vp.p + nI, vq.p + nI, 1, 1.0, vq.p + nI, 1.0, st);
    launch_seg_dot(vp.p, vq.p, chF.d, d_pq, bwork.p, st);
    launch_seg_ratio(d_rz, d_pq, bactive.p, nseg, d_al, st);
    launch_seg_axpby(chF.d, d_al, 1.0, vp.p, 1.0, vx.p, st);
    launch_seg_axpby(chF.d, d_al, -1.0, vq.p, 1.0, vr.p, st);
    launch_seg_dot(vr.p, vr.p, chF.d, d_rr, bwork.p, st);
    launch_seg_converge(d_rr, bfn.p, rtol, maxit, bactive.p, bits.p, brel.p, bany.p, nseg, st);
    // z = M r (block-factorization preconditioner with M2 of every matrix)
    double *t = pfull_t.p;
    solve_I64(vr.p, t);
    launch_spmm<double>(A_GI.d64(), t, t + nI, 1, -1.0, vr.p + nI, 1.0, st);
    m2_batched(t + nI, vz.p + nI);
    launch_spmm<double>(A_IG.d64(), vz.p + nI, t, 1, -1.0, vr.p, 1.0, st);
    solve_I64(t, vz.p);
    launch_seg_dot(vr.p, vz.p, chF.d, d_rzn, bwork.p, st);
    launch_seg_ratio(d_rzn, d_rz, bactive.p, nseg, d_be, st);
    launch_seg_axpby(chF.d, d_be, 1.0, vp.p, 0.0, vp.p, st);     // p = beta p
    launch_seg_axpby(chF.d, nullptr, 1.0, vz.p, 1.0, vp.p, st);  // p += z
    NSP_CUDA(cudaMemcpyAsync(d_rz, d_rzn, nseg * sizeof(double), cudaMemcpyDeviceToDevice, st));
    (void)n;
  }

  void solve_batched(const double *b_user, double *x_user, double rtol, int maxit) override {
    auto t0 = Clock::now();
    const int64_t n = an.n, nI = an.nI, nG = an.nG;
    vb.ensure(n); vx.ensure(n); vt.ensure(n); vu.ensure(n); vf.ensure(n);
    vr.ensure(n); vz.ensure(n); vp.ensure(n); vq.ensure(n); pfull_t.ensure(n);
    bfn.ensure(nseg); brel.ensure(nseg); bits.ensure(nseg); bany.ensure(1);
    if (!h_any) NSP_CUDA(cudaMallocHost(&h_any, sizeof(int32_t)));
    ensure_ws(1);
    double *sc = bscal.p;  // per matrix: rz, pq, alpha, beta, rr, rznew, ff, bb (8 x nseg)
    double *d_rz = sc, *d_rr = sc + 4 * nseg, *d_ff = sc + 6 * nseg, *d_bb = sc + 7 * nseg;
    double *bI = vb.p, *bG = vb.p + nI;
    launch_gather_rows<double, double>(i2g_I.p, nI, b_user, bI, 1, st);
    launch_gather_rows<double, double>(i2g_G.p, nG, b_user, bG, 1, st);
    // x0 = (A_I^{-1} b_I, 0); r0 = b - A x0
    double *x0 = vu.p;
    solve_I64(bI, x0);
    NSP_CUDA(cudaMemsetAsync(x0 + nI, 0, nG * sizeof(double), st));
    launch_spmm<double>(A_I.d64(), x0, vf.p, 1, 1.0, nullptr, 0.0, st);
    launch_spmm<double>(A_GI.d64(), x0, vf.p + nI, 1, 1.0, nullptr, 0.0, st);
    launch_axpby(n, nullptr, 1.0, vb.p, -1.0, vf.p, st);
    NSP_CUDA(cudaMemsetAsync(vx.p, 0, n * sizeof(double), st));
    NSP_CUDA(cudaMemcpyAsync(vr.p, vf.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_seg_dot(vf.p, vf.p, chF.d, d_ff, bwork.p, st);
    launch_seg_pcg_init(d_ff, nseg, bfn.p, bactive.p, bits.p, brel.p, st);
    // z0 = M r0, p0 = z0, rz = r0^T z0
    {
      double *t = pfull_t.p;
      solve_I64(vr.p, t);
      launch_spmm<double>(A_GI.d64(), t, t + nI, 1, -1.0, vr.p + nI, 1.0, st);
      m2_batched(t + nI, vz.p + nI);
      launch_spmm<double>(A_IG.d64(), vz.p + nI, t, 1, -1.0, vr.p, 1.0, st);
      solve_I64(t, vz.p);
    }
    NSP_CUDA(cudaMemcpyAsync(vp.p, vz.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_seg_dot(vr.p, vz.p, chF.d, d_rz, bwork.p, st);
    // one eager iteration (every workspace and sweep plan then exists), then the rest as a
    // device-driven CUDA graph loop: k_seg_converge's flag ends it, with no host decision
    pcg_batched_iteration(rtol, maxit);
    NSP_CUDA(cudaMemcpyAsync(h_any, bany.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    sync();
    if (*h_any != 0 && maxit > 1) {
      bpass.ensure(2);
      NSP_CUDA(cudaMemsetAsync(bpass.p + 1, 0, sizeof(int32_t), st));
      device_while(
          [&](cudaGraphConditionalHandle h) {
            pcg_batched_iteration(rtol, maxit);
            launch_loop_condition(bany.p, bpass.p + 1, h, st);
          },
          bpass.p + 1);
    }
    launch_axpby(n, nullptr, 1.0, x0, 1.0, vx.p, st);
    launch_scatter_rows<double, double>(i2g_I.p, nI, vx.p, x_user, 1, st);
    launch_scatter_rows<double, double>(i2g_G.p, nG, vx.p + nI, x_user, 1, st);
    CsrDev<double> Af{(int32_t)n, (int32_t)n, an.nnz, full_rowptr.p, full_col.p, Aval.p};
    launch_spmm<double>(Af, x_user, vt.p, 1, -1.0, b_user, 1.0, st);
    launch_seg_dot(vt.p, vt.p, chU.d, d_rr, bwork.p, st);
    launch_seg_dot(b_user, b_user, chU.d, d_bb, bwork.p, st);
    std::vector<double> rr(nseg), bb(nseg), rel(nseg);
    std::vector<int32_t> its(nseg);
    NSP_CUDA(cudaMemcpyAsync(rr.data(), d_rr, nseg * sizeof(double), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaMemcpyAsync(bb.data(), d_bb, nseg * sizeof(double), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaMemcpyAsync(rel.data(), brel.p, nseg * sizeof(double), cudaMemcpyDeviceToHost, st));
    NSP_CUDA(cudaMemcpyAsync(its.data(), bits.p, nseg * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    sync();
    check_status();
    bool ok = true;
    for (int g = 0; g < nseg; ++g) {
      binfo[g].it_pcg = its[g];
      binfo[g].pcg_residual = rel[g];
      binfo[g].final_residual = bb[g] > 0 ? std::sqrt(rr[g] / bb[g]) : 0.0;
      binfo[g].ms_solve = ms_since(t0);
      ok &= !(rel[g] > rtol);
    }
    info.ms_solve = ms_since(t0);
    if (!ok) throw Error(NSP_ERR_NOT_CONVERGED, "outer PCG did not converge for every matrix");
  }

  // Failure-detection check of the sweeps, on the handle's own interior forest: the plan's
  // epoch is moved 2^20 launches ahead of its counters, so every dependency wait of one sweep
  // is unreachable; the bounded waits (max_spins polls) must run out, abort the launch and
  // record DEV_TIMEOUT. The plan's counters and the status word are then reset, so the
  // handle stays usable. Returns the status the sweep reported.
  nsp_status timeout_selftest(int max_spins) override {
    FI.elem_bytes = (int)sizeof(T);
    auto &P = FI.plan(true, st);
    ensure_ws(1);
    sT.ensure(std::max(an.nI, an.nG));
    sT2.ensure(std::max(an.nI, an.nG));
    NSP_CUDA(cudaMemsetAsync(sT.p, 0, an.nI * sizeof(T), st));
    NSP_CUDA(cudaMemsetAsync(dstat.p, 0, sizeof(DevStatus), st));
    const uint32_t far = 1u << 20;
    NSP_CUDA(cudaMemcpyAsync(P.d.epoch, &far, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    launch_sweep<T>(FI.dev, P.d, panelI.p, sT.p, Yw.p, Uw.p, sT2.p, 1, dstat.p, st, 0, max_spins);
    NSP_CUDA(cudaMemcpyAsync(hstat, dstat.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    sync();
    const int32_t code = hstat->code;
    NSP_CUDA(cudaMemsetAsync(P.counters.p, 0, P.counters.bytes(), st));
    NSP_CUDA(cudaMemsetAsync(dstat.p, 0, sizeof(DevStatus), st));
    sync();
    return code == DEV_TIMEOUT ? NSP_ERR_TIMEOUT : code == DEV_OK ? NSP_OK : NSP_ERR_CUDA;
  }

  // ---- caller-order wrappers (asynchronous on the handle's stream, no allocation after
  // the first call with a given width)
  DBuf<T> io_a, io_b;
  void schur_apply_user(const void *X, void *Yv, int sc) override {
    ensure_ws(sc);
    io_a.ensure((size_t)an.nG * sc);
    io_b.ensure((size_t)an.nG * sc);
    launch_gather_rows<T, T>(i2u_G.p, an.nG, (const T *)X, io_a.p, sc, st);
    schur_apply(io_a.p, io_b.p, sc, true);
    launch_scatter_rows<T, T>(i2u_G.p, an.nG, io_b.p, (T *)Yv, sc, st);
  }
  void factor_solve_user(int which, const void *B, void *X, int sc) override {
    ensure_ws(sc);
    const int64_t nn = which == 0 ? an.nI : an.nG;
    const int64_t *perm = which == 0 ? i2u_I.p : i2u_G.p;
    io_a.ensure((size_t)std::max(an.nI, an.nG) * sc);
    io_b.ensure((size_t)std::max(an.nI, an.nG) * sc);
    launch_gather_rows<T, T>(perm, nn, (const T *)B, io_a.p, sc, st);
    if (which == 0) solve_I(io_a.p, io_b.p, sc);
    else solve_G(io_a.p, io_b.p, sc);
    launch_scatter_rows<T, T>(perm, nn, io_b.p, (T *)X, sc, st);
  }
  void get_basis(double *Zh, double *Sh, int32_t *rk) override {
    if (nseg > 1) {  // batch: all k columns, Sigma per matrix (nseg x k, zero beyond its rank)
      if (rk) *rk = k;
      if (Sh) {
        NSP_CUDA(cudaMemcpyAsync(Sh, bSig.p, (size_t)nseg * k * sizeof(double), cudaMemcpyDeviceToHost, st));
      }
      if (Zh) {
        DBuf<double> zu((size_t)an.nG * k);
        launch_scatter_rows<T, double>(i2u_G.p, an.nG, Zt.p, zu.p, k, st);
        NSP_CUDA(cudaMemcpyAsync(Zh, zu.p, (size_t)an.nG * k * sizeof(double), cudaMemcpyDeviceToHost, st));
      }
      sync();
      return;
    }
    if (rk) *rk = rank;
    if (rank <= 0) return;
    if (Sh) {
      NSP_CUDA(cudaMemcpyAsync(Sh, Sigma.p, rank * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (Zh) {
      DBuf<double> zu((size_t)an.nG * k);
      launch_scatter_rows<T, double>(i2u_G.p, an.nG, Zt.p, zu.p, k, st);
      std::vector<double> hz((size_t)an.nG * k);
      NSP_CUDA(cudaMemcpyAsync(hz.data(), zu.p, hz.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      sync();
      for (int64_t i = 0; i < an.nG; ++i)
        for (int j = 0; j < rank; ++j) Zh[i * rank + j] = hz[(size_t)i * k + j];
    }
    sync();
  }
  void get_intermediate(int which, double *out) override {
    require(keep, NSP_ERR_INVALID_ARG, "build without keep_intermediates");
    require(which >= 0 && which <= 3, NSP_ERR_INVALID_ARG, "intermediate id");
    require(which != 1 || inner_form == NSP_FORM_SGAMMA, NSP_ERR_INVALID_ARG,
            "the S_I form keeps no n_Gamma x s block E");
    require(!m3, NSP_ERR_INVALID_ARG, "M3 keeps no n_Gamma x s intermediates");
    const T *src = which == 0 ? G.p : which == 1 ? E.p : which == 2 ? Y.p : U.p;
    const int cols = which == 3 ? k : s;
    DBuf<double> o((size_t)an.nG * std::max(cols, 1));
    launch_scatter_rows<T, double>(i2u_G.p, an.nG, src, o.p, cols, st);
    std::vector<double> h((size_t)an.nG * cols);
    NSP_CUDA(cudaMemcpyAsync(h.data(), o.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    const int oc = which == 3 ? rank : s;
    for (int64_t i = 0; i < an.nG; ++i)
      for (int j = 0; j < oc; ++j) out[i * oc + j] = h[(size_t)i * cols + j];
  }
  void get_factor(int block, int64_t *order, double *L, int64_t nb) override {
    require(block >= 0 && block <= an.nblocks, NSP_ERR_INVALID_ARG, "block id");
    const bool g = block == an.nblocks;
    require(!(g && gnest), NSP_ERR_UNSUPPORTED, "A_G is not factorized (gamma_levels = 1)");
    join_fg();
    const Forest &F = g ? FG.h : FI.h;
    const int b = g ? 0 : block;
    const int64_t off = F.block_off[b], n_b = F.block_off[b + 1] - off;
    require(nb == n_b, NSP_ERR_INVALID_ARG, "n_b does not match the block size");
    std::vector<T> pan(F.panel_size);
    NSP_CUDA(cudaMemcpyAsync(pan.data(), g ? panelG.p : panelI.p, F.panel_size * sizeof(T),
                             cudaMemcpyDeviceToHost, st));
    sync();
    for (int64_t t = 0; t < n_b; ++t) order[t] = g ? an.i2g_G[off + t] : an.i2g_I[off + t];
    std::fill(L, L + n_b * n_b, 0.0);
    for (int J = 0; J < F.nsn; ++J) {
      if (F.sn_block[J] != b) continue;
      const int w = F.sn_w[J], m = F.sn_m[J], ld = panel_ld(m);
      const T *Pj = pan.data() + F.sn_panel[J];
      // L11 = inv(Pj_top) by forward substitution; L21 = Pj_bot L11
      std::vector<double> Li((size_t)w * w, 0.0), L11((size_t)w * w, 0.0);
      for (int r = 0; r < w; ++r)
        for (int c = 0; c <= r; ++c) Li[r + (size_t)c * w] = (double)Pj[r + (size_t)c * ld];
      for (int c = 0; c < w; ++c)
        for (int r = c; r < w; ++r) {
          double v = (r == c) ? 1.0 : 0.0;
          for (int t = c; t < r; ++t) v -= Li[r + (size_t)t * w] * L11[t + (size_t)c * w];
          L11[r + (size_t)c * w] = v / Li[r + (size_t)r * w];
        }
      const int64_t first = F.sn_first[J] - off;
      for (int c = 0; c < w; ++c) {
        for (int r = c; r < w; ++r)
          L[(first + r) + (first + c) * n_b] = L11[r + (size_t)c * w];
        for (int r = w; r < m; ++r) {
          double v = 0.0;
          for (int t = c; t < w; ++t) v += (double)Pj[r + (size_t)t * ld] * L11[t + (size_t)c * w];
          const int64_t row = F.rows[F.sn_rowptr[J] + r] - off;
          L[row + (first + c) * n_b] = v;
        }
      }
    }
  }
};

}  // namespace nsp

// ------------------------------------------------------------------ C ABI
struct nsp_handle {
  std::unique_ptr<nsp::EngineBase> eng;
  nsp_params prm{};
  int32_t batch = 0;   // number of matrices of a batched handle (0: single matrix)
};

namespace nsp {
static thread_local std::string g_last_error;
void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }
}  // namespace nsp

static nsp_status guard(const std::function<void()> &f) {
  try {
    f();
    return NSP_OK;
  } catch (const nsp::Error &e) {
    nsp::set_last_error(e.what());
    return e.status;
  } catch (const std::bad_alloc &) {
    nsp::set_last_error("host allocation failed");
    return NSP_ERR_OOM;
  } catch (const std::exception &e) {
    nsp::set_last_error(e.what());
    return NSP_ERR_INVALID_ARG;
  } catch (...) {
    nsp::set_last_error("unknown exception");
    return NSP_ERR_INVALID_ARG;
  }
}

extern "C" {

void nsp_default_params(nsp_params *prm) {
  if (!prm) return;
  std::memset(prm, 0, sizeof(*prm));
  prm->k = 16;
  prm->p = 10;
  prm->eps_inner = 0.1;
  prm->eps_trunc_rel = 1e-10;
  prm->drop_tol = 1e-6;
  prm->max_inner_it = 500;
  prm->seed = 210112164ull;
  prm->sketch = nullptr;
  prm->precision = NSP_FP32;
  prm->outer_form = NSP_OUTER_AUTO;
  prm->inner_form = NSP_FORM_SGAMMA;
  prm->keep_intermediates = 0;
  prm->stream = nullptr;
  prm->gamma_levels = 0;
  prm->gamma_k = 16;
  prm->gamma_p = 8;
  prm->gamma_eps_inner = 0.1;
}

const char *nsp_last_error(void) { return nsp::g_last_error.c_str(); }

const char *nsp_status_string(nsp_status s) {
  switch (s) {
    case NSP_OK: return "ok";
    case NSP_ERR_INVALID_ARG: return "invalid argument";
    case NSP_ERR_NOT_DBBD: return "partition is not doubly bordered block diagonal";
    case NSP_ERR_NOT_SPD: return "matrix block is not positive definite";
    case NSP_ERR_BREAKDOWN: return "block PCG breakdown";
    case NSP_ERR_NOT_CONVERGED: return "iteration did not converge";
    case NSP_ERR_TIMEOUT: return "device wait timed out";
    case NSP_ERR_CUDA: return "CUDA error";
    case NSP_ERR_OOM: return "out of device memory";
    case NSP_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static nsp::EngineBase *make_engine(const nsp_csr *A, const int64_t *rp, const int32_t *ci,
                                    const nsp_partition *P, const nsp_params *prm) {
  cudaStream_t st = (cudaStream_t)prm->stream;
  if (prm->precision == NSP_FP64) return new nsp::Engine<double>(A, rp, ci, P, st);
  if (prm->precision == NSP_FP32) return new nsp::Engine<float>(A, rp, ci, P, st);
  throw nsp::Error(NSP_ERR_INVALID_ARG, "precision");
}

// The parameter checks of Engine::construct / construct_batched that need no analysis, in the
// same order and with the same status codes, run on the host before any device work so that
// a malformed request fails fast (the engine repeats them).
static void validate_params(const nsp_params *prm, bool batched) {
  nsp::require(prm != nullptr, NSP_ERR_INVALID_ARG, "params");
  nsp::require(prm->precision == NSP_FP64 || prm->precision == NSP_FP32, NSP_ERR_INVALID_ARG,
               "precision");
  nsp::require(prm->gamma_levels == 0 || prm->gamma_levels == 1, NSP_ERR_INVALID_ARG,
               "gamma_levels must be 0 or 1");
  if (batched) {
    nsp::require(prm->gamma_levels == 0, NSP_ERR_UNSUPPORTED,
                 "batched handles factorize A_G directly (gamma_levels = 0)");
    nsp::require(prm->variant == NSP_VARIANT_M2, NSP_ERR_UNSUPPORTED,
                 "batched handles build M2 only");
    nsp::require(prm->q == 0, NSP_ERR_UNSUPPORTED, "batched handles take no power iterations");
    nsp::require(prm->k > 0 && prm->p >= 0, NSP_ERR_INVALID_ARG, "k > 0 and p >= 0 required");
    nsp::require(prm->k + prm->p <= 96, NSP_ERR_UNSUPPORTED, "batched handles support k + p <= 96");
    return;
  }
  nsp::require(prm->k > 0 && prm->p >= 0, NSP_ERR_INVALID_ARG, "k > 0 and p >= 0 required");
  nsp::require(prm->k + prm->p <= 256, NSP_ERR_UNSUPPORTED, "k + p > 256");
  // the engine's next checks (k + p <= n_Gamma, then these) all answer NSP_ERR_INVALID_ARG
  nsp::require(prm->inner_form == NSP_FORM_SGAMMA || prm->inner_form == NSP_FORM_SI,
               NSP_ERR_INVALID_ARG, "unknown inner form");
  nsp::require(prm->variant >= NSP_VARIANT_M2 && prm->variant <= NSP_VARIANT_M1,
               NSP_ERR_INVALID_ARG, "unknown preconditioner variant");
  nsp::require(prm->q >= 0 && prm->q <= 16, NSP_ERR_INVALID_ARG, "power iterations q in [0, 16]");
  if (prm->gamma_levels == 1) {
    nsp::require(prm->variant == NSP_VARIANT_M2 && prm->inner_form == NSP_FORM_SGAMMA &&
                     prm->q == 0,
                 NSP_ERR_UNSUPPORTED,
                 "the recursive A_G takes the M2 variant, the S_Gamma inner form and q = 0");
    nsp::require(prm->gamma_k > 0 && prm->gamma_p >= 0, NSP_ERR_INVALID_ARG,
                 "gamma_k > 0 and gamma_p >= 0 required");
    nsp::require(prm->gamma_k + prm->gamma_p <= 256, NSP_ERR_UNSUPPORTED, "gamma_k + gamma_p > 256");
  }
}

// the A_G split of a recursive build (nsp_build only: nsp_rebuild keeps the build's split)
static void validate_gamma_split(const nsp_params *prm) {
  if (prm->gamma_levels == 1)
    nsp::require(prm->gamma_part && prm->gamma_nblocks >= 1, NSP_ERR_INVALID_ARG,
                 "gamma_levels = 1 needs gamma_part and gamma_nblocks >= 1");
}

nsp_status nsp_build(const nsp_csr *A, const nsp_partition *P, const nsp_params *prm,
                     nsp_handle **out) {
  if (!out) return NSP_ERR_INVALID_ARG;
  *out = nullptr;
  auto h = std::make_unique<nsp_handle>();
  nsp_status s = guard([&] {
    nsp::validate_csr(A);
    validate_params(prm, false);
    validate_gamma_split(prm);
    h->prm = *prm;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    const int64_t *rpp = A->rowptr;
    const int32_t *cip = A->col;
    if (A->on_device) {  // pattern is analysed on the host
      rp.resize(A->n + 1);
      NSP_CUDA(cudaMemcpy(rp.data(), A->rowptr, (A->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
      ci.resize(rp[A->n]);
      NSP_CUDA(cudaMemcpy(ci.data(), A->col, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
      rpp = rp.data();
      cip = ci.data();
    }
    h->eng.reset(make_engine(A, rpp, cip, P, prm));
    if (prm->gamma_levels == 1) h->eng->attach_gamma(*prm);
    h->eng->factorize(A->val, A->on_device != 0);
    h->eng->construct(h->prm);
  });
  if (s == NSP_OK) *out = h.release();
  return s;
}

nsp_status nsp_build_batched(int32_t count, const nsp_csr *A, const nsp_partition *P,
                             const nsp_params *prm, nsp_handle **out) {
  if (!out || count < 1 || !A || !P || !prm) return NSP_ERR_INVALID_ARG;
  *out = nullptr;
  auto h = std::make_unique<nsp_handle>();
  nsp_status s = guard([&] {
    validate_params(prm, true);
    h->prm = *prm;
    h->batch = count;
    // block-diagonal concatenation: unknowns and interior blocks renumbered matrix by matrix
    int64_t n = 0, nnz = 0;
    int32_t nb = 0;
    std::vector<int64_t> off(count + 1, 0);
    for (int m = 0; m < count; ++m) {
      nsp::validate_csr(&A[m]);
      nsp::require(!A[m].on_device, NSP_ERR_INVALID_ARG, "batched build needs host CSR");
      nsp::require(P[m].part && P[m].nblocks >= 1, NSP_ERR_INVALID_ARG, "partition");
      off[m + 1] = off[m] + A[m].n;
      nnz += A[m].rowptr[A[m].n];
      nb += P[m].nblocks;
    }
    n = off[count];
    std::vector<int64_t> rp(n + 1, 0), perm;
    std::vector<int32_t> col, part(n);
    std::vector<double> val;
    col.reserve(nnz);
    val.reserve(nnz);
    bool any_perm = false, all_perm = true;
    for (int m = 0; m < count; ++m) { any_perm |= P[m].perm != nullptr; all_perm &= P[m].perm != nullptr; }
    nsp::require(any_perm == all_perm, NSP_ERR_INVALID_ARG, "batched: give perm for all matrices or none");
    int32_t boff = 0;
    for (int m = 0; m < count; ++m) {
      const nsp_csr &a = A[m];
      for (int64_t i = 0; i < a.n; ++i) {
        for (int64_t e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
          col.push_back((int32_t)(a.col[e] + off[m]));
          val.push_back(a.val[e]);
        }
        rp[off[m] + i + 1] = (int64_t)col.size();
        const int32_t pt = P[m].part[i];
        part[off[m] + i] = pt < 0 ? -1 : pt + boff;
      }
      if (all_perm) {
        int64_t ni = 0;
        for (int64_t i = 0; i < a.n; ++i) ni += P[m].part[i] >= 0;
        for (int64_t q = 0; q < ni; ++q) perm.push_back(P[m].perm[q] + off[m]);
      }
      boff += P[m].nblocks;
    }
    nsp_csr Asup{n, rp.data(), col.data(), val.data(), 0};
    nsp_partition Psup{nb, part.data(), all_perm ? perm.data() : nullptr};
    h->eng.reset(make_engine(&Asup, rp.data(), col.data(), &Psup, prm));
    h->eng->setup_batch(off);
    h->eng->factorize(val.data(), false);
    h->eng->construct_batched(h->prm);
  });
  if (s == NSP_OK) *out = h.release();
  return s;
}

nsp_status nsp_solve_batched(const nsp_handle *h, const double *b, double *x, double rtol,
                             int32_t maxit, nsp_info *infos) {
  if (!h || !h->eng || h->batch < 1 || !b || !x || !(rtol > 0) || maxit < 1)
    return NSP_ERR_INVALID_ARG;
  nsp_status s = guard([&] {
    const int64_t n = h->eng->info.n;
    cudaStream_t st = h->eng->st;
    const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
    const double *bp = b;
    double *xp = x;
    if (!bd) {
      h->eng->stage_b.ensure(n);
      NSP_CUDA(cudaMemcpyAsync(h->eng->stage_b.p, b, n * sizeof(double), cudaMemcpyHostToDevice, st));
      bp = h->eng->stage_b.p;
    }
    if (!xd) {
      h->eng->stage_x.ensure(n);
      xp = h->eng->stage_x.p;
    }
    nsp_status inner = NSP_OK;
    try {
      h->eng->solve_batched(bp, xp, rtol, maxit);
    } catch (const nsp::Error &e) {
      if (e.status != NSP_ERR_NOT_CONVERGED) throw;
      inner = e.status;
    }
    if (!xd) {
      NSP_CUDA(cudaMemcpyAsync(x, xp, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      NSP_CUDA(cudaStreamSynchronize(st));
    }
    if (inner != NSP_OK) throw nsp::Error(inner, "not converged");
  });
  if (infos)
    for (int m = 0; m < h->batch && m < (int)h->eng->binfo.size(); ++m) infos[m] = h->eng->binfo[m];
  return s;
}

nsp_status nsp_rebuild(nsp_handle *h, const double *val, int32_t on_device, const nsp_params *prm) {
  if (!h || !h->eng || !val) return NSP_ERR_INVALID_ARG;
  return guard([&] {
    if (prm) {
      nsp::require(prm->precision == h->prm.precision, NSP_ERR_INVALID_ARG, "precision change");
      nsp::require(prm->gamma_levels == h->prm.gamma_levels, NSP_ERR_INVALID_ARG,
                   "gamma_levels change");
      validate_params(prm, h->batch > 0);
      void *stream = h->prm.stream;
      h->prm = *prm;
      h->prm.stream = stream;
    }
    h->eng->factorize(val, on_device != 0);
    if (h->batch > 0)
      h->eng->construct_batched(h->prm);
    else
      h->eng->construct(h->prm);
  });
}

nsp_status nsp_check_timeout_path(const nsp_handle *h, int32_t max_spins, int32_t *observed) {
  if (!h || !h->eng || !observed || max_spins < 1) return NSP_ERR_INVALID_ARG;
  return guard([&] { *observed = h->eng->timeout_selftest(max_spins); });
}

nsp_status nsp_apply(const nsp_handle *h, const double *r, double *z) {
  if (!h || !h->eng || !r || !z) return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->apply_m2(r, z); });
}


nsp_status nsp_solve(const nsp_handle *h, const double *b, double *x, double rtol, int32_t maxit,
                     nsp_info *info) {
  if (!h || !h->eng || !b || !x || !(rtol > 0) || maxit < 1) return NSP_ERR_INVALID_ARG;
  if (h->batch > 0) return NSP_ERR_INVALID_ARG;   // batched handles: nsp_solve_batched
  nsp_status s = guard([&] {
    const int64_t n = h->eng->info.n;
    cudaStream_t st = h->eng->st;
    const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
    const double *bp = b;
    double *xp = x;
    if (!bd) {
      h->eng->stage_b.ensure(n);
      NSP_CUDA(cudaMemcpyAsync(h->eng->stage_b.p, b, n * sizeof(double), cudaMemcpyHostToDevice, st));
      bp = h->eng->stage_b.p;
    }
    if (!xd) {
      h->eng->stage_x.ensure(n);
      xp = h->eng->stage_x.p;
    }
    nsp_status inner = NSP_OK;
    try {
      h->eng->solve(bp, xp, rtol, maxit, h->prm.outer_form);
    } catch (const nsp::Error &e) {
      if (e.status != NSP_ERR_NOT_CONVERGED) throw;
      inner = e.status;
    }
    if (!xd) {
      NSP_CUDA(cudaMemcpyAsync(x, xp, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      NSP_CUDA(cudaStreamSynchronize(st));
    }
    if (inner != NSP_OK) throw nsp::Error(inner, "not converged");
  });
  if (info) *info = h->eng->info;
  return s;
}

nsp_status nsp_schur_apply(const nsp_handle *h, const void *X, void *Y, int32_t s) {
  if (!h || !h->eng || !X || !Y || s < 1 || s > 256) return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->schur_apply_user(X, Y, s); });
}

nsp_status nsp_factor_solve(const nsp_handle *h, int32_t which, const void *B, void *X, int32_t s) {
  if (!h || !h->eng || !B || !X || s < 1 || s > 256 || (which != 0 && which != 1))
    return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->factor_solve_user(which, B, X, s); });
}

nsp_status nsp_get_basis(const nsp_handle *h, double *Z, double *Sigma, int32_t *rank) {
  if (!h || !h->eng) return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->get_basis(Z, Sigma, rank); });
}

nsp_status nsp_get_intermediate(const nsp_handle *h, int32_t which, double *out) {
  if (!h || !h->eng || !out) return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->get_intermediate(which, out); });
}

nsp_status nsp_get_factor(const nsp_handle *h, int32_t block, int64_t *order, double *L, int64_t n_b) {
  if (!h || !h->eng || !order || !L) return NSP_ERR_INVALID_ARG;
  return guard([&] { h->eng->get_factor(block, order, L, n_b); });
}

nsp_status nsp_get_info(const nsp_handle *h, nsp_info *info) {
  if (!h || !h->eng || !info) return NSP_ERR_INVALID_ARG;
  *info = h->eng->info;
  return NSP_OK;
}

nsp_status nsp_destroy(nsp_handle *h) {
  if (!h) return NSP_ERR_INVALID_ARG;
  delete h;
  return NSP_OK;
}

int64_t nsp_kernel_launches(void) { return nsp::g_launches.load(); }

}  // extern "C"

// Scratch of nsp_schur_apply_noalloc: a fixed device array that every GPU using this library
// holds until the process exits. Host code must not use the symbol as an address: the device
// address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_schur_scratch[NSP_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mutex;
void *g_scratch_ptr[128] = {nullptr};

unsigned char *scratch_for_current_device() {
  int dev = 0;
  NSP_CUDA(cudaGetDevice(&dev));
  nsp::require(dev >= 0 && dev < 128, NSP_ERR_UNSUPPORTED, "device ordinal beyond 127");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    NSP_CUDA(cudaGetSymbolAddress(&p, g_schur_scratch));
    g_scratch_ptr[dev] = p;
  }
  return static_cast<unsigned char *>(g_scratch_ptr[dev]);
}
}  // namespace

extern "C" {

nsp_status nsp_schur_apply_noalloc(const nsp_handle *h, const void *X, void *Y, int32_t s) {
  if (!h || !h->eng || !X || !Y || s < 1 || s > 256) return NSP_ERR_INVALID_ARG;
  return guard([&] {
    nsp::require(h->eng->schur_noalloc_bytes(s) <= (size_t)NSP_NOALLOC_SCRATCH_BYTES,
                 NSP_ERR_INVALID_ARG,
                 "problem too large for the fixed scratch of nsp_schur_apply_noalloc");
    unsigned char *scratch = scratch_for_current_device();
    h->eng->schur_apply_noalloc(X, Y, s, scratch);
  });
}

// partials of either Gram kernel, then the status word
static size_t gram_partials_bytes(int64_t n, int32_t s1, int32_t s2) {
  return nsp::gram_work_size(n, s1, s2) * sizeof(double);
}
int64_t nsp_gram_work_bytes(int64_t n, int32_t s1, int32_t s2) {
  if (n < 0 || s1 < 1 || s2 < 1 || s1 > 256 || s2 > 256) return -1;
  return (int64_t)gram_partials_bytes(n, s1, s2) + 256;
}
nsp_status nsp_gram_compensated(const float *X, const float *Y, int64_t n, int32_t s1,
                                int32_t s2, double *C, void *work, void *stream) {
  if (!X || !Y || !C || !work || n < 0 || s1 < 1 || s2 < 1 || s1 > 256 || s2 > 256)
    return NSP_ERR_INVALID_ARG;
  return guard([&] {
    const cudaStream_t st = (cudaStream_t)stream;
    auto *status = reinterpret_cast<nsp::DevStatus *>(static_cast<unsigned char *>(work) +
                                                      gram_partials_bytes(n, s1, s2));
    NSP_CUDA(cudaMemsetAsync(status, 0, sizeof(nsp::DevStatus), st));
    nsp::launch_gram<float, double>(X, Y, n, s1, s2, C, static_cast<double *>(work), st);
  });
}
nsp_status nsp_gram(const float *X, const float *Y, int64_t n, int32_t s1, int32_t s2,
                    double *C, void *work, void *stream) {
  if (!X || !Y || !C || !work || n < 0 || s1 < 1 || s2 < 1 || s1 > 256 || s2 > 256)
    return NSP_ERR_INVALID_ARG;
  return guard([&] {
    const cudaStream_t st = (cudaStream_t)stream;
    auto *status = reinterpret_cast<nsp::DevStatus *>(static_cast<unsigned char *>(work) +
                                                      gram_partials_bytes(n, s1, s2));
    NSP_CUDA(cudaMemsetAsync(status, 0, sizeof(nsp::DevStatus), st));
    nsp::launch_tc_gram(X, Y, n, s1, s2, C, static_cast<double *>(work), status, st);
  });
}
int64_t nsp_block_update_work_bytes(int32_t s1, int32_t s2) {
  if (s1 < 1 || s2 < 1 || s1 > 256 || s2 > 256) return -1;
  return (int64_t)(nsp::tc_update_work_floats(s1, s2) * sizeof(float)) + 256;
}
nsp_status nsp_block_update(const float *A, const double *M, int64_t n, int32_t s1, int32_t s2,
                            float scale, const float *Cin, float beta, float *Out, void *work,
                            void *stream) {
  if (!A || !M || !Out || !work || n < 0 || s1 < 1 || s2 < 1 || s1 > 256 || s2 > 256)
    return NSP_ERR_INVALID_ARG;
  return guard([&] {
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t off = nsp::tc_update_work_floats(s1, s2) * sizeof(float);
    auto *status = reinterpret_cast<nsp::DevStatus *>(static_cast<unsigned char *>(work) + off);
    NSP_CUDA(cudaMemsetAsync(status, 0, sizeof(nsp::DevStatus), st));
    nsp::launch_tc_block_update(A, M, n, s1, s2, scale, Cin, beta, Out,
                                static_cast<float *>(work), status, st);
  });
}

nsp_status nsp_gaussian(uint64_t seed, int64_t count, double *out, void *stream) {
  if (!out || count < 0) return NSP_ERR_INVALID_ARG;
  return guard([&] {
    nsp::launch_gaussian<double>(seed, count, out, (cudaStream_t)stream);
    NSP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

// Host-only analysis (no CUDA call): validation, DBBD check, orderings and symbolic
// factorization statistics.
nsp_status nsp_analyze(const nsp_csr *A, const nsp_partition *P, nsp_info *info) {
  if (!info) return NSP_ERR_INVALID_ARG;
  return guard([&] {
    nsp::validate_csr(A);
    nsp::require(!A->on_device, NSP_ERR_INVALID_ARG, "nsp_analyze needs host CSR");
    nsp::Analysis an;
    nsp::analyze(A, A->rowptr, A->col, P, an);
    std::memset(info, 0, sizeof(*info));
    info->n = an.n;
    info->n_interior = an.nI;
    info->n_gamma = an.nG;
    info->nblocks = an.nblocks;
    info->nnz_L_interior = an.FI.nnz_L;
    info->nnz_L_gamma = an.FG.nnz_L;
    info->n_supernodes = an.FI.nsn + an.FG.nsn;
    info->ms_analyze = an.ms;
    info->failed_block = -1;
  });
}

}  // extern "C"
