// Symbolic analysis for the supernodal multifrontal Cholesky factors (see symbolic.h).
//
// Textbook building blocks, written from their definitions:
//  * elimination tree by Liu's ancestor/path-compression algorithm;
//  * postorder by depth-first search (children before parents);
//  * column counts by row subtrees: row k of L has a nonzero in column j exactly when j is
//    on a path of the elimination tree from some j' (A(k, j') != 0, j' < k) up to k;
//  * fundamental supernodes (j-1 the only child of j and cc(j-1) = cc(j) + 1), then relaxed
//    amalgamation of a supernode with its last child when few explicit zeros are added;
//  * supernode row structure = own columns + A's rows + children's structures;
//  * nested dissection by level-structure bisection from a pseudo-peripheral vertex.
#include "symbolic.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <functional>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <thread>

namespace nsp {

// ------------------------------------------------------------------ nested dissection
namespace {

struct NDState {
  const Graph &g;
  std::vector<int32_t> label;   // current part of each vertex, -1 = already ordered
  std::vector<int32_t> dist;
  std::vector<int32_t> queue;
  std::vector<int32_t> out;
  int32_t next_label = 1;
  int32_t leaf;
  explicit NDState(const Graph &gr, int32_t lf) : g(gr), label(gr.n, 0), dist(gr.n, -1), leaf(lf) {
    queue.reserve(gr.n);
    out.reserve(gr.n);
  }

  int32_t degree_in(int32_t v, int32_t lab) const {
    int32_t d = 0;
    for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) d += label[g.adj[e]] == lab;
    return d;
  }

  // BFS over vertices labelled lab from src; fills queue (visit order) and dist.
  // Returns eccentricity. Resets dist of visited vertices only at the next call's start.
  int32_t bfs(int32_t src, int32_t lab) {
    for (int32_t v : queue) dist[v] = -1;
    queue.clear();
    queue.push_back(src);
    dist[src] = 0;
    size_t h = 0;
    while (h < queue.size()) {
      int32_t v = queue[h++];
      for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
        int32_t u = g.adj[e];
        if (label[u] == lab && dist[u] < 0) {
          dist[u] = dist[v] + 1;
          queue.push_back(u);
        }
      }
    }
    return dist[queue.back()];
  }

  void order(std::vector<int32_t> verts, int32_t lab) {
    if (verts.empty()) return;
    if ((int32_t)verts.size() <= leaf) {
      // leaf: breadth-first order from a minimum-degree vertex (keeps the leaf banded)
      int32_t s = verts[0], dmin = 1 << 30;
      for (int32_t v : verts) {
        int32_t d = degree_in(v, lab);
        if (d < dmin) { dmin = d; s = v; }
      }
      std::vector<int32_t> acc;
      while (true) {
        bfs(s, lab);
        for (int32_t v : queue) { acc.push_back(v); label[v] = -1; }
        s = -1;
        for (int32_t v : verts) if (label[v] == lab) { s = v; break; }
        if (s < 0) break;
      }
      for (int32_t v : acc) out.push_back(v);
      for (int32_t v : queue) dist[v] = -1;
      queue.clear();
      return;
    }
    // connected components of the set
    {
      int32_t s = verts[0];
      bfs(s, lab);
      if (queue.size() < verts.size()) {
        std::vector<std::vector<int32_t>> comps;
        std::vector<int32_t> comp_label;
        for (int32_t v : verts) {
          if (label[v] != lab) continue;
          bfs(v, lab);
          int32_t nl = next_label++;
          for (int32_t u : queue) label[u] = nl;
          comps.emplace_back(queue.begin(), queue.end());
          comp_label.push_back(nl);
        }
        for (size_t c = 0; c < comps.size(); ++c) order(std::move(comps[c]), comp_label[c]);
        return;
      }
    }
    // pseudo-peripheral vertex (George & Liu)
    int32_t start = verts[0], dmin = 1 << 30;
    for (int32_t v : verts) {
      int32_t d = degree_in(v, lab);
      if (d < dmin) { dmin = d; start = v; }
    }
    int32_t ecc = bfs(start, lab);
    for (int iter = 0; iter < 8; ++iter) {
      int32_t best = -1, bd = 1 << 30;
      for (int32_t v : queue)
        if (dist[v] == ecc) {
          int32_t d = degree_in(v, lab);
          if (d < bd) { bd = d; best = v; }
        }
      int32_t e2 = bfs(best, lab);
      if (e2 <= ecc) { bfs(start, lab); break; }
      start = best;
      ecc = e2;
    }
    int32_t nv = (int32_t)queue.size();
    if (ecc < 2) {  // nearly complete graph: treat as a leaf
      int32_t keep = leaf;
      leaf = nv;
      order(std::move(verts), lab);
      leaf = keep;
      return;
    }
    std::vector<int32_t> cnt(ecc + 1, 0);
    for (int32_t v : queue) cnt[dist[v]]++;
    // separator level: smallest level among balanced candidates, else the median level
    int32_t best_l = -1, best_c = 1 << 30, below = 0, med = -1;
    for (int32_t l = 0; l <= ecc; ++l) {
      int32_t above = nv - below - cnt[l];
      if (med < 0 && below + cnt[l] >= nv / 2) med = l;
      if (l >= 1 && l <= ecc - 1) {
        int32_t rest = nv - cnt[l];
        if (below >= 0.3 * rest && above >= 0.3 * rest && cnt[l] < best_c) {
          best_c = cnt[l];
          best_l = l;
        }
      }
      below += cnt[l];
    }
    if (best_l < 0) best_l = std::min(std::max(med, 1), ecc - 1);
    std::vector<int32_t> A, B, S;
    std::vector<int32_t> vis(queue.begin(), queue.end());
    for (int32_t v : vis) {
      int32_t d = dist[v];
      if (d < best_l) {
        A.push_back(v);
      } else if (d > best_l) {
        B.push_back(v);
      } else {
        bool touches = false;
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
          int32_t u = g.adj[e];
          if (label[u] == lab && dist[u] == best_l + 1) { touches = true; break; }
        }
        (touches ? S : A).push_back(v);
      }
    }
    for (int32_t v : vis) dist[v] = -1;
    queue.clear();
    int32_t la = next_label++, lb = next_label++;
    for (int32_t v : A) label[v] = la;
    for (int32_t v : B) label[v] = lb;
    for (int32_t v : S) label[v] = -1;
    order(std::move(A), la);
    order(std::move(B), lb);
    for (int32_t v : S) out.push_back(v);
  }
};

}  // namespace

std::vector<int32_t> nested_dissection(const Graph &g, int32_t leaf) {
  NDState st(g, std::max<int32_t>(leaf, 1));
  std::vector<int32_t> all(g.n);
  std::iota(all.begin(), all.end(), 0);
  st.order(std::move(all), 0);
  if ((int32_t)st.out.size() != g.n) throw std::runtime_error("nested_dissection: lost vertices");
  return st.out;
}

// ------------------------------------------------------------------ forest analysis
namespace {

struct LocalSym {
  std::vector<int32_t> post;      // new -> old (postorder of the elimination tree)
  std::vector<int32_t> parent;    // new numbering
  std::vector<int64_t> cc;        // column counts (diagonal included)
  // lower triangle by columns in new numbering
  std::vector<int64_t> colptr;
  std::vector<int32_t> rowidx;
  std::vector<int64_t> src;
};

void local_symbolic(const BlockPattern &P, LocalSym &L) {
  const int32_t n = P.n;
  // strict lower triangle by rows (row i -> columns j < i), old numbering
  std::vector<int64_t> rp(n + 1, 0);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t e = P.colptr[j]; e < P.colptr[j + 1]; ++e)
      if (P.rowidx[e] > j) rp[P.rowidx[e] + 1]++;
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  std::vector<int32_t> ci(rp[n]);
  {
    std::vector<int64_t> pos(rp.begin(), rp.end() - 1);
    for (int32_t j = 0; j < n; ++j)
      for (int64_t e = P.colptr[j]; e < P.colptr[j + 1]; ++e)
        if (P.rowidx[e] > j) ci[pos[P.rowidx[e]]++] = j;
  }
  // elimination tree (Liu)
  std::vector<int32_t> parent(n, -1), anc(n, -1);
  for (int32_t k = 0; k < n; ++k) {
    for (int64_t e = rp[k]; e < rp[k + 1]; ++e) {
      int32_t i = ci[e];
      while (i != -1 && i < k) {
        int32_t inext = anc[i];
        anc[i] = k;
        if (inext == -1) parent[i] = k;
        i = inext;
      }
    }
  }
  // postorder (children visited in increasing order)
  std::vector<int32_t> head(n, -1), next(n, -1);
  for (int32_t j = n - 1; j >= 0; --j)
    if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
  L.post.clear();
  L.post.reserve(n);
  std::vector<int32_t> stack;
  for (int32_t r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      int32_t v = stack.back();
      int32_t c = head[v];
      if (c == -1) {
        stack.pop_back();
        L.post.push_back(v);
      } else {
        head[v] = next[c];
        stack.push_back(c);
      }
    }
  }
  std::vector<int32_t> ipost(n);
  for (int32_t k = 0; k < n; ++k) ipost[L.post[k]] = k;
  L.parent.assign(n, -1);
  for (int32_t k = 0; k < n; ++k) {
    int32_t p = parent[L.post[k]];
    L.parent[k] = p < 0 ? -1 : ipost[p];
  }
  // lower triangle by columns in new numbering (rows sorted)
  L.colptr.assign(n + 1, 0);
  for (int32_t jn = 0; jn < n; ++jn) {
    int32_t jo = L.post[jn];
    L.colptr[jn + 1] = L.colptr[jn] + (P.colptr[jo + 1] - P.colptr[jo]);
  }
  L.rowidx.resize(L.colptr[n]);
  L.src.resize(L.colptr[n]);
  std::vector<std::pair<int32_t, int64_t>> tmp;
  for (int32_t jn = 0; jn < n; ++jn) {
    int32_t jo = L.post[jn];
    tmp.clear();
    for (int64_t e = P.colptr[jo]; e < P.colptr[jo + 1]; ++e) {
      int32_t in = ipost[P.rowidx[e]];
      if (in < jn) throw std::runtime_error("postorder broke the lower triangle");
      tmp.emplace_back(in, P.src[e]);
    }
    std::sort(tmp.begin(), tmp.end());
    int64_t o = L.colptr[jn];
    for (size_t t = 0; t < tmp.size(); ++t) { L.rowidx[o + t] = tmp[t].first; L.src[o + t] = tmp[t].second; }
  }
  // column counts by row subtrees
  std::vector<int64_t> rpn(n + 1, 0);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t e = L.colptr[j]; e < L.colptr[j + 1]; ++e)
      if (L.rowidx[e] > j) rpn[L.rowidx[e] + 1]++;
  for (int32_t i = 0; i < n; ++i) rpn[i + 1] += rpn[i];
  std::vector<int32_t> cin(rpn[n]);
  {
    std::vector<int64_t> pos(rpn.begin(), rpn.end() - 1);
    for (int32_t j = 0; j < n; ++j)
      for (int64_t e = L.colptr[j]; e < L.colptr[j + 1]; ++e)
        if (L.rowidx[e] > j) cin[pos[L.rowidx[e]]++] = j;
  }
  L.cc.assign(n, 0);
  std::vector<int32_t> mark(n, -1);
  for (int32_t k = 0; k < n; ++k) {
    mark[k] = k;
    L.cc[k] += 1;
    for (int64_t e = rpn[k]; e < rpn[k + 1]; ++e) {
      int32_t i = cin[e];
      while (mark[i] != k) {
        mark[i] = k;
        L.cc[i] += 1;
        i = L.parent[i];
        if (i < 0) throw std::runtime_error("row subtree left the tree");
      }
    }
  }
}

// Allowed fraction of explicit zeros in a merged supernode by merged width (<=16, <=32,
// <=64, larger), per relaxation level.
const double kRelax[4][4] = {{0, 0, 0, 0},
                             {0.5, 0.15, 0.1, 0.05},
                             {0.8, 0.5, 0.25, 0.05},
                             {0.9, 0.7, 0.4, 0.1}};

// Whether merging (child C immediately before J) is acceptable.
bool accept_merge(int relax, int64_t wc, int64_t wj, int64_t mj, int64_t nz) {
  if (relax <= 0) return false;
  const int64_t w = wc + wj, m = wc + mj;
  const int64_t ent = w * m - w * (w - 1) / 2;
  const double zf = double(ent - nz) / double(ent);
  const double *tab = kRelax[relax > 3 ? 3 : relax];
  if (w <= 8) return true;
  if (w <= 16) return zf < tab[0];
  if (w <= 32) return zf < tab[1];
  if (w <= 64) return zf < tab[2];
  return zf < tab[3];
}

}  // namespace

// Symbolic analysis of one block in block-local numbering (offsets from 0): supernodes,
// their row structures, levels, panel / front / update-row offsets, relative maps and
// assembly lists. analyze_forest concatenates the blocks.
static void analyze_block(const BlockPattern &P, int relax, Forest &f) {
  f = Forest();
  f.nblocks = 1;
  f.block_off = {0, (int64_t)P.n};
  f.n = P.n;
  f.order.resize(f.n);
  f.sn_rowptr.push_back(0);
  f.asm_ptr.push_back(0);
  std::vector<int32_t> pos(f.n, -1);   // block index -> position in the current front
  int64_t panel = 0, front = 0, upd = 0;
  const int32_t b = 0;
  {
    const int32_t n = P.n;
    const int64_t off = 0;
    if (n == 0) return;
    LocalSym L;
    local_symbolic(P, L);
    for (int32_t k = 0; k < n; ++k) f.order[off + k] = L.post[k];
    for (int32_t k = 0; k < n; ++k) f.nnz_L += L.cc[k];
    // fundamental supernodes
    std::vector<int32_t> nchild(n, 0);
    for (int32_t k = 0; k < n; ++k) if (L.parent[k] >= 0) nchild[L.parent[k]]++;
    std::vector<int32_t> sfirst;            // supernode start columns (local)
    for (int32_t j = 0; j < n; ++j) {
      bool cont = j > 0 && L.parent[j - 1] == j && nchild[j] == 1 && L.cc[j - 1] == L.cc[j] + 1;
      if (!cont) sfirst.push_back(j);
    }
    int32_t ns = (int32_t)sfirst.size();
    std::vector<int32_t> sw(ns), sm(ns), spar(ns, -1), snode_of(n);
    std::vector<int64_t> snz(ns, 0);
    for (int32_t s = 0; s < ns; ++s) {
      int32_t e = s + 1 < ns ? sfirst[s + 1] : n;
      sw[s] = e - sfirst[s];
      sm[s] = (int32_t)L.cc[sfirst[s]];
      for (int32_t j = sfirst[s]; j < e; ++j) { snode_of[j] = s; snz[s] += L.cc[j]; }
    }
    for (int32_t s = 0; s < ns; ++s) {
      int32_t last = sfirst[s] + sw[s] - 1;
      spar[s] = L.parent[last] < 0 ? -1 : snode_of[L.parent[last]];
    }
    // relaxed amalgamation: merge J with the supernode just before it when that is a child
    std::vector<int32_t> alive(ns, 1), rep(ns);
    std::iota(rep.begin(), rep.end(), 0);
    std::vector<int32_t> mfirst(sfirst), mw(sw), mm(sm);
    std::vector<int64_t> mnz(snz);
    std::vector<int32_t> prev_alive(ns, -1);   // previous alive supernode in column order
    {
      int32_t pa = -1;
      for (int32_t s = 0; s < ns; ++s) { prev_alive[s] = pa; pa = s; }
    }
    auto find = [&](int32_t s) {
      while (rep[s] != s) { rep[s] = rep[rep[s]]; s = rep[s]; }
      return s;
    };
    for (int32_t J = 0; J < ns; ++J) {
      while (true) {
        int32_t C = prev_alive[J];
        if (C < 0) break;
        if (spar[C] < 0 || find(spar[C]) != J) break;
        if (!accept_merge(relax, mw[C], mw[J], mm[J], mnz[C] + mnz[J])) break;
        // merge C into J: J now starts at C's first column
        mfirst[J] = mfirst[C];
        mm[J] = mw[C] + mm[J];
        mw[J] = mw[C] + mw[J];
        mnz[J] += mnz[C];
        alive[C] = 0;
        rep[C] = J;
        prev_alive[J] = prev_alive[C];
      }
    }
    // final supernodes of this block (in column order), their parents
    std::vector<int32_t> fid(ns, -1);
    std::vector<int32_t> list;
    for (int32_t s = 0; s < ns; ++s) if (alive[s]) { fid[s] = (int32_t)list.size(); list.push_back(s); }
    const int32_t base = f.nsn;
    const int32_t nf = (int32_t)list.size();
    std::vector<int32_t> col_sn(n);
    for (int32_t t = 0; t < nf; ++t) {
      int32_t s = list[t];
      for (int32_t j = mfirst[s]; j < mfirst[s] + mw[s]; ++j) col_sn[j] = t;
    }
    for (int32_t t = 0; t < nf; ++t) {
      int32_t s = list[t];
      int32_t last = mfirst[s] + mw[s] - 1;
      int32_t par = L.parent[last] < 0 ? -1 : base + col_sn[L.parent[last]];
      f.sn_first.push_back((int32_t)(off + mfirst[s]));
      f.sn_w.push_back(mw[s]);
      f.sn_m.push_back(0);
      f.sn_parent.push_back(par);
      f.sn_block.push_back(b);
      f.sn_level.push_back(0);
    }
    f.nsn += nf;
    // children (local, for structures)
    std::vector<std::vector<int32_t>> kids(nf);
    for (int32_t t = 0; t < nf; ++t) {
      int32_t p = f.sn_parent[base + t];
      if (p >= 0) kids[p - base].push_back(base + t);
    }
    // structures, levels, relative maps, assembly lists (children precede parents)
    std::vector<int32_t> mark(n, -1);
    std::vector<int32_t> extra;
    for (int32_t t = 0; t < nf; ++t) {
      const int32_t J = base + t;
      const int32_t first = f.sn_first[J];
      const int32_t w = f.sn_w[J];
      const int32_t lfirst = first - (int32_t)off, llast = lfirst + w - 1;
      extra.clear();
      for (int32_t j = lfirst; j <= llast; ++j) {
        mark[j] = J;
        for (int64_t e = L.colptr[j]; e < L.colptr[j + 1]; ++e) {
          int32_t i = L.rowidx[e];
          if (i > llast && mark[i] != J) { mark[i] = J; extra.push_back(i); }
        }
      }
      int32_t lvl = 0;
      for (int32_t C : kids[t]) {
        lvl = std::max(lvl, f.sn_level[C] + 1);
        for (int64_t e = f.sn_rowptr[C] + f.sn_w[C]; e < f.sn_rowptr[C + 1]; ++e) {
          int32_t i = f.rows[e] - (int32_t)off;
          if (i > llast && mark[i] != J) { mark[i] = J; extra.push_back(i); }
          if (i < lfirst) throw std::runtime_error("child structure below parent columns");
        }
      }
      std::sort(extra.begin(), extra.end());
      f.sn_level[J] = lvl;
      const int32_t m = w + (int32_t)extra.size();
      f.sn_m[J] = m;
      const int64_t r0 = f.sn_rowptr[J];
      for (int32_t j = 0; j < w; ++j) f.rows.push_back(first + j);
      for (int32_t i : extra) f.rows.push_back((int32_t)(off + i));
      f.sn_rowptr.push_back(r0 + m);
      for (int32_t r = 0; r < m; ++r) pos[f.rows[r0 + r]] = r;
      f.sn_panel.push_back(panel);
      f.sn_front.push_back(front);
      f.sn_upd.push_back(upd);
      panel += (int64_t)panel_ld(m) * w;
      front += (int64_t)m * m;
      upd += m - w;
      for (int32_t r = w; r < m; ++r) f.relmap.push_back(-1);
      // children's update rows land at these positions of J's front
      for (int32_t C : kids[t])
        for (int64_t e = f.sn_rowptr[C] + f.sn_w[C]; e < f.sn_rowptr[C + 1]; ++e)
          f.relmap[f.sn_upd[C] + (e - f.sn_rowptr[C] - f.sn_w[C])] = pos[f.rows[e]];
      // A entries of J's columns
      for (int32_t j = lfirst; j <= llast; ++j)
        for (int64_t e = L.colptr[j]; e < L.colptr[j + 1]; ++e) {
          int32_t r = pos[off + L.rowidx[e]];
          f.asm_dst.push_back((int64_t)r + (int64_t)(j - lfirst) * m);
          f.asm_src.push_back(L.src[e]);
        }
      f.asm_ptr.push_back((int64_t)f.asm_dst.size());
      // partial Cholesky flops of the front (2 per multiply-add)
      for (int32_t c = 0; c < w; ++c) {
        double r = m - c - 1;
        f.flops_factor += r + r * (r + 1);
      }
    }
    }
  f.panel_size = panel;
  f.front_size = front;
  f.upd_rows = upd;
}

void parallel_for(int64_t count, const std::function<void(int64_t)> &body) {
  int nt = (int)std::thread::hardware_concurrency();
  if (const char *e = std::getenv("NSP_THREADS")) nt = std::atoi(e);
  nt = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::max(nt, 1), count, 64}));
  if (nt <= 1) {
    for (int64_t i = 0; i < count; ++i) body(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto work = [&] {
    for (int64_t i = next++; i < count; i = next++) {
      try {
        body(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err) err = std::current_exception();
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto &t : th) t.join();
  if (err) std::rethrow_exception(err);
}

void analyze_forest(const std::vector<BlockPattern> &blocks, int relax, Forest &f) {
  f = Forest();
  f.nblocks = (int32_t)blocks.size();
  f.block_off.assign(f.nblocks + 1, 0);
  for (int32_t b = 0; b < f.nblocks; ++b) f.block_off[b + 1] = f.block_off[b] + blocks[b].n;
  f.n = f.block_off[f.nblocks];
  f.order.resize(f.n);
  f.sn_rowptr.push_back(0);
  f.asm_ptr.push_back(0);
  // blocks are independent: analyze them in parallel, then concatenate in block order
  std::vector<Forest> part(f.nblocks);
  parallel_for(f.nblocks, [&](int64_t b) { analyze_block(blocks[b], relax, part[b]); });
  // offsets of every block's pieces in the concatenation, then a parallel copy with shifts
  const int32_t nb = f.nblocks;
  std::vector<int64_t> sn0(nb + 1, 0), row0(nb + 1, 0), asm0(nb + 1, 0), upd0(nb + 1, 0),
      pan0(nb + 1, 0), fr0(nb + 1, 0);
  for (int32_t b = 0; b < nb; ++b) {
    const Forest &q = part[b];
    sn0[b + 1] = sn0[b] + q.nsn;
    row0[b + 1] = row0[b] + (int64_t)q.rows.size();
    asm0[b + 1] = asm0[b] + (int64_t)q.asm_dst.size();
    upd0[b + 1] = upd0[b] + q.upd_rows;
    pan0[b + 1] = pan0[b] + q.panel_size;
    fr0[b + 1] = fr0[b] + q.front_size;
    f.nnz_L += q.nnz_L;
    f.flops_factor += q.flops_factor;
  }
  const int64_t nsn = sn0[nb];
  f.nsn = (int32_t)nsn;
  f.sn_first.resize(nsn);
  f.sn_w.resize(nsn);
  f.sn_m.resize(nsn);
  f.sn_parent.resize(nsn);
  f.sn_block.resize(nsn);
  f.sn_level.resize(nsn);
  f.sn_rowptr.resize(nsn + 1);
  f.sn_panel.resize(nsn);
  f.sn_front.resize(nsn);
  f.sn_upd.resize(nsn);
  f.asm_ptr.resize(nsn + 1);
  f.rows.resize(row0[nb]);
  f.relmap.resize(upd0[nb]);
  f.asm_dst.resize(asm0[nb]);
  f.asm_src.resize(asm0[nb]);
  parallel_for(nb, [&](int64_t b) {
    Forest &q = part[b];
    const int64_t off = f.block_off[b], base = sn0[b];
    for (int64_t k = 0; k < (int64_t)q.order.size(); ++k) f.order[off + k] = q.order[k];
    for (int32_t J = 0; J < q.nsn; ++J) {
      const int64_t g = base + J;
      f.sn_first[g] = (int32_t)(off + q.sn_first[J]);
      f.sn_w[g] = q.sn_w[J];
      f.sn_m[g] = q.sn_m[J];
      f.sn_parent[g] = q.sn_parent[J] < 0 ? -1 : (int32_t)(base + q.sn_parent[J]);
      f.sn_block[g] = (int32_t)b;
      f.sn_level[g] = q.sn_level[J];
      f.sn_rowptr[g + 1] = row0[b] + q.sn_rowptr[J + 1];
      f.sn_panel[g] = pan0[b] + q.sn_panel[J];
      f.sn_front[g] = fr0[b] + q.sn_front[J];
      f.sn_upd[g] = upd0[b] + q.sn_upd[J];
      f.asm_ptr[g + 1] = asm0[b] + q.asm_ptr[J + 1];
    }
    for (size_t r = 0; r < q.rows.size(); ++r) f.rows[row0[b] + r] = (int32_t)(off + q.rows[r]);
    std::copy(q.relmap.begin(), q.relmap.end(), f.relmap.begin() + upd0[b]);
    std::copy(q.asm_dst.begin(), q.asm_dst.end(), f.asm_dst.begin() + asm0[b]);
    std::copy(q.asm_src.begin(), q.asm_src.end(), f.asm_src.begin() + asm0[b]);
    q = Forest();
  });
  const int64_t panel = pan0[nb], front = fr0[nb], upd = upd0[nb];
  f.panel_size = panel;
  f.front_size = front;
  f.upd_rows = upd;
  // children CSR (forest)
  f.ch_ptr.assign(f.nsn + 1, 0);
  for (int32_t J = 0; J < f.nsn; ++J) if (f.sn_parent[J] >= 0) f.ch_ptr[f.sn_parent[J] + 1]++;
  for (int32_t J = 0; J < f.nsn; ++J) f.ch_ptr[J + 1] += f.ch_ptr[J];
  f.ch_list.resize(f.ch_ptr[f.nsn]);
  {
    std::vector<int32_t> p(f.ch_ptr.begin(), f.ch_ptr.end() - 1);
    for (int32_t J = 0; J < f.nsn; ++J) if (f.sn_parent[J] >= 0) f.ch_list[p[f.sn_parent[J]]++] = J;
  }
  // gather lists: for each front position, the children's update rows that land there
  const int64_t npos = f.sn_rowptr[f.nsn];
  f.gptr.assign(npos + 1, 0);
  for (int32_t C = 0; C < f.nsn; ++C) {
    int32_t P = f.sn_parent[C];
    if (P < 0) continue;
    for (int64_t u = f.sn_upd[C]; u < f.sn_upd[C] + f.sn_m[C] - f.sn_w[C]; ++u)
      f.gptr[f.sn_rowptr[P] + f.relmap[u] + 1]++;
  }
  for (int64_t q = 0; q < npos; ++q) f.gptr[q + 1] += f.gptr[q];
  f.gsrc.resize(f.gptr[npos]);
  {
    std::vector<int64_t> p(f.gptr.begin(), f.gptr.end() - 1);
    for (int32_t C = 0; C < f.nsn; ++C) {
      int32_t P = f.sn_parent[C];
      if (P < 0) continue;
      for (int64_t u = f.sn_upd[C]; u < f.sn_upd[C] + f.sn_m[C] - f.sn_w[C]; ++u)
        f.gsrc[p[f.sn_rowptr[P] + f.relmap[u]]++] = u;
    }
  }
  // level schedule
  f.nlevels = 0;
  for (int32_t J = 0; J < f.nsn; ++J) f.nlevels = std::max(f.nlevels, f.sn_level[J] + 1);
  f.level_ptr.assign(f.nlevels + 1, 0);
  for (int32_t J = 0; J < f.nsn; ++J) f.level_ptr[f.sn_level[J] + 1]++;
  for (int32_t l = 0; l < f.nlevels; ++l) f.level_ptr[l + 1] += f.level_ptr[l];
  f.level_sn.resize(f.nsn);
  {
    std::vector<int32_t> p(f.level_ptr.begin(), f.level_ptr.end() - 1);
    for (int32_t J = 0; J < f.nsn; ++J) f.level_sn[p[f.sn_level[J]]++] = J;
  }
}

}  // namespace nsp
