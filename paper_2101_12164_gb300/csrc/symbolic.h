// Host-side symbolic analysis of the sparse Cholesky factors of A_1..A_N (the diagonal
// blocks of A_I) and of A_G, which Algorithm 2 needs for A_I^{-1} and A_G^{-1}
// ("factorized cheaply in parallel using a direct algorithm", §2.3).
//
// A "forest" is a set of independent SPD blocks whose unknowns are numbered
// consecutively (block b owns [off_b, off_b + n_b)). Each block is ordered (caller order or
// nested dissection), its elimination tree is postordered, and columns are grouped into
// relaxed supernodes. Supernode J owns columns [first, first + w) and a sorted row
// structure of m >= w rows whose first w entries are its own columns.
#pragma once
#include <cstdint>
#include <functional>
#include <vector>

namespace nsp {

// Leading dimension of a supernode panel with m rows: rounded up to 4 elements so that every
// panel column starts on a 16-byte boundary (vector loads in the solve sweeps).
inline int32_t panel_ld(int32_t m) { return (m + 3) & ~3; }

// Lower triangle (diagonal included) of one block by columns, in the block's initial order.
struct BlockPattern {
  int32_t n = 0;
  std::vector<int64_t> colptr;   // n + 1
  std::vector<int32_t> rowidx;   // row >= column
  std::vector<int64_t> src;      // index of the value in the caller's CSR value array
};

struct Forest {
  int64_t n = 0;                         // total unknowns of the forest
  int32_t nblocks = 0;
  std::vector<int64_t> block_off;        // nblocks + 1
  std::vector<int64_t> order;            // internal index -> index in the block's initial order

  int32_t nsn = 0;
  std::vector<int32_t> sn_first, sn_w, sn_m, sn_parent, sn_block, sn_level;
  std::vector<int64_t> sn_rowptr;        // nsn + 1, into rows
  std::vector<int32_t> rows;             // internal indices (forest numbering)
  std::vector<int64_t> sn_panel;         // offset of the panel_ld(m) x w panel (column-major)
  std::vector<int64_t> sn_front;         // offset of the m x m front (column-major)
  std::vector<int64_t> sn_upd;           // first update row (the m - w rows below the panel)
  std::vector<int32_t> relmap;           // update row -> position in the parent's front
  std::vector<int32_t> ch_ptr, ch_list;  // children of each supernode
  std::vector<int64_t> gptr;             // per front position (sn_rowptr numbering) + 1
  std::vector<int64_t> gsrc;             // update rows of children landing on that position
  std::vector<int64_t> asm_ptr;          // per supernode, A entries to scatter into its front
  std::vector<int64_t> asm_dst;          // front offset (r + c*m) relative to sn_front
  std::vector<int64_t> asm_src;          // caller CSR value index
  int32_t nlevels = 0;
  std::vector<int32_t> level_ptr, level_sn;   // supernodes grouped by height (leaves = 0)

  int64_t nnz_L = 0;                     // structural nonzeros (true column counts)
  int64_t panel_size = 0, front_size = 0, upd_rows = 0;
  double flops_factor = 0;               // multiply-add pairs x 2 of the partial Cholesky
};

struct Graph {                            // symmetric adjacency, no self loops
  int32_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
};

// body(i) for i in [0, count) on up to hardware_concurrency() host threads (NSP_THREADS
// overrides; 1 runs serially); the first exception of a body is rethrown after all end.
void parallel_for(int64_t count, const std::function<void(int64_t)> &body);

// Nested-dissection order (new -> old) of a graph by level-structure bisection.
std::vector<int32_t> nested_dissection(const Graph &g, int32_t leaf);

// Full symbolic analysis of a forest of blocks (each pattern in its initial order).
// relax: amalgamation aggressiveness (0 = fundamental supernodes only).
void analyze_forest(const std::vector<BlockPattern> &blocks, int relax, Forest &f);

}  // namespace nsp
