// Host-side symbolic analysis: block elimination tree, fill, tile task graph (B-DAG) and the
// level sets of the solve sweeps.  Pure C++ (no CUDA), shared by d3m_analyze and d3m_create.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "d3m.h"

namespace d3m {

// Task flags.
enum : int32_t {
  TF_DIAG = 1,        // I == J
  TF_SAME_BLOCK = 2,  // p == q: padding unknowns get a unit diagonal
  TF_UPDATE = 4,      // partial-update task (else: the tile's final task)
  TF_S_IN = 8,        // start from the tile's accumulator S (else from K_IJ)
  TF_PRIO = 16,       // on or near the critical path: served from the priority lane
  TF_PAIR = 32,       // update task over two tiles (I, J) and (I, J + 1) that share the L_IK operand
};

// One task of the factorization DAG.  The paper's task model (Sec. II: one task per nonzero
// block of the dual matrix, covering its update, triangular solve and factorization) at tile
// granularity: the updates of lower tile (I, J), S_IJ = K_IJ - sum_K L_IK D_K L_JK^T, are cut
// into segments, one per source block column; every segment but the last is an UPDATE task
// (S <- S_in - sum over the segment, kept in the tile's accumulator; segments chained in
// increasing K), and the FINAL task (task id == tile id) applies the last segment and then
// factors the diagonal tile (I == J) or applies the triangular solve (I != J).
struct TileTask {
  int32_t tile;        // tile id (== id of the tile's final task)
  int32_t diag;        // tile id of (J, J)
  int32_t col;         // global tile column J
  int32_t nk;          // tile updates of this task's segment
  int64_t kl_off;      // offset of the segment in the klist array
  int64_t k_off;       // element (c128) offset of the stored K block, -1 for a fill block
  int32_t k_ld;        // leading dimension of the stored K block
  int32_t k_tr;        // 1: entry (r, c) of block (p, q) is stored(c, r) (use the transpose)
  int32_t r0, c0;      // first row / column of the tile inside block (p, q)
  int32_t rv, cv;      // valid rows / columns (the rest is padding up to the tile edge)
  int32_t flags;       // TF_* bits
  int32_t sidx;        // accumulator slot of the tile, -1 if it has a single segment
  // TF_PAIR: the second tile (I, J + 1), its first column inside block (p, q), valid columns and
  // accumulator slot; its K-list entries are those of the first tile with b2_tile = (J + 1, K)
  int32_t tile2, c0_2, cv2, sidx2;
  int32_t kseq;        // position of the stored K block in the upload order (-1: fill block)
  int32_t pad_;
};
static_assert(sizeof(TileTask) == 88, "TileTask layout");

// One K-list entry: S_IJ -= L_IK D_K L_JK^T uses tiles a = (I, K), b = (J, K), column K; in a
// paired segment b2 = (J + 1, K) for the second tile (else -1).
struct KEntry {
  int32_t a_tile, b_tile, kcol, b2_tile;
};

// One solve gather item: partial = L(tile) * y(src tile) (forward) or L(tile)^T * w(src)
// (backward), written to partial slot `slot` of destination tile row/column `dst`.
struct SolveItem {
  int32_t tile, src, dst, slot;
};

// Consecutive items of one destination whose products one gather block sums into one partial.
struct SolveGroup {
  int32_t first, count, slot, dst;   // items [first, first + count) (global index), partial slot
};

struct Symbolic {
  // block level (NEW numbering)
  int N = 0;
  int b = 64;                                // tile edge
  std::vector<int32_t> perm, inv;            // perm[new] = old
  std::vector<int32_t> m, ntile, tstart;     // block size, tiles per block, first tile
  std::vector<int64_t> xoff;                 // first unknown of block (padded, new order)
  std::vector<int64_t> xoff_orig;            // first unknown of ORIGINAL block f
  std::vector<std::vector<int32_t>> str;     // struct(k): rows i > k with L_ik != 0
  std::vector<std::vector<int32_t>> rowlist; // blocks k < q with q in struct(k)
  std::vector<int32_t> parent, level;
  int depth = 0, max_height = 0, nlevels = 0;
  int64_t n = 0, npad = 0;                   // unknowns (unpadded / padded)
  int64_t nnzb_K = 0, nL_off = 0, n_upd_off = 0;
  int64_t n_tile_updates = 0, n_edges = 0;
  double factor_flops = 0, solve_flops_rhs = 0, residual_flops_rhs = 0;

  // K layout (caller numbering, lower block-CSC)
  std::vector<int64_t> colptr;
  std::vector<int32_t> rowidx;
  std::vector<int64_t> kblk_off;             // [nnzb+1] element offsets
  // upload order of the stored blocks (a host K is copied in this order while the factorization
  // runs): blocks sorted by the elimination position of their lower column, merged into runs
  // that are contiguous in storage; run r covers blocks up to sequence number kc_seq_end[r] - 1
  std::vector<int32_t> kseq;                 // [nnzb] sequence number of each stored block
  std::vector<int64_t> kc_off, kc_len;       // runs: element offset and length
  std::vector<int32_t> kc_seq_end;
  std::vector<int32_t> m_orig;               // block sizes, caller numbering

  // tile level
  int NT = 0;                                // tile columns
  std::vector<int64_t> tcolptr;              // [NT+1]
  std::vector<int32_t> trow;                 // tile row of each tile
  std::vector<int32_t> tblk;                 // block of each tile row/column index
  std::vector<TileTask> tasks;             // [ntiles final tasks, then update tasks]
  int64_t ntiles = 0;
  int64_t n_acc = 0;                         // tiles with an accumulator slot
  std::vector<KEntry> klist;
  std::vector<int32_t> ndeps;
  std::vector<int64_t> succ_ptr;
  std::vector<int32_t> succ;
  std::vector<int32_t> init_ready;           // tasks ready at launch, normal lane
  std::vector<int32_t> init_ready_hi;        // tasks ready at launch, priority lane
  int64_t n_prio = 0;                        // tasks flagged TF_PRIO
  std::vector<int32_t> diag_tile;            // tile column J -> tile id of (J, J)

  // solve level sets (forward uses levels ascending, backward descending)
  std::vector<std::vector<int32_t>> lev_blocks;      // blocks of each level
  std::vector<int64_t> fwd_item_ptr, bwd_item_ptr;   // per level, into fwd_items / bwd_items
  std::vector<SolveItem> fwd_items, bwd_items;
  std::vector<int64_t> fwd_slot_ptr, bwd_slot_ptr;   // [NT] first slot | count << 32
  int64_t max_level_items = 0;
  std::vector<int64_t> fwd_group_ptr, bwd_group_ptr;  // per level, into fwd_groups / bwd_groups
  std::vector<SolveGroup> fwd_groups, bwd_groups;
  int64_t max_level_groups = 0;
  int32_t max_group = 1;                     // most items in one group

  // residual (caller numbering): per output block f, the stored blocks contributing to r_f
  std::vector<int64_t> res_ptr;              // [N+1]
  std::vector<int32_t> res_blk;              // stored block index e
  std::vector<int32_t> res_src;              // source block g (x_g)
  std::vector<int32_t> res_tr;               // 1: use stored block transposed

  int64_t tile_of(int I, int J) const;       // -1 if (I, J) not in the tile pattern
};

// Validate the pattern and permutation, then run the full analysis for tile edge b.  Tasks whose
// estimated slack is within prio_slack of the critical path are flagged TF_PRIO.
// Returns D3M_OK or an error code with a message in `err`.
// task_cost (6 values or nullptr): the duration model of the priority estimate, cost = base +
// per_k * nk (nk = tile products of the task) for update tasks (task_cost[0], [1]), diagonal
// final tasks ([2], [3]) and off-diagonal final tasks ([4], [5]), in any common unit; nullptr or
// all zeros = the built-in model.
// pair_updates: the source-block update segments of tiles (I, J) and (I, J + 1) (J at an even
// tile offset in its block) become one TF_PAIR task that reads each L_IK tile once for both.
int analyze(const d3m_pattern* pat, const int32_t* perm, int b, bool build_tasks,
            Symbolic& s, std::string& err, double prio_slack = 0.08, int seg_group = 1,
            const double* task_cost = nullptr, int gather_group = 1, bool pair_updates = false);

// Grid nested dissection (see d3m_order_grid_nd).
int order_grid_nd(int nx, int ny, int nz, std::vector<int32_t>& perm);

}  // namespace d3m
