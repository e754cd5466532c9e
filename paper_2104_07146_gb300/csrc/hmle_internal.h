// Internal types of libhmle: device descriptors shared by the planner
// (host C++) and the kernels, and the handle structs behind the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hmle.h"

namespace hmle {

constexpr int kMaxLevels = 24;      // depth limit (n / leaf <= 2^23)
constexpr int kMaxLeaf = 128;       // leaf_size upper bound
constexpr int kMaxRank = 64;        // max_rank upper bound
constexpr int kMaxSample = 64;      // max_rank + oversample upper bound

// Block kinds.
constexpr int32_t kDense = 0;       // leaf x leaf, kept dense (incl. diagonal)
constexpr int32_t kLowRank = 1;     // admissible, U W^T

// One block of the lower triangle of the block tree.  Point ranges are in
// cluster order.  Dense blocks are stored column-major with ld = leaf_size.
struct BlockDesc {
  int32_t kind;
  int32_t level;
  int32_t rbeg, rend;      // rows (points)
  int32_t cbeg, cend;      // columns (points)
  int32_t rleaf, cleaf;    // first leaf of the row / column cluster
  int64_t off_d;           // dense: L / C storage (b x b, ld = b)
  int64_t off_uc, off_vc;  // low-rank: ACA factors of C (m x kc, p x kc)
  int64_t off_u;           // low-rank: U of L (m x kcap, ld = m)
  int32_t panel;           // low-rank: W-panel holding W of L; dense: -1
  int32_t slot;            // low-rank: first column of this block in the panel
};

// A W-panel: all low-rank blocks (rho, sigma) of one column cluster sigma
// keep their right factor W (|sigma| x kcap) side by side in one
// |sigma| x width column-major matrix (ld = |sigma|).  The last panel is the
// right-hand side Z (root cluster, width nrhs).
struct PanelDesc {
  int32_t rbeg, rend;
  int32_t width;
  int32_t leaf0;           // first leaf of the cluster
  int64_t off;
};

// --- per-step task records (all indices into the step's own arrays) -----

// Gram of two low-rank factors over their overlapping columns:
// G = W_A[ov]^T W_B[ov] (kcap x kcap), written at goff.
struct GramTask {
  int32_t a, b;            // block ids
  int32_t ovb, ove;        // overlapping point range
  int64_t goff;            // offset in the gram workspace
};

// A row chunk of a gram: rows [r0, r1) of the overlap, written to out
// (the gram itself when it has one chunk, else a partial sum).
struct GramChunk {
  int32_t g;               // index of the GramTask
  int32_t r0, r1;
  int64_t out;
};

// Sum of a gram's partial chunks (fixed order) into the gram.
struct GramReduce {
  int32_t g;
  int32_t nchunk;
  int64_t poff;
};

// Pair (A, B) contributing -U_A G_AB U_B^T to a low-rank target; a and b
// are indices of the A- and B-entries (SideEntry) of that target.
struct LrPair {
  int32_t ae, be;
  int64_t goff;            // LR x LR: gram offset; otherwise -1
};

// Pair (A, B) contributing -U_A G_AB U_B^T to a dense target; a and b are
// block ids (A covers the target's rows, B its columns).
struct DPair {
  int32_t a, b;
  int64_t goff;            // LR x LR: gram offset; otherwise -1
};

// Low-rank target compressed at this step (S = C_T - sum pairs).
struct LrTarget {
  int32_t blk;             // target block id
  int32_t m, p;            // rows, cols
  int32_t a0, a1;          // its A-entries [a0, a1) in the step's A list
  int32_t b0, b1;          // its B-entries
  int64_t yoff;            // Y / Q workspace (m x r, ld m)
  int64_t zoff;            // Z workspace (p x r, ld p)
  int64_t soff;            // small r x r workspace (4 r x r)
  int64_t tcoff;           // t_C workspace (kc x r)
  int32_t gm, gp;          // row groups of the tall QR of Y (m rows) and Z (p rows)
  int64_t roff;            // partial R factors (max(gm, gp) x r x r)
};

// An A- (or B-) entry of a target: a block covering some rows of the
// target's row (column) cluster, with its own small workspaces.
struct SideEntry {
  int32_t target;          // index into the step's LrTarget list
  int32_t blk;             // block id
  int64_t toff;            // t workspace (k x r): U^T x restricted
  int64_t soff;            // s workspace (k x r): sum of G t
  int32_t p0, p1;          // pairs of this entry in the step's pair-index list
};

// Rows of a target's Y (or Z) written by one CTA: one leaf of the target's
// row (column) cluster and the side entries covering it.
struct RowTask {
  int32_t target;
  int32_t leaf;
  int32_t e0, e1;          // entries in the step's row-entry index list
};

// Dense target (I, K) at step K (incl. the diagonal).
struct DenseTarget {
  int32_t blk;
  int32_t p0, p1;          // pairs in the step's dense pair list
};

// Deferred update of a W-panel by a block A whose columns end at this step.
struct HTask {
  int32_t a;               // block id (low-rank)
  int32_t panel;
  int64_t hoff;            // H = W_A^T W_panel[cols A]  (kcap x width)
};

struct UpdRow {
  int32_t panel;
  int32_t leaf;
  int32_t e0, e1;          // update entries (UpdEntry) for this panel row
};

struct UpdEntry {
  int32_t a;               // block id
  int64_t hoff;            // low-rank: H offset; dense: -1
};

// Ranges of one step's tasks in the flat arrays.
struct StepRange {
  int32_t gram0, gram1;
  int32_t gch0, gch1;      // gram row chunks
  int32_t gred0, gred1;    // grams needing a reduction of their chunks
  int32_t lrt0, lrt1;
  int32_t aent0, aent1;
  int32_t bent0, bent1;
  int32_t arow0, arow1;    // Y row tasks
  int32_t brow0, brow1;    // Z row tasks
  int32_t dns0, dns1;      // dense targets (diagonal first)
  int32_t wpan0, wpan1;    // panels solved at this step
  int32_t ht0, ht1;
  int32_t ur0, ur1;
  int64_t dpws;            // workspace of the dense pairs' partial products (b x b each)
  int64_t ws_words;        // workspace doubles needed by this step
};

// The θ-independent plan of one tree.
struct Plan {
  int32_t n, d, b, depth, nleaf, kcap, kc, r;
  std::vector<int32_t> cl_beg, cl_end;          // heap-indexed clusters
  std::vector<BlockDesc> blocks;
  std::vector<int32_t> diag_of_leaf;            // block id of (K, K)
  std::vector<PanelDesc> panels;
  int32_t rhs_panel;
  int64_t dense_words, uc_words, u_words, w_words;
  // flat task arrays
  std::vector<GramTask> grams;
  std::vector<GramChunk> gchunks;
  std::vector<GramReduce> greds;
  std::vector<LrTarget> lrt;
  std::vector<SideEntry> aent, bent;
  std::vector<int32_t> apair, bpair;            // pair indices per entry
  std::vector<LrPair> lrpairs;                  // pairs of LR targets
  std::vector<RowTask> arow, brow;
  std::vector<int32_t> arow_ent, brow_ent;
  std::vector<DenseTarget> dns;
  std::vector<DPair> dpairs;
  std::vector<int32_t> wpan;
  std::vector<HTask> hts;
  std::vector<UpdRow> urows;
  std::vector<UpdEntry> uents;
  std::vector<StepRange> steps;
  // forward solve of a new right-hand side through a finished factor: per
  // step, the deferred updates restricted to the right-hand-side panel
  std::vector<HTask> hts_rhs;
  std::vector<UpdRow> urows_rhs;
  std::vector<UpdEntry> uents_rhs;
  std::vector<int32_t> ht_rhs0, ur_rhs0;   // per step ranges (nleaf + 1 entries)
  // backward solve v = L^{-T} w (reverse sweep).  At step K (leaves in
  // reverse order), after v_K is solved, every block A whose row cluster
  // starts at K pushes v[cols A] -= A^T v[rows A]: low-rank blocks through
  // h_A = U_A^T v[rows A] (bh_blocks), then per column leaf J the entries
  // touching it (bupd rows: UpdRow with panel unused, entries UpdEntry with
  // hoff = index into the h workspace, or -1 for a dense block).
  std::vector<int32_t> bh_blocks, bh0;      // per step: LR blocks whose rows start at K
  std::vector<UpdRow> bupd;
  std::vector<UpdEntry> bents;
  std::vector<int32_t> bupd0;               // per step ranges of bupd
  // triangular H-matvec y = L x (simulation): per leaf row, the blocks of L
  // covering it (diagonal first)
  std::vector<int32_t> mv_row0, mv_blocks;
  // per leaf I: off-diagonal blocks whose columns cover I (symmetric C x)
  std::vector<int32_t> mvt_row0, mvt_blocks;
  int64_t ws_max;
  int64_t n_lr_blocks, n_dense_blocks;
};

// Depth of the cluster tree of n points with leaves of at most leaf_size
// points (every level halves the clusters), and the clusters' point ranges
// in heap order (cluster h splits at b + (e - b) / 2 into 2h + 1, 2h + 2).
int32_t tree_depth(int64_t n, int32_t leaf_size);
void cluster_ranges(int64_t n, int32_t depth, std::vector<int32_t> &cl_beg,
                    std::vector<int32_t> &cl_end);

// Build the plan from the cluster ranges and the block list (host).
// Returns an empty string on success, else an error message.
std::string build_plan(Plan &P, int32_t n, int32_t d, int32_t b, int32_t depth,
                       const std::vector<int32_t> &cl_beg,
                       const std::vector<int32_t> &cl_end,
                       const std::vector<int4> &blocks_lij,  // (level, i, j, kind)
                       int32_t kcap, int32_t kc, int32_t r, int32_t nrhs);

}  // namespace hmle
