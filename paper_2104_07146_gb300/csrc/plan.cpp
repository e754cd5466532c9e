// Host planner: the θ-independent schedule of the left-looking leaf sweep.
//
// The H-Cholesky factor L~ of C~ (Sec. 2) has the block structure of C~:
// dense leaf blocks near the diagonal, and admissible blocks (rho, sigma)
// held as U W^T.  With S_{rho,sigma} = C_{rho,sigma} - L_{rho,<s} L_{sigma,<s}^T
// (s = first column of sigma) the factor block is
//     L_{rho,sigma} = S_{rho,sigma} L_{sigma,sigma}^{-T},
// so the sweep over leaves K = 0..N-1 does, at step K:
//   1. compress S of every low-rank block whose column cluster starts at K
//      (all its updates come from columns < s, finished earlier) into
//      U W0^T and start W = W0;
//   2. form the dense blocks of column K (S = C - updates), POTRF the
//      diagonal leaf, TRSM the others;
//   3. forward-solve the rows of leaf K of every open W-panel
//      (W <- L_{sigma,sigma}^{-1} W0 advances one leaf; the right-hand side
//      Z is the panel of the root cluster, which gives w = L^{-1} Z);
//   4. push the contribution of every block whose columns end at K into the
//      rows below it of every open W-panel containing it.
// Every update L_{X,<s} L_{Y,<s}^T is a sum over pairs of blocks (A, B)
// covering rows X and Y and overlapping columns: U_A G_AB U_B^T with
// G_AB = W_A[ov]^T W_B[ov] (a dense leaf block acts as U = D, W = I).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <tuple>
#include <unordered_map>

#include "hmle_internal.h"

namespace hmle {

namespace {

inline int cid(int l, int i) { return (1 << l) - 1 + i; }

struct Builder {
  Plan &P;
  std::vector<std::vector<int32_t>> rowlist;  // blocks whose rows contain leaf I
  std::vector<int32_t> stampA, stampB;
  int32_t stamp = 0;
  explicit Builder(Plan &p) : P(p) {}

  int span(const BlockDesc &B) const { return 1 << (P.depth - B.level); }
  bool overlap(const BlockDesc &A, const BlockDesc &B) const {
    return std::max(A.cbeg, B.cbeg) < std::min(A.cend, B.cend);
  }
  int64_t kof(const BlockDesc &B) const { return B.kind == kLowRank ? P.kcap : P.b; }

  // blocks covering leaves [l0, l1) with columns ending at or before s
  void collect(int l0, int l1, int32_t s, std::vector<int32_t> &out,
               std::vector<int32_t> &stampv) {
    ++stamp;
    out.clear();
    for (int I = l0; I < l1; ++I)
      for (int32_t x : rowlist[I]) {
        const BlockDesc &X = P.blocks[x];
        if (X.cend <= s && stampv[x] != stamp) {
          stampv[x] = stamp;
          out.push_back(x);
        }
      }
    std::sort(out.begin(), out.end());
  }

  // Column overlaps through the cluster tree.  Block column ranges are
  // clusters, which are nested or disjoint, so the blocks of a list whose
  // columns overlap A's are those whose column cluster is A's, one of its
  // ancestors, or a cluster inside A's.  index_columns() indexes a list;
  // overlapping() returns the positions of the overlapping blocks in
  // ascending order (the order a scan of the whole list would give).
  int colcid(const BlockDesc &B) const {
    return (1 << B.level) - 1 + (B.cleaf >> (P.depth - B.level));
  }
  std::unordered_map<int32_t, std::vector<int32_t>> bycol;   // column cluster -> positions
  std::vector<std::pair<int32_t, int32_t>> byleaf;            // (first column leaf, position)
  const std::vector<int32_t> *ilist = nullptr;
  void index_columns(const std::vector<int32_t> &list) {
    ilist = &list;
    bycol.clear();
    byleaf.clear();
    for (size_t i = 0; i < list.size(); ++i) {
      const BlockDesc &B = P.blocks[list[i]];
      bycol[colcid(B)].push_back((int32_t)i);
      byleaf.emplace_back(B.cleaf, (int32_t)i);
    }
    std::sort(byleaf.begin(), byleaf.end());
  }
  void overlapping(const BlockDesc &A, std::vector<int32_t> &out) const {
    out.clear();
    for (int h = colcid(A);; h = (h - 1) / 2) {
      auto it = bycol.find(h);
      if (it != bycol.end()) out.insert(out.end(), it->second.begin(), it->second.end());
      if (h == 0) break;
    }
    const int32_t l1 = A.cleaf + span(A);
    auto it = std::lower_bound(byleaf.begin(), byleaf.end(),
                               std::make_pair(A.cleaf, std::numeric_limits<int32_t>::min()));
    for (; it != byleaf.end() && it->first < l1; ++it)
      if (P.blocks[(*ilist)[it->second]].level > A.level) out.push_back(it->second);
    std::sort(out.begin(), out.end());
  }
};

}  // namespace

int32_t tree_depth(int64_t n, int32_t leaf_size) {
  int32_t depth = 0;
  while (((n + (1LL << depth) - 1) >> depth) > leaf_size) ++depth;
  return depth;
}

void cluster_ranges(int64_t n, int32_t depth, std::vector<int32_t> &cb, std::vector<int32_t> &ce) {
  const int ncl = (2 << depth) - 1;
  cb.assign(ncl, 0);
  ce.assign(ncl, 0);
  cb[0] = 0;
  ce[0] = (int32_t)n;
  for (int h = 0; h < (1 << depth) - 1; ++h) {
    const int32_t b = cb[h], e = ce[h], mid = b + (e - b) / 2;
    cb[2 * h + 1] = b; ce[2 * h + 1] = mid;
    cb[2 * h + 2] = mid; ce[2 * h + 2] = e;
  }
}

std::string build_plan(Plan &P, int32_t n, int32_t d, int32_t b, int32_t depth,
                       const std::vector<int32_t> &cl_beg,
                       const std::vector<int32_t> &cl_end,
                       const std::vector<int4> &blk, int32_t kcap, int32_t kc,
                       int32_t r, int32_t nrhs) {
  P.n = n; P.d = d; P.b = b; P.depth = depth; P.nleaf = 1 << depth;
  P.kcap = kcap; P.kc = kc; P.r = r;
  P.cl_beg = cl_beg; P.cl_end = cl_end;
  const int N = P.nleaf;
  // The overlap searches below go through the cluster tree (nested or
  // disjoint column clusters) instead of comparing point ranges.  The two
  // agree only while no cluster is empty: an empty cluster nested inside
  // another overlaps nothing by point range, yet the tree search would report
  // it.  The halving rule with leaf_size >= 16 never empties a cluster, and a
  // caller's partition that would is refused here.
  if ((int)cl_beg.size() < (2 << depth) - 1 || (int)cl_end.size() < (2 << depth) - 1)
    return "cluster arrays shorter than the tree";
  for (int h = 0; h < (2 << depth) - 1; ++h)
    if (!(cl_beg[h] < cl_end[h])) return "empty cluster";

  // --- blocks, in a fixed order: by column leaf, then dense before
  // low-rank, then row leaf (the device block tree is already deterministic;
  // this order only fixes storage offsets).
  std::vector<int4> order(blk);
  auto key = [&](const int4 &q) {
    int sh = depth - q.x;
    return std::make_tuple(q.z << sh, q.w, q.y << sh, q.x);
  };
  std::sort(order.begin(), order.end(),
            [&](const int4 &a, const int4 &c) { return key(a) < key(c); });
  P.blocks.clear();
  P.diag_of_leaf.assign(N, -1);
  int64_t dw = 0, ucw = 0, uw = 0;
  P.n_lr_blocks = P.n_dense_blocks = 0;
  for (const int4 &q : order) {
    BlockDesc B{};
    B.level = q.x;
    B.kind = q.w;
    int hr = cid(q.x, q.y), hc = cid(q.x, q.z);
    B.rbeg = cl_beg[hr]; B.rend = cl_end[hr];
    B.cbeg = cl_beg[hc]; B.cend = cl_end[hc];
    B.rleaf = q.y << (depth - q.x);
    B.cleaf = q.z << (depth - q.x);
    B.panel = -1; B.slot = 0;
    B.off_d = B.off_uc = B.off_vc = B.off_u = -1;
    if (B.kind == kDense) {
      if (q.x != depth) return "dense block above the leaf level";
      if (q.y < q.z) return "dense block above the diagonal";
      B.off_d = dw; dw += (int64_t)b * b;
      if (q.y == q.z) P.diag_of_leaf[q.y] = (int32_t)P.blocks.size();
      ++P.n_dense_blocks;
    } else {
      if (q.y <= q.z) return "admissible block on or above the diagonal";
      int64_t m = B.rend - B.rbeg, p = B.cend - B.cbeg;
      B.off_uc = ucw; ucw += m * kc;
      B.off_vc = ucw; ucw += p * kc;
      B.off_u = uw; uw += m * kcap;
      ++P.n_lr_blocks;
    }
    P.blocks.push_back(B);
  }
  for (int K = 0; K < N; ++K)
    if (P.diag_of_leaf[K] < 0) return "missing diagonal block";
  P.dense_words = dw; P.uc_words = ucw; P.u_words = uw;

  // --- W-panels: one per column cluster holding low-rank blocks
  std::vector<int32_t> panel_of(2 * N, -1);
  P.panels.clear();
  int64_t ww = 0;
  for (size_t x = 0; x < P.blocks.size(); ++x) {
    BlockDesc &B = P.blocks[x];
    if (B.kind != kLowRank) continue;
    int hc = cid(B.level, B.cleaf >> (depth - B.level));
    if (panel_of[hc] < 0) {
      PanelDesc pd{};
      pd.rbeg = B.cbeg; pd.rend = B.cend; pd.width = 0;
      pd.leaf0 = B.cleaf; pd.off = 0;
      panel_of[hc] = (int32_t)P.panels.size();
      P.panels.push_back(pd);
    }
    PanelDesc &pd = P.panels[panel_of[hc]];
    B.panel = panel_of[hc];
    B.slot = pd.width;
    pd.width += kcap;
  }
  // right-hand side panel: the root cluster
  {
    PanelDesc pd{};
    pd.rbeg = 0; pd.rend = n; pd.width = std::max(nrhs, 1); pd.leaf0 = 0;
    P.rhs_panel = (int32_t)P.panels.size();
    panel_of[0] = panel_of[0] < 0 ? P.rhs_panel : panel_of[0];
    P.panels.push_back(pd);
  }
  for (PanelDesc &pd : P.panels) {
    pd.off = ww;
    ww += (int64_t)(pd.rend - pd.rbeg) * pd.width;
  }
  P.w_words = ww;
  // the panels of cluster h and of its ancestors, in panel order (cluster
  // ranges are nested or disjoint, so these are exactly the panels whose
  // range contains cluster h's); the root's panel is the right-hand side
  std::vector<int32_t> pans, cand;
  auto panels_above = [&](int h, std::vector<int32_t> &out) {
    out.clear();
    for (;; h = (h - 1) / 2) {
      if (panel_of[h] >= 0) out.push_back(panel_of[h]);
      if (h == 0) break;
    }
    std::sort(out.begin(), out.end());
  };

  Builder Bd(P);
  Bd.rowlist.assign(N, {});
  for (size_t x = 0; x < P.blocks.size(); ++x) {
    const BlockDesc &B = P.blocks[x];
    if (B.kind == kDense && B.rleaf == B.cleaf) continue;  // diagonal
    for (int I = B.rleaf; I < B.rleaf + Bd.span(B); ++I) Bd.rowlist[I].push_back((int32_t)x);
  }
  Bd.stampA.assign(P.blocks.size(), 0);
  Bd.stampB.assign(P.blocks.size(), 0);

  // rows of L for the triangular matvec: diagonal block, then the rest
  P.mv_row0.assign(N + 1, 0);
  P.mv_blocks.clear();
  for (int I = 0; I < N; ++I) {
    P.mv_row0[I] = (int32_t)P.mv_blocks.size();
    P.mv_blocks.push_back(P.diag_of_leaf[I]);
    P.mv_blocks.insert(P.mv_blocks.end(), Bd.rowlist[I].begin(), Bd.rowlist[I].end());
  }
  P.mv_row0[N] = (int32_t)P.mv_blocks.size();
  {
    std::vector<std::vector<int32_t>> collist(N);
    for (size_t x = 0; x < P.blocks.size(); ++x) {
      const BlockDesc &B = P.blocks[x];
      if (B.kind == kDense && B.rleaf == B.cleaf) continue;
      for (int J = B.cleaf; J < B.cleaf + Bd.span(B); ++J) collist[J].push_back((int32_t)x);
    }
    P.mvt_row0.assign(N + 1, 0);
    P.mvt_blocks.clear();
    for (int I = 0; I < N; ++I) {
      P.mvt_row0[I] = (int32_t)P.mvt_blocks.size();
      P.mvt_blocks.insert(P.mvt_blocks.end(), collist[I].begin(), collist[I].end());
    }
    P.mvt_row0[N] = (int32_t)P.mvt_blocks.size();
  }

  // blocks grouped by first column leaf / by last column leaf
  std::vector<std::vector<int32_t>> starts(N), ends(N);
  for (size_t x = 0; x < P.blocks.size(); ++x) {
    const BlockDesc &B = P.blocks[x];
    starts[B.cleaf].push_back((int32_t)x);
    if (!(B.kind == kDense && B.rleaf == B.cleaf))
      ends[B.cleaf + Bd.span(B) - 1].push_back((int32_t)x);
  }

  P.grams.clear(); P.gchunks.clear(); P.greds.clear(); P.lrt.clear(); P.aent.clear(); P.bent.clear();
  P.apair.clear(); P.bpair.clear(); P.lrpairs.clear();
  P.arow.clear(); P.brow.clear(); P.arow_ent.clear(); P.brow_ent.clear();
  P.dns.clear(); P.dpairs.clear(); P.wpan.clear(); P.hts.clear();
  P.urows.clear(); P.uents.clear(); P.steps.clear();
  P.ws_max = 0;

  std::vector<int32_t> Aset, Bset;
  std::unordered_map<int64_t, int64_t> gram_of;  // (a, b) -> offset, per step
  const int64_t kk = (int64_t)kcap * kcap;

  for (int K = 0; K < N; ++K) {
    StepRange st{};
    int64_t ws = 0;
    gram_of.clear();
    st.gram0 = (int32_t)P.grams.size();
    auto gram = [&](int32_t a, int32_t c) -> int64_t {
      const BlockDesc &A = P.blocks[a], &C = P.blocks[c];
      if (A.kind != kLowRank || C.kind != kLowRank) return -1;
      int64_t key = (int64_t)a * (int64_t)P.blocks.size() + c;
      auto it = gram_of.find(key);
      if (it != gram_of.end()) return it->second;
      GramTask g{};
      g.a = a; g.b = c;
      g.ovb = std::max(A.cbeg, C.cbeg); g.ove = std::min(A.cend, C.cend);
      g.goff = ws; ws += kk;
      P.grams.push_back(g);
      gram_of[key] = g.goff;
      return g.goff;
    };

    // 1. low-rank targets whose column cluster starts at leaf K
    st.lrt0 = (int32_t)P.lrt.size();
    st.aent0 = (int32_t)P.aent.size();
    st.bent0 = (int32_t)P.bent.size();
    st.arow0 = (int32_t)P.arow.size();
    st.brow0 = (int32_t)P.brow.size();
    for (int32_t t : starts[K]) {
      const BlockDesc &T = P.blocks[t];
      if (T.kind != kLowRank) continue;
      LrTarget L{};
      L.blk = t;
      L.m = T.rend - T.rbeg; L.p = T.cend - T.cbeg;
      const int sp = Bd.span(T);
      Bd.collect(T.rleaf, T.rleaf + sp, T.cbeg, Aset, Bd.stampA);
      Bd.collect(T.cleaf, T.cleaf + sp, T.cbeg, Bset, Bd.stampB);
      int32_t ti = (int32_t)P.lrt.size();
      L.a0 = (int32_t)P.aent.size();
      std::unordered_map<int32_t, int32_t> aidx, bidx;
      for (int32_t a : Aset) {
        SideEntry e{};
        e.target = ti; e.blk = a;
        e.toff = ws; ws += Bd.kof(P.blocks[a]) * r;
        e.soff = ws; ws += Bd.kof(P.blocks[a]) * r;
        aidx[a] = (int32_t)P.aent.size();
        P.aent.push_back(e);
      }
      L.a1 = (int32_t)P.aent.size();
      L.b0 = (int32_t)P.bent.size();
      for (int32_t c : Bset) {
        SideEntry e{};
        e.target = ti; e.blk = c;
        e.toff = ws; ws += Bd.kof(P.blocks[c]) * r;
        e.soff = ws; ws += Bd.kof(P.blocks[c]) * r;
        bidx[c] = (int32_t)P.bent.size();
        P.bent.push_back(e);
      }
      L.b1 = (int32_t)P.bent.size();
      // pairs, grouped per A-entry and per B-entry
      std::vector<std::vector<int32_t>> pa(Aset.size()), pb(Bset.size());
      Bd.index_columns(Bset);
      for (size_t ia = 0; ia < Aset.size(); ++ia) {
        Bd.overlapping(P.blocks[Aset[ia]], cand);
        for (int32_t ib : cand) {
          LrPair pr{};
          pr.ae = L.a0 + (int32_t)ia; pr.be = L.b0 + (int32_t)ib;
          pr.goff = gram(Aset[ia], Bset[ib]);
          int32_t pi = (int32_t)P.lrpairs.size();
          P.lrpairs.push_back(pr);
          pa[ia].push_back(pi);
          pb[ib].push_back(pi);
        }
      }
      for (size_t ia = 0; ia < Aset.size(); ++ia) {
        SideEntry &e = P.aent[L.a0 + ia];
        e.p0 = (int32_t)P.apair.size();
        P.apair.insert(P.apair.end(), pa[ia].begin(), pa[ia].end());
        e.p1 = (int32_t)P.apair.size();
      }
      for (size_t ib = 0; ib < Bset.size(); ++ib) {
        SideEntry &e = P.bent[L.b0 + ib];
        e.p0 = (int32_t)P.bpair.size();
        P.bpair.insert(P.bpair.end(), pb[ib].begin(), pb[ib].end());
        e.p1 = (int32_t)P.bpair.size();
      }
      // row tasks
      for (int I = T.rleaf; I < T.rleaf + sp; ++I) {
        RowTask rt{};
        rt.target = ti; rt.leaf = I;
        rt.e0 = (int32_t)P.arow_ent.size();
        for (int32_t x : Bd.rowlist[I]) {
          auto it = aidx.find(x);
          if (it != aidx.end()) P.arow_ent.push_back(it->second);
        }
        rt.e1 = (int32_t)P.arow_ent.size();
        if (rt.e1 - rt.e0 > 512) return "more than 512 blocks cover one leaf row of a target";
        P.arow.push_back(rt);
      }
      for (int J = T.cleaf; J < T.cleaf + sp; ++J) {
        RowTask rt{};
        rt.target = ti; rt.leaf = J;
        rt.e0 = (int32_t)P.brow_ent.size();
        for (int32_t x : Bd.rowlist[J]) {
          auto it = bidx.find(x);
          if (it != bidx.end()) P.brow_ent.push_back(it->second);
        }
        rt.e1 = (int32_t)P.brow_ent.size();
        if (rt.e1 - rt.e0 > 512) return "more than 512 blocks cover one leaf row of a target";
        P.brow.push_back(rt);
      }
      L.yoff = ws; ws += (int64_t)L.m * r;
      L.zoff = ws; ws += (int64_t)L.p * r;
      L.soff = ws; ws += 4LL * r * r;
      L.tcoff = ws; ws += (int64_t)std::max(kc, r) * r;
      // TSQR row groups: a group streams its rows 64 at a time through one
      // CTA, and the final combine stacks the groups' R factors one after
      // another, so about sqrt(rows / 64) groups balance the two chains
      auto groups = [](int rows) {
        int g = (int)std::ceil(std::sqrt((double)rows / 64.0));
        return std::max(1, std::min(32, g));
      };
      L.gm = groups(L.m);
      L.gp = groups(L.p);
      L.roff = ws; ws += (int64_t)std::max(L.gm, L.gp) * r * r;
      P.lrt.push_back(L);
    }
    st.lrt1 = (int32_t)P.lrt.size();
    st.aent1 = (int32_t)P.aent.size();
    st.bent1 = (int32_t)P.bent.size();
    st.arow1 = (int32_t)P.arow.size();
    st.brow1 = (int32_t)P.brow.size();

    // 2. dense targets of column K, the diagonal first
    st.dns0 = (int32_t)P.dns.size();
    std::vector<int32_t> dlist;
    dlist.push_back(P.diag_of_leaf[K]);
    for (int32_t t : starts[K])
      if (P.blocks[t].kind == kDense && t != P.diag_of_leaf[K]) dlist.push_back(t);
    for (int32_t t : dlist) {
      const BlockDesc &T = P.blocks[t];
      DenseTarget dt{};
      dt.blk = t;
      dt.p0 = (int32_t)P.dpairs.size();
      Bd.collect(T.rleaf, T.rleaf + 1, T.cbeg, Aset, Bd.stampA);
      Bd.collect(T.cleaf, T.cleaf + 1, T.cbeg, Bset, Bd.stampB);
      Bd.index_columns(Bset);
      for (int32_t a : Aset) {
        Bd.overlapping(P.blocks[a], cand);
        for (int32_t q : cand) {
          const int32_t c = Bset[q];
          DPair pr{};
          pr.a = a; pr.b = c; pr.goff = gram(a, c);
          P.dpairs.push_back(pr);
        }
      }
      dt.p1 = (int32_t)P.dpairs.size();
      P.dns.push_back(dt);
    }
    st.dns1 = (int32_t)P.dns.size();
    st.gram1 = (int32_t)P.grams.size();
    st.dpws = ws;
    ws += (int64_t)(P.dns[st.dns1 - 1].p1 - P.dns[st.dns0].p0) * b * b;
    // row chunks of the grams (512 rows each), partial sums reduced in order
    st.gch0 = (int32_t)P.gchunks.size();
    st.gred0 = (int32_t)P.greds.size();
    for (int gi = st.gram0; gi < st.gram1; ++gi) {
      const GramTask &g = P.grams[gi];
      const int len = g.ove - g.ovb, nch = std::max(1, (len + 511) / 512);
      int64_t poff = -1;
      if (nch > 1) {
        poff = ws;
        ws += (int64_t)nch * kk;
        P.greds.push_back(GramReduce{gi, nch, poff});
      }
      for (int c = 0; c < nch; ++c) {
        GramChunk ch{};
        ch.g = gi;
        ch.r0 = g.ovb + c * 512;
        ch.r1 = std::min(g.ove, ch.r0 + 512);
        ch.out = nch > 1 ? poff + (int64_t)c * kk : g.goff;
        P.gchunks.push_back(ch);
      }
    }
    st.gch1 = (int32_t)P.gchunks.size();
    st.gred1 = (int32_t)P.greds.size();

    // 3. panels advanced by the forward solve of leaf K
    st.wpan0 = (int32_t)P.wpan.size();
    panels_above(N - 1 + K, pans);   // the panels whose cluster holds leaf K
    P.wpan.insert(P.wpan.end(), pans.begin(), pans.end());
    st.wpan1 = (int32_t)P.wpan.size();

    // 4. deferred updates by blocks whose columns end at leaf K
    st.ht0 = (int32_t)P.hts.size();
    st.ur0 = (int32_t)P.urows.size();
    std::map<std::pair<int32_t, int32_t>, std::vector<UpdEntry>> rows;  // (panel, leaf)
    for (int32_t a : ends[K]) {
      const BlockDesc &A = P.blocks[a];
      // the panels containing A: clusters holding both its rows and columns
      int hr = cid(A.level, A.rleaf >> (depth - A.level));
      int hc = cid(A.level, A.cleaf >> (depth - A.level));
      while (hr != hc) { hr = (hr - 1) / 2; hc = (hc - 1) / 2; }
      panels_above(hr, pans);
      for (int32_t pi : pans) {
        UpdEntry ue{};
        ue.a = a; ue.hoff = -1;
        if (A.kind == kLowRank) {
          HTask h{};
          h.a = a; h.panel = pi;
          h.hoff = ws; ws += (int64_t)kcap * P.panels[pi].width;
          P.hts.push_back(h);
          ue.hoff = h.hoff;
        }
        for (int I = A.rleaf; I < A.rleaf + Bd.span(A); ++I)
          rows[{pi, I}].push_back(ue);
      }
    }
    st.ht1 = (int32_t)P.hts.size();
    for (auto &kv : rows) {
      UpdRow ur{};
      ur.panel = kv.first.first; ur.leaf = kv.first.second;
      ur.e0 = (int32_t)P.uents.size();
      P.uents.insert(P.uents.end(), kv.second.begin(), kv.second.end());
      ur.e1 = (int32_t)P.uents.size();
      P.urows.push_back(ur);
    }
    st.ur1 = (int32_t)P.urows.size();
    st.ws_words = ws;
    P.ws_max = std::max(P.ws_max, ws);
    P.steps.push_back(st);
  }
  // the right-hand-side panel's share of the deferred updates
  P.hts_rhs.clear(); P.urows_rhs.clear(); P.uents_rhs.clear();
  P.ht_rhs0.assign(N + 1, 0);
  P.ur_rhs0.assign(N + 1, 0);
  for (int K = 0; K < N; ++K) {
    const StepRange &st = P.steps[K];
    P.ht_rhs0[K] = (int32_t)P.hts_rhs.size();
    for (int q = st.ht0; q < st.ht1; ++q)
      if (P.hts[q].panel == P.rhs_panel) P.hts_rhs.push_back(P.hts[q]);
    P.ur_rhs0[K] = (int32_t)P.urows_rhs.size();
    for (int q = st.ur0; q < st.ur1; ++q) {
      if (P.urows[q].panel != P.rhs_panel) continue;
      UpdRow u = P.urows[q];
      const int e0 = (int32_t)P.uents_rhs.size();
      P.uents_rhs.insert(P.uents_rhs.end(), P.uents.begin() + u.e0, P.uents.begin() + u.e1);
      u.e0 = e0;
      u.e1 = (int32_t)P.uents_rhs.size();
      P.urows_rhs.push_back(u);
    }
  }
  P.ht_rhs0[N] = (int32_t)P.hts_rhs.size();
  P.ur_rhs0[N] = (int32_t)P.urows_rhs.size();

  // backward solve: blocks grouped by the first leaf of their rows
  {
    std::vector<std::vector<int32_t>> rstart(N);
    for (size_t x = 0; x < P.blocks.size(); ++x) {
      const BlockDesc &B = P.blocks[x];
      if (B.kind == kDense && B.rleaf == B.cleaf) continue;  // diagonal
      rstart[B.rleaf].push_back((int32_t)x);
    }
    P.bh_blocks.clear(); P.bh0.assign(N + 1, 0);
    P.bupd.clear(); P.bents.clear(); P.bupd0.assign(N + 1, 0);
    for (int K = 0; K < N; ++K) {
      P.bh0[K] = (int32_t)P.bh_blocks.size();
      std::map<int32_t, std::vector<UpdEntry>> cols;   // column leaf -> entries
      for (int32_t x : rstart[K]) {
        const BlockDesc &A = P.blocks[x];
        UpdEntry ue{};
        ue.a = x;
        ue.hoff = -1;
        if (A.kind == kLowRank) {
          ue.hoff = (int64_t)(P.bh_blocks.size() - P.bh0[K]);
          P.bh_blocks.push_back(x);
        }
        for (int J = A.cleaf; J < A.cleaf + Bd.span(A); ++J) cols[J].push_back(ue);
      }
      P.bupd0[K] = (int32_t)P.bupd.size();
      for (auto &kv : cols) {
        UpdRow u{};
        u.panel = -1;
        u.leaf = kv.first;
        u.e0 = (int32_t)P.bents.size();
        P.bents.insert(P.bents.end(), kv.second.begin(), kv.second.end());
        u.e1 = (int32_t)P.bents.size();
        P.bupd.push_back(u);
      }
    }
    P.bh0[N] = (int32_t)P.bh_blocks.size();
    P.bupd0[N] = (int32_t)P.bupd.size();
  }
  return "";
}

}  // namespace hmle
