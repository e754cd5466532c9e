// Algorithmic FP64 work of one evaluation, per kernel kind, tallied on the
// host from the θ-independent plan and the ranks that evaluation produced.
// This is the flop counter per phase: it counts the arithmetic the
// left-looking sweep must do with the actual ranks (not the padded block
// capacities).  The assembly (Matern entries, ACA) is not part of the sweep
// and is not counted here.  Used for the achieved-throughput side of the
// roofline.
#include <algorithm>

#include "hmle_internal.h"
#include "tally.h"

namespace hmle {

double tally_flops(const Plan &P, int kind, const std::vector<int32_t> &rc,
                   const std::vector<int32_t> &rl, const std::vector<int32_t> &kept, int osamp,
                   double jacobi_flops) {
  const int r = P.r, b = P.b, qr = 64;
  auto sw = [&](int blk) { return std::min(r, std::max(8, rc[blk]) + osamp); };
  auto keff = [&](int blk) {
    const BlockDesc &B = P.blocks[blk];
    return (double)(B.kind == kLowRank ? rl[blk] : B.cend - B.cbeg);
  };
  auto rows_in = [&](int blk, int lo, int hi) {
    const BlockDesc &B = P.blocks[blk];
    return (double)std::max(0, std::min(hi, B.rend) - std::max(lo, B.rbeg));
  };
  auto hh = [&](double h, double c) { return 2.0 * h * c * c - 2.0 * c * c * c / 3.0; };
  double f = 0.0;
  switch (kind) {
    case 0:  // k_gram
      for (const GramTask &g : P.grams) f += 2.0 * (g.ove - g.ovb) * rl[g.a] * rl[g.b];
      break;
    case 1:  // k_side_t (both passes)
      for (const LrTarget &L : P.lrt) {
        const BlockDesc &T = P.blocks[L.blk];
        const double rt = sw(L.blk);
        for (int e = L.b0; e < L.b1; ++e)
          f += 2.0 * rows_in(P.bent[e].blk, T.cbeg, T.cend) * keff(P.bent[e].blk) * rt;
        for (int e = L.a0; e < L.a1; ++e)
          f += 2.0 * rows_in(P.aent[e].blk, T.rbeg, T.rend) * keff(P.aent[e].blk) * rt;
        f += 2.0 * (L.m + L.p) * rc[L.blk] * rt;
      }
      break;
    case 2:  // k_side_s (both passes)
      for (const LrPair &pr : P.lrpairs) {
        const int a = P.aent[pr.ae].blk, c = P.bent[pr.be].blk;
        const double rt = sw(P.lrt[P.aent[pr.ae].target].blk);
        const BlockDesc &A = P.blocks[a], &B = P.blocks[c];
        if (A.kind == kDense && B.kind == kDense) f += 2.0 * (A.cend - A.cbeg) * rt;
        else f += 2.0 * 2.0 * keff(a) * keff(c) * rt;
      }
      break;
    case 3:  // k_rows (both passes)
      for (int pass = 0; pass < 2; ++pass) {
        const std::vector<RowTask> &rows = pass ? P.brow : P.arow;
        const std::vector<int32_t> &ents = pass ? P.brow_ent : P.arow_ent;
        const std::vector<SideEntry> &side = pass ? P.bent : P.aent;
        for (const RowTask &R : rows) {
          const LrTarget &L = P.lrt[R.target];
          const double mi = P.cl_end[(1 << P.depth) - 1 + R.leaf] - P.cl_beg[(1 << P.depth) - 1 + R.leaf];
          double k = rc[L.blk];
          for (int q = R.e0; q < R.e1; ++q) k += keff(side[ents[q]].blk);
          f += 2.0 * mi * sw(L.blk) * k;
        }
      }
      break;
    case 4:  // k_tsqr_part (Y and Z)
      for (const LrTarget &L : P.lrt) {
        const double rt = sw(L.blk);
        f += (std::ceil(L.m / 64.0) + L.gm + std::ceil(L.p / 64.0) + L.gp) * hh(rt + qr, rt);
      }
      break;
    case 5:  // k_tsqr_final: QR of the stacked group factors, the pivoted QR of
             // each r x r R (Y and Z), and the Jacobi sweeps (device count)
      for (const LrTarget &L : P.lrt) {
        const double rt = sw(L.blk);
        f += (L.gm + L.gp) * hh(rt + qr, rt) + 2.0 * hh(rt, rt);
      }
      f += jacobi_flops;
      break;
    case 6:  // k_tall_apply
      for (size_t t = 0; t < P.lrt.size(); ++t) {
        const LrTarget &L = P.lrt[t];
        const double rt = sw(L.blk), k1 = kept[t], k = rl[L.blk];
        f += 2.0 * L.m * rt * k1 * 2.0 + 2.0 * (L.m + L.p) * rt * k;
      }
      break;
    case 7:  // k_cholqr_part
      for (size_t t = 0; t < P.lrt.size(); ++t) f += 2.0 * P.lrt[t].m * kept[t] * kept[t];
      break;
    case 8:  // k_cholqr_final
      for (size_t t = 0; t < P.lrt.size(); ++t) f += 2.0 * std::pow((double)kept[t], 3) / 3.0;
      break;
    case 9:  // k_dense_pair
      for (const DenseTarget &dt : P.dns) {
        const BlockDesc &T = P.blocks[dt.blk];
        const double m = T.rend - T.rbeg, p = T.cend - T.cbeg;
        for (int q = dt.p0; q < dt.p1; ++q) {
          const DPair &pr = P.dpairs[q];
          const BlockDesc &A = P.blocks[pr.a], &B = P.blocks[pr.b];
          const double ka = keff(pr.a), kb = keff(pr.b);
          if (A.kind == kDense && B.kind == kDense) f += 2.0 * m * ka * p;
          else f += 2.0 * ka * kb * p + 2.0 * m * ka * p;
        }
      }
      break;
    case 10:  // k_dense_reduce: the pair products subtracted from the assembled C_IK
      for (const DenseTarget &dt : P.dns) {
        const BlockDesc &T = P.blocks[dt.blk];
        f += (double)(T.rend - T.rbeg) * (T.cend - T.cbeg) * (dt.p1 - dt.p0);
      }
      break;
    case 11:  // k_potrf
      for (int K = 0; K < P.nleaf; ++K) {
        const BlockDesc &D = P.blocks[P.diag_of_leaf[K]];
        f += std::pow((double)(D.rend - D.rbeg), 3) / 3.0;
      }
      break;
    case 12:  // k_trsm
      for (const DenseTarget &dt : P.dns) {
        const BlockDesc &T = P.blocks[dt.blk];
        if (T.rbeg == T.cbeg) continue;
        const double mk = T.cend - T.cbeg;
        f += (double)(T.rend - T.rbeg) * mk * mk;
      }
      break;
    case 13:  // k_wsolve
      for (size_t K = 0; K < P.steps.size(); ++K) {
        const BlockDesc &D = P.blocks[P.diag_of_leaf[K]];
        const double mk = D.rend - D.rbeg;
        for (int q = P.steps[K].wpan0; q < P.steps[K].wpan1; ++q) f += mk * mk * P.panels[P.wpan[q]].width;
      }
      break;
    case 14:  // k_htask
      for (const HTask &h : P.hts) {
        const BlockDesc &A = P.blocks[h.a];
        f += 2.0 * (A.cend - A.cbeg) * rl[h.a] * P.panels[h.panel].width;
      }
      break;
    case 15:  // k_updrow
      for (const UpdRow &R : P.urows) {
        const double mi = P.cl_end[(1 << P.depth) - 1 + R.leaf] - P.cl_beg[(1 << P.depth) - 1 + R.leaf];
        const double w = P.panels[R.panel].width;
        for (int q = R.e0; q < R.e1; ++q) f += 2.0 * mi * keff(P.uents[q].a) * w;
      }
      break;
    default:
      break;
  }
  (void)b;
  return f;
}

}  // namespace hmle
