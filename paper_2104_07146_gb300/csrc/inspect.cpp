// Host-only inspection of the factorisation schedule: build the planner's
// task lists for a given block partition without a device, and copy them
// out as flat integer records (hmle_plan_build / hmle_plan_list).  The
// records are the planner's own (hmle_internal.h); the field order of every
// list is stated in include/hmle.h.
#include <cstring>
#include <new>

#include "hmle_internal.h"

struct hmle_plan {
  hmle::Plan P;
};

namespace {

using hmle::Plan;

// Copies records of `width` int64 fields; f(i, row) fills record i.
template <class F>
hmle_status emit(size_t count, int width, int64_t *out, int64_t cap, int64_t *nrec, int32_t *w,
                 F f) {
  if (nrec) *nrec = (int64_t)count;
  if (w) *w = width;
  if (!out) return HMLE_OK;
  if (cap < (int64_t)count * width) return HMLE_ERR_INVALID_ARG;
  for (size_t i = 0; i < count; ++i) f(i, out + (int64_t)i * width);
  return HMLE_OK;
}

hmle_status ints(const std::vector<int32_t> &v, int64_t *out, int64_t cap, int64_t *nrec,
                 int32_t *w) {
  return emit(v.size(), 1, out, cap, nrec, w, [&](size_t i, int64_t *r) { r[0] = v[i]; });
}

hmle_status upd_rows(const std::vector<hmle::UpdRow> &v, int64_t *out, int64_t cap,
                     int64_t *nrec, int32_t *w) {
  return emit(v.size(), 4, out, cap, nrec, w, [&](size_t i, int64_t *r) {
    r[0] = v[i].panel; r[1] = v[i].leaf; r[2] = v[i].e0; r[3] = v[i].e1;
  });
}

hmle_status upd_ents(const std::vector<hmle::UpdEntry> &v, int64_t *out, int64_t cap,
                     int64_t *nrec, int32_t *w) {
  return emit(v.size(), 2, out, cap, nrec, w, [&](size_t i, int64_t *r) {
    r[0] = v[i].a; r[1] = v[i].hoff;
  });
}

hmle_status hts(const std::vector<hmle::HTask> &v, int64_t *out, int64_t cap, int64_t *nrec,
                int32_t *w) {
  return emit(v.size(), 3, out, cap, nrec, w, [&](size_t i, int64_t *r) {
    r[0] = v[i].a; r[1] = v[i].panel; r[2] = v[i].hoff;
  });
}

hmle_status side(const std::vector<hmle::SideEntry> &v, int64_t *out, int64_t cap,
                 int64_t *nrec, int32_t *w) {
  return emit(v.size(), 6, out, cap, nrec, w, [&](size_t i, int64_t *r) {
    r[0] = v[i].target; r[1] = v[i].blk; r[2] = v[i].toff; r[3] = v[i].soff;
    r[4] = v[i].p0; r[5] = v[i].p1;
  });
}

hmle_status rowtasks(const std::vector<hmle::RowTask> &v, int64_t *out, int64_t cap,
                     int64_t *nrec, int32_t *w) {
  return emit(v.size(), 4, out, cap, nrec, w, [&](size_t i, int64_t *r) {
    r[0] = v[i].target; r[1] = v[i].leaf; r[2] = v[i].e0; r[3] = v[i].e1;
  });
}

}  // namespace

extern "C" {

hmle_status hmle_plan_build(int64_t n, int32_t d, int32_t leaf_size, const int32_t *blocks,
                            int32_t nblocks, int32_t max_rank, int32_t oversample,
                            hmle_plan **out) {
  using namespace hmle;
  if (!blocks || !out || nblocks < 1) return HMLE_ERR_INVALID_ARG;
  if (n < 2 || n > (1LL << 30) || (d != 2 && d != 3)) return HMLE_ERR_INVALID_ARG;
  if (leaf_size < 16 || leaf_size > kMaxLeaf || leaf_size % 16 != 0) return HMLE_ERR_INVALID_ARG;
  if (max_rank < 8 || max_rank > kMaxRank || max_rank % 8 != 0) return HMLE_ERR_INVALID_ARG;
  if (oversample < 4 || max_rank + oversample > kMaxSample) return HMLE_ERR_INVALID_ARG;
  const int32_t depth = tree_depth(n, leaf_size);
  if (depth > kMaxLevels - 2) return HMLE_ERR_INVALID_ARG;
  std::vector<int4> blk((size_t)nblocks);
  for (int32_t x = 0; x < nblocks; ++x) {
    const int32_t l = blocks[4 * x], i = blocks[4 * x + 1], j = blocks[4 * x + 2],
                  k = blocks[4 * x + 3];
    if (l < 0 || l > depth || i < 0 || j < 0 || i >= (1 << l) || j > i || (k != 0 && k != 1))
      return HMLE_ERR_INVALID_ARG;
    blk[x] = make_int4(l, i, j, k);
  }
  hmle_plan *p = new (std::nothrow) hmle_plan();
  if (!p) return HMLE_ERR_OOM;
  std::vector<int32_t> cb, ce;
  cluster_ranges(n, depth, cb, ce);
  const int32_t kc = max_rank + 16 <= kMaxRank ? max_rank + 16 : kMaxRank;
  const std::string err = build_plan(p->P, (int32_t)n, d, leaf_size, depth, cb, ce, blk, max_rank,
                                     kc, max_rank + oversample, 1);
  if (!err.empty()) {
    delete p;
    return HMLE_ERR_INVALID_ARG;
  }
  *out = p;
  return HMLE_OK;
}

void hmle_plan_destroy(hmle_plan *p) { delete p; }

hmle_status hmle_plan_list(const hmle_plan *pl, int32_t which, int64_t *out, int64_t cap,
                           int64_t *nrec, int32_t *width) {
  if (!pl) return HMLE_ERR_INVALID_ARG;
  const Plan &P = pl->P;
  switch (which) {
    case HMLE_PLAN_SCALARS:
      return emit(1, 14, out, cap, nrec, width, [&](size_t, int64_t *r) {
        const int64_t v[14] = {P.n, P.d, P.b, P.depth, P.nleaf, P.kcap, P.kc, P.r, P.rhs_panel,
                               P.ws_max, P.dense_words, P.uc_words, P.u_words, P.w_words};
        std::memcpy(r, v, sizeof(v));
      });
    case HMLE_PLAN_BLOCKS:
      return emit(P.blocks.size(), 14, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::BlockDesc &B = P.blocks[i];
        const int64_t v[14] = {B.kind, B.level, B.rbeg, B.rend, B.cbeg, B.cend, B.rleaf,
                               B.cleaf, B.off_d, B.off_uc, B.off_vc, B.off_u, B.panel, B.slot};
        std::memcpy(r, v, sizeof(v));
      });
    case HMLE_PLAN_STEPS:
      return emit(P.steps.size(), 26, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::StepRange &S = P.steps[i];
        const int64_t v[26] = {S.gram0, S.gram1, S.gch0, S.gch1, S.gred0, S.gred1, S.lrt0,
                               S.lrt1, S.aent0, S.aent1, S.bent0, S.bent1, S.arow0, S.arow1,
                               S.brow0, S.brow1, S.dns0, S.dns1, S.wpan0, S.wpan1, S.ht0,
                               S.ht1, S.ur0, S.ur1, S.dpws, S.ws_words};
        std::memcpy(r, v, sizeof(v));
      });
    case HMLE_PLAN_LRT:
      return emit(P.lrt.size(), 14, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::LrTarget &L = P.lrt[i];
        const int64_t v[14] = {L.blk, L.m, L.p, L.a0, L.a1, L.b0, L.b1, L.yoff, L.zoff, L.soff,
                               L.tcoff, L.gm, L.gp, L.roff};
        std::memcpy(r, v, sizeof(v));
      });
    case HMLE_PLAN_AENT: return side(P.aent, out, cap, nrec, width);
    case HMLE_PLAN_BENT: return side(P.bent, out, cap, nrec, width);
    case HMLE_PLAN_LRPAIRS:
      return emit(P.lrpairs.size(), 3, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        r[0] = P.lrpairs[i].ae; r[1] = P.lrpairs[i].be; r[2] = P.lrpairs[i].goff;
      });
    case HMLE_PLAN_DNS:
      return emit(P.dns.size(), 3, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        r[0] = P.dns[i].blk; r[1] = P.dns[i].p0; r[2] = P.dns[i].p1;
      });
    case HMLE_PLAN_DPAIRS:
      return emit(P.dpairs.size(), 3, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        r[0] = P.dpairs[i].a; r[1] = P.dpairs[i].b; r[2] = P.dpairs[i].goff;
      });
    case HMLE_PLAN_PANELS:
      return emit(P.panels.size(), 5, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::PanelDesc &D = P.panels[i];
        r[0] = D.rbeg; r[1] = D.rend; r[2] = D.width; r[3] = D.leaf0; r[4] = D.off;
      });
    case HMLE_PLAN_WPAN: return ints(P.wpan, out, cap, nrec, width);
    case HMLE_PLAN_HTS: return hts(P.hts, out, cap, nrec, width);
    case HMLE_PLAN_UROWS: return upd_rows(P.urows, out, cap, nrec, width);
    case HMLE_PLAN_UENTS: return upd_ents(P.uents, out, cap, nrec, width);
    case HMLE_PLAN_GRAMS:
      return emit(P.grams.size(), 5, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::GramTask &g = P.grams[i];
        r[0] = g.a; r[1] = g.b; r[2] = g.ovb; r[3] = g.ove; r[4] = g.goff;
      });
    case HMLE_PLAN_GCHUNKS:
      return emit(P.gchunks.size(), 4, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        const hmle::GramChunk &c = P.gchunks[i];
        r[0] = c.g; r[1] = c.r0; r[2] = c.r1; r[3] = c.out;
      });
    case HMLE_PLAN_GREDS:
      return emit(P.greds.size(), 3, out, cap, nrec, width, [&](size_t i, int64_t *r) {
        r[0] = P.greds[i].g; r[1] = P.greds[i].nchunk; r[2] = P.greds[i].poff;
      });
    case HMLE_PLAN_AROW: return rowtasks(P.arow, out, cap, nrec, width);
    case HMLE_PLAN_BROW: return rowtasks(P.brow, out, cap, nrec, width);
    case HMLE_PLAN_AROW_ENT: return ints(P.arow_ent, out, cap, nrec, width);
    case HMLE_PLAN_BROW_ENT: return ints(P.brow_ent, out, cap, nrec, width);
    case HMLE_PLAN_APAIR: return ints(P.apair, out, cap, nrec, width);
    case HMLE_PLAN_BPAIR: return ints(P.bpair, out, cap, nrec, width);
    case HMLE_PLAN_HTS_RHS: return hts(P.hts_rhs, out, cap, nrec, width);
    case HMLE_PLAN_UROWS_RHS: return upd_rows(P.urows_rhs, out, cap, nrec, width);
    case HMLE_PLAN_UENTS_RHS: return upd_ents(P.uents_rhs, out, cap, nrec, width);
    case HMLE_PLAN_HT_RHS0: return ints(P.ht_rhs0, out, cap, nrec, width);
    case HMLE_PLAN_UR_RHS0: return ints(P.ur_rhs0, out, cap, nrec, width);
    case HMLE_PLAN_BH_BLOCKS: return ints(P.bh_blocks, out, cap, nrec, width);
    case HMLE_PLAN_BH0: return ints(P.bh0, out, cap, nrec, width);
    case HMLE_PLAN_BUPD: return upd_rows(P.bupd, out, cap, nrec, width);
    case HMLE_PLAN_BENTS: return upd_ents(P.bents, out, cap, nrec, width);
    case HMLE_PLAN_BUPD0: return ints(P.bupd0, out, cap, nrec, width);
    case HMLE_PLAN_MV_ROW0: return ints(P.mv_row0, out, cap, nrec, width);
    case HMLE_PLAN_MV_BLOCKS: return ints(P.mv_blocks, out, cap, nrec, width);
    case HMLE_PLAN_MVT_ROW0: return ints(P.mvt_row0, out, cap, nrec, width);
    case HMLE_PLAN_MVT_BLOCKS: return ints(P.mvt_blocks, out, cap, nrec, width);
    default: return HMLE_ERR_INVALID_ARG;
  }
}

}  // extern "C"
