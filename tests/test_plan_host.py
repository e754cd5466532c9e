"""The planner (host logic of the leaf sweep) against the definitions it
implements, on random block partitions, without a GPU.

The left-looking H-Cholesky (Sec. 2) needs, for every block T of the lower
triangle with first column s,

    S_T = C_T - sum_{k < s} L[rows T, k] L[cols T, k]^T,

so the pairs of factor blocks that update T are exactly those (X, Y) with X
holding an entry (i, k) and Y an entry (j, k), i in rows T, j in cols T,
k < s.  The blocks tile the lower triangle, so at leaf resolution every
(I, K) with K <= I has one owner block, and the pair set of T is
{(owner(I, K), owner(J, K)) : I in rows T, J in cols T, K < s}.  These tests
derive every list of the schedule that way (targets per step, side entries,
pairs, row tasks, W-panels, deferred updates, backward and matvec lists)
and compare them with hmle_plan_list, and check that every step's
workspace regions are disjoint and inside the step's workspace.
"""
import itertools

import numpy as np
import pytest

from paper_2104_07146_gb300 import hmle


def partition(depth, rng, p_adm=0.5, leaf_lowrank=False):
    """A random block tree: diagonal pairs split into three children, an
    off-diagonal pair is low-rank with probability p_adm (at level >= 1)
    or splits into four; leaf pairs are dense (or low-rank off the diagonal
    when leaf_lowrank)."""
    out = []

    def rec(lv, i, j):
        if i == j:
            if lv == depth:
                out.append((lv, i, j, 0))
                return
            rec(lv + 1, 2 * i, 2 * j)
            rec(lv + 1, 2 * i + 1, 2 * j)
            rec(lv + 1, 2 * i + 1, 2 * j + 1)
            return
        if lv == depth:
            out.append((lv, i, j, 1 if (leaf_lowrank and rng.random() < p_adm) else 0))
            return
        if lv >= 1 and rng.random() < p_adm:
            out.append((lv, i, j, 1))
            return
        for a, c in itertools.product((0, 1), (0, 1)):
            rec(lv + 1, 2 * i + a, 2 * j + c)

    rec(0, 0, 0)
    order = rng.permutation(len(out))          # the planner must not rely on input order
    return [out[k] for k in order]


def clusters(n, depth):
    """The documented halving rule: heap order, cluster h splits at b + (e - b) // 2."""
    cb, ce = [0] * ((2 << depth) - 1), [0] * ((2 << depth) - 1)
    ce[0] = n
    for h in range((1 << depth) - 1):
        b, e = cb[h], ce[h]
        mid = b + (e - b) // 2
        cb[2 * h + 1], ce[2 * h + 1] = b, mid
        cb[2 * h + 2], ce[2 * h + 2] = mid, e
    return cb, ce


def depth_of(n, leaf):
    d = 0
    while -(-n // (1 << d)) > leaf:
        d += 1
    return d


CASES = [  # n, leaf, max_rank, oversample, p_adm, leaf_lowrank, seed
    (16, 16, 8, 4, 0.5, False, 9),         # one leaf: the diagonal block only
    (40, 32, 32, 8, 0.5, False, 1),
    (100, 16, 16, 8, 0.5, False, 2),
    (250, 16, 32, 8, 0.6, False, 3),
    (500, 32, 48, 16, 0.4, False, 4),
    (333, 16, 8, 4, 0.7, True, 5),
    (1000, 32, 32, 8, 0.5, True, 6),
    (1023, 32, 24, 8, 0.3, False, 7),
    (4096, 64, 32, 8, 0.6, False, 8),      # overlaps above 512 points: chunked grams
    # the smallest n of each leaf size at depth 1 and 2 (the smallest clusters)
    (17, 16, 8, 4, 0.5, False, 10),
    (33, 16, 8, 4, 0.5, True, 11),
    (33, 32, 16, 8, 0.5, False, 12),
    (65, 32, 16, 8, 0.5, True, 13),
    (65, 64, 32, 8, 0.5, False, 14),
    (129, 64, 32, 8, 0.5, True, 15),
    (129, 128, 32, 8, 0.5, False, 16),
    (257, 128, 32, 8, 0.5, True, 17),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "n%d_leaf%d_s%d" % (c[0], c[1], c[6]))
def case(request):
    n, leaf, kcap, osamp, p_adm, llr, seed = request.param
    depth = depth_of(n, leaf)
    rng = np.random.default_rng(seed)
    blocks = partition(depth, rng, p_adm, llr)
    plan = hmle.Plan(n, 2, leaf, blocks, max_rank=kcap, oversample=osamp)
    L = {name: plan.list(name) for name in hmle.PLAN_LISTS}
    plan.close()
    return dict(n=n, leaf=leaf, kcap=kcap, osamp=osamp, depth=depth, input=blocks, L=L)


def _blocks(case):
    """Exported blocks as dicts, with their leaf spans and the owner map."""
    depth = case["depth"]
    N = 1 << depth
    B = []
    owner = {}
    for x, rec in enumerate(case["L"]["blocks"]):
        kind, lv, rb, re_, cb, ce, rl, cl = (int(v) for v in rec[:8])
        sp = 1 << (depth - lv)
        B.append(dict(kind=kind, level=lv, rbeg=rb, rend=re_, cbeg=cb, cend=ce, rleaf=rl,
                      cleaf=cl, span=sp, off_d=int(rec[8]), off_uc=int(rec[9]),
                      off_vc=int(rec[10]), off_u=int(rec[11]), panel=int(rec[12]),
                      slot=int(rec[13]), diag=(kind == 0 and rl == cl)))
        for I in range(rl, rl + sp):
            for J in range(cl, cl + sp):
                assert (I, J) not in owner, "blocks overlap"
                owner[(I, J)] = x
    assert len(owner) == N * (N + 1) // 2, "blocks do not tile the lower triangle"
    for (I, J) in owner:
        assert J <= I
    return B, owner, N


def test_scalars_blocks_and_clusters(case):
    L, depth, n, leaf = case["L"], case["depth"], case["n"], case["leaf"]
    s = L["scalars"][0]
    assert list(s[:9]) == [n, 2, leaf, depth, 1 << depth, case["kcap"],
                           min(case["kcap"] + 16, 64), case["kcap"] + case["osamp"],
                           len(L["panels"]) - 1]
    B, owner, N = _blocks(case)
    assert len(B) == len(case["input"])
    assert sorted((b["level"], b["rleaf"] >> (depth - b["level"]), b["cleaf"] >> (depth - b["level"]),
                   b["kind"]) for b in B) == sorted(tuple(t) for t in case["input"])
    cb, ce = clusters(n, depth)
    for b in B:
        lv = b["level"]
        hr = (1 << lv) - 1 + (b["rleaf"] >> (depth - lv))
        hc = (1 << lv) - 1 + (b["cleaf"] >> (depth - lv))
        assert (b["rbeg"], b["rend"], b["cbeg"], b["cend"]) == (cb[hr], ce[hr], cb[hc], ce[hc])
    # storage: dense slots are distinct b x b slots; low-rank regions disjoint
    dn = sorted(b["off_d"] for b in B if b["kind"] == 0)
    assert dn == [k * leaf * leaf for k in range(len(dn))] and s[10] == len(dn) * leaf * leaf
    uc = []
    for b in B:
        if b["kind"] == 1:
            m, p = b["rend"] - b["rbeg"], b["cend"] - b["cbeg"]
            uc += [(b["off_uc"], m * s[6]), (b["off_vc"], p * s[6])]
    _disjoint(uc, s[11])
    _disjoint([(b["off_u"], (b["rend"] - b["rbeg"]) * s[5]) for b in B if b["kind"] == 1], s[12])


def _disjoint(regions, limit):
    regions = sorted((o, o + ln) for o, ln in regions if ln > 0)
    for (a0, a1), (b0, b1) in zip(regions, regions[1:]):
        assert a1 <= b0, ((a0, a1), (b0, b1))
    if regions:
        assert regions[0][0] >= 0 and regions[-1][1] <= limit, (regions[-1], limit)


def _rows(b):
    return range(b["rleaf"], b["rleaf"] + b["span"])


def _cols(b):
    return range(b["cleaf"], b["cleaf"] + b["span"])


def test_cluster_nesting_agrees_with_point_ranges(case):
    """The planner finds column overlaps through the cluster tree (nested or
    disjoint clusters).  That equals the point-range definition
    max(begin) < min(end) only if no cluster is empty: check both on every
    pair of exported blocks, rows and columns."""
    B, _, _ = _blocks(case)
    for b in B:
        assert b["rbeg"] < b["rend"] and b["cbeg"] < b["cend"]
    for a in B:
        for b in B:
            by_points = max(a["cbeg"], b["cbeg"]) < min(a["cend"], b["cend"])
            by_leaves = max(a["cleaf"], b["cleaf"]) < min(a["cleaf"] + a["span"], b["cleaf"] + b["span"])
            assert by_points == by_leaves
            by_points = max(a["rbeg"], b["rbeg"]) < min(a["rend"], b["rend"])
            by_leaves = max(a["rleaf"], b["rleaf"]) < min(a["rleaf"] + a["span"], b["rleaf"] + b["span"])
            assert by_points == by_leaves


def test_targets_per_step(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    steps = L["steps"]
    assert len(steps) == N
    lrt, dns = L["lrt"], L["dns"]
    for K in range(N):
        st = steps[K]
        got = sorted(int(lrt[t][0]) for t in range(st[6], st[7]))
        want = sorted(x for x, b in enumerate(B) if b["kind"] == 1 and b["cleaf"] == K)
        assert got == want
        dl = [int(dns[t][0]) for t in range(st[16], st[17])]
        assert dl[0] == owner[(K, K)] and B[dl[0]]["diag"]
        assert sorted(dl) == sorted(x for x, b in enumerate(B) if b["kind"] == 0 and b["cleaf"] == K)
    # every target once, steps in order
    assert sorted(int(t[0]) for t in lrt) == sorted(x for x, b in enumerate(B) if b["kind"] == 1)


def _pairs_by_definition(owner, rows, cols, s_leaf):
    return {(owner[(I, K)], owner[(J, K)]) for I in rows for J in cols for K in range(s_leaf)}


def test_low_rank_targets_have_exactly_their_updates(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    aent, bent, lrp, apair, bpair = L["aent"], L["bent"], L["lrpairs"], L["apair"], L["bpair"]
    for ti, t in enumerate(L["lrt"]):
        T = B[int(t[0])]
        assert (int(t[1]), int(t[2])) == (T["rend"] - T["rbeg"], T["cend"] - T["cbeg"])
        s = T["cleaf"]
        a_blk = [int(aent[e][1]) for e in range(t[3], t[4])]
        b_blk = [int(bent[e][1]) for e in range(t[5], t[6])]
        assert all(int(aent[e][0]) == ti for e in range(t[3], t[4]))
        assert all(int(bent[e][0]) == ti for e in range(t[5], t[6]))
        assert sorted(a_blk) == sorted({owner[(I, K)] for I in _rows(T) for K in range(s)})
        assert sorted(b_blk) == sorted({owner[(J, K)] for J in _cols(T) for K in range(s)})
        want = _pairs_by_definition(owner, _rows(T), _cols(T), s)
        got = [(int(aent[p[0]][1]), int(bent[p[1]][1])) for p in lrp
               if t[3] <= p[0] < t[4]]
        assert len(got) == len(set(got)) and set(got) == want
        for p in lrp:
            if t[3] <= p[0] < t[4]:
                assert t[5] <= p[1] < t[6]
                both_lr = B[int(aent[p[0]][1])]["kind"] == 1 and B[int(bent[p[1]][1])]["kind"] == 1
                assert (p[2] >= 0) == both_lr
        # each entry lists exactly the pairs it takes part in
        for e in range(t[3], t[4]):
            mine = sorted(int(apair[q][0]) for q in range(aent[e][4], aent[e][5]))
            assert mine == sorted(k for k, p in enumerate(lrp) if p[0] == e)
        for e in range(t[5], t[6]):
            mine = sorted(int(bpair[q][0]) for q in range(bent[e][4], bent[e][5]))
            assert mine == sorted(k for k, p in enumerate(lrp) if p[1] == e)


def test_row_tasks_cover_each_leaf_row_of_a_target(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    for which, ent, ents, span in (("arow", L["aent"], L["arow_ent"], _rows),
                                   ("brow", L["bent"], L["brow_ent"], _cols)):
        tasks = L[which]
        for ti, t in enumerate(L["lrt"]):
            T = B[int(t[0])]
            mine = [r for r in tasks if r[0] == ti]
            assert sorted(int(r[1]) for r in mine) == list(span(T))
            lo, hi = (t[3], t[4]) if which == "arow" else (t[5], t[6])
            for r in mine:
                got = sorted(int(ent[int(ents[q][0])][1]) for q in range(r[2], r[3]))
                assert all(lo <= int(ents[q][0]) < hi for q in range(r[2], r[3]))
                want = sorted(int(ent[e][1]) for e in range(lo, hi)
                              if int(r[1]) in _rows(B[int(ent[e][1])]))
                assert got == want


def test_dense_targets_have_exactly_their_updates(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    dp = L["dpairs"]
    for d in L["dns"]:
        T = B[int(d[0])]
        want = _pairs_by_definition(owner, _rows(T), _cols(T), T["cleaf"])
        got = [(int(dp[q][0]), int(dp[q][1])) for q in range(d[1], d[2])]
        assert len(got) == len(set(got)) and set(got) == want


def test_panels_and_forward_solve_order(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    depth, kcap, n = case["depth"], case["kcap"], case["n"]
    panels = L["panels"]
    rhs = len(panels) - 1
    assert (panels[rhs][0], panels[rhs][1], panels[rhs][3]) == (0, n, 0)
    lr = [b for b in B if b["kind"] == 1]
    by_panel = {}
    for b in lr:
        by_panel.setdefault(b["panel"], []).append(b)
    assert set(by_panel) == set(range(rhs))
    for pi, bl in by_panel.items():
        P = panels[pi]
        assert all((P[0], P[1]) == (b["cbeg"], b["cend"]) for b in bl)
        assert P[2] == kcap * len(bl)
        assert sorted(b["slot"] for b in bl) == [kcap * k for k in range(len(bl))]
    _disjoint([(int(P[4]), int((P[1] - P[0]) * P[2])) for P in panels], L["scalars"][0][13])
    # step K solves the leaf-K rows of every panel whose leaf range holds K
    lv = {pi: bl[0]["level"] for pi, bl in by_panel.items()}
    for K, st in enumerate(L["steps"]):
        got = sorted(int(L["wpan"][q][0]) for q in range(st[18], st[19]))
        want = sorted([pi for pi in range(rhs)
                       if panels[pi][3] <= K < panels[pi][3] + (1 << (depth - lv[pi]))] + [rhs])
        assert got == want


def test_deferred_updates_reach_every_panel_row_once_before_its_solve(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    panels, hts, urows, uents = L["panels"], L["hts"], L["urows"], L["uents"]
    pushed = {}
    for K, st in enumerate(L["steps"]):
        step_h = {int(hts[q][2]): (int(hts[q][0]), int(hts[q][1])) for q in range(st[20], st[21])}
        for q in range(st[22], st[23]):
            pi, I, e0, e1 = (int(v) for v in urows[q])
            assert K < I, "a row is updated before the step that solves it"
            for e in range(e0, e1):
                a, hoff = int(uents[e][0]), int(uents[e][1])
                A = B[a]
                assert A["cleaf"] + A["span"] - 1 == K        # pushed when its columns end
                if A["kind"] == 1:
                    assert step_h[hoff] == (a, pi)
                else:
                    assert hoff == -1
                key = (pi, I, a)
                assert key not in pushed
                pushed[key] = K
    want = set()
    for pi, P in enumerate(panels):
        for a, A in enumerate(B):
            if A["diag"] or not (P[0] <= A["cbeg"] and A["rend"] <= P[1]):
                continue
            for I in _rows(A):
                want.add((pi, I, a))
    assert set(pushed) == want
    # the right-hand-side panel's share, step by step
    rhs = len(panels) - 1
    for K, st in enumerate(L["steps"]):
        h0, h1 = L["ht_rhs0"][K][0], L["ht_rhs0"][K + 1][0]
        assert [tuple(r) for r in L["hts_rhs"][h0:h1]] == \
            [tuple(hts[q]) for q in range(st[20], st[21]) if hts[q][1] == rhs]
        u0, u1 = L["ur_rhs0"][K][0], L["ur_rhs0"][K + 1][0]
        mine = [urows[q] for q in range(st[22], st[23]) if urows[q][0] == rhs]
        assert len(mine) == u1 - u0
        for r, q in zip(mine, L["urows_rhs"][u0:u1]):
            assert (r[0], r[1]) == (q[0], q[1])
            assert [tuple(x) for x in uents[r[2]:r[3]]] == [tuple(x) for x in L["uents_rhs"][q[2]:q[3]]]


def test_forward_rhs_updates_use_their_own_steps_products(case):
    # the multi-vector sweeps (hmle_prediction_errors) give each vector kcap
    # doubles per right-hand-side product of a step instead of the factor's
    # workspace: every low-rank entry of a step's right-hand-side rows must
    # use one of that same step's products, and each product's offset is
    # distinct within the step
    L = case["L"]
    hts, uents, urows = L["hts_rhs"], L["uents_rhs"], L["urows_rhs"]
    N = 1 << case["depth"]
    for K in range(N):
        h0, h1 = L["ht_rhs0"][K][0], L["ht_rhs0"][K + 1][0]
        offs = [int(hts[q][2]) for q in range(h0, h1)]
        assert len(set(offs)) == len(offs)
        for q in range(L["ur_rhs0"][K][0], L["ur_rhs0"][K + 1][0]):
            for e in range(int(urows[q][2]), int(urows[q][3])):
                h = int(uents[e][1])
                assert h == -1 or h in offs


def test_backward_sweep_lists(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    bh, bh0, bupd, bents, bupd0 = L["bh_blocks"], L["bh0"], L["bupd"], L["bents"], L["bupd0"]
    for K in range(N):
        starting = [a for a, A in enumerate(B) if not A["diag"] and A["rleaf"] == K]
        lr = [int(v[0]) for v in bh[bh0[K][0]:bh0[K + 1][0]]]
        assert sorted(lr) == sorted(a for a in starting if B[a]["kind"] == 1)
        got = {}
        for q in range(bupd0[K][0], bupd0[K + 1][0]):
            _, J, e0, e1 = (int(v) for v in bupd[q])
            for e in range(e0, e1):
                a, h = int(bents[e][0]), int(bents[e][1])
                assert (h == -1) == (B[a]["kind"] == 0)
                if h >= 0:
                    assert lr[h] == a
                got.setdefault(J, []).append(a)
        want = {}
        for a in starting:
            for J in _cols(B[a]):
                want.setdefault(J, []).append(a)
        assert {J: sorted(v) for J, v in got.items()} == {J: sorted(v) for J, v in want.items()}


def test_matvec_lists(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    r0, mb, t0, tb = L["mv_row0"], L["mv_blocks"], L["mvt_row0"], L["mvt_blocks"]
    for I in range(N):
        row = [int(v[0]) for v in mb[r0[I][0]:r0[I + 1][0]]]
        assert row[0] == owner[(I, I)]
        assert sorted(row[1:]) == sorted(a for a, A in enumerate(B) if not A["diag"] and I in _rows(A))
        col = [int(v[0]) for v in tb[t0[I][0]:t0[I + 1][0]]]
        assert sorted(col) == sorted(a for a, A in enumerate(B) if not A["diag"] and I in _cols(A))


def test_step_workspaces_are_disjoint(case):
    L = case["L"]
    B, owner, N = _blocks(case)
    s = L["scalars"][0]
    b, kcap, kc, r, ws_max = int(s[2]), int(s[5]), int(s[6]), int(s[7]), int(s[9])
    kof = lambda x: kcap if B[x]["kind"] == 1 else b
    for K, st in enumerate(L["steps"]):
        reg = []
        for t in L["lrt"][st[6]:st[7]]:
            m, p, gm, gp = int(t[1]), int(t[2]), int(t[11]), int(t[12])
            reg += [(t[7], m * r), (t[8], p * r), (t[9], 4 * r * r), (t[10], max(kc, r) * r),
                    (t[13], max(gm, gp) * r * r)]
        for e in list(L["aent"][st[8]:st[9]]) + list(L["bent"][st[10]:st[11]]):
            reg += [(e[2], kof(int(e[1])) * r), (e[3], kof(int(e[1])) * r)]
        reg += [(g[4], kcap * kcap) for g in L["grams"][st[0]:st[1]]]
        reg += [(g[2], g[1] * kcap * kcap) for g in L["greds"][st[4]:st[5]]]
        npair = int(L["dns"][st[17] - 1][2] - L["dns"][st[16]][1])
        reg += [(st[24], npair * b * b)]
        panels = L["panels"]
        reg += [(h[2], kcap * int(panels[int(h[1])][2])) for h in L["hts"][st[20]:st[21]]]
        _disjoint([(int(o), int(ln)) for o, ln in reg], int(st[25]))
        assert st[25] <= ws_max
        # gram chunks: 512-row pieces of each gram's overlap, in order
        for gi in range(st[0], st[1]):
            g = L["grams"][gi]
            ch = [c for c in L["gchunks"][st[2]:st[3]] if c[0] == gi]
            assert [int(c[1]) for c in ch] == list(range(int(g[2]), int(g[3]), 512)) or \
                (g[2] == g[3] and len(ch) == 1)
            assert int(ch[-1][2]) == int(g[3])


def test_rejects_out_of_range_records():
    with pytest.raises(hmle.HmleError):
        hmle.Plan(100, 2, 16, [(0, 0, 0, 0)])                    # a dense block above the leaf level
    with pytest.raises(hmle.HmleError):
        hmle.Plan(40, 2, 32, [(1, 0, 1, 0), (1, 0, 0, 0), (1, 1, 1, 0)])   # above the diagonal
    with pytest.raises(hmle.HmleError):
        hmle.Plan(40, 2, 32, [(5, 0, 0, 0)])                     # level beyond the depth
    with pytest.raises(hmle.HmleError):
        hmle.Plan(40, 2, 24, [(0, 0, 0, 0)])                     # leaf size not a multiple of 16
