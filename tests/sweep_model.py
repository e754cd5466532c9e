"""A numpy interpreter of the factorisation schedule (test infrastructure).

It runs the task lists that the library's planner produces (hmle.Plan) in
their order, with dense numpy arithmetic: the Schur complement of every
target from its pair list, an exact SVD truncation in place of the kernels'
randomised compression, POTRF / TRSM of the dense blocks, the leaf-by-leaf
forward solves of the W-panels and the deferred updates.  The result is the
H-Cholesky factor of Sec. 2 as the schedule defines it, so a wrong or missing
task shows up as a factor that does not reproduce C.  It shares nothing with
the CUDA kernels; the cluster and block trees are built here in numpy.
"""
from __future__ import annotations


import numpy as np
import scipy.linalg as sla

import oracle
from paper_2104_07146_gb300 import hmle


def cluster_tree(locs, leaf):
    """Median bisection along the longest bounding-box side (ties: the first
    axis), stable within a cluster; cluster ranges halve as in the library."""
    n = locs.shape[0]
    depth = 0
    while -(-n // (1 << depth)) > leaf:
        depth += 1
    perm = np.arange(n)
    levels = [[(0, n)]]
    for _ in range(depth):
        nxt = []
        for b, e in levels[-1]:
            idx = perm[b:e]
            pts = locs[idx]
            ax = int(np.argmax(pts.max(0) - pts.min(0)))
            perm[b:e] = idx[np.argsort(pts[:, ax], kind="stable")]
            mid = b + (e - b) // 2
            nxt += [(b, mid), (mid, e)]
        levels.append(nxt)
    boxes = [[(locs[perm[b:e]].min(0), locs[perm[b:e]].max(0)) for b, e in lv] for lv in levels]
    return depth, perm, boxes


def block_tree(depth, boxes, eta):
    """(level, i, j, kind) of the lower triangle: admissible when
    min(diam) <= eta dist (boxes); leaf-level admissible pairs stay dense."""
    def diam(l, i):
        lo, hi = boxes[l][i]
        return float(np.linalg.norm(hi - lo))

    def dist(l, i, j):
        (lo1, hi1), (lo2, hi2) = boxes[l][i], boxes[l][j]
        return float(np.linalg.norm(np.maximum(0.0, np.maximum(lo1 - hi2, lo2 - hi1))))

    out, stack = [], [(0, 0, 0)]
    while stack:
        l, i, j = stack.pop()
        if i != j and min(diam(l, i), diam(l, j)) <= eta * dist(l, i, j):
            out.append((l, i, j, 1 if l < depth else 0))
            continue
        if l == depth:
            out.append((l, i, j, 0))
            continue
        for a in (0, 1):
            for c in (0, 1):
                if 2 * i + a >= 2 * j + c:
                    stack.append((l + 1, 2 * i + a, 2 * j + c))
    return out


def execute(locs, Z, theta, leaf=32, eta=2.0, eps=1e-8, max_rank=48, form="llt"):
    """Factor C~ by the planner's schedule (rank capacity max_rank per block).

    form "llt": C~ = L L^T (H-Cholesky).  form "ldlt": C~ = L D L^T with L
    unit lower triangular and D diagonal (Sec. 2, no square roots), on the
    same schedule: every block is held as M = L D (the diagonal leaves as
    their unit factors, d apart), and every product over a column index k
    carries the weight 1 / d_k (M_X D^{-1} M_Y^T = L_X D L_Y^T).  The leaf
    factorisation is a pivot-free LDL^T, the off-diagonal solves and W-panel
    solves use the unit factors, log|C~| = sum log d and the quadratic form is
    sum w_k^2 / d_k.

    Returns (log|C~|, Z^T C~^{-1} Z, dense L~ (for "ldlt": L D^(1/2), the
    Cholesky factor it equals), C in cluster order, permutation, number of
    low-rank blocks, largest rank)."""
    n, d = locs.shape
    depth, perm, boxes = cluster_tree(locs, leaf)
    blocks = block_tree(depth, boxes, eta)
    plan = hmle.Plan(n, d, leaf, blocks, max_rank=max_rank, oversample=64 - max_rank)
    Ls = {k: plan.list(k) for k in hmle.PLAN_LISTS}
    plan.close()
    lp = locs[perm]
    C = oracle.matern_matrix(lp, theta)
    B = [dict(kind=int(r[0]), rb=int(r[2]), re=int(r[3]), cb=int(r[4]), ce=int(r[5]),
              panel=int(r[12]), slot=int(r[13])) for r in Ls["blocks"]]
    panels = [dict(rb=int(p[0]), re=int(p[1]), W=np.zeros((int(p[1] - p[0]), int(p[2]))))
              for p in Ls["panels"]]
    rhs = len(panels) - 1
    panels[rhs]["W"][:, 0] = np.asarray(Z, dtype=np.float64)[perm]
    Dn, U, rank = {}, {}, {}
    ldlt = form == "ldlt"
    dinv = np.ones(n)                  # 1 / d_k (all ones for L L^T)

    def W_of(x):                       # right factor of a low-rank block, rows = its columns
        b = B[x]
        P = panels[b["panel"]]
        return P["W"][b["cb"] - P["rb"]:b["ce"] - P["rb"], b["slot"]:b["slot"] + rank[x]]

    def L_dense(x):                    # L_X as a dense (rows x cols) array
        return Dn[x] if B[x]["kind"] == 0 else U[x] @ W_of(x).T

    def schur(x, pairs):               # S_X = C_X - sum over its pairs
        T = B[x]
        S = C[T["rb"]:T["re"], T["cb"]:T["ce"]].copy()
        for a, c in pairs:
            A, Y = B[a], B[c]
            o0, o1 = max(A["cb"], Y["cb"]), min(A["ce"], Y["ce"])
            r0, r1 = max(A["rb"], T["rb"]), min(A["re"], T["re"])
            s0, s1 = max(Y["rb"], T["cb"]), min(Y["re"], T["ce"])
            LA, LY = L_dense(a), L_dense(c)
            S[r0 - T["rb"]:r1 - T["rb"], s0 - T["cb"]:s1 - T["cb"]] -= \
                (LA[r0 - A["rb"]:r1 - A["rb"], o0 - A["cb"]:o1 - A["cb"]] * dinv[o0:o1]) @ \
                LY[s0 - Y["rb"]:s1 - Y["rb"], o0 - Y["cb"]:o1 - Y["cb"]].T
        return S

    logdet = 0.0
    aent, bent, lrp, dp = Ls["aent"], Ls["bent"], Ls["lrpairs"], Ls["dpairs"]
    for K, st in enumerate(Ls["steps"]):
        # 1. low-rank targets: S_T from its pairs, truncated SVD, W0 = S_T^T U_T
        for t in Ls["lrt"][st[6]:st[7]]:
            x = int(t[0])
            pairs = [(int(aent[p[0]][1]), int(bent[p[1]][1])) for p in lrp if t[3] <= p[0] < t[4]]
            S = schur(x, pairs)
            Uu, sv, _ = np.linalg.svd(S, full_matrices=False)
            T = B[x]
            cn = np.linalg.norm(C[T["rb"]:T["re"], T["cb"]:T["ce"]])
            thr = eps * eps * max(float(np.sum(sv ** 2)), cn * cn)
            tail = np.cumsum((sv ** 2)[::-1])[::-1]          # tail[k] = sum_{i >= k} sigma_i^2
            k = int(np.sum(tail > thr))
            assert k <= max_rank, "rank above the capacity"
            U[x] = Uu[:, :k]
            rank[x] = k
            P = panels[T["panel"]]
            P["W"][T["cb"] - P["rb"]:T["ce"] - P["rb"], T["slot"]:T["slot"] + k] = S.T @ U[x]
        # 2. dense targets of column K, the diagonal first
        Lkk = None
        for q in Ls["dns"][st[16]:st[17]]:
            x = int(q[0])
            S = schur(x, [(int(p[0]), int(p[1])) for p in dp[q[1]:q[2]]])
            if Lkk is None:
                if ldlt:
                    Lkk, dk = oracle.ldlt(S)             # unit lower, pivots d
                    assert np.all(dk > 0.0), "non-positive pivot"
                    T = B[x]
                    dinv[T["rb"]:T["re"]] = 1.0 / dk
                    logdet += float(np.sum(np.log(dk)))
                    Dn[x] = Lkk * dk[None, :]            # M = L D; the solves use Lkk
                else:
                    Lkk = np.linalg.cholesky(S)
                    logdet += 2.0 * float(np.sum(np.log(np.diag(Lkk))))
                    Dn[x] = Lkk
            else:
                Dn[x] = sla.solve_triangular(Lkk, S.T, lower=True, unit_diagonal=ldlt).T
        kb, ke = B[int(Ls["dns"][st[16]][0])]["rb"], B[int(Ls["dns"][st[16]][0])]["re"]
        # 3. rows of leaf K of every open W-panel: W <- L_KK^{-1} W
        for pi in Ls["wpan"][st[18]:st[19]]:
            P = panels[int(pi[0])]
            r0 = kb - P["rb"]
            P["W"][r0:r0 + ke - kb] = sla.solve_triangular(Lkk, P["W"][r0:r0 + ke - kb], lower=True,
                                                           unit_diagonal=ldlt)
        # 4. deferred updates by the blocks whose columns end at K
        for ur in Ls["urows"][st[22]:st[23]]:
            pi, I, e0, e1 = (int(v) for v in ur)
            P = panels[pi]
            ib, ie = _leaf_range(Ls, I)
            for e in range(e0, e1):
                a = int(Ls["uents"][e][0])
                A = B[a]
                LA = L_dense(a)
                P["W"][ib - P["rb"]:ie - P["rb"]] -= \
                    (LA[ib - A["rb"]:ie - A["rb"]] * dinv[A["cb"]:A["ce"]]) @ \
                    P["W"][A["cb"] - P["rb"]:A["ce"] - P["rb"]]
    w = panels[rhs]["W"][:, 0]
    Ld = np.zeros((n, n))
    for x, b in enumerate(B):
        Ld[b["rb"]:b["re"], b["cb"]:b["ce"]] = L_dense(x)
    Ld = np.tril(Ld)                   # the diagonal leaves' upper triangles are zero already
    if ldlt:
        Ld = Ld * np.sqrt(dinv)[None, :]   # M D^{-1/2} = L D^{1/2}
    q = float(np.sum(w * w * dinv))
    return logdet, q, Ld, C, perm, len(rank), max(rank.values(), default=0)


def _leaf_range(Ls, I):
    s = Ls["scalars"][0]
    depth, n = int(s[3]), int(s[0])
    b, e = 0, n
    for lv in range(depth):
        mid = b + (e - b) // 2
        if (I >> (depth - 1 - lv)) & 1:
            b = mid
        else:
            e = mid
    return b, e
