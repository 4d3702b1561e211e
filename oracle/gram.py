"""A^T A of the join matrix by factorized aggregation over the join tree, without
materialising the join and without FiGaRo's Alg. 3/4 (an independent route).

Test infrastructure only (see ``oracle/__init__.py``).

A^T A = sum over join tuples of y y^T, where y is the concatenation of the data rows
of the joined tuples.  For a block (k, l) of relations:
    sum over join tuples of y_k y_l^T = sum_{t in S_k} y_t m_l(t)^T,
where m_l(t) is the sum of y_l over the join tuples that contain t (for l = k it is
c(t) y_t with c(t) the number of such tuples).  c and m_l are computed by message
passing on the join tree re-rooted at S_k: the message of a subtree to its parent,
grouped by the attributes they share, is (number of join tuples of the subtree,
sum of y_l over them for every S_l of the subtree).  This is the standard sum-product
evaluation of group-by aggregates over acyclic joins that the paper's §5 cites.
Accumulation is in float64 (counts as float64: relative rounding 2^-53).
"""
from __future__ import annotations

import numpy as np

from . import relational as rl


def _neighbors(db):
    nb = {i: set() for i in range(len(db.relations))}
    for i, p in enumerate(db.parent):
        if p >= 0:
            nb[i].add(p)
            nb[p].add(i)
    return nb


def _aggregate(db, k):
    """For every tuple t of S_k: (c(t), {l: m_l(t)} for every l != k)."""
    nb = _neighbors(db)

    def message(j, parent):
        """Message from the subtree of S_j (tree rooted at S_k) to S_parent."""
        rel = db.relations[j]
        M = rel.n_rows
        cnt = np.ones(M)
        sums = {}
        kids = [c for c in nb[j] if c != parent]
        msgs = {}
        for c in kids:
            attrs = rl.shared_attrs(db, j, c)
            mc = message(c, j)
            idx = rl.match_rows(rl.key_columns(rel, attrs), mc["keys"])
            msgs[c] = (mc, idx)
        for c, (mc, idx) in msgs.items():
            ok = idx >= 0
            cnt = cnt * np.where(ok, mc["cnt"][np.maximum(idx, 0)], 0.0)
        for c, (mc, idx) in msgs.items():
            ok = idx >= 0
            other = np.ones(M)
            for c2, (mc2, idx2) in msgs.items():
                if c2 != c:
                    other = other * np.where(idx2 >= 0, mc2["cnt"][np.maximum(idx2, 0)], 0.0)
            for l, s in mc["sums"].items():
                sums[l] = np.where(ok[:, None], s[np.maximum(idx, 0)], 0.0) * other[:, None]
        if parent is None:
            return cnt, sums
        sums[j] = rel.data * cnt[:, None]
        attrs = rl.shared_attrs(db, j, parent)
        kc = rl.key_columns(rel, attrs)
        order, starts, uniq = rl.group_rows(kc)
        G = len(starts) - 1
        gid = np.empty(M, np.int64)
        gid[order] = np.repeat(np.arange(G), np.diff(starts))     # group of every row
        out_cnt = np.bincount(gid, weights=cnt, minlength=G)
        out_sums = {}
        for l, s in sums.items():
            acc = np.zeros((G, s.shape[1]))
            for c in range(s.shape[1]):
                acc[:, c] = np.bincount(gid, weights=s[:, c], minlength=G)
            out_sums[l] = acc
        return {"keys": uniq, "cnt": out_cnt, "sums": out_sums}

    return message(k, None)


def factorized_gram(db) -> np.ndarray:
    """A^T A (N x N) of the natural join, columns in relation order."""
    off = rl.col_offsets(db)
    N = db.n_cols
    G = np.zeros((N, N))
    for k, rel in enumerate(db.relations):
        cnt, sums = _aggregate(db, k)
        ck = slice(off[k], off[k] + rel.n_data)
        G[ck, ck] = rel.data.T @ (rel.data * cnt[:, None])
        for l, s in sums.items():
            cl = slice(off[l], off[l] + db.relations[l].n_data)
            G[ck, cl] = rel.data.T @ s
    return G


def join_size(db) -> int:
    """Number of tuples of the natural join (exact, via Alg.-independent message passing
    with Python integers on the tree rooted at the root)."""
    nb = _neighbors(db)

    def message(j, parent):
        rel = db.relations[j]
        cnt = [1] * rel.n_rows
        for c in nb[j]:
            if c == parent:
                continue
            attrs = rl.shared_attrs(db, j, c)
            mc = message(c, j)
            kc = rl.key_columns(rel, attrs).tolist()
            for t, key in enumerate(kc):
                cnt[t] *= mc.get(tuple(key), 0)
        if parent is None:
            return sum(cnt)
        attrs = rl.shared_attrs(db, j, parent)
        out = {}
        for t, key in enumerate(rl.key_columns(rel, attrs).tolist()):
            out[tuple(key)] = out.get(tuple(key), 0) + cnt[t]
        return out

    return message(db.root, None)
