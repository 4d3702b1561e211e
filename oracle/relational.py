"""Relations as matrices (paper §2 "Setup"): grouping by key attributes, the natural
join that defines the matrix A, and full reduction (removal of dangling tuples).

Test infrastructure only (see ``oracle/__init__.py``).

A database is the ``synth.Database`` container: relations S_1..S_r with key columns
identified by global attribute ids and data columns Y_i, plus a join tree given as a
parent array.  The column order of A[:, Y] is relation order, then data-column order
inside each relation (the [T_1 ... T_r] layout of Alg. 4).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- tree structure

def children(db, i):
    return [j for j, p in enumerate(db.parent) if p == i]


def subtree(db, i):
    """Relations in the subtree of S_i (S_i included), in relation order."""
    out = {i}
    stack = [i]
    while stack:
        u = stack.pop()
        for c in children(db, u):
            out.add(c)
            stack.append(c)
    return sorted(out)


def shared_attrs(db, i, j):
    """X_ij: the join attributes common to S_i and S_j, in ascending attribute id."""
    return sorted(set(db.relations[i].key_attrs) & set(db.relations[j].key_attrs))


def parent_attrs(db, i):
    """X_p for S_i: the attributes S_i shares with its parent (empty for the root)."""
    p = db.parent[i]
    return [] if p < 0 else shared_attrs(db, i, p)


def sort_attrs(db, i):
    """The order in which S_i is sorted and grouped.  The paper (§5) assumes S_i sorted
    on X_i with a child first sorted on the attributes shared with its parent; the
    order of attributes within each part is not fixed there, and this oracle takes
    ascending attribute id: X_p first, then the rest of X_i."""
    xp = parent_attrs(db, i)
    rest = sorted(set(db.relations[i].key_attrs) - set(xp))
    return xp + rest


def col_offsets(db):
    """Global column offset of each relation's Y_i in A[:, Y]."""
    off, acc = [], 0
    for r in db.relations:
        off.append(acc)
        acc += r.n_data
    return off


def cols_of(db, rels):
    off = col_offsets(db)
    return [off[k] + c for k in sorted(rels) for c in range(db.relations[k].n_data)]


def key_columns(rel, attrs):
    """The key matrix of ``rel`` restricted to ``attrs`` (in that order), int64 [M, len]."""
    idx = [rel.key_attrs.index(a) for a in attrs]
    return rel.keys[:, idx] if idx else np.zeros((rel.n_rows, 0), np.int64)


def group_rows(keys: np.ndarray):
    """Group the rows of an int64 key matrix by equal key tuples.

    Returns (order, starts, uniq): ``order`` lists the row indices sorted
    lexicographically by key with ties kept in input order (a stable sort),
    ``starts`` the group boundaries in ``order`` (length G+1) and ``uniq`` the G
    distinct key tuples in ascending lexicographic order."""
    m, k = keys.shape
    if k == 0:
        order = np.arange(m)
        return order, np.array([0, m]) if m else np.array([0]), np.zeros((1 if m else 0, 0), np.int64)
    order = np.lexsort(keys.T[::-1])                       # numpy lexsort is stable
    sk = keys[order]
    head = np.ones(m, dtype=bool)
    head[1:] = np.any(sk[1:] != sk[:-1], axis=1)
    starts = np.concatenate([np.flatnonzero(head), [m]])
    return order, starts, sk[head]


def _row_ids(a: np.ndarray, b: np.ndarray):
    """Number the distinct rows of the int64 matrices ``a`` and ``b`` (same width) jointly:
    equal rows get equal ids.  Returns (ids of a's rows, ids of b's rows, number of ids)."""
    both = np.concatenate([a, b], axis=0)
    order, starts, _ = group_rows(both)
    G = len(starts) - 1
    ids = np.empty(both.shape[0], np.int64)
    ids[order] = np.repeat(np.arange(G), np.diff(starts))
    return ids[:a.shape[0]], ids[a.shape[0]:], G


def match_rows(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """For every row of the int64 matrix ``a``, the index of the equal row of ``b`` (whose
    rows are distinct), or -1."""
    if a.shape[1] == 0:
        return np.zeros(a.shape[0], np.int64) if b.shape[0] == 1 else np.full(a.shape[0], -1)
    ia, ib, u = _row_ids(a, b)
    lut = np.full(u, -1, np.int64)
    lut[ib] = np.arange(b.shape[0])
    return lut[ia]


# ---------------------------------------------------------------- natural join

def natural_join(db, rels=None):
    """The natural join of the relations ``rels`` (all by default): a dict with the
    row index of each participating relation for every output tuple, and the value of
    every attribute.  Relations that share no attribute with the partial result are
    joined by Cartesian product.  Plain hash join; small inputs only."""
    rels = list(range(len(db.relations))) if rels is None else list(rels)
    if not rels:
        return {"rows": {}, "attrs": {}, "size": 1}
    # order: start from the first relation, then repeatedly take one that shares attributes
    todo = rels[1:]
    cur_rows = {rels[0]: np.arange(db.relations[rels[0]].n_rows)}
    r0 = db.relations[rels[0]]
    cur_attr = {a: r0.keys[:, c].copy() for c, a in enumerate(r0.key_attrs)}
    size = r0.n_rows
    while todo:
        pick = next((j for j in todo if set(db.relations[j].key_attrs) & set(cur_attr)), todo[0])
        todo.remove(pick)
        R = db.relations[pick]
        common = sorted(set(R.key_attrs) & set(cur_attr))
        # bucket R's rows by the common attributes
        buckets = {}
        rk = key_columns(R, common)
        for t, key in enumerate(map(tuple, rk.tolist())):
            buckets.setdefault(key, []).append(t)
        left, right = [], []
        ck = np.stack([cur_attr[a] for a in common], axis=1) if common else np.zeros((size, 0), np.int64)
        for u, key in enumerate(map(tuple, ck.tolist())):
            for t in buckets.get(key, ()):
                left.append(u)
                right.append(t)
        left = np.array(left, dtype=np.int64)
        right = np.array(right, dtype=np.int64)
        cur_rows = {k: v[left] for k, v in cur_rows.items()}
        cur_rows[pick] = right
        cur_attr = {a: v[left] for a, v in cur_attr.items()}
        for c, a in enumerate(R.key_attrs):
            if a not in cur_attr:
                cur_attr[a] = R.keys[right, c]
        size = len(left)
    return {"rows": cur_rows, "attrs": cur_attr, "size": size}


def join_matrix(db) -> np.ndarray:
    """A[:, Y] (§2 "From Relations to Matrices"): one row per tuple of the natural join,
    the data columns of every relation in relation order."""
    J = natural_join(db)
    parts = [db.relations[k].data[J["rows"][k]] for k in range(len(db.relations))]
    return np.concatenate(parts, axis=1) if parts else np.zeros((J["size"], 0))


# ---------------------------------------------------------------- full reduction

def semijoin_keep(db_rel, other_rel, attrs):
    """Rows of ``db_rel`` whose projection on ``attrs`` occurs in ``other_rel``."""
    a = key_columns(db_rel, attrs)
    b = key_columns(other_rel, attrs)
    if len(attrs) == 0:
        return np.full(db_rel.n_rows, other_rel.n_rows > 0)
    ia, ib, u = _row_ids(a, b)
    present = np.zeros(u, dtype=bool)
    present[ib] = True
    return present[ia]


def full_reduce(db):
    """Remove dangling tuples (§2: a database is fully reduced if every tuple contributes
    to the join output).  For an acyclic join with join tree tau, a bottom-up pass of
    semijoins (parent <- child) followed by a top-down pass (child <- parent) leaves
    exactly the tuples that occur in the join (Yannakakis' full reducer, the calibration
    step mentioned in §8.1).  Returns a new Database."""
    import copy
    out = copy.deepcopy(db)
    rels = out.relations

    def restrict(i, keep):
        r = rels[i]
        r.keys, r.data = r.keys[keep], r.data[keep]

    order = []
    def post(i):
        for c in children(out, i):
            post(c)
        order.append(i)
    post(out.root)
    for i in order:                                       # bottom-up
        p = out.parent[i]
        if p >= 0:
            restrict(p, semijoin_keep(rels[p], rels[i], shared_attrs(out, i, p)))
    for i in reversed(order):                             # top-down
        p = out.parent[i]
        if p >= 0:
            restrict(i, semijoin_keep(rels[i], rels[p], shared_attrs(out, i, p)))
    return out


def is_valid_join_tree(db) -> bool:
    """§2: tau is a join tree iff it is a tree over the relations and, for every pair
    S_i, S_j, every relation on the path between them contains X_ij (equivalently: the
    relations containing any given attribute form a connected subtree)."""
    r = len(db.relations)
    if sorted(db.parent).count(-1) != 1 or len(db.parent) != r:
        return False
    seen = set()
    def dfs(i):
        if i in seen:
            return False
        seen.add(i)
        return all(dfs(c) for c in children(db, i))
    if not dfs(db.root) or len(seen) != r:
        return False
    attrs = {a for rel in db.relations for a in rel.key_attrs}
    for a in attrs:
        holders = {i for i, rel in enumerate(db.relations) if a in rel.key_attrs}
        # connected iff exactly one holder has no holder parent
        tops = [i for i in holders if db.parent[i] not in holders]
        if len(tops) != 1:
            return False
    return True
