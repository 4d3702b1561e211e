"""Count queries Phi_circ, Phi_up, Phi_down (paper §5, Fig. 4) and Alg. 3.

Test infrastructure only (see ``oracle/__init__.py``).

Counts are Python integers (exact at any size).  Maps are dicts keyed by key tuples
ordered as ``relational.sort_attrs`` (X_i) or ``relational.parent_attrs`` (X_p / X_ij).
"""
from __future__ import annotations

from collections import defaultdict

from . import relational as rl


def _group_counts(db, J, attrs):
    """|sigma_{attrs = x}(J)| for every x, from a materialised join J."""
    out = defaultdict(int)
    if J["size"] == 0:
        return dict(out)
    cols = [J["attrs"][a] for a in attrs]
    for t in range(J["size"]):
        out[tuple(int(c[t]) for c in cols)] += 1
    return dict(out)


def counts_bruteforce(db):
    """Fig. 4 by definition, materialising each sub-join (tiny inputs only):
      Phi_circ_i(x_i) = |sigma_{X_i=x_i}( join of all S_j, j != i )|
      Phi_up_i(x_p)   = |sigma_{X_p=x_p}( join of the S_j not in the subtree of S_i )|
      Phi_down_i(x_p) = |sigma_{X_p=x_p}( join of the S_j in the subtree of S_i )|
    Returns {i: {"circ": ..., "up": ..., "down": ...}} (up/down absent for the root)."""
    r = len(db.relations)
    out = {}
    for i in range(r):
        xi = rl.sort_attrs(db, i)
        others = [j for j in range(r) if j != i]
        res = {"circ": _group_counts(db, rl.natural_join(db, others), xi)}
        if db.parent[i] >= 0:
            xp = rl.parent_attrs(db, i)
            sub = rl.subtree(db, i)
            outside = [j for j in range(r) if j not in sub]
            res["up"] = _group_counts(db, rl.natural_join(db, outside), xp)
            res["down"] = _group_counts(db, rl.natural_join(db, sub), xp)
        out[i] = res
    return out


def _keys_by_group(db, i):
    """Distinct X_i values of S_i with their row counts (the rows_per_key map)."""
    rel = db.relations[i]
    xi = rl.sort_attrs(db, i)
    kc = rl.key_columns(rel, xi)
    rows = defaultdict(int)
    for key in map(tuple, kc.tolist()):
        rows[key] += 1
    return xi, dict(sorted(rows.items()))


def _projector(db):
    """Projection of a key tuple x_i (ordered by sort_attrs(i)) onto a list of attributes;
    the attribute positions are computed once per (i, attrs)."""
    cache = {}

    def project(i, key, attrs):
        ck = (i, tuple(attrs))
        pos = cache.get(ck)
        if pos is None:
            xi = rl.sort_attrs(db, i)
            pos = tuple(xi.index(a) for a in attrs)
            cache[ck] = pos
        return tuple(key[p] for p in pos)
    return project


def compute_counts(db):
    """Alg. 3 (compute-counts): pass_1 bottom-up computes rows_per_key_i,
    Theta_down_i(x_i) = rows_per_key_i(x_i) * prod_children Phi_down_j(x_ij) and
    Phi_down_i(x_p) = sum of Theta_down_i over the x_i that project to x_p; pass_2
    top-down computes full_join_size_i(x_i) = Theta_down_i(x_i) * Phi_up_i(x_p) (1 at
    the root), accumulates it into Phi_up_j(x_ij) of every child j, sets
    Phi_circ_i(x_i) = full_join_size_i(x_i) / rows_per_key_i(x_i), and divides each
    child's accumulated Phi_up_j by Phi_down_j just before recursing.

    Returns {i: {"rows", "theta", "down", "up", "circ", "full"}}."""
    r = len(db.relations)
    project = _projector(db)
    st = {i: {"rows": {}, "theta": {}, "down": defaultdict(int), "up": defaultdict(int),
              "circ": {}, "full": {}} for i in range(r)}

    def pass1(i):
        for j in rl.children(db, i):
            pass1(j)
        _, rows = _keys_by_group(db, i)
        for x, cnt in rows.items():                               # loop over values x_i
            st[i]["rows"][x] = cnt
            theta = cnt
            for j in rl.children(db, i):
                xij = project(i, x, rl.shared_attrs(db, i, j))
                theta = theta * st[j]["down"].get(xij, 0)
            st[i]["theta"][x] = theta
            if db.parent[i] >= 0:
                xp = project(i, x, rl.parent_attrs(db, i))
                st[i]["down"][xp] += theta

    def pass2(i):
        for x in st[i]["rows"]:                                   # loop over values x_i
            if db.parent[i] >= 0:
                up_count = st[i]["up"].get(project(i, x, rl.parent_attrs(db, i)), 0)
            else:
                up_count = 1
            full = st[i]["theta"][x] * up_count
            st[i]["full"][x] = full
            for j in rl.children(db, i):
                xij = project(i, x, rl.shared_attrs(db, i, j))
                st[j]["up"][xij] += full
            st[i]["circ"][x] = full // st[i]["rows"][x]
            assert full % st[i]["rows"][x] == 0
        for j in rl.children(db, i):
            for xij in list(st[j]["up"].keys()):
                d = st[j]["down"].get(xij, 0)
                st[j]["up"][xij] = st[j]["up"][xij] // d if d else 0
            pass2(j)

    pass1(db.root)
    pass2(db.root)
    for i in range(r):
        st[i]["down"] = dict(st[i]["down"])
        st[i]["up"] = dict(st[i]["up"])
    return st
