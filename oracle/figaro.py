"""Alg. 4 (FiGaRo) and the §7 post-processing.

Test infrastructure only (see ``oracle/__init__.py``).

``figaro_r0`` follows Alg. 4 procedure by procedure on a fully reduced database:
  heads_and_tails              tails sqrt(Phi_circ_i(x_i)) T(S_i^{x_i}) go to Out,
                               Data[x_i : Y_i] = H(S_i^{x_i}), scales[x_i] = sqrt|S_i^{x_i}|
  process_and_join_children    recurse into every child j; Data[x_i : Y_k] =
                               Data_j[x_ij : Y_k] * scales[x_i] * prod_{other children j'}
                               scales_j'[x_ij'] for S_k in the subtree of S_j; then
                               Data[x_i : Y_i] and scales[x_i] are multiplied by
                               prod_j scales_j[x_ij]
  project_away_join_attributes for every x_p: Out gets sqrt(Phi_up_i(x_p)) T(Data[x_p,*],
                               scales[x_p,*]); Data'[x_p] = H(Data[x_p,*], scales[x_p,*]),
                               scales'[x_p] = sqrt(Phi_down_i(x_p))
  root                         Out.append(Data)

Readings of the paper taken here:
  * the product "j' in [r] \\ {j}" in process_and_join_children ranges over the other
    children of S_i (the text after Alg. 4 and the beta_{jkl} factors of the §6 example
    fix this);
  * the rows appended to Out with the same column support (all tails of one relation;
    all generalized tails of one node; the root Data) form one block of R0 for the
    post-processing;
  * groups are visited in ascending key order with X_p first (relational.sort_attrs),
    rows inside a group in input order.
"""
from __future__ import annotations

import numpy as np

from . import relational as rl
from .counts import compute_counts
from .givens import head, tail, gen_head, gen_tail
from .householder import householder_r


class Block:
    """A block of R0: ``rows`` (float64 [rows, len(cols)]) living on the global columns
    ``cols`` of A[:, Y]."""

    def __init__(self, kind, rel, cols, rows):
        self.kind, self.rel, self.cols, self.rows = kind, rel, list(cols), rows

    def __repr__(self):
        return f"Block({self.kind}, S{self.rel + 1}, {self.rows.shape})"


def figaro_r0(db, counts=None, record=None):
    """Alg. 4 on a fully reduced database: returns the list of R0 blocks.  If ``record``
    is a dict, record[i] receives the (Data, scales) that S_i returns to its parent."""
    counts = compute_counts(db) if counts is None else counts
    blocks = []

    def figaro(i):
        rel = db.relations[i]
        xi_attrs = rl.sort_attrs(db, i)
        order, starts, uniq = rl.group_rows(rl.key_columns(rel, xi_attrs))
        G = len(starts) - 1
        keys = [tuple(u) for u in uniq.tolist()]
        own_cols = rl.cols_of(db, [i])
        sub_cols = rl.cols_of(db, rl.subtree(db, i))
        pos = {c: k for k, c in enumerate(sub_cols)}
        own = [pos[c] for c in own_cols]
        Data = np.zeros((G, len(sub_cols)))
        scales = np.zeros(G)

        # heads_and_tails
        tails = [np.zeros((0, len(own_cols)))]
        for g in range(G):
            S_x = rel.data[order[starts[g]:starts[g + 1]]]
            tails.append(tail(S_x) * np.sqrt(counts[i]["circ"][keys[g]]))
            Data[g, own] = head(S_x)[0]
            scales[g] = np.sqrt(S_x.shape[0])
        blocks.append(Block("tails", i, own_cols, np.concatenate(tails)))

        ch = rl.children(db, i)
        if ch:
            # process_and_join_children
            res = {j: figaro(j) for j in ch}
            proj = {j: [xi_attrs.index(a) for a in rl.shared_attrs(db, i, j)] for j in ch}
            for g in range(G):
                idx, s = {}, {}
                for j in ch:
                    xij = tuple(keys[g][p] for p in proj[j])
                    idx[j] = res[j]["index"][xij]
                    s[j] = res[j]["scales"][idx[j]]
                for j in ch:
                    other = 1.0
                    for jj in ch:
                        if jj != j:
                            other *= s[jj]
                    for c_pos, c in enumerate(res[j]["cols"]):
                        Data[g, pos[c]] = res[j]["Data"][idx[j], c_pos] * scales[g] * other
                prod_all = 1.0
                for j in ch:
                    prod_all *= s[j]
                Data[g, own] *= prod_all
                scales[g] *= prod_all

        if db.parent[i] >= 0 and not ch:
            # a leaf: X_i = X_p (every join attribute of a leaf is shared with its
            # parent), so Data already has one row per x_p and Alg. 4 returns it as is.
            index = {keys[g]: g for g in range(G)}
            if record is not None:
                record[i] = (Data.copy(), scales.copy())
            return {"Data": Data, "scales": scales, "index": index, "cols": sub_cols}
        if db.parent[i] >= 0:
            # project_away_join_attributes: groups are sorted with X_p first, so the
            # x_i sharing one x_p are consecutive.
            n_xp = len(rl.parent_attrs(db, i))
            xp_keys = [k[:n_xp] for k in keys]
            seg = [0] + [g for g in range(1, G) if xp_keys[g] != xp_keys[g - 1]] + [G]
            P = len(seg) - 1
            Data2 = np.zeros((P, len(sub_cols)))
            scales2 = np.zeros(P)
            index = {}
            gts = [np.zeros((0, len(sub_cols)))]
            for p in range(P):
                a, b = seg[p], seg[p + 1]
                xp = xp_keys[a]
                D, v = Data[a:b], scales[a:b]
                gts.append(gen_tail(D, v) * np.sqrt(counts[i]["up"][xp]))
                Data2[p] = gen_head(D, v)[0]
                scales2[p] = np.sqrt(counts[i]["down"][xp])
                index[xp] = p
            blocks.append(Block("gen_tails", i, sub_cols, np.concatenate(gts)))
            if record is not None:
                record[i] = (Data2.copy(), scales2.copy())
            return {"Data": Data2, "scales": scales2, "index": index, "cols": sub_cols}
        blocks.append(Block("root", i, sub_cols, Data))
        return None

    figaro(db.root)
    return blocks


def postprocess(blocks, n_cols):
    """§7: triangularize every non-zero block of R0 on its own columns (dropping the
    zero rows that arise), stack the triangles in global column positions and
    triangularize the stack.  Householder QR is used for both steps."""
    tris = []
    for b in blocks:
        if b.rows.shape[0] == 0:
            continue
        Rb = householder_r(b.rows)
        full = np.zeros((Rb.shape[0], n_cols))
        full[:, b.cols] = Rb
        tris.append(full)
    if not tris:
        return np.zeros((n_cols, n_cols))
    return householder_r(np.concatenate(tris))


def figaro_r(db):
    """R of A[:, Y] by FiGaRo: full reduction (§2 assumes a fully reduced database),
    Alg. 3, Alg. 4, then the §7 post-processing."""
    red = rl.full_reduce(db)
    return postprocess(figaro_r0(red), db.n_cols)


def materialized_r(db):
    """R of A[:, Y] by Householder QR of the materialised join (small inputs only)."""
    A = rl.join_matrix(db)
    return householder_r(A)
