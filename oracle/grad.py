"""Gradients of a loss on R with respect to the data columns of the input relations.

Test infrastructure only (see ``oracle/__init__.py``).

The paper computes R (§7) but does not differentiate it; this follows from standard
matrix calculus.  R is the upper-triangular factor, with non-negative diagonal, of A's
QR decomposition (§2 "Output"); R depends on A only through A^T A, and for full column
rank (from dA = dQ R + Q dR with Q^T dQ skew-symmetric and dR upper triangular)

    dL = tr(Rbar^T dR)  =>  Abar = Q copyltu(R Rbar^T) R^-T = A W,
    W = R^-1 copyltu(R Rbar^T) R^-T                                   (N x N, symmetric)

where copyltu(M) keeps the lower triangle of M and mirrors it above the diagonal and
Rbar = dL/dR.  A is the natural join: row tau of A concatenates the data rows of the
tuples that form tau, so the gradient for tuple t of relation S_k is the sum over the
join rows containing t,

    dL/dy_t = sum_{tau contains t} Abar[tau, Y_k] = m(t)^T W[:, Y_k],

with m(t) = sum_{tau contains t} A[tau, :] the join-sum of the rows containing t: on
Y_k it is c(t) y_t (c(t) = number of such rows), on the columns of another relation S_l
the sum of y_l over them.  m(t) comes from the same message passing over the join tree
as ``gram.py`` (independent of Alg. 3/4).  Two special cases have closed forms (pinned
in the tests): L = ||R||_F^2 gives W = 2I and dL/dy_t = 2 c(t) y_t; L = sigma_i gives
W = v_i v_i^T / sigma_i.
"""
from __future__ import annotations

import numpy as np

from . import gram
from . import relational as rl


def copyltu(M: np.ndarray) -> np.ndarray:
    """Lower triangle of M (with the diagonal) mirrored above the diagonal."""
    L = np.tril(M)
    return L + np.tril(M, -1).T


def w_matrix(R: np.ndarray, Rbar: np.ndarray) -> np.ndarray:
    """W = R^-1 copyltu(R Rbar^T) R^-T (R upper triangular, invertible)."""
    S = copyltu(R @ Rbar.T)
    X = np.linalg.solve(R, S)                 # R^-1 S   (library solve)
    return np.linalg.solve(R, X.T).T          # (R^-1 (R^-1 S)^T)^T = R^-1 S R^-T


def join_sums(db, k: int):
    """(c, m) for every tuple t of relation k: c(t) = number of join rows containing t,
    m (M_k x N) = the sum of those join rows of A[:, Y]."""
    off = rl.col_offsets(db)
    N = db.n_cols
    rel = db.relations[k]
    cnt, sums = gram._aggregate(db, k)
    m = np.zeros((rel.n_rows, N))
    m[:, off[k]:off[k] + rel.n_data] = rel.data * cnt[:, None]
    for l, s in sums.items():
        m[:, off[l]:off[l] + db.relations[l].n_data] = s
    return cnt, m


def data_gradient(db, R: np.ndarray, Rbar: np.ndarray):
    """[dL/dY_k for every relation k] (M_k x N_k each) for dL/dR = Rbar."""
    W = w_matrix(R, Rbar)
    off = rl.col_offsets(db)
    out = []
    for k, rel in enumerate(db.relations):
        _, m = join_sums(db, k)
        out.append(m @ W[:, off[k]:off[k] + rel.n_data])
    return out
