"""Givens rotations, heads and tails (paper §1.1 and §3).

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np


def givens_matrix(d: int, i: int, j: int, sin: float, cos: float) -> np.ndarray:
    """Def. "Givens rotation" (§3): the d x d identity with G[i,i] = G[j,j] = cos,
    G[i,j] = -sin, G[j,i] = sin.  Indices are 0-based here (the paper's are 1-based)."""
    G = np.eye(d)
    G[i, i] = cos
    G[j, j] = cos
    G[i, j] = -sin
    G[j, i] = sin
    return G


def bindel_rotation(a: float, b: float):
    """§1.1: the rotation that maps (a, b) to (r, 0): sin = -sign(a) b / sqrt(a^2+b^2),
    cos = |a| / sqrt(a^2+b^2), r = sign(a) sqrt(a^2+b^2) (sign(0) taken as +1)."""
    h = np.hypot(a, b)
    sg = 1.0 if a >= 0 else -1.0
    return -sg * b / h, abs(a) / h, sg * h


def head(A: np.ndarray) -> np.ndarray:
    """Def. "Head and Tail" (§3): H(A) = (1/sqrt(m)) * sum of the rows of A (a 1 x n row)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    return A.sum(axis=0, keepdims=True) / np.sqrt(m)


def tail(A: np.ndarray) -> np.ndarray:
    """Def. "Head and Tail" (§3): for j = 1..m-1 (1-based),
    T(A)[j] = ( sqrt(j) A[j+1] - (sum_{i<=j} A[i]) / sqrt(j) ) / sqrt(j+1).
    The prefix sums are taken with numpy.cumsum (a library prefix sum)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    if m <= 1:
        return np.zeros((0, A.shape[1]))
    j = np.arange(1, m, dtype=np.float64)[:, None]        # j = 1..m-1
    prefix = np.cumsum(A, axis=0)[:-1]                     # sum_{i<=j} A[i], j = 1..m-1
    return (np.sqrt(j) * A[1:] - prefix / np.sqrt(j)) / np.sqrt(j + 1.0)


def gen_head(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Def. "Generalized Head and Tail" (§3): H(A, v) = (1/||v||) sum_i v[i] A[i]."""
    A = np.asarray(A, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    return (v[:, None] * A).sum(axis=0, keepdims=True) / np.sqrt(np.sum(v * v))


def gen_tail_def(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Def. "Generalized Head and Tail" (§3), row j = 1..m-1 (1-based), in the reading
    that the ungarbled Alg. 2 confirms:
      T(A, v)[j] = ( ||v[1..j]|| A[j+1] - v[j+1] (sum_{i<=j} v[i] A[i]) / ||v[1..j]|| )
                   / ||v[1..j+1]||.
    Norms and prefix sums use numpy (sqrt, cumsum)."""
    A = np.asarray(A, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    m = A.shape[0]
    if m <= 1:
        return np.zeros((0, A.shape[1]))
    nv = np.sqrt(np.cumsum(v * v))                         # ||v[1..k]||, k = 1..m
    pref = np.cumsum(v[:, None] * A, axis=0)               # sum_{i<=k} v[i] A[i]
    out = np.empty((m - 1, A.shape[1]))
    for j in range(1, m):                                   # 1-based j
        out[j - 1] = (nv[j - 1] * A[j] - v[j] * pref[j - 1] / nv[j - 1]) / nv[j]
    return out


def gen_tail(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Alg. 2 (GenTail), step by step: a running ssum_v += v[j]^2 and
    sum_A += v[j] A[j]; row j is (sqrt(ssum_v) A[j+1] - v[j+1] sum_A / sqrt(ssum_v))
    divided by sqrt(ssum_v + v[j+1]^2).  The loop runs over rows; each step is
    vectorised over the columns."""
    A = np.asarray(A, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    m, n = A.shape
    T = np.zeros((max(m - 1, 0), n))
    sum_A = np.zeros(n)
    ssum_v = 0.0
    for j in range(m - 1):                                  # 0-based: rows j+1 of the paper
        ssum_v = ssum_v + v[j] ** 2
        sum_A = sum_A + v[j] * A[j]
        T[j] = np.sqrt(ssum_v) * A[j + 1] - v[j + 1] * sum_A / np.sqrt(ssum_v)
        T[j] = T[j] / np.sqrt(ssum_v + v[j + 1] ** 2)
    return T


def lemma1_rotations(m: int):
    """Lemma 1 (Cartesian product): R_i = Giv_m(1, i, -1/sqrt(i), sqrt(i-1)/sqrt(i)) for
    i = 2..m (1-based); returned as a list of (i, sin, cos) with 0-based i."""
    return [(i - 1, -1.0 / np.sqrt(i), np.sqrt(i - 1) / np.sqrt(i)) for i in range(2, m + 1)]


def lemma2_rotations(v: np.ndarray):
    """Lemma 2 (scaled Cartesian product): R_i = Giv_m(1, i, -v[i]/||v[1..i]||,
    ||v[1..i-1]|| / ||v[1..i]||) for i = 2..m (1-based), as (i0, sin, cos)."""
    v = np.asarray(v, dtype=np.float64)
    out = []
    for i in range(2, len(v) + 1):
        n_i = np.sqrt(np.sum(v[:i] ** 2))
        n_im1 = np.sqrt(np.sum(v[:i - 1] ** 2))
        out.append((i - 1, -v[i - 1] / n_i, n_im1 / n_i))
    return out


def apply_rotations(A: np.ndarray, rotations) -> np.ndarray:
    """Left-multiply A by the explicit d x d Givens matrices R_2, then R_3, ... (each
    rotating row 1 with row i), i.e. compute G A with G = R_m ... R_2 by brute force."""
    A = np.asarray(A, dtype=np.float64)
    d = A.shape[0]
    U = A.copy()
    for (i, s, c) in rotations:
        U = givens_matrix(d, 0, i, s, c) @ U
    return U
