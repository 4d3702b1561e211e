"""Textbook Householder QR (the off-the-shelf QR that the paper's §7 post-processing
uses for its blocks), returning only R.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np


def householder_r(A: np.ndarray) -> np.ndarray:
    """R of the QR decomposition of A (m x n), as an n x n upper-triangular matrix
    (rows below min(m, n) are zero), normalised to a non-negative diagonal (the
    uniqueness condition of §2 "Output": R with positive diagonal is unique when A has
    full rank; a zero diagonal entry keeps its row as computed).

    For k = 0..min(m,n)-1: x = A[k:, k]; the reflector I - 2 v v^T / (v^T v) with
    v = x - alpha e_1, alpha = -sign(x_0) ||x||, maps x to alpha e_1 and is applied to
    the trailing columns A[k:, k:]."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    for k in range(min(m, n)):
        x = A[k:, k]
        normx = np.sqrt(np.dot(x, x))
        if normx == 0.0:
            continue
        alpha = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= alpha
        vv = np.dot(v, v)
        if vv == 0.0:
            continue
        w = v @ A[k:, k:]
        A[k:, k:] -= np.outer(v, (2.0 / vv) * w)
        A[k + 1:, k] = 0.0
    R = np.zeros((n, n))
    r = min(m, n)
    R[:r] = np.triu(A[:r])
    return sign_normalize(R)


def sign_normalize(R: np.ndarray) -> np.ndarray:
    """Multiply row k of R by the sign of R[k, k] (zero counts as positive)."""
    R = np.array(R, dtype=np.float64, copy=True)
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return R * s[:, None]
