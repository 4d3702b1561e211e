"""SVD and PCA of the join matrix through R (paper §8.2-8.3).

Test infrastructure only (see ``oracle/__init__.py``).

§8.2: with A = Q R and R = U_R Sigma_R V_R^T, the singular values of A are those of R
and its right singular vectors are V_R.  §8.3: the principal components of A are the
columns of V for the largest singular values, with eigenvalues sigma^2 of A^T A (the
paper's experiments do not centre the data, and neither does this oracle).
The SVD of the n x n matrix R is numpy.linalg.svd (LAPACK), a library step.
"""
from __future__ import annotations

import numpy as np


def normalize_columns_sign(V: np.ndarray) -> np.ndarray:
    """Make the largest-magnitude entry of every column positive (first one on ties)."""
    V = np.array(V, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V


def svd_of_r(R: np.ndarray):
    """(sigma descending, V) of R: the singular values and right singular vectors of A."""
    _, s, Vt = np.linalg.svd(np.asarray(R, dtype=np.float64))
    return s, normalize_columns_sign(Vt.T)


def pca_of_r(R: np.ndarray, k: int):
    """Top-k principal components (columns of V) and their eigenvalues sigma^2."""
    s, V = svd_of_r(R)
    k = min(k, len(s))
    return V[:, :k], s[:k] ** 2
