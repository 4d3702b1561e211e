"""SVD and PCA of the join matrix through R (paper §8.2-8.3).

Test infrastructure only (see ``oracle/__init__.py``).

§8.2: with A = Q R and R = U_R Sigma_R V_R^T, the singular values of A are those of R
and its right singular vectors are V_R.  §8.3: the principal components of A are the
columns of V for the largest singular values, with eigenvalues sigma^2 of A^T A (the
paper's experiments do not centre the data).  Centred PCA (not in the paper) takes the
eigenvectors of the scatter matrix of the centred join rows,
(A - 1 mu^T)^T (A - 1 mu^T) = A^T A - |J| mu mu^T (mu = column means over the join, |J|
its row count): a rank-1 downdate of A^T A = R^T R.
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


def _eig_desc(C: np.ndarray, k: int):
    lam, W = np.linalg.eigh(C)
    lam, W = lam[::-1], W[:, ::-1]
    k = min(k, len(lam))
    return normalize_columns_sign(W[:, :k]), lam[:k]


def centered_pca_materialized(A: np.ndarray, k: int):
    """Top-k principal components and eigenvalues of the scatter matrix of the centred rows
    of a materialised A (the definition; small joins only)."""
    Ac = A - A.mean(axis=0, keepdims=True)
    return _eig_desc(Ac.T @ Ac, k)


def centered_pca_of_r(R: np.ndarray, colsum: np.ndarray, n_rows: int, k: int):
    """The same from R (R^T R = A^T A), the join's column sums and its row count |J|:
    A^T A - |J| mu mu^T = R^T R - colsum colsum^T / |J|."""
    C = R.T @ R - np.outer(colsum, colsum) / float(n_rows)
    return _eig_desc(C, k)

