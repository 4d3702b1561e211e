"""FiGaRo on GB300: the R of the QR decomposition, the SVD and the PCA of the matrix
defined by an acyclic natural join, computed without materialising the join
(arXiv 2204.00525), in CUDA kernels for sm_103a behind the C ABI of include/figaro.h.

``binding`` holds the ctypes binding (same names as the C entry points) and the
``JoinPlan`` helper for torch tensors; ``build_lib`` builds the library in-tree.
"""
from . import build_lib  # noqa: F401
