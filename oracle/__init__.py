"""CPU oracle for FiGaRo (Olteanu, Vortmeier, Zivanovic: "Givens Rotations for QR
Decomposition, SVD and PCA over Database Joins", arXiv 2204.00525).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run anything
in this package.  The product path (``paper_2204_00525_gb300``) never imports it and
shares no code with it; the only common dependency is ``synth`` (seeded inputs, no
method arithmetic).

Everything here is plain, slow and in float64 (Python integers for the count
aggregates).  Each function cites the passage of the paper it follows:

  givens.py       Def. of Givens rotations (§3), Def. of head/tail and generalized
                  head/tail, Alg. 2 (GenTail), the rotation sequences of Lemmas 1-2
  relational.py   §2 data model: grouping by key attributes, natural join
                  (materialisation of A), full reduction (removal of dangling tuples)
  counts.py       Fig. 4 count queries (brute force from the definitions) and
                  Alg. 3 (compute-counts)
  figaro.py       Alg. 4 (FiGaRo: heads_and_tails, process_and_join_children,
                  project_away_join_attributes) and the §7 post-processing
  householder.py  textbook Householder QR (the QR used by the post-processing)
  gram.py         A^T A by factorized aggregation over the join tree (independent of
                  Alg. 3/4), used to check R^T R = A^T A at any size
  spectral.py     §8.2-8.3: SVD and PCA of A through the SVD of R
  grad.py         gradients of a loss on R with respect to the relations' data columns
                  (matrix calculus of the QR factor; join sums by message passing)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, brute force, library routines or
values the paper prints; none is "parity unpinned".
"""
