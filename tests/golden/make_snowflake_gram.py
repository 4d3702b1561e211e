"""Writes tests/golden/snowflake_gram.npz: A^T A of the 10M-row snowflake workload
(D3(c) 100k rows - D1(a, c) 1M - F(a, b) 10M - D2(b) 1M, 50 U[-1,1] columns each, 10 of the
200 columns x 1e4; synth.snowflake() with its default seed) by the oracle's factorized
aggregation over the join tree (oracle.gram.factorized_gram, independent of Alg. 3/4),
with the input fingerprint (synth.fingerprint) it belongs to.

The benchmark measures the R^T R error of its FP64 and mixed runs against this matrix
instead of against another GPU result.  Calls only oracle/ and synth/.  Run from the
repository root:  python tests/golden/make_snowflake_gram.py   (a few minutes)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np

import synth
from oracle import gram, relational

OUT = os.path.join(ROOT, "tests", "golden", "snowflake_gram.npz")


def main():
    db = synth.snowflake()
    G = gram.factorized_gram(relational.full_reduce(db))
    np.savez_compressed(OUT, gram=G, fingerprint=np.array(synth.fingerprint(db)),
                        workload=np.array(db.description))
    print(f"wrote {OUT}: {G.shape}, fingerprint {synth.fingerprint(db)}")


if __name__ == "__main__":
    main()
