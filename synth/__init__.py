"""Seeded synthetic databases for the FiGaRo join-QR workloads.

This module only draws random numbers and arranges them into relations; it holds
none of the method's arithmetic.  Both the CPU oracle (``oracle/``) and the GPU path
(``paper_2204_00525_gb300``) consume what it produces, so it is the one piece of code
the two sides share.

Data model (the paper's §2 "Setup"):
  * a database is a list of relations S_1..S_r plus a join tree tau given as a
    parent array (``parent[root] == -1``);
  * every relation has key (join) attributes X_i, identified by global integer
    attribute ids, and data attributes Y_i (real numbers);
  * the natural join joins on equal attribute ids.

Workload shapes follow the paper's experiments (§9: key-fkey snowflake and star
schemas, a many-to-many star schema, and the synthetic Cartesian product with
U[-3,3) data) at the sizes of the benchmark configurations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Relation:
    name: str
    key_attrs: tuple          # global attribute ids of the key columns, in column order
    keys: np.ndarray          # int64 [M, K]
    data: np.ndarray          # float64 [M, N]

    @property
    def n_rows(self) -> int:
        return int(self.data.shape[0])

    @property
    def n_data(self) -> int:
        return int(self.data.shape[1])


@dataclass
class Database:
    relations: list
    parent: list              # join tree: parent index, -1 for the root
    attr_names: list = field(default_factory=list)
    description: str = ""

    @property
    def root(self) -> int:
        return self.parent.index(-1)

    @property
    def n_cols(self) -> int:
        return sum(r.n_data for r in self.relations)

    def input_cells(self) -> int:
        """Cells of the input database: sum over relations of M_i * (N_i + K_i)."""
        return sum(r.n_rows * (r.n_data + len(r.key_attrs)) for r in self.relations)

    def input_bytes(self) -> int:
        return 8 * self.input_cells()


# ----------------------------------------------------------------------------- helpers

def zipf_keys(rng: np.random.Generator, n: int, domain: int, s: float) -> np.ndarray:
    """n draws from a truncated Zipf law P(k) ~ k^-s over k = 1..domain, returned 0-based."""
    p = np.arange(1, domain + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    return rng.choice(domain, size=n, p=p).astype(np.int64)


def covering_keys(rng: np.random.Generator, n: int, domain: int, draw) -> np.ndarray:
    """Every key of [0, domain) appears at least once (domain <= n); the remaining
    n - domain keys come from ``draw(rng, count)``; the result is shuffled."""
    assert domain <= n
    rest = draw(rng, n - domain)
    k = np.concatenate([np.arange(domain, dtype=np.int64), rest.astype(np.int64)])
    rng.shuffle(k)
    return k


def _normal(rng, m, n):
    return rng.standard_normal((m, n))


# ----------------------------------------------------------------------------- workloads

def two_relation(seed: int = 1, rows: int = 1000, keys: int = 100, n_s: int = 3, n_t: int = 2,
                 cover: bool = True) -> Database:
    """S(a; x1..x3) root joined with T(a; y1..y2): uniform key a over ``keys`` values,
    N(0,1) data.  With ``cover`` every key occurs in both relations (fully reduced)."""
    rng = np.random.default_rng(seed)
    draw = lambda g, c: g.integers(0, keys, size=c)
    if cover:
        ka = covering_keys(rng, rows, keys, draw)
        kb = covering_keys(rng, rows, keys, draw)
    else:
        ka, kb = draw(rng, rows), draw(rng, rows)
    S = Relation("S", (0,), ka[:, None], _normal(rng, rows, n_s))
    T = Relation("T", (0,), kb[:, None], _normal(rng, rows, n_t))
    return Database([S, T], [-1, 0], ["a"],
                    f"two-relation S(a;{n_s}) x T(a;{n_t}), {rows} rows each, a uniform over {keys}")


def path3(seed: int = 2, rows: int = 2_000_000, keys: int = 2000, s: float = 1.1,
          n_cols: int = 8, root: int = 0) -> Database:
    """Acyclic path join R1(a; x1..x8) - R2(a, b; y1..y8) - R3(b; z1..z8).

    a and b are i.i.d. Zipf(s) over ``keys`` values (independent inside R2), data
    N(0,1).  ``root`` picks the join-tree root among the three relations (R is the
    same for every join tree of the same join)."""
    rng = np.random.default_rng(seed)
    a1 = zipf_keys(rng, rows, keys, s)
    a2 = zipf_keys(rng, rows, keys, s)
    b2 = zipf_keys(rng, rows, keys, s)
    b3 = zipf_keys(rng, rows, keys, s)
    R1 = Relation("R1", (0,), a1[:, None], _normal(rng, rows, n_cols))
    R2 = Relation("R2", (0, 1), np.stack([a2, b2], axis=1), _normal(rng, rows, n_cols))
    R3 = Relation("R3", (1,), b3[:, None], _normal(rng, rows, n_cols))
    parents = {0: [-1, 0, 1], 1: [1, -1, 1], 2: [1, 2, -1]}[root]
    return Database([R1, R2, R3], parents, ["a", "b"],
                    f"path join R1(a)-R2(a,b)-R3(b), {rows} rows each, Zipf({s}) over {keys} keys, "
                    f"{n_cols} N(0,1) cols each, root R{root + 1}")


def star(seed: int = 3, fact_rows: int = 5_000_000, dim_rows: int = 50_000, keys: int = 10_000,
         n_cols: int = 16) -> Database:
    """Many-to-many star: dimension D1 (root) - Fact(k1, k2, k3) - {D2, D3}.

    Dimensions hold ``dim_rows`` rows over ``keys`` distinct keys (every key present);
    fact keys are uniform.  The fact data is drawn in FP32 and widened exactly to FP64."""
    rng = np.random.default_rng(seed)
    uni = lambda g, c: g.integers(0, keys, size=c)
    dk = [covering_keys(rng, dim_rows, keys, uni) for _ in range(3)]
    fk = [covering_keys(rng, fact_rows, keys, uni) for _ in range(3)]
    fdata = rng.standard_normal((fact_rows, n_cols), dtype=np.float32).astype(np.float64)
    D1 = Relation("D1", (0,), dk[0][:, None], _normal(rng, dim_rows, n_cols))
    F = Relation("F", (0, 1, 2), np.stack(fk, axis=1), fdata)
    D2 = Relation("D2", (1,), dk[1][:, None], _normal(rng, dim_rows, n_cols))
    D3 = Relation("D3", (2,), dk[2][:, None], _normal(rng, dim_rows, n_cols))
    return Database([D1, F, D2, D3], [-1, 0, 1, 1], ["k1", "k2", "k3"],
                    f"many-to-many star, fact {fact_rows} rows, dims {dim_rows} rows over {keys} keys")


def snowflake(seed: int = 4, f_rows: int = 10_000_000, d1_rows: int = 1_000_000,
              d2_rows: int = 1_000_000, d3_rows: int = 100_000, n_cols: int = 50,
              n_scaled: int = 10, scale: float = 1e4) -> Database:
    """Key-fkey snowflake D3(c) root - D1(a, c) - F(a, b) - D2(b).

    D1, D2, D3 have unique keys a, b, c; F.a, F.b, D1.c are uniform foreign keys with
    every key referenced at least once.  Data U[-1,1]; ``n_scaled`` of the columns
    (a seeded choice) are multiplied by ``scale``."""
    rng = np.random.default_rng(seed)
    fa = covering_keys(rng, f_rows, d1_rows, lambda g, c: g.integers(0, d1_rows, size=c))
    fb = covering_keys(rng, f_rows, d2_rows, lambda g, c: g.integers(0, d2_rows, size=c))
    d1c = covering_keys(rng, d1_rows, d3_rows, lambda g, c: g.integers(0, d3_rows, size=c))
    d1a = rng.permutation(d1_rows).astype(np.int64)
    d2b = rng.permutation(d2_rows).astype(np.int64)
    d3c = rng.permutation(d3_rows).astype(np.int64)
    u = lambda m: rng.uniform(-1.0, 1.0, size=(m, n_cols))
    D3 = Relation("D3", (2,), d3c[:, None], u(d3_rows))
    D1 = Relation("D1", (0, 2), np.stack([d1a, d1c], axis=1), u(d1_rows))
    F = Relation("F", (0, 1), np.stack([fa, fb], axis=1), u(f_rows))
    D2 = Relation("D2", (1,), d2b[:, None], u(d2_rows))
    rels = [D3, D1, F, D2]
    scaled = rng.choice(4 * n_cols, size=n_scaled, replace=False)
    for c in scaled:
        rels[c // n_cols].data[:, c % n_cols] *= scale
    return Database(rels, [-1, 0, 1, 2], ["a", "b", "c"],
                    f"snowflake D3-D1-F-D2, F {f_rows} rows, {n_cols} U[-1,1] cols each, "
                    f"{n_scaled} cols x{scale:g}")


def batch_instance(inst: int, seed: int = 5, lo: int = 1000, hi: int = 1_000_000,
                   n_lo: int = 8, n_hi: int = 64, s: float = 1.1) -> Database:
    """Instance ``inst`` of the batch of independent two-relation joins: log-uniform rows
    per side in [lo, hi], Zipf(s) keys over ceil(max(m_S, m_T)/100) values with every key
    present in both sides; n total data columns in U{n_lo..n_hi}, split floor(n/2) / rest.
    Each instance has its own seeded generator, so instances can be drawn one at a time."""
    rng = np.random.default_rng(seed * 100_003 + inst)
    mS = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    mT = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    n = int(rng.integers(n_lo, n_hi + 1))
    nS = n // 2
    dom = max(1, -(-max(mS, mT) // 100))
    dom = min(dom, mS, mT)
    draw = lambda g, c: zipf_keys(g, c, dom, s)
    kS = covering_keys(rng, mS, dom, draw)
    kT = covering_keys(rng, mT, dom, draw)
    S = Relation("S", (0,), kS[:, None], _normal(rng, mS, nS))
    T = Relation("T", (0,), kT[:, None], _normal(rng, mT, n - nS))
    return Database([S, T], [-1, 0], ["a"], f"batch instance {inst}")


def batch_instances(seed: int = 5, count: int = 256, lo: int = 1000, hi: int = 1_000_000,
                    n_lo: int = 8, n_hi: int = 64, s: float = 1.1):
    """The first ``count`` instances of the batch (see ``batch_instance``)."""
    return [batch_instance(i, seed, lo, hi, n_lo, n_hi, s) for i in range(count)]


def cartesian(seed: int = 6, m: int = 512, n: int = 64, m2: int = None, n2: int = None) -> Database:
    """Cartesian product S x T of two relations without join attributes, data U[-3,3)
    (the synthetic setting of the paper's Exp. 1)."""
    rng = np.random.default_rng(seed)
    m2 = m if m2 is None else m2
    n2 = n if n2 is None else n2
    S = Relation("S", (), np.zeros((m, 0), np.int64), rng.uniform(-3.0, 3.0, size=(m, n)))
    T = Relation("T", (), np.zeros((m2, 0), np.int64), rng.uniform(-3.0, 3.0, size=(m2, n2)))
    return Database([S, T], [-1, 0], [], f"Cartesian product {m}x{n} times {m2}x{n2}, U[-3,3)")


def four_relation(seed: int = 7, domain: int = 2, rows=(6, 9, 5, 4), n_cols=(2, 2, 1, 2)) -> Database:
    """The shape of the paper's §4 example: S1(a) root - S2(a, b, c) - {S3(b), S4(c)},
    keys drawn from a small domain with every key present where it is needed for the
    database to be fully reduced."""
    rng = np.random.default_rng(seed)
    dom = domain
    m1, m2, m3, m4 = rows
    # S2 holds every (a, b, c) combination once, then random extra rows.
    combos = np.array([(a, b, c) for a in range(dom) for b in range(dom) for c in range(dom)], np.int64)
    extra = rng.integers(0, dom, size=(max(0, m2 - len(combos)), 3))
    k2 = np.concatenate([combos, extra])[:max(m2, len(combos))]
    rng.shuffle(k2)
    k1 = covering_keys(rng, m1, dom, lambda g, c: g.integers(0, dom, size=c))
    k3 = covering_keys(rng, m3, dom, lambda g, c: g.integers(0, dom, size=c))
    k4 = covering_keys(rng, m4, dom, lambda g, c: g.integers(0, dom, size=c))
    S1 = Relation("S1", (0,), k1[:, None], _normal(rng, m1, n_cols[0]))
    S2 = Relation("S2", (0, 1, 2), k2, _normal(rng, len(k2), n_cols[1]))
    S3 = Relation("S3", (1,), k3[:, None], _normal(rng, m3, n_cols[2]))
    S4 = Relation("S4", (2,), k4[:, None], _normal(rng, m4, n_cols[3]))
    return Database([S1, S2, S3, S4], [-1, 0, 1, 1], ["a", "b", "c"],
                    "four-relation tree S1(a)-S2(a,b,c)-{S3(b),S4(c)}")


def random_tree_db(seed: int, n_rel: int = 4, rows_lo: int = 1, rows_hi: int = 12,
                   domain: int = 3, cols_hi: int = 3, dangling: bool = False) -> Database:
    """A random acyclic database for property tests: a random tree over ``n_rel``
    relations, one fresh join attribute per tree edge (a relation holds the attributes
    of its incident edges), keys uniform over ``domain``.  Unless ``dangling`` is set,
    tuples that do not join are allowed to exist only if they are later removed by the
    caller; this generator does not reduce the database itself."""
    rng = np.random.default_rng(seed)
    parent = [-1] + [int(rng.integers(0, i)) for i in range(1, n_rel)]
    edges = {i: i - 1 for i in range(1, n_rel)}        # child i uses attribute id i-1
    rels = []
    for i in range(n_rel):
        attrs = []
        if parent[i] >= 0:
            attrs.append(edges[i])
        attrs += [edges[c] for c in range(1, n_rel) if parent[c] == i]
        attrs = tuple(sorted(attrs))
        m = int(rng.integers(rows_lo, rows_hi + 1))
        keys = rng.integers(0, domain, size=(m, len(attrs))).astype(np.int64)
        if not dangling and len(attrs) > 0:
            # make every key value of every attribute present in this relation
            full = np.array(np.meshgrid(*[np.arange(domain)] * len(attrs), indexing="ij")).reshape(len(attrs), -1).T
            keys = np.concatenate([full, keys]).astype(np.int64)
            m = keys.shape[0]
        n = int(rng.integers(1, cols_hi + 1))
        rels.append(Relation(f"S{i + 1}", attrs, keys, _normal(rng, m, n)))
    return Database(rels, parent, [f"e{i}" for i in range(n_rel - 1)], f"random tree seed {seed}")


def app_a_cartesian(seed: int = 8, m1: int = 16, n1: int = 4, m2: int = 16, n2: int = 4,
                    int_range: int = 5):
    """The paper's Appendix A accuracy construction (a Cartesian product whose R has a
    known top-left block).

    Draws a rational unit vector v (v_1 != -1), an upper-triangular integer R_S with
    positive diagonal and an m2 x n2 matrix T of natural numbers (m2 a perfect square).
    Q_S is the first n1 columns of the rational orthogonal matrix
        Qhat = [[v_1, v_2 .. v_m1], [v_2..v_m1, v_i v_j / (v_1 + 1) - delta_ij]]
    (its first row ends with v_m1: the matrix is m1 x m1), and S = Q_S R_S is formed in
    exact rational arithmetic and rounded once to float64.  By the appendix's corollary
    the R of S x T has top-left block R_S * sqrt(m2).

    v is the first column of the reflection I - 2 w w^T / (w^T w) for an integer w,
    v_i = delta_i1 - 2 w_1 w_i / |w|^2, which is a rational unit vector.

    Returns (Database, R_fixed) with R_fixed = R_S * sqrt(m2) as float64.
    """
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    r = int(round(np.sqrt(m2)))
    assert r * r == m2, "m2 must be a perfect square"
    assert n1 <= m1
    while True:
        w = [int(x) for x in rng.integers(-3, 4, size=m1)]
        w[0] = int(rng.integers(1, 4))
        ww = sum(x * x for x in w)
        v = [Fraction((ww if i == 0 else 0) - 2 * w[0] * w[i], ww) for i in range(m1)]
        if v[0] != -1:
            break
    R_S = [[0] * n1 for _ in range(n1)]
    for i in range(n1):
        R_S[i][i] = int(rng.integers(1, int_range + 1))
        for j in range(i + 1, n1):
            R_S[i][j] = int(rng.integers(-int_range, int_range + 1))
    T = rng.integers(0, int_range + 1, size=(m2, n2)).astype(np.float64)
    d = v[0] + 1

    def qhat(i, j):
        if i == 0:
            return v[j]
        if j == 0:
            return v[i]
        return v[i] * v[j] / d - (1 if i == j else 0)

    S = np.empty((m1, n1))
    for i in range(m1):
        row = [qhat(i, k) for k in range(n1)]
        for j in range(n1):
            S[i, j] = float(sum(row[k] * R_S[k][j] for k in range(j + 1)))
    R_fixed = np.array(R_S, dtype=np.float64) * float(r)
    rel_S = Relation("S", (), np.zeros((m1, 0), np.int64), S)
    rel_T = Relation("T", (), np.zeros((m2, 0), np.int64), T)
    db = Database([rel_S, rel_T], [-1, 0], [], f"Appendix A construction m1={m1} n1={n1} m2={m2} n2={n2}")
    return db, R_fixed


CONFIGS = {
    "two_relation_1k": lambda **kw: two_relation(seed=1, **kw),
    "path3_2m": lambda **kw: path3(seed=2, **kw),
    "star_5m": lambda **kw: star(seed=3, **kw),
    "snowflake_10m": lambda **kw: snowflake(seed=4, **kw),
}


def presorted(db: Database) -> Database:
    """A copy of ``db`` whose relations are stored in join-key order, the paper's input
    convention (§5 assumes S_i sorted on X_i, a child first on the attributes it shares
    with its parent; §9 times pre-sorted inputs): the attributes shared with the parent
    first, then the relation's other key attributes, each part by ascending attribute id,
    values ascending, ties in input order."""
    rels = []
    for i, r in enumerate(db.relations):
        p = db.parent[i]
        shared = sorted(set(r.key_attrs) & set(db.relations[p].key_attrs)) if p >= 0 else []
        rest = sorted(set(r.key_attrs) - set(shared))
        cols = [r.key_attrs.index(a) for a in shared + rest]
        if cols:
            order = np.lexsort(tuple(r.keys[:, c] for c in reversed(cols)))   # stable
        else:
            order = np.arange(r.n_rows)
        rels.append(Relation(r.name, r.key_attrs, np.ascontiguousarray(r.keys[order]),
                             np.ascontiguousarray(r.data[order])))
    return Database(rels, list(db.parent), list(db.attr_names), db.description + " (pre-sorted)")


def fingerprint(db: Database, stride: int = 9973) -> str:
    """A short hash of a database's keys and data (every ``stride``-th row of every
    relation, plus the shapes): it ties a stored expected value to the inputs it was
    computed from, so that a changed generator is noticed instead of compared against."""
    import hashlib
    h = hashlib.sha256()
    h.update(repr(list(db.parent)).encode())
    for r in db.relations:
        h.update(repr((r.name, tuple(r.key_attrs), r.keys.shape, r.data.shape)).encode())
        h.update(np.ascontiguousarray(r.keys[::stride]).tobytes())
        h.update(np.ascontiguousarray(r.data[::stride]).tobytes())
    return h.hexdigest()[:16]
