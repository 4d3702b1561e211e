"""CPU FiGaRo in C with OpenMP (figaro_cpu.c): the paper's method on the host cores.

TEST INFRASTRUCTURE AND CPU BASELINE ONLY (see ``oracle/__init__.py``).  It serves as the
timed CPU baseline of the benchmark: the paper's own system is multicore C++ (§9
"Experimental Setup"), and this is Alg. 3, Alg. 4 (with Alg. 2) and the §7
post-processing written in C, with OpenMP over relations, groups and row tiles.  Its R is
pinned against the Python oracle (``oracle.figaro.figaro_r``) and the paper's closed forms
by ``tests/test_oracle_cfigaro.py``.

``build()`` compiles the library with gcc (``-O3 -fopenmp``, no fast-math) into
``_build/`` beside this file; ``figaro_r(db)`` runs it on a ``synth.Database``.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import platform
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "figaro_cpu.c")
HDR = os.path.join(HERE, "figaro_cpu.h")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcfigaro.so")
CFLAGS = ["-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall"]

STATUS = {0: "ok", 1: "invalid input", 2: "not fully reduced", 3: "count overflow", 4: "out of host memory",
          5: "not sorted"}


class CFigaroError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"cfig_figaro_r: {STATUS.get(status, status)}")
        self.status = status


class cfig_relation(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_keys", C.c_int32), ("key_attr", C.POINTER(C.c_int32)),
                ("keys", C.POINTER(C.c_void_p)), ("n_data", C.c_int32), ("data", C.c_void_p),
                ("ld", C.c_int64)]


def _stamp() -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(CFLAGS).encode())
    for p in (SRC, HDR):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile figaro_cpu.c into _build/libcfigaro.so (skipped when current)."""
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == _stamp():
                return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler found for the CPU FiGaRo baseline")
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp"
    r = subprocess.run([cc] + CFLAGS + [SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gcc failed on figaro_cpu.c:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(_stamp())
    return LIB


_LIB = None


def load():
    global _LIB
    if _LIB is None:
        lib = C.CDLL(build())
        lib.cfig_figaro_r.restype = C.c_int
        lib.cfig_figaro_r.argtypes = [C.c_int32, C.POINTER(cfig_relation), C.POINTER(C.c_int32), C.c_int32,
                                      C.c_int32, C.c_void_p, C.c_void_p]
        lib.cfig_max_threads.restype = C.c_int
        lib.cfig_max_threads.argtypes = []
        _LIB = lib
    return _LIB


def max_threads() -> int:
    return int(load().cfig_max_threads())


class Prepared:
    """A database marshalled once for repeated runs (the timed region then covers the C
    call only): column-major data copies, key arrays and the relation table."""

    def __init__(self, db):
        n = len(db.relations)
        self.n, self.N = n, db.n_cols
        self.rels = (cfig_relation * n)()
        self._keep = []
        for i, r in enumerate(db.relations):
            keys = [np.ascontiguousarray(r.keys[:, k], dtype=np.int64) for k in range(r.keys.shape[1])]
            data = np.asfortranarray(r.data, dtype=np.float64)
            attrs = (C.c_int32 * max(len(keys), 1))(*r.key_attrs)
            kp = (C.c_void_p * max(len(keys), 1))(*[k.ctypes.data for k in keys])
            self._keep += [keys, data, attrs, kp]
            self.rels[i] = cfig_relation(r.n_rows, len(keys), attrs, kp, r.n_data,
                                         data.ctypes.data if r.n_data else None, max(r.n_rows, 1))
        self.parent = (C.c_int32 * n)(*db.parent)

    def run(self, threads: int = 0, presorted: bool = False):
        """(R, seconds): see ``figaro_r``."""
        R = np.zeros((self.N, self.N))
        sec = np.zeros(4)
        st = load().cfig_figaro_r(self.n, self.rels, self.parent, int(presorted), int(threads), R.ctypes.data,
                                  sec.ctypes.data)
        if st != 0:
            raise CFigaroError(st)
        return R, sec


def figaro_r(db, threads: int = 0, presorted: bool = False):
    """(R, seconds) of a ``synth.Database``: R (n_cols x n_cols, non-negative diagonal) and
    the wall seconds of [sort + grouping, Alg. 3, Alg. 4, post-processing]."""
    return Prepared(db).run(threads, presorted)
