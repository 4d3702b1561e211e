"""Thin ctypes binding of include/figaro.h (argument marshalling only).

The functions carry the C names; every computation runs in the CUDA library.  If the
library is not built, ``load()`` raises: there is no CPU fallback.

``JoinPlan`` is a convenience wrapper for torch tensors: it keeps the tensors the plan
reads alive, passes their device pointers and the current torch stream, and allocates
outputs.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build_lib

FIGARO_OK = 0
FIGARO_ERR_INVALID_ARG = 1
FIGARO_ERR_OVERFLOW, FIGARO_ERR_NOMEM, FIGARO_ERR_TIMEOUT = 4, 5, 6
FIGARO_ERR_UNSUPPORTED = 10
FIGARO_KEY_I64, FIGARO_KEY_I32 = 0, 1
FIGARO_COL_MAJOR, FIGARO_ROW_MAJOR = 0, 1
FIGARO_PREC_FP64, FIGARO_PREC_MIXED, FIGARO_PREC_MIXED_REFINED = 0, 1, 2
FIGARO_PROJ_X, FIGARO_PROJ_Q, FIGARO_PROJ_U, FIGARO_PROJ_SCORES = 0, 1, 2, 3
FIGARO_LEAF_HOUSEHOLDER, FIGARO_LEAF_GIVENS, FIGARO_LEAF_TCGEN05, FIGARO_LEAF_MMA_SYNC = 0, 1, 2, 3
FIGARO_MEM_DEVICE, FIGARO_MEM_HOST = 0, 1
DBG = {"sizes": 0, "perm": 1, "group_off": 2, "counts": 3, "pcounts": 4, "tails": 5, "heads": 6,
       "gen_tails": 7, "data": 8, "root_rows": 9}
STAGES = ["sort", "segment", "counts", "heads_tails", "join_project", "tsqr_leaf", "tsqr_tree", "svd"]


class figaro_relation(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_keys", C.c_int32), ("key_type", C.c_int32),
                ("key_attr", C.POINTER(C.c_int32)), ("key_cols", C.POINTER(C.c_void_p)),
                ("n_data", C.c_int32), ("layout", C.c_int32), ("ld", C.c_int64),
                ("data", C.c_void_p)]


class figaro_join_tree(C.Structure):
    _fields_ = [("n_rel", C.c_int32), ("rels", C.POINTER(figaro_relation)),
                ("parent", C.POINTER(C.c_int32))]


class figaro_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("presorted", C.c_int32), ("require_reduced", C.c_int32),
                ("mem", C.c_int32), ("stage_timing", C.c_int32), ("gradients", C.c_int32),
                ("leaf", C.c_int32), ("workspace_limit_mib", C.c_int32), ("svd_max_sweeps", C.c_int32),
                ("fuse_tails", C.c_int32), ("autotune", C.c_int32), ("reserved", C.c_int32 * 5)]


class figaro_plan_info(C.Structure):
    _fields_ = [("n_rel", C.c_int32), ("n_cols", C.c_int32), ("input_cells", C.c_int64),
                ("input_bytes", C.c_int64), ("workspace_bytes", C.c_int64), ("r0_rows", C.c_int64),
                ("launches", C.c_int64), ("tsqr_leaf_flops", C.c_double), ("refined", C.c_int32),
                ("reserved", C.c_int32)]


class FigaroError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_LIB = None


def load(build_if_missing: bool = False):
    """The loaded library.  Raises if it is not built (or builds it on request)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not build_lib.is_current():
        if not build_if_missing:
            raise RuntimeError("libfigaro.so is not built for this machine: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        build_lib.build()
    lib = C.CDLL(build_lib.LIB)
    P = C.c_void_p
    sig = {
        "figaro_default_options": (None, [C.POINTER(figaro_options)]),
        "figaro_plan": (C.c_int, [C.POINTER(figaro_join_tree), C.POINTER(figaro_options), P, C.POINTER(P)]),
        "figaro_qr_r": (C.c_int, [P, P, C.c_int64]),
        "figaro_svd": (C.c_int, [P, P, P, P]),
        "figaro_pca": (C.c_int, [P, C.c_int32, P, P]),
        "figaro_plan_destroy": (C.c_int, [P]),
        "figaro_plan_get_info": (C.c_int, [P, C.POINTER(figaro_plan_info)]),
        "figaro_stage_times": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
        "figaro_reset_stage_times": (C.c_int, [P]),
        "figaro_block_times": (C.c_int, [P, C.c_int32, P, P, P]),
        "figaro_debug_read": (C.c_int64, [P, C.c_int32, C.c_int32, P, C.c_int64]),
        "figaro_svd_from_r_static": (C.c_int, [P, C.c_int64, C.c_int32, P, P, P]),
        "figaro_backward": (C.c_int, [P, P, C.c_int64, P, C.c_int64, P, P]),
        "figaro_pca_centered": (C.c_int, [P, C.c_int32, P, P]),
        "figaro_qr_r_async": (C.c_int, [P, P, C.c_int64]),
        "figaro_plan_sync": (C.c_int, [P]),
        "figaro_join_size": (C.c_int, [P, C.POINTER(C.c_uint64)]),
        "figaro_project": (C.c_int, [P, C.c_int32, P, C.c_int64, P, C.c_int64, C.c_int32, P, C.c_int64, C.c_int64,
                                     C.POINTER(C.c_int64)]),
        "figaro_batch_create": (C.c_int, [C.c_int32, P, P, P, P, P, C.POINTER(P)]),
        "figaro_batch_run": (C.c_int, [P, P]),
        "figaro_batch_launches": (C.c_int64, [P]),
        "figaro_batch_destroy": (C.c_int, [P]),
        "figaro_fp64_fma_rate": (C.c_int, [C.POINTER(C.c_double), P]),
        "figaro_error_string": (C.c_char_p, [C.c_int]),
        "figaro_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def check(status):
    if status != FIGARO_OK:
        lib = load()
        raise FigaroError(status, f"{lib.figaro_error_string(status).decode()}: "
                                  f"{lib.figaro_last_error().decode()}")
    return status


# ----------------------------------------------------------------------------- C names

def figaro_default_options():
    o = figaro_options()
    load().figaro_default_options(C.byref(o))
    return o


def figaro_plan(tree: figaro_join_tree, opt: figaro_options, stream: int):
    h = C.c_void_p()
    check(load().figaro_plan(C.byref(tree), C.byref(opt), C.c_void_p(stream), C.byref(h)))
    return h


def figaro_qr_r(plan, R_ptr: int, ldr: int):
    return check(load().figaro_qr_r(plan, C.c_void_p(R_ptr), ldr))


def figaro_svd(plan, sigma_ptr: int, V_ptr: int, R_ptr: int = 0):
    return check(load().figaro_svd(plan, C.c_void_p(sigma_ptr), C.c_void_p(V_ptr), C.c_void_p(R_ptr or None)))


def figaro_pca(plan, k: int, comp_ptr: int, eig_ptr: int):
    return check(load().figaro_pca(plan, k, C.c_void_p(comp_ptr), C.c_void_p(eig_ptr)))


def figaro_fp64_fma_rate(stream: int) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s."""
    v = C.c_double()
    check(load().figaro_fp64_fma_rate(C.byref(v), C.c_void_p(stream)))
    return v.value


def figaro_svd_from_r_static(R_ptr: int, ldr: int, n: int, sigma_ptr: int, V_ptr: int, stream: int):
    return check(load().figaro_svd_from_r_static(C.c_void_p(R_ptr), ldr, n, C.c_void_p(sigma_ptr),
                                                 C.c_void_p(V_ptr), C.c_void_p(stream)))


def figaro_backward(plan, R_ptr: int, ldr: int, Rbar_ptr: int, ldb: int, grad_ptrs, ldgs):
    n = len(grad_ptrs)
    ptrs = (C.c_void_p * max(n, 1))(*[C.c_void_p(p) if p else None for p in grad_ptrs])
    lds = (C.c_int64 * max(n, 1))(*ldgs)
    return check(load().figaro_backward(plan, C.c_void_p(R_ptr), ldr, C.c_void_p(Rbar_ptr), ldb,
                                        C.cast(ptrs, C.c_void_p), C.cast(lds, C.c_void_p)))


def figaro_plan_destroy(plan):
    return check(load().figaro_plan_destroy(plan))


def figaro_plan_get_info(plan) -> dict:
    info = figaro_plan_info()
    check(load().figaro_plan_get_info(plan, C.byref(info)))
    return {k: getattr(info, k) for k, _ in figaro_plan_info._fields_}


def figaro_stage_times(plan):
    ms = (C.c_double * 8)()
    cnt = (C.c_int64 * 8)()
    load().figaro_stage_times(plan, ms, cnt, 8)
    return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}


def figaro_block_times(plan):
    """[(leaf_ms, n_cols, rows)] per R0 block (see the header)."""
    lib = load()
    nb = lib.figaro_block_times(plan, 0, None, None, None)
    if nb < 0:
        check(-nb)
    ms, nc, rows = (C.c_double * max(nb, 1))(), (C.c_int32 * max(nb, 1))(), (C.c_int64 * max(nb, 1))()
    lib.figaro_block_times(plan, nb, C.cast(ms, C.c_void_p), C.cast(nc, C.c_void_p), C.cast(rows, C.c_void_p))
    return [(ms[i], nc[i], rows[i]) for i in range(nb)]


def figaro_reset_stage_times(plan):
    return check(load().figaro_reset_stage_times(plan))


def figaro_debug_read(plan, rel: int, what: str, dtype):
    """Copy an intermediate array to a new numpy array of ``dtype``."""
    import numpy as np
    lib = load()
    n = lib.figaro_debug_read(plan, rel, DBG[what], None, 0)
    if n < 0:
        raise FigaroError(-n, "figaro_debug_read failed")
    out = np.empty(n // np.dtype(dtype).itemsize, dtype=dtype)
    if n:
        lib.figaro_debug_read(plan, rel, DBG[what], out.ctypes.data_as(C.c_void_p), n)
    return out


# ----------------------------------------------------------------------------- torch helper

class JoinPlan:
    """A plan over torch tensors.

    relations: list of dicts with ``keys`` (list of 1-D int64/int32 tensors), ``key_attrs``
    (list of ints) and ``data`` (2-D float64 tensor, row- or column-major, may have 0
    columns).  Tensors must live on the current CUDA device (or on the host, pinned for
    asynchronous copies, with ``mem=FIGARO_MEM_HOST``)."""

    def __init__(self, relations, parent, precision=FIGARO_PREC_FP64, presorted=False,
                 require_reduced=False, mem=FIGARO_MEM_DEVICE, stage_timing=False, stream=None,
                 gradients=False, leaf=FIGARO_LEAF_HOUSEHOLDER, workspace_limit_mib=0, svd_max_sweeps=0,
                 fuse_tails=False, autotune=False):
        import torch
        self._keep = []
        self._data = []
        n = len(relations)
        rels = (figaro_relation * n)()
        self._arrays = []
        for i, r in enumerate(relations):
            keys = [k.contiguous() for k in r["keys"]]
            data = r["data"]
            if data.dim() != 2 or data.dtype != torch.float64:
                raise ValueError("data must be a 2-D float64 tensor")
            m, nd = data.shape
            if nd > 0 and data.stride(0) == 1 and (nd == 1 or data.stride(1) >= m):
                layout, ld = FIGARO_COL_MAJOR, (data.stride(1) if nd > 1 else m)
            else:
                data = data.contiguous()
                layout, ld = FIGARO_ROW_MAJOR, max(nd, 1)
            kt = FIGARO_KEY_I32 if (keys and keys[0].dtype == torch.int32) else FIGARO_KEY_I64
            attrs = (C.c_int32 * max(len(keys), 1))(*r["key_attrs"])
            cols = (C.c_void_p * max(len(keys), 1))(*[k.data_ptr() for k in keys])
            self._arrays += [attrs, cols]
            self._keep += keys + [data]
            self._data.append(data)
            rels[i] = figaro_relation(m, len(keys), kt, attrs, cols, nd, layout, ld,
                                      data.data_ptr() if nd > 0 else None)
        par = (C.c_int32 * n)(*parent)
        self._arrays += [rels, par]
        tree = figaro_join_tree(n, rels, par)
        opt = figaro_default_options()
        opt.precision = precision
        opt.presorted = int(presorted)
        opt.require_reduced = int(require_reduced)
        opt.mem = mem
        opt.stage_timing = int(stage_timing)
        opt.gradients = int(gradients)
        opt.leaf = int(leaf)
        opt.workspace_limit_mib = int(workspace_limit_mib)
        opt.svd_max_sweeps = int(svd_max_sweeps)
        opt.fuse_tails = int(fuse_tails)
        opt.autotune = int(autotune)
        self.mem = mem
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = figaro_plan(tree, opt, self.stream.cuda_stream)
        self.n_cols = figaro_plan_get_info(self.handle)["n_cols"]

    def _out(self, *shape):
        import torch
        if self.mem == FIGARO_MEM_HOST:
            return torch.empty(*shape, dtype=torch.float64).pin_memory()
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    def qr_r(self, out=None):
        R = self._out(self.n_cols, self.n_cols) if out is None else out
        figaro_qr_r(self.handle, R.data_ptr(), R.stride(0))
        return R

    def qr_r_async(self, out):
        """Enqueue a figaro_qr_r into `out` and return at once (see figaro_plan_sync)."""
        check(load().figaro_qr_r_async(self.handle, C.c_void_p(out.data_ptr()), out.stride(0)))
        return out

    def sync(self):
        check(load().figaro_plan_sync(self.handle))

    def svd(self, with_r=False):
        N = self.n_cols
        s, V = self._out(N), self._out(N, N)
        R = self._out(N, N) if with_r else None
        figaro_svd(self.handle, s.data_ptr(), V.data_ptr(), R.data_ptr() if with_r else 0)
        return (s, V, R) if with_r else (s, V)

    def pca(self, k):
        comp, ev = self._out(self.n_cols, k), self._out(k)
        figaro_pca(self.handle, k, comp.data_ptr(), ev.data_ptr())
        return comp, ev

    def join_size(self):
        n = C.c_uint64()
        check(load().figaro_join_size(self.handle, C.byref(n)))
        return int(n.value)

    def project(self, R, mode=FIGARO_PROJ_Q, X=None, k=None, max_rows=1 << 27):
        """A X for the last call's data (see figaro_project): Q (mode FIGARO_PROJ_Q), the
        first k columns of U, the top-k PCA scores, or A X for a given X (N x k)."""
        import torch
        N = self.n_cols
        if mode == FIGARO_PROJ_Q:
            k = N
        elif mode == FIGARO_PROJ_X:
            X = X.to(device=R.device, dtype=torch.float64).contiguous()
            k = X.shape[1]
        rows = self.join_size()
        if rows > max_rows:
            raise FigaroError(FIGARO_ERR_UNSUPPORTED, f"the join has {rows} rows (max_rows {max_rows})")
        out = torch.empty(max(rows, 1), k, dtype=torch.float64, device=R.device)
        n = C.c_int64()
        check(load().figaro_project(self.handle, mode, C.c_void_p(R.data_ptr()), R.stride(0),
                                    C.c_void_p(X.data_ptr()) if X is not None else None, k if X is None else X.stride(0),
                                    k, C.c_void_p(out.data_ptr()), k, max_rows, C.byref(n)))
        return out[:rows]

    def pca_centered(self, k):
        comp, ev = self._out(self.n_cols, k), self._out(k)
        check(load().figaro_pca_centered(self.handle, k, C.c_void_p(comp.data_ptr()), C.c_void_p(ev.data_ptr())))
        return comp, ev

    def backward(self, R, Rbar):
        """Gradients of a loss with dL/dR = Rbar at the last call's data: one
        column-major (M_i, N_i) float64 tensor per relation (None without data columns)."""
        import torch
        R = R.contiguous()
        Rbar = Rbar.to(device=R.device, dtype=torch.float64).contiguous()
        grads, ptrs, lds = [], [], []
        for d in self._data:
            m, nd = d.shape
            if nd == 0:
                grads.append(None)
                ptrs.append(0)
                lds.append(max(m, 1))
                continue
            g = torch.empty(nd, m, dtype=torch.float64, device=R.device).t()   # column-major
            grads.append(g)
            ptrs.append(g.data_ptr())
            lds.append(max(m, 1))
        figaro_backward(self.handle, R.data_ptr(), R.stride(0), Rbar.data_ptr(), Rbar.stride(0), ptrs, lds)
        return grads

    def info(self):
        return figaro_plan_get_info(self.handle)

    def stage_times(self):
        return figaro_stage_times(self.handle)

    def block_times(self):
        return figaro_block_times(self.handle)

    def reset_stage_times(self):
        figaro_reset_stage_times(self.handle)

    def debug(self, rel, what, dtype):
        return figaro_debug_read(self.handle, rel, what, dtype)

    def close(self):
        if getattr(self, "handle", None) is not None:
            figaro_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_from_db(db, device="cuda", precision=FIGARO_PREC_FP64, col_major=True, **kw):
    """A JoinPlan over a ``synth.Database`` copied to ``device`` (``"cpu"`` pins host
    memory and selects FIGARO_MEM_HOST)."""
    import torch
    host = device == "cpu"
    rels = []
    for r in db.relations:
        keys = [torch.from_numpy(r.keys[:, k].copy()) for k in range(r.keys.shape[1])]
        data = torch.from_numpy(r.data)
        if col_major:
            data = data.t().contiguous().t()
        if host:
            keys = [k.pin_memory() for k in keys]
            data = data.pin_memory() if data.numel() else data
        else:
            keys = [k.to(device) for k in keys]
            data = data.to(device)
            if col_major and data.shape[1] > 1 and data.stride(0) != 1:
                data = data.t().contiguous().t()
        rels.append({"keys": keys, "key_attrs": list(r.key_attrs), "data": data})
    return JoinPlan(rels, list(db.parent), precision=precision,
                    mem=FIGARO_MEM_HOST if host else FIGARO_MEM_DEVICE, **kw)


class FigaroR:
    """R of the join as a differentiable function of the relations' data tensors.

    ``FigaroR(plan)(*datas)`` runs figaro_qr_r (the plan must have been made over exactly
    these tensors, with gradients=True) and returns R; its backward calls figaro_backward
    with the incoming dL/dR."""

    def __init__(self, plan):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, *datas):
                R = plan.qr_r()
                ctx.save_for_backward(R)
                return R

            @staticmethod
            def backward(ctx, Rbar):
                (R,) = ctx.saved_tensors
                grads = plan.backward(R, Rbar)
                return tuple(grads)

        self._fn = _Fn
        self.plan = plan

    def __call__(self, *datas):
        return self._fn.apply(*datas)


class Batch:
    """Many JoinPlans run as one CUDA graph (figaro_batch_*): R of every instance, and the
    top-k principal components where k[i] > 0."""

    def __init__(self, plans, k=None):
        import torch
        lib = load()
        n = len(plans)
        self.plans = plans
        self.R = [torch.empty(p.n_cols, p.n_cols, dtype=torch.float64, device="cuda") for p in plans]
        self.k = [0] * n if k is None else [int(x) for x in k]
        self.comps = [torch.empty(p.n_cols, max(ki, 1), dtype=torch.float64, device="cuda")
                      for p, ki in zip(plans, self.k)]
        self.eig = [torch.empty(max(ki, 1), dtype=torch.float64, device="cuda") for ki in self.k]
        arr = lambda xs: (C.c_void_p * n)(*[x for x in xs])
        self._arrays = [arr([p.handle for p in plans]), arr([t.data_ptr() for t in self.R]),
                        arr([t.data_ptr() for t in self.comps]), arr([t.data_ptr() for t in self.eig]),
                        (C.c_int32 * n)(*self.k)]
        h = C.c_void_p()
        check(lib.figaro_batch_create(n, C.cast(self._arrays[0], C.c_void_p), C.cast(self._arrays[1], C.c_void_p),
                                      C.cast(self._arrays[2], C.c_void_p), C.cast(self._arrays[3], C.c_void_p),
                                      C.cast(self._arrays[4], C.c_void_p), C.byref(h)))
        self.handle = h

    def run(self):
        """Launch every instance and wait; returns the per-instance status list."""
        n = len(self.plans)
        st = (C.c_int32 * n)()
        rc = load().figaro_batch_run(self.handle, C.cast(st, C.c_void_p))
        self.status = list(st)
        check(rc)
        return self.status

    def launches(self):
        return int(load().figaro_batch_launches(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None:
            load().figaro_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

