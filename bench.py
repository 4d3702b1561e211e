#!/usr/bin/env python
"""Benchmark: input cells per second to R for the 4-relation snowflake join
D3(c) 100k rows - D1(a, c) 1M - F(a, b) 10M - D2(b) 1M, 50 U[-1,1] float64 columns each
(200 in all, 10 of them x 1e4), key-fkey with every key referenced; the join has 10M
rows x 200 columns and is never materialised.  One step = sort, segment, count (Alg. 3),
heads/tails and joins (Alg. 4), TSQR (§7) -> R, on inputs already resident in HBM.  This
is the largest single-GPU workload of the benchmark set (628 M input cells, 5 GB).

Also measured on it: the mixed-precision path against the FP64 path (whole step and TSQR
alone), R^T R errors against the oracle's factorized A^T A (stored in tests/golden), the
same steps on pre-sorted inputs (the paper's timing convention), end-to-end throughput
through the C ABI with host buffers, stage times with their rooflines, the dominant
kernel's roofline against a live FP64 rate measurement, the gradient of ||R||_F^2, the
CPU FiGaRo baseline (C with OpenMP on all host cores) on the same workload, and the
2M-row path join as a second workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl figaro|reference]
Under torchrun every rank runs an independent instance (weak scaling; the path has no
data exchange) and rank 0 prints one JSON line.

Other workloads (one JSON line each, not the benchmark line): --batch-instances K (the
batch of independent two-relation joins as one graph launch) and --wide (the star and
snowflake joins, one call at a time).  --plan-only runs one plan on a chosen workload
without output, for ncu captures.
"""
import os

for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

import synth

METRIC = "input cells/sec to R (GB/s vs HBM peak); mixed vs FP64 speedup at rel err ≤1e-6"
WORKLOAD = ("snowflake_10m: D3(c) 100k - D1(a,c) 1M - F(a,b) 10M - D2(b) 1M rows, 50 U[-1,1] float64 "
            "cols each (200; 10 cols x1e4), key-fkey, every key referenced; join 10M rows x 200 cols")
PATH3 = ("path3_2m: R1(a;x1..x8) - R2(a,b;y1..y8) - R3(b;z1..z8), 2,000,000 rows each, "
         "a,b Zipf(1.1) over 2,000 keys, N(0,1) float64 data; join ~1.5e16 rows")
FP64_PEAK_DERIVED = 152 * 2070e6 * 4 / 1e12   # 152 SMs x 2.07 GHz x 2 DFMA/clk/SM x 2 flop
REF_SAMPLE = 4                                # the reference arm's rows: the workload's / 4
GOLDEN_GRAM = os.path.join(ROOT, "tests", "golden", "snowflake_gram.npz")
# DRAM bytes per row of the dominant kernel (k_tsqr_fold<double>, leaf of the 100-column
# generalized-tail block): (dram__bytes_read.sum + dram__bytes_write.sum) / rows of the ncu
# capture of the same kernel on the snowflake with a fifth of the rows, summarised in
# profiles/tsqr_fold_f64_snowflake.md; the traffic grows with the rows.
DOMINANT_DRAM_BYTES_PER_ROW = (1.443330e9 + 9.190912e6) / 1_799_944


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock samples (every 100 ms) over the measured region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.2)
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
        return False

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def make_inputs(db, torch, device):
    rels = []
    for r in db.relations:
        keys = [torch.from_numpy(np.ascontiguousarray(r.keys[:, k])) for k in range(r.keys.shape[1])]
        data = torch.from_numpy(np.asfortranarray(r.data))
        data = torch.as_strided(data, r.data.shape, (1, r.data.shape[0]))
        if device == "cpu":
            keys = [k.pin_memory() for k in keys]
            pinned = torch.empty_strided(r.data.shape, (1, r.data.shape[0]), dtype=torch.float64).pin_memory()
            pinned.copy_(data)
            data = pinned
        else:
            keys = [k.to(device) for k in keys]
            dd = torch.empty_strided(r.data.shape, (1, r.data.shape[0]), dtype=torch.float64, device=device)
            dd.copy_(data)
            data = dd
        rels.append({"keys": keys, "key_attrs": list(r.key_attrs), "data": data})
    return rels


def time_steps(plan, torch, steps, warmup, barrier):
    """W untimed steps, then exactly K steps between CUDA events on the plan's stream."""
    for _ in range(warmup):
        plan.qr_r(out=plan._R)
    plan.reset_stage_times()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(plan.stream)
    for _ in range(steps):
        plan.qr_r(out=plan._R)
    e1.record(plan.stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps


def time_steps_pipelined(plans, torch, steps, warmup, barrier):
    """Throughput with two calls in flight: the plans (each on its own stream) alternate
    figaro_qr_r_async / figaro_plan_sync; a plan is synced before it is reused, so every
    step is one complete pass.  CUDA events on a third stream that waits for both."""
    for i in range(max(warmup, 2)):
        plans[i % 2].qr_r_async(plans[i % 2]._R)
        plans[i % 2].sync()
    barrier()
    torch.cuda.synchronize()
    ts = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ts)
    for p in plans:
        p.stream.wait_event(e0)
    for i in range(steps):
        p = plans[i % 2]
        if i >= 2:
            p.sync()
        p.qr_r_async(p._R)
    for p in plans:
        ev = torch.cuda.Event()
        ev.record(p.stream)
        ts.wait_event(ev)
    e1.record(ts)
    for p in plans:
        p.sync()
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps


def run_plan_only(args):
    """--plan-only: W + K calls of one plan on the benchmark workload and nothing else
    (no JSON line): a short, deterministic launch sequence for ncu captures."""
    import torch
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = wide_workload(args.workload) if args.workload != "path3" else synth.path3(seed=2, rows=args.rows)
    dev_inputs = make_inputs(db, torch, "cuda")
    prec = binding.FIGARO_PREC_MIXED if args.plan_only.startswith("mixed") else binding.FIGARO_PREC_FP64
    p = binding.JoinPlan(dev_inputs, db.parent, precision=prec, stage_timing=args.plan_only.endswith("staged"),
                         stream=torch.cuda.current_stream(), fuse_tails=args.fuse_tails,
                         autotune=args.autotune)
    p._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    ms = time_steps(p, torch, args.steps, args.warmup, lambda: None)
    p.close()
    log(f"{args.plan_only}: {ms:.3f} ms per step")


# FiGaRo-MKL seconds for R on the Cartesian product S x T (paper's Exp. 1 grid, its own
# 24-core Xeon Silver 4214 machine): rows per relation -> {columns per relation: seconds}
PAPER_CARTESIAN_S = {512: {64: 0.10, 256: 0.13}, 1024: {64: 0.10, 256: 0.13}, 2048: {64: 0.12, 256: 0.15},
                     4096: {64: 0.12, 256: 0.14}, 8192: {64: 0.13, 256: 0.18}}


def run_cartesian(args):
    """--cartesian: R of the Cartesian product S x T with U[-3,3) data over the paper's
    Exp. 1 grid (2^9..2^13 rows and 2^6, 2^8 columns per relation; 2^10 and 2^12 columns
    per relation exceed this library's 1024 columns of R), FP64 and mixed, one call at a
    time with CUDA events, beside the paper's FiGaRo-MKL times on its own CPU machine
    (context, not a target: other hardware).  Prints one JSON line."""
    import torch
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    stream = torch.cuda.current_stream()
    rows = []
    for m in sorted(PAPER_CARTESIAN_S):
        for n in (64, 256):
            db = synth.cartesian(seed=6, m=m, n=n)
            dev = make_inputs(db, torch, "cuda")
            rec = {"rows_per_relation": m, "cols_per_relation": n, "join_rows": m * m,
                   "paper_figaro_mkl_s": PAPER_CARTESIAN_S[m][n]}
            for tag, prec in (("fp64", binding.FIGARO_PREC_FP64), ("mixed", binding.FIGARO_PREC_MIXED)):
                p = one_plan(binding, torch, dev, db.parent, stream, precision=prec)
                rec[tag + "_ms"] = time_steps(p, torch, args.steps, args.warmup, lambda: None)
                p.close()
            rec["paper_over_fp64"] = rec["paper_figaro_mkl_s"] * 1e3 / rec["fp64_ms"]
            rows.append(rec)
            del dev
    print(json.dumps({"metric": "time to R, Cartesian product S x T (paper Exp. 1 grid)", "unit": "ms",
                      "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic U[-3,3) (seeded)", "paper_hardware": "Xeon Silver 4214, 24 cores, MKL",
                      "grid": rows}), flush=True)


def wide_workload(name):
    """The wide-block workloads: the 5M-row many-to-many star (16 columns per relation,
    a 48-column generalized-tail block of ~5M rows) and the 10M-row snowflake (50 columns per
    relation, 10 of the 200 scaled by 1e4; 100-, 150- and 200-column blocks)."""
    if name == "snowflake-small":    # a fifth of the rows: small ncu captures of the same kernels
        return synth.snowflake(f_rows=2_000_000, d1_rows=200_000, d2_rows=200_000, d3_rows=20_000)
    return synth.star() if name == "star" else synth.snowflake()


def run_wide(args):
    """--wide: R of the star and snowflake workloads (blocks wider than 32 columns, reduced
    by the streamed fold), FP64 and mixed, one call at a time (CUDA events), with the
    dominant block's leaf time from a stage-timed plan.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    out = []
    for name in ("star", "snowflake"):
        db = wide_workload(name)
        dev_inputs = make_inputs(db, torch, "cuda")
        cells = db.input_cells()
        row = {"workload": db.description, "input_cells": cells}
        Rs = {}
        for tag, prec in (("fp64", binding.FIGARO_PREC_FP64), ("mixed", binding.FIGARO_PREC_MIXED)):
            p = binding.JoinPlan(dev_inputs, db.parent, precision=prec, stream=torch.cuda.current_stream())
            p._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
            ms = time_steps(p, torch, args.steps, args.warmup, lambda: None)
            Rs[tag] = p.qr_r().cpu().numpy()
            p.close()
            ps = binding.JoinPlan(dev_inputs, db.parent, precision=prec, stage_timing=True,
                                  stream=torch.cuda.current_stream())
            ps.qr_r()
            ps.reset_stage_times()
            ps.qr_r()
            blocks = ps.block_times()
            ps.close()
            leaf_ms, n_cols, rows = max(blocks)
            flops = 2.0 * rows * n_cols * n_cols
            row[tag] = {"ms_per_step": ms, "cells_per_s": cells / (ms * 1e-3),
                        "dominant_block": {"n_cols": n_cols, "rows": rows, "leaf_ms": leaf_ms,
                                           "leaf_tflops": flops / (leaf_ms * 1e-3) / 1e12}}
        G = Rs["fp64"].T @ Rs["fp64"]
        row["mixed"]["rel_err_RtR_vs_fp64"] = float(np.linalg.norm(Rs["mixed"].T @ Rs["mixed"] - G) /
                                                    np.linalg.norm(G))
        row["mixed"]["speedup_vs_fp64"] = row["fp64"]["ms_per_step"] / row["mixed"]["ms_per_step"]
        out.append(row)
        del dev_inputs
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "wide-block workloads: time to R, one call at a time", "unit": "ms",
                      "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic (seeded)", "fp64_peak_tflops_derived": FP64_PEAK_DERIVED,
                      "leaf_flops": "2 rows n^2 per block (Householder on the block's rows)",
                      "workloads": out}), flush=True)


def run_batch(args):
    """--batch-instances K: the first K instances of the 256-instance batch workload
    (two-relation joins, 1k-1M rows per side, 8-64 columns): R and the top-min(10, n)
    principal components of every instance, as one graph launch (figaro_batch_run)
    against the same plans called one after another.  Prints one JSON line."""
    import torch
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    t0 = time.time()
    dbs = [synth.batch_instance(i) for i in range(args.batch_instances)]
    cells = sum(db.input_cells() for db in dbs)
    t1 = time.time()
    plans = [binding.plan_from_db(db, autotune=args.autotune) for db in dbs]
    plan_s = time.time() - t1
    ks = [min(10, db.n_cols) for db in dbs]
    log(f"batch: {len(dbs)} instances, {cells / 1e6:.1f}M cells, setup {time.time() - t0:.1f}s")
    for _ in range(args.warmup):                      # one call each: graphs captured
        for p, k in zip(plans, ks):
            p.pca(k)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        for p, k in zip(plans, ks):
            p.qr_r()
            p.pca(k)
    loop_ms = (time.perf_counter() - t) * 1e3 / args.steps
    bt = binding.Batch(plans, k=ks)
    for _ in range(args.warmup):
        bt.run()
    t = time.perf_counter()
    for _ in range(args.steps):
        bt.run()
    batch_ms = (time.perf_counter() - t) * 1e3 / args.steps
    out = {"metric": "batched instances: R and top-10 PCA of every instance", "impl": "figaro-batch",
           "value": len(dbs) / (batch_ms * 1e-3), "unit": "instances/s", "ms_per_batch": batch_ms,
           "cells_per_s": cells / (batch_ms * 1e-3), "loop_ms": loop_ms, "speedup_vs_loop": loop_ms / batch_ms,
           "launches_per_batch": bt.launches(), "instances": len(dbs), "input_cells": cells,
           "autotune": bool(args.autotune), "plans_s": plan_s,
           "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic (seeded)",
           "timing": "host clock around figaro_batch_run (launch + wait) / around the loop of "
                     "figaro_qr_r + figaro_pca calls (each waits)"}
    bt.close()
    for p in plans:
        p.close()
    print(json.dumps(out), flush=True)


def rank_context(torch, device_type="cuda"):
    """(rank, world size, barrier, max over ranks) of the process group that torchrun's
    environment describes: NCCL on GPUs, gloo on the CPU; a world of one needs no group.
    Replicas exchange nothing but these two timing collectives."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return rank, 1, (lambda: None), (lambda x: x)
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device(f"cuda:{local}") if device_type == "cuda" else torch.device("cpu")
    if not dist.is_initialized():
        if device_type == "cuda":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group("gloo")

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return rank, world, (lambda: dist.barrier()), max_over_ranks


def gram_errors(R, G):
    """||R^T R - G||_F / ||G||_F, plain and with rows and columns scaled by 1/sqrt(G_jj)
    (the 1e4 columns dominate the plain norm)."""
    E = R.T @ R - G
    d = np.sqrt(np.maximum(np.diag(G), 1e-300))
    Es, Gs = E / d[:, None] / d[None, :], G / d[:, None] / d[None, :]
    return float(np.linalg.norm(E) / np.linalg.norm(G)), float(np.linalg.norm(Es) / np.linalg.norm(Gs))


def load_golden_gram(db):
    """The oracle's A^T A of the snowflake workload, if it was computed from these inputs."""
    try:
        z = np.load(GOLDEN_GRAM)
    except OSError:
        return None, "tests/golden/snowflake_gram.npz missing"
    if str(z["fingerprint"]) != synth.fingerprint(db):
        return None, "stored oracle Gram belongs to other inputs (generator changed)"
    return z["gram"], "oracle factorized A^T A (tests/golden/snowflake_gram.npz)"


def stage_rooflines(plan, stages, db, hbm, fp64_peak, mixed):
    """Per-stage algorithmic bytes (HBM-bound stages) or flops (TSQR) over the stage's
    time in a stage-timed plan.  Bytes count what the stage must move at least: sort reads
    the keys and writes a permutation; heads/tails read the data and write tails and heads;
    joins read the joined Data and write generalized tails and heads."""
    esz_t = 4 if mixed else 8
    sz = []
    for i, r in enumerate(db.relations):
        v = plan.debug(i, "sizes", "int64")
        sz.append({"M": int(v[0]), "G": int(v[1]), "P": int(v[2]), "K": int(v[6]), "N": r.n_data,
                   "N_sub": int(v[7]), "gen": int(v[4]), "root": int(v[5])})
    b_sort = sum(s["M"] * (8 * s["K"] + 4) for s in sz)
    b_seg = sum(s["M"] * 8 + s["G"] * 4 for s in sz)
    b_ht = sum(s["M"] * s["N"] * 8 + (s["M"] - s["G"]) * s["N"] * esz_t + s["G"] * s["N"] * 8 for s in sz)
    b_join = sum((s["G"] * s["N_sub"] * 8 + s["gen"] * s["N_sub"] * esz_t + s["P"] * s["N_sub"] * 8)
                 for s in sz if s["gen"] > 0 or s["root"] > 0)
    out = {}
    for name, b in (("sort", b_sort), ("segment", b_seg), ("heads_tails", b_ht), ("join_project", b_join)):
        ms = stages[name]
        out[name] = {"ms": ms, "algorithmic_bytes": b, "gbs": b / (ms * 1e-3) / 1e9 if ms > 0 else None,
                     "bound": "hbm", "frac": (b / (ms * 1e-3) / 1e9) / hbm if ms > 0 else None}
    info = plan.info()
    ms = stages["tsqr_tree"]
    fl = info["tsqr_leaf_flops"]
    out["tsqr"] = {"ms": ms, "algorithmic_flops": fl, "tflops": fl / (ms * 1e-3) / 1e12,
                   "bound": "fp32 pipe / tensor" if mixed else "fp64 pipe",
                   "frac_of_measured_fp64": None if mixed else fl / (ms * 1e-3) / 1e12 / fp64_peak,
                   "note": "leaf flops sum_b 2 rows_b n_b^2 - 2/3 n_b^3 over the whole TSQR section (leaf + tree + final QR)"}
    out["counts"] = {"ms": stages["counts"], "bound": "latency (per-group kernels over <= 10M groups)"}
    return out, sz


def plan_pair(binding, torch, inputs, parent, **kw):
    ps = []
    for _ in range(2):
        p = binding.JoinPlan(inputs, parent, stream=torch.cuda.Stream(), **kw)
        p._R = torch.empty(p.n_cols, p.n_cols, dtype=torch.float64, device="cuda")
        ps.append(p)
    return ps


def one_plan(binding, torch, inputs, parent, stream, **kw):
    p = binding.JoinPlan(inputs, parent, stream=stream, **kw)
    p._R = torch.empty(p.n_cols, p.n_cols, dtype=torch.float64, device="cuda")
    return p


def staged_run(binding, torch, inputs, parent, stream, steps, warmup, barrier, **kw):
    """Stage times (ms per call), block leaf times and the plan of a stage-timed run."""
    p = one_plan(binding, torch, inputs, parent, stream, stage_timing=True, **kw)
    ms = time_steps(p, torch, steps, warmup, barrier)
    st = {k: v[0] / steps for k, v in p.stage_times().items()}
    blocks = [(a / steps, n, r) for a, n, r in p.block_times()]
    return p, ms, st, blocks


def time_spectral(plan, torch, steps, warmup, stream, G_ref):
    """figaro_svd (R and its Jacobi SVD) and figaro_pca (k = 10) per call with CUDA events on
    the plan's stream; sigma against the square roots of the oracle's factorized A^T A."""
    out = {}
    for name, call in (("svd", lambda: plan.svd()), ("pca_k10", lambda: plan.pca(10))):
        for _ in range(max(1, warmup)):
            res = call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            res = call()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms_per_call"] = e0.elapsed_time(e1) / steps
        if name == "svd":
            sig = res[0].cpu().numpy()
    if G_ref is not None:
        lam = np.sort(np.linalg.eigvalsh(G_ref))[::-1]
        ref = np.sqrt(np.maximum(lam, 0.0))
        out["sigma_max_rel_err_vs_oracle_gram"] = float(np.max(np.abs(sig - ref)) / ref[0])
        out["sigma_ref"] = "square roots of the eigenvalues of the stored oracle A^T A (tests/golden)"
    out["includes"] = "R (as figaro_qr_r) and the Jacobi SVD of R; FP64"
    return out


def run_figaro(args):
    import torch
    from paper_2204_00525_gb300 import binding

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank, world, barrier, max_over_ranks = rank_context(torch, "cuda")
    torch.cuda.set_device(local)
    binding.load(build_if_missing=True)
    K, W = args.steps, args.warmup
    K2 = max(3, min(K, 5))          # secondary measurements (stages, pre-sorted, refined, backward)

    t0 = time.time()
    db = synth.snowflake(seed=4 + rank)
    dbs = synth.presorted(db)
    cells, in_bytes = db.input_cells(), db.input_bytes()
    log(f"[rank {rank}] generated {cells / 1e6:.1f}M cells (+ pre-sorted copy) in {time.time() - t0:.1f}s")
    G_ref, g_src = load_golden_gram(db) if rank == 0 else (None, "rank > 0")
    dev = make_inputs(db, torch, "cuda")
    stream = torch.cuda.current_stream()
    fp64_rate = binding.figaro_fp64_fma_rate(stream.cuda_stream)
    hbm, hbm_kind = peaks()

    # --- FP64 path (the headline): throughput with two calls in flight, latency of one call
    pair = plan_pair(binding, torch, dev, db.parent)
    with ClockSampler(local) as clk:
        ms64 = time_steps_pipelined(pair, torch, K, W, barrier)
    clocks = clk.summary()
    ms64 = max_over_ranks(ms64)
    assert torch.equal(pair[0]._R, pair[1]._R)
    for p in pair:
        p.close()
    p64 = one_plan(binding, torch, dev, db.parent, stream)
    lat64 = max_over_ranks(time_steps(p64, torch, K, W, barrier))
    info = p64.info()
    R64 = p64._R.cpu().numpy()
    svd_rec = time_spectral(p64, torch, K2, W, stream, G_ref)
    p64.close()
    pst, ms_st64, st64, blk64 = staged_run(binding, torch, dev, db.parent, stream, K2, W, barrier)
    roof64, sizes = stage_rooflines(pst, st64, db, hbm, fp64_rate, False)
    pst.close()

    # --- mixed path
    mpair = plan_pair(binding, torch, dev, db.parent, precision=binding.FIGARO_PREC_MIXED)
    msmx_tp = max_over_ranks(time_steps_pipelined(mpair, torch, K, W, barrier))
    for p in mpair:
        p.close()
    pmx = one_plan(binding, torch, dev, db.parent, stream, precision=binding.FIGARO_PREC_MIXED)
    latmx = max_over_ranks(time_steps(pmx, torch, K, W, barrier))
    Rmx = pmx._R.cpu().numpy()
    pmx.close()
    pms, ms_stmx, stmx, blkmx = staged_run(binding, torch, dev, db.parent, stream, K2, W, barrier,
                                           precision=binding.FIGARO_PREC_MIXED)
    roofmx, _ = stage_rooflines(pms, stmx, db, hbm, fp64_rate, True)
    pms.close()
    pmr = one_plan(binding, torch, dev, db.parent, stream, precision=binding.FIGARO_PREC_MIXED_REFINED)
    latmr = max_over_ranks(time_steps(pmr, torch, K2, W, barrier))
    Rmr = pmr._R.cpu().numpy()
    refined = int(pmr.info()["refined"])
    pmr.close()

    # --- pre-sorted inputs (the paper's convention: sorting excluded)
    del dev
    torch.cuda.empty_cache()
    devs = make_inputs(dbs, torch, "cuda")
    pps = plan_pair(binding, torch, devs, dbs.parent, presorted=True)
    ms64_ps = max_over_ranks(time_steps_pipelined(pps, torch, K2, W, barrier))
    R64_ps = pps[0]._R.cpu().numpy()
    for p in pps:
        p.close()
    ppm = plan_pair(binding, torch, devs, dbs.parent, presorted=True, precision=binding.FIGARO_PREC_MIXED)
    msmx_ps = max_over_ranks(time_steps_pipelined(ppm, torch, K2, W, barrier))
    for p in ppm:
        p.close()
    # stage rooflines without the sort and its permutation gathers (the paper's convention)
    roof_ps = {}
    for tag, prec in (("fp64", binding.FIGARO_PREC_FP64), ("mixed", binding.FIGARO_PREC_MIXED)):
        pps_st, _, st_ps, _ = staged_run(binding, torch, devs, dbs.parent, stream, K2, W, barrier,
                                         presorted=True, precision=prec)
        roof_ps[tag], _ = stage_rooflines(pps_st, st_ps, dbs, hbm, fp64_rate, prec != binding.FIGARO_PREC_FP64)
        pps_st.close()

    # --- gradient of ||R||_F^2 with respect to all data columns (figaro_backward)
    pg = binding.JoinPlan(devs, dbs.parent, presorted=True, gradients=True, stream=stream)
    Rg = pg.qr_r()
    Rbar = 2.0 * Rg
    for _ in range(W):
        pg.backward(Rg, Rbar)
    torch.cuda.synchronize()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    for _ in range(K2):
        grads = pg.backward(Rg, Rbar)
    eb1.record(stream)
    torch.cuda.synchronize()
    bwd_ms = max_over_ranks(eb0.elapsed_time(eb1) / K2)
    pg.close()
    del grads, devs
    torch.cuda.empty_cache()

    # --- end to end through the C ABI with pinned host buffers: every step copies all
    # keys and data in and R out; two plans on two streams alternate so that one step's
    # copies overlap the other's computation
    host = make_inputs(db, torch, "cpu")
    ph = binding.JoinPlan(host, db.parent, mem=binding.FIGARO_MEM_HOST, stream=stream)
    Rh = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64).pin_memory()
    for _ in range(W):
        ph.qr_r(out=Rh)
    barrier()
    t = time.perf_counter()
    for _ in range(K2):
        ph.qr_r(out=Rh)
    e2e_seq_ms = max_over_ranks((time.perf_counter() - t) * 1e3 / K2)
    ph.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pp = [binding.JoinPlan(host, db.parent, mem=binding.FIGARO_MEM_HOST, stream=s) for s in streams]
    Rp = [torch.empty(db.n_cols, db.n_cols, dtype=torch.float64).pin_memory() for _ in pp]
    for i in range(max(W, 2)):
        pp[i % 2].qr_r_async(Rp[i % 2])
        pp[i % 2].sync()
    barrier()
    t = time.perf_counter()
    for i in range(K):
        p_i = pp[i % 2]
        if i >= 2:
            p_i.sync()
        p_i.qr_r_async(Rp[i % 2])
    for p_i in pp:
        p_i.sync()
    e2e_ms = max_over_ranks((time.perf_counter() - t) * 1e3 / K)
    assert np.array_equal(Rp[0].numpy(), Rp[1].numpy())
    for p_i in pp:
        p_i.close()
    del host
    torch.cuda.empty_cache()

    # --- the 2M-row path join (second workload): FP64 throughput, mixed latency
    p3 = path3_numbers(binding, torch, rank, K, W, barrier, max_over_ranks, world)

    # --- errors against the oracle's A^T A (or the FP64 path where it is missing)
    G = G_ref if G_ref is not None else R64.T @ R64
    e64 = gram_errors(R64, G) if G_ref is not None else (None, None)
    emx, emr, e64ps = gram_errors(Rmx, G), gram_errors(Rmr, G), gram_errors(R64_ps, G)

    # --- the dominant kernel: the FP64 fold leaf of the 100-column generalized-tail block
    leaf_ms, n_dom, rows_dom = max(blk64)
    dom_flops = 2.0 * rows_dom * n_dom * n_dom - 2.0 / 3.0 * n_dom ** 3
    dom_tflops = dom_flops / (leaf_ms * 1e-3) / 1e12
    roofline = {"kernel": f"k_tsqr_fold<double> leaf of the {n_dom}-column block ({rows_dom} rows): streamed "
                          "Householder fold, FP64", "bound": "alu", "achieved": dom_tflops,
                "peak": fp64_rate, "unit": "TFLOP/s", "frac": dom_tflops / fp64_rate,
                "traffic": (DOMINANT_DRAM_BYTES_PER_ROW * rows_dom if DOMINANT_DRAM_BYTES_PER_ROW else None),
                "peak_kind": "measured in this run: FP64 FMA loop (figaro_fp64_fma_rate), burst",
                "frac_of_derived_peak": dom_tflops / FP64_PEAK_DERIVED,
                "derived_peak": FP64_PEAK_DERIVED, "flops_per_launch": dom_flops, "rows_per_launch": rows_dom,
                "ms_per_launch": leaf_ms, "launches_per_step": 1,
                "algorithmic_bytes_per_launch": rows_dom * n_dom * 8,
                "timing": "CUDA events around the launch on its stream in the stage-timed plan"}
    tsqr64, tsqrmx = st64["tsqr_tree"], stmx["tsqr_tree"]
    value = cells * world / (ms64 * 1e-3)
    gbs = in_bytes * world / (ms64 * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "throughput_mode": "two calls in flight (two plans, two streams, figaro_qr_r_async / figaro_plan_sync)",
        "latency_ms_per_step": lat64, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded snowflake generator, see config)",
        "config": {"workload": WORKLOAD, "rows": [r.n_rows for r in db.relations],
                   "cols": db.n_cols, "input_cells_per_gpu": cells, "input_bytes_per_gpu": in_bytes,
                   "l2": "inputs exceed L2 (5.0 GB > 129 MB); no flush", "sort": "included (pre-sorted below)",
                   "parallelism": f"replicas x{world} (independent instances)"},
        "gbs": gbs, "hbm_frac": gbs / hbm, "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind,
        "errors_vs": g_src,
        "rel_err_RtR": e64[0], "rel_err_RtR_col_scaled": e64[1],
        "presorted": {"ms_per_step": ms64_ps, "value": cells * world / (ms64_ps * 1e-3),
                      "mixed_ms_per_step": msmx_ps, "mixed_value": cells * world / (msmx_ps * 1e-3),
                      "rel_err_RtR": e64ps[0], "mode": "inputs stored in join-key order, figaro_options.presorted "
                                                       "= 1 (order verified, sort skipped); two calls in flight",
                      "stage_rooflines": roof_ps},
        "mixed": {"ms_per_step": msmx_tp, "value": cells * world / (msmx_tp * 1e-3),
                  "speedup_vs_fp64": ms64 / msmx_tp, "basis": "throughput, two calls in flight, vs ms_per_step",
                  "latency_ms_per_step": latmx, "latency_speedup_vs_fp64": lat64 / latmx,
                  "tsqr_ms": tsqrmx, "tsqr_ms_fp64": tsqr64, "tsqr_speedup_vs_fp64": tsqr64 / tsqrmx,
                  "tsqr_basis": "a5+a6 (TSQR section) of the stage-timed plans",
                  "rel_err_RtR": emx[0], "rel_err_RtR_col_scaled": emx[1],
                  "stages_ms": stmx, "stage_rooflines": roofmx,
                  "refined": {"ms_per_step": latmr, "speedup_vs_fp64": lat64 / latmr, "applied": refined,
                              "rel_err_RtR": emr[0], "rel_err_RtR_col_scaled": emr[1]},
                  "dtype": "double-float head/tail sums, f32 tails and TSQR (split-tf32 tensor-core trailing "
                           "updates on wide blocks), f64 counts, joins, final QR"},
        "stages_ms": st64, "stage_rooflines": roof64,
        "stage_note": "stage-timed plans (CUDA events around every stage, TSQR chains serialised); "
                      "tsqr_tree is the whole TSQR section, tsqr_leaf its leaf launches",
        "blocks": [{"n": n, "rows": r, "leaf_ms": m} for m, n, r in blk64 if r > 0],
        "r0_rows": info["r0_rows"],
        "roofline": roofline,
        "spectral": svd_rec,
        "backward": {"ms_per_call": bwd_ms, "loss": "||R||_F^2", "value": cells * world / (bwd_ms * 1e-3),
                     "unit": "cells/s", "note": "figaro_backward after a forward call (pre-sorted plan)"},
        "e2e": {"value": cells * world / (e2e_ms * 1e-3), "unit": "cells/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": db.n_cols * db.n_cols * 8 + 4,
                "mode": "two plans on two streams alternating figaro_qr_r_async / figaro_plan_sync",
                "sequential_ms_per_step": e2e_seq_ms},
        "path3_2m": p3,
        "gpu_launches": int(info["launches"]) * K,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(db, dbs)
    if world > 1:
        import torch.distributed as dist
        barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def path3_numbers(binding, torch, rank, K, W, barrier, max_over_ranks, world):
    db = synth.path3(seed=2 + rank)
    dev = make_inputs(db, torch, "cuda")
    pair = plan_pair(binding, torch, dev, db.parent)
    ms = max_over_ranks(time_steps_pipelined(pair, torch, K, W, barrier))
    R = pair[0]._R.cpu().numpy()
    for p in pair:
        p.close()
    pm = one_plan(binding, torch, dev, db.parent, torch.cuda.current_stream(), precision=binding.FIGARO_PREC_MIXED)
    msm = max_over_ranks(time_steps(pm, torch, K, W, barrier))
    Rm = pm._R.cpu().numpy()
    pm.close()
    del dev
    torch.cuda.empty_cache()
    cells = db.input_cells()
    G = R.T @ R
    return {"workload": PATH3, "input_cells": cells, "ms_per_step": ms, "value": cells * world / (ms * 1e-3),
            "unit": "cells/s", "mixed_latency_ms": msm,
            "mixed_rel_err_RtR_vs_fp64_path": float(np.linalg.norm(Rm.T @ Rm - G) / np.linalg.norm(G))}


def host_threads():
    """All host cores this process may run on (the CPU baseline's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2"}


def cpu_facts():
    model = platform_model()
    return {"nproc": os.cpu_count(), "cpu": model}


def platform_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                for key in ("model name", "Model", "CPU part"):
                    if line.startswith(key):
                        v = line.split(":", 1)[1].strip()
                        return f"{ARM_PARTS[v]} (CPU part {v})" if v in ARM_PARTS else v
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(db, dbs):
    """The CPU FiGaRo baseline (oracle/cfigaro: C with OpenMP, all host cores) on the same
    workload: one run with the sort, one on the pre-sorted copy."""
    from oracle import cfigaro
    prep, preps = cfigaro.Prepared(db), cfigaro.Prepared(dbs)
    threads = host_threads()
    t = time.perf_counter()
    _, sec = prep.run(threads=threads)
    dt = time.perf_counter() - t
    t = time.perf_counter()
    _, secs = preps.run(threads=threads, presorted=True)
    dts = time.perf_counter() - t
    cells = db.input_cells()
    return {"value": cells / dt, "unit": "cells/s", "cores": threads,
            "kind": "oracle: CPU FiGaRo (Alg. 3, Alg. 4, Householder post-processing) in C with OpenMP",
            "sample": f"the full workload ({cells} cells), one run: {dt:.2f} s with sort, "
                      f"{dts:.2f} s pre-sorted; stage seconds [sort, counts, heads/tails+joins, QR] = "
                      f"{[round(float(x), 3) for x in sec]}",
            "presorted_value": cells / dts, "same_config": True, **cpu_facts()}


def run_reference(args):
    """--impl reference: the CPU FiGaRo baseline (there is no reference implementation to
    install: the paper's code is not provided) on the host cores, each step one run on a
    row sample (1/--ref-divisor, a quarter by default) of the snowflake workload (same
    schema, key law and columns)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cfigaro
    div = max(1, args.ref_divisor)
    db = synth.snowflake(f_rows=10_000_000 // div, d1_rows=1_000_000 // div, d2_rows=1_000_000 // div,
                         d3_rows=max(100_000 // div, 1))
    cells = db.input_cells()
    prep = cfigaro.Prepared(db)
    threads = host_threads()
    for _ in range(args.warmup):
        prep.run(threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        prep.run(threads=threads)
    dt = (time.perf_counter() - t) / args.steps
    value = cells / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "rows": [r.n_rows for r in db.relations],
                   "note": f"CPU FiGaRo baseline on a 1/{div} row sample of the same workload"},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": threads,
                         "kind": "oracle: CPU FiGaRo in C with OpenMP",
                         "sample": f"snowflake with 1/{div} of the rows ({cells} cells), sort included",
                         **cpu_facts()},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="figaro", choices=["figaro", "reference"])
    ap.add_argument("--rows", type=int, default=2_000_000, help="rows per relation of --workload path3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-divisor", type=int, default=REF_SAMPLE,
                    help="--impl reference: rows of the workload divided by this")
    ap.add_argument("--plan-only", choices=["fp64", "mixed", "fp64-staged", "mixed-staged"],
                    help="profiling aid: run one plan only and print no JSON line")
    ap.add_argument("--autotune", action="store_true",
                    help="--plan-only / --batch-instances: TSQR plans picked by the autotuner (options.autotune)")
    ap.add_argument("--fuse-tails", action="store_true",
                    help="--plan-only: tails of relations with <= 32 columns formed inside the TSQR leaf")
    ap.add_argument("--workload", choices=["path3", "star", "snowflake", "snowflake-small"], default="snowflake",
                    help="workload of --plan-only")
    ap.add_argument("--wide", action="store_true",
                    help="measure the wide-block workloads (star, snowflake) instead")
    ap.add_argument("--cartesian", action="store_true",
                    help="measure the Cartesian-product grid of the paper's first experiment instead")
    ap.add_argument("--batch-instances", type=int, default=0,
                    help="measure the batched-instances workload (first K of 256) instead")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    if args.plan_only:
        run_plan_only(args)
    elif args.batch_instances:
        run_batch(args)
    elif args.wide:
        run_wide(args)
    elif args.cartesian:
        run_cartesian(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_figaro(args)


if __name__ == "__main__":
    main()
