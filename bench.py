#!/usr/bin/env python
"""Benchmark: input cells per second to R for the acyclic path join
R1(a; 8 cols) - R2(a, b; 8 cols) - R3(b; 8 cols), 2M rows per relation, a and b
Zipf(1.1) over 2,000 keys, N(0,1) float64 data (the join has ~1.5e16 rows and is never
materialised).  One step = sort, segment, count (Alg. 3), heads/tails (Alg. 4), TSQR (§7)
-> R, on inputs already resident in HBM.

Also measured: the mixed-precision path (float32 TSQR leaves) against the FP64 path,
end-to-end throughput through the C ABI with host buffers, the dominant kernel's
roofline, and the CPU oracle on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl figaro|reference]
Under torchrun every rank runs an independent instance (weak scaling; the path has no
data exchange) and rank 0 prints one JSON line.

Other workloads (one JSON line each, not the benchmark line): --batch-instances K (the
batch of independent two-relation joins as one graph launch) and --wide (the star and
snowflake joins, whose blocks of 33-256 columns go through the streamed fold).
--plan-only runs one plan on a chosen workload without output, for ncu captures.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
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
WORKLOAD = ("path3_2m: R1(a;x1..x8) - R2(a,b;y1..y8) - R3(b;z1..z8), 2,000,000 rows each, "
            "a,b Zipf(1.1) over 2,000 keys, N(0,1) float64 data, column-major; join ~1.5e16 rows")
ROWS = 2_000_000
SAMPLE_ROWS = 100_000          # oracle sample per relation (same shape and key distribution)
FP64_PEAK_TFLOPS = 152 * 2070e6 * 4 / 1e12   # 152 SMs x 2.07 GHz x 2 DFMA/clk/SM x 2 flop
# DRAM bytes per input row of the dominant kernel (k_tsqr_reg<double, 8>, leaf of a tails
# block), from the ncu capture summarised in profiles/tsqr_reg8_fp64_path3_2m.md:
# (dram__bytes_read.sum + dram__bytes_write.sum) / rows = 132.37 MB / 1,998,000 rows.
DOMINANT_DRAM_BYTES_PER_ROW = 132.37e6 / 1_998_000


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
                         stream=torch.cuda.current_stream())
    p._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    ms = time_steps(p, torch, args.steps, args.warmup, lambda: None)
    p.close()
    log(f"{args.plan_only}: {ms:.3f} ms per step")


def wide_workload(name):
    """The wide-block workloads: the 5M-row many-to-many star (16 columns per relation,
    a 48-column generalized-tail block of ~5M rows) and the 10M-row snowflake (50 columns per
    relation, 10 of the 200 scaled by 1e4; 100-, 150- and 200-column blocks)."""
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
                      "data": "synthetic (seeded)", "fp64_peak_tflops_derived": FP64_PEAK_TFLOPS,
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
    plans = [binding.plan_from_db(db) for db in dbs]
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


def run_figaro(args):
    import torch
    from paper_2204_00525_gb300 import binding

    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank, world, barrier, max_over_ranks = rank_context(torch, "cuda")
    torch.cuda.set_device(local)
    binding.load(build_if_missing=True)

    t0 = time.time()
    db = synth.path3(seed=2 + rank, rows=args.rows)
    cells = db.input_cells()
    in_bytes = db.input_bytes()
    log(f"[rank {rank}] generated {cells / 1e6:.1f}M cells in {time.time() - t0:.1f}s")
    dev_inputs = make_inputs(db, torch, "cuda")
    stream = torch.cuda.current_stream()

    # --- FP64 path (the headline): production plans, kernels as a user gets them.
    # Throughput: two calls in flight (two plans on two streams); latency: one plan alone.
    pair = []
    for _ in range(2):
        p = binding.JoinPlan(dev_inputs, db.parent, stream=torch.cuda.Stream())
        p._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
        pair.append(p)
    with ClockSampler(local) as clk:
        ms64 = time_steps_pipelined(pair, torch, args.steps, args.warmup, barrier)
    clocks = clk.summary()
    ms64 = max_over_ranks(ms64)
    assert torch.equal(pair[0]._R, pair[1]._R)
    for p in pair:
        p.close()
    p64 = binding.JoinPlan(dev_inputs, db.parent, stream=stream)
    p64._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    lat64 = max_over_ranks(time_steps(p64, torch, args.steps, args.warmup, barrier))
    info = p64.info()
    R64 = p64._R.cpu().numpy()
    p64.close()

    # --- stage breakdown and the leaf roofline: a second plan with CUDA events around
    # every stage (its TSQR chains run serialised so that kernel times are not shared)
    pst = binding.JoinPlan(dev_inputs, db.parent, stage_timing=True, stream=stream)
    pst._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    ms_staged = time_steps(pst, torch, args.steps, args.warmup, barrier)
    stages = pst.stage_times()
    block_times = pst.block_times()
    pst.close()

    # --- mixed path
    mx_pair = []
    for _ in range(2):
        p = binding.JoinPlan(dev_inputs, db.parent, precision=binding.FIGARO_PREC_MIXED, stream=torch.cuda.Stream())
        p._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
        mx_pair.append(p)
    msmx_tp = max_over_ranks(time_steps_pipelined(mx_pair, torch, args.steps, args.warmup, barrier))
    for p in mx_pair:
        p.close()
    pmx = binding.JoinPlan(dev_inputs, db.parent, precision=binding.FIGARO_PREC_MIXED, stream=stream)
    pmx._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    msmx = max_over_ranks(time_steps(pmx, torch, args.steps, args.warmup, barrier))
    Rmx = pmx._R.cpu().numpy()
    G64 = R64.T @ R64
    err_mx = float(np.linalg.norm(Rmx.T @ Rmx - G64) / np.linalg.norm(G64))
    pmx.close()
    pmxs = binding.JoinPlan(dev_inputs, db.parent, precision=binding.FIGARO_PREC_MIXED, stage_timing=True,
                            stream=stream)
    pmxs._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    time_steps(pmxs, torch, args.steps, args.warmup, barrier)
    mx_stages = {k: v[0] / args.steps for k, v in pmxs.stage_times().items()}
    pmxs.close()

    # --- mixed path with the CholeskyQR2-style refinement
    pmr = binding.JoinPlan(dev_inputs, db.parent, precision=binding.FIGARO_PREC_MIXED_REFINED, stream=stream)
    pmr._R = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64, device="cuda")
    msmr = max_over_ranks(time_steps(pmr, torch, args.steps, args.warmup, barrier))
    Rmr = pmr._R.cpu().numpy()
    refined = int(pmr.info()["refined"])
    pmr.close()
    err_mr = float(np.linalg.norm(Rmr.T @ Rmr - G64) / np.linalg.norm(G64))
    err_mr_r = float(np.linalg.norm(Rmr - R64) / np.linalg.norm(R64))

    # --- gradient of ||R||_F^2 with respect to all data columns (figaro_backward)
    pg = binding.JoinPlan(dev_inputs, db.parent, gradients=True, stream=stream)
    Rg = pg.qr_r()
    Rbar = 2.0 * Rg
    for _ in range(args.warmup):
        pg.backward(Rg, Rbar)
    torch.cuda.synchronize()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    for _ in range(args.steps):
        grads = pg.backward(Rg, Rbar)
    eb1.record(stream)
    torch.cuda.synchronize()
    bwd_ms = max_over_ranks(eb0.elapsed_time(eb1) / args.steps)
    pg.close()
    del grads

    # --- end to end through the C ABI with pinned host buffers
    host_inputs = make_inputs(db, torch, "cpu")
    ph = binding.JoinPlan(host_inputs, db.parent, mem=binding.FIGARO_MEM_HOST, stream=stream)
    Rh = torch.empty(db.n_cols, db.n_cols, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        ph.qr_r(out=Rh)
    barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        ph.qr_r(out=Rh)          # H2D copies, the whole path, D2H of R, final sync
    e2e_seq_ms = max_over_ranks((time.perf_counter() - t) * 1e3 / args.steps)
    ph.close()
    # pipelined: two plans on two streams alternate (figaro_qr_r_async / figaro_plan_sync),
    # so one step's host-to-device copies overlap the other's computation; every step still
    # copies its inputs in and its R out
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pp = [binding.JoinPlan(host_inputs, db.parent, mem=binding.FIGARO_MEM_HOST, stream=s) for s in streams]
    Rp = [torch.empty(db.n_cols, db.n_cols, dtype=torch.float64).pin_memory() for _ in pp]
    for i in range(max(args.warmup, 2)):
        pp[i % 2].qr_r_async(Rp[i % 2])
        pp[i % 2].sync()
    barrier()
    t = time.perf_counter()
    for i in range(args.steps):
        p_i = pp[i % 2]
        if i >= 2:
            p_i.sync()                 # its previous step (two steps back) is complete
        p_i.qr_r_async(Rp[i % 2])
    for p_i in pp:
        p_i.sync()
    e2e_ms = max_over_ranks((time.perf_counter() - t) * 1e3 / args.steps)
    assert np.array_equal(Rp[0].numpy(), Rp[1].numpy())
    for p_i in pp:
        p_i.close()

    hbm, hbm_kind = peaks()
    value = cells * world / (ms64 * 1e-3)
    gbs = in_bytes * world / (ms64 * 1e-3) / 1e9
    steps_timed = args.steps
    # stage breakdown of the FP64 step (serialised TSQR; "tsqr_tree" is the whole TSQR section)
    per_stage = {k: v[0] / steps_timed for k, v in stages.items()}
    launches = {k: v[1] / steps_timed for k, v in stages.items()}
    dom = max((k for k in per_stage if k != "tsqr_leaf"), key=per_stage.get)
    leaf_ms = per_stage["tsqr_leaf"]
    # the dominant kernel: the register TSQR leaf of the 8-column tails blocks (one launch
    # per block per step, timed by CUDA events around it on its stream in the stage-timed
    # plan).  Algorithmic flops per launch: 2 rows n^2 - 2/3 n^3 (Householder, R only).
    dom_blocks = [(ms / steps_timed, n, rows) for ms, n, rows in block_times if n == 8 and rows > 0]
    dom_flops = sum(2.0 * rows * n * n - 2.0 / 3.0 * n ** 3 for _, n, rows in dom_blocks) / len(dom_blocks)
    dom_ms = sum(ms for ms, _, _ in dom_blocks) / len(dom_blocks)
    dom_rows = sum(rows for _, _, rows in dom_blocks) / len(dom_blocks)
    dom_tflops = dom_flops / (dom_ms * 1e-3) / 1e12
    roofline = {"kernel": "k_tsqr_reg<double, 8> (TSQR leaf of a tails block: warp-per-tile Householder "
                          "in registers, FP64)",
                "bound": "alu", "achieved": dom_tflops, "peak": round(FP64_PEAK_TFLOPS, 3),
                "unit": "TFLOP/s", "frac": dom_tflops / FP64_PEAK_TFLOPS,
                "traffic": DOMINANT_DRAM_BYTES_PER_ROW * dom_rows,
                "peak_kind": "derived FP64 pipe peak: 152 SMs x 2 DFMA/clk x 2070 MHz",
                "flops_per_launch": dom_flops, "rows_per_launch": dom_rows, "ms_per_launch": dom_ms,
                "launches_per_step": len(dom_blocks),
                "algorithmic_bytes_per_launch": dom_rows * 8 * 8,
                "all_leaf_launches": {"ms_per_step": leaf_ms, "flops_per_step": info["tsqr_leaf_flops"],
                                      "tflops": info["tsqr_leaf_flops"] / (leaf_ms * 1e-3) / 1e12,
                                      "launches_per_step": launches["tsqr_leaf"]},
                "staged_ms_per_step": ms_staged, "largest_stage": dom}
    out = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "throughput_mode": "two calls in flight (two plans, two streams, figaro_qr_r_async / figaro_plan_sync)",
        "latency_ms_per_step": lat64,
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, see config)",
        "config": {"workload": WORKLOAD, "rows_per_relation": args.rows, "cols": db.n_cols,
                   "input_cells_per_gpu": cells, "input_bytes_per_gpu": in_bytes,
                   "l2": "inputs exceed L2 (448 MB > 129 MB); no flush", "sort": "included",
                   "parallelism": f"replicas x{world} (independent instances)"},
        "gbs": gbs, "hbm_frac": gbs / hbm, "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind,
        "backward": {"ms_per_call": bwd_ms, "loss": "||R||_F^2", "value": cells * world / (bwd_ms * 1e-3),
                     "unit": "cells/s", "note": "figaro_backward after a forward call: gradients of all "
                                                "data columns, FP64 (includes output allocation)"},
        "mixed": {"ms_per_step": msmx, "value": cells * world / (msmx * 1e-3), "speedup_vs_fp64": lat64 / msmx,
                  "basis": "one plan, one call at a time (latency), against latency_ms_per_step",
                  "throughput_ms_per_step": msmx_tp, "throughput_value": cells * world / (msmx_tp * 1e-3),
                  "throughput_speedup_vs_fp64": ms64 / msmx_tp,
                  "rel_err_RtR_vs_fp64_path": err_mx, "stages_ms_per_step": mx_stages,
                  "refined": {"ms_per_step": msmr, "value": cells * world / (msmr * 1e-3),
                              "speedup_vs_fp64": lat64 / msmr, "refinement_applied": refined,
                              "rel_err_RtR_vs_fp64_path": err_mr, "rel_err_R_vs_fp64_path": err_mr_r,
                              "dtype": "mixed path + one CholeskyQR2-style correction with A^T A in "
                                       "double-float"},
                  "dtype": "double-float head/tail sums, f32 tails and TSQR leaf/tree, f64 counts, join, final QR"},
        "stages_ms_per_step": per_stage,
        "stage_note": "from a stage-timed plan with serialised TSQR chains; tsqr_tree = whole TSQR section, tsqr_leaf = its leaf launches",
        "r0_rows": info["r0_rows"],
        "roofline": roofline,
        "e2e": {"value": cells * world / (e2e_ms * 1e-3), "unit": "cells/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": db.n_cols * db.n_cols * 8 + 4,
                "mode": "two plans on two streams alternating figaro_qr_r_async / figaro_plan_sync",
                "sequential_ms_per_step": e2e_seq_ms, "h2d_note": "pinned H2D measured at ~210 GB/s: "
                                                                  "2.2 ms of copies per step"},
        "gpu_launches": int(info["launches"]) * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.sample_rows)
    if world > 1:
        import torch.distributed as dist
        barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def oracle_step(db):
    from oracle import figaro as ofg
    return ofg.figaro_r(db)


def cpu_baseline(sample_rows, repeats=1):
    db = synth.path3(seed=2, rows=sample_rows)
    t = time.perf_counter()
    for _ in range(repeats):
        oracle_step(db)
    dt = (time.perf_counter() - t) / repeats
    return {"value": db.input_cells() / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": f"path3 with {sample_rows} rows per relation (same key law and columns), "
                      f"{db.input_cells()} cells, oracle FiGaRo R (Alg. 3, Alg. 4, §7 Householder), "
                      f"{dt:.2f} s per run"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    db = synth.path3(seed=2, rows=args.sample_rows)
    cells = db.input_cells()
    for _ in range(args.warmup):
        oracle_step(db)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(db)
    dt = (time.perf_counter() - t) / args.steps
    value = cells / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "rows_per_relation": args.sample_rows,
                   "note": "CPU oracle on a bounded sample of the same workload"},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": f"path3 with {args.sample_rows} rows per relation, {cells} cells"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="figaro", choices=["figaro", "reference"])
    ap.add_argument("--rows", type=int, default=ROWS)
    ap.add_argument("--sample-rows", type=int, default=SAMPLE_ROWS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plan-only", choices=["fp64", "mixed", "fp64-staged", "mixed-staged"],
                    help="profiling aid: run one plan only and print no JSON line")
    ap.add_argument("--workload", choices=["path3", "star", "snowflake"], default="path3",
                    help="workload of --plan-only")
    ap.add_argument("--wide", action="store_true",
                    help="measure the wide-block workloads (star, snowflake) instead")
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
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_figaro(args)


if __name__ == "__main__":
    main()
