#!/usr/bin/env python3
"""Benchmark of the generalized sparse contraction path on one B300.

Workload (default ``rmat18``): R-MAT scale 18 (262,144 vertices, edge factor 16,
a/b/c/d = 0.57/0.19/0.19/0.05, self-loops and duplicates removed), weights
uniform (0,1] as (m+1)*2^-24.  One step is the whole path over that graph:
(+,x) SpGEMM C = A.A in fp64, the same in fp32, and Bellman-Ford single-source
shortest paths from vertex 0 over the (min,+) fp32 semiring.  The metric is
semiring operations per second: the products of the two SpGEMMs (each one
multiply and one add of the algebra) plus the edge relaxations of Bellman-Ford,
divided by the step time.  ``er4096`` is the small (min,+) int32 SpGEMM case.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SpGEMM semiring-ops/s & MFBC GTEPS, learned+batched vs plain form on one B300"
UNIT = "semiring-ops/s"
L2_BYTES = 126 * 1024 * 1024
# DRAM bytes (read + write) per output entry of the fp64 numeric rank kernel, from
# one ncu capture of that kernel at R-MAT scale 16.
# Traffic grows with the output (B stays in L2), so a full launch is scaled by its
# nnz(C): 0.346 GB read + 1.848 GB written for 163,809,247 entries.
NUMERIC_FP64_DRAM_BYTES_PER_ENTRY = (0.346040e9 + 1.848326e9) / 163809247
# FP64 peak of the B300 part: 2 FP64 instructions (DADD, DMUL or DFMA) per clock per SM,
# 148 SMs, 2032 MHz maximum clock.  FP64_PEAK_TFLOPS is that instruction rate (in units
# of 1e12 instructions per second); FP64_FMA_PEAK_TFLOPS counts a DFMA as two flops
# (the nominal 1.25 TFLOP/s), the peak of a multiply-add per product.
FP64_OPS_PER_CLK_SM = 2
NUM_SMS = 148
SM_MAX_MHZ = 2032
FP64_PEAK_TFLOPS = FP64_OPS_PER_CLK_SM * NUM_SMS * SM_MAX_MHZ * 1e6 / 1e12
FP64_FMA_PEAK_TFLOPS = 2 * FP64_PEAK_TFLOPS


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def build_workload(name: str):
    if name.startswith("rmat"):
        scale = int(name[4:])
        A = W.rmat(scale, seed=0)
        w = W.weights_unit01(A.nnz, seed=0)
        g = W.weights_unit01(A.nnz, seed=1).astype(np.float32)
        return {"A": A, "w64": w, "w32": w.astype(np.float32), "g32": g, "scale": scale}
    if name == "er4096":
        A = W.er_fixed_degree(4096, 8, seed=0)
        return {"A": A, "wi32": W.weights_int(A.nnz, 1, 1000, seed=0), "scale": None}
    raise SystemExit(f"unknown workload {name}")


def products(A: W.Csr, rows=None) -> int:
    lens = np.diff(A.rowptr)
    if rows is None:
        return int(lens[A.col].sum())
    return int(sum(lens[A.col[A.rowptr[i]:A.rowptr[i + 1]]].sum() for i in rows))


_NPROD = {}


def nprod_of(A: W.Csr) -> int:
    key = id(A)
    if key not in _NPROD:
        _NPROD[key] = products(A)
    return _NPROD[key]


def csr_bytes(n, nnz, s):
    return 8 * (n + 1) + (4 + s) * nnz


# Betweenness centrality: algorithmic bytes per (edge, source) traversal in each
# direction -- the target's 4-byte distance read and its 8-byte multiplicity (forward)
# or dependency (backward) updated; the edge's column and length are shared by the
# batch's sources and not counted.
MFBC_BYTES_PER_TRAVERSAL = 12


def gustavson_bytes(A: W.Csr, B: W.Csr, nnzC: int, s: int) -> int:
    """Algorithmic bytes of C = A B in the row-wise (Gustavson) model: read A, for
    every stored A_ik the pointer pair of B_k (8 B) and B_k's columns and values,
    write C; s = bytes per value."""
    lens = np.diff(B.rowptr)
    gathered = int(lens[A.col].sum())
    return csr_bytes(A.nrows, A.nnz, s) + 8 * A.nnz + (4 + s) * gathered + csr_bytes(A.nrows, nnzC, s)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle arm

def oracle_sample(wl, budget_rows_stride=16):
    """Time the oracle on a bounded sample of the workload; returns (ops, seconds, desc)."""
    import oracle as O
    A = wl["A"]
    if wl["scale"] is None:
        a = A.with_val(wl["wi32"])
        t = time.perf_counter()
        O.spgemm(O.MP_I32, a, a)
        dt = time.perf_counter() - t
        return products(A), dt, "full er4096 (min,+) SpGEMM"
    nz = np.nonzero(np.diff(A.rowptr) > 0)[0]
    rows = nz[::budget_rows_stride]
    ops = 0
    t = time.perf_counter()
    a64 = A.with_val(wl["w64"])
    O.spgemm(O.PT_F64, a64, a64, rows=rows)
    a32 = A.with_val(wl["w32"])
    O.spgemm(O.PT_F32, a32, a32, rows=rows)
    g = A.with_val(wl["g32"])
    _, _, relax = O.bellman_ford(O.MP_F32, g, 0, with_relaxations=True)
    dt = time.perf_counter() - t
    ops = 2 * products(A, rows) + relax
    desc = (f"every {budget_rows_stride}th non-empty row of both (+,x) SpGEMMs "
            f"({rows.size} rows) plus full Bellman-Ford (full relaxation rounds)")
    return ops, dt, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    wl = build_workload(args.workload)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(wl)
    tot_ops, tot_t = 0, 0.0
    desc = ""
    for _ in range(args.steps):
        ops, dt, desc = oracle_sample(wl)
        tot_ops += ops
        tot_t += dt
    v = tot_ops / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------- GPU arm

def aggregate_ranks(ops, seconds, dist=None, device="cpu"):
    """Whole-job throughput of N replicas: the semiring operations of every rank over
    the slowest rank's timed span.  Returns (ops/s, max seconds, summed ops); with no
    process group, this rank's own figures."""
    if dist is None:
        return ops / seconds, seconds, ops
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    o = torch.tensor([float(ops)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(o, op=dist.ReduceOp.SUM)
    return o.item() / t.item(), t.item(), o.item()


def run_stc(args):
    import torch
    import paper_1512_00066_b300 as stc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = build_workload(args.workload)
    A = wl["A"]
    H = stc.Handle()
    H.set_timing(True)
    dev = torch.device("cuda", local)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    if wl["scale"] is None:
        ops_step = products(A)
        dA = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["wi32"])

        def step():
            C = H.spgemm(stc.MIN_PLUS_I32, dA, dA)
            t = H.phase_times()
            return ops_step, {"numeric_ms": t[4], "spgemm_ms": sum(t[:5]), "nnzC": C.nnz, "s": 4}
        dom_val_bytes = 4
    else:
        nprod = products(A)
        d64 = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["w64"])
        d32 = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["w32"])
        dg = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["g32"])

        def step():
            C = H.spgemm(stc.PLUS_TIMES_F64, d64, d64)
            t64 = H.phase_times()
            nnz64 = C.nnz
            del C
            C = H.spgemm(stc.PLUS_TIMES_F32, d32, d32)
            t32 = H.phase_times()
            del C
            dist_, rounds = H.bellman_ford(stc.MIN_PLUS_F32, dg, 0, persistent=True)
            tbf = H.phase_times()
            relax = H.last_relaxations
            return 2 * nprod + relax, {"numeric_ms": t64[4], "phases64": t64, "phases32": t32,
                                       "bf_ms": tbf, "nnzC": nnz64, "rounds": rounds,
                                       "relax": relax, "s": 8}
        dom_val_bytes = 8

    # setup, outside the timed region: the autotuner picks the light-row threshold of
    # each SpGEMM of the step (cached in the handle for later calls)
    tuning = None
    if not args.no_tune and A.ncols <= (1 << 18):
        if wl["scale"] is None:
            tuning = {"int32": H.autotune_spgemm(stc.MIN_PLUS_I32, dA, dA)}
        else:
            tuning = {"fp64": H.autotune_spgemm(stc.PLUS_TIMES_F64, d64, d64),
                      "fp32": H.autotune_spgemm(stc.PLUS_TIMES_F32, d32, d32)}
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos, ops_total = [], 0
    launches0 = H.kernel_launches()
    barrier()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between timed steps (outside the timed span)
            ev[k][0].record()
            ops, info = step()
            ev[k][1].record()
            ops_total += ops
            infos.append(info)
        barrier()
    launches = H.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, t_total, _ = aggregate_ranks(ops_total, sum(step_ms) / 1e3, dist, dev)

    # roofline of the dominant kernel: the numeric phase of the first SpGEMM of the
    # step.  Algorithmic bytes follow the row-wise (Gustavson) traffic model: read A,
    # for every stored A_ik its B row's pointer pair (8 B) and the row's columns and
    # values, write C (gustavson_bytes).  The compulsory bytes (A, B and C once, plus
    # the cell table and C.rowptr read back) are reported beside them.
    n, nnzA = A.nrows, A.nnz
    nnzC = infos[0]["nnzC"]
    s = dom_val_bytes
    ncell = -(-A.ncols // 1024)
    compulsory = (csr_bytes(n, nnzA, s) * 2 + 4 * A.nrows * (ncell + 1)
                  + 8 * (n + 1) + (4 + s) * nnzC)
    num_ms = statistics.mean(i["numeric_ms"] for i in infos)
    hbm, peak_kind = peaks()
    gbytes = gustavson_bytes(A, A, nnzC, s)
    achieved = gbytes / (num_ms / 1e3) / 1e9
    if wl["scale"]:
        sp_ms = statistics.mean(sum(i["phases64"][:5]) for i in infos)
    else:
        sp_ms = statistics.mean(i["spgemm_ms"] for i in infos)
    # fp64 instruction rate of the numeric phase (one DFMA per product), informational
    dfma_per_s = nprod_of(A) / (num_ms / 1e3)
    # the accumulator bound: products per second that shared-memory accumulation
    # with the algebra's (+) absorbs on this device (calibration kernel of the library)
    acc_alg = stc.PLUS_TIMES_F64 if wl["scale"] else stc.MIN_PLUS_I32
    acc_rate = H.calibrate_accumulate(acc_alg)
    acc_achieved = nprod_of(A) / (num_ms / 1e3)

    # end to end: host (pinned) inputs -> device -> the same step -> results back to host
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, stc, H, wl, dev)
    forms = {}
    if not args.no_forms and rank == 0:
        H.set_timing(False)
        want = set(args.forms.split(","))
        rmat = wl["scale"] is not None  # forms that run on the step's own R-MAT graph
        if "bf" in want and rmat:
            forms["bellman_ford_drivers"] = measure_bf_drivers(stc, H, wl)
        if "er4096" in want:
            forms["er4096"] = measure_er4096(stc, H)
        if "learned" in want and rmat:
            forms["learned_vs_plain"] = measure_learned(stc, H, wl, dev)
        if "masked" in want and rmat:
            forms["masked_vs_plain"] = measure_masked(stc, H, wl)
        if "apsp" in want:
            forms["apsp_path_doubling"] = measure_apsp(stc, H)
        if "spmm" in want:
            forms["spmm_e1"] = measure_spmm_e1(stc, H)
        if "mlp" in want:
            forms["mlp_forward"] = measure_mlp(stc, H)
        if "batched" in want:
            forms["batched_vs_per_call"] = measure_batched(stc, H, args.batched_pairs, not args.batched_no_per_call)
        if "mfbc" in want:
            forms["mfbc"] = measure_mfbc(stc, H, scale=args.mfbc_scale, nsrc=args.mfbc_sources)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32" if wl["scale"] else "int32",
            "data": "synthetic",
            "config": {"workload": (f"rmat{wl['scale']}: (+,x) SpGEMM A.A fp64 and fp32 + Bellman-Ford "
                                    "(min,+) fp32 from vertex 0" if wl["scale"] else
                                    "er4096: (min,+) int32 SpGEMM A(x)A"),
                       "n": A.nrows, "nnz": A.nnz, "nnzC": nnzC, "parallelism": "replicas" if world > 1 else "1gpu",
                       "l2": "flushed between timed steps (write of 2x L2)",
                       "ops_per_step": ops_total // args.steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                         if peak_kind == "measured" else "fallback 6.4 TB/s",
                         "traffic": (NUMERIC_FP64_DRAM_BYTES_PER_ENTRY * nnzC
                                     if (NUMERIC_FP64_DRAM_BYTES_PER_ENTRY and wl["scale"]) else None),
                         "traffic_note": "ncu DRAM bytes of the numeric kernel at R-MAT scale 16 scaled by nnz(C)",
                         "kernel": ("k_numeric_rank + k_copy_rows (numeric phase of the fp64 SpGEMM)"
                                    if wl["scale"] else "numeric phase of the (min,+) int32 SpGEMM"),
                         "kernel_ms": num_ms, "algorithmic_bytes": gbytes,
                         "bytes_model": "|A| + sum over stored A_ik of (8 + nnz(B_k)(4+s)) + |C|",
                         "whole_spgemm": {"ms": sp_ms, "frac": gbytes / (sp_ms / 1e3) / 1e9 / hbm},
                         "compulsory": {"bytes": compulsory,
                                        "frac": compulsory / (num_ms / 1e3) / 1e9 / hbm},
                         "fp64_dfma_per_s": dfma_per_s if wl["scale"] else None,
                         "smem_accumulate": {"achieved": acc_achieved, "peak": acc_rate,
                                             "unit": "products/s", "frac": acc_achieved / acc_rate,
                                             "peak_source": "stc_calibrate_accumulate on this device"}},
            "gpu_launches": launches,
            "tuning": tuning,
            "clocks": clk.summary(),
            "phases_ms": infos[-1],
        }
        if e2e is not None:
            out["e2e"] = e2e
        if forms:
            out["forms"] = forms
        if not args.no_cpu_baseline and world == 1:
            import oracle as O
            cores = len(os.sched_getaffinity(0))
            O.set_threads(cores)
            ops, dt, desc = oracle_sample(wl)
            out["cpu_baseline"] = {"value": ops / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": desc}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def _timed(fn, reps):
    """Median wall time (s) of fn() over reps runs, each bracketed by device syncs."""
    import torch
    ts = []
    out = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
        if out is not None and not isinstance(out, tuple):
            del out
            out = None
    return statistics.median(ts)


def measure_learned(stc, H, wl, dev):
    """Plain two-pass vs learned single pass (trained model) vs upper-bound single
    pass on (+,x) fp32 A.A for the workload's graph and for R-MAT scale 20 (2^20
    output columns: four column slabs).  The model is trained on about 1.1M rows of
    R-MAT scales 14-18 (seeds 1-5), ER and banded matrices, never on a measured
    graph (seed 0)."""
    import torch
    pairs = []
    specs = [W.rmat(14, seed=1), W.rmat(15, seed=2), W.rmat(16, seed=3), W.rmat(17, seed=4), W.rmat(18, seed=5),
             W.er_fixed_degree(1 << 18, 8, seed=1), W.er_fixed_degree(1 << 17, 16, seed=2),
             W.banded(1 << 17, 16, 0.5, seed=3), W.banded(1 << 16, 4, 0.5, seed=4)]
    for m in specs:
        d = stc.DeviceCsr.from_host(m.nrows, m.ncols, m.rowptr, m.col, None)
        pairs.append((d, d))
    t0 = time.perf_counter()
    feat, target = stc.training_rows(H, pairs)
    n_train = int(target.numel())
    w = stc.mlp_init(seed=1)
    losses = H.mlp_train(w, feat, target, batch=8192, epochs=20, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del feat, target, pairs
    torch.cuda.empty_cache()
    out = {"unit": UNIT,
           "training": {"rows": n_train, "seconds": t_train, "final_loss": losses[-1] if losses else None,
                        "epochs": len(losses)}}
    graphs = [("rmat18", wl["A"] if wl["scale"] == 18 else W.rmat(18, seed=0)), ("rmat20", W.rmat(20, seed=0))]
    for name, A in graphs:
        d32 = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col,
                                      W.weights_unit01(A.nnz, seed=0).astype(np.float32))
        nprod = products(A)
        res = {"workload": f"{name} (+,x) fp32 A.A", "columns": A.ncols}
        stats = {}

        def learned(weights, margin, key):
            C, st = H.spgemm_learned(stc.PLUS_TIMES_F32, d32, d32, weights, margin)
            stats[key] = st
            return C

        for key, fn in (("plain", lambda: H.spgemm(stc.PLUS_TIMES_F32, d32, d32)),
                        ("learned", lambda: learned(w, 0.5, "model")),
                        ("upper_bound", lambda: learned(None, 0.0, "upper_bound"))):
            try:
                t = _timed(fn, 3)
                res[key + "_ms"] = 1e3 * t
                res[key] = nprod / t
            except Exception as e:  # the upper-bound scratch can exceed device memory
                res[key] = None
                res[key + "_error"] = str(e)[:120]
            torch.cuda.empty_cache()
        res["model_stats"] = stats.get("model")
        res["upper_bound_stats"] = stats.get("upper_bound")
        nnzC = (stats.get("model") or {}).get("nnz")
        if nnzC:
            hbm, peak_kind = peaks()
            gb = gustavson_bytes(A, A, int(nnzC), 4)
            res["roofline"] = {"bound": "hbm", "algorithmic_bytes": gb, "unit": "GB/s", "peak": hbm,
                               "peak_source": peak_kind}
            for key in ("plain", "learned", "upper_bound"):
                if res.get(key + "_ms"):
                    res["roofline"][key + "_frac"] = gb / (res[key + "_ms"] / 1e3) / 1e9 / hbm
        out[name] = res
        del d32
        torch.cuda.empty_cache()
    return out


def measure_masked(stc, H, wl):
    """Masked product C<A> = A.A (the output structure given: A's own, the
    triangle-counting shape) against the plain A.A, (+,x) fp64 on the workload's
    graph."""
    import torch
    A = wl["A"]
    d64 = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["w64"])
    M = stc.DeviceCsr(A.nrows, A.ncols, d64.rowptr, d64.col, None)
    nprod = products(A)
    t_plain = _timed(lambda: H.spgemm(stc.PLUS_TIMES_F64, d64, d64), 3)
    t_mask = _timed(lambda: H.spgemm_masked(stc.PLUS_TIMES_F64, d64, d64, M), 3)
    torch.cuda.empty_cache()
    return {"unit": UNIT, "workload": f"rmat{wl['scale']} (+,x) fp64: C<A> = A.A vs A.A",
            "products": nprod, "mask_entries": A.nnz,
            "masked": nprod / t_mask, "plain": nprod / t_plain,
            "ms": {"masked": 1e3 * t_mask, "plain": 1e3 * t_plain}}


def measure_apsp(stc, H, n=2048):
    """All-pairs shortest paths by path doubling on the paper's APSP workload:
    a dense graph on n = 2048 vertices with int32 lengths U[1, n^2].  Ops = the
    (min,+) products of all squarings."""
    import torch
    rng = np.random.default_rng(0)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    keep = rows != cols
    G = W.csr_from_coo(rows[keep], cols[keep], n, n)
    G.val = rng.integers(1, n * n + 1, G.nnz).astype(np.int32)
    d = stc.DeviceCsr.from_host(G.nrows, G.ncols, G.rowptr, G.col, G.val)
    res = {}

    def run():
        P, sq = H.apsp(d)
        res["squarings"] = sq
        res["nnz"] = P.nnz
        return P

    t = _timed(run, 3)
    ops = res["squarings"] * n ** 3  # every squaring of a full matrix: n^3 products
    tk = {}

    def run_tiskin():
        P, rounds, prods = H.apsp_tiskin(d)
        tk["rounds"] = rounds
        tk["products"] = prods
        return P

    t_tk = _timed(run_tiskin, 3)
    torch.cuda.empty_cache()
    return {"unit": UNIT, "workload": f"dense n={n}, int32 lengths U[1, n^2]",
            "path_doubling": {"ms": 1e3 * t, "squarings": res["squarings"], "products": ops, "value": ops / t,
                              "closure_nnz": res["nnz"]},
            "tiskin": {"ms": 1e3 * t_tk, "rounds": tk["rounds"], "products": tk["products"],
                       "value": tk["products"] / t_tk}}


def measure_mlp(stc, H, scale=20):
    """Row-size perceptron forward over the features of every row of A.A (R-MAT
    scale 20, 2^20 rows): the CUDA-core kernel against the tcgen05 one, timed with
    CUDA events on the launching stream (the 285 MB feature matrix is larger than
    L2).  Algorithmic bytes per row: 272 of features read, 4 of prediction written."""
    import torch
    A = W.rmat(scale, seed=0)
    dA = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, np.ones(A.nnz, np.float32))
    feat = H.row_features(dA, dA)
    n = feat.shape[0]
    w = stc.mlp_init(seed=1)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    hbm, peak_kind = peaks()
    L = stc.lib()
    s = torch.cuda.current_stream()
    out = {"workload": f"features of R-MAT {scale} A.A rows ({n} rows x 68 fp32)", "rows": n,
           "bytes_per_row": 276}
    for name, fn in (("cuda_cores", L.stc_mlp_forward), ("tcgen05", L.stc_mlp_forward_tc)):
        def run():
            st = fn(H._h, w.data_ptr(), feat.data_ptr(), n, y.data_ptr(), s.cuda_stream)
            if st != 0:
                raise stc.StcError(st, name)
        for _ in range(3):
            run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(10):
            run()
        e1.record(s)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 10 / 1e3
        gbs = n * 276 / t / 1e9
        out[name] = {"us": 1e6 * t, "GB/s": gbs, "hbm_frac": gbs / hbm, "peak_source": peak_kind}
        out[name]["y"] = y.clone()
    H.check_device_status()
    yc, yt = out["cuda_cores"].pop("y"), out["tcgen05"].pop("y")
    out["max_rel_diff"] = float(((yc - yt).abs() / (1 + yc.abs())).max())
    out["speedup"] = out["cuda_cores"]["us"] / out["tcgen05"]["us"]
    del feat, dA, y, yc, yt
    torch.cuda.empty_cache()
    return out


def measure_spmm_e1(stc, H, n=16384, k=8192, densities=(0.01, 0.16)):
    """The paper's SpMM experiment shape: an n x n sparse matrix with independent
    density d times a dense n x k block (n = 16384, k = 8192), fp64.  Each product
    is one DFMA instruction (2 flops); the fraction is of the FP64 instruction
    peak (2 per clock per SM, the same unit as the numeric kernel's roofline)."""
    import torch
    X = torch.rand((n, k), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    Y = torch.empty((n, k), dtype=torch.float64, device="cuda")
    out = {"workload": f"A {n}x{n} sparse (independent density), X {n}x{k} dense, fp64", "unit": "TFLOP/s"}
    for dens in densities:
        rng = np.random.default_rng(0)
        A = W.distinct_columns(rng, rng.binomial(n, dens, size=n), n)
        A.val = W.weights_unit01(A.nnz, 1)
        d = stc.DeviceCsr.from_host(n, n, A.rowptr, A.col, A.val)
        t = _timed(lambda: H.spmm(stc.PLUS_TIMES_F64, d, X, Y), 3)
        fma_t = A.nnz * k / t / 1e12  # DFMA instructions, in units of 1e12 per second
        out[f"density_{dens}"] = {"nnz": A.nnz, "ms": 1e3 * t, "tflops": 2.0 * fma_t,
                                  "fp64_frac": fma_t / FP64_PEAK_TFLOPS}
        del d
    del X, Y
    torch.cuda.empty_cache()
    return out


def measure_batched(stc, H, npairs=4096, with_per_call=True):
    """4096 independent (+,x) fp32 pairs: one batched call vs one call per pair.
    Roofline: the row-wise traffic model summed over the pairs (gustavson_bytes)
    over the batched call's time, against the measured HBM bandwidth.  npairs and
    with_per_call select a smaller batch and skip the per-call loop (profiling runs)."""
    import torch
    sizes, As, Bs = W.powerlaw_batch(npairs, 64, 16384, 2.1, 4, 64, seed=0)
    dA = [stc.DeviceCsr.from_host(a.nrows, a.ncols, a.rowptr, a.col, a.val) for a in As]
    dB = [stc.DeviceCsr.from_host(b.nrows, b.ncols, b.rowptr, b.col, b.val) for b in Bs]
    nprod = sum(int(np.diff(b.rowptr)[a.col].sum()) for a, b in zip(As, Bs))
    nnz = {}

    def batched():
        Cs = H.spgemm_batched(stc.PLUS_TIMES_F32, dA, dB)
        nnz["c"] = Cs._nnz
    t_b = _timed(batched, 3)
    gbytes = sum(gustavson_bytes(a, b, int(c), 4) for a, b, c in zip(As, Bs, nnz["c"]))
    hbm, peak_kind = peaks()

    def per_call():
        for a, b in zip(dA, dB):
            H.spgemm(stc.PLUS_TIMES_F32, a, b)
    t_p = _timed(per_call, 1) if with_per_call else None
    torch.cuda.empty_cache()
    return {"unit": UNIT, "workload": f"{npairs} pairs, rows power-law [64,16384] exp 2.1, U{{4..64}}/row, N(0,1) fp32",
            "products": nprod, "nnzC": int(nnz["c"].sum()), "batched": nprod / t_b,
            "per_call": nprod / t_p if t_p else None,
            "ms": {"batched": 1e3 * t_b, "per_call": 1e3 * t_p if t_p else None},
            "roofline": {"bound": "hbm", "algorithmic_bytes": gbytes, "achieved": gbytes / t_b / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": gbytes / t_b / 1e9 / hbm, "peak_source": peak_kind,
                         "time": "whole batched call (wall clock, device synchronised)"}}


def measure_er4096(stc, H, reps=20):
    """The small (min,+) int32 case: C = A (x) A for an Erdos-Renyi digraph on 4096
    vertices with exactly 8 distinct uniform columns per row, weights U[1,1000]
    (seed 0); plain two-pass call, wall clock per call and the numeric phase from the
    library's events, each against the row-wise traffic model."""
    import torch
    A = W.er_fixed_degree(4096, 8, seed=0)
    A.val = W.weights_int(A.nnz, 1, 1000, seed=0)
    d = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, A.val)
    nprod = products(A)
    for _ in range(3):
        C = H.spgemm(stc.MIN_PLUS_I32, d, d)
    nnzC = C.nnz
    t = _timed(lambda: H.spgemm(stc.MIN_PLUS_I32, d, d), reps)
    H.set_timing(True)
    ph = []
    for _ in range(reps):
        H.spgemm(stc.MIN_PLUS_I32, d, d)
        ph.append(H.phase_times())
    H.set_timing(False)
    num_ms = statistics.median(p[4] for p in ph)
    gbytes = gustavson_bytes(A, A, nnzC, 4)
    hbm, peak_kind = peaks()
    torch.cuda.empty_cache()
    return {"unit": UNIT, "workload": "er4096: (min,+) int32 A(x)A, 8 distinct columns per row, U[1,1000]",
            "products": nprod, "nnzC": nnzC, "ms": 1e3 * t, "value": nprod / t, "numeric_ms": num_ms,
            "roofline": {"bound": "hbm", "algorithmic_bytes": gbytes, "unit": "GB/s", "peak": hbm,
                         "peak_source": peak_kind, "call_frac": gbytes / t / 1e9 / hbm,
                         "numeric_frac": gbytes / (num_ms / 1e3) / 1e9 / hbm,
                         "note": "4.7 MB of traffic: launch- and latency-bound at any speed"}}


def measure_bf_drivers(stc, H, wl):
    """Bellman-Ford (min,+) fp32 from vertex 0 on the workload graph with the three
    drivers: host loop (one launch + one read-back per round), one cooperative
    persistent launch, one CUDA graph with a conditional WHILE node."""
    A = wl["A"]
    dg = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, wl["g32"])
    out = {"unit": "ms", "workload": "rmat18 (min,+) fp32 from vertex 0"}
    for name, mode in (("host_loop", 0), ("persistent", 1), ("cuda_graph", 2)):
        H.bellman_ford(stc.MIN_PLUS_F32, dg, 0, persistent=mode)  # warm
        out[name] = 1e3 * _timed(lambda: H.bellman_ford(stc.MIN_PLUS_F32, dg, 0, persistent=mode), 5)
    # many short calls: R-MAT 14, 1000 sources one call each (the graph is
    # instantiated once per handle and reused; each call rewrites its parameters)
    G = W.rmat(14, seed=0)
    d14 = stc.DeviceCsr.from_host(G.nrows, G.ncols, G.rowptr, G.col, W.weights_unit01(G.nnz, seed=1).astype(np.float32))
    srcs = W.sample_sources(G, 1000, seed=0)
    short = {"workload": "rmat14 (min,+) fp32, 1000 calls from sampled sources", "unit": "ms per call"}
    for name, mode in (("host_loop", 0), ("persistent", 1), ("cuda_graph", 2)):
        H.bellman_ford(stc.MIN_PLUS_F32, d14, int(srcs[0]), persistent=mode)

        def many():
            for v in srcs:
                H.bellman_ford(stc.MIN_PLUS_F32, d14, int(v), persistent=mode)
        short[name] = 1e3 * _timed(many, 1) / len(srcs)
    out["short_calls"] = short
    return out


def measure_mfbc(stc, H, scale=22, nsrc=4096, batch=256):
    """Betweenness centrality on R-MAT scale 22 over a 4096-source sample (16
    batches of 256; other sizes through --mfbc-scale / --mfbc-sources):
    GTEPS = sources * edges / time (forward + backward + reduction), with unit and
    int32 [1, 255] lengths; the host-driven round loop is timed on one batch beside
    the graph driver."""
    import torch
    G = W.rmat(scale, seed=0)
    src = W.sample_sources(G, nsrc, seed=0)
    out = {"unit": "GTEPS", "workload": f"rmat{scale}, {nsrc} sources in batches of {batch}", "edges": G.nnz}
    for name, val in (("unit_lengths", None), ("int_lengths_1_255", W.weights_int(G.nnz, 1, 255, seed=1))):
        d = stc.DeviceCsr.from_host(G.nrows, G.ncols, G.rowptr, G.col, val)
        H.set_round_driver("graph")
        t = _timed(lambda: H.mfbc(d, src, batch=batch), 1)
        out[name] = len(src) * G.nnz / t / 1e9
        out[name + "_ms"] = 1e3 * t
        hbm, peak_kind = peaks()
        gb = MFBC_BYTES_PER_TRAVERSAL * 2 * len(src) * G.nnz
        out[name + "_roofline"] = {"bound": "hbm", "algorithmic_bytes": gb, "unit": "GB/s",
                                   "achieved": gb / t / 1e9, "peak": hbm, "frac": gb / t / 1e9 / hbm,
                                   "peak_source": peak_kind,
                                   "model": f"{MFBC_BYTES_PER_TRAVERSAL} B per (edge, source), forward and backward"}
        one = src[:batch]
        for drv in ("graph", "host"):
            H.set_round_driver(drv)
            t1 = _timed(lambda: H.mfbc(d, one, batch=batch), 1)
            out[f"{name}_one_batch_{drv}_ms"] = 1e3 * t1
        H.set_round_driver("graph")
        del d
        torch.cuda.empty_cache()
    # many small batches: the per-round host round trip against one graph per batch
    Gs = W.rmat(16, seed=0)
    srcs = W.sample_sources(Gs, 1024, seed=0)
    ds = stc.DeviceCsr.from_host(Gs.nrows, Gs.ncols, Gs.rowptr, Gs.col, W.weights_int(Gs.nnz, 1, 255, seed=1))
    small = {"workload": "rmat16, int lengths 1..255, 1024 sources in batches of 64"}
    for drv in ("graph", "host"):
        H.set_round_driver(drv)
        t = _timed(lambda: H.mfbc(ds, srcs, batch=64), 3)
        small[drv + "_ms"] = 1e3 * t
        small[drv + "_gteps"] = len(srcs) * Gs.nnz / t / 1e9
    H.set_round_driver("graph")
    out["small_batches"] = small
    return out


def measure_e2e(args, stc, H, wl, dev):
    """Same metric through the public API with host inputs and host results."""
    import torch
    A = wl["A"]
    if wl["scale"] is None:
        return None
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_ptr, h_col = pin(A.rowptr), pin(A.col)
    h_w64, h_w32, h_g = pin(wl["w64"]), pin(wl["w32"]), pin(wl["g32"])
    nprod = products(A)
    # the step's inputs: the graph's structure (shared by its three operations) and
    # three value arrays
    h2d = h_ptr.numel() * 8 + h_col.numel() * 4 + h_w64.numel() * 8 + h_w32.numel() * 4 + h_g.numel() * 4
    out_bufs = {}
    side = torch.cuda.Stream(device=dev)  # results go back to the host while the next operation runs

    def host_buf(key, t):
        b = out_bufs.get(key)
        if b is None or b.numel() < t.numel() or b.dtype != t.dtype:
            b = out_bufs[key] = torch.empty(t.numel(), dtype=t.dtype).pin_memory()
        return b[: t.numel()]

    def back(items):
        ev = torch.cuda.Event()
        ev.record()
        side.wait_event(ev)
        n = 0
        with torch.cuda.stream(side):
            for key, t in items:
                host_buf(key, t).copy_(t, non_blocking=True)
                t.record_stream(side)
                n += t.numel() * t.element_size()
        return n

    def one():
        ptr_d = h_ptr.to(dev, non_blocking=True)
        col_d = h_col.to(dev, non_blocking=True)
        v64 = h_w64.to(dev, non_blocking=True)
        C = H.spgemm(stc.PLUS_TIMES_F64, stc.DeviceCsr(A.nrows, A.ncols, ptr_d, col_d, v64),
                     stc.DeviceCsr(A.nrows, A.ncols, ptr_d, col_d, v64))
        d2h = back((("p64", C.rowptr), ("c64", C.col), ("v64", C.val)))
        del C
        v32 = h_w32.to(dev, non_blocking=True)
        C = H.spgemm(stc.PLUS_TIMES_F32, stc.DeviceCsr(A.nrows, A.ncols, ptr_d, col_d, v32),
                     stc.DeviceCsr(A.nrows, A.ncols, ptr_d, col_d, v32))
        d2h += back((("p32", C.rowptr), ("c32", C.col), ("v32", C.val)))
        del C
        G = stc.DeviceCsr(A.nrows, A.ncols, ptr_d, col_d, h_g.to(dev, non_blocking=True))
        d, _ = H.bellman_ford(stc.MIN_PLUS_F32, G, 0)
        d2h += back((("dist", d),))
        torch.cuda.synchronize()
        return 2 * nprod + H.last_relaxations, d2h

    one()  # warm (allocates the pinned result buffers)
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t = time.perf_counter()
    ops = 0
    d2h = 0
    for _ in range(steps):
        o, d2h = one()
        ops += o
    dt = time.perf_counter() - t
    return {"value": ops / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="stc", choices=["stc", "reference"])
    ap.add_argument("--workload", default="rmat18",
                    help="rmat<scale> (the R-MAT step; rmat18 is the benchmark) or er4096")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the light-row autotuning before the warm-up")
    ap.add_argument("--forms", default="bf,er4096,learned,masked,apsp,spmm,mlp,batched,mfbc",
                    help="comma-separated subset of the comparison forms to run after the timed steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mfbc-scale", type=int, default=22, help="R-MAT scale of the mfbc form")
    ap.add_argument("--mfbc-sources", type=int, default=4096, help="sampled sources of the mfbc form")
    ap.add_argument("--batched-pairs", type=int, default=4096, help="pairs of the batched form")
    ap.add_argument("--batched-no-per-call", action="store_true",
                    help="skip the one-call-per-pair comparison of the batched form")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the learned / batched / centrality measurements")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_stc(args)


if __name__ == "__main__":
    main()
