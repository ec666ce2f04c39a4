#!/usr/bin/env python
"""pMMF benchmark: factor throughput (nnz/s) at the stated Frobenius error, plus
matrix-free apply GB/s against the HBM peak.

Workload (the metric's configuration): the Laplacian + 1e-3 I of the
symmetrised 10-nearest-neighbour graph of 65,536 uniform points in the unit
square (seed 1, about 12 nonzeros per row), FP64 CSR; clusters of about 256
coordinates by k-means on the points, Givens rotations (k = 2), eta = 0.5,
core size 256.  One step = one full factorization (every stage: clustering,
Gram, rotation search, blocked update, accounting) with the input resident in
device memory.  A 256 MiB buffer is written between timed steps to flush L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload knn|er_batch]

--workload er_batch times the batched factorization of 4,096 independent
Erdos-Renyi Laplacians (sizes 64..1024, core 16 each) held as one
block-diagonal matrix, next to the same matrices factored one call each.

--impl reference times the plain CPU oracle (the reference arm) on the host.
With N > 1 (torchrun) every rank factors its own replica: the factorization
of one matrix has no data-parallel split without an exchange step, so the job
scales by replicas (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pMMF factor time & nnz/s at stated Frobenius error; apply GB/s vs HBM peak"
UNIT = "nnz/s"
WORK = dict(n=65536, knn=10, gen_seed=1, k=2, eta=0.5, cluster_size=256, core_size=256, seed=0)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 rate (vector), used for ALU-bound kernels
NRHS_APPLY = 8


def workload_name(n):
    return (f"knn_laplacian n={n} (10-NN, 2-D uniform points, seed 1) + 1e-3 I, FP64 CSR; "
            f"k-means clusters ~{WORK['cluster_size']}, k=2 Givens, eta={WORK['eta']}, "
            f"core {WORK['core_size']}")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_run(a, runs=3):
    from oracle import oracle as O
    ts = []
    err = None
    for _ in range(runs):
        t0 = time.perf_counter()
        f = O.factor(a.n, a.rowptr, a.col, a.val, a.coords, k=WORK["k"], eta=WORK["eta"],
                     cluster_size=WORK["cluster_size"], core_size=WORK["core_size"], seed=WORK["seed"])
        ts.append(time.perf_counter() - t0)
        assert f.status == 0
        err = f.error
    return statistics.median(ts), err


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1507_04396_gb300 import inputs as I
    a = I.knn_laplacian(args.n, WORK["knn"], seed=WORK["gen_seed"])
    from oracle import oracle as O
    O.build()
    kw = dict(k=WORK["k"], eta=WORK["eta"], cluster_size=WORK["cluster_size"],
              core_size=WORK["core_size"], seed=WORK["seed"])
    for _ in range(args.warmup):
        O.factor(a.n, a.rowptr, a.col, a.val, a.coords, **kw)
    t0 = time.perf_counter()
    err = None
    for _ in range(args.steps):
        f = O.factor(a.n, a.rowptr, a.col, a.val, a.coords, **kw)
        err = f.error
    dt = time.perf_counter() - t0
    value = a.nnz * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(a.n), "n": a.n, "nnz": a.nnz,
                   "frobenius_error": err},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full workload, {args.steps} factorizations, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count(), model


def fp64_peak(stream):
    """Measured FP64 FMA throughput (TFLOP/s) of this GPU from the library's
    probe, else GB300's nominal rate."""
    from paper_1507_04396_gb300 import pmmf
    try:
        return pmmf.pmmf_probe_fp64(stream), "measured (pmmf_probe_fp64, FP64 FMA throughput)"
    except Exception:
        return FP64_NOMINAL_TFLOPS, "nominal FP64"


def roofline_of(dominant, prof, hbm, hbm_kind, f64, f64_kind):
    """Roofline object of one kernel family from its profiled launches."""
    if dominant in ("gram", "rows", "apply"):
        ach = prof["bytes"] / (prof["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel_family": dominant, "peak_kind": hbm_kind}
    else:
        ach = prof["flops"] / (prof["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": f64, "unit": "TFLOP/s", "frac": ach / f64,
                "traffic": None, "kernel_family": dominant, "peak_kind": f64_kind}
    roof["launches_profiled"] = prof["launches"]
    roof["avg_launch_ms"] = prof["ms"] / max(prof["launches"], 1)
    return roof


def poisson_extras(dev, stream, flush, hbm):
    """The 128^3 Poisson workload beside the headline: factor time, the
    blocked update's GB/s on its first two stages, the matrix-free A~^-1 x
    GB/s on 8 right-hand sides."""
    import torch
    from paper_1507_04396_gb300 import inputs as I, pmmf
    a = I.poisson3d(POISSON["nx"], seed=POISSON["gen_seed"])
    A = I.SymCSR(a.n, torch.from_numpy(a.rowptr).to(dev), torch.from_numpy(a.col).to(dev),
                 torch.from_numpy(a.val).to(dev))
    co = torch.from_numpy(a.coords).to(dev)
    nx = POISSON["nx"]
    bricks = torch.from_numpy(I.grid_bricks(nx, nx, nx, 8, 8, 4)).to(dev)
    kw = dict(k=POISSON["k"], eta=POISSON["eta"], cluster_size=POISSON["cluster_size"],
              core_size=POISSON["core_size"], seed=POISSON["seed"])
    fac = lambda **x: pmmf.factor(A, coords=co, labels=bricks, stream=stream, **dict(kw, **x))
    fac().close()
    ts = []
    for _ in range(3):
        ms, f = _timed(stream, fac, 1, flush)
        ts.append(ms)
        info = f.info()
        if _ < 2:
            f.close()
    # the blocked update's launches that carry >= 100 MB of algorithmic bytes
    # (the first two stages)
    pmmf.pmmf_profile_begin(["rows"])
    fac().close()
    recs = [r for r in pmmf.pmmf_profile_records() if r[0] == "rows" and r[2] >= 100e6]
    pmmf.pmmf_profile_end()
    rows = {"ms": sum(r[1] for r in recs), "bytes": sum(r[2] for r in recs), "launches": len(recs)}
    rows_gbs = rows["bytes"] / (rows["ms"] / 1e3) / 1e9 if rows["ms"] > 0 else 0.0
    x = torch.randn(a.n, POISSON["nrhs"], dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        f.apply(pmmf.OP_A_INV, x, y, stream)
    torch.cuda.synchronize()
    pmmf.pmmf_profile_begin(["apply"])
    for _ in range(10):
        f.apply(pmmf.OP_A_INV, x, y, stream)
    ap = pmmf.pmmf_profile_end()["apply"]
    f.close()
    apply_gbs = ap["bytes"] / (ap["ms"] / 1e3) / 1e9
    return {
        "workload": "poisson3d 128^3 (7-point FV, log-normal sigma=1, seed 4), FP64 CSR; stage 1: "
                    "8x8x4 grid bricks, then k-means clusters of 256; k=2, eta=0.5, core 1024",
        "n": a.n, "nnz": a.nnz, "stages": info.stages, "frobenius_error": info.error,
        "factor_ms": sorted(ts)[1], "nnz_per_s": a.nnz / (sorted(ts)[1] / 1e3),
        "update_launches_over_100MB": {"gbs": rows_gbs, "frac_of_hbm": rows_gbs / hbm,
                              "algorithmic_bytes": rows["bytes"], "ms": rows["ms"],
                              "launches": rows["launches"]},
        "apply_a_inv_8rhs": {"gbs": apply_gbs, "frac_of_hbm": apply_gbs / hbm,
                             "ms_per_apply": ap["ms"] / 10},
    }


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()

    a = I.knn_laplacian(args.n, WORK["knn"], seed=WORK["gen_seed"])
    kw = dict(k=WORK["k"], eta=WORK["eta"], cluster_size=WORK["cluster_size"],
              core_size=WORK["core_size"], seed=WORK["seed"])
    rp = torch.from_numpy(a.rowptr).to(dev)
    ci = torch.from_numpy(a.col).to(dev)
    va = torch.from_numpy(a.val).to(dev)
    co = torch.from_numpy(a.coords).to(dev)
    A = I.SymCSR(a.n, rp, ci, va)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def factor():
        return pmmf.factor(A, coords=co, stream=stream, **kw)

    for _ in range(max(args.warmup, 0)):
        factor().close()

    # timed region: the product path as shipped (no profiling hooks)
    clocks = Clocks(local)
    l0 = pmmf.pmmf_launch_count()
    total_ms = 0.0
    err = None
    info = None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = factor()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        info = f.info()
        err = info.error
        f.close()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = pmmf.pmmf_launch_count() - l0
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = a.nnz * args.steps * ws / (total_ms / 1e3)

    # per-kernel figures from a separate profiled pass (CUDA events around
    # every launch on its stream; the search's flop count needs a readback,
    # so this pass is slower than the timed one and is not the headline)
    prof_steps = 3
    pmmf.pmmf_profile_begin(pmmf.FAMILIES)
    for _ in range(prof_steps):
        flush.zero_()
        factor().close()
    breakdown = pmmf.pmmf_profile_end()
    dominant = max((f for f in breakdown if breakdown[f]["launches"] > 0),
                   key=lambda f: breakdown[f]["ms"])
    hbm, hbm_kind = peaks()
    f64, f64_kind = fp64_peak(stream)
    roof = roofline_of(dominant, breakdown[dominant], hbm, hbm_kind, f64, f64_kind)

    # matrix-free apply: y = U^T H U x on 8 right-hand sides
    f = factor()
    if dominant == "select":
        # DRAM bytes per launch of the rotation search, measured with ncu on
        # this workload's stage-2 launch: 157.6 MB = 1.158 x 16 B per Gram
        # entry (G and M streamed once, plus the prefetched rows of candidate
        # partners that were not chosen); scaled to every launch by its Gram
        # entries
        sq = [int((np.diff(f.clusters(p)[0]) ** 2).sum()) for p in range(f.info().stages)]
        roof["traffic"] = 1.158 * 16.0 * sum(sq) / max(len(sq), 1)
        roof["traffic_basis"] = ("ncu DRAM bytes of the stage-2 launch at n=65536 scaled by "
                                 "Gram entries per launch")
    x = torch.randn(a.n, NRHS_APPLY, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        f.apply(pmmf.OP_A, x, y, stream)
    torch.cuda.synchronize()
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        f.apply(pmmf.OP_A, x, y, stream)
    e1.record(stream)
    e1.synchronize()
    apply_ms = e0.elapsed_time(e1) / reps
    pmmf.pmmf_profile_begin(["apply"])
    for _ in range(reps):
        f.apply(pmmf.OP_A, x, y, stream)
    ap = pmmf.pmmf_profile_end()["apply"]
    apply_gbs = ap["bytes"] / (ap["ms"] / 1e3) / 1e9 if ap["ms"] > 0 else None
    f.close()

    # end to end through the C-ABI with host buffers (pinned), H diagonal read back
    hp = [torch.from_numpy(v).pin_memory() for v in (a.rowptr, a.col, a.val, a.coords)]
    Ah = I.SymCSR(a.n, hp[0], hp[1], hp[2])
    h2d = sum(t.numel() * t.element_size() for t in hp)
    hd = np.empty(a.n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g = pmmf.factor(Ah, coords=hp[3], stream=stream, **kw)
        hd[:] = g.h()[0]
        g.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": a.nnz * args.steps * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(hd.nbytes)}

    poisson = None
    if rank == 0 and not args.no_extras:
        poisson = poisson_extras(dev, stream, flush, hbm)

    cpu = cpu_omp = None
    oracle_err = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        from oracle import oracle as O
        O.build()
        t, oracle_err = cpu_oracle_run(a, runs=3)
        cores, model = host_cpu()
        cpu = {"value": a.nnz / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "full workload, median of 3 single-thread factorizations",
               "host_cores": cores, "cpu_model": model}
        r = O.time_factor_openmp(a.n, a.rowptr, a.col, a.val, a.coords, runs=3, **kw)
        if r is not None:
            tt, e_omp, threads = r
            cpu_omp = {"value": a.nnz / tt, "unit": UNIT, "cores": threads, "kind": "oracle (OpenMP)",
                       "sample": "full workload, median of 3 factorizations, clusters and rows "
                                 "spread over the host's cores",
                       "frobenius_error": e_omp, "host_cores": cores, "cpu_model": model}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a.n), "n": a.n, "nnz": a.nnz,
                       "stages": info.stages, "rotations": info.rotations,
                       "frobenius_error": err, "oracle_frobenius_error": oracle_err,
                       "l2": "256 MiB buffer written between timed steps",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "timed_region": "no profiling hooks; per-kernel figures from a separate "
                                       f"profiled pass of {prof_steps} factorizations"},
            "roofline": roof,
            "apply": {"op": "U^T H U x", "nrhs": NRHS_APPLY, "ms": apply_ms,
                      "rotation_pass_gbs": apply_gbs,
                      "frac_of_hbm": (apply_gbs / hbm) if apply_gbs else None},
            "kernel_breakdown_ms": {k: round(v["ms"] / prof_steps, 4)
                                    for k, v in breakdown.items() if v["launches"]},
            "poisson_128": poisson,
            "cpu_baseline": cpu, "cpu_baseline_openmp": cpu_omp, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


BATCH = dict(count=4096, lo=64, hi=1024, gen_seed=3, k=2, eta=0.5, core_size=16, seed=0)


def batch_name():
    return (f"er_laplacian batch: {BATCH['count']} Erdos-Renyi graphs (p = 8/n, weights U(0.5,1.5)) "
            f"+ 1e-3 I, sizes U[{BATCH['lo']},{BATCH['hi']}], seed {BATCH['gen_seed']}, FP64 CSR, "
            f"one block-diagonal matrix; one cluster per matrix, k=2 Givens, eta={BATCH['eta']}, "
            f"core {BATCH['core_size']} per matrix")


def batch_inputs():
    from paper_1507_04396_gb300 import inputs as I
    mats = I.er_laplacian_batch(BATCH["count"], BATCH["lo"], BATCH["hi"], seed=BATCH["gen_seed"])
    big, off = I.blockdiag(mats)
    return mats, big, off


def batch_oracle_sample(mats, stride):
    """Oracle on every stride-th matrix of the batch: (seconds, nnz, count)."""
    from oracle import oracle as O
    O.build()
    t, nnz, cnt = 0.0, 0, 0
    for b in range(0, len(mats), stride):
        m = mats[b]
        t0 = time.perf_counter()
        f = O.factor(m.n, m.rowptr, m.col, m.val, None, k=BATCH["k"], eta=BATCH["eta"],
                     cluster_size=max(m.n, 2), core_size=min(BATCH["core_size"], m.n),
                     seed=BATCH["seed"] + b)
        t += time.perf_counter() - t0
        assert f.status == 0
        nnz += m.nnz
        cnt += 1
    return t, nnz, cnt


def run_reference_batch(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    mats, big, off = batch_inputs()
    stride = 64
    batch_oracle_sample(mats[:1], 1)
    ts = []
    for _ in range(args.steps):
        t, nnz, cnt = batch_oracle_sample(mats, stride)
        ts.append(t)
    t = statistics.median(ts)
    value = nnz / t
    sample = f"every {stride}th matrix of the batch ({cnt} matrices, {nnz} nnz), single thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t * len(mats) / cnt,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": batch_name(), "n": big.n, "nnz": big.nnz},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu_batch(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    mats, big, off = batch_inputs()
    A = I.SymCSR(big.n, torch.from_numpy(big.rowptr).to(dev), torch.from_numpy(big.col).to(dev),
                 torch.from_numpy(big.val).to(dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kw = dict(k=BATCH["k"], eta=BATCH["eta"], core_size=BATCH["core_size"], seed=BATCH["seed"])

    def factor():
        return pmmf.factor_blockdiag(A, off, stream=stream, **kw)

    for _ in range(max(args.warmup, 0)):
        factor().close()
    pmmf.pmmf_profile_begin(pmmf.FAMILIES)
    factor().close()
    breakdown = pmmf.pmmf_profile_end()
    dominant = max((f for f in breakdown if breakdown[f]["launches"] > 0),
                   key=lambda f: breakdown[f]["ms"])

    clocks = Clocks(local)
    l0 = pmmf.pmmf_launch_count()
    total_ms = 0.0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    info = errs = None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = factor()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        info = f.info()
        errs = f.batch()["errors"]
        f.close()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = pmmf.pmmf_launch_count() - l0
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = big.nnz * args.steps * ws / (total_ms / 1e3)

    hbm, hbm_kind = peaks()
    f64, f64_kind = fp64_peak(stream)
    roof = roofline_of(dominant, breakdown[dominant], hbm, hbm_kind, f64, f64_kind)

    # the same matrices factored one pmmf_factor call each (per-matrix launches),
    # on every 16th matrix of the batch
    stride = 16
    singles = [(b, I.SymCSR(mats[b].n, torch.from_numpy(mats[b].rowptr).to(dev),
                            torch.from_numpy(mats[b].col).to(dev), torch.from_numpy(mats[b].val).to(dev)))
               for b in range(0, len(mats), stride)]
    for b, m in singles[:4]:
        pmmf.factor(m, coords=None, cluster_size=max(m.n, 2), stream=stream,
                    **dict(kw, seed=BATCH["seed"] + b)).close()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for b, m in singles:
        pmmf.factor(m, coords=None, cluster_size=max(m.n, 2), stream=stream,
                    **dict(kw, seed=BATCH["seed"] + b)).close()
    e1.record(stream)
    e1.synchronize()
    single_ms = e0.elapsed_time(e1)
    single_nnz = sum(mats[b].nnz for b, _ in singles)
    per_matrix = {"value": single_nnz / (single_ms / 1e3), "unit": UNIT,
                  "sample": f"every {stride}th matrix ({len(singles)} matrices), one pmmf_factor each"}

    # end to end: pinned host CSR in, H diagonal out
    hp = [torch.from_numpy(v).pin_memory() for v in (big.rowptr, big.col, big.val)]
    Ah = I.SymCSR(big.n, hp[0], hp[1], hp[2])
    h2d = sum(t.numel() * t.element_size() for t in hp)
    hd = np.empty(big.n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g = pmmf.factor_blockdiag(Ah, off, stream=stream, **kw)
        g.hdiag(hd)
        g.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": big.nnz * args.steps * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(hd.nbytes)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        t, nnz, cnt = batch_oracle_sample(mats, 64)
        cpu = {"value": nnz / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"every 64th matrix of the batch ({cnt} matrices), single thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batch_name(), "n": big.n, "nnz": big.nnz, "matrices": len(mats),
                       "stages": info.stages, "rotations": info.rotations,
                       "frobenius_error": info.error,
                       "matrix_error_max": float(np.max(errs)),
                       "l2": "256 MiB buffer written between timed steps",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roof,
            "per_matrix_launches": per_matrix,
            "batched_vs_per_matrix": value / per_matrix["value"],
            "kernel_breakdown_ms": {k: round(v["ms"], 4) for k, v in breakdown.items() if v["launches"]},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


RBF = dict(n=16384, components=20, gen_seed=2, k=3, eta=0.5, cluster_size=512, core_size=512, seed=0)
POISSON = dict(nx=128, gen_seed=4, k=2, eta=0.5, cluster_size=256, core_size=1024, seed=0, nrhs=8,
               rtol=1e-8)
PREC = {"fp64": 0, "tf32": 1, "bf16": 2}


def _timed(stream, fn, steps, flush):
    """Run fn() steps times with an L2 flush before each, CUDA events on stream."""
    import torch
    total, out = 0.0, None
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
        if hasattr(out, "close") and _ < steps - 1:
            out.close()
    return total, out


def tf32_peak(dev):
    """Measured TF32 tensor throughput (TFLOP/s): cuBLAS FP32 GEMM with TF32
    allowed, 8192^3, best of 5 after warm-up (CUDA events)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device=dev)
        b = torch.randn(n, n, device=dev)
        for _ in range(3):
            a @ b
        best = None
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return 2.0 * n ** 3 / (best / 1e3) / 1e12, "measured tf32 (cuBLAS FP32 GEMM, TF32 allowed)"
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def run_gpu_rbf(args):
    """Dense Gaussian RBF kernel (3-D mixture), k = 3, clusters of 512: the
    dense path in FP64 and, with --precision, the tensor-core Gram shortlist."""
    import numpy as np
    import torch
    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    dev = torch.device("cuda", 0)
    n = args.n if args.n != WORK["n"] else RBF["n"]
    a = I.rbf_mixture(n, RBF["components"], seed=RBF["gen_seed"])
    D = torch.from_numpy(a.to_dense()).to(dev)
    co = torch.from_numpy(a.coords).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kw = dict(k=RBF["k"], eta=RBF["eta"], cluster_size=RBF["cluster_size"],
              core_size=RBF["core_size"], seed=RBF["seed"])
    prec = PREC[args.precision]

    def run(p):
        return lambda: pmmf.factor(D, coords=co, precision=p, stream=stream, **kw)

    for _ in range(max(args.warmup, 0)):
        run(prec)().close()
    pmmf.pmmf_profile_begin(pmmf.FAMILIES)
    run(prec)().close()
    recs = [r for r in pmmf.pmmf_profile_records() if r[0] == "gram"]
    breakdown = pmmf.pmmf_profile_end()
    gram = breakdown["gram"]
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    l0 = pmmf.pmmf_launch_count()
    ms, f = _timed(stream, run(prec), args.steps, flush)
    launches = pmmf.pmmf_launch_count() - l0
    clk = clocks.stop()
    info, st = f.info(), f.precision_stats()
    rots = [f.rotations(p) for p in range(info.stages)]
    f.close()
    ref = None
    if prec != 0:
        # the FP64 mode on the same input: time and identical selections
        run(0)().close()
        ms64, g = _timed(stream, run(0), 1, flush)
        same = sum(int((r[2] == q[2]).all(axis=1).sum()) for r, q in
                   zip(rots, [g.rotations(p) for p in range(g.info().stages)]))
        ref = {"fp64_ms_per_step": ms64, "fp64_frobenius_error": g.info().error,
               "identical_tuples": same, "rotations": info.rotations}
        g.close()
    value = n * n * args.steps / (ms / 1e3)
    if prec != 0 and st["steps"] > 0:
        if prec == 1:
            pk, pk_kind = tf32_peak(dev)
        else:
            pk = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]) \
                if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
            pk_kind = "measured bf16 (cuBLAS)"
        # the first stage's Gram is the tensor-core split product (stages with
        # fewer clusters take the FP64 Gram)
        r0 = recs[0] if recs else ("gram", gram["ms"], 0.0, gram["flops"])
        ach = r0[3] / (r0[1] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": None, "kernel_family": "gram (tensor-core split product, stage 1)",
                "peak_kind": pk_kind}
    else:
        # FP64 mode, or a reduced-precision mode whose stages all had fewer
        # clusters than the shortlist threshold (every Gram in FP64)
        f64, f64_kind = fp64_peak(stream)
        ach = gram["flops"] / (gram["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": f64, "unit": "TFLOP/s",
                "frac": ach / f64, "traffic": None, "kernel_family": "gram (FP64)",
                "peak_kind": f64_kind}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else f"f64 + {args.precision} Gram",
        "data": "synthetic",
        "config": {"workload": f"rbf_mixture n={n} (20-component 3-D Gaussian mixture, seed 2), dense "
                               f"FP64 Gaussian kernel, sigma = median distance; k-means clusters of 512, "
                               f"k=3, eta=0.5, core 512", "n": n, "nnz": n * n,
                   "stages": info.stages, "rotations": info.rotations, "frobenius_error": info.error,
                   "precision": args.precision, "l2": "256 MiB buffer written between timed steps"},
        "roofline": roof, "shortlist": st, "fp64_mode": ref,
        "kernel_breakdown_ms": {k: round(v["ms"], 3) for k, v in breakdown.items() if v["launches"]},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def run_gpu_poisson(args):
    """3-D variable-coefficient Poisson (log-normal, 128^3), pMMF as the PCG
    preconditioner for 8 right-hand sides to 1e-8."""
    import numpy as np
    import torch
    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    dev = torch.device("cuda", 0)
    nx = args.nx
    a = I.poisson3d(nx, seed=POISSON["gen_seed"])
    A = I.SymCSR(a.n, torch.from_numpy(a.rowptr).to(dev), torch.from_numpy(a.col).to(dev),
                 torch.from_numpy(a.val).to(dev))
    co = torch.from_numpy(a.coords).to(dev)
    bricks = torch.from_numpy(I.grid_bricks(nx, nx, nx, 8, 8, 4)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kw = dict(k=POISSON["k"], eta=POISSON["eta"], cluster_size=POISSON["cluster_size"],
              core_size=POISSON["core_size"], seed=POISSON["seed"])
    fac = lambda: pmmf.factor(A, coords=co, labels=bricks, stream=stream, **kw)
    for _ in range(max(args.warmup, 0)):
        fac().close()
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    l0 = pmmf.pmmf_launch_count()
    ms, f = _timed(stream, fac, args.steps, flush)
    rng = np.random.default_rng(POISSON["gen_seed"])
    rng.standard_normal(a.n)
    b = torch.from_numpy(rng.standard_normal((a.n, POISSON["nrhs"]))).to(dev)
    f.solve(A, b, rtol=POISSON["rtol"], maxit=3000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, x, iters, relres = f.solve(A, b, rtol=POISSON["rtol"], maxit=3000)
    torch.cuda.synchronize()
    pcg_s = time.perf_counter() - t0
    launches = pmmf.pmmf_launch_count() - l0
    xx = torch.randn(a.n, POISSON["nrhs"], dtype=torch.float64, device=dev)
    yy = torch.empty_like(xx)
    # xi = 1/2: forming core^{-1/2} (first request), then the split-system CG
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f.apply(pmmf.OP_A_INV_SQRT, xx, yy)
    torch.cuda.synchronize()
    isqrt_s = time.perf_counter() - t0
    f.solve(A, b, rtol=POISSON["rtol"], maxit=3000, xi=0.5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st2, x2, iters2, relres2 = f.solve(A, b, rtol=POISSON["rtol"], maxit=3000, xi=0.5)
    torch.cuda.synchronize()
    sym_s = time.perf_counter() - t0
    for _ in range(3):
        f.apply(pmmf.OP_A_INV, xx, yy)
    pmmf.pmmf_profile_begin(["apply"])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        f.apply(pmmf.OP_A_INV, xx, yy)
    e1.record(stream)
    e1.synchronize()
    ap = pmmf.pmmf_profile_end()["apply"]
    clk = clocks.stop()
    info = f.info()
    hbm, hbm_kind = peaks()
    ach = ap["bytes"] / (ap["ms"] / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": a.nnz * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"poisson3d {nx}^3 (7-point FV, log-normal sigma=1, seed 4), FP64 CSR; "
                               f"stage 1: 8x8x4 grid bricks ({nx ** 3 // 256:,} clusters), then k-means "
                               "clusters of 256 on cell centres; k=2, eta=0.5, core 1024",
                   "n": a.n, "nnz": a.nnz, "stages": info.stages, "frobenius_error": info.error,
                   "l2": "256 MiB buffer written between timed steps"},
        "pcg": {"nrhs": POISSON["nrhs"], "rtol": POISSON["rtol"], "status": st, "seconds": pcg_s,
                "iterations": [int(v) for v in iters], "max_relres": float(np.max(relres))},
        "pcg_xi_half": {"status": st2, "seconds": sym_s, "core_isqrt_seconds": isqrt_s,
                        "iterations": [int(v) for v in iters2],
                        "max_relres": float(np.max(relres2))},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "kernel_family": "apply (rotation passes of A~^-1 x, 8 RHS)",
                     "peak_kind": hbm_kind},
        "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line))
    f.close()
    return 0


def run_gpu_scaling(args):
    """Factor time against input size (the linear-scaling claim): kNN Laplacians
    of 2^14 .. 2^20 points, clusters of 256, core 256, median of 3 runs each."""
    import numpy as np
    import torch
    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rows = []
    for lg in range(14, 21):
        n = 1 << lg
        a = I.knn_laplacian(n, WORK["knn"], seed=WORK["gen_seed"])
        A = I.SymCSR(a.n, torch.from_numpy(a.rowptr).to(dev), torch.from_numpy(a.col).to(dev),
                     torch.from_numpy(a.val).to(dev))
        co = torch.from_numpy(a.coords).to(dev)
        kw = dict(k=2, eta=0.5, cluster_size=256, core_size=256, seed=0)
        fac = lambda: pmmf.factor(A, coords=co, stream=stream, **kw)
        fac().close()
        ts = []
        for _ in range(3):
            ms, f = _timed(stream, fac, 1, flush)
            ts.append(ms)
            err = f.info().error
            f.close()
        ms = sorted(ts)[1]
        rows.append({"n": n, "nnz": a.nnz, "ms": round(ms, 3), "nnz_per_s": a.nnz / (ms / 1e3),
                     "error": err})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    # least-squares slope of log(time) against log(nnz) over the four largest sizes
    x = np.log([r["nnz"] for r in rows[-4:]])
    y = np.log([r["ms"] for r in rows[-4:]])
    slope = float(np.polyfit(x, y, 1)[0])
    big = rows[-1]
    line = {"metric": METRIC, "value": big["nnz_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 3,
            "warmup": 1, "ms_per_step": big["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "knn_laplacian n = 2^14 .. 2^20 (10-NN, 2-D uniform points, seed 1), "
                                   "clusters ~256, k=2, eta=0.5, core 256; median of 3 per size",
                       "log_log_slope_time_vs_nnz": slope},
            "sizes": rows}
    print(json.dumps(line))
    return 0


def run_gpu_quality(args):
    """Compression quality against core size: ||A - A~||_F / ||A - A_r||_F with
    A_r the best rank-r approximation (r = core size), on a kNN Laplacian and a
    dense RBF kernel matrix (eigenvalues by numpy on the host)."""
    import numpy as np
    import torch
    from paper_1507_04396_gb300 import build, inputs as I, pmmf
    build.build()
    pmmf.load()
    dev = torch.device("cuda", 0)
    cases = [("knn_laplacian n=4096 (10-NN), clusters 256, k=2",
              I.knn_laplacian(4096, 10, seed=1), dict(k=2, cluster_size=256)),
             ("rbf_mixture n=2048 (dense), clusters 256, k=3",
              I.rbf_mixture(2048, 20, seed=2), dict(k=3, cluster_size=256))]
    out = []
    for name, a, kw in cases:
        dense = a.to_dense()
        ev = np.linalg.eigvalsh(dense)
        order = np.sort(np.abs(ev))[::-1]
        nrm = float(np.sqrt(np.sum(ev ** 2)))
        for core in (64, 128, 256, 512):
            f = pmmf.factor(torch.from_numpy(dense).to(dev) if kw["k"] == 3 else a, coords=a.coords,
                            eta=0.5, core_size=core, seed=0, **kw)
            e = f.info().error
            f.close()
            best = float(np.sqrt(np.sum(order[core:] ** 2))) / nrm
            out.append({"matrix": name, "core": core, "pmmf_rel_error": e,
                        "best_rank_r_rel_error": best, "ratio": e / best if best > 0 else None})
            print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    line = {"metric": "||A - A~||_F / ||A - A_r||_F against core size", "value": out[-1]["ratio"],
            "unit": "ratio", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "compression quality"},
            "results": out}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=WORK["n"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 128^3 Poisson figures beside the headline")
    ap.add_argument("--workload", choices=["knn", "er_batch", "rbf_dense", "poisson", "scaling",
                                           "quality"],
                    default="knn",
                    help="knn: the kNN Laplacian (default); er_batch: 4,096 independent ER "
                         "Laplacians factored as one batch; rbf_dense: dense RBF kernel, k = 3; "
                         "poisson: 128^3 Poisson factorization and PCG")
    ap.add_argument("--precision", choices=list(PREC), default="fp64",
                    help="Gram precision of the rbf_dense workload")
    ap.add_argument("--nx", type=int, default=POISSON["nx"],
                    help="grid edge of the poisson workload (a multiple of 8)")
    ap.add_argument("--tune", action="append", default=[], metavar="NAME=VALUE",
                    help="library knob for every cluster size, e.g. dense_tiles=1 (repeatable)")
    args = ap.parse_args()
    if args.nx <= 0 or args.nx % 8:
        ap.error("--nx must be a positive multiple of 8")
    if args.tune and args.impl == "gpu":
        from paper_1507_04396_gb300 import build, pmmf
        build.build()
        for kv in args.tune:
            name, _, value = kv.partition("=")
            if name not in pmmf.TUNE_PARAMS or not value.lstrip("-").isdigit():
                ap.error(f"--tune {kv}: expected one of {sorted(pmmf.TUNE_PARAMS)}=<int>")
            pmmf.set_tuning(name, int(value))
    if args.workload == "rbf_dense":
        return run_gpu_rbf(args)
    if args.workload == "scaling":
        return run_gpu_scaling(args)
    if args.workload == "quality":
        return run_gpu_quality(args)
    if args.workload == "poisson":
        return run_gpu_poisson(args)
    if args.workload == "er_batch":
        return run_reference_batch(args) if args.impl == "reference" else run_gpu_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
