#!/usr/bin/env python3
"""Benchmark of the isoperimetric clustering hot path on GB300.

One step = one call of isoclust_cluster on the 100,000-point, d = 64
anisotropic-blob workload (FP32 storage, k = 20, sigma = 1): minimum spanning
tree, vertex weights, tree orientation, the bisection of Algorithm 2 and the
labels.  Inputs are resident in HBM; L2 is flushed (a 256 MiB write) before
every step inside the timed region.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload blobs_n100k_d64|sparse_n50k_d4096|batched_4096_d32|moons_n20k_d128]

--workload sparse_n50k_d4096 times the same call on 50,000 sparse-like rows
of 4,096 features (L2-normalised log-normal values at 1 % density, 10
groups, k = 10), where the sweep's Gram tiles dominate the MST stage.

--workload batched_4096_d32 times isoclust_cluster_batched on 4,096
independent sets (sizes log-uniform in [64, 8192], d = 32, 2-8 blobs each,
k = blob count): one step = one call over all sets.  --workload
moons_n20k_d128 times the differentiable path on 20,000 interleaved-moons
points in 128 dimensions (k = 3): one step = the scaled forward call plus
the FP64 backward of i_k in X, the per-feature scale and sigma.

N > 1 (torchrun, one rank per GPU): every rank clusters its own independent
point set (replicas; the path has no cross-GPU exchange), value = total
points over the slowest rank's time.  --impl reference times the FP64 CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "points/s end-to-end"
UNIT = "points/s"
WORKLOAD = "blobs_n100k_d64"
SPARSE = "sparse_n50k_d4096"
BATCHED = "batched_4096_d32"
MOONS = "moons_n20k_d128"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) of one full-size launch of the roofline kernel,
# measured by a one-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel as it stands; other workloads report null
OMEGA_TRAFFIC = {"blobs_n100k_d64": 51293952 + 242455808}
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def _oracle_time(X, k, sigma, n_sample, threads):
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    Xs = np.ascontiguousarray(X[:n_sample])
    t0 = time.perf_counter()
    oracle.cluster(Xs, k, sigma)
    return time.perf_counter() - t0


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _sample_rows(d, base=30000):
    """Oracle sample size: about the cost of 30,000 points at d = 64 (the
    path costs n^2 d)."""
    return int(max(2000, min(base, base * (64.0 / max(d, 1)) ** 0.5)))


def cpu_baseline(X, k, sigma, n_sample=None):
    """The oracle as it stands, on a bounded sample, scaled to full n by the
    O(n^2) cost of the path (all pairs for omega, Prim's n min-reductions)."""
    n = X.shape[0]
    if n_sample is None:
        n_sample = _sample_rows(X.shape[1])
    n_sample = min(n_sample, n)
    cores = _cpu_cores()
    t = _oracle_time(X, k, sigma, n_sample, cores)
    t_full = t * (n / n_sample) ** 2
    return {"value": n / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample} of the {n} points (full pipeline: Prim MST, omega, Algorithms 1-2) took "
                      f"{t:.2f} s on {cores} threads; value = n / (t * (n/{n_sample})^2), the O(n^2) cost law"}


def run_reference(args, X, k, sigma):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps_total = args.steps + args.warmup
    n = X.shape[0]
    n_sample = min(n, int(max(2000, _sample_rows(X.shape[1]) * min(1.0, (8.0 / max(steps_total, 1)) ** 0.5))))
    cores = _cpu_cores()
    for _ in range(args.warmup):
        _oracle_time(X, k, sigma, n_sample, cores)
    times = [_oracle_time(X, k, sigma, n_sample, cores) for _ in range(args.steps)]
    t = sum(times) / len(times)
    value = n / (t * (n / n_sample) ** 2)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1000.0 * (n / n_sample) ** 2,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "d": X.shape[1], "k": k, "sigma": sigma},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: oracle on the first {n_sample} points, {t:.2f} s mean; "
                                   f"scaled to n={n} by the O(n^2) cost law"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mst-compare", action="store_true")
    ap.add_argument("--n", type=int, default=0,
                    help="points of the same generator (profiling of a smaller case); default: the full 100,000")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, SPARSE, BATCHED, MOONS])
    ap.add_argument("--nsets", type=int, default=0, help="batched: fewer sets of the same recipe (profiling)")
    ap.add_argument("--sweep-variant", type=int, default=-1,
                    help="force the MST sweep's tile variant 0..3 (profiling: a profiler distorts the autotuner's "
                         "trial timings); -1 = the library's own choice")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.workload == BATCHED:
        return main_batched(args)
    if args.workload == MOONS:
        return main_moons(args)

    from paper_1702_04739_gb300 import workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    X, k, sigma = workloads.make(args.workload, seed=rank)
    if args.n:
        X = workloads.blobs_anisotropic(seed=rank, n=args.n)[0] if args.workload == WORKLOAD else X[:args.n]
    if args.impl == "reference":
        return run_reference(args, X, k, sigma)

    import torch
    from paper_1702_04739_gb300 import isoclust
    torch.cuda.set_device(local_rank)
    isoclust.set_sweep_variant(args.sweep_variant)
    dev = torch.device("cuda", local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    residual = torch.empty(n, dtype=torch.uint8, device=dev)
    ik = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        flush.zero_()
        isoclust.cluster_into(Xd, k, sigma, labels, residual, ik)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if pg is not None:
            pg.barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    prof = []
    barrier()
    torch.cuda.synchronize(dev)
    l0 = isoclust.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        prof.append(isoclust.last_profile())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = isoclust.kernel_launches() - l0
    clk = clocks.stop()
    sweep_variant = isoclust.last_sweep_variant()
    t_ms = ev0.elapsed_time(ev1)
    if pg is not None:
        tt = torch.tensor([t_ms], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_ms = float(tt.item())
    ms_per_step = t_ms / args.steps
    value = world * n / (ms_per_step / 1000.0)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        lh = torch.empty(n, dtype=torch.int32).pin_memory()
        rh = torch.empty(n, dtype=torch.uint8).pin_memory()
        ih = torch.empty(1, dtype=torch.float64).pin_memory()

        def e2e_step():
            flush.zero_()
            Xd.copy_(Xh, non_blocking=True)
            isoclust.cluster_into(Xd, k, sigma, labels, residual, ik)
            lh.copy_(labels, non_blocking=True)
            rh.copy_(residual, non_blocking=True)
            ih.copy_(ik, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        te = e0.elapsed_time(e1)
        if pg is not None:
            tt = torch.tensor([te], device=dev)
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": world * n / (te / args.steps / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(n * 4 + n + 8)}

    # roofline of the dominant kernel: the screened double-word omega sweep
    peaks, src = _peaks()
    # the kernel's own CUDA-event time (the omega stage time when it was not
    # the symmetric kernel)
    w_ms = statistics.mean(p["omega_kernel_ms"] or p["weights_ms"] for p in prof)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12   # T instr/s
    tiles, tiles_dw = prof[-1]["omega_tiles"], prof[-1]["omega_tiles_dw"]
    sym = prof[-1]["omega_symmetric"]
    # FP32 screen of one pair (both directions if sym); none when the tensor
    # cores screened the tile pairs (sym == 2)
    screen_ops = 0.0 if sym == 2 else 2.0 * d + (12.0 if sym else 8.0)
    # d2 (18.75/dim in the symmetric sweep: renormalised every 4 dimensions;
    # 21/dim in the ordered one), then sqrt and one double-word exp per pair,
    # accumulated in one direction (ordered sweep) or both (symmetric sweep)
    dw_ops = (18.75 * d + 95.0) if sym else (21.0 * d + 75.0)
    work = tiles * 4096.0 * screen_ops + tiles_dw * 4096.0 * dw_ops
    achieved = work / (w_ms / 1000.0) / 1e12
    # MST stage: tensor-core work and the BF16 + FP64-recheck path against the FP32 SIMT path
    mst_ms = statistics.mean(p["mst_ms"] for p in prof)
    rounds = prof[-1]["boruvka_rounds"]
    n_pad = -(-n // 128) * 128
    d_pad = -(-d // 64) * 64
    alg_flop = rounds * 2.0 * n * n * d                  # one Gram term per round over all ordered pairs
    exe_flop = rounds * 3 * 2.0 * n_pad * n_pad * d_pad  # hi.hi + hi.lo + lo.hi MMAs as issued
    mst_cmp = None
    if not args.no_mst_compare:
        ref_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_BF16_TC))
        t_tc = isoclust.last_profile()["mst_ms"]
        fp_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_FP32))
        t_fp = isoclust.last_profile()["mst_ms"]
        same = all(torch.equal(a, b) for a, b in zip(ref_edges, fp_edges))
        mst_cmp = {"bf16_tc_fp64_recheck_ms": t_tc, "fp32_simt_fp64_recheck_ms": t_fp,
                   "speedup_vs_fp32": t_fp / t_tc if t_tc > 0 else None, "identical_edges": bool(same)}
    mst = {"stage_ms": mst_ms, "rounds": rounds, "sweep_variant": sweep_variant,
           "algorithmic_tflops": alg_flop / (mst_ms / 1000.0) / 1e12,
           "executed_tensor_tflops": exe_flop / (mst_ms / 1000.0) / 1e12,
           "peak_bf16_tflops": peaks.get("bf16_tflops"), "peak_source": src,
           "frac_executed_of_peak": exe_flop / (mst_ms / 1000.0) / 1e12 / peaks.get("bf16_tflops", 1900.0),
           "note": "stage time includes the FP64 recheck and union-find; algorithmic = rounds x 2 n^2 d"}
    if mst_cmp:
        mst["compare"] = mst_cmp
    stages = {key: round(statistics.mean(p[key] for p in prof), 3)
              for key in ("validate_ms", "weights_ms", "mst_ms", "orient_ms", "search_ms", "labels_ms")}
    counts = {key: prof[-1][key] for key in ("boruvka_rounds", "rescanned_rows", "alg1_passes", "tree_depth")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "d": d, "k": k, "sigma": sigma, "storage": "f32",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed by a 256 MiB write before every step (inside the timed region)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak,
                     "traffic": OMEGA_TRAFFIC.get(args.workload) if (sym and not args.n) else None,
                     "kernel": "k_weights_sym (omega, double-word FP32)" if sym else "k_weights_dw (omega, double-word FP32)",
                     "note": f"FP32-pipe instructions of the algorithm: every {'unordered' if sym else 'ordered'} "
                             f"pair of the 64x64 tile grid screened ("
                             f"{'on the tensor cores' if sym == 2 else 'in FP32, %.0f each' % screen_ops}, {tiles} tiles), "
                             f"double-word evaluation ({dw_ops:.0f} per pair) of the {tiles_dw} tiles the screen "
                             f"keeps; over the kernel's CUDA-event time ({w_ms:.2f} ms, launch on the call's stream); "
                             f"peak = {sms} SMs x {FP32_LANES_PER_SM} lanes x max SM clock ({src} sm_max_mhz)"},
        "stages_ms": stages, "counts": counts, "mst": mst,
        "omega_tiles": {"screened": prof[-1]["omega_tiles"], "double_word": prof[-1]["omega_tiles_dw"]},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X, k, sigma)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------- independent sets
def _oracle_sets_time(X, offs, ks, sigma, sets, threads):
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    for b in sets:
        oracle.cluster(np.ascontiguousarray(X[offs[b]:offs[b + 1]]), int(ks[b]), sigma)
    return time.perf_counter() - t0


def _sets_sample(offs, budget_pairs=1.5e9):
    """The first sets whose n^2 sum stays within the budget (about 10-30 s of
    oracle work on 16 cores)."""
    sizes = np.diff(offs).astype(np.float64)
    c = np.cumsum(sizes ** 2)
    m = int(np.searchsorted(c, budget_pairs)) + 1
    return list(range(min(m, sizes.size)))


def _sets_cpu(X, offs, ks, sigma, steps=1, warmup=0):
    sizes = np.diff(offs).astype(np.float64)
    sets = _sets_sample(offs)
    cores = _cpu_cores()
    for _ in range(warmup):
        _oracle_sets_time(X, offs, ks, sigma, sets, cores)
    t = statistics.mean(_oracle_sets_time(X, offs, ks, sigma, sets, cores) for _ in range(max(steps, 1)))
    scale = float((sizes ** 2).sum() / (sizes[sets] ** 2).sum())
    value = float(offs[-1]) / (t * scale)
    return value, t, scale, sets, cores


def main_batched(args):
    from paper_1702_04739_gb300 import workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    X, offs, ks, sigma = workloads.make_batched(BATCHED, seed=rank, nsets=args.nsets or None)
    N, d = X.shape
    nsets = ks.size
    cfg = {"workload": BATCHED, "nsets": int(nsets), "points": int(N), "d": int(d), "sigma": sigma,
           "sizes": "log-uniform in [64, 8192]", "k": "blob count (2-8)", "storage": "f32"}
    if args.impl == "reference":
        if rank != 0:
            return 0
        value, t, scale, sets, cores = _sets_cpu(X, offs, ks, sigma, args.steps, args.warmup)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * scale * 1000.0,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"each step: oracle on the first {len(sets)} sets, {t:.2f} s mean; "
                                           f"scaled to all {nsets} sets by their n^2 sum (x{scale:.1f})"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    from paper_1702_04739_gb300 import isoclust
    torch.cuda.set_device(local_rank)
    isoclust.set_sweep_variant(args.sweep_variant)
    dev = torch.device("cuda", local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    plan = isoclust.BatchPlan(offs, ks)
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    residual = torch.empty(N, dtype=torch.uint8, device=dev)
    ik = torch.empty(nsets, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        flush.zero_()
        isoclust.cluster_batched_into(Xd, plan, sigma, labels, residual, ik)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    prof = []
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize(dev)
    l0 = isoclust.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        prof.append(isoclust.last_profile())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg is not None:
        pg.barrier()
    launches = isoclust.kernel_launches() - l0
    clk = clocks.stop()
    sweep_variant = isoclust.last_sweep_variant()
    t_ms = ev0.elapsed_time(ev1)
    if pg is not None:
        tt = torch.tensor([t_ms], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_ms = float(tt.item())
    ms_per_step = t_ms / args.steps
    value = world * N / (ms_per_step / 1000.0)

    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        lh = torch.empty(N, dtype=torch.int32).pin_memory()
        rh = torch.empty(N, dtype=torch.uint8).pin_memory()
        ih = torch.empty(nsets, dtype=torch.float64).pin_memory()

        def e2e_step():
            flush.zero_()
            Xd.copy_(Xh, non_blocking=True)
            isoclust.cluster_batched_into(Xd, plan, sigma, labels, residual, ik)
            lh.copy_(labels, non_blocking=True)
            rh.copy_(residual, non_blocking=True)
            ih.copy_(ik, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        te = e0.elapsed_time(e1)
        e2e = {"value": world * N / (te / args.steps / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(N * 5 + nsets * 8)}

    peaks, src = _peaks()
    w_ms = statistics.mean(p["omega_kernel_ms"] or p["weights_ms"] for p in prof)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * FP32_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    tiles, tiles_dw = prof[-1]["omega_tiles"], prof[-1]["omega_tiles_dw"]
    # independent sets: the tile bound is the only screen (no FP32 pair screen
    # runs), so only the double-word pass counts
    dw_ops = 18.75 * d + 95.0
    work = tiles_dw * 4096.0 * dw_ops
    achieved = work / (w_ms / 1000.0) / 1e12
    sizes = np.diff(offs)
    rounds = prof[-1]["boruvka_rounds"]
    mst_ms = statistics.mean(p["mst_ms"] for p in prof)
    pad128 = -(-sizes // 128) * 128
    exe_flop = rounds * 3 * 2.0 * float((pad128.astype(np.float64) ** 2).sum()) * (-(-d // 64) * 64)
    stages = {key: round(statistics.mean(p[key] for p in prof), 3)
              for key in ("validate_ms", "weights_ms", "mst_ms", "orient_ms", "search_ms", "labels_ms")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(cfg, parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       l2="flushed by a 256 MiB write before every step (inside the timed region)"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "kernel": "k_weights_sym (omega over the sets' tile pairs, double-word FP32)",
                     "note": f"FP32-pipe instructions of the algorithm ({dw_ops:.0f} per double-word pair; "
                             f"{tiles} tile pairs within the sets' tile bound, all {tiles_dw} taken to the double-word "
                             f"pass without a pair screen) "
                             f"over the kernel's CUDA-event time ({w_ms:.2f} ms); peak = {sms} SMs x {FP32_LANES_PER_SM} lanes x "
                             f"max SM clock ({src})"},
        "stages_ms": stages,
        "mst": {"stage_ms": mst_ms, "rounds": rounds, "sweep_variant": sweep_variant,
                "executed_tensor_tflops": exe_flop / (mst_ms / 1000.0) / 1e12,
                "peak_bf16_tflops": peaks.get("bf16_tflops"), "peak_source": src},
        "omega_tiles": {"screened": tiles, "double_word": tiles_dw},
        "gpu_launches": int(launches), "clocks": clk,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if rank == 0 and not args.no_cpu_baseline:
        value_c, t, scale, sets, cores = _sets_cpu(X, offs, ks, sigma)
        line["cpu_baseline"] = {"value": value_c, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"oracle on the first {len(sets)} sets took {t:.2f} s on {cores} threads; "
                                          f"scaled to all {nsets} sets by their n^2 sum (x{scale:.1f})"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------- differentiation
def _moons_cpu(X, k, sigma, n_sample=12000):
    """Oracle forward + FP64 gradient on the first n_sample points, scaled to
    n by the O(n^2) cost of both."""
    import oracle
    oracle.build()
    cores = _cpu_cores()
    oracle.set_threads(cores)
    Xs = np.ascontiguousarray(X[:n_sample]).astype(np.float64)
    s = np.ones(X.shape[1])
    t0 = time.perf_counter()
    f = oracle.cluster(Xs * s, k, sigma)
    fx = oracle.ik_fixed(Xs, s, sigma, f["parent"], f["labels"], k)
    oracle.ik_grad(Xs, s, sigma, f["parent"], f["labels"], fx["jstar"])
    t = time.perf_counter() - t0
    scale = (X.shape[0] / n_sample) ** 2
    return X.shape[0] / (t * scale), t, cores, n_sample


def main_moons(args):
    from paper_1702_04739_gb300 import workloads
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    X, k, sigma = workloads.make(MOONS, seed=rank)
    n, d = X.shape
    cfg = {"workload": MOONS, "n": n, "d": d, "k": k, "sigma": sigma, "storage": "f32",
           "gradient": "FP64, d i_k / d(X, scale, sigma) through the fixed tree and subpartition"}
    if args.impl == "reference":
        if rank != 0:
            return 0
        vals = [_moons_cpu(X, k, sigma) for _ in range(max(args.steps, 1))]
        value = statistics.mean(v[0] for v in vals)
        t, cores, ns = vals[-1][1], vals[-1][2], vals[-1][3]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": 0, "ms_per_step": n / value * 1000.0, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"forward + gradient on the first {ns} points, {t:.2f} s; scaled by (n/{ns})^2"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    import torch
    from paper_1702_04739_gb300 import isoclust
    torch.cuda.set_device(local_rank)
    isoclust.set_sweep_variant(args.sweep_variant)
    dev = torch.device("cuda", local_rank)
    Xd = torch.from_numpy(X).to(dev)
    sd = torch.ones(d, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    times = {}

    def step():
        flush.zero_()
        Z = isoclust.scale_features(Xd, sd)
        out = isoclust.cluster_detail(Z, k, sigma)
        times["fwd"] = isoclust.last_profile()
        g = isoclust.ik_backward(Xd, sd, sigma, out["parent"], out["labels"], k, out["phi_par"], out["omega"], 1.0)
        pb = isoclust.last_profile()
        times["bwd_ms"] = pb["search_ms"]
        times["pair_ms"] = pb["omega_kernel_ms"]
        return out, g

    for _ in range(args.warmup):
        out, g = step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = isoclust.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    bwd, pair = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        out, g = step()
        bwd.append(times["bwd_ms"])
        pair.append(times["pair_ms"])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = isoclust.kernel_launches() - l0
    clk = clocks.stop()
    ms_per_step = ev0.elapsed_time(ev1) / args.steps
    value = world * n / (ms_per_step / 1000.0)

    e2e = None
    if not args.no_e2e:
        # the same step from pinned host memory: H2D of X, forward + backward,
        # D2H of labels, i_k and the FP64 gradient (dX, dscale, dsigma)
        Xh = torch.from_numpy(X).pin_memory()
        Xe = torch.empty_like(Xd)
        lh = torch.empty(n, dtype=torch.int32).pin_memory()
        gh = torch.empty((n, d), dtype=torch.float64).pin_memory()
        sh = torch.empty(d + 2, dtype=torch.float64).pin_memory()

        def e2e_step():
            flush.zero_()
            Xe.copy_(Xh, non_blocking=True)
            Z = isoclust.scale_features(Xe, sd)
            o = isoclust.cluster_detail(Z, k, sigma)
            ge = isoclust.ik_backward(Xe, sd, sigma, o["parent"], o["labels"], k, o["phi_par"], o["omega"], 1.0)
            lh.copy_(o["labels"], non_blocking=True)
            gh.copy_(ge["dX"], non_blocking=True)
            sh[:d].copy_(ge["dscale"], non_blocking=True)
            sh[d:d + 1].copy_(ge["dsigma"], non_blocking=True)
            sh[d + 1:].copy_(o["i_k"], non_blocking=True)
        e2e_step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        te = e0.elapsed_time(e1)
        e2e = {"value": world * n / (te / args.steps / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(X.nbytes),
               "d2h_bytes_per_step": int(lh.numel() * 4 + gh.numel() * 8 + sh.numel() * 8)}
    # work of the pair kernel: |A*| n + (n - |A*|) |A*| ordered pairs, each a
    # d-long dot product and a d-long accumulation in double-word FP32 (12
    # FP32-pipe instructions per step) and the pair's coefficient (norms,
    # root, reciprocal, exp, products: ~115 double-word FP32 instructions)
    lab = out["labels"].cpu().numpy()
    par = out["parent"].cpu().numpy()
    phi = out["phi_par"].cpu().numpy()
    om = out["omega"].cpu().numpy()
    ratios = []
    for j in range(k):
        inj = lab == j
        cross = (par >= 0) & (inj != inj[np.maximum(par, 0)])
        ratios.append(phi[cross].sum() / om[inj].sum())
    a = int((lab == int(np.argmax(ratios))).sum())
    pairs = a * n + (n - a) * a
    ops = pairs * (24.0 * d + 115.0)
    b_ms = statistics.mean(bwd)
    k_ms = statistics.mean(pair)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, src = _peaks()
    alu_peak = sms * FP32_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 forward, f64 gradient", "data": "synthetic",
        "config": dict(cfg, l2="flushed by a 256 MiB write before every step (inside the timed region)"),
        "roofline": {"bound": "alu", "achieved": ops / (k_ms / 1000.0) / 1e12, "peak": alu_peak,
                     "unit": "TFLOP/s", "frac": ops / (k_ms / 1000.0) / 1e12 / alu_peak, "traffic": None,
                     "kernel": "k_pair_grad (backward pair sums, double-word FP32)",
                     "note": f"{pairs} ordered pairs (|A*| = {a}) x (24 d + 115) FP32-pipe instructions (two "
                             f"d-long double-word sums and the pair's coefficient) over the kernel's CUDA-event "
                             f"time ({k_ms:.2f} ms of the backward's {b_ms:.2f} ms); peak = {sms} SMs x "
                             f"{FP32_LANES_PER_SM} lanes x max SM clock ({src})"},
        "stages_ms": {"forward_ms": round(sum(times["fwd"][key] for key in ("validate_ms", "weights_ms", "mst_ms",
                                                                          "orient_ms", "search_ms", "labels_ms")), 3),
                      "backward_ms": round(b_ms, 3)},
        "gpu_launches": int(launches), "clocks": clk, "e2e": e2e,
        "mst_sweep_variant": isoclust.last_sweep_variant(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, t, cores, ns = _moons_cpu(X, k, sigma)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"oracle forward + FP64 gradient on the first {ns} points took {t:.2f} s "
                                          f"on {cores} threads; scaled by (n/{ns})^2"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
