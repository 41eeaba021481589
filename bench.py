#!/usr/bin/env python3
"""Benchmark of the isoperimetric clustering hot path on GB300.

One step = one call of isoclust_cluster on the 100,000-point, d = 64
anisotropic-blob workload (FP32 storage, k = 20, sigma = 1): minimum spanning
tree, vertex weights, tree orientation, the bisection of Algorithm 2 and the
labels.  Inputs are resident in HBM; L2 is flushed (a 256 MiB write) before
every step inside the timed region.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload blobs_n100k_d64|sparse_n50k_d4096|batched_4096_d32|moons_n20k_d128]

The default line also carries, under "workloads", the other three benchmark
workloads measured the same way with fewer steps (--extra-steps):
  sparse_n50k_d4096  50,000 sparse-like rows of 4,096 features (L2-normalised
                     log-normal values at 1 % density, 10 groups, k = 10),
                     where the sweep's Gram tiles dominate the MST stage;
  batched_4096_d32   isoclust_cluster_batched on 4,096 independent sets (sizes
                     log-uniform in [64, 8192], d = 32, 2-8 blobs each, k =
                     blob count): one step = one call over all sets;
  moons_n20k_d128    the differentiable path on 20,000 interleaved-moons points
                     in 128 dimensions (k = 3): one step = the scaled forward
                     call plus the FP64 backward of i_k in X, scale and sigma.
--workload selects one of them as the headline instead.

cpu_baseline (rank 0 at N = 1) runs the FP64 CPU oracle once on the whole
workload on the host cores (about a minute for the default workload on 16
cores) and compares the GPU's result with it ("parity": edges, parent and
labels bit for bit, the largest omega / i_k errors, the decision margin).
--impl reference times that same oracle run as the reference arm (one step).

N > 1 (torchrun, one rank per GPU): every rank clusters its own independent
point set (replicas; the path's units shard with no exchange), value = total
points over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
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
L2_NOTE = "flushed by a 256 MiB write before every step (inside the timed region)"
# DRAM bytes (read + write) of one full-size launch of the symmetric omega
# kernel as it stands, from a one-pass ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum); workloads without a capture report null
OMEGA_TRAFFIC: dict[str, int] = {}
# DRAM bytes per unit of the two omega kernels with the Gram on the tensor cores, from their
# full-section capture at 40,000 x 64 (profiles/k_weights_sym_gram_k_oz_gram_blobs_n40k_d64.md):
# the sweep 1.504621 + 0.045260 GB over 42,831 kept 64 x 64 tile pairs (their 32 KB Gram tiles,
# mostly), the Gram kernel 0.236092 + 1.348661 GB over 22,524 blocks of 128 x 64 (its G written).
# Both grow with those units at this row length; other row lengths read other plane and row
# bytes, so the line's traffic is null there.
OMEGA_GRAM_TRAFFIC_D = 64
OMEGA_SWEEP_BYTES_PER_TILE_PAIR = (1.504621e9 + 0.045260e9) / 42831
OMEGA_GRAM_BYTES_PER_BLOCK = (0.236092e9 + 1.348661e9) / 22524
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64, nominal (context for the FP64-equivalent rate)


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

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


# ---------------------------------------------------------------- timing
class Timer:
    """CUDA events on the launching stream around K steps, after W warm-ups,
    with a synchronize (and a barrier across ranks) on both sides."""

    def __init__(self, torch, dev, pg=None):
        self.torch, self.dev, self.pg = torch, dev, pg

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def run(self, step, steps, warmup, after=None):
        torch = self.torch
        for _ in range(warmup):
            step()
        torch.cuda.synchronize(self.dev)
        stream = torch.cuda.current_stream(self.dev)
        clocks = ClockSampler(self.dev.index or 0).start()
        self.barrier()
        torch.cuda.synchronize(self.dev)
        from paper_1702_04739_gb300 import isoclust
        l0 = isoclust.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
            if after:
                after()
        e1.record(stream)
        torch.cuda.synchronize(self.dev)
        self.barrier()
        launches = isoclust.kernel_launches() - l0
        clk = clocks.stop()
        t_ms = e0.elapsed_time(e1)
        if self.pg is not None:
            tt = torch.tensor([t_ms], device=self.dev)
            self.pg.all_reduce(tt, op=self.pg.ReduceOp.MAX)
            t_ms = float(tt.item())
        return t_ms / steps, int(launches), clk


def _alu_peak(torch, dev, peaks):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms, sms * FP32_LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def _stages(prof):
    return {key: round(statistics.mean(p[key] for p in prof), 3)
            for key in ("validate_ms", "weights_ms", "mst_ms", "orient_ms", "search_ms", "labels_ms")}


def omega_roofline(torch, dev, prof, n_pairs_alg, d, workload, sets=False):
    """Roofline of the symmetric omega kernel (the dominant kernel).

    Primary: FP32-pipe instructions of the algorithm as built (double-word
    FP32, the fastest FP64-grade arithmetic on this chip) per evaluated tile
    pair, over the kernel's CUDA-event time, against 152 SMs x 128 lanes x
    the max SM clock.  Beside it, the method's own work: n(n-1)/2 pairs x
    (2d + 25) FP64-equivalent flop per launch, over the same time; there is
    no measured peak in that unit (native FP64 is nominally 1.25 TFLOP/s)."""
    peaks, src = _peaks()
    sms, alu_peak = _alu_peak(torch, dev, peaks)
    w_ms = statistics.mean(p["omega_kernel_ms"] or p["weights_ms"] for p in prof)
    tiles, tiles_dw, sym = prof[-1]["omega_tiles"], prof[-1]["omega_tiles_dw"], prof[-1]["omega_symmetric"]
    alg_flop = n_pairs_alg * (2.0 * d + 25.0)
    if sym == 3:
        return omega_gram_roofline(prof, peaks, src, alu_peak, sms, w_ms, tiles_dw, d, alg_flop)
    screen_ops = 0.0 if (sym == 2 or sets) else 2.0 * d + (12.0 if sym else 8.0)
    dw_ops = (18.75 * d + 95.0) if (sym or sets) else (21.0 * d + 75.0)
    work = tiles * 4096.0 * screen_ops + tiles_dw * 4096.0 * dw_ops
    achieved = work / (w_ms / 1000.0) / 1e12
    alg = alg_flop / (w_ms / 1000.0) / 1e12
    return {
        "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
        "traffic": OMEGA_TRAFFIC.get(workload),
        "kernel": "k_weights_sym (omega, double-word FP32)",
        "kernel_ms": w_ms,
        "note": f"FP32-pipe instructions of the algorithm as built: {dw_ops:.0f} per double-word pair for the "
                f"{tiles_dw} 64x64 tile pairs evaluated (of {tiles} "
                f"{'within the sets tile bound' if sets else 'screened on the tensor cores' if sym == 2 else 'screened'}"
                f"{'' if screen_ops == 0 else ', plus %.0f per screened pair' % screen_ops}), over the kernel's "
                f"CUDA-event time ({w_ms:.2f} ms); peak = {sms} SMs x {FP32_LANES_PER_SM} lanes x max SM clock "
                f"({src} sm_max_mhz); 'unit' counts FP32-pipe instructions",
        "algorithmic": {"achieved": alg, "unit": "FP64-equivalent TFLOP/s", "peak": None,
                        "flop_per_launch": alg_flop,
                        "note": f"the method's work: {n_pairs_alg:.4g} pairs x (2d + 25) FP64-equivalent flop (eq. "
                                f"omega over all pairs) per launch over the same time; no measured peak exists in "
                                f"this unit (native FP64 is {FP64_NOMINAL_TFLOPS} TFLOP/s nominal, "
                                f"{alg / FP64_NOMINAL_TFLOPS:.1f}x of it)"},
    }


def omega_gram_roofline(prof, peaks, src, alu_peak, sms, sweep_ms, items, d, alg_flop):
    """omega with the Gram on the tensor cores: two kernels.  The Gram kernel
    (tensor-bound: 34 BF16 digit-plane products of 2 x 128 x 64 x d_pad
    flop per 128 x 64 block, executed) and the sweep that reads it
    (ALU-bound, FP32-pipe instructions of the algorithm as built: per pair of
    a kept 64 x 64 tile pair 155 (d2 from G and the parts' size 40, root and
    Newton correction 25, shift 20, double-word exp 50, two accumulations
    20); per off-diagonal tile pair with tile centres (d < 1024) 128 cross
    terms of 14 d and |D|^2 of 12 d; per pair that took the direct sum
    18.75 d + 60).  The line's roofline is the slower of the two."""
    g_ms = statistics.mean(p["omega_gram_ms"] for p in prof)
    blocks = prof[-1]["omega_gram_blocks"]
    d_pad = -(-d // 64) * 64
    tc_flop = blocks * 34 * 2.0 * 128 * 64 * d_pad
    bf16 = peaks.get("bf16_tflops", 1900.0)
    tc = tc_flop / (g_ms / 1000.0) / 1e12 if g_ms > 0 else 0.0
    direct = prof[-1].get("omega_gram_direct_pairs", 0)
    cross = 0.0 if d >= 1024 else items * (128.0 * 14.0 * d + 12.0 * d)
    sw_ops = items * 4096.0 * 155.0 + cross + direct * (18.75 * d + 60.0)
    sw = sw_ops / (sweep_ms / 1000.0) / 1e12 if sweep_ms > 0 else 0.0
    scaled = d == OMEGA_GRAM_TRAFFIC_D
    gram_k = {"kernel": "k_oz_gram (omega Gram, tcgen05 BF16 digit planes)", "bound": "tensor", "kernel_ms": g_ms,
              "achieved": tc, "peak": bf16, "unit": "TFLOP/s", "frac": tc / bf16, "blocks": blocks,
              "traffic": blocks * OMEGA_GRAM_BYTES_PER_BLOCK if scaled else None}
    sweep_k = {"kernel": "k_weights_sym<GRAM> (omega terms from the Gram, double-word FP32)", "bound": "alu",
               "kernel_ms": sweep_ms, "achieved": sw, "peak": alu_peak, "unit": "TFLOP/s", "frac": sw / alu_peak,
               "direct_pairs": direct, "direct_share": direct / max(1.0, items * 4096.0),
               "traffic": items * OMEGA_SWEEP_BYTES_PER_TILE_PAIR if scaled else None}
    top, other = (gram_k, sweep_k) if g_ms >= sweep_ms else (sweep_k, gram_k)
    both_ms = g_ms + sweep_ms
    alg = alg_flop / (both_ms / 1000.0) / 1e12
    out = dict(top,
               traffic_note=("DRAM bytes per launch: the 40,000 x 64 full-section capture's bytes per kept tile pair "
                             "(sweep) or per block (Gram), times this launch's count" if scaled else
                             "no capture at this row length"),
               note=f"omega's Gram on the tensor cores: the Gram kernel {g_ms:.2f} ms ({blocks} blocks of 128 x 64, 34 "
                    f"digit-plane MMAs per 16 dimensions, executed flop over the measured BF16 peak, {src}) and the "
                    f"sweep reading it {sweep_ms:.2f} ms (FP32-pipe instructions of the algorithm as built - 155 per "
                    f"pair, cross terms {'none: one centre' if d >= 1024 else '128 x 14 d per tile pair'}, "
                    f"18.75 d + 60 per direct pair - over "
                    f"{sms} SMs x 128 lanes x max SM clock); the line reports the slower one",
               other_kernel=other,
               algorithmic={"achieved": alg, "unit": "FP64-equivalent TFLOP/s", "peak": None,
                            "flop_per_launch": alg_flop,
                            "note": "the method's work (eq. omega over all pairs, (2d + 25) FP64-equivalent flop each) "
                                    "over both kernels' time; no measured peak exists in this unit"})
    return out


def mst_summary(prof, n_pairs_alg, pad_pairs_exe, d, sweep_variant):
    """MST stage: the brute-force Boruvka Gram work (n(n-1)/2 pairs x 2d
    flop per round) and the tensor-core MMAs as issued (3 BF16 products over
    the 128 x 128 tile pairs actually swept: all of them per round without
    pruning), both against the measured BF16 peak."""
    peaks, src = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    mst_ms = statistics.mean(p["mst_ms"] for p in prof)
    rounds = prof[-1]["boruvka_rounds"]
    d_pad = -(-d // 64) * 64
    swept, full = prof[-1].get("mst_tiles_swept", 0), prof[-1].get("mst_tiles_full", 0)
    tile_pairs = swept if full else rounds * pad_pairs_exe / (128.0 * 128.0)
    alg = rounds * n_pairs_alg * 2.0 * d / (mst_ms / 1000.0) / 1e12
    exe = 3 * 2.0 * tile_pairs * 128.0 * 128.0 * d_pad / (mst_ms / 1000.0) / 1e12
    return {"stage_ms": mst_ms, "rounds": rounds, "sweep_variant": sweep_variant,
            "tile_pairs_swept": swept, "tile_pairs_full": full,
            "swept_share": (swept / full) if full else None,
            "algorithmic_tflops": alg, "frac_algorithmic_of_peak": alg / peak,
            "executed_tensor_tflops": exe, "frac_executed_of_peak": exe / peak,
            "peak_bf16_tflops": peak, "peak_source": src,
            "note": "stage time includes the row order, the FP64 recheck and union-find; algorithmic = rounds x "
                    "n(n-1)/2 x 2d (brute-force Boruvka: pruned rounds skip tile pairs that cannot hold a "
                    "component's lightest edge, so this rate can exceed the peak); executed = 3 MMAs (hi.hi, "
                    "hi.lo, lo.hi) x 2 x 128 x 128 x padded d per 128 x 128 tile pair swept"}


# ---------------------------------------------------------------- GPU measurements
def measure_single(torch, dev, X, k, sigma, workload, steps, warmup, pg=None, world=1, e2e=True,
                   mst_compare=True, want_detail=True):
    from paper_1702_04739_gb300 import isoclust
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    residual = torch.empty(n, dtype=torch.uint8, device=dev)
    ik = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    prof = []

    def step():
        flush.zero_()
        isoclust.cluster_into(Xd, k, sigma, labels, residual, ik)

    T = Timer(torch, dev, pg)
    ms, launches, clk = T.run(step, steps, warmup, after=lambda: prof.append(isoclust.last_profile()))
    sweep_variant = isoclust.last_sweep_variant()
    out = {"ms_per_step": ms, "value": world * n / (ms / 1000.0), "steps": steps, "warmup": warmup,
           "gpu_launches": launches, "clocks": clk}
    if e2e:
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
        te, _, _ = T.run(e2e_step, steps, 1)
        out["e2e"] = {"value": world * n / (te / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
                      "d2h_bytes_per_step": int(n * 4 + n + 8)}
    pairs = n * (n - 1) / 2.0
    out["roofline"] = omega_roofline(torch, dev, prof, pairs, d, workload)
    n_pad = -(-n // 128) * 128
    out["mst"] = mst_summary(prof, pairs, float(n_pad) * n_pad, d, sweep_variant)
    if mst_compare:
        ref_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_BF16_TC))
        t_tc = isoclust.last_profile()["mst_ms"]
        fp_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_FP32))
        t_fp = isoclust.last_profile()["mst_ms"]
        same = all(torch.equal(a, b) for a, b in zip(ref_edges, fp_edges))
        isoclust.set_mst_prune(0)
        full_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_BF16_TC))
        full_edges = isoclust.cluster_mst(Xd, isoclust.opts(precision=isoclust.PREC_BF16_TC))
        t_full = isoclust.last_profile()["mst_ms"]
        isoclust.set_mst_prune(-1)
        same_full = all(torch.equal(a, b) for a, b in zip(ref_edges, full_edges))
        out["mst"]["compare"] = {"bf16_tc_fp64_recheck_ms": t_tc, "fp32_simt_fp64_recheck_ms": t_fp,
                                 "speedup_vs_fp32": t_fp / t_tc if t_tc > 0 else None, "identical_edges": bool(same),
                                 "every_tile_pair_ms": t_full, "identical_to_every_tile_pair": bool(same_full)}
    out["stages_ms"] = _stages(prof)
    out["counts"] = {key: prof[-1][key] for key in ("boruvka_rounds", "rescanned_rows", "alg1_passes", "tree_depth")}
    out["omega_tiles"] = {"screened": prof[-1]["omega_tiles"], "double_word": prof[-1]["omega_tiles_dw"]}
    detail = None
    if want_detail:
        detail = {key: v.cpu().numpy() for key, v in isoclust.cluster_detail(Xd, k, sigma).items()}
    del Xd, flush
    return out, detail


def measure_batched(torch, dev, X, offs, ks, sigma, steps, warmup, pg=None, world=1, e2e=True, want_detail=True):
    from paper_1702_04739_gb300 import isoclust
    N, d = X.shape
    nsets = ks.size
    plan = isoclust.BatchPlan(offs, ks)
    Xd = torch.from_numpy(X).to(dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    residual = torch.empty(N, dtype=torch.uint8, device=dev)
    ik = torch.empty(nsets, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    prof = []

    def step():
        flush.zero_()
        isoclust.cluster_batched_into(Xd, plan, sigma, labels, residual, ik)

    T = Timer(torch, dev, pg)
    ms, launches, clk = T.run(step, steps, warmup, after=lambda: prof.append(isoclust.last_profile()))
    out = {"ms_per_step": ms, "value": world * N / (ms / 1000.0), "steps": steps, "warmup": warmup,
           "gpu_launches": launches, "clocks": clk, "graph_mode": isoclust.last_batched_graph_mode()}
    if e2e:
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
        te, _, _ = T.run(e2e_step, steps, 1)
        out["e2e"] = {"value": world * N / (te / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
                      "d2h_bytes_per_step": int(N * 5 + nsets * 8)}
    sizes = np.diff(offs).astype(np.float64)
    pairs = float((sizes * (sizes - 1) / 2).sum())
    out["roofline"] = omega_roofline(torch, dev, prof, pairs, d, BATCHED, sets=True)
    pad = -(-sizes // 128) * 128
    out["mst"] = mst_summary(prof, pairs, float((pad ** 2).sum()), d, isoclust.last_sweep_variant())
    out["stages_ms"] = _stages(prof)
    detail = None
    if want_detail:
        res = isoclust.cluster_batched(Xd, offs, ks, sigma)
        detail = {"labels": res["labels"].cpu().numpy(), "i_k": res["i_k"].cpu().numpy()}
    del Xd, flush
    return out, detail


def measure_moons(torch, dev, X, k, sigma, steps, warmup, world=1, e2e=True):
    from paper_1702_04739_gb300 import isoclust
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    sd = torch.ones(d, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    state = {}
    fwd, bwd, pair = [], [], []

    def step():
        flush.zero_()
        Z = isoclust.scale_features(Xd, sd)
        o = isoclust.cluster_detail(Z, k, sigma)
        state["fwd"] = isoclust.last_profile()
        g = isoclust.ik_backward(Xd, sd, sigma, o["parent"], o["labels"], k, o["phi_par"], o["omega"], 1.0)
        state["bwd"] = isoclust.last_profile()
        state["out"], state["g"] = o, g

    def after():
        fwd.append(state["fwd"])
        bwd.append(state["bwd"]["search_ms"])
        pair.append(state["bwd"]["omega_kernel_ms"])

    T = Timer(torch, dev)
    ms, launches, clk = T.run(step, steps, warmup, after=after)
    out = {"ms_per_step": ms, "value": world * n / (ms / 1000.0), "steps": steps, "warmup": warmup,
           "gpu_launches": launches, "clocks": clk}
    if e2e:
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
        te, _, _ = T.run(e2e_step, steps, 1)
        out["e2e"] = {"value": world * n / (te / 1000.0), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
                      "d2h_bytes_per_step": int(lh.numel() * 4 + gh.numel() * 8 + sh.numel() * 8)}
    # the backward's pair kernel: |A*| n + (n - |A*|) |A*| ordered pairs, each
    # two d-long double-word sums (12 FP32-pipe instructions per step) and the
    # pair's coefficient (~115)
    o = {key: v.cpu().numpy() for key, v in state["out"].items()}
    ratios = []
    for j in range(k):
        inj = o["labels"] == j
        cross = (o["parent"] >= 0) & (inj != inj[np.maximum(o["parent"], 0)])
        ratios.append(o["phi_par"][cross].sum() / o["omega"][inj].sum())
    a = int((o["labels"] == int(np.argmax(ratios))).sum())
    pairs = a * n + (n - a) * a
    ops = pairs * (24.0 * d + 115.0)
    k_ms = statistics.mean(pair)
    peaks, src = _peaks()
    sms, alu_peak = _alu_peak(torch, dev, peaks)
    out["roofline"] = {
        "bound": "alu", "achieved": ops / (k_ms / 1000.0) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
        "frac": ops / (k_ms / 1000.0) / 1e12 / alu_peak, "traffic": None,
        "kernel": "k_pair_grad (backward pair sums, double-word FP32)", "kernel_ms": k_ms,
        "note": f"{pairs} ordered pairs (|A*| = {a}) x (24 d + 115) FP32-pipe instructions (two d-long double-word "
                f"sums and the pair's coefficient) over the kernel's CUDA-event time ({k_ms:.2f} ms of the "
                f"backward's {statistics.mean(bwd):.2f} ms); peak = {sms} SMs x {FP32_LANES_PER_SM} lanes x max SM "
                f"clock ({src})"}
    fw = _stages(fwd)
    out["stages_ms"] = {"forward_ms": round(sum(fw.values()), 3), "backward_ms": round(statistics.mean(bwd), 3),
                        "forward_stages_ms": fw}
    out["mst_sweep_variant"] = isoclust.last_sweep_variant()
    detail = dict(o, dX=state["g"]["dX"].cpu().numpy(), dscale=state["g"]["dscale"].cpu().numpy(),
                  dsigma=float(state["g"]["dsigma"].cpu()[0]))
    del Xd, flush
    return out, detail


# ---------------------------------------------------------------- the oracle (CPU baseline / reference arm)
def _oracle():
    import oracle
    oracle.build()
    oracle.set_threads(_cpu_cores())
    return oracle


def oracle_single(X, k, sigma):
    """One full oracle run on the whole workload: (result, seconds)."""
    orc = _oracle()
    t0 = time.perf_counter()
    r = orc.cluster(X, k, sigma)
    return r, time.perf_counter() - t0


def oracle_single_sampled(X, k, sigma, n_sample):
    """The oracle on the first n_sample points (workloads whose full oracle
    run takes tens of minutes): (seconds, n_sample)."""
    orc = _oracle()
    Xs = np.ascontiguousarray(X[:n_sample])
    t0 = time.perf_counter()
    orc.cluster(Xs, k, sigma)
    return time.perf_counter() - t0


def oracle_sets(X, offs, ks, sigma):
    orc = _oracle()
    t0 = time.perf_counter()
    res = [orc.cluster(np.ascontiguousarray(X[offs[b]:offs[b + 1]]), int(ks[b]), sigma) for b in range(ks.size)]
    return res, time.perf_counter() - t0


def oracle_moons(X, k, sigma):
    orc = _oracle()
    s = np.ones(X.shape[1])
    t0 = time.perf_counter()
    f = orc.cluster(X, k, sigma)
    fx = orc.ik_fixed(X, s, sigma, f["parent"], f["labels"], k)
    g = orc.ik_grad(X, s, sigma, f["parent"], f["labels"], fx["jstar"])
    return f, g, time.perf_counter() - t0


def _omega_bound(n, d, eu, ev, ed2, sigma):
    nn = np.full(n, np.inf)
    np.minimum.at(nn, eu, ed2)
    np.minimum.at(nn, ev, ed2)
    return 2.0 ** -45 * max(1.0, math.sqrt(d / 64.0)) * (np.sqrt(nn) / sigma + 4.0)


def parity_single(r, g, X, k, sigma):
    """The GPU's result g against the oracle's r on the same input."""
    orc = _oracle()
    n, d = X.shape
    rel = np.abs(g["omega"] - r["omega"]) / r["omega"]
    bound = _omega_bound(n, d, r["edge_u"], r["edge_v"], r["edge_d2"], sigma)
    det = orc.decision_detail(r["parent"], r["phi_par"], r["omega"], None, k, r["beta"])
    vis = det["code"] >= 0
    beta = r["beta"]
    margin, at_beta = None, 0
    if beta > 0:
        m = np.minimum(np.abs(det["ncut"][vis] - beta), np.abs(det["njoin"][vis] - beta)) / beta
        at_beta = int((m <= 1e-15).sum())
        margin = float(m[m > 1e-15].min()) if (m > 1e-15).any() else None
    nz = r["parent"] >= 0
    return {
        "edges_identical": bool((g["edge_u"] == r["edge_u"]).all() and (g["edge_v"] == r["edge_v"]).all()
                                and (g["edge_d2"] == r["edge_d2"]).all()),
        "parent_identical": bool((g["parent"] == r["parent"]).all()),
        "labels_identical": bool((g["labels"] == r["labels"]).all()),
        "i_k_rel_err": abs(float(g["i_k"][0]) - r["i_k"]) / r["i_k"] if r["i_k"] else abs(float(g["i_k"][0])),
        "beta_rel_err": abs(float(g["beta"][0]) - beta) / beta if beta else abs(float(g["beta"][0])),
        "phi_max_rel_err": float((np.abs(g["phi_par"][nz] - r["phi_par"][nz]) / r["phi_par"][nz]).max()),
        "omega_max_rel_err": float(rel.max()),
        "omega_max_share_of_bound": float((rel / bound).max()),
        "decision_margin": margin, "decisions_at_beta": at_beta,
        "note": "omega bound per row 2^-45 max(1, sqrt(d/64)) (y_nn + 4); decision margin = smallest "
                "|N_crit - beta| / beta over Algorithm 1's decisions before its k-th cut, apart from those at beta",
    }


def parity_sets(res, g):
    ik_o = np.array([r["i_k"] for r in res])
    same = all((g["labels"][a:a + r["labels"].size] == r["labels"]).all()
               for a, r in zip(np.concatenate([[0], np.cumsum([r["labels"].size for r in res])[:-1]]), res))
    return {"labels_identical_all_sets": bool(same),
            "i_k_max_rel_err": float((np.abs(g["i_k"] - ik_o) / ik_o).max())}


def parity_moons(f, gr, g):
    return {"labels_identical": bool((g["labels"] == f["labels"]).all()),
            "parent_identical": bool((g["parent"] == f["parent"]).all()),
            "i_k_rel_err": abs(float(g["i_k"][0]) - f["i_k"]) / f["i_k"],
            "dX_max_err_rel_to_max": float(np.abs(g["dX"] - gr["dX"]).max() / np.abs(gr["dX"]).max()),
            "dscale_max_err_rel_to_max": float(np.abs(g["dscale"] - gr["dscale"]).max()
                                               / np.abs(gr["dscale"]).max()),
            "dsigma_rel_err": abs(g["dsigma"] - gr["dsigma"]) / abs(gr["dsigma"])}


SPARSE_SAMPLE = 6000


def cpu_baseline(workload, data, k, sigma, gpu_detail):
    """The oracle as it stands on the host cores, once on the whole workload
    (the sparse-like workload: a stated sample, its full run taking tens of
    minutes), and the GPU's result compared with it."""
    cores = _cpu_cores()
    if workload == BATCHED:
        X, offs, ks = data
        res, t = oracle_sets(X, offs, ks, sigma)
        cb = {"value": X.shape[0] / t, "unit": UNIT, "cores": cores, "kind": "oracle",
              "sample": f"the whole workload: the oracle on each of the {ks.size} sets (Prim MST, omega, "
                        f"Algorithms 1-2) took {t:.1f} s on {cores} threads, measured, not scaled"}
        return cb, (parity_sets(res, gpu_detail) if gpu_detail is not None else None)
    X = data
    n = X.shape[0]
    if workload == MOONS:
        f, gr, t = oracle_moons(X, k, sigma)
        cb = {"value": n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
              "sample": f"the whole workload: oracle forward (Prim MST, omega, Algorithms 1-2) and FP64 gradient "
                        f"took {t:.1f} s on {cores} threads, measured, not scaled"}
        return cb, (parity_moons(f, gr, gpu_detail) if gpu_detail is not None else None)
    if workload == SPARSE:
        ns = min(SPARSE_SAMPLE, n)
        t = oracle_single_sampled(X, k, sigma, ns)
        cb = {"value": n / (t * (n / ns) ** 2), "unit": UNIT, "cores": cores, "kind": "oracle",
              "sample": f"first {ns} of the {n} points took {t:.1f} s on {cores} threads; value = n / (t (n/{ns})^2), "
                        f"the path's O(n^2) cost (the full run takes tens of minutes; its result is the stored "
                        f"full-size golden the parity tests use)"}
        return cb, None
    r, t = oracle_single(X, k, sigma)
    cb = {"value": n / t, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": f"the whole workload: one oracle run (Prim MST, omega, Algorithms 1-2) took {t:.1f} s on "
                    f"{cores} threads, measured, not scaled"}
    return cb, (parity_single(r, gpu_detail, X, k, sigma) if gpu_detail is not None else None)


def load_workload(name, seed=0, n=0, nsets=0):
    from paper_1702_04739_gb300 import workloads
    if name == BATCHED:
        X, offs, ks, sigma = workloads.make_batched(BATCHED, seed=seed, nsets=nsets or None)
        return (X, offs, ks), None, sigma
    X, k, sigma = workloads.make(name, seed=seed)
    if n:
        X = workloads.blobs_anisotropic(seed=seed, n=n)[0] if name == WORKLOAD else np.ascontiguousarray(X[:n])
    return X, k, sigma


def config_of(name, data, k, sigma, world):
    par = f"replicas x{world}" if world > 1 else "single GPU"
    if name == BATCHED:
        X, offs, ks = data
        return {"workload": BATCHED, "nsets": int(ks.size), "points": int(X.shape[0]), "d": int(X.shape[1]),
                "sigma": sigma, "sizes": "log-uniform in [64, 8192]", "k": "blob count (2-8)", "storage": "f32",
                "parallelism": par, "l2": L2_NOTE}
    c = {"workload": name, "n": int(data.shape[0]), "d": int(data.shape[1]), "k": k, "sigma": sigma,
         "storage": "f64" if data.dtype == np.float64 else "f32", "parallelism": par, "l2": L2_NOTE}
    if name == MOONS:
        c["gradient"] = "FP64, d i_k / d(X, scale, sigma) through the fixed tree and subpartition"
    return c


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, one step = one
    oracle run on the whole workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    data, k, sigma = load_workload(args.workload, n=args.n, nsets=args.nsets)
    cb, _ = cpu_baseline(args.workload, data, k, sigma, None)
    n = data[0].shape[0] if args.workload == BATCHED else data.shape[0]
    value = cb["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": n / value * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, data, k, sigma, 1),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": f"one oracle run (requested --steps {args.steps} --warmup {args.warmup}): a run on the whole "
                f"workload takes about a minute or more, so it is timed once and not repeated"
                + ("; the sparse-like workload times a stated sample (see cpu_baseline)" if args.workload == SPARSE
                   else ""),
    }
    print(json.dumps(line), flush=True)
    return 0


def profile_mst(torch, dev, X, args):
    """Profiling aid: the MST stage alone (the library's cluster_mst), W untimed
    and K timed calls, CUDA events on the current stream, L2 flushed before
    each.  Not a benchmark line: it prints its own keys."""
    from paper_1702_04739_gb300 import isoclust
    if args.workload not in (WORKLOAD, SPARSE, MOONS):
        raise SystemExit("--mst-only takes a one-set workload")
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    isoclust.set_mst_prune(args.mst_prune)
    times = []
    try:
        for it in range(args.warmup + args.steps):
            flush.fill_(it & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            isoclust.cluster_mst(Xd)
            b.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(a.elapsed_time(b))
        prof = isoclust.last_profile()
    finally:
        isoclust.set_mst_prune(-1)
    print(json.dumps({"profile": "mst", "workload": args.workload, "n": int(X.shape[0]), "d": int(X.shape[1]),
                      "mst_prune": args.mst_prune, "ms_per_call": float(np.median(times)),
                      "tiles_swept": prof.get("mst_tiles_swept"), "tiles_full": prof.get("mst_tiles_full")}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mst-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="default workload only (no 'workloads' key)")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed steps of each extra workload")
    ap.add_argument("--n", type=int, default=0,
                    help="points of the same generator (profiling of a smaller case); default: the full workload")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, SPARSE, BATCHED, MOONS])
    ap.add_argument("--nsets", type=int, default=0, help="batched: fewer sets of the same recipe (profiling)")
    ap.add_argument("--sweep-variant", type=int, default=-1,
                    help="force the MST sweep's tile variant 0..3 (profiling: a profiler distorts the autotuner's "
                         "trial timings); -1 = the library's own choice")
    ap.add_argument("--mst-only", action="store_true",
                    help="profiling: time only the minimum spanning tree of the workload's points (no omega "
                         "buffers on the device) and print one line of its own")
    ap.add_argument("--mst-prune", type=int, default=-1, choices=[-1, 0, 1],
                    help="with --mst-only: pruned Boruvka rounds -1 auto, 0 never, 1 whenever supported")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    from paper_1702_04739_gb300 import isoclust
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    isoclust.set_sweep_variant(args.sweep_variant)
    dev = torch.device("cuda", local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    data, k, sigma = load_workload(args.workload, seed=rank, n=args.n, nsets=args.nsets)
    if args.mst_only:
        return profile_mst(torch, dev, data, args)
    e2e = not args.no_e2e
    if args.workload == BATCHED:
        X, offs, ks = data
        res, detail = measure_batched(torch, dev, X, offs, ks, sigma, args.steps, args.warmup, pg, world, e2e)
    elif args.workload == MOONS:
        res, detail = measure_moons(torch, dev, data, k, sigma, args.steps, args.warmup, world, e2e)
    else:
        res, detail = measure_single(torch, dev, data, k, sigma, args.workload, args.steps, args.warmup, pg, world,
                                     e2e, mst_compare=not args.no_mst_compare)
    line = {"metric": METRIC, "value": res.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 forward, f64 gradient" if args.workload == MOONS else "f32+f64", "data": "synthetic",
            "config": config_of(args.workload, data, k, sigma, world)}
    res.pop("steps", None)
    res.pop("warmup", None)
    line.update(res)

    # the other benchmark workloads, fewer steps, one GPU
    if world == 1 and args.workload == WORKLOAD and not args.no_extras and not args.n:
        extras = {}
        ew = 3
        Xs, ks_, ss = load_workload(SPARSE)
        r3, _ = measure_single(torch, dev, Xs, ks_, ss, SPARSE, args.extra_steps, ew, e2e=False, mst_compare=True,
                               want_detail=False)
        extras[SPARSE] = dict(r3, config=config_of(SPARSE, Xs, ks_, ss, 1))
        del Xs
        (Xb, ob, kb), _, sb = load_workload(BATCHED)
        r4, _ = measure_batched(torch, dev, Xb, ob, kb, sb, args.extra_steps, ew, e2e=False, want_detail=False)
        extras[BATCHED] = dict(r4, config=config_of(BATCHED, (Xb, ob, kb), None, sb, 1))
        del Xb
        Xm, km, sm = load_workload(MOONS)
        r5, _ = measure_moons(torch, dev, Xm, km, sm, args.extra_steps, ew, e2e=False)
        extras[MOONS] = dict(r5, config=config_of(MOONS, Xm, km, sm, 1))
        for v in extras.values():
            v["note"] = "device-timed value, steps and warm-ups as given; L2 flushed before every step"
        line["workloads"] = extras

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, par = cpu_baseline(args.workload, data, k, sigma, detail)
        line["cpu_baseline"] = cb
        if par is not None:
            line["parity"] = par
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
