#!/usr/bin/env python3
"""Throughput of the NPCF hot path on one GB300 (or N, one process per GPU).

Workload: 200,000 log-normal points in a periodic 1000 Mpc/h cube, 10 linear shells
20-160 Mpc/h, lmax = 5, 4PCF + 3PCF (all parity-even multiplets). One step = one
npcf_accumulate of the whole catalog: cell list, pair kernel (a_lm of every primary),
3PCF and 4PCF contraction, FP64 reduction. Metric: primaries per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16]
    python bench.py --workload batch64 ...  # 64 catalogs in one batch (CUDA graph)
    python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "primaries/sec for 4PCF (lmax=5, 10 shells); split-BF16 vs FP32 at stated error"
WORKLOAD = "lognormal_200k_L1000_4pcf3pcf_lmax5_nr10_20-160"
FOURPCF_ALG_FLOP_PER_PRIMARY = 405_360 + 126_240   # P-build + final contraction (lmax 5, N_r 10)
PAIR_ALG_FLOP = 180                                  # per accepted pair at lmax 5
FP32_LANES = 128                                     # FP32 lanes per SM (used only if the probe fails)
KERNELS_PER_STEP = 10  # k_sumw, 4 cell-list kernels, pair, contract3, contract4, one reduce per order

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu pass) on the
# 200k workload, with the SHA-256 prefix of the kernel's source when they were taken; the
# roofline reports them only while the source is unchanged (profiles/ has the captures).
TRAFFIC = {
    "pair": {"bytes": 12_835_072 + 428_769_536, "source": "paper_2105_08722_gb300/csrc/npcf_pair.cu",
             "sha256": "5ab3768ce8a30c34"},
    "contraction/fp32": {"bytes": 338_221_568 + 141_824, "source": "paper_2105_08722_gb300/csrc/npcf_contract4.cu",
                         "sha256": "ec635d2be4d339ba"},
    "contraction/bf16": {"bytes": 338_193_920 + 3_255_552,
                         "source": "paper_2105_08722_gb300/csrc/npcf_contract_tc.cu", "sha256": "9e25cf7cd3089fa9"},
}


def _traffic(kernel):
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    try:
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != t["sha256"]:
                return None
    except OSError:
        return None
    return t["bytes"]


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(wl, sample_n: int, seed: int = 77, nthreads: int = 0, want_zeta: bool = False):
    """The oracle as it stands (OpenMP over primaries), timed on a sample of primaries
    against the full catalog. Returns (primaries/s, threads, sample description) and, with
    want_zeta, also (sample indices, the oracle's raw zeta of that sample)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(wl.n, sample_n, replace=False))
    cores = nthreads or (os.cpu_count() or 1)
    t0 = time.perf_counter()
    zeta, _ = oracle.npcf(wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, prim=sample, nthreads=cores)
    dt = time.perf_counter() - t0
    desc = "%d seeded primaries of the %dk catalog against all %dk secondaries" % (sample_n, wl.n // 1000,
                                                                                  wl.n // 1000)
    if want_zeta:
        return sample_n / dt, cores, desc, sample, zeta
    return sample_n / dt, cores, desc


def fp32_peak_tflops(dev):
    """Measured FP32 FMA throughput of this GPU (the library's probe), with the SM count
    read from the device; falls back to SMs x 128 lanes x 2 x max clock if the probe fails."""
    import torch
    from paper_2105_08722_gb300._lib import probe_fp32_peak
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        t, _ = probe_fp32_peak()
        return t, "measured: FMA-chain probe (npcf_probe_fp32_peak), %d SMs" % nsm, nsm
    except Exception as e:   # noqa: BLE001
        mhz = float(_peaks().get("sm_max_mhz", 2070.0))
        return (nsm * FP32_LANES * 2 * mhz * 1e6 / 1e12,
                "derived: %d SMs x %d lanes x 2 x %.0f MHz (probe failed: %s)" % (nsm, FP32_LANES, mhz, e), nsm)


def order_errors(got, want, orders, lmax, nr):
    """max |got - want| / RMS(want) per order (the oracle's layout)."""
    import oracle
    g = oracle.split_orders(got, orders, lmax, nr)
    o = oracle.split_orders(want, orders, lmax, nr)
    out = {}
    for N in orders:
        rms = math.sqrt(float(np.mean(o[N] ** 2)))
        out[str(N)] = float(np.max(np.abs(g[N] - o[N]))) / rms if rms > 0 else None
    return out


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the slowest rank sets the
    time of a step); identity on one rank."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processes its own replica of units_per_rank
    (weak scaling), and the step takes the slowest rank's time ms."""
    return units_per_rank * world / (ms * 1e-3)


def lognormal_workload(n_points):
    """The 200k log-normal workload, or the same density and spectrum at n_points (box
    scaled by (n/200k)^(1/3); a smaller case for profiling)."""
    from paper_2105_08722_gb300 import catalogs
    if not n_points or n_points == 200_000:
        return catalogs.lognormal200k_4pcf()
    box = 1000.0 * (n_points / 200_000) ** (1.0 / 3.0)
    pos = catalogs.lognormal_box(n_points, box, 256, seed=1002)
    return catalogs.Workload("lognormal_%dk_L%d_4pcf3pcf_lmax5_nr10_20-160" % (n_points // 1000, round(box)), pos,
                             np.ones(n_points, np.float32), catalogs.linear_edges(20.0, 160.0, 10), 5, (3, 4), box)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2105_08722_gb300 import catalogs
    wl = lognormal_workload(args.n)
    sample_n = args.ref_sample
    times = []
    for step in range(args.warmup + args.steps):
        rate, cores, desc = cpu_oracle_rate(wl, sample_n, seed=1000 + step)
        if step >= args.warmup:
            times.append(sample_n / rate)
    ms_per_primary = 1e3 * sum(times) / (sample_n * len(times))
    value = 1e3 / ms_per_primary
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "primaries/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if wl.n == 200_000 else wl.name, "n_points": wl.n, "lmax": wl.lmax, "nr": 10,
                   "orders": [3, 4], "step": "%d primaries (bounded sample)" % sample_n},
        "cpu_baseline": {"value": value, "unit": "primaries/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "primaries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32, SPLIT_BF16

    wl = lognormal_workload(args.n)
    prec = SPLIT_BF16 if args.precision == "bf16" else FP32
    est = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, prec)
    pos = torch.from_numpy(wl.pos).to(dev)
    w = torch.from_numpy(wl.w).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        est.accumulate(pos, w)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage_ms = []
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                      # evict the catalog and a_lm from L2 between steps
        starts[k].record(stream)
        est.accumulate(pos, w)
        ends[k].record(stream)
        stage_ms.append(est.timings())     # per-stage events of this step (same stream)
    torch.cuda.synchronize()
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    counts = est.pair_counts()

    # end to end: host buffers through the C ABI, copies and result read-back inside
    pos_h = np.ascontiguousarray(wl.pos)
    w_h = np.ascontiguousarray(wl.w)

    def e2e_ms_of(p):
        e = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, p)
        e.accumulate_host(pos_h, w_h)
        e.finalize()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e.reset()
            e.accumulate_host(pos_h, w_h)
            e.finalize()
        dt = (time.perf_counter() - t0) / args.steps
        size = e.size
        e.close()
        return dt * 1e3, size

    e2e_ms_local, out_size = e2e_ms_of(prec)
    barrier()
    clk = clocks.stop()

    ms, e2e_ms = max_over_ranks([float(np.mean(step_ms)), e2e_ms_local], world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    st = np.mean(np.array(stage_ms, dtype=np.float64), axis=0)   # [cell list, pair, contraction, reduction]
    npairs_per_step = float(counts.sum()) / (args.warmup + args.steps)
    pair_tflops = npairs_per_step * PAIR_ALG_FLOP / (st[1] * 1e-3) / 1e12
    con_tflops = wl.n * FOURPCF_ALG_FLOP_PER_PRIMARY / (st[2] * 1e-3) / 1e12
    fp32_peak, peak_source, nsm = fp32_peak_tflops(dev)
    dominant = "pair" if st[1] >= st[2] else "contraction"
    achieved = pair_tflops if dominant == "pair" else con_tflops
    achieved = float(achieved)
    other = None
    oprec = FP32 if prec == SPLIT_BF16 else SPLIT_BF16
    if not args.no_other_precision:
        # the other contraction arithmetic on the same workload (same timing protocol)
        oest = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, oprec)
        for _ in range(args.warmup):
            oest.accumulate(pos, w)
        torch.cuda.synchronize()
        oms, ost = [], []
        for k in range(args.steps):
            flush.zero_()
            s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s_ev.record(stream)
            oest.accumulate(pos, w)
            e_ev.record(stream)
            ost.append(oest.timings())
            torch.cuda.synchronize()
            oms.append(s_ev.elapsed_time(e_ev))
        ost = np.mean(np.array(ost, dtype=np.float64), axis=0)
        o_e2e_ms, _ = e2e_ms_of(oprec)
        other = {"precision": "bf16" if oprec == SPLIT_BF16 else "fp32",
                 "value": wl.n / (float(np.mean(oms)) * 1e-3), "ms_per_step": float(np.mean(oms)),
                 "e2e": {"value": wl.n / (o_e2e_ms * 1e-3), "unit": "primaries/s",
                         "h2d_bytes_per_step": int(wl.pos.nbytes + wl.w.nbytes),
                         "d2h_bytes_per_step": int(8 * out_size)},
                 "stages_ms": {"pair": float(ost[1]), "contraction": float(ost[2])},
                 "contraction_tflops": float(wl.n * FOURPCF_ALG_FLOP_PER_PRIMARY / (ost[2] * 1e-3) / 1e12)}
        oest.close()
    line = {
        "metric": METRIC,
        "value": aggregate_rate(wl.n, world, ms),
        "unit": "primaries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == FP32 else "bf16x3",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if wl.n == 200_000 else wl.name, "n_points": wl.n, "lmax": wl.lmax,
                   "nr": 10, "orders": [3, 4],
                   "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "e2e": {"value": aggregate_rate(wl.n, world, e2e_ms), "unit": "primaries/s",
                "h2d_bytes_per_step": int(wl.pos.nbytes + wl.w.nbytes),
                "d2h_bytes_per_step": int(8 * out_size)},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "pairs_per_step": npairs_per_step,
        "roofline": {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": (_traffic(dominant if dominant == "pair" else "contraction/" + args.precision)
                                 if wl.n == 200_000 else None),
                     "peak_source": peak_source,
                     "contraction_tflops": float(con_tflops),
                     "contraction_frac": float(con_tflops / fp32_peak)},
        "clocks": clk,
        "other_precision": other,
    }
    if not args.no_cpu_baseline:
        rate, cores, desc, sample, zwant = cpu_oracle_rate(wl, args.cpu_sample, want_zeta=True)
        rate1, _, desc1 = cpu_oracle_rate(wl, args.cpu_sample_1core, seed=78, nthreads=1)
        line["cpu_baseline"] = {"value": rate, "unit": "primaries/s", "cores": cores, "kind": "oracle",
                                "sample": desc, "value_1core": rate1, "sample_1core": desc1}
        # measured error of both contraction arithmetics against the oracle on that sample:
        # the sampled primaries (weight w, every other primary 0) against all secondaries
        wprim = np.zeros(wl.n, np.float32)
        wprim[sample] = wl.w[sample]
        twp = torch.from_numpy(wprim).to(dev)
        errs = {}
        for p_, name in ((FP32, "fp32"), (SPLIT_BF16, "bf16")):
            e = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, p_)
            e.accumulate(pos, w, wprim=twp)
            errs[name] = order_errors(e.finalize(), zwant, wl.orders, wl.lmax, len(wl.edges) - 1)
            e.close()
        line["stated_error"] = {
            "measure": "max |gpu - oracle| / RMS(oracle) per zeta order, raw sums of %d seeded primaries "
                       "against the full catalog" % len(sample),
            "fp32": errs["fp32"], "bf16": errs["bf16"], "bar": {"fp32": 1e-5, "bf16": 3e-5}}
    print(json.dumps(line))
    sys.stdout.flush()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_gpu_batch(args):
    """64 log-normal periodic catalogs (20k-300k points, log-uniform sizes) in one batch:
    autotuned on the largest catalog, captured into a CUDA graph, replayed every step."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32, SPLIT_BF16

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    cats, edges = catalogs.batch64_lognormal()
    sizes = np.array([len(c) for c in cats])
    off = np.concatenate([[0], np.cumsum(sizes)])
    n = int(off[-1])
    lmax, orders, box = 5, (3, 4), 1000.0
    prec = FP32 if args.precision == "fp32" else SPLIT_BF16
    pos_h = np.ascontiguousarray(np.concatenate(cats), np.float32)
    w_h = np.ones(n, np.float32)
    pos = torch.from_numpy(pos_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)

    big = int(np.argmax(sizes))
    tuner = NPCF(lmax, orders, edges, box, prec)
    chosen = tuner.autotune(pos[off[big]:off[big + 1]], w[off[big]:off[big + 1]])
    tuner.close()
    est = NPCF(lmax, orders, edges, box, prec)
    for key, name in ((0, "cells_per_rmax"), (5, "pair_chunk"), (3, "pair_cap"), (2, "chunk")):
        est.set_tuning(key, chosen[name])

    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            est.accumulate_batch(pos, w, off, stream=stream)
    stream.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            starts[k].record(stream)
            est.accumulate_batch(pos, w, off, stream=stream)
            ends[k].record(stream)
    stream.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    got = est.finalize_batch() / (args.warmup + args.steps)
    ncat, graphs = est.batch_info()

    # end to end: pinned host buffers copied in, the batch, every catalog's multiplets out
    pos_p = torch.from_numpy(pos_h).pin_memory()
    w_p = torch.from_numpy(w_h).pin_memory()
    e2e = NPCF(lmax, orders, edges, box, prec)
    for key, name in ((0, "cells_per_rmax"), (5, "pair_chunk"), (3, "pair_cap"), (2, "chunk")):
        e2e.set_tuning(key, chosen[name])
    dpos = torch.empty_like(pos)
    dw = torch.empty_like(w)
    t0 = None
    for k in range(args.steps + 1):
        if k == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            dpos.copy_(pos_p, non_blocking=True)
            dw.copy_(w_p, non_blocking=True)
            e2e.accumulate_batch(dpos, dw, off, stream=stream)
        e2e.finalize_batch()
    e2e_ms = (time.perf_counter() - t0) / args.steps * 1e3
    clk = clocks.stop()

    # per-catalog error of this precision against the FP32 path (itself held to the
    # oracle by the GPU tests)
    ref = NPCF(lmax, orders, edges, box, FP32)
    with torch.cuda.stream(stream):
        ref.accumulate_batch(pos, w, off, stream=stream)
    stream.synchronize()
    want = ref.finalize_batch()
    errs = {3: [], 4: []}
    for k in range(ncat):
        gs, ws = est.split(got[k]), ref.split(want[k])
        for N in (3, 4):
            rms = math.sqrt(float(np.mean(ws[N] ** 2)))
            errs[N].append(float(np.max(np.abs(gs[N] - ws[N]))) / rms if rms > 0 else 0.0)
    ms = float(np.mean(step_ms))
    counts = est.pair_counts_batch().sum() / (args.warmup + args.steps)
    alg = counts * PAIR_ALG_FLOP + n * FOURPCF_ALG_FLOP_PER_PRIMARY
    fp32_peak, peak_source, _ = fp32_peak_tflops(dev)
    achieved = alg / (ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": n / (ms * 1e-3), "unit": "primaries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == FP32 else "bf16x3",
        "data": "synthetic",
        "config": {"workload": "batch64_lognormal_20k-300k_L1000_4pcf3pcf_lmax5_nr10_20-160",
                   "n_catalogs": ncat, "n_points": n, "precision": "fp32" if prec == FP32 else "bf16",
                   "l2": "inputs (positions, a_lm) larger than L2", "parallelism": "single GPU",
                   "autotuned": chosen, "graph_launches": graphs},
        "e2e": {"value": n / (e2e_ms * 1e-3), "unit": "primaries/s", "h2d_bytes_per_step": int(pos_h.nbytes + w_h.nbytes),
                "d2h_bytes_per_step": int(8 * ncat * est.size)},
        "gpu_launches": args.steps,   # one CUDA-graph launch per step (KERNELS_PER_STEP kernels inside)
        "roofline": {"bound": "alu", "kernel": "whole batch (pair + contraction)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_source": peak_source},
        "clocks": clk,
        "per_catalog_error_vs_fp32": {str(N): {"max": max(errs[N]), "median": statistics.median(errs[N])}
                                      for N in (3, 4)},
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def _timed_steps(args, step, dev):
    """W untimed warm-up steps, then K steps each timed with CUDA events on the current
    stream (L2 flushed in between, untimed); returns (mean ms, clocks)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.mean(ms)), clocks.stop()


def run_gpu_uniform4k(args):
    """3PCF: 4,096 uniform points in a periodic 250 Mpc/h cube, 10 shells 0-50, lmax 5."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    wl = catalogs.uniform4k_3pcf()
    est = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, FP32)
    pos, w = torch.from_numpy(wl.pos).to(dev), torch.from_numpy(wl.w).to(dev)
    ms, clk = _timed_steps(args, lambda: est.accumulate(pos, w), dev)
    st = est.timings()
    line = {
        "metric": "primaries/sec for the 3PCF (lmax=5, 10 shells)", "value": wl.n / (ms * 1e-3),
        "unit": "primaries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uniform_4096_L250_3pcf_lmax5_nr10_0-50", "n_points": wl.n,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "gpu_launches": (KERNELS_PER_STEP - 2) * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


# The paper's own timings on its Table 2 catalog (16-core CPU), as primaries/s = 5e4 / T
PAPER_TABLE2_CPU = {4: 5.0e4 / 4.8, 5: 5.0e4 / 741.8}


def run_gpu_paper(args, order):
    """The paper's timing setting (Table 2): 5e4 uniform points, periodic 1500 Mpc/h box,
    10 shells to 200 Mpc/h, lmax 5; order 4 (with the 3PCF) or order 5."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32, SPLIT_BF16

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    orders = (3, 4) if order == 4 else (5,)
    wl = catalogs.paper_uniform_1500(orders=orders)
    prec = SPLIT_BF16 if (args.precision == "bf16" and order == 4) else FP32
    est = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, prec)
    pos, w = torch.from_numpy(wl.pos).to(dev), torch.from_numpy(wl.w).to(dev)
    ms, clk = _timed_steps(args, lambda: est.accumulate(pos, w), dev)
    st = est.timings()   # stages of the last timed step
    value = wl.n / (ms * 1e-3)
    name = "4PCF (with the 3PCF)" if order == 4 else "5PCF"
    line = {
        "metric": "primaries/sec for the %s (lmax=5, 10 shells) on the paper's timing catalog" % name,
        "value": value, "unit": "primaries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_TABLE2_CPU[order],
        "dtype": "bf16x3" if prec == SPLIT_BF16 else "f32", "data": "synthetic",
        "config": {"workload": "uniform_50k_L1500_%s_lmax5_nr10_0-200" % ("4pcf3pcf" if order == 4 else "5pcf"),
                   "n_points": wl.n, "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU",
                   "baseline": "the paper's 16-core CPU time on this catalog (Table 2): %.4g primaries/s"
                               % PAPER_TABLE2_CPU[order]},
        "gpu_launches": (KERNELS_PER_STEP - (0 if order == 4 else 2)) * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_gpu_survey(args):
    """Survey D - R: 400k log-normal data + 1.6M randoms (weights +1, -N_D/N_R) inside a
    60 degree cap, 600-1400 Mpc/h, non-periodic; the 1.6M randoms-only run; the GPU edge
    correction. One step = both accumulate calls and the edge-correction solve."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32, SPLIT_BF16

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    dr, rr = catalogs.survey_dmr_and_randoms()
    prec = FP32 if args.precision == "fp32" else SPLIT_BF16
    nest = NPCF(dr.lmax, dr.orders, dr.edges, 0.0, prec)
    rest = NPCF(rr.lmax, rr.orders, rr.edges, 0.0, prec)
    dpos, dw = torch.from_numpy(dr.pos).to(dev), torch.from_numpy(dr.w).to(dev)
    rpos, rw = torch.from_numpy(rr.pos).to(dev), torch.from_numpy(rr.w).to(dev)
    stages = []

    def step():
        nest.reset()
        rest.reset()
        nest.accumulate(dpos, dw)
        rest.accumulate(rpos, rw)
        nest.edge_correct(rest)
        stages.append(np.array(nest.timings(), np.float64) + np.array(rest.timings(), np.float64))

    ms, clk = _timed_steps(args, step, dev)
    st = np.mean(np.array(stages[-args.steps:]), axis=0)
    n = dr.n + rr.n
    line = {
        "metric": "primaries/sec for the survey D-R 4PCF + 3PCF with edge correction (lmax=5, 10 shells)",
        "value": n / (ms * 1e-3), "unit": "primaries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == FP32 else "bf16x3", "data": "synthetic",
        "config": {"workload": "survey_DmR_400k_1600k_plus_R_1600k_4pcf3pcf_lmax5_nr10_20-160_edge",
                   "n_points": n, "precision": args.precision, "l2": "inputs larger than L2",
                   "parallelism": "single GPU"},
        "gpu_launches": 2 * KERNELS_PER_STEP * args.steps + 2 * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_gpu_5pcf(args):
    """5PCF: 100k log-normal points, periodic 1000 Mpc/h, 8 shells 20-160, lmax 4 (all
    5PCF multiplets with l12 <= 2 lmax). One step = one npcf_accumulate."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    wl = catalogs.lognormal100k_5pcf()
    est = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, FP32)
    pos = torch.from_numpy(wl.pos).to(dev)
    w = torch.from_numpy(wl.w).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        est.accumulate(pos, w)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ms, st = [], []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        est.accumulate(pos, w)
        b.record(stream)
        st.append(est.timings())
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    clk = clocks.stop()
    st = np.mean(np.array(st, dtype=np.float64), axis=0)
    t = float(np.mean(ms))
    # algorithmic 5PCF flop per primary: the P12 and P34 builds and the final products
    alg = wl.n * (543_200 * 2 + 1_110_200)
    fp32_peak, peak_source, _ = fp32_peak_tflops(dev)
    achieved = alg / (st[2] * 1e-3) / 1e12
    line = {
        "metric": "primaries/sec for the 5PCF (lmax=4, 8 shells)", "value": wl.n / (t * 1e-3),
        "unit": "primaries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "lognormal_100k_L1000_5pcf_lmax4_nr8_20-160", "n_points": wl.n,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "gpu_launches": (KERNELS_PER_STEP - 2) * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "roofline": {"bound": "alu", "kernel": "contraction (5PCF)", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_source": peak_source},
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_gpu_6pcf(args):
    """6PCF: 50k log-normal points, periodic 1000 Mpc/h, 8 shells 20-160, lmax 2 (327
    parity-even multiplets with intermediates up to 2 lmax, 56 bin tuples). One step = one
    npcf_accumulate."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    wl = catalogs.lognormal_6pcf()
    est = NPCF(wl.lmax, wl.orders, wl.edges, wl.box, FP32)
    pos, w = torch.from_numpy(wl.pos).to(dev), torch.from_numpy(wl.w).to(dev)
    ms, clk = _timed_steps(args, lambda: est.accumulate(pos, w), dev)
    st = est.timings()
    line = {
        "metric": "primaries/sec for the 6PCF (lmax=2, 8 shells)", "value": wl.n / (ms * 1e-3),
        "unit": "primaries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "lognormal_50k_L1000_6pcf_lmax2_nr8_20-160", "n_points": wl.n,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "gpu_launches": (KERNELS_PER_STEP - 2) * args.steps,
        "stages_ms": {"cell_list": float(st[0]), "pair": float(st[1]), "contraction": float(st[2]),
                      "reduction": float(st[3])},
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_gpu_survey_splits(args):
    """Survey data (400k, weight +1) with 1.6M randoms in 4 splits (weights -N_D/N_k), 3PCF +
    4PCF, lmax 5, 10 shells, open geometry: the 4 data-minus-randoms splits co-added (Sec.
    4.2), once through npcf_accumulate of each concatenated split and once with the data
    harmonics kept (npcf_cache_data once, then npcf_accumulate_split per split). One step =
    the whole set of splits (the cached arm includes its npcf_cache_data)."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    d, wd, splits, edges = catalogs.survey_splits()
    lmax, orders = 5, (3, 4)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dd, dw = t(d), t(wd)
    cat = [(t(np.concatenate([d, r])), t(np.concatenate([wd, wr]))) for r, wr in splits]
    rs = [(t(r), t(wr)) for r, wr in splits]
    plain = NPCF(lmax, orders, edges, 0.0, FP32)
    cached = NPCF(lmax, orders, edges, 0.0, FP32)

    def step_plain():
        plain.reset()
        for p_, w_ in cat:
            plain.accumulate(p_, w_)

    def step_cached():
        cached.reset()
        cached.cache_data(dd, dw)
        for p_, w_ in rs:
            cached.accumulate_split(p_, w_)

    ms_plain, _ = _timed_steps(args, step_plain, dev)
    ms_cached, clk = _timed_steps(args, step_cached, dev)
    a, b = plain.finalize(), cached.finalize()
    rel = float(np.max(np.abs(a - b)) / np.sqrt(np.mean(a ** 2)))
    prim = sum(len(d) + len(r) for r, _ in splits)
    line = {
        "metric": "primaries/sec for the survey D-R 4PCF + 3PCF over 4 random splits (lmax=5, 10 shells)",
        "value": prim / (ms_cached * 1e-3), "unit": "primaries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_cached, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "survey_400k_data_4x400k_random_splits_4pcf3pcf_lmax5_nr10_20-160",
                   "n_primaries_per_step": prim, "l2": "inputs larger than L2", "parallelism": "single GPU"},
        "without_cache": {"value": prim / (ms_plain * 1e-3), "ms_per_step": ms_plain},
        "max_diff_vs_without_cache_over_rms": rel,
        "gpu_launches": None,
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_gpu_grid(args):
    """Gridded field (Sec. 3.2.2): the log-normal overdensity on a 64^3 mesh in a periodic
    1000 Mpc/h box, 3PCF + 4PCF, lmax 5, 10 shells 20-160; a_lm of every cell by FFT, cells
    as primaries. One step = one npcf_accumulate_grid (kernel spectra kept from warm-up)."""
    import torch

    from paper_2105_08722_gb300 import build, catalogs
    build()
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    n = args.ngrid
    delta = torch.from_numpy(catalogs.lognormal_mesh(n, 1000.0, seed=1007)).to(dev)
    est = NPCF(5, (3, 4), catalogs.linear_edges(20.0, 160.0, 10), 1000.0, FP32)
    ms, clk = _timed_steps(args, lambda: est.accumulate_grid(delta), dev)
    st = est.timings()
    cells = n ** 3
    line = {
        "metric": "cells/sec for the 4PCF + 3PCF of a gridded field (lmax=5, 10 shells)",
        "value": cells / (ms * 1e-3), "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "lognormal_mesh_%d3_L1000_4pcf3pcf_lmax5_nr10_20-160" % n, "cells": cells,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "single GPU"},
        "stages_ms": {"fft_alm": float(st[1]), "contraction": float(st[2]), "reduction": float(st[3])},
        "gpu_launches": None,
        "clocks": clk,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def run_fp16_range(args):
    """Range of the contraction operands the FP16-scaled precision would have to hold, on
    the 200k log-normal workload: for a seeded sample of primaries, their a_lm (from the
    GPU, npcf_debug_alm) as the contraction kernels hold them (reduced harmonics a_lm /
    sqrt((2l+1)/(4 pi))) and the 4PCF products P^{L,m3}(b1,b2) = sum_m1 E C a^{b1} a^{b2} of
    those (couplings from the library, npcf_coupling); per primary the largest |P| and |a|.
    A GEMM over primaries with one scale s_p per primary (A = P / s_p, B = a s_p) fits FP16
    only if max|P| max|a| <= 65504^2."""
    import torch

    from paper_2105_08722_gb300 import build
    build()
    from paper_2105_08722_gb300 import _lib
    from paper_2105_08722_gb300._lib import NPCF, FP32

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    wl = lognormal_workload(args.n)
    est = NPCF(wl.lmax, (3,), wl.edges, wl.box, FP32)
    est.accumulate(torch.from_numpy(wl.pos).to(dev), torch.from_numpy(wl.w).to(dev))
    rng = np.random.default_rng(909)
    sample = np.sort(rng.choice(wl.n, args.fp16_sample, replace=False))
    a_pos, _ = est.debug_alm(sample)                    # [k, nr, nlm] complex, m >= 0
    k, nr, lmax = len(sample), len(wl.edges) - 1, wl.lmax
    a = {}
    for l in range(lmax + 1):
        for m in range(l + 1):
            v = a_pos[:, :, l * (l + 1) // 2 + m].astype(np.complex128)
            a[(l, m)] = v
            if m:
                a[(l, -m)] = ((-1) ** m) * np.conj(v)
    # the contraction kernels work on the reduced harmonics a_lm / sqrt((2l+1)/(4 pi))
    red = np.array([math.sqrt(4.0 * math.pi / (2 * l + 1)) for l in range(lmax + 1) for m in range(l + 1)])
    for key in list(a):
        a[key] = a[key] * math.sqrt(4.0 * math.pi / (2 * key[0] + 1))
    amax = np.max(np.abs(a_pos * red[None, None, :]), axis=(1, 2))
    pmax = np.zeros(k)
    iu = np.triu_indices(nr, 1)
    for L in _lib.multiplets(4, lmax):
        l1, l2, l3 = (int(x) for x in L)
        E = (-1) ** (l1 + l2 + l3)
        for m3 in range(l3 + 1):
            P = np.zeros((k, nr, nr), np.complex128)
            for m1 in range(-l1, l1 + 1):
                m2 = -m1 - m3
                if abs(m2) > l2:
                    continue
                c = E * _lib.coupling(4, [l1, l2, l3], [m1, m2, m3])
                if c:
                    P += c * a[(l1, m1)][:, :, None] * a[(l2, m2)][:, None, :]
            pmax = np.maximum(pmax, np.max(np.abs(P[:, iu[0], iu[1]]), axis=1))
    prod = pmax * amax
    edges_hist = [0, 3, 4, 5, 6, 7, 8, 9, 9.63, 10, 11, 12, 13, 14]
    hist, _ = np.histogram(np.log10(np.maximum(prod, 1e-30)), bins=edges_hist)
    limit = 65504.0 ** 2
    line = {
        "metric": "FP16 range of the 4PCF contraction operands (reduced harmonics; lmax=5, 10 shells)",
        "config": {"workload": wl.name if wl.n != 200_000 else WORKLOAD, "primaries_sampled": int(k)},
        "max_abs_a": {"median": float(np.median(amax)), "p99": float(np.percentile(amax, 99)), "max": float(amax.max())},
        "max_abs_P": {"median": float(np.median(pmax)), "p99": float(np.percentile(pmax, 99)), "max": float(pmax.max())},
        "max_P_times_max_a": {"median": float(np.median(prod)), "p99": float(np.percentile(prod, 99)),
                              "max": float(prod.max())},
        "log10_histogram": {"bin_edges": edges_hist, "counts": [int(x) for x in hist]},
        "fraction_beyond_one_fp16_scale": float(np.mean(prod > limit)),
        "fp16_limit_65504_squared": limit,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16"],
                    help="contraction arithmetic (default fp32; bf16 for the batch workload)")
    ap.add_argument("--n", type=int, default=0,
                    help="points of the 200k log-normal workload at the same density (default 200,000)")
    ap.add_argument("--workload", default="lognormal200k",
                    choices=["uniform4k", "lognormal200k", "survey", "lognormal100k-5pcf", "batch64", "paper4",
                             "paper5", "lognormal50k-6pcf", "survey-splits", "grid", "fp16-range"],
                    help="uniform4k: 4,096 uniform points, 3PCF; lognormal200k: one 200k log-normal catalog "
                         "(4PCF + 3PCF); survey: 400k data + 1.6M randoms (D-R and R runs) with edge correction; "
                         "lognormal100k-5pcf: 100k points, 5PCF; batch64: 64 catalogs in one batch; "
                         "paper4 / paper5: the paper's timing catalog (5e4 uniform, L 1500), 4PCF / 5PCF; "
                         "lognormal50k-6pcf: 50k points, 6PCF; survey-splits: 4 random splits with and without "
                         "the data harmonics kept; grid: a log-normal field on an ngrid^3 mesh by FFT")
    ap.add_argument("--ngrid", type=int, default=64, help="mesh side of the grid workload")
    ap.add_argument("--fp16-sample", type=int, default=4096, help="primaries sampled by fp16-range")
    ap.add_argument("--cpu-sample", type=int, default=1500)
    ap.add_argument("--cpu-sample-1core", type=int, default=120)
    ap.add_argument("--ref-sample", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-precision", action="store_true",
                    help="skip timing the other contraction precision")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.precision is None:
        args.precision = "bf16" if args.workload == "batch64" else "fp32"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_gpu_batch(args)
    if args.workload == "lognormal100k-5pcf":
        return run_gpu_5pcf(args)
    if args.workload == "uniform4k":
        return run_gpu_uniform4k(args)
    if args.workload in ("paper4", "paper5"):
        return run_gpu_paper(args, 4 if args.workload == "paper4" else 5)
    if args.workload == "survey":
        return run_gpu_survey(args)
    if args.workload == "lognormal50k-6pcf":
        return run_gpu_6pcf(args)
    if args.workload == "survey-splits":
        return run_gpu_survey_splits(args)
    if args.workload == "grid":
        return run_gpu_grid(args)
    if args.workload == "fp16-range":
        return run_fp16_range(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
