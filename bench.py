"""Benchmark of the hot path: all-pairs windowed DTW matrix, then k-medoids.

One step = dtw_pairwise over a set of 2000 series of length 512 (five seeded
class generators, z-normalised, window w = 51), one dtw_query of a series of
the set against the set, and kmedoids_fit with k = 5 from seeded initial
medoids.  The metric is throughput in GCUPS: in-band DP cells of the all-pairs
matrix per second of whole-step time.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead, on a
bounded sample of the same workload, and prints the same line with
"impl": "reference".  Under torchrun every rank runs its own independent
problem (seed 1 + rank); value = all ranks' cells / the slowest rank's time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SERIES, LENGTH, WINDOW, K_CLUSTERS = 2000, 512, 51, 5
FP32_LANES_PER_SM = 128   # FP32 ALU lanes per Blackwell SM
OPS_PER_CELL = 4          # FADD (x-y), two FMNMX, FFMA: the 4-op cell of the roofline
WORKLOAD = "N=2000 series x L=512, five-class synthetic, w=51, k=5"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dtw_band_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2307_04904_gb300", "csrc", f)
                  for f in ("band_kernels.cuh", "band_tworow.cuh", "band2r.cu", "common.cuh")]


def band_cells(L: int, w: int) -> int:
    """In-band cells of one L x L pair: L(2w+1) - w(w+1)."""
    w = min(w, L - 1)
    return L * (2 * w + 1) - w * (w + 1)


def cells_per_step() -> int:
    return N_SERIES * (N_SERIES - 1) // 2 * band_cells(LENGTH, WINDOW)


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the DTW kernel from the committed ncu summary,
    or None if the kernel source changed since it was captured."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha") != kernel_source_sha():
            return None
        return float(kv["dram_bytes_per_launch_full_workload"])
    except (OSError, KeyError, ValueError):
        return None


# ----------------------------------------------------------------- helpers


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step: float, steps: int, world: int, t_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return units_per_rank_step * steps * world / t_max


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------- CPU oracle


def cpu_oracle_rate(seed: int, budget_s: float = 12.0):
    """Oracle GCUPS on a bounded random sample of the pairs of the workload."""
    import numpy as np

    import oracle
    from paper_2307_04904_gb300 import synth

    values, offsets, _ = synth.five_class_set(N_SERIES, LENGTH, seed=seed)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1234)

    def sample(n):
        a = rng.integers(0, N_SERIES - 1, n)
        b = rng.integers(0, N_SERIES, n)
        b = np.where(b <= a, a + 1 + (b % (N_SERIES - 1 - a)), b)
        return a, b

    a, b = sample(2000)
    t = time.perf_counter()
    oracle.pairs(values, offsets, a, b, WINDOW, threads=cores)
    dt = time.perf_counter() - t
    n = int(max(2000, min(N_SERIES * (N_SERIES - 1) // 2, 2000 * budget_s / max(dt, 1e-6))))
    a, b = sample(n)
    t = time.perf_counter()
    oracle.pairs(values, offsets, a, b, WINDOW, threads=cores)
    dt = time.perf_counter() - t
    cells = n * band_cells(LENGTH, WINDOW)
    # the same oracle on one thread, on a sample of about 3 s
    n1 = int(max(50, min(n, n * 3.0 / max(dt * cores, 1e-6))))
    a1, b1 = sample(n1)
    t = time.perf_counter()
    oracle.pairs(values, offsets, a1, b1, WINDOW, threads=1)
    dt1 = time.perf_counter() - t
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} random pairs of the {WORKLOAD} set, float64 DP, OpenMP over pairs; "
                      f"{dt:.2f} s",
            "single_thread": {"value": round(n1 * band_cells(LENGTH, WINDOW) / dt1 / 1e9, 4),
                              "unit": "GCUPS", "sample": f"{n1} random pairs, {dt1:.2f} s"}}


# --------------------------------------------------------------- GPU arm


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2307_04904_gb300 import api, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    seed = 1 + rank
    values, offsets, _ = synth.five_class_set(N_SERIES, LENGTH, seed=seed)
    init_h = synth.init_medoids(N_SERIES, K_CLUSTERS, seed)
    v = torch.from_numpy(values).to(dev)
    o = torch.from_numpy(offsets).to(dev)
    init = torch.as_tensor(init_h, dtype=torch.int32, device=dev)
    q = v[int(offsets[7]):int(offsets[8])].clone()
    D = torch.empty((N_SERIES, N_SERIES), dtype=torch.float32, device=dev)
    qrow = torch.empty(N_SERIES, dtype=torch.float32, device=dev)
    med = torch.empty(K_CLUSTERS, dtype=torch.int32, device=dev)
    lab = torch.empty(N_SERIES, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(values_t, offsets_t):
        api.dtw_pairwise(values_t, offsets_t, WINDOW, out=D)
        api.dtw_query(q, values_t, offsets_t, WINDOW, out=qrow)
        _, _, cost, iters = api.kmedoids_fit(D, K_CLUSTERS, init, out_medoids=med, out_labels=lab)
        return cost, iters

    for _ in range(args.warmup):
        step(v, o)
    torch.cuda.synchronize()

    # device-resident inputs: per-step CUDA events, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            cost, iters = step(v, o)
            ends[i].record(stream)
            # dtw_pairwise: staging, band kernel, zero diagonal; dtw_query: set and query
            # staging, band kernel; k-medoids: 3 per sweep, then assign and 2 cost kernels
            launches += 3 + 3 + 3 * iters + 3
        torch.cuda.synchronize()
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, world)
    cells = cells_per_step()
    value = whole_job_value(cells, args.steps, world, t_max) / 1e9
    clocks = clk.summary()

    # the DTW kernel alone (dominant kernel), on the stream it is launched on
    ks, ke = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kreps = max(3, args.steps)
    kms = []
    for _ in range(kreps):
        flush.zero_()
        ks.record(stream)
        api.dtw_pairwise(v, o, WINDOW, out=D)
        ke.record(stream)
        torch.cuda.synchronize()
        kms.append(ks.elapsed_time(ke))
    k_ms = statistics.median(kms)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak_gcups = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / OPS_PER_CELL / 1e9
    achieved = cells / (k_ms / 1e3) / 1e9
    med_mhz = clocks.get("sm_mhz")
    roofline = {
        "bound": "alu", "achieved": round(achieved, 1), "peak": round(peak_gcups, 1),
        "unit": "GCUPS", "frac": round(achieved / peak_gcups, 4),
        "traffic": recorded_traffic(),
        "kernel": api.describe_shape(LENGTH, LENGTH, WINDOW) + " (+ staging, zero_diagonal)",
        "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz:.0f} MHz / "
                      f"{OPS_PER_CELL} ops per cell",
        "frac_at_median_clock": (round(achieved / (sms * FP32_LANES_PER_SM * med_mhz * 1e6
                                                   / OPS_PER_CELL / 1e9), 4)
                                 if med_mhz else None),
        "kernel_ms": round(k_ms, 4),
        # the stricter ceiling the kernel's own instruction mix allows: a cell issues three
        # instructions (subtraction, three-input minimum, fused multiply-add) and an SM issues
        # one warp instruction per scheduler per clock, 4 x 32 thread instructions
        "issue_ceiling": round(sms * 4 * 32 * max_mhz * 1e6 / 3 / 1e9, 1),
        "frac_of_issue_ceiling": round(achieved / (sms * 4 * 32 * max_mhz * 1e6 / 3 / 1e9), 4),
    }

    # end to end through the library's host-buffer route (DTW_HOST_IO) from pinned host
    # arrays: the matrix and the query row come back to the host; k-medoids (device D in the
    # C ABI) runs on the host matrix uploaded again, and its medoids and labels come back
    hv = torch.from_numpy(values).pin_memory()
    ho = torch.from_numpy(offsets).pin_memory()
    hq = q.cpu().pin_memory()
    hD = torch.empty((N_SERIES, N_SERIES), dtype=torch.float32).pin_memory()
    hrow = torch.empty(N_SERIES, dtype=torch.float32).pin_memory()
    hmed = torch.empty(K_CLUSTERS, dtype=torch.int32).pin_memory()
    hlab = torch.empty(N_SERIES, dtype=torch.int32).pin_memory()
    nv, no, nq, nD, nrow = hv.numpy(), ho.numpy(), hq.numpy(), hD.numpy(), hrow.numpy()
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.dtw_pairwise_host(nv, no, WINDOW, out=nD)
        api.dtw_query_host(nq, nv, no, WINDOW, out=nrow)
        D.copy_(hD, non_blocking=True)
        api.kmedoids_fit(D, K_CLUSTERS, init, out_medoids=med, out_labels=lab)
        hmed.copy_(med, non_blocking=True)
        hlab.copy_(lab, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(sum(e2e_times), world)
    set_bytes = hv.numel() * 4 + ho.numel() * 8
    h2d = 2 * set_bytes + hq.numel() * 4 + hD.numel() * 4
    d2h = hD.numel() * 4 + hrow.numel() * 4 + hmed.numel() * 4 + hlab.numel() * 4 + 8
    e2e = {"value": round(cells * args.steps * world / e2e_t / 1e9, 2), "unit": "GCUPS",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "route": "dtw_pairwise and dtw_query with DTW_HOST_IO from pinned host arrays; "
                    "kmedoids_fit on the host matrix uploaded again"}

    cpu = cpu_oracle_rate(seed) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    line = {
        "metric": "all-pairs DTW GCUPS (whole step: matrix + query + k-medoids)",
        "value": round(value, 2), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded five-class generator; the UCR archive is not available)",
        "config": {"workload": WORKLOAD, "cells_per_step": cells, "pairs": N_SERIES * (N_SERIES - 1) // 2,
                   "band": "Sakoe-Chiba |i-j|<=51, squared-difference cost",
                   "l2": "flushed (256 MB write) before every timed step",
                   "kmedoids_iters": iters, "kmedoids_cost": cost,
                   "parallelism": f"replicas x{world} (independent problem per rank)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "impl": "dtwgb",
    }
    return line


def run_reference(args, world, rank):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    if rank != 0:
        return None
    per = []
    cpu = None
    for i in range(args.warmup + args.steps):
        budget = 2.0 if i < args.warmup else 8.0
        cpu = cpu_oracle_rate(1, budget_s=budget)
        if i >= args.warmup:
            per.append(cpu["value"])
    value = statistics.median(per)
    cpu["value"] = round(value, 3)
    return {
        "metric": "all-pairs DTW GCUPS (whole step: matrix + query + k-medoids)",
        "value": round(value, 3), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "random pairs per step, ~8 s of CPU work"},
        "impl": "reference", "cpu_baseline": cpu,
        "e2e": {"value": round(value, 3), "unit": "GCUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------- batched ragged sets

RAGGED_N, RAGGED_LO, RAGGED_HI, RAGGED_PERMILLE = 4000, 64, 2048, 50
RAGGED_WORKLOAD = ("N=4000 series, lengths uniform in [64, 2048], five-class synthetic, per-pair "
                   "window 5 % of the longer series widened to |n-m|")


def _event_time(fn, steps, flush, stream):
    import torch

    ms = []
    for _ in range(steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(s.elapsed_time(e))
    return ms


def run_ragged(args):
    import numpy as np
    import torch

    import oracle
    from paper_2307_04904_gb300 import api, synth

    dev = torch.device("cuda", 0)
    lens = synth.ragged_lengths(RAGGED_N, RAGGED_LO, RAGGED_HI, seed=2)
    values, offsets, _ = synth.five_class_set(RAGGED_N, lens, seed=2)
    v = torch.from_numpy(values).to(dev)
    o = torch.from_numpy(offsets).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    job = {"values": v, "offsets": o, "window_permille": RAGGED_PERMILLE}
    t0 = time.perf_counter()
    batch = api.Batch([job], graph=True, autotune=True)
    plan_s = time.perf_counter() - t0
    info = batch.info()
    cells = info["cells"]
    for _ in range(max(1, args.warmup - 2)):
        batch.run()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        ms = _event_time(batch.run, args.steps, flush, stream)
    t_batch = statistics.median(ms)

    D2 = torch.empty((RAGGED_N, RAGGED_N), dtype=torch.float32, device=dev)
    plain = lambda: api.dtw_pairwise(v, o, RAGGED_PERMILLE, permille=True, out=D2)
    plain()
    t_plain = statistics.median(_event_time(plain, 2, flush, stream))
    same = bool(torch.equal(D2, batch.outputs[0]))

    b2 = api.Batch([job], graph=False, autotune=False, unsorted=True)
    b2.run()
    t_unsorted = statistics.median(_event_time(b2.run, 2, flush, stream))
    b2.close()
    b3 = api.Batch([job], graph=True, autotune=False)
    b3.run()
    t_model = statistics.median(_event_time(b3.run, 2, flush, stream))
    b3.close()

    # per-pair launches on a sample: one dtw_pairwise call per pair
    rng = np.random.default_rng(7)
    a = rng.integers(0, RAGGED_N - 1, 500)
    c = np.minimum(RAGGED_N - 1, a + 1 + rng.integers(0, RAGGED_N, 500) % (RAGGED_N - 1 - a))
    pv = [torch.from_numpy(np.concatenate([values[offsets[i]:offsets[i + 1]],
                                           values[offsets[j]:offsets[j + 1]]])).to(dev)
          for i, j in zip(a, c)]
    po = [torch.tensor([0, int(lens[i]), int(lens[i] + lens[j])], dtype=torch.int64, device=dev)
          for i, j in zip(a, c)]
    torch.cuda.synchronize()
    tp = time.perf_counter()
    for x, y in zip(pv, po):
        api.dtw_pairwise(x, y, RAGGED_PERMILLE, permille=True)
    torch.cuda.synchronize()
    per_pair_s = (time.perf_counter() - tp) / len(pv)

    # the oracle on sampled pairs, including the extreme lengths
    order = np.argsort(lens)
    sa = np.concatenate([rng.integers(0, RAGGED_N, 3000), order[:20], order[-20:]])
    sb = np.concatenate([rng.integers(0, RAGGED_N, 3000), order[-20:], order[-40:-20]])
    keep = sa != sb
    sa, sb = sa[keep], sb[keep]
    wl = np.maximum(lens[sa], lens[sb]) * RAGGED_PERMILLE // 1000
    cores = os.cpu_count() or 1
    tc = time.perf_counter()
    ref = oracle.pairs_w(values, offsets, sa, sb, wl, threads=cores)
    cpu_s = time.perf_counter() - tc
    scells = sum(oracle.band_cells(int(lens[i]), int(lens[j]), int(w)) for i, j, w in zip(sa, sb, wl))
    got = batch.outputs[0].cpu().numpy()[sa, sb].astype(np.float64)
    max_rel = float(np.max(np.abs(got - ref) / ref))

    classes = batch.classes()
    top = max(classes, key=lambda c: c["cells"])
    by_kernel = {}
    for c in classes:
        key = "rotated (all K, G)" if c["kind"] == "rotated" else f"{c['kind']} K={c['K']}"
        by_kernel[key] = by_kernel.get(key, 0) + c["cells"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / OPS_PER_CELL / 1e9
    value = cells / (t_batch / 1e3) / 1e9
    return {
        "metric": "batched ragged DTW GCUPS (one graph replay: staging + all shape classes)",
        "value": round(value, 1), "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_batch, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": RAGGED_WORKLOAD, "pairs": info["pairs"], "cells_per_step": cells,
                   "classes": info["classes"], "buckets_tuned": info["buckets_tuned"],
                   "cell_share_by_kernel": {k: round(v / cells, 4) for k, v in
                                            sorted(by_kernel.items(), key=lambda kv: -kv[1])},
                   "plan_s": round(plan_s, 2), "l2": "flushed before every timed step"},
        "compare": {
            "plain_dtw_pairwise_ms": round(t_plain, 3),
            "plain_gcups": round(cells / (t_plain / 1e3) / 1e9, 1),
            "unsorted_model_shapes_ms": round(t_unsorted, 3),
            "sorted_model_shapes_graph_ms": round(t_model, 3),
            "per_pair_launch_us": round(per_pair_s * 1e6, 1),
            "per_pair_launches_extrapolated_s": round(per_pair_s * info["pairs"], 1),
            "batch_equals_plain_bitwise": same,
        },
        "roofline": {"bound": "alu", "achieved": round(value, 1), "peak": round(peak, 1),
                     "unit": "GCUPS", "frac": round(value / peak, 4), "traffic": None,
                     "kernel": f"largest class: {top['kind']} K={top['K']} G={top['G']} "
                               f"({top['cells'] / cells:.0%} of cells)"},
        "parity": {"sampled_pairs": int(len(sa)), "max_rel_vs_oracle": max_rel},
        "cpu_baseline": {"value": round(scells / cpu_s / 1e9, 3), "unit": "GCUPS", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{len(sa)} pairs incl. the 20 shortest and longest series, "
                                   f"{cpu_s:.1f} s"},
        "clocks": clocks, "impl": "dtwgb",
    }


# ----------------------------------------------------------------- serving

SERVING_JOBS, SERVING_RATE = 120, 20.0
SERVING_WORKLOAD = ("Poisson stream, 20 jobs/s: clustering jobs with N ~ U[100, 5000] series of "
                    "length L ~ U[128, 1024] (five-class synthetic), w = floor(0.1 L), "
                    "k ~ U[2, 12]; 30 % of jobs are 1-vs-N queries against resident sets")


def run_serving(args):
    import torch

    from paper_2307_04904_gb300 import serving

    arrivals = serving.poisson_stream(SERVING_JOBS, rate=SERVING_RATE, seed=4)
    # warm the kernels and the pools with a small stream first (not timed)
    warm = serving.poisson_stream(6, rate=100.0, seed=5, n_range=(50, 120), len_range=(64, 128))
    srv = serving.DTWServer(slots=4, hbm_budget=32 << 30)
    for f in serving.replay(srv, warm, realtime=False):
        f.result()
    srv.drain()
    srv.close()
    span = arrivals[-1][0] - arrivals[0][0]
    srv = serving.DTWServer(slots=4, hbm_budget=32 << 30)
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        futs = serving.replay(srv, arrivals, realtime=True)
        for f in futs:
            f.result()
        srv.drain()
        wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    cl = st.get("cluster", {})
    return {
        "metric": "serving p99 job latency (clustering jobs, arrival to result)",
        "value": round(cl.get("p99_ms", float("nan")), 1), "unit": "ms", "n_gpus": 1,
        "steps": len(arrivals), "warmup": len(warm), "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": SERVING_WORKLOAD, "slots": 4,
                                        "hbm_budget_gb": 32},
        "latency_ms": {k: st[k] for k in ("cluster", "query") if k in st},
        # both over the cells of every job (clustering and query): offered over the
        # arrival span, served over first start to last result, which includes the
        # drain after the last arrival
        "served_gcups": round(st.get("served_gcups", 0.0), 1),
        "offered_gcups": round(st.get("cells", 0) / span / 1e9, 1),
        "jobs": {"offered": len(arrivals), "completed": st.get("jobs", 0)},
        "drain_s": round(st.get("drain_s", float("nan")), 3),
        "wall_s": round(wall, 2), "arrival_span_s": round(span, 2),
        "queue_high_water": st["queue_high_water"], "clocks": clk.summary(), "impl": "dtwgb",
    }


# ----------------------------------------------------------------- learned proposals

LEARNED_N, LEARNED_T, LEARNED_W, LEARNED_K = 20000, 256, 25, 10
LEARNED_WORKLOAD = ("N=20000 series x L=256, five-class synthetic, w=25 (10 %), k=10; encoder "
                    "trained on the exact DTW of 633 series (200,028 pairs)")


def encoder_train_flops(S: int, T: int) -> float:
    """Algorithmic FLOPs of one full-batch training step: per series, the two 64->64
    convolutions forward, backward-data and weight-gradient (6 x T*64*64*7*2) plus the
    1->64 convolution forward and weight-gradient (2 x T*64*7*2)."""
    return S * (6 * T * 64 * 64 * 7 * 2 + 2 * T * 64 * 7 * 2)


def encoder_step_ms(v, o, S, T, w, steps, warm=3, graph=True):
    """Mean CUDA-event time of one full-batch training step (S series of length T)."""
    import torch

    from paper_2307_04904_gb300 import api

    n = o.numel() - 1
    enc = api.Encoder(T, max(S, 2))
    enc.init_params(0)
    D = api.dtw_pairwise(v[:S * T], o[:S + 1], w)
    tgt = api.Encoder.targets(D)
    x = v.view(n, T)[:S]
    enc.train(x, tgt, 3e-3, warm, graph=graph)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    enc.train(x, tgt, 3e-3, steps, graph=graph)
    e1.record(st)
    torch.cuda.synchronize()
    enc.close()
    return e0.elapsed_time(e1) / steps


def run_encoder(args):
    """The encoder's training step alone: S=633 series (200,028 target pairs) of length 256."""
    import torch

    from paper_2307_04904_gb300 import synth

    dev = torch.device("cuda", 0)
    S, T = 633, LEARNED_T
    values, offsets, _ = synth.five_class_set(S, T, seed=3)
    v = torch.from_numpy(values).to(dev)
    o = torch.from_numpy(offsets).to(dev)
    with ClockSampler(0) as clk:
        step_ms = encoder_step_ms(v, o, S, T, LEARNED_W, steps=args.steps, warm=args.warmup)
    flops = encoder_train_flops(S, T)
    tflops = flops / (step_ms / 1e3) / 1e12
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
    cpu = None
    if not args.no_cpu_baseline:
        import numpy as np

        from oracle import encoder_ref

        Sc = 12  # a bounded sample: the float64 reference step on 12 series
        xs = values[:Sc * T].reshape(Sc, T).astype(np.float64)
        pa, pb = np.triu_indices(Sc, 1)
        tc0 = time.perf_counter()
        encoder_ref.backward(encoder_ref.init_params(0).astype(np.float64), xs, pa, pb,
                             np.ones(len(pa)))
        dt = time.perf_counter() - tc0
        cpu = {"value": round(encoder_train_flops(Sc, T) / dt / 1e12, 6), "unit": "TFLOP/s",
               "cores": 1, "kind": "oracle",
               "sample": f"float64 numpy reference (single-threaded einsum), forward + backward of "
                         f"{Sc} series x {T}: {dt:.2f} s"}
    return {
        "metric": "encoder training step TFLOP/s (algorithmic convolution FLOPs)",
        "value": round(tflops, 2), "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"encoder full-batch Adam step, S={S} series x T={T}, "
                               "one CUDA graph replay per step",
                   "flops_per_step": flops,
                   "l2": "activations (about 0.3 GB) exceed L2"},
        "roofline": {"bound": "tensor", "achieved": round(tflops, 2), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(tflops / peak, 4), "traffic": None,
                     "kernel": "whole training step, bf16 of measured cuBLAS burst"},
        "cpu_baseline": cpu, "clocks": clk.summary(), "impl": "dtwgb",
    }


def embedding_rank_correlation(emb, values_t, offsets_t, w, n, pairs=20000, seed=5):
    """Spearman correlation between embedding distance and sqrt(exact DTW) over random pairs
    (ties broken by position; the distances are continuous)."""
    import numpy as np
    import torch

    from paper_2307_04904_gb300 import api

    rng = np.random.default_rng(seed)
    pa = torch.as_tensor(rng.integers(0, n, pairs), dtype=torch.int32, device=emb.device)
    pb = torch.as_tensor(rng.integers(0, n, pairs), dtype=torch.int32, device=emb.device)
    d = api.dtw_pairs(values_t, offsets_t, pa, pb, w).double().cpu().numpy()
    e = emb.double()
    de = (e[pa.long()] - e[pb.long()]).norm(dim=1).cpu().numpy()

    def rank(a):
        r = np.empty(len(a))
        r[np.argsort(a, kind="stable")] = np.arange(len(a))
        return r

    return float(np.corrcoef(rank(de), rank(np.sqrt(d)))[0, 1])


def run_learned(args):
    """Learned-proposal k-medoids on the 20000 x 256 set (k = 10) against plain k-medoids,
    the same pipeline with the encoder untrained, and the pipeline without embeddings
    (screening-only lazy fit from seeded random medoids), on the same seeds."""
    import numpy as np
    import torch

    from paper_2307_04904_gb300 import api, learned, synth

    dev = torch.device("cuda", 0)
    values, offsets, _ = synth.five_class_set(LEARNED_N, LEARNED_T, seed=3)
    v = torch.from_numpy(values).to(dev)
    o = torch.from_numpy(offsets).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    n, T, w, k = LEARNED_N, LEARNED_T, LEARNED_W, LEARNED_K
    for _ in range(args.warmup):  # kernels, pools and graphs warm (not timed)
        learned.fit(v[:2000 * T], o[:2001], w, k, train_series=200, steps=5)
    learned.plain_fit(v, o, w, k, torch.arange(k, dtype=torch.int32, device=dev))

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    legs = {"trained": dict(), "untrained": dict(steps=0), "no_embedding": dict(embed=False)}
    rows = []
    rho = {}
    with ClockSampler(0) as clk:
        for s in range(args.steps):
            init = torch.as_tensor(synth.init_medoids(n, k, s), dtype=torch.int32, device=dev)
            p, tp = timed(lambda: learned.plain_fit(v, o, w, k, init))
            row = dict(seed=s, plain_s=tp, plain_cost=p["cost"], plain_iters=p["iters"])
            for name, kw in legs.items():
                r, t = timed(lambda: learned.fit(v, o, w, k, seed=s, rounds=4,
                                                 target_cost=p["cost"], **kw))
                row[name] = dict(s=t, cost=r["cost"], rounds=r["rounds"], pairs=r["pairs"],
                                 reached=r["cost"] <= p["cost"] * (1 + learned.REACH_RTOL),
                                 stage_ms=r["times_ms"])
                if s == 0 and r["embeddings"] is not None:
                    rho[name] = round(embedding_rank_correlation(r["embeddings"], v, o, w, n), 4)
            rows.append(row)
    S = 633
    step_ms = encoder_step_ms(v, o, S, T, w, steps=20)
    tflops = encoder_train_flops(S, T) / (step_ms / 1e3) / 1e12
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]

    def leg_summary(name):
        ts = [r[name]["s"] for r in rows]
        # a leg that does not reach the plain cost falls back to plain k-medoids
        tf = [r[name]["s"] + (0.0 if r[name]["reached"] else r["plain_s"]) for r in rows]
        return {"reached": f"{sum(r[name]['reached'] for r in rows)}/{len(rows)}",
                "median_s": round(float(np.median(ts)), 4),
                "mean_s_with_plain_fallback": round(float(np.mean(tf)), 4),
                "median_s_with_plain_fallback": round(float(np.median(tf)), 4),
                "cost_mean": round(float(np.mean([r[name]["cost"] for r in rows])), 1),
                "dtw_pairs_median": int(np.median([r[name]["pairs"] for r in rows]))}

    plain_med = float(np.median([r["plain_s"] for r in rows]))
    value = leg_summary("trained")["median_s"]
    pairs_full = n * (n - 1) // 2
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        rng = np.random.default_rng(11)
        cores = os.cpu_count() or 1
        a = rng.integers(0, n, 20000)
        b = rng.integers(0, n, 20000)
        tc0 = time.perf_counter()
        oracle.pairs(values, offsets, a, b, w, threads=cores)
        dt = time.perf_counter() - tc0
        cpu = {"value": round(dt / len(a) * pairs_full, 1), "unit": "s", "cores": cores,
               "kind": "oracle",
               "sample": f"float64 DTW of 20000 random pairs in {dt:.2f} s, scaled to the "
                         f"{pairs_full} pairs of the plain method's matrix (k-medoids excluded)"}
    return {
        "metric": "k-medoids seconds to reach the plain method's exact DTW cost (learned proposals)",
        "value": value, "unit": "s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(value * 1e3, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 DTW, bf16 encoder",
        "data": "synthetic",
        "config": {"workload": LEARNED_WORKLOAD, "train_steps": 20, "candidates": 8,
                   "screen_sample": 32, "screen_keep": 8, "max_rounds": 4,
                   "reach_rtol": learned.REACH_RTOL, "seeds": args.steps,
                   "l2": "flushed before every timed fit; the 1.6 GB matrix exceeds L2"},
        "compare": {
            "plain_s_median": round(plain_med, 4),
            "speedup_vs_plain": round(plain_med / value, 2),
            "dtw_pairs_plain": pairs_full,
            "legs": {name: leg_summary(name) for name in legs},
            "embedding_rank_correlation_with_dtw": rho,
            "plain_cost_mean": round(float(np.mean([r["plain_cost"] for r in rows])), 1),
        },
        "per_seed": rows,
        "cpu_baseline": cpu,
        "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak,
                     "unit": "TFLOP/s", "frac": round(tflops / peak, 4), "traffic": None,
                     "kernel": f"encoder training step (S={S}, T={T}), {step_ms:.3f} ms, "
                               "bf16 of measured cuBLAS burst"},
        "clocks": clk.summary(), "impl": "dtwgb",
    }


# ------------------------------------------------------- cluster quality, PAM

def run_cluster(args):
    """Silhouette, elbow curve and PAM swap refinement on the DTW matrix of the
    20000 x 256 set (w = 25): the matrix (1.6 GB) exceeds L2, so each PAM pass and
    the silhouette stream it from HBM."""
    import torch

    from paper_2307_04904_gb300 import api, quality, synth

    dev = torch.device("cuda", 0)
    n, T, w, k = args.n or LEARNED_N, LEARNED_T, LEARNED_W, LEARNED_K
    values, offsets, _ = synth.five_class_set(n, T, seed=3)
    v = torch.from_numpy(values).to(dev)
    o = torch.from_numpy(offsets).to(dev)
    D = api.dtw_pairwise(v, o, w)
    init = torch.as_tensor(synth.init_medoids(n, k, 0), dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):  # kernels and pools warm (small problem)
        api.kmedoids_pam(D[:512, :512].contiguous(), 3)
    with ClockSampler(0) as clk:
        (med, lab, alt_cost, alt_iters), t_alt = timed(lambda: api.kmedoids_fit(D, k, init))
        (pm, pl, pam_cost, swaps), t_pam = timed(lambda: api.kmedoids_pam(D, k, med))
        (_, sil), t_sil = timed(lambda: api.kmedoids_silhouette(D, pl, k))
        (_, _, build_cost, build_swaps), t_build = timed(lambda: api.kmedoids_pam(D, k, None, 0))
        el, t_elbow = timed(lambda: quality.elbow(D, 12, seed=0))
    passes = swaps + 1
    pass_s = t_pam / passes
    cpu = None
    if not args.no_cpu_baseline:
        import numpy as np

        import oracle
        from oracle import cluster_ref

        # a bounded sample: float64 reference swap passes over the exact DTW matrix of the
        # first ns series, each from another seeded medoid set (about 10 s of CPU work)
        ns, reps = min(n, 1000), 5
        a, b = np.triu_indices(ns, 1)
        Ds = np.zeros((ns, ns))
        Ds[a, b] = Ds[b, a] = oracle.pairs_f32_mirror(values, offsets, a, b, w)
        tc0 = time.perf_counter()
        for r in range(reps):
            cluster_ref.swap_deltas(Ds, list(synth.init_medoids(ns, k, r)))
        dt = (time.perf_counter() - tc0) / reps
        cpu = {"value": round(dt * (n / ns) ** 2, 1), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"float64 reference swap pass on the first {ns} series, {reps} passes "
                         f"from seeded medoid sets, {dt:.2f} s each, scaled by (n / {ns})^2 to one "
                         f"pass at n = {n}"}
    gbs = n * n * 4 / pass_s / 1e9
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    return {
        "metric": "PAM swap pass over the DTW matrix (s per pass, every delta(o, i) from one read of D)",
        "value": round(pass_s, 6), "unit": "s", "n_gpus": 1, "steps": passes, "warmup": args.warmup,
        "ms_per_step": round(pass_s * 1e3, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 D, compensated f32 segment sums, f64 across segments",
        "data": "synthetic",
        "config": {"workload": f"N={n} x L={T} five-class synthetic, w={w}, k={k}; "
                               f"D is {n * n * 4 / 1e9:.2f} GB",
                   "l2": "D exceeds L2: every pass reads it from HBM"},
        "compare": {
            "alternate_cost": round(alt_cost, 1), "alternate_s": round(t_alt, 4),
            "pam_from_alternate_cost": round(pam_cost, 1), "pam_swaps": swaps,
            "pam_total_s": round(t_pam, 3),
            "pam_build_cost": round(build_cost, 1), "pam_build_s": round(t_build, 3),
            "silhouette_of_pam": round(sil, 6), "silhouette_s": round(t_sil, 4),
            "silhouette_gbs": round(n * n * 4 / t_sil / 1e9, 1),
            "elbow_k": el["elbow"], "elbow_costs": {str(a): round(b, 1) for a, b in el["costs"].items()},
            "elbow_silhouette": {str(a): round(b, 4) for a, b in el["silhouette"].items()},
            "elbow_s": round(t_elbow, 3),
        },
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "traffic": None,
                     "kernel": "PAM swap pass (nearest medoids, member lists, segment sums of the "
                               "two FastPAM1 terms, deltas, argmin, host check): n^2 x 4 B of D "
                               "per pass, of measured copy bandwidth"},
        "cpu_baseline": cpu, "clocks": clk.summary(), "impl": "dtwgb",
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="pairwise",
                    choices=["pairwise", "ragged", "serving", "learned", "encoder", "cluster"],
                    help="pairwise: the benchmark line (2000 x 512); ragged: the batched "
                         "ragged-set measurement; serving: the Poisson job stream; learned: "
                         "k-medoids with learned proposals against the plain method; encoder: "
                         "the proposal encoder's training step; cluster: PAM, silhouette and "
                         "elbow over the 20000-series matrix")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dtwgb", choices=["dtwgb", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0,
                    help="cluster workload only: series count in place of 20000 (a smaller "
                         "case for profiler captures)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "ragged":
        print(json.dumps(run_ragged(args)), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "learned":
        print(json.dumps(run_learned(args)), flush=True)
        return
    if args.workload == "encoder":
        print(json.dumps(run_encoder(args)), flush=True)
        return
    if args.workload == "cluster":
        print(json.dumps(run_cluster(args)), flush=True)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_gpu(args, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
