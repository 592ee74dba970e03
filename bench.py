#!/usr/bin/env python
"""Throughput of FFT-accelerated Core AFD (arXiv:1711.08604) on GB300.

Workload (default): one signal of N = 4096 samples (20 seeded tones with
amplitude 1/f plus noise, positive-frequency projected), M = 200 radii i/200,
K = 50 greedy steps, FP32 grid with FP64 guard and update.  One bench step is
one whole decomposition (all K greedy steps: forward FFT, M inverse FFTs with
the fused objective and argmax, FP64 guard, remainder update, energy).

Metric: grid evaluations per second, M * N * K / time, with the input resident
in device memory when the timed region starts; L2 is flushed (a 256 MiB write)
between timed steps, outside the timed intervals.  Also reported: signals/s,
p50/p99 latency per decomposition, end-to-end figures through the C ABI from
pinned host memory, the grid kernel's roofline, SM clocks sampled during the
timed region, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl afd|reference]
                  [--precision fp32|fp64]
For N > 1 launch with torch.distributed.run; every rank decomposes its own
copy of the workload (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
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

METRIC = "AFD grid evals/s (M*N*K/s)"
UNIT = "grid_evals/s"
N_SIG, M_RAD, K_STEPS = 4096, 200, 50
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128
STEPREC_BYTES, SLOTCTL_BYTES = 80, 64  # StepRec, SlotCtl


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("afd_kernels.cu", "afd_device.cuh", "afd_fft.cuh", "afd_internal.h"):
        with open(os.path.join(ROOT, "paper_1711_08604_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel sources changed since that capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_sources_sha256_16") != kernel_sources_hash():
        return None
    return rec["dram_bytes_per_launch"]


def workload():
    from paper_1711_08604_gb300 import workloads as W
    return W.tones(N=N_SIG, M=M_RAD, K=K_STEPS)


def workload_name(prec: str) -> str:
    return (f"tones: single signal N={N_SIG}, M={M_RAD} radii i/{M_RAD}, K={K_STEPS} steps, "
            + ("FP32 grid + FP64 guard/update" if prec == "fp32" else "FP64 plain"))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.file = gpu, None, None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.proc or not self.file:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = [float(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(rows),
                "reasons": reasons}


def aggregate(local_ms: float, local_units: float, world_size: int):
    """Whole-job time and units over the ranks of an independent-replica run:
    the slowest rank's time (MAX) and the units of all ranks (SUM).  With one
    rank, the local figures."""
    if world_size <= 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_baseline(s, sample_steps: int = 2) -> dict:
    """The FP64 oracle, as it stands, on the host cores: the first sample_steps
    greedy steps of the same workload (full M x N grid each)."""
    import oracle
    t0 = time.perf_counter()
    d = oracle.decompose(s.G, s.radii, sample_steps)
    dt = time.perf_counter() - t0
    evals = s.M * s.N * d["steps"]
    out = {"value": evals / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"first {d['steps']} of {s.K} greedy steps of the same workload "
                     f"(direct O(M N^2) grid, {evals} grid evals, {dt:.2f} s)"}
    out["single_thread"] = _oracle_single_thread(oracle, s)
    out["other_configs"] = _oracle_other_configs(oracle)
    return out


def _oracle_single_thread(oracle, s) -> dict:
    """The same oracle on one host thread: one greedy step over every 8th radius."""
    sub = s.radii[::8]
    n0 = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        d = oracle.decompose(s.G, sub, 1)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(n0)
    evals = len(sub) * s.N * d["steps"]
    return {"value": evals / dt, "unit": UNIT, "cores": 1,
            "sample": f"1 greedy step over {len(sub)} of the {s.M} radii ({evals} grid evals, {dt:.2f} s)"}


def _oracle_other_configs(oracle) -> dict:
    """The oracle on all host threads for the other workloads: the kernel sum
    (N = 256, M = 50, K = 10) in full; the batch and the chirp (N = 65536,
    M = 1000, K = 100) on bounded samples, extrapolated by their M N^2 K."""
    from paper_1711_08604_gb300 import workloads as W
    k1 = W.kernel_sum()
    t0 = time.perf_counter()
    d = oracle.decompose(k1.G, k1.radii, k1.K)
    dt1 = time.perf_counter() - t0
    c5 = W.chirp()
    sub = c5.radii[::500]
    t0 = time.perf_counter()
    d5 = oracle.decompose(c5.G, sub, 1)
    dt5 = time.perf_counter() - t0
    # the batch workload (1024 signals, N in {1024..8192}, M = 100, K = 30): one
    # greedy step over 10 radii of its first 16 signals gives the oracle's rate
    # in terms (grid evals x N) per second, extrapolated to the whole batch
    sigs = W.batch()
    t0 = time.perf_counter()
    terms = 0
    for sg in sigs[:16]:
        db = oracle.decompose(sg.G, sg.radii[::10], 1)
        terms += len(sg.radii[::10]) * sg.N * sg.N * db["steps"]
    dtb = time.perf_counter() - t0
    rate = terms / dtb
    total = sum(sg.M * sg.N * sg.N * sg.K for sg in sigs)
    return {
        "batch_extrapolated": {"value": sum(sg.M * sg.N * sg.K for sg in sigs) / (total / rate), "unit": UNIT,
                               "s_per_batch": total / rate,
                               "sample": f"1 greedy step over 10 radii of 16 of the {len(sigs)} signals "
                                         f"({dtb:.2f} s), extrapolated by M N^2 K per signal"},
        "kernel_sum_full": {"value": k1.M * k1.N * d["steps"] / dt1, "unit": UNIT,
                            "s_per_decomposition": dt1, "sample": "N=256, M=50, K=10 in full"},
        "chirp_extrapolated": {"value": len(sub) * c5.N * d5["steps"] / dt5, "unit": UNIT,
                               "s_per_decomposition": dt5 * (c5.M / len(sub)) * (c5.K / d5["steps"]),
                               "sample": f"1 greedy step over {len(sub)} of the {c5.M} radii "
                                         f"({dt5:.2f} s), extrapolated linearly in M K"},
    }


def _run_batch(afd, torch, sigs, packed, persistent, reps: int):
    b = afd.afd_batch_create([x.N for x in sigs], sigs[0].radii, 30, persistent=persistent)
    afd.afd_batch_run(b, packed)  # warm-up (graph capture, autotuner)
    torch.cuda.synchronize()
    l0 = afd.afd_batch_counters(b)["kernel_launches"]
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        r = afd.afd_batch_run(b, packed)
        times.append(time.perf_counter() - t0)
    tuning = afd.afd_batch_tuning(b)
    launches = afd.afd_batch_counters(b)["kernel_launches"] - l0
    b.close()
    return r, min(times), tuning, launches


def bench_batch(afd, torch, dev, reps: int = 3) -> dict:
    """Workload 3: 1024 signals of uneven N in {1024..8192}, M = 100, K = 30, one
    batch: per-N launches on parallel streams replayed as a CUDA graph (the
    default; grid-kernel variants by the autotuner), and, for comparison, all K
    steps of every signal in one multi-signal persistent launch
    (persistent=2)."""
    from paper_1711_08604_gb300 import workloads as W
    sigs = W.batch()
    packed = torch.from_numpy(np.concatenate([x.G for x in sigs])).to(dev)
    r2, t2, _, launches2 = _run_batch(afd, torch, sigs, packed, 2, reps)
    r, t, tuning, launches = _run_batch(afd, torch, sigs, packed, True, reps)
    assert all(np.array_equal(a, b) for a, b in zip(r["coeff"], r2["coeff"]))
    evals = sum(int(x.M) * x.N * int(st) for x, st in zip(sigs, r["steps"]))
    flops = sum(int(x.M) * x.N * int(st) * (5 * int(np.log2(x.N)) + 6) for x, st in zip(sigs, r["steps"]))
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    return {"workload": "batch: 1024 signals, N in {1024,2048,4096,8192}, M=100, K=30, FP32+FP64 guard",
            "grid_evals_per_s": evals / t, "signals_per_s": len(sigs) / t, "s_per_batch": t,
            "path": "per-N kernels on parallel streams, replayed as a CUDA graph (grid variants by the autotuner)",
            "launches_per_batch": launches / reps,
            "timing": "host wall clock around afd_batch_run (device-resident input), best of %d" % reps,
            "grid_fp32_tflops": flops / t / 1e12,
            "grid_fp32_frac_of_peak": flops / t / 1e12 / peak,
            "autotuner": {str(q["N"]): {"variant": ["default", "32 points/thread", "512-thread CTAs"][q["variant"]],
                                        "grid_us": q["us"]} for q in tuning},
            "multi_signal_path": {"grid_evals_per_s": evals / t2, "s_per_batch": t2,
                                  "launches_per_batch": launches2 / reps,
                                  "note": "all K steps of every signal in one cooperative persistent launch "
                                          "(persistent=2; the serving ticks' path); bitwise the same results"},
            "fp32_note": "grid flops (5 log2 N + 6 per grid evaluation) over the whole batch time, "
                         "FP64 guard/update and forward FFTs included in the time; peak derived: "
                         f"{sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x 2070 MHz"}


def hbm_peak_gbs() -> tuple:
    """Measured HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json), else
    the fallback figure of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (earlier GB300 copy measurement)"


def bench_chirp(afd, torch, dev, reps: int = 3) -> dict:
    """Workload 5: one decomposition of N = 65536 (two-pass HBM-staged FFT),
    M = 1000 radii i/1000, K = 100.  Grid evals/s over the whole decomposition,
    and the two-pass grid stage against HBM bandwidth: pass 1 writes and pass 2
    reads the M x N FP32 intermediate, 16 M N bytes per step."""
    from paper_1711_08604_gb300 import workloads as W
    s = W.chirp()
    stream = torch.cuda.Stream(device=dev)
    plan = afd.afd_plan_create(s.N, s.radii, device=dev.index, stream=stream.cuda_stream, use_graph=True)
    Gd = torch.from_numpy(s.G).to(dev)
    K = s.K
    out = {"a": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "coeff": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "delta": torch.zeros(K + 1, dtype=torch.float64, device=dev),
           "idx": torch.zeros(2 * K, dtype=torch.int32, device=dev)}

    def once():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = afd.afd_decompose(plan, Gd, K, 0.0, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        assert r["steps"] == K
        return e0.elapsed_time(e1)

    once()
    ms = min(once() for _ in range(reps))
    afd.afd_plan_set_profiling(plan, True)
    once()
    afd.afd_plan_reset_counters(plan)
    once()
    kt = afd.afd_plan_kernel_times(plan)
    afd.afd_plan_set_profiling(plan, False)
    plan.close()
    grid_ms, grid_launches = kt["grid"]
    steps = grid_launches // 2  # pass 1 + pass 2 per step
    bytes_per_step = 16 * s.M * s.N
    gbs = bytes_per_step * steps / (grid_ms * 1e-3) / 1e9 if grid_ms > 0 else 0.0
    peak, src = hbm_peak_gbs()
    return {"workload": "large: N=65536 two-pass FFT, M=1000 radii i/1000, K=100, FP32 grid + FP64 guard/update",
            "ms_per_decomposition": ms, "grid_evals_per_s": s.M * s.N * K / (ms * 1e-3),
            "timing": "CUDA events around afd_decompose (device-resident input), best of %d" % reps,
            "kernels_ms": {k: {"launches": n, "total_ms": t} for k, (t, n) in kt.items()},
            "roofline_two_pass_grid": {"bound": "hbm", "kernel": "k_grid2_pass1 + k_grid2_pass2",
                                       "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                       "peak_source": src,
                                       "bytes_per_step": bytes_per_step,
                                       "bytes_note": "pass-1 write + pass-2 read of the M x N FP32 "
                                                     "intermediate; the spectrum and tables are L2-resident",
                                       "ms_per_step": grid_ms / max(1, steps)}}


def bench_single(afd, torch, dev, sig, precision, reps: int = 20, plan=None, grid_angles=None, **plan_kw) -> dict:
    """One signal's whole decomposition through afd_decompose (device-resident
    input; CUDA events on the plan's stream), best of `reps`.  plan: an
    existing plan (its stream is used); grid_angles: angles of the grid when
    they are not the samples (non-uniform plans)."""
    if plan is None:
        stream = torch.cuda.Stream(device=dev)
        plan = afd.afd_plan_create(sig.N, sig.radii, precision=precision, device=dev.index,
                                   stream=stream.cuda_stream, use_graph=True, **plan_kw)
    else:
        stream = torch.cuda.ExternalStream(afd.afd_plan_get_stream(plan), device=dev)
    Gd = torch.from_numpy(sig.G).to(dev)
    K = sig.K
    out = {"a": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "coeff": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "delta": torch.zeros(K + 1, dtype=torch.float64, device=dev),
           "idx": torch.zeros(2 * K, dtype=torch.int32, device=dev)}
    times = []
    for i in range(reps + 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        afd.afd_decompose(plan, Gd, K, 0.0, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            times.append(e0.elapsed_time(e1))
    plan.close()
    ms = min(times)
    L = grid_angles or sig.N
    return {"ms_per_decomposition": ms, "p50_ms": float(np.percentile(times, 50)),
            "p99_ms": float(np.percentile(times, 99)), "grid_evals_per_s": sig.M * L * K / (ms * 1e-3),
            "signals_per_s": 1e3 / ms,
            "timing": "CUDA events around afd_decompose (device-resident input), min / p50 / p99 of %d" % reps}


def bench_next(afd, torch, dev, reps: int = 10) -> dict:
    """The NEXT rows, one signal each, FP32 grid + FP64 guard: a mixed-radix
    size (N = 3000 = 2^3 3 5^3), non-uniform samples (3000 jittered angles,
    L = 1024 grid angles), the renormalised objective and the off-grid
    refinement on workload 2."""
    from paper_1711_08604_gb300 import workloads as W
    fp32 = afd.AFD_FP32_GUARDED
    out = {}
    mixed = W.tones(item=5, N=3000, M=100, K=20)
    out["mixed_radix"] = dict(bench_single(afd, torch, dev, mixed, fp32, reps=reps),
                              workload="tones: N=3000 (2^3 3 5^3, mixed radix), M=100, K=20")
    x = W.nonuniform()
    stream = torch.cuda.Stream(device=dev)
    plan = afd.afd_plan_create_nonuniform(x.theta, x.radii, x.L, weights=x.weights, device=dev.index,
                                          stream=stream.cuda_stream, use_graph=True)
    out["nonuniform"] = dict(bench_single(afd, torch, dev, x, fp32, reps=reps, plan=plan, grid_angles=x.L),
                             workload="non-uniform: %d jittered samples, L=%d grid angles, M=%d, K=%d"
                                      % (x.N, x.L, x.M, x.K))
    t = W.tones()
    out["renormalised"] = dict(bench_single(afd, torch, dev, t, fp32, reps=reps, renormalise=True),
                               workload="tones: N=4096, M=200, K=50, renormalised objective")
    # off-grid refinement of every step's point (not in the paper): time, and
    # the relative error after K steps against the grid-only decomposition
    out["offgrid"] = dict(bench_single(afd, torch, dev, t, fp32, reps=reps, offgrid_iters=20),
                          workload="tones: N=4096, M=200, K=50, points refined off the grid (<= 20 Newton steps)")
    for key, kw in (("delta_K_offgrid", {"offgrid_iters": 20}), ("delta_K_grid", {})):
        plan = afd.afd_plan_create(t.N, t.radii, precision=fp32, device=dev.index, **kw)
        out["offgrid"][key] = float(afd.afd_decompose(plan, t.G, t.K)["delta"][-1])
        plan.close()
    return out


def bench_serve(afd, duration: float = 10.0, fp64_every: int = 25) -> dict:
    """Workload 4: Poisson arrivals at 2000 req/s for `duration` seconds; N in
    {512..16384}, M = 128, stop at delta <= 1e-4 or K = 64; 40 GB admission
    budget.  Latency is submission to completion.  Every fp64_every-th request
    of the same stream (a systematic sample of the whole mix, N = 16384
    included) is also run one by one through FP64-plain plans for the
    signals/s comparison."""
    import threading
    from paper_1711_08604_gb300 import workloads as W
    reqs = W.serving_requests(duration=duration)
    srv = afd.afd_serve_create(40 << 30)
    # warm the plan cache so table building is not inside the measurement
    warm = {}
    for _, x in reqs:
        warm.setdefault(x.N, x)
    for x in warm.values():
        afd.afd_serve_wait(srv, afd.afd_serve_submit(srv, x.G, x.radii, 2, 0.0), 120.0)
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def submit():
        for i, (t, x) in enumerate(reqs):
            while time.perf_counter() - t0 < t:
                time.sleep(0.0002)
            ids[i] = afd.afd_serve_submit(srv, x.G, x.radii, x.K, x.tol)

    th = threading.Thread(target=submit)
    th.start()
    th.join()
    outs = [afd.afd_serve_wait(srv, i, 600.0) for i in ids]
    t_all = time.perf_counter() - t0
    st = afd.afd_serve_get_stats(srv)
    # capacity: the same requests all submitted at once
    t2 = time.perf_counter()
    ids2 = [afd.afd_serve_submit(srv, x.G, x.radii, x.K, x.tol) for _, x in reqs]
    for i in ids2:
        afd.afd_serve_wait(srv, i, 600.0)
    capacity = len(reqs) / (time.perf_counter() - t2)
    srv.close()
    lat = np.array([o["latency_ms"] for o in outs])
    evals = sum(x.M * x.N * o["steps"] for (_, x), o in zip(reqs, outs))
    served = len(reqs) / t_all
    # plain FP64 single-signal path, requests one after another
    sample = [x for _, x in reqs][::fp64_every]
    plans = {}
    t1 = time.perf_counter()
    for x in sample:
        if x.N not in plans:
            plans[x.N] = afd.afd_plan_create(x.N, x.radii, precision=afd.AFD_FP64_PLAIN)
            afd.afd_decompose(plans[x.N], x.G, 2, 0.0)
    t1 = time.perf_counter()
    for x in sample:
        afd.afd_decompose(plans[x.N], x.G, x.K, x.tol)
    fp64_rate = len(sample) / (time.perf_counter() - t1)
    for p in plans.values():
        p.close()
    return {"workload": f"serving: Poisson 2000 req/s for {duration:g} s, N in 512..16384, M=128, "
                        "delta<=1e-4 or K=64, 40 GB budget",
            "requests": len(reqs), "signals_per_s": served, "grid_evals_per_s": evals / t_all,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "ticks": st["ticks"], "kernel_launches": st["kernel_launches"], "failed": st["failed"],
            "capacity_signals_per_s": capacity,
            "fp64_plain_single_signal_per_s": fp64_rate,
            "capacity_vs_fp64_plain": capacity / fp64_rate,
            "fp64_plain_sample": f"every {fp64_every}th request of the same stream ({len(sample)} requests, "
                                 f"N = {min(x.N for x in sample)}..{max(x.N for x in sample)}), "
                                 "one after another, one FP64-plain plan per N",
            "note": "served signals/s is bounded by the offered 2000 req/s; capacity: all requests "
                    "submitted at once (FP32+FP64-guarded continuous batching)"}


def bench_paper_sweep(afd, reps: int = 20) -> dict:
    """The N-sweep of Table 9 (Sec. 4.2): f1 on N = 128..4096 points, radii
    0, 0.1, ..., 0.8, 10 steps (a_1 = 0 imposed, as Tables 4 and 6 read);
    milliseconds per decomposition, FP32 + FP64 guard.  The paper's Matlab
    times on one CPU thread are context, not a target."""
    from paper_1711_08604_gb300 import workloads as W
    out = {}
    for N in (128, 256, 512, 1024, 2048, 4096):
        G = W.paper_f1(N)
        plan = afd.afd_plan_create(N, W.radii_paper(), force_a1_zero=True)
        afd.afd_decompose(plan, G, 10)
        t0 = time.perf_counter()
        for _ in range(reps):
            afd.afd_decompose(plan, G, 10)
        out[str(N)] = 1e3 * (time.perf_counter() - t0) / reps
        plan.close()
    return {"workload": "Table 9 sweep: f1, radii 0..0.8, 10 steps", "ms_per_decomposition": out,
            "timing": f"host wall clock per afd_decompose call (host input and outputs), mean of {reps}"}


def run_reference(args):
    """Reference arm: the CPU oracle on a bounded sample of the workload per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    s = workload()
    sub = s.radii[:: 8]                       # 25 of the 200 radii
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.decompose(s.G, sub, 1)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    evals = sub.size * s.N
    value = evals * len(times) / sum(times)
    sample = (f"one greedy step of the workload over {sub.size} of its {s.M} radii "
              f"(every 8th), direct O(M N^2) grid")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.precision), "N": s.N,
                                            "M": s.M, "K": s.K, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_afd(args):
    import torch
    import paper_1711_08604_gb300 as afd

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    afd._native.load()
    s = workload()
    prec = afd.AFD_FP32_GUARDED if args.precision == "fp32" else afd.AFD_FP64_PLAIN
    stream = torch.cuda.Stream(device=dev)
    plan = afd.afd_plan_create(s.N, s.radii, precision=prec, device=local, stream=stream.cuda_stream,
                               use_graph=True)
    K = s.K
    Gd = torch.from_numpy(s.G).to(dev)
    out = {"a": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "coeff": torch.zeros(2 * K, dtype=torch.float64, device=dev),
           "delta": torch.zeros(K + 1, dtype=torch.float64, device=dev),
           "idx": torch.zeros(2 * K, dtype=torch.int32, device=dev)}
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2
    torch.cuda.synchronize()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed_loop(n, G_in, outs):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for e0, e1 in ev:
            with torch.cuda.stream(stream):
                flush.zero_()
            e0.record(stream)
            r = afd.afd_decompose(plan, G_in, K, 0.0, out=outs)
            e1.record(stream)
            assert r["steps"] == K
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    for _ in range(args.warmup):
        timed_loop(1, Gd, out)
    # device-resident timed region
    afd.afd_plan_reset_counters(plan)
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        ms = timed_loop(args.steps, Gd, out)
        barrier()
        t_wall = time.perf_counter() - t_wall
    launches = afd.afd_plan_counters(plan)["kernel_launches"]
    evals_per_step = s.M * s.N * K
    total_ms, total_evals = aggregate(sum(ms), evals_per_step * args.steps, ws)
    value = total_evals / (total_ms * 1e-3)

    # Per-kernel device times: the same K steps again, with CUDA events recorded
    # between consecutive kernels inside the replayed graph (event-record nodes
    # on the plan's stream).
    afd.afd_plan_set_profiling(plan, True)
    timed_loop(1, Gd, out)
    afd.afd_plan_reset_counters(plan)
    ms_prof = timed_loop(args.steps, Gd, out)
    ktimes = afd.afd_plan_kernel_times(plan)
    phases = afd.afd_plan_phase_cycles(plan)
    afd.afd_plan_set_profiling(plan, False)

    logn = int(np.log2(s.N))
    flops_per_eval = 5 * logn + 6
    if ktimes["persistent"][1] > 0:
        # one cooperative launch per decomposition: all K steps' grid evaluations
        kname = f"k_persistent<{logn}>"
        k_ms, k_n = ktimes["persistent"]
        evals_per_launch = s.M * s.N * K
    else:
        kname = f"k_grid<float,{logn}>"
        k_ms, k_n = ktimes["grid"]
        evals_per_launch = s.M * s.N
    avg_ms = k_ms / max(1, k_n)
    flops_per_launch = evals_per_launch * flops_per_eval
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    achieved_tflops = flops_per_launch / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved_tflops,
                "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops,
                "traffic": ncu_traffic(kname),
                "traffic_note": "dram read+write bytes per launch from one cold-cache ncu capture "
                                "(profiles/); null if the kernel changed since",
                "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz",
                "grid_evals_per_launch": evals_per_launch,
                "flops_per_eval": f"5*log2(N)+6 = {flops_per_eval}",
                "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_ms}
    prof_total = sum(ms_prof)
    kernel_us = {k: {"launches": n, "avg_us": 1e3 * t / max(1, n), "share": t / max(prof_total, 1e-9)}
                 for k, (t, n) in ktimes.items()}

    # end to end through the C ABI: pinned host input, host outputs, copies timed
    G_pin = torch.from_numpy(s.G).pin_memory()
    for _ in range(2):
        timed_loop(1, G_pin, None)
    barrier()
    e2e_ms = timed_loop(args.steps, G_pin, None)
    e2e_total, e2e_evals = aggregate(sum(e2e_ms), evals_per_step * args.steps, ws)
    e2e = {"value": e2e_evals / (e2e_total * 1e-3), "unit": UNIT,
           # the signal; the slot descriptor is copied only when it changed
           # (first call), not per step
           "h2d_bytes_per_step": 16 * s.N,
           "d2h_bytes_per_step": STEPREC_BYTES * K + SLOTCTL_BYTES}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.precision), "N": s.N, "M": s.M, "K": K,
                       "precision": "f32 grid + f64 guard/update" if args.precision == "fp32" else "f64",
                       "parallelism": f"replicas x{ws}",
                       "l2": "flushed (256 MiB write) between timed steps, outside the timed intervals"},
            "signals_per_s": total_evals / evals_per_step / (total_ms * 1e-3),
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "min": min(ms), "max": max(ms)},
            "wall_s": t_wall,
            "kernels": kernel_us,
            "persistent_phase_cycles_per_step": phases,
            "kernels_note": "device time per kernel from CUDA events inside the replayed graph, "
                            "a second pass of the same steps; share = fraction of that pass",
            "gpu_launches": int(launches),
            "roofline": roofline,
            "e2e": e2e,
            "clocks": clocks,
        }
        # the CPU baseline and the other workloads at N = 1 only: with more
        # ranks they would hold every GPU while rank 0 alone works
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(s)
        if ws == 1 and not args.no_extra:
            from paper_1711_08604_gb300 import workloads as W
            line["other_workloads"] = {
                "c1_kernel_sum": dict(bench_single(afd, torch, dev, W.kernel_sum(), afd.AFD_FP64_PLAIN),
                                      workload="kernel sum: N=256, M=50 radii i/50, K=10, FP64 plain"),
                "c1_kernel_sum_fp32": dict(bench_single(afd, torch, dev, W.kernel_sum(), afd.AFD_FP32_GUARDED),
                                           workload="kernel sum: N=256, M=50 radii i/50, K=10, FP32 grid + FP64 guard"),
                "c2_tones_fp64_plain": dict(bench_single(afd, torch, dev, s, afd.AFD_FP64_PLAIN, reps=10),
                                            workload="tones: N=4096, M=200, K=50, FP64 plain (the comparator)"),
                "batch": bench_batch(afd, torch, dev),
                "large_two_pass": bench_chirp(afd, torch, dev),
                "serving": bench_serve(afd, args.serve_seconds),
                "paper_table9": bench_paper_sweep(afd),
                "next_rows": bench_next(afd, torch, dev)}
        print(json.dumps(line))
    plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["afd", "reference"], default="afd")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch and serving workloads")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--workload", choices=["main", "batch", "serve", "sweep", "large", "next"], default="main",
                    help="main: the contract line; batch / serve / sweep: only that workload's figures "
                         "(for profiling), printed as one JSON object")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "main":
        import torch
        import paper_1711_08604_gb300 as afd
        afd._native.load()
        dev = torch.device("cuda", 0)
        fn = {"batch": lambda: bench_batch(afd, torch, dev), "serve": lambda: bench_serve(afd, args.serve_seconds),
              "sweep": lambda: bench_paper_sweep(afd), "large": lambda: bench_chirp(afd, torch, dev),
              "next": lambda: bench_next(afd, torch, dev)}[args.workload]
        print(json.dumps(fn()))
        return 0
    return run_afd(args)


if __name__ == "__main__":
    sys.exit(main())
