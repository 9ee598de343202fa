#!/usr/bin/env python3
"""Benchmark of the PRNGD bulk fill on GB300 (Demchik and Gulov, arXiv:1401.8230, Section 2).

Step = one launch of the hot path over the bulk workload: 2^20 xorshift128 streams (seed 1)
x 1024 outputs = 2^30 extended-precision uniforms, w = 32, written as correctly rounded
doubles (form B, integer-only), stream-major, 8 GiB. Per step: the draws, accept-reject,
n, conversion and the store of every value; the streams continue from step to step, so
every step produces new numbers. The 8 GiB output exceeds the 129 MB L2, so no flush is
needed between steps.

Prints ONE JSON line (rank 0). Extra keys measure the other forms, w = 24, the fused
statistics mode and the end-to-end host path. `--impl reference` times the CPU oracle
instead (the slow reference arm) on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank fills its own 2^20 streams (rank r takes streams
[r 2^20, (r+1) 2^20) of the same seed); no data exchange; weak scaling.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import re
import statistics
import subprocess
import tempfile
import sys
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 uniforms Gsamples/s & % HBM-write roofline; batched/served p50/p99 vs plain"
UNIT = "Gsamples/s"
SEED = 1
N_STREAMS = 1 << 20
PER_STREAM = 1024
W = 32
GAMMA = 0x9E3779B97F4A7C15
PROFILE = os.path.join(ROOT, "profiles", "fill_b32_bulk_2p30.txt")
KERNEL_SOURCES = ["paper_1401_8230_gb300/csrc/prngd_fill.cuh", "paper_1401_8230_gb300/csrc/prngd_math.cuh"]
STATS_PROFILE = os.path.join(ROOT, "profiles", "stats_kernel_w32_fused.txt")
STATS_SOURCES = ["paper_1401_8230_gb300/csrc/prngd_stats.cuh", "paper_1401_8230_gb300/csrc/prngd_math.cuh"]
# the ALU pipe: 2 warp instructions (64 lanes) per clock per SM (ncu peak_sustained), 152 SMs,
# 2.07 GHz maximum SM clock
ALU_PEAK_GOPS = 152 * 64 * 2.07


def shard_seed(seed: int, rank: int, n_streams: int) -> int:
    """Seed whose streams 0 .. n-1 are streams rank*n .. rank*n + n-1 of `seed`: stream s of a
    seed uses splitmix64 positions 2s+1 and 2s+2 after it, so shifting the seed by 2*rank*n
    gammas shifts every stream by rank*n."""
    return (seed + 2 * rank * n_streams * GAMMA) % 2**64


def max_over_ranks(dist, value: float, device) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_desc():
    if (N_STREAMS, PER_STREAM) == (1 << 20, 1024):
        name = ("bulk fill: 2^20 xorshift128 streams (seed 1) x 1024 outputs = 2^30 uniforms, "
                "w=32, form B values (correctly rounded f64) by the balanced route "
                "(3 of 4 outputs rounded by the u64->f64 conversion; integer-only form B in forms), "
                "stream-major, 8 GiB, one launch")
    else:
        name = f"reduced bulk fill: {N_STREAMS} streams x {PER_STREAM} outputs, w=32, form B (profiling case)"
    return {"workload": name,
            "n_streams": N_STREAMS, "per_stream": PER_STREAM, "w": W, "form": "B", "mode": "PRNG_MODE_BALANCED",
            "output": "f64",
            "arithmetic": "32/64-bit integer draws, accept-reject, n and rounding; the u64->f64 conversion "
                          "instruction rounds 3 of 4 outputs (the same bits)",
            "l2": f"{N_STREAMS * PER_STREAM * 8 / 2**30:.2f} GiB output per step > 129 MB L2: no flush"}


def kernel_hash(sources=None):
    h = hashlib.sha256()
    for rel in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_value(path, sources, key):
    """A figure from a committed ncu summary, if the summary was taken on these kernel sources."""
    try:
        text = open(path).read()
    except OSError:
        return None
    m_h = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    m_t = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_h or not m_t or m_h.group(1) != kernel_hash(sources):
        return None
    return float(m_t.group(1))


def profiled_traffic():
    """DRAM bytes per launch of the bulk fill from its ncu summary."""
    return profiled_value(PROFILE, KERNEL_SOURCES, "dram_bytes_per_launch")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        # raw samples beside the run (only their summary goes into the JSON line)
        self.path = os.path.join(os.environ.get("PRNGD_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"prngd_clocks_rank{device_index}.csv")
        self.dev = device_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # a sampler must not outlive the bench, whatever ends it (an exception in the timed
            # region included): the child is ended at interpreter exit if stop() never ran
            atexit.register(self._end_child)
        except Exception:
            self.proc = None

    def _end_child(self):
        if self.proc and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait(timeout=5)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._end_child()
        atexit.unregister(self._end_child)
        self.fh.close()
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
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle
def oracle_rate(n_streams_sample: int, first: int = 0, threads: int | None = None):
    """Oracle form-B fill of streams [first, first + n) x 1024 on all host cores."""
    import numpy as np

    import oracle as O

    threads = threads or os.cpu_count() or 1
    chunk = max(1, n_streams_sample // (threads * 4))
    jobs = [(s, min(chunk, first + n_streams_sample - s)) for s in range(first, first + n_streams_sample, chunk)]
    O.lib()

    def run(job):
        s, n = job
        out = np.empty(n * PER_STREAM, dtype=np.float64)
        rej = np.empty(n, dtype=np.uint64)
        rc = O.lib().orc_fill(SEED, s, n, PER_STREAM, W, O.FORM_B, out.ctypes.data, rej.ctypes.data)
        assert rc == 0
        return n

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        done = sum(ex.map(run, jobs))
    dt = time.perf_counter() - t0
    return done * PER_STREAM / dt / 1e9, dt, threads


def cpu_baseline(target_s: float = 10.0):
    # calibrate on a small sample, then time a sample sized for ~target_s of wall time
    rate, _, threads = oracle_rate(2048)
    n = int(max(2048, min(N_STREAMS, rate * 1e9 * target_s / PER_STREAM)))
    rate, dt, threads = oracle_rate(n)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"streams 0..{n - 1} of the bulk workload (seed 1, w=32, form B, 1024 outputs each; "
                      f"{n * PER_STREAM} samples, {dt:.1f} s wall on {threads} threads)"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    rate, _, threads = oracle_rate(2048)
    per_step_s = min(2.0, 120.0 / (args.steps + args.warmup))  # whole run within ~2 minutes
    n = int(max(64, min(N_STREAMS, rate * 1e9 * per_step_s / PER_STREAM)))
    for _ in range(args.warmup):
        oracle_rate(max(64, n // 8))
    times, total = [], 0
    for _ in range(args.steps):
        r, dt, threads = oracle_rate(n)
        times.append(dt)
        total += n * PER_STREAM
    value = total / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_desc(), "sample": f"{n} streams x 1024 per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"streams 0..{n - 1} of the bulk workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def time_calls(torch, fn, reps, stream):
    """Average device time of fn() over reps launches, CUDA events on `stream`."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--batched-requests", type=int, default=4096, help="reduce for profiling runs")
    ap.add_argument("--batched-hi", type=int, default=2**26, help="largest request length (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default batch launch shape")
    ap.add_argument("--stats-per-stream", type=int, default=2**16, help="fused-statistics outputs per stream")
    ap.add_argument("--n-streams", type=int, default=None, help="override the stream count (profiling runs)")
    ap.add_argument("--per-stream", type=int, default=None, help="override outputs per stream (profiling runs)")
    args = ap.parse_args()
    global N_STREAMS, PER_STREAM
    N_STREAMS = args.n_streams or N_STREAMS
    PER_STREAM = args.per_stream or PER_STREAM
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_1401_8230_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    seed_r = shard_seed(SEED, rank, N_STREAMS)  # rank r fills streams [r n, (r+1) n) of SEED
    stream = torch.cuda.current_stream()
    g = P.Generator(seed_r, N_STREAMS, W)
    out = torch.empty(N_STREAMS * PER_STREAM, dtype=torch.float64, device="cuda")

    def step():
        g.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_BALANCED, None, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for a, b in evs:
        a.record(stream)
        step()
        b.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in evs]
    if dist:
        total_ms = max_over_ranks(dist, total_ms, "cuda")
    samples_step = N_STREAMS * PER_STREAM
    value = world * samples_step * args.steps / (total_ms * 1e-3) / 1e9
    avg_launch_ms = sum(launch_ms) / len(launch_ms)
    peak, peak_kind = load_peaks()
    alg_bytes = samples_step * 8 + N_STREAMS * 32  # outputs written + state read and written
    achieved = alg_bytes / (avg_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(), "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)",
                "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_ms}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_desc(), "parallelism": f"replicas x{world} (disjoint stream ranges)"},
            "roofline": roofline, "clocks": clk, "gpu_launches": args.steps}

    if rank == 0 and not args.no_extras:
        line["forms"] = extras(torch, P, g, out, stream, peak, args.stats_per_stream)
    plain_rate = value / world
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e(torch, P, g, samples_step)
    del out
    g.close()
    if rank == 0 and not args.no_batched:
        torch.cuda.empty_cache()
        forms = line.get("forms", {})
        rates = {k: forms.get(k, {}).get("gsamples_s") for k in ("w32_formB_intbits", "w32_eq5_formB_balanced")}
        line["batched"] = batched(torch, P, stream, plain_rate, args.batched_requests, args.batched_hi,
                                  not args.no_autotune, rates)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_served:
        mix_rate = None
        forms = line.get("forms", {})
        if all(k in forms for k in ("w32_formA_fp64", "w32_formB_intbits", "w32_formC_f32pair")):
            # plain-fill rate of the served form mix (a third of the outputs in each form)
            mix_rate = 3.0 / sum(1.0 / forms[k]["gsamples_s"] for k in ("w32_formA_fp64", "w32_formB_intbits",
                                                                         "w32_formC_f32pair"))
        line["served"] = served(torch, P, plain_rate, args.serve_seconds, mix_rate)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def extras(torch, P, g, out, stream, peak, stats_per_stream=1 << 16):
    """The other forms and modes on the same sizes (average device time of a few launches)."""
    res = {}
    n = N_STREAMS * PER_STREAM
    reps = 10

    def rate(ms):
        return n / (ms * 1e-3) / 1e9

    for name, fn in [
        ("w32_formA_fp64", lambda: g.fill_f64(out, PER_STREAM, P.FORM_A_FP64, None, stream)),
        ("w32_formA_balanced",
         lambda: g.fill_mode(out, PER_STREAM, P.FORM_A_FP64, P.MODE_BALANCED, None, stream)),
        ("w32_formB_intbits", lambda: g.fill_f64(out, PER_STREAM, P.FORM_B_INTBITS, None, stream)),
        ("w32_formC_f32pair", lambda: g.fill_f32pair(out, PER_STREAM, None, stream)),
        # Section 2's other maps and Algorithm 1's literal FP64 evaluation
        ("w32_eq5_formB", lambda: g.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_EQ5, None, stream)),
        ("w32_eq5_formB_balanced",
         lambda: g.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_EQ5 | P.MODE_BALANCED, None, stream)),
        ("w32_one_minus_formB", lambda: g.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_ONE_MINUS, None, stream)),
        ("w32_eq5_one_minus_formB",
         lambda: g.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_EQ5 | P.MODE_ONE_MINUS, None, stream)),
        ("w32_formL_algorithm1_single_redraw",
         lambda: g.fill_mode(out, PER_STREAM, P.FORM_L_ALGO1, P.MODE_SINGLE_REDRAW, None, stream)),
    ]:
        fn()
        ms = sum(time_calls(torch, fn, reps, stream)) / reps
        res[name] = {"gsamples_s": rate(ms), "ms": ms, "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak}
    # the bench step's fill into an output that starts 16 bytes into a 32-byte sector (a view of
    # a larger buffer): rows then start mid-sector and take the map shifted by two outputs
    off_buf = torch.empty(n + 4, dtype=torch.float64, device="cuda")
    o16 = off_buf[2:2 + n]
    fn = lambda: g.fill_mode(o16, PER_STREAM, P.FORM_B_INTBITS, P.MODE_BALANCED, None, stream)  # noqa: E731
    fn()
    ms = sum(time_calls(torch, fn, reps, stream)) / reps
    res["w32_formB_balanced_at_16B_offset"] = {"gsamples_s": rate(ms), "ms": ms,
                                               "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak,
                                               "note": "output 16 bytes into a 32-byte sector"}
    del o16, off_buf
    # a few long streams: 64 streams x 2^24 outputs (the same 2^30 outputs), cut into pieces by
    # jump-ahead so that they fill the GPU (prng_fill_split, automatic piece count)
    gl = P.Generator(SEED, 64, W)
    fn = lambda: gl.fill_split(out, n // 64, P.FORM_B_INTBITS, P.MODE_BALANCED, 0, None, stream)  # noqa: E731
    fn()
    ms = sum(time_calls(torch, fn, reps, stream)) / reps
    res["w32_split_64_streams_formB"] = {"gsamples_s": rate(ms), "ms": ms, "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak,
                                         "note": "64 streams x 2^24 outputs, jump-ahead pieces"}
    gl.close()
    # MRG32k3a base streams (Section 2's recommended generators), same sizes, form B
    gm = P.Generator(SEED, N_STREAMS, generator=P.GEN_MRG32K3A)
    fn = lambda: gm.fill_f64(out, PER_STREAM, P.FORM_B_INTBITS, None, stream)  # noqa: E731
    fn()
    ms = sum(time_calls(torch, fn, reps, stream)) / reps
    res["mrg32k3a_formB"] = {"gsamples_s": rate(ms), "ms": ms, "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak,
                             "note": "2^20 MRG32k3a streams x 1024, M = m1 grid, series fast path"}
    fn = lambda: gm.fill_mode(out, PER_STREAM, P.FORM_B_INTBITS, P.MODE_BALANCED, None, stream)  # noqa: E731
    fn()
    ms = sum(time_calls(torch, fn, reps, stream)) / reps
    res["mrg32k3a_formB_balanced"] = {"gsamples_s": rate(ms), "ms": ms,
                                      "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak}
    gm.close()
    g24 = P.Generator(SEED, N_STREAMS, 24)
    for name, form, mode in [("w24_formB_intbits", P.FORM_B_INTBITS, 0),
                             ("w24_formB_balanced", P.FORM_B_INTBITS, P.MODE_BALANCED),
                             ("w24_formA_fp64", P.FORM_A_FP64, 0),
                             ("w24_formA_balanced", P.FORM_A_FP64, P.MODE_BALANCED)]:
        fn = lambda form=form, mode=mode: g24.fill_mode(out, PER_STREAM, form, mode, None, stream)  # noqa: E731
        fn()
        ms = sum(time_calls(torch, fn, reps, stream)) / reps
        res[name] = {"gsamples_s": rate(ms), "ms": ms, "hbm_frac": n * 8 / (ms * 1e-3) / 1e9 / peak}
    g24.close()
    # fused statistics, 2^20 streams x 2^16 = 2^36 samples, no store
    gs = P.Generator(SEED, N_STREAMS, 32)
    hist = torch.zeros(65536, dtype=torch.int64, device="cuda")
    sums = torch.zeros(8, dtype=torch.int64, device="cuda")
    per = stats_per_stream
    fn = lambda: gs.fused_stats(per, hist, sums, None, stream)  # noqa: E731
    fn()
    ms = sum(time_calls(torch, fn, 3, stream)) / 3
    rate = N_STREAMS * per / (ms * 1e-3) / 1e9
    res["w32_fused_stats"] = {"gsamples_s": rate, "ms": ms,
                              "outputs": N_STREAMS * per, "note": "2^20 streams x per_stream, no store"}
    alu = profiled_value(STATS_PROFILE, STATS_SOURCES, "alu_warp_instructions_per_32_outputs")
    if alu:  # ALU lane operations per output = ALU warp instructions per 32 outputs
        res["w32_fused_stats"]["roofline"] = {
            "bound": "alu", "achieved": rate * alu, "peak": ALU_PEAK_GOPS, "unit": "Gop/s",
            "frac": rate * alu / ALU_PEAK_GOPS, "alu_ops_per_output": alu,
            "peak_kind": "ALU pipe: 64 lanes per clock per SM x 152 SMs x 2.07 GHz (ncu peak_sustained, max clock)"}
    gs.close()
    res["precision"] = precision(torch, P)
    return res


def precision(torch, P):
    """Steps (differences of the bit patterns) of forms A and C from form B's correctly rounded
    double, over every output of the bulk workload: fresh handles, so each form rounds the
    same draws. Form B is RN(n/D) (the GPU tests compare it with the oracle's exact division);
    its balanced route is compared with the integer-only one here. Bounds in ulp(n/D): form A
    < 1.5 (1 step), B < 0.5 (0), C < 8.5 (8)."""
    n = N_STREAMS * PER_STREAM

    def fill(form, mode=0):
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        gg = P.Generator(SEED, N_STREAMS, W)
        gg.fill_mode(out, PER_STREAM, form, mode)
        torch.cuda.synchronize()
        gg.close()
        return out

    b = fill(P.FORM_B_INTBITS).view(torch.int64)
    res = {}
    for name, form, mode, bound, steps_bound in [
            ("formA_fp64", P.FORM_A_FP64, 0, 1.5, 1), ("formB_balanced", P.FORM_B_INTBITS, P.MODE_BALANCED, 0.5, 0),
            ("formC_f32pair", P.FORM_C_F32PAIR, 0, 8.5, 8)]:
        x = fill(form, mode)
        worst, at_worst = 0, 0
        for lo in range(0, n, 1 << 27):
            hi_ = min(n, lo + (1 << 27))
            if form == P.FORM_C_F32PAIR:
                pair = x[lo:hi_].view(torch.float32).view(-1, 2).to(torch.float64)
                xi = (pair[:, 0] + pair[:, 1]).view(torch.int64)  # exact: at most 48 significant bits
            else:
                xi = x[lo:hi_].view(torch.int64)
            d = (xi - b[lo:hi_]).abs()
            m = int(d.max())
            if m > worst:
                worst, at_worst = m, 0
            if m == worst:
                at_worst += int((d == worst).sum())
        del x
        res[name] = {"max_ulp_vs_rn": worst, "share_at_max": at_worst / n, "outputs": n,
                     "bound_steps_from_rn": steps_bound, "bound_err_ulp_vs_exact": bound}
    res["formB_intbits"] = {"max_ulp_vs_rn": 0, "bound_steps_from_rn": 0, "bound_err_ulp_vs_exact": 0.5,
                            "note": "the reference of the steps above; equal to the oracle's exact RN(n/D) in "
                                    "the GPU tests"}
    del b
    torch.cuda.empty_cache()
    return res


TUNE_TABLE = os.path.join(ROOT, "paper_1401_8230_gb300", "lib", "autotune.txt")


def batched(torch, P, stream, plain_rate, n_req=4096, hi=2**26, tune=True, rates=None):
    """4096 fresh requests, log-uniform lengths in [2^8, 2^26], own seeds and stream offsets,
    w = 32 form B by the balanced route (as the bench step), one persistent launch (graph
    replay) with the autotuned shape; against the same requests as 4096 single-request
    launches. Each request's output starts on a 256-byte boundary of one pool (as separately
    allocated outputs would). Also timed: the same batch packed at 16-byte offsets, with
    integer-only form B (the single-form kernel), and under the Eq. 5 map."""
    rates = rates or {}
    from paper_1401_8230_gb300 import workloads

    spec = workloads.batched_requests(n=n_req, lo=2**8, hi=hi, seed=1)
    total = sum(r["length"] for r in spec)
    g = P.Generator(SEED, 1, W)
    tuned = P.prng_batch_autotune(g.h, P.FORM_B_INTBITS, 2**8, hi, TUNE_TABLE) if tune else None
    F = P.MODE_BALANCED

    def place(align, mode=0):
        """One pool, request i at a multiple of `align` outputs; returns (pool, request array)."""
        sizes = [((r["length"] + 1) // 2 * 2 + align - 1) // align * align for r in spec]
        pool = torch.empty(sum(sizes) + 32, dtype=torch.float64, device="cuda")
        reqs, off = [], 0
        for r, sz in zip(spec, sizes):
            reqs.append(P.fresh_request(pool[off:], r["length"], r["seed"], r["first_stream"], P.FORM_B_INTBITS,
                                        0, None, mode))
            off += sz
        return pool, reqs, (P.Request * len(reqs))(*reqs)

    def batch_ms(arr):
        P.prng_submit(g.h, arr, stream)
        return sorted(time_calls(torch, lambda: P.prng_submit(g.h, arr, stream), 3, stream))[1]

    pool, reqs, arr = place(2, F)  # 16-byte packing
    packed_ms = batch_ms(arr)
    del pool, reqs, arr
    torch.cuda.empty_cache()
    pool, reqs, arr = place(32, P.MODE_EQ5 | F)  # the Eq. 5 map
    eq5_ms = batch_ms(arr)
    del pool, reqs, arr
    torch.cuda.empty_cache()
    pool, reqs, arr = place(32)  # integer-only form B: the single-form kernel
    int_ms = batch_ms(arr)
    del pool, reqs, arr
    torch.cuda.empty_cache()
    pool, reqs, arr = place(32, F)  # 256-byte aligned, the bench step's route
    ms = batch_ms(arr)
    default_shape = P.prng_batch_get_shape(g.h)
    default_ms = None
    if tuned:  # the same batch with the untuned shape
        P.prng_batch_set_shape(g.h, 8, 3, 4, 16)
        default_shape = P.prng_batch_get_shape(g.h)
        default_ms = batch_ms(arr)
        P.prng_batch_set_shape(g.h, tuned["warps_per_block"], tuned["blocks_per_sm"], tuned["items_per_ticket"],
                               tuned["outputs_per_chunk"])
    # plain: one launch per request on the same stream
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    for k in range(2):
        torch.cuda.synchronize()
        t0.record(stream)
        for q in reqs:
            while True:
                try:
                    P.prng_submit(g.h, [q], stream)
                    break
                except P.PrngError as e:
                    if e.code != P.PRNG_EBUSY:
                        raise
        t1.record(stream)
        torch.cuda.synchronize()
    plain_ms = t0.elapsed_time(t1)
    del pool
    g.close()
    rate = total / (ms * 1e-3) / 1e9
    packed = total / (packed_ms * 1e-3) / 1e9
    eq5 = total / (eq5_ms * 1e-3) / 1e9
    intb = total / (int_ms * 1e-3) / 1e9
    int_plain, eq5_plain = rates.get("w32_formB_intbits"), rates.get("w32_eq5_formB_balanced")
    return {"requests": len(spec), "outputs": total, "placement": "256-byte aligned outputs in one pool",
            "gsamples_s": rate, "ms": ms, "vs_plain_fill": rate / plain_rate,
            "packed_16B": {"gsamples_s": packed, "ms": packed_ms, "vs_plain_fill": packed / plain_rate},
            "kernel": "single-form (form B, PRNG_MODE_BALANCED)",
            "integer_only": {"gsamples_s": intb, "ms": int_ms, "kernel": "single-form",
                             "vs_plain_integer_only_fill": (intb / int_plain) if int_plain else None},
            "eq5_map": {"gsamples_s": eq5, "ms": eq5_ms, "kernel": "any-mode",
                        "vs_plain_eq5_fill": (eq5 / eq5_plain) if eq5_plain else None},
            "per_request_launches_gsamples_s": total / (plain_ms * 1e-3) / 1e9,
            "per_request_launches_ms": plain_ms, "shape": tuned, "graph": True,
            "default_shape": {"warps_per_block": default_shape[0], "blocks_per_sm": default_shape[1],
                              "items_per_ticket": default_shape[2], "outputs_per_chunk": default_shape[3],
                              "ms": default_ms,
                              "gsamples_s": (total / (default_ms * 1e-3) / 1e9) if default_ms else None}}


def served(torch, P, plain_rate, seconds, mix_rate=None, streams_per_client=32768):
    """Poisson arrivals at 20k requests/s for `seconds`, lengths log-uniform in [2^10, 2^28],
    form uniform over A/B/C, 2^16 clients with `streams_per_client` resident streams each (16 B
    of state a stream), 32 GiB output pool; requests replayed in real time by the library's
    serving loop. Then the same server at saturation (all of a fixed request set arriving at
    once)."""
    import numpy as np

    from paper_1401_8230_gb300 import workloads

    clients, S = 2**16, streams_per_client
    g = P.Generator(SEED, clients * S, W)
    srv = P.prng_server_create(g.h, S, 1024, 32 << 30)
    try:
        P.prng_batch_autotune(g.h, P.FORM_B_INTBITS, 2**10, 2**28, TUNE_TABLE)
        trace = workloads.serving_arrivals(seconds, 20000.0, 2**10, 2**28, clients, seed=1)
        items = [(r["t"], r["client"], r["length"], r["form"]) for r in trace]
        lat, makespan = P.prng_server_run_trace(srv, items, 600)
        total = sum(r["length"] for r in trace)
        info = P.prng_server_info(srv)
        sat = workloads.serving_arrivals(1.0, 4000.0, 2**10, 2**28, clients, seed=2)
        sat_items = [(0.0, r["client"], r["length"], r["form"]) for r in sat]
        _, sat_makespan = P.prng_server_run_trace(srv, sat_items, 600)
        sat_total = sum(r["length"] for r in sat)
    finally:
        P.prng_server_destroy(srv)
        g.close()
    rate = total / makespan / 1e9
    sat_rate = sat_total / sat_makespan / 1e9
    lat = np.asarray(lat)
    length = np.array([r["length"] for r in trace])  # the server's lanes by request length
    classes = (("le_2p20", length <= 2**20), ("2p20_to_2p24", (length > 2**20) & (length <= 2**24)),
               ("2p24_to_2p26", (length > 2**24) & (length <= 2**26)), ("gt_2p26", length > 2**26))
    lanes = {name: {"requests": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50) * 1e3),
                    "p99_ms": float(np.percentile(lat[m], 99) * 1e3)}
             for name, m in classes if m.any()}
    return {"requests": len(trace), "outputs": total, "offered_gsamples_s": total / seconds / 1e9,
            "gsamples_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "by_lane": lanes,
            "makespan_s": makespan, "batches": info["batches"],
            "saturation_gsamples_s": sat_rate, "saturation_vs_plain_fill": sat_rate / plain_rate,
            "plain_fill_of_form_mix_gsamples_s": mix_rate,
            "saturation_vs_plain_fill_of_form_mix": (sat_rate / mix_rate) if mix_rate else None,
            "saturation_requests": len(sat),
            "workload": f"Poisson 20k req/s, log-uniform [2^10, 2^28], forms A/B/C, 2^16 clients x {S} streams, "
                        "32 GiB pool"}


def e2e(torch, P, g, samples_step):
    """End to end through the public API: prng_fill_f64_host into pinned host memory (device
    slices generated and copied back inside the call), one full 2^30-sample step per call."""
    host = torch.empty(samples_step, dtype=torch.float64, pin_memory=True)
    g.fill_f64_host(host, PER_STREAM, P.FORM_B_INTBITS)  # warm-up (staging buffers)
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        g.fill_f64_host(host, PER_STREAM, P.FORM_B_INTBITS)
    dt = (time.perf_counter() - t0) / reps
    # the host link itself: plain device-to-pinned-host copies of the same bytes into the same
    # buffer (copy engines; one stream, and four streams over quarters), best of three each
    dev = torch.empty(samples_step, dtype=torch.float64, device="cuda")
    best = float("inf")
    for n_st in (1, 4):
        streams = [torch.cuda.Stream() for _ in range(n_st)]
        parts = list(zip(dev.chunk(n_st), host.chunk(n_st)))
        for rep in range(4):  # the first round warms up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for st, (d, h) in zip(streams, parts):
                with torch.cuda.stream(st):
                    h.copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            if rep:
                best = min(best, time.perf_counter() - t0)
    del dev, host
    # the same call into pageable memory (staged slices and copies), for comparison
    import numpy as np

    pageable = np.empty(samples_step, dtype=np.float64)
    g.fill_f64_host(pageable, PER_STREAM, P.FORM_B_INTBITS)
    t0 = time.perf_counter()
    g.fill_f64_host(pageable, PER_STREAM, P.FORM_B_INTBITS)
    dt_pageable = time.perf_counter() - t0
    del pageable
    link_gbs = samples_step * 8 / best / 1e9
    return {"value": samples_step / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": samples_step * 8, "ms_per_step": dt * 1e3,
            "api": "prng_fill_f64_host (pinned host buffer: device slices, copy-engine DMA)",
            "pageable_gsamples_s": samples_step / dt_pageable / 1e9,
            "host_link_copy_gbs": link_gbs,
            "host_link_frac": samples_step * 8 / dt / 1e9 / link_gbs}


if __name__ == "__main__":
    sys.exit(main())
