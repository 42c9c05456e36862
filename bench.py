#!/usr/bin/env python3
"""Benchmark of the event-parallel parton shower on GB300.

One step = one pass of the whole hot path over one batch of synthetic events
(the paper's workload is itself generated, so synthetic inputs are the
workload): LO matrix element, the plain per-cycle shower (one launch per veto
cycle, host all-done check), validation, observables (Durham y23..y56, 1-T,
rho_H) and histograms.  Default workload: 10^6 LEP events at sqrt(s) = 91.2
GeV, alpha_s(m_Z) = 0.118, t_C = 1 GeV^2, seed 2, 128 parton slots.

Prints one JSON line (rank 0).  `--impl reference` times the oracle (the plain
serial CPU implementation) on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "showered events/sec on 1 GB300 (10^6 LEP events) vs plain GPU; p50/p99 job latency"
UNIT = "events/s"

# Required FP64 work of the shower cycle: the FP64 arithmetic an
# oracle-exact result cannot avoid, counted from the oracle's formulas.
# Trial ranking and veto decisions give the same outcome in FP32 and are not
# counted.  "simple" = +, -, x or a fused a*b+c; the other operations are
# converted to DFMA-equivalents with their throughput measured on the device
# in the same run (gaps_probe_fp64_rates; a log at the rate of the faster of
# the library's and the shower's own table-driven log).
#   per winner:   ln r and the scaled update of ln t
#   per emission: t = exp(ln t), z (expm1), y, the azimuth (sincospi), the
#                 dipole map (transverse frame, k_perp, three momenta) and
#                 four dipole-cache refreshes (Q^2, z+, ln(z+/z-), 1/ln)
WORK_PER_WINNER = {"simple": 5, "log": 1}
WORK_PER_EMISSION = {"simple": 164, "div": 18, "sqrt": 7, "log": 4, "exp": 2, "sincospi": 1}
# FP64 units: two DFMA per SM per clock (the sm__sass_thread_inst_executed_op_dfma
# peak ncu reports for this GB300), two flops per DFMA.
DFMA_PER_SM_PER_CLOCK = 2

# The oracle's arithmetic, unit by unit, as the oracle does it: every trial,
# dipole, veto and splitting in FP64 with the library's transcendentals.
#   per trial:    c from its kernel integral (log of (1-z-)/(1-z+), a
#                 division), t' = t r^(1/c) = t exp(ln r / c) (log, exp,
#                 division), the comparison
#   per dipole:   Q^2 = 2 p_i.p_k and z+- = (1 +- sqrt(1 - 4 t_C/Q^2)) / 2
#   per winner:   z (the kernel's inverse integral), y, alpha_s(t), and the
#                 acceptance ratio (1-y) alpha_s P / (alpha_s^over P^over)
#   per emission: the azimuth and the dipole map (transverse frame, k_perp,
#                 three momenta), colours
ORACLE_PER_TRIAL = {"simple": 4, "log": 2, "exp": 1, "div": 2}
ORACLE_PER_DIPOLE = {"simple": 10, "div": 1, "sqrt": 1}
ORACLE_PER_WINNER = {"simple": 20, "log": 1, "exp": 1, "div": 4}
ORACLE_PER_EMISSION = {"simple": 140, "div": 6, "sqrt": 3, "sincospi": 1}
# Algorithmic bytes of a pass: the final event records, 44 bytes per parton
# (four momentum components, flavour, colour lines, links, with the event's
# share of its scalars), for the final partons and the two initial ones.
RECORD_BYTES_PER_PARTON = 44


def step_kernel_profile():
    """Figures of the committed ncu captures of the plain-form step kernel
    (profiles/k_step_deferred_1e5.md): DRAM bytes per event-cycle of a whole
    pass and the FP64-pipe, issue-slot and SM-active fractions of mid-shower
    launches; None once the kernel sources differ from the captured ones."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "k_step_deferred_1e5.md")
    try:
        text = open(path).read()
        want = re.search(r"source_sha256:\s*([0-9a-f]+)", text).group(1)
        files = re.search(r"sources:\s*(.+)", text).group(1).split()
        h = hashlib.sha256()
        for f in files:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != want:
            return None
        keys = ("dram_bytes_per_event_cycle", "dram_bytes_per_event_cycle_warm", "fp64_pipe_active_frac",
                "issue_active_frac", "sm_active_frac")
        return {k: float(re.search(k + r":\s*([0-9.]+)", text).group(1)) for k in keys}
    except (OSError, AttributeError, ValueError):
        return None


def step_kernel_traffic(event_cycles_per_launch, warm=False):
    """DRAM bytes per launch of the plain-form step kernel: the per-event-cycle
    traffic of the committed ncu capture (all step launches of one pass at
    10^5 events, the deferred emissions included; cold caches as ncu runs by
    default, or warm: caches as the pass leaves them) times this run's
    event-cycles per launch; None once the kernel sources differ from the
    captured ones."""
    prof = step_kernel_profile()
    key = "dram_bytes_per_event_cycle_warm" if warm else "dram_bytes_per_event_cycle"
    return None if prof is None else prof[key] * event_cycles_per_launch


def pipe_fractions():
    """The FP64-pipe and issue-slot fractions of the step kernel (ncu, two
    mid-shower launches at 10^5 events), as the profile records them."""
    prof = step_kernel_profile()
    if prof is None:
        return None
    return {"fp64_pipe_of_active_cycles": prof["fp64_pipe_active_frac"],
            "issue_slots_of_active_cycles": prof["issue_active_frac"],
            "sm_active_of_elapsed_cycles": prof["sm_active_frac"],
            "source": "profiles/k_step_deferred_1e5.md (ncu --set full, launches 21-22 of a 10^5-event pass)"}


def dfma_equivalents(counts, rates, library_log=False):
    """DFMA-equivalents of an operation count; a logarithm costs what the
    faster of the library's log and the shower's table-driven one costs (the
    library's alone with library_log)."""
    def rate(op):
        if op == "log" and not library_log:
            return max(rates["log"], rates.get("log_fp64", 0.0))
        return rates[op]
    return sum(n * (1.0 if op == "simple" else rates["dfma"] / rate(op)) for op, n in counts.items())


def kernels_outside_shower(capacity):
    """Library kernels per pass besides the shower cycles: matrix element,
    validation, the three bucketing kernels and one event-shape kernel per
    multiplicity class (16, 32, 64, 128, 256 slots), the fixed-point
    histogram fill and its conversion."""
    classes = sum(1 for lo in (0, 16, 32, 64, 128) if capacity > lo)
    return 1 + 1 + 3 + classes + 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gaps", choices=["gaps", "reference"])
    ap.add_argument("--events", type=int, default=1_000_000)
    ap.add_argument("--capacity", type=int, default=128)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=10_000_000,
                    help="oracle events for the CPU baseline on all host cores (about 10 s on 16 Grace cores; "
                         "one core gets 1/16 of them)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-variants", action="store_true", help="skip the persistent-form variants")
    ap.add_argument("--batched-events", type=int, default=10_000_000,
                    help="events of the batched persistent variant (0: skip it)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival schedule of the serving variant (0: skip it)")
    ap.add_argument("--uneven-jobs", type=int, default=64,
                    help="jobs of the uneven multi-job batch variant (0: skip it)")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="device memory of the serving pool")
    ap.add_argument("--serve-cycles-per-round", type=int, default=32)
    ap.add_argument("--serve-max-jobs", type=int, default=256, help="job slots of the serving pool")
    ap.add_argument("--serve-mode", default="slice", choices=["slice", "steps"])
    ap.add_argument("--early-stop", action="store_true",
                    help="instead of the benchmark line: the early-termination trade-off, pass time against "
                         "the bias of the histograms when the shower stops after k veto cycles")
    ap.add_argument("--scan", action="store_true",
                    help="instead of the benchmark line: events/s of the plain and persistent passes for "
                         "1 .. 10^7 events (median and IQR of --steps passes), one JSON line per size")
    return ap.parse_args()


def workload_config(args, world):
    return {"workload": f"LEP e+e- -> q qbar, sqrt(s)=91.2 GeV, alpha_s(mZ)=0.118, t_C=1 GeV^2, "
                        f"{args.events} events per GPU, seed {args.seed}, {args.capacity} parton slots, "
                        f"plain per-cycle shower + observables + histograms",
            "events_per_gpu": args.events, "capacity": args.capacity, "seed": args.seed,
            "shower_form": "plain (one launch per veto cycle, host all-done check)",
            "parallelism": f"event ranges, {world} GPU(s), no collective on the data path",
            "l2": "flushed (512 MiB write) before every timed step; the event record is also larger than L2"}


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="gaps_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# --------------------------------------------------------- CPU oracle
def oracle_rate(seed, n_events, capacity, threads, first_event=0, chunk=1_000_000):
    """The oracle's full pipeline (ME, shower, validation, observables,
    histograms) over n_events events of the workload, in chunks of at most
    `chunk` events so that host memory stays bounded; events/s and seconds."""
    from oracle import oracle as O
    p = O.make_params(seed=seed, capacity=capacity)
    t0 = time.perf_counter()
    done = 0
    while done < n_events:
        k = min(chunk, n_events - done)
        O.run(p, first_event + done, k, threads=threads, want_obs=True, want_hist=True)
        done += k
    dt = time.perf_counter() - t0
    return n_events / dt, dt


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def run_reference(args, rank, world):
    """The oracle on the host cores as the reference arm: every step showers
    a bounded sample of the same workload (same seed, event ids continuing
    from step to step)."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.lib()
    cores = host_cores()
    sample = max(1000, args.cpu_sample // 20)
    for w in range(args.warmup):
        oracle_rate(args.seed, sample // 10, args.capacity, cores, first_event=w * sample)
    times = []
    for k in range(args.steps):
        _, dt = oracle_rate(args.seed, sample, args.capacity, cores, first_event=k * sample)
        times.append(dt)
    total = sum(times)
    value = args.steps * sample / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (generated events; the paper's workload is itself generated)",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} events per step of the same workload (seed {args.seed}), "
                                       f"event ranges split over {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- size scan
def run_scan(args, g, torch, np):
    """Throughput against batch size (the paper's scan over N): the whole
    pass, plain and persistent forms, median and IQR over args.steps passes
    after args.warmup, one JSON line per size."""
    stream = torch.cuda.current_stream()
    p = g.make_params(seed=args.seed)
    for n in (1, 10, 100, 1_000, 10_000, 100_000, 1_000_000, 10_000_000):
        ws = g.Workspace(n, args.capacity)
        hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
        line = {"impl": "scan", "events": n, "unit": UNIT}
        for form, mode in (("plain", g.SHOWER_PLAIN), ("persistent", g.SHOWER_PERSISTENT)):
            def one():
                hist.zero_()
                g.generate_me(p, ws, stream)
                if mode == g.SHOWER_PERSISTENT:
                    g.shower_persistent(p, ws, None, stream)
                else:
                    g.shower(p, ws, mode, stream)
                g.validate(p, ws, stream)
                g.observables(p, ws, stream)
                g.histograms(p, ws, hist, stream)
            for _ in range(max(1, args.warmup)):
                one()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            med = float(np.median(ms))
            line[form] = {"ms_median": med, "ms_iqr": [float(np.percentile(ms, 25)), float(np.percentile(ms, 75))],
                          "events_per_s": n / (med / 1e3)}
        print(json.dumps(line), flush=True)
        del ws
        torch.cuda.empty_cache()


# ------------------------------------------------------------ early stop
def hist_chi2(h1, h2):
    """chi^2/ndf between two weighted histograms [obs][bin][3] (summed
    variances, bins empty in both skipped)."""
    import numpy as np
    w1, v1, w2, v2 = h1[:, :, 0], h1[:, :, 1], h2[:, :, 0], h2[:, :, 1]
    m = (v1 + v2) > 0
    return float(np.sum((w1[m] - w2[m]) ** 2 / (v1[m] + v2[m])) / max(1, m.sum())), int(m.sum())


def run_early_stop(args, g, torch, np):
    """Early termination (a measured trade-off, never the default): the plain
    form with the veto cycles capped at k, so events still showering after k
    cycles stop with the step-limit status and are left out of the
    histograms.  Per k: the pass time, the events left out, and the bias of
    the histograms against the full run's, as chi^2/ndf and per observable
    as the relative change of the mean."""
    stream = torch.cuda.current_stream()
    n = args.events
    ws = g.Workspace(n, args.capacity)
    hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device="cuda")
    centres = np.zeros((g.N_OBS, g.HIST_ROW))

    def one(p):
        hist.zero_()
        g.generate_me(p, ws, stream)
        g.shower(p, ws, g.SHOWER_PLAIN, stream)
        g.validate(p, ws, stream)
        g.observables(p, ws, stream)
        g.histograms(p, ws, hist, stream)

    def timed(p):
        for _ in range(2):
            one(p)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one(p)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms)), hist.cpu().numpy().reshape(g.N_OBS, g.HIST_ROW, 3).copy()

    full_ms, full = timed(g.make_params(seed=args.seed))
    means_full = (full[:, :, 0] * np.arange(g.HIST_ROW)).sum(axis=1) / np.maximum(full[:, :, 0].sum(axis=1), 1e-300)
    for k in (100000, 80, 60, 50, 40, 35, 30, 25):
        ms, h = timed(g.make_params(seed=args.seed, max_steps=k))
        status = ws.scalars()["status"].cpu().numpy()
        chi2, ndf = hist_chi2(h, full)
        means = (h[:, :, 0] * np.arange(g.HIST_ROW)).sum(axis=1) / np.maximum(h[:, :, 0].sum(axis=1), 1e-300)
        print(json.dumps({"impl": "early_stop", "events": n, "max_cycles": k, "ms_median": ms,
                          "time_saved": 1.0 - ms / full_ms, "events_stopped": int((status == g.STEP_LIMIT).sum()),
                          "chi2_per_ndf_vs_full": chi2, "ndf": ndf,
                          "mean_bin_shift": [float(x) for x in (means - means_full)]}), flush=True)


# ------------------------------------------------------------- serving
def serve_c(server, jobs, realtime):
    """Serve (arrival s, events, seed) jobs at LEP energy through the C
    scheduler: each job is submitted at its arrival time (all at once unless
    realtime); the schedule advances one step at a time (gaps_server_step)
    and every job it reports finished is polled for its histograms.  Latency
    runs from the scheduled arrival to the moment they are on the host."""
    import numpy as np
    import paper_2403_08692_gb300 as g
    pending = sorted(jobs, key=lambda j: j[0])
    open_jobs, lat, done_events = {}, [], 0
    i = 0
    t0 = time.perf_counter()
    while i < len(pending) or open_jobs:
        now = time.perf_counter() - t0
        while i < len(pending) and (not realtime or pending[i][0] <= now):
            arr, nev, sd = pending[i]
            jid = server.submit(g.make_params(seed=sd), nev, 0)
            open_jobs[jid] = (arr if realtime else 0.0, nev)
            i += 1
        if not open_jobs:
            time.sleep(max(0.0, pending[i][0] - (time.perf_counter() - t0)))
            continue
        # one step of the schedule, then every job it reports finished
        for jid in server.step():
            if server.poll(jid) is not None:
                arr, nev = open_jobs.pop(jid)
                lat.append(time.perf_counter() - t0 - arr)
                done_events += nev
    wall = time.perf_counter() - t0
    lat = np.array(lat) if lat else np.zeros(1)
    return {"jobs": len(jobs), "events": done_events, "wall_s": wall, "events_per_s": done_events / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "max_latency_s": float(lat.max())}


# ------------------------------------------------------------- GPU arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import paper_2403_08692_gb300 as g
    from paper_2403_08692_gb300 import sharding

    torch.cuda.set_device(local_rank)
    if args.scan:
        g.load()
        run_scan(args, g, torch, np)
        return
    if args.early_stop:
        g.load()
        run_early_stop(args, g, torch, np)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    g.load()
    dev = torch.device("cuda", local_rank)
    p = g.make_params(seed=args.seed)
    n = args.events
    first_event, _ = sharding.shard(rank, world, n)
    ws = g.Workspace(n, args.capacity, first_event=first_event, device=dev)
    hist_dev = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64, device=dev)
    stats_dev = torch.zeros(16, dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    STAGES = ("me", "shower", "validate", "observables", "histograms")

    def step(marks=None, kernel_times=False):
        # marks: CUDA events recorded after each stage (per-stage times);
        # kernel_times: time every step launch with its own events (a pass
        # that does so runs a little slower, so the timed passes do not)
        g.generate_me(p, ws, stream)
        if marks:
            marks[0].record(stream)
        if kernel_times:
            rc, launches, kms = g.shower_timed(p, ws, g.SHOWER_PLAIN, stream)
        else:
            (rc, launches), kms = g.shower(p, ws, g.SHOWER_PLAIN, stream), 0.0
        if marks:
            marks[1].record(stream)
        g.validate(p, ws, stream)
        if marks:
            marks[2].record(stream)
        g.observables(p, ws, stream)
        if marks:
            marks[3].record(stream)
        g.histograms(p, ws, hist_dev, stream)
        if marks:
            marks[4].record(stream)
        return launches, kms

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        hist_dev.zero_()
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, launches_total, kernel_ms_total = [], 0, 0.0
    stage_ms = {k: [] for k in STAGES}
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        hist_dev.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in STAGES]
        e0.record(stream)
        launches, kms = step(marks)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(marks[-1]))
        prev = e0
        for name, m in zip(STAGES, marks):
            stage_ms[name].append(prev.elapsed_time(m))
            prev = m
        launches_total += launches
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    total_ms = sharding.job_time_ms(sum(step_ms), dist, dev)
    # the step kernels' own time (for the roofline), from as many more passes
    # with every launch bracketed by events
    for _ in range(args.steps):
        flush.zero_()
        hist_dev.zero_()
        torch.cuda.synchronize()
        kernel_ms_total += step(kernel_times=True)[1]
    torch.cuda.synchronize()

    # FP32-screen fallbacks of the last pass (cycles redone in FP64, vetoes
    # decided in FP64)
    counters = ws.view("counters", torch.int64, (32,)).cpu().numpy()
    # per-event work units of one pass (identical every step)
    g.reduce_stats(ws, stats_dev, stream)
    st = g.Stats.from_buffer_copy(stats_dev.cpu().numpy().tobytes()[:len(bytes(g.Stats()))])
    rates = g.probe_fp64_rates(stream)
    dfma_per_winner = dfma_equivalents(WORK_PER_WINNER, rates)
    dfma_per_emission = dfma_equivalents(WORK_PER_EMISSION, rates)
    dfma_per_pass = dfma_per_winner * st.sum_winners + dfma_per_emission * st.sum_emissions
    launches_per_pass = launches_total / args.steps
    kernel_s_per_launch = kernel_ms_total / 1e3 / launches_total
    achieved_tflops = 2.0 * dfma_per_pass / (kernel_ms_total / 1e3 / args.steps) / 1e12
    # the oracle's arithmetic on the same units, at the same kernel time
    oracle_dfma_per_pass = (dfma_equivalents(ORACLE_PER_TRIAL, rates, True) * st.sum_trials +
                            dfma_equivalents(ORACLE_PER_DIPOLE, rates, True) * st.sum_dipoles +
                            dfma_equivalents(ORACLE_PER_WINNER, rates, True) * st.sum_winners +
                            dfma_equivalents(ORACLE_PER_EMISSION, rates, True) * st.sum_emissions)
    oracle_tflops = 2.0 * oracle_dfma_per_pass / (kernel_ms_total / 1e3 / args.steps) / 1e12
    record_bytes = RECORD_BYTES_PER_PARTON * (st.sum_partons + 2 * st.n_events)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clock_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = 2.0 * DFMA_PER_SM_PER_CLOCK * sms * clock_mhz * 1e6 / 1e12

    # The batched persistent form on the same workload: autotuned launch shape,
    # the whole pass captured once in a CUDA graph and replayed (no host
    # synchronisation inside the pass).  Same events as the plain form.
    variants = {}
    if not args.no_variants:
        cfg, _ = g.autotune_persistent(p, ws, stream)
        ws.record_layout = cfg.layout  # the record layout the autotuner picked, for every persistent pass

        def pass_persistent():
            hist_dev.zero_()
            g.generate_me(p, ws, stream)
            g.shower_persistent(p, ws, cfg, stream)
            g.validate(p, ws, stream)
            g.observables(p, ws, stream)
            g.histograms(p, ws, hist_dev, stream)

        for _ in range(3):
            pass_persistent()
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pass_persistent()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        variants["persistent"] = {"value": n * args.steps / (sum(times) / 1e3), "unit": UNIT,
                                  "ms_per_step": sum(times) / args.steps, "config": cfg.as_dict(),
                                  "launches_per_pass": kernels_outside_shower(args.capacity) + 1}
        # CUDA graph of the whole pass
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            pass_persistent()  # warm-up on the capture stream
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=side):
                hist_dev.zero_()
                g.generate_me(p, ws, side)
                g.shower_persistent(p, ws, cfg, side)
                g.validate(p, ws, side)
                g.observables(p, ws, side)
                g.histograms(p, ws, hist_dev, side)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            replay_stream = torch.cuda.current_stream()  # replay() launches on the current stream
            e0.record(replay_stream)
            graph.replay()
            e1.record(replay_stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        variants["persistent_graph"] = {"value": n * args.steps / (sum(times) / 1e3), "unit": UNIT,
                                        "ms_per_step": sum(times) / args.steps,
                                        "layout": g.LAYOUT_NAMES[cfg.layout]}
        del graph
        ws.record_layout = g.LAYOUT_SOA

    # The per-dipole trial mode (one trial per dipole with the summed
    # overestimate; the same distribution, other events) on the same
    # workload, plain and persistent forms.
    if not args.no_variants:
        pd = g.make_params(seed=args.seed, trial_mode=g.TRIALS_PER_DIPOLE)
        cfg_pd, _ = g.autotune_persistent(pd, ws, stream)
        for name, persistent in (("plain_per_dipole", False), ("persistent_per_dipole", True)):
            ws.record_layout = cfg_pd.layout if persistent else g.LAYOUT_SOA

            def pass_pd():
                hist_dev.zero_()
                g.generate_me(pd, ws, stream)
                if persistent:
                    g.shower_persistent(pd, ws, cfg_pd, stream)
                else:
                    g.shower(pd, ws, g.SHOWER_PLAIN, stream)
                g.validate(pd, ws, stream)
                g.observables(pd, ws, stream)
                g.histograms(pd, ws, hist_dev, stream)
            for _ in range(3):
                pass_pd()
            torch.cuda.synchronize()
            times = []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pass_pd()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            variants[name] = {"workload": f"{n} LEP events per GPU, seed {args.seed}, per-dipole trials",
                              "value": world * n * args.steps / (sharding.job_time_ms(sum(times), dist, dev) / 1e3),
                              "unit": UNIT, "ms_per_step": sum(times) / args.steps}
            if persistent:
                variants[name]["config"] = cfg_pd.as_dict()
        ws.record_layout = g.LAYOUT_SOA

    # The batched persistent form at its own paper-scale workload (10^7 LEP
    # events, seed 3): autotuned shape, the whole pass in one CUDA graph.
    if not args.no_variants and args.batched_events > 0:
        del ws
        torch.cuda.empty_cache()
        nb = args.batched_events
        pb = g.make_params(seed=3)
        wsb = g.Workspace(nb, args.capacity, first_event=sharding.shard(rank, world, nb)[0], device=dev)
        cfg_b, _ = g.autotune_persistent(pb, wsb, stream)
        wsb.record_layout = cfg_b.layout
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                hist_dev.zero_()
                g.generate_me(pb, wsb, side)
                g.shower_persistent(pb, wsb, cfg_b, side)
                g.validate(pb, wsb, side)
                g.observables(pb, wsb, side)
                g.histograms(pb, wsb, hist_dev, side)
        torch.cuda.synchronize()
        replay_stream = torch.cuda.current_stream()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(replay_stream)
            graph.replay()
            e1.record(replay_stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        variants["persistent_graph_1e7"] = {
            "workload": f"{nb} LEP events per GPU, seed 3, same physics and observables",
            "value": world * nb * args.steps / (sharding.job_time_ms(sum(times), dist, dev) / 1e3), "unit": UNIT,
            "ms_per_step": sum(times) / args.steps, "config": cfg_b.as_dict()}
        del graph, wsb
        torch.cuda.empty_cache()
        ws = g.Workspace(n, args.capacity, first_event=first_event, device=dev)

    # The uneven multi-job batch: 64 jobs of 10^3..10^6 events (log-uniform),
    # sqrt(s) in {91.2, 133, 200} GeV, t_C in {0.5, 1, 2} GeV^2, a Philox key
    # per job, showered in one persistent launch with per-job histograms.
    if not args.no_variants and args.uneven_jobs > 0:
        from paper_2403_08692_gb300 import workloads
        try:
            del ws
        except NameError:
            pass
        torch.cuda.empty_cache()
        jobs = workloads.uneven_batch(n_jobs=args.uneven_jobs, seed=4)
        nu = sum(j["n_events"] for j in jobs)
        wsu = g.Workspace(nu, args.capacity, device=dev,
                          layout=cfg_b.layout if args.batched_events > 0 else g.LAYOUT_SOA)
        g.set_jobs([(g.make_params(sqrt_s=j["sqrt_s"], t_cutoff=j["t_cutoff"], alphas_mz=j["alphas_mz"],
                                   seed=j["seed"]), j["n_events"], j["first_event"]) for j in jobs], wsu, stream)
        hist_u = torch.zeros(len(jobs) * g.HIST_DOUBLES, dtype=torch.float64, device=dev)
        cfg_u = cfg_b.as_dict() if args.batched_events > 0 else None

        def pass_uneven():
            hist_u.zero_()
            g.generate_me(None, wsu, stream)
            g.shower_persistent(None, wsu, cfg_u, stream)
            g.validate(None, wsu, stream)
            g.observables(None, wsu, stream)
            g.histograms(None, wsu, hist_u, stream)

        for _ in range(2):
            pass_uneven()
        torch.cuda.synchronize()
        times = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pass_uneven()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        # per-job shower lengths: the longest event of each job (all jobs run
        # together, so a job's share of the launch follows its events' cycles)
        job_of = wsu.view("job_of", torch.int16, (nu,)).to(torch.int64) & 0xFFFF
        steps = wsu.scalars()["n_steps"].to(torch.int64)
        job_max = torch.zeros(len(jobs), dtype=torch.int64, device=dev).scatter_reduce(0, job_of, steps, "amax")
        job_sum = torch.zeros(len(jobs), dtype=torch.int64, device=dev).scatter_add(0, job_of, steps)
        sizes = np.array([j["n_events"] for j in jobs])
        mean_cycles = job_sum.cpu().numpy() / sizes
        variants["uneven_64"] = {
            "workload": f"{len(jobs)} jobs, {nu} events (10^3-10^6 per job, log-uniform, seed 4), sqrt(s) in "
                        f"{{91.2, 133, 200}} GeV, t_C in {{0.5, 1, 2}} GeV^2, one persistent launch, "
                        f"per-job histograms",
            "value": nu * len(times) / (sum(times) / 1e3), "unit": UNIT, "ms_per_step": sum(times) / len(times),
            "ms_iqr": [float(np.percentile(times, 25)), float(np.percentile(times, 75))],
            "config": cfg_u, "jobs": len(jobs), "events": nu,
            "job_events_min_median_max": [int(sizes.min()), int(np.median(sizes)), int(sizes.max())],
            "job_mean_cycles_min_median_max": [float(mean_cycles.min()), float(np.median(mean_cycles)),
                                               float(mean_cycles.max())],
            "job_max_cycles_min_median_max": [int(x) for x in np.percentile(job_max.cpu().numpy(), [0, 50, 100])]}
        del wsu, hist_u
        torch.cuda.empty_cache()
        ws = g.Workspace(n, args.capacity, first_event=first_event, device=dev)

    # The serving loop: Poisson job arrivals served in real time by
    # continuous batching over a resident pool (histograms of every job back
    # on the host), and the same jobs all queued at once (saturated).
    if args.serve_seconds > 0:
        from paper_2403_08692_gb300 import workloads
        try:
            del ws
        except NameError:
            pass
        torch.cuda.empty_cache()
        arrivals = workloads.poisson_arrivals(rate_per_s=50.0, duration_s=args.serve_seconds, seed=5)
        per_event = g.workspace_bytes(1 << 20, args.capacity) / float(1 << 20)
        pool_events = int(args.serve_budget_gb * 2**30 // per_event)
        mode = g.SERVE_SLICE if args.serve_mode == "slice" else g.SERVE_STEPS
        server = g.CServer(pool_events, args.capacity, max_jobs=args.serve_max_jobs,
                           cycles_per_round=args.serve_cycles_per_round, mode=mode, stream=stream)
        serve_c(server, [(0.0, 20000, 7)] * 4, realtime=False)  # warm-up
        jobs = [(t, nev, sd) for (t, nev, sd) in arrivals]
        offered = sum(j[1] for j in jobs) / args.serve_seconds
        s = serve_c(server, jobs, realtime=True)
        variants["serving"] = {
            "workload": f"Poisson arrivals, 50 jobs/s for {args.serve_seconds:g} s (seed 5), 10^3-10^6 events "
                        f"per job log-uniform, sqrt(s)=91.2 GeV, each job its own Philox key",
            "api": "C scheduler: gaps_submit at each arrival, gaps_poll until done (gaps_server_*)",
            "value": s["events_per_s"], "unit": UNIT, "offered_events_per_s": offered,
            "p50_latency_ms": 1e3 * s["p50_latency_s"], "p99_latency_ms": 1e3 * s["p99_latency_s"],
            "max_latency_ms": 1e3 * s["max_latency_s"], "jobs": s["jobs"], "events": s["events"],
            "wall_s": s["wall_s"], "pool_events": pool_events, "memory_budget_gb": args.serve_budget_gb,
            "cycles_per_round": args.serve_cycles_per_round, "max_jobs": args.serve_max_jobs,
            "mode": args.serve_mode + (" (one persistent launch per round)" if args.serve_mode == "slice"
                                       else " (plain-form steps)")}
        sat_jobs = [(0.0, nev, sd) for (t, nev, sd) in jobs if t < args.serve_seconds / 6.0]
        s = serve_c(server, sat_jobs, realtime=False)
        variants["serving_saturated"] = {
            "workload": f"the jobs arriving in the first {args.serve_seconds / 6.0:g} s of the serving workload, "
                        f"all queued at time 0",
            "api": "C scheduler (gaps_submit / gaps_poll)",
            "value": s["events_per_s"], "unit": UNIT, "jobs": s["jobs"], "events": s["events"], "wall_s": s["wall_s"],
            "p50_latency_ms": 1e3 * s["p50_latency_s"], "p99_latency_ms": 1e3 * s["p99_latency_s"]}
        server.close()
        del server
        torch.cuda.empty_cache()
        ws = g.Workspace(n, args.capacity, first_event=first_event, device=dev)

    # end to end through the C ABI with host buffers: params in, histograms and
    # statistics out, every step
    host_hist = torch.zeros(g.HIST_DOUBLES, dtype=torch.float64).pin_memory()
    for _ in range(max(3, args.warmup)):  # the same warm-up as the device-timed passes
        g.run(p, ws, host_hist, g.SHOWER_PLAIN, stream)
    e2e_times = []
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.run(p, ws, host_hist, g.SHOWER_PLAIN, stream)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = world * n * len(e2e_times) / sum(e2e_times)

    value = world * n * args.steps / (total_ms / 1e3)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, dt = oracle_rate(args.seed, args.cpu_sample, args.capacity, cores)
        one = max(1000, args.cpu_sample // 16)
        rate1, dt1 = oracle_rate(args.seed, one, args.capacity, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample} events of the same workload (seed {args.seed}), full "
                         f"pipeline (ME, shower, validation, observables, histograms), event ranges over "
                         f"{cores} threads, {dt:.1f} s wall",
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                               "sample": f"first {one} events, one thread, {dt1:.1f} s wall"},
               "gpu_over_single_core": value / rate1,
               "paper_context": "the paper quotes 295x for its shower stage on a V100 against one Xeon "
                                "E5-2620 core (context only: other hardware, other code)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (generated events; the paper's workload is itself generated)",
        "config": workload_config(args, world),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 48,
                "d2h_bytes_per_step": 8 * g.HIST_DOUBLES + len(bytes(g.Stats())),
                "api": "gaps_run (parameters from host, histograms and statistics back to host)"},
        "gpu_launches": int(args.steps * (kernels_outside_shower(args.capacity) + int(counters[27]))
                            + launches_total),
        "roofline": {"bound": "alu", "kernel": "k_step_deferred (plain-form step: select/veto + deferred emissions)",
                     "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak_tflops,
                     "frac_of_probe": achieved_tflops / (2.0 * rates["dfma"] / 1e12),
                     "oracle_arithmetic": {
                         "label": "FP64-equivalent rate of the oracle's arithmetic: every trial, dipole, veto and "
                                  "splitting of the run evaluated in FP64 as the oracle does it, at the library's "
                                  "measured transcendental costs, over the step kernels' time; above the FP64 peak "
                                  "because the kernels rank trials and decide vetoes in FP32 under error bounds "
                                  "and redo only undecided cases in FP64",
                         "achieved": oracle_tflops, "unit": "TFLOP/s", "over_peak": oracle_tflops / peak_tflops,
                         "dfma_equivalents": {"per_trial": dfma_equivalents(ORACLE_PER_TRIAL, rates, True),
                                              "per_dipole": dfma_equivalents(ORACLE_PER_DIPOLE, rates, True),
                                              "per_winner": dfma_equivalents(ORACLE_PER_WINNER, rates, True),
                                              "per_emission": dfma_equivalents(ORACLE_PER_EMISSION, rates, True)}},
                     "algorithmic_record_bytes_per_pass": record_bytes,
                     "dram_over_algorithmic": (None if step_kernel_traffic(1.0) is None else
                                               step_kernel_traffic(float(st.sum_steps)) / record_bytes),
                     "traffic": step_kernel_traffic(st.sum_steps / max(1.0, launches_per_pass)),
                     "traffic_warm": step_kernel_traffic(st.sum_steps / max(1.0, launches_per_pass), warm=True),
                     "traffic_source": "profiles/k_step_deferred_1e5.md: DRAM bytes per event-cycle from one ncu "
                                       "capture x this run's event-cycles per launch (traffic: caches flushed "
                                       "before each launch, ncu's default; traffic_warm: caches as the pass "
                                       "leaves them, which at 10^5 events hold most of the record)",
                     "pipes": pipe_fractions(),
                     "peak_source": f"FP64 unit count x clock: {DFMA_PER_SM_PER_CLOCK} DFMA/SM/clock x {sms} SMs "
                                    f"x {clock_mhz:.0f} MHz (median SM clock under load) x 2 flops; "
                                    f"MEASURED_PEAKS.json has no FP64 entry",
                     "work_model": f"required FP64 work: {dfma_per_winner:.1f} DFMA-equivalents per winner, "
                                   f"{dfma_per_emission:.1f} per accepted emission (oracle formulas; "
                                   f"transcendentals at their measured cost, a log at the faster of "
                                   f"the library's and the table-driven one), x2 flops",
                     "launches_per_pass": launches_per_pass,
                     "avg_launch_ms": kernel_s_per_launch * 1e3,
                     "fp64_probe_per_s": {k: float(f"{v:.4g}") for k, v in rates.items()},
                     "probe_dfma_tflops": 2.0 * rates["dfma"] / 1e12},
        "clocks": clocks,
        "stages_ms": {k: {"median": float(np.median(v)), "iqr": [float(np.percentile(v, 25)),
                                                                 float(np.percentile(v, 75))]}
                      for k, v in stage_ms.items()},
        "variants": variants,
        "shower": {"kernel_ms_per_pass": kernel_ms_total / args.steps, "launches_per_pass": launches_per_pass,
                   "units_per_pass": {"dipoles": st.sum_dipoles, "trials": st.sum_trials,
                                      "winners": st.sum_winners, "emissions": st.sum_emissions},
                   "max_steps": st.max_steps, "event_cycles": st.sum_steps,
                   "mean_partons": st.sum_partons / max(1, st.n_events),
                   "fp64_fallback_cycles": int(counters[2]), "fp64_vetoes": int(counters[3]),
                   "fp64_thrust_searches": int(counters[4]), "durham_multi_candidate_merges": int(counters[5])},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
