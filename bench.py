"""Benchmark: ParRep SSA events/s on the Schloegl workload with 4096 replicas.

Workload (one "step"): a full ParRep run of the Schloegl network
(k = 0.03, 1e-4, 200, 3.5; regions x < 250 / x >= 250) with N = 4096
replicas, t_corr = t_phase = 1 (time thresholds), T_end = 1e6, x_0 drawn
uniformly from {0..1000}, FIM / RER window [5e5, 1e6].  Each step uses its own
seed.  value = serial-equivalent SSA events (the jumps whose holding time
enters the ParRep clock: decorrelation + parallel-step contributions) per
second of device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f64]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Under torchrun every rank runs its own seeds on its own GPU (independent
ParRep instances, no collective on the data path; weak scaling); rank 0
prints the JSON line with the maximum time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAK_SM_CLOCK_HZ = 2.07e9  # maximum SM clock of a GB300 (used only if the device does not report one)
N_SM = 152  # SMs of a GB300 (used only if the device does not report its count)
# Thread-instructions per event of the FP32 form, counted from the operations
# an event needs (see the design notes): Philox4x32-10 = 10 rounds x (2 wide
# multiplies, 2 three-way XORs, 2 key adds) = 60; two uniforms 8; Schloegl
# propensities 8; a0 3; tau (log, negate, divide, scale, convert) 14;
# selection 10; update and region 4; histogram address + shared atomic 3;
# clock sum, counters and exit tests 10.  Dephasing jumps skip tau and the
# histogram (-17) but add the Fleming-Viot ballots (+4).
OPS_PER_EVENT = 120
OPS_PER_DEPHASE_EVENT = 107
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the staged FP32
# run kernel on the n = 4096 Schloegl workload (ncu launch list, mean of 4
# launches of the default command)
RUN_KERNEL_TRAFFIC = 1.1667e6


def issue_peak(clocks=None):
    """Thread-instruction issue peak of the device: SMs x 4 schedulers x 32
    lanes x the maximum SM clock.  The SM count comes from the device, the
    clock from nvidia-smi's clocks.max.sm sampled during the run, else the
    measured-peaks file, else the GB300 maximum."""
    n_sm, mhz, src = N_SM, None, "GB300 maximum"
    try:
        import torch

        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        pass
    if clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    else:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz, src = float(json.load(f)["sm_max_mhz"]), "measured peaks file"
        except Exception:
            mhz = PEAK_SM_CLOCK_HZ / 1e6
    return n_sm * 4 * 32 * mhz * 1e6, f"{n_sm} SM x 4 schedulers x 32 lanes x {mhz:g} MHz ({src})"


def rank_seed(rank: int, i: int) -> int:
    """Seed of run i on a rank: ranks never share a seed (independent
    instances, weak scaling)."""
    return 1_000_003 * (rank + 1) + i


EXACT_REFS = os.path.join(ROOT, "tests", "golden", "exact_references.json")


def exact_refs():
    """Exact values of the truncated chains (stationary laws, rates, FIM),
    stored by tests/golden/make_exact_references.py from the oracle's exact
    references."""
    with open(EXACT_REFS) as f:
        return json.load(f)


def accuracy_summary(hists, T, escapes, fims, t_corr, ref=None, esc_by_region=None):
    """Accuracy of independent runs of the classic Schloegl workload against
    the exact chain.  hists: per-run time-weighted histograms normalised by
    their clocks T; escapes: per-run parallel-step escapes; fims: per-run FIM
    diagonals (or None).  Pooled estimates weight runs by their clocks; the
    standard errors come from the spread over runs (batch means) and, for the
    TV, from a bootstrap over runs.
      escape_rate_ratio: escapes per unit time over the exact rate of exits
        that follow a completed decorrelation of length t_corr (1 for an
        exact ParRep; Sec. III.B: exact only as the thresholds grow);
      well_mass: time fraction in x < 250 against the exact 0.22026;
      tv: total variation between the pooled histogram and the exact law;
      escape_rate_ratio_lower / _upper (with esc_by_region, per-run escape
        counts out of x < 250 and x >= 250): escapes per unit time spent in
        the region over the exact rate, with Poisson standard errors."""
    import numpy as np

    ref = ref or exact_refs()["schlogl_classic"]
    pi = np.asarray(ref["pi"])
    split = ref["split"]
    H = np.asarray(hists, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    esc = np.asarray(escapes, dtype=np.float64)
    n = len(T)
    w = T / T.sum()
    pooled = w @ H

    def se(v):
        v = np.asarray(v, dtype=np.float64)
        return float(v.std(ddof=1) / np.sqrt(len(v))) if len(v) > 1 else None

    exact_rate = ref["decorrelated_exit_rate"].get(f"{t_corr:g}")
    rate = esc.sum() / T.sum()
    masses = H[:, :split].sum(1)
    tv = 0.5 * float(np.abs(pooled - pi).sum())
    rng = np.random.default_rng(0)
    boot = []
    for _ in range(200 if n > 1 else 0):
        k = rng.integers(0, n, n)
        wk = T[k] / T[k].sum()
        boot.append(0.5 * float(np.abs(wk @ H[k] - pi).sum()))
    out = {
        "runs": n, "T_pooled": float(T.sum()), "t_corr": t_corr,
        "escapes_per_1e6": 1e6 * rate, "escapes_per_1e6_se": None if se(esc / T) is None else 1e6 * se(esc / T),
        "exact_escapes_per_1e6": None if exact_rate is None else 1e6 * exact_rate,
        "escape_rate_ratio": None if exact_rate is None else rate / exact_rate,
        "escape_rate_ratio_se": None if (exact_rate is None or se(esc / T) is None) else se(esc / T) / exact_rate,
        "well_mass": float(pooled[:split].sum()), "well_mass_se": se(masses), "well_mass_exact": ref["mass_lower"],
        "tv": tv, "tv_se": float(np.std(boot, ddof=1)) if boot else None,
    }
    if esc_by_region is not None:
        eb = np.asarray(esc_by_region, dtype=np.float64).sum(0)
        ex2 = ref.get("decorrelated_exit_rates_lower_upper", {}).get(f"{t_corr:g}")
        t_lo = float((H[:, :split].sum(1) * T).sum())
        t_hi = float(T.sum()) - t_lo
        for i, (name, tw, mw) in enumerate((("lower", t_lo, ref["mass_lower"]), ("upper", t_hi, 1.0 - ref["mass_lower"]))):
            out[f"escapes_{name}"] = int(eb[i])
            if ex2 is not None and tw > 0:
                r = (eb[i] / tw) / (ex2[i] / mw)
                out[f"escape_rate_ratio_{name}"] = r
                out[f"escape_rate_ratio_{name}_se"] = r / np.sqrt(max(eb[i], 1.0))
    if fims is not None and len(fims):
        Fd = np.asarray(fims, dtype=np.float64)
        ex = np.asarray(ref["fim_diag"])
        out["fim_diag_rel_error"] = (Fd.mean(0) / ex - 1.0).tolist()
        out["fim_diag_rel_se"] = [None if se(Fd[:, j]) is None else se(Fd[:, j]) / ex[j] for j in range(len(ex))]
    return out


def combine_ranks(dist, t_total, counts, device):
    """Whole-job figures over the ranks: the maximum of the timed seconds and
    the sums of the event counts.  Without a process group, the rank's own."""
    if dist is None:
        return float(t_total), [int(c) for c in counts]
    import torch

    t = torch.tensor([float(t_total)] + [float(c) for c in counts], device=device, dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
    return float(tmax[0]), [int(v) for v in t[1:].tolist()]


def workload(name="schlogl_n4096"):
    """The single-run workloads: the Schloegl run with 4096 replicas (the
    default) or the toggle-switch run with 16384 replicas."""
    from paper_1705_06807_gb300 import configs as K

    c = dict(K.C3 if name == "toggle_n16384" else K.C2)
    c.setdefault("x0_uniform_hi", 0)
    c.setdefault("T_burn", c["T_end"] / 2)
    return c


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--T_end", type=float, default=None, help="override T_end (small profiling cases only)")
    ap.add_argument("--x0", type=int, default=None, help="fixed x_0 instead of the uniform draw (profiling)")
    ap.add_argument("--t_corr", type=float, default=None, help="override t_corr (profiling)")
    ap.add_argument("--t_phase", type=float, default=None, help="override t_phase (profiling)")
    ap.add_argument("--block_threads", type=int, default=0, help="CUDA block size (0 = library default)")
    ap.add_argument("--chunk_steps", type=int, default=0, help="steps between escape votes (0 = default)")
    ap.add_argument("--workload", default="schlogl_n4096", choices=["schlogl_n4096", "toggle_n16384", "batch256", "serve", "speedup", "uq", "sweep",
                             "accuracy"],
                    help="schlogl_n4096: one ParRep run of 4096 replicas to T_end = 1e6 per step; toggle_n16384: "
                         "one run of the toggle switch (alpha = 50, n = 2.5) with 16384 replicas to T_end = 1e5; "
                         "batch256: "
                         "256 mixed Schloegl / toggle instances (64..65536 replicas, T_end = 1e4) in one launch; "
                         "serve: Poisson-arriving requests through the continuous-batching server; speedup: "
                         "ParRep vs plain SSA to the same simulated time at TV <= 1e-2 (Schloegl V=25); uq: the "
                         "Sec. V.A IAF / FIM / information-bound experiment (100 samples to T = 2e5); sweep: the "
                         "Sec. V.A accuracy and speedup studies over n_c = n_p and R; accuracy: the Schloegl n=4096 "
                         "workload's escape rate, well mass and TV against the exact chain over t_corr = t_phase")
    ap.add_argument("--serve_rate", type=float, default=200.0, help="request arrivals per second (serve)")
    ap.add_argument("--serve_seconds", type=float, default=20.0, help="length of the arrival stream (serve)")
    ap.add_argument("--batch_n", type=int, default=256, help="instances of the batch workload")
    ap.add_argument("--accuracy_t", default="1,2,4,6,8", help="t_corr = t_phase values (accuracy)")
    ap.add_argument("--accuracy_seeds", type=int, default=64, help="runs per threshold (accuracy)")
    ap.add_argument("--fv_group", type=int, default=32, help="Fleming-Viot group size (accuracy)")
    ap.add_argument("--f32_layout", default="auto", choices=["auto", "staged", "direct", "mixed"],
                    help="FP32 kernel layout (auto: direct from 16384 replicas on, staged below; batches and "
                         "the server choose per instance)")
    ap.add_argument("--serve_seconds_default", type=float, default=5.0,
                    help="length of the request stream measured beside the headline (0 = none)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the side measurements (accurate threshold, FP64 form, serve stream)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [t.strip() for t in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.remove(self.path)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


def cpu_baseline(c, sample_T=1000.0, seed=0):
    """The oracle as it stands, single-threaded, on the first sample_T time
    units of the same workload (same network, replicas, thresholds, x_0 law)."""
    import oracle as O

    t0 = time.perf_counter()
    r = O.parrep_run(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], sample_T, seed, c["x0"],
                     x0_uniform_hi=c.get("x0_uniform_hi", 0), precision="f64", T_burn=sample_T / 2)
    dt = time.perf_counter() - t0
    useful = r["events_decorr"] + r["events_parallel_useful"]
    return dict(value=useful / dt, unit="events/s", cores=1, kind="oracle",
                sample=f"{c['name']} truncated to T_end={sample_T:g} (seed {seed}, binary64), "
                       f"{useful} useful + {r['events_dephase']} dephasing events in {dt:.2f} s")


def cpu_baseline_all_cores(c, sample_T=1000.0, seed0=100):
    """The oracle as it stands on every host core at once: one thread per core,
    each running its own seed of the same truncated workload (the C oracle
    releases the interpreter lock while it runs)."""
    import threading

    import oracle as O

    O.lib()  # build / load once before the threads start
    n = os.cpu_count() or 1
    out = [None] * n

    def work(i):
        r = O.parrep_run(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], sample_T, seed0 + i, c["x0"],
                         x0_uniform_hi=c.get("x0_uniform_hi", 0), precision="f64", T_burn=sample_T / 2)
        out[i] = r["events_decorr"] + r["events_parallel_useful"]

    th = [threading.Thread(target=work, args=(i,)) for i in range(n)]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    dt = time.perf_counter() - t0
    useful = sum(out)
    return dict(value=useful / dt, unit="events/s", cores=n, kind="oracle",
                sample=f"{n} threads, one per host core, each {c['name']} truncated to T_end={sample_T:g} "
                       f"(seeds {seed0}..{seed0 + n - 1}, binary64): {useful} useful events in {dt:.2f} s")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = workload()
    vals, secs = [], []
    sample_T = 1000.0  # about 2 s of one host core per step
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        b = cpu_baseline(c, sample_T=sample_T, seed=1000 + i)
        if i >= args.warmup:
            vals.append(b)
            secs.append(time.perf_counter() - t0)
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": "SSA events/s", "value": v, "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c["name"], "replicas": c["n_replicas"], "T_end_sample": sample_T},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batch(args, world, rank, local, dist):
    """The batched workload: every step runs all instances in one launch."""
    import numpy as np
    import torch

    from paper_1705_06807_gb300 import ParRep, ParRepBatch
    from paper_1705_06807_gb300 import configs as K

    T_end = args.T_end or 1e4
    insts = K.batch_instances(n=args.batch_n, seed=0, T_end=T_end)

    def make():
        hs = [ParRep(d["network"], d["n_replicas"], d["t_corr"], d["t_phase"], x0=d["x0"], thresh=d["thresh"],
                     precision=args.precision, T_burn=0.5 * d["T_end"]) for d in insts]
        return hs, ParRepBatch(hs, block_threads=args.block_threads, f32_layout=args.f32_layout)

    handles, batch = make()
    Ts = [d["T_end"] for d in insts]
    seeds0 = [(d["seed"] + 7919 * rank) & 0xFFFFFFFFFFFFFFFF for d in insts]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(i):
        flush.fill_(float(i))  # evicts L2 between steps, outside the timed region
        torch.cuda.synchronize()
        info = batch.run(Ts, [s + i for s in seeds0])
        return info["kernel_ms"], [h.stats() for h in handles], info

    for i in range(args.warmup):
        one(i)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats, info = [], [], None
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ms, st, info = one(args.warmup + i)
            times.append(ms)
            stats.append(st)
    t_total = sum(times) / 1e3
    flat = [x for st in stats for x in st]
    useful = sum(x["events_decorr"] + x["events_parallel_useful"] for x in flat)
    executed = sum(x["events_decorr"] + x["events_parallel_executed"] + x["events_replay"] + x["events_dephase"]
                   for x in flat)
    dephase = sum(x["events_dephase"] for x in flat)
    breakdown = {k: sum(x[k] for x in flat) // max(1, len(stats)) for k in
                 ("events_decorr", "events_dephase", "events_parallel_useful", "events_parallel_executed",
                  "events_replay", "cycles", "escapes")}
    ph = {}
    for x in flat:
        for k, v in x["phase_cycles"].items():
            ph[k] = ph.get(k, 0.0) + v
    ph_tot = sum(v for k, v in ph.items() if not k.startswith("dec_")) or 1.0
    t_total, (useful, executed, dephase) = combine_ranks(dist, t_total, [useful, executed, dephase], "cuda")
    clocks = clk.summary()
    e2e = None
    if not args.no_e2e:
        # through the public API with host structs in and host results out:
        # create every handle and the batch, run, read histograms and FIMs
        t0 = time.perf_counter()
        hs2, b2 = make()
        b2.run(Ts, [s + args.warmup for s in seeds0])
        d2h = 0
        for h in hs2:
            hist = h.histogram()
            fim = h.fim()
            d2h += hist.nbytes + fim.nbytes
        wall = time.perf_counter() - t0
        ev = sum(h.stats()["events_decorr"] + h.stats()["events_parallel_useful"] for h in hs2)
        b2.close()
        for h in hs2:
            h.close()
        e2e = {"value": ev / wall, "unit": "events/s", "h2d_bytes_per_step": len(insts) * (96 + 56 + 16),
               "d2h_bytes_per_step": d2h, "note": "includes creating the 256 handles (device allocation) and "
                                                   "the autotuner's trial runs"}
    peak_ops, peak_note = issue_peak(clocks)
    ops = (executed - dephase) * OPS_PER_EVENT + dephase * OPS_PER_DEPHASE_EVENT
    achieved = ops / t_total if t_total > 0 else None
    R = [d["n_replicas"] for d in insts]
    line = {
        "metric": "SSA events/s", "value": useful / t_total, "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": f"batch{len(insts)}_mixed_T{T_end:g}", "instances": len(insts),
                   "replicas_total": int(sum(R)), "replicas_min_max": [int(min(R)), int(max(R))],
                   "mix": "half Schloegl V in {0.5,1,2,4,8}, half toggle n~U[2,3] alpha~U[30,80]",
                   "thresholds": "time t_corr=t_phase=1", "fim_window": "[T_end/2, T_end]",
                   "l2": "flushed (256 MiB write) between steps", "parallelism": f"independent batches x{world}"},
        "executed_events_per_s": executed / t_total,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12 if achieved else None, "peak": peak_ops / 1e12,
                     "unit": "Tinst/s", "frac": achieved / peak_ops if achieved else None, "traffic": None,
                     "note": "thread-instructions at 120 per event (107 per dephasing jump) over the device time "
                             "of the launch sequence; peak = " + peak_note},
        "batch": {k: info[k] for k in ("block_threads", "replicas_per_block", "grid_blocks", "n_items", "graph",
                                        "tuned_trials", "tune_ms", "est_balance", "f32_layout")},
        "events_per_step": breakdown,
        "phase_share": {k: round(v / ph_tot, 4) for k, v in ph.items()},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0:
        if not args.no_cpu and world == 1:
            import oracle as O

            t0 = time.perf_counter()
            ev = 0
            small = [d for d in insts if d["n_replicas"] <= 2048][:4]
            for d in small:
                r = O.parrep_run(d["network"], d["n_replicas"], d["t_corr"], d["t_phase"], 20.0, d["seed"],
                                 d["x0"], precision="f64", T_burn=10.0)
                ev += r["events_decorr"] + r["events_parallel_useful"]
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": ev / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
                                    "sample": f"first 4 instances with <= 2048 replicas truncated to T_end=20 "
                                              f"(binary64): {ev} useful "
                                              f"events in {dt:.2f} s"}
        print(json.dumps(line), flush=True)
    batch.close()


def bench_serve(args, local):
    """The serving workload: requests arrive at their Poisson times, are
    submitted from host structs and their results (histogram, FIM, stats)
    read back to host memory as they complete."""
    print(json.dumps(serve_stream(args, local, args.serve_rate, args.serve_seconds)), flush=True)


def serve_stream(args, local, rate, seconds):
    """Runs one seeded Poisson request stream through the server; returns the
    JSON line (p50/p99 latency, events/s over the stream's wall time)."""
    import numpy as np
    import torch

    from paper_1705_06807_gb300 import ParRepServer
    from paper_1705_06807_gb300 import configs as K

    stream = K.serve_requests(rate=rate, seconds=seconds, seed=0)
    srv = ParRepServer(precision=args.precision, f32_layout=args.f32_layout)
    # warm-up: a few small requests (module load, first launches)
    for i in range(max(args.warmup, 1)):
        d = stream[i][1]
        srv.result(srv.submit(d["network"], 64, d["t_corr"], d["t_phase"], 100.0, 1000 + i, x0=d["x0"],
                              T_burn=50.0))
    torch.cuda.synchronize()
    pending, lat, useful, executed, dephase = {}, [], 0, 0, 0

    tm = {"submit": 0.0, "poll": 0.0, "result": 0.0}

    def collect(block=False):
        nonlocal useful, executed, dephase
        for rid in list(pending):
            t1 = time.perf_counter()
            ready = block or srv.poll(rid) == 2
            t2 = time.perf_counter()
            tm["poll"] += t2 - t1
            if ready:
                r = srv.result(rid)
                tm["result"] += time.perf_counter() - t2
                assert r["status"] == 0, r["status"]
                st = r["stats"]
                lat.append(r["latency_s"])
                useful += st["events_decorr"] + st["events_parallel_useful"]
                executed += (st["events_decorr"] + st["events_parallel_executed"] + st["events_replay"] +
                             st["events_dephase"])
                dephase += st["events_dephase"]
                del pending[rid]

    launches0 = srv.stats()["launches"]
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for t_arr, d in stream:
            while time.perf_counter() - t0 < t_arr:
                collect()
                time.sleep(0.0002)
            t1 = time.perf_counter()
            rid = srv.submit(d["network"], d["n_replicas"], d["t_corr"], d["t_phase"], d["T_end"], d["seed"],
                             x0=d["x0"], T_burn=0.5 * d["T_end"])
            tm["submit"] += time.perf_counter() - t1
            pending[rid] = t_arr
        t_stream = time.perf_counter() - t0
        collect(block=True)
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    st = srv.stats()
    srv.close()
    lat_a = np.array(lat)
    peak_ops, peak_note = issue_peak(clocks)
    ops = (executed - dephase) * OPS_PER_EVENT + dephase * OPS_PER_DEPHASE_EVENT
    line = {
        "metric": "SSA events/s", "value": useful / wall, "unit": "events/s", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"serve_poisson{rate:g}_{seconds:g}s",
                   "requests": len(stream), "mix": "Schloegl V in {0.5,1,2,4,8} / toggle n~U[2,3] alpha~U[30,80], "
                   "replicas log-uniform 64..65536, T_end log-uniform 1e3..1e5, t_corr=t_phase=1",
                   "timing": "wall clock from the first arrival to the last result on the host"},
        "latency_s": {"p50": float(np.percentile(lat_a, 50)), "p99": float(np.percentile(lat_a, 99)),
                      "mean": float(lat_a.mean()), "max": float(lat_a.max())},
        "executed_events_per_s": executed / wall,
        "roofline": {"bound": "alu", "achieved": ops / wall / 1e12, "peak": peak_ops / 1e12, "unit": "Tinst/s",
                     "frac": ops / wall / peak_ops, "traffic": None,
                     "note": "over the wall time of the stream, idle gaps between arrivals included"},
        "gpu_launches": st["launches"] - launches0,
        "server": {k: st[k] for k in ("submitted", "admitted", "completed", "launches", "grid_blocks")},
        "host_s": {"stream": t_stream, **{k: round(v, 3) for k, v in tm.items()}},
        "clocks": clocks,
        "e2e": {"value": useful / wall, "unit": "events/s", "h2d_bytes_per_step": len(stream) * 600,
                "d2h_bytes_per_step": None, "note": "the served path is end to end: host requests in, host results out"},
    }
    return line


def accuracy_runs(c, t, n, precision, seed0, batched=True, fv_group=32, by_region=None):
    """n independent runs of the classic Schloegl workload c with t_corr =
    t_phase = t, in one batch launch (or one after another).  Returns the
    per-run histograms, clocks, escapes and FIM diagonals, the useful events
    and the device seconds; with by_region (a list), also appends each run's
    escape counts out of region 0 and region 1 (from its cycle log)."""
    import numpy as np

    from paper_1705_06807_gb300 import ParRep, ParRepBatch

    hs = [ParRep(c["network"], c["n_replicas"], t, t, x0=c["x0"], x0_uniform_hi=c["x0_uniform_hi"],
                 thresh=c["thresh"], precision=precision, T_burn=c["T_burn"], fv_group=fv_group)
          for _ in range(n)]
    seeds = [seed0 + i for i in range(n)]
    if batched:
        b = ParRepBatch(hs, autotune=False)
        info = b.run([c["T_end"]] * n, seeds)
        assert b.status() == [0] * n
        dev_s = info["kernel_ms"] / 1e3
        b.close()
    else:
        dev_s = 0.0
        for h, sd in zip(hs, seeds):
            dev_s += h.run(c["T_end"], sd)["kernel_ms"] / 1e3
    hists, T, esc, fims, useful = [], [], [], [], 0
    for h in hs:
        st = h.stats()
        hists.append(h.histogram())
        T.append(st["T_s"])
        esc.append(st["escapes"])
        fims.append(np.diag(h.fim()))
        useful += st["events_decorr"] + st["events_parallel_useful"]
        if by_region is not None:
            cnt = [0, 0]
            for cy in h.cycle_log():
                if cy["k"] >= 0 and cy["W"] in (0, 1):
                    cnt[cy["W"]] += 1
            by_region.append(cnt)
        h.close()
    return hists, T, esc, fims, useful, dev_s


def bench_accuracy(args):
    """Accuracy of the benchmarked Schloegl workload against the exact chain,
    over t_corr = t_phase (Sec. III.B: ParRep is exact only as the
    decorrelation and dephasing grow).  For each threshold, `accuracy_seeds`
    independent runs of the headline configuration (4096 replicas, x_0 ~
    U{0..1000}, T_end = 1e6, FIM window [5e5, 1e6]) in one batch launch: the
    parallel-step escape rate against the exact rate of exits that follow a
    completed decorrelation, the lower-well mass against 0.22026, the pooled
    histogram's TV against the exact law (with standard errors), the FIM
    diagonal's relative error, and useful events/s."""
    c = workload("schlogl_n4096")
    rows = []
    ts = [float(v) for v in args.accuracy_t.split(",")]
    for i, t in enumerate(ts):
        byr = []
        hists, T, esc, fims, useful, dev_s = accuracy_runs(c, t, args.accuracy_seeds, args.precision,
                                                           7_000_000 + 100_000 * i, fv_group=args.fv_group,
                                                           by_region=byr)
        row = accuracy_summary(hists, T, esc, fims, t, esc_by_region=byr)
        row["fv_group"] = args.fv_group
        row["useful_events_per_s"] = useful / dev_s
        row["device_s"] = dev_s
        rows.append(row)
        print(json.dumps({"partial": row}), file=sys.stderr, flush=True)
    ok = [r for r in rows if r["tv"] <= 1e-2]
    line = {
        "metric": "accuracy of the Schloegl n=4096 workload vs t_corr=t_phase", "value": ok[0]["t_corr"] if ok else None,
        "unit": "smallest t_corr=t_phase with pooled TV <= 1e-2", "n_gpus": 1, "steps": len(ts), "warmup": 0,
        "ms_per_step": 1e3 * sum(r["device_s"] for r in rows) / len(rows), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": "schlogl_n4096_T1e6_accuracy_sweep", "runs_per_threshold": args.accuracy_seeds,
                   "thresholds": ts, "exact": "product-formula law truncated at 1500; exact decorrelated-exit rate"},
        "rows": rows,
    }
    print(json.dumps(line), flush=True)


def bench_speedup(args):
    """ParRep speedup over plain SSA at TV <= 1e-2 against the exact law, on
    the V = 25 Schloegl network with the paper's Sec. V.A settings (R = 100,
    n_c = n_p = 5000): 128 seeds x 1.25e5 time units in one batch (the pooled
    histogram's TV is measured and reported; its well-mass standard error is
    about 1.3e-3, so sampling noise alone leaves a TV of a few 1e-3), against
    one plain-SSA trajectory over the same 1.6e7 time units -- as a
    one-thread GPU SSA and as the oracle on one core, both timed on a shorter
    stretch and scaled by simulated time."""
    import numpy as np

    import oracle as O
    from paper_1705_06807_gb300 import ParRep, ParRepBatch, parrep_ssa
    from paper_1705_06807_gb300 import configs as K

    net = K.schlogl_paper(V=25)
    n, T_each = 128, 1.25e5
    T_total = n * T_each
    pi = np.asarray(exact_refs()["schlogl_v25"]["pi"])
    hs = [ParRep(net, 100, 5000, 5000, x0=[4], thresh="steps", precision=args.precision) for _ in range(n)]
    b = ParRepBatch(hs)
    b.run([T_each] * n, [77 + i for i in range(n)])  # warm-up and autotuning
    t0 = time.perf_counter()
    info = b.run([T_each] * n, [5000 + i for i in range(n)])
    wall = time.perf_counter() - t0
    pooled = sum(h.histogram() * h.stats()["T_s"] for h in hs) / T_total
    tv = 0.5 * float(np.abs(pooled - pi).sum())
    useful = sum(h.stats()["events_decorr"] + h.stats()["events_parallel_useful"] for h in hs)
    b.close()
    # plain SSA, one trajectory on one GPU thread
    parrep_ssa(net, 1, [4], 100.0, 1, precision=args.precision)
    T_gpu = 2e4
    _, ev_gpu, ms_gpu = parrep_ssa(net, 1, [4], T_gpu, 2, precision=args.precision)
    t_ssa_gpu = ms_gpu / 1e3 * T_total / T_gpu
    # plain SSA, the oracle on one host core
    T_cpu = 2e3
    t1 = time.perf_counter()
    _, ev_cpu, _ = O.ssa_run(net, 1, [4], T_cpu, 3)
    t_ssa_cpu = (time.perf_counter() - t1) * T_total / T_cpu
    line = {
        "metric": "ParRep speedup vs plain SSA at TV<=1e-2", "value": t_ssa_gpu / (info["kernel_ms"] / 1e3),
        "unit": "x", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": info["kernel_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": "schlogl_V25_paper_settings", "R": 100, "n_c": 5000, "n_p": 5000, "seeds": n,
                   "T_each": T_each, "T_total": T_total},
        "tv_vs_exact": tv,
        "parrep": {"device_s": info["kernel_ms"] / 1e3, "wall_s": wall, "useful_events": useful},
        "plain_ssa_gpu_thread": {"s_to_T_total": t_ssa_gpu, "events_per_s": ev_gpu / (ms_gpu / 1e3),
                                 "timed_T": T_gpu},
        "plain_ssa_oracle_1core": {"s_to_T_total": t_ssa_cpu, "events_per_s": ev_cpu / (t_ssa_cpu * T_cpu / T_total),
                                   "timed_T": T_cpu},
        "speedup_vs_oracle_1core": t_ssa_cpu / (info["kernel_ms"] / 1e3),
    }
    print(json.dumps(line), flush=True)


def bench_uq(args):
    """The stationary UQ experiment of Sec. V.A (its Tables II and III):
    100 independent ParRep samples of the V = 25 Schloegl network (R = 100,
    n_c = n_p = 5000), each to T = 2e5 with [0, 1e5] as burn-in, in one batch;
    then parrep_uq for f = x: the IAF, the stationary mean, the FIM with 95%
    half widths and the information bounds.  value = device seconds of the
    batch run plus the UQ call's wall time; the estimates are reported beside
    the exact values of the truncated chain and the paper's printed ones."""
    import numpy as np

    import oracle as O
    from paper_1705_06807_gb300 import ParRep, ParRepBatch, parrep_uq
    from paper_1705_06807_gb300 import configs as K

    net = K.schlogl_paper(V=25, hist_max=255)
    n, T, Tb = 100, 2e5, 1e5
    hs = [ParRep(net, 100, 5000, 5000, x0=[4], thresh="steps", precision=args.precision, T_burn=Tb)
          for _ in range(n)]
    b = ParRepBatch(hs)
    b.run([T] * n, [91 + i for i in range(n)])  # warm-up and autotuning
    x = np.arange(256.0)
    parrep_uq(hs, x)
    info = b.run([T] * n, [60000 + i for i in range(n)])
    assert b.status() == [0] * n
    t0 = time.perf_counter()
    r = parrep_uq(hs, x)
    t_uq = time.perf_counter() - t0
    useful = sum(h.stats()["events_decorr"] + h.stats()["events_parallel_useful"] for h in hs)
    b.close()
    ex = exact_refs()["schlogl_v25"]
    pi = np.asarray(ex["pi"])
    tau = ex["iaf_x"]
    S = np.asarray(ex["sensitivity_x"])
    Fd = np.asarray(ex["fim_diag"])
    # the oracle (one host core) on one sample over 2e4 time units, scaled to the experiment
    T_cpu = 2e4
    t1 = time.perf_counter()
    O.parrep_run(net, 100, 5000, 5000, T_cpu, 1, [4], thresh="steps")
    t_cpu = (time.perf_counter() - t1) * n * T / T_cpu
    dev_s = info["kernel_ms"] / 1e3 + t_uq
    line = {
        "metric": "Sec. V.A UQ experiment time (100 samples to T=2e5)", "value": dev_s, "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": dev_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": "schlogl_V25_uq_100x2e5", "R": 100, "n_c": 5000, "n_p": 5000, "samples": n,
                   "T": T, "T_burn": Tb, "f": "x"},
        "batch_s": info["kernel_ms"] / 1e3, "uq_call_s": t_uq, "useful_events_per_s": useful / (info["kernel_ms"] / 1e3),
        "estimate": {"iaf": r["iaf"], "mean_f": r["mean_f"], "fim_diag": np.diag(r["fim"]).tolist(),
                     "fim_half_width_diag": np.diag(r["fim_half_width"]).tolist(), "bounds": r["bounds"].tolist()},
        "exact": {"iaf": tau, "mean_f": float(pi @ x), "fim_diag": Fd.tolist(), "sensitivity": S.tolist(),
                  "bounds": (np.sqrt(tau) * np.sqrt(Fd)).tolist()},
        "paper": {"iaf": 5.87e5, "fim_diag": [87.5, 1670.0, 200.0, 24.6], "bounds": [7.16e3, 3.09e4, 1.08e4, 3.80e3]},
        "oracle_1core_s_estimate": t_cpu,
    }
    print(json.dumps(line), flush=True)


def bench_sweep(args):
    """The STEPS-mode studies of Sec. V.A: the stationary mean of the V = 25
    Schloegl network estimated from 100 samples to T = 1e5 (R = 100) for
    n_c = n_p = 1000 .. 5000, and for R = 20 .. 100 at n_c = n_p = 5000.  For
    each setting: the mean with its 95% half width against the exact value,
    and the paper's speedup -- serial SSA jumps over the jumps on ParRep's
    critical path (decorrelation + dephasing + parallel lockstep steps), i.e.
    the speedup on R ideal processors -- next to the GPU time."""
    import numpy as np

    from paper_1705_06807_gb300 import ParRep, ParRepBatch
    from paper_1705_06807_gb300 import configs as K

    net = K.schlogl_paper(V=25, hist_max=255)
    x = np.arange(256.0)
    exact = exact_refs()["schlogl_v25"]["mean"]
    n, T = 100, 1e5
    settings = [(100, nc) for nc in (1000, 2000, 3000, 4000, 5000)] + [(R, 5000) for R in (20, 40, 60, 80)]
    rows, t_total = [], 0.0
    for i, (R, nc) in enumerate(settings):
        hs = [ParRep(net, R, nc, nc, x0=[4], thresh="steps", precision=args.precision) for _ in range(n)]
        b = ParRepBatch(hs)
        info = b.run([T] * n, [100000 * (i + 1) + k for k in range(n)])
        assert b.status() == [0] * n
        means = np.array([h.histogram() @ x for h in hs])
        useful = crit = 0
        for h in hs:
            st = h.stats()
            useful += st["events_decorr"] + st["events_parallel_useful"]
            crit += sum(c["decorr_steps"] + c["dephase_steps"] + c["n_star"] for c in h.cycle_log())
        b.close()
        t_total += info["kernel_ms"] / 1e3
        rows.append({"R": R, "n_c": nc, "mean": float(means.mean()),
                     "half_width_95": float(1.96 * means.std(ddof=1) / np.sqrt(n)),
                     "rel_error": float(means.mean() / exact - 1.0), "paper_speedup": useful / crit,
                     "gpu_s": info["kernel_ms"] / 1e3, "useful_events_per_s": useful / (info["kernel_ms"] / 1e3)})
    line = {
        "metric": "Sec. V.A sweeps: ParRep speedup on R ideal processors (R=100, n_c=n_p=5000)",
        "value": rows[4]["paper_speedup"], "unit": "x", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": t_total * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": "schlogl_V25_sweeps_100x1e5", "samples": n, "T": T, "exact_mean": exact},
        "rows": rows,
        "paper": {"rel_error_nc5000": 4e-4, "speedup_R20_to_R100": [7, 20]},
    }
    print(json.dumps(line), flush=True)


ACCURATE_T = 12.0  # the smallest t_corr = t_phase of the accuracy sweep with TV <= 1e-2 and exact escape rates


def side_measurements(args, c, rank, local, stream, flush):
    """Measurements printed beside the headline, outside its timed region:
      accurate_threshold: the same workload at t_corr = t_phase = ACCURATE_T,
        events/s over its own timed runs with their accuracy keys;
      fp64: the plain binary64 form of the headline workload (one timed run);
      serve: a short Poisson request stream through the server (p50/p99)."""
    import numpy as np
    import torch

    from paper_1705_06807_gb300 import ParRep

    out = {}

    def timed_runs(g, n, seed0, T_end):
        ms, sts, acc = [], [], ([], [], [], [])
        for i in range(n):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.run(T_end, seed0 + i)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = g.stats()
            sts.append(st)
            acc[0].append(g.histogram())
            acc[1].append(st["T_s"])
            acc[2].append(st["escapes"])
            acc[3].append(np.diag(g.fim()))
        useful = sum(s_["events_decorr"] + s_["events_parallel_useful"] for s_ in sts)
        return useful / (sum(ms) / 1e3), sum(ms) / n, acc

    T_end = c["T_end"]

    def handle(t, precision, T_burn):
        return ParRep(c["network"], c["n_replicas"], t, t, x0=c["x0"], x0_uniform_hi=c["x0_uniform_hi"],
                      thresh=c["thresh"], precision=precision, T_burn=T_burn, stream=stream)

    # warm-up on a shortened run (its own handle: the burn-in must stay inside it)
    handle(ACCURATE_T, args.precision, 0.0).run(T_end / 10, 1)
    g = handle(ACCURATE_T, args.precision, c["T_burn"])
    n = max(3, args.steps)
    v, ms, acc = timed_runs(g, n, rank_seed(rank, 50_000), T_end)
    g.close()
    out["accurate_threshold"] = {
        "t_corr": ACCURATE_T, "t_phase": ACCURATE_T, "value": v, "unit": "events/s", "steps": n, "ms_per_step": ms,
        "dtype": args.precision, "accuracy": accuracy_summary(acc[0], acc[1], acc[2], acc[3], ACCURATE_T),
        "note": "same workload and launch as the headline with longer thresholds; pooled over 1024 runs "
                "(bench.py --workload accuracy) this threshold gives TV 0.001 +- 0.002 and escape rates "
                "within 1% of the exact ones"}
    if args.precision != "f64":
        handle(c["t_corr"], "f64", 0.0).run(T_end / 100, 2)  # warm-up
        g = handle(c["t_corr"], "f64", c["T_burn"])
        v, ms, acc = timed_runs(g, 1, rank_seed(rank, 60_000), T_end)
        g.close()
        out["fp64"] = {"value": v, "unit": "events/s", "steps": 1, "ms_per_step": ms, "dtype": "f64",
                       "accuracy": accuracy_summary(acc[0], acc[1], acc[2], acc[3], c["t_corr"]),
                       "note": "the plain binary64 form of the headline workload (one thread per replica)"}
    if rank == 0 and args.serve_seconds_default > 0:
        sv = serve_stream(args, local, 200.0, args.serve_seconds_default)
        out["serve"] = {k: sv[k] for k in ("value", "unit", "latency_s", "config", "server", "gpu_launches")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch

    from paper_1705_06807_gb300 import ParRep
    from paper_1705_06807_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload in ("speedup", "uq", "sweep", "accuracy"):
        if rank == 0:
            dict(speedup=bench_speedup, uq=bench_uq, sweep=bench_sweep, accuracy=bench_accuracy)[args.workload](args)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "serve":
        if rank == 0:
            bench_serve(args, local)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "batch256":
        bench_batch(args, world, rank, local, dist)
        if dist:
            dist.destroy_process_group()
        return
    c = workload(args.workload)
    T_end = args.T_end or c["T_end"]
    if args.x0 is not None:
        c["x0"], c["x0_uniform_hi"] = [args.x0], 0
    if args.t_corr is not None:
        c["t_corr"] = args.t_corr
    if args.t_phase is not None:
        c["t_phase"] = args.t_phase
    stream = torch.cuda.Stream()
    g = ParRep(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], x0=c["x0"],
               x0_uniform_hi=c["x0_uniform_hi"], thresh=c["thresh"], precision=args.precision,
               T_burn=c["T_burn"] * T_end / c["T_end"], stream=stream, block_threads=args.block_threads,
               chunk_steps=args.chunk_steps, f32_layout=args.f32_layout)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    seed0 = rank_seed(rank, 0)

    def one(i):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))  # evicts L2 (129 MB) between steps, outside the timed region
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.run(T_end, seed0 + i)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), g.stats()

    for i in range(args.warmup):
        one(i)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats, acc = [], [], ([], [], [], [])
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ms, st = one(args.warmup + i)
            times.append(ms)
            stats.append(st)
            # outside the timed region: the run's outputs for the accuracy keys
            acc[0].append(g.histogram())
            acc[1].append(st["T_s"])
            acc[2].append(st["escapes"])
            acc[3].append(np.diag(g.fim()) if c["network"]["kind"] == "schlogl" else None)
    torch.cuda.synchronize()
    t_total = sum(times) / 1e3
    useful = sum(s["events_decorr"] + s["events_parallel_useful"] for s in stats)
    executed = sum(s["events_decorr"] + s["events_parallel_executed"] + s["events_replay"] + s["events_dephase"]
                   for s in stats)
    dephase = sum(s["events_dephase"] for s in stats)
    kernel_s = sum(s["kernel_ms"] for s in stats) / 1e3
    ph = {}
    for s_ in stats:
        for k, v in s_["phase_cycles"].items():
            ph[k] = ph.get(k, 0.0) + v
    main_phases = [k for k in ph if not k.startswith("dec_")]
    ph_tot = sum(ph[k] for k in main_phases) or 1.0
    phase_share = {k: round(v / ph_tot, 4) for k, v in ph.items()}
    events = {k: sum(s_[k] for s_ in stats) // max(1, len(stats)) for k in
              ("events_decorr", "events_dephase", "events_parallel_useful", "events_parallel_executed",
               "events_replay", "cycles", "escapes")}
    t_total, (useful, executed) = combine_ranks(dist, t_total, [useful, executed], "cuda")
    clocks = clk.summary()
    value = useful / t_total

    # e2e through the public API with host buffers: create (host structs and
    # tables copied in), run, histogram + FIM read back into host memory.
    e2e = None
    if not args.no_e2e:
        e_times, e_useful = [], 0
        nb = g.n_bins
        for i in range(max(1, min(args.steps, 3))):
            t0 = time.perf_counter()
            h = ParRep(c["network"], c["n_replicas"], c["t_corr"], c["t_phase"], x0=c["x0"],
                       x0_uniform_hi=c["x0_uniform_hi"], thresh=c["thresh"], precision=args.precision,
                       T_burn=c["T_burn"] * T_end / c["T_end"], block_threads=args.block_threads,
                       chunk_steps=args.chunk_steps, f32_layout=args.f32_layout)
            st = h.run(T_end, seed0 + args.warmup + i)  # the timed steps' seeds: the same work
            hist = h.histogram()
            fim = h.fim()
            h.close()
            e_times.append(time.perf_counter() - t0)
            e_useful += st["events_decorr"] + st["events_parallel_useful"]
            assert hist.shape == (nb,) and np.isfinite(fim).all()
        e2e = {"value": e_useful / sum(e_times), "unit": "events/s",
               "h2d_bytes_per_step": 8 * (6 + 4) + 4 * 8,
               "d2h_bytes_per_step": 8 * nb + 8 * 16 + 512}
    # roofline: issue rate of plain ALU instructions
    peak_ops, peak_note = issue_peak(clocks)
    ops = (executed - dephase) * OPS_PER_EVENT + dephase * OPS_PER_DEPHASE_EVENT
    achieved = ops / kernel_s if kernel_s > 0 else None
    schlogl = args.workload == "schlogl_n4096"
    accuracy = accuracy_summary(acc[0], acc[1], acc[2], acc[3], c["t_corr"]) if schlogl and args.T_end is None \
        else None
    line = {
        "metric": "SSA events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": c["name"], "replicas": c["n_replicas"], "T_end": T_end,
                   "thresholds": "time t_corr=t_phase=1",
                   "x0": f"uniform {{0..{c['x0_uniform_hi']}}}" if c["x0_uniform_hi"] else str(c["x0"]),
                   "fim_window": [c["T_burn"] * T_end / c["T_end"], T_end],
                   "accumulators": "64-bit fixed point 2^-40", "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"independent instances x{world}",
                   "launch": f"{stats[-1]['grid_blocks']} blocks x {stats[-1]['block_threads']} threads "
                             f"({args.precision}, layout {args.f32_layout})"},
        "executed_events_per_s": executed / t_total,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12 if achieved else None,
                     "peak": peak_ops / 1e12, "unit": "Tinst/s",
                     "frac": achieved / peak_ops if achieved else None,
                     "traffic": RUN_KERNEL_TRAFFIC if (schlogl and args.T_end is None and args.precision == "f32"
                                                       and args.f32_layout != "direct") else None,
                     "note": "thread-instructions at 120 per event (107 per dephasing jump) over the run kernel "
                             "time; peak = " + peak_note + "; traffic = DRAM bytes read + written per launch "
                             "(ncu launch list of this command, profiles/)"},
        "phase_share": phase_share,
        "events_per_step": events,
        "accuracy": accuracy,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if schlogl and args.T_end is None and not args.no_extras:
        line.update(side_measurements(args, c, rank, local, stream, flush))
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(c)
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(c)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
