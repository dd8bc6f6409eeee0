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

PEAK_SM_CLOCK_HZ = 2.07e9  # maximum SM clock of a GB300
N_SM = 152
# Thread-instructions per event of the FP32 form, counted from the operations
# an event needs (see the design notes): Philox4x32-10 = 10 rounds x (2 wide
# multiplies, 2 three-way XORs, 2 key adds) = 60; two uniforms 8; Schloegl
# propensities 8; a0 3; tau (log, negate, divide, scale, convert) 14;
# selection 10; update and region 4; histogram address + shared atomic 3;
# clock sum, counters and exit tests 10.  Dephasing jumps skip tau and the
# histogram (-17) but add the Fleming-Viot ballots (+4).
OPS_PER_EVENT = 120
OPS_PER_DEPHASE_EVENT = 107


def workload():
    from paper_1705_06807_gb300 import configs as K

    return K.C2


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


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = workload()
    vals, tot_t, tot_ev = [], 0.0, 0
    sample_T = 300.0
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(c, sample_T=sample_T, seed=1000 + i)
        if i >= args.warmup:
            vals.append(b)
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": "SSA events/s", "value": v, "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c["name"], "replicas": c["n_replicas"], "T_end_sample": sample_T},
            "cpu_baseline": {"value": v, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    c = dict(workload())
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
               chunk_steps=args.chunk_steps)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    seed0 = 1_000_003 * (rank + 1)

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
    times, stats = [], []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ms, st = one(args.warmup + i)
            times.append(ms)
            stats.append(st)
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
    if dist:
        t = torch.tensor([t_total, float(useful), float(executed)], device="cuda", dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        t_total, useful, executed = float(tmax[0]), int(t[1]), int(t[2])
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
                       chunk_steps=args.chunk_steps)
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
    peak_ops = N_SM * 4 * 32 * PEAK_SM_CLOCK_HZ
    ops = (useful_ops := (executed - dephase) * OPS_PER_EVENT) + dephase * OPS_PER_DEPHASE_EVENT
    achieved = ops / kernel_s if kernel_s > 0 else None
    line = {
        "metric": "SSA events/s", "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": c["name"], "replicas": c["n_replicas"], "T_end": T_end,
                   "thresholds": "time t_corr=t_phase=1", "x0": "uniform {0..1000}",
                   "fim_window": [c["T_burn"] * T_end / c["T_end"], T_end],
                   "accumulators": "64-bit fixed point 2^-40", "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"independent instances x{world}"},
        "executed_events_per_s": executed / t_total,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12 if achieved else None,
                     "peak": peak_ops / 1e12, "unit": "Tinst/s",
                     "frac": achieved / peak_ops if achieved else None, "traffic": None,
                     "note": "thread-instructions at 120 per event (107 per dephasing jump) over the run kernel "
                             "time; peak = 152 SM x 4 schedulers x 32 lanes x 2.07 GHz"},
        "phase_share": phase_share,
        "events_per_step": events,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(c)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
