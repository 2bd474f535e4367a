"""Benchmark: exact min-cut of the gaze-line stereo graph, 384x288 pair, 16 depth numbers.

One step = the whole hot path on one synthetic stereo pair already resident in
device memory: data-term cost volume, chain-graph build, push-relabel max-flow
to the exact cut, label extraction.  The metric is milliseconds per pair (lower
is better).  L2 is flushed (a 512 MiB write) before every timed step, outside
the timed events.

Extra keys on the JSON line:
  e2e           the same metric through the public API from pinned host images
                to host labels (H2D + four C-ABI calls + D2H inside the timing)
  roofline      the push-relabel sweep kernel: algorithmic bytes (72 B per node
                per sweep) / its average launch time, measured with CUDA events
                on the solve's stream during the timed steps, against the
                measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (Boykov-Kolmogorov) on a bounded sample
  clocks        SM clocks and throttle reasons sampled during the timed steps

--impl reference times the CPU oracle on the same workload (the reference arm).
Multi-GPU (torchrun): replicas, each rank solves its own pairs; no collective
on the data path (weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_01516_gb300 import synth  # noqa: E402

METRIC = "ms/pair exact min-cut at 384x288x16"
UNIT = "ms/pair"
BYTES_PER_NODE_SWEEP = 72      # 9 int32 words read and written once per node per sweep
N_PAIRS = 4                    # distinct seeded pairs, cycled over the steps


def _workload():
    return synth.MAIN


def _config(wl, extra=None):
    c = {"workload": wl.name, "w": wl.w, "h": wl.h, "D": wl.D, "tau": wl.tau,
         "lambda": wl.lam, "inhibit": wl.inhibit, "vertical_inhibit": 1, "pairs_per_step": 1,
         "distinct_pairs": N_PAIRS, "l2": "flushed before each timed step (512 MiB write)"}
    if extra:
        c.update(extra)
    return c


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"gs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_baseline(wl, budget_s=20.0):
    """Time the CPU oracle (cost volume + Boykov-Kolmogorov) on whole pairs
    until about budget_s seconds of CPU work have been spent."""
    import oracle
    oracle.build()
    times = []
    t_all = time.perf_counter()
    i = 0
    while True:
        L, R, _ = synth.make_pair(wl, i % N_PAIRS)
        t0 = time.perf_counter()
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        oracle.solve(C, wl.lam, wl.inhibit, 1, "bk")
        times.append(time.perf_counter() - t0)
        i += 1
        if time.perf_counter() - t_all > budget_s or i >= 16:
            break
    return {"value": 1e3 * float(np.mean(times)), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} whole {wl.w}x{wl.h}x{wl.D} pairs, single-threaded "
                      f"Boykov-Kolmogorov + cost volume, mean ms/pair"}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only)."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    wl = _workload()
    import oracle
    oracle.build()
    pairs = [synth.make_pair(wl, i) for i in range(N_PAIRS)]

    def step(i):
        L, R, _ = pairs[i % N_PAIRS]
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        oracle.solve(C, wl.lam, wl.inhibit, 1, "bk")

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    ms = 1e3 * dt / max(args.steps, 1)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": _config(wl),
            "cpu_baseline": {"value": ms, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole pairs, single-threaded "
                                       "Boykov-Kolmogorov (the CPU oracle) + cost volume"},
            "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch

    from paper_1803_01516_gb300 import gazecut as gc

    rank, world, local = _dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    wl = _workload()
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                  vertical_inhibit=1)
    o = gc.SolveOpts(sweeps_per_relabel=args.sweeps_per_relabel)
    # each rank solves its own pairs (replicas)
    pairs = [synth.make_pair(wl, rank * N_PAIRS + i) for i in range(N_PAIRS)]
    Ld = [torch.from_numpy(L).to(dev) for L, _, _ in pairs]
    Rd = [torch.from_numpy(R).to(dev) for _, R, _ in pairs]
    buf = gc.Buffers(p, o, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        gc.solve_pair(Ld[i % N_PAIRS], Rd[i % N_PAIRS], p, o, buf)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    if int(buf.status.item()) != gc.GS_OK:
        raise RuntimeError(f"solve status {buf.status.item()}")

    clocks = ClockSampler(dev.index if world == 1 else local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches0 = gc.gs_kernel_launches()
    sweep_ns = relabel_ns = sweeps = relabels = passes = 0
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
        st = gc.gs_solve_stats(buf.work)
        sweep_ns += st["sweep_ns"]
        relabel_ns += st["relabel_ns"]
        sweeps += st["sweeps"]
        relabels += st["relabels"]
        passes += st["bfs_passes"]
    torch.cuda.synchronize(dev)
    launches = gc.gs_kernel_launches() - launches0
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    my_ms = float(sum(ms_steps))
    clk = clocks.stop() if rank == 0 else None
    if int(buf.status.item()) != gc.GS_OK:
        raise RuntimeError(f"solve status {buf.status.item()}")
    if dist:
        t = torch.tensor([my_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    else:
        tot_ms = my_ms
    total_pairs = args.steps * world
    value = tot_ms / total_pairs

    # ----- e2e through the public API from pinned host memory -----
    e2e = None
    if rank == 0:
        Lh = [torch.from_numpy(L).pin_memory() for L, _, _ in pairs]
        Rh = [torch.from_numpy(R).pin_memory() for _, R, _ in pairs]
        lab_h = torch.empty((p.h, p.ng), dtype=torch.int32).pin_memory()
        flow_h = torch.empty(1, dtype=torch.int64).pin_memory()
        Lbuf = torch.empty((p.h, p.w), dtype=torch.uint8, device=dev)
        Rbuf = torch.empty((p.h, p.w), dtype=torch.uint8, device=dev)
        e2e_ms = []
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Lbuf.copy_(Lh[i % N_PAIRS], non_blocking=True)
            Rbuf.copy_(Rh[i % N_PAIRS], non_blocking=True)
            labels, flow, _ = gc.solve_pair(Lbuf, Rbuf, p, o, buf)
            lab_h.copy_(labels, non_blocking=True)
            flow_h.copy_(flow, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e = {"value": float(np.mean(e2e_ms)), "unit": UNIT,
               "h2d_bytes_per_step": 2 * p.w * p.h,
               "d2h_bytes_per_step": 4 * p.h * p.ng + 8}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    nodes = gc.gs_num_nodes(p)
    bytes_per_sweep = BYTES_PER_NODE_SWEEP * nodes
    sweep_launch_s = (sweep_ns * 1e-9) / max(sweeps, 1)
    achieved = bytes_per_sweep / sweep_launch_s / 1e9 if sweeps else 0.0
    cpu = None if args.no_cpu_baseline or world > 1 else _cpu_baseline(wl)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": _config(wl, {"sweeps_per_relabel": o.sweeps_per_relabel,
                               "replicas": world}),
        "e2e": e2e,
        "roofline": {"bound": "hbm", "kernel": "k_sweep", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"{peak_kind} HBM copy",
                     "bytes_per_launch": bytes_per_sweep,
                     "avg_launch_us": sweep_launch_s * 1e6},
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": int(launches),
        "solver": {"sweeps_per_pair": sweeps / args.steps, "relabels_per_pair": relabels / args.steps,
                   "bfs_passes_per_pair": passes / args.steps,
                   "sweep_ms_per_pair": sweep_ns * 1e-6 / args.steps,
                   "relabel_ms_per_pair": relabel_ns * 1e-6 / args.steps},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gazecut", choices=["gazecut", "reference"])
    ap.add_argument("--sweeps-per-relabel", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
