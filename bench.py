"""Benchmark: exact min-cut of the gaze-line stereo graph, 384x288 pair, 16 depth numbers.

One step = the whole hot path on one synthetic stereo pair already resident in
device memory: data-term cost volume, chain-graph build, push-relabel max-flow
to the exact cut, label extraction.  The metric is milliseconds per pair (lower
is better).  L2 is flushed (a 512 MiB write) before every timed step, outside
the timed events.

Extra keys on the JSON line:
  e2e           the same metric through the public API from pinned host images
                to host labels (H2D + four C-ABI calls + D2H inside the timing)
  roofline      the persistent solve kernel (the dominant one): algorithmic
                bytes (72 B per node of every tile a sweep round visits, 40 B
                per node of every tile a relabel pass visits) / its launch
                time, measured with CUDA events on the solve's stream during
                the timed steps, against the L2-resident copy bandwidth
                measured in the same run (the state fits in L2) and the
                measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (Boykov-Kolmogorov) on the bench's distinct pairs,
                whose results also check the timed GPU results (parity_vs_oracle)
  clocks        SM clocks and throttle reasons sampled during the timed steps
  batched       64 uneven pairs in one batched call replayed as a CUDA graph
                (pairs/s) vs one call per pair
  differentiated  forward exact solve + backward, 16 pairs at 384x288x32,
                device-timed, next to the plain exact solve of the same pairs
  learning      200 Adam steps on (w1, w2, tau, lambda) by the structured hinge
                loss over 16 pairs at 384x288x32; Eq. 2 error before and after
  fixed_sweeps  integer energy gap and ms of the fixed-sweep approximate mode
  rgb_data_term the paper's colour data term on colour versions of the pairs
  level1_approximation / level2_approximation  §4.5's approximate modes (ms,
                energy gap against the exact minimum, oracle parity of one pair)
  large         one 1920x1080x128 exact solve (228.5 M nodes) with its roofline

--impl reference times the CPU oracle on the same workload (the reference arm).
Multi-GPU (torchrun): replicas, each rank solves its own pairs; no collective
on the data path (weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
BYTES_PER_NODE_BFS = 40        # 9 words read, the height written, per node per BFS level
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


def _profiled_traffic():
    """DRAM bytes per launch of the solve kernel from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_batch_main-384x288x16.md")
    src = os.path.join(ROOT, "paper_1803_01516_gb300", "csrc", "tile.cu")
    try:
        kv = {}
        for line in open(prof):
            if ":" in line and not line.startswith(("|", " ", "#")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if kv.get("kernel_source_sha256_16") != sha:
            return None
        return int(kv["traffic_bytes_per_launch"])
    except Exception:
        return None


def _l2_copy_gbs(dev, mib: int = 32, reps: int = 200, trials: int = 5) -> float:
    """Streaming bandwidth of an L2-resident working set through the SMs,
    measured here: an elementwise kernel (dst = src + 1, int32) over a
    `mib` MiB buffer into another (2 x 32 MiB, well under the 129 MB L2),
    `reps` launches back to back after a warm-up, CUDA events, best of
    `trials`; read + write bytes.  (A plain same-type copy_ would go to the
    driver's device-to-device memcpy, not through the SMs.)"""
    import torch
    src = torch.ones((mib << 20) // 4, dtype=torch.int32, device=dev)
    dst = torch.empty_like(src)
    for _ in range(20):
        torch.add(src, 1, out=dst)
    best = 0.0
    for _ in range(trials):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            torch.add(src, 1, out=dst)
        b.record()
        b.synchronize()
        best = max(best, 2.0 * 4 * src.numel() * reps / (a.elapsed_time(b) * 1e-3) / 1e9)
    return best


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


def _cpu_info() -> dict:
    """Host CPU model (first model line of /proc/cpuinfo) and core count."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "hardware", "cpu part", "processor name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    # Arm hosts list a part number instead of a name
    model = {"0xd4f": "Arm Neoverse V2 (part 0xd4f)", "0xd40": "Arm Neoverse V1 (part 0xd40)",
             "0xd0c": "Arm Neoverse N1 (part 0xd0c)"}.get(model.lower(), model)
    return {"cpu_model": model, "nproc": os.cpu_count()}


def _oracle_pair_ms(item):
    """One whole pair through the CPU oracle (a pool worker; no GPU)."""
    D, dis0, tau, lam, inhibit, L, R = item
    import oracle
    t0 = time.perf_counter()
    C = oracle.cost_volume(L, R, D, dis0, tau)
    oracle.solve(C, lam, inhibit, 1, "bk")
    return 1e3 * (time.perf_counter() - t0)


def _batched_cpu_baseline(batch, n_sample=2):
    """The oracle on the batch's n_sample pairs nearest its lower-quartile node
    count (a pair near the median takes the oracle most of a minute), one pair
    per process on the host cores (a spawn pool: no process forked from one
    that holds a GPU context).  pairs/s = cores / mean time per pair, i.e. the
    whole batch spread over all cores; the sample leaves out the batch's larger
    pairs, on which Boykov-Kolmogorov is slower, so this rate favours the CPU."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    nodes = np.array([(wl.w - 2 * (wl.D - 1)) * wl.h * (wl.D - 1) for wl, _, _, _ in batch])
    target = np.percentile(nodes, 25)
    pick = [int(k) for k in np.argsort(np.abs(nodes - target))[:n_sample]]
    items = [(batch[k][0].D, 2 * (batch[k][0].D - 1), batch[k][0].tau, batch[k][0].lam,
              batch[k][0].inhibit, batch[k][1], batch[k][2]) for k in pick]
    cores = os.cpu_count() or 1
    workers = min(cores, n_sample)
    with mp.get_context("spawn").Pool(workers) as pool:
        ms = pool.map(_oracle_pair_ms, items)
    return {"value": 1e3 * cores / float(np.mean(ms)), "unit": "pairs/s", "cores": cores,
            "kind": "oracle",
            "sample": f"the {n_sample} of the {len(batch)} pairs nearest the lower-quartile node "
                      f"count ({int(target)}; median {int(np.median(nodes))}), single-threaded "
                      f"Boykov-Kolmogorov + cost volume "
                      f"each, {workers} at a time; pairs/s = cores / mean time per pair "
                      f"({float(np.mean(ms)):.0f} ms)", **_cpu_info()}


def _cpu_baseline(wl, pairs):
    """The CPU oracle (cost volume + Boykov-Kolmogorov, single-threaded) on the
    bench's distinct pairs; returns the timing line and the oracle solutions."""
    import oracle
    oracle.build()
    times, refs = [], []
    for L, R, _ in pairs:
        t0 = time.perf_counter()
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        refs.append(oracle.solve(C, wl.lam, wl.inhibit, 1, "bk"))
        times.append(time.perf_counter() - t0)
    cpu = {"value": 1e3 * float(np.mean(times)), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the {len(pairs)} distinct {wl.w}x{wl.h}x{wl.D} pairs of the timed steps, "
                     "whole pairs, single-threaded Boykov-Kolmogorov + cost volume, mean ms/pair",
           **_cpu_info()}
    return cpu, refs


def _reduce_max(ms: float, dist, device) -> float:
    """The job's time is the slowest replica's: max over ranks (no other
    collective: each rank solves its own pairs)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_pairs(rank: int, n: int = None):
    """Seeded pair indices of a replica: disjoint across ranks."""
    n = N_PAIRS if n is None else n
    return [rank * n + i for i in range(n)]


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


def _batched(gc, dev, args, stream, flush):
    """64 synthetic pairs of uneven size and depth range in one batched call
    (two persistent launches) vs the same pairs solved one call at a time."""
    import torch
    from paper_1803_01516_gb300 import autotune
    batch = synth.make_batch(args.batch_pairs)
    params = [gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                        vertical_inhibit=1) for wl, _, _, _ in batch]
    opts = [autotune.tuned_opts(p) for p in params]
    B = gc.Batch(params, opts, device=dev)
    Ls = [torch.from_numpy(L).to(dev) for _, L, _, _ in batch]
    Rs = [torch.from_numpy(R).to(dev) for _, _, R, _ in batch]
    gc.gs_solve_batched(B, Ls, Rs)                    # warm-up (and set-up outside capture)
    torch.cuda.synchronize(dev)
    # the whole batched call captured once in a CUDA graph, then replayed
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            gc.gs_solve_batched(B, Ls, Rs)
    stream.wait_stream(cap)
    graph.replay()
    torch.cuda.synchronize(dev)
    times, times_uncaptured = [], []
    for i in range(args.batch_steps):
        for captured in (True, False):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if captured:
                graph.replay()
            else:
                gc.gs_solve_batched(B, Ls, Rs)
            b.record(stream)
            b.synchronize()
            (times if captured else times_uncaptured).append(a.elapsed_time(b))
    graph.replay()
    torch.cuda.synchronize(dev)
    ok = all(int(b.status.item()) == gc.GS_OK for b in B.bufs)
    flows = [int(b.flow.item()) for b in B.bufs]
    # the same pairs, one call each (same buffers, same options)
    t_single = 0.0
    for i, (p, o, buf) in enumerate(zip(params, opts, B.bufs)):
        flush.fill_(i & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gc.solve_pair(Ls[i], Rs[i], p, o, buf)
        b.record(stream)
        b.synchronize()
        t_single += a.elapsed_time(b)
        ok &= int(buf.flow.item()) == flows[i]
    nodes = sum(gc.gs_num_nodes(p) for p in params)
    out = {"pairs": len(params), "nodes": nodes, "ms_per_batch": float(np.mean(times)),
           "pairs_per_s": 1e3 * len(params) / float(np.mean(times)),
           "timed_as": "replay of one CUDA graph holding the whole batched call",
           "uncaptured_ms_per_batch": float(np.mean(times_uncaptured)),
           "single_call_loop_ms": t_single,
           "single_call_pairs_per_s": 1e3 * len(params) / t_single,
           "flows_match_single_calls": bool(ok),
           "workload": "64 pairs, w~U[160,640], h~U[120,480], D~U[16,64], layered scenes"}
    if not args.no_batched_cpu_baseline and not args.no_cpu_baseline:
        out["cpu_baseline"] = _batched_cpu_baseline(batch)
    if not args.no_cpu_baseline:
        import oracle
        order = np.argsort([gc.gs_num_nodes(p) for p in params])[:2]
        good = True
        for k in order:
            wl, L, R, _ = batch[k]
            C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
            ref = oracle.solve(C, wl.lam, wl.inhibit, 1, "bk")
            good &= flows[k] == ref["flow"] and bool(np.array_equal(
                B.bufs[k].labels.cpu().numpy(), ref["labels"]))
        out["parity_vs_oracle"] = {"pairs_checked": len(order), "equal": good}
    return out


def _learned_workload():
    return synth.Workload("learned-384x288x32", 384, 288, 32, tau=30, lam=8, sigma=2.0,
                          scene="layers", n_layers=5, n_slanted=2, max_disp=31, seed_base=5)


def _differentiated(gc, dev, args, stream):
    """Forward exact solve + backward on 16 pairs at 384x288 with 32 depth
    numbers (learned FP32 data term, scale 256), device-timed with CUDA
    events around the whole loop (the forward never waits for the device; the
    only host reads are the gradient transfers of the backward), next to the
    plain exact solve of the same pairs and cost volumes (no gradient)."""
    import torch
    from paper_1803_01516_gb300 import learn
    from paper_1803_01516_gb300 import autotune
    wl = _learned_workload()
    probs = []
    for i in range(args.diff_pairs):
        L, R, _ = synth.make_pair(wl, i)
        p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=0, lam=0, inhibit=1023 * 256)
        probs.append(learn.problem(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), p,
                                   autotune.tuned_opts(p)))
    theta = torch.tensor([1.0, 1.0, 30.0, 8.0], dtype=torch.float64, requires_grad=True)
    learn.min_energy(theta, probs[0]).backward()        # warm-up
    torch.cuda.synchronize(dev)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    def fwd_bwd():
        theta.grad = None
        E = sum(learn.min_energy(theta, pr) for pr in probs)
        E.backward()

    def plain():
        for pr in probs:
            learn.labels_at(theta, pr)

    t_fb = min(timed(fwd_bwd) for _ in range(2))
    t_plain = min(timed(plain) for _ in range(2))
    for pr in probs:
        pr.check()
    n = len(probs)
    return {"pairs": n, "ms_per_pair_fwd_bwd": t_fb / n, "pairs_per_s": 1e3 * n / t_fb,
            "plain_exact_ms_per_pair": t_plain / n,
            "backward_overhead": t_fb / t_plain - 1.0,
            "timed_as": "CUDA events around all pairs (best of 2); forward = FP32 cost volume, "
                        "graph, exact solve, labels, adjoint kernels; plain = the same without "
                        "the adjoint",
            "workload": "384x288, 32 depth numbers, learned FP32 cost at scale 256"}


def _learning(gc, dev, args):
    """The learning workload: Adam on (w1, w2, tau, lambda) from (1, 1, 30, 8)
    against the synthetic ground-truth depth of 16 pairs at 384x288x32 by the
    structured hinge loss (exact loss-augmented cuts), theta projected to >= 0
    after each step; Eq. 2 error and exact-site fraction before and after."""
    import torch
    from paper_1803_01516_gb300 import learn, metrics
    from paper_1803_01516_gb300 import autotune
    wl = _learned_workload()
    probs, gts, gts_np = [], [], []
    for i in range(args.diff_pairs):
        L, R, dR = synth.make_pair(wl, 100 + i)
        p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=0, lam=0, inhibit=1023 * 256)
        probs.append(learn.problem(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), p,
                                   autotune.tuned_opts(p)))
        gt = metrics.gt_depth(dR, wl.D, 2 * (wl.D - 1))
        gts_np.append(gt)
        gts.append(torch.from_numpy(gt).to(dev))

    def accuracy(theta):
        err, exact, sites = 0, 0, 0
        for pr, gt in zip(probs, gts_np):
            X = learn.labels_at(theta, pr).cpu().numpy()
            hist = metrics.depth_error_hist(X, gt)
            err += metrics.depth_error_from_hist(hist)
            exact += int(hist[0])
            sites += int(hist.sum())
        return {"eq2_error": err, "exact_fraction": exact / sites, "sites": sites}

    theta0 = (1.0, 1.0, 30.0, 8.0)
    before = accuracy(torch.tensor(theta0, dtype=torch.float64))
    t0 = time.perf_counter()
    theta, losses = learn.fit(theta0, probs, gts, steps=args.learn_steps, lr=args.learn_lr)
    wall = time.perf_counter() - t0
    after = accuracy(theta)
    marks = sorted(set([0, len(losses) - 1] + list(range(0, len(losses), 20))))
    return {"pairs": len(probs), "steps": len(losses), "optimizer": f"Adam lr={args.learn_lr}",
            "theta0": {"w1": theta0[0], "w2": theta0[1], "tau": theta0[2], "lambda": theta0[3]},
            "theta": dict(zip(["w1", "w2", "tau", "lambda"], [float(x) for x in theta])),
            "hinge_loss": {str(k): losses[k] for k in marks},
            "before": before, "after": after, "wall_s": wall,
            "workload": "16 pairs at 384x288, 32 depth numbers (seeds disjoint from the "
                        "differentiated leg), ground truth = the scene generator's depth"}


def _rgb(gc, dev, flush, stream, with_oracle):
    """The paper's colour data term (§4.3: |dR|+|dG|+|dB|, 0..765, no
    truncation, lambda = 14) on colour versions of the main workload's pairs:
    device ms of the whole path per pair, one pair checked against the oracle."""
    import torch
    from paper_1803_01516_gb300 import autotune
    wl = synth.MAIN
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=765, lam=14, inhibit=wl.inhibit,
                  vertical_inhibit=1)
    o = autotune.tuned_opts(p)
    buf = gc.Buffers(p, o, device=dev)
    pairs = [synth.make_pair_rgb(wl, i) for i in range(N_PAIRS)]
    Ld = [torch.from_numpy(L).to(dev) for L, _, _ in pairs]
    Rd = [torch.from_numpy(R).to(dev) for _, R, _ in pairs]
    ms, cost_ms = [], []
    for rep_ in range(3):
        for k in range(N_PAIRS):
            flush.fill_(k & 0xff)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            gc.gs_stereo_cost_volume_rgb(Ld[k], Rd[k], p, buf.cost)
            ev[1].record(stream)
            gc.solve_costs(buf.cost, p, o, buf)
            ev[2].record(stream)
            ev[2].synchronize()
            if int(buf.status.item()) != gc.GS_OK:
                raise RuntimeError("rgb solve status")
            if rep_:
                ms.append(ev[0].elapsed_time(ev[2]))
                cost_ms.append(ev[0].elapsed_time(ev[1]))
    out = {"workload": "colour versions of the main workload's pairs (384x288x16), tau 765, "
                       "lambda 14", "ms_per_pair": float(np.mean(ms)),
           "cost_volume_ms": float(np.mean(cost_ms))}
    if with_oracle:
        import oracle
        L, R, _ = pairs[0]
        gc.gs_stereo_cost_volume_rgb(Ld[0], Rd[0], p, buf.cost)
        gc.solve_costs(buf.cost, p, o, buf)
        C = oracle.cost_volume_rgb(L, R, wl.D, 2 * (wl.D - 1), 765)
        ref = oracle.solve(C, 14, wl.inhibit, 1)
        out["parity_vs_oracle"] = {
            "pairs_checked": 1,
            "cost_volume_equal": bool(np.array_equal(buf.cost.cpu().numpy().reshape(C.shape), C)),
            "flow_equal": int(buf.flow.item()) == ref["flow"],
            "labels_equal": bool(np.array_equal(buf.labels.cpu().numpy(), ref["labels"]))}
    return out


def _fixed_sweeps(gc, dev, p, o, Ld, Rd, exact_flows, flush, stream):
    """Fixed-sweep approximate mode on the main pairs: integer energy gap of its
    labels against the exact minimum, and device ms of solve + labels."""
    import torch
    buf = gc.Buffers(p, o, device=dev)
    E = torch.zeros(1, dtype=torch.int64, device=dev)
    out = {}
    for n in (8, 32, 128):
        of = gc.SolveOpts(mode=gc.GS_MODE_FIXED_SWEEPS, fixed_sweeps=n,
                          sweeps_per_relabel=min(n, o.sweeps_per_relabel),
                          local_iters=o.local_iters, relabel_passes=o.relabel_passes,
                          tile_w=o.tile_w, tile_h=o.tile_h)
        ms, gaps, rel, lows = [], [], [], []
        for rep_ in range(2):
            for k in range(len(Ld)):
                gc.gs_stereo_cost_volume(Ld[k], Rd[k], p, buf.cost)
                gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
                flush.fill_(k & 0xff)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gc.gs_maxflow_solve(buf.graph, p, of, buf.work, buf.status)
                gc.gs_extract_labels(buf.graph, p, of, buf.work, buf.labels, buf.flow, buf.status)
                c.record(stream)
                gc.gs_energy(buf.cost, buf.labels, p, E)
                c.synchronize()
                if int(buf.status.item()) != gc.GS_OK:
                    raise RuntimeError("fixed-sweep status")
                if rep_ == 0:
                    continue
                ms.append(a.elapsed_time(c))
                gap = int(E.item()) - exact_flows[k]
                if gap < 0 or int(buf.flow.item()) > exact_flows[k]:
                    raise RuntimeError("fixed-sweep bounds violated")
                gaps.append(gap)
                rel.append(gap / exact_flows[k])
                lows.append((exact_flows[k] - int(buf.flow.item())) / exact_flows[k])
        out[str(n)] = {"ms_per_pair": float(np.mean(ms)), "energy_gap_mean": float(np.mean(gaps)),
                       "energy_gap_rel_mean": float(np.mean(rel)), "max_gap": int(max(gaps)),
                       "flow_shortfall_rel_mean": float(np.mean(lows))}
    return {"workload": "the main workload's pairs", "sweeps": out,
            "gap": "E(labels) - exact min E (integer, >= 0); labels from the nodes that "
                   "cannot reach remaining sink capacity"}


def _large(gc, dev, flush, stream, peak):
    """One 1920x1080 pair with 128 depth numbers (228.5 M graph nodes): device
    time of each step of the path, solver statistics and the solve kernel's
    algorithmic bytes against the HBM peak (the 8.2 GB state does not fit in
    L2); flow == E(labels) checked on the device (the oracle cannot solve this
    size; tests/test_large.py certifies it on the CPU)."""
    import torch
    from paper_1803_01516_gb300 import autotune
    wl = synth.LARGE
    L, R, _ = synth.make_pair(wl, 0)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit,
                  vertical_inhibit=1)
    o = autotune.tuned_opts(p)
    buf = gc.Buffers(p, o, device=dev)
    Ld, Rd = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
    E = torch.zeros(1, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    flush.fill_(1)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    gc.gs_stereo_cost_volume(Ld, Rd, p, buf.cost)
    gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
    ev[1].record(stream)
    gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
    ev[2].record(stream)
    gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
    ev[3].record(stream)
    gc.gs_energy(buf.cost, buf.labels, p, E)
    ev[3].synchronize()
    st = gc.gs_solve_stats(buf.work)
    status = int(buf.status.item())
    flow = int(buf.flow.item())
    nodes = gc.gs_num_nodes(p)
    ti = gc.gs_tile_info(p, o)
    npt = nodes / ti["tiles"]
    alg = (BYTES_PER_NODE_SWEEP * st["sweep_visits"] + BYTES_PER_NODE_BFS * st["relabel_visits"]) \
        * npt
    solve_ms = ev[1].elapsed_time(ev[2])
    achieved = alg / (solve_ms * 1e-3) / 1e9
    out = {"workload": wl.name, "nodes": nodes, "status": gc.STATUS_NAMES[status],
           "ms_total": ev[0].elapsed_time(ev[3]),
           "phases_ms": {"cost_volume+build": ev[0].elapsed_time(ev[1]), "maxflow_solve": solve_ms,
                         "extract_labels": ev[2].elapsed_time(ev[3])},
           "solver": {k: st[k] for k in ("relabels", "sweeps", "bfs_passes", "sweep_visits",
                                          "relabel_visits")},
           "tile": [ti["tile_w"], ti["tile_h"]],
           "flow": flow, "flow_equals_energy_of_labels": flow == int(E.item()),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "alg_bytes": alg,
                        "accounting": "72 B/node per tile visit of a sweep round + 40 B/node "
                                      "per tile visit of a relabel pass"}}
    del buf
    torch.cuda.empty_cache()
    return out


def _level1(gc, dev, p, Ld, Rd, exact_flows, flush, stream, with_oracle):
    """Level-1 approximation (§4.5) on the main workload's pairs, block sizes
    2 and 3: device time per pair from the images (cost volume, delegate cut,
    skin, second cut, labels), energy gap against the exact minimum, and one
    pair checked against the oracle."""
    import torch
    from paper_1803_01516_gb300 import autotune
    out = {"workload": "the main workload's pairs", "block_sizes": {}}
    cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device=dev)
    E = torch.zeros(1, dtype=torch.int64, device=dev)
    for b in (2, 3):
        pc = gc.gs_delegate_params(p, b)
        bufs = gc.Level1Buffers(p, b, autotune.tuned_opts(p), autotune.tuned_opts(pc), device=dev)
        ms, gaps, rel = [], [], []
        for rep_ in range(4):
            for k in range(len(Ld)):
                flush.fill_(k & 0xff)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gc.gs_stereo_cost_volume(Ld[k], Rd[k], p, cost)
                X, _, st = gc.solve_level1(cost, p, b, bufs.o, bufs)
                c.record(stream)
                c.synchronize()
                if int(st.item()) != gc.GS_OK:
                    raise RuntimeError(f"level-1 status {int(st.item())}")
                if rep_ == 0:
                    continue                      # warm-up round
                ms.append(a.elapsed_time(c))
                gc.gs_energy(cost, X, p, E)
                gap = int(E.item()) - exact_flows[k]
                gaps.append(gap)
                rel.append(gap / exact_flows[k])
        entry = {"ms_per_pair": float(np.mean(ms)), "energy_gap_mean": float(np.mean(gaps)),
                 "energy_gap_rel_mean": float(np.mean(rel)), "min_gap": int(min(gaps))}
        if with_oracle and b == 2:
            import oracle
            from oracle import level1 as l1
            gc.gs_stereo_cost_volume(Ld[0], Rd[0], p, cost)
            X, Xc, _ = gc.solve_level1(cost, p, b, bufs.o, bufs)
            C = cost.cpu().numpy().reshape(p.h, p.ng, p.D)
            ref = l1.level1(C, p.lam, p.inhibit, 1, b)
            entry["parity_vs_oracle"] = {
                "pairs_checked": 1,
                "labels_equal": bool(np.array_equal(X.cpu().numpy(), ref["labels"])),
                "coarse_labels_equal": bool(np.array_equal(Xc.cpu().numpy(), ref["coarse_labels"]))}
        out["block_sizes"][str(b)] = entry
    return out


def _level2(gc, dev, p, Ld, Rd, exact_flows, flush, stream, with_oracle, passes=2):
    """Level-2 approximation (§4.5) on the main workload's pairs, block sizes 2
    and 3: device time per pair from the images (cost volume, delegate cut,
    skin, start labels, two passes of block cuts), energy gap against the
    exact minimum, and one pair checked against the oracle."""
    import torch
    from paper_1803_01516_gb300 import autotune
    out = {"workload": "the main workload's pairs", "passes": passes, "block_sizes": {}}
    cost = torch.empty(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device=dev)
    E = torch.zeros(1, dtype=torch.int64, device=dev)
    for b in (2, 3):
        pc = gc.gs_delegate_params(p, b)
        bufs = gc.Level1Buffers(p, b, autotune.tuned_opts(p), autotune.tuned_opts(pc), device=dev)
        ms, gaps, rel = [], [], []
        for rep_ in range(4):
            for k in range(len(Ld)):
                flush.fill_(k & 0xff)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gc.gs_stereo_cost_volume(Ld[k], Rd[k], p, cost)
                X, _, st = gc.solve_level2(cost, p, b, passes, bufs.o, bufs)
                c.record(stream)
                c.synchronize()
                if int(st.item()) != gc.GS_OK:
                    raise RuntimeError(f"level-2 status {int(st.item())}")
                if rep_ == 0:
                    continue
                ms.append(a.elapsed_time(c))
                gc.gs_energy(cost, X, p, E)
                gap = int(E.item()) - exact_flows[k]
                gaps.append(gap)
                rel.append(gap / exact_flows[k])
        entry = {"ms_per_pair": float(np.mean(ms)), "energy_gap_mean": float(np.mean(gaps)),
                 "energy_gap_rel_mean": float(np.mean(rel)), "min_gap": int(min(gaps))}
        if with_oracle:
            import oracle
            from oracle import level2 as l2
            gc.gs_stereo_cost_volume(Ld[0], Rd[0], p, cost)
            X, Xc, _ = gc.solve_level2(cost, p, b, passes, bufs.o, bufs)
            C = cost.cpu().numpy().reshape(p.h, p.ng, p.D)
            ref = l2.level2(C, p.lam, p.inhibit, 1, b, passes)
            entry["parity_vs_oracle"] = {
                "pairs_checked": 1,
                "labels_equal": bool(np.array_equal(X.cpu().numpy(), ref["labels"])),
                "coarse_labels_equal": bool(np.array_equal(Xc.cpu().numpy(), ref["coarse_labels"]))}
        out["block_sizes"][str(b)] = entry
    return out


def _prepass(gc, dev, p, o, Ld, Rd, flush, stream):
    """Max-flow time with and without the chain-local initial flow (the
    build's stand-in for the paper's wave-front pre-pass), same pairs."""
    import torch
    buf = gc.Buffers(p, o, device=dev)
    out = {}
    for name, flags in (("with_chain_prepass", gc.GS_BUILD_CHAIN_PREFLOW), ("without", 0)):
        ms, flows = [], []
        for rep_ in range(3):
            for k in range(len(Ld)):
                gc.gs_stereo_cost_volume(Ld[k], Rd[k], p, buf.cost)
                gc.gs_build_graph_flags(buf.cost, p, flags, buf.graph, buf.status)
                flush.fill_(k & 0xff)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
                c.record(stream)
                gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
                c.synchronize()
                if int(buf.status.item()) != gc.GS_OK:
                    raise RuntimeError("solve status")
                if rep_:
                    ms.append(a.elapsed_time(c))
                    flows.append(int(buf.flow.item()))
        out[name] = {"maxflow_ms": float(np.mean(ms)), "flows": flows[:len(Ld)]}
    out["same_flows"] = out["with_chain_prepass"]["flows"] == out["without"]["flows"]
    return out


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
    from paper_1803_01516_gb300 import autotune
    o = autotune.tuned_opts(p)               # tile shape and schedule for this size bucket
    if args.sweeps_per_relabel:
        o.sweeps_per_relabel = args.sweeps_per_relabel
    if args.local_iters:
        o.local_iters = args.local_iters
    if args.relabel_passes:
        o.relabel_passes = args.relabel_passes
    # each rank solves its own pairs (replicas)
    pairs = [synth.make_pair(wl, i) for i in replica_pairs(rank)]
    Ld = [torch.from_numpy(L).to(dev) for L, _, _ in pairs]
    Rd = [torch.from_numpy(R).to(dev) for _, R, _ in pairs]
    buf = gc.Buffers(p, o, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def step(i, evs=None):
        """One pair: cost volume + graph build | max-flow solve | label extraction."""
        k = i % N_PAIRS
        if evs:
            evs[0].record(stream)
        gc.gs_stereo_cost_volume(Ld[k], Rd[k], p, buf.cost)
        gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
        if evs:
            evs[1].record(stream)
        gc.gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status)
        if evs:
            evs[2].record(stream)
        gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
        if evs:
            evs[3].record(stream)

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
    evs = [[ev() for _ in range(4)] for _ in range(args.steps)]
    launches0 = gc.gs_kernel_launches()
    stats = []
    bad_status = 0
    for i in range(args.steps):
        flush.fill_(i & 0xff)                       # L2 flush, outside the timed events
        step(i, evs[i])
        stats.append(gc.gs_solve_stats(buf.work))   # synchronises, after the last event
        bad_status |= int(buf.status.item()) != gc.GS_OK
    torch.cuda.synchronize(dev)
    launches = gc.gs_kernel_launches() - launches0
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    solve_ms = [e[1].elapsed_time(e[2]) for e in evs]
    extract_ms = [e[2].elapsed_time(e[3]) for e in evs]
    my_ms = float(sum(step_ms))
    clk = clocks.stop() if rank == 0 else None
    if bad_status:
        raise RuntimeError("a timed solve did not end with GS_OK")
    tot_ms = _reduce_max(my_ms, dist, dev)
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
            a, b = ev(), ev()
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

    # ----- roofline of the dominant kernel (the persistent solve) -----
    peak, peak_kind = _peaks()
    l2_peak = _l2_copy_gbs(dev)
    nodes = gc.gs_num_nodes(p)
    ti = gc.gs_tile_info(p, o)
    nodes_per_tile = nodes / ti["tiles"]
    sweep_visits = float(np.mean([s["sweep_visits"] for s in stats]))
    relabel_visits = float(np.mean([s["relabel_visits"] for s in stats]))
    alg_bytes = (BYTES_PER_NODE_SWEEP * sweep_visits + BYTES_PER_NODE_BFS * relabel_visits) \
        * nodes_per_tile
    solve_s = float(np.mean(solve_ms)) * 1e-3
    achieved = alg_bytes / solve_s / 1e9
    # per phase, over the device time the solver spent in each (its own clock)
    sweep_ns = float(np.mean([s["sweep_ns"] for s in stats]))
    relabel_ns = float(np.mean([s["relabel_ns"] for s in stats]))
    per_phase = {
        "sweep_rounds": {"achieved": BYTES_PER_NODE_SWEEP * sweep_visits * nodes_per_tile
                         / max(sweep_ns, 1.0), "ms": sweep_ns * 1e-6},
        "relabel_passes": {"achieved": BYTES_PER_NODE_BFS * relabel_visits * nodes_per_tile
                           / max(relabel_ns, 1.0), "ms": relabel_ns * 1e-6}}
    for v in per_phase.values():
        v["frac_l2"] = v["achieved"] / l2_peak
        v["frac_hbm"] = v["achieved"] / peak

    # ----- CPU oracle on the same pairs: baseline time and parity of the timed pairs -----
    cpu = None
    parity = None
    if not args.no_cpu_baseline and world == 1:
        cpu, refs = _cpu_baseline(wl, pairs)
        ok_flow = ok_lab = True
        for k, ref in enumerate(refs):
            step(k)
            torch.cuda.synchronize(dev)
            ok_flow &= int(buf.flow.item()) == ref["flow"]
            ok_lab &= bool(np.array_equal(buf.labels.cpu().numpy(), ref["labels"]))
        parity = {"pairs": len(refs), "flow_equal": ok_flow, "labels_equal": ok_lab}

    level1 = level2 = prepass = None
    if not args.no_batched and world == 1:
        exact_flows = []
        for k in range(len(Ld)):
            step(k)
            torch.cuda.synchronize(dev)
            exact_flows.append(int(buf.flow.item()))
        level1 = _level1(gc, dev, p, Ld, Rd, exact_flows, flush, stream,
                         not args.no_cpu_baseline)
        level2 = _level2(gc, dev, p, Ld, Rd, exact_flows, flush, stream,
                         not args.no_cpu_baseline)
        prepass = _prepass(gc, dev, p, o, Ld, Rd, flush, stream)
    fixed = rgb = None
    if not args.no_batched and world == 1:
        fixed = _fixed_sweeps(gc, dev, p, o, Ld, Rd, exact_flows, flush, stream)
        rgb = _rgb(gc, dev, flush, stream, not args.no_cpu_baseline)
    batched = None if args.no_batched or world > 1 else _batched(gc, dev, args, stream, flush)
    diff = None if args.no_batched or world > 1 else _differentiated(gc, dev, args, stream)
    large = None
    if not args.no_large and world == 1:
        large = _large(gc, dev, flush, stream, peak)
    learning = None
    if not args.no_learning and world == 1:
        learning = _learning(gc, dev, args)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": _config(wl, {"sweeps_per_relabel": o.sweeps_per_relabel,
                               "local_iters": o.local_iters, "relabel_passes": o.relabel_passes,
                               "replicas": world, "tile": [ti["tile_w"], ti["tile_h"]],
                               "direction": "auto"}),
        "e2e": e2e,
        # the 55 MB state of this workload stays in L2 (DRAM traffic per launch is a
        # small fraction of the state, profiles/): L2 is the binding ceiling; the HBM
        # copy peak is reported beside it
        "roofline": {"bound": "l2", "kernel": "k_batch (max-flow)", "achieved": achieved,
                     "peak": l2_peak, "unit": "GB/s", "frac": achieved / l2_peak,
                     "traffic": _profiled_traffic(),
                     "peak_kind": "measured in this run: L2-resident elementwise stream "
                                  "through the SMs (int32 add, 2 x 32 MiB), best of 5 x 200",
                     "hbm": {"peak": peak, "frac": achieved / peak,
                             "peak_kind": f"{peak_kind} HBM copy (MEASURED_PEAKS.json)"},
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": solve_s * 1e3,
                     "accounting": "72 B/node per tile visit of a sweep round + 40 B/node per "
                                   "tile visit of a relabel pass",
                     "per_phase": per_phase},
        "phases_ms": {"cost_volume+build": float(np.mean(build_ms)),
                      "maxflow_solve": float(np.mean(solve_ms)),
                      "extract_labels": float(np.mean(extract_ms))},
        "cpu_baseline": cpu,
        "parity_vs_oracle": parity,
        "batched": batched,
        "differentiated": diff,
        "level1_approximation": level1,
        "level2_approximation": level2,
        "fixed_sweeps": fixed,
        "rgb_data_term": rgb,
        "large": large,
        "learning": learning,
        "initial_flow_prepass": prepass,
        "clocks": clk,
        "gpu_launches": int(launches),
        "solver": {k: float(np.mean([s[k] for s in stats])) for k in
                   ("relabels", "sweeps", "bfs_passes", "label_passes", "sweep_visits",
                    "relabel_visits")},
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
    ap.add_argument("--sweeps-per-relabel", type=int, default=0, help="0: autotuned")
    ap.add_argument("--local-iters", type=int, default=0, help="0: autotuned")
    ap.add_argument("--relabel-passes", type=int, default=0, help="0: autotuned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--diff-pairs", type=int, default=16)
    ap.add_argument("--no-large", action="store_true", help="skip the 1920x1080x128 solve")
    ap.add_argument("--no-learning", action="store_true", help="skip the learning run")
    ap.add_argument("--learn-steps", type=int, default=200)
    ap.add_argument("--learn-lr", type=float, default=0.1)
    ap.add_argument("--no-batched-cpu-baseline", action="store_true",
                    help="skip the CPU oracle on two batch pairs (about 20 s)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
