#!/usr/bin/env python
"""Benchmark: exact w(theta) pair counts (DD + DR + RR) on one GB300.

A step is one whole w(theta): DD, DR and RR of the survey-scale workload
(1M clustered + 1M uniform points in a 60 deg polar cap, 32 log bins
0.5'-20 deg), with the catalogues resident in HBM.  The metric is algorithmic
pair evaluations per second: (n(n-1)/2 + n n_r + n_r(n_r-1)/2) / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload survey|small|largest]

Under torchrun (N > 1) the survey w(theta) is sharded: every rank holds both
whole catalogues, counts the pairs whose first point lies in its share of the
tile rows (wtheta_count_wtheta_shard: rows split by kept tile pairs, so equal
work), and one NCCL all-reduce of the 3 (K+2) counts combines them inside the
timed step (strong scaling: the total work is fixed); the step time is the
maximum over ranks.  --replicas runs N independent w(theta) instead (weak
scaling, no collective).  --impl reference times the CPU oracle instead, on a
bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-evals/s for w(θ) 1M×1M (exact counts); batched p50/p99 latency vs plain"
UNIT = "pair-evals/s"
FP32_OPS_PER_PAIR = 6       # 3 FADD + 1 FMUL + 2 FFMA per squared chord
FP32_LANES_PER_SM = 128
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_pairs_survey.md")
KERNEL_SOURCE = os.path.join(ROOT, "paper_1208_3658_gb300", "csrc", "wtheta_count.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["survey", "small", "largest", "batch", "serve",
                                           "jackknife"],
                    default="survey")
    ap.add_argument("--requests", type=int, default=2000, help="serve workload: requests")
    ap.add_argument("--load", type=float, default=0.7,
                    help="serve workload: offered load as a fraction of plain throughput")
    ap.add_argument("--mocks", type=int, default=256, help="batch workload: number of mocks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", default="",
                    help="threads,points_per_thread,hist_mode of the pair kernel (default: library's)")
    ap.add_argument("--no-skip-far", action="store_true",
                    help="evaluate every tile pair (no bounding-cap skipping): brute force")
    ap.add_argument("--separate-counts", action="store_true",
                    help="count DD, DR and RR with three wtheta_count calls (each catalogue "
                         "prepared per call) instead of one wtheta_count_wtheta call")
    ap.add_argument("--no-span-bins", action="store_true",
                    help="bin every evaluated pair through the table (no per-chunk settling)")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent replicas of the workload (weak scaling) instead "
                         "of one w(theta) sharded over the ranks")
    ap.add_argument("--bins", type=int, default=0,
                    help="number of log bins over the workload's range (default: the "
                         "workload's own; e.g. 256 for the large-K span path)")
    ap.add_argument("--n", type=int, default=0,
                    help="points per catalogue (same shape, smaller: profiling cases)")
    return ap.parse_args()


def make_workload(name, seed, n=0, bins=0):
    from paper_1208_3658_gb300 import synth
    if bins:
        wl, desc = make_workload(name, seed, n)
        wl.n_bins = bins
        return wl, desc.replace("%d log bins" % {"small": 16, "survey": 32, "largest": 64}.get(
            name, 0), "%d log bins" % bins) + (" (%d log bins)" % bins if n else "")
    if n:
        wl = {"small": synth.small, "survey": synth.survey, "largest": synth.largest}[name](
            seed=seed, n=n)
        return wl, "%s-shaped, %d + %d points" % (name, wl.n_d, wl.n_r)
    if name == "small":
        wl = synth.small(seed=seed)
        desc = ("small: 10k clustered (200 centres, sigma 3') + 10k uniform, 10x10 deg patch, "
                "16 log bins 1'-5 deg")
    elif name == "largest":
        wl = synth.largest(seed=seed)
        desc = ("largest: 10M clustered (200k centres, sigma 1') + 10M uniform full sky, "
                "64 log bins 0.2'-30 deg")
    else:
        wl = synth.survey(seed=seed)
        desc = ("survey: 1M clustered (20k centres, Poisson(50), sigma 2') + 1M uniform in a "
                "60 deg polar cap, 32 log bins 0.5'-20 deg")
    return wl, desc


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200", "-f", self.path]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                    power.append(float(f[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_median": statistics.median(power), "samples": len(sm),
                "reasons": sorted(reasons)}


def shared_atomic_roofline(W, sm_count, clk_mhz, st, pairs, tile):
    """The histogram's roofline: measured shared reductions per SM per clock
    (own word per thread, as the kernel's private columns; and one word for
    all, the worst case), against the reductions the step issued at most: one
    per pair binned through the table plus three per settled chunk and thread."""
    private = W.wtheta_probe_shared_atomics(False)
    same = W.wtheta_probe_shared_atomics(True)
    binned = max(0.0, float(st[W.STAT_TILES]) * tile * tile - float(st[W.STAT_SPAN]))
    reductions = binned + 3.0 * float(st[W.STAT_SPAN]) / 256.0   # thread-level
    per_pair = reductions / max(1.0, float(pairs))
    peak_lanes = sm_count * 32.0 * private * clk_mhz * 1e6      # thread reductions / s
    return {"warp_reductions_per_sm_clock": {"own_word": private, "one_word": same},
            "reductions_per_algorithmic_pair": per_pair,
            "peak_algorithmic_pairs_per_s": peak_lanes / max(per_pair, 1e-30),
            "note": "upper bound on the reductions: pairs of the kept tile pairs minus the "
                    "pairs settled by span, plus 3 per settled chunk and thread"}


def kernel_code_sha():
    """Hash of the device code of the pair kernel's source file: the text from
    the namespace opening to the host launch code (so host-only edits keep a
    measurement valid, any kernel edit voids it)."""
    t = open(KERNEL_SOURCE, "rb").read()
    start = t.index(b"namespace wtheta {")
    return hashlib.sha256(t[start:t.index(b"// launch plumbing")]).hexdigest()[:16]


def kernel_traffic():
    """DRAM bytes per launch of the pair kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    src = kernel_code_sha()
    m_sha = re.search(r"kernel_code_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != src:
        return None
    return float(m_tr.group(1))


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline only)
# ---------------------------------------------------------------------------
def oracle_sample_rate(wl, e, target_s=15.0):
    """Times the oracle's cross count on a sample of data rows against all
    randoms, sized to take about target_s seconds.  Returns a dict."""
    import numpy as np
    from oracle import oracle as O
    D = O.radec_to_xyz(wl.data)
    R = O.radec_to_xyz(wl.rand)
    cores = O.num_threads()
    m = max(64, min(wl.n_d, 4 * cores))
    t0 = time.perf_counter()
    O.count_xyz(np.ascontiguousarray(D[:, :m]), R, e, False)
    dt = time.perf_counter() - t0
    rate = m * wl.n_r / max(dt, 1e-6)
    m2 = int(min(wl.n_d, max(m, rate * target_s / wl.n_r)))
    rows = np.ascontiguousarray(D[:, :m2])
    t0 = time.perf_counter()
    O.count_xyz(rows, R, e, False)
    dt = time.perf_counter() - t0
    pairs = m2 * wl.n_r
    return {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "DR: %d data rows x %d randoms (%.3g pairs, %.1f s)" % (m2, wl.n_r, pairs, dt)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    sharded = world > 1 and not args.replicas and not args.separate_counts
    wl, desc = make_workload(args.workload, seed=1 if sharded else 1 + rank, n=args.n,
                             bins=args.bins)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    K = wl.n_bins
    d_data = torch.from_numpy(wl.data).to(dev)
    d_rand = torch.from_numpy(wl.rand).to(dev)
    counts = torch.zeros((3, K + 2), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (126 MB)
    pairs = wl.pairs

    tune = None
    if args.tune:
        t = [int(x) for x in args.tune.split(",")]
        tune = dict(threads=t[0], points_per_thread=t[1], hist_mode=t[2])
    if args.no_skip_far:
        tune = dict(tune or {}, skip_far=2)
    if args.no_span_bins:
        tune = dict(tune or {}, span_bins=2)

    n_calls = 3 if args.separate_counts else 1

    def step(evs=None, stats=None):
        if sharded:
            # this rank's tile rows of every count, then one all-reduce of the
            # 3 (K+2) counts over NCCL
            if evs is not None:
                evs[0][0].record(stream)
            W.wtheta_count_wtheta_shard(d_data, d_rand, False, e, rank, world, counts, tune=tune,
                                        stats=stats, stream=stream)
            dist.all_reduce(counts, op=dist.ReduceOp.SUM)
            if evs is not None:
                evs[0][1].record(stream)
            return
        if not args.separate_counts:
            # one w(theta): both catalogues prepared once, DD, DR, RR in one launch
            if evs is not None:
                evs[0][0].record(stream)
            W.wtheta_count_wtheta(d_data, d_rand, False, e, counts, tune=tune, stats=stats,
                                  stream=stream)
            if evs is not None:
                evs[0][1].record(stream)
            return
        calls = [(d_data, None, True), (d_data, d_rand, False), (d_rand, None, True)]
        for q, (a, b, auto) in enumerate(calls):
            if evs is not None:
                evs[q][0].record(stream)
            if tune is None and stats is None:
                W.wtheta_count(a, b, e, auto, counts[q], stream=stream)
            else:
                W.wtheta_count_ex(a, b, False, e, auto, counts[q], tune=tune, stats=stats,
                                  stream=stream)
            if evs is not None:
                evs[q][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    gpu_id = None
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        gpu_id = u if u.startswith("GPU-") else "GPU-" + u
    sampler = ClockSampler(gpu_id if world == 1 else None)
    sampler.start()
    step_evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)]
                 for _ in range(n_calls)] for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = W.wtheta_kernel_launches()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict the catalogues from L2 between steps (not timed)
        step(step_evs[k])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = W.wtheta_kernel_launches() - launches0
    clocks = sampler.stop()

    call_ms = [[step_evs[k][q][0].elapsed_time(step_evs[k][q][1]) for q in range(n_calls)]
               for k in range(args.steps)]
    step_ms = [sum(c) for c in call_ms]
    ms = sum(step_ms) / args.steps
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = (1 if sharded else world) * pairs / (ms / 1e3)

    # exactness checks on the benchmark's own output (cheap, exact integers)
    c = counts.cpu().numpy().astype(np.uint64)
    nd, nr = wl.n_d, wl.n_r
    totals_ok = (int(c[0].sum()) == nd * (nd - 1) // 2 and int(c[1].sum()) == nd * nr
                 and int(c[2].sum()) == nr * (nr - 1) // 2)

    # statistics of one untimed step: binned and rechecked fractions
    stats = torch.zeros(W.NSTATS, dtype=torch.int64, device=dev)
    step(stats=stats)
    torch.cuda.synchronize()
    st = stats.cpu().numpy()

    # roofline of the pair kernel: FP32 pipe, 6 FP32 instructions per pair
    sm_count = props.multi_processor_count
    clk = clocks.get("sm_mhz") or 2070.0
    clk_max = clocks.get("sm_max_mhz") or 2070.0
    peak = sm_count * FP32_LANES_PER_SM * clk * 1e6 / FP32_OPS_PER_PAIR
    peak_max = sm_count * FP32_LANES_PER_SM * clk_max * 1e6 / FP32_OPS_PER_PAIR
    per_launch_ms = [c for row in call_ms for c in row]
    # the roofline counts the pairs the kernel evaluates (tile padding included,
    # tile pairs skipped by their bounding caps excluded); value counts the
    # algorithmic pairs of the w(theta)
    evaluated = float(st[W.STAT_PAIRS])
    achieved = (evaluated * args.steps) / (sum(per_launch_ms) / 1e3)
    traffic = kernel_traffic()
    roofline = {
        "bound": "alu",
        "achieved": achieved / 1e9,
        "peak": peak / 1e9,
        "unit": "Gpair/s",
        "frac": achieved / peak,
        "traffic": traffic,
        "peak_basis": ("FP32 pipe: %d SMs x %d lanes x %.0f MHz (median sampled under load) / "
                       "%d FP32 instructions per pair; achieved counts evaluated pairs "
                       "(%.3g per step of %.3g algorithmic)" % (
                           sm_count, FP32_LANES_PER_SM, clk, FP32_OPS_PER_PAIR, evaluated,
                           float(pairs))),
        "frac_at_max_clock": achieved / peak_max,
        "shared_atomic": shared_atomic_roofline(
            W, sm_count, clk, st, pairs,
            (lambda t: t[0] * t[1])([int(x) for x in args.tune.split(",")]) if args.tune
            else 1024),
        "kernel_ms_per_launch": ({"DD": statistics.mean(r[0] for r in call_ms),
                                  "DR": statistics.mean(r[1] for r in call_ms),
                                  "RR": statistics.mean(r[2] for r in call_ms)}
                                 if args.separate_counts else
                                 {"DD+DR+RR": statistics.mean(r[0] for r in call_ms)}),
    }

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n_data": nd, "n_rand": nr, "n_bins": K,
                   "tune": args.tune or "library default",
                   "skip_far_tile_pairs": not args.no_skip_far,
                   "span_bins": not args.no_span_bins,
                   "api": ("three wtheta_count calls" if args.separate_counts else
                           "wtheta_count_wtheta (DD, DR, RR in one launch)"),
                   "pairs_per_step": pairs, "l2": "flushed between steps (512 MB write)",
                   "inputs": "resident in HBM (FP64 RA/Dec), converted inside each call",
                   "parallelism": ("dp%d: tile rows sharded by kept tile pairs, NCCL all-reduce "
                                   "of the counts" % world if sharded else
                                   "replicas" if world > 1 else "single GPU")},
        "roofline": roofline,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "counts_total_exact": bool(totals_ok),
        "evaluated_pair_evals_per_s": (1 if sharded else world) * evaluated / (ms / 1e3),
        "stats": {"in_range_frac": float(sum(int(x[:-1].sum()) for x in c)) / pairs,
                  "recheck_frac": float(st[W.STAT_RECHECK]) / max(1, float(pairs)),
                  "evaluated_over_algorithmic": float(st[W.STAT_PAIRS]) / pairs,
                  "tile_pairs_evaluated": int(st[W.STAT_TILES]),
                  "tile_pairs_skipped": int(st[W.STAT_SKIPPED]),
                  "evaluated_pairs": int(evaluated),
                  "span_settled_pairs": int(st[W.STAT_SPAN])},
        "wall_s_timed_region": t_wall,
    }

    # end to end through the host-buffer C-ABI call (H2D + count + D2H + LS)
    if args.no_e2e:
        return out
    h_data = torch.from_numpy(wl.data).pin_memory()
    h_rand = torch.from_numpy(wl.rand).pin_memory()

    def e2e_step():
        if not sharded:
            W.wtheta_correlate(h_data.numpy(), h_rand.numpy(), e, stream=stream)
            return
        # each rank: pinned host catalogues in, its shard, the all-reduce, counts
        # out, Eq. 2 on the host
        dd = h_data.to(dev, non_blocking=True)
        dr = h_rand.to(dev, non_blocking=True)
        W.wtheta_count_wtheta_shard(dd, dr, False, e, rank, world, counts, stream=stream)
        dist.all_reduce(counts, op=dist.ReduceOp.SUM)
        hc = counts.cpu().numpy().astype(np.uint64)
        W.wtheta_ls(hc[0], hc[1], hc[2], nd, nr)

    e2e_step()
    e2e_t = []
    for _ in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t)
    if dist is not None:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    out["e2e"] = {"value": (1 if sharded else world) * pairs / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": (nd + nr) * 16, "d2h_bytes_per_step": 3 * (K + 2) * 8,
                  "api": ("per rank: pinned host RA/Dec in, wtheta_count_wtheta_shard, NCCL "
                          "all-reduce, counts out, wtheta_ls" if sharded else
                          "wtheta_correlate (pinned host RA/Dec in, counts + w out)"),
                  "skip_far_tile_pairs": True}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample_rate(wl, e)
    return out


def run_batch(args, rank, world, dist):
    """256 mocks (sizes log-uniform in [20k, 400k], 2x randoms, own 15 deg
    patches, 16 log bins 1'-5 deg): every DD, DR, RR in one graph replay of
    one persistent launch; compared with the same counts as serial
    one-count-per-launch calls."""
    import numpy as np
    import torch

    from paper_1208_3658_gb300 import build, synth
    build.build()
    from paper_1208_3658_gb300 import wtheta as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    t0 = time.perf_counter()
    mocks, (lo, hi, K) = synth.batch_mocks(seed=1 + rank, n_mocks=args.mocks)
    gen_s = time.perf_counter() - t0
    e = W.wtheta_edges(lo, hi, K)
    cats = [(torch.from_numpy(m.data).to(dev), torch.from_numpy(m.rand).to(dev)) for m in mocks]
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    plan = W.wtheta_batch_plan(cats, e, stream=stream)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    info = W.wtheta_batch_info(plan)
    counts = torch.zeros((len(cats), 3, K + 2), dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        W.wtheta_batch_run(plan, counts, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = W.wtheta_kernel_launches()
    for k in range(args.steps):
        evs[k][0].record(stream)
        W.wtheta_batch_run(plan, counts, stream=stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = W.wtheta_kernel_launches() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    pairs = info["pairs"]
    evaluated = W.wtheta_batch_info(plan)["evaluated_pairs"]   # computed by the last run
    # the same counts, one count per launch, serially
    plain = torch.zeros_like(counts)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for m, (d, r) in enumerate(cats):
        W.wtheta_count(d, None, e, True, plain[m, 0], stream=stream)
        W.wtheta_count(d, r, e, False, plain[m, 1], stream=stream)
        W.wtheta_count(r, None, e, True, plain[m, 2], stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    same = bool(torch.equal(plain, counts))
    sm_count = props.multi_processor_count
    clk = clocks.get("sm_mhz") or 2070.0
    peak = sm_count * FP32_LANES_PER_SM * clk * 1e6 / FP32_OPS_PER_PAIR
    achieved = evaluated / (ms / 1e3)
    return {
        "metric": METRIC, "value": world * pairs / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch: %d mocks, n log-uniform in [20k, 400k], 2x randoms, own "
                               "15x15 deg patches, 16 log bins 1'-5 deg" % len(cats),
                   "pairs_per_step": pairs, "items": info["n_items"], "tune": info["tune"],
                   "autotuned": info["autotuned"], "autotune_ms": info["autotune_ms"],
                   "graph_kernels": info["graph_kernels"],
                   "l2": "inputs (~1.6 GB FP32 copies) larger than L2"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                     "unit": "Gpair/s", "frac": achieved / peak, "traffic": None,
                     "note": "achieved counts the pairs whose squared chord the run computed "
                             "(%.3g of %.3g algorithmic; far tile pairs and settled chunks "
                             "skipped)" % (evaluated, pairs)},
        "batched_vs_plain": {"batched_ms": ms, "plain_ms": plain_ms,
                             "speedup": plain_ms / ms, "counts_identical": same},
        "gpu_launches": int(launches), "clocks": clocks,
        "host_s": {"generate": gen_s, "plan_incl_autotune": plan_s},
    }


def run_jackknife(args, rank, world, dist):
    """The survey workload split into 64 jackknife regions (8 RA sectors x 8
    Dec rings of the 60 deg cap): DD, DR and RR of every region pair in one
    launch, then the jackknife covariance of w(theta) on the host; against the
    plain w(theta) (three counts) on the same catalogues."""
    import numpy as np
    import torch

    from paper_1208_3658_gb300 import build, synth
    build.build()
    from paper_1208_3658_gb300 import wtheta as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.survey(seed=1 + rank, n=args.n or 1_000_000)
    R = 64
    ld = synth.grid_labels(wl.data, 0.0, 360.0, 30.0, 90.0, 8, 8)
    lr = synth.grid_labels(wl.rand, 0.0, 360.0, 30.0, 90.0, 8, 8)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    K = wl.n_bins
    d, r = torch.from_numpy(wl.data).to(dev), torch.from_numpy(wl.rand).to(dev)
    dl, rl = torch.from_numpy(ld).to(dev), torch.from_numpy(lr).to(dev)
    counts = torch.zeros((3, R, R, K + 2), dtype=torch.int64, device=dev)
    plain = torch.zeros((3, K + 2), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def jk():
        return W.wtheta_count_regions(d, dl, r, rl, e, R, counts, stream=stream)

    def pl():
        W.wtheta_count(d, None, e, True, plain[0], stream=stream)
        W.wtheta_count(d, r, e, False, plain[1], stream=stream)
        W.wtheta_count(r, None, e, True, plain[2], stream=stream)

    for _ in range(args.warmup):
        jk()
        pl()
    torch.cuda.synchronize()
    sampler = ClockSampler()
    sampler.start()
    launches0 = W.wtheta_kernel_launches()
    t_jk = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sizes = jk()
        torch.cuda.synchronize()
        t_jk.append(time.perf_counter() - t0)
    launches = W.wtheta_kernel_launches() - launches0
    clocks = sampler.stop()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        pl()
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b) / args.steps
    c = counts.cpu().numpy().astype(np.uint64)
    p = plain.cpu().numpy().astype(np.uint64)
    sums_equal = all(np.array_equal(c[k].sum(axis=(0, 1), dtype=np.uint64), p[k]) for k in range(3))
    t0 = time.perf_counter()
    w, w_k, cov = W.wtheta_jackknife(c, sizes, R)
    host_s = time.perf_counter() - t0
    ms = 1e3 * sum(t_jk) / len(t_jk)
    pairs = wl.pairs
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return {
        "metric": METRIC, "value": world * pairs / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "jackknife: survey catalogues (%d + %d points) in 64 regions "
                               "(8 RA sectors x 8 Dec rings of the cap), region-pair DD/DR/RR "
                               "in one launch" % (wl.n_d, wl.n_r),
                   "pairs_per_step": pairs, "regions": R,
                   "timing": "wall clock of the call (it synchronises once for the region "
                             "sizes)"},
        "vs_plain_w": {"region_split_ms": ms, "plain_ms": plain_ms,
                       "overhead": ms / plain_ms, "sums_equal_plain_counts": bool(sums_equal),
                       "jackknife_host_ms": 1e3 * host_s},
        "w_and_sigma_sample": {"theta_bin": [1, K // 2, K],
                               "w": [float(w[0]), float(w[K // 2 - 1]), float(w[K - 1])],
                               "sigma_jk": [float(sig[0]), float(sig[K // 2 - 1]),
                                            float(sig[K - 1])]},
        "gpu_launches": int(launches), "clocks": clocks,
    }


def run_serve(args, rank, world, dist):
    """w(theta) requests with Poisson arrivals: sizes log-uniform in [1k, 2M]
    points with 1:1 randoms, 70% auto / 30% cross, 15x15 deg patches,
    24 log bins 1'-10 deg.  Request catalogues are random slices of
    pre-generated clustered and uniform pools, rotated in RA (a rotation about
    the pole keeps them equal-area and clustered).  Plain: one request at a
    time, each count one launch, FIFO; served: the continuous-batching server
    at the same arrival times.  Latency = done - arrival."""
    import math
    import threading

    import numpy as np
    import torch

    from paper_1208_3658_gb300 import build, synth
    build.build()
    from paper_1208_3658_gb300 import wtheta as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nmax = 2_000_000
    fp = synth.Patch(100.0, 15.0, 10.0, 25.0)
    pools = {
        "d": synth.clustered(fp, nmax, nmax // 50, 3.0, 1 + rank, "serve", "data"),
        "r": synth.uniform(fp, nmax, 1 + rank, "serve", "random"),
        "d2": synth.clustered(fp, nmax, nmax // 50, 3.0, 1 + rank, "serve", "data2"),
        "r2": synth.uniform(fp, nmax, 1 + rank, "serve", "random2"),
    }
    e = W.wtheta_edges(1.0 / 60.0, 10.0, 24)
    K = 24
    rng = synth.rng_for(1 + rank, "serve", "sizes")
    nreq = args.requests
    sizes = np.rint(np.exp(rng.uniform(math.log(1_000), math.log(nmax), nreq))).astype(np.int64)
    kinds = synth.rng_for(1 + rank, "serve", "kinds").random(nreq) < 0.7
    offs = rng.integers(0, 1 << 30, (nreq, 4))
    rot = rng.uniform(0.0, 360.0, nreq)

    def cut(pool, n, off, shift):
        a = pools[pool].reshape(-1, 2)
        start = int(off % (nmax - n + 1))
        out = a[start:start + n].copy()
        out[:, 0] = np.mod(out[:, 0] + shift, 360.0)
        return out.reshape(-1)

    def materialize(q):
        n = int(sizes[q])
        d = cut("d", n, offs[q, 0], rot[q])
        r = cut("r", n, offs[q, 1], rot[q])
        if kinds[q]:
            return d, r, None, None
        return d, r, cut("d2", n, offs[q, 2], rot[q]), cut("r2", n, offs[q, 3], rot[q])

    def pairs_of(q):
        n = int(sizes[q])
        return n * (n - 1) + n * n if kinds[q] else 4 * n * n

    # plain: each request alone (host -> device, one launch per count, counts back)
    stream = torch.cuda.current_stream(dev)
    service, plain_counts = [], []
    for q in range(nreq):
        d, r, d2, r2 = materialize(q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = [torch.from_numpy(x).pin_memory() if x is not None else None for x in (d, r, d2, r2)]
        ds = [x.to(dev, non_blocking=True) if x is not None else None for x in hs]
        if d2 is None:
            c = torch.zeros((3, K + 2), dtype=torch.int64, device=dev)
            W.wtheta_count(ds[0], None, e, True, c[0], stream=stream)
            W.wtheta_count(ds[0], ds[1], e, False, c[1], stream=stream)
            W.wtheta_count(ds[1], None, e, True, c[2], stream=stream)
        else:
            c = torch.zeros((4, K + 2), dtype=torch.int64, device=dev)
            for k, (a, b) in enumerate([(0, 2), (0, 3), (1, 2), (1, 3)]):
                W.wtheta_count(ds[a], ds[b], e, False, c[k], stream=stream)
        ch = c.cpu().numpy().astype(np.uint64)
        service.append(time.perf_counter() - t0)
        plain_counts.append(ch)
    total_pairs = sum(pairs_of(q) for q in range(nreq))
    plain_rate = total_pairs / sum(service)
    lam = args.load * plain_rate / (total_pairs / nreq)          # requests per second
    gaps = synth.rng_for(1 + rank, "serve", "arrivals").exponential(1.0 / lam, nreq)
    arrival = np.cumsum(gaps) - gaps[0]
    finish, lat_plain = 0.0, []
    for q in range(nreq):
        finish = max(arrival[q], finish) + service[q]
        lat_plain.append(finish - arrival[q])

    # served: submit at the arrival times from a client thread
    srv = W.wtheta_server_create(e, 120 << 30)
    mats = [None] * nreq
    ids = [None] * nreq
    submit_err = []

    def client():
        t0 = time.perf_counter()
        for q in range(nreq):
            m = materialize(q)
            dt = arrival[q] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            try:
                ids[q] = W.wtheta_server_submit(srv, *m)
            except Exception as ex:  # noqa: BLE001
                submit_err.append(repr(ex))
                return

    launches0 = W.wtheta_kernel_launches()
    sampler = ClockSampler()
    sampler.start()
    th = threading.Thread(target=client)
    t_start = time.perf_counter()
    th.start()
    th.join()
    lat_served, identical = [], True
    t_first, t_last = None, 0.0
    for q in range(nreq):
        done, c, w = W.wtheta_server_wait(srv, ids[q], timeout_ms=-1)
        info = W.wtheta_server_request_info(srv, ids[q])
        lat_served.append(info["t_done"] - info["t_submit"])
        t_first = info["t_submit"] if t_first is None else min(t_first, info["t_submit"])
        t_last = max(t_last, info["t_done"])
        identical &= bool(np.array_equal(c, plain_counts[q]))
        W.wtheta_server_release(srv, ids[q])
    wall = time.perf_counter() - t_start
    clocks = sampler.stop()
    st = W.wtheta_server_stats(srv)
    W.wtheta_server_destroy(srv)
    served_rate = total_pairs / (t_last - t_first)

    # saturated: every request submitted at once; makespan against the plain
    # service time of the same requests
    srv = W.wtheta_server_create(e, 120 << 30)
    mats = [materialize(q) for q in range(nreq)]   # host catalogues ready, as for plain
    t0 = time.perf_counter()
    sat_ids = [W.wtheta_server_submit(srv, *mats[q]) for q in range(nreq)]
    for i in sat_ids:
        W.wtheta_server_wait(srv, i, timeout_ms=-1)
    makespan = time.perf_counter() - t0
    W.wtheta_server_destroy(srv)

    def pct(x, p):
        return float(np.percentile(np.asarray(x), p))

    return {
        "metric": METRIC, "value": world * total_pairs / makespan, "unit": UNIT,
        "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": makespan * 1e3,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve: %d Poisson requests, n log-uniform in [1k, 2M], 1:1 "
                               "randoms, 70%% auto / 30%% cross, 15x15 deg patches, 24 log bins "
                               "1'-10 deg, 120 GB budget, offered load %.2f of plain throughput"
                               % (nreq, args.load),
                   "pairs": total_pairs, "arrival_rate_hz": lam},
        "latency_s": {"served_p50": pct(lat_served, 50), "served_p99": pct(lat_served, 99),
                      "plain_p50": pct(lat_plain, 50), "plain_p99": pct(lat_plain, 99)},
        "throughput": {"served_at_offered_load": served_rate,
                       "served_saturated": total_pairs / makespan,
                       "plain_saturated": plain_rate,
                       "saturated_speedup": (total_pairs / makespan) / plain_rate,
                       "note": "saturated: all requests submitted at once from ready host "
                               "arrays, makespan incl. the copies to pinned memory and the "
                               "device; "
                               "plain: sum of one-request-at-a-time service times"},
        "counts_identical_to_plain": identical, "submit_errors": submit_err[:3],
        "server": st, "gpu_launches": int(W.wtheta_kernel_launches() - launches0),
        "clocks": clocks, "wall_s": wall,
    }


def run_reference(args, rank, world):
    """The CPU oracle on the host cores, each step a bounded sample (data rows
    against all randoms) of the same workload."""
    from oracle import oracle as O
    wl, desc = make_workload(args.workload, seed=1, n=args.n, bins=args.bins)
    e = O.edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    cal = oracle_sample_rate(wl, e, target_s=4.0)
    import numpy as np
    D = O.radec_to_xyz(wl.data)
    R = O.radec_to_xyz(wl.rand)
    m = int(cal["sample"].split(":")[1].split("data rows")[0])
    rows = np.ascontiguousarray(D[:, :m])
    for _ in range(args.warmup):
        O.count_xyz(rows, R, e, False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.count_xyz(rows, R, e, False)
    dt = time.perf_counter() - t0
    pairs = m * wl.n_r * args.steps
    value = pairs / dt
    sample = "DR: %d data rows x %d randoms per step (%.3g pairs per step)" % (m, wl.n_r, m * wl.n_r)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "n_data": wl.n_d, "n_rand": wl.n_r,
                                        "n_bins": wl.n_bins},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, world)))
        return 0
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    if args.workload == "batch":
        out = run_batch(args, rank, world, dist)
    elif args.workload == "jackknife":
        out = run_jackknife(args, rank, world, dist)
    elif args.workload == "serve":
        out = run_serve(args, rank, world, dist)
    else:
        out = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
