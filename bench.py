"""Benchmark: GaBP edge-message updates/s and time to a 1e-10 relative residual.

Workload: random sparse symmetric diagonally dominant system, Erdos-Renyi
pattern with n = 1,000,000 and average degree 8, off-diagonals N(0,1),
A_ii = 1.1 sum_j |A_ij|, b ~ N(0,1) (synthetic, seeded).

One step = one complete solve to ||b - A x||_inf / ||b||_inf < 1e-10 with the
mixed-precision path (FP32 messages, FP64 residual refinement), inputs
already resident in HBM.  L2 is flushed (a 256 MiB write) before every step,
outside the timed events.  The plain FP64 sweep solve of the same system is
timed the same way for the comparison the metric asks for.

value   = directed edges x sweeps / solve time (edge-message updates/s),
          summed over ranks, divided by the slowest rank's time.
e2e     = the same metric through gabp_solve_host (host b and x, the copies
          inside the timed call), timed with the host clock.
roofline: the kernel with the largest device time inside the timed region,
          its algorithmic bytes per launch over its mean event-timed
          duration, against the measured HBM copy bandwidth.

Multi-GPU (torchrun): every rank solves its own system (same matrix, its own
right-hand side); no data moves between ranks ("replicas", weak scaling).

--impl reference times the CPU oracle (plain FP64 synchronous GaBP) on the
host cores, on a bounded number of rounds of the same system per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_NODES = 1_000_000
AVG_DEGREE = 8
DOMINANCE = 1.1
SCHEDULES = {0: "synchronous (Alg. 2)", 1: "colour-serial (Section III-C)"}
TOL = 1e-10
METRIC = "GaBP edge-message updates/s (mixed FP32+FP64 refinement solve to 1e-10 rel. residual)"
UNIT = "edge-updates/s"
WORKLOAD = "ER n=1e6 avg-degree 8 SDD (dominance 1.1), b~N(0,1), solve to 1e-10 rel. residual"

# Algorithmic bytes per launch of each kernel kind: values and indices the
# method must move (per directed edge, per node).
BYTES = {
    "mean": (16, 12),      # c 4 + eta in 4 + rev 4 + eta out 4 | rhs 4 + 1/P 4 + d out 4
    "full32": (24, 16),    # A 4 + (P,eta) in 8 + rev 4 + (P,eta) out 8 | diag 4 + rhs 4 + (P,d) out 8
    # in-place form: A 4 + col 4 + (P,eta) in 8 + out 8 | diag 4 + rhs 4 + totals in 8 + out 8
    # + monitors in 8 + out 8 (the gathered totals of the senders, an L2-resident n-entry
    # table, are not counted)
    "full32_inplace": (24, 40),
    "full64": (44, 24),    # A 8 + (P,eta) in 16 + rev 4 + (P,eta) out 16 | diag 8 + b 8 + x out 8
    "residual": (20, 32),  # A 8 + col 4 + x[col] 8 | diag 8 + x 8 + b 8 + r 8
}
# The grid form (per-direction planes) has no reverse index to read.
BYTES_GRID = {
    "mean": (12, 12),      # c 4 + eta in 4 + eta out 4 | rhs 4 + 1/P 4 + d out 4
    "full64": (40, 24),    # A 8 + (P,eta) in 16 + (P,eta) out 16 | diag 8 + b 8 + x out 8
}


# DRAM traffic of the dominant kernels from ncu captures (dram__bytes_read.sum
# + dram__bytes_write.sum per launch; ncu flushes caches between replays, so
# these are cold-cache figures), valid only for the kernel sources they were
# taken on: a changed source makes the figure null.
TRAFFIC = {
    "mean": {"sources": ("gabp_kernels.cu", "gabp_device.cuh"), "sha": "b04585fc006c2b3e",
             "bytes_per_launch": 171.9e6},
    "mean_win": {"sources": ("gabp_window.cu", "gabp_device.cuh"), "sha": "b584bc04817140ca",
                 "bytes_per_launch": 121.1e6},
    "full32_inplace": {"sources": ("gabp_kernels.cu", "gabp_device.cuh"), "sha": "fe67705660b1de65",
                       "bytes_per_launch": 203.5e6},
    "dense_mean": {"sources": ("gabp_dense.cu", "gabp_device.cuh"), "sha": "60dde3d85b4a733b",
                   "bytes_per_pair": 23.14},
    "dense_mean_serial": {"sources": ("gabp_dense.cu", "gabp_device.cuh"), "sha": "60dde3d85b4a733b",
                          "bytes_per_pair": 15.16},
}


def _traffic(kind, units=None):
    import hashlib
    t = TRAFFIC.get(kind)
    if t is None:
        return None
    d = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_0810_1119_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    if d.hexdigest()[:16] != t["sha"]:
        return None
    if "bytes_per_launch" in t:
        return t["bytes_per_launch"]
    return t["bytes_per_pair"] * units


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _workload(seed_rhs: int):
    from paper_0810_1119_gb300 import workloads as W
    m = W.er_sdd(N_NODES, AVG_DEGREE, DOMINANCE, 0)
    b = W.normal_rhs(m.n, 1 + seed_rhs)
    return m, b


def _scatter_floor_us(m, dev, reps=20):
    """Device time of one torch index_copy_ that stores the E off-diagonal
    four-byte values through the workload's reverse-edge permutation: the
    random scatter a mean sweep makes, with nothing else (warm L2, int64
    indices).  A reference for the mean sweep's floor, outside the timed
    region; not the library's code."""
    import torch
    from paper_0810_1119_gb300 import workloads as W
    rev = W.reverse_index(m)
    r = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    idx = torch.tensor(rev[m.col != r], dtype=torch.int64, device=dev)
    src = torch.rand(idx.numel(), device=dev)
    dst = torch.zeros(m.nnz, device=dev)
    for _ in range(3):
        dst.index_copy_(0, idx, src)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        dst.index_copy_(0, idx, src)
    z.record()
    torch.cuda.synchronize()
    return 1e3 * a.elapsed_time(z) / reps


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _cpu_baseline(m, b, rounds: int):
    """The oracle on the host cores: edge-updates/s over `rounds` fixed rounds
    on all cores and over 2 rounds on one core, and the time to the 1e-10
    relative residual on all cores (measured; on one core estimated from its
    time per round, labelled as such)."""
    import oracle
    E = m.n_directed_edges
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    r = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED, max_rounds=rounds)
    dt = time.perf_counter() - t0
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED, max_rounds=2)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    t0 = time.perf_counter()
    rs = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=5000, tol=TOL)
    dts = time.perf_counter() - t0
    return {"value": E * r["rounds"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{r['rounds']} synchronous FP64 rounds (Alg. 2) of the n=1e6 ER system, "
                      f"{dt:.2f} s",
            "single_thread": {"value": E * 2 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"2 rounds, {dt1:.2f} s"},
            "time_to_1e-10_s": {"all_cores": dts, "rounds": rs["rounds"], "status": rs["status"],
                                "single_thread_estimate": dt1 / 2 * rs["rounds"],
                                "note": "all cores measured (a full oracle solve with its residual "
                                        "check every round); one core = its time per round x rounds"}}


def _emit(line, args):
    """Print a workload's JSON line, or hand it back when the default run
    collects it into its `configs` entry."""
    if getattr(args, "collect", False):
        return line
    print(json.dumps(line), flush=True)
    return 0


def reduce_over_ranks(dist, times, counts, device):
    """Whole-job figures of a replicated run: the slowest rank's times (MAX)
    and the units of work of all ranks (SUM).  Works with any process group
    (NCCL with CUDA tensors, gloo with CPU tensors)."""
    import torch
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(list(counts), dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()], [float(v) for v in c.cpu()]


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    m, b = _workload(0)
    E = m.n_directed_edges
    rounds = args.ref_rounds
    for _ in range(args.warmup):
        _cpu_baseline(m, b, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        import oracle
        oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_FIXED, max_rounds=rounds)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = E * rounds * args.steps / tot
    import oracle
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"{rounds} FP64 oracle rounds on host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{rounds} synchronous FP64 rounds per step, n=1e6 ER"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _collect_configs(args):
    """The other configurations of the workload list, each run the way its
    own --workload run does it with 1-3 timed steps, and each with its error
    against the oracle or the closed form: 2D Poisson 32x32 (FP64, absolute
    1e-10), 64 right-hand sides on ER n=2e6, the 4096-system detection batch
    (colour-serial, damping 0.2 on the z -> x^ messages), and 3D Poisson 256^3
    in the grid form (red-black, mixed precision, with and without Aitken's
    Delta^2 on the inner solves).  Clocks are sampled over all of them."""
    import copy
    import torch
    base = copy.copy(args)
    base.collect = True
    base.warmup = 1
    jobs = (
        ("poisson32", run_poisson32, {"steps": 3}),
        ("multi64", run_multi, {"steps": 1, "n": 2_000_000, "oracle_check": True}),
        ("detect", run_detect, {"steps": 2, "schedule": 1, "damp_scope": 1, "damping": 0.2,
                                "psi_zero": False, "lsq_form": 0, "nsys": 4096}),
        ("poisson3d_256_grid", run_poisson3d, {"steps": 1, "p": 256, "form": "grid", "schedule": 1,
                                               "only": ("mixed_fp32", "mixed_fp32_aitken"), "oracle_residual": True,
                                               "max_iter": 400000}),
    )
    out = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for name, fn, kw in jobs:
        a = copy.copy(base)
        for k, v in kw.items():
            setattr(a, k, v)
        t0 = time.perf_counter()
        try:
            line = fn(a)
            line.pop("tuning", None)
            for r in line.get("runs", {}).values():
                r.pop("tuning", None)
            out[name] = line
        except Exception as e:   # a failing configuration must not drop the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    out["clocks"] = sampler.stop()
    return out


def run_gabp(args):
    import torch
    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp

    m, b = _workload(rank)
    E = m.n_directed_edges
    bt = torch.tensor(b, device=dev)
    xt = torch.empty_like(bt)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    # Timed solves run the graph driver (one CUDA graph launch per solve).
    # A second handle with profile=1 runs the same kernels from the host
    # driver with CUDA events around every kernel: it gives the per-kernel
    # device times of the roofline figure.
    # Launch shapes are picked by the library's autotuner at create time
    # (outside the timed region); the profiled pass reuses the same handle.
    mixed = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=gabp.PREC_MIXED_FP32,
                                 autotune=True, schedule=args.schedule, pull_lanes=args.pull_lanes,
                                 mean_window=args.mean_window)
    fp64 = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=gabp.PREC_FP64, autotune=True,
                                schedule=args.schedule)
    stream = torch.cuda.current_stream()

    def timed_solves(solver, steps):
        evs = []
        stats = []
        for _ in range(steps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            it = gabp.gabp_solve(solver.handle, bt, xt, TOL, 5000)
            z.record(stream)
            evs.append((a, z))
            st = solver.stats()
            st["iters"] = it
            stats.append(st)
        torch.cuda.synchronize()
        return [a.elapsed_time(z) for a, z in evs], stats

    for _ in range(args.warmup):
        timed_solves(mixed, 1)
        timed_solves(fp64, 1)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier()
    ms_mixed, st_mixed = timed_solves(mixed, args.steps)
    barrier()
    ms_fp64, st_fp64 = timed_solves(fp64, max(1, min(args.steps, args.fp64_steps)))
    barrier()
    clocks = sampler.stop() if sampler else None
    gabp.gabp_set_profile(mixed.handle, True)
    _, st_prof = timed_solves(mixed, args.steps)
    gabp.gabp_set_profile(mixed.handle, False)

    # end to end through the host-buffer entry point
    b_host = torch.tensor(b, dtype=torch.float64).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    bh, xh = b_host.numpy(), x_host.numpy()
    gabp.gabp_solve_host(mixed.handle, bh, TOL, 5000, x=xh)
    barrier()
    e2e_t, e2e_sweeps = [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it = gabp.gabp_solve_host(mixed.handle, bh, TOL, 5000, x=xh)
        e2e_t.append(time.perf_counter() - t0)
        e2e_sweeps.append(it)
    barrier()

    tot_ms = sum(ms_mixed)
    updates = sum(E * s["iters"] for s in st_mixed)
    launches = sum(s["kernel_launches"] for s in st_mixed)
    e2e_updates = sum(E * it for it in e2e_sweeps)
    e2e_s = sum(e2e_t)
    if dist is not None:
        (tot_ms, e2e_s), (updates, e2e_updates, launches) = reduce_over_ranks(
            dist, [tot_ms, e2e_s], [updates, e2e_updates, launches], dev)
        launches = int(launches)

    if rank == 0:
        hbm, peak_kind = _peaks()
        # roofline of the dominant kernel kind inside the timed mixed solves
        kinds = {
            "mean": (sum(s["ms_mean"] for s in st_prof), sum(s["sweeps_mean"] for s in st_prof)),
            "full32": (sum(s["ms_full"] for s in st_prof), sum(s["sweeps_full"] for s in st_prof)),
            "residual": (sum(s["ms_residual"] for s in st_prof),
                         sum(s["residual_checks"] for s in st_prof)),
        }
        dom = max(kinds, key=lambda k: kinds[k][0])
        ms_k, n_k = kinds[dom]
        lanes = mixed.tuning()["pull_lanes"]   # FP32 full sweep: 0 = scatter form
        per_edge, per_node = BYTES["full32_inplace" if dom == "full32" and lanes > 0 else dom]
        bytes_launch = per_edge * E + per_node * m.n
        achieved = bytes_launch * n_k / (ms_k * 1e-3) / 1e9 if ms_k > 0 else None
        kernel_names = {"mean": "mean_kernel<float> (FP32 mean-only sweep)",
                        "full32": "sweep32_kernel (FP32 full sweep)",
                        "residual": "residual64_kernel (FP64 residual)"}
        fp64_ms = statistics.mean(ms_fp64)
        mixed_ms = tot_ms / args.steps
        scatter_us = _scatter_floor_us(m, dev)
        # the FP32 full sweep in the form the autotuner kept
        fe, fn = BYTES["full32_inplace" if lanes > 0 else "full32"]
        ms_f, n_f = kinds["full32"]
        full_sweep = {"form": f"in place, {lanes} lanes per row" if lanes > 0 else "scatter",
                      "us_per_launch": 1e3 * ms_f / max(n_f, 1),
                      "bytes_per_launch": fe * E + fn * m.n,
                      "traffic": _traffic("full32_inplace") if lanes > 0 else None,
                      "hbm_frac": ((fe * E + fn * m.n) * n_f / (ms_f * 1e-3) / 1e9 / hbm) if ms_f > 0 else None}
        if lanes > 0:
            kernel_names["full32"] = "pull32_kernel (FP32 full sweep, in place)"
        mwin = mixed.tuning()["mean_window"]
        if mwin > 0:
            kernel_names["mean"] = (f"mean_win_kernel<float> (FP32 mean-only sweep, window form, "
                                    f"{mixed.tuning()['windows']} windows of about {mwin} slots)")
        line = {
            "metric": METRIC, "value": updates / (tot_ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": m.n, "directed_edges": E, "schedule": SCHEDULES[args.schedule],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed (256 MiB write) before every step",
                       "precision": "FP32 messages, FP64 residual refinement"},
            "time_to_solution_ms": {"mixed_fp32": mixed_ms, "fp64_sweep": fp64_ms,
                                    "speedup_vs_fp64": fp64_ms / mixed_ms},
            "sweeps": {"mixed_total": st_mixed[-1]["sweeps_total"],
                       "mixed_full": st_mixed[-1]["sweeps_full"],
                       "mixed_mean": st_mixed[-1]["sweeps_mean"],
                       "mixed_outer": st_mixed[-1]["outer_steps"],
                       "fp64": st_fp64[-1]["sweeps_total"]},
            "fp64_edge_updates_per_s": E * st_fp64[-1]["sweeps_total"] / (fp64_ms * 1e-3),
            "final_rel_residual": st_mixed[-1]["residual"] / st_mixed[-1]["rhs_norm"],
            "roofline": {"bound": "hbm", "kernel": kernel_names[dom],
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None,
                         "peak_source": peak_kind,
                         "traffic": _traffic("mean_win" if (dom == "mean" and mwin > 0) else dom),
                         "bytes_per_launch": bytes_launch, "launches": n_k,
                         "mean_launch_us": 1e3 * ms_k / max(n_k, 1),
                         "random_scatter_us": scatter_us,
                         "timing": "CUDA events around every kernel in a profiled pass "
                                   "of the same solves (host driver)"},
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kinds.items()},
            "full_sweep": full_sweep,
            "e2e": {"value": e2e_updates / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * m.n, "d2h_bytes_per_step": 8 * m.n,
                    "ms_per_step": 1e3 * e2e_s / args.steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "tuning": {"mixed": mixed.tuning(), "fp64": fp64.tuning()},
        }
        if not args.no_cpu_baseline:
            # the mixed solution against the oracle's FP64 solution to 1e-13
            import oracle
            ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_REL, max_rounds=5000,
                              tol=1e-13)
            xg = xt.cpu().numpy()
            line["max_rel_err_vs_oracle"] = float(np.abs(xg - ref["x"]).max() / np.abs(ref["x"]).max())
            line["oracle_reference"] = {"rounds": ref["rounds"], "status": ref["status"],
                                        "stop": "relative residual 1e-13"}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(m, b, args.cpu_rounds)
        if world == 1 and not args.no_configs:
            line["configs"] = _collect_configs(args)
        print(json.dumps(line), flush=True)
    mixed.close()
    fp64.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_multi(args):
    """Multi right-hand-side workload: ER n=2e6, average degree 10, dominance
    1.05, 64 columns b ~ N(0,1) (row-major n x 64).  One step = one
    gabp_solve_multi (precisions once, then all 64 columns together, FP64
    refinement per column) to 1e-10 relative residual in every column."""
    import torch
    torch.cuda.set_device(0)
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    from paper_0810_1119_gb300 import workloads as W
    n, K = args.n, 64
    m = W.er_sdd(n, 10, 1.05, 0)
    E = m.n_directed_edges
    B = torch.tensor(W.normal_rhs(n, 5, k=K), device="cuda")
    X = torch.empty_like(B)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    s = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=gabp.PREC_MIXED_FP32, autotune=True,
                             schedule=args.schedule)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        gabp.gabp_solve_multi(s.handle, B, X, TOL, 5000)
    ms, st = [], None
    for _ in range(args.steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gabp.gabp_solve_multi(s.handle, B, X, TOL, 5000)
        z.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(z))
        st = s.stats()
    t = statistics.mean(ms)
    updates = E * st["sweeps_full"] + E * K * st["sweeps_mean"]
    # profiled pass of the same handle: per-kind kernel times
    gabp.gabp_set_profile(s.handle, True)
    gabp.gabp_solve_multi(s.handle, B, X, TOL, 5000)
    sp = s.stats()
    gabp.gabp_set_profile(s.handle, False)
    hbm, peak_src = _peaks()
    # K-column mean sweep: eta in 4 K + eta out 4 K per edge, c and rev once
    # (8 B), per row the K-column rhs, d in and d out (12 K B)
    bytes_meanK = (8 * K + 8) * E + 12 * K * n
    meanK_us = 1e3 * sp["ms_mean"] / max(1, sp["sweeps_mean"])
    roof = {"bound": "hbm", "kernel": "mean_multi_kernel (K-column mean-only sweep)",
            "achieved": bytes_meanK / (meanK_us * 1e-6) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_meanK / (meanK_us * 1e-6) / 1e9 / hbm, "peak_source": peak_src,
            "traffic": None, "bytes_per_launch": bytes_meanK, "mean_launch_us": meanK_us,
            "timing": "CUDA events around every kernel in a profiled pass of the same solve (host driver)"}
    # FP64 comparison: the 64 columns solved one after another by FP64 sweeps
    s64 = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=gabp.PREC_FP64, schedule=args.schedule)
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    gabp.gabp_solve_multi(s64.handle, B, X, TOL, 5000)
    z.record(stream)
    torch.cuda.synchronize()
    t64 = a.elapsed_time(z)
    err_col0 = None
    if getattr(args, "oracle_check", False):
        # column 0 of the mixed solve against the oracle's FP64 solution to 1e-13
        import oracle
        gabp.gabp_solve_multi(s.handle, B, X, TOL, 5000)
        x0 = X[:, 0].cpu().numpy()
        ref = oracle.gabp(m.row_ptr, m.col, m.val, B[:, 0].cpu().numpy(), stop=oracle.STOP_RES_REL,
                          max_rounds=5000, tol=1e-13)
        err_col0 = float(np.abs(x0 - ref["x"]).max() / np.abs(ref["x"]).max())
    line = {"metric": "GaBP edge x RHS message updates/s (64 right-hand sides, mixed FP32 + FP64 refinement to 1e-10)",
            "value": updates / (t * 1e-3), "unit": "edge-rhs-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"multi-RHS: ER n={n:.0e} avg-degree 10 SDD (dominance 1.05), 64 RHS b~N(0,1), 1e-10 rel. residual per column",
                       "n": n, "directed_edges": E, "nrhs": K, "schedule": SCHEDULES[args.schedule]},
            "sweeps": {"precision": st["sweeps_full"], "mean_K_columns": st["sweeps_mean"],
                       "outer": st["outer_steps"]},
            "time_to_solution_ms": {"mixed_multi": t, "fp64_column_by_column": t64,
                                    "speedup_vs_fp64": t64 / t},
            "algorithmic_bytes_per_mean_sweep": bytes_meanK, "roofline": roof,
            "max_rel_err_vs_oracle_column0": err_col0,
            "kernel_ms_per_step": {"mean_K": sp["ms_mean"], "precision": sp["ms_full"],
                                   "residual": sp["ms_residual"], "other": sp["ms_other"]},
            "tuning": s.tuning()}
    s.close()
    s64.close()
    return _emit(line, args)


def run_poisson32(args):
    """2D Poisson 5-point Laplacian on a 32 x 32 grid (n = 1024, 3968 directed
    edges), b ~ U[-1, 1]; plain synchronous FP64 GaBP until ||A x - b||_inf <
    1e-10 (absolute).  The system is ~100 KB, so the solve is latency-bound
    (thousands of short sweeps): reported as time to solution and sweeps/s,
    with the mixed-precision solve of the same system and the oracle's
    solve on the host cores beside it."""
    import torch
    import oracle
    torch.cuda.set_device(0)
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    from paper_0810_1119_gb300 import workloads as W
    m = W.poisson2d(32)
    b = W.uniform_rhs(m.n, 0)
    E = m.n_directed_edges
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec, ait in (("fp64", gabp.PREC_FP64, 0), ("fp64_aitken2", gabp.PREC_FP64, 2),
                            ("mixed_fp32", gabp.PREC_MIXED_FP32, 0)):
        s = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=prec,
                                 residual_kind=gabp.RESIDUAL_ABS, autotune=True, aitken=ait,
                                 schedule=args.schedule)
        for _ in range(args.warmup):
            gabp.gabp_solve(s.handle, bt, xt, TOL, 100000)
        ms = []
        for _ in range(args.steps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gabp.gabp_solve(s.handle, bt, xt, TOL, 100000)
            z.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(z))
        st = s.stats()
        out[name] = {"ms": statistics.mean(ms), "stats": st, "x": xt.cpu().numpy(),
                     "tuning": s.tuning()}
        s.close()
    t0 = time.perf_counter()
    ref = oracle.gabp(m.row_ptr, m.col, m.val, b, stop=oracle.STOP_RES_ABS, max_rounds=100000, tol=TOL)
    cpu_s = time.perf_counter() - t0
    f = out["fp64"]
    st = f["stats"]
    line = {"metric": "time to ||Ax-b||_inf < 1e-10, plain FP64 GaBP (2D Poisson 32x32)",
            "value": f["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f["ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "2D Poisson 5-point 32x32 (n=1024), b~U[-1,1], abs 1e-10",
                       "schedule": SCHEDULES[args.schedule],
                       "n": m.n, "directed_edges": E, "bound": "latency (system fits in L2)"},
            "sweeps": st["sweeps_total"], "residual_checks": st["residual_checks"],
            "sweeps_per_s": st["sweeps_total"] / (f["ms"] * 1e-3),
            "edge_updates_per_s": E * st["sweeps_total"] / (f["ms"] * 1e-3),
            "us_per_sweep": 1e3 * f["ms"] / st["sweeps_total"],
            "final_abs_residual": st["residual"],
            "max_rel_err_vs_oracle": float(np.abs(f["x"] - ref["x"]).max() / np.abs(ref["x"]).max()),
            "mixed_fp32": {"ms": out["mixed_fp32"]["ms"],
                           "sweeps": out["mixed_fp32"]["stats"]["sweeps_total"],
                           "outer": out["mixed_fp32"]["stats"]["outer_steps"]},
            "fp64_aitken2": {"ms": out["fp64_aitken2"]["ms"],
                             "sweeps": out["fp64_aitken2"]["stats"]["sweeps_total"],
                             "max_rel_err_vs_oracle": float(np.abs(out["fp64_aitken2"]["x"] - ref["x"]).max()
                                                            / np.abs(ref["x"]).max()),
                             "note": "Aitken's Delta^2 on the means of rounds t-4, t-2, t (Section IV-A)"},
            "tuning": f["tuning"],
            "cpu_baseline": {"value": 1e3 * cpu_s, "unit": "ms", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"the full solve ({ref['rounds']} rounds)"}}
    return _emit(line, args)


def run_poisson3d(args):
    """3D Poisson 7-point Laplacian on a p^3 grid (p = 256: n = 16.8M, 100M
    directed edges), b ~ U[-1, 1]; FP32 messages (and the BF16 mean-storage
    variant) inside FP64 refinement to 1e-10 relative residual, beside the
    plain FP64 sweep, and the mixed FP32 solve with Aitken's Delta^2 on the
    means of every inner solve; the line's value is the faster of the two
    mixed FP32 solves that meets 1e-10.  Convergence takes O(p^2) sweeps (~1e5 at p = 256), so
    with --max-iter below that the run reports the measured per-sweep times
    and the residual reached, and extrapolates the time to 1e-10 from the
    observed FP64 residual contraction (labelled as such)."""
    import torch
    torch.cuda.set_device(0)
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    from paper_0810_1119_gb300 import workloads as W
    p = args.p
    t0 = time.perf_counter()
    m = W.poisson3d(p)
    b = W.uniform_rhs(m.n, 0)
    gen_s = time.perf_counter() - t0
    E = m.n_directed_edges
    bt = torch.tensor(b, device="cuda")
    xt = torch.empty_like(bt)
    stream = torch.cuda.current_stream()
    hbm, peak_src = _peaks()
    res = {}
    only = getattr(args, "only", None)
    # mixed_fp32_aitken: Aitken's Delta^2 (Section IV-A) on the means of
    # every inner solve, spacing chosen by the library
    for name, prec, ait in (("mixed_fp32", gabp.PREC_MIXED_FP32, 0),
                            ("mixed_fp32_aitken", gabp.PREC_MIXED_FP32, 2),
                            ("mixed_bf16", gabp.PREC_MIXED_BF16, 0), ("fp64", gabp.PREC_FP64, 0)):
        if only and name not in only:
            continue
        t0 = time.perf_counter()
        if args.form == "grid":
            s = gabp.Solver.from_grid([p, p, p], m.row_ptr, m.col, m.val, precision=prec,
                                      schedule=args.schedule, aitken=ait)
        else:
            s = gabp.Solver.from_csr(m.row_ptr, m.col, m.val, precision=prec, autotune=True,
                                     schedule=args.schedule, aitken=ait)
        build_s = time.perf_counter() - t0
        ms, st, err = [], None, ""
        cap = args.fp64_max_iter if (prec == gabp.PREC_FP64 and args.fp64_max_iter) else args.max_iter
        if prec == gabp.PREC_MIXED_BF16 and args.skip_bf16:
            s.close()
            continue
        for step in range(max(1, args.steps)):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            try:
                gabp.gabp_solve(s.handle, bt, xt, TOL, cap)
            except gabp.GabpError as e:
                err = e.name
            z.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(z))
            st = s.stats()
        r = {"ms": statistics.mean(ms), "status": err or "GABP_OK", "sweeps": st["sweeps_total"],
             "sweeps_full": st["sweeps_full"], "sweeps_mean": st["sweeps_mean"],
             "sweeps_mean_fp32_after_ladder": st["sweeps_wide"], "aitken_steps": st["aitken_steps"],
             "outer": st["outer_steps"], "rel_residual": st["residual"] / st["rhs_norm"],
             "handle_build_s": build_s, "tuning": s.tuning()}
        if getattr(args, "oracle_residual", False):
            # the reached x checked by the oracle's own residual routine (the
            # oracle cannot iterate this system to convergence in bench time)
            import oracle
            xr = xt.cpu().numpy()
            r["rel_residual_by_oracle"] = (oracle.residual_inf(m.row_ptr, m.col, m.val, b, xr)
                                           / float(np.abs(b).max()))
        # per-kernel times from a profiled pass capped at a few hundred sweeps
        gabp.gabp_set_profile(s.handle, True)
        try:
            gabp.gabp_solve(s.handle, bt, xt, TOL, min(args.max_iter, 300))
        except gabp.GabpError:
            pass
        sp = s.stats()
        gabp.gabp_set_profile(s.handle, False)
        if prec == gabp.PREC_FP64:
            per = 1e3 * sp["ms_full"] / max(1, sp["sweeps_full"])
            r["us_per_full_sweep"] = per
            bm = BYTES_GRID if args.form == "grid" else BYTES
            r["full_sweep_frac"] = (bm["full64"][0] * E + bm["full64"][1] * m.n) / (per * 1e-6) / 1e9 / hbm
        else:
            if sp["sweeps_mean"]:
                per = 1e3 * sp["ms_mean"] / sp["sweeps_mean"]
                eb = 14 if prec == gabp.PREC_MIXED_BF16 else 16   # BF16: eta in/out 2 + 2
                if args.form == "grid":
                    eb -= 4                                        # no reverse index
                r["us_per_mean_sweep"] = per
                r["mean_sweep_frac"] = (eb * E + BYTES["mean"][1] * m.n) / (per * 1e-6) / 1e9 / hbm
            if sp["sweeps_full"]:
                r["us_per_full_sweep"] = 1e3 * sp["ms_full"] / sp["sweeps_full"]
        res[name] = r
        s.close()
    f64 = res.get("fp64")
    ait = res.get("mixed_fp32_aitken")
    mixed = res.get("mixed_fp32") or ait or res.get("mixed_bf16") or f64
    best = ait if (ait is not None and ait["status"] == "GABP_OK" and ait["ms"] < mixed["ms"]) else mixed
    extrap = None
    if f64 is not None and f64["status"] != "GABP_OK" and mixed["status"] == "GABP_OK":
        # FP64 capped: its time to 1e-10 estimated from its measured time per
        # sweep and the FP64 / mixed sweep-count ratio measured at p = 64 and
        # 128 (0.77, 0.79)
        need = 0.79 * mixed["sweeps"]
        extrap = {"fp64_sweeps_to_1e-10_estimate": need,
                  "fp64_ms_estimate": need * f64["ms"] / f64["sweeps"],
                  "basis": "FP64 time per sweep measured over the capped run x (0.79 x the mixed "
                           "solve's sweeps, the FP64/mixed ratio measured at p = 64 and 128)"}
    line = {"metric": f"time to 1e-10 relative residual, 3D Poisson {p}^3 (mixed FP32 + FP64 refinement"
                      + (", Aitken on the inner solves)" if best is ait else ")"),
            "value": best["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": 0,
            "ms_per_step": best["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3D Poisson 7-point {p}^3, b~U[-1,1], 1e-10 rel. residual",
                       "schedule": SCHEDULES[args.schedule],
                       "form": "grid (per-direction planes, no index arrays)" if args.form == "grid" else "CSR tiles",
                       "n": m.n, "directed_edges": E, "max_iter": args.max_iter,
                       "generate_s": gen_s},
            "runs": res, "extrapolation": extrap,
            "edge_updates_per_s_mixed": E * mixed["sweeps"] / (mixed["ms"] * 1e-3)}
    return _emit(line, args)


def run_detect(args):
    """Batched uneven linear detection: 4096 systems, K ~ U{16..256}, N = 2K,
    S = +-1/sqrt(N), x in {+-1}, y = S x + noise at 10 dB.  Every system is
    solved through its Section VII augmented form in one batched handle (one
    CUDA graph per solve, one persistent launch per sweep over all systems);
    one step = one gabp_solve_lsq_batched to 1e-10 relative residual per
    augmented system.  Reports the MMSE solution's agreement with the
    closed form on a sample of systems.  With --psi-zero every system asks
    for the Moore-Penrose solution S^+ y (Psi = 0, the zero-forcing
    detector): one step is then the whole iteration to
    ||S^T (y - S x^)|| <= 1e-10 ||S^T y|| per system, checked against a
    least-squares solve on the sample.

    Per-system control (--batch-control 0, the default): each system leaves
    the sweeps when it meets its own rule, so the value counts the edge
    updates the solve actually made (2 x grid positions swept).  The same
    batch under one controller for the whole batch (batch_control 1) is
    timed beside it, and its profiled pass, where every launch sweeps every
    system, gives the kernel roofline."""
    import torch
    torch.cuda.set_device(0)
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    from paper_0810_1119_gb300 import workloads as W
    nsys = args.nsys
    systems = W.detection_batch(nsys, 16, 256, 10.0, seed=0)
    o = gabp.gabp_default_options()
    o.precision = gabp.PREC_MIXED_FP32
    o.damping = args.damping
    o.lsq_form = args.lsq_form
    o.schedule = args.schedule
    o.damp_scope = args.damp_scope
    o.autotune = 1
    o.pinv_shift = args.pinv_shift
    o.stream = gabp.current_stream_handle()
    psi = [0.0 if args.psi_zero else d.sigma2 for d in systems]
    max_iter = 2_000_000 if args.psi_zero else 20000
    y = torch.tensor(np.concatenate([d.y for d in systems]), device="cuda")
    xh = torch.empty(sum(d.K for d in systems), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(batch_control, steps, warmup):
        o.batch_control = batch_control
        t0 = time.perf_counter()
        hh = gabp.gabp_create_lsq_batched([d.S for d in systems], psi, o)
        bs = time.perf_counter() - t0
        for _ in range(warmup):
            gabp.gabp_solve_lsq_batched(hh, y, xh, TOL, max_iter)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gabp.gabp_solve_lsq_batched(hh, y, xh, TOL, max_iter)
            z.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(z))
        return hh, statistics.mean(ms), bs

    h, t, build_s = timed(args.batch_control, args.steps, args.warmup)
    st = gabp.gabp_get_stats(h)
    sys_sweeps = gabp.gabp_get_system_sweeps(h, nsys)
    E = st["edges"]
    got = xh.cpu().numpy()
    offs = np.cumsum([0] + [d.K for d in systems])
    errs = []
    for k in range(0, nsys, max(1, nsys // 32)):
        if args.psi_zero:
            closed = np.linalg.lstsq(systems[k].S, systems[k].y, rcond=None)[0]
        else:
            A, bb = systems[k].dense_system()
            closed = np.linalg.solve(A, bb)
        errs.append(float(np.abs(got[offs[k]:offs[k + 1]] - closed).max() / np.abs(closed).max()))
    tuning = gabp.gabp_get_tuning(h)
    gabp.gabp_destroy(h)
    # the same batch under one controller (every system sweeps until the last
    # one is done); its profiled pass (host driver, CUDA events around every
    # kernel) gives per-kind kernel times with every launch over every system
    h1, t1, _ = timed(1, max(1, min(args.steps, 3)), 1)
    st1 = gabp.gabp_get_stats(h1)
    gabp.gabp_set_profile(h1, True)
    sp = None
    for _ in range(2):   # events around host-driven launches absorb host delays: keep the faster pass
        gabp.gabp_solve_lsq_batched(h1, y, xh, TOL, max_iter)
        s2 = gabp.gabp_get_stats(h1)
        if sp is None or s2["ms_mean"] < sp["ms_mean"]:
            sp = s2
    gabp.gabp_destroy(h1)
    hbm, peak_src = _peaks()
    pairs = E // 2
    dense = args.lsq_form == 0
    serial = args.schedule == 1
    # dense form, per grid position (two directed edges), synchronous: mean sweep
    # c 8 + eta in 8 + eta out 8; full sweep S 4 + messages in 16 + out 16.
    # Serial: only the z -> x^ messages are read and written (mean c 8 + 4 + 4,
    # full S 4 + 8 + 8); damping on every message adds the x^ -> z ones (mean 8,
    # full 16).  Per node ~ 24 B.
    if dense and serial:
        damped = args.damping > 0 and args.damp_scope == 0
        per_mean, per_full = (24, 36) if damped else (16, 20)
    else:
        per_mean, per_full = (24, 36) if dense else (16, 24)
    bytes_mean = (per_mean * pairs if dense else per_mean * E) + 24 * st["n"]
    bytes_full = (per_full * pairs if dense else per_full * E) + 24 * st["n"]
    mean_us = 1e3 * sp["ms_mean"] / max(1, sp["sweeps_mean"])
    full_us = 1e3 * sp["ms_full"] / max(1, sp["sweeps_full"])
    kname = ("dense_mean_serial_kernel" if serial else "dense_mean_kernel") if dense else "mean_kernel"
    roof = {"bound": "hbm", "kernel": kname + " (mean-only sweep)",
            "achieved": bytes_mean / (mean_us * 1e-6) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_mean / (mean_us * 1e-6) / 1e9 / hbm, "peak_source": peak_src,
            "traffic": _traffic("dense_mean_serial" if serial else "dense_mean", pairs) if dense else None,
            "bytes_per_launch": bytes_mean, "mean_launch_us": mean_us,
            "full_sweep_us": full_us,
            "full_sweep_frac": bytes_full / (full_us * 1e-6) / 1e9 / hbm,
            "timing": "CUDA events around every kernel in a profiled pass of the solve under one "
                      "controller for the whole batch (every launch sweeps every system; host driver)"}
    what = ("batched zero-forcing detection, Section VII with Psi = 0 (S^+ y), normal equations to 1e-10"
            if args.psi_zero else "batched detection, Section VII augmented systems, to 1e-10")
    line = {"metric": f"GaBP edge-message updates/s ({what})",
            "value": 2 * st["positions_swept"] / (t * 1e-3), "unit": "edge-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched detection: {nsys} systems, K~U{{16..256}}, N=2K, 10 dB, augmented form",
                       "augmented_rows": st["n"], "directed_edges": E, "systems": nsys,
                       "damping": args.damping, "schedule": SCHEDULES[args.schedule],
                       "damp_scope": "z -> x^ messages only" if args.damp_scope else "every message"},
            "sweeps": {"full": st["sweeps_full"], "mean": st["sweeps_mean"], "outer": st["outer_steps"]},
            "batch_control": "per system" if args.batch_control == 0 else "whole batch",
            "grid_positions_swept_per_solve": st["positions_swept"],
            "system_sweeps": {"min": int(sys_sweeps.min()), "median": float(np.median(sys_sweeps)),
                              "max": int(sys_sweeps.max()), "solve": st["sweeps_total"]},
            "whole_batch_control": {"time_to_solution_ms": t1, "sweeps": st1["sweeps_total"],
                                    "grid_positions_swept_per_solve": st1["positions_swept"],
                                    "edge_updates_per_s": 2 * st1["positions_swept"] / (t1 * 1e-3)},
            "psi": "0 for every system (Moore-Penrose)" if args.psi_zero else "sigma^2 = 0.1 (MMSE)",
            "time_to_solution_ms": t, "handle_build_s": build_s,
            "form": "dense bipartite grid" if dense else "CSR tiles",
            ("max_rel_err_vs_lstsq_sample" if args.psi_zero else "max_rel_err_vs_closed_form_sample"): max(errs),
            "roofline": roof,
            "kernel_ms_per_step": {"mean": sp["ms_mean"], "full32": sp["ms_full"],
                                   "residual": sp["ms_residual"], "other": sp["ms_other"]},
            "tuning": tuning}
    return _emit(line, args)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gabp", choices=["gabp", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-rounds", type=int, default=10)
    ap.add_argument("--ref-rounds", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="er1e6: leave out the other configurations (configs entry of the line)")
    ap.add_argument("--p", type=int, default=128, help="poisson3d: grid side")
    ap.add_argument("--max-iter", type=int, default=200000, help="poisson3d: sweep cap per solve")
    ap.add_argument("--fp64-max-iter", type=int, default=0,
                    help="poisson3d: separate sweep cap for the FP64 comparison (0 = --max-iter)")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1],
                    help="all workloads: 0 synchronous (Alg. 2), 1 colour-serial (Section III-C)")
    ap.add_argument("--form", default="grid", choices=["csr", "grid"],
                    help="poisson3d: the grid form (gabp_create_grid, default) or the general CSR handle")
    ap.add_argument("--n", type=int, default=2_000_000, help="multi64: unknowns (smaller for profiling)")
    ap.add_argument("--damp-scope", type=int, default=0, choices=[0, 1],
                    help="detect with --schedule 1: 0 damp every message, 1 only those the last class sends")
    ap.add_argument("--skip-bf16", action="store_true", help="poisson3d: leave out the BF16 variant")
    ap.add_argument("--runs", default="",
                    help="poisson3d: comma list of the solves to run (mixed_fp32, mixed_fp32_aitken, mixed_bf16, fp64); "
                         "default all")
    ap.add_argument("--pull-lanes", type=int, default=0, choices=[-1, 0, 2, 4, 8, 16, 32],
                    help="er1e6: form of the FP32 full sweep: 0 = autotuned, -1 = scatter, "
                         "2..32 = in place with that many lanes per row")
    ap.add_argument("--mean-window", type=int, default=0,
                    help="er1e6: form of the mean sweep: 0 = autotuned, -1 = tiles, "
                         "256..65536 = windows of about that many slots")
    ap.add_argument("--workload", default="er1e6",
                    choices=["er1e6", "multi64", "detect", "poisson32", "poisson3d"],
                    help="er1e6: the headline line; multi64 / detect / poisson32 / poisson3d: extra lines")
    ap.add_argument("--nsys", type=int, default=4096)
    ap.add_argument("--batch-control", type=int, default=0, choices=[0, 1],
                    help="detect: 0 = per-system control (systems leave when done), 1 = whole batch")
    ap.add_argument("--lsq-form", type=int, default=0, choices=[0, 1],
                    help="detect: 0 = dense bipartite kernels, 1 = general CSR path")
    ap.add_argument("--psi-zero", action="store_true",
                    help="detect: Psi = 0 for every system, i.e. the Moore-Penrose solution S^+ y")
    ap.add_argument("--pinv-shift", type=float, default=0.0,
                    help="detect --psi-zero: Psi_0 relative to the mean squared column norm (0 = 0.1)")
    ap.add_argument("--damping", type=float, default=0.3,
                    help="detect workload: message damping (plain GaBP diverges on some systems)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "multi64":
        return run_multi(args)
    if args.workload == "detect":
        return run_detect(args)
    if args.workload == "poisson32":
        return run_poisson32(args)
    if args.workload == "poisson3d":
        if args.runs:
            args.only = tuple(r.strip() for r in args.runs.split(",") if r.strip())
        return run_poisson3d(args)
    return run_gabp(args)


if __name__ == "__main__":
    sys.exit(main())
