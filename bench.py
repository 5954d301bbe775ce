#!/usr/bin/env python
"""Benchmark of the on-line SBD matvec (Gpts/s = N * nrhs / matvec time).

Default workload: Laplace kernel, N = 10^6 points uniform in arc length on 8
random star-shaped curves in [0, 10]^2, f ~ N(0, 1), eps = 1e-6, delta_min from
Theorem 1 (alpha = 0), FP32 form (FP64 near field and accumulation).  One step =
one sbd_matvec over the whole point set, inputs resident in HBM.  The grids
(~0.8 GB each) and D (~2.1 GB) exceed the 129 MB L2, so no flush is needed.

The default line also carries (N = 1 only, after the headline's timed region):
balanced_delta_min (delta_min by measurement), uniform_grid (the same workload with the
node step replaced by a multiplication on the frequency grid), near_fp32 (the same plan with D f in
float32), fp64_form (the same workload in the FP64 form), eps_sweep (the same points and f at
eps = 1e-3 and 1e-9, with the fit's Gram factorisation time), helmholtz (kappa delta_max
= 500, FP32 and FP64 forms), table2 (separate targets and sources, the Table 2 setting),
served and served_batched (a short serving run, the second with the solves' matvecs merged into
batched launches: p50/p99 latency with a queue / plan / solve breakdown), and
cpu_baseline (the oracle's direct sum over all host cores, plus the oracle SBD timed on
the N = 2000 disk).

  python bench.py [--gpus N --steps K --warmup W] [--form fp32|fp64] [--impl reference]

Multi-GPU: the matvec does not shard (replicas only); each rank runs its own
instance (seed 2 + rank) and value is the sum over ranks (weak scaling).
--impl reference times the CPU oracle (direct sum) on the host cores instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SBD matvec Gpts/s at rel.err 1e-6 (FP32 vs FP64 form); served p50/p99 latency"
UNIT = "Gpts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workload", default="laplace_curves",
                    choices=["laplace_curves", "helmholtz_curves", "laplace_square", "serve", "batch"])
    ap.add_argument("--instances", type=int, default=64, help="batch: number of plans in the graph")
    ap.add_argument("--n", type=int, default=0, help="points (0: the workload's own size)")
    ap.add_argument("--nrhs", type=int, default=0, help="right-hand sides (0: the workload's own)")
    ap.add_argument("--requests", type=int, default=256, help="serve: number of solve requests")
    ap.add_argument("--slots", type=int, default=8, help="serve: concurrent requests")
    ap.add_argument("--batch-matvecs", action="store_true",
                    help="serve: merge the solves' matvecs into batched launches (iteration-level batching)")
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--alpha", type=float, default=0.0,
                    help="curve workloads: delta_min by Theorem 1 with this alpha in [0, 1/6]")
    ap.add_argument("--cpu-targets", type=int, default=400, help="targets of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-balance", action="store_true", help="skip the delta_min balance (sbd_plan_balanced)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-form, near-FP32, Helmholtz and serving keys of the default line")
    ap.add_argument("--served-requests", type=int, default=64, help="requests of the serving key")
    return ap.parse_args()


WORKLOADS = {
    # name: (default N, default nrhs, seed, description)
    "laplace_curves": (1_000_000, 1, 2, "Laplace, 8 star-shaped curves in [0,10]^2, delta_min by Theorem 1 alpha=0"),
    "helmholtz_curves": (1_000_000, 1, 3, "Helmholtz kappa*delta_max=500 on the curve family, complex f, "
                                          "delta_min by Theorem 1 alpha=0"),
    "laplace_square": (10_000_000, 16, 4, "Laplace, uniform in the unit square, ~20 neighbours within delta_min"),
}


def resolve(args):
    n0, r0, _, _ = WORKLOADS.get(args.workload, (0, 1, 0, ""))
    args.n = args.n or n0
    args.nrhs = args.nrhs or r0
    return args


def make_workload(args, rank):
    import workloads as W
    seed = WORKLOADS[args.workload][2] + rank
    if args.workload == "laplace_curves":
        return W.laplace_curves(args.n, seed, args.eps, args.alpha)
    if args.workload == "helmholtz_curves":
        return W.helmholtz_curves(args.n, seed, args.eps, alpha=args.alpha)
    return W.laplace_square(args.n, seed, args.eps, args.nrhs)


def workload_config(args, rank):
    desc = WORKLOADS[args.workload][3]
    if args.alpha and args.workload.endswith("curves"):
        desc = desc.replace("alpha=0", f"alpha={args.alpha:g}")
    return {"workload": f"{args.workload} N={args.n} nrhs={args.nrhs} eps={args.eps:g} ({desc})",
            "kernel": "helmholtz" if args.workload.startswith("helmholtz") else "laplace",
            "n_points": args.n, "nrhs": args.nrhs, "eps": args.eps, "seed": WORKLOADS[args.workload][2] + rank,
            "alpha": args.alpha if args.workload.endswith("curves") else None,
            "form": args.form, "l2_policy": "inputs larger than L2 (each grid and D exceed 129 MB)",
            "scaling_mode": "replicas (one independent instance per rank)"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stage_bytes(info, n, nrhs, form, esz=8, near32=False):
    """Algorithmic bytes per launch of each on-line step (see the design notes).
    esz: bytes of one input/output value (8 real Laplace, 16 complex Helmholtz).
    The node step counts a read and a write of the frequency cells it covers (the half plane for
    Laplace) and no node data: the nodes and their weights are a function of (p, m) and a P-vector,
    so the method need not move them (the plan's stored records, which the kernels do stream, are
    reported apart as node_records_bytes).
    near32: D's values stored in float32 (SBD_FLAG_NEAR_FP32), else float64."""
    c = 8 if form == "fp32" else 16          # complex grid element
    pr = 16 if form == "fp32" else 24        # point record: int2 cell + fractions
    m, nk, nnz, P = info["grid_x"], info["grid_k"], info["nnz"], info["stencil_x"]
    touched = min(m * m, n * P * P)
    vb = (16 if esz == 16 else 8) // (2 if near32 else 1)   # D value: complex for Helmholtz, float32 with the flag
    r = nrhs   # every step takes all right-hand sides in one launch: grid and value terms scale with r
    if info.get("uniform_grid"):
        # uniform-grid variant: the node step is one multiplication per stored frequency (grid in and
        # out, and the coefficients: real for Laplace over the half plane, complex for Helmholtz)
        cb = c // 2 if esz == 8 else c
        node = (c * nk * nk + cb * nk * nk // 2) if esz == 8 else (2 * c * nk * nk + cb * nk * nk)
        out = stage_bytes(dict(info, uniform_grid=0), n, nrhs, form, esz, near32)
        out["node"] = node * r if esz == 8 else node * r
        return out
    if esz == 8:
        # Laplace: real spreading grid (half a complex element per cell), Hermitian K of
        # which the half plane kx >= 0 is transformed, half the node records
        return {
            "sum": esz * n * r,
            "spread": pr * n + (esz * n + c * m * m // 2) * r,
            "fft_fwd": c * (m * m // 2 + nk * nk // 2) * r,
            "node": c * nk * nk * r,
            "fft_inv": c * (nk * nk // 2 + m * m // 2) * r,
            "interp": pr * n + (esz * n + c * touched // 2) * r,
            "spmv": (4 + vb) * nnz + 8 * (n + 1) + 2 * esz * n * r,
        }
    return {
        "sum": esz * n * r,
        "spread": pr * n + (esz * n + c * m * m) * r,
        "fft_fwd": c * (m * m + nk * nk) * r,
        "node": 2 * c * nk * nk * r,
        "fft_inv": c * (nk * nk + m * m) * r,
        "interp": pr * n + (esz * n + c * touched) * r,
        "spmv": (4 + vb) * nnz + 8 * (n + 1) + 2 * esz * n * r,
    }


def node_records_bytes(info, form):
    """Bytes of the node records the node step streams per launch (stored at plan time)."""
    return (24 if form == "fp32" else 32) * info["n_records"]


def traffic_key(args, alpha):
    """Key of a workload's entries in the committed traffic table: the workload at its own size
    and right-hand sides, delta_min by Theorem 1 at alpha (curve workloads)."""
    n0, r0, _, _ = WORKLOADS[args.workload]
    key = args.workload
    if args.n != n0 or args.nrhs != r0:
        key += f"_n{args.n}_rhs{args.nrhs}"
    return key if not alpha else f"{key}_alpha{alpha:g}"


def traffic_for(stage, workload, form):
    """dram bytes per launch from a committed ncu summary, if it covers this stage's kernels
    on this workload and form and the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        ent = d.get(f"{workload}/{form}/{stage}")
        if not ent:
            return None
        import hashlib
        src = os.path.join(ROOT, ent["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent["source_sha"]:
            return None   # kernel changed since the counters were taken
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_ORACLE_DATA = None


def _oracle_init(z, f, kind, kappa, y):
    global _ORACLE_DATA
    _ORACLE_DATA = (z, f, kind, kappa, y)


def _oracle_direct(idx):
    from oracle import sbd_oracle as O
    z, f, kind, kappa, y = _ORACLE_DATA
    if y is not None:
        return O.direct_sum_st(z, y, f, kind, kappa, targets=idx, chunk=16)
    return O.direct_sum(z, f, kind, kappa, targets=idx, chunk=16)


class OraclePool:
    """The oracle's direct sum over the host cores: one spawned worker process per core (single-
    threaded numpy each), every worker holding the points and f, targets split evenly.  With y
    given, z are the targets and y the sources (the direct sum of separate sets)."""

    def __init__(self, z, f, kind="laplace", kappa=0.0, cores=None, y=None):
        import multiprocessing as mp
        self.cores = max(1, cores or os.cpu_count() or 1)
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                      initargs=(z, f, kind, kappa, y))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.n = len(z) if y is None else len(y)      # sources: pairs per target
        self.nrhs = 1 if np.ndim(f) == 1 else f.shape[0]
        self.pool.map(_oracle_direct, [np.array([i]) for i in range(self.cores)], chunksize=1)   # warm

    def direct_sum(self, idx):
        """(q at the targets, seconds, workers used)."""
        parts = [c for c in np.array_split(np.asarray(idx), min(self.cores, len(idx))) if len(c)]
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_direct, parts, chunksize=1)
        dt = time.perf_counter() - t0
        return np.concatenate(out, axis=-1), dt, len(parts)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(pool, targets_idx):
    """Time the oracle's direct sum on a sample of targets over the host cores; return (rate info, q)."""
    q, dt, used = pool.direct_sum(targets_idx)
    pairs = len(targets_idx) * pool.n * pool.nrhs
    # a full matvec needs N^2 pair evaluations: Gpts/s = N / (N^2 / pair rate)
    value = (pairs / dt) / pool.n / 1e9
    return {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"direct sum (Eq. discreteConv) at {len(targets_idx)} sampled targets over all {pool.n} "
                      f"sources x {pool.nrhs} rhs in {dt:.2f} s on {used} worker processes (one per host core, "
                      f"os.cpu_count() = {os.cpu_count()}); value = pair rate / N (extrapolated to a full matvec)"}, q


def oracle_sbd_timing(n=2000, seed=1, eps=1e-6):
    """The oracle SBD (plain SBD: direct exponential sums, brute-force near pairs) on the
    N = 2000 disk workload, timed whole on one core: plan (fit, circles, D) and one matvec."""
    import workloads as W
    from oracle import sbd_oracle as O
    wl = W.laplace_disk(n, seed, eps)
    t0 = time.perf_counter()
    pl = O.make_plan(wl.z, "laplace", wl.delta_min, wl.eps)
    pl.D = O.close_matrix(pl)
    t1 = time.perf_counter()
    O.sbd_matvec(pl, wl.f)
    t2 = time.perf_counter()
    return {"workload": f"laplace_disk N={n} eps={eps:g}", "cores": 1, "plan_s": t1 - t0, "matvec_s": t2 - t1,
            "value": n / (t2 - t1) / 1e9, "unit": UNIT, "P": int(pl.P), "n_xi": int(len(pl.xi))}


def stage_report(S, plan, step, f_dev, args, info, nrhs, esz, workload_key, form=None, near32=False, steps=None):
    """Per-step device times of `steps` matvecs (library events on the launching stream),
    algorithmic bytes per step and the roofline entry of the step that takes longest."""
    import torch
    form = form or args.form
    steps = steps or args.steps
    S.sbd_profile(plan, True)
    for _ in range(steps):
        step(f_dev)
    torch.cuda.synchronize()
    prof = S.sbd_profile_read(plan)
    S.sbd_profile(plan, False)
    sb = stage_bytes(info, args.n, nrhs, form, esz, near32)
    hbm, peak_src = measured_peaks()
    stages = {}
    for st, (tot, cnt) in prof.items():
        if cnt:
            avg = tot / cnt
            stages[st] = {"ms": avg, "launches_per_step": cnt // steps, "algorithmic_bytes": sb[st],
                          "GBps": sb[st] / (avg * 1e-3) / 1e9}
    if "node" in stages and not info.get("uniform_grid"):
        stages["node"]["node_records_bytes"] = node_records_bytes(info, form)
    dom = max(stages, key=lambda s_: stages[s_]["ms"] * stages[s_]["launches_per_step"])
    achieved = stages[dom]["GBps"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic_for(dom, workload_key, form),
                "peak_source": f"{peak_src} (hbm_gbs)"}
    return stages, roofline


def max_over_ranks(ms, world, device):
    """The slowest rank's time (the whole job finishes when it does); ms on one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput (Gpts/s) of `world` replicas, each doing units_per_rank in ms."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload in ("serve", "batch"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no solve server or batch runner; "
                                                              "those lines are compared against matvec lines"}))
        return
    wl = make_workload(args, 0)
    pool = OraclePool(wl.z, wl.f, wl.kernel, wl.kappa)
    rng = np.random.default_rng(123)
    k = max(4 * pool.cores, args.cpu_targets // max(args.steps, 1) // args.nrhs)
    for _ in range(args.warmup):
        cpu_baseline(pool, rng.choice(args.n, pool.cores, replace=False))
    times, used = [], pool.cores
    for _ in range(args.steps):
        info, _ = cpu_baseline(pool, rng.choice(args.n, k, replace=False))
        times.append(info["value"])
        used = info["cores"]
    pool.close()
    value = statistics.median(times)
    ms = args.n * args.nrhs / (value * 1e9) * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": workload_config(args, 0),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"direct sum at {k} sampled targets per step over all {args.n} sources "
                                   f"x {args.nrhs} rhs, targets split over {used} worker processes; "
                                   f"ms_per_step extrapolates the pair rate to a full N x N matvec"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def accuracy(q, qref, f, idx):
    """Errors at the sampled targets against the oracle's direct sum: rel-L2 and max / sum|f|."""
    qs = q[..., idx]
    f_abs = np.abs(f).sum(axis=-1, keepdims=True) if np.ndim(f) > 1 else np.abs(f).sum()
    return {"targets": len(idx), "reference": "oracle direct sum (FP64)",
            "rel_l2_vs_direct_sum": float(np.linalg.norm(qs - qref) / np.linalg.norm(qref)),
            "max_err_over_sum_abs_f": float(np.max(np.abs(qs - qref) / f_abs))}


class Runner:
    """One plan of a workload on the device: planned, tuned, warmed up and timed with CUDA events
    on the launching stream (the same protocol as the headline)."""

    def __init__(self, S, torch, stream, zt, ft, wl, form, nrhs, flags=0, tune=True):
        self.S, self.torch, self.stream, self.ft, self.nrhs = S, torch, stream, ft, nrhs
        kind = S.SBD_HELMHOLTZ if wl.kernel == "helmholtz" else S.SBD_LAPLACE
        self.plan = S.sbd_plan(zt, len(wl.z), kind, wl.kappa, wl.delta_min, wl.eps,
                               S.make_options(form=form, max_nrhs=nrhs, flags=flags))
        self.tune_ms = S.sbd_tune(self.plan, 3, stream.cuda_stream) if tune else None
        self.info = S.sbd_plan_info(self.plan)
        self.q = torch.empty_like(ft)

    def step(self, f_in):
        self.S.sbd_matvec(self.plan, f_in, self.q, self.nrhs, self.stream.cuda_stream)

    def time(self, steps, warmup):
        torch = self.torch
        for _ in range(warmup):
            self.step(self.ft)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            self.step(self.ft)
        e1.record(self.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def close(self):
        self.S.sbd_destroy(self.plan)
        self.q = None


def plan_keys(info):
    return {k: info[k] for k in ("P", "n_xi", "nnz", "grid_x", "grid_k", "fft_n", "fit_err", "device_bytes",
                                 "plan_seconds")}


def main():
    args = resolve(parse())
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serve":
        out = run_serve(args, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    import torch
    import torch.distributed as dist

    import paper_1711_07877_gb300 as S

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = make_workload(args, rank)
    helm = wl.kernel == "helmholtz"
    esz = 16 if helm else 8
    nrhs = args.nrhs
    form = S.SBD_FORM_FP32 if args.form == "fp32" else S.SBD_FORM_FP64
    zt = torch.from_numpy(wl.z).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(wl.f)).cuda()
    stream = torch.cuda.current_stream()
    t_tune = time.perf_counter()
    head = Runner(S, torch, stream, zt, ft, wl, form, nrhs)
    t_tune = time.perf_counter() - t_tune - head.info["plan_seconds"]
    plan, qt, info, step = head.plan, head.q, head.info, head.step

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(ft)
    barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(ft)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    value = job_rate(args.n * nrhs, world, ms)

    # per-step device times on the same stream (library events), for the roofline
    stages, roofline = stage_report(S, plan, step, ft, args, info, nrhs, esz, traffic_key(args, args.alpha))

    # delta_min by measurement (Theorem 1 leaves alpha in [0, 1/6] free): the same points, f,
    # eps and form, planned at the fastest alpha; reported beside the headline (alpha = 0)
    balanced, q_bal = None, None
    if args.workload in ("laplace_curves", "helmholtz_curves") and not args.no_balance:
        alphas = [0.0, 1 / 24, 1 / 12, 5 / 48, 1 / 8, 1 / 6]
        pb, cand_ms, ci = S.sbd_plan_balanced(zt, args.n, S.SBD_HELMHOLTZ if helm else S.SBD_LAPLACE, wl.kappa,
                                              wl.eps, alphas, nrhs, 5, S.make_options(form=form, max_nrhs=nrhs),
                                              stream.cuda_stream)
        infob = S.sbd_plan_info(pb)
        qb = torch.empty_like(ft)

        def step_b(f_in):
            S.sbd_matvec(pb, f_in, qb, nrhs, stream.cuda_stream)
        for _ in range(args.warmup):
            step_b(ft)
        barrier()
        e0b, e1b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0b.record(stream)
        for _ in range(args.steps):
            step_b(ft)
        e1b.record(stream)
        barrier()
        msb = max_over_ranks(e0b.elapsed_time(e1b) / args.steps, world, "cuda")
        stages_b, roof_b = stage_report(S, pb, step_b, ft, args, infob, nrhs, esz,
                                        traffic_key(args, alphas[ci]))
        balanced = {"alpha": alphas[ci], "delta_min": infob["delta_min"], "a": infob["a"],
                    "value": job_rate(args.n * nrhs, world, msb), "unit": UNIT, "ms_per_step": msb,
                    "candidates": [{"alpha": a_, "ms": m_} for a_, m_ in zip(alphas, cand_ms)],
                    "roofline": roof_b, "stages": stages_b, "plan": plan_keys(infob),
                    "note": "delta_min = a delta_max, a = |log eps|^(2/3) / N^(2/3 - alpha) (Theorem 1) at the "
                            "fastest alpha of the candidates (sbd_plan_balanced: each planned, tuned and timed); "
                            "same points, f, eps and form as the headline line, which keeps alpha = 0"}
        q_bal = qb.cpu().numpy()
        S.sbd_destroy(pb)
        del qb

    # cuFFT (through torch.fft), timed only as a comparison for the forward transform: the
    # same row transforms (length n, the rows that carry data), full outputs, plus the
    # transpose between the two passes
    fft_cmp = None
    try:
        m_, nk_, n_ = info["grid_x"], info["grid_k"], info["fft_n"]
        rows1 = m_ // 2 if not helm else m_
        rows2 = nk_ // 2 + info["stencil_k"] // 2 + 2 if not helm else nk_
        cdt = torch.complex64 if args.form == "fp32" else torch.complex128
        a1 = torch.randn(rows1, m_, dtype=cdt, device="cuda")
        a2 = torch.randn(rows2, m_, dtype=cdt, device="cuda")

        def cufft_fwd():
            y1 = torch.fft.fft(a1, n=n_, dim=1)
            t = y1[:, :rows2].t().contiguous() if rows2 <= n_ else y1.t().contiguous()
            return torch.fft.fft(a2, n=n_, dim=1), t
        for _ in range(2):
            cufft_fwd()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            cufft_fwd()
        e1.record(stream)
        torch.cuda.synchronize()
        fft_cmp = {"ours_fft_fwd_ms": stages["fft_fwd"]["ms"], "cufft_ms": e0.elapsed_time(e1) / 5,
                   "note": "torch.fft (cuFFT) on the same row counts and length, full outputs, plus one "
                           "transpose; comparison only, not on the matvec path"}
        del a1, a2
        torch.cuda.empty_cache()
    except Exception as exc:  # a comparison only
        fft_cmp = {"error": str(exc)[:200]}

    # end to end through the public API: pinned host f -> device, matvec, q -> pinned host
    fh = torch.from_numpy(np.ascontiguousarray(wl.f)).pin_memory()
    qh = torch.empty_like(fh).pin_memory()
    fd = torch.empty_like(ft)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        fd.copy_(fh, non_blocking=True)
        step(fd)
        qh.copy_(qt, non_blocking=True)
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    io_bytes = esz * args.n * nrhs
    e2e = {"value": job_rate(args.n * nrhs, world, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.form == "fp32" else "f64", "data": "synthetic",
           "config": workload_config(args, rank), "clocks": clk, "e2e": e2e,
           # per matvec, all right-hand sides together: f gather, D f, sum of f, spread, 2 row FFT
           # passes on each side of the node step, and the interpolation (the ncu launch list shows 10)
           "gpu_launches": 10 * args.steps, "roofline": roofline, "stages": stages,
           "fft_comparison": fft_cmp, "balanced_delta_min": balanced,
           "plan": dict({k: info[k] for k in ("P", "n_xi", "n_records", "nnz", "grid_x", "grid_k", "fft_n",
                                              "stencil_x", "stencil_k", "nufft_tol", "fit_err", "device_bytes",
                                              "plan_seconds", "node_acc", "node_sched")},
                        tune_seconds=t_tune, tune_node_ms=head.tune_ms)}
    q_head = qt.cpu().numpy()
    head.close()
    extra = rank == 0 and world == 1 and not args.no_extras
    pool, idx, qref = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool(wl.z, wl.f, wl.kernel, wl.kappa)
        targets = args.cpu_targets if args.n * nrhs <= 2_000_000 else max(8, args.cpu_targets // 20)
        idx = np.random.default_rng(7).choice(args.n, targets, replace=False)
        cb, qref = cpu_baseline(pool, idx)
        if extra:
            cb["oracle_sbd"] = oracle_sbd_timing()
        out["cpu_baseline"] = cb
        out["accuracy"] = accuracy(q_head, qref, wl.f, idx)
        if balanced is not None:
            balanced["accuracy"] = accuracy(q_bal, qref, wl.f, idx)
    if extra and args.workload == "laplace_curves":
        out["uniform_grid"] = uniform_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, pool, idx, qref, value)
        out["near_fp32"] = near_fp32_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, stages, pool, idx, qref)
        out["fp64_form"] = form_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, S.SBD_FORM_FP64, pool, idx,
                                     qref, value)
        out["eps_sweep"] = eps_sweep(S, torch, stream, zt, ft, wl, args, nrhs, pool, idx, qref)
    if pool is not None:
        pool.close()
    del zt, ft
    torch.cuda.empty_cache()
    if extra and args.workload == "laplace_curves":
        out["helmholtz"] = helmholtz_lines(S, torch, stream, args)
        out["table2"] = table2_line(S, torch, stream, args)
        out["served"] = run_serve(args, rank, world, local, requests=args.served_requests, short=True,
                                  batch_matvecs=False)
        out["served_batched"] = run_serve(args, rank, world, local, requests=args.served_requests, short=True,
                                          batch_matvecs=True)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def uniform_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, pool, idx, qref, type3_value):
    """The headline workload with SBD_FLAG_UNIFORM_GRID: the node step replaced by a multiplication by
    the Fourier coefficients of the windowed series (no circle quadrature), FP32 form."""
    r = Runner(S, torch, stream, zt, ft, wl, S.SBD_FORM_FP32, nrhs, flags=S.SBD_FLAG_UNIFORM_GRID)
    try:
        ms = r.time(min(args.steps, 20), 3)
        st, roof = stage_report(S, r.plan, r.step, ft, args, r.info, nrhs, esz, "none", form="fp32", steps=3)
        value = args.n * nrhs / (ms * 1e-3) / 1e9
        line = {"flags": "SBD_FLAG_UNIFORM_GRID", "ms_per_step": ms, "value": value, "unit": UNIT,
                "over_type3": value / type3_value, "stages": st, "roofline": roof,
                "plan": dict(plan_keys(r.info), n_records=r.info["n_records"]),
                "note": "node step = multiplication by the coefficients of the windowed, periodised series G_fit "
                        "(each J0 term whole, no circle quadrature); stage 'node' is that multiplication"}
        if pool is not None:
            line["accuracy"] = accuracy(r.q.cpu().numpy(), qref, wl.f, idx)
        return line
    finally:
        r.close()


def near_fp32_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, stages, pool, idx, qref):
    """The headline plan with SBD_FLAG_NEAR_FP32: D f in float32 beside the default float64 D f."""
    r = Runner(S, torch, stream, zt, ft, wl, S.SBD_FORM_FP32, nrhs, flags=S.SBD_FLAG_NEAR_FP32)
    try:
        ms = r.time(min(args.steps, 10), 2)
        st, _ = stage_report(S, r.plan, r.step, ft, args, r.info, nrhs, esz, "none", form="fp32", near32=True,
                             steps=3)
        line = {"flags": "SBD_FLAG_NEAR_FP32", "ms_per_step": ms, "value": args.n * nrhs / (ms * 1e-3) / 1e9,
                "unit": UNIT, "spmv_ms": st["spmv"]["ms"], "spmv_GBps": st["spmv"]["GBps"],
                "spmv_ms_fp64_near": stages["spmv"]["ms"], "spmv_GBps_fp64_near": stages["spmv"]["GBps"],
                "note": "D rounded to float32 and applied to float32 f (row partials in float64) against the "
                        "default float64 D f of the headline"}
        if pool is not None:
            line["accuracy"] = accuracy(r.q.cpu().numpy(), qref, wl.f, idx)
        return line
    finally:
        r.close()


def form_line(S, torch, stream, zt, ft, wl, args, nrhs, esz, form, pool, idx, qref, fp32_value):
    """The same workload in the FP64 form (spread, FFT, node step and interpolation in float64)."""
    r = Runner(S, torch, stream, zt, ft, wl, form, nrhs)
    try:
        ms = r.time(min(args.steps, 5), 2)
        st, roof = stage_report(S, r.plan, r.step, ft, args, r.info, nrhs, esz, "none", form="fp64", steps=2)
        value = args.n * nrhs / (ms * 1e-3) / 1e9
        line = {"form": "fp64", "dtype": "f64", "ms_per_step": ms, "value": value, "unit": UNIT,
                "fp32_over_fp64": fp32_value / value, "stages": st, "roofline": roof, "plan": plan_keys(r.info)}
        if pool is not None:
            line["accuracy"] = accuracy(r.q.cpu().numpy(), qref, wl.f, idx)
        return line
    finally:
        r.close()


def eps_sweep(S, torch, stream, zt, ft, wl, args, nrhs, pool, idx, qref):
    """The headline points and f at the other tolerances of the curve workload, eps = 1e-3 and 1e-9
    (delta_min by Theorem 1 at each eps): the FP64 form at both, the FP32 form at 1e-3 (its floor is
    ~3e-7).  At 1e-9 the fit needs its full Gram Cholesky (P ~ 7000), factored on the device."""
    import workloads as W
    out = {}
    for eps, forms in ((1e-3, ("fp32", "fp64")), (1e-9, ("fp64",))):
        w = dataclasses.replace(wl, delta_min=W.theorem1_delta_min(args.n, eps, wl.meta["delta_max"], args.alpha),
                                eps=eps)
        line = {"delta_min": w.delta_min}
        for name in forms:
            S.sbd_fit_cache_clear()
            r = Runner(S, torch, stream, zt, ft, w, S.SBD_FORM_FP32 if name == "fp32" else S.SBD_FORM_FP64, nrhs)
            try:
                fit_s, fit_where = S.sbd_fit_last_factorisation()
                ms = r.time(min(args.steps, 5 if name == "fp64" else 20), 2)
                d = {"ms_per_step": ms, "value": args.n * nrhs / (ms * 1e-3) / 1e9, "unit": UNIT,
                     "plan": plan_keys(r.info)}
                if fit_where:
                    d["fit_factorisation"] = {"seconds": fit_s, "on": "device" if fit_where == 2 else "host"}
                if pool is not None:
                    d["accuracy"] = accuracy(r.q.cpu().numpy(), qref, w.f, idx)
                line[name] = d
            finally:
                r.close()
        out[f"{eps:g}"] = line
    return out


def table2_line(S, torch, stream, args):
    """Separate targets and sources, the Sec. 7.1 / Table 2 benchmark: N targets and N sources
    uniform in the unit square (independent), Laplace, FP32 form, delta_min by Theorem 1."""
    import workloads as W
    wl = W.laplace_square_st(args.n, 6, args.eps)
    xt = torch.from_numpy(wl.z).cuda()
    yt = torch.from_numpy(wl.y).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(wl.f)).cuda()
    plan = S.sbd_plan_st(xt, args.n, yt, args.n, S.SBD_LAPLACE, 0.0, wl.delta_min, wl.eps,
                         S.make_options(form=S.SBD_FORM_FP32))
    try:
        S.sbd_tune(plan, 3, stream.cuda_stream)
        info = S.sbd_plan_info(plan)
        q = torch.empty(args.n, dtype=torch.float64, device="cuda")
        for _ in range(2):
            S.sbd_matvec(plan, ft, q, 1, stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = min(args.steps, 10)
        e0.record(stream)
        for _ in range(steps):
            S.sbd_matvec(plan, ft, q, 1, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out = {"workload": f"laplace_square_st N={args.n} targets and N sources uniform in [0,1]^2 (independent), "
                           f"eps={args.eps:g}, FP32 form, delta_min by Theorem 1 alpha=0",
               "ms_per_step": ms, "value": args.n / (ms * 1e-3) / 1e9, "unit": UNIT,
               "plan": plan_keys(info),
               "paper_table2": {"N": 1_000_000, "online_s": 2.6, "hardware": "a laptop at 1.6 GHz, 32 GB (Table 2)",
                                "note": "context only: another machine, precision and eps not stated"}}
        if not args.no_cpu_baseline:
            idx = np.random.default_rng(13).choice(args.n, 64, replace=False)
            pool = OraclePool(wl.z, wl.f, "laplace", 0.0, y=wl.y)
            try:
                qref, _, _ = pool.direct_sum(idx)
            finally:
                pool.close()
            out["accuracy"] = accuracy(q.cpu().numpy(), qref, wl.f, idx)
        return out
    finally:
        S.sbd_destroy(plan)
        del xt, yt, ft
        torch.cuda.empty_cache()


def helmholtz_lines(S, torch, stream, args):
    """Helmholtz, kappa delta_max = 500, N = 10^6 on the curves (eps = 1e-6): FP32 and FP64 forms,
    errors against the oracle's direct sum at sampled targets (over the host cores)."""
    import workloads as W
    wl = W.helmholtz_curves(args.n, 3, args.eps)
    zt = torch.from_numpy(wl.z).cuda()
    ft = torch.from_numpy(np.ascontiguousarray(wl.f)).cuda()
    out = {"workload": f"helmholtz_curves N={args.n} nrhs=1 eps={args.eps:g} (kappa delta_max = 500, complex f, "
                       "delta_min by Theorem 1 alpha=0)"}
    qs = {}
    for name, form in (("fp32", S.SBD_FORM_FP32), ("fp64", S.SBD_FORM_FP64)):
        r = Runner(S, torch, stream, zt, ft, wl, form, 1)
        try:
            ms = r.time(min(args.steps, 10 if name == "fp32" else 4), 2)
            st, roof = stage_report(S, r.plan, r.step, ft, args, r.info, 1, 16, "none", form=name, steps=2)
            out[name] = {"ms_per_step": ms, "value": args.n / (ms * 1e-3) / 1e9, "unit": UNIT, "stages": st,
                         "roofline": roof, "plan": plan_keys(r.info)}
            qs[name] = r.q.cpu().numpy()
        finally:
            r.close()
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    if not args.no_cpu_baseline:
        idx = np.random.default_rng(8).choice(args.n, 64, replace=False)
        pool = OraclePool(wl.z, wl.f, "helmholtz", wl.kappa)
        try:
            qref, dt, used = pool.direct_sum(idx)
        finally:
            pool.close()
        for name in qs:
            out[name]["accuracy"] = accuracy(qs[name], qref, wl.f, idx)
        out["oracle_seconds"] = dt
    del zt, ft
    torch.cuda.empty_cache()
    return out


def run_batch(args, rank, world, local):
    """Many small plans of uneven size: one batch-graph launch against one matvec after another."""
    import torch

    import paper_1711_07877_gb300 as S
    import workloads as W

    torch.cuda.set_device(local)
    rng = np.random.default_rng(11 + rank)
    form = S.SBD_FORM_FP32 if args.form == "fp32" else S.SBD_FORM_FP64
    plans, fs, qs, ns = [], [], [], []
    for i in range(args.instances):
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5)))))
        z = W.curve_points(n, 20_000 + 100 * rank + i)
        dmax = W.enclosing_diameter(z)
        p = S.sbd_plan(torch.from_numpy(z).cuda(), n, S.SBD_LAPLACE, 0.0, W.theorem1_delta_min(n, args.eps, dmax),
                       args.eps, S.make_options(form=form))
        plans.append(p)
        ns.append(n)
        fs.append(torch.from_numpy(W.rhs(n, 30_000 + i)).cuda())
        qs.append(torch.empty_like(fs[-1]))
    units = sum(ns)
    stream = torch.cuda.current_stream()
    b = S.sbd_batch_create(plans, fs, qs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def seq():
        for p, f, q in zip(plans, fs, qs):
            S.sbd_matvec(p, f, q, 1, stream.cuda_stream)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    ms_batch = max_over_ranks(timed(lambda: S.sbd_batch_launch(b, stream.cuda_stream)), world, "cuda")
    ms_seq = max_over_ranks(timed(seq), world, "cuda")
    ms_batched = max_over_ranks(timed(lambda: S.sbd_matvec_batched(plans, fs, qs, stream=stream.cuda_stream)),
                                world, "cuda")
    batched_status = S.sbd_device_status(stream.cuda_stream)
    clk = clocks.stop()
    # end to end: host f in, batch launch, host q out (pinned buffers)
    fh = [f.cpu().pin_memory() for f in fs]
    qh = [torch.empty_like(x).pin_memory() for x in fh]

    def e2e():
        for f, h in zip(fs, fh):
            f.copy_(h, non_blocking=True)
        S.sbd_batch_launch(b, stream.cuda_stream)
        for q, h in zip(qs, qh):
            h.copy_(q, non_blocking=True)
    ms_e2e = max_over_ranks(timed(e2e), world, "cuda")
    S.sbd_batch_destroy(b)
    for p in plans:
        S.sbd_destroy(p)
    out = {"metric": METRIC, "value": job_rate(units, world, ms_batch), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.form == "fp32" else "f64",
           "data": "synthetic",
           "config": {"workload": f"batch of {args.instances} Laplace plans, N log-uniform in [1e3, 1e5] on curve "
                                  f"geometries, eps={args.eps:g}, one CUDA-graph launch per step",
                      "instances": args.instances, "points_total": units, "form": args.form,
                      "l2_policy": "per-instance grids small; the whole batch exceeds L2"},
           "sequential": {"ms_per_step": ms_seq, "value": job_rate(units, world, ms_seq),
                          "note": "the same matvecs, one sbd_matvec after another on one stream"},
           "matvec_batched": {"ms_per_step": ms_batched, "value": job_rate(units, world, ms_batched),
                              "status": batched_status,
                              "note": "sbd_matvec_batched: one spreading, one node-step and one interpolation "
                                      "launch over all instances (persistent CTAs, work queues), the FFTs per "
                                      "instance on their own streams"},
           "e2e": {"value": job_rate(units, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": 8 * units,
                   "d2h_bytes_per_step": 8 * units},
           "clocks": clk, "roofline": None, "gpu_launches": 10 * args.instances * args.steps}
    if rank == 0:
        print(json.dumps(out))


def run_serve(args, rank, world, local, requests=None, short=False, batch_matvecs=None):
    """Continuous-batching solve server over a Poisson stream of GMRES requests; returns the line
    (or, with short, the key the default line carries) with p50/p99 latency and a per-request
    breakdown into queueing (arrival to admission), planning and solving."""
    import torch

    import paper_1711_07877_gb300 as S
    from paper_1711_07877_gb300 import serve
    import workloads as W

    torch.cuda.set_device(local)
    count = requests or args.requests
    specs = W.serve_requests(count, seed=5 + rank, eps=args.eps)
    form = S.SBD_FORM_FP32 if args.form == "fp32" else S.SBD_FORM_FP64
    reqs = [serve.Request(rid=i, z=r["z"], b=r["b"],
                          kind=S.SBD_HELMHOLTZ if r["kernel"] == "helmholtz" else S.SBD_LAPLACE,
                          kappa=r["kappa"], delta_min=r["delta_min"], eps=r["eps"], shift=r["shift"],
                          scale=r["scale"]) for i, r in enumerate(specs)]
    # warm-up: a few small requests (library load, kernel attributes, allocator)
    warm = [serve.Request(rid=-1 - i, z=r.z, b=r.b, kind=r.kind, kappa=r.kappa, delta_min=r.delta_min,
                          eps=r.eps, shift=r.shift, scale=r.scale)
            for i, r in enumerate(sorted(reqs, key=lambda q: len(q.z))[:max(args.warmup, 3)])]
    serve.run_poisson(warm, mean_gap_s=0.002, seed=1, slots=args.slots, form=form, tol=1e-6, max_iter=600)
    S.sbd_fit_cache_clear()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    torch.cuda.synchronize()
    batched = args.batch_matvecs if batch_matvecs is None else batch_matvecs
    srv, summ = serve.run_poisson(reqs, mean_gap_s=0.002, seed=9 + rank, slots=args.slots, form=form, tol=1e-6,
                                  max_iter=600, timeout_s=600.0, batch_matvecs=batched)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ok = [r for r in reqs if r.error is None]
    its = [r.iterations for r in ok]
    plan_s = [r.plan_seconds for r in ok]
    cache = S.sbd_fit_cache_stats()
    h2d = sum(r.z.nbytes + r.b.nbytes for r in ok)
    d2h = sum(r.b.nbytes for r in ok)

    def pct(xs):
        return {"p50_ms": float(np.percentile(xs, 50) * 1e3), "p99_ms": float(np.percentile(xs, 99) * 1e3),
                "mean_ms": float(np.mean(xs) * 1e3)} if xs else None
    breakdown = {"queue": pct([r.start - r.arrival for r in ok]), "plan": pct(plan_s),
                 "solve": pct([r.done - r.start - r.plan_seconds for r in ok]),
                 "note": "queue = arrival to admission, plan = sbd_plan, solve = the rest of the request "
                         "(GMRES, copies); arrivals of all requests span ~2 ms x count"}
    workload = (f"serve {len(reqs)} GMRES requests, Poisson arrivals mean 2 ms, curve geometries "
                "N log-uniform [1e3, 1e6], 50/50 Laplace/Helmholtz kappa*delta_max U[50, 500], "
                "(I/2 + (L/N) A) x = b (L = arc length) to relative residual 1e-6, GMRES(30)")
    served = {"requests_ok": len(ok), "errors": len(reqs) - len(ok), "incomplete": summ.get("incomplete"),
              "wall_s": summ.get("wall_s"),
              "matvecs_mean": float(np.mean(its)) if its else None,
              "matvecs_max": int(max(its)) if its else None,
              "points_mean": float(np.mean([len(r.z) for r in ok])) if ok else None,
              "max_residual": float(max(r.residual for r in ok)) if ok else None,
              "requeued_after_enomem": summ.get("requeued"), "deadline_dropped": summ.get("deadline_dropped"),
              "batch_matvecs": batched, "matvec_batches": summ.get("matvec_batches"),
              "matvecs_batched": summ.get("matvecs_batched"),
              "fit_cache": cache, "breakdown": breakdown}
    latency = {"p50_ms": summ.get("p50_ms"), "p99_ms": summ.get("p99_ms"), "mean_ms": summ.get("mean_ms")}
    if short:
        return {"workload": workload, "slots": args.slots, "form": args.form, "value": summ.get("gpts_per_s"),
                "unit": UNIT, "latency": latency, "served": served, "clocks": clk}
    return {"metric": METRIC, "value": summ["gpts_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": len(reqs), "warmup": len(warm), "ms_per_step": summ["wall_s"] * 1e3 / max(len(reqs), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.form == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": workload, "slots": args.slots, "eps": args.eps, "form": args.form,
                       "l2_policy": "n/a (serving)"},
            "latency": latency, "served": served,
            "e2e": {"value": summ["gpts_per_s"], "unit": UNIT, "h2d_bytes_per_step": h2d // max(len(ok), 1),
                    "d2h_bytes_per_step": d2h // max(len(ok), 1),
                    "note": "each request copies points and b from host and reads x back"},
            "clocks": clk, "roofline": None, "gpu_launches": None}


if __name__ == "__main__":
    main()
