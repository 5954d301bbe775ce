"""Continuous-batching solve server over the C ABI.

Each request is a boundary-integral-like system (shift I + scale A) x = b on its own
point cloud, A the SBD convolution of that cloud (Introduction: iterative solvers
whose cost is the discrete convolution).  The server keeps `slots` worker threads,
each with its own CUDA stream; a request is admitted when a slot is free and its
estimated device footprint fits the HBM budget, then planned (sbd_plan), solved
(sbd_gmres) and released (sbd_destroy) on that slot's stream.  Requests that arrive
while others run are admitted as slots and memory free up, so their device work
overlaps.  The library calls release the GIL; the arithmetic is all in libsbd.so.
"""
from __future__ import annotations

import os
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np

from . import sbd as S


def enclosing_diameter(z: np.ndarray) -> float:
    """2 max |z - c| with c the centre of the bounding box: the plan's delta_max (R2)."""
    lo, hi = z.min(axis=0), z.max(axis=0)
    c = 0.5 * (lo + hi)
    return float(2.0 * np.sqrt(np.max(np.sum((z - c) ** 2, axis=1))))


def fit_grid_scales(kind: int, kappa: float, delta_min: float, diameter: float, a_steps: int = 8,
                    root_step: int = 4) -> tuple[float, float]:
    """(delta_min', delta_max') on fixed grids, so that requests on different geometries
    reuse the library's cached normalised fit.

    The fit depends on a = delta_min / scale_R and, for Helmholtz, on k' (Sec. 4.1-4.2).
    a is rounded down to a power of 2^(1/a_steps): a smaller delta_min keeps the eps
    bound (the fit is made at the new a) and only moves work from the near field to the
    far field.  For Helmholtz, delta_max is raised until k' is a zero of Y0 whose index
    is a multiple of root_step (delta_max' sits just below k' / kappa, so the plan's
    first zero >= kappa delta_max' is that one), and delta_min is capped at one
    wavelength 2 pi / kappa: the Y0 fit needs P a >= k' a / pi + gamma(eps), and past
    P a ~ 6.7 the Gram matrix reaches the FP64 conditioning floor (Sec. 4.1), so a
    delta_min several wavelengths long (small N at large kappa delta_max) cannot be fitted."""
    dmax = diameter * (1.0 + 1e-9)
    if kind == S.SBD_LAPLACE:
        scale_R = dmax
    else:
        x = kappa * dmax
        k = max(1, int(x / np.pi) - 2)
        while S.sbd_y0_root(k) < x:
            k += 1
        k = -(-k // root_step) * root_step
        while True:
            root = S.sbd_y0_root(k)
            dmax_q = root * (1.0 - 1e-12) / kappa
            if dmax_q >= dmax and kappa * dmax_q > S.sbd_y0_root(k - 1):
                break
            k += root_step
        dmax = dmax_q
        scale_R = root / kappa
        delta_min = min(delta_min, 2.0 * np.pi / kappa)
    a = delta_min / scale_R
    a_q = 2.0 ** (np.floor(np.log2(a) * a_steps) / a_steps)
    return float(a_q * scale_R), float(dmax)


@dataclass
class Request:
    rid: int
    z: np.ndarray                 # (N, 2) float64 points
    b: np.ndarray                 # (N,) float64 or complex128
    kind: int                     # S.SBD_LAPLACE / S.SBD_HELMHOLTZ
    kappa: float
    delta_min: float
    eps: float
    shift: complex = 0.5
    scale: complex = 1.0
    geometry: object = None       # hashable key: requests with the same key share points,
                                  # kernel and tolerances, and reuse one resident plan
    arrival: float = 0.0          # seconds after the server's start
    # results
    x: np.ndarray | None = None
    iterations: int = 0
    residual: float = float("nan")
    start: float = 0.0
    done: float = 0.0
    plan_seconds: float = 0.0
    device_bytes: int = 0
    error: str | None = None
    attempts: int = 0             # re-admissions after running out of device memory
    deadline_s: float | None = None   # give up if still queued this long after arrival
    late: bool = False            # finished after its deadline


@dataclass
class ServerStats:
    latencies: list = field(default_factory=list)
    points_matvecs: float = 0.0
    wall: float = 0.0

    def summary(self) -> dict:
        lat = np.sort(np.asarray(self.latencies))
        if lat.size == 0:
            return {"requests": 0}
        return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "wall_s": self.wall, "gpts_per_s": self.points_matvecs / max(self.wall, 1e-9) / 1e9}


class Admission:
    """Device-memory admission for the server (host logic only).

    Requests wait in arrival order; `admit` returns the first waiting request whose
    estimated footprint fits the free budget (a smaller request may pass a larger one
    at the head), or the head itself when nothing is running, so that a request larger
    than the whole budget still runs, alone.  The per-point estimate only grows, from
    the footprints that finished plans report.

    Resident plans: a request with a geometry key keeps its plan on the device after it
    finishes (its bytes stay counted); a later request with the same key reuses it and
    needs only solver workspace, but waits while another request uses that plan.  When
    a request does not fit, idle resident plans are evicted oldest-use first; `admit`
    hands them back so that the caller frees them.
    """

    def __init__(self, budget: int, bytes_per_point: float = 8000.0, fixed_bytes: int = 64 << 20,
                 solve_bytes_per_point: float = 32 * 16.0):
        self.budget = int(budget)
        self.bytes_per_point = float(bytes_per_point)
        self.fixed_bytes = int(fixed_bytes)
        self.solve_bytes_per_point = float(solve_bytes_per_point)
        self.in_use = 0
        self.running = 0
        self.pending: list = []
        self.resident: "OrderedDict" = OrderedDict()   # key -> {"bytes", "busy", "plan"}
        self.building: set = set()                     # keys whose plan a running request builds

    def estimate(self, n_points: int) -> int:
        return int(self.bytes_per_point * n_points) + self.fixed_bytes

    def solve_estimate(self, n_points: int) -> int:
        return int(self.solve_bytes_per_point * n_points)

    def push(self, req) -> None:
        self.pending.append(req)

    def _idle_bytes(self, keep) -> int:
        return sum(v["bytes"] for k, v in self.resident.items() if not v["busy"] and k != keep)

    def admit(self):
        """(request, estimate, [(key, plan) to free]) or None."""
        for i, r in enumerate(self.pending):
            key = getattr(r, "geometry", None)
            if key is not None and key in self.building:
                continue                                # its plan is being built: wait for it
            reuse = key is not None and key in self.resident
            if reuse and self.resident[key]["busy"]:
                continue
            est = self.solve_estimate(len(r.z)) if reuse else self.estimate(len(r.z))
            evict = []
            if self.in_use + est > self.budget and self.running > 0:
                if self.in_use - self._idle_bytes(key) + est > self.budget:
                    continue
                for k in list(self.resident):
                    if self.in_use + est <= self.budget:
                        break
                    v = self.resident[k]
                    if v["busy"] or k == key:
                        continue
                    self.in_use -= v["bytes"]
                    evict.append((k, v["plan"]))
                    del self.resident[k]
            elif self.running == 0 and self.in_use + est > self.budget:
                # alone on the device: free every idle resident plan first
                for k in list(self.resident):
                    v = self.resident[k]
                    if k == key:
                        continue
                    self.in_use -= v["bytes"]
                    evict.append((k, v["plan"]))
                    del self.resident[k]
            self.pending.pop(i)
            self.in_use += est
            self.running += 1
            if reuse:
                self.resident[key]["busy"] = True
                self.resident.move_to_end(key)
            elif key is not None:
                self.building.add(key)
            return r, est, evict
        return None

    def release(self, est: int, n_points: int = 0, device_bytes: int = 0, key=None, plan=None,
                keep: bool = True) -> None:
        """The request is done.  With a key and keep, its plan (device_bytes) stays
        resident; keep = False (the build failed) only ends the build."""
        self.in_use -= est
        self.running -= 1
        if n_points and device_bytes:
            self.bytes_per_point = max(self.bytes_per_point, 1.2 * device_bytes / n_points)
        if key is not None:
            self.building.discard(key)
        if key is not None and keep:
            if key in self.resident:
                self.resident[key]["busy"] = False
            else:
                self.resident[key] = {"bytes": int(device_bytes), "busy": False, "plan": plan}
                self.in_use += int(device_bytes)
            self.resident.move_to_end(key)

    def plan_of(self, key):
        v = self.resident.get(key)
        return v["plan"] if v else None


class CudaBackend:
    """The device side of a request, through the library's entry points (the server's host
    logic talks only to this, so that it can be exercised on the host with a stand-in)."""

    def __init__(self):
        import torch
        self.torch = torch

    def stream(self):
        return self.torch.cuda.Stream()

    def free_bytes(self) -> int:
        return int(self.torch.cuda.mem_get_info()[0])

    def plan(self, req, stream, delta_min: float, delta_max: float, form: int, host_threads: int):
        torch = self.torch
        with torch.cuda.stream(stream):
            zt = torch.from_numpy(req.z).to("cuda", non_blocking=True)
        opt = S.make_options(form=form, delta_max=delta_max, host_threads=host_threads)
        plan = S.sbd_plan(zt, len(req.z), req.kind, req.kappa, delta_min, req.eps, opt, stream.cuda_stream)
        return plan, S.sbd_plan_info(plan)

    def solve(self, plan, req, stream, tol: float, restart: int, max_iter: int):
        torch = self.torch
        with torch.cuda.stream(stream):
            bt = torch.from_numpy(req.b).to("cuda", non_blocking=True)
            xt = torch.zeros_like(bt)
        it, res = S.sbd_gmres(plan, bt, xt, req.shift, req.scale, tol, restart, max_iter, stream.cuda_stream)
        stream.synchronize()
        return xt.cpu().numpy(), it, res

    def solve_batched(self, plan, req, stream, tol: float, restart: int, max_iter: int, sched):
        """GMRES as a session whose matvecs go through the scheduler (merged with other solves')."""
        torch = self.torch
        with torch.cuda.stream(stream):
            bt = torch.from_numpy(req.b).to("cuda", non_blocking=True)
            xt = torch.zeros_like(bt)
        sess = S.sbd_gmres_begin(plan, bt, xt, req.shift, req.scale, tol, restart, max_iter, stream.cuda_stream)
        try:
            while True:
                io = S.sbd_gmres_next(sess)
                if io is None:
                    break
                ready = torch.cuda.Event()
                ready.record(stream)
                done = sched.submit(plan, io[0], io[1], ready)
                stream.wait_event(done)
                S.sbd_gmres_advance(sess)
        finally:
            it, res = S.sbd_gmres_end(sess)
        stream.synchronize()
        return xt.cpu().numpy(), it, res

    def matvec_batched(self, tickets, stream):
        """One sbd_matvec_batched for the tickets' matvecs (distinct plans) on stream, after each
        ticket's ready event; returns the event that marks the batch done."""
        for t in tickets:
            stream.wait_event(t.ready)
        S.sbd_matvec_batched([t.plan for t in tickets], [t.inp for t in tickets], [t.out for t in tickets],
                             stream=stream.cuda_stream)
        done = self.torch.cuda.Event()
        done.record(stream)
        return done

    def synchronize(self, stream) -> None:
        stream.synchronize()

    def destroy(self, plan, stream) -> None:
        S.sbd_destroy_async(plan, stream.cuda_stream)   # no device-wide wait

    def destroy_now(self, plan) -> None:
        S.sbd_destroy(plan)


@dataclass
class _Ticket:
    plan: object
    inp: object
    out: object
    ready: object
    done: object = None
    error: Exception | None = None
    flag: threading.Event = field(default_factory=threading.Event)


class MatvecScheduler:
    """Iteration-level batching of the server's solves: a worker whose GMRES session needs a
    matvec submits it (plan, in, out, an event on its stream) and waits until the batch that
    holds it is enqueued; the scheduler thread takes the pending matvecs of distinct plans
    (at most max_batch), waiting up to window_s for every solving worker to submit, launches
    them as one sbd_matvec_batched on its own stream and hands each worker the batch's event,
    which the worker's stream waits on before the session continues."""

    def __init__(self, backend, max_batch: int = 64, window_s: float = 0.0005):
        self.backend = backend
        self.max_batch = max_batch
        self.window_s = window_s
        self.stream = backend.stream()
        self.cv = threading.Condition()
        self.pending: list[_Ticket] = []
        self.active = 0          # workers inside a solve
        self.closed = False
        self.batches = 0
        self.matvecs = 0
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def enter(self) -> None:
        with self.cv:
            self.active += 1

    def leave(self) -> None:
        with self.cv:
            self.active -= 1
            self.cv.notify_all()

    def submit(self, plan, inp, out, ready):
        t = _Ticket(plan, inp, out, ready)
        with self.cv:
            self.pending.append(t)
            self.cv.notify_all()
        t.flag.wait()
        if t.error is not None:
            raise t.error
        return t.done

    def close(self) -> None:
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self.thread.join()

    def _run(self) -> None:
        while True:
            with self.cv:
                while not self.pending and not self.closed:
                    self.cv.wait(timeout=0.05)
                if self.closed and not self.pending:
                    return
                end = time.perf_counter() + self.window_s
                while len(self.pending) < self.active and not self.closed:
                    left = end - time.perf_counter()
                    if left <= 0:
                        break
                    self.cv.wait(timeout=left)
                take, seen = [], set()
                for t in list(self.pending):
                    if len(take) < self.max_batch and t.plan not in seen:
                        take.append(t)
                        seen.add(t.plan)
                        self.pending.remove(t)
            try:
                done = self.backend.matvec_batched(take, self.stream)
                for t in take:
                    t.done = done
            except Exception as e:   # every matvec of the batch fails with it
                for t in take:
                    t.error = e
            self.batches += 1
            self.matvecs += len(take)
            for t in take:
                t.flag.set()


class Server:
    """slots worker threads; admission by a device-memory budget (bytes).

    Failure handling on the host: a request whose plan or solve runs out of device memory
    (SBD_ENOMEM) goes back to the head of the queue, at most `retries` times, after the
    admission's per-point estimate grows by half (so that it next waits for more room); a
    request with a deadline (Request.deadline_s, seconds after arrival) that is still queued
    when it passes is dropped by a watchdog thread with an error, and one that finishes after
    it is marked late (its result is kept)."""

    def __init__(self, slots: int = 4, hbm_budget: int | None = None, form: int = S.SBD_FORM_FP32,
                 tol: float = 1e-6, restart: int = 30, max_iter: int = 300, fit_grid: bool = True,
                 backend=None, retries: int = 3, watchdog_s: float = 0.01, batch_matvecs: bool = False):
        self.backend = backend or CudaBackend()
        # batch_matvecs: the solves' matvecs merge into batched launches (MatvecScheduler)
        self.sched = MatvecScheduler(self.backend) if batch_matvecs else None
        self.slots = slots
        self.form = form
        self.tol, self.restart, self.max_iter = tol, restart, max_iter
        self.fit_grid = fit_grid
        self.retries = retries
        # the host part of concurrent plan builds shares the cores
        self.host_threads = max(1, (os.cpu_count() or slots) // slots)
        if hbm_budget is None:
            hbm_budget = int(self.backend.free_bytes() * 0.8)
        self.adm = Admission(hbm_budget)
        self.cv = threading.Condition()
        self.stats = ServerStats()
        self.t0 = time.perf_counter()
        self.closed = False
        self.requeued = 0
        self.dropped = 0
        self.workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for w in self.workers:
            w.start()
        self.watchdog = threading.Thread(target=self._watch, args=(watchdog_s,), daemon=True)
        self.watchdog.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> None:
        with self.cv:
            req.arrival = self.now() if req.arrival == 0.0 else req.arrival
            self.adm.push(req)
            self.cv.notify_all()

    def _watch(self, period: float) -> None:
        """Drops queued requests whose deadline has passed."""
        while True:
            with self.cv:
                if self.closed:
                    return
                now = self.now()
                late = [r for r in self.adm.pending
                        if getattr(r, "deadline_s", None) is not None and now - r.arrival > r.deadline_s]
                for r in late:
                    self.adm.pending.remove(r)
                    r.error = f"deadline of {r.deadline_s:.3f} s passed while queued"
                    r.done = now
                    self.dropped += 1
                if late:
                    self.cv.notify_all()
            time.sleep(period)

    def _worker(self):
        be = self.backend
        stream = be.stream()
        while True:
            with self.cv:
                got = None
                while not self.closed:
                    got = self.adm.admit()
                    if got:
                        break
                    self.cv.wait(timeout=0.05)
                if not got:
                    return
            req, est, evict = got
            for _, old_plan in evict:            # idle resident plans that made room
                be.destroy(old_plan, stream)
            req.start = self.now()
            key = req.geometry
            with self.cv:
                plan = self.adm.plan_of(key) if key is not None else None
            reused = plan is not None
            requeue = False
            try:
                if not reused:
                    dmin, dmax = req.delta_min, 0.0
                    if self.fit_grid:
                        dmin, dmax = fit_grid_scales(req.kind, req.kappa, req.delta_min,
                                                     enclosing_diameter(req.z))
                    plan, info = be.plan(req, stream, dmin, dmax, self.form, self.host_threads)
                    req.plan_seconds = info["plan_seconds"]
                    req.device_bytes = info["device_bytes"]
                if self.sched is not None:
                    self.sched.enter()
                    try:
                        req.x, req.iterations, req.residual = be.solve_batched(plan, req, stream, self.tol,
                                                                               self.restart, self.max_iter, self.sched)
                    finally:
                        self.sched.leave()
                else:
                    req.x, req.iterations, req.residual = be.solve(plan, req, stream, self.tol, self.restart,
                                                                   self.max_iter)
            except Exception as e:  # the request fails (or waits again), the server keeps serving
                if getattr(e, "code", None) == S.SBD_ENOMEM and req.attempts < self.retries:
                    requeue = True
                    req.attempts += 1
                else:
                    req.error = str(e)
            finally:
                failed = req.error is not None or requeue
                keep = key is not None and plan is not None and not failed
                if plan is not None and not keep and not reused:
                    be.synchronize(stream)
                    be.destroy(plan, stream)
                    if not reused:
                        plan = None
                if not requeue:
                    req.done = self.now()
                    if getattr(req, "deadline_s", None) is not None and req.done - req.arrival > req.deadline_s:
                        req.late = True
                with self.cv:
                    if keep:
                        self.adm.release(est, len(req.z), req.device_bytes, key=key, plan=plan)
                    elif reused:
                        # a reused plan whose solve failed stays resident
                        self.adm.release(est, key=key, plan=plan)
                    else:
                        self.adm.release(est, len(req.z), req.device_bytes, key=key, keep=False)
                    if requeue:
                        # out of memory: the footprint was underestimated; wait for more room
                        self.adm.bytes_per_point *= 1.5
                        self.adm.pending.insert(0, req)
                        self.requeued += 1
                    elif req.error is None:
                        self.stats.latencies.append(req.done - req.arrival)
                        self.stats.points_matvecs += len(req.z) * (req.iterations + 2)
                    self.cv.notify_all()

    def close(self) -> None:
        """Stop the workers and free every resident plan."""
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()
        self.watchdog.join()
        if self.sched is not None:
            self.sched.close()
        for v in list(self.adm.resident.values()):
            if v["plan"]:
                self.backend.destroy_now(v["plan"])
        self.adm.resident.clear()

    def drain(self, requests: list[Request], timeout_s: float | None = None) -> bool:
        """Wait until every request in the list is done, then stop the workers.  With a
        timeout, give up after timeout_s seconds: the requests still open are marked
        failed, the workers are left running (daemon threads) and False is returned."""
        t0 = time.perf_counter()
        while any(r.done == 0.0 for r in requests):
            if timeout_s is not None and time.perf_counter() - t0 > timeout_s:
                for r in requests:
                    if r.done == 0.0:
                        r.error = "not finished within the drain timeout"
                done = [r.done for r in requests if r.done > 0.0]
                self.stats.wall = (max(done) if done else self.now()) - min(r.arrival for r in requests)
                return False
            time.sleep(0.002)
        self.close()
        self.stats.wall = max(r.done for r in requests) - min(r.arrival for r in requests)
        return True


def run_poisson(requests: list[Request], mean_gap_s: float, seed: int = 0, timeout_s: float | None = None,
                **server_kw) -> tuple[Server, dict]:
    """Submit requests with exponential inter-arrival times; return the server and its summary
    (with "incomplete": the number of requests still open when timeout_s ran out)."""
    rng = np.random.default_rng(seed)
    srv = Server(**server_kw)
    t = 0.0
    for r in requests:
        t += rng.exponential(mean_gap_s)
        while True:
            dt = t - srv.now()
            if dt <= 0:
                break
            time.sleep(min(0.001, dt))
        r.arrival = 0.0
        srv.submit(r)
    finished = srv.drain(requests, timeout_s)
    summ = srv.stats.summary()
    summ["incomplete"] = 0 if finished else sum(r.error == "not finished within the drain timeout" for r in requests)
    summ["requeued"] = srv.requeued
    if srv.sched is not None:
        summ["matvec_batches"] = srv.sched.batches
        summ["matvecs_batched"] = srv.sched.matvecs
    summ["deadline_dropped"] = srv.dropped
    summ["late"] = sum(1 for r in requests if r.late)
    return srv, summ
