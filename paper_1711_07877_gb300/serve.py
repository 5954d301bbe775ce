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


class Server:
    """slots worker threads; admission by a device-memory budget (bytes)."""

    def __init__(self, slots: int = 4, hbm_budget: int | None = None, form: int = S.SBD_FORM_FP32,
                 tol: float = 1e-6, restart: int = 30, max_iter: int = 300, fit_grid: bool = True):
        import torch
        self.torch = torch
        self.slots = slots
        self.form = form
        self.tol, self.restart, self.max_iter = tol, restart, max_iter
        self.fit_grid = fit_grid
        # the host part of concurrent plan builds shares the cores
        self.host_threads = max(1, (os.cpu_count() or slots) // slots)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(free * 0.8)
        self.adm = Admission(hbm_budget)
        self.cv = threading.Condition()
        self.stats = ServerStats()
        self.t0 = time.perf_counter()
        self.closed = False
        self.workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(slots)]
        for w in self.workers:
            w.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request) -> None:
        with self.cv:
            req.arrival = self.now() if req.arrival == 0.0 else req.arrival
            self.adm.push(req)
            self.cv.notify_all()

    def _worker(self):
        torch = self.torch
        stream = torch.cuda.Stream()
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
                S.sbd_destroy_async(old_plan, stream.cuda_stream)
            req.start = self.now()
            key = req.geometry
            with self.cv:
                plan = self.adm.plan_of(key) if key is not None else None
            reused = plan is not None
            try:
                with torch.cuda.stream(stream):
                    bt = torch.from_numpy(req.b).to("cuda", non_blocking=True)
                    xt = torch.zeros_like(bt)
                if not reused:
                    with torch.cuda.stream(stream):
                        zt = torch.from_numpy(req.z).to("cuda", non_blocking=True)
                    dmin, dmax = req.delta_min, 0.0
                    if self.fit_grid:
                        dmin, dmax = fit_grid_scales(req.kind, req.kappa, req.delta_min,
                                                     enclosing_diameter(req.z))
                    opt = S.make_options(form=self.form, delta_max=dmax, host_threads=self.host_threads)
                    plan = S.sbd_plan(zt, len(req.z), req.kind, req.kappa, dmin, req.eps, opt, stream.cuda_stream)
                    info = S.sbd_plan_info(plan)
                    req.plan_seconds = info["plan_seconds"]
                    req.device_bytes = info["device_bytes"]
                it, res = S.sbd_gmres(plan, bt, xt, req.shift, req.scale, self.tol, self.restart, self.max_iter,
                                      stream.cuda_stream)
                stream.synchronize()
                req.x = xt.cpu().numpy()
                req.iterations, req.residual = it, res
            except Exception as e:  # the request fails, the server keeps serving
                req.error = str(e)
            finally:
                keep = key is not None and plan is not None and req.error is None
                if plan is not None and not keep and not reused:
                    stream.synchronize()
                    S.sbd_destroy_async(plan, stream.cuda_stream)   # no device-wide wait
                req.done = self.now()
                with self.cv:
                    if keep:
                        self.adm.release(est, len(req.z), req.device_bytes, key=key, plan=plan)
                    elif reused:
                        # a reused plan whose solve failed stays resident
                        self.adm.release(est, key=key, plan=plan)
                    else:
                        self.adm.release(est, len(req.z), req.device_bytes, key=key, keep=False)
                    if req.error is None:
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
        for v in list(self.adm.resident.values()):
            if v["plan"]:
                S.sbd_destroy(v["plan"])
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
    return srv, summ
