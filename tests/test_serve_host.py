"""Host logic of the solve server: device-memory admission (no GPU needed)."""
from types import SimpleNamespace

import numpy as np

from paper_1711_07877_gb300.serve import Admission


def req(n, geometry=None):
    return SimpleNamespace(z=np.zeros((n, 2)), geometry=geometry)


def test_admission_fifo_with_skip_ahead():
    a = Admission(budget=1000, bytes_per_point=1.0, fixed_bytes=0)
    for n in (600, 500, 300, 100):
        a.push(req(n))
    r1, e1, _ = a.admit()
    assert len(r1.z) == 600 and e1 == 600
    r2, e2, _ = a.admit()          # 500 does not fit beside 600; 300 does
    assert len(r2.z) == 300
    r3, e3, _ = a.admit()
    assert len(r3.z) == 100
    assert a.admit() is None       # 500 waits
    a.release(e1)
    r4, _, _ = a.admit()
    assert len(r4.z) == 500
    assert a.in_use == 900 and a.running == 3


def test_admission_oversize_runs_alone():
    a = Admission(budget=10, bytes_per_point=1.0, fixed_bytes=0)
    a.push(req(50))
    a.push(req(60))
    r, e, _ = a.admit()
    assert len(r.z) == 50
    assert a.admit() is None       # nothing else while the oversize one runs
    a.release(e)
    r, e, _ = a.admit()
    assert len(r.z) == 60


def test_admission_estimate_grows_from_reports():
    a = Admission(budget=10**9, bytes_per_point=100.0, fixed_bytes=0)
    a.push(req(10))
    r, e, _ = a.admit()
    a.release(e, n_points=10, device_bytes=5000)
    assert a.bytes_per_point == 600.0
    assert a.estimate(10) == 6000


def test_fit_grid_scales_laplace():
    from paper_1711_07877_gb300 import serve, sbd as S
    d1, D1 = serve.fit_grid_scales(S.SBD_LAPLACE, 0.0, 0.0123, 7.9)
    assert D1 >= 7.9 and D1 < 7.9 * (1 + 1e-8)
    assert d1 <= 0.0123 and d1 > 0.0123 * 2 ** (-1 / 8)
    a = d1 / D1
    assert abs(np.log2(a) * 8 - round(np.log2(a) * 8)) < 1e-9
    d2, D2 = serve.fit_grid_scales(S.SBD_LAPLACE, 0.0, 0.0124, 8.0)
    assert abs(d2 / D2 - a) < 1e-15 * a * 8


def test_fit_grid_scales_helmholtz():
    from paper_1711_07877_gb300 import serve, sbd as S
    for kappa, diam, dmin in ((30.0, 7.9, 0.02), (61.3, 3.1, 0.004), (6.0, 8.5, 0.05)):
        d, D = serve.fit_grid_scales(S.SBD_HELMHOLTZ, kappa, dmin, diam)
        assert D >= diam and d <= min(dmin, 2 * np.pi / kappa)
        x = kappa * D
        # the plan's k' (first zero of Y0 >= kappa delta_max) has an index that is a multiple of 4
        k = 1
        while S.sbd_y0_root(k) < x:
            k += 1
        assert k % 4 == 0, (kappa, k)
        assert D < diam * 1.0 + 4.5 * np.pi / kappa
        a = d * kappa / S.sbd_y0_root(k)
        assert abs(np.log2(a) * 8 - round(np.log2(a) * 8)) < 1e-9


def test_fit_grid_caps_delta_min_at_a_wavelength():
    """Small N at large kappa delta_max: Theorem 1 gives delta_min of several wavelengths,
    which the Y0 fit cannot reach (conditioning floor); the server caps it."""
    from paper_1711_07877_gb300 import serve, sbd as S
    kappa, diam = 437.6 / 9.62, 9.62
    d, D = serve.fit_grid_scales(S.SBD_HELMHOLTZ, kappa, 0.4639, diam)
    assert d <= 2 * np.pi / kappa
    fit = S.sbd_offline_fit(S.SBD_HELMHOLTZ, kappa, d, D, 1e-6)
    assert fit["fit_err"] <= 1e-6 / 3


def test_resident_plans_are_reused_and_evicted_oldest_first():
    a = Admission(budget=1000, bytes_per_point=1.0, fixed_bytes=0, solve_bytes_per_point=0.1)
    a.push(req(300, "A"))
    r, e, ev = a.admit()
    assert ev == [] and e == 300
    a.release(e, 300, device_bytes=250, key="A", plan="plan-A")
    assert a.in_use == 250 and a.plan_of("A") == "plan-A"
    # same geometry: only solver workspace, the plan is marked busy
    a.push(req(300, "A"))
    a.push(req(300, "A"))
    r, e, ev = a.admit()
    assert e == 30 and ev == []
    assert a.admit() is None            # the second "A" waits for the plan
    a.release(e, key="A", plan="plan-A")
    r, e, ev = a.admit()
    assert e == 30
    a.release(e, key="A", plan="plan-A")
    # fill with B, then C needs room: the oldest idle resident (A) goes first
    a.push(req(400, "B"))
    r, e, ev = a.admit()
    a.release(e, 400, device_bytes=300, key="B", plan="plan-B")
    assert a.in_use == 550
    a.push(req(300))
    a.push(req(200))
    r, e, ev = a.admit()                # 300 fits beside the residents: 550 + 300 <= 1000
    assert ev == [] and len(r.z) == 300
    r2, e2, ev2 = a.admit()             # 200: needs eviction of A (oldest idle)
    assert [k for k, _ in ev2] == ["A"] and a.plan_of("A") is None
    assert a.in_use <= 1000


def test_resident_plan_in_use_is_never_evicted():
    a = Admission(budget=500, bytes_per_point=1.0, fixed_bytes=0, solve_bytes_per_point=0.1)
    a.push(req(400, "A"))
    r, e, _ = a.admit()
    a.release(e, 400, device_bytes=400, key="A", plan="plan-A")
    a.push(req(400, "A"))
    r, e, _ = a.admit()                 # A busy now
    a.push(req(300))
    assert a.admit() is None            # would need A's bytes, but A is in use
    a.release(e, key="A", plan="plan-A")
    r, e2, ev = a.admit()
    assert [k for k, _ in ev] == ["A"]


def test_second_request_waits_while_its_plan_is_built():
    a = Admission(budget=10_000, bytes_per_point=1.0, fixed_bytes=0, solve_bytes_per_point=0.1)
    a.push(req(300, "A"))
    a.push(req(300, "A"))
    a.push(req(100))
    r, e, _ = a.admit()
    r2, e2, _ = a.admit()
    assert r2.geometry is None               # the second "A" waits, the other one passes
    assert a.admit() is None
    a.release(e, 300, device_bytes=300, key="A", plan="pA")
    r3, e3, _ = a.admit()
    assert r3.geometry == "A" and e3 == 30   # reuses the resident plan
    # a failed build releases the key without a resident plan
    a.push(req(50, "B"))
    rb, eb, _ = a.admit()
    a.release(eb, key="B", keep=False)
    assert "B" not in a.building and a.plan_of("B") is None


# --- failure paths of the server, on the host: a stand-in backend raises the library's errors ----

import threading
import time

from paper_1711_07877_gb300 import sbd as S
from paper_1711_07877_gb300.serve import Request, Server


class FakeBackend:
    """Host stand-in for the device: plans fail with SBD_ENOMEM a set number of times, solves
    take a set time; records what happened."""

    def __init__(self, enomem=0, solve_s=0.0):
        self.enomem = enomem
        self.solve_s = solve_s
        self.plans = 0
        self.destroyed = 0
        self.lock = threading.Lock()

    def stream(self):
        return object()

    def free_bytes(self):
        return 10 ** 12

    def plan(self, req, stream, delta_min, delta_max, form, host_threads):
        with self.lock:
            self.plans += 1
            if self.enomem > 0:
                self.enomem -= 1
                raise S.SbdError(S.SBD_ENOMEM, "sbd_plan", "out of memory: cudaMallocAsync")
        return object(), {"plan_seconds": 1e-3, "device_bytes": 1000 * len(req.z)}

    def solve(self, plan, req, stream, tol, restart, max_iter):
        time.sleep(self.solve_s)
        return np.zeros_like(req.b), 3, 1e-7

    def synchronize(self, stream):
        pass

    def destroy(self, plan, stream):
        with self.lock:
            self.destroyed += 1

    def destroy_now(self, plan):
        self.destroy(plan, None)


def mk(i, n=100, deadline=None):
    return Request(rid=i, z=np.zeros((n, 2)), b=np.ones(n), kind=S.SBD_LAPLACE, kappa=0.0, delta_min=0.1,
                   eps=1e-6, deadline_s=deadline)


def test_out_of_memory_requeues_then_succeeds():
    be = FakeBackend(enomem=2)
    srv = Server(slots=1, hbm_budget=10 ** 9, backend=be, fit_grid=False)
    r = mk(0)
    srv.submit(r)
    assert srv.drain([r], timeout_s=10)
    assert r.error is None and r.attempts == 2 and srv.requeued == 2
    assert be.plans == 3
    assert srv.adm.bytes_per_point >= 8000.0 * 1.5 ** 2   # the estimate grew by half per retry


def test_out_of_memory_fails_after_the_retries():
    be = FakeBackend(enomem=10)
    srv = Server(slots=1, hbm_budget=10 ** 9, backend=be, fit_grid=False, retries=3)
    r = mk(0)
    srv.submit(r)
    assert srv.drain([r], timeout_s=10)
    assert r.error is not None and "out of memory" in r.error and r.attempts == 3
    assert be.plans == 4 and srv.adm.running == 0 and srv.adm.in_use == 0


def test_deadline_drops_queued_requests_and_marks_late_ones():
    be = FakeBackend(solve_s=0.3)
    srv = Server(slots=1, hbm_budget=10 ** 9, backend=be, fit_grid=False)
    slow = mk(0, deadline=0.1)          # admitted at once, finishes after its deadline: late
    queued = mk(1, deadline=0.1)        # waits behind it past its deadline: dropped
    free = mk(2)                        # no deadline: served after the slow one
    for r in (slow, queued, free):
        srv.submit(r)
    assert srv.drain([slow, queued, free], timeout_s=10)
    assert slow.error is None and slow.late
    assert queued.error is not None and "deadline" in queued.error and srv.dropped == 1
    assert free.error is None and not free.late
    assert be.destroyed == 2            # the two solved requests released their plans


class FakeBatchedBackend(FakeBackend):
    """Stand-in whose solves ask for `steps` matvecs through the scheduler."""

    def __init__(self, steps=20):
        super().__init__()
        self.steps = steps
        self.batch_sizes = []

    def solve_batched(self, plan, req, stream, tol, restart, max_iter, sched):
        for _ in range(self.steps):
            sched.submit(plan, None, None, None)
            time.sleep(0.0005)                 # the session's own work between matvecs
        return np.zeros_like(req.b), self.steps, 1e-7

    def matvec_batched(self, tickets, stream):
        assert len({id(t.plan) for t in tickets}) == len(tickets)   # distinct plans per batch
        self.batch_sizes.append(len(tickets))
        return None


def test_scheduler_merges_the_solves_matvecs():
    be = FakeBatchedBackend(steps=20)
    srv = Server(slots=4, hbm_budget=10 ** 9, backend=be, fit_grid=False, batch_matvecs=True)
    reqs = [mk(i) for i in range(8)]
    for r in reqs:
        srv.submit(r)
    assert srv.drain(reqs, timeout_s=30)
    assert all(r.error is None and r.iterations == 20 for r in reqs)
    assert srv.sched.matvecs == 8 * 20 == sum(be.batch_sizes)
    assert srv.sched.batches < srv.sched.matvecs / 2          # most launches carry several solves
    assert max(be.batch_sizes) <= 4                           # at most one matvec per solving worker
