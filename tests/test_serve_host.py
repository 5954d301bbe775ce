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
