"""Host logic of the solve server: device-memory admission (no GPU needed)."""
from types import SimpleNamespace

import numpy as np

from paper_1711_07877_gb300.serve import Admission


def req(n):
    return SimpleNamespace(z=np.zeros((n, 2)))


def test_admission_fifo_with_skip_ahead():
    a = Admission(budget=1000, bytes_per_point=1.0, fixed_bytes=0)
    for n in (600, 500, 300, 100):
        a.push(req(n))
    r1, e1 = a.admit()
    assert len(r1.z) == 600 and e1 == 600
    r2, e2 = a.admit()             # 500 does not fit beside 600; 300 does
    assert len(r2.z) == 300
    r3, e3 = a.admit()
    assert len(r3.z) == 100
    assert a.admit() is None       # 500 waits
    a.release(e1)
    r4, _ = a.admit()
    assert len(r4.z) == 500
    assert a.in_use == 900 and a.running == 3


def test_admission_oversize_runs_alone():
    a = Admission(budget=10, bytes_per_point=1.0, fixed_bytes=0)
    a.push(req(50))
    a.push(req(60))
    r, e = a.admit()
    assert len(r.z) == 50
    assert a.admit() is None       # nothing else while the oversize one runs
    a.release(e)
    r, e = a.admit()
    assert len(r.z) == 60


def test_admission_estimate_grows_from_reports():
    a = Admission(budget=10**9, bytes_per_point=100.0, fixed_bytes=0)
    a.push(req(10))
    r, e = a.admit()
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
