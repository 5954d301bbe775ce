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
