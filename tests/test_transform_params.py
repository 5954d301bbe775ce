"""Host sizing of the type-3 transforms (sbd_transform_params, no GPU): the rules the plan
follows for the spreading window, its oversampling and the grid sizes, checked against their
definitions (Sec. 1 steps (i)-(iii) realised by window spreading + FFT + node windows)."""
import math

import numpy as np
import pytest

import workloads as W

S = pytest.importorskip("paper_1711_07877_gb300.sbd")

EPS = 1e-6


def _even(x):
    return x + (x & 1)


def _good(n):
    """Smallest even 5-smooth integer >= n."""
    while True:
        m = n + (n & 1)
        k = m
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        n = m + 2


@pytest.fixture(scope="module")
def curves():
    n = 200_000
    wl = W.laplace_curves(n, 2, EPS)
    c = 0.5 * (wl.z.min(axis=0) + wl.z.max(axis=0))
    half = float(np.max(wl.z.max(axis=0) - c))
    return n, wl.meta["delta_max"], half


def _params(curves, alpha=0.0, form=1, flags=0, kind=0, kappa=0.0):
    n, dmax, half = curves
    dmin = W.theorem1_delta_min(n, EPS, dmax, alpha)
    return S.sbd_transform_params(kind, kappa, dmin, dmax, EPS, n, half, S.make_options(form=form, flags=flags)), dmin


def test_sizes_follow_their_definitions(curves):
    n, dmax, half = curves
    t, dmin = _params(curves)
    fit = S.sbd_offline_fit(S.SBD_LAPLACE, 0.0, dmin, dmax, EPS)
    assert fit["P"] == t["P"] and int(np.sum(fit["M"])) == t["n_xi"]
    s_max = fit["rho"][-1] / dmax
    # the oversampling rule: cells per point of the grid at 2 past 60 -> 1.25, past 20 -> 1.5, else 2
    cells = (2 * half * 2 * s_max / math.pi) ** 2 / n
    sig = 1.25 if cells > 60 else 1.5 if cells > 20 else 2.0
    assert cells > 60 and t["sigma_s"] == sig and t["spread_window"] == 1   # a large grid per point at alpha = 0
    assert t["nufft_tol"] == pytest.approx(3e-7)            # the FP32 floor
    assert t["stencil_x"] == _even(math.ceil(math.log(10 / 3e-7) / (math.pi * math.sqrt(1 - 1 / sig))))
    assert t["stencil_k"] == _even(math.ceil(-math.log10(3e-7)))
    # h = pi / (sigma S), S = largest circle radius rho_P / delta_max (Laplace: scale delta_max)
    assert t["h"] == pytest.approx(math.pi / (sig * s_max), rel=1e-12)
    assert t["grid_x"] == _good(math.ceil(2 * half / t["h"]) + t["stencil_x"] + 4)
    assert t["fft_n"] == 2 * t["grid_x"]
    assert t["deta"] == pytest.approx(2 * math.pi / (t["fft_n"] * t["h"]), rel=1e-12)
    # the stored frequency grid holds every node (|xi| <= S) with its stencil, inside the FFT length
    assert t["grid_k"] >= 2 * s_max / t["deta"] + t["stencil_k"] + 4 - 1e-9
    assert t["grid_k"] <= t["fft_n"] and t["grid_k"] % 2 == 0


def test_oversampling_choice_and_flags(curves):
    auto, _ = _params(curves)
    two, _ = _params(curves, flags=S.SBD_FLAG_SPREAD_SIGMA_2)
    one5, _ = _params(curves, flags=S.SBD_FLAG_SPREAD_SIGMA_15)
    assert two["sigma_s"] == 2.0 and two["stencil_x"] == 8
    assert one5["sigma_s"] == 1.5 and one5["stencil_x"] == 10
    assert auto["sigma_s"] == 1.25 and auto["stencil_x"] == 14
    # the smaller spreading grid, the same frequency grid (it is set by S and the point extent)
    assert 1.2 < two["grid_x"] / one5["grid_x"] < 1.45 and 1.1 < one5["grid_x"] / auto["grid_x"] < 1.3
    assert abs(two["grid_k"] - auto["grid_k"]) <= 0.05 * two["grid_k"]
    # few cells per point (alpha = 1/8: larger delta_min, fewer circles, a coarser grid): oversampling 2,
    # and the grid at 2 indeed holds fewer than ~20 cells per point
    coarse, _ = _params(curves, alpha=0.125)
    n, half = curves[0], curves[2]
    assert coarse["sigma_s"] == 2.0 and (2 * half / coarse["h"]) ** 2 < 20 * n
    assert (2 * half / two["h"]) ** 2 > 20 * n             # and at alpha = 0 more
    # Gaussian spreading: oversampling 2, its own width rule
    g, _ = _params(curves, flags=S.SBD_FLAG_GAUSSIAN_SPREAD)
    assert g["sigma_s"] == 2.0 and g["spread_window"] == 0
    assert g["stencil_x"] == _even(math.ceil(3 / math.pi * math.log(0.1 / 3e-7)))
    # FP64 form: the transform tolerance is eps / (6 sum |w|), not floored at 3e-7; the widths follow
    # the same rules at that tolerance
    f64, _ = _params(curves, form=0)
    tol = f64["nufft_tol"]
    assert tol < 3e-7
    assert f64["stencil_k"] == _even(math.ceil(-math.log10(tol)))
    sig = f64["sigma_s"]
    assert f64["stencil_x"] == _even(math.ceil(math.log(10 / tol) / (math.pi * math.sqrt(1 - 1 / sig))))
    opt = S.make_options(form=0, nufft_tol=1e-13)
    n, dmax, half = curves
    t13 = S.sbd_transform_params(0, 0.0, W.theorem1_delta_min(n, EPS, dmax), dmax, EPS, n, half, opt)
    assert t13["nufft_tol"] == 1e-13 and t13["stencil_k"] == 14 and t13["stencil_x"] > f64["stencil_x"]


def test_helmholtz_adds_the_j0_circle(curves):
    n, dmax, half = curves
    t, _ = _params(curves, kind=S.SBD_HELMHOLTZ, kappa=500.0 / dmax)
    assert t["n_circles"] == t["P"] + 1
    assert t["grid_k"] <= t["fft_n"]


def test_invalid_arguments(curves):
    n, dmax, half = curves
    dmin = W.theorem1_delta_min(n, EPS, dmax)
    bad = [
        dict(flags=S.SBD_FLAG_SPREAD_SIGMA_2 | S.SBD_FLAG_SPREAD_SIGMA_15),
        dict(flags=S.SBD_FLAG_GAUSSIAN_SPREAD | S.SBD_FLAG_SPREAD_SIGMA_15),
        dict(flags=1 << 20),
    ]
    for kw in bad:
        with pytest.raises(S.SbdError) as e:
            S.sbd_transform_params(0, 0.0, dmin, dmax, EPS, n, half, S.make_options(form=1, **kw))
        assert e.value.code == S.SBD_EINVAL
    for args in [(0, 0.0, dmin, dmax, EPS, 0, half), (0, 0.0, dmin, dmax, EPS, n, 0.0),
                 (0, 0.0, dmax, dmax, EPS, n, half), (0, 0.0, dmin, dmax, 1e-12, n, half),
                 (1, 0.0, dmin, dmax, EPS, n, half)]:
        with pytest.raises(S.SbdError) as e:
            S.sbd_transform_params(*args)
        assert e.value.code == S.SBD_EINVAL
