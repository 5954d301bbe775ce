"""GPU parity of the FP32 form against the oracle SBD, element by element.

The oracle SBD (Sec. 1 on-line part by direct exponential sums, D by the plane-wave sum
of Eq. defD) and the GPU plan pick the same P and circle sizes M_p (asserted first), so
the difference between the two is the error of the fast transforms and the FP32
rounding only, without the fit and quadrature error that a comparison with the direct
sum also contains.

FP32 bound (rel-L2 and max|dq| / max|q| <= 1e-6, the accuracy the FP32 form is specified
at): the FP32 form runs each type-3 transform at the tolerance 3e-7 (its floor; relative
to sum|omega| sum|f|) with float32 window weights and grid sums (unit roundoff 6e-8,
growing like sqrt(log n) through the FFT passes), while D f, the xi = 0 term and the
final sums are float64 (SBD_FLAG_NEAR_FP32 adds float32 rounding of D's values and of f,
about 6e-8 of the near term).  The measured errors sit near 1e-7.

Where the oracle's D would cost too much (N = 6000: ~10^5 near pairs x 3 10^4 nodes),
the far part alone (sbd_far) is compared with the oracle's far part.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sbd_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_REL = 1e-6


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_07877_gb300 import build
    build.build_library()
    import paper_1711_07877_gb300 as pkg
    return pkg


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def plan(S, z, kind, dmin, eps, kappa=0.0, flags=0):
    opt = S.make_options(form=S.SBD_FORM_FP32, flags=flags)
    p = S.sbd_plan(dev(z), len(z), S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE, kappa, dmin, eps, opt)
    torch.cuda.synchronize()
    return p


def run(S, p, f, fn=None):
    ft = dev(f)
    q = torch.empty_like(ft)
    (fn or S.sbd_matvec)(p, ft, q, 1)
    torch.cuda.synchronize()
    return q.cpu().numpy()


def same_fit(S, p, pl):
    info = S.sbd_plan_info(p)
    assert info["P"] == pl.P and np.array_equal(S.sbd_plan_export(p)["M"], pl.M), "plans differ: no parity compare"


def assert_close(q, want, bound=FP32_REL):
    rel = np.linalg.norm(q - want) / np.linalg.norm(want)
    worst = np.max(np.abs(q - want)) / np.max(np.abs(want))
    assert rel <= bound and worst <= bound, (rel, worst)
    return rel, worst


@pytest.fixture(scope="module")
def config1():
    wl = W.laplace_disk(2000, 1, 1e-6)
    pl = O.make_plan(wl.z, "laplace", wl.delta_min, wl.eps)
    return wl, pl, O.sbd_matvec(pl, wl.f), O.direct_sum(wl.z, wl.f, "laplace")


# flags: default (ES windows, automatic oversampling), near field in float32 (16),
# spreading oversampling forced to 2 (4) or 1.5 (8), Gaussian node window (1)
@pytest.mark.parametrize("flags", [0, 16, 4, 8, 1])
def test_fp32_matvec_matches_oracle_sbd_config1(S, config1, flags):
    wl, pl, q_sbd, q_dir = config1
    p = plan(S, wl.z, "laplace", wl.delta_min, wl.eps, flags=flags)
    try:
        same_fit(S, p, pl)
        q = run(S, p, wl.f)
        assert_close(q, q_sbd)
        assert np.linalg.norm(q - q_dir) / np.linalg.norm(q_dir) <= FP32_REL
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("acc", [3, 4])
@pytest.mark.parametrize("sched", [0, 1])
def test_fp32_binned_node_kernel_matches_oracle_far_part(S, sched, acc):
    """The binned node kernels (variants acc 3 and 4, the ones the tuner picks from at N = 10^6)
    against the oracle's far part by direct sums, N = 6000 in the disk."""
    wl = W.laplace_disk(6000, 51, 1e-6)
    pl = O.make_plan(wl.z, "laplace", wl.delta_min, wl.eps)
    p = plan(S, wl.z, "laplace", wl.delta_min, wl.eps)
    try:
        same_fit(S, p, pl)
        assert S.sbd_plan_info(p)["node_binned"] == 1
        S.sbd_set_tuning(p, acc, sched, 0)
        far = run(S, p, wl.f, fn=S.sbd_far)
        want = O.far_part(pl, wl.f).real
        assert_close(far, want)
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("flags", [0, 16])
def test_fp32_helmholtz_matches_oracle_sbd(S, flags):
    z = W.disk_points(600, 21)
    f = W.rhs(600, 22, complex_valued=True)
    dmin, kappa = math.sqrt(20 / 600), 25.0
    pl = O.make_plan(z, "helmholtz", dmin, 1e-6, kappa=kappa)
    q_sbd = O.sbd_matvec(pl, f)
    p = plan(S, z, "helmholtz", dmin, 1e-6, kappa=kappa, flags=flags)
    try:
        same_fit(S, p, pl)
        assert_close(run(S, p, f), q_sbd)
    finally:
        S.sbd_destroy(p)


def test_near_fp32_flag_needs_fp32_form(S):
    z = W.disk_points(100, 3)
    with pytest.raises(S.SbdError) as e:
        S.sbd_plan(dev(z), 100, S.SBD_LAPLACE, 0.0, 0.3, 1e-6, S.make_options(form=S.SBD_FORM_FP64, flags=16))
    assert e.value.code == S.SBD_EINVAL


def test_fp32_form_keeps_close_matrix_in_fp64(S):
    """Without SBD_FLAG_NEAR_FP32 the FP32 form's D holds float64 values: identical to the
    FP64 form's D entry by entry (same points, delta_min and fit); with the flag the values
    are those rounded to float32."""
    z = W.disk_points(500, 7)
    dmin = math.sqrt(20 / 500)
    p64 = S.sbd_plan(dev(z), 500, S.SBD_LAPLACE, 0.0, dmin, 1e-6, S.make_options(form=S.SBD_FORM_FP64))
    p32 = plan(S, z, "laplace", dmin, 1e-6)
    p32n = plan(S, z, "laplace", dmin, 1e-6, flags=16)
    try:
        r64, c64, v64 = S.sbd_close_export(p64)
        r32, c32, v32 = S.sbd_close_export(p32)
        r3n, c3n, v3n = S.sbd_close_export(p32n)
        assert np.array_equal(r64, r32) and np.array_equal(c64, c32) and np.array_equal(c64, c3n)
        assert np.array_equal(v64, v32)
        assert np.array_equal(v3n, v64.astype(np.float32).astype(np.float64))
    finally:
        for p in (p64, p32, p32n):
            S.sbd_destroy(p)
