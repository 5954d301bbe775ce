"""GPU parity of the uniform-grid multiplier variant (SBD_FLAG_UNIFORM_GRID) against the oracle.

The variant's operator is the SBD without its circle quadrature: G_fit beyond delta_min and G on
the near pairs, which the oracle computes by definition (series_matvec, direct O(N^2 P) sums).
The plan and the oracle pick the same P (asserted first).  Bars:
  * FP64 form vs series_matvec: rel-L2 <= 1e-10 with the transforms and the window at 1e-13;
  * FP32 form vs series_matvec: rel-L2 and max|dq| / max|q| <= 1e-6 (the FP32 bound);
  * both vs the direct sum: max |q - q*| <= eps sum|f| (Sec. 1 bound), rel-L2 <= 1e-6;
  * D = G - G_fit on the near pairs: pairs bit-exact, values within 1e-11 of max|D|.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sbd_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UNIFORM = 32


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


def plan(S, z, kind, dmin, eps, kappa=0.0, form=0, nufft_tol=0.0, max_nrhs=1, flags=UNIFORM):
    opt = S.make_options(form=form, nufft_tol=nufft_tol, max_nrhs=max_nrhs, flags=flags)
    p = S.sbd_plan(dev(z), len(z), S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE, kappa, dmin, eps, opt)
    torch.cuda.synchronize()
    return p


def run(S, p, f, nrhs=1):
    ft = dev(f)
    q = torch.empty_like(ft)
    S.sbd_matvec(p, ft, q, nrhs)
    torch.cuda.synchronize()
    return q.cpu().numpy()


@pytest.fixture(scope="module")
def config1():
    wl = W.laplace_disk(2000, 1, 1e-6)
    pl = O.make_plan(wl.z, "laplace", wl.delta_min, wl.eps)
    return wl, pl, O.series_matvec(pl, wl.f), O.direct_sum(wl.z, wl.f, "laplace")


@pytest.mark.parametrize("form", [0, 1])
def test_uniform_matches_oracle_series_laplace(S, config1, form):
    wl, pl, q_ser, q_dir = config1
    p = plan(S, wl.z, "laplace", wl.delta_min, wl.eps, form=form, nufft_tol=1e-13 if form == 0 else 0.0)
    try:
        info = S.sbd_plan_info(p)
        assert info["uniform_grid"] == 1 and info["P"] == pl.P and info["n_records"] == 0
        q = run(S, p, wl.f)
        rel = np.linalg.norm(q - q_ser) / np.linalg.norm(q_ser)
        worst = np.max(np.abs(q - q_ser)) / np.max(np.abs(q_ser))
        bound = 1e-10 if form == 0 else 1e-6
        assert rel <= bound and worst <= bound * (10 if form == 0 else 1), (rel, worst)
        assert np.max(np.abs(q - q_dir)) <= wl.eps * np.abs(wl.f).sum()
        assert np.linalg.norm(q - q_dir) / np.linalg.norm(q_dir) <= 1e-6
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("form", [0, 1])
def test_uniform_matches_oracle_series_helmholtz(S, form):
    z = W.disk_points(600, 71)
    f = W.rhs(600, 72, complex_valued=True)
    dmin, kappa = math.sqrt(20 / 600), 25.0
    pl = O.make_plan(z, "helmholtz", dmin, 1e-6, kappa=kappa)
    q_ser = O.series_matvec(pl, f)
    p = plan(S, z, "helmholtz", dmin, 1e-6, kappa=kappa, form=form, nufft_tol=1e-13 if form == 0 else 0.0)
    try:
        assert S.sbd_plan_info(p)["P"] == pl.P
        q = run(S, p, f)
        rel = np.linalg.norm(q - q_ser) / np.linalg.norm(q_ser)
        assert rel <= (1e-10 if form == 0 else 1e-6), rel
        assert np.max(np.abs(q - O.direct_sum(z, f, "helmholtz", kappa))) <= 1e-6 * np.abs(f).sum()
    finally:
        S.sbd_destroy(p)


def test_uniform_close_matrix_is_g_minus_the_series(S):
    """D against G - G_fit by the oracle's series_kernel evaluated with the plan's own exported
    coefficients (two independent fits differ along the Gram matrix's small eigenvectors, Sec. 3.3)."""
    import dataclasses
    z = W.disk_points(500, 73)
    dmin = math.sqrt(20 / 500)
    pl = O.make_plan(z, "laplace", dmin, 1e-6)
    p = plan(S, z, "laplace", dmin, 1e-6)
    try:
        ex = S.sbd_plan_export(p)
        P = S.sbd_plan_info(p)["P"]
        pl = dataclasses.replace(pl, P=P, rho=ex["rho"][:P], alpha=ex["alpha"][:P], C=O.normalisation_C(ex["rho"][:P]))
        rowptr, col, val = S.sbd_close_export(p)
        k, l = O.near_pairs(z, dmin)
        r = np.hypot(*(z[k] - z[l]).T)
        want = {(int(a), int(b)): v for a, b, v in
                zip(k, l, O.kernel_G(r, "laplace") - O.series_kernel(pl, r))}
        g0 = O.series_kernel(pl, 0.0)[0]
        for i in range(500):
            want[(i, i)] = -g0
        got = {}
        for i in range(500):
            for j in range(rowptr[i], rowptr[i + 1]):
                got[(i, int(col[j]))] = val[j]
        assert set(got) == set(want)
        scale = max(abs(v) for v in want.values())
        assert max(abs(got[q] - want[q]) for q in want) <= 1e-11 * scale
    finally:
        S.sbd_destroy(p)


def test_uniform_batches_and_argument_rules(S):
    z = W.disk_points(700, 74)
    dmin = math.sqrt(20 / 700)
    F = np.stack([W.rhs(700, 75 + r) for r in range(3)])
    p = plan(S, z, "laplace", dmin, 1e-6, form=1, max_nrhs=3)
    try:
        qb = run(S, p, F, nrhs=3)
        for r in range(3):
            qs = run(S, p, F[r])
            assert np.max(np.abs(qb[r] - qs)) <= 2e-6 * np.abs(qs).max()
        # the batched call runs the multiplication on the plan's stream
        q2 = torch.empty(700, dtype=torch.float64, device="cuda")
        zt = W.curve_points(900, 76)
        p2 = S.sbd_plan(dev(zt), 900, S.SBD_LAPLACE, 0.0, float(np.sqrt(20 / 900)), 1e-6,
                        S.make_options(form=1))
        try:
            f2 = dev(W.rhs(900, 77))
            q3 = torch.empty_like(f2)
            S.sbd_matvec_batched([p, p2], [dev(F[0]), f2], [q2, q3])
            assert S.sbd_device_status() == S.SBD_OK
            assert np.max(np.abs(q2.cpu().numpy() - run(S, p, F[0]))) <= 2e-6 * np.abs(qb[0]).max()
        finally:
            S.sbd_destroy(p2)
        with pytest.raises(S.SbdError) as e:       # no quadrature nodes to transform to
            S.sbd_nufft_minus(p, dev(F[0] + 0j), torch.empty(10, dtype=torch.complex128, device="cuda"))
        assert e.value.code == S.SBD_ENOTSUP
    finally:
        S.sbd_destroy(p)
    for flags in (UNIFORM | 1, UNIFORM | 2):       # the Gaussian windows are not part of the variant
        with pytest.raises(S.SbdError) as e:
            plan(S, z, "laplace", dmin, 1e-6, flags=flags)
        assert e.value.code == S.SBD_EINVAL


def test_uniform_curves_sampled_against_direct_sum(S):
    """Laplace on the curve family, N = 3 10^5, FP32 form: 300 sampled outputs against the
    oracle's direct sum over all sources."""
    wl = W.laplace_curves(300_000, 2, 1e-6)
    p = plan(S, wl.z, "laplace", wl.delta_min, wl.eps, form=1)
    try:
        S.sbd_tune(p, 1)
        q = run(S, p, wl.f)
        idx = np.random.default_rng(14).choice(len(wl.z), 300, replace=False)
        qd = O.direct_sum(wl.z, wl.f, "laplace", targets=idx, chunk=32)
        assert np.max(np.abs(q[idx] - qd)) <= wl.eps * np.abs(wl.f).sum()
        assert np.linalg.norm(q[idx] - qd) / np.linalg.norm(qd) <= 1e-6
    finally:
        S.sbd_destroy(p)
