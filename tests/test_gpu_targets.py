"""GPU parity of plans with separate targets and sources (Sec. 7.1, Table 2) against the oracle.

sbd_plan_st fits the union of the two sets, so the oracle's make_plan_st picks the same P and
circle sizes (asserted first); then
  * FP64 form vs the oracle SBD (sbd_matvec_st): rel-L2 <= 1e-10 with the transforms at 1e-13;
  * FP32 form vs the oracle SBD: rel-L2 and max|dq| / max|q| <= 1e-6 (the FP32 bound of
    test_gpu_fp32_parity.py);
  * both forms vs the oracle's direct sum: max |q - q*| <= eps sum|f| (Sec. 1 output bound);
  * the rectangular D: identical pairs (bit-exact), values within 1e-11 of the oracle's
    plane-wave sum taken with the plan's own weights;
  * with targets = sources, the plan equals sbd_plan's up to the summation order.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sbd_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def plan_st(S, x, y, kind, dmin, eps, kappa=0.0, form=0, nufft_tol=0.0, max_nrhs=1, flags=0):
    opt = S.make_options(form=form, nufft_tol=nufft_tol, max_nrhs=max_nrhs, flags=flags)
    p = S.sbd_plan_st(dev(x), len(x), dev(y), len(y), S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE,
                      kappa, dmin, eps, opt)
    torch.cuda.synchronize()
    return p


def run(S, p, f, n_out, nrhs=1, fn=None):
    ft = dev(f)
    shape = (nrhs, n_out) if nrhs > 1 else (n_out,)
    q = torch.empty(shape, dtype=ft.dtype, device="cuda")
    (fn or S.sbd_matvec)(p, ft, q, nrhs)
    torch.cuda.synchronize()
    return q.cpu().numpy()


def same_fit(S, p, pl):
    info = S.sbd_plan_info(p)
    assert info["P"] == pl.P and np.array_equal(S.sbd_plan_export(p)["M"], pl.M)
    assert info["separate_targets"] == 1


@pytest.fixture(scope="module")
def lap_st():
    x = W.square_points(500, 41)
    y = W.square_points(700, 42)
    f = W.rhs(700, 43)
    dmin = 0.06
    pl = O.make_plan_st(x, y, "laplace", dmin, 1e-6)
    return x, y, f, dmin, pl, O.sbd_matvec_st(pl, f), O.direct_sum_st(x, y, f, "laplace")


def test_fp64_matches_oracle_sbd_laplace(S, lap_st):
    x, y, f, dmin, pl, q_sbd, q_dir = lap_st
    p = plan_st(S, x, y, "laplace", dmin, 1e-6, form=0, nufft_tol=1e-13)
    try:
        same_fit(S, p, pl)
        info = S.sbd_plan_info(p)
        assert (info["n_points"], info["n_targets"]) == (700, 500)
        q = run(S, p, f, 500)
        assert np.linalg.norm(q - q_sbd) / np.linalg.norm(q_sbd) <= 1e-10
        assert np.max(np.abs(q - q_dir)) <= 1e-6 * np.abs(f).sum()
        # the halves add up, and the transforms take sources forward and targets backward
        far = run(S, p, f, 500, fn=S.sbd_far)
        close = run(S, p, f, 500, fn=S.sbd_close)
        assert np.max(np.abs(far + close - q)) <= 1e-11 * np.abs(q).max()
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("flags", [0, 16])
def test_fp32_matches_oracle_sbd_laplace(S, lap_st, flags):
    x, y, f, dmin, pl, q_sbd, q_dir = lap_st
    p = plan_st(S, x, y, "laplace", dmin, 1e-6, form=1, flags=flags)
    try:
        same_fit(S, p, pl)
        q = run(S, p, f, 500)
        rel = np.linalg.norm(q - q_sbd) / np.linalg.norm(q_sbd)
        worst = np.max(np.abs(q - q_sbd)) / np.max(np.abs(q_sbd))
        assert rel <= 1e-6 and worst <= 1e-6, (rel, worst)
        assert np.max(np.abs(q - q_dir)) <= 1e-6 * np.abs(f).sum()
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("form", [0, 1])
def test_helmholtz_matches_oracle_sbd(S, form):
    x = W.square_points(300, 44)
    y = W.square_points(450, 45)
    f = W.rhs(450, 46, complex_valued=True)
    kappa, dmin = 30.0, 0.08
    pl = O.make_plan_st(x, y, "helmholtz", dmin, 1e-6, kappa=kappa)
    q_sbd = O.sbd_matvec_st(pl, f)
    p = plan_st(S, x, y, "helmholtz", dmin, 1e-6, kappa=kappa, form=form, nufft_tol=1e-13 if form == 0 else 0.0)
    try:
        same_fit(S, p, pl)
        q = run(S, p, f, 300)
        rel = np.linalg.norm(q - q_sbd) / np.linalg.norm(q_sbd)
        assert rel <= (1e-10 if form == 0 else 1e-6), rel
        q_dir = O.direct_sum_st(x, y, f, "helmholtz", kappa)
        assert np.max(np.abs(q - q_dir)) <= 1e-6 * np.abs(f).sum()
    finally:
        S.sbd_destroy(p)


def test_rectangular_close_matrix_matches_oracle(S, lap_st):
    import dataclasses
    x, y, f, dmin, pl, _, _ = lap_st
    p = plan_st(S, x, y, "laplace", dmin, 1e-6)
    try:
        ex = S.sbd_plan_export(p)
        info = S.sbd_plan_info(p)
        xi = [np.zeros((1, 2))] + [O.circle_nodes(float(r), int(M)) for r, M in zip(ex["radius"], ex["M"])]
        om = [np.array([complex(info["w0_re"], info["w0_im"])])] + [
            np.full(int(M), w, dtype=np.complex128) for M, w in zip(ex["M"], ex["weight"])]
        pl2 = dataclasses.replace(pl, xi=np.concatenate(xi), omega=np.concatenate(om), D_st=None)
        rows, cols, vals = O.close_matrix_st(pl2)
        rowptr, col, val = S.sbd_close_export(p)
        assert len(rowptr) == 501 and rowptr[-1] == len(rows) == info["nnz"]
        got = {}
        for k in range(500):
            for j in range(rowptr[k], rowptr[k + 1]):
                got[(k, int(col[j]))] = val[j]
        want = {(int(r), int(c)): v for r, c, v in zip(rows, cols, vals)}
        assert set(got) == set(want)
        scale = max(abs(v) for v in want.values())
        assert max(abs(got[k] - want[k]) for k in want) <= 1e-11 * scale
    finally:
        S.sbd_destroy(p)


def test_equal_sets_reduce_to_the_square_plan(S):
    z = W.disk_points(600, 47)
    f = W.rhs(600, 48)
    dmin = math.sqrt(20 / 600)
    p1 = S.sbd_plan(dev(z), 600, S.SBD_LAPLACE, 0.0, dmin, 1e-6, S.make_options(form=0))
    p2 = plan_st(S, z, z, "laplace", dmin, 1e-6, form=0)
    try:
        assert S.sbd_plan_info(p2)["n_coincident"] == 600          # each target is its own source
        q1, q2 = run(S, p1, f, 600), run(S, p2, f, 600)
        assert np.max(np.abs(q1 - q2)) <= 1e-12 * np.abs(q1).max()
    finally:
        S.sbd_destroy(p1)
        S.sbd_destroy(p2)


def test_coincident_pairs_batches_and_errors(S, lap_st):
    x, y, f, dmin, pl, _, _ = lap_st
    x2 = x.copy()
    x2[:4] = y[10:14]                                              # four targets sit on sources
    F = np.stack([f, W.rhs(700, 49), W.rhs(700, 50)])
    p = plan_st(S, x2, y, "laplace", dmin, 1e-6, form=1, max_nrhs=3)
    try:
        assert S.sbd_plan_info(p)["n_coincident"] == 4
        qb = run(S, p, F, 500, nrhs=3)
        for r in range(3):
            qs = run(S, p, F[r], 500)
            assert np.max(np.abs(qb[r] - qs)) <= 2e-6 * np.abs(qs).max()
            qd = O.direct_sum_st(x2, y, F[r], "laplace")
            assert np.max(np.abs(qb[r] - qd)) <= 1e-6 * np.abs(F[r]).sum()
        with pytest.raises(S.SbdError) as e:                        # not a square system
            S.sbd_gmres(p, dev(f[:500]), torch.zeros(500, dtype=torch.float64, device="cuda"))
        assert e.value.code == S.SBD_EINVAL
    finally:
        S.sbd_destroy(p)
    for args in [(0, 5, dev(y), 700), (dev(x), 0, dev(y), 700), (dev(x), 500, 0, 700)]:
        with pytest.raises(S.SbdError) as e:
            S.sbd_plan_st(*args, S.SBD_LAPLACE, 0.0, dmin, 1e-6)
        assert e.value.code == S.SBD_EINVAL


def test_table2_workload_sampled_against_direct_sum(S):
    """The Table 2 setting at N = 3 10^5 targets and sources (FP32 form, tuned): 200 sampled
    targets against the oracle's direct sum over all sources."""
    wl = W.laplace_square_st(300_000, 6, 1e-6)
    p = plan_st(S, wl.z, wl.y, "laplace", wl.delta_min, wl.eps, form=1)
    try:
        S.sbd_tune(p, 1)
        q = run(S, p, wl.f, len(wl.z))
        idx = np.random.default_rng(12).choice(len(wl.z), 200, replace=False)
        qd = O.direct_sum_st(wl.z, wl.y, wl.f, "laplace", targets=idx, chunk=32)
        assert np.max(np.abs(q[idx] - qd)) <= wl.eps * np.abs(wl.f).sum()
        assert np.linalg.norm(q[idx] - qd) / np.linalg.norm(qd) <= 1e-6
    finally:
        S.sbd_destroy(p)
