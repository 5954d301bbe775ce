"""GPU: delta_min chosen by measurement (sbd_plan_balanced).

Theorem 1 sets delta_min = a delta_max with a = |log eps|^(2/3) / N^(2/3 - alpha) for any
alpha in [0, 1/6]; the library plans each candidate alpha, times it and keeps the fastest.
Whatever it keeps, the output bound of Sec. 1 (|q - q*| <= eps sum|f|) must hold, and the
kept plan must be the one sbd_plan builds at that delta_min.  Expected values come from the
oracle's direct sum only.
"""
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


def run(S, p, f, nrhs=1):
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    q = torch.empty_like(ft)
    S.sbd_matvec(p, ft, q, nrhs)
    torch.cuda.synchronize()
    return q.cpu().numpy()


@pytest.mark.parametrize("form", [1, 0])
def test_balanced_laplace_within_eps_and_equal_to_plain_plan(S, form):
    n = 40_000
    wl = W.laplace_curves(n, 2, 1e-6)
    alphas = [0.0, 1 / 12, 1 / 6]
    zt = torch.from_numpy(wl.z).cuda()
    p, ms, k = S.sbd_plan_balanced(zt, n, S.SBD_LAPLACE, 0.0, wl.eps, alphas, nrhs=1, reps=2,
                                   options=S.make_options(form=form))
    try:
        assert len(ms) == 3 and all(m > 0 for m in ms), ms
        assert ms[k] == min(ms)
        info = S.sbd_plan_info(p)
        want = W.theorem1_delta_min(n, wl.eps, info["delta_max"], alphas[k])
        assert abs(info["delta_min"] - want) <= 1e-12 * want
        assert abs(info["delta_max"] - wl.meta["delta_max"]) <= 1e-12 * wl.meta["delta_max"]
        q = run(S, p, wl.f)
        idx = np.random.default_rng(11).choice(n, 300, replace=False)
        qd = O.direct_sum(wl.z, wl.f, "laplace", targets=idx, chunk=64)
        assert np.max(np.abs(q[idx] - qd)) <= wl.eps * np.abs(wl.f).sum()
        # the kept plan is the plain plan at that delta_min (node-kernel variants agree to rounding)
        p2 = S.sbd_plan(zt, n, S.SBD_LAPLACE, 0.0, info["delta_min"], wl.eps, S.make_options(form=form))
        try:
            info2 = S.sbd_plan_info(p2)
            assert (info2["P"], info2["nnz"], info2["n_xi"]) == (info["P"], info["nnz"], info["n_xi"])
            q2 = run(S, p2, wl.f)
            rel = np.linalg.norm(q - q2) / np.linalg.norm(q2)
            assert rel <= (2e-6 if form == 1 else 1e-12), rel
        finally:
            S.sbd_destroy(p2)
    finally:
        S.sbd_destroy(p)


def test_balanced_helmholtz_two_rhs(S):
    n = 20_000
    wl = W.helmholtz_curves(n, 3, 1e-6)
    f = np.stack([wl.f, np.conj(wl.f[::-1])])
    zt = torch.from_numpy(wl.z).cuda()
    p, ms, k = S.sbd_plan_balanced(zt, n, S.SBD_HELMHOLTZ, wl.kappa, wl.eps, [0.0, 1 / 24], nrhs=2, reps=1,
                                   options=S.make_options(form=1))
    try:
        assert ms[k] == min(m for m in ms if m > 0)
        q = run(S, p, f, nrhs=2)
        idx = np.random.default_rng(12).choice(n, 60, replace=False)
        for r in range(2):
            qd = O.direct_sum(wl.z, f[r], "helmholtz", wl.kappa, targets=idx, chunk=30)
            assert np.max(np.abs(q[r][idx] - qd)) <= wl.eps * np.abs(f[r]).sum(), r
    finally:
        S.sbd_destroy(p)


def test_balanced_rejects_bad_arguments(S):
    z = W.disk_points(500, 1)
    zt = torch.from_numpy(z).cuda()
    for alphas, nrhs, reps, eps in [([0.2], 1, 1, 1e-6), ([], 1, 1, 1e-6), ([-0.01], 1, 1, 1e-6),
                                    ([0.0], 0, 1, 1e-6), ([0.0], 1, 0, 1e-6), ([0.0], 1, 1, 1e-12),
                                    ([0.0] * 17, 1, 1, 1e-6)]:
        with pytest.raises(S.SbdError) as e:
            S.sbd_plan_balanced(zt, 500, S.SBD_LAPLACE, 0.0, eps, alphas, nrhs=nrhs, reps=reps)
        assert e.value.code == S.SBD_EINVAL
