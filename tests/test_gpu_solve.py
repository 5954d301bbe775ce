"""GPU: the GMRES entry point and the continuous-batching server.

Expected solutions come from a dense solve of the same system built with the oracle's
exact kernel G (no SBD anywhere): (shift I + scale A) x = b, A_kl = G(|z_k - z_l|) for
k != l (Eq. discrete convolution, self term excluded).  The SBD matvec differs from A x
by at most eps sum|x| per entry (Sec. 1), so with scale = 1/N and shift = 1 the system
is well conditioned and the solution moves by O(eps); GMRES stops at `tol`.
Bar: ||x - x_dense|| / ||x_dense|| <= 20 (tol + eps).
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


def dense_matrix(z, kind, kappa=0.0):
    d = np.hypot(z[:, None, 0] - z[None, :, 0], z[:, None, 1] - z[None, :, 1])
    np.fill_diagonal(d, 1.0)
    A = O.kernel_G(d, kind, kappa)
    np.fill_diagonal(A, 0.0)
    return A


def system(kind, n, seed):
    if kind == "laplace":
        z = W.disk_points(n, seed)
        kappa = 0.0
        b = W.rhs(n, seed + 100)
    else:
        z = W.curve_points(n, seed)
        kappa = 40.0 / W.enclosing_diameter(z)
        b = W.rhs(n, seed + 100, complex_valued=True)
    dmin = float(np.sqrt(20.0 / n))
    return z, kappa, dmin, b


def solve_gpu(S, z, kind, kappa, dmin, eps, b, form, tol, shift, scale, restart=30, max_iter=400):
    zt = torch.from_numpy(z).cuda()
    opt = S.make_options(form=form)
    p = S.sbd_plan(zt, len(z), S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE, kappa, dmin, eps, opt)
    try:
        bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        xt = torch.zeros_like(bt)
        it, res = S.sbd_gmres(p, bt, xt, shift, scale, tol, restart, max_iter)
        torch.cuda.synchronize()
        return xt.cpu().numpy(), it, res
    finally:
        S.sbd_destroy(p)


@pytest.mark.parametrize("kind,form,eps,tol", [
    ("laplace", 0, 1e-10, 1e-9),
    ("laplace", 1, 1e-6, 1e-5),
    ("helmholtz", 0, 1e-10, 1e-9),
    ("helmholtz", 1, 1e-6, 1e-5),
])
def test_gmres_matches_dense_solve(S, kind, form, eps, tol):
    n = 1800
    z, kappa, dmin, b = system(kind, n, 11)
    shift, scale = 1.0, 1.0 / n
    x, it, res = solve_gpu(S, z, kind, kappa, dmin, eps, b, form, tol, shift, scale)
    assert 0 < it < 400 and res <= tol * 1.0001, (it, res)
    A = dense_matrix(z, kind, kappa)
    M = shift * np.eye(n) + scale * A
    x_ref = np.linalg.solve(M, b)
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err <= 20 * (tol + eps), err
    # the residual of the GPU solution against the exact operator
    r = np.linalg.norm(b - M @ x) / np.linalg.norm(b)
    assert r <= 20 * (tol + eps), r


def test_gmres_restart_small_subspace(S):
    """restart = 3 forces several cycles; the answer must not change."""
    n = 1200
    z, kappa, dmin, b = system("laplace", n, 12)
    x3, it3, _ = solve_gpu(S, z, "laplace", kappa, dmin, 1e-10, b, 0, 1e-9, 1.0, 1.0 / n, restart=3, max_iter=600)
    x30, it30, _ = solve_gpu(S, z, "laplace", kappa, dmin, 1e-10, b, 0, 1e-9, 1.0, 1.0 / n, restart=30)
    assert it3 >= it30
    assert np.linalg.norm(x3 - x30) / np.linalg.norm(x30) < 1e-7


def test_gmres_zero_rhs_and_bad_args(S):
    n = 500
    z, kappa, dmin, _ = system("laplace", n, 13)
    zt = torch.from_numpy(z).cuda()
    p = S.sbd_plan(zt, n, S.SBD_LAPLACE, 0.0, dmin, 1e-6, S.make_options(form=0))
    try:
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        x = torch.ones(n, dtype=torch.float64, device="cuda")
        it, res = S.sbd_gmres(p, b, x, 1.0, 1.0, 1e-8)
        torch.cuda.synchronize()
        assert it == 0 and res == 0.0 and float(x.abs().max()) == 0.0
        for kw in ({"tol": 0.0}, {"restart": 0}, {"max_iter": -1}):
            args = dict(shift=1.0, scale=1.0, tol=1e-6, restart=10, max_iter=10)
            args.update(kw)
            with pytest.raises(S.SbdError) as e:
                S.sbd_gmres(p, b, x, **args)
            assert e.value.code == S.SBD_EINVAL
    finally:
        S.sbd_destroy(p)


def test_gmres_max_iter_reports_residual(S):
    n = 1500
    z, kappa, dmin, b = system("helmholtz", n, 14)
    x, it, res = solve_gpu(S, z, "helmholtz", kappa, dmin, 1e-8, b, 0, 1e-14, 1.0, 1.0 / n, restart=5, max_iter=4)
    assert it == 4 and res > 1e-14


def test_server_results_match_solo_solves(S):
    """Requests served concurrently (3 slots, Poisson arrivals) give the answers they give alone."""
    from paper_1711_07877_gb300 import serve
    reqs, solo = [], []
    specs = [("laplace", 1500), ("helmholtz", 2000), ("laplace", 3000), ("helmholtz", 1200),
             ("laplace", 2500), ("laplace", 1000)]
    tol = 1e-8
    for i, (kind, n) in enumerate(specs):
        z, kappa, dmin, b = system(kind, n, 20 + i)
        reqs.append(serve.Request(rid=i, z=z, b=b, kind=S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE,
                                  kappa=kappa, delta_min=dmin, eps=1e-10, shift=1.0, scale=1.0 / n))
        solo.append(solve_gpu(S, z, kind, kappa, dmin, 1e-10, b, 0, tol, 1.0, 1.0 / n)[0])
    srv, summary = serve.run_poisson(reqs, mean_gap_s=0.004, seed=5, slots=3, form=S.SBD_FORM_FP64, tol=tol)
    assert [r.error for r in reqs] == [None] * len(reqs)
    assert summary["requests"] == len(specs)
    assert 0 < summary["p50_ms"] <= summary["p99_ms"]
    assert summary["gpts_per_s"] > 0
    for r, xs in zip(reqs, solo):
        assert r.error is None, r.error
        assert r.residual <= tol * 1.0001
        assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-6, r.rid


def test_server_batched_matvecs_match_solo_solves(S):
    """The same requests with the solves' matvecs merged into batched launches (iteration-level
    batching): the answers of the solo solves, and most launches carry several solves."""
    from paper_1711_07877_gb300 import serve
    reqs, solo = [], []
    specs = [("laplace", 1500), ("helmholtz", 2000), ("laplace", 3000), ("helmholtz", 1200),
             ("laplace", 2500), ("laplace", 1000)]
    tol = 1e-8
    for i, (kind, n) in enumerate(specs):
        z, kappa, dmin, b = system(kind, n, 20 + i)
        reqs.append(serve.Request(rid=i, z=z, b=b, kind=S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE,
                                  kappa=kappa, delta_min=dmin, eps=1e-10, shift=1.0, scale=1.0 / n))
        solo.append(solve_gpu(S, z, kind, kappa, dmin, 1e-10, b, 0, tol, 1.0, 1.0 / n)[0])
    srv, summary = serve.run_poisson(reqs, mean_gap_s=0.0005, seed=5, slots=6, form=S.SBD_FORM_FP64, tol=tol,
                                     batch_matvecs=True)
    assert [r.error for r in reqs] == [None] * len(reqs)
    assert summary["matvecs_batched"] >= sum(r.iterations for r in reqs)
    assert summary["matvec_batches"] < summary["matvecs_batched"]
    for r, xs in zip(reqs, solo):
        assert r.residual <= tol * 1.0001
        assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-6, r.rid


def test_gmres_session_equals_gmres(S):
    """The session API driven by hand (plain matvecs) gives sbd_gmres's answer."""
    z, kappa, dmin, b = system("helmholtz", 1800, 60)
    x_ref, it_ref, res_ref = solve_gpu(S, z, "helmholtz", kappa, dmin, 1e-8, b, 0, 1e-6, 0.5, 1.0 / 1800)
    p = S.sbd_plan(torch.from_numpy(z).cuda(), 1800, S.SBD_HELMHOLTZ, kappa, dmin, 1e-8, S.make_options(form=0))
    try:
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        sess = S.sbd_gmres_begin(p, bt, xt, 0.5, 1.0 / 1800, 1e-6)
        steps = 0
        while True:
            io = S.sbd_gmres_next(sess)
            if io is None:
                break
            S.sbd_matvec(p, io[0], io[1])
            S.sbd_gmres_advance(sess)
            steps += 1
        it, res = S.sbd_gmres_end(sess)
        torch.cuda.synchronize()
        assert abs(it - it_ref) <= 1 and res <= 1e-6 and steps >= it
        assert np.linalg.norm(xt.cpu().numpy() - x_ref) / np.linalg.norm(x_ref) < 1e-6
    finally:
        S.sbd_destroy(p)


def test_server_budget_serialises(S):
    """A budget smaller than any request admits one request at a time."""
    from paper_1711_07877_gb300 import serve
    reqs = []
    for i in range(4):
        z, kappa, dmin, b = system("laplace", 800 + 200 * i, 40 + i)
        reqs.append(serve.Request(rid=i, z=z, b=b, kind=S.SBD_LAPLACE, kappa=0.0, delta_min=dmin, eps=1e-6,
                                  shift=1.0, scale=1.0 / len(z)))
    srv, summary = serve.run_poisson(reqs, mean_gap_s=0.0005, seed=6, slots=4, hbm_budget=1,
                                     form=S.SBD_FORM_FP32, tol=1e-5)
    spans = sorted((r.start, r.done) for r in reqs)
    for (s0, d0), (s1, d1) in zip(spans, spans[1:]):
        assert s1 >= d0 - 1e-6
    assert all(r.error is None for r in reqs)


def test_plan_delta_max_option_and_fit_cache(S):
    """A larger delta_max (options.delta_max) keeps the eps bound; one below 2 max|z - c| is
    rejected; a second plan with the same normalised fit is a fit-cache hit."""
    n = 3000
    z, _, dmin, _ = system("laplace", n, 31)
    f = W.rhs(n, 131)
    zt = torch.from_numpy(z).cuda()
    ft = torch.from_numpy(f).cuda()
    lo, hi = z.min(0), z.max(0)
    diam = 2 * np.sqrt(np.max(np.sum((z - 0.5 * (lo + hi)) ** 2, axis=1)))
    q_ref = O.direct_sum(z, f, "laplace")
    S.sbd_fit_cache_clear()
    for dmax in (0.0, 1.5 * diam):
        p = S.sbd_plan(zt, n, S.SBD_LAPLACE, 0.0, dmin, 1e-8, S.make_options(form=0, delta_max=dmax))
        q = torch.empty_like(ft)
        S.sbd_matvec(p, ft, q)
        torch.cuda.synchronize()
        info = S.sbd_plan_info(p)
        S.sbd_destroy(p)
        if dmax:
            assert abs(info["delta_max"] - dmax) < 1e-15 * dmax
        err = np.max(np.abs(q.cpu().numpy() - q_ref)) / np.abs(f).sum()
        assert err <= 1e-8, (dmax, err)
    with pytest.raises(S.SbdError) as e:
        S.sbd_plan(zt, n, S.SBD_LAPLACE, 0.0, dmin, 1e-8, S.make_options(form=0, delta_max=0.99 * diam))
    assert e.value.code == S.SBD_EINVAL
    # same a = delta_min / delta_max on a rescaled copy of the points: a cache hit
    before = S.sbd_fit_cache_stats()
    z2 = torch.from_numpy(np.ascontiguousarray(2.0 * z)).cuda()
    p = S.sbd_plan(z2, n, S.SBD_LAPLACE, 0.0, 2.0 * dmin, 1e-8, S.make_options(form=0, delta_max=2.0 * 1.5 * diam))
    S.sbd_destroy(p)
    after = S.sbd_fit_cache_stats()
    assert after["hits"] == before["hits"] + 1


@pytest.mark.parametrize("kind,form", [("laplace", 0), ("laplace", 1), ("helmholtz", 0), ("helmholtz", 1)])
def test_matvec_graph_equals_matvec(S, kind, form):
    """The graph replay computes the same matvec, on the default stream and on a side
    stream, for several inputs and for nrhs = 1 and 2."""
    n = 2500
    z, kappa, dmin, _ = system(kind, n, 61)
    zt = torch.from_numpy(z).cuda()
    p = S.sbd_plan(zt, n, S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE, kappa, dmin, 1e-8,
                   S.make_options(form=form, max_nrhs=2))
    try:
        side = torch.cuda.Stream()
        for trial, stream in enumerate((None, side, None)):
            for nrhs in (1, 2):
                f = W.rhs(n, 70 + trial, nrhs=nrhs, complex_valued=kind == "helmholtz")
                ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
                q0, q1 = torch.empty_like(ft), torch.empty_like(ft)
                S.sbd_matvec(p, ft, q0, nrhs)
                torch.cuda.synchronize()
                sid = None if stream is None else stream.cuda_stream
                if stream is not None:
                    stream.wait_stream(torch.cuda.current_stream())
                S.sbd_matvec_graph(p, ft, q1, nrhs, sid)
                torch.cuda.synchronize()
                a, b = q0.cpu().numpy(), q1.cpu().numpy()
                tol = 1e-12 if form == 0 else 2e-6
                assert np.linalg.norm(a - b) / np.linalg.norm(a) < tol, (trial, nrhs)
    finally:
        S.sbd_destroy(p)


def test_server_reuses_resident_plans(S):
    """Requests with the same geometry key reuse one resident plan (no second plan build)
    and give the answer of a fresh solve."""
    from paper_1711_07877_gb300 import serve
    z, kappa, dmin, b = system("laplace", 2000, 81)
    b2 = W.rhs(2000, 82)
    mk = lambda rid, rhs: serve.Request(rid=rid, z=z, b=rhs, kind=S.SBD_LAPLACE, kappa=0.0, delta_min=dmin,
                                        eps=1e-10, shift=1.0, scale=1.0 / 2000, geometry="g1")
    reqs = [mk(0, b), mk(1, b2), mk(2, b)]
    srv, summary = serve.run_poisson(reqs, mean_gap_s=0.001, seed=3, slots=2, form=S.SBD_FORM_FP64, tol=1e-9)
    assert all(r.error is None for r in reqs)
    built = [r for r in reqs if r.plan_seconds > 0]
    assert len(built) == 1                      # one plan build, two reuses
    assert np.linalg.norm(reqs[0].x - reqs[2].x) / np.linalg.norm(reqs[0].x) < 1e-8
    solo = solve_gpu(S, z, "laplace", 0.0, dmin, 1e-10, b2, 0, 1e-9, 1.0, 1.0 / 2000)[0]
    assert np.linalg.norm(reqs[1].x - solo) / np.linalg.norm(solo) < 1e-6
    assert not srv.adm.resident                # close() freed the resident plan
