"""GPU: a batch graph runs several plans' matvecs in one launch and gives each plan's
own matvec (same kernels, same order within a plan; FP32 node-step atomics may reorder
additions, so FP32 agrees to rounding)."""
import numpy as np
import pytest

import workloads as W

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


def test_batch_equals_single_matvecs(S):
    specs = [("laplace", 1200, 1, 1), ("helmholtz", 3000, 1, 1), ("laplace", 5000, 0, 1), ("laplace", 2000, 1, 2)]
    plans, fs, qs = [], [], []
    try:
        for i, (kind, n, form, nrhs) in enumerate(specs):
            z = W.curve_points(n, 90 + i)
            kappa = 80.0 / W.enclosing_diameter(z) if kind == "helmholtz" else 0.0
            p = S.sbd_plan(torch.from_numpy(z).cuda(), n, S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE,
                           kappa, float(np.sqrt(20.0 / n)), 1e-6, S.make_options(form=form, max_nrhs=nrhs))
            plans.append(p)
            f = W.rhs(n, 95 + i, nrhs=nrhs, complex_valued=kind == "helmholtz")
            fs.append(torch.from_numpy(np.ascontiguousarray(f)).cuda())
            qs.append(torch.empty_like(fs[-1]))
        b = S.sbd_batch_create(plans, fs, qs, [s[3] for s in specs])
        try:
            for trial in range(2):
                if trial:
                    for f in fs:
                        f.mul_(-0.5)                       # new inputs in the same buffers
                S.sbd_batch_launch(b)
                torch.cuda.synchronize()
                for (kind, n, form, nrhs), p, f, q in zip(specs, plans, fs, qs):
                    ref = torch.empty_like(f)
                    S.sbd_matvec(p, f, ref, nrhs)
                    torch.cuda.synchronize()
                    a, r = q.cpu().numpy(), ref.cpu().numpy()
                    tol = 1e-12 if form == 0 else 2e-6
                    assert np.linalg.norm(a - r) / np.linalg.norm(r) < tol, (kind, n, form, trial)
        finally:
            S.sbd_batch_destroy(b)
        with pytest.raises(S.SbdError) as e:
            S.sbd_batch_create([plans[0], plans[0]], [fs[0], fs[0]], [qs[0], qs[0]])
        assert e.value.code == S.SBD_EINVAL
    finally:
        for p in plans:
            S.sbd_destroy(p)


def _plans(S, specs, seed):
    plans, fs, qs = [], [], []
    for i, (kind, n, form, nrhs, n_t) in enumerate(specs):
        z = W.curve_points(n, seed + i)
        kappa = 80.0 / W.enclosing_diameter(z) if kind == "helmholtz" else 0.0
        k = S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE
        opt = S.make_options(form=form, max_nrhs=nrhs)
        dmin = float(np.sqrt(20.0 / n))
        if n_t:
            x = W.curve_points(n_t, seed + 50 + i)
            p = S.sbd_plan_st(torch.from_numpy(x).cuda(), n_t, torch.from_numpy(z).cuda(), n, k, kappa, dmin, 1e-6,
                              opt)
        else:
            p = S.sbd_plan(torch.from_numpy(z).cuda(), n, k, kappa, dmin, 1e-6, opt)
        plans.append(p)
        f = W.rhs(n, seed + 20 + i, nrhs=nrhs, complex_valued=kind == "helmholtz")
        fs.append(torch.from_numpy(np.ascontiguousarray(f)).cuda())
        shape = (nrhs, n_t or n) if nrhs > 1 else (n_t or n,)
        qs.append(torch.empty(shape, dtype=fs[-1].dtype, device="cuda"))
    return plans, fs, qs


# sbd_matvec_batched: uneven instances (Laplace and Helmholtz, several right-hand sides, a plan
# with separate targets, the binned and the fused node kernels) in one call; each result equals
# the plan's own sbd_matvec (the batched kernels run the same bodies; FP32 atomics may reorder
# additions, so FP32 agrees to rounding)
@pytest.mark.parametrize("form", [1, 0])
def test_matvec_batched_equals_single_matvecs(S, form):
    specs = [("laplace", 1500, form, 1, 0), ("helmholtz", 2500, form, 2, 0), ("laplace", 6000, form, 3, 0),
             ("laplace", 800, form, 1, 1100), ("helmholtz", 900, form, 1, 0)]
    plans, fs, qs = _plans(S, specs, 300 + 10 * form)
    try:
        if form == 1:
            S.sbd_set_tuning(plans[2], 0, 0, 0)          # one plan on the fused node kernel, the rest binned
        for trial in range(2):
            if trial:
                for f in fs:
                    f.mul_(-0.5)
            S.sbd_matvec_batched(plans, fs, qs, [s[3] for s in specs])
            assert S.sbd_device_status() == S.SBD_OK
            for spec, p, f, q in zip(specs, plans, fs, qs):
                ref = torch.empty_like(q)
                S.sbd_matvec(p, f, ref, spec[3])
                torch.cuda.synchronize()
                a, r = q.cpu().numpy(), ref.cpu().numpy()
                tol = 1e-12 if form == 0 else 2e-6
                assert np.linalg.norm(a - r) / np.linalg.norm(r) < tol, (spec, trial)
    finally:
        for p in plans:
            S.sbd_destroy(p)


def test_matvec_batched_rejects_bad_batches(S):
    specs = [("laplace", 700, 1, 1, 0), ("laplace", 900, 0, 1, 0)]
    plans, fs, qs = _plans(S, specs, 400)
    try:
        with pytest.raises(S.SbdError) as e:
            S.sbd_matvec_batched([plans[0], plans[0]], [fs[0], fs[0]], [qs[0], qs[0]])
        assert e.value.code == S.SBD_EINVAL
        with pytest.raises(S.SbdError) as e:                 # mixed forms
            S.sbd_matvec_batched(plans, fs, qs)
        assert e.value.code == S.SBD_ENOTSUP
        with pytest.raises(S.SbdError) as e:                 # nrhs beyond the plan's max_nrhs
            S.sbd_matvec_batched(plans[:1], fs[:1], qs[:1], [2])
        assert e.value.code == S.SBD_EINVAL
        with pytest.raises(S.SbdError) as e:
            S.sbd_set_device_wait(0.0, 0)
        assert e.value.code == S.SBD_EINVAL
    finally:
        for p in plans:
            S.sbd_destroy(p)


def test_batched_device_wait_runs_out_and_reports(S):
    """Fault injection on the host's terms: the grid barriers of the batched kernels wait for
    one phantom CTA that never arrives; every wait gives up after 50 ms, the kernels return,
    sbd_device_status reports SBD_ETIMEOUT once, and the next batched call is correct."""
    specs = [("laplace", 1500, 1, 1, 0), ("helmholtz", 1200, 1, 1, 0)]
    plans, fs, qs = _plans(S, specs, 500)
    try:
        assert S.sbd_device_status() == S.SBD_OK
        S.sbd_set_device_wait(0.05, 1)
        try:
            S.sbd_matvec_batched(plans, fs, qs)
            assert S.sbd_device_status() == S.SBD_ETIMEOUT
            assert S.sbd_device_status() == S.SBD_OK           # reported once
        finally:
            S.sbd_set_device_wait(2.0, 0)
        S.sbd_matvec_batched(plans, fs, qs)
        assert S.sbd_device_status() == S.SBD_OK
        for spec, p, f, q in zip(specs, plans, fs, qs):
            ref = torch.empty_like(q)
            S.sbd_matvec(p, f, ref)
            torch.cuda.synchronize()
            a, r = q.cpu().numpy(), ref.cpu().numpy()
            assert np.linalg.norm(a - r) / np.linalg.norm(r) < 2e-6
    finally:
        for p in plans:
            S.sbd_destroy(p)
