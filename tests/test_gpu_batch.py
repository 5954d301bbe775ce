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
