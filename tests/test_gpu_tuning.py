"""GPU: the node-kernel variants chosen by sbd_tune compute the same matvec.

Each variant sums the same products in another order (with another atomic, or bin by
bin without atomics), so results agree to FP32 rounding (rel-L2 <= 2e-6 between
variants) and each stays within eps sum|f| of the oracle's direct sum (Sec. 1 output
bound)."""
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


@pytest.mark.parametrize("kind", ["laplace", "helmholtz"])
def test_variants_agree_and_tune_picks_one(S, kind):
    n = 6000
    wl = W.laplace_disk(n, 51, 1e-6) if kind == "laplace" else None
    if kind == "laplace":
        z, f, kappa, dmin = wl.z, wl.f, 0.0, wl.delta_min
    else:
        z = W.curve_points(n, 52)
        f = W.rhs(n, 53, complex_valued=True)
        kappa = 60.0 / W.enclosing_diameter(z)
        dmin = float(np.sqrt(20.0 / n))
    zt = torch.from_numpy(z).cuda()
    ft = torch.from_numpy(f).cuda()
    S.sbd_tune_cache_clear()                                  # time every variant (no cached choice)
    p = S.sbd_plan(zt, n, S.SBD_HELMHOLTZ if kind == "helmholtz" else S.SBD_LAPLACE, kappa, dmin, 1e-6,
                   S.make_options(form=S.SBD_FORM_FP32))
    try:
        assert S.sbd_plan_info(p)["node_binned"] == 1          # FP32, 8-cell stencils, small tiles
        outs = {}
        for acc in (0, 1, 2, 3, 4):
            for sched in (0, 1):
                for split in (0, 2):
                    S.sbd_set_tuning(p, acc, sched, split)
                    info = S.sbd_plan_info(p)
                    assert (info["node_acc"], info["node_sched"], info["fft_split"]) == (acc, sched, split)
                    q = torch.empty_like(ft)
                    S.sbd_matvec(p, ft, q)
                    torch.cuda.synchronize()
                    outs[(acc, sched, split)] = q.cpu().numpy()
        base = outs[(0, 0, 0)]
        for k, v in outs.items():
            assert np.linalg.norm(v - base) / np.linalg.norm(base) < 2e-6, k
        idx = np.random.default_rng(5).choice(n, 300, replace=False)
        ref = O.direct_sum(z, f, kind, kappa, targets=idx)
        for k, v in outs.items():
            assert np.max(np.abs(v[idx] - ref)) <= 1e-6 * np.abs(f).sum(), k
        ms = S.sbd_tune(p, reps=2)
        assert len(ms) == 12 and all(t > 0 for t in ms)
        info = S.sbd_plan_info(p)
        node = {(a, sc): ms[a * 2 + sc] if a < 4 else ms[10 + sc] for a in range(5) for sc in (0, 1)}
        assert (info["node_acc"], info["node_sched"]) == min(node, key=node.get)
    finally:
        S.sbd_destroy(p)


def test_fp64_rejects_cas_variant(S):
    wl = W.laplace_disk(500, 54, 1e-6)
    S.sbd_tune_cache_clear()
    zt = torch.from_numpy(wl.z).cuda()
    p = S.sbd_plan(zt, 500, S.SBD_LAPLACE, 0.0, wl.delta_min, 1e-6, S.make_options(form=S.SBD_FORM_FP64))
    try:
        assert S.sbd_plan_info(p)["node_binned"] == 0
        for acc in (1, 2, 3, 4, 5):
            with pytest.raises(S.SbdError) as e:
                S.sbd_set_tuning(p, acc, 0, 0)
            assert e.value.code == S.SBD_EINVAL
        ms = S.sbd_tune(p, reps=1)
        assert ms[0] > 0 and ms[1] > 0 and all(t == -1 for t in ms[2:8]) and ms[8] > 0 and ms[9] > 0
        assert ms[10] == -1 and ms[11] == -1
    finally:
        S.sbd_destroy(p)


def test_point_chunk_search_and_tuning_cache(S):
    """sbd_tune also picks the point chunk; a second plan of the same class takes the cached
    choice without timing (tuned = 2); every chunk gives the same matvec to FP32 rounding."""
    S.sbd_tune_cache_clear()
    wl = W.laplace_curves(120_000, 81, 1e-6)
    zt = torch.from_numpy(wl.z).cuda()
    ft = torch.from_numpy(wl.f).cuda()
    opt = S.make_options(form=S.SBD_FORM_FP32)
    p1 = S.sbd_plan(zt, len(wl.z), S.SBD_LAPLACE, 0.0, wl.delta_min, wl.eps, opt)
    p2 = S.sbd_plan(zt, len(wl.z), S.SBD_LAPLACE, 0.0, wl.delta_min, wl.eps, opt)
    try:
        ms = S.sbd_tune_points(p1, 2)
        assert len(ms) == 5 and all(t > 0 for t in ms)
        outs = []
        for chunk in (128, 512, 2048):
            S.sbd_set_point_chunk(p1, chunk)
            assert S.sbd_plan_info(p1)["point_chunk"] == chunk
            q = torch.empty_like(ft)
            S.sbd_matvec(p1, ft, q)
            torch.cuda.synchronize()
            outs.append(q.cpu().numpy())
        for o in outs[1:]:
            assert np.linalg.norm(o - outs[0]) / np.linalg.norm(outs[0]) < 2e-6
        S.sbd_tune(p1, 2)
        i1 = S.sbd_plan_info(p1)
        assert i1["tuned"] == 1 and S.sbd_tune_cache_stats()["misses"] == 1
        S.sbd_tune(p2, 2)
        i2 = S.sbd_plan_info(p2)
        assert i2["tuned"] == 2 and S.sbd_tune_cache_stats()["hits"] == 1
        for k in ("node_acc", "node_sched", "fft_split", "point_chunk"):
            assert i1[k] == i2[k], k
        with pytest.raises(S.SbdError) as e:
            S.sbd_set_point_chunk(p1, 64)
        assert e.value.code == S.SBD_EINVAL
    finally:
        S.sbd_destroy(p1)
        S.sbd_destroy(p2)
        S.sbd_tune_cache_clear()
