"""GPU: the off-line fit's Cholesky of the Gram matrix (Sec. 3.2, Eq. LinearSystem; the O(P^3)
step of Sec. 6.1) on the device gives the same fit as on the host.

Two factorisations of one ill-conditioned Gram matrix differ by rounding, which the solve
amplifies along the matrix's small eigenvectors (Sec. 3.3), so the coefficients are not
compared one by one.  What both must satisfy is the fit itself: the same P from the search,
each fit error within the tolerance, and the two series G_fit(r) = sum_p alpha_p C_p J0(rho_p r)
within the sum of their errors of each other on [delta_min, delta_max] (both are within their
own error of G there).  For Laplace the series fits log r on [a, 1] (delta_max = 1 here), and
fit_err is reported in kernel units, i.e. divided by 2 pi (G = -log r / (2 pi) + w0, Sec. 4.1)."""
import numpy as np
import pytest

from oracle import sbd_oracle as O

torch = pytest.importorskip("torch")
scipy_special = pytest.importorskip("scipy.special")
pytestmark = pytest.mark.gpu
TWO_PI = 2 * np.pi


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_07877_gb300 import build
    build.build_library()
    import paper_1711_07877_gb300 as pkg
    yield pkg
    pkg.sbd_set_fit_device(0)
    pkg.sbd_fit_cache_clear()


def fit(S, mode, dmin, eps=1e-9, kind=0, kappa=0.0):
    S.sbd_set_fit_device(mode)
    S.sbd_fit_cache_clear()
    f = S.sbd_offline_fit(kind, kappa, dmin, 1.0, eps)
    return f, S.sbd_fit_last_factorisation()


def series(f, r):
    P = f["P"]
    rho, alpha = f["rho"][:P], f["alpha"][:P]
    C = O.normalisation_C(rho)
    return scipy_special.j0(np.outer(r, rho)) @ (alpha * C)


@pytest.mark.parametrize("dmin", [0.05, 0.002])
def test_device_factor_gives_the_host_fit(S, dmin):
    fh, (th, wh) = fit(S, 1, dmin)
    fd, (td, wd) = fit(S, 2, dmin)
    assert wh == 1 and wd == 2 and th > 0 and td > 0
    assert fd["P"] == fh["P"]
    tol = 1e-9 / 3                        # the fit's share of eps
    assert fh["fit_err"] <= tol and fd["fit_err"] <= tol
    assert abs(fd["fit_err"] - fh["fit_err"]) <= 0.1 * fh["fit_err"]
    r = np.geomspace(dmin, 1.0, 3001)
    gh, gd = series(fh, r) / TWO_PI, series(fd, r) / TWO_PI
    assert np.max(np.abs(gh - gd)) <= fh["fit_err"] + fd["fit_err"]
    # and each against the kernel itself
    g = np.log(r) / TWO_PI
    assert np.max(np.abs(gd - g)) <= 1.05 * fd["fit_err"] + 1e-13


def test_auto_mode_uses_the_device_from_p_3000_and_helmholtz(S):
    f, (t, where) = fit(S, 0, 0.0015)
    assert f["P"] >= 3000 and where == 2
    f2, (t2, where2) = fit(S, 0, 0.05)
    assert f2["P"] < 3000 and where2 == 1
    # Helmholtz (Sec. 4.2): the same Gram matrix in k' units; device and host agree on P and error
    kappa = 400.0
    hh, _ = fit(S, 1, 0.004, kind=1, kappa=kappa)
    hd, (_, wd) = fit(S, 2, 0.004, kind=1, kappa=kappa)
    assert wd == 2 and hh["P"] == hd["P"]
    assert abs(hh["fit_err"] - hd["fit_err"]) <= 0.1 * hh["fit_err"]


def test_large_fit_on_the_device(S):
    """eps = 1e-9 at a = delta_min / delta_max = 7.7e-4 (the N = 10^6 curves at eps 1e-9): P ~ 7200,
    the size where the host's packed Cholesky takes tens of seconds."""
    f, (t, where) = fit(S, 0, 0.00077)
    assert where == 2 and f["P"] > 7000
    assert f["fit_err"] <= 1e-9 / 3
    r = np.geomspace(0.00077, 1.0, 4001)
    assert np.max(np.abs(series(f, r) - np.log(r)) / TWO_PI) <= 1.05 * f["fit_err"] + 1e-13
