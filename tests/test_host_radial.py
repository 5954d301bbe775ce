"""Host (no GPU): the library's fit of a general real radial kernel (sbd_offline_fit_radial,
Sec. 4.3) against the oracle's radial_fit: the same P, the same J1 frequencies and correction
weights mu_t / J0(omega_t), the same constant c, fit errors that agree (the coefficients alpha
themselves are compared only through the fit, as two Cholesky solves of the ill-conditioned Gram
matrix differ along its small eigenvectors, Sec. 3.3); the Laplace kernel written as a radial
kernel reproduces the Laplace fit; argument errors."""
import math

import numpy as np
import pytest
from scipy.special import j0, j1

from oracle import sbd_oracle as O

S = pytest.importorskip("paper_1711_07877_gb300.sbd")


def kernel_a(beta):
    """G(r) = log r + J0(beta r) + r^2 / 2: its radial-Laplacian iterates in closed form
    (Delta log r = 0, Delta^j J0(beta r) = (-beta^2)^j J0(beta r), Delta r^2 / 2 = 2)."""
    value = lambda r: np.log(r) + j0(beta * r) + 0.5 * np.square(r)  # noqa: E731
    deriv = lambda r: 1.0 / np.asarray(r) - beta * j1(beta * r) + np.asarray(r)  # noqa: E731
    lap = lambda j, r: (-beta * beta) ** j * j0(beta * r) + (2.0 if j == 1 else 0.0)  # noqa: E731
    return value, deriv, lap


def both(value, deriv, lap, log_coef, n):
    ok = O.RadialKernel(value, deriv, lap, log_coef)
    ck = S.radial_kernel(lambda r: value(r), lambda r: deriv(r), lambda j, r: lap(j, r), log_coef, n)
    return ok, ck


@pytest.mark.parametrize("beta,n,dmin,eps", [(9.0, 1, 0.1, 1e-6), (9.0, 3, 0.05, 1e-6), (40.0, 3, 0.08, 3e-9),
                                            (2.0, 2, 0.2, 1e-3)])
def test_host_radial_fit_matches_oracle(beta, n, dmin, eps):
    R = 2.0
    ok, ck = both(*kernel_a(beta), 1.0, n)
    h = S.sbd_offline_fit_radial(ck, dmin, R, eps)
    P, rho, C, alpha, err, omega, mu, c = O.radial_fit(ok, R, dmin / R, eps / 3, n)
    assert h["P"] == P and h["n_circles"] == P + n
    np.testing.assert_allclose(h["rho"][P:], omega, rtol=1e-14)
    np.testing.assert_allclose(h["alpha"][P:], mu / j0(omega), rtol=1e-9)
    assert abs(h["w0"] - c) <= 1e-12 * max(1.0, abs(c))
    assert abs(h["fit_err"] - err) <= 1e-3 * err + 1e-15
    assert h["fit_err"] <= eps / 3
    np.testing.assert_allclose(h["rho"][:P], rho, rtol=1e-14)


def test_fit_floor_reported_like_the_oracle():
    """With two iterates enforced, J0(40 r) leaves h rough enough at r = delta_max that the fit
    meets the Gram conditioning floor (Sec. 3.3) before 1e-9 / 3: the oracle's search fails there
    too, and the library says so (SBD_EFIT) instead of returning a worse fit."""
    ok, ck = both(*kernel_a(40.0), 1.0, 2)
    with pytest.raises(Exception):
        O.radial_fit(ok, 2.0, 0.04, 1e-9 / 3, 2)
    with pytest.raises(S.SbdError) as e:
        S.sbd_offline_fit_radial(ck, 0.08, 2.0, 1e-9)
    assert e.value.code == S.SBD_EFIT


def test_laplace_as_a_radial_kernel():
    """-log(r)/(2 pi) has no iterate to enforce: the radial fit is the Laplace fit of Sec. 4.1 (the
    same P and circle sizes, coefficients -alpha / (2 pi), the constant G(delta_max))."""
    R, dmin, eps = 3.0, 0.1, 1e-6
    value = lambda r: -np.log(r) / (2 * math.pi)  # noqa: E731
    deriv = lambda r: -1.0 / (2 * math.pi * np.asarray(r))  # noqa: E731
    ck = S.radial_kernel(value, deriv, None, -1.0 / (2 * math.pi), 0)
    h = S.sbd_offline_fit_radial(ck, dmin, R, eps)
    lap = S.sbd_offline_fit(S.SBD_LAPLACE, 0.0, dmin, R, eps)
    assert h["P"] == lap["P"] and np.array_equal(h["M"], lap["M"])
    np.testing.assert_allclose(h["alpha"], -lap["alpha"] / (2 * math.pi), rtol=1e-8, atol=1e-15)
    assert abs(h["w0"] - value(R)) < 1e-15


def test_radial_argument_errors():
    value, deriv, lap = kernel_a(9.0)
    for n in (-1, 9):
        with pytest.raises(S.SbdError) as e:
            S.sbd_offline_fit_radial(S.radial_kernel(value, deriv, lap, 1.0, n), 0.1, 2.0, 1e-6)
        assert e.value.code == S.SBD_EINVAL
    with pytest.raises(S.SbdError) as e:                   # iterates asked for, no laplacian
        S.sbd_offline_fit_radial(S.radial_kernel(value, deriv, None, 1.0, 2), 0.1, 2.0, 1e-6)
    assert e.value.code == S.SBD_EINVAL
    with pytest.raises(S.SbdError) as e:
        S.sbd_offline_fit_radial(S.radial_kernel(value, deriv, lap, 1.0, 1), 2.5, 2.0, 1e-6)
    assert e.value.code == S.SBD_EINVAL
    host = np.zeros((4, 2))
    with pytest.raises(S.SbdError) as e:                   # the uniform-grid variant is not offered
        S.sbd_plan_radial(host, 4, S.radial_kernel(value, deriv, lap, 1.0, 1), 0.1, 1e-6,
                          S.make_options(form=1, flags=S.SBD_FLAG_UNIFORM_GRID), stream=0)
    assert e.value.code == S.SBD_ENOTSUP


@pytest.mark.parametrize("kappa,dmin,eps", [(0.05, 0.1, 1e-6), (0.2, 0.05, 1e-6), (0.1, 0.1, 1e-9), (0.02, 0.2, 1e-3)])
def test_low_wavenumber_helmholtz_fit_matches_oracle(kappa, dmin, eps):
    """kappa delta_max below half the first Y0 root: the Dini (Robin) fit of Y0 at scale delta_max
    (reading R15), the library's against the oracle's: the same P, Dini roots and fit error."""
    import scipy.special as sp
    dmax = 2.0
    h = S.sbd_offline_fit(S.SBD_HELMHOLTZ, kappa, dmin, dmax, eps)
    k, a = kappa * dmax, dmin / dmax
    H = O.robin_H(k)
    g = lambda s: sp.y0(k * s)  # noqa: E731
    gp = lambda s: -k * sp.y1(k * s)  # noqa: E731
    tol = eps / 3 / 0.25
    P, rho, C, alpha, err = O.choose_P(g, gp, a, tol, O.initial_P(a, tol, 2 * k), 2 * k,
                                       coefficients=lambda q: O.robin_coefficients(g, gp, a, q, H, 2 * k))
    assert h["P"] == P and h["n_circles"] == P + 1
    np.testing.assert_allclose(h["rho"][:P], rho, rtol=1e-13)
    assert abs(h["fit_err"] - 0.25 * err) <= 1e-3 * h["fit_err"]     # the 1e-9 case sits at the Gram floor
