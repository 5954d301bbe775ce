"""CPU pins of the oracle's Robin / Dini branch for low-wavenumber Helmholtz (Sec. 2.3, Sec. 4.2
third case; reading R15), each fixed independently of the oracle's own formulas:
  * Dini roots: the limits H -> infinity (roots of J0) and H -> 0 (roots of J1, the first ~ sqrt(2H)),
    from scipy's own zero tables;
  * orthonormality of the Dini basis in a_H (Sec. 2.3 Theorem), by scipy.integrate.quad;
  * Y0(k s) meets the Robin condition with H = k Y1(k) / Y0(k) (central difference of Y0);
  * the fit of Y0(k s) needs far fewer terms than the first-root scaling of Sec. 4.2 at the same
    geometry, and its error falls exponentially with P;
  * the SBD with the Robin branch meets the Sec. 1 output bound against the direct sum."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import workloads as W
from oracle import sbd_oracle as O


def test_dini_root_limits():
    big = O.dini_roots(1e9, 6)
    np.testing.assert_allclose(big, sp.jn_zeros(0, 6), rtol=1e-8)
    small = O.dini_roots(1e-10, 6)
    assert abs(small[0] - math.sqrt(2e-10)) < 1e-9
    np.testing.assert_allclose(small[1:], sp.jn_zeros(1, 5), rtol=1e-9)


@pytest.mark.parametrize("H", [0.3, 1.2, 7.0])
def test_dini_basis_is_orthonormal_in_a_H(H):
    rho = O.dini_roots(H, 5)
    C = O.dini_C(rho, H)
    for p in range(5):
        for q in range(p, 5):
            grad = si.quad(lambda s: 2 * math.pi * s * C[p] * C[q] * rho[p] * rho[q] * sp.j1(rho[p] * s)
                           * sp.j1(rho[q] * s), 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
            bnd = 2 * math.pi * H * C[p] * C[q] * sp.j0(rho[p]) * sp.j0(rho[q])
            assert abs(grad + bnd - (1.0 if p == q else 0.0)) < 1e-11, (p, q)


@pytest.mark.parametrize("k", [0.05, 0.3])
def test_y0_meets_the_robin_condition(k):
    H = O.robin_H(k)
    h = 1e-5 * k
    d = (sp.y0(k * (1 + h / k)) - sp.y0(k * (1 - h / k))) / (2 * h / k)   # d/ds Y0(k s) at s = 1
    assert abs(d + H * sp.y0(k)) < 1e-8 * abs(H * sp.y0(k))
    assert H > 0 and O.robin_applies(k) and not O.robin_applies(0.5)


def test_robin_fit_is_short_and_converges():
    k, a = 0.1, 0.03
    H = O.robin_H(k)
    g = lambda s: sp.y0(k * s)  # noqa: E731
    gp = lambda s: -k * sp.y1(k * s)  # noqa: E731
    errs = []
    for P in (10, 20, 40, 80):
        rho, C, alpha = O.robin_coefficients(g, gp, a, P, H, 2 * k)
        errs.append(O.fit_linf_error(g, rho, C, alpha, a, 2 * k))
    assert all(e2 < e1 / 5 for e1, e2 in zip(errs[:-1], errs[1:3])), errs
    # the first-root scaling of Sec. 4.2 (R9) for the same geometry: R = k' / kappa stretches the
    # interval by k' / k ~ 9, and reaching the same error takes many times more terms
    tol = errs[2]
    kp = O.y0_first_root_at_least(k)
    a2 = a * k / kp
    g2 = lambda s: sp.y0(kp * s)  # noqa: E731
    g2p = lambda s: -kp * sp.y1(kp * s)  # noqa: E731
    P2, *_ = O.choose_P(g2, g2p, a2, tol, O.initial_P(a2, tol, 2 * kp), 2 * kp)
    assert P2 > 4 * 40, P2


@pytest.mark.parametrize("kappa", [0.05, 0.2])
def test_robin_sbd_meets_the_output_bound(kappa):
    z = W.disk_points(800, 43)
    f = W.rhs(800, 44, complex_valued=True)
    dmin = math.sqrt(20 / 800)
    pl = O.make_plan(z, "helmholtz", dmin, 1e-6, kappa=kappa)
    assert pl.scale_R == pl.delta_max and O.robin_applies(kappa * pl.delta_max)
    q = O.sbd_matvec(pl, f)
    qd = O.direct_sum(z, f, "helmholtz", kappa)
    assert np.max(np.abs(q - qd)) <= 1e-6 * np.abs(f).sum()
