"""CPU FP64 oracle for the Sparse Bessel Decomposition (SBD) discrete convolution.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (no kernels, tables or helpers); the two meet only
in the seeded input generators of ``workloads``.

It is deliberately plain and slow: NumPy/SciPy in float64, library special
functions, Gauss-Legendre quadrature, a Cholesky solve, and direct exponential
sums in place of any fast transform.  Every function names the passage of
M. Averseng, "Fast discrete convolution in R^2 using Sparse Bessel
Decomposition" (arXiv:1711.07877) that it restates.

Readings taken where the paper is silent or ambiguous (each also listed in the
design notes):
  R1  The self interaction l = k is excluded from the sum of Eq. (discreteConv)
      (G is singular at 0); D_kk = -G_approx(0) cancels the far part's self term.
  R2  delta_max is taken as 2 max_k |z_k - c| (c = bounding-box centre), an upper
      bound of the diameter (Sec. 3.1 allows any bound).
  R3  The Bessel argument of the Sec. 1 series reads J0(rho_p r / delta_max).
  R4  Coefficients are expressed on the normalised basis e_p = C_p J0(rho_p r)
      (Sec. 2.1), so omega_hat = alpha_p C_p / M_p (Sec. 6.2).
  R5  The off-diagonal closed form of A^P (Sec. 3.2) is used with the opposite
      sign (denominator rho_i^2 - rho_j^2); the printed sign disagrees with the
      integral definition, which the quadrature Gram follows.
  R6  The circle size M_p is the smallest even M >= rho_p with
      2 sum_{j>=1} |J_{jM}(rho_p)| |alpha_p C_p| <= eps_q / P  (the exact aliasing
      series of Sec. 5, worst case at |x| = delta_max); evenness makes the node
      set symmetric under xi -> -xi so G_approx is real for a real kernel.
  R7  eps is split into eps/3 for the fit, eps/3 for the circular quadrature and
      eps/3 left to the fast transform of the CUDA path (the paper splits
      eps/2 + eps/2 between fit and quadrature, Sec. 6.1).
  R8  Pairs at distance exactly delta_min are near pairs (<=, Sec. 1).
  R9  Helmholtz: G(x) = (i/4) H0^(1)(kappa |x|) = (i/4) J0 - (1/4) Y0; the J0 part is
      one circle of radius kappa (Sec. 1 circle identity), the Y0 part is an SBD
      of Y0(k' s) with k' the first root of Y0 >= kappa delta_max, scaled by
      R = k'/kappa (Sec. 4.2).
  R10 The L_inf stopping test of the P search (Sec. 1) is evaluated on the
      fixed sample set ``fit_error_samples`` of [a, 1], dense near a (where the
      paper advises to monitor it), and the dichotomy stops at a resolution of
      max(1, P // 128) terms (``choose_P``).
  R14 General radial kernels (Sec. 4.3), in the scaled variable s = r / delta_max:
      K(s) = sum_t mu_t J0(omega_t s) / J0(omega_t) with the n conditions
      (-Delta)^j (g - K)(1) = 0, j = 1..n, i.e. M mu = lambda with M_jt =
      (-1)^j omega_t^(2j) and lambda_j = Delta^j g(1) (the printed system pairs
      (-1)^j in M with (-Delta)^j in lambda, which differ by (-1)^j; the
      condition itself is the multi-Dirichlet one of Sec. 2.2).  The order-0
      condition is met by the constant c = g(1) - K(1), carried by the xi = 0
      node.  omega' = sqrt of the mean |lambda_{j+1} / lambda_j| over
      j = 1..n (n + 1 iterates); omega_1..omega_n are the roots of J1 nearest
      omega', nearest first.  The SBD then fits h = g - K - c.
  R15 Low-wavenumber Helmholtz (Sec. 4.2, third case, with the Dini series of
      Sec. 2.3): used when kappa delta_max is below half the first root of Y0
      (where the first-root scaling of R9 would stretch R beyond 2 delta_max).
      g(s) = Y0(k s), k = kappa delta_max, fitted on (a, 1) in the Dini basis
      e_p = C_p J0(rho_p s), rho_p the positive roots of rho J1(rho) = H J0(rho)
      (rho J0'(rho) + H J0(rho) = 0), H = k Y1(k) / Y0(k) (> 0 there), C_p
      normalising e_p in a_H(u, v) = int_B grad u . grad v + H int_C u v.  The
      coefficients minimise the same form restricted to the annulus: the
      gradient term over A(a) plus the boundary term H int_C at r = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.special as sp

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# Kernels and the direct sum (Introduction, Eq. discreteConv; Sec. 4.1, 4.2, 4.3)
# ---------------------------------------------------------------------------

@dataclass
class RadialKernel:
    """A real radial kernel of Sec. 4.3, given by functions of r > 0: value(r) = G(r),
    deriv(r) = G'(r), and lap(j, r) = (Delta^j G)(r) for j >= 1, Delta = d^2/dr^2 + (1/r) d/dr
    the radial Laplacian.  log_coef is c in G = c log r + (a function smooth at 0); the oracle
    does not use it (the CUDA path tabulates the near field with it)."""
    value: object
    deriv: object
    lap: object
    log_coef: float = 0.0


def is_complex_kind(kind) -> bool:
    return isinstance(kind, str) and kind == "helmholtz"


def kernel_G(r: np.ndarray, kind, kappa: float = 0.0) -> np.ndarray:
    """G(r): Laplace -log(r)/(2 pi) (Introduction) or Helmholtz (i/4) H0^(1)(kappa r) (R9); for a
    RadialKernel (Sec. 4.3) its own value."""
    r = np.asarray(r, dtype=np.float64)
    if isinstance(kind, RadialKernel):
        return kind.value(r)
    if kind == "laplace":
        return -np.log(r) / TWO_PI
    if kind == "helmholtz":
        return 0.25j * sp.hankel1(0, kappa * r)
    raise ValueError(kind)


def direct_sum(z: np.ndarray, f: np.ndarray, kind: str, kappa: float = 0.0,
               targets: np.ndarray | None = None, chunk: int = 512) -> np.ndarray:
    """q_k = sum_{l != k} G(z_k - z_l) f_l, Eq. (discreteConv), reading R1.

    ``targets`` (indices into z) restricts k to a subsample; all l are summed.
    f may be (N,) or (nrhs, N); the result has the matching leading shape.
    """
    z = np.asarray(z, dtype=np.float64)
    f = np.asarray(f)
    single = f.ndim == 1
    F = f[None, :] if single else f
    idx = np.arange(len(z)) if targets is None else np.asarray(targets)
    out_dtype = np.complex128 if (is_complex_kind(kind) or np.iscomplexobj(F)) else np.float64
    q = np.zeros((F.shape[0], len(idx)), dtype=out_dtype)
    for s in range(0, len(idx), chunk):
        ks = idx[s:s + chunk]
        d = np.hypot(z[ks, 0][:, None] - z[None, :, 0], z[ks, 1][:, None] - z[None, :, 1])
        self_mask = d == 0.0
        d_safe = np.where(self_mask, 1.0, d)
        g = kernel_G(d_safe, kind, kappa)
        g = np.where(self_mask, 0.0, g)
        q[:, s:s + len(ks)] = (g @ F.T).T
    return q[0] if single else q


# ---------------------------------------------------------------------------
# Bessel roots and the normalised basis (Sec. 2.1)
# ---------------------------------------------------------------------------

def j0_roots(P: int) -> np.ndarray:
    """rho_1 < ... < rho_P, the positive roots of J0 (Definition of Sec. 2.1)."""
    return sp.jn_zeros(0, P).astype(np.float64)


def y0_first_root_at_least(x: float) -> float:
    """The first root of Y0 that is >= x (Sec. 4.2, choice of k')."""
    s = max(1, int(x / math.pi) - 2)
    while True:
        roots = sp.yn_zeros(0, s + 8)
        hit = roots[roots >= x]
        if hit.size:
            return float(hit[0])
        s += 8


def normalisation_C(rho: np.ndarray) -> np.ndarray:
    """C_p = 1 / (sqrt(pi) rho_p |J1(rho_p)|) so that ||e_p||_{H^1_0} = 1 (Sec. 2.1)."""
    return 1.0 / (math.sqrt(math.pi) * rho * np.abs(sp.j1(rho)))


# ---------------------------------------------------------------------------
# Gauss-Legendre quadrature on [a, 1] (composite, graded panels)
# ---------------------------------------------------------------------------

def gauss_legendre(a: float, b: float, h: float, order: int = 24):
    """Composite Gauss-Legendre rule on [a, b] with panels of length <= h.

    Panels grow geometrically (ratio 2) from a until they reach h, so that
    integrands with a singularity at 0 (1/s, Y1) stay resolved next to a.
    """
    x, w = sp.roots_legendre(order)
    edges = [a]
    step = min(h, a) if a > 0 else h
    while edges[-1] < b:
        edges.append(min(b, edges[-1] + step))
        step = min(h, 2.0 * step)
    edges = np.asarray(edges)
    half = 0.5 * np.diff(edges)
    mid = 0.5 * (edges[1:] + edges[:-1])
    nodes = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    weights = (half[:, None] * w[None, :]).ravel()
    return nodes, weights


def _panel_length(rho_max: float, extra_freq: float = 0.0) -> float:
    # integrands oscillate with angular frequency <= 2 rho_max (+ extra_freq);
    # a 24-point Gauss panel spanning about one period integrates that to rounding
    return min(0.125, 6.0 / (2.0 * rho_max + extra_freq))


# ---------------------------------------------------------------------------
# The SBD fit: Gram matrix, right-hand side, solve (Sec. 3.1, 3.2)
# ---------------------------------------------------------------------------

def gram_quadrature(rho: np.ndarray, a: float, C: np.ndarray | None = None) -> np.ndarray:
    """A_pq = int_{A(a)} grad e_p . grad e_q = 2 pi C_p C_q rho_p rho_q int_a^1 s J1(rho_p s) J1(rho_q s) ds.

    Gram matrix of the quadratic form Q^P (Sec. 3.1) on the annulus A(a), by
    composite Gauss-Legendre quadrature of its integral definition (Sec. 3.2).
    """
    C = normalisation_C(rho) if C is None else C
    s, w = gauss_legendre(a, 1.0, _panel_length(float(rho.max())))
    B = (C * rho)[:, None] * sp.j1(rho[:, None] * s[None, :])  # (P, nq): -(d/ds) e_p
    return TWO_PI * (B * (w * s)[None, :]) @ B.T


def gram_closed_form(rho: np.ndarray, a: float) -> np.ndarray:
    """The explicit A^P of Sec. 3.2 (Green's formula), reading R5 for the off-diagonal sign.

    F_ij(r) = rho_i r J0(rho_i r) J0'(rho_j r), F_i(r) as printed; valid for any rho.
    """
    C = normalisation_C(rho)
    P = len(rho)

    def F_ij(ri, rj, r):
        return ri * r * sp.j0(ri * r) * (-sp.j1(rj * r))

    def F_i(ri, r):
        j0v = sp.j0(ri * r)
        dj0 = -sp.j1(ri * r)
        return ri * ri * r * r * (0.5 * j0v * j0v + 0.5 * dj0 * dj0) + ri * r * j0v * dj0

    A = np.empty((P, P))
    ri = rho[:, None]
    rj = rho[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        bracket = (F_ij(ri, rj, 1.0) - F_ij(rj, ri, 1.0) - F_ij(ri, rj, a) + F_ij(rj, ri, a))
        off = TWO_PI * C[:, None] * C[None, :] * ri * rj / (ri * ri - rj * rj) * bracket
    A[:] = off
    diag = TWO_PI * C * C * (F_i(rho, 1.0) - F_i(rho, a))
    A[np.arange(P), np.arange(P)] = diag
    return A


def rhs_quadrature(g_prime, rho: np.ndarray, a: float, C: np.ndarray | None = None,
                   extra_freq: float = 0.0) -> np.ndarray:
    """b_p = int_{A(a)} grad g . grad e_p = 2 pi int_a^1 s g'(s) (-C_p rho_p J1(rho_p s)) ds.

    Right-hand side of the normal equations Eq. (LinearSystem) in the e_p basis.
    """
    C = normalisation_C(rho) if C is None else C
    s, w = gauss_legendre(a, 1.0, _panel_length(float(rho.max()), extra_freq))
    B = (C * rho)[:, None] * sp.j1(rho[:, None] * s[None, :])
    return -TWO_PI * (B * (w * s * g_prime(s))[None, :]).sum(axis=1)


def sbd_coefficients(g_prime, a: float, P: int, extra_freq: float = 0.0):
    """SBD coefficients of order P: minimiser of Q^P (Sec. 3.1) by Cholesky (Sec. 3.2).

    Returns (rho, C, alpha) with g(s) ~ sum_p alpha_p C_p J0(rho_p s) on (a, 1).
    """
    rho = j0_roots(P)
    C = normalisation_C(rho)
    A = gram_quadrature(rho, a, C)
    b = rhs_quadrature(g_prime, rho, a, C, extra_freq)
    L = np.linalg.cholesky(A)
    y = sla.solve_triangular(L, b, lower=True)
    alpha = sla.solve_triangular(L.T, y, lower=False)
    return rho, C, alpha


def fit_error_samples(a: float, extra_freq: float = 0.0) -> np.ndarray:
    """Sample set of [a, 1] for the L_inf stopping test (reading R10).

    512 points a + d (i/511)^2 with d = min(1 - a, 30 a), dense next to a where the
    paper advises to monitor the error (Sec. 1), plus U = 256 + 4 ceil(extra_freq/pi)
    uniform points a + (1 - a) j / (U - 1) (extra_freq = 2 k' for the Y0 fit, whose
    error oscillates at that frequency over the whole interval).
    """
    d = min(1.0 - a, 30.0 * a)
    near = a + d * (np.arange(512) / 511.0) ** 2
    U = 256 + 4 * int(math.ceil(extra_freq / math.pi))
    uni = a + (1.0 - a) * np.arange(U) / (U - 1.0)
    return np.unique(np.concatenate([near, uni]))


def series_value(s: np.ndarray, rho: np.ndarray, C: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """sum_p alpha_p C_p J0(rho_p s)."""
    s = np.atleast_1d(s)
    out = np.zeros(s.shape, dtype=np.result_type(alpha.dtype, np.float64))
    for i in range(0, len(rho), 256):
        out += (alpha[i:i + 256] * C[i:i + 256]) @ sp.j0(rho[i:i + 256, None] * s[None, :])
    return out


def fit_linf_error(g, rho, C, alpha, a: float, extra_freq: float = 0.0) -> float:
    """max_{s in samples} |g(s) - sum_p alpha_p C_p J0(rho_p s)| (reading R10)."""
    s = fit_error_samples(a, extra_freq)
    return float(np.max(np.abs(g(s) - series_value(s, rho, C, alpha))))


def initial_P(a: float, tol: float, extra_freq: float = 0.0) -> int:
    """Starting P of the search: gamma = P a from the observed Laplace rate (Sec. 4.1,
    log10 err ~ -0.5 - 1.5 gamma), plus k'/pi Bessel terms for the Y0 fit (Sec. 4.2)."""
    gamma = max(0.5, (-math.log10(tol) - 0.5) / 1.5)
    return max(2, int(math.ceil(gamma / a)) + int(math.ceil(extra_freq / (2.0 * math.pi))))


def choose_P(g, g_prime, a: float, tol: float, P_start: int, extra_freq: float = 0.0,
             P_max: int = 20000, coefficients=None):
    """A P whose fit error is <= tol, by bracketing then dichotomy (Sec. 1).

    Bracket: from P_start, grow by factors 1.1 (ceil) while the error is above tol,
    or shrink by factors 0.9 (floor) while it is below.  Dichotomy on the bracket
    (lo fails, hi passes) until hi - lo <= max(1, hi // 128): the smallest
    passing P when P < 256, within 1% above it beyond.
    ``coefficients(P)`` replaces the Dirichlet fit (the Robin basis of R15).
    Returns (P, rho, C, alpha, err).
    """
    cache = {}

    def err_of(P):
        if P not in cache:
            rho, C, alpha = (coefficients(P) if coefficients is not None
                             else sbd_coefficients(g_prime, a, P, extra_freq))
            cache[P] = (fit_linf_error(g, rho, C, alpha, a, extra_freq), rho, C, alpha)
        return cache[P][0]

    P = max(1, P_start)
    if err_of(P) > tol:
        lo, hi = P, int(math.ceil(P * 1.1))
        while err_of(hi) > tol:
            if hi >= P_max:
                raise RuntimeError(f"SBD fit does not reach {tol:g} with P <= {P_max}")
            lo, hi = hi, min(P_max, int(math.ceil(hi * 1.1)))
    else:
        hi, lo = P, int(math.floor(P * 0.9))
        while lo >= 1 and err_of(lo) <= tol:
            hi, lo = lo, int(math.floor(lo * 0.9))
        lo = max(lo, 0)
    res = max(1, hi // 128)
    while hi - lo > res:
        mid = (lo + hi) // 2
        if mid >= 1 and err_of(mid) <= tol:
            hi = mid
        else:
            lo = mid
    e, rho, C, alpha = cache[hi]
    return hi, rho, C, alpha, e


# ---------------------------------------------------------------------------
# Robin boundary condition: the Dini series (Sec. 2.3) for low-wavenumber Helmholtz (Sec. 4.2, R15)
# ---------------------------------------------------------------------------

def robin_applies(k: float) -> bool:
    """R15: the Dini series of Y0(k s) is used when k = kappa delta_max is below half the first
    root of Y0."""
    return k < 0.5 * float(sp.y0_zeros(1)[0][0].real)


def robin_H(k: float) -> float:
    """H = -k Y0'(k) / Y0(k) = k Y1(k) / Y0(k): the Robin constant that Y0(k s) satisfies at s = 1
    (Sec. 4.2)."""
    return float(k * sp.y1(k) / sp.y0(k))


def dini_roots(H: float, P: int) -> np.ndarray:
    """The first P positive roots of rho J0'(rho) + H J0(rho) = 0, i.e. rho J1(rho) = H J0(rho)
    (Sec. 2.3), H > 0: the p-th lies between the (p-1)-th root of J1 (0 for p = 1) and the p-th
    root of J0, where the function changes sign; brentq on each bracket."""
    from scipy.optimize import brentq
    f = lambda x: x * sp.j1(x) - H * sp.j0(x)  # noqa: E731
    j1z = np.concatenate([[0.0], sp.jn_zeros(1, P)])
    j0z = sp.jn_zeros(0, P)
    return np.array([brentq(f, j1z[p], j0z[p], xtol=1e-15, rtol=1e-15, maxiter=200) for p in range(P)])


def dini_C(rho: np.ndarray, H: float) -> np.ndarray:
    """C_p with a_H(e_p, e_p) = 1 (Sec. 2.3): 1 / C_p^2 = 2 pi (rho_p^2 int_0^1 s J1(rho_p s)^2 ds
    + H J0(rho_p)^2), the integral by Gauss-Legendre quadrature of its definition."""
    s, w = gauss_legendre(0.0, 1.0, _panel_length(float(rho.max())))
    J = sp.j1(rho[:, None] * s[None, :])
    integ = (J * J * (w * s)[None, :]).sum(axis=1)
    return 1.0 / np.sqrt(TWO_PI * (rho * rho * integ + H * sp.j0(rho) ** 2))


def robin_coefficients(g, g_prime, a: float, P: int, H: float, extra_freq: float = 0.0):
    """Coefficients of g in the Dini basis e_p = C_p J0(rho_p s) (R15): the minimiser of
    int_{A(a)} |grad(g - sum t_p e_p)|^2 + H int_C (g - sum t_p e_p)^2, by Cholesky of its Gram
    matrix (quadrature of the gradient term, the boundary term 2 pi H e_p(1) e_q(1))."""
    rho = dini_roots(H, P)
    C = dini_C(rho, H)
    s, w = gauss_legendre(a, 1.0, _panel_length(float(rho.max()), extra_freq))
    B = (C * rho)[:, None] * sp.j1(rho[:, None] * s[None, :])
    A = TWO_PI * (B * (w * s)[None, :]) @ B.T
    e1 = C * sp.j0(rho)
    A += TWO_PI * H * np.outer(e1, e1)
    b = -TWO_PI * (B * (w * s * g_prime(s))[None, :]).sum(axis=1) + TWO_PI * H * float(g(1.0)) * e1
    L = np.linalg.cholesky(A)
    alpha = sla.solve_triangular(L.T, sla.solve_triangular(L, b, lower=True), lower=False)
    return rho, C, alpha


# ---------------------------------------------------------------------------
# Circular quadrature (Sec. 5; nodes Eq. defXimp)
# ---------------------------------------------------------------------------

def aliasing_bound(M: int, r: float, n_terms: int = 4) -> float:
    """2 sum_{j=1..n_terms} |J_{jM}(r)|: the modulus bound of the aliasing series of Sec. 5."""
    return 2.0 * float(sum(abs(sp.jv(j * M, r)) for j in range(1, n_terms + 1)))


def circle_size(r: float, weight: float, tol: float) -> int:
    """Smallest even M >= r with aliasing_bound(M, r) * |weight| <= tol (reading R6).

    For M >= r every |J_{jM}| is increasing on [0, r] (its first maximum lies
    beyond order jM), so the aliasing error of Sec. 5 over all |x| <= scale is
    largest at the circle argument r itself.
    """
    M = max(2, 2 * int(math.ceil(0.5 * r)))
    while aliasing_bound(M, r) * abs(weight) > tol:
        M += 2
    return M


def circle_nodes(radius: float, M: int) -> np.ndarray:
    """xi_m = radius (cos 2 pi m / M, sin 2 pi m / M), m = 0..M-1 (Eq. defXimp)."""
    t = TWO_PI * np.arange(M) / M
    return radius * np.stack([np.cos(t), np.sin(t)], axis=1)


# ---------------------------------------------------------------------------
# The plan: weights omega_hat and frequencies xi (Sec. 1, Sec. 6.1, 6.2)
# ---------------------------------------------------------------------------

@dataclass
class OraclePlan:
    kind: str
    kappa: float
    z: np.ndarray
    delta_min: float
    delta_max: float
    eps: float
    scale_R: float          # radius scale of the Bessel circles (delta_max, or R for Y0)
    a: float                # delta_min / scale_R
    P: int
    rho: np.ndarray
    C: np.ndarray
    alpha: np.ndarray
    fit_err: float          # L_inf error of the fitted g on the sample set (g units)
    M: np.ndarray           # nodes per circle (Bessel circles first; Helmholtz J0 circle last)
    circle_radius: np.ndarray
    circle_weight: np.ndarray   # omega_hat per node of each circle (complex)
    w0: complex             # weight of the xi = 0 node (G(delta_max), Laplace)
    xi: np.ndarray          # (N_xi, 2)
    omega: np.ndarray       # (N_xi,) complex
    pairs: tuple | None = None
    D: np.ndarray | None = None   # values per pair (k, l), aligned with pairs
    x: np.ndarray | None = None   # targets, when they differ from the sources (make_plan_st)
    y: np.ndarray | None = None   # sources (make_plan_st)
    D_st: tuple | None = None     # rectangular close matrix (close_matrix_st)
    enforce: tuple | None = None  # general kernel (make_plan_radial): (omega, mu, c) of reading R14


def make_plan(z: np.ndarray, kind: str, delta_min: float, eps: float, kappa: float = 0.0,
              P: int | None = None, P_start: int | None = None) -> OraclePlan:
    """Off-line part (Sec. 1): SBD fit, circular quadrature, weights and frequencies.

    ``P`` fixes the number of Bessel terms; otherwise it is chosen by choose_P.
    """
    z = np.asarray(z, dtype=np.float64)
    c = 0.5 * (z.min(axis=0) + z.max(axis=0))
    delta_max = 2.0 * float(np.sqrt(np.max(np.sum((z - c) ** 2, axis=1))))   # R2
    if not (0.0 < delta_min < delta_max):
        raise ValueError("need 0 < delta_min < delta_max")
    eps_fit = eps / 3.0        # R7
    eps_q = eps / 3.0
    if kind == "laplace":
        # -log(r)/(2pi) = -(1/2pi) [log(delta_max) + log(s)], s = r / delta_max  (Sec. 4.1)
        scale_R = delta_max
        g = np.log
        g_prime = lambda s: 1.0 / s  # noqa: E731
        gscale = -1.0 / TWO_PI
        extra = 0.0
        w0 = complex(-math.log(delta_max) / TWO_PI)      # G(delta_max): the xi = 0 term (Sec. 1)
    elif kind == "helmholtz" and robin_applies(kappa * delta_max):
        # low wavenumber: Dini series of Y0(k s), k = kappa delta_max, on (a, 1)  (R15)
        k = kappa * delta_max
        scale_R = delta_max
        g = lambda s: sp.y0(k * s)  # noqa: E731
        g_prime = lambda s: -k * sp.y1(k * s)  # noqa: E731
        gscale = -0.25
        extra = 2.0 * k
        w0 = 0.0j
    elif kind == "helmholtz":
        kp = y0_first_root_at_least(kappa * delta_max)   # k' (Sec. 4.2)
        scale_R = kp / kappa
        g = lambda s: sp.y0(kp * s)  # noqa: E731
        g_prime = lambda s: -kp * sp.y1(kp * s)  # noqa: E731
        gscale = -0.25
        extra = 2.0 * kp
        w0 = 0.0j
    else:
        raise ValueError(kind)
    a = delta_min / scale_R
    tol_fit = eps_fit / abs(gscale)
    robin = kind == "helmholtz" and robin_applies(kappa * delta_max)
    coefficients = None
    if robin:
        H = robin_H(kappa * delta_max)
        coefficients = lambda Pq: robin_coefficients(g, g_prime, a, Pq, H, extra)  # noqa: E731
    if P is None:
        if P_start is None:
            P_start = initial_P(a, tol_fit, extra)
        P, rho, C, alpha, err = choose_P(g, g_prime, a, tol_fit, P_start, extra, coefficients=coefficients)
    else:
        rho, C, alpha = coefficients(P) if robin else sbd_coefficients(g_prime, a, P, extra)
        err = fit_linf_error(g, rho, C, alpha, a, extra)
    coef = gscale * alpha * C      # kernel units: G ~ const + sum_p coef_p J0(rho_p r / scale_R)
    n_circles = P + (1 if kind == "helmholtz" else 0)
    M = np.array([circle_size(float(rho[p]), float(coef[p]), eps_q / n_circles) for p in range(P)],
                 dtype=np.int64)
    radius = rho / scale_R
    weight = (coef / M).astype(np.complex128)                # omega_hat = alpha_p C_p / M_p (Sec. 6.2)
    if kind == "helmholtz":
        # (i/4) J0(kappa r): one circle of radius kappa, exact by the identity of Sec. 1
        kd = kappa * delta_max
        Mj = circle_size(kd, 0.25, eps_q / n_circles)
        M = np.append(M, Mj)
        radius = np.append(radius, kappa)
        weight = np.append(weight, 0.25j / Mj)
    xi = [np.zeros((1, 2))] if w0 != 0 else []
    om = [np.array([w0])] if w0 != 0 else []
    for Mp, rp, wp in zip(M, radius, weight):
        xi.append(circle_nodes(float(rp), int(Mp)))
        om.append(np.full(int(Mp), wp, dtype=np.complex128))
    xi = np.concatenate(xi, axis=0)
    om = np.concatenate(om)
    return OraclePlan(kind, kappa, z, delta_min, delta_max, eps, scale_R, a, P, rho, C, alpha, err,
                      M, radius, weight, w0, xi, om)


# ---------------------------------------------------------------------------
# Type-3 transforms by definition (Introduction: NUFFT_{+-}[z, xi])
# ---------------------------------------------------------------------------

def nufft_direct(src: np.ndarray, dst: np.ndarray, c: np.ndarray, sign: int, chunk: int = 2048) -> np.ndarray:
    """out_j = sum_k exp(sign * i src_k . dst_j) c_k, by direct summation.

    NUFFT_{+-}[z, xi] of the Introduction: with src = z, dst = xi it maps C^{N_z}
    to C^{N_xi}; Eq. (far convolution) also applies it with the roles of z and
    xi exchanged (src = xi, dst = z), which is the same exponential sum.
    """
    c = np.asarray(c, dtype=np.complex128)
    out = np.zeros(len(dst), dtype=np.complex128)
    for s in range(0, len(dst), chunk):
        ph = dst[s:s + chunk] @ src.T
        out[s:s + chunk] = np.exp(sign * 1j * ph) @ c
    return out


# ---------------------------------------------------------------------------
# Near pairs and the close-correction matrix D (Sec. 1 Eq. defD; Sec. 6.1)
# ---------------------------------------------------------------------------

def near_pairs(z: np.ndarray, delta_min: float):
    """All ordered pairs (k, l), k != l, with |z_k - z_l| <= delta_min (R8), by brute force."""
    rows, cols = [], []
    for s in range(0, len(z), 1024):
        d2 = (z[s:s + 1024, 0][:, None] - z[None, :, 0]) ** 2 + (z[s:s + 1024, 1][:, None] - z[None, :, 1]) ** 2
        k, l = np.nonzero(d2 <= delta_min * delta_min)
        keep = (k + s) != l
        rows.append(k[keep] + s)
        cols.append(l[keep])
    return np.concatenate(rows), np.concatenate(cols)


def g_approx_direct(y: np.ndarray, xi: np.ndarray, omega: np.ndarray, chunk: int = 1024) -> np.ndarray:
    """G_approx(y) = sum_nu omega_nu exp(i y . xi_nu), Eq. (Gapprox), by direct summation."""
    out = np.zeros(len(y), dtype=np.complex128)
    for s in range(0, len(y), chunk):
        out[s:s + chunk] = np.exp(1j * (y[s:s + chunk] @ xi.T)) @ omega
    return out


def close_matrix(plan: OraclePlan):
    """D of Eq. (defD): G(z_k - z_l) - G_approx(z_k - z_l) on near pairs; D_kk = -G_approx(0) (R1).

    Returns (rows, cols, values) including the diagonal.
    """
    z = plan.z
    k, l = near_pairs(z, plan.delta_min)
    y = z[k] - z[l]
    r = np.hypot(y[:, 0], y[:, 1])
    gap = g_approx_direct(y, plan.xi, plan.omega)
    coincide = r == 0.0
    gval = np.where(coincide, 0.0, kernel_G(np.where(coincide, 1.0, r), plan.kind, plan.kappa))
    vals = gval - gap
    n = len(z)
    g0 = plan.omega.sum()
    rows = np.concatenate([k, np.arange(n)])
    cols = np.concatenate([l, np.arange(n)])
    vals = np.concatenate([vals, np.full(n, -g0)])
    return rows, cols, vals


# ---------------------------------------------------------------------------
# On-line part (Sec. 1; Sec. 6.2)
# ---------------------------------------------------------------------------

def far_part(plan: OraclePlan, f: np.ndarray) -> np.ndarray:
    """q_far = NUFFT_+[z, xi](omega_hat . NUFFT_-[z, xi](f)), Eq. (far convolution), steps (i)-(iii)."""
    fhat = nufft_direct(plan.z, plan.xi, f, -1)       # (i)  space -> Fourier
    ghat = plan.omega * fhat                         # (ii) Fourier multiply
    return nufft_direct(plan.xi, plan.z, ghat, +1)   # (iii) Fourier -> space


def close_part(plan: OraclePlan, f: np.ndarray) -> np.ndarray:
    """q_close = D f (Sec. 1, close correction)."""
    if plan.D is None:
        plan.D = close_matrix(plan)
    rows, cols, vals = plan.D
    out = np.zeros(len(plan.z), dtype=np.complex128)
    np.add.at(out, rows, vals * f[cols])
    return out


def sbd_matvec(plan: OraclePlan, f: np.ndarray) -> np.ndarray:
    """q = q_far + q_close (Sec. 1, on-line output).  Real for a real kernel and real f."""
    f = np.asarray(f)
    if f.ndim == 2:
        return np.stack([sbd_matvec(plan, fi) for fi in f])
    q = far_part(plan, f) + close_part(plan, f)
    if not is_complex_kind(plan.kind) and not np.iscomplexobj(f):
        return q.real
    return q


# ---------------------------------------------------------------------------
# Separate targets and sources (Sec. 7.1 and Table 2: q_k = sum_l G(x_k - y_l) f_l for two
# independent point sets x and y)
# ---------------------------------------------------------------------------

def direct_sum_st(x: np.ndarray, y: np.ndarray, f: np.ndarray, kind: str, kappa: float = 0.0,
                  targets: np.ndarray | None = None, chunk: int = 512) -> np.ndarray:
    """q_k = sum_l G(x_k - y_l) f_l over all sources y_l, for targets x_k (Sec. 7.1).

    A target that coincides with a source takes no contribution from it (reading R1 carried
    over: G is singular there; with x = y this is Eq. discreteConv).  ``targets`` (indices
    into x) restricts k; f may be (N_y,) or (nrhs, N_y).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    f = np.asarray(f)
    single = f.ndim == 1
    F = f[None, :] if single else f
    idx = np.arange(len(x)) if targets is None else np.asarray(targets)
    out_dtype = np.complex128 if (kind == "helmholtz" or np.iscomplexobj(F)) else np.float64
    q = np.zeros((F.shape[0], len(idx)), dtype=out_dtype)
    for s in range(0, len(idx), chunk):
        ks = idx[s:s + chunk]
        d = np.hypot(x[ks, 0][:, None] - y[None, :, 0], x[ks, 1][:, None] - y[None, :, 1])
        zero = d == 0.0
        g = kernel_G(np.where(zero, 1.0, d), kind, kappa)
        g = np.where(zero, 0.0, g)
        q[:, s:s + len(ks)] = (g @ F.T).T
    return q[0] if single else q


def make_plan_st(x: np.ndarray, y: np.ndarray, kind: str, delta_min: float, eps: float, kappa: float = 0.0,
                 P: int | None = None) -> OraclePlan:
    """Off-line part for targets x and sources y: the fit, circles and weights of make_plan
    taken for the union of the two sets, whose delta_max (R2) bounds every |x_k - y_l|."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    pl = make_plan(np.concatenate([x, y]), kind, delta_min, eps, kappa, P=P)
    pl.x, pl.y = x, y
    return pl


def near_pairs_st(x: np.ndarray, y: np.ndarray, delta_min: float):
    """All pairs (k, l) with |x_k - y_l| <= delta_min (R8), by brute force, coincident ones included."""
    rows, cols = [], []
    for s in range(0, len(x), 1024):
        d2 = (x[s:s + 1024, 0][:, None] - y[None, :, 0]) ** 2 + (x[s:s + 1024, 1][:, None] - y[None, :, 1]) ** 2
        k, l = np.nonzero(d2 <= delta_min * delta_min)
        rows.append(k + s)
        cols.append(l)
    return np.concatenate(rows), np.concatenate(cols)


def close_matrix_st(plan: OraclePlan):
    """Rectangular D of Eq. (defD): G(x_k - y_l) - G_approx(x_k - y_l) on near pairs, with G taken
    as 0 at distance 0 (so that D_kl = -G_approx(0) cancels the far part there, as the diagonal
    of the square case does).  Returns (rows, cols, values)."""
    k, l = near_pairs_st(plan.x, plan.y, plan.delta_min)
    d = plan.x[k] - plan.y[l]
    r = np.hypot(d[:, 0], d[:, 1])
    gap = g_approx_direct(d, plan.xi, plan.omega)
    zero = r == 0.0
    gval = np.where(zero, 0.0, kernel_G(np.where(zero, 1.0, r), plan.kind, plan.kappa))
    return k, l, gval - gap


def sbd_matvec_st(plan: OraclePlan, f: np.ndarray) -> np.ndarray:
    """q = NUFFT_+[x, xi](omega_hat . NUFFT_-[y, xi](f)) + D f (Sec. 1 on-line part with the
    sources y in the forward transform and the targets x in the backward one)."""
    f = np.asarray(f)
    if f.ndim == 2:
        return np.stack([sbd_matvec_st(plan, fi) for fi in f])
    fhat = nufft_direct(plan.y, plan.xi, f, -1)                  # (i)  sources -> Fourier
    q = nufft_direct(plan.xi, plan.x, plan.omega * fhat, +1)     # (ii), (iii) Fourier -> targets
    if plan.D_st is None:
        plan.D_st = close_matrix_st(plan)
    rows, cols, vals = plan.D_st
    np.add.at(q, rows, vals * f[cols])
    if plan.kind == "laplace" and not np.iscomplexobj(f):
        return q.real
    return q


# ---------------------------------------------------------------------------
# The SBD without its circular quadrature (the uniform-grid multiplier variant): the far
# part uses the fitted series itself, G_fit(r) = const + sum_p c_p J0(rho_p r / R) (Sec. 1,
# before the J0 terms are turned into plane waves on circles in Sec. 5), the near pairs G.
# ---------------------------------------------------------------------------

def series_kernel(plan: OraclePlan, r: np.ndarray) -> np.ndarray:
    """G_fit(r) in kernel units: Laplace w0 - (1/2pi) sum_p alpha_p C_p J0(rho_p r / delta_max)
    (Sec. 4.1, reading R4); Helmholtz -(1/4) sum_p alpha_p C_p J0(rho_p r / R) + (i/4) J0(kappa r)
    (Sec. 4.2, reading R9: the J0 part is exact, without its circle)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    s = r / plan.scale_R
    if plan.kind == "laplace":   # a real kernel (Sec. 4.1): w0 is stored as a complex weight
        return complex(plan.w0).real - series_value(s, plan.rho, plan.C, plan.alpha) / TWO_PI
    return -0.25 * series_value(s, plan.rho, plan.C, plan.alpha) + 0.25j * sp.j0(plan.kappa * r)


def series_matvec(plan: OraclePlan, f: np.ndarray, chunk: int = 256) -> np.ndarray:
    """q_k = sum_{l != k} K(|z_k - z_l|) f_l with K = G on the near pairs (|z_k - z_l| <= delta_min,
    reading R8) and K = G_fit beyond: the on-line output of the SBD when each J0 term is summed
    exactly instead of by its circle of plane waves (coincident points as the self pair, R1)."""
    z = plan.z
    f = np.asarray(f)
    if f.ndim == 2:
        return np.stack([series_matvec(plan, fi, chunk) for fi in f])
    out_dtype = np.complex128 if (plan.kind == "helmholtz" or np.iscomplexobj(f)) else np.float64
    q = np.zeros(len(z), dtype=out_dtype)
    for s in range(0, len(z), chunk):
        d = np.hypot(z[s:s + chunk, 0][:, None] - z[None, :, 0], z[s:s + chunk, 1][:, None] - z[None, :, 1])
        near = d <= plan.delta_min
        zero = d == 0.0
        kfit = series_kernel(plan, d.ravel()).reshape(d.shape)
        kg = kernel_G(np.where(zero, 1.0, d), plan.kind, plan.kappa)
        k = np.where(near, kg, kfit)
        k = np.where(zero, 0.0, k)
        q[s:s + chunk] = k @ f
    if plan.kind == "laplace" and not np.iscomplexobj(f):
        return q.real
    return q


# ---------------------------------------------------------------------------
# General radial kernels: the multi-Dirichlet condition enforced by a few J0 terms (Sec. 4.3)
# ---------------------------------------------------------------------------

def dirichlet_frequencies(lam: np.ndarray, n: int) -> np.ndarray:
    """omega_1..omega_n of Sec. 4.3 (reading R14): omega' = sqrt of the mean ratio |lam_{j+1} /
    lam_j| of successive iterates (lam holds Delta^j g(1) for j = 1..n+1), then the roots of J1
    nearest omega', nearest first."""
    ratios = [abs(lam[j + 1] / lam[j]) for j in range(n) if lam[j] != 0.0]
    w = math.sqrt(sum(ratios) / len(ratios)) if ratios else 1.0
    roots = sp.jn_zeros(1, int(w / math.pi) + n + 4)
    order = np.argsort(np.abs(roots - w), kind="stable")
    return np.sort(roots[order[:n]])


def dirichlet_correction(lam: np.ndarray, n: int):
    """(omega, mu) of K(s) = sum_t mu_t J0(omega_t s) / J0(omega_t) with Delta^j K(1) = lam_j for
    j = 1..n: the system M mu = lam of Sec. 4.3, M_jt = (-1)^j omega_t^(2j) (reading R14)."""
    if n == 0:
        return np.zeros(0), np.zeros(0)
    omega = dirichlet_frequencies(lam, n)
    j = np.arange(1, n + 1)[:, None]
    M = (-1.0) ** j * omega[None, :] ** (2 * j)
    mu = np.linalg.solve(M, np.asarray(lam[:n], dtype=np.float64))
    return omega, mu


def correction_value(s, omega, mu):
    """K(s) = sum_t mu_t J0(omega_t s) / J0(omega_t)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    if len(omega) == 0:
        return np.zeros(s.shape)
    return (sp.j0(np.outer(s, omega)) / sp.j0(omega)[None, :]) @ mu


def correction_deriv(s, omega, mu):
    """K'(s) = -sum_t mu_t omega_t J1(omega_t s) / J0(omega_t)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    if len(omega) == 0:
        return np.zeros(s.shape)
    return -(sp.j1(np.outer(s, omega)) * (omega / sp.j0(omega))[None, :]) @ mu


def radial_fit(kern: RadialKernel, R: float, a: float, tol: float, n_enforce: int = 0, P: int | None = None):
    """The SBD of a general real radial kernel on (a, 1) in s = r / R (Sec. 4.3 with Sec. 3):
    lambda_j = Delta_s^j g(1) = R^(2j) (Delta^j G)(R) for j = 1..n+1, the correction K and constant
    c of reading R14, then the Sec. 3 fit of h = g - K - c, its P chosen by choose_P against tol
    (kernel units) unless given.  Returns (P, rho, C, alpha, err, omega, mu, c)."""
    lam = np.array([R ** (2 * j) * float(kern.lap(j, R)) for j in range(1, n_enforce + 2)])
    omega, mu = dirichlet_correction(lam, n_enforce)
    cst = float(kern.value(R)) - float(correction_value(1.0, omega, mu)[0])
    h = lambda s: kern.value(R * s) - correction_value(s, omega, mu) - cst  # noqa: E731
    h_prime = lambda s: R * kern.deriv(R * s) - correction_deriv(s, omega, mu)  # noqa: E731
    extra = 2.0 * float(omega.max()) if len(omega) else 0.0
    if P is None:
        P, rho, C, alpha, err = choose_P(h, h_prime, a, tol, initial_P(a, tol, extra), extra)
    else:
        rho, C, alpha = sbd_coefficients(h_prime, a, P, extra)
        err = fit_linf_error(h, rho, C, alpha, a, extra)
    return P, rho, C, alpha, err, omega, mu, cst


def make_plan_radial(z: np.ndarray, kern: RadialKernel, delta_min: float, eps: float, n_enforce: int = 0,
                     P: int | None = None) -> OraclePlan:
    """Off-line part for a general real radial kernel (Sec. 4.3; circles of Sec. 5): radial_fit
    with R = delta_max, one circle per Bessel term of h and per term of K (Sec. 1 identity), and
    the constant c at xi = 0.  The plan's alpha holds h's coefficients in the e_p basis."""
    z = np.asarray(z, dtype=np.float64)
    c0 = 0.5 * (z.min(axis=0) + z.max(axis=0))
    delta_max = 2.0 * float(np.sqrt(np.max(np.sum((z - c0) ** 2, axis=1))))   # R2
    if not (0.0 < delta_min < delta_max):
        raise ValueError("need 0 < delta_min < delta_max")
    eps_fit, eps_q = eps / 3.0, eps / 3.0      # R7
    R = delta_max
    a = delta_min / R
    P, rho, C, alpha, err, omega, mu, cst = radial_fit(kern, R, a, eps_fit, n_enforce, P)
    coef = alpha * C                          # kernel units (no scale: the kernel is G itself)
    n_circles = P + len(omega)
    M = [circle_size(float(rho[p]), float(coef[p]), eps_q / n_circles) for p in range(P)]
    radius = list(rho / R)
    weight = list(coef / np.array(M, dtype=np.float64))
    for om, m in zip(omega, mu):
        wt = float(m / sp.j0(om))
        Mt = circle_size(float(om), wt, eps_q / n_circles)
        M.append(Mt)
        radius.append(om / R)
        weight.append(wt / Mt)
    M = np.array(M, dtype=np.int64)
    radius = np.array(radius)
    weight = np.array(weight, dtype=np.complex128)
    w0 = complex(cst)
    xi = [np.zeros((1, 2))]
    om_list = [np.array([w0])]
    for Mp, rp, wp in zip(M, radius, weight):
        xi.append(circle_nodes(float(rp), int(Mp)))
        om_list.append(np.full(int(Mp), wp, dtype=np.complex128))
    return OraclePlan(kern, 0.0, z, delta_min, delta_max, eps, R, a, P, rho, C, alpha, err, M, radius, weight,
                      w0, np.concatenate(xi, axis=0), np.concatenate(om_list), enforce=(omega, mu, cst))


def radial_series_kernel(plan: OraclePlan, r) -> np.ndarray:
    """G_fit(r) = c + K(s) + sum_p alpha_p C_p J0(rho_p s), s = r / delta_max: the general-kernel
    series whose circles the plan quadratures (Sec. 4.3, R14)."""
    omega, mu, cst = plan.enforce
    s = np.atleast_1d(np.asarray(r, dtype=np.float64)) / plan.scale_R
    return cst + correction_value(s, omega, mu) + series_value(s, plan.rho, plan.C, plan.alpha)
