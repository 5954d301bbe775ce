"""Seeded synthetic inputs for the SBD matvec (points, right-hand sides, delta_min).

This module holds no arithmetic of the method itself: it only draws point
clouds and vectors shaped like the paper's numerical tests (Sec. 7: points
uniform in a square; boundary-integral setting of the Introduction: points
on closed curves) and the workload parameters that go with them.  It is
shared by the oracle-based tests and by the CUDA path's tests and bench,
and imports neither.

Recipes (all FP64, all seeded with numpy's PCG64 via default_rng):

* ``disk``   - N points uniform in the unit disk (radius sqrt(u), angle 2 pi v).
* ``curves`` - N points uniform in arc length on 8 random star-shaped closed
  curves r(theta) = 1 + 0.3 sum_{m<=5} a_m cos(m theta + phi_m), a_m ~ U(0,1)/m,
  phi_m ~ U(0, 2 pi), centres uniform in [1.7, 8.3]^2 (so every curve stays in
  [0, 10]^2); N is split between curves in proportion to their length.
* ``square`` - N points uniform in [0, 1]^2.
* right-hand sides: f ~ N(0, 1), real or complex (re, im independent).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def disk_points(n: int, seed: int) -> np.ndarray:
    """N points uniform in the unit disk, shape (n, 2), float64."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.random(n))
    t = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def square_points(n: int, seed: int) -> np.ndarray:
    """N points uniform in [0, 1]^2, shape (n, 2), float64."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 2))


def _star_curve(rng: np.random.Generator):
    a = rng.random(5) / np.arange(1, 6)
    phi = 2.0 * np.pi * rng.random(5)
    centre = 1.7 + 6.6 * rng.random(2)
    m = np.arange(1, 6)

    def radius(t):
        return 1.0 + 0.3 * np.sum(a[None, :] * np.cos(m[None, :] * t[:, None] + phi[None, :]), axis=1)

    def dradius(t):
        return -0.3 * np.sum(a[None, :] * m[None, :] * np.sin(m[None, :] * t[:, None] + phi[None, :]), axis=1)

    return centre, radius, dradius


def _curve_tables(rng: np.random.Generator, n_curves: int, n_table: int):
    curves = [_star_curve(rng) for _ in range(n_curves)]
    t = np.linspace(0.0, 2.0 * np.pi, n_table + 1)
    tables = []
    for centre, radius, dradius in curves:
        r = radius(t)
        dr = dradius(t)
        speed = np.sqrt(r * r + dr * dr)
        tables.append(np.concatenate([[0.0], np.cumsum(0.5 * (speed[1:] + speed[:-1]) * np.diff(t))]))
    return curves, t, tables


def curve_length(seed: int, n_curves: int = 8, n_table: int = 1 << 16) -> float:
    """Total arc length of the curves that ``curve_points(., seed)`` samples."""
    _, _, tables = _curve_tables(np.random.default_rng(seed), n_curves, n_table)
    return float(sum(c[-1] for c in tables))


def curve_points(n: int, seed: int, n_curves: int = 8, n_table: int = 1 << 16) -> np.ndarray:
    """N points uniform in arc length on ``n_curves`` random star-shaped curves."""
    rng = np.random.default_rng(seed)
    curves, t, tables = _curve_tables(rng, n_curves, n_table)
    lengths = np.asarray([c[-1] for c in tables])
    counts = np.floor(n * lengths / lengths.sum()).astype(np.int64)
    counts[: n - counts.sum()] += 1
    pts = []
    for (centre, radius, _), cum, cnt in zip(curves, tables, counts):
        s = (np.arange(cnt) + rng.random(cnt)) * (cum[-1] / max(cnt, 1))
        s = np.clip(s, 0.0, cum[-1])
        tt = np.interp(s, cum, t)
        r = radius(tt)
        pts.append(np.stack([centre[0] + r * np.cos(tt), centre[1] + r * np.sin(tt)], axis=1))
    z = np.concatenate(pts, axis=0)
    return z[rng.permutation(len(z))]


def rhs(n: int, seed: int, nrhs: int = 1, complex_valued: bool = False) -> np.ndarray:
    """f ~ N(0, 1): shape (n,) for nrhs == 1, else (nrhs, n) (one row per RHS)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs == 1 else (nrhs, n)
    f = rng.standard_normal(shape)
    if complex_valued:
        f = f + 1j * rng.standard_normal(shape)
    return f


def enclosing_diameter(z: np.ndarray) -> float:
    """2 max_k |z_k - c| with c the bounding-box centre: an upper bound of the diameter."""
    c = 0.5 * (z.min(axis=0) + z.max(axis=0))
    return 2.0 * float(np.sqrt(np.max(np.sum((z - c) ** 2, axis=1))))


def theorem1_delta_min(n: int, eps: float, delta_max: float, alpha: float = 0.0) -> float:
    """delta_min = a delta_max with a = |log eps|^(2/3) / N^(2/3 - alpha) (Theorem 1)."""
    a = abs(math.log(eps)) ** (2.0 / 3.0) / n ** (2.0 / 3.0 - alpha)
    return a * delta_max


@dataclass
class Workload:
    """One seeded problem instance: points, rhs, kernel and tolerances."""

    name: str
    z: np.ndarray
    f: np.ndarray
    kernel: str  # "laplace" | "helmholtz"
    kappa: float
    delta_min: float
    eps: float
    meta: dict = field(default_factory=dict)
    y: np.ndarray | None = None   # sources when they differ from the targets z (else None)


def laplace_disk(n: int = 2000, seed: int = 1, eps: float = 1e-6, neighbours: float = 20.0) -> Workload:
    """Laplace kernel, N points uniform in the unit disk, delta_min giving ~20 neighbours."""
    z = disk_points(n, seed)
    f = rhs(n, seed + 1000)
    delta_min = math.sqrt(neighbours / n)
    return Workload(f"laplace_disk_n{n}", z, f, "laplace", 0.0, delta_min, eps,
                    {"seed": seed, "neighbours": neighbours})


def laplace_curves(n: int = 1_000_000, seed: int = 2, eps: float = 1e-6, alpha: float = 0.0) -> Workload:
    """Laplace kernel, N points on 8 random star-shaped curves, delta_min from Theorem 1."""
    z = curve_points(n, seed)
    f = rhs(n, seed + 1000)
    dmax = enclosing_diameter(z)
    return Workload(f"laplace_curves_n{n}", z, f, "laplace", 0.0,
                    theorem1_delta_min(n, eps, dmax, alpha), eps,
                    {"seed": seed, "delta_max": dmax, "alpha": alpha})


def helmholtz_curves(n: int = 1_000_000, seed: int = 3, eps: float = 1e-6,
                     kappa_delta_max: float = 500.0, alpha: float = 0.0) -> Workload:
    """Helmholtz kernel, kappa * delta_max fixed, N points on the curve family, complex f."""
    z = curve_points(n, seed)
    f = rhs(n, seed + 1000, complex_valued=True)
    dmax = enclosing_diameter(z)
    return Workload(f"helmholtz_curves_n{n}", z, f, "helmholtz", kappa_delta_max / dmax,
                    theorem1_delta_min(n, eps, dmax, alpha), eps,
                    {"seed": seed, "delta_max": dmax, "kappa_delta_max": kappa_delta_max})


def laplace_square(n: int = 10_000_000, seed: int = 4, eps: float = 1e-6, nrhs: int = 16,
                   neighbours: float = 20.0) -> Workload:
    """Laplace kernel, N points uniform in [0,1]^2, nrhs right-hand sides."""
    z = square_points(n, seed)
    f = rhs(n, seed + 1000, nrhs=nrhs)
    delta_min = math.sqrt(neighbours / (math.pi * n))
    return Workload(f"laplace_square_n{n}", z, f, "laplace", 0.0, delta_min, eps,
                    {"seed": seed, "nrhs": nrhs})


def laplace_square_st(n: int = 1_000_000, seed: int = 6, eps: float = 1e-6, alpha: float = 0.0) -> Workload:
    """Laplace kernel with separate targets and sources (the Sec. 7.1 / Table 2 setting): targets
    z and sources y, each N points uniform in [0,1]^2 and drawn independently, f ~ N(0, 1) on the
    sources, delta_min by Theorem 1 with delta_max bounding the union of the two sets."""
    x = square_points(n, seed)
    y = square_points(n, seed + 500)
    f = rhs(n, seed + 1000)
    dmax = enclosing_diameter(np.concatenate([x, y]))
    return Workload(f"laplace_square_st_n{n}", x, f, "laplace", 0.0, theorem1_delta_min(n, eps, dmax, alpha), eps,
                    {"seed": seed, "delta_max": dmax, "alpha": alpha}, y=y)


def serve_requests(count: int = 256, seed: int = 5, n_lo: int = 1_000, n_hi: int = 1_000_000, eps: float = 1e-6,
                   kd_lo: float = 50.0, kd_hi: float = 500.0) -> list[dict]:
    """Solve requests for the server: each a random curve geometry (8 star-shaped curves in
    [0, 10]^2) with N log-uniform in [n_lo, n_hi], Laplace or Helmholtz with equal odds
    (kappa * delta_max uniform in [kd_lo, kd_hi]), delta_min from Theorem 1, and the
    second-kind-like system (I / 2 + (L / N) A) x = b, L the total arc length (the
    quadrature weight of a point), b ~ N(0, 1) (complex for Helmholtz)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        helm = bool(rng.random() < 0.5)
        kd = float(rng.uniform(kd_lo, kd_hi))
        gseed = 10_000 + seed * 1_000 + i
        z = curve_points(n, gseed)
        dmax = enclosing_diameter(z)
        out.append({"z": z, "b": rhs(n, gseed + 500_000, complex_valued=helm),
                    "kernel": "helmholtz" if helm else "laplace", "kappa": kd / dmax if helm else 0.0,
                    "delta_min": theorem1_delta_min(n, eps, dmax), "eps": eps, "shift": 0.5,
                    "scale": curve_length(gseed) / n})
    return out
