"""Seeded synthetic inputs for the filtered-AIM EFIE workloads.

This module is shared by the CPU oracle tests, the GPU parity tests and the benchmark.
It holds none of the method's arithmetic: it only produces scatterer outlines (closed
polygons given by their vertices), incidence angles, random coefficient vectors, and the
table of workload sizes. Everything the method computes from these (quadrature, grid,
interpolation, kernel, spectrum, operators) is done separately by each side.

Units: lengths in wavelengths, so the free-space wavenumber is k = 2*pi.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------------------
# Contours
# --------------------------------------------------------------------------------------
def circle_polygon(radius: float, n_seg: int) -> np.ndarray:
    """Vertices of the regular n_seg-gon inscribed in a circle, counter-clockwise.

    Returns an (n_seg, 2) float64 array; vertex i sits at angle 2*pi*i/n_seg.
    """
    phi = TWO_PI * np.arange(n_seg) / n_seg
    return np.stack([radius * np.cos(phi), radius * np.sin(phi)], axis=1)


@dataclasses.dataclass(frozen=True)
class StarContour:
    """r(phi) = a * (1 + sum_{m=1..M} eps_m cos(m phi + theta_m)) drawn from a seed.

    eps_m ~ U[0, eps_max), theta_m ~ U[0, 2pi) from numpy default_rng(seed), in that order.
    """

    eps: np.ndarray
    theta: np.ndarray

    @staticmethod
    def from_seed(seed: int, n_modes: int = 8, eps_max: float = 0.08) -> "StarContour":
        rng = np.random.default_rng(seed)
        eps = rng.uniform(0.0, eps_max, n_modes)
        theta = rng.uniform(0.0, TWO_PI, n_modes)
        return StarContour(eps=eps, theta=theta)

    def radius(self, phi: np.ndarray, a: float = 1.0) -> np.ndarray:
        mm = np.arange(1, len(self.eps) + 1)[:, None]
        return a * (1.0 + np.sum(self.eps[:, None] * np.cos(mm * phi[None, :] + self.theta[:, None]), axis=0))

    def _fine(self, n_fine: int):
        phi = TWO_PI * np.arange(n_fine) / n_fine
        r = self.radius(phi)
        xy = np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)
        d = np.roll(xy, -1, axis=0) - xy
        ds = np.hypot(d[:, 0], d[:, 1])
        return phi, xy, ds

    def polygon(self, perimeter: float, n_seg: int, oversample: int = 64) -> np.ndarray:
        """Vertices (n_seg, 2), counter-clockwise, at (nearly) equal arc length.

        The unit-a curve is sampled finely, its length measured, the curve scaled so its
        perimeter is `perimeter`, and vertices placed at equal fractions of arc length by
        linear interpolation along the fine polyline.
        """
        n_fine = max(4096, oversample * n_seg)
        phi, xy, ds = self._fine(n_fine)
        total = ds.sum()
        scale = perimeter / total
        s = np.concatenate([[0.0], np.cumsum(ds)])
        target = total * np.arange(n_seg) / n_seg
        idx = np.searchsorted(s, target, side="right") - 1
        idx = np.clip(idx, 0, n_fine - 1)
        frac = (target - s[idx]) / ds[idx]
        nxt = (idx + 1) % n_fine
        pts = xy[idx] + frac[:, None] * (xy[nxt] - xy[idx])
        return scale * pts


# --------------------------------------------------------------------------------------
# Right-hand sides and probe vectors
# --------------------------------------------------------------------------------------
def equispaced_angles(n: int) -> np.ndarray:
    """Incidence angles 2*pi*r/n, r = 0..n-1."""
    return TWO_PI * np.arange(n) / n


def random_angles(n: int, seed: int = 7) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, TWO_PI, n)


def random_coeffs(n: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """Complex standard-normal coefficient vectors, shape (nrhs, n), complex128."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))) / math.sqrt(2.0)


def random_grid(m: int, nrhs: int = 1, seed: int = 0, density: float = 1.0) -> np.ndarray:
    """Complex grid samples of shape (nrhs, m, m); a fraction `density` of points nonzero."""
    rng = np.random.default_rng(seed)
    u = (rng.standard_normal((nrhs, m, m)) + 1j * rng.standard_normal((nrhs, m, m))) / math.sqrt(2.0)
    if density < 1.0:
        u *= rng.uniform(size=(nrhs, m, m)) < density
    return u


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    form: str            # "tm" (pulse basis, point collocation) or "te" (P1 hats, Galerkin)
    nodes: np.ndarray    # (N, 2) polygon vertices, counter-clockwise
    k: float             # wavenumber (rad / wavelength)
    m: int               # grid points per side
    fft_P: int           # circulant embedding size per side
    s: int               # interpolation points per axis
    p: int               # Gauss-Legendre nodes per segment
    alpha: float         # filter radius (rad / wavelength)
    angles: np.ndarray   # plane-wave incidence angles

    @property
    def n(self) -> int:
        return self.nodes.shape[0]


def _pow2_at_least(x: int) -> int:
    p = 1
    while p < x:
        p *= 2
    return p


def tm_circle(n_seg: int = 256, m: int = 64, radius: float = 1.0, alpha_over_k: float = 8.0) -> Workload:
    """TM, pulse/collocation, PEC circle of radius 1 wavelength, N=256, 64x64 grid."""
    k = TWO_PI
    return Workload("tm_circle_n%d_m%d" % (n_seg, m), "tm", circle_polygon(radius, n_seg), k, m,
                    _pow2_at_least(2 * m), 4, 4, alpha_over_k * k, equispaced_angles(1))


def te_circle(n_seg: int, m: int, radius: float = 1.0, alpha_over_k: float = 8.0, s: int = 4, p: int = 4) -> Workload:
    k = TWO_PI
    return Workload("te_circle_n%d_m%d" % (n_seg, m), "te", circle_polygon(radius, n_seg), k, m,
                    _pow2_at_least(2 * m), s, p, alpha_over_k * k, equispaced_angles(1))


def te_star(perimeter: float, n_seg: int, m: int, seed: int = 0, alpha_over_k: float = 2.0,
            nrhs: int = 1, s: int = 4, p: int = 4) -> Workload:
    """TE Calderon workload on the seeded star-contour family at the given perimeter."""
    k = TWO_PI
    nodes = StarContour.from_seed(seed).polygon(perimeter, n_seg)
    return Workload("te_star_p%g_n%d_m%d_s%d" % (perimeter, n_seg, m, seed), "te", nodes, k, m,
                    _pow2_at_least(2 * m), s, p, alpha_over_k * k, equispaced_angles(nrhs))


def single_solve_scale(seed: int = 0) -> Workload:
    """Perimeter 1000 wavelengths, 10 segments per wavelength (N=10000), 2048^2 grid, alpha=2k."""
    return te_star(1000.0, 10000, 2048, seed=seed, alpha_over_k=2.0, nrhs=1)


def batching_scale(seed: int = 0, nrhs: int = 64) -> Workload:
    """Perimeter 400 wavelengths (N=4000), 1024^2 grid, 64 equispaced incidence angles."""
    return te_star(400.0, 4000, 1024, seed=seed, alpha_over_k=2.0, nrhs=nrhs)


@dataclasses.dataclass(frozen=True)
class ServingRequest:
    t_arrival: float
    perimeter: float
    seed: int
    k: float
    n_seg: int
    m: int
    nrhs: int
    alpha: float


def serving_stream(n_requests: int, rate: float = 200.0, seed: int = 11) -> list:
    """Poisson arrivals; perimeter log-uniform in [5, 500] wavelengths-at-k, N = 10 per wavelength,
    k ~ U[pi, 4pi], grid m = smallest power of two in [32, 1024] with spacing <= 0.16 wavelength,
    1..16 right-hand sides, alpha = min(8k, (2/3) pi / spacing)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        per_wl = math.exp(rng.uniform(math.log(5.0), math.log(500.0)))
        k = rng.uniform(math.pi, 4.0 * math.pi)
        nrhs = int(rng.integers(1, 17))
        geo_seed = int(rng.integers(0, 2**31 - 1))
        wl = TWO_PI / k
        n_seg = max(50, int(round(10.0 * per_wl)))
        # grid: the contour's diameter is about perimeter/pi; pick m so the spacing is <= 0.16 wl
        diam = 1.25 * per_wl * wl / math.pi
        m = 32
        while m < 1024 and diam / (m - 8) > 0.16 * wl:
            m *= 2
        eps = diam / (m - 8)
        alpha = min(8.0 * k, (2.0 / 3.0) * math.pi / eps)
        alpha = max(alpha, 1.05 * k)
        out.append(ServingRequest(t, per_wl * wl, geo_seed, k, n_seg, m, nrhs, alpha))
    return out
