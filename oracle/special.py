"""Green's function, quadrature rules and closed-form circle results (oracle).

TEST INFRASTRUCTURE ONLY: used by tests, smoke() and the benchmark's CPU baseline.

* g(r) = -(j/4) H0^(2)(k r)                                  (Sec. II, below Eq. 2)
* Circle eigenvalues of S and N and of the analytically filtered S^alpha (Sec. II,
  Eqs. 4-6), derived with Graf's addition theorem; pinned in the tests against the
  dense operators on regular polygons and against each other (lambda_n mu_n -> 1/4).
* The analytically filtered kernel g^alpha of Eq. 6 at a distance (a principal-value integral).
* PEC circular-cylinder series currents (TM, TE) for the same time convention.

Pins: g against the small-argument expansion of H0^(2); Gauss rules against exact
polynomial moments and the log moment; closed forms against the dense oracle operators.
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate, special

EULER_GAMMA = 0.57721566490153286061


# --------------------------------------------------------------------------------------
# Green's function (Sec. II): g(r, r') = -(j/4) H0^(2)(k |r - r'|), H0^(2) = J0 - j Y0
# --------------------------------------------------------------------------------------
def green(k: float, r: np.ndarray) -> np.ndarray:
    """g at distance r > 0 (complex128)."""
    x = k * np.asarray(r, dtype=np.float64)
    return -0.25j * (special.j0(x) - 1j * special.y0(x))


# --------------------------------------------------------------------------------------
# Quadrature rules
# --------------------------------------------------------------------------------------
def gauss01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def graded01(levels: int = 30, n: int = 14, ratio: float = 0.3):
    """Composite Gauss-Legendre on [0, 1], geometrically graded toward 0.

    Sub-intervals [ratio^(l+1), ratio^l] for l = 0..levels-1 plus [0, ratio^levels],
    each with n Gauss points. Integrates x^b log(x) * smooth to ~1e-15 for b >= 0.
    """
    xs, ws = [], []
    g, gw = gauss01(n)
    edges = [ratio ** l for l in range(levels + 1)] + [0.0]
    for hi, lo in zip(edges[:-1], edges[1:]):
        xs.append(lo + (hi - lo) * g)
        ws.append((hi - lo) * gw)
    return np.concatenate(xs), np.concatenate(ws)


# --------------------------------------------------------------------------------------
# Closed forms on a circle of radius a (modes e^{j n phi})
# --------------------------------------------------------------------------------------
def _h2(n, x):
    return special.jv(n, x) - 1j * special.yv(n, x)


def _h2p(n, x):
    return special.jvp(n, x) - 1j * special.yvp(n, x)


def circle_lambda(n, ka: float, a: float) -> np.ndarray:
    """Eigenvalue of the single layer S (Eq. 4) for e^{j n phi}: -(j pi a/2) J_n(ka) H_n^(2)(ka)."""
    n = np.asarray(n)
    return -0.5j * math.pi * a * special.jv(n, ka) * _h2(n, ka)


def circle_mu(n, ka: float, a: float) -> np.ndarray:
    """Eigenvalue of the hypersingular N (Eq. 2): (j pi a k^2/2) J_n'(ka) H_n^(2)'(ka)."""
    n = np.asarray(n)
    k = ka / a
    return 0.5j * math.pi * a * k * k * special.jvp(n, ka) * _h2p(n, ka)


def circle_lambda_filtered(n: int, k: float, a: float, alpha: float) -> complex:
    """Eigenvalue of the analytically filtered S^alpha (Eqs. 5-6) for e^{j n phi}.

    Graf's theorem gives the eigenvalue of the subtracted tail of Eq. 6 as
    -a int_alpha^inf J_n(sa)^2 s/(s^2-k^2) ds; with PV int_0^inf J_n(sa)^2 s/(s^2-k^2) ds
    = -(pi/2) J_n(ka) Y_n(ka) this leaves
        a PV int_0^alpha J_n(sa)^2 s/(s^2-k^2) ds - j (pi a/2) J_n(ka)^2 .
    """
    f = lambda s: special.jv(n, s * a) ** 2 * s / (s + k)
    # PV int f(s)/(s-k) ds by QUADPACK's Cauchy weight; split the range for oscillations
    edges = np.linspace(0.0, alpha, 2 + int(alpha * a / 2.0))
    pv = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        if lo < k < hi:
            val, _ = integrate.quad(f, lo, hi, weight="cauchy", wvar=k, limit=400)
        else:
            val, _ = integrate.quad(lambda s: f(s) / (s - k), lo, hi, limit=400, epsabs=1e-14, epsrel=1e-13)
        pv += val
    return a * pv - 0.5j * math.pi * a * special.jv(n, k * a) ** 2


def filtered_green(k: float, alpha: float, r: float) -> complex:
    """The analytically filtered kernel g^alpha of Eq. 6 at distance r >= 0.

    Eq. 6 writes g^alpha = -(j/4) H0^(2)(kr) - (1/2 pi) int_alpha^inf J0(sr) s/(s^2-k^2) ds. With the
    integral representation PV int_0^inf J0(sr) s/(s^2-k^2) ds = -(pi/2) Y0(kr) (DLMF 10.9, the
    same identity behind circle_lambda_filtered) and H0^(2) = J0 - j Y0, the Y0 terms cancel:
        g^alpha(r) = -(j/4) J0(kr) + (1/2 pi) PV int_0^alpha J0(sr) s/(s^2-k^2) ds,
    a finite integral, regular at r = 0 (Sec. III-C: the filtered kernel has no singularity).
    The principal value is QUADPACK's Cauchy-weight rule on the panel that holds s = k; the range is
    cut into panels of about two oscillations of J0(sr).
    """
    r = float(r)
    f = lambda s: special.j0(s * r) * s / (s + k)
    edges = list(np.linspace(0.0, alpha, 2 + int(alpha * r / 4.0)))
    # keep s = k strictly inside a panel
    for i in range(1, len(edges) - 1):
        if abs(edges[i] - k) < 1e-6 * k:
            del edges[i]
            break
    pv = 0.0
    with np.errstate(all="ignore"), warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        for lo, hi in zip(edges[:-1], edges[1:]):
            if lo < k < hi:
                val, _ = integrate.quad(f, lo, hi, weight="cauchy", wvar=k, limit=400, epsabs=1e-15, epsrel=1e-13)
            else:
                val, _ = integrate.quad(lambda s: f(s) / (s - k), lo, hi, limit=400, epsabs=1e-15, epsrel=1e-13)
            pv += val
    return complex(pv / (2.0 * math.pi), -0.25 * special.j0(k * r))


def tm_cylinder_current(phi: np.ndarray, ka: float, a: float, theta: float = 0.0, eta: float = 1.0,
                        nmax: int | None = None) -> np.ndarray:
    """Surface current J_z on a PEC circle for E^i_z = exp(-j k khat.r), khat = (cos th, sin th).

    From j k eta lambda_n c_n = j^{-n} J_n(ka) e^{-j n theta}:  c_n = 2 j^{-n} e^{-j n th} / (pi k a eta H_n(ka)).
    """
    k = ka / a
    if nmax is None:
        nmax = int(ka + 10.0 * ka ** (1.0 / 3.0) + 20)
    n = np.arange(-nmax, nmax + 1)
    c = 2.0 * (1j ** (-n)) * np.exp(-1j * n * theta) / (math.pi * k * a * eta * _h2(n, ka))
    return (c[None, :] * np.exp(1j * np.outer(phi, n))).sum(axis=1)


def circle_mu_filtered(n: int, k: float, a: float, alpha: float) -> complex:
    """Eigenvalue of N (Maue form) built on the analytically filtered kernel g^alpha (Eqs. 5-6).

    On the circle the Maue form pairs the tangential derivatives, (n/a)^2 times the single-layer
    eigenvalue of the mode, with the term -k^2 (n.n') g, where n.n' = cos(phi - phi') couples
    modes n -+ 1: mu_n = (n/a)^2 lambda_n - k^2 (lambda_{n-1} + lambda_{n+1})/2. That identity
    holds for any radial kernel, so with lambda^alpha it gives the filtered eigenvalue.
    """
    lam = lambda m: circle_lambda_filtered(abs(m), k, a, alpha)
    return (n / a) ** 2 * lam(n) - k * k * (lam(n - 1) + lam(n + 1)) / 2.0


def te_cylinder_current(phi: np.ndarray, ka: float, a: float, theta: float = 0.0,
                        nmax: int | None = None) -> np.ndarray:
    """Tangential current j_t on a PEC circle solving (eta/(j k)) N j_t = E_t (Eq. 1), H^i_z = exp(-j k khat.r).

    With E^i = eta H^i_z (z x khat) the tangential field on the circle (t = (-sin, cos)) is
    E_t = eta e^{-j ka cos(phi-th)} cos(phi-th) = eta sum_n j^{1-n} J_n'(ka) e^{j n (phi-th)}, and
    N e^{j n phi} = mu_n e^{j n phi}, so c_n = j k j^{1-n} J_n'(ka) e^{-j n th} / mu_n.
    """
    k = ka / a
    if nmax is None:
        nmax = int(ka + 10.0 * ka ** (1.0 / 3.0) + 20)
    n = np.arange(-nmax, nmax + 1)
    c = 1j * k * (1j ** (1 - n)) * special.jvp(n, ka) * np.exp(-1j * n * theta) / circle_mu(n, ka, a)
    return (c[None, :] * np.exp(1j * np.outer(phi, n))).sum(axis=1)
