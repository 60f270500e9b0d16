"""Mesh quantities of a closed polygonal contour (oracle).

TEST INFRASTRUCTURE ONLY.

Sec. II: the curve gamma is cut into N segments; the current is expanded in piecewise
linear Lagrange hats phi_i (one per vertex). Segment e runs from vertex e to vertex e+1
(indices mod N); its unit tangent t_e follows the counter-clockwise orientation and its
outward normal is n_e = t_e x z = (t_y, -t_x).

On segment e (local coordinate sigma in [0,1]) two hats are nonzero:
    phi_e     = 1 - sigma   ("falling" piece, a = 0),  d/ds = -1/h_e
    phi_{e+1} = sigma       ("rising"  piece, a = 1),  d/ds = +1/h_e
so hat i consists of the pieces (segment i, a=0) and (segment i-1, a=1).

Pins: exact integrals of polynomials under the Gauss rules; Gram entries against closed form.
"""
from __future__ import annotations

import numpy as np

from . import special


def segments(nodes: np.ndarray):
    """Return d (N,2) segment vectors, h (N,) lengths, t (N,2) tangents, n (N,2) outward normals."""
    nodes = np.asarray(nodes, dtype=np.float64)
    d = np.roll(nodes, -1, axis=0) - nodes
    h = np.hypot(d[:, 0], d[:, 1])
    t = d / h[:, None]
    n = np.stack([t[:, 1], -t[:, 0]], axis=1)
    return d, h, t, n


def gauss_nodes(nodes: np.ndarray, p: int):
    """Quadrature nodes r_{e,u} = v_e + xi_u d_e and weights w_{e,u} = omega_u h_e (Eq. 7).

    Returns r (N,p,2), w (N,p), xi (p,).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    d, h, _, _ = segments(nodes)
    xi, om = special.gauss01(p)
    r = nodes[:, None, :] + xi[None, :, None] * d[:, None, :]
    w = om[None, :] * h[:, None]
    return r, w, xi


def midpoints(nodes: np.ndarray) -> np.ndarray:
    nodes = np.asarray(nodes, dtype=np.float64)
    return 0.5 * (nodes + np.roll(nodes, -1, axis=0))


def gram_dense(nodes: np.ndarray) -> np.ndarray:
    """[G]_ij = <phi_i, phi_j> (Eq. 3): cyclic tridiagonal, (h_{i-1}+h_i)/3 on the diagonal, h/6 beside."""
    _, h, _, _ = segments(nodes)
    n = len(h)
    g = np.zeros((n, n))
    for i in range(n):
        g[i, i] = (h[i - 1] + h[i]) / 3.0
        g[i, (i + 1) % n] += h[i] / 6.0
        g[(i + 1) % n, i] += h[i] / 6.0
    return g
