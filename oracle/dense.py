"""Exact dense operators on a flat-segment mesh (oracle tier O1).

TEST INFRASTRUCTURE ONLY.

TE, Galerkin with P1 hats (Sec. II):
    [S]_ij = <phi_i, S phi_j>           single layer, Eq. 4, with g of Sec. II
    [N]_ij = <phi_i, N phi_j>           hypersingular, Eq. 2, evaluated in the
             = int int g(r,r') [phi_i'(r) phi_j'(r') - k^2 (n.n') phi_i(r) phi_j(r')]
             (integration by parts along the closed curve; the circle test pins it)
    E_i    = <phi_i, (jk/eta) E_t>      excitation of Eq. 1 / Sec. II
TM, pulse basis and midpoint collocation (the small TM workload):
    Z_ij   = jk eta int_{seg j} g(r_i, r') dl'   ,  E_i = E^i_z(r_i)

All singular and nearly singular integrals are computed to ~1e-14 relative:
* self pairs reduce exactly to a 1-D integral in t = |sigma - tau| with a polynomial
  weight, integrated with geometrically graded Gauss toward t = 0;
* pairs sharing a vertex use the Duffy split at the shared vertex plus graded Gauss;
* other pairs use tensor Gauss-Legendre with an order chosen from their distance.

Pins: the circle eigenvalue tests (lambda_n, mu_n), quadrature-order convergence, and
the cylinder-series solutions.
"""
from __future__ import annotations

import numpy as np

from . import geometry, special


def _psi(a: int, s: np.ndarray) -> np.ndarray:
    return s if a == 1 else 1.0 - s


def _seg_seg_distance(p0, p1, q0, q1):
    """Minimum distance between segments [p0,p1] and [q0,q1] (vectorised, non-crossing)."""
    def pt_seg(x, a, b):
        ab = b - a
        tt = np.clip(np.einsum("ij,ij->i", x - a, ab) / np.einsum("ij,ij->i", ab, ab), 0.0, 1.0)
        c = a + tt[:, None] * ab
        return np.hypot(*(x - c).T)
    return np.minimum.reduce([pt_seg(p0, q0, q1), pt_seg(p1, q0, q1), pt_seg(q0, p0, p1), pt_seg(q1, p0, p1)])


def pair_integrals(nodes: np.ndarray, k: float, e: np.ndarray, f: np.ndarray,
                   n_close: int = 14, n_far: int = 8, close_factor: float = 3.0,
                   levels: int = 30, n_graded: int = 14, n_y: int = 16) -> np.ndarray:
    """I[q, a, b] = int_seg e int_seg f psi_a(sigma) g(|r - r'|) psi_b(tau) dl dl'  for pairs (e_q, f_q).

    psi_0 = 1 - sigma (falling hat piece), psi_1 = sigma (rising hat piece).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    d, h, _, _ = geometry.segments(nodes)
    e = np.asarray(e, dtype=np.int64)
    f = np.asarray(f, dtype=np.int64)
    out = np.zeros((len(e), 2, 2), dtype=np.complex128)

    is_self = e == f
    is_next = f == (e + 1) % nseg
    is_prev = e == (f + 1) % nseg
    rest = ~(is_self | is_next | is_prev)

    # --- self pairs: I_ab = h^2 int_0^1 g(h t) Q_ab(t) dt
    if is_self.any():
        q = np.nonzero(is_self)[0]
        tg, tw = special.graded01(levels, n_graded)
        g2, g2w = special.gauss01(2)
        # Q_ab(t) = int_t^1 [psi_a(s) psi_b(s-t) + psi_a(s-t) psi_b(s)] ds  (2-pt Gauss is exact)
        s = tg[:, None] + (1.0 - tg[:, None]) * g2[None, :]
        ws = (1.0 - tg[:, None]) * g2w[None, :]
        Q = np.zeros((2, 2, len(tg)))
        for a in range(2):
            for b in range(2):
                Q[a, b] = np.sum(ws * (_psi(a, s) * _psi(b, s - tg[:, None]) + _psi(a, s - tg[:, None]) * _psi(b, s)), axis=1)
        hq = h[e[q]]
        gv = special.green(k, hq[:, None] * tg[None, :])            # (nq, nt)
        out[q] = (hq ** 2)[:, None, None] * np.einsum("qt,abt->qab", gv * tw[None, :], Q)

    # --- vertex-sharing pairs: Duffy split at the shared vertex
    def adjacent(eq, fq):
        # f = e + 1, shared vertex V = v_{e+1} = v_f; x = distance fraction from V back along e
        X, Xw = special.graded01(levels, n_graded)
        Y, Yw = special.gauss01(n_y)
        de = d[eq]
        df = d[fq]
        res = np.zeros((len(eq), 2, 2), dtype=np.complex128)
        for tri in range(2):
            if tri == 0:    # tau <= x :  x = X, tau = X Y
                xe = X[:, None] * np.ones_like(Y)[None, :]
                tau = X[:, None] * Y[None, :]
            else:           # x <= tau :  tau = X, x = X Y
                tau = X[:, None] * np.ones_like(Y)[None, :]
                xe = X[:, None] * Y[None, :]
            jac = (X[:, None] * Xw[:, None] * Yw[None, :])
            vec = xe[None, :, :, None] * de[:, None, None, :] + tau[None, :, :, None] * df[:, None, None, :]
            r = np.sqrt(np.sum(vec * vec, axis=-1))
            gv = special.green(k, r) * jac[None]
            sig_e = 1.0 - xe
            for a in range(2):
                for b in range(2):
                    res[:, a, b] += np.sum(gv * (_psi(a, sig_e) * _psi(b, tau))[None], axis=(1, 2))
        return res * (h[eq] * h[fq])[:, None, None]

    if is_next.any():
        q = np.nonzero(is_next)[0]
        out[q] = adjacent(e[q], f[q])
    if is_prev.any():
        q = np.nonzero(is_prev)[0]
        out[q] = np.transpose(adjacent(f[q], e[q]), (0, 2, 1))

    # --- separated pairs: tensor Gauss, order by distance
    if rest.any():
        q = np.nonzero(rest)[0]
        dist = _seg_seg_distance(nodes[e[q]], nodes[(e[q] + 1) % nseg], nodes[f[q]], nodes[(f[q] + 1) % nseg])
        close = dist < close_factor * np.maximum(h[e[q]], h[f[q]])
        for sel, n in ((close, n_close), (~close, n_far)):
            qq = q[sel]
            if len(qq) == 0:
                continue
            sg, sw = special.gauss01(n)
            for c0 in range(0, len(qq), 4096):
                qc = qq[c0:c0 + 4096]
                re = nodes[e[qc]][:, None, :] + sg[None, :, None] * d[e[qc]][:, None, :]
                rf = nodes[f[qc]][:, None, :] + sg[None, :, None] * d[f[qc]][:, None, :]
                diff = re[:, :, None, :] - rf[:, None, :, :]
                r = np.sqrt(np.sum(diff * diff, axis=-1))
                gv = special.green(k, r) * (sw[:, None] * sw[None, :])[None]
                for a in range(2):
                    for b in range(2):
                        out[qc, a, b] = np.einsum("qst,s,t->q", gv, _psi(a, sg), _psi(b, sg))
                out[qc] *= (h[e[qc]] * h[f[qc]])[:, None, None]
    return out


def te_piece_terms(nodes: np.ndarray, k: float, e, f, I):
    """Per segment pair, the S and N (Maue form) contributions of the hat pieces (a on e, b on f)."""
    _, h, _, nrm = geometry.segments(nodes)
    e = np.asarray(e)
    f = np.asarray(f)
    J = I.sum(axis=(1, 2))
    sgn = np.array([-1.0, 1.0])
    nn = np.sum(nrm[e] * nrm[f], axis=1)
    dd = (sgn[None, :, None] / h[e][:, None, None]) * (sgn[None, None, :] / h[f][:, None, None])
    Nt = dd * J[:, None, None] - (k * k) * nn[:, None, None] * I
    return I, Nt


def _assemble_pieces(T: np.ndarray) -> np.ndarray:
    """Hat i = (segment i, a=0) + (segment i-1, a=1). T is (N, N, 2, 2) over segment pairs."""
    A = T[:, :, 0, 0].copy()
    A += np.roll(T[:, :, 0, 1], 1, axis=1)        # (e=i, f=j-1, b=1)
    A += np.roll(T[:, :, 1, 0], 1, axis=0)        # (e=i-1, f=j, a=1)
    A += np.roll(np.roll(T[:, :, 1, 1], 1, axis=0), 1, axis=1)
    return A


def te_dense(nodes: np.ndarray, k: float, **quad):
    """Exact dense Galerkin S and N (Eqs. 2, 4) for P1 hats; returns (S, N)."""
    nseg = np.asarray(nodes).shape[0]
    ee, ff = np.meshgrid(np.arange(nseg), np.arange(nseg), indexing="ij")
    I = pair_integrals(nodes, k, ee.ravel(), ff.ravel(), **quad)
    Is, Nt = te_piece_terms(nodes, k, ee.ravel(), ff.ravel(), I)
    S = _assemble_pieces(Is.reshape(nseg, nseg, 2, 2))
    N = _assemble_pieces(Nt.reshape(nseg, nseg, 2, 2))
    return S, N


def te_entries(nodes: np.ndarray, k: float, rows: np.ndarray, cols: np.ndarray, **quad):
    """Exact [S]_ij and [N]_ij for listed hat pairs (i, j)."""
    nseg = np.asarray(nodes).shape[0]
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    S = np.zeros(len(rows), dtype=np.complex128)
    N = np.zeros(len(rows), dtype=np.complex128)
    for (de, a) in ((0, 0), (-1, 1)):
        for (df, b) in ((0, 0), (-1, 1)):
            e = (rows + de) % nseg
            f = (cols + df) % nseg
            I = pair_integrals(nodes, k, e, f, **quad)
            Is, Nt = te_piece_terms(nodes, k, e, f, I)
            S += Is[:, a, b]
            N += Nt[:, a, b]
    return S, N


def tm_point_segment(nodes: np.ndarray, k: float, i: np.ndarray, j: np.ndarray,
                     n_close: int = 16, n_far: int = 8, close_factor: float = 3.0,
                     levels: int = 30, n_graded: int = 14) -> np.ndarray:
    """int_{seg j} g(|r_i - r'|) dl' with r_i the midpoint of segment i."""
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    d, h, _, _ = geometry.segments(nodes)
    mid = geometry.midpoints(nodes)
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    out = np.zeros(len(i), dtype=np.complex128)
    is_self = i == j
    if is_self.any():
        q = np.nonzero(is_self)[0]
        tg, tw = special.graded01(levels, n_graded)
        half = 0.5 * h[j[q]]
        out[q] = 2.0 * half * np.sum(special.green(k, half[:, None] * tg[None, :]) * tw[None, :], axis=1)
    rest = ~is_self
    if rest.any():
        q = np.nonzero(rest)[0]
        p0 = nodes[j[q]]
        ab = d[j[q]]
        x = mid[i[q]]
        tt = np.clip(np.einsum("ij,ij->i", x - p0, ab) / np.einsum("ij,ij->i", ab, ab), 0.0, 1.0)
        dist = np.hypot(*(x - (p0 + tt[:, None] * ab)).T)
        close = dist < close_factor * h[j[q]]
        for sel, n in ((close, n_close), (~close, n_far)):
            qq = q[sel]
            if len(qq) == 0:
                continue
            sg, sw = special.gauss01(n)
            rr = nodes[j[qq]][:, None, :] + sg[None, :, None] * d[j[qq]][:, None, :]
            diff = mid[i[qq]][:, None, :] - rr
            r = np.hypot(diff[..., 0], diff[..., 1])
            out[qq] = h[j[qq]] * np.sum(special.green(k, r) * sw[None, :], axis=1)
    return out


def tm_dense(nodes: np.ndarray, k: float, eta: float = 1.0, **quad) -> np.ndarray:
    """Z_ij = j k eta int_{seg j} g(r_i, r') dl' (pulse basis, midpoint collocation)."""
    nseg = np.asarray(nodes).shape[0]
    ii, jj = np.meshgrid(np.arange(nseg), np.arange(nseg), indexing="ij")
    return 1j * k * eta * tm_point_segment(nodes, k, ii.ravel(), jj.ravel(), **quad).reshape(nseg, nseg)


# --------------------------------------------------------------------------------------
# Excitations
# --------------------------------------------------------------------------------------
def te_rhs(nodes: np.ndarray, k: float, theta: float, n_quad: int = 10) -> np.ndarray:
    """E_i = <phi_i, (jk/eta) E_t> with H^i_z = exp(-jk khat.r), E^i = eta H^i_z (z x khat) (Sec. II)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    d, h, t, _ = geometry.segments(nodes)
    kh = np.array([np.cos(theta), np.sin(theta)])
    xi, om = special.gauss01(n_quad)
    r = nodes[:, None, :] + xi[None, :, None] * d[:, None, :]
    hz = np.exp(-1j * k * (r @ kh))
    et = hz * (kh[0] * t[:, 1] - kh[1] * t[:, 0])[:, None]           # E_t / eta
    piece0 = 1j * k * h * np.sum(om[None, :] * (1.0 - xi)[None, :] * et, axis=1)
    piece1 = 1j * k * h * np.sum(om[None, :] * xi[None, :] * et, axis=1)
    return piece0 + np.roll(piece1, 1)


def tm_rhs(nodes: np.ndarray, k: float, theta: float) -> np.ndarray:
    """E_i = E^i_z(r_i) = exp(-jk khat.r_i) at segment midpoints."""
    mid = geometry.midpoints(nodes)
    kh = np.array([np.cos(theta), np.sin(theta)])
    return np.exp(-1j * k * (mid @ kh))
