"""The AIM-defined operators, unfiltered and numerically filtered (oracle tier O2).

TEST INFRASTRUCTURE ONLY.

Steps, in the paper's order (Sec. III):
1. Eq. 7: [S]_ij = sum_u sum_v w_u phi_i(r_u) g(r_u, r_v) w_v phi_j(r_v) over Gauss nodes.
2. Sec. III-A: a 2L x 2L grid centred at the origin, m points per side, spacing
   eps = 2L/(m-1); G_nodes ~ Lambda^T G_grid Lambda with Lambda the sparse interpolation
   from nodes to grid points (tensor-product Lagrange, s points per axis) and G_grid the
   Toeplitz matrix of grid-point interactions. The composed projection is P = Lambda W Phi.
3. Sec. III-A / Eq. 8: G_grid u is computed by embedding the kernel in a circulant:
   c_grid is the grid kernel mirrored about its last row and column, u is zero-padded, and
   v = [F^-1(F(c_grid) .* F(b))]_restr.
4. Sec. III-B: the filter is a circular truncation of F(c_grid) at radius alpha,
   giving F(c_grid^alpha); Eq. 10 then uses it in place of F(c_grid). For comparison
   (Fig. 1a) the analytically filtered kernel g^alpha of Eq. 6 can instead be sampled on
   the grid and transformed (filter_kind="analytic").
5. Sec. III-C: the self interaction of G_grid is set to zero (before the FFT and mask).

Readings taken where the paper leaves a choice (all listed in the design notes):
* embedding side P (power of two, P >= 2m-1); c[i,j] = g(eps*sqrt(i~^2+j~^2)) with
  i~ = i for i <= P/2 and i - P otherwise (so every mirrored sample is the kernel at
  that distance); the filtered result depends on P, the unfiltered one does not;
* DFT bin (p,q) has wavenumber kappa = 2 pi sqrt(p~^2+q~^2)/(P eps); bins with
  kappa <= alpha are kept, all others zeroed; only F(c) is masked;
* Lagrange stencil: for even s the indices floor(xi)-s/2+1 .. floor(xi)+s/2, for odd s
  round(xi)-(s-1)/2 .. round(xi)+(s-1)/2, with xi = (x+L)/eps;
* L = R/(1 - (s+2)/(m-1)) with R = max |coordinate| of the contour vertices, so every
  stencil lies inside the grid with one spare point;
* near-field correction (not in the paper): for the unfiltered operators only, the
  entries of hat pairs whose supports lie within `near_radius` (default s*eps) are
  replaced by the exact dense entries. The filtered S^alpha is exactly Eq. 10.

Two independent evaluations of the grid product are provided: by FFT (Eq. 8, a
library FFT as one step) and by a direct Toeplitz sum over grid-point pairs, with the
filtered kernel obtained by an explicit DFT matrix. Tests check one against the other.

Pins: Lagrange exactness on polynomials; direct sum == FFT product; filter idempotence
and identity for alpha above the grid Nyquist radius; unfiltered AIM -> dense exact
operator as m and s grow, for TE (S, N) and TM (Z, on a circle and a star); the TM AIM
solution against the cylinder series; filtered spectrum on a circle against the closed form.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft
import scipy.sparse as sp

from . import dense, geometry, special


# --------------------------------------------------------------------------------------
# Grid and interpolation (Sec. III-A)
# --------------------------------------------------------------------------------------
def grid_half_side(nodes: np.ndarray, m: int, s: int) -> float:
    R = float(np.max(np.abs(np.asarray(nodes, dtype=np.float64))))
    return R / (1.0 - (s + 2.0) / (m - 1.0))


def grid_spacing(L: float, m: int) -> float:
    return 2.0 * L / (m - 1)


def lagrange_1d(xi: np.ndarray, s: int):
    """Stencil start index and the s Lagrange weights at fractional grid coordinate xi."""
    xi = np.asarray(xi, dtype=np.float64)
    if s % 2 == 0:
        base = np.floor(xi).astype(np.int64) - s // 2 + 1
    else:
        base = np.floor(xi + 0.5).astype(np.int64) - (s - 1) // 2
    loc = xi - base                                   # position within the stencil, in [.., ..]
    w = np.ones(xi.shape + (s,))
    for a in range(s):
        for b in range(s):
            if b != a:
                w[..., a] *= (loc - b) / (a - b)
    return base, w


def stencils(points: np.ndarray, L: float, eps: float, s: int):
    """2D stencils: (ix0, iy0, W) with W[..., b, a] the weight of grid point (ix0+a, iy0+b)."""
    pts = np.asarray(points, dtype=np.float64)
    bx, wx = lagrange_1d((pts[..., 0] + L) / eps, s)
    by, wy = lagrange_1d((pts[..., 1] + L) / eps, s)
    W = wy[..., :, None] * wx[..., None, :]
    return bx, by, W


def _coo_from_stencils(ix0, iy0, W, col, val, m, s):
    """Rows: linear grid index iy*m + ix. One column index and one scalar per stencil."""
    a = np.arange(s)
    ix = ix0[..., None, None] + a[None, :]
    iy = iy0[..., None, None] + a[:, None]
    rows = (iy * m + ix).ravel()
    cols = np.broadcast_to(np.asarray(col)[..., None, None], W.shape).ravel()
    data = (W * np.asarray(val)[..., None, None]).ravel()
    return rows, cols, data


def te_projections(nodes: np.ndarray, p: int, L: float, eps: float, m: int, s: int):
    """P = Lambda W Phi for the four hat projections used by S and by N (Maue form).

    Returns csr matrices (m*m, N) with identical sparsity: 'S' (phi), 'd' (phi'),
    'nx' (n_x phi), 'ny' (n_y phi).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    _, h, _, nrm = geometry.segments(nodes)
    r, w, xi = geometry.gauss_nodes(nodes, p)
    ix0, iy0, W = stencils(r, L, eps, s)                           # (N, p), (N, p, s, s)
    seg = np.arange(nseg)[:, None] * np.ones((1, p), dtype=np.int64)
    out = {}
    for name in ("S", "d", "nx", "ny"):
        rows_all, cols_all, data_all = [], [], []
        for piece in (0, 1):                                       # 0: hat e (falling), 1: hat e+1 (rising)
            hat = (seg + piece) % nseg
            phi = (1.0 - xi)[None, :] if piece == 0 else xi[None, :]
            dphi = (-1.0 if piece == 0 else 1.0) / h[:, None]
            if name == "S":
                val = w * phi
            elif name == "d":
                val = w * dphi * np.ones_like(phi)
            elif name == "nx":
                val = w * phi * nrm[:, 0:1]
            else:
                val = w * phi * nrm[:, 1:2]
            rr, cc, dd = _coo_from_stencils(ix0, iy0, W, hat, val, m, s)
            rows_all.append(rr); cols_all.append(cc); data_all.append(dd)
        out[name] = sp.csr_matrix((np.concatenate(data_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                                  shape=(m * m, nseg))
    return out


def tm_projections(nodes: np.ndarray, p: int, L: float, eps: float, m: int, s: int):
    """Pulse sources (Gauss nodes of each segment) and midpoint collocation tests."""
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    r, w, _ = geometry.gauss_nodes(nodes, p)
    ix0, iy0, W = stencils(r, L, eps, s)
    seg = np.arange(nseg)[:, None] * np.ones((1, p), dtype=np.int64)
    rr, cc, dd = _coo_from_stencils(ix0, iy0, W, seg, w, m, s)
    src = sp.csr_matrix((dd, (rr, cc)), shape=(m * m, nseg))
    mid = geometry.midpoints(nodes)
    jx0, jy0, V = stencils(mid, L, eps, s)
    rr, cc, dd = _coo_from_stencils(jx0, jy0, V, np.arange(nseg), np.ones(nseg), m, s)
    tst = sp.csr_matrix((dd, (rr, cc)), shape=(m * m, nseg))
    return {"src": src, "tst": tst}


# --------------------------------------------------------------------------------------
# Grid kernel, circulant embedding, filter (Sec. III-A, III-B, III-C)
# --------------------------------------------------------------------------------------
def signed_index(P: int) -> np.ndarray:
    i = np.arange(P)
    return np.where(i <= P // 2, i, i - P)


def grid_kernel(k: float, eps: float, P: int) -> np.ndarray:
    """c_grid on the P x P periodic cell: c[i,j] = g(eps*sqrt(i~^2 + j~^2)), c[0,0] = 0 (Sec. III-C)."""
    t = signed_index(P).astype(np.float64)
    r = eps * np.sqrt(t[:, None] ** 2 + t[None, :] ** 2)
    r[0, 0] = 1.0
    c = special.green(k, r)
    c[0, 0] = 0.0
    return c


def analytic_grid_kernel(k: float, eps: float, P: int, alpha: float) -> np.ndarray:
    """The analytically filtered kernel of Eq. 6 sampled on the P x P periodic cell:
    c^alpha_an[i,j] = g^alpha(eps*sqrt(i~^2 + j~^2)). g^alpha is regular at the origin, so the
    self term keeps its value g^alpha(0) (nothing to zero, Sec. III-C). Each distinct distance is
    evaluated once (the cell is even in both indices and symmetric under i <-> j)."""
    t = np.abs(signed_index(P))
    H = P // 2
    quarter = np.zeros((H + 1, H + 1), dtype=np.complex128)
    for i in range(H + 1):
        for j in range(i, H + 1):
            quarter[i, j] = quarter[j, i] = special.filtered_green(k, alpha, eps * math.hypot(i, j))
    return quarter[t[:, None], t[None, :]]


def dft_matrix(P: int) -> np.ndarray:
    j = np.arange(P)
    return np.exp(-2j * math.pi * np.outer(j, j) / P)


def dft2(x: np.ndarray, direct: bool) -> np.ndarray:
    """2-D DFT F(x)[p,q] = sum_ij x[i,j] e^{-2 pi j (p i + q j)/P}."""
    if direct:
        F = dft_matrix(x.shape[0])
        return F @ x @ F
    return scipy.fft.fft2(x, workers=-1)


def idft2(X: np.ndarray, direct: bool) -> np.ndarray:
    if direct:
        F = dft_matrix(X.shape[0]).conj()
        return (F @ X @ F) / (X.shape[0] * X.shape[1])
    return scipy.fft.ifft2(X, workers=-1)


def filter_mask(P: int, eps: float, alpha: float) -> np.ndarray:
    """Circular truncation of Sec. III-B: keep bins with kappa <= alpha."""
    t = signed_index(P).astype(np.float64)
    kappa = (2.0 * math.pi / (P * eps)) * np.sqrt(t[:, None] ** 2 + t[None, :] ** 2)
    return kappa <= alpha


# --------------------------------------------------------------------------------------
# Grid products
# --------------------------------------------------------------------------------------
def conv_fft(u: np.ndarray, Chat: np.ndarray) -> np.ndarray:
    """Eq. 8 bracket: [F^-1(Chat .* F(b))]_restr with b = u zero-padded to P x P. u: (..., m, m)."""
    m = u.shape[-1]
    P = Chat.shape[0]
    b = np.zeros(u.shape[:-2] + (P, P), dtype=np.complex128)
    b[..., :m, :m] = u
    v = scipy.fft.ifft2(Chat * scipy.fft.fft2(b, workers=-1), workers=-1)
    return v[..., :m, :m]


def conv_direct(u: np.ndarray, t: np.ndarray, out_idx: np.ndarray | None = None, chunk: int = 2048) -> np.ndarray:
    """v[a] = sum_b t[(a - b) mod P] u[b] by a direct sum over grid-point pairs.

    u: (m, m) grid; t: (P, P) periodic kernel. Returns v at the linear grid indices
    `out_idx` (all m*m points if None). Only nonzero u[b] are visited.
    """
    m = u.shape[-1]
    P = t.shape[0]
    uf = u.reshape(-1)
    nz = np.nonzero(uf)[0]
    by, bx = np.divmod(nz, m)
    if out_idx is None:
        out_idx = np.arange(m * m)
    ay, ax = np.divmod(np.asarray(out_idx), m)
    v = np.zeros(len(out_idx), dtype=np.complex128)
    for c0 in range(0, len(out_idx), chunk):
        sl = slice(c0, c0 + chunk)
        T = t[(ay[sl, None] - by[None, :]) % P, (ax[sl, None] - bx[None, :]) % P]
        v[sl] = T @ uf[nz]
    return v


# --------------------------------------------------------------------------------------
# Near field (not in the paper; replaces AIM entries of close pairs by exact ones)
# --------------------------------------------------------------------------------------
def near_pairs_te(nodes: np.ndarray, radius: float):
    """Hat pairs (i, j) whose supports (segments i-1, i and j-1, j) come within `radius`."""
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    a0 = nodes
    a1 = np.roll(nodes, -1, axis=0)
    ee, ff = [], []
    mid = 0.5 * (a0 + a1)
    _, h, _, _ = geometry.segments(nodes)
    reach = radius + h.max() * 1.01
    for e in range(nseg):
        cand = np.nonzero(np.hypot(*(mid - mid[e]).T) <= reach)[0]
        dist = dense._seg_seg_distance(np.repeat(a0[e:e + 1], len(cand), 0), np.repeat(a1[e:e + 1], len(cand), 0),
                                       a0[cand], a1[cand])
        sel = cand[dist <= radius]
        ee.append(np.full(len(sel), e)); ff.append(sel)
    ee = np.concatenate(ee); ff = np.concatenate(ff)
    # segment pair (e, f) touches hats {e, e+1} x {f, f+1}
    hi = np.concatenate([ee, ee, (ee + 1) % nseg, (ee + 1) % nseg])
    hj = np.concatenate([ff, (ff + 1) % nseg, ff, (ff + 1) % nseg])
    key = np.unique(hi * nseg + hj)
    return key // nseg, key % nseg


def near_pairs_tm(nodes: np.ndarray, radius: float):
    """(test i, source segment j) pairs with dist(midpoint_i, segment j) <= radius."""
    nodes = np.asarray(nodes, dtype=np.float64)
    nseg = nodes.shape[0]
    mid = geometry.midpoints(nodes)
    a0 = nodes
    d = np.roll(nodes, -1, axis=0) - nodes
    ii, jj = [], []
    _, h, _, _ = geometry.segments(nodes)
    for i in range(nseg):
        cand = np.nonzero(np.hypot(*(mid - mid[i]).T) <= radius + h.max())[0]
        x = mid[i]
        tt = np.clip(np.einsum("ij,ij->i", x - a0[cand], d[cand]) / np.einsum("ij,ij->i", d[cand], d[cand]), 0.0, 1.0)
        dist = np.hypot(*(x - (a0[cand] + tt[:, None] * d[cand])).T)
        sel = cand[dist <= radius]
        ii.append(np.full(len(sel), i)); jj.append(sel)
    return np.concatenate(ii), np.concatenate(jj)


def aim_entries(Pt: sp.csr_matrix, Ps: sp.csr_matrix, t: np.ndarray, m: int, rows: np.ndarray, cols: np.ndarray):
    """[Pt^T T Ps]_ij for listed pairs, with T the Toeplitz operator of the periodic kernel t."""
    P = t.shape[0]
    Ptc = Pt.tocsc()
    Psc = Ps.tocsc()
    out = np.zeros(len(rows), dtype=np.complex128)
    order = np.argsort(cols, kind="stable")
    rows_s = np.asarray(rows)[order]
    cols_s = np.asarray(cols)[order]
    bounds = np.flatnonzero(np.diff(np.concatenate([[-1], cols_s, [-1]])))
    for s0, s1 in zip(bounds[:-1], bounds[1:]):
        j = cols_s[s0]
        bj = Psc.indices[Psc.indptr[j]:Psc.indptr[j + 1]]
        vj = Psc.data[Psc.indptr[j]:Psc.indptr[j + 1]]
        by, bx = np.divmod(bj, m)
        for q in range(s0, s1):
            i = rows_s[q]
            ai = Ptc.indices[Ptc.indptr[i]:Ptc.indptr[i + 1]]
            vi = Ptc.data[Ptc.indptr[i]:Ptc.indptr[i + 1]]
            ay, ax = np.divmod(ai, m)
            T = t[(ay[:, None] - by[None, :]) % P, (ax[:, None] - bx[None, :]) % P]
            out[order[q]] = vi @ (T @ vj)
    return out


# --------------------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------------------
class _AimBase:
    def _grid_setup(self, nodes, k, m, P, s, p, alpha, L, near_radius, direct_dft, filter_kind="numerical"):
        self.nodes = np.asarray(nodes, dtype=np.float64)
        self.n = self.nodes.shape[0]
        self.k, self.m, self.P, self.s, self.p, self.alpha = float(k), int(m), int(P), int(s), int(p), float(alpha)
        if P < 2 * m - 1:
            raise ValueError("embedding side P must be >= 2m-1")
        self.L = grid_half_side(self.nodes, m, s) if L is None else float(L)
        self.eps = grid_spacing(self.L, m)
        self.near_radius = s * self.eps if near_radius is None else float(near_radius)
        self.direct = (P <= 256) if direct_dft is None else bool(direct_dft)
        self.c = grid_kernel(self.k, self.eps, self.P)
        self.Chat = dft2(self.c, self.direct)
        self.filter_kind = filter_kind
        self.mask = filter_mask(self.P, self.eps, self.alpha)
        if filter_kind == "numerical":          # Sec. III-B: circular truncation of F(c_grid) (Eq. 10)
            self.Chat_alpha = self.Chat * self.mask
        elif filter_kind == "analytic":         # Eq. 6 sampled on the grid, then transformed
            self.c_an = analytic_grid_kernel(self.k, self.eps, self.P, self.alpha)
            self.Chat_alpha = dft2(self.c_an, self.direct)
        else:
            raise ValueError("filter_kind must be 'numerical' or 'analytic'")
        self._c_alpha = None

    @property
    def c_alpha(self) -> np.ndarray:
        """Spatial filtered kernel c^alpha = F^-1(mask .* F(c)) (explicit DFT when P is small)."""
        if self._c_alpha is None:
            self._c_alpha = idft2(self.Chat_alpha, self.direct)
        return self._c_alpha

    def grid_product(self, u: np.ndarray, filtered: bool, method: str = "fft", out_idx=None) -> np.ndarray:
        """G_grid u (Eq. 8) or its filtered version (Eq. 10) on an (..., m, m) grid."""
        if method == "fft":
            v = conv_fft(u, self.Chat_alpha if filtered else self.Chat)
            return v if out_idx is None else v.reshape(v.shape[:-2] + (-1,))[..., out_idx]
        t = self.c_alpha if filtered else self.c
        if u.ndim == 2:
            v = conv_direct(u, t, out_idx)
            return v.reshape(self.m, self.m) if out_idx is None else v
        return np.stack([self.grid_product(x, filtered, method, out_idx) for x in u])

    def _apply(self, Pt, Ps, x, filtered, method):
        x = np.asarray(x, dtype=np.complex128)
        single = x.ndim == 1
        X = x[None] if single else x
        out = []
        for xv in X:
            u = (Ps @ xv).reshape(self.m, self.m)
            if method == "fft":
                v = self.grid_product(u, filtered, "fft").reshape(-1)
                out.append(Pt.T @ v)
            else:
                act = np.flatnonzero(np.diff(Pt.indptr))      # grid points the test side reads
                v = np.zeros(self.m * self.m, dtype=np.complex128)
                v[act] = self.grid_product(u, filtered, "direct", out_idx=act)
                out.append(Pt.T @ v)
        out = np.stack(out)
        return out[0] if single else out


class TEOperators(_AimBase):
    """TE, P1 hats, Galerkin: S, S^alpha (Eq. 10), N (Maue form), G, and the Calderon products (Eq. 3)."""

    def __init__(self, nodes, k, m, P, s=4, p=4, alpha=None, L=None, near_radius=None, direct_dft=None,
                 near=True, filter_kind="numerical"):
        self._grid_setup(nodes, k, m, P, s, p, alpha if alpha is not None else 8.0 * k, L, near_radius, direct_dft,
                         filter_kind)
        self.proj = te_projections(self.nodes, self.p, self.L, self.eps, self.m, self.s)
        self.G = sp.csc_matrix(geometry.gram_dense(self.nodes)) if self.n <= 2048 else self._gram_sparse()
        self.near_rows = self.near_cols = None
        self.CS = self.CN = sp.csr_matrix((self.n, self.n), dtype=np.complex128)
        if near:
            self._near_setup()

    def _gram_sparse(self):
        _, h, _, _ = geometry.segments(self.nodes)
        n = self.n
        i = np.arange(n)
        rows = np.concatenate([i, i, (i + 1) % n])
        cols = np.concatenate([i, (i + 1) % n, i])
        data = np.concatenate([(np.roll(h, 1) + h) / 3.0, h / 6.0, h / 6.0])
        return sp.csc_matrix((data, (rows, cols)), shape=(n, n))

    def _near_setup(self, rows=None):
        if rows is None:
            ni, nj = near_pairs_te(self.nodes, self.near_radius)
        else:
            ni, nj = near_pairs_te(self.nodes, self.near_radius)
            keep = np.isin(ni, rows)
            ni, nj = ni[keep], nj[keep]
        self.near_rows, self.near_cols = ni, nj
        Sx, Nx = dense.te_entries(self.nodes, self.k, ni, nj)
        A = {key: aim_entries(self.proj[key], self.proj[key], self.c, self.m, ni, nj) for key in ("S", "d", "nx", "ny")}
        cS = Sx - A["S"]
        cN = Nx - (A["d"] - self.k ** 2 * (A["nx"] + A["ny"]))
        self.CS = sp.csr_matrix((cS, (ni, nj)), shape=(self.n, self.n))
        self.CN = sp.csr_matrix((cN, (ni, nj)), shape=(self.n, self.n))

    # operators
    def S(self, x, method="fft"):
        return self._apply(self.proj["S"], self.proj["S"], x, False, method) + (self.CS @ np.asarray(x).T).T

    def S_alpha(self, x, method="fft"):
        return self._apply(self.proj["S"], self.proj["S"], x, True, method)

    def N(self, x, method="fft"):
        pr = self.proj
        y = self._apply(pr["d"], pr["d"], x, False, method)
        y = y - self.k ** 2 * (self._apply(pr["nx"], pr["nx"], x, False, method) + self._apply(pr["ny"], pr["ny"], x, False, method))
        return y + (self.CN @ np.asarray(x).T).T

    def N_alpha(self, x, method="fft"):
        """N (Maue form) with the numerically filtered kernel c^alpha of Eq. 10 in all three
        projections and no near-field correction: the filter applied to the hypersingular operator
        as Eq. 10 applies it to S."""
        pr = self.proj
        y = self._apply(pr["d"], pr["d"], x, True, method)
        return y - self.k ** 2 * (self._apply(pr["nx"], pr["nx"], x, True, method) +
                                  self._apply(pr["ny"], pr["ny"], x, True, method))

    def gram_solve(self, x):
        from scipy.sparse.linalg import splu
        if not hasattr(self, "_Glu"):
            self._Glu = splu(sp.csc_matrix(self.G, dtype=np.complex128))
        x = np.asarray(x, dtype=np.complex128)
        return self._Glu.solve(x.T).T if x.ndim > 1 else self._Glu.solve(x)

    def calderon(self, x, filtered=True, method="fft"):
        """G^-1 S G^-1 N x (Eq. 3), with S^alpha of Eq. 10 when filtered."""
        z = self.gram_solve(self.N(x, method))
        w = self.S_alpha(z, method) if filtered else self.S(z, method)
        return self.gram_solve(w)

    def calderon_both(self, x, method="fft"):
        """G^-1 S^alpha G^-1 N^alpha x: Eq. 3 with both operators filtered."""
        return self.gram_solve(self.S_alpha(self.gram_solve(self.N_alpha(x, method)), method))


class TMOperators(_AimBase):
    """TM, pulse basis, midpoint collocation: Z = j k eta S (unfiltered + near field) and Z^alpha."""

    def __init__(self, nodes, k, m, P, s=4, p=4, alpha=None, L=None, near_radius=None, direct_dft=None,
                 eta=1.0, near=True, filter_kind="numerical"):
        self._grid_setup(nodes, k, m, P, s, p, alpha if alpha is not None else 8.0 * k, L, near_radius, direct_dft,
                         filter_kind)
        self.eta = float(eta)
        self.proj = tm_projections(self.nodes, self.p, self.L, self.eps, self.m, self.s)
        self.CZ = sp.csr_matrix((self.n, self.n), dtype=np.complex128)
        if near:
            ni, nj = near_pairs_tm(self.nodes, self.near_radius)
            self.near_rows, self.near_cols = ni, nj
            zx = 1j * self.k * self.eta * dense.tm_point_segment(self.nodes, self.k, ni, nj)
            za = 1j * self.k * self.eta * aim_entries(self.proj["tst"], self.proj["src"], self.c, self.m, ni, nj)
            self.CZ = sp.csr_matrix((zx - za, (ni, nj)), shape=(self.n, self.n))

    def Z(self, x, method="fft"):
        y = 1j * self.k * self.eta * self._apply(self.proj["tst"], self.proj["src"], x, False, method)
        return y + (self.CZ @ np.asarray(x).T).T

    def Z_alpha(self, x, method="fft"):
        return 1j * self.k * self.eta * self._apply(self.proj["tst"], self.proj["src"], x, True, method)
