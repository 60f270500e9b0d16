"""Planted mistakes: each test plants one plausible error in the oracle (on the CPU) and
checks that a pin of `test_oracle_pins.py` would catch it. This shows the pins are tight
enough that a dropped term, a wrong sign, a swapped index or a transposed operand fails."""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.sparse as sp

import synth
from oracle import aim, dense, geometry, special

K = 2.0 * math.pi


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def circle_mu_error(mode=3, n=128):
    nodes = synth.circle_polygon(1.0, n)
    S, N = dense.te_dense(nodes, K)
    G = geometry.gram_dense(nodes)
    v = np.exp(1j * mode * 2 * math.pi * np.arange(n) / n)
    lam = (S[0] @ v) / (G[0] @ v)
    mu = (N[0] @ v) / (G[0] @ v)
    return (abs(lam - special.circle_lambda(mode, K, 1.0)) / abs(special.circle_lambda(mode, K, 1.0)),
            abs(mu - special.circle_mu(mode, K, 1.0)) / abs(special.circle_mu(mode, K, 1.0)))


def aim_vs_dense_error():
    nodes = synth.StarContour.from_seed(0).polygon(3.0, 48)
    S, N = dense.te_dense(nodes, K)
    op = aim.TEOperators(nodes, K, 40, 80)
    x = synth.random_coeffs(48, 1, 1)[0]
    return rel(op.S(x), S @ x), rel(op.N(x), N @ x)


def test_baseline_errors_small():
    e_lam, e_mu = circle_mu_error()
    assert e_lam < 2e-2 and e_mu < 2e-2
    es, en = aim_vs_dense_error()
    assert es < 2e-3 and en < 2e-3


def test_planted_wrong_sign_of_k2_term_in_N(monkeypatch):
    orig = dense.te_piece_terms

    def bad(nodes, k, e, f, I):
        Is, Nt = orig(nodes, k, e, f, I)
        _, h, _, nrm = geometry.segments(nodes)
        nn = np.sum(nrm[np.asarray(e)] * nrm[np.asarray(f)], axis=1)
        return Is, Nt + 2 * k * k * nn[:, None, None] * I        # flips the sign of -k^2 (n.n') phi phi
    monkeypatch.setattr(dense, "te_piece_terms", bad)
    assert circle_mu_error()[1] > 0.1


def test_planted_hankel_of_first_kind(monkeypatch):
    monkeypatch.setattr(special, "green", lambda k, r: -0.25j * (scipy.special.j0(k * np.asarray(r)) + 1j * scipy.special.y0(k * np.asarray(r))))
    assert circle_mu_error()[0] > 0.1


def test_planted_dropped_segment_length(monkeypatch):
    orig = dense.pair_integrals

    def bad(nodes, k, e, f, **kw):
        _, h, _, _ = geometry.segments(nodes)
        return orig(nodes, k, e, f, **kw) / h[np.asarray(f)][:, None, None]
    monkeypatch.setattr(dense, "pair_integrals", bad)
    assert circle_mu_error()[0] > 0.1


def test_planted_transposed_stencil(monkeypatch):
    orig = aim.stencils

    def bad(points, L, eps, s):
        bx, by, W = orig(points, L, eps, s)
        return bx, by, np.swapaxes(W, -1, -2)
    monkeypatch.setattr(aim, "stencils", bad)
    es, en = aim_vs_dense_error()
    assert es > 1e-2 or en > 1e-2


def test_planted_swapped_hat_pieces(monkeypatch):
    orig = geometry.gauss_nodes

    def bad(nodes, p):
        r, w, xi = orig(nodes, p)
        return r, w, 1.0 - xi          # hat values taken at the mirrored node
    monkeypatch.setattr(geometry, "gauss_nodes", bad)
    es, en = aim_vs_dense_error()
    assert es > 1e-2 or en > 1e-2


def test_planted_stencil_off_by_one(monkeypatch):
    orig = aim.lagrange_1d

    def bad(xi, s):
        base, w = orig(xi, s)
        return base + 1, w
    monkeypatch.setattr(aim, "lagrange_1d", bad)
    # a uniform shift of every stencil preserves relative positions, so the operator pins
    # cannot see it; the polynomial-reproduction pin does
    xi = np.linspace(20.1, 29.9, 17)
    base, w = aim.lagrange_1d(xi, 4)
    nodes = base[:, None] + np.arange(4)[None, :]
    assert np.max(np.abs(np.sum(w * nodes, axis=1) - xi)) > 0.5


def test_planted_self_term_not_zeroed(monkeypatch):
    orig = aim.grid_kernel

    def bad(k, eps, P):
        c = orig(k, eps, P)
        c[0, 0] = special.green(k, 0.5 * eps)
        return c
    monkeypatch.setattr(aim, "grid_kernel", bad)
    c = aim.grid_kernel(K, 0.07, 32)
    Chat = aim.dft2(c, direct=True)
    assert abs(Chat.sum()) > 1e-6 * np.abs(Chat).max() * 32


def test_planted_missing_mask_or_wrong_radius(monkeypatch):
    nodes = synth.circle_polygon(1.0, 256)
    G = geometry.gram_dense(nodes)
    v = np.exp(1j * 80 * 2 * math.pi * np.arange(256) / 256)
    for bad in (lambda P, eps, alpha: np.ones((P, P), bool),
                lambda P, eps, alpha: (2 * math.pi / P) * np.hypot(*np.meshgrid(aim.signed_index(P), aim.signed_index(P))) <= alpha):
        monkeypatch.setattr(aim, "filter_mask", bad)
        op = aim.TEOperators(nodes, K, 128, 256, alpha=8 * K, near=False, direct_dft=False)
        high = abs(np.vdot(v, op.S_alpha(v)) / np.vdot(v, G @ v))
        assert high > 1e-3 * abs(special.circle_lambda(80, K, 1.0))


def test_planted_forward_transform_used_as_inverse(monkeypatch):
    m, P, eps = 10, 20, 0.05
    u = synth.random_grid(m, 1, seed=3)[0]
    c = aim.grid_kernel(K, eps, P)
    iy, ix = np.divmod(np.arange(m * m), m)
    r = eps * np.hypot(iy[:, None] - iy[None, :], ix[:, None] - ix[None, :])
    T = np.where(r > 0, special.green(K, np.where(r > 0, r, 1.0)), 0.0)
    brute = (T @ u.ravel()).reshape(m, m)
    monkeypatch.setattr(scipy.fft, "ifft2", lambda X, workers=None: scipy.fft.fft2(X) / (X.shape[-1] * X.shape[-2]))
    assert rel(aim.conv_fft(u, aim.dft2(c, direct=True)), brute) > 0.1


# --------------------------------------------------------------------------------------
# TM projections (pulse sources, midpoint collocation): each plant fails the TM pins
# --------------------------------------------------------------------------------------
def _tm_pin_fails():
    from test_oracle_pins import _tm_aim_errors
    return any(e48 >= 0.1 * e24 or e48 >= 3e-4 for e24, e48 in _tm_aim_errors())


def test_planted_equal_pulse_weights(monkeypatch):
    orig = aim.tm_projections

    def bad(nodes, p, L, eps, m, s):
        out = orig(nodes, p, L, eps, m, s)
        nodes = np.asarray(nodes)
        r, w, _ = geometry.gauss_nodes(nodes, p)
        w = np.repeat(w.sum(axis=1, keepdims=True) / p, p, axis=1)   # Gauss weights replaced by h/p
        ix0, iy0, W = aim.stencils(r, L, eps, s)
        seg = np.arange(len(nodes))[:, None] * np.ones((1, p), dtype=np.int64)
        rr, cc, dd = aim._coo_from_stencils(ix0, iy0, W, seg, w, m, s)
        out["src"] = sp.csr_matrix((dd, (rr, cc)), shape=(m * m, len(nodes)))
        return out
    monkeypatch.setattr(aim, "tm_projections", bad)
    assert _tm_pin_fails()


def test_planted_collocation_at_vertex(monkeypatch):
    orig = aim.tm_projections

    def bad(nodes, p, L, eps, m, s):
        out = orig(nodes, p, L, eps, m, s)
        nodes = np.asarray(nodes)
        jx0, jy0, V = aim.stencils(nodes, L, eps, s)                     # vertex instead of midpoint
        rr, cc, dd = aim._coo_from_stencils(jx0, jy0, V, np.arange(len(nodes)), np.ones(len(nodes)), m, s)
        out["tst"] = sp.csr_matrix((dd, (rr, cc)), shape=(m * m, len(nodes)))
        return out
    monkeypatch.setattr(aim, "tm_projections", bad)
    assert _tm_pin_fails()


def test_planted_swapped_source_and_test(monkeypatch):
    orig = aim.tm_projections
    monkeypatch.setattr(aim, "tm_projections",
                        lambda *a: {"src": orig(*a)["tst"], "tst": orig(*a)["src"]})
    assert _tm_pin_fails()


def test_planted_shifted_segment_index(monkeypatch):
    orig = aim.tm_projections

    def bad(nodes, p, L, eps, m, s):
        out = orig(nodes, p, L, eps, m, s)
        src = out["src"].tocsc()
        out["src"] = src[:, np.roll(np.arange(src.shape[1]), 1)].tocsr()
        return out
    monkeypatch.setattr(aim, "tm_projections", bad)
    assert _tm_pin_fails()


def test_planted_sign_of_the_filtered_tail(monkeypatch):
    # Eq. 6 subtracts the tail beyond alpha; adding it instead flips the sign of the principal-value
    # part of the regular form; the analytic-filter pin against lambda_n^alpha catches it
    orig = special.filtered_green

    def bad(k, alpha, r):
        v = orig(k, alpha, r)
        return complex(-v.real, v.imag)
    monkeypatch.setattr(special, "filtered_green", bad)
    N = 128
    nodes = synth.circle_polygon(1.0, N)
    G = geometry.gram_dense(nodes)
    op = aim.TEOperators(nodes, K, 48, 96, alpha=4 * K, near=False, direct_dft=False, filter_kind="analytic")
    v = np.ones(N, dtype=np.complex128)
    lam0 = np.vdot(v, op.S_alpha(v)) / np.vdot(v, G @ v)
    exact = special.circle_lambda_filtered(0, K, 1.0, 4 * K)
    assert abs(lam0 - exact) > 0.1 * abs(exact)
