"""Host logic of the spectral diagnostics (no GPU): the Laplace-Beltrami eigenpairs that order
the singular values of Figs. 2-3."""
import numpy as np
import pytest

pytest.importorskip("torch")


def test_laplace_beltrami_modes_of_a_regular_polygon():
    # P1 hats on N equal segments of length h: K and G are circulant, with eigenvalues
    # (2/h)(1 - cos t) and (h/3)(2 + cos t) at t = 2 pi n/N, so lam_n = 6 (1 - cos t)/(h^2 (2 + cos t))
    import math
    import synth
    from paper_2606_10784_gb300 import diagnostics
    N = 48
    nodes = synth.circle_polygon(1.0, N)
    h = 2.0 * math.sin(math.pi / N)
    lam, X, G = diagnostics.laplace_beltrami(nodes)
    t = 2 * math.pi * np.arange(N) / N
    want = np.sort(6 * (1 - np.cos(t)) / (h * h * (2 + np.cos(t))))
    assert np.max(np.abs(lam - want)) < 1e-10 * want.max()
    assert np.allclose(X.T @ G @ X, np.eye(N), atol=1e-12)
