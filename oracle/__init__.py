"""Plain, slow CPU oracle for the numerically filtered AIM operators of the 2D EFIE.

TEST INFRASTRUCTURE ONLY. Nothing in the product (the CUDA library and its Python
binding) imports, links or runs this package. Only the tests, the `smoke()` check and
the benchmark's CPU-baseline leg may use it.

Everything here is numpy/scipy in float64 / complex128 and follows the paper
(Pignatelli et al., "A Numerical Approach to Operator Filtering within the Adaptive
Integral Method for Electromagnetic Integral Equations") step by step:

* `geometry`   - flat-segment mesh of the contour, Gauss nodes, P1 hats (Sec. II)
* `special`    - Green's function g (Sec. II), Gauss rules, closed-form circle results
* `dense`      - exact dense Galerkin S, N, G (Eqs. 2-4, Eq. 7) and TM collocation
* `aim`        - the AIM factorisation G_nodes ~ Lambda^T G_grid Lambda (Sec. III-A),
                 circulant embedding and FFT product (Eq. 8), circular spectral
                 truncation (Sec. III-B), the filtered operator (Eq. 10), the zeroed
                 self term (Sec. III-C), and the near-field correction
* `solve`      - Calderon composition (Eq. 3) and a plain restarted GMRES

Parity status per function is listed in each module's header.
"""
