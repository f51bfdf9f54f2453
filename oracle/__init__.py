"""Plain, slow FP64 CPU oracle of the contour-integral (CISS) hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package. The
product (the CUDA library and its Python binding) never calls it and shares no
code with it.

What it computes, step by step, in complex128 (each module cites its passage):
  contour.py    quadrature nodes/weights on an ellipse (trapezoid rule) and the
                coefficient table F[i, j] = f_i(z_j) (split form, Sec. 2 Eq. (split));
  fn.py         the scalar function classes of Sec. 3.2.2 and their derivatives;
  band_lu.c     banded LU with partial pivoting and the banded solve (plain C);
  band.py       band storage assembly of T(z_j) = sum_i f_i(z_j) A_i and ctypes glue;
  ciss.py       solves T(z_j) Y_j = V with FP64 refinement, moments, block Hankel
                SVD, reduced eigenproblem, Rayleigh-Ritz projection (Eq. (narnoldi-split))
                with Newton (Eq. (newton)) and the scaled residual (Eq. (sressplit));
  count.py      eigenvalue count inside the contour by the argument principle;
  interpol.py   the polynomial interpolation solver of Sec. 4.4 (Chebyshev coefficients, Eq.
                (polinterpcoef), and the dense Chebyshev-basis linearisation of P_d).

Parity status of each function is listed in its docstring; all intermediate
Hankel/Rayleigh-Ritz matrices depend on the random probe block V and are
"parity unpinned" beyond agreement with this oracle: only end results
(eigenvalues, residuals, moments of closed-form cases, counts) are pinned.
"""
