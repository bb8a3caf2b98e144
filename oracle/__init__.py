"""FP64 CPU oracle for the decoupled phase-field scheme of Yang, Christov & Dong
(arXiv 2305.09020), Algorithms 1 (2D) and 2 (3D hybrid Fourier/spectral element).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.

It is deliberately plain: every discrete operator is assembled as a global
sparse matrix from element-by-element GLL quadrature (Section 3.2.1), every
linear system of the time step is solved by a direct sparse LU of the
assembled matrix with Dirichlet rows eliminated, and the 3D algorithm reduces
to per-mode 2D problems through numpy's real FFT (Section 3.2.2, eqs. 74-78).
It shares no code with the CUDA path.

Modules:
  gll.py           Gauss-Lobatto-Legendre nodes, weights, differentiation.
  sem.py           tensor-product spectral-element mesh and sparse operators.
  scheme.py        the time step (Alg. 1 / Alg. 2), the initial potential
                   fixed point (Remark in Sec. 3.1), diagnostics.
  manufactured.py  sympy-derived source terms for the manufactured solutions
                   of eq. (80) and eq. (81).

Parity status per function is stated in each module header.
"""
