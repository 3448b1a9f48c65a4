"""FP64 CPU oracle for the high-dimensional DG advection operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything in this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously-correct restatement of the method of
Munch, Kormann & Kronbichler, "hyper.deal: An efficient, matrix-free
finite-element library for high-dimensional partial differential equations"
(arXiv 2002.08110):

* ``quadrature``  -- 1D Gauss-Legendre / Gauss-Lobatto rules and Lagrange
  bases (Sec. 2.3 "Elements and degrees of freedom", Sec. 2.5 "Quadrature").
* ``dg``          -- the weak form of the advection equation in reference
  coordinates (Sec. 1.3, Eq. "into:adv:ref") with the phase-space
  block-diagonal Jacobian (Sec. 3, first display), upwind flux, element-centric
  evaluation over cell pairs (Algorithms 1 and 2), the mass matrix and its
  inverse (Algorithm 2 step 4).  Operators are written as Kronecker products of
  1D matrices and applied either as dense matrices (``dense_cell_operator``,
  tiny cells only) or axis by axis with ``numpy.tensordot`` (``apply``); the
  two routes are checked against each other in the tests.
* ``lsrk``        -- the five-stage, fourth-order low-storage Runge-Kutta
  scheme cited in Sec. 5.4 (Kennedy, Carpenter & Lewis 2000).

Every floating-point computation here is FP64.
"""
