"""Vlasov-Poisson coupling for one configuration dimension (oracle; test
infrastructure only -- the product path never imports this module).

Sec. 6 of arXiv 2002.08110 advances electrons in a neutralising background:
    df/dt + (v, -E(t, x)) . grad f = 0,
    rho = 1 - int f dv,   -phi'' = rho,   E = -phi'   (Eq. vp:close),
with LSRK(5,4) time stepping whose every stage (i) reduces f to rho over
velocity space, (ii)-(iv) solves the Poisson problem for E and (v) applies
the advection operator with the field a = (v, -E).

Written from those definitions:
* ``charge_density`` is ``Problem.charge_density`` (the v integral by the v
  cell quadrature, Sec. 2.5).
* ``poisson_periodic_1d``: E' = rho in the physical coordinate, periodic.
  rho is the nodal degree-k polynomial of each x cell; its mean is removed
  (a periodic solution needs a neutral right-hand side) and E is its exact
  antiderivative, fixed to zero mean (phi periodic).  Each cell's polynomial
  is recovered in the monomial basis by solving the Vandermonde system at the
  nodes and integrated with numpy's polynomial routines; E is returned as a
  callable piecewise polynomial (the advection operator evaluates it wherever
  it needs the field) and at the nodes.
* ``vp_rhs`` / ``vp_step``: the stage right-hand side with the field
  recomputed from the stage's own input, inside ``lsrk.step``.

Readings: the paper gives no discretisation of the Poisson problem for
d_x = 1 (its solver is multigrid on the x mesh); the exact antiderivative of
the DG charge density is the reading taken here.  The field enters the
advection operator as its v components a_v = -E (component 1) and 0 for any
further velocity dimension (no magnetic field).
"""
import numpy as np
from numpy.polynomial import polynomial as P

from . import lsrk
from .dg import PhaseSpaceField


class PiecewiseField:
    """E(y) on a periodic 1D lattice: per cell, coefficients in the local
    variable xi = 2 (y - y_c) / h_y - 1 in [-1, 1]."""

    def __init__(self, y_lo, h_y, coeffs):
        self.y_lo, self.h_y, self.coeffs = y_lo, h_y, coeffs
        self.ncells = len(coeffs)

    def __call__(self, y):
        y = np.asarray(y, dtype=np.float64)
        s = (y - self.y_lo) / self.h_y
        # points on a cell boundary take the cell to their left when the
        # right one would wrap past the box (E is continuous there anyway)
        c = np.clip(np.floor(s), 0, self.ncells - 1).astype(np.int64)
        xi = 2.0 * (s - c) - 1.0
        C = np.asarray(self.coeffs)[c]                    # (..., degree + 1)
        powers = xi[..., None] ** np.arange(C.shape[-1])
        return np.sum(C * powers, axis=-1)


def poisson_periodic_1d(p, rho):
    """E with E' = rho - mean(rho), zero mean, for the x mesh of ``p``
    (dim_x = 1).  ``rho`` has shape (x cells, n).  Returns (E callable of the
    lattice coordinate, E at the x nodes with the shape of rho)."""
    assert p.dx == 1
    n, zeta = p.n, p.T.nodes
    ncx = int(p.cells[0])
    hy = p.h[0]
    hx = p.S[0, 0] * hy                       # physical cell length (signed)
    V = np.vander(zeta, n, increasing=True)   # V[q, m] = zeta_q^m
    coef = [np.linalg.solve(V, rho[c]) for c in range(ncx)]
    # mean of rho over the period: sum of the cell integrals / length
    ints = [P.polyval(1.0, P.polyint(a)) - P.polyval(-1.0, P.polyint(a)) for a in coef]
    rho_bar = np.sum(ints) / (2.0 * ncx)
    E_coef = []
    left = 0.0                                # E at the left end of the cell
    for c in range(ncx):
        a = coef[c].copy()
        a[0] -= rho_bar
        # dE/dxi = (h_x / 2) (rho - rho_bar)
        anti = P.polyint(a) * (hx / 2.0)
        anti[0] += left - P.polyval(-1.0, anti)
        E_coef.append(anti)
        left = P.polyval(1.0, anti)
    # zero mean: subtract (1 / L) int E dy
    mean = np.sum([(P.polyval(1.0, P.polyint(a)) - P.polyval(-1.0, P.polyint(a))) / 2.0
                   for a in E_coef]) / ncx
    for a in E_coef:
        a[0] -= mean
    field = PiecewiseField(p.lo[0], hy, E_coef)
    nodal = np.array([P.polyval(zeta, a) for a in E_coef])
    return field, nodal


def field_from(p, u):
    """The Vlasov field (v, -E) with E from the state u (Sec. 6, steps 1-4)."""
    rho = p.charge_density(u)
    E, _ = poisson_periodic_1d(p, rho)
    dv = p.dv

    def a_v(yx):
        e = -E(yx[..., 0])
        out = np.zeros(e.shape + (dv,))
        out[..., 0] = e
        return out

    return PhaseSpaceField(1, dv, a_v)


def vp_rhs(p, u):
    """M^{-1} A(u) with the field of u (one stage right-hand side)."""
    return p.with_field(field_from(p, u)).apply(u)


def vp_step(p, u, dt):
    """One LSRK(5,4) step of the Vlasov-Poisson system."""
    return lsrk.step(lambda w: vp_rhs(p, w), u, dt)
