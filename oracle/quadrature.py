"""1D quadrature rules and nodal Lagrange bases (oracle; test infrastructure only).

Sec. 2.3 of the paper uses tensor products of 1D shape functions of degree k
(``P_k^d = P_k^1 x ... x P_k^1``); Sec. 2.5 builds cell and face quadrature as
tensor products of 1D rules and names the two families used here:
Gauss-Legendre (exact to degree 2 n_q - 1) and Gauss-Lobatto (exact to degree
2 n_q - 3, endpoints included).

Everything is FP64.  Gauss-Legendre points come from numpy's library routine
``leggauss``; Gauss-Lobatto points are the endpoints plus the roots of
P'_{n-1}, with the classical weights 2 / (n (n-1) P_{n-1}(x)^2).
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes and weights on [-1, 1] (Sec. 2.5)."""
    if n < 1:
        raise ValueError("n >= 1 required")
    x, w = _leg.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gauss_lobatto(n):
    """n-point Gauss-Lobatto nodes and weights on [-1, 1] (Sec. 2.3, 2.5)."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs n >= 2")
    pn1 = _leg.Legendre.basis(n - 1)
    inner = np.sort(np.real(pn1.deriv().roots())) if n > 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (n * (n - 1) * pn1(x) ** 2)
    return x.astype(np.float64), w.astype(np.float64)


def lagrange_values(nodes, x):
    """Matrix V[i, p] = phi_p(x_i) of the Lagrange polynomials through ``nodes``.

    phi_p(x) = prod_{m != p} (x - z_m) / (z_p - z_m).
    """
    z = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(z)
    V = np.ones((len(x), n))
    for p in range(n):
        for m in range(n):
            if m != p:
                V[:, p] *= (x - z[m]) / (z[p] - z[m])
    return V


def lagrange_derivatives(nodes, x):
    """Matrix D[i, p] = phi_p'(x_i) (product rule applied to the formula above)."""
    z = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(z)
    D = np.zeros((len(x), n))
    for p in range(n):
        for r in range(n):
            if r == p:
                continue
            term = np.full(len(x), 1.0 / (z[p] - z[r]))
            for m in range(n):
                if m != p and m != r:
                    term *= (x - z[m]) / (z[p] - z[m])
            D[:, p] += term
    return D


class Tables1D:
    """1D ingredients of the tensor-product element of degree k.

    basis="gl":  nodal basis at the n = k+1 Gauss-Legendre points with the same
                 points as quadrature (collocation; mass matrix diagonal).
    basis="gll": nodal basis at the Gauss-Lobatto points with n_q = k+1
                 Gauss-Legendre quadrature (the paper's default configuration,
                 Sec. 1.3 and 2.5, kept in Sec. 5.3), i.e. a non-trivial basis
                 change.
    basis="gllc": nodal basis at the n = k+1 Gauss-Lobatto points with the same
                 points as quadrature (the collocation variant the paper
                 mentions as an alternative, Sec. 2.5 and 5.3; exact to degree 2k-1,
                 mass matrix diagonal).

    B[q, p]  = phi_p(zeta_q)      basis at quadrature points
    Bd[q, p] = phi_p'(zeta_q)     derivative at quadrature points
    lp[p]    = phi_p(+1), lm[p] = phi_p(-1)   face values
    w[q]     = quadrature weights, zeta[q] = quadrature points
    """

    def __init__(self, k, basis="gl"):
        if k < 0:
            raise ValueError("degree k >= 0 required")
        n = k + 1
        self.k, self.n, self.basis = k, n, basis
        if basis in ("gll", "gllc") and n < 2:
            raise ValueError("GLL basis needs k >= 1")
        if basis == "gllc":
            self.zeta, self.w = gauss_lobatto(n)
        else:
            self.zeta, self.w = gauss_legendre(n)
        if basis in ("gl", "gllc"):
            self.nodes = self.zeta.copy()
        elif basis == "gll":
            self.nodes, _ = gauss_lobatto(n)
        else:
            raise ValueError(basis)
        self.B = lagrange_values(self.nodes, self.zeta)
        self.Bd = lagrange_derivatives(self.nodes, self.zeta)
        self.lp = lagrange_values(self.nodes, [1.0])[0]
        self.lm = lagrange_values(self.nodes, [-1.0])[0]
