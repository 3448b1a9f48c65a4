"""Five-stage, fourth-order low-storage Runge-Kutta scheme (oracle; test
infrastructure only).

Sec. 5.4 of the paper embeds the advection operator in "a low-storage
Runge-Kutta scheme of order 4 with 5 stages, which uses two auxiliary vectors
besides the solution vector" and cites Kennedy, Carpenter & Lewis (2000).  The
paper prints no coefficients; the values below are that publication's
five-stage fourth-order "2R" scheme.  They are pinned in the tests by the eight
fourth-order conditions, which a wrong digit anywhere would break.

2R form: with the stage vector w (initially the solution u), for stage s
    K   = L(w)
    w   = u + a_s dt K        (s < 5; uses u before this stage's update)
    u   = u + b_s dt K
which is the explicit scheme with Butcher matrix A[i, i-1] = a_{i-1},
A[i, j] = b_j for j < i-1, and weights b.
"""
from fractions import Fraction

import numpy as np

A_FRAC = [
    Fraction(970286171893, 4311952581923),
    Fraction(6584761158862, 12103376702013),
    Fraction(2251764453980, 15575788980749),
    Fraction(26877169314380, 34165994151039),
]
B_FRAC = [
    Fraction(1153189308089, 22510343858157),
    Fraction(1772645290293, 4653164025191),
    Fraction(-1672844663538, 4480602732383),
    Fraction(2114624349019, 3568978502595),
    Fraction(5198255086312, 14908931495163),
]
A = np.array([float(x) for x in A_FRAC])
B = np.array([float(x) for x in B_FRAC])
STAGES = 5


def butcher(frac=False):
    """Butcher tableau (A, b, c) of the 2R scheme."""
    z = Fraction(0) if frac else 0.0
    a = A_FRAC if frac else list(A)
    b = B_FRAC if frac else list(B)
    M = [[z] * STAGES for _ in range(STAGES)]
    for i in range(1, STAGES):
        M[i][i - 1] = a[i - 1]
        for j in range(i - 1):
            M[i][j] = b[j]
    c = [sum(row, z) for row in M]
    return M, b, c


def step(L, u, dt):
    """One LSRK(5,4) step in 2R form for du/dt = L(u)."""
    u = np.array(u, dtype=np.result_type(np.asarray(u), np.float64))
    w = u.copy()
    for s in range(STAGES):
        K = L(w)
        if s < STAGES - 1:
            w = u + A[s] * dt * K
        u = u + B[s] * dt * K
    return u


def step_butcher(L, u, dt):
    """The same step written with the full Butcher tableau (cross-check)."""
    M, b, _ = butcher()
    u = np.array(u, dtype=np.result_type(np.asarray(u), np.float64))
    Ks = []
    for i in range(STAGES):
        y = u.copy()
        for j in range(i):
            if M[i][j] != 0.0:
                y = y + dt * M[i][j] * Ks[j]
        Ks.append(L(y))
    return u + dt * sum(b[i] * Ks[i] for i in range(STAGES))


def stability_polynomial_coeffs():
    """Coefficients of R(z) = sum_m gamma_m z^m, gamma_m = b^T A^{m-1} 1."""
    M, b, _ = butcher(frac=True)
    vec = [Fraction(1)] * STAGES
    coeffs = [Fraction(1)]
    for _ in range(STAGES):
        coeffs.append(sum(bi * vi for bi, vi in zip(b, vec)))
        vec = [sum(M[i][j] * vec[j] for j in range(STAGES)) for i in range(STAGES)]
    return coeffs
