"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, textbook special cases, exact identities of the upwind DG operator,
values printed in the paper, and brute force on tiny inputs.  A dropped term,
a wrong sign or index, or a transposed operand in ``oracle/`` breaks at least
one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as P

from oracle import lsrk
from oracle.dg import ConstantField, PhaseSpaceField, Problem
from oracle.quadrature import (Tables1D, gauss_legendre, gauss_lobatto,
                               lagrange_derivatives, lagrange_values)
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _problem(w, basis="gl", field=None):
    if field is None:
        if w.field_kind == 0:
            field = ConstantField(w.a_const)
        else:
            field = PhaseSpaceField(w.dx, w.dv, W.e_function(w))
    shear = None if w.shear is None else np.array(w.shear).reshape(w.dx, w.dx)
    return Problem(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                   field, shear=shear, basis=basis)


# ---------------------------------------------------------------------------
# 1D tables (Sec. 2.5: Gauss exact to 2n-1, Gauss-Lobatto to 2n-3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exactness(n):
    x, w = gauss_legendre(n)
    for m in range(2 * n):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x ** m) - exact) < 1e-14
    # and not exact one degree higher (even monomial 2n)
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gauss_lobatto_exactness(n):
    x, w = gauss_lobatto(n)
    assert x[0] == -1.0 and x[-1] == 1.0
    for m in range(2 * n - 2):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x ** m) - exact) < 1e-13
    m = 2 * n - 2
    assert abs(np.sum(w * x ** m) - 2.0 / (m + 1)) > 1e-6


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("basis", ["gl", "gll"])
def test_lagrange_tables_reproduce_polynomials(k, basis):
    T = Tables1D(k, basis)
    rng = np.random.default_rng(k)
    coef = rng.standard_normal(k + 1)                 # random degree-k polynomial
    vals = P.polyval(T.nodes, coef)
    dcoef = P.polyder(coef)
    x = np.linspace(-1, 1, 7)
    assert np.allclose(lagrange_values(T.nodes, x) @ vals, P.polyval(x, coef), atol=1e-12)
    assert np.allclose(lagrange_derivatives(T.nodes, x) @ vals, P.polyval(x, dcoef), atol=1e-11)
    assert np.allclose(lagrange_values(T.nodes, T.nodes), np.eye(k + 1), atol=1e-14)
    assert abs(T.lp @ vals - P.polyval(1.0, coef)) < 1e-12
    assert abs(T.lm @ vals - P.polyval(-1.0, coef)) < 1e-12


# ---------------------------------------------------------------------------
# values printed in the paper
# ---------------------------------------------------------------------------
def test_paper_table_dofs_per_cell():
    g = json.load(open(GOLDEN))["dofs_per_cell"]
    for i, k in enumerate(g["k_rows"]):
        for j, d in enumerate(g["d_cols"]):
            dx = d // 2
            p = Problem(dx, d - dx, k, [1] * dx, [1] * (d - dx), [0] * dx, [1] * dx,
                        [0] * (d - dx), [1] * (d - dx), ConstantField(np.zeros(d)))
            assert p.dofs_per_cell == g["values"][i][j]


def test_paper_table_mapping_memory():
    g = json.load(open(GOLDEN))["mapping_doubles_per_qpoint"]
    n, dx, dv = g["k"] + 1, g["dx"], g["dv"]
    tensor = (n ** dx * dx ** 2 + n ** dv * dv ** 2) / n ** (dx + dv)
    assert round(tensor, 2) == g["tensor_product"]
    assert (dx + dv) ** 2 == g["full_jacobian"]


def test_paper_table_scaling_sizes():
    g = json.load(open(GOLDEN))["strong_scaling_dofs"]
    n = g["k"] + 1
    for row in g["rows"]:
        cells = [c // n for c in row["dofs_per_direction"]]
        p = Problem(3, 3, g["k"], cells[:3], cells[3:], [0] * 3, [1] * 3, [0] * 3, [1] * 3,
                    ConstantField(np.zeros(6)))
        assert abs(p.n_dofs / row["dofs"] - 1.0) < 0.03


# ---------------------------------------------------------------------------
# brute force: axis-by-axis evaluation == dense Kronecker matrices
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dx,dv,k,cells", [
    (1, 1, 3, (3, 2)), (1, 1, 1, (1, 2)), (2, 1, 2, (2, 1, 3)), (1, 2, 4, (2, 2, 1)),
    (2, 2, 1, (2, 1, 2, 1)), (2, 3, 1, (1, 2, 1, 2, 1)), (3, 3, 1, (1, 1, 2, 1, 1, 2)),
    (3, 2, 2, (1, 1, 1, 1, 1)), (1, 1, 5, (2, 2)),
])
@pytest.mark.parametrize("kind", ["const", "phase"])
def test_axiswise_equals_dense(dx, dv, k, cells, kind):
    rng = np.random.default_rng(dx * 10 + dv)
    d = dx + dv
    if kind == "const":
        field = ConstantField(rng.uniform(-1, 1, d))
    else:
        if dv < dx:
            pytest.skip("phase-space field needs dv >= dx")
        amp = rng.uniform(0.2, 1, dv)
        field = PhaseSpaceField(dx, dv, lambda y: amp * np.cos(2 * np.pi * y.sum(-1, keepdims=True) + np.arange(dv)))
    shear = np.eye(dx) + 0.1 * np.triu(np.ones((dx, dx)), 1)
    p = Problem(dx, dv, k, cells[:dx], cells[dx:], [0] * dx, [1] * dx, [-1] * dv, [1] * dv,
                field, shear=shear)
    u = rng.standard_normal(p.n_dofs)
    a = p.apply(u)
    b = p.apply_dense(u)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


# ---------------------------------------------------------------------------
# textbook special case: k = 0 is first-order upwind finite volumes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [(1.0, 0.5), (-0.7, 0.3), (0.4, -1.2), (-1.0, -2.0)])
def test_k0_is_upwind_finite_volume(a):
    nx, nv = 5, 4
    p = Problem(1, 1, 0, (nx,), (nv,), (0,), (2,), (0,), (1,), ConstantField(a))
    rng = np.random.default_rng(3)
    u = rng.standard_normal(p.n_dofs)
    U = u.reshape(nv, nx)                           # cell = ix + nx * iv
    h = (2.0 / nx, 1.0 / nv)
    du = np.zeros_like(U)
    for axis, aj, hj in ((1, a[0], h[0]), (0, a[1], h[1])):
        if aj > 0:
            du -= aj / hj * (U - np.roll(U, 1, axis=axis))
        else:
            du -= aj / hj * (np.roll(U, -1, axis=axis) - U)
    assert np.allclose(p.apply(u), du.reshape(-1), atol=1e-13)


# ---------------------------------------------------------------------------
# invariants of the upwind DG operator
# ---------------------------------------------------------------------------
def _small_workloads():
    return [
        W.shrink(W.config_2d(), cells_x=(3,), cells_v=(4,)),
        W.shrink(W.config_4d(), cells_x=(2, 3), cells_v=(3, 2), k=2),
        W.shrink(W.config_6d(), cells_x=(2, 1, 1), cells_v=(1, 2, 1), k=1),
        W.shrink(W.config_adjoint(), cells_x=(2, 1), cells_v=(1, 2, 1), k=2),
    ]


@pytest.mark.parametrize("basis", ["gl", "gllc"])
@pytest.mark.parametrize("w", _small_workloads(), ids=lambda w: w.name)
def test_annihilates_constants(w, basis):
    p = _problem(w, basis=basis)
    r = p.apply(np.ones(p.n_dofs))
    scale = np.max(np.abs(p.apply(np.random.default_rng(0).standard_normal(p.n_dofs))))
    assert np.max(np.abs(r)) <= 1e-13 * scale


@pytest.mark.parametrize("basis", ["gl", "gllc"])
@pytest.mark.parametrize("w", _small_workloads(), ids=lambda w: w.name)
def test_conserves_mass(w, basis):
    p = _problem(w, basis=basis)
    u = np.random.default_rng(1).standard_normal(p.n_dofs)
    Mdiag = p.mass_diagonal()
    Lu = p.apply(u)
    assert abs(Mdiag @ Lu) <= 1e-13 * (np.abs(Mdiag) @ np.abs(Lu))


def _independent_traces(vals, nodes):
    """Value at -1 and +1 of the degree-k interpolant through (nodes, vals),
    by a monomial fit (independent of the oracle's Lagrange tables)."""
    c = P.polyfit(nodes, vals, len(nodes) - 1)
    return P.polyval(-1.0, c), P.polyval(1.0, c)


@pytest.mark.parametrize("basis", ["gl", "gllc"])
@pytest.mark.parametrize("w", _small_workloads()[:3], ids=lambda w: w.name)
def test_energy_identity(w, basis):
    """u^T M L u = -1/2 sum over faces of |J| W_perp |c_n| [u]^2 (upwind flux,
    divergence-free speed that does not vary along its own direction).  For
    the Gauss-Lobatto collocation it holds because that rule integrates
    u du/dx (degree 2k-1) exactly: the summation-by-parts property."""
    p = _problem(w, basis=basis)
    u = np.random.default_rng(2).standard_normal(p.n_dofs)
    lhs = u @ (p.mass_diagonal() * p.apply(u))
    zeta, wq = npleg.leggauss(p.n) if basis == "gl" else gauss_lobatto(p.n)
    d, n = p.d, p.n
    h = np.array(w.h)
    S = np.eye(w.dx) if w.shear is None else np.array(w.shear).reshape(w.dx, w.dx)
    Sinv = np.linalg.inv(S)
    detJ = np.linalg.det(S) * np.prod(h / 2)
    E = W.e_function(w) if w.field_kind == 1 else None
    rhs = 0.0
    for e in range(p.ncells):
        cc = (e // p.strides) % p.cells
        Ue = u[e * n ** d:(e + 1) * n ** d].reshape([n] * d, order="F")
        for j in range(d):
            # this cell is the left side of its +face along j
            cr = cc.copy()
            cr[j] = (cr[j] + 1) % p.cells[j]
            er = int(np.sum(cr * p.strides))
            Ur = u[er * n ** d:(er + 1) * n ** d].reshape([n] * d, order="F")
            for idx in np.ndindex(*([n] * (d - 1))):
                full = list(idx[:j]) + [slice(None)] + list(idx[j:])
                _, tl = _independent_traces(Ue[tuple(full)], zeta)
                tr, _ = _independent_traces(Ur[tuple(full)], zeta)
                q = [zeta[i] for i in idx]
                pos = q[:j] + [1.0] + q[j:]            # reference face point
                y = np.array([w.lo[m] + h[m] * (cc[m] + (pos[m] + 1) / 2) for m in range(d)])
                if w.field_kind == 0:
                    a = np.array(w.a_const)
                else:
                    a = np.concatenate([y[w.dx:2 * w.dx], E(y[None, :w.dx])[0]])
                c = np.concatenate([(2 / h[:w.dx]) * (Sinv @ a[:w.dx]), (2 / h[w.dx:]) * a[w.dx:]])
                wperp = np.prod([wq[i] for i in idx])
                rhs += -0.5 * detJ * wperp * abs(c[j]) * (tl - tr) ** 2
    assert lhs < 0
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


@pytest.mark.parametrize("w", _small_workloads(), ids=lambda w: w.name)
def test_transpose_is_mass_scaled_negated_field(w):
    """L^T = M L(-a) M^{-1} for the upwind flux (exact, cell by cell)."""
    p = _problem(w)
    L = p.assemble().toarray()
    pn = p.with_field(p.field.negated())
    Ln = pn.assemble().toarray()
    Md = p.mass_diagonal()
    rhs = (Md[:, None] * Ln) / Md[None, :]
    assert np.max(np.abs(L.T - rhs)) <= 1e-12 * np.max(np.abs(L))
    # the oracle's adjoint routine is the transpose
    y = np.random.default_rng(4).standard_normal(p.n_dofs)
    assert np.allclose(p.apply_adjoint(y), L.T @ y, rtol=0, atol=1e-12 * np.max(np.abs(L.T @ y)))


@pytest.mark.parametrize("w", _small_workloads()[:2], ids=lambda w: w.name)
def test_gl_collocation_similar_to_gll_gauss(w):
    """GL collocation and the paper's GLL basis with Gauss quadrature span the
    same space with the same quadrature: L_GL = V L_GLL V^{-1} with
    V_qi = phi^GLL_i(zeta_q) applied cell by cell."""
    pg = _problem(w, "gl")
    pl = _problem(w, "gll")
    Lg = pg.assemble().toarray()
    Ll = pl.assemble().toarray()
    T = Tables1D(w.k, "gll")
    V1 = lagrange_values(T.nodes, T.zeta)
    V = np.ones((1, 1))
    for _ in range(pg.d):
        V = np.kron(V1, V)
    Vg = np.kron(np.eye(pg.ncells), V)
    assert np.max(np.abs(Lg @ Vg - Vg @ Ll)) <= 1e-11 * np.max(np.abs(Lg))


def test_consistency_with_the_pde():
    """L u -> -a . grad u for smooth u; a wrong sign gives relative error ~2."""
    errs = []
    for N in (8, 16):
        w = W.config_2d(cells=N)
        p = _problem(w)
        zeta = npleg.leggauss(w.n)[0]
        u = W.separable_state(w, zeta)
        # exact: -(a1 d/dx + a2 d/dv) sin(2 pi x) sin(2 pi v)
        fx = [lambda y: 2 * np.pi * np.cos(2 * np.pi * y), lambda y: np.sin(2 * np.pi * y)]
        fv = [lambda y: np.sin(2 * np.pi * y), lambda y: 2 * np.pi * np.cos(2 * np.pi * y)]
        ux = W.separable_state(W.Workload(**{**w.__dict__, "u0_factors": fx}), zeta)
        uv = W.separable_state(W.Workload(**{**w.__dict__, "u0_factors": fv}), zeta)
        exact = -(w.a_const[0] * ux + w.a_const[1] * uv)
        errs.append(np.linalg.norm(p.apply(u) - exact) / np.linalg.norm(exact))
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] > 4.0


# ---------------------------------------------------------------------------
# LSRK(5,4) (Sec. 5.4, Kennedy-Carpenter-Lewis 2R scheme)
# ---------------------------------------------------------------------------
def test_lsrk_order_conditions():
    A, b, c = lsrk.butcher(frac=True)
    s = lsrk.STAGES
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(s)) for i in range(s)]
    conds = [
        (sum(b), 1), (sum(b[i] * c[i] for i in range(s)), 0.5),
        (sum(b[i] * c[i] ** 2 for i in range(s)), 1 / 3), (sum(b[i] * Ac[i] for i in range(s)), 1 / 6),
        (sum(b[i] * c[i] ** 3 for i in range(s)), 0.25), (sum(b[i] * c[i] * Ac[i] for i in range(s)), 1 / 8),
        (sum(b[i] * Ac2[i] for i in range(s)), 1 / 12), (sum(b[i] * AAc[i] for i in range(s)), 1 / 24),
    ]
    from fractions import Fraction
    for val, target in conds:
        t = Fraction(target).limit_denominator(100)
        assert abs(float(val - t)) < 1e-18


def test_lsrk_low_storage_equals_butcher_form():
    rng = np.random.default_rng(5)
    Lm = rng.standard_normal((7, 7))
    u = rng.standard_normal(7)
    a = lsrk.step(lambda x: Lm @ x, u, 0.05)
    b = lsrk.step_butcher(lambda x: Lm @ x, u, 0.05)
    assert np.allclose(a, b, atol=1e-14)


def test_lsrk_stability_polynomial():
    g = lsrk.stability_polynomial_coeffs()
    for m in range(5):
        assert abs(float(g[m]) - 1.0 / math.factorial(m)) < 1e-15
    lam, dt = -3.0 + 2.0j, 0.1
    z = lam * dt
    R = sum(float(g[m]) * z ** m for m in range(6))
    y = lsrk.step(lambda x: lam * x, np.array([1.0 + 0j]), dt)
    assert abs(y[0] - R) < 1e-14


def test_lsrk_temporal_order_four():
    import scipy.sparse.linalg as spla
    w = W.shrink(W.config_2d(), cells_x=(4,), cells_v=(4,))
    p = _problem(w)
    L = p.assemble()
    zeta = npleg.leggauss(w.n)[0]
    u0 = W.separable_state(w, zeta)
    T = 0.05
    exact = spla.expm_multiply(L * T, u0)
    errs = []
    for nsteps in (8, 16):
        u = u0.copy()
        for _ in range(nsteps):
            u = lsrk.step(lambda x: L @ x, u, T / nsteps)
        errs.append(np.linalg.norm(u - exact))
    assert 3.6 < math.log2(errs[0] / errs[1]) < 4.6


def _rk_run(p, u, dt, steps):
    L = p.assemble()
    for _ in range(steps):
        u = lsrk.step(lambda x: L @ x, u, dt)
    return u


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_order_k_plus_one(k):
    """Product of sines transported by a constant field; the L2 error at a
    fixed time falls like h^{k+1} (smooth data, upwind DG)."""
    errs = []
    for N in (4, 8, 16):
        w = W.config_2d(cells=N)
        w = W.Workload(**{**w.__dict__, "k": k, "final_time": 0.25})
        p = _problem(w)
        zeta = npleg.leggauss(w.n)[0]
        u0 = W.separable_state(w, zeta)
        dt, steps = W.time_step(w)
        dt, steps = dt / 4, steps * 4
        u = _rk_run(p, u0, dt, steps)
        T = dt * steps
        shifted = W.Workload(**{**w.__dict__, "u0_factors": (
            lambda y: np.sin(2 * np.pi * (y - w.a_const[0] * T)),
            lambda y: np.sin(2 * np.pi * (y - w.a_const[1] * T)))})
        exact = W.separable_state(shifted, zeta)
        diff = u - exact
        errs.append(math.sqrt(diff @ (p.mass_diagonal() * diff)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k + 1 - 0.3, rates


def test_one_period_return_2d_config():
    """The 2D workload (16 x 16, k = 3, a = (1, 0.5)) returns to its initial
    state after T = 2 up to the discretisation error."""
    w = W.config_2d()
    p = _problem(w)
    zeta = npleg.leggauss(w.n)[0]
    u0 = W.separable_state(w, zeta)
    dt, steps = W.time_step(w)
    assert steps == 240
    u = _rk_run(p, u0, dt, steps)
    Md = p.mass_diagonal()
    rel = math.sqrt((u - u0) @ (Md * (u - u0)) / (u0 @ (Md * u0)))
    assert rel < 2e-4
    # mass conserved to round-off, energy non-increasing
    assert abs(Md @ u - Md @ u0) < 1e-13
    assert u @ (Md * u) <= u0 @ (Md * u0)


# ---------------------------------------------------------------------------
# Vlasov-Poisson charge density rho = 1 - int f dv (Sec. 6)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dx,dv,k", [(1, 1, 2), (1, 2, 3), (2, 2, 1), (2, 3, 2)])
def test_charge_density_closed_form(dx, dv, k):
    """f = g(x) prod_j (a_j + b_j v_j^2 + c_j v_j^3): the Gauss rule of a v
    cell is exact for degree 2k+1 >= 3, so int f dv = g(x) prod_j I_j with
    I_j the integral over [v_lo_j, v_hi_j] written out by hand."""
    rng = np.random.default_rng(11 + 7 * dx + dv + k)
    cells_x = [3, 2][:dx]
    cells_v = [3, 2, 2][:dv]
    v_lo = -rng.uniform(1.0, 3.0, dv)
    v_hi = rng.uniform(1.0, 3.0, dv)
    p = Problem(dx, dv, k, cells_x, cells_v, [0.0] * dx, [2 * np.pi] * dx, v_lo, v_hi,
                ConstantField([1.0] * (dx + dv)))
    a, b, c = rng.uniform(0.5, 1.5, dv), rng.uniform(-1, 1, dv), rng.uniform(-1, 1, dv)
    kx = np.arange(1, dx + 1)

    def g(yx):
        return 0.3 + np.cos(yx @ kx + 0.2)

    def f(yx, v):
        return g(yx) * np.prod(a + b * v ** 2 + c * v ** 3, axis=-1)

    u = p.interpolate(f)
    rho = p.charge_density(u)
    I = np.prod(a * (v_hi - v_lo) + b * (v_hi ** 3 - v_lo ** 3) / 3 + c * (v_hi ** 4 - v_lo ** 4) / 4)
    ncx = int(np.prod(cells_x))
    for cx in range(ncx):
        # the first v cell shares this x cell's x nodes
        yx, _ = p.node_coordinates(cx)
        gx = g(yx)[(slice(None),) * dx + (0,) * dv].reshape(-1, order="F")
        np.testing.assert_allclose(rho[cx], 1.0 - gx * I, rtol=0, atol=1e-12 * abs(I) + 1e-14)


def test_charge_density_maxwellian():
    """A Landau-damping profile (1 + alpha cos(kx)) e^{-v^2/2} / sqrt(2 pi)^dv on
    a wide v box: rho = -alpha cos(kx) up to the quadrature error and the
    Gaussian tail beyond +-8."""
    alpha, kk = 0.01, 0.5
    p = Problem(1, 2, 3, [4], [16, 16], [0.0], [2 * np.pi / kk], [-8.0] * 2, [8.0] * 2,
                ConstantField([1.0, 1.0, 1.0]))

    def f(yx, v):
        return (1 + alpha * np.cos(kk * yx[..., 0])) * np.exp(-0.5 * np.sum(v ** 2, -1)) / (2 * np.pi)

    rho = p.charge_density(p.interpolate(f))
    for cx in range(4):
        yx, _ = p.node_coordinates(cx)
        x = yx[:, 0, 0, 0]
        np.testing.assert_allclose(rho[cx], -alpha * np.cos(kk * x), atol=2e-6)


def test_charge_density_layout_x_cells_and_nodes():
    """Brute force on a tiny mesh: rho at (x cell, x node) sums exactly the
    DoFs with that x cell and x node, weighted by the v quadrature."""
    p = Problem(2, 2, 1, [2, 3], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], ConstantField([1] * 4))
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    rho = p.charge_density(u)
    n, npc = p.n, p.dofs_per_cell
    wv = p.T.w
    ref = np.ones((6, n * n))
    for e in range(p.ncells):
        cc = p.cell_coords(e)
        cx = cc[0] + 2 * cc[1]
        for q in range(npc):
            q0, q1, q2, q3 = q % n, (q // n) % n, (q // n ** 2) % n, q // n ** 3
            w = wv[q2] * wv[q3] * (p.h[2] / 2) * (p.h[3] / 2)
            ref[cx, q0 + n * q1] -= w * u[e * npc + q]
    np.testing.assert_allclose(rho, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# Vlasov-Poisson for dim_x = 1 (Sec. 6)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k,shear", [(1, None), (3, None), (2, [[1.7]]), (5, [[-0.8]])])
def test_poisson_periodic_closed_form(k, shear):
    """rho = c0 + alpha cos(kappa x) on the period: E = alpha sin(kappa x) /
    kappa (E' = rho - c0, zero mean), up to the interpolation error of rho."""
    from oracle.vp import poisson_periodic_1d
    s = 1.0 if shear is None else shear[0][0]
    kappa, alpha, c0 = 0.5, 0.3, 0.7
    L = 2 * np.pi / kappa
    ncx = 24
    p = Problem(1, 1, k, [ncx], [2], [0.0], [L / s], [-1.0], [1.0], ConstantField([1.0, 1.0]),
                shear=shear)
    xs = np.array([p.node_coordinates(c)[0][:, 0, 0] * s for c in range(ncx)])   # physical x
    rho = c0 + alpha * np.cos(kappa * xs)
    E, nodal = poisson_periodic_1d(p, rho)
    tol = {1: 3e-3, 2: 2e-4, 3: 1e-5, 5: 1e-8}[k]
    np.testing.assert_allclose(nodal, alpha * np.sin(kappa * xs) / kappa, atol=tol)
    # the callable agrees with the nodal values and is continuous and periodic
    ys = np.array([p.node_coordinates(c)[0][:, 0, 0] for c in range(ncx)])
    np.testing.assert_allclose(E(ys), nodal, atol=1e-14)
    edges = p.lo[0] + p.h[0] * np.arange(ncx + 1)
    left = E(edges[1:-1] - 1e-12)
    right = E(edges[1:-1] + 1e-12)
    np.testing.assert_allclose(left, right, atol=1e-9)
    np.testing.assert_allclose(E(np.array([edges[0]])), E(np.array([edges[-1] - 1e-13])), atol=1e-9)


def test_poisson_periodic_polynomial_exact():
    """A charge density that is a single polynomial of degree k in every cell
    and already neutral: E is exact to rounding (degree k+1 antiderivative),
    checked against the antiderivative written out by hand."""
    from oracle.vp import poisson_periodic_1d
    k = 3
    p = Problem(1, 1, k, [4], [1], [0.0], [4.0], [-1.0], [1.0], ConstantField([1.0, 1.0]))
    # on each unit cell [c, c+1]: rho = (t - 1/2)^3 with t = x - c (zero mean per cell);
    # E = ((t - 1/2)^4 - 1/16) / 4 + const, the const making the mean zero
    xs = np.array([p.node_coordinates(c)[0][:, 0, 0] for c in range(4)])
    t = xs - np.floor(xs)
    rho = (t - 0.5) ** 3
    _, nodal = poisson_periodic_1d(p, rho)
    exact = ((t - 0.5) ** 4 - 1.0 / 16) / 4
    exact -= (1.0 / 80 - 1.0 / 16) / 4        # int_0^1 ((t - 1/2)^4 - 1/16) dt = 1/80 - 1/16
    np.testing.assert_allclose(nodal, exact, atol=1e-14)


def test_vp_uniform_maxwellian_is_stationary():
    """A spatially uniform, neutral Maxwellian has rho = 0 up to its
    quadrature error, hence E = 0 exactly (the mean is removed) and no
    x-gradient: one step leaves it unchanged."""
    from oracle.vp import vp_step
    p = Problem(1, 1, 3, [4], [12], [0.0], [4 * np.pi], [-6.0], [6.0], ConstantField([1.0, 1.0]))
    u = p.interpolate(lambda yx, v: np.exp(-0.5 * v[..., 0] ** 2) / np.sqrt(2 * np.pi))
    u1 = vp_step(p, u, 0.05)
    np.testing.assert_allclose(u1, u, atol=1e-14)


def test_vp_field_uses_minus_e_and_conserves_mass():
    """With a density bump the field is (v, -E): the operator of vp_rhs equals
    the advection operator with a_v = -E(y) written with the closed-form E of
    the nodal rho; the step conserves mass."""
    from oracle.vp import field_from, poisson_periodic_1d, vp_step
    p = Problem(1, 1, 2, [6], [8], [0.0], [2 * np.pi], [-4.0], [4.0], ConstantField([1.0, 1.0]))
    f = lambda yx, v: (1 + 0.2 * np.cos(yx[..., 0])) * np.exp(-0.5 * v[..., 0] ** 2) / np.sqrt(2 * np.pi)
    u = p.interpolate(f)
    rho = p.charge_density(u)
    E, nodal = poisson_periodic_1d(p, rho)
    fld = field_from(p, u)
    ys = np.linspace(0.0, 2 * np.pi, 7, endpoint=False)[:, None]
    a = fld(ys, np.zeros((7, 1)))
    np.testing.assert_allclose(a[:, 1], -E(ys[:, 0]), atol=0)
    np.testing.assert_allclose(a[:, 0], 0.0, atol=0)
    # rho = 1 - int f dv is close to -0.2 cos(x) (the Maxwellian integrates to ~1)
    xs = np.array([p.node_coordinates(c)[0][:, 0, 0] for c in range(6)])
    np.testing.assert_allclose(rho, -0.2 * np.cos(xs), atol=2e-3)
    np.testing.assert_allclose(nodal, -0.2 * np.sin(xs), atol=5e-3)
    m0 = p.integrals(u)[0]
    u1 = vp_step(p, u, 0.02)
    assert abs(p.integrals(u1)[0] - m0) <= 1e-13 * abs(m0)


# ---------------------------------------------------------------------------
# Gauss-Lobatto collocation (the paper's alternative basis, Sec. 2.5 and 5.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [2.0, -1.5])
def test_gllc_k1_operator_by_hand(a):
    """k = 1, nodes -1, +1, weights 1, 1, speed c = 2a/h along x only.  Worked
    by hand from the weak form: with the upwind neighbour's facing node value
    u_nb, c > 0: K = c (u_nb - (u0+u1)/2, (u0-u1)/2);
    c < 0: K = c ((u0-u1)/2, (u0+u1)/2 - u_nb)."""
    h = 1.0
    p = Problem(1, 1, 1, [3], [1], [0.0], [3.0], [-1.0], [1.0], ConstantField([a, 0.0]),
                basis="gllc")
    u = np.random.default_rng(5).standard_normal(p.n_dofs)
    K = p.apply(u).reshape(3, 2, 2)        # cell, v node, x node
    U = u.reshape(3, 2, 2)
    c = 2 * a / h
    for e in range(3):
        for qv in range(2):
            u0, u1 = U[e, qv]
            if c > 0:
                unb = U[(e - 1) % 3, qv, 1]
                ref = (c * (unb - (u0 + u1) / 2), c * (u0 - u1) / 2)
            else:
                unb = U[(e + 1) % 3, qv, 0]
                ref = (c * (u0 - u1) / 2, c * ((u0 + u1) / 2 - unb))
            np.testing.assert_allclose(K[e, qv], ref, atol=1e-13)


@pytest.mark.parametrize("k", [2, 3])
def test_gllc_convergence_order(k):
    """Gauss-Lobatto collocation transports a product of sines at order k+1."""
    from oracle.quadrature import gauss_lobatto as gl_nodes
    errs = []
    for N in (4, 8, 16):
        w = W.config_2d(cells=N)
        w = W.Workload(**{**w.__dict__, "k": k, "final_time": 0.25})
        p = _problem(w, basis="gllc")
        zeta = gl_nodes(w.n)[0]
        u0 = W.separable_state(w, zeta)
        dt, steps = W.time_step(w)
        dt, steps = dt / 4, steps * 4
        L = p.assemble()
        u = u0.copy()
        for _ in range(steps):
            u = lsrk.step(lambda x: L @ x, u, dt)
        T = dt * steps
        shifted = W.Workload(**{**w.__dict__, "u0_factors": (
            lambda y: np.sin(2 * np.pi * (y - w.a_const[0] * T)),
            lambda y: np.sin(2 * np.pi * (y - w.a_const[1] * T)))})
        diff = u - W.separable_state(shifted, zeta)
        errs.append(math.sqrt(diff @ (p.mass_diagonal() * diff)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k + 1 - 0.3, rates


# ---------------------------------------------------------------------------
# curved (non-affine) x-mesh: a Jacobian per quadrature point (Sec. 5.1)
# ---------------------------------------------------------------------------
def test_curved_zero_deformation_is_the_affine_operator():
    f = ConstantField([0.7, -0.4, 0.3, 0.5])
    pa = Problem(2, 2, 2, [2, 3], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], f)
    pc = Problem(2, 2, 2, [2, 3], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], f, deform=[0.0, 0.0])
    u = np.random.default_rng(0).standard_normal(pa.n_dofs)
    np.testing.assert_allclose(pc.apply(u), pa.apply(u), rtol=0, atol=1e-13 * np.abs(pa.apply(u)).max())


@pytest.mark.parametrize("dx,dv", [(1, 1), (2, 1), (1, 2)])
def test_curved_conserves_mass(dx, dv):
    """The face geometry is evaluated at the same physical point from both
    sides, so the upwind flux is single-valued and mass is conserved exactly."""
    rng = np.random.default_rng(dx + 2 * dv)
    a = rng.uniform(-1, 1, dx + dv)
    p = Problem(dx, dv, 2, [3] * dx, [2] * dv, [0] * dx, [1] * dx, [-1] * dv, [1] * dv,
                ConstantField(a), deform=rng.uniform(-0.3, 0.3, dx))
    u = rng.standard_normal(p.n_dofs)
    Md = p.mass_diagonal()
    Lu = p.apply(u)
    assert abs(Md @ Lu) <= 1e-13 * (np.abs(Md) @ np.abs(Lu))


def test_curved_translation_order():
    """A product of sines in PHYSICAL coordinates translated by a constant
    velocity on a strongly deformed 1x1v mesh (delta = 0.3): the L2 error at
    T = 1/4 against the exact translate falls at order k+1."""
    a = np.array([1.0, 0.5])
    k = 2

    def f(x, v):
        return np.sin(2 * np.pi * x) * np.sin(2 * np.pi * v)

    errs = []
    for N in (4, 8, 16):
        p = Problem(1, 1, k, [N], [N], [0.0], [1.0], [0.0], [1.0], ConstantField(a), deform=[0.3])
        X = lambda yx: p.physical_x(yx)[..., 0]
        u = p.interpolate(lambda yx, v: f(X(yx), v[..., 0]))
        T = 0.25
        steps = int(math.ceil(T / (0.2 * 1.0 / (a[0] * N * 1.5 + a[1] * N))))
        dt = T / steps
        L = p.assemble()
        for _ in range(steps):
            u = lsrk.step(lambda x: L @ x, u, dt)
        ex = p.interpolate(lambda yx, v: f(X(yx) - a[0] * T, v[..., 0] - a[1] * T))
        diff = u - ex
        errs.append(math.sqrt(diff @ (p.mass_diagonal() * diff)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k + 1 - 0.3, rates


def test_curved_consistency_two_x_directions():
    """L u against -a . grad u (physical gradient) for a smooth u on a 2x1v
    mesh whose x directions are coupled by the deformation (off-diagonal,
    point-dependent J_x): the error falls at order >= k - 1/2."""
    a = np.array([0.7, -0.4, 0.3])
    tp = 2 * np.pi
    k = 2

    def parts(x1, x2, v):
        s1, c1, s2, c2, sv, cv = (np.sin(tp * x1), np.cos(tp * x1), np.sin(tp * x2),
                                  np.cos(tp * x2), np.sin(tp * v), np.cos(tp * v))
        return s1 * c2 * sv, -tp * (a[0] * c1 * c2 * sv - a[1] * s1 * s2 * sv + a[2] * s1 * c2 * cv)

    errs = []
    for N in (3, 6, 12):
        p = Problem(2, 1, k, [N, N], [N], [0, 0], [1, 1], [0], [1], ConstantField(a),
                    deform=[0.25, -0.2])

        def ev(i):
            return lambda yx, v: parts(*np.moveaxis(p.physical_x(yx), -1, 0), v[..., 0])[i]

        diff = p.apply(p.interpolate(ev(0))) - p.interpolate(ev(1))
        errs.append(math.sqrt(diff @ (p.mass_diagonal() * diff)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] > k - 0.5, rates


# ---------------------------------------------------------------------------
# the term scale |L| |u| (``Problem.apply_abs``): the yardstick of every
# reduced-precision parity test.  The weak form (Sec. 1.3, Eq. into:adv:ref)
# evaluated with the absolute value of every factor and term.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a", [(1.0, 0.5), (-0.7, 0.3), (0.4, -1.2)])
def test_term_scale_k0_closed_form(a):
    """k = 0 (first-order upwind finite volumes): the operator is
    -a_j (u_i - u_up) / h_j per direction, whose terms in absolute value are
    |a_j| (|u_i| + |u_up|) / h_j -- no volume term (the derivative of a
    constant is zero), the outflow trace and the upwind neighbour's trace."""
    nx, nv = 5, 4
    p = Problem(1, 1, 0, (nx,), (nv,), (0,), (2,), (0,), (1,), ConstantField(a))
    U = np.random.default_rng(13).standard_normal(p.n_dofs).reshape(nv, nx)
    h = (2.0 / nx, 1.0 / nv)
    ref = np.zeros_like(U)
    for axis, aj, hj in ((1, a[0], h[0]), (0, a[1], h[1])):
        up = np.roll(U, 1 if aj > 0 else -1, axis=axis)
        ref += abs(aj) / hj * (np.abs(U) + np.abs(up))
    got = p.apply_abs(U.reshape(-1))
    np.testing.assert_allclose(got, ref.reshape(-1), rtol=1e-14, atol=0)


def _lagrange_1d_by_fit(nodes, x):
    """Values and derivatives at x of the Lagrange polynomials through
    ``nodes``, by monomial fits of the unit vectors (independent of the
    oracle's product formulas)."""
    n = len(nodes)
    V = np.zeros((len(x), n))
    D = np.zeros((len(x), n))
    for p_ in range(n):
        c = P.polyfit(nodes, np.eye(n)[p_], n - 1)
        V[:, p_] = P.polyval(x, c)
        D[:, p_] = P.polyval(x, P.polyder(c))
    return V, D


def _rule_independent(n, basis):
    """The n-point Gauss-Legendre ("gl") or Gauss-Lobatto ("gllc") rule from
    scipy's Golub-Welsch roots (the Lobatto interior points are the
    Gauss-Jacobi(1, 1) points) with weights from the moment equations, not
    from the oracle's quadrature module."""
    from scipy.special import roots_jacobi, roots_legendre
    if basis == "gl":
        x, w = roots_legendre(n)
        return np.asarray(x), np.asarray(w)
    x = np.concatenate([[-1.0], roots_jacobi(n - 2, 1.0, 1.0)[0] if n > 2 else [], [1.0]])
    V = np.vander(x, n, increasing=True).T            # V[m, i] = x_i^m
    mom = np.array([(1 - (-1) ** (m + 1)) / (m + 1) for m in range(n)])
    return x, np.linalg.solve(V, mom)


def _term_scale_dense(p, u):
    """|M^{-1}| sum over terms |T_t| |u| with every term of the weak form as a
    dense Kronecker matrix (cell terms per direction, outflow-face terms and
    upwind-neighbour face terms per face), built from independently fitted
    1D tables.  Collocation bases only (M diagonal)."""
    d, n = p.d, p.n
    zeta, wq = _rule_independent(n, p.basis)
    B, Bd = _lagrange_1d_by_fit(zeta, zeta)
    lp, _ = _lagrange_1d_by_fit(zeta, np.array([1.0]))
    lm, _ = _lagrange_1d_by_fit(zeta, np.array([-1.0]))

    def kron(mats):
        K = np.ones((1, 1))
        for M in mats:
            K = np.kron(M, K)
        return K

    def weights(ws):
        return kron([np.asarray(w_)[:, None] for w_ in ws])[:, 0]

    npc = n ** d
    out = np.zeros(p.n_dofs)
    aB, aBd = np.abs(B), np.abs(Bd)
    for e in range(p.ncells):
        cc = (e // p.strides) % p.cells
        # physical points of the cell: speeds c = J^{-1} a from the field
        def speeds(pts):
            axes = [p.lo[j] + p.h[j] * (cc[j] + (np.asarray(pts[j]) + 1) / 2) for j in range(d)]
            Y = np.stack(np.meshgrid(*axes, indexing="ij"), -1)
            a = p.field(Y[..., :p.dx], Y[..., p.dx:])
            return (a @ np.linalg.inv(p.J).T).reshape(-1, d, order="F")
        detJ = abs(np.linalg.det(p.J))
        ue = np.abs(u[e * npc:(e + 1) * npc])
        acc = np.zeros(npc)
        Wc = weights([wq] * d)
        C = speeds([zeta] * d)
        for j in range(d):
            Kd = kron([aBd if m == j else aB for m in range(d)])
            acc += Kd.T @ (Wc * detJ * np.abs(C[:, j]) * (kron([aB] * d) @ ue))
        for j in range(d):
            for s in (1, -1):
                ls, lo = (lp, lm) if s > 0 else (lm, lp)
                pts = [zeta] * d
                pts[j] = np.array([float(s)])
                cj = speeds(pts)[:, j]
                wf = weights([np.ones(1) if m == j else wq for m in range(d)])
                Ts = kron([np.abs(ls) if m == j else aB for m in range(d)])
                To = kron([np.abs(lo) if m == j else aB for m in range(d)])
                nb = (e + 0)
                cn = cc.copy()
                cn[j] = (cn[j] + s) % p.cells[j]
                nb = int(np.sum(cn * p.strides))
                un = np.abs(u[nb * npc:(nb + 1) * npc])
                own = (s * cj > 0)
                acc += Ts.T @ (wf * detJ * np.abs(cj) * np.where(own, Ts @ ue, To @ un))
        out[e * npc:(e + 1) * npc] = acc / (Wc * detJ)
    return out


def _term_scale_problems():
    rng = np.random.default_rng(21)
    out = []
    for dx, dv, k, cells, kind, basis in [
            (1, 1, 3, (3, 2), "const", "gl"), (1, 1, 2, (2, 3), "phase", "gllc"),
            (2, 1, 2, (2, 1, 3), "const", "gl"), (1, 2, 1, (2, 2, 1), "phase", "gl"),
            (2, 2, 1, (2, 1, 2, 1), "phase", "gl"), (1, 2, 3, (1, 2, 2), "phase", "gllc")]:
        d = dx + dv
        if kind == "const":
            field = ConstantField(rng.uniform(-1, 1, d))
        else:
            amp = rng.uniform(0.3, 1, dv)
            field = PhaseSpaceField(dx, dv, lambda y, amp=amp: amp * np.sin(
                2 * np.pi * y.sum(-1, keepdims=True) + 0.3))
        shear = None if dx == 1 else np.eye(dx) + 0.1 * np.eye(dx, k=1)
        out.append(Problem(dx, dv, k, cells[:dx], cells[dx:], [0] * dx, [1] * dx, [-1] * dv,
                           [1.5] * dv, field, shear=shear, basis=basis))
    return out


@pytest.mark.parametrize("p", _term_scale_problems(), ids=lambda p: f"{p.dx}x{p.dv}v_k{p.k}_{p.basis}")
def test_term_scale_equals_termwise_dense_route(p):
    """apply_abs (axis-wise sums) equals the same terms as dense Kronecker
    matrices from independently fitted 1D tables: a term dropped, counted
    twice, or taken from the wrong side fails."""
    u = np.random.default_rng(22).standard_normal(p.n_dofs)
    got = p.apply_abs(u)
    ref = _term_scale_dense(p, u)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("p", _term_scale_problems(), ids=lambda p: f"{p.dx}x{p.dv}v_k{p.k}_{p.basis}")
def test_term_scale_bounds_the_assembled_operator(p):
    """|L| |u| <= apply_abs(u) row by row (the triangle inequality over the
    terms that the assembled entries of L sum), and the bound is not loose by
    more than the cancellation inside the collocated 1D operators: every row
    sum of the scale stays within a factor 4 of |L| |u|."""
    L = p.assemble()
    u = np.random.default_rng(23).standard_normal(p.n_dofs)
    lo = abs(L) @ np.abs(u)
    hi = p.apply_abs(u)
    assert np.all(lo <= hi * (1 + 1e-12))
    assert np.all(hi <= 4 * lo)


# ---------------------------------------------------------------------------
# integrals with the cell quadrature (``Problem.integrals``; Sec. 2.5, the
# tensor-product rules, and Sec. 1.3, the |J| of the reference map)
# ---------------------------------------------------------------------------
def _poly_integral(coef, lo, hi):
    ci = P.polyint(coef)
    return P.polyval(hi, ci) - P.polyval(lo, ci)


@pytest.mark.parametrize("basis", ["gl", "gll", "gllc"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_integrals_of_polynomials_exact(basis, k):
    """u = prod_j p_j(y_j), each p_j of degree k (gllc: k - 1 for the square)
    on a sheared 2x + 1v box.  The nodal interpolant is u itself, and the
    rule integrates degree 2k+1 (Gauss) or 2k-1 (Lobatto) exactly, so
    int u = det(S) prod_j int p_j and int u^2 = det(S) prod_j int p_j^2 to
    round-off; max |u| is the largest nodal value."""
    rng = np.random.default_rng(31 + k)
    dx, dv = 2, 1
    S = np.array([[1.0, 0.1], [0.0, 1.0]]) * np.array([[1.0], [1.3]])   # det = 1.3
    lo, hi = np.array([0.0, 0.5, -1.0]), np.array([1.0, 2.0, 1.5])
    p = Problem(dx, dv, k, (3, 2), (2,), lo[:2], hi[:2], lo[2:], hi[2:],
                ConstantField([1.0, 1.0, 1.0]), shear=S, basis=basis)
    for deg, check_sq in ((k, basis != "gllc"), (k - 1, True)):
        coefs = [rng.standard_normal(deg + 1) for _ in range(3)]

        def f(yx, v):
            return (P.polyval(yx[..., 0], coefs[0]) * P.polyval(yx[..., 1], coefs[1])
                    * P.polyval(v[..., 0], coefs[2]))
        u = p.interpolate(f)
        mass, l2, umax = p.integrals(u)
        ex_mass = np.linalg.det(S) * np.prod([_poly_integral(c, a, b)
                                              for c, a, b in zip(coefs, lo, hi)])
        assert abs(mass - ex_mass) <= 1e-12 * max(1.0, abs(ex_mass))
        if check_sq:
            ex_l2 = np.linalg.det(S) * np.prod([_poly_integral(P.polymul(c, c), a, b)
                                                for c, a, b in zip(coefs, lo, hi)])
            assert abs(l2 - ex_l2) <= 1e-12 * ex_l2
        assert umax == np.max(np.abs(u))


def test_integrals_of_squared_sines_exact():
    """sin^2(2 pi y1) sin^2(2 pi y2) sin^2(2 pi v) = (1 - cos 4 pi y)/2 per
    factor: on N >= 3 cells per period the composite Gauss rule sums each
    cosine to zero (roots of unity), so int u^2 over the sheared box is
    det(S) |box| / 8 and int u = 0 exactly.  A missing |J| factor, a wrong
    weight or the wrong cell size fails."""
    S = np.array([[1.0, 0.2], [0.0, 0.8]])
    p = Problem(2, 1, 3, (3, 4), (5,), (0.0, 0.0), (1.0, 1.0), (-1.0,), (1.0,),
                ConstantField([1.0, 1.0, 1.0]), shear=S)
    u = p.interpolate(lambda yx, v: np.sin(2 * np.pi * yx[..., 0]) * np.sin(2 * np.pi * yx[..., 1])
                      * np.sin(2 * np.pi * v[..., 0]))
    mass, l2, _ = p.integrals(u)
    vol = np.linalg.det(S) * 1.0 * 1.0 * 2.0
    assert abs(mass) <= 1e-14
    assert abs(l2 - vol / 8) <= 1e-13


@pytest.mark.parametrize("basis", ["gl", "gllc"])
def test_integrals_curved_mesh_volume(basis):
    """The periodic deformation maps the lattice onto itself, so the physical
    volume is the lattice volume: int 1 = |box| and int p(v) = |box_x| int p
    exactly (the cos(2 pi y) term of |J_x| sums to zero over N >= 2 cells).
    A missing per-point |J_x| (or one taken at the wrong point) fails."""
    rng = np.random.default_rng(41)
    p = Problem(2, 1, 2, (3, 2), (2,), (0.0, 0.0), (1.0, 2.0), (-1.0,), (1.0,),
                ConstantField([1.0, 1.0, 1.0]), basis=basis, deform=[0.3, -0.25])
    c = rng.standard_normal(2)                  # degree 1 in v: exact in both rules
    mass1, _, _ = p.integrals(np.ones(p.n_dofs))
    assert abs(mass1 - 2.0 * 2.0) <= 1e-13
    u = p.interpolate(lambda yx, v: P.polyval(v[..., 0], c) + 0 * yx[..., 0])
    mass, _, _ = p.integrals(u)
    assert abs(mass - 2.0 * _poly_integral(c, -1.0, 1.0)) <= 1e-13
    # and the |J_x| really varies on this mesh (the pin would be vacuous otherwise)
    _, dj = p.jacobian(0, [p.T.zeta] * 3)
    assert np.ptp(dj) > 0.1 * np.mean(dj)


@pytest.mark.parametrize("mistake", ["no_volume", "no_faces", "own_trace_on_inflow",
                                     "no_jacobian", "unit_weights"])
def test_term_scale_and_integral_pins_catch_planted_mistakes(mistake, monkeypatch):
    """Each mistake planted in the oracle (on the CPU) fails at least one of
    the pins above: the term scale against the dense route and the bounds,
    or the integrals against the closed forms."""
    p = _term_scale_problems()[2]
    u = np.random.default_rng(24).standard_normal(p.n_dofs)
    dense = _term_scale_dense(p, u)
    lo = abs(p.assemble()) @ np.abs(u)
    q = Problem(1, 1, 3, (3,), (2,), (0.0,), (1.0,), (-1.0,), (1.0,), ConstantField([1.0, 1.0]))
    cx, cv = np.array([0.3, -1.0, 0.5, 0.2]), np.array([1.0, 0.4, -0.7, 0.1])
    uq = q.interpolate(lambda yx, v: P.polyval(yx[..., 0], cx) * P.polyval(v[..., 0], cv))
    ex = _poly_integral(cx, 0.0, 1.0) * _poly_integral(cv, -1.0, 1.0)
    if mistake == "no_volume":
        monkeypatch.setattr(p.T, "Bd", np.zeros_like(p.T.Bd))
    elif mistake == "no_faces":
        monkeypatch.setattr(p, "_face_trace_abs", lambda U, j, l: np.zeros_like(
            np.take(U, [0], axis=j)))
    elif mistake == "own_trace_on_inflow":
        monkeypatch.setattr(p, "neighbour", lambda cell, j, s: cell)
    elif mistake == "no_jacobian":
        monkeypatch.setattr(p, "_detJ", lambda cell, pts: 1.0)
        monkeypatch.setattr(q, "_detJ", lambda cell, pts: 1.0)
    else:
        monkeypatch.setattr(p.T, "w", np.ones_like(p.T.w))
        monkeypatch.setattr(q.T, "w", np.ones_like(q.T.w))
    hi = p.apply_abs(u)
    scale_ok = (np.allclose(hi, dense, rtol=1e-12, atol=0) and np.all(lo <= hi * (1 + 1e-12))
                and np.all(hi <= 4 * lo))
    integral_ok = abs(q.integrals(uq)[0] - ex) <= 1e-12
    assert not (scale_ok and integral_ok), mistake
