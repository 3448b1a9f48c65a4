"""The Gauss-Lobatto bases on the GPU against the oracle: the collocation
variant (DG_BASIS_GLL, oracle basis "gllc") in the generic and the 6D
kernels, and the paper's default element (DG_BASIS_GLL_GAUSS, oracle basis
"gll": Lobatto nodes, Gauss quadrature) through the library's change of basis.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsrk  # noqa: E402
from oracle import vp as ovp  # noqa: E402
from oracle.dg import ConstantField, PhaseSpaceField, Problem  # noqa: E402
from dg_helpers import assert_term_scale  # noqa: E402

pytestmark = pytest.mark.gpu

ORACLE_BASIS = {1: "gllc", 2: "gll"}
TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _field_table(p, E):
    """E at the x quadrature points (where the library samples the field), in
    the library's layout (x cell, point, component), from the oracle's own
    point coordinates."""
    dx, dv, n = p.dx, p.dv, p.n
    ncx = int(np.prod(p.cells[:dx]))
    tab = np.zeros((ncx, n ** dx, dv))
    for e in range(ncx):
        yx, _ = p.coordinates(e, [p.T.zeta] * p.d)
        sub = yx[tuple([slice(None)] * dx + [0] * dv)]
        tab[e] = E(sub.reshape(-1, dx, order="F"))
    return tab


def _pair(basis, dx, dv, k, cells, kind, seed=0):
    from paper_2002_08110_gb300 import DG
    rng = np.random.default_rng(seed)
    d = dx + dv
    x_lo, x_hi = [0.0] * dx, [1.0] * dx
    v_lo, v_hi = [-1.0] * dv, [1.5] * dv
    kw = dict(dim_x=dx, dim_v=dv, degree=k, cells_x=cells[:dx], cells_v=cells[dx:], x_lo=x_lo,
              x_hi=x_hi, v_lo=v_lo, v_hi=v_hi, basis=basis)
    if kind == "const":
        a = rng.uniform(-1, 1, d)
        field = ConstantField(a)
        dg = DG(field_kind=0, a_const=a, **kw)
    else:
        amp, ph = rng.uniform(0.3, 1.0, dv), rng.uniform(0, 1, dv)

        def E(yx):
            s = np.asarray(yx).sum(-1, keepdims=True)
            return amp * np.sin(2 * np.pi * (s + ph))

        field = PhaseSpaceField(dx, dv, E)
        p0 = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, field,
                     basis=ORACLE_BASIS[basis])
        dg = DG(field_kind=1, e_nodes=_field_table(p0, E), **kw)
    p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, field,
                basis=ORACLE_BASIS[basis])
    return dg, p


CASES = [(1, 1, 1, (5, 3)), (1, 1, 3, (4, 3)), (1, 2, 2, (2, 3, 2)), (2, 2, 3, (2, 1, 2, 3)),
         (2, 3, 2, (1, 2, 2, 1, 2)), (3, 3, 1, (2, 1, 2, 1, 2, 2)), (3, 3, 3, (1, 2, 1, 2, 1, 2))]


@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
def test_gll_collocation_apply(case, kind):
    dx, dv, k, cells = case
    if kind == "phase" and dv < dx:
        pytest.skip("phase-space field needs dim_v >= dim_x")
    dg, p = _pair(1, dx, dv, k, cells, kind, seed=k + 3 * dx)
    assert dg.info.basis == 1
    u = np.random.default_rng(4).standard_normal(p.n_dofs)
    ref = p.apply(u)
    out = dg.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.linalg.norm(out - ref) <= TOL64 * np.linalg.norm(ref)
    assert_term_scale(out, ref, p.apply_abs(u), TOL64, what="gllc fp64")
    u32 = torch.tensor(u, device="cuda", dtype=torch.float32)
    uin = u32.double().cpu().numpy()
    out32 = dg.apply(u32, prec=1).double().cpu().numpy()
    assert_term_scale(out32, p.apply(uin), p.apply_abs(uin), TOL32, what="gllc fp32")
    dg.check()
    dg.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_gll_collocation_6d_kernels(prec):
    """The 6D, k = 3 kernels (64 and 128 threads per cell) with the Lobatto
    tables agree with the generic kernel and the oracle."""
    dg, p = _pair(1, 3, 3, 3, (2, 3, 1, 2, 1, 3), "const", seed=7)
    assert dg.info.uniform_sides == 1
    u = np.random.default_rng(8).standard_normal(p.n_dofs)
    dt = torch.float32 if prec == 1 else torch.float64
    ut = torch.tensor(u, device="cuda", dtype=dt)
    uin = ut.double().cpu().numpy()
    ref = p.apply(uin)
    scale = p.apply_abs(uin)
    for variant in (0, 1, 2):
        dg.set_launch(prec, threads=256, cells_per_block=1, variant=variant)
        out = dg.apply(ut, prec=prec).double().cpu().numpy()
        assert_term_scale(out, ref, scale, TOL32, what=f"variant {variant}")
    dg.check()
    dg.close()


def test_gll_collocation_6d_adjoint():
    """The transposed operator of the 6D kernels in the Lobatto collocation
    (face-layer loads for the v neighbours) agrees with the generic kernel."""
    dg, p = _pair(1, 3, 3, 3, (2, 1, 2, 3, 2, 2), "const", seed=11)
    assert dg.info.uniform_sides == 1
    y = torch.tensor(np.random.default_rng(9).standard_normal(p.n_dofs), device="cuda",
                     dtype=torch.float32)
    outs = []
    for variant in (0, 2):
        dg.set_launch(1, threads=256, cells_per_block=1, variant=variant)
        outs.append(dg.apply_adjoint(y, prec=1).double().cpu().numpy())
    dg.check()
    # term scale of L^T = M L(-a) M^{-1}: M |L(-a)| M^{-1} |y|
    Md = p.mass_diagonal()
    yy = np.abs(y.double().cpu().numpy())
    scale = Md * p.with_field(p.field.negated()).apply_abs(yy / Md)
    ref = Md * p.with_field(p.field.negated()).apply(y.double().cpu().numpy() / Md)
    for v, o in enumerate(outs):
        assert_term_scale(o, ref, scale, TOL32, what=f"adjoint variant {v}")
    dg.close()


def test_gll_collocation_rk_steps():
    dg, p = _pair(1, 2, 2, 2, (3, 2, 2, 3), "phase", seed=2)
    u0 = np.random.default_rng(1).standard_normal(p.n_dofs)
    dt = 0.01
    ref = u0.copy()
    for _ in range(3):
        ref = lsrk.step(p.apply, ref, dt)
    u = torch.tensor(u0, device="cuda")
    dg.rk_step(u, dt, nsteps=3)
    dg.check()
    assert np.linalg.norm(u.cpu().numpy() - ref) <= TOL64 * np.linalg.norm(ref - u0) + 1e-14 * np.linalg.norm(u0)
    dg.close()


@pytest.mark.parametrize("case", [(1, 1, 3, (4, 3)), (2, 2, 2, (2, 3, 2, 2)), (3, 3, 3, (1, 2, 1, 2, 1, 2))],
                         ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("kind", ["const", "phase"])
def test_gll_gauss_apply_and_adjoint(case, kind):
    """The paper's default element: V^{-1} L_GL V on the GPU against the
    oracle's Lobatto-node, Gauss-quadrature operator; the adjoint by the
    dot-product identity."""
    dx, dv, k, cells = case
    dg, p = _pair(2, dx, dv, k, cells, kind, seed=5 + k)
    assert dg.info.basis == 2
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal(p.n_dofs), rng.standard_normal(p.n_dofs)
    ref = p.apply(x)
    Lx = dg.apply(torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.linalg.norm(Lx - ref) <= TOL64 * np.linalg.norm(ref)
    LTy = dg.apply_adjoint(torch.tensor(y, device="cuda")).cpu().numpy()
    lhs, rhs = y @ Lx, LTy @ x
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(y) @ np.abs(Lx) + np.abs(LTy) @ np.abs(x))
    dg.check()
    dg.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_gll_gauss_stage_and_steps(prec):
    dg, p = _pair(2, 2, 2, 3, (2, 2, 3, 2), "phase", seed=3)
    rng = np.random.default_rng(2)
    w, u = rng.standard_normal(p.n_dofs), rng.standard_normal(p.n_dofs)
    dt, stage = 0.01, 2
    wdt = torch.float64 if prec == 0 else torch.float32
    wt = torch.tensor(w, device="cuda", dtype=wdt)
    ut = torch.tensor(u, device="cuda")
    wo = torch.empty_like(wt)
    dg.rk_stage(wt, wo, ut, stage, dt, prec=prec)
    dg.check()
    K = p.apply(wt.double().cpu().numpy())
    u_ref = u + lsrk.B[stage] * dt * K
    w_ref = u + lsrk.A[stage] * dt * K
    tol = TOL64 if prec == 0 else 3e-6
    assert np.linalg.norm(ut.cpu().numpy() - u_ref) <= tol * np.linalg.norm(u_ref)
    assert np.linalg.norm(wo.double().cpu().numpy() - w_ref) <= tol * np.linalg.norm(w_ref)
    if prec == 0:
        ref = u.copy()
        for _ in range(2):
            ref = lsrk.step(p.apply, ref, dt)
        x = torch.tensor(u, device="cuda")
        dg.rk_step(x, dt, nsteps=2)
        dg.check()
        assert np.linalg.norm(x.cpu().numpy() - ref) <= TOL64 * np.linalg.norm(ref)
        m, l2, _ = dg.integrals(torch.tensor(u, device="cuda"))
        mo, lo, _ = p.integrals(u)
        assert abs(m - mo) <= 1e-12 * np.sum(np.abs(u)) * p.detJ * 2 ** p.d
        assert abs(l2 - lo) <= 1e-12 * abs(lo)
    dg.close()


def test_gll_gauss_refuses_vlasov_poisson():
    from paper_2002_08110_gb300 import DGError
    dg, _ = _pair(2, 1, 1, 2, (3, 4), "phase", seed=1)
    f = torch.zeros(dg.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(DGError):
        dg.charge_density(f)
    dg.close()


def test_gll_collocation_vlasov_poisson_pieces():
    """rho and E with the Lobatto nodes and weights (1D1V) against the oracle."""
    dg, p = _pair(1, 1, 1, 3, (6, 5), "phase", seed=9)
    u = np.random.default_rng(3).standard_normal(p.n_dofs) * 0.1 + 1.0
    rho = dg.charge_density(torch.tensor(u, device="cuda"))
    ref = p.charge_density(u).reshape(-1)
    assert np.max(np.abs(rho.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref) + 1)
    e = dg.poisson_periodic_1d(torch.tensor(ref, device="cuda"))
    _, eref = ovp.poisson_periodic_1d(p, ref.reshape(6, 4))
    assert np.max(np.abs(e.cpu().numpy() - eref.reshape(-1))) <= 1e-13 * (np.max(np.abs(eref)) + 1)
    dg.close()


def test_gll_6d_workload_keeps_the_specialised_kernel():
    """The 6D workload in the Lobatto collocation has field zeros on face
    nodes (v = 0, and E = 0.05 sin 2 pi x at x = 1/2 up to rounding, a tiny
    speed of either sign).  Such speeds carry no flux at FP32 precision; they
    take the cell's side, the specialised kernel still runs, and the result
    matches the oracle."""
    import workloads as W
    from paper_2002_08110_gb300 import DG, basis_nodes
    w = W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, 2))
    nodes, qpts, _ = basis_nodes(1, w.k)
    dg = DG(e_nodes=W.e_table(w, qpts), basis=1, **W.dg_kwargs(w))
    assert dg.info.uniform_sides == 1
    p = Problem(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                PhaseSpaceField(w.dx, w.dv, W.e_function(w)), basis="gllc")
    u = W.separable_state(w, nodes, xp=torch, device="cuda").float()
    uin = u.double().cpu().numpy()
    ref = p.apply(uin)
    scale = p.apply_abs(uin)
    # speeds below 1e-12 of a cell's largest carry no flux in the FP32 tables:
    # entries whose every term comes from such speeds (v = 0 and x at a zero
    # of E) are exact only to that level, an absolute floor far below FP32
    floor = 1e-12 * np.max(np.abs(scale))
    for variant in (0, 2):
        dg.set_launch(1, threads=256, cells_per_block=1, variant=variant)
        out = dg.apply(u, prec=1).double().cpu().numpy()
        assert_term_scale(out, ref, scale, TOL32, floor=floor, what=f"6d gllc variant {variant}")
    dg.check()
    dg.close()
