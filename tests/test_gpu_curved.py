"""Curved (non-affine) x-meshes on the GPU against the oracle: a Jacobian
per quadrature point (Sec. 5.1 deforms the Cartesian mesh), in the generic
kernel, FP64 and FP32 sweeps, operator, LSRK steps and integrals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsrk  # noqa: E402
from oracle.dg import ConstantField, PhaseSpaceField, Problem  # noqa: E402
from dg_helpers import assert_term_scale  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _pair(dx, dv, k, cells, kind, seed=0, basis=0):
    from paper_2002_08110_gb300 import DG
    rng = np.random.default_rng(seed)
    d = dx + dv
    deform = rng.uniform(-0.3, 0.3, dx)
    x_lo, x_hi = [0.0] * dx, [1.0] * dx
    v_lo, v_hi = [-1.0] * dv, [1.5] * dv
    kw = dict(dim_x=dx, dim_v=dv, degree=k, cells_x=cells[:dx], cells_v=cells[dx:], x_lo=x_lo,
              x_hi=x_hi, v_lo=v_lo, v_hi=v_hi, deform=list(deform), basis=basis)
    ob = "gl" if basis == 0 else "gllc"
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
                     deform=deform, basis=ob)
        ncx = int(np.prod(cells[:dx]))
        tab = np.zeros((ncx, (k + 1) ** dx, dv))
        for e in range(ncx):
            yx, _ = p0.node_coordinates(e)
            tab[e] = E(yx[tuple([slice(None)] * dx + [0] * dv)].reshape(-1, dx, order="F"))
        dg = DG(field_kind=1, e_nodes=tab, **kw)
    p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, field, deform=deform,
                basis=ob)
    return dg, p


CASES = [(1, 1, 3, (5, 3)), (1, 2, 2, (3, 2, 2)), (2, 1, 2, (3, 2, 3)), (2, 2, 1, (2, 3, 2, 2)),
         (2, 3, 2, (2, 2, 1, 2, 2)), (3, 3, 1, (2, 1, 2, 1, 2, 2))]


@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
def test_curved_apply(case, kind):
    dx, dv, k, cells = case
    if kind == "phase" and dv < dx:
        pytest.skip("phase-space field needs dim_v >= dim_x")
    dg, p = _pair(dx, dv, k, cells, kind, seed=k + 5 * dx + dv)
    assert dg.info.uniform_sides == 0          # the generic kernel runs
    u = np.random.default_rng(2).standard_normal(p.n_dofs)
    ref = p.apply(u)
    out = dg.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    assert_term_scale(out, ref, p.apply_abs(u), 1e-12, what="curved fp64")
    for prec in (1, 2):
        x = torch.tensor(u, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
        uin = x.double().cpu().numpy()
        o = dg.apply(x, prec=prec).double().cpu().numpy()
        assert_term_scale(o, p.apply(uin), p.apply_abs(uin), 1e-5, what=f"curved prec {prec}")
    dg.check()
    dg.close()


def test_curved_gll_collocation_apply():
    dg, p = _pair(2, 2, 3, (2, 3, 2, 2), "phase", seed=4, basis=1)
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    ref = p.apply(u)
    out = dg.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    assert_term_scale(out, ref, p.apply_abs(u), 1e-12, what="curved gllc fp64")
    dg.close()


def test_curved_steps_integrals_and_coordinates():
    dg, p = _pair(2, 2, 2, (3, 2, 2, 3), "phase", seed=6)
    u0 = np.random.default_rng(5).standard_normal(p.n_dofs)
    dt = 0.005
    ref = u0.copy()
    for _ in range(2):
        ref = lsrk.step(p.apply, ref, dt)
    u = torch.tensor(u0, device="cuda")
    dg.rk_step(u, dt, nsteps=2)
    dg.check()
    assert np.linalg.norm(u.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    m, l2, mx = dg.integrals(torch.tensor(u0, device="cuda"))
    mo, lo, mxo = p.integrals(u0)
    assert abs(m - mo) <= 1e-12 * np.sum(np.abs(u0)) * abs(lo) / max(np.sum(u0 ** 2), 1e-300)
    assert abs(l2 - lo) <= 1e-12 * lo
    # mass is conserved by the steps (single-valued face geometry)
    m1, _, _ = dg.integrals(u)
    assert abs(m1 - m) <= 1e-12 * (abs(m) + lo)
    # physical node coordinates
    X = dg.node_coordinates(4)
    for e in (0, 5):
        yx, _ = p.node_coordinates(e)
        xs = p.physical_x(yx[:, :, 0, 0, :]).reshape(-1, 2, order="F")
        np.testing.assert_allclose(X[e * 9:(e + 1) * 9], xs, atol=1e-14)
    dg.close()


def test_curved_refuses_adjoint_and_poisson():
    from paper_2002_08110_gb300 import DGError
    dg, _ = _pair(1, 1, 2, (4, 3), "phase", seed=1)
    y = torch.zeros(dg.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(DGError):
        dg.apply_adjoint(y)
    with pytest.raises(DGError):
        dg.poisson_periodic_1d(torch.zeros(12, dtype=torch.float64, device="cuda"))
    dg.close()
