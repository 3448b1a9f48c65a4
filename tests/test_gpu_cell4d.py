"""GPU parity of the specialised 4D kernel (dim_x = dim_v = 2, FP32 sweeps,
n = 2..6; the cell's columns and rows in registers) against the FP64 oracle,
and against the generic kernel on the same inputs.

Meshes span several blocks with a ragged last block and include directions
with one cell (the periodic neighbour is the cell itself).  The phase-space
field changes sign inside cells (the upwind side is chosen per thread) and
the x mesh is sheared.  n = 6 runs the pair-split kernel (two threads per
column and row, 3 cells per block).  Tolerance, element by element:
|K_i - K_ref,i| <= 1e-5 (|L| |u|)_i.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from dg_helpers import assert_term_scale, random_problem  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
# (degree, cells): several blocks of the kernel, a ragged tail, a direction of one cell
CASES = [(1, (5, 3, 4, 3)), (2, (3, 4, 2, 3)), (3, (3, 2, 1, 3)), (3, (4, 4, 3, 5)),
         (4, (2, 3, 1, 2)), (5, (2, 1, 2, 3)), (5, (2, 2, 1, 5))]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _problem(k, cells, kind):
    shear = np.eye(2) + 0.1 * np.eye(2, k=1)
    return random_problem(2, 2, k, cells, kind, seed=20 + k, shear=shear)


def _set_variant(dg, prec, variant):
    c = dg.get_launch(prec)
    dg.set_launch(prec, c["threads"], c["cells_per_block"], c["order"], variant)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"k{c[0]}_{'x'.join(map(str, c[1]))}")
@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("prec", [1, 2])
def test_apply_4d_kernel(case, kind, prec):
    k, cells = case
    dg, p = _problem(k, cells, kind)
    assert dg.get_launch(prec)["variant"] == 2          # the default for 4D
    u = np.random.default_rng(k).standard_normal(p.n_dofs)
    dt = torch.float32 if prec == 1 else torch.float64
    ut = torch.tensor(u, device="cuda", dtype=dt)
    uin = ut.double().cpu().numpy()
    ref = p.apply(uin)
    scale = p.apply_abs(uin)
    outs = []
    for variant in (2, 0):
        _set_variant(dg, prec, variant)
        outs.append(dg.apply(ut, prec=prec).double().cpu().numpy())
    dg.check()
    for v, o in zip((2, 0), outs):
        assert_term_scale(o, ref, scale, TOL32, what=f"variant {v}")
    dg.close()


@pytest.mark.parametrize("case", CASES[1:4] + CASES[6:], ids=lambda c: f"k{c[0]}_{'x'.join(map(str, c[1]))}")
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("stage", [0, 4])
def test_stage_4d_kernel(case, prec, stage):
    """Fused stage: u <- u + b_s dt K (FP64), w_out = u_old + a_s dt K, or u_new
    at the last stage."""
    k, cells = case
    dg, p = _problem(k, cells, "phase")
    rng = np.random.default_rng(30 + k)
    w = rng.standard_normal(p.n_dofs)
    u = rng.standard_normal(p.n_dofs)
    dt = 1e-2
    wdt = torch.float32 if prec == 1 else torch.float64
    wt = torch.tensor(w, device="cuda", dtype=wdt)
    ut = torch.tensor(u, device="cuda", dtype=torch.float64)
    wo = torch.empty_like(wt)
    dg.rk_stage(wt, wo, ut, stage, dt, prec=prec)
    dg.check()
    win = wt.double().cpu().numpy()
    K = p.apply(win)
    scale = np.abs(p.apply_abs(win))
    u_ref = u + lsrk.B[stage] * dt * K
    w_ref = u_ref if stage == 4 else u + lsrk.A[stage] * dt * K
    err_u = np.abs(ut.cpu().numpy() - u_ref)
    err_w = np.abs(wo.double().cpu().numpy() - w_ref)
    # K error (term scale) times dt, plus the rounding of w_out to its type
    bound_u = 1e-14 * np.abs(u_ref) + TOL32 * dt * (scale + np.abs(K))
    assert np.all(err_u <= bound_u + 1e-300)
    if prec == 1:
        a_dtK = np.abs((lsrk.B[4] if stage == 4 else lsrk.A[stage]) * dt * K)
        assert np.all(err_w <= bound_u + 2.5e-7 * (np.abs(u) + a_dtK) + 1e-30)
    else:
        assert np.all(err_w <= bound_u + 1e-14 * np.abs(w_ref))
    dg.close()


def test_4d_kernel_zero_speed_lines():
    """A constant field with a zero component: those lines contribute nothing
    in both kernels (the direction is skipped), and the rest still matches."""
    from paper_2002_08110_gb300 import DG
    from oracle.dg import ConstantField, Problem
    a = np.array([0.7, 0.0, -0.4, 0.0])
    cells = (3, 2, 2, 3)
    args = ([0.0] * 2, [1.0] * 2, [-1.0] * 2, [1.5] * 2)
    p = Problem(2, 2, 3, cells[:2], cells[2:], *args, ConstantField(a))
    dg = DG(2, 2, 3, cells[:2], cells[2:], *args, field_kind=0, a_const=a)
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    out = dg.apply(torch.tensor(u, device="cuda", dtype=torch.float32), prec=1)
    dg.check()
    uin = u.astype(np.float32).astype(np.float64)
    assert_term_scale(out.double().cpu().numpy(), p.apply(uin), p.apply_abs(uin), TOL32,
                      what="zero-speed lines")
    dg.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4], CASES[6]],
                         ids=lambda c: f"k{c[0]}_{'x'.join(map(str, c[1]))}")
@pytest.mark.parametrize("prec", [1, 2])
def test_adjoint_4d_kernel(case, prec):
    """L^T = M L(-a) M^{-1} in the 4D kernel: the transpose identity
    <y, L x> = <L^T y, x> against the oracle's L, and agreement with the
    generic kernel's transpose."""
    k, cells = case
    dg, p = _problem(k, cells, "phase")
    rng = np.random.default_rng(40 + k)
    dt = torch.float32 if prec == 1 else torch.float64
    x = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda", dtype=dt)
    y = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda", dtype=dt)
    xh, yh = x.double().cpu().numpy(), y.double().cpu().numpy()
    outs = []
    for variant in (2, 0):
        _set_variant(dg, prec, variant)
        outs.append(dg.apply_adjoint(y, prec=prec).double().cpu().numpy())
    dg.check()
    lhs = yh @ p.apply(xh)
    scale = np.abs(yh) @ p.apply_abs(xh)
    for o in outs:
        assert abs(lhs - o @ xh) <= TOL32 * scale
    ref = p.apply_adjoint(yh)
    # term scale of L^T = M L(-a) M^{-1}: M |L(-a)| M^{-1} |y|
    Md = p.mass_diagonal()
    tscale = Md * p.with_field(p.field.negated()).apply_abs(np.abs(yh) / Md)
    for v, o in zip((2, 0), outs):
        assert_term_scale(o, ref, tscale, TOL32, what=f"adjoint variant {v}")
    dg.close()
