"""GPU parity of the operator application against the FP64 oracle.

Every (d, k) the library supports, every precision, the adjoint, with
ragged meshes that span several blocks and include directions with one and
two cells (the periodic neighbour is the cell itself or the same cell on
both sides).  Tolerances (stated per apply), element by element against the
term scale S = |L| |u| (the oracle's evaluation with the absolute value of
every factor; rounding errors of an entry scale with the terms it sums):
  FP64:             |K_i - K_ref,i| <= 1e-12 S_i, and ||K - K_ref|| <= 1e-12 ||K_ref||
  FP32 / mixed:     |K_i - K_ref,i| <= 1e-5 S_i
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from dg_helpers import assert_term_scale, random_problem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


CASES = [
    # (dx, dv, k, cells)
    (1, 1, 1, (13, 11)), (1, 1, 3, (16, 9)), (1, 1, 5, (7, 2)),
    (2, 1, 2, (5, 3, 4)), (1, 2, 4, (3, 1, 5)), (2, 1, 5, (2, 3, 2)),
    (2, 2, 1, (3, 4, 2, 3)), (2, 2, 3, (3, 2, 1, 3)), (2, 2, 5, (2, 1, 2, 1)),
    (2, 3, 2, (2, 3, 1, 2, 2)), (3, 2, 3, (2, 1, 2, 2, 1)), (2, 3, 5, (1, 2, 1, 1, 2)),
    (3, 3, 1, (2, 3, 2, 2, 1, 2)), (3, 3, 2, (2, 1, 2, 1, 2, 1)), (3, 3, 3, (2, 2, 1, 1, 2, 3)),
    (3, 3, 4, (1, 2, 1, 1, 1, 2)), (3, 3, 5, (1, 1, 2, 1, 2, 1)),
]


def _run(dg, p, prec, adjoint, seed=1):
    from paper_2002_08110_gb300 import PREC_FP32
    u = np.random.default_rng(seed).standard_normal(p.n_dofs)
    dt = torch.float32 if prec == PREC_FP32 else torch.float64
    ut = torch.tensor(u, device="cuda", dtype=dt)
    uin = ut.double().cpu().numpy()
    out = (dg.apply_adjoint(ut, prec=prec) if adjoint else dg.apply(ut, prec=prec))
    dg.check()
    return uin, out.double().cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_parity(case, kind, prec):
    dx, dv, k, cells = case
    if kind == "phase" and dv < dx:
        pytest.skip("phase-space field needs dv >= dx")
    shear = None if dx == 1 else np.eye(dx) + 0.1 * np.eye(dx, k=1)
    dg, p = random_problem(dx, dv, k, cells, kind, shear=shear)
    u, out = _run(dg, p, prec, adjoint=False)
    ref = p.apply(u)
    scale = p.apply_abs(u)
    if prec == 0:
        assert np.linalg.norm(out - ref) <= TOL64 * np.linalg.norm(ref)
        assert_term_scale(out, ref, scale, TOL64, what="fp64 apply")
    else:
        assert_term_scale(out, ref, scale, TOL32, what=f"prec {prec} apply")
    dg.close()


ADJ_CASES = [(1, 1, 3, (5, 4)), (2, 2, 2, (3, 2, 2, 3)), (2, 3, 3, (2, 1, 2, 1, 2)),
             (3, 3, 2, (2, 1, 2, 2, 1, 2)), (3, 3, 1, (2, 2, 1, 1, 2, 2))]


@pytest.mark.parametrize("case", ADJ_CASES, ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_adjoint_parity(case, kind, prec):
    """dg_apply_adjoint == the oracle's transposed operator (dense cell blocks)."""
    dx, dv, k, cells = case
    shear = None if dx == 1 else np.eye(dx) + 0.1 * np.eye(dx, k=1)
    dg, p = random_problem(dx, dv, k, cells, kind, seed=3, shear=shear)
    y, out = _run(dg, p, prec, adjoint=True, seed=4)
    ref = p.apply_adjoint(y)
    # term scale of the transpose: M |L(-a)| M^{-1} |y| (L^T = M L(-a) M^{-1})
    Md = p.mass_diagonal()
    scale = Md * p.with_field(p.field.negated()).apply_abs(np.abs(y) / Md)
    if prec == 0:
        assert np.linalg.norm(out - ref) <= TOL64 * np.linalg.norm(ref)
        assert_term_scale(out, ref, scale, TOL64, what="fp64 adjoint")
    else:
        assert_term_scale(out, ref, scale, TOL32, what=f"prec {prec} adjoint")
    dg.close()


def _dot_identity(dg, p, prec, seed):
    """<y, L x> (oracle) against <L^T y, x> (library): the adjoint is the
    transpose at any size, without assembling L."""
    rng = np.random.default_rng(seed)
    dt = torch.float32 if prec == 1 else torch.float64
    x = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda", dtype=dt)
    y = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda", dtype=dt)
    ltx = dg.apply_adjoint(y, prec=prec).double().cpu().numpy()
    xh, yh = x.double().cpu().numpy(), y.double().cpu().numpy()
    lhs = yh @ p.apply(xh)
    rhs = ltx @ xh
    scale = np.abs(yh) @ p.apply_abs(xh)
    return abs(lhs - rhs), scale


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_adjoint_dot_identity_6d(prec):
    dg, p = random_problem(3, 3, 3, (2, 1, 2, 2, 1, 3), "phase", seed=5)
    err, scale = _dot_identity(dg, p, prec, seed=6)
    assert err <= (1e-12 if prec == 0 else TOL32) * scale
    dg.close()


def _uniform_6d_problems():
    """6D, k = 3 problems in which no speed changes sign inside a cell, so the
    specialised kernel runs: the 6D workload on 2^6 cells (v = 0 and the zeros
    of E lie on cell faces) and a constant field on a ragged mesh."""
    import workloads as W
    from dg_helpers import dg_for
    w = W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, 2))
    yield "6d_config", dg_for(w)
    yield "const_ragged", random_problem(3, 3, 3, (2, 3, 1, 2, 1, 3), "const", seed=7)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("adjoint", [False, True])
def test_specialised_6d_kernel_matches_generic(prec, adjoint):
    """The 6D, k = 3 specialised kernel and the generic kernel agree; both
    match the oracle (forward) or satisfy the transpose identity (adjoint)."""
    for name, (dg, p) in _uniform_6d_problems():
        assert dg.info.uniform_sides == 1, name
        u = np.random.default_rng(8).standard_normal(p.n_dofs)
        dt = torch.float32 if prec == 1 else torch.float64
        ut = torch.tensor(u, device="cuda", dtype=dt)
        uin = ut.double().cpu().numpy()
        outs = []
        for variant in (0, 1, 2):
            dg.set_launch(prec, threads=256, cells_per_block=1, variant=variant)
            f = dg.apply_adjoint if adjoint else dg.apply
            outs.append(f(ut, prec=prec).double().cpu().numpy())
            if adjoint:
                err, scale = _dot_identity(dg, p, prec, seed=10 + variant)
                assert err <= TOL32 * scale, name
        dg.check()
        if adjoint:
            Md = p.mass_diagonal()
            scale = Md * p.with_field(p.field.negated()).apply_abs(np.abs(uin) / Md)
            ref = Md * p.with_field(p.field.negated()).apply(uin / Md)
        else:
            scale = p.apply_abs(uin)
            ref = p.apply(uin)
        for v, o in enumerate(outs):
            assert_term_scale(o, ref, scale, TOL32, what=f"{name} variant {v}")
        dg.close()


def test_sign_change_inside_cells_uses_generic_path():
    """A field whose speeds change sign inside cells is still applied exactly
    (the specialised kernel is bypassed)."""
    dg, p = random_problem(3, 3, 3, (2, 1, 2, 2, 1, 3), "phase", seed=5)
    assert dg.info.uniform_sides == 0
    u = np.random.default_rng(1).standard_normal(p.n_dofs)
    out = dg.apply(torch.tensor(u, device="cuda", dtype=torch.float32), prec=1)
    uin = u.astype(np.float32).astype(np.float64)
    assert_term_scale(out.double().cpu().numpy(), p.apply(uin), p.apply_abs(uin), TOL32,
                      what="sign change inside cells")
    dg.close()


def test_launch_configurations_agree():
    """Every cells-per-block / thread count / sweep order gives the same result."""
    dg, p = random_problem(2, 2, 2, (3, 2, 3, 2), "phase", seed=9)
    u = torch.tensor(np.random.default_rng(1).standard_normal(p.n_dofs), device="cuda")
    ref = dg.apply(u).cpu().numpy()
    for threads in (64, 128, 512):
        for cpb in (1, 3, 8):
            for order in ([0, 1, 2, 3], [3, 2, 1, 0], [2, 0, 3, 1]):
                dg.set_launch(0, threads=threads, cells_per_block=cpb, order=order)
                out = dg.apply(u).cpu().numpy()
                assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))
    best = dg.autotune(u, torch.empty_like(u), 0)
    assert best > 0
    out = dg.apply(u).cpu().numpy()
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))
    dg.close()


@pytest.mark.parametrize("cells", [(2, 2, 2, 2, 2, 2), (1, 3, 1, 2, 1, 1)])
def test_zero_velocity_gives_exact_zero(cells):
    """a = 0 (the degenerate field): the operator is exactly zero in every
    precision and kernel, and a stage leaves the state unchanged."""
    from paper_2002_08110_gb300 import DG
    dg = DG(3, 3, 3, cells[:3], cells[3:], [0] * 3, [1] * 3, [-1] * 3, [1] * 3, field_kind=0,
            a_const=[0.0] * 6)
    u = torch.tensor(np.random.default_rng(2).standard_normal(dg.n_dofs), device="cuda")
    for prec, x in ((0, u), (1, u.float()), (2, u)):
        for variant in (0, 1, 2):
            if prec == 0 and variant:
                continue
            dg.set_launch(prec, threads=256, cells_per_block=1, variant=variant)
            assert torch.count_nonzero(dg.apply(x, prec=prec)) == 0, (prec, variant)
    w_in, w_out, uu = u.float(), torch.empty(dg.n_dofs, dtype=torch.float32, device="cuda"), u.clone()
    dg.rk_stage(w_in, w_out, uu, 1, 0.1, prec=1)
    dg.check()
    assert torch.equal(uu, u)
    dg.close()

