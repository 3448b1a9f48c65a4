"""The sum-factorised FP64 OpenMP CPU evaluation (``oracle/cpu_sumfac.cpp``)
against the oracle's axis-wise and dense Kronecker routes on small meshes:
the same operator to round-off (1e-13 of the term scale, element by
element), in every dimension split and degree, with constant and
phase-space fields, sheared x-meshes and one- and two-cell directions; and
the fused LSRK stage; its term scale against ``Problem.apply_abs``.  It is
the timed CPU baseline and the full-size parity reference, so it is pinned
here against the plain definition first."""
import numpy as np
import pytest

from dg_helpers import assert_term_scale, e_table_from_oracle
from oracle import lsrk
from oracle.dg import ConstantField, PhaseSpaceField, Problem
from oracle.sumfac import SumFac

CASES = [
    (1, 1, 0, (4, 3)), (1, 1, 3, (5, 2)), (1, 1, 5, (2, 3)), (2, 1, 2, (3, 1, 2)),
    (1, 2, 4, (2, 2, 1)), (2, 2, 1, (2, 3, 1, 2)), (2, 2, 3, (1, 2, 2, 1)),
    (2, 3, 2, (2, 1, 1, 2, 1)), (3, 2, 1, (1, 2, 1, 2, 1)), (3, 3, 1, (1, 2, 1, 1, 2, 1)),
    (3, 3, 3, (1, 1, 1, 1, 1, 2)),
]


def _pair(dx, dv, k, cells, kind, seed, basis="gl"):
    rng = np.random.default_rng(seed)
    d = dx + dv
    x_lo, x_hi, v_lo, v_hi = [0.0] * dx, [1.0] * dx, [-1.0] * dv, [1.5] * dv
    shear = None if dx == 1 else np.eye(dx) + 0.15 * np.eye(dx, k=1) - 0.05 * np.eye(dx, k=-1)
    if kind == "const":
        a = rng.uniform(-1, 1, d)
        p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, ConstantField(a),
                    shear=shear, basis=basis)
        sf = SumFac(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, a=a, shear=shear,
                    basis=basis)
    else:
        amp, ph = rng.uniform(0.3, 1.0, dv), rng.uniform(0, 1, dv)

        def E(yx):
            return amp * np.sin(2 * np.pi * (np.asarray(yx).sum(-1, keepdims=True) + ph))
        p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi,
                    PhaseSpaceField(dx, dv, E), shear=shear, basis=basis)
        sf = SumFac(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi,
                    e_nodes=e_table_from_oracle(p, E), shear=shear, basis=basis)
    return sf, p


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("kind", ["const", "phase"])
def test_sumfac_equals_oracle(case, kind):
    dx, dv, k, cells = case
    if kind == "phase" and dv < dx:
        pytest.skip("phase-space field needs dv >= dx")
    sf, p = _pair(dx, dv, k, cells, kind, seed=3 * k + dx + 7 * dv)
    u = np.random.default_rng(1).standard_normal(p.n_dofs)
    got = sf.apply(u)
    ref = p.apply(u)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    scale = p.apply_abs(u)
    assert_term_scale(got, ref, scale, 1e-13, what="sum factorisation vs oracle")
    # the term scale (the tolerance of the full-size GPU parity tests)
    got_abs = sf.apply_abs(u)
    assert np.all(got_abs >= 0)
    assert np.max(np.abs(got_abs - scale) / np.maximum(scale, 1e-300)) <= 1e-13
    if p.dofs_per_cell <= 64:
        dense = p.apply_dense(u)
        assert np.linalg.norm(got - dense) <= 1e-13 * np.linalg.norm(dense)
    sf.close()


@pytest.mark.parametrize("stage", [0, 3, 4])
def test_sumfac_stage_equals_oracle(stage):
    sf, p = _pair(2, 2, 2, (2, 3, 2, 2), "phase", seed=9)
    rng = np.random.default_rng(stage)
    w, u = rng.standard_normal(p.n_dofs), rng.standard_normal(p.n_dofs)
    dt = 0.01
    K = p.apply(w)
    u_ref = u + lsrk.B[stage] * dt * K
    w_ref = u_ref if stage == 4 else u + lsrk.A[stage] * dt * K
    wo = np.empty_like(w)
    uu = u.copy()
    sf.rk_stage(w, wo, uu, lsrk.A[stage] * dt if stage < 4 else 0.0, lsrk.B[stage] * dt,
                last=stage == 4)
    scale = dt * p.apply_abs(w)
    assert_term_scale(uu, u_ref, scale + 1e-16 * np.abs(u), 1e-13, what="u")
    assert_term_scale(wo, w_ref, scale + 1e-16 * np.abs(u), 1e-13, what="w_out")
    sf.close()


def test_sumfac_stage_on_a_cell_range():
    """A stage restricted to a range of cells updates exactly those cells, as
    the full stage does, and reads neighbours outside the range."""
    sf, p = _pair(1, 2, 2, (3, 2, 4), "phase", seed=4)
    rng = np.random.default_rng(8)
    w, u = rng.standard_normal(p.n_dofs), rng.standard_normal(p.n_dofs)
    full_w, full_u = np.empty_like(w), u.copy()
    sf.rk_stage(w, full_w, full_u, 0.02, 0.03)
    part_w, part_u = np.zeros_like(w), u.copy()
    lo, hi = 6, 18                              # v2 cell 1 of 4 (6 cells per v2 slab) and more
    sf.rk_stage(w, part_w, part_u, 0.02, 0.03, cells=(lo, hi))
    npc = p.dofs_per_cell
    sl = slice(lo * npc, hi * npc)
    assert np.array_equal(part_u[sl], full_u[sl]) and np.array_equal(part_w[sl], full_w[sl])
    assert np.array_equal(part_u[:lo * npc], u[:lo * npc])
    assert np.array_equal(part_u[hi * npc:], u[hi * npc:])
    sf.close()


@pytest.mark.parametrize("case", [c for c in CASES if c[2] >= 1], ids=lambda c: f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("kind", ["const", "phase"])
def test_sumfac_gauss_lobatto_collocation_equals_oracle(case, kind):
    """The Gauss-Lobatto collocation (nodes and quadrature at the Lobatto
    points; the traces are the face nodes) against the oracle's "gllc"
    element, operator and term scale to round-off."""
    dx, dv, k, cells = case
    if kind == "phase" and dv < dx:
        pytest.skip("phase-space field needs dv >= dx")
    sf, p = _pair(dx, dv, k, cells, kind, seed=5 * k + dx + 3 * dv, basis="gllc")
    u = np.random.default_rng(2).standard_normal(p.n_dofs)
    scale = p.apply_abs(u)
    assert_term_scale(sf.apply(u), p.apply(u), scale, 1e-13, what="Lobatto collocation")
    assert np.max(np.abs(sf.apply_abs(u) - scale) / np.maximum(scale, 1e-300)) <= 1e-13
