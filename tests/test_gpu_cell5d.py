"""GPU parity of the specialised 5D kernels (dim_x = 2, dim_v = 3, k = 3, FP32
sweeps; three register phases: the x block of a v node, the v1-v2 plane of
an x node, the v3 lines; FP32 input: the persistent kernel whose cells
arrive by tensor copies) against the FP64 oracle, element by element against
the term scale, and against the generic kernel.  Ragged meshes over several
blocks with one- and two-cell directions; the phase-space field changes sign
inside cells (the upwind side is chosen per thread); sheared x-mesh.  The
adjoint steps run the kernel on the negated field with weight-scaled states
and are checked against the oracle's L^T steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from dg_helpers import assert_term_scale, random_problem  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
CASES = [(2, 3, 2, 1, 3), (1, 2, 2, 3, 1), (3, 1, 1, 2, 2)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _problem(cells, kind, seed):
    shear = np.eye(2) + 0.15 * np.eye(2, k=1)
    return random_problem(2, 3, 3, cells, kind, seed=seed, shear=shear)


def _variant(dg, prec, v):
    c = dg.get_launch(prec)
    dg.set_launch(prec, c["threads"], c["cells_per_block"], c["order"], v)


@pytest.mark.parametrize("cells", CASES, ids=lambda c: "x".join(map(str, c)))
@pytest.mark.parametrize("kind", ["const", "phase"])
@pytest.mark.parametrize("prec", [1, 2])
def test_apply_5d_kernel(cells, kind, prec):
    dg, p = _problem(cells, kind, seed=sum(cells))
    assert dg.get_launch(prec)["variant"] == 2          # the default for this 5D split
    u = np.random.default_rng(1).standard_normal(p.n_dofs)
    x = torch.tensor(u, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
    xin = x.double().cpu().numpy()
    ref, scale = p.apply(xin), p.apply_abs(xin)
    for v in (2, 0):
        _variant(dg, prec, v)
        out = dg.apply(x, prec=prec).double().cpu().numpy()
        dg.check()
        assert_term_scale(out, ref, scale, TOL32, what=f"5D variant {v}")
    dg.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_apply_5d_zero_speed_directions(prec):
    """Directions whose speed is zero everywhere (x2 and v2 here) need no
    neighbour: the persistent kernel copies none for them and waits for none."""
    from oracle.dg import ConstantField, Problem
    from paper_2002_08110_gb300 import DG
    a = np.array([0.3, 0.0, -0.7, 0.0, 0.2])
    cells = (2, 3, 2, 1, 3)
    args = (2, 3, 3, cells[:2], cells[2:], [0.0] * 2, [1.0] * 2, [-1.0] * 3, [1.5] * 3)
    p = Problem(*args, ConstantField(a))
    dg = DG(*args, field_kind=0, a_const=a)
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    x = torch.tensor(u, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
    xin = x.double().cpu().numpy()
    out = dg.apply(x, prec=prec).double().cpu().numpy()
    dg.check()
    assert_term_scale(out, p.apply(xin), p.apply_abs(xin), TOL32, what="5D, zero-speed directions")
    dg.close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("stage", [1, 4])
def test_stage_5d_kernel(prec, stage):
    dg, p = _problem(CASES[0], "phase", seed=5)
    rng = np.random.default_rng(6)
    w, u = rng.standard_normal(p.n_dofs), rng.standard_normal(p.n_dofs)
    dt = 1e-2
    wt = torch.tensor(w, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
    ut = torch.tensor(u, device="cuda")
    wo = torch.empty_like(wt)
    dg.rk_stage(wt, wo, ut, stage, dt, prec=prec)
    dg.check()
    win = wt.double().cpu().numpy()
    K = p.apply(win)
    S = p.apply_abs(win)
    u_ref = u + lsrk.B[stage] * dt * K
    w_ref = u_ref if stage == 4 else u + lsrk.A[stage] * dt * K
    bound_u = 1e-14 * np.abs(u_ref) + TOL32 * dt * (S + np.abs(K))
    assert_term_scale(ut.cpu().numpy(), u_ref, bound_u, 1.0, what="u")
    a_dtK = np.abs((lsrk.B[4] if stage == 4 else lsrk.A[stage]) * dt * K)
    bound_w = bound_u + (2.5e-7 * (np.abs(u) + a_dtK) if prec == 1 else 1e-14 * np.abs(w_ref))
    assert_term_scale(wo.double().cpu().numpy(), w_ref, bound_w, 1.0, floor=1e-30, what="w_out")
    dg.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_steps_5d(prec):
    """LSRK steps with L^T (the adjoint of a linear autonomous problem) against
    the oracle's steps with the assembled transpose."""
    dg, p = _problem((2, 1, 2, 1, 2), "phase", seed=9)
    LT = p.assemble().T.tocsr()
    u0 = np.random.default_rng(10).standard_normal(p.n_dofs)
    dt, nsteps = 2e-3, 3
    ref = u0.copy()
    for _ in range(nsteps):
        ref = lsrk.step(lambda x: LT @ x, ref, dt)
    ut = torch.tensor(u0, device="cuda")
    dg.rk_step(ut, dt, nsteps=nsteps, prec=prec, adjoint=True)
    dg.check()
    rel = np.linalg.norm(ut.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel < (1e-13 if prec == 0 else 1e-5), rel
    dg.close()
