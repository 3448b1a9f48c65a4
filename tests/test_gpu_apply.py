"""GPU parity of the operator application against the FP64 oracle.

Every (d, k) the library supports, every precision, the adjoint, with
ragged meshes that span several blocks and include directions with one and
two cells (the periodic neighbour is the cell itself or the same cell on
both sides).  Tolerances (stated per apply):
  FP64:             ||K - K_ref|| / ||K_ref|| <= 1e-12
  FP32 / mixed:     ||K - K_ref|| / || |L| |u| || <= 1e-5   (term scale: the
                    oracle's evaluation with the absolute value of every
                    factor; rounding errors scale with it, not with K)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from dg_helpers import random_problem  # noqa: E402

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
    if prec == 0:
        assert np.linalg.norm(out - ref) <= TOL64 * np.linalg.norm(ref)
    else:
        scale = np.linalg.norm(p.apply_abs(u))
        assert np.linalg.norm(out - ref) <= TOL32 * scale
    dg.close()
