"""Gradient of the final-time misfit through LSRK(5,4) (autograd over the
library's adjoint): against central finite differences (exact up to rounding
for this quadratic functional of a linear map), against the oracle's
assembled transpose, and with checkpointed recomputation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from dg_helpers import dg_for  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _setup(k=2):
    w = W.shrink(W.config_adjoint(), cells_x=(3, 2), cells_v=(2, 1, 2), k=k)
    dg, p = dg_for(w)
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    u0 = W.separable_state(w, zeta)
    pert = W.noise(w)
    dt = 0.5 * W.time_step(w)[0]
    return w, dg, p, u0, pert, dt


@pytest.mark.parametrize("prec", [0, 1])
def test_gradient_against_oracle_transpose(prec):
    from paper_2002_08110_gb300.autograd import misfit_gradient
    w, dg, p, u0, pert, dt = _setup()
    nsteps = 7
    L = p.assemble()
    LT = L.T.tocsr()
    tgt = u0 + pert
    for _ in range(nsteps):
        tgt = lsrk.step(lambda x: L @ x, tgt, dt)
    uT = u0.copy()
    for _ in range(nsteps):
        uT = lsrk.step(lambda x: L @ x, uT, dt)
    g_ref = uT - tgt
    for _ in range(nsteps):
        g_ref = lsrk.step(lambda x: LT @ x, g_ref, dt)
    J, g = misfit_gradient(torch.tensor(u0, device="cuda"), torch.tensor(tgt, device="cuda"),
                           dg, dt, nsteps, prec=prec, checkpoint_every=3)
    g = g.cpu().numpy()
    J_ref = 0.5 * np.sum((uT - tgt) ** 2)
    tol = 1e-11 if prec == 0 else 2e-4
    assert abs(J - J_ref) <= tol * J_ref
    assert np.linalg.norm(g - g_ref) <= tol * np.linalg.norm(g_ref)
    dg.close()


def test_gradient_against_finite_differences():
    """J is quadratic in u0, so central differences are exact up to rounding."""
    from paper_2002_08110_gb300.autograd import final_state, misfit_gradient
    w, dg, p, u0, pert, dt = _setup(k=3)
    nsteps = 5
    u0t = torch.tensor(u0, device="cuda")
    tgt = torch.tensor(u0 + pert, device="cuda")
    dg.rk_step(tgt, dt, nsteps=nsteps, prec=0)
    J, g = misfit_gradient(u0t, tgt, dg, dt, nsteps, prec=0, checkpoint_every=2)
    rng = np.random.default_rng(4)
    for _ in range(3):
        e = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda")
        eps = 1e-3

        def Jf(x):
            with torch.no_grad():
                y = final_state(x, dg, dt, nsteps, 0, 100)
                return 0.5 * torch.sum((y - tgt) ** 2).item()
        fd = (Jf(u0t + eps * e) - Jf(u0t - eps * e)) / (2 * eps)
        an = torch.dot(g, e).item()
        assert abs(fd - an) <= 1e-8 * max(abs(an), 1e-30) + 1e-12 * abs(J)
    dg.close()


def test_checkpoint_recomputation_detects_corruption():
    from paper_2002_08110_gb300.autograd import CheckpointMismatch, RKForward
    w, dg, p, u0, pert, dt = _setup()
    x = torch.tensor(u0, device="cuda", requires_grad=True)
    uT = RKForward.apply(x, dg, dt, 6, 0, 2)
    uT.sum().backward()                    # consistent trajectory: passes
    assert x.grad is not None
    y = torch.tensor(u0, device="cuda", requires_grad=True)
    vT = RKForward.apply(y, dg, dt, 6, 0, 2)
    vT.grad_fn.checkpoints[1].add_(1e-3)   # corrupt a stored checkpoint
    with pytest.raises(CheckpointMismatch):
        vT.sum().backward()
    dg.close()
