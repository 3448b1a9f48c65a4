"""Adjoint of the coupled Vlasov-Poisson steps (Sec. 6) on the GPU
(``dg_vp_step_adjoint`` and the checkpointed ``VPForward``): the step is
nonlinear in the state (its field follows the state at every stage), so its
adjoint is the transposed Jacobian at the step's own stage inputs.

* The transpose identity <Phi'(u) d, lam> = <d, Phi'(u)^T lam> for one step,
  with Phi'(u) d taken by central differences of the GPU's own FP64 steps.
* The gradient of J = 0.5 ||u(T) - u_target||^2 after several steps against
  central differences of J through the oracle's Vlasov-Poisson steps.
* Checkpoint segmentation does not change the gradient (bit for bit).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dg import PhaseSpaceField, Problem  # noqa: E402
from oracle import vp as ovp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _vp_pair(k, ncx, ncv, dv, L=4 * np.pi, vmax=5.0):
    from paper_2002_08110_gb300 import DG
    zero_e = np.zeros((ncx, k + 1, dv))
    dg = DG(1, dv, k, [ncx], [ncv] * dv, [0.0], [L], [-vmax] * dv, [vmax] * dv, field_kind=1,
            e_nodes=zero_e)
    p = Problem(1, dv, k, [ncx], [ncv] * dv, [0.0], [L], [-vmax] * dv, [vmax] * dv,
                PhaseSpaceField(1, dv, lambda yx: np.zeros(yx.shape[:-1] + (dv,))))
    return dg, p


def _landau(alpha, kappa, dv, phase=0.3):
    """A perturbed Maxwellian.  The phase keeps the zeros of E off the x nodes:
    where E vanishes at a node the step is not differentiable (the upwind side
    flips), and a central difference there averages two one-sided slopes."""
    def f(yx, v):
        return ((1 + alpha * np.cos(kappa * yx[..., 0] + phase)) * np.exp(-0.5 * np.sum(v ** 2, -1))
                / (2 * np.pi) ** (dv / 2))
    return f


@pytest.mark.parametrize("dv,k,ncx,ncv", [(1, 2, 5, 8), (1, 3, 4, 6), (2, 2, 3, 4)])
def test_vp_step_adjoint_transpose_identity(dv, k, ncx, ncv):
    dg, p = _vp_pair(k, ncx, ncv, dv)
    u0 = torch.tensor(p.interpolate(_landau(0.3, 0.5, dv)), device="cuda")
    rng = np.random.default_rng(20 + k + dv)
    d = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda")
    d *= torch.linalg.vector_norm(u0) / torch.linalg.vector_norm(d)
    lam = torch.tensor(rng.standard_normal(p.n_dofs), device="cuda")
    dt = 0.05

    def step(x):
        y = x.clone()
        dg.vp_rk_step(y, dt, nsteps=1, prec=0)
        return y

    eps = 1e-6
    Jd = (step(u0 + eps * d) - step(u0 - eps * d)) / (2 * eps)
    ubar = lam.clone()
    dg.vp_step_adjoint(u0, ubar, dt)
    dg.check()
    lhs = float(torch.dot(Jd, lam))
    rhs = float(torch.dot(d, ubar))
    scale = float(torch.linalg.vector_norm(Jd) * torch.linalg.vector_norm(lam))
    assert abs(lhs - rhs) <= 1e-8 * scale, (lhs, rhs, scale)
    dg.close()


def test_vp_misfit_gradient_matches_oracle_differences():
    from paper_2002_08110_gb300.autograd import vp_misfit_gradient
    dv, k, ncx, ncv = 1, 2, 4, 6
    dg, p = _vp_pair(k, ncx, ncv, dv)
    u0 = p.interpolate(_landau(0.3, 0.5, dv))
    rng = np.random.default_rng(5)
    target = u0 + 0.05 * rng.standard_normal(p.n_dofs)
    dt, nsteps = 0.05, 4
    J, g = vp_misfit_gradient(torch.tensor(u0, device="cuda"), torch.tensor(target, device="cuda"),
                              dg, dt, nsteps, checkpoint_every=3)
    g = g.cpu().numpy()

    def J_oracle(x):
        for _ in range(nsteps):
            x = ovp.vp_step(p, x, dt)
        return 0.5 * float(np.sum((x - target) ** 2))

    assert abs(J - J_oracle(u0)) <= 1e-10 * abs(J)
    for i in range(3):
        d = rng.standard_normal(p.n_dofs)
        d *= np.linalg.norm(u0) / np.linalg.norm(d)
        eps = 1e-6
        fd = (J_oracle(u0 + eps * d) - J_oracle(u0 - eps * d)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * np.linalg.norm(g) * np.linalg.norm(d), (i, fd, g @ d)
    dg.close()


def test_vp_gradient_independent_of_checkpoint_segments():
    from paper_2002_08110_gb300.autograd import vp_misfit_gradient
    dg, p = _vp_pair(2, 5, 8, 1)
    u0 = torch.tensor(p.interpolate(_landau(0.2, 0.5, 1)), device="cuda")
    target = u0 * 0.9
    grads = [vp_misfit_gradient(u0, target, dg, 0.05, 5, checkpoint_every=e)[1] for e in (1, 2, 5)]
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])
    dg.close()
