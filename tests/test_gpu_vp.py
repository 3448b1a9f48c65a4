"""Vlasov-Poisson coupling on the GPU (Sec. 6) against the oracle: the charge
density reduction, the 1D periodic Poisson solve, the device-fed field and
whole coupled LSRK steps; and the linear Landau damping rate as a property of
the coupled GPU run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from dg_helpers import random_problem  # noqa: E402
from oracle.dg import ConstantField, PhaseSpaceField, Problem  # noqa: E402
from oracle import vp as ovp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _vp_pair(k, ncx, ncv, dv=1, L=4 * np.pi, vmax=6.0, shear=None):
    from paper_2002_08110_gb300 import DG
    nq = (k + 1) ** 1
    zero_e = np.zeros((ncx, nq, dv))
    dg = DG(1, dv, k, [ncx], [ncv] * dv, [0.0], [L], [-vmax] * dv, [vmax] * dv, field_kind=1,
            e_nodes=zero_e, shear=shear)
    p = Problem(1, dv, k, [ncx], [ncv] * dv, [0.0], [L], [-vmax] * dv, [vmax] * dv,
                PhaseSpaceField(1, dv, lambda yx: np.zeros(yx.shape[:-1] + (dv,))), shear=shear)
    return dg, p


def _landau(alpha, kappa, dv):
    def f(yx, v):
        return ((1 + alpha * np.cos(kappa * yx[..., 0])) * np.exp(-0.5 * np.sum(v ** 2, -1))
                / (2 * np.pi) ** (dv / 2))
    return f


# -- charge density -----------------------------------------------------------
@pytest.mark.parametrize("dx,dv,k,cells", [
    (1, 1, 3, [5, 7]), (1, 2, 2, [3, 5, 4]), (2, 2, 1, [3, 2, 5, 3]),
    (2, 3, 2, [2, 3, 3, 2, 3]), (3, 3, 3, [2, 3, 2, 2, 2, 3]), (1, 3, 5, [2, 3, 2, 2]),
])
@pytest.mark.parametrize("prec", [0, 1])
def test_charge_density_matches_oracle(dx, dv, k, cells, prec):
    dg, p = random_problem(dx, dv, k, cells, "const", seed=dx + 3 * dv + k)
    rng = np.random.default_rng(7 + prec)
    u = rng.standard_normal(p.n_dofs)
    dt = torch.float64 if prec == 0 else torch.float32
    ut = torch.tensor(u, device="cuda").to(dt)
    rho = dg.charge_density(ut, prec=prec)
    ref = p.charge_density(ut.double().cpu().numpy()).reshape(-1)
    scale = p.charge_density(np.abs(ut.double().cpu().numpy())).reshape(-1)   # 1 - int |f|
    # both sides sum the same FP64 products; only the summation order differs
    bound = 1e-13 * (np.abs(1 - scale) + 1)
    assert np.all(np.abs(rho.cpu().numpy() - ref) <= bound)
    dg.close()


def test_charge_density_6d_fullsize_sampled():
    """8^6 cells, k = 3 (the 6D workload) on three sampled x cells; the oracle
    reads only those cells' rows of f from the device."""
    import workloads as W
    from paper_2002_08110_gb300 import DG, reference_nodes
    w = W.config_6d()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    f = W.separable_state(w, zeta, xp=torch, device="cuda").float()
    rho = dg.charge_density(f, prec=1)
    torch.cuda.synchronize()
    shear = None if w.shear is None else np.array(w.shear).reshape(w.dx, w.dx)
    p = Problem(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                ConstantField([1.0] * 6), shear=shear)

    class Rows:
        def __init__(self, t):
            self.t = t

        def __getitem__(self, s):
            return self.t[s].double().cpu().numpy()

    ncx = int(np.prod(w.cells_x))
    nqx = (w.k + 1) ** 3
    cells = [0, 137, ncx - 1]
    ref = p.charge_density(Rows(f), x_cells=cells)
    got = rho.view(ncx, nqx)[cells].cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    dg.close()


# -- Poisson ------------------------------------------------------------------
@pytest.mark.parametrize("k,ncx,shear", [(1, 3, None), (3, 37, None), (2, 2500, [[1.3]]),
                                         (5, 1031, [[-0.7]])])
def test_poisson_matches_oracle(k, ncx, shear):
    """Random nodal rho; sizes span several 1024-cell chunks of the scan."""
    dg, p = _vp_pair(k, ncx, 2, L=3.0, shear=shear)
    rho = np.random.default_rng(ncx).standard_normal((ncx, k + 1)) + 0.5
    _, ref = ovp.poisson_periodic_1d(p, rho)
    e = dg.poisson_periodic_1d(torch.tensor(rho.reshape(-1), device="cuda"))
    scale = np.abs(p.h[0] * (1.0 if shear is None else shear[0][0])) * np.abs(rho).sum()
    np.testing.assert_allclose(e.cpu().numpy(), ref.reshape(-1), rtol=0, atol=1e-13 * scale)
    dg.close()


# -- device-fed field ---------------------------------------------------------
def test_set_field_device_equals_host_field():
    """The same field from host and device memory gives bit-identical applies
    (FP64 and FP32); components beyond the given ones are zero."""
    from paper_2002_08110_gb300 import DG
    k, cells_x, cells_v = 2, [4, 3], [3, 4]
    rng = np.random.default_rng(5)
    nq = (k + 1) ** 2
    e1 = rng.uniform(-1, 1, (12, nq, 1))
    full = np.concatenate([e1, np.zeros_like(e1)], axis=-1)
    kw = dict(dim_x=2, dim_v=2, degree=k, cells_x=cells_x, cells_v=cells_v, x_lo=[0, 0],
              x_hi=[1, 1], v_lo=[-1, -1], v_hi=[1, 1], field_kind=1)
    host = DG(e_nodes=full, **kw)
    dev = DG(e_nodes=np.zeros_like(full), **kw)
    dev.set_field_device(torch.tensor(-e1.reshape(-1), device="cuda"), components=1, scale=-1.0)
    u = torch.tensor(rng.standard_normal(host.n_dofs), device="cuda")
    for prec, src in ((0, u), (1, u.float())):
        a = host.apply(src, prec=prec)
        b = dev.apply(src, prec=prec)
        assert torch.equal(a, b)
    dev.check()
    host.close()
    dev.close()


def test_set_field_device_6d_kernel_choice():
    """d = 6, k = 3: a device field whose sign changes inside a cell turns the
    specialised kernel off (uniform_sides 0) and back on; results follow the
    oracle either way."""
    from paper_2002_08110_gb300 import DG
    cells = [2, 2, 2, 2, 2, 2]
    kw = dict(dim_x=3, dim_v=3, degree=3, cells_x=cells[:3], cells_v=cells[3:], x_lo=[0] * 3,
              x_hi=[1] * 3, v_lo=[-1] * 3, v_hi=[1] * 3, field_kind=1)
    nq = 64
    dg = DG(e_nodes=np.full((8, nq, 3), 0.5), **kw)
    assert dg.info.uniform_sides == 1
    p0 = Problem(3, 3, 3, cells[:3], cells[3:], [0] * 3, [1] * 3, [-1] * 3, [1] * 3,
                 ConstantField([1.0] * 6))
    xs = np.array([p0.node_coordinates(c)[0][..., 0, 0, 0, :].reshape(-1, 3, order="F")
                   for c in range(8)])                    # (x cell, x node, 3)
    def mixed_fn(yx):
        return np.stack([np.sin(2 * np.pi * yx[..., 0] + 0.3), 0.4 + 0 * yx[..., 1],
                         -0.2 + 0 * yx[..., 2]], -1)

    def const_fn(yx):
        return np.full(yx.shape[:-1] + (3,), -0.3)

    rng = np.random.default_rng(1)
    u = rng.standard_normal(dg.n_dofs)
    ut = torch.tensor(u, device="cuda", dtype=torch.float32)
    # the oracle evaluates the same functions at its own nodes (the v faces'
    # quadrature points are the x nodes)
    for fn, uniform in ((mixed_fn, 0), (const_fn, 1)):
        table = fn(xs)
        dg.set_field_device(torch.tensor(table.reshape(-1), device="cuda"))
        assert dg.info.uniform_sides == uniform
        got = dg.apply(ut, prec=1).double().cpu().numpy()

        p = p0.with_field(PhaseSpaceField(3, 3, fn))
        uu = ut.double().cpu().numpy()
        ref = p.apply(uu)
        scale = p.apply_abs(uu)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(scale)
    dg.check()
    dg.close()


# -- coupled steps --------------------------------------------------------------
@pytest.mark.parametrize("dv,k,ncx,ncv,prec", [(1, 3, 6, 10, 0), (1, 2, 5, 9, 1), (2, 2, 4, 5, 0),
                                               (1, 3, 6, 10, 2)])
def test_vp_steps_match_oracle(dv, k, ncx, ncv, prec):
    dg, p = _vp_pair(k, ncx, ncv, dv=dv, L=4 * np.pi, vmax=5.0)
    u0 = p.interpolate(_landau(0.2, 0.5, dv))
    dt = 0.04
    ref = u0.copy()
    for _ in range(2):
        ref = ovp.vp_step(p, ref, dt)
    u = torch.tensor(u0, device="cuda")
    dg.vp_rk_step(u, dt, nsteps=2, prec=prec)
    dg.check()
    got = u.cpu().numpy()
    if prec == 0:
        tol = 1e-11 * np.linalg.norm(ref - u0) + 1e-14 * np.linalg.norm(u0)
    else:
        # FP32 sweeps: 1e-5 of the term scale |L| |u| per stage, over the
        # 2 steps' stage weights (sum |b_s| < 2)
        S = p.with_field(ovp.field_from(p, u0)).apply_abs(u0)
        tol = 1e-5 * 2 * 2 * dt * np.linalg.norm(S)
    assert np.linalg.norm(got - ref) <= tol
    dg.close()


def test_vp_rejects_bad_handles():
    from paper_2002_08110_gb300 import DG, DGError
    dg = DG(2, 2, 1, [2, 2], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], field_kind=1,
            e_nodes=np.zeros((4, 4, 2)))
    u = torch.zeros(dg.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(DGError):
        dg.vp_rk_step(u, 0.1)
    with pytest.raises(DGError):
        # sized as for a 1D x mesh of the same cells so that the library itself refuses
        dg.poisson_periodic_1d(torch.zeros(8, dtype=torch.float64, device="cuda"),
                               torch.zeros(8, dtype=torch.float64, device="cuda"))
    dg.close()


def test_landau_damping_rate():
    """Linear Landau damping (alpha = 0.01, kappa = 0.5): the electric field's
    L2 norm decays like exp(gamma t) with gamma = -0.1533 (the root of the
    Vlasov-Poisson dispersion relation for kappa = 0.5), oscillating at
    2 omega = 2.83.  The maxima over t in [2, 18] give the rate."""
    k, ncx, ncv = 3, 16, 64
    dg, p = _vp_pair(k, ncx, ncv, dv=1, L=4 * np.pi, vmax=6.0)
    u = torch.tensor(p.interpolate(_landau(0.01, 0.5, 1)), device="cuda")
    w = torch.tensor(p.T.w, device="cuda").repeat(ncx) * (p.h[0] / 2)
    dt, T = 0.025, 18.0
    ts, en = [], []
    w0 = dg.empty(0)
    w1 = dg.empty(0)
    for i in range(int(round(T / dt)) + 1):
        rho = dg.charge_density(u)
        e = dg.poisson_periodic_1d(rho)
        ts.append(i * dt)
        en.append(float(torch.sqrt(torch.sum(w * e * e))))
        dg.vp_rk_step(u, dt, nsteps=1, w0=w0, w1=w1)
    dg.check()
    ts, en = np.array(ts), np.log(np.array(en))
    peaks = [i for i in range(1, len(en) - 1) if en[i] > en[i - 1] and en[i] >= en[i + 1]
             and ts[i] >= 2.0]
    assert len(peaks) >= 5
    gamma = np.polyfit(ts[peaks], en[peaks], 1)[0]
    assert abs(gamma + 0.1533) < 0.01, gamma
    dg.close()
