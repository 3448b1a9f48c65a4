"""The delta-f form (FP32 sweeps around an FP64 reference operator) against
the FP64 oracle on the smooth 6D workload, where plain FP32 sweeps lose
relative accuracy because L u is much smaller than its terms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from dg_helpers import oracle_for  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


@pytest.fixture(scope="module")
def small6d():
    from paper_2002_08110_gb300 import DG, reference_nodes
    w = W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, 2))
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    p = oracle_for(w)
    u = W.separable_state(w, zeta, xp=torch, device="cuda")
    u_ref = W.separable_state(W.equilibrium_6d(w), zeta, xp=torch, device="cuda")
    yield w, dg, p, u, u_ref
    dg.close()


@pytest.mark.parametrize("variant", [0, 2])
def test_apply_df_meets_plain_relative_tolerance(small6d, variant):
    from paper_2002_08110_gb300 import PREC_FP32
    w, dg, p, u, u_ref = small6d
    dg.set_launch(PREC_FP32, threads=256, cells_per_block=1, variant=variant)
    dg.set_reference(u_ref)
    ref = p.apply(u.cpu().numpy())
    kdf = dg.apply_df(u).cpu().numpy()
    k32 = dg.apply(u.float(), prec=PREC_FP32).double().cpu().numpy()
    dg.check()
    err_df = np.linalg.norm(kdf - ref) / np.linalg.norm(ref)
    err_32 = np.linalg.norm(k32 - ref) / np.linalg.norm(ref)
    assert err_df <= 1e-5, err_df
    assert err_df * 10 <= err_32, (err_df, err_32)


@pytest.mark.parametrize("variant", [0, 2])
def test_rk_step_df_against_oracle(small6d, variant):
    """Two LSRK steps: the state change matches the FP64 oracle to 1e-5 of
    itself (plain relative), and the stage kernels took the delta-f path on
    the specialised (variant 2) and generic (variant 0) kernels."""
    from paper_2002_08110_gb300 import PREC_FP32
    w, dg, p, u, u_ref = small6d
    dg.set_launch(PREC_FP32, threads=256, cells_per_block=1, variant=variant)
    dg.set_reference(u_ref)
    dt, _ = W.time_step(w)
    u0 = u.cpu().numpy()
    ref = u0.copy()
    for _ in range(2):
        ref = lsrk.step(p.apply, ref, dt)
    x = u.clone()
    dg.rk_step_df(x, dt, nsteps=2)
    dg.check()
    inc = np.linalg.norm(ref - u0)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-5 * inc
    # the plain FP32 steps are visibly worse on this smooth state
    y = u.clone()
    dg.rk_step(y, dt, nsteps=2, prec=PREC_FP32)
    assert np.linalg.norm(x.cpu().numpy() - ref) * 10 <= np.linalg.norm(y.cpu().numpy() - ref)


def test_df_requires_reference():
    from paper_2002_08110_gb300 import DG, DGError
    dg = DG(2, 2, 1, [2, 2], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], field_kind=0, a_const=[1, 1, 1, 1])
    u = torch.zeros(dg.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(DGError):
        dg.apply_df(u)
    dg.close()
