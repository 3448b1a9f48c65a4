"""Batched persistent execution: every member of a batch advances exactly as
the single-problem path (itself checked against the oracle), for both
precisions, any tile size, and after autotuning; one member is also checked
against the oracle's time integration directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


def _members(count=6, seed=3):
    ws = W.batched_instances(count=count, seed=seed, cells_lo=2, cells_hi=5)
    # include the smallest degree too
    ws[0] = W.Workload(**{**ws[0].__dict__, "k": 1})
    return ws


def _states(ws, zeta_of):
    return [torch.tensor(W.separable_state(w, zeta_of(w.k)) +
                         0.1 * np.random.default_rng(i).standard_normal(w.n_dofs), device="cuda")
            for i, w in enumerate(ws)]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_single_problem_path(prec):
    from paper_2002_08110_gb300 import DG, DGBatch, reference_nodes
    ws = _members()
    dgs = [DG(**W.dg_kwargs(w)) for w in ws]
    zeta_of = lambda k: reference_nodes(k)[0]
    u0 = _states(ws, zeta_of)
    dts = [0.5 * W.time_step(w)[0] for w in ws]
    wdt = torch.float32 if prec == 1 else torch.float64
    nsteps = 3
    refs = []
    for dg, u, dt in zip(dgs, u0, dts):
        x = u.clone()
        dg.rk_step(x, dt, nsteps=nsteps, prec=prec)
        refs.append(x)
    batch = DGBatch(dgs)
    assert batch.n_dofs == sum(w.n_dofs for w in ws)
    for tile, threads in [(4096, 256), (256, 64), (1024, 512)]:
        batch.set_launch(tile, threads)
        us = [u.clone() for u in u0]
        w0s = [torch.empty(w.n_dofs, device="cuda", dtype=wdt) for w in ws]
        w1s = [torch.empty(w.n_dofs, device="cuda", dtype=wdt) for w in ws]
        batch.rk_step(us, w0s, w1s, dts, nsteps=nsteps, prec=prec)
        batch.check()
        for u, ref in zip(us, refs):
            tol = 1e-13 if prec == 0 else 1e-6
            assert torch.max(torch.abs(u - ref)) <= tol * torch.max(torch.abs(ref))
    # autotuner picks a configuration; results stay the same afterwards
    us = [u.clone() for u in u0]
    w0s = [torch.empty(w.n_dofs, device="cuda", dtype=wdt) for w in ws]
    w1s = [torch.empty(w.n_dofs, device="cuda", dtype=wdt) for w in ws]
    best = batch.autotune(us, w0s, w1s, dts, prec=prec)
    assert best > 0
    us = [u.clone() for u in u0]
    batch.rk_step(us, w0s, w1s, dts, nsteps=nsteps, prec=prec)
    batch.check()
    for u, ref in zip(us, refs):
        tol = 1e-13 if prec == 0 else 1e-6
        assert torch.max(torch.abs(u - ref)) <= tol * torch.max(torch.abs(ref))
    batch.close()
    for dg in dgs:
        dg.close()


def test_batch_member_against_oracle():
    from paper_2002_08110_gb300 import DG, DGBatch
    from dg_helpers import oracle_for
    # small members only: the oracle assembles each operator densely by cell
    ws = [w for w in _members(count=12, seed=5) if w.n_dofs <= 30000][:4]
    assert len(ws) >= 2
    dgs = [DG(**W.dg_kwargs(w)) for w in ws]
    zeta = lambda k: np.polynomial.legendre.leggauss(k + 1)[0]
    u0 = [W.separable_state(w, zeta(w.k)) for w in ws]
    dts = [0.5 * W.time_step(w)[0] for w in ws]
    batch = DGBatch(dgs)
    us = [torch.tensor(u, device="cuda") for u in u0]
    w0s = [torch.empty(w.n_dofs, device="cuda", dtype=torch.float64) for w in ws]
    w1s = [torch.empty(w.n_dofs, device="cuda", dtype=torch.float64) for w in ws]
    batch.rk_step(us, w0s, w1s, dts, nsteps=2, prec=0)
    batch.check()
    for w, u, ug, dt in zip(ws, u0, us, dts):
        L = oracle_for(w).assemble()
        ref = u
        for _ in range(2):
            ref = lsrk.step(lambda x: L @ x, ref, dt)
        assert np.linalg.norm(ug.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    batch.close()


def test_batch_rejects_unsupported_members():
    from paper_2002_08110_gb300 import DG, DGBatch, DGError
    w = W.shrink(W.config_4d(), cells_x=(2, 2), cells_v=(2, 2), k=1)
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    with pytest.raises(DGError):
        DGBatch([dg])
    dg.close()
