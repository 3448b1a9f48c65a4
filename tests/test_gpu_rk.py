"""GPU parity of the fused LSRK(5,4) stages and of whole time steps, the
invariants over time, integrals and the device error latch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from dg_helpers import dg_for, oracle_for, random_problem  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


@pytest.mark.parametrize("case", [(1, 1, 3, (6, 5)), (2, 2, 2, (2, 3, 2, 2)),
                                  (3, 3, 3, (2, 1, 2, 1, 2, 2)), "6d_uniform", "6d_uniform_v1"],
                         ids=lambda c: c if isinstance(c, str) else f"{c[0]}x{c[1]}v_k{c[2]}")
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("stage", [0, 2, 4])
def test_fused_stage(case, prec, stage):
    """K = L(w); u <- u + b_s dt K; w_out = u_old + a_s dt K (s < 4) or u_new.
    "6d_uniform*" run the specialised 6D kernels (no sign change inside cells)."""
    if case.__class__ is str:
        # the specialised 6D kernels: 128 threads per cell (default) or 64 ("_v1")
        dg, p = dg_for(W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, 2)))
        assert dg.info.uniform_sides == 1
        if case.endswith("_v1") and prec != 0:
            c = dg.get_launch(prec)
            dg.set_launch(prec, c["threads"], c["cells_per_block"], c["order"], 1)
    else:
        dx, dv, k, cells = case
        dg, p = random_problem(dx, dv, k, cells, "phase", seed=11)
    rng = np.random.default_rng(12)
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
    u_ref = u + lsrk.B[stage] * dt * K
    w_ref = u_ref if stage == 4 else u + lsrk.A[stage] * dt * K
    scale = 1.0 if prec == 0 else np.abs(p.apply_abs(win))
    tol = 1e-13 if prec == 0 else 1e-5
    err_u = np.abs(ut.cpu().numpy() - u_ref)
    err_w = np.abs(wo.double().cpu().numpy() - w_ref)
    if prec == 0:
        assert np.max(err_u) <= tol * np.max(np.abs(u_ref))
        assert np.max(err_w) <= tol * np.max(np.abs(w_ref))
    else:
        # K error (term scale) times dt, plus the FP32 rounding of w_out
        bound_u = 1e-14 * np.abs(u_ref) + tol * dt * (scale + np.abs(K))
        assert np.all(err_u <= bound_u + 1e-300)
        if prec == 1:
            a_dtK = np.abs((lsrk.B[4] if stage == 4 else lsrk.A[stage]) * dt * K)
            assert np.all(err_w <= bound_u + 2.5e-7 * (np.abs(u) + a_dtK) + 1e-30)
        else:
            assert np.all(err_w <= bound_u + 1e-14 * np.abs(w_ref))
    dg.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_rk_steps_match_oracle(prec, adjoint):
    """nsteps full LSRK(5,4) steps (graph replay) == the oracle's steps with
    the assembled L (or L^T)."""
    w = W.shrink(W.config_4d(), cells_x=(3, 2), cells_v=(2, 3), k=2)
    dg, p = dg_for(w)
    L = p.assemble()
    A = L.T.tocsr() if adjoint else L
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    u0 = W.initial_state(w, zeta)
    dt = 0.5 * W.time_step(w)[0]
    nsteps = 7
    ref = u0.copy()
    for _ in range(nsteps):
        ref = lsrk.step(lambda x: A @ x, ref, dt)
    ut = torch.tensor(u0, device="cuda")
    dg.rk_step(ut, dt, nsteps=nsteps, prec=prec, adjoint=adjoint)
    dg.check()
    out = ut.cpu().numpy()
    rel = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert rel < (1e-13 if prec == 0 else 1e-5), rel
    # replay again from the same start (graphs cached) gives the same result
    ut2 = torch.tensor(u0, device="cuda")
    dg.rk_step(ut2, dt, nsteps=nsteps, prec=prec, adjoint=adjoint)
    assert torch.equal(ut, ut2)
    dg.close()


def test_rk_2d_config_one_period():
    """The 2D workload through the library: after T = 2 (240 steps) the state
    matches the oracle's time integration and returns to u0 up to the
    discretisation error; mass is conserved and the L2 norm does not grow."""
    w = W.config_2d()
    dg, p = dg_for(w)
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    u0 = W.separable_state(w, zeta)
    dt, steps = W.time_step(w)
    ut = torch.tensor(u0, device="cuda")
    m0, l0, _ = dg.integrals(ut)
    dg.rk_step(ut, dt, nsteps=steps)
    dg.check()
    m1, l1, _ = dg.integrals(ut)
    L = p.assemble()
    ref = u0.copy()
    for _ in range(steps):
        ref = lsrk.step(lambda x: L @ x, ref, dt)
    out = ut.cpu().numpy()
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    Md = p.mass_diagonal()
    assert math.sqrt((out - u0) @ (Md * (out - u0)) / (u0 @ (Md * u0))) < 2e-4
    assert abs(m1 - m0) < 1e-13
    assert l1 <= l0 * (1 + 1e-14)
    dg.close()


def test_integrals_match_oracle():
    w = W.shrink(W.config_4d(), cells_x=(3, 2), cells_v=(2, 3), k=3)
    dg, p = dg_for(w)
    u = np.random.default_rng(3).standard_normal(p.n_dofs)
    m, l2, mx = dg.integrals(torch.tensor(u, device="cuda"))
    rm, rl2, rmx = p.integrals(u)
    assert abs(m - rm) <= 1e-12 * abs(rl2) and abs(l2 - rl2) <= 1e-12 * rl2 and mx == rmx
    dg.close()


def test_nonfinite_is_latched_and_cleared():
    from paper_2002_08110_gb300 import DGError
    dg, p = random_problem(2, 2, 1, (2, 2, 2, 2), "const", seed=1)
    u = torch.zeros(p.n_dofs, device="cuda", dtype=torch.float64)
    u[5] = float("nan")
    dg.apply(u)
    with pytest.raises(DGError) as ei:
        dg.check()
    assert ei.value.status == 5
    u[5] = 0.0
    dg.apply(u)
    dg.check()          # latch cleared
    dg.close()


def test_host_argument_errors():
    from paper_2002_08110_gb300 import DGError
    dg, p = random_problem(1, 1, 2, (3, 3), "const", seed=1)
    u = torch.zeros(p.n_dofs, device="cuda", dtype=torch.float64)
    lib = dg.lib
    import ctypes
    ptr = ctypes.c_void_p(u.data_ptr())
    assert lib.dg_apply(dg.handle, ptr, ptr, 0, None) == 1            # aliasing
    assert lib.dg_apply(dg.handle, ptr, ctypes.c_void_p(u.data_ptr() + 8 * p.n_dofs // 2),
                        0, None) == 1                                  # overlap
    assert lib.dg_apply(dg.handle, ptr, ctypes.c_void_p(u.data_ptr() + 4), 0, None) == 1
    assert lib.dg_apply(dg.handle, ptr, None, 0, None) == 1
    assert lib.dg_apply(dg.handle, ptr, ptr, 3, None) == 1             # precision
    assert lib.dg_rk_stage(dg.handle, ptr, ptr, ptr, 5, 0.1, 0, 0, None) == 1
    with pytest.raises(DGError):
        dg.set_launch(0, threads=48, cells_per_block=1)
    with pytest.raises(DGError):
        dg.set_launch(0, threads=64, cells_per_block=1, order=[0, 0])
    dg.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_host_buffer_stage_equals_device_stage(prec):
    """dg_rk_stage_host (pinned host buffers, library-owned staging) gives the
    same bits as dg_rk_stage on device buffers, twice in a row (the staging is
    reused)."""
    dg, p = random_problem(2, 2, 3, [3, 4, 3, 5], "phase", seed=9)
    rng = np.random.default_rng(4)
    wdt = torch.float64 if prec == 0 else torch.float32
    u0 = torch.tensor(rng.standard_normal(dg.n_dofs))
    w_in = torch.tensor(rng.standard_normal(dg.n_dofs)).to(wdt)
    for stage in (1, 4):
        du, dw_in = u0.cuda(), w_in.cuda()
        dw_out = torch.empty_like(dw_in)
        dg.rk_stage(dw_in, dw_out, du, stage, 0.01, prec=prec)
        hu = u0.clone().pin_memory()
        hw_in = w_in.clone().pin_memory()
        hw_out = torch.empty_like(hw_in).pin_memory()
        dg.rk_stage_host(hw_in, hw_out, hu, stage, 0.01, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(hu, du.cpu())
        assert torch.equal(hw_out, dw_out.cpu())
    dg.check()
    dg.close()


def test_bounded_wait_gives_up_and_reports_timeout():
    """A kernel wait that cannot complete (an mbarrier expecting bytes that no
    copy delivers) gives up after its limit and latches DG_ERR_TIMEOUT; the
    latch clears and the context keeps working."""
    import ctypes
    from paper_2002_08110_gb300 import DGError
    dg, p = random_problem(2, 2, 2, (2, 3, 2, 2), "phase", seed=3)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert dg.lib.dg_selftest_wait(dg.handle, stream) == 0
    with pytest.raises(DGError) as err:
        dg.check()
    assert err.value.status == 6            # DG_ERR_TIMEOUT
    dg.check()                              # cleared
    u = torch.tensor(np.random.default_rng(0).standard_normal(p.n_dofs), device="cuda")
    ref = p.apply(u.cpu().numpy())
    assert np.linalg.norm(dg.apply(u).cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    dg.close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n3", [2, 6, 10])
def test_host_buffer_stage_pipelined_6d(prec, n3):
    """The 6D host-buffer stage runs as a pipeline over slabs of v3 cells
    (one slab per v3 cell up to 8, uneven slabs beyond); every slab's kernel
    walks part of each pencil and reads the v3 neighbour of its first cell.
    The bits equal the one-launch device stage's, for both pencil directions
    (the v3 speed changes sign across x3 cells)."""
    dg, p = dg_for(W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, n3)))
    assert dg.info.uniform_sides == 1
    rng = np.random.default_rng(n3)
    wdt = torch.float32 if prec == 1 else torch.float64
    u0 = torch.tensor(rng.standard_normal(dg.n_dofs))
    w_in = torch.tensor(rng.standard_normal(dg.n_dofs)).to(wdt)
    for stage in (0, 4):
        du, dw_in = u0.cuda(), w_in.cuda()
        dw_out = torch.empty_like(dw_in)
        dg.rk_stage(dw_in, dw_out, du, stage, 0.01, prec=prec)
        hu = u0.clone().pin_memory()
        hw_in = w_in.clone().pin_memory()
        hw_out = torch.empty_like(hw_in).pin_memory()
        dg.rk_stage_host(hw_in, hw_out, hu, stage, 0.01, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(hu, du.cpu())
        assert torch.equal(hw_out, dw_out.cpu())
        assert not torch.equal(hu, u0)
    dg.check()
    dg.close()
