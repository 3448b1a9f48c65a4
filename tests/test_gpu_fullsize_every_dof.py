"""Parity of every value at the workloads' full sizes: a fused FP32-sweep LSRK
stage on the GPU, in the launch configuration the benchmark times, against
the sum-factorised FP64 CPU oracle (``oracle/cpu_sumfac.cpp``, all host
cores) evaluated on the same stage vector, element by element against its
term scale M^{-1} |A| |w| (``apply_abs``; the oracle is pinned to the dense
and axis-wise routes, and its term scale to ``Problem.apply_abs``, in
``test_oracle_sumfac.py``).

6D: 8^6 cells, k = 3 (1.07e9 values; the 128-thread pencil kernel), in the
Gauss-Legendre and the Gauss-Lobatto collocation (the face-layer variant).
5D adjoint workload: 12^2 x 8^3 cells (the persistent 5D kernel).
4D at k = 5: 16^4 cells (the pair kernel).
The host holds the stage vector, the oracle's K and term scale, and the GPU's
u and w_out (about 47 GB for 6D): a host with less free memory skips.
"""
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


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def _stage_every_dof(w, stage, state, basis=0, floor_rel=0.0):
    """One FP32-sweep stage of workload ``w`` on the GPU from the FP64 state
    ``state`` (host array), checked value by value against the CPU oracle.
    basis 1: Gauss-Lobatto collocation.  floor_rel: an allowance on K relative
    to the largest term scale (see the Lobatto test)."""
    from oracle.sumfac import SumFac
    from paper_2002_08110_gb300 import DG, PREC_FP32, basis_nodes
    n = w.n_dofs
    if _mem_available_gb() < 48.0 * n / 1.0e9 + 8.0:
        pytest.skip(f"needs ~{48 * n / 1e9 + 8:.0f} GB of free host memory")
    _, qpts, _ = basis_nodes(basis, w.k)
    e = W.e_table(w, qpts)
    dt, _ = W.time_step(w)
    dg = DG(e_nodes=e, basis=basis, **W.dg_kwargs(w))
    assert dg.get_launch(PREC_FP32)["variant"] >= 1
    u = torch.from_numpy(state).to("cuda")
    w_in = u.float()
    w_out = torch.empty_like(w_in)
    uu = u.clone()
    dg.rk_stage(w_in, w_out, uu, stage, dt, prec=PREC_FP32)
    dg.check()
    dg.close()
    win = w_in.double().cpu().numpy()
    u_new = uu.cpu().numpy()
    wo = w_out.cpu().numpy()
    del u, w_in, w_out, uu
    torch.cuda.empty_cache()
    kw = dict(e_nodes=e) if w.field_kind == 1 else dict(a=w.a_const)
    sf = SumFac(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                shear=W.dg_kwargs(w).get("shear"), basis="gllc" if basis == 1 else "gl", **kw)
    K = sf.apply(win)
    S = sf.apply_abs(win)
    sf.close()
    del win
    floor = floor_rel * float(S.max())
    a = lsrk.B[4] if stage == 4 else lsrk.A[stage]
    chunk = 1 << 24
    worst_u = worst_w = 0.0
    for lo in range(0, n, chunk):
        sl = slice(lo, min(n, lo + chunk))
        uo, Kc, Sc = state[sl], K[sl], S[sl]
        u_ref = uo + lsrk.B[stage] * dt * Kc
        w_ref = u_ref if stage == 4 else uo + a * dt * Kc
        # K to 1e-5 of its term scale (the FP32 sweeps), u in FP64 on top
        bound_u = 1e-14 * np.abs(u_ref) + 1e-5 * dt * (Sc + np.abs(Kc)) + dt * floor
        ru = np.abs(u_new[sl] - u_ref) / bound_u
        # w_out adds its own FP32 rounding
        bound_w = bound_u + 2.5e-7 * (np.abs(uo) + np.abs(a * dt * Kc)) + 1e-30
        rw = np.abs(wo[sl].astype(np.float64) - w_ref) / bound_w
        worst_u, worst_w = max(worst_u, float(ru.max())), max(worst_w, float(rw.max()))
        if worst_u > 1.0 or worst_w > 1.0:
            i = lo + int(np.argmax(ru if worst_u > 1.0 else rw))
            raise AssertionError(f"value {i}: error / bound u {worst_u:.3g}, w_out {worst_w:.3g} "
                                 f"(K {K[i]:.3e}, term scale {S[i]:.3e})")
    return worst_u, worst_w


def test_6d_stage_every_value():
    w = W.config_6d()
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    _stage_every_dof(w, 1, W.separable_state(w, zeta))


def test_6d_gauss_lobatto_collocation_stage_every_value():
    """The Lobatto-collocation stage at 8^6 (the face-layer kernel).  Speeds
    below 1e-12 of a cell's largest (v = 0 on Lobatto face nodes, E at its
    zeros) carry no flux in the FP32 tables: entries made only of such terms
    are exact to 1e-12 of the largest term scale."""
    from paper_2002_08110_gb300 import basis_nodes
    w = W.config_6d()
    nodes, _, _ = basis_nodes(1, w.k)
    _stage_every_dof(w, 2, W.separable_state(w, nodes), basis=1, floor_rel=1e-12)


def test_5d_adjoint_workload_stage_every_value():
    w = W.config_adjoint()
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    _stage_every_dof(w, 4, W.initial_state(w, zeta))


def test_4d_k5_stage_every_value():
    w = W.config_4d(k=5)
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    _stage_every_dof(w, 2, W.initial_state(w, zeta))


def test_6d_applies_every_value():
    """The operator alone at 8^6, every value: FP64 (to 1e-12 of the term
    scale), FP32 sweeps with FP64 input and output, and FP32 throughout (to
    1e-5), each against the oracle on the input it was given."""
    from oracle.sumfac import SumFac
    from paper_2002_08110_gb300 import DG, PREC_FP32, PREC_FP64, PREC_MIXED, reference_nodes
    w = W.config_6d()
    n = w.n_dofs
    if _mem_available_gb() < 40.0 * n / 1.0e9 + 8.0:
        pytest.skip(f"needs ~{40 * n / 1e9 + 8:.0f} GB of free host memory")
    zeta = np.polynomial.legendre.leggauss(w.n)[0]
    state = W.separable_state(w, zeta)
    e = W.e_table(w, reference_nodes(w.k)[0])
    dg = DG(e_nodes=e, **W.dg_kwargs(w))
    sf = SumFac(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi, e_nodes=e)
    x64 = torch.from_numpy(state).to("cuda")
    chunk = 1 << 24

    def check(got, K, S, tol, what):
        for lo in range(0, n, chunk):
            sl = slice(lo, min(n, lo + chunk))
            r = np.abs(got[sl].astype(np.float64) - K[sl]) / (tol * S[sl] + 1e-300)
            if r.max() > 1.0:
                i = lo + int(np.argmax(r))
                raise AssertionError(f"{what}: value {i}: error {abs(got[i] - K[i]):.3e}, "
                                     f"term scale {S[i]:.3e}, bound {tol:g}")

    K, S = sf.apply(state), sf.apply_abs(state)
    for prec, tol, what in ((PREC_FP64, 1e-12, "FP64 apply"), (PREC_MIXED, 1e-5, "FP32 sweeps, FP64 I/O")):
        out = dg.apply(x64, prec=prec)
        dg.check()
        check(out.cpu().numpy(), K, S, tol, what)
        del out
    x32 = x64.float()
    del x64
    src32 = x32.double().cpu().numpy()
    K, S = sf.apply(src32, K), sf.apply_abs(src32, S)
    out = dg.apply(x32, prec=PREC_FP32)
    dg.check()
    check(out.cpu().numpy(), K, S, 1e-5, "FP32 apply")
    sf.close()
    dg.close()
