"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times, on sampled cells the oracle evaluates one by one, and an
invariant that holds at any size.

6D: 8^6 cells, k = 3 (1.07e9 DoFs), the specialised kernel: fused LSRK stage
(FP32 sweeps, FP32 stage vector, FP64 state), FP32 apply and FP64-I/O apply.
4D: 16^4 cells, sheared, FP64 apply and the 4D kernel's FP32-sweep stage.
5D adjoint workload: L^T on a sampled cell against the oracle's transposed
blocks.  Mass conservation of FP64 steps
on the full 6D mesh.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from dg_helpers import assert_term_scale, oracle_for  # noqa: E402
from oracle import lsrk  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()


class DeviceVector:
    """Read-only view of a device tensor for the oracle: slices are copied to
    the host on demand, so only the cells the oracle touches move."""

    def __init__(self, t):
        self.t = t
        self.shape = (t.numel(),)

    def __getitem__(self, s):
        return self.t[s].double().cpu().numpy()


def _sample_cells(p, count, seed):
    """``count`` random cells plus every corner of the cell grid (2^d cells
    whose neighbours wrap around the periodic boundary in every direction)."""
    rng = np.random.default_rng(seed)
    cells = set(int(c) for c in rng.choice(p.ncells, size=count, replace=False))
    for corner in np.ndindex(*([2] * p.d)):
        cells.add(p.cell_index([(p.cells[j] - 1) * corner[j] for j in range(p.d)]))
    return sorted(cells)


def _sample_cells_6d(p, seed):
    """Cells chosen for the paths of the 6D kernel (x1..x3, v1..v3 cell
    coordinates; pencils are the lines of cells along v3, walked from the
    upwind end, in tiles of 2 cells per direction of the other five):
      * all 2^6 corners (wrap-around neighbours in every direction);
      * four whole pencils, two walked forwards (E_3 > 0: x3 cells 0..3) and two
        backwards (x3 cells 4..7): the first cell of each reads its upwind v3
        neighbour, the other seven take the carried traces; v3 = 0 and v3 = 7
        are also the edge slabs of the host-buffer pipeline;
      * cells with every other coordinate on a pencil-tile boundary (1|2, 3|4,
        5|6 and the wrap 7|0);
      * random cells."""
    rng = np.random.default_rng(seed)
    N = p.cells
    cells = set()
    for corner in np.ndindex(*([2] * 6)):
        cells.add(p.cell_index([(N[j] - 1) * corner[j] for j in range(6)]))
    for x3 in (1, 2, 5, 6):
        c5 = list(rng.integers(0, N[:5]))
        c5[2] = x3
        for v3 in range(N[5]):
            cells.add(p.cell_index(c5 + [v3]))
    for _ in range(8):
        cc = [int(rng.choice([1, 2, 3, 4, 5, 6, 7, 0])) for _ in range(5)] + [int(rng.integers(N[5]))]
        cells.add(p.cell_index(cc))
    for c in rng.choice(p.ncells, size=8, replace=False):
        cells.add(int(c))
    return sorted(cells)


def _oracle_cells(p, u, cells):
    K = [p.apply_mass_inverse(p.cell_residual(u, e)).reshape(-1, order="F") for e in cells]
    S = [p.apply_mass_inverse(p.cell_residual(u, e, absolute=True)).reshape(-1, order="F")
         for e in cells]
    return K, S


@pytest.fixture(scope="module")
def six():
    from paper_2002_08110_gb300 import DG, reference_nodes
    w = W.config_6d()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    assert dg.info.uniform_sides == 1          # the specialised kernel runs
    # the oracle evaluates the same field and state functions at its own nodes
    p = oracle_for(w)
    u = W.separable_state(w, zeta, xp=torch, device="cuda")
    yield w, dg, p, u
    dg.close()


def test_6d_fused_stage_sampled(six):
    from paper_2002_08110_gb300 import PREC_FP32
    w, dg, p, u = six
    npc = p.dofs_per_cell
    dt, _ = W.time_step(w)
    w_in = u.float()
    w_out = torch.empty_like(w_in)
    uu = u.clone()
    stage = 1
    dg.rk_stage(w_in, w_out, uu, stage, dt, prec=PREC_FP32)
    dg.check()
    cells = _sample_cells_6d(p, seed=0)
    assert len(cells) >= 64
    _check_stage_cells(p, u, uu, w_out, DeviceVector(w_in), cells, stage, dt)


def _check_stage_cells(p, u, uu, w_out, w_in, cells, stage, dt, floor_rel=0.0):
    """Element by element on the sampled cells: u_new = u + b_s dt K and
    w_out = u + a_s dt K with K from the oracle; the error of K is bounded by
    1e-5 of its term scale, w_out adds its own FP32 rounding.  ``floor_rel``:
    an absolute allowance on K, relative to the largest term scale (see the
    Gauss-Lobatto test)."""
    npc = p.dofs_per_cell
    K, S = _oracle_cells(p, w_in, cells)
    floor = floor_rel * max(float(np.max(np.abs(Se))) for Se in S)
    for e, Ke, Se in zip(cells, K, S):
        sl = slice(e * npc, (e + 1) * npc)
        u_old = u[sl].cpu().numpy()
        u_ref = u_old + lsrk.B[stage] * dt * Ke
        w_ref = u_old + lsrk.A[stage] * dt * Ke
        bound_u = 1e-14 * np.abs(u_ref) + 1e-5 * dt * (np.abs(Se) + np.abs(Ke)) + dt * floor
        assert_term_scale(uu[sl].cpu().numpy(), u_ref, bound_u, 1.0, what=f"u, cell {e}")
        bound_w = bound_u + 2.5e-7 * (np.abs(u_old) + np.abs(lsrk.A[stage] * dt * Ke))
        assert_term_scale(w_out[sl].double().cpu().numpy(), w_ref, bound_w, 1.0,
                          floor=1e-30, what=f"w_out, cell {e}")


@pytest.mark.parametrize("prec", [1, 2])
def test_6d_apply_sampled(six, prec):
    w, dg, p, u = six
    npc = p.dofs_per_cell
    src = u.float() if prec == 1 else u
    out = dg.apply(src, prec=prec)
    dg.check()
    cells = _sample_cells_6d(p, seed=1)
    K, S = _oracle_cells(p, DeviceVector(src), cells)
    for e, Ke, Se in zip(cells, K, S):
        got = out[e * npc:(e + 1) * npc].double().cpu().numpy()
        assert_term_scale(got, Ke, Se, 1e-5, what=f"prec {prec} apply, cell {e}")


def test_6d_host_buffer_stage_sampled(six):
    """The host-buffer stage (pipelined over the slabs of v3 cells) at the
    full size: sampled cells, including both edge slabs (v3 = 0 and 7) of
    pencils walked in both directions, against the oracle."""
    from paper_2002_08110_gb300 import PREC_FP32
    w, dg, p, u = six
    dt, _ = W.time_step(w)
    stage = 2
    h_w = u.float().cpu().pin_memory()
    h_out = torch.empty_like(h_w).pin_memory()
    h_u = u.cpu().pin_memory()
    dg.rk_stage_host(h_w, h_out, h_u, stage, dt, prec=PREC_FP32)
    torch.cuda.synchronize()
    dg.check()
    cells = [c for c in _sample_cells_6d(p, seed=6) if (c // 32768) in (0, 1, 6, 7)]
    assert len(cells) >= 32
    _check_stage_cells(p, u, h_u, h_out, DeviceVector(h_w), cells, stage, dt)
    del h_w, h_out, h_u


def test_6d_mass_conserved_fp64(six):
    from paper_2002_08110_gb300 import PREC_FP64
    w, dg, p, u = six
    dt, _ = W.time_step(w)
    x = u.clone()
    m0, l0, _ = dg.integrals(x)
    dg.rk_step(x, dt, nsteps=1, prec=PREC_FP64)
    dg.check()
    m1, l1, _ = dg.integrals(x)
    assert abs(m1 - m0) <= 1e-12 * abs(m0)
    assert l1 <= l0 * (1 + 1e-13)


def test_4d_fullsize_apply_sampled():
    from paper_2002_08110_gb300 import DG, PREC_FP64, reference_nodes
    w = W.config_4d()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    p = oracle_for(w)
    u = torch.tensor(W.initial_state(w, zeta), device="cuda")
    out = dg.apply(u, prec=PREC_FP64)
    dg.check()
    npc = p.dofs_per_cell
    cells = _sample_cells(p, 20, seed=2)
    K, S = _oracle_cells(p, DeviceVector(u), cells)
    for e, Ke, Se in zip(cells, K, S):
        got = out[e * npc:(e + 1) * npc].cpu().numpy()
        assert np.linalg.norm(got - Ke) <= 1e-12 * np.linalg.norm(Ke)
        assert_term_scale(got, Ke, Se, 1e-12, what=f"fp64 apply, cell {e}")
    dg.close()


def test_4d_fullsize_stage_fp32_sampled():
    """The 4D kernel (the default for dim_x = dim_v = 2) at the 4D workload's
    full size: a fused FP32-sweep stage on sampled cells."""
    from paper_2002_08110_gb300 import DG, PREC_FP32, reference_nodes
    w = W.config_4d()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    assert dg.get_launch(PREC_FP32)["variant"] == 2
    p = oracle_for(w)
    u = torch.tensor(W.initial_state(w, zeta), device="cuda")
    w_in = u.float()
    w_out = torch.empty_like(w_in)
    uu = u.clone()
    dt, _ = W.time_step(w)
    stage = 3
    dg.rk_stage(w_in, w_out, uu, stage, dt, prec=PREC_FP32)
    dg.check()
    npc = p.dofs_per_cell
    cells = _sample_cells(p, 20, seed=3)
    _check_stage_cells(p, u, uu, w_out, DeviceVector(w_in), cells, stage, dt)
    dg.close()


def test_5d_fullsize_stage_fp32_sampled():
    """The persistent 5D kernel at the 5D workload's full size (73,728 cells,
    each block walks ~80 of them with the next cell's copies in flight; E_3
    changes sign inside a third of the x cells, and its v3 neighbours are read
    per thread): a fused FP32-sweep stage on all 2^5 corner cells and 40
    random ones."""
    from paper_2002_08110_gb300 import DG, PREC_FP32, reference_nodes
    w = W.config_adjoint()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    assert dg.get_launch(PREC_FP32)["variant"] == 2
    p = oracle_for(w)
    u = torch.tensor(W.initial_state(w, zeta), device="cuda")
    w_in = u.float()
    w_out = torch.empty_like(w_in)
    uu = u.clone()
    dt, _ = W.time_step(w)
    stage = 2
    dg.rk_stage(w_in, w_out, uu, stage, dt, prec=PREC_FP32)
    dg.check()
    cells = _sample_cells(p, 40, seed=7)
    _check_stage_cells(p, u, uu, w_out, DeviceVector(w_in), cells, stage, dt)
    dg.close()


def test_5d_adjoint_fullsize_sampled():
    from paper_2002_08110_gb300 import DG, PREC_FP32, reference_nodes
    w = W.config_adjoint()
    zeta, _ = reference_nodes(w.k)
    dg = DG(e_nodes=W.e_table(w, zeta), **W.dg_kwargs(w))
    p = oracle_for(w)
    y = torch.tensor(W.initial_state(w, zeta), device="cuda", dtype=torch.float32)
    out = dg.apply_adjoint(y, prec=PREC_FP32)
    dg.check()
    npc = p.dofs_per_cell
    yv = DeviceVector(y)
    e = 12345
    rows = {e} | {p.neighbour(e, j, s) for j in range(p.d) for s in (1, -1)}
    ref = np.zeros(npc)
    scale = np.zeros(npc)
    for r in rows:
        blocks = p.dense_cell_blocks(r)
        if e in blocks:
            yr = yv[slice(r * npc, (r + 1) * npc)]
            ref += blocks[e].T @ yr
            scale += np.abs(blocks[e].T) @ np.abs(yr)
    got = out[e * npc:(e + 1) * npc].double().cpu().numpy()
    assert_term_scale(got, ref, scale, 4e-5, what="5D adjoint cell")
    dg.close()


def test_6d_gll_collocation_stage_sampled():
    """The Lobatto-collocation stage at 8^6 (face-layer kernel) on sampled
    cells against the oracle's gllc operator."""
    from paper_2002_08110_gb300 import DG, PREC_FP32, basis_nodes
    from oracle.dg import PhaseSpaceField, Problem
    w = W.config_6d()
    nodes, qpts, _ = basis_nodes(1, w.k)
    dg = DG(e_nodes=W.e_table(w, qpts), basis=1, **W.dg_kwargs(w))
    assert dg.info.uniform_sides == 1
    p = Problem(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                PhaseSpaceField(w.dx, w.dv, W.e_function(w)), basis="gllc")
    u = W.separable_state(w, nodes, xp=torch, device="cuda")
    npc = p.dofs_per_cell
    dt, _ = W.time_step(w)
    w_in = u.float()
    w_out = torch.empty_like(w_in)
    uu = u.clone()
    stage = 2
    dg.rk_stage(w_in, w_out, uu, stage, dt, prec=PREC_FP32)
    dg.check()
    cells = _sample_cells_6d(p, seed=4)
    # speeds below 1e-12 of a cell's largest (v = 0 on Lobatto face nodes, E at
    # its zeros) carry no flux in the FP32 tables: entries made only of such
    # terms are exact to 1e-12 of the largest term scale
    _check_stage_cells(p, u, uu, w_out, DeviceVector(w_in), cells, stage, dt, floor_rel=1e-12)
    dg.close()


def test_6d_deltaf_apply_sampled(six):
    """The delta-f operator at 8^6 around the Maxwellian: plain relative error
    against the oracle on sampled cells below 1e-5 of the sampled K."""
    w, dg, p, u = six
    from paper_2002_08110_gb300 import reference_nodes
    zeta, _ = reference_nodes(w.k)
    u_eq = W.separable_state(W.equilibrium_6d(w), zeta, xp=torch, device="cuda")
    dg.set_reference(u_eq)
    k = dg.apply_df(u)
    dg.check()
    npc = p.dofs_per_cell
    cells = _sample_cells(p, 3, seed=5)[::4]
    K, _ = _oracle_cells(p, DeviceVector(u), cells)
    got = np.concatenate([k[e * npc:(e + 1) * npc].cpu().numpy() for e in cells])
    ref = np.concatenate(K)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    del k, u_eq
