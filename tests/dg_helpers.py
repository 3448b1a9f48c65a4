"""Shared helpers of the GPU tests: build the library handle and the oracle
problem for the same synthetic inputs.  Inputs (fields, states) are computed
from the oracle's own node coordinates or seeded generators, never from the
CUDA path."""
import numpy as np

import workloads as W
from oracle.dg import ConstantField, PhaseSpaceField, Problem


def e_table_from_oracle(p, E):
    """E at the x nodes in the library's layout (x-cell, x-node, component),
    evaluated at the oracle's node coordinates."""
    dx, dv, n = p.dx, p.dv, p.n
    ncx = int(np.prod(p.cells[:dx]))
    tab = np.zeros((ncx, n ** dx, dv))
    for e in range(ncx):                      # cells e < ncx have c_v = 0
        yx, _ = p.node_coordinates(e)
        sub = yx[tuple([slice(None)] * dx + [0] * dv)]
        tab[e] = E(sub.reshape(-1, dx, order="F"))
    return tab


def oracle_for(w, basis="gl"):
    field = (ConstantField(w.a_const) if w.field_kind == 0
             else PhaseSpaceField(w.dx, w.dv, W.e_function(w)))
    shear = None if w.shear is None else np.array(w.shear).reshape(w.dx, w.dx)
    return Problem(w.dx, w.dv, w.k, w.cells_x, w.cells_v, w.x_lo, w.x_hi, w.v_lo, w.v_hi,
                   field, shear=shear, basis=basis)


def dg_for(w, p=None):
    from paper_2002_08110_gb300 import DG
    p = p or oracle_for(w)
    e = None
    if w.field_kind == 1:
        e = e_table_from_oracle(p, W.e_function(w))
    return DG(e_nodes=e, **W.dg_kwargs(w)), p


def random_problem(dx, dv, k, cells, kind, seed=0, shear=None):
    """A (library handle, oracle problem) pair with a seeded random field."""
    from paper_2002_08110_gb300 import DG
    rng = np.random.default_rng(seed)
    d = dx + dv
    x_lo, x_hi = [0.0] * dx, [1.0] * dx
    v_lo, v_hi = [-1.0] * dv, [1.5] * dv
    if kind == "const":
        a = rng.uniform(-1, 1, d)
        p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi,
                    ConstantField(a), shear=shear)
        dg = DG(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, field_kind=0,
                a_const=a, shear=shear)
        return dg, p
    amp = rng.uniform(0.3, 1.0, dv)
    ph = rng.uniform(0, 1, dv)

    def E(yx):
        s = np.asarray(yx).sum(-1, keepdims=True)
        return amp * np.sin(2 * np.pi * (s + ph))
    p = Problem(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi,
                PhaseSpaceField(dx, dv, E), shear=shear)
    dg = DG(dx, dv, k, cells[:dx], cells[dx:], x_lo, x_hi, v_lo, v_hi, field_kind=1,
            e_nodes=e_table_from_oracle(p, E), shear=shear)
    return dg, p


def assert_term_scale(got, ref, scale, tol, floor=1e-300, what=""):
    """Element by element: |got_i - ref_i| <= tol * scale_i + floor, where
    scale is the term scale of each entry (the oracle's evaluation with the
    absolute value of every factor, ``Problem.apply_abs``): rounding errors
    of an entry scale with the terms that entry sums, not with the entry or
    the norm of the whole vector.  Reports the worst entry on failure."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    scale = np.abs(np.asarray(scale, dtype=np.float64)).reshape(-1)
    err = np.abs(got - ref)
    bound = tol * scale + floor
    bad = err > bound
    if np.any(bad):
        i = int(np.argmax(err / bound))
        raise AssertionError(
            f"{what}: {int(bad.sum())} of {err.size} entries exceed tol {tol:g} x term scale; "
            f"worst index {i}: |err| {err[i]:.3e}, scale {scale[i]:.3e}, ratio "
            f"{err[i] / max(scale[i], 1e-300):.3e}")
