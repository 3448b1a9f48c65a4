"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only states the problems
(mesh sizes, boxes, velocity fields, initial states, seeds, step counts) and
evaluates user-level functions at coordinates that the caller supplies.  Node
positions come from whichever side uses the workload (the oracle's own tables,
or the CUDA library's exported reference nodes), so neither side depends on
the other.

The shapes follow the paper's experiments (hypercube meshes of degree 3 in
2 to 6 dimensions, phase-space velocity fields a = (v, E(x)); Sec. 5.1 and
Sec. 6), at sizes chosen for one GPU.  No public dataset is involved; every
input is synthetic and seeded.
"""
from dataclasses import dataclass, field, replace
import math

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass
class Workload:
    name: str
    dx: int
    dv: int
    k: int
    cells_x: tuple
    cells_v: tuple
    x_lo: tuple
    x_hi: tuple
    v_lo: tuple
    v_hi: tuple
    field_kind: int                      # 0: constant a, 1: a = (v[:dx], E(y_x))
    a_const: tuple = ()
    E: object = None                     # callable: (yx1, ..., yx_dx) -> list of dv arrays
    shear: tuple = None                  # row-major dx*dx, None = identity
    u0_factors: tuple = ()               # d callables, u0 = prod_j f_j(y_j)
    noise_amp: float = 0.0
    noise_seed: int = 0
    steps: int = 1
    final_time: float = None             # if set, steps are derived from it
    cfl: float = 0.2
    amax: tuple = ()                     # max |a_j| over the domain, per dimension
    extra: dict = field(default_factory=dict)

    @property
    def d(self):
        return self.dx + self.dv

    @property
    def n(self):
        return self.k + 1

    @property
    def cells(self):
        return tuple(self.cells_x) + tuple(self.cells_v)

    @property
    def lo(self):
        return tuple(self.x_lo) + tuple(self.v_lo)

    @property
    def hi(self):
        return tuple(self.x_hi) + tuple(self.v_hi)

    @property
    def h(self):
        return tuple((b - a) / c for a, b, c in zip(self.lo, self.hi, self.cells))

    @property
    def ncells(self):
        return int(np.prod(self.cells))

    @property
    def n_dofs(self):
        return self.ncells * self.n ** self.d


# -- time step: CFL recipe ----------------------------------------------------
def time_step(w: Workload):
    """dt = CFL * min(1, (4/(k+1))^2) / sum_j max|a_j| / h_j, then shortened so
    that an integer number of steps reaches ``final_time`` (if given)."""
    rate = sum(a / h for a, h in zip(w.amax, w.h))
    dt = w.cfl * min(1.0, (4.0 / (w.k + 1)) ** 2) / rate
    if w.final_time is not None:
        steps = int(math.ceil(w.final_time / dt - 1e-9))
        return w.final_time / steps, steps
    return dt, w.steps


# -- evaluation at caller-supplied node positions -----------------------------
def axis_coordinates(w: Workload, zeta):
    """Per-dimension coordinates of all nodes, shape (cells_j, n) each
    (lattice coordinates in x, velocity coordinates in v)."""
    zeta = np.asarray(zeta, dtype=np.float64)
    out = []
    for j in range(w.d):
        c = np.arange(w.cells[j], dtype=np.float64)[:, None]
        out.append(w.lo[j] + w.h[j] * (c + (zeta[None, :] + 1.0) / 2.0))
    return out


def separable_state(w: Workload, zeta, xp=np, device=None, dtype=None):
    """u0 = prod_j f_j(y_j) at all nodes, flat in the library's vector layout
    (index = cell * n^d + q; cells and nodes lexicographic, first dimension
    fastest).  ``xp`` is numpy or torch (then ``device``/``dtype`` apply)."""
    d, n = w.d, w.n
    coords = axis_coordinates(w, zeta)
    # C-order tensor with axes (c_d, ..., c_1, q_d, ..., q_1): the flat index
    # is then cell * n^d + q with the first dimension fastest in both parts.
    out = None
    for j in range(d):
        vals = np.asarray(w.u0_factors[j](coords[j]), dtype=np.float64).reshape(w.cells[j], n)
        full = [1] * (2 * d)
        full[d - 1 - j] = w.cells[j]
        full[2 * d - 1 - j] = n
        if xp is np:
            t = _place(vals, full, d - 1 - j, 2 * d - 1 - j)
        else:
            t = xp.as_tensor(_place(vals, full, d - 1 - j, 2 * d - 1 - j),
                             device=device, dtype=dtype or xp.float64)
        out = t if out is None else out * t
    full_shape = [w.cells[j] for j in reversed(range(d))] + [n] * d
    if xp is np:
        return np.broadcast_to(out, full_shape).reshape(-1).copy()
    return out.expand(full_shape).reshape(-1).contiguous()


def _place(vals, full, axis_c, axis_q):
    """Reshape vals[c, q] into a tensor of shape ``full`` whose only
    non-singleton axes are axis_c (cells) and axis_q (nodes)."""
    t = vals.reshape(vals.shape[0], 1, vals.shape[1])
    # t axes: (c, gap, q); build the full shape with c at axis_c and q at axis_q
    return t.reshape([1] * axis_c + [vals.shape[0]] + [1] * (axis_q - axis_c - 1)
                     + [vals.shape[1]] + [1] * (len(full) - axis_q - 1))


def noise(w: Workload):
    """Seeded uniform noise U(-1, 1) * amp per DoF (numpy, FP64), or None."""
    if w.noise_amp == 0.0:
        return None
    rng = np.random.default_rng(w.noise_seed)
    return w.noise_amp * rng.uniform(-1.0, 1.0, w.n_dofs)


def initial_state(w: Workload, zeta):
    """Full initial state on the host (numpy FP64): separable part + noise."""
    u = separable_state(w, zeta)
    z = noise(w)
    return u if z is None else u + z


def e_table(w: Workload, zeta):
    """E at every x-node, layout (x-cell, x-node, component), x-cells and
    x-nodes lexicographic with x_1 fastest (numpy FP64).  Zero for
    constant-velocity workloads."""
    zeta = np.asarray(zeta, dtype=np.float64)
    dx, dv, n = w.dx, w.dv, w.n
    if w.field_kind != 1:
        return None
    coords = axis_coordinates(w, zeta)[:dx]       # each (cells_j, n)
    # grid over (c_x lexicographic) x (q_x lexicographic), x_1 fastest
    cx_grid = np.meshgrid(*[np.arange(w.cells_x[j]) for j in range(dx)], indexing="ij")
    cx_flat = [g.reshape(-1, order="F") for g in cx_grid]
    q_grid = np.meshgrid(*[np.arange(n) for _ in range(dx)], indexing="ij")
    q_flat = [g.reshape(-1, order="F") for g in q_grid]
    ys = [coords[j][cx_flat[j][:, None], q_flat[j][None, :]] for j in range(dx)]
    comps = w.E(*ys)
    return np.stack([np.asarray(c, dtype=np.float64) * np.ones_like(ys[0]) for c in comps], axis=-1)


def e_function(w: Workload):
    """E as a function of lattice x-coordinates (..., dx) -> (..., dv)."""
    def E(yx):
        comps = w.E(*[yx[..., j] for j in range(w.dx)])
        return np.stack([np.asarray(c, dtype=np.float64) * np.ones(yx.shape[:-1]) for c in comps],
                        axis=-1)
    return E


def dg_kwargs(w: Workload):
    """Constructor arguments of the library's problem handle (plain data)."""
    return dict(dim_x=w.dx, dim_v=w.dv, degree=w.k, cells_x=tuple(w.cells_x),
                cells_v=tuple(w.cells_v), x_lo=tuple(w.x_lo), x_hi=tuple(w.x_hi),
                v_lo=tuple(w.v_lo), v_hi=tuple(w.v_hi), field_kind=w.field_kind,
                a_const=tuple(w.a_const) if w.field_kind == 0 else None,
                shear=None if w.shear is None else np.array(w.shear).reshape(w.dx, w.dx))


# -- the five problems --------------------------------------------------------
def _sin2pi(y):
    return np.sin(TWO_PI * y)


def _gauss(mu, sigma):
    return lambda y: np.exp(-((y - mu) ** 2) / (2.0 * sigma * sigma))


def config_2d(cells=16):
    """2D (1x + 1v), k = 3, 16 x 16 cells on [0,1]^2, a = (1, 0.5),
    u0 = sin(2 pi x) sin(2 pi v), one period T = 2, CFL 0.2."""
    return Workload(
        name="2d_k3_16x16", dx=1, dv=1, k=3, cells_x=(cells,), cells_v=(cells,),
        x_lo=(0.0,), x_hi=(1.0,), v_lo=(0.0,), v_hi=(1.0,),
        field_kind=0, a_const=(1.0, 0.5),
        u0_factors=(_sin2pi, _sin2pi), final_time=2.0, cfl=0.2, amax=(1.0, 0.5))


def _E4(y1, y2):
    return [0.1 * np.sin(TWO_PI * y1), 0.1 * np.cos(TWO_PI * y2)]


def config_4d(cells=16, k=3):
    """4D (2x + 2v), 16^2 x 16^2 cells, x in [0,1]^2 sheared by 0.1,
    v in [0,1]^2, a = (v, 0.1 (sin 2 pi y1, cos 2 pi y2)); u0 = Gaussian
    product (sigma 0.1, centred) + 1e-2 U(-1,1) noise (seed 0); 200 steps."""
    g = _gauss(0.5, 0.1)
    return Workload(
        name=f"4d_k{k}_{cells}^4_shear0.1", dx=2, dv=2, k=k,
        cells_x=(cells, cells), cells_v=(cells, cells),
        x_lo=(0.0, 0.0), x_hi=(1.0, 1.0), v_lo=(0.0, 0.0), v_hi=(1.0, 1.0),
        field_kind=1, E=_E4, shear=(1.0, 0.1, 0.0, 1.0),
        u0_factors=(g, g, g, g), noise_amp=1e-2, noise_seed=0, steps=200, cfl=0.2,
        amax=(1.1, 1.0, 0.1, 0.1))


def _E6(y1, y2, y3):
    return [0.05 * np.sin(TWO_PI * y1), 0.05 * np.sin(TWO_PI * y2), 0.05 * np.sin(TWO_PI * y3)]


def config_6d(cells=8, k=3):
    """6D (3x + 3v), 8^3 x 8^3 cells, x in [0,1]^3, v in [-6,6]^3,
    a = (v, 0.05 sin 2 pi x_i); u0 = Maxwellian in v times (1 + 0.01 cos 2 pi x1);
    50 steps."""
    maxw = lambda y: np.exp(-0.5 * y * y) / math.sqrt(TWO_PI)
    one = lambda y: np.ones_like(y)
    return Workload(
        name=f"6d_k{k}_{cells}^6", dx=3, dv=3, k=k,
        cells_x=(cells,) * 3, cells_v=(cells,) * 3,
        x_lo=(0.0,) * 3, x_hi=(1.0,) * 3, v_lo=(-6.0,) * 3, v_hi=(6.0,) * 3,
        field_kind=1, E=_E6,
        u0_factors=(lambda y: 1.0 + 0.01 * np.cos(TWO_PI * y), one, one, maxw, maxw, maxw),
        steps=50, cfl=0.2, amax=(6.0, 6.0, 6.0, 0.05, 0.05, 0.05))


def equilibrium_6d(w: Workload):
    """The 6D workload's spatially uniform Maxwellian (its state without the
    1% density perturbation): the reference state of the delta-f form."""
    one = lambda y: np.ones_like(y)
    return Workload(**{**w.__dict__, "u0_factors": (one,) + tuple(w.u0_factors[1:])})


def _E5(y1, y2):
    return [0.1 * np.sin(TWO_PI * y1), 0.1 * np.cos(TWO_PI * y2), 0.1 * np.sin(TWO_PI * (y1 + y2))]


def config_adjoint(cells_x=12, cells_v=8, noise_seed=2):
    """5D (2x + 3v), 12^2 x 8^3 cells, k = 3, x in [0,1]^2, v in [-1,1]^3,
    a = ((v1, v2), 0.1 (sin 2 pi y1, cos 2 pi y2, sin 2 pi (y1 + y2)));
    u0 = Gaussian product sigma 0.1 centred in the box; the target comes from
    the perturbed state u0 + 1e-2 U(-1,1) (seed 2); 200 steps, checkpoint
    every 20."""
    gx = _gauss(0.5, 0.1)
    gv = _gauss(0.0, 0.1)
    return Workload(
        name=f"5d_k3_{cells_x}^2x{cells_v}^3_adjoint", dx=2, dv=3, k=3,
        cells_x=(cells_x,) * 2, cells_v=(cells_v,) * 3,
        x_lo=(0.0, 0.0), x_hi=(1.0, 1.0), v_lo=(-1.0,) * 3, v_hi=(1.0,) * 3,
        field_kind=1, E=_E5,
        u0_factors=(gx, gx, gv, gv, gv), noise_amp=1e-2, noise_seed=noise_seed,
        steps=200, cfl=0.2, amax=(1.0, 1.0, 0.1, 0.1, 0.1),
        extra={"checkpoint_every": 20})


def batched_instances(count=64, seed=1, cells_lo=8, cells_hi=24):
    """``count`` independent constant-velocity problems: d alternates between
    3 (2x + 1v) and 4 (2x + 2v); k ~ U{2..5}; cells per direction ~
    U{cells_lo..cells_hi}; a ~ U[-1, 1]^d; u0 = prod sin(2 pi y_j) on [0,1]^d."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dv = 1 if i % 2 == 0 else 2
        dx = 2
        d = dx + dv
        k = int(rng.integers(2, 6))
        cells = tuple(int(c) for c in rng.integers(cells_lo, cells_hi + 1, size=d))
        a = tuple(float(x) for x in rng.uniform(-1.0, 1.0, size=d))
        out.append(Workload(
            name=f"batch{i}_{d}d_k{k}", dx=dx, dv=dv, k=k,
            cells_x=cells[:dx], cells_v=cells[dx:],
            x_lo=(0.0,) * dx, x_hi=(1.0,) * dx, v_lo=(0.0,) * dv, v_hi=(1.0,) * dv,
            field_kind=0, a_const=a, u0_factors=tuple([_sin2pi] * d),
            steps=1, cfl=0.2, amax=tuple(abs(x) for x in a)))
    return out


def shrink(w: Workload, cells_x=None, cells_v=None, k=None):
    """The same problem on a smaller mesh (parity-test sizes)."""
    cx = tuple(cells_x) if cells_x is not None else w.cells_x
    cv = tuple(cells_v) if cells_v is not None else w.cells_v
    return replace(w, cells_x=cx, cells_v=cv, k=w.k if k is None else k,
                   name=w.name + f"_small{cx}x{cv}")
