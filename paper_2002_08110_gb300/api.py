"""Python binding of the DG advection library (argument marshalling only).

``DG`` wraps one ``dg_handle``; vectors are torch CUDA tensors owned by the
caller.  Every numerical step runs in ``libdg.so``; if the library is missing
the import fails (no CPU fallback exists).
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import BASIS_GL, PREC_FP32, PREC_FP64, PREC_MIXED, DGError, check

_WDTYPE = {PREC_FP64: torch.float64, PREC_FP32: torch.float32, PREC_MIXED: torch.float64}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def basis_nodes(basis, degree):
    """(DoF nodes, quadrature points, quadrature weights) of a basis (numpy)."""
    lib = _lib.load()
    arrs = [np.zeros(degree + 1) for _ in range(3)]
    check(lib.dg_basis_nodes(int(basis), int(degree),
                             *[a.ctypes.data_as(_lib.c_double_p) for a in arrs]))
    return tuple(arrs)


def reference_nodes(degree):
    """Gauss-Legendre nodes and weights of the library (numpy, FP64)."""
    lib = _lib.load()
    x = np.zeros(degree + 1)
    w = np.zeros(degree + 1)
    check(lib.dg_reference_nodes(degree, x.ctypes.data_as(_lib.c_double_p),
                                 w.ctypes.data_as(_lib.c_double_p)))
    return x, w


class DG:
    """One advection problem on the tensor product of an x mesh and a v mesh.

    field_kind 0: constant velocity ``a_const`` (d entries);
    field_kind 1: a = (v[:dim_x], E(x)) with ``e_nodes`` of shape
    (n_xcells, (k+1)^dim_x, dim_v) at the x nodes (``node_coordinates(0)``).
    ``shear``: dim_x x dim_x matrix S of x = S y (None: identity).
    """

    def __init__(self, dim_x, dim_v, degree, cells_x, cells_v, x_lo, x_hi, v_lo, v_hi,
                 field_kind=0, a_const=None, e_nodes=None, shear=None, basis=BASIS_GL,
                 deform=None):
        self.lib = _lib.load()
        self.dim_x, self.dim_v, self.degree = int(dim_x), int(dim_v), int(degree)
        g = _lib.Geometry()
        for j in range(self.dim_x):
            g.x_lo[j], g.x_hi[j] = float(x_lo[j]), float(x_hi[j])
        for j in range(self.dim_v):
            g.v_lo[j], g.v_hi[j] = float(v_lo[j]), float(v_hi[j])
        if shear is not None:
            S = np.asarray(shear, dtype=np.float64).reshape(self.dim_x, self.dim_x)
            for i in range(self.dim_x):
                for m in range(self.dim_x):
                    g.shear_x[i * self.dim_x + m] = S[i, m]
        g.field_kind = int(field_kind)
        g.basis = int(basis)
        if deform is not None:
            for j, dl in enumerate(deform):
                g.deform[j] = float(dl)
        self.basis = int(basis)
        if a_const is not None:
            for j, a in enumerate(a_const):
                g.a_const[j] = float(a)
        self._e_keep = None
        if e_nodes is not None:
            self._e_keep = np.ascontiguousarray(e_nodes, dtype=np.float64).reshape(-1)
            g.e_nodes = self._e_keep.ctypes.data_as(_lib.c_double_p)
        cx = (ctypes.c_int * self.dim_x)(*[int(c) for c in cells_x])
        cv = (ctypes.c_int * self.dim_v)(*[int(c) for c in cells_v])
        h = ctypes.c_void_p()
        check(self.lib.dg_create(self.dim_x, self.dim_v, self.degree, cx, cv, ctypes.byref(g),
                                 ctypes.byref(h)))
        self.handle = h
        info = _lib.Info()
        check(self.lib.dg_info(self.handle, ctypes.byref(info)))
        self.info = info
        self.n_dofs = int(info.n_dofs)
        self.n_cells = int(info.n_cells)
        self.dofs_per_cell = int(info.dofs_per_cell)

    # -- lifetime --------------------------------------------------------------
    def close(self):
        """Release the handle (dg_destroy); idempotent."""
        if getattr(self, "handle", None):
            self.lib.dg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -----------------------------------------------------------------
    def node_coordinates(self, space):
        """x nodes (space 0, lattice coordinates), v nodes (space 1), the x / v
        quadrature points (spaces 2, 3; the nodes except for the GLL-Gauss
        basis), or the physical coordinates of the x nodes (space 4)."""
        if space % 2 == 0:
            rows, cols = int(self.info.n_xcells) * (self.degree + 1) ** self.dim_x, self.dim_x
        else:
            rows, cols = int(self.info.n_vcells) * (self.degree + 1) ** self.dim_v, self.dim_v
        out = np.zeros((rows, cols))
        check(self.lib.dg_node_coordinates(self.handle, space, out.ctypes.data_as(_lib.c_double_p)))
        return out

    def set_field(self, e_nodes):
        """Replace the phase-space field's E at the x quadrature nodes (host
        array, layout of ``node_coordinates(2)`` by component); dg_set_field."""
        e = np.ascontiguousarray(e_nodes, dtype=np.float64).reshape(-1)
        check(self.lib.dg_set_field(self.handle, e.ctypes.data_as(_lib.c_double_p), _stream()))

    def empty(self, prec=PREC_FP64, device="cuda"):
        """An uninitialised vector of n_dofs elements of the precision's type."""
        return torch.empty(self.n_dofs, dtype=_WDTYPE[prec], device=device)

    def _vec(self, t, prec, name):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != _WDTYPE[prec]:
            raise TypeError(f"{name} must be {_WDTYPE[prec]} for precision {prec}")
        if not t.is_contiguous() or t.numel() != self.n_dofs:
            raise ValueError(f"{name} must be contiguous with {self.n_dofs} elements")
        return _ptr(t)

    # -- the operator ------------------------------------------------------------
    def apply(self, src, dst=None, prec=PREC_FP64):
        """dst = M^{-1} A(src)."""
        if dst is None:
            dst = torch.empty_like(src)
        check(self.lib.dg_apply(self.handle, self._vec(src, prec, "src"),
                                self._vec(dst, prec, "dst"), prec, _stream()))
        return dst

    def apply_adjoint(self, src, dst=None, prec=PREC_FP64):
        """dst = L^T src (transpose of ``apply``)."""
        if dst is None:
            dst = torch.empty_like(src)
        check(self.lib.dg_apply_adjoint(self.handle, self._vec(src, prec, "src"),
                                        self._vec(dst, prec, "dst"), prec, _stream()))
        return dst

    def rk_stage(self, w_in, w_out, u, stage, dt, prec=PREC_FP64, adjoint=False):
        """One fused LSRK(5,4) stage (dg_rk_stage): K = L(w_in) (L^T if
        adjoint), u += b_s dt K in FP64, w_out = u_old + a_s dt K (or u_new at
        the last stage)."""
        check(self.lib.dg_rk_stage(self.handle, self._vec(w_in, prec, "w_in"),
                                   self._vec(w_out, prec, "w_out"),
                                   self._vec(u, PREC_FP64, "u"), int(stage), float(dt), prec,
                                   int(bool(adjoint)), _stream()))

    # -- delta-f form -----------------------------------------------------------
    def set_reference(self, u_ref):
        """Keep u_ref and K_ref = L(u_ref) (FP64) for the delta-f calls."""
        check(self.lib.dg_set_reference(self.handle, self._vec(u_ref, PREC_FP64, "u_ref"), _stream()))

    def apply_df(self, src, dst=None):
        """dst = L(u_ref) + L(src - u_ref) with FP32 sweeps (FP64 vectors)."""
        if dst is None:
            dst = torch.empty_like(src)
        check(self.lib.dg_apply_df(self.handle, self._vec(src, PREC_FP64, "src"),
                                   self._vec(dst, PREC_FP64, "dst"), _stream()))
        return dst

    def rk_step_df(self, u, dt, nsteps=1, w0=None, w1=None):
        """LSRK(5,4) steps in the delta-f form (FP32 stage vectors)."""
        if w0 is None:
            w0 = self.empty(PREC_FP32, u.device)
        if w1 is None:
            w1 = self.empty(PREC_FP32, u.device)
        check(self.lib.dg_rk_step_df(self.handle, self._vec(u, PREC_FP64, "u"),
                                     self._vec(w0, PREC_FP32, "w0"), self._vec(w1, PREC_FP32, "w1"),
                                     float(dt), int(nsteps), _stream()))
        return u

    def rk_stage_host(self, w_in, w_out, u, stage, dt, prec=PREC_FP32):
        """One fused stage on host (CPU, preferably pinned) tensors; the library
        stages them through device memory it owns."""
        for name, t, want in (("w_in", w_in, _WDTYPE[prec]), ("w_out", w_out, _WDTYPE[prec]),
                              ("u", u, torch.float64)):
            if t.is_cuda or t.dtype != want or not t.is_contiguous() or t.numel() != self.n_dofs:
                raise ValueError(f"{name} must be a contiguous host tensor of {self.n_dofs} {want}")
        check(self.lib.dg_rk_stage_host(self.handle, _ptr(w_in), _ptr(w_out), _ptr(u), int(stage),
                                        float(dt), prec, _stream()))

    def rk_step(self, u, dt, nsteps=1, prec=PREC_FP64, adjoint=False, w0=None, w1=None):
        """Advance the FP64 state u in place by nsteps LSRK(5,4) steps."""
        if w0 is None:
            w0 = self.empty(prec, u.device)
        if w1 is None:
            w1 = self.empty(prec, u.device)
        check(self.lib.dg_rk_step(self.handle, self._vec(u, PREC_FP64, "u"),
                                  self._vec(w0, prec, "w0"), self._vec(w1, prec, "w1"),
                                  float(dt), int(nsteps), prec, int(bool(adjoint)), _stream()))
        return u

    def integrals(self, u):
        """(int u, int u^2, max |u|) with the cell quadrature (synchronises)."""
        out = np.zeros(3)
        check(self.lib.dg_integrals(self.handle, self._vec(u, PREC_FP64, "u"),
                                    out.ctypes.data_as(_lib.c_double_p), _stream()))
        return tuple(float(x) for x in out)

    def charge_density(self, f, prec=PREC_FP64, rho=None):
        """rho = 1 - int f dv at the x nodes, shape (n_xcells * (k+1)^dim_x,) FP64."""
        nrho = int(self.info.n_xcells) * (self.degree + 1) ** self.dim_x
        if rho is None:
            rho = torch.empty(nrho, dtype=torch.float64, device=f.device)
        if rho.numel() != nrho or rho.dtype != torch.float64 or not rho.is_contiguous():
            raise ValueError(f"rho must be a contiguous FP64 tensor of {nrho} elements")
        check(self.lib.dg_charge_density(self.handle, self._vec(f, prec, "f"), prec, _ptr(rho),
                                         _stream()))
        return rho

    def poisson_periodic_1d(self, rho, e=None):
        """E at the x nodes with E' = rho - mean(rho), zero mean (dim_x = 1)."""
        if e is None:
            e = torch.empty_like(rho)
        for name, t in (("rho", rho), ("e", e)):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                    and t.numel() == int(self.info.n_xcells) * (self.degree + 1)):
                raise ValueError(f"{name} must be a contiguous CUDA FP64 tensor of one value per x node")
        check(self.lib.dg_poisson_periodic_1d(self.handle, _ptr(rho), _ptr(e), _stream()))
        return e

    def set_field_device(self, e, components=None, scale=1.0):
        """a_v = scale * e from a device tensor (x cell, x node, component)."""
        comps = self.dim_v if components is None else int(components)
        nx = int(self.info.n_xcells) * (self.degree + 1) ** self.dim_x
        if not (e.is_cuda and e.dtype == torch.float64 and e.is_contiguous()
                and e.numel() == nx * comps):
            raise ValueError(f"e must be a contiguous CUDA FP64 tensor of {nx * comps} values")
        check(self.lib.dg_set_field_device(self.handle, _ptr(e), comps, float(scale), _stream()))
        info = _lib.Info()
        check(self.lib.dg_info(self.handle, ctypes.byref(info)))
        self.info = info

    def vp_rk_step(self, u, dt, nsteps=1, prec=PREC_FP64, w0=None, w1=None):
        """Vlasov-Poisson LSRK(5,4) steps (dim_x = 1): the field follows f at every stage."""
        if w0 is None:
            w0 = self.empty(prec, u.device)
        if w1 is None:
            w1 = self.empty(prec, u.device)
        check(self.lib.dg_vp_rk_step(self.handle, self._vec(u, PREC_FP64, "u"),
                                     self._vec(w0, prec, "w0"), self._vec(w1, prec, "w1"),
                                     float(dt), int(nsteps), prec, _stream()))
        return u

    def vp_step_adjoint(self, u, ubar, dt):
        """Adjoint of one FP64 Vlasov-Poisson step from the state ``u`` at its
        start: ``ubar`` (dJ/du after the step) becomes dJ/du before it, in place."""
        check(self.lib.dg_vp_step_adjoint(self.handle, self._vec(u, PREC_FP64, "u"),
                                          self._vec(ubar, PREC_FP64, "ubar"), float(dt), _stream()))
        return ubar

    def check(self):
        """Synchronise and raise DGError(DG_ERR_NONFINITE) if a kernel saw NaN/Inf."""
        check(self.lib.dg_check(self.handle, _stream()))

    # -- launch configuration -----------------------------------------------------
    def get_launch(self, prec):
        """The cell-kernel launch configuration used for ``prec``."""
        c = _lib.Launch()
        check(self.lib.dg_get_launch(self.handle, prec, ctypes.byref(c)))
        return {"threads": c.threads, "cells_per_block": c.cells_per_block,
                "order": list(c.order)[: self.dim_x + self.dim_v], "variant": c.variant}

    def set_launch(self, prec, threads, cells_per_block, order=None, variant=0):
        """Set the launch configuration for ``prec`` (validated by the library;
        captured graphs are dropped)."""
        c = _lib.Launch()
        c.threads, c.cells_per_block, c.variant = int(threads), int(cells_per_block), int(variant)
        order = list(range(self.dim_x + self.dim_v)) if order is None else list(order)
        for j in range(6):
            c.order[j] = order[j] if j < len(order) else j
        check(self.lib.dg_set_launch(self.handle, prec, ctypes.byref(c)))

    def autotune(self, src, dst, prec):
        """Time the candidate launch configurations on apply(src, dst), keep the
        fastest for ``prec`` and return its time in ms."""
        best = ctypes.c_double()
        check(self.lib.dg_autotune(self.handle, self._vec(src, prec, "src"),
                                   self._vec(dst, prec, "dst"), prec, _stream(), ctypes.byref(best)))
        return float(best.value)


def from_spec(spec, e_nodes=None):
    """Build a DG from a plain description (dict with the constructor's keys)."""
    return DG(e_nodes=e_nodes, **spec)


class DGBatch:
    """Independent constant-velocity problems (d = 3 or 4) advanced together:
    one persistent launch per LSRK stage over all members, replayed from a
    CUDA graph.  The member handles stay owned by the caller."""

    def __init__(self, members):
        self.lib = _lib.load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle for m in self.members])
        h = ctypes.c_void_p()
        check(self.lib.dg_batch_create(len(self.members), arr, ctypes.byref(h)))
        self.handle = h
        tiles, nd = ctypes.c_longlong(), ctypes.c_longlong()
        check(self.lib.dg_batch_info(self.handle, ctypes.byref(tiles), ctypes.byref(nd)))
        self.tiles, self.n_dofs = int(tiles.value), int(nd.value)

    def close(self):
        """Release the batch (the member handles stay open); idempotent."""
        if getattr(self, "handle", None):
            self.lib.dg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, us, w0s, w1s, dts, prec):
        n = len(self.members)
        if not (len(us) == len(w0s) == len(w1s) == len(dts) == n):
            raise ValueError("one u, w0, w1 and dt per member")
        for m, u, a, b in zip(self.members, us, w0s, w1s):
            m._vec(u, PREC_FP64, "u")
            m._vec(a, prec, "w0")
            m._vec(b, prec, "w1")
        U = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
        A = (ctypes.c_void_p * n)(*[w.data_ptr() for w in w0s])
        B = (ctypes.c_void_p * n)(*[w.data_ptr() for w in w1s])
        D = (ctypes.c_double * n)(*[float(x) for x in dts])
        return U, A, B, D

    def rk_step(self, us, w0s, w1s, dts, nsteps=1, prec=PREC_FP32):
        """Advance every member's FP64 state by nsteps LSRK(5,4) steps of its
        own dt (w0s, w1s: per-member stage vectors of the precision's type)."""
        U, A, B, D = self._arrays(us, w0s, w1s, dts, prec)
        check(self.lib.dg_batch_rk_step(self.handle, U, A, B, D, int(nsteps), prec, _stream()))

    def set_launch(self, tile_dofs, threads, threads4=None, order=None, r4_max_n=None):
        """Launch configuration of the batched kernels: DoFs per work tile and
        threads per block of the shared-memory kernel, threads per block of the
        4D register kernel (n^2 per cell), the direction-order bits, and the
        largest n of the FP32 4D groups that run the register kernel
        (dg_batch_launch)."""
        c = self.get_launch()
        c.update(tile_dofs=int(tile_dofs), threads=int(threads))
        for k, v in (("threads4", threads4), ("order", order), ("r4_max_n", r4_max_n)):
            if v is not None:
                c[k] = int(v)
        check(self.lib.dg_batch_set_launch_ex(self.handle, ctypes.byref(_lib.BatchLaunch(**c))))

    def get_launch(self):
        """The current dg_batch_launch as a dict."""
        c = _lib.BatchLaunch()
        check(self.lib.dg_batch_get_launch(self.handle, ctypes.byref(c)))
        return {"tile_dofs": c.tile_dofs, "threads": c.threads, "threads4": c.threads4,
                "order": c.order, "r4_max_n": c.r4_max_n}

    def autotune_record(self):
        """The configurations the last autotune timed (list of dicts with ms)."""
        n = ctypes.c_int()
        check(self.lib.dg_batch_autotune_record(self.handle, None, 0, ctypes.byref(n)))
        arr = (_lib.BatchTrial * max(1, n.value))()
        check(self.lib.dg_batch_autotune_record(self.handle, arr, n.value, ctypes.byref(n)))
        return [{"tile_dofs": t.tile_dofs, "threads": t.threads, "threads4": t.threads4,
                 "order": t.order, "r4_max_n": t.r4_max_n, "ms": t.ms} for t in arr[:n.value]]

    def autotune(self, us, w0s, w1s, dts, prec=PREC_FP32):
        """Time launch configurations (block sizes, so cells per block; tile
        size; direction order) on one step each, keep the fastest and return
        its time per step in ms (the states are advanced by the trials); the
        record of what was timed is ``autotune_record()``."""
        U, A, B, D = self._arrays(us, w0s, w1s, dts, prec)
        best = ctypes.c_double()
        check(self.lib.dg_batch_autotune(self.handle, U, A, B, D, prec, _stream(),
                                         ctypes.byref(best)))
        return float(best.value)

    def check(self):
        """Synchronise and raise DGError if a batched kernel saw NaN/Inf."""
        check(self.lib.dg_batch_check(self.handle, _stream()))
