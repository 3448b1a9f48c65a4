"""ctypes binding of the sum-factorised FP64 OpenMP CPU evaluation
(``cpu_sumfac.cpp``; oracle, test infrastructure only).

The same operator as ``dg.Problem.apply`` (Gauss-Legendre collocation,
affine x-mesh x = S y, constant or phase-space field), evaluated the way the
paper's CPU code does it: cell by cell with 1D sweeps (Sec. 2.4,
Algorithms 1 and 2), in FP64 on all host cores.  It serves as the timed CPU
baseline at the workloads' full sizes and is checked against the dense and
axis-wise routes of ``dg.Problem`` on small meshes.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_sumfac.cpp")
LIB = os.path.join(HERE, "libsumfac.so")


class Problem_(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int), ("dv", ctypes.c_int), ("k", ctypes.c_int),
                ("cells", ctypes.c_int * 6), ("lo", ctypes.c_double * 6),
                ("hi", ctypes.c_double * 6), ("S", ctypes.c_double * 9),
                ("field_kind", ctypes.c_int), ("a", ctypes.c_double * 6),
                ("e_nodes", ctypes.POINTER(ctypes.c_double)), ("basis", ctypes.c_int)]


def build():
    """Compile cpu_sumfac.cpp into libsumfac.so (g++, OpenMP) if it is missing
    or older than its source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["g++", "-O3", "-fopenmp", "-std=c++17", "-shared", "-fPIC", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the CPU sum-factorisation oracle failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        vp, d = ctypes.c_void_p, ctypes.c_double
        lib.sf_create.restype = vp
        lib.sf_create.argtypes = [ctypes.POINTER(Problem_)]
        lib.sf_destroy.restype = None
        lib.sf_destroy.argtypes = [vp]
        lib.sf_apply.restype = ctypes.c_int
        lib.sf_apply.argtypes = [vp, vp, vp]
        lib.sf_apply_abs.restype = ctypes.c_int
        lib.sf_apply_abs.argtypes = [vp, vp, vp]
        lib.sf_rk_stage.restype = ctypes.c_int
        lib.sf_rk_stage.argtypes = [vp, vp, vp, vp, d, d, ctypes.c_int, ctypes.c_longlong,
                                    ctypes.c_longlong]
        lib.sf_threads.restype = ctypes.c_int
        lib.sf_threads.argtypes = []
        _lib = lib
    return _lib


def threads():
    """OpenMP threads the evaluation uses."""
    return load().sf_threads()


class SumFac:
    """Plan for one mesh and field.  ``e_nodes`` (phase-space field): E at
    the x nodes, array (x cells, x nodes, dv) with cells and nodes
    lexicographic (first direction fastest).  ``basis``: "gl" (Gauss-Legendre
    collocation) or "gllc" (Gauss-Lobatto collocation, k >= 1)."""

    def __init__(self, dx, dv, k, cells_x, cells_v, x_lo, x_hi, v_lo, v_hi, a=None,
                 e_nodes=None, shear=None, basis="gl"):
        lib = load()
        pb = Problem_()
        pb.dx, pb.dv, pb.k = dx, dv, k
        if basis not in ("gl", "gllc"):
            raise ValueError("basis must be 'gl' or 'gllc'")
        pb.basis = 0 if basis == "gl" else 1
        for j, c in enumerate(list(cells_x) + list(cells_v)):
            pb.cells[j] = int(c)
        for j, (a_, b_) in enumerate(zip(list(x_lo) + list(v_lo), list(x_hi) + list(v_hi))):
            pb.lo[j], pb.hi[j] = float(a_), float(b_)
        if shear is not None:
            S = np.asarray(shear, dtype=np.float64).reshape(dx, dx)
            for i in range(dx):
                for m in range(dx):
                    pb.S[i * dx + m] = S[i, m]
        self._e = None
        if e_nodes is not None:
            pb.field_kind = 1
            self._e = np.ascontiguousarray(e_nodes, dtype=np.float64).reshape(-1)
            pb.e_nodes = self._e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            pb.field_kind = 0 if a is not None else 1
            for j, x in enumerate(a if a is not None else []):
                pb.a[j] = float(x)
        self.plan = lib.sf_create(ctypes.byref(pb))
        if not self.plan:
            raise ValueError("unsupported dimensions or degree")
        self.lib = lib
        self.ncells = int(np.prod(list(cells_x) + list(cells_v)))
        self.n_dofs = self.ncells * (k + 1) ** (dx + dv)

    def apply(self, src, dst=None):
        src = np.ascontiguousarray(src, dtype=np.float64)
        assert src.shape == (self.n_dofs,)
        dst = np.empty_like(src) if dst is None else dst
        assert self.lib.sf_apply(self.plan, src.ctypes.data, dst.ctypes.data) == 0
        return dst

    def apply_abs(self, src, dst=None):
        """The term scale M^{-1} |A| |src| (every factor and term in absolute
        value, upwind choices unchanged), as ``dg.Problem.apply_abs``."""
        src = np.ascontiguousarray(src, dtype=np.float64)
        assert src.shape == (self.n_dofs,)
        dst = np.empty_like(src) if dst is None else dst
        assert self.lib.sf_apply_abs(self.plan, src.ctypes.data, dst.ctypes.data) == 0
        return dst

    def rk_stage(self, w_in, w_out, u, a_dt, b_dt, last=False, cells=None):
        """In place: w_out = u + a_dt K (u_new if last), u += b_dt K, on the
        cells [cells[0], cells[1]) (default: all)."""
        for x in (w_in, w_out, u):
            assert x.dtype == np.float64 and x.flags.c_contiguous and x.shape == (self.n_dofs,)
        lo, hi = (0, self.ncells) if cells is None else cells
        assert self.lib.sf_rk_stage(self.plan, w_in.ctypes.data, w_out.ctypes.data,
                                    u.ctypes.data, float(a_dt), float(b_dt), int(last),
                                    int(lo), int(hi)) == 0

    def close(self):
        if self.plan:
            self.lib.sf_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
