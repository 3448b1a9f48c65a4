"""The allocation-free integrals entry point against dg_integrals and the
oracle.

dg_integrals_noalloc serves callers that cannot allocate device memory: code
inside a framework whose allocator owns all device memory, or a long run that
must not call cudaMalloc after start-up.  It keeps its scratch in a fixed
array inside the library, shared by every call, so calls in a row must not
see each other's leftovers.  It covers the collocated bases on affine meshes
(Gauss-Legendre or Gauss-Lobatto weights, one |J| per cell).  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as entry
    entry.build()
    from paper_2002_08110_gb300 import _lib
    return _lib.load()


def _noalloc(lib, u, dg, basis=None):
    out = np.zeros(3)
    basis = dg.info.basis if basis is None else basis
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(u.data_ptr()), dg.n_cells,
                                  dg.dim_x + dg.dim_v, dg.degree, basis, dg.info.det_jacobian,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def _close(out, ref, what):
    assert abs(out[0] - ref[0]) <= 1e-12 * abs(ref[1]) + 1e-300, what
    assert abs(out[1] - ref[1]) <= 1e-12 * abs(ref[1]), what
    assert out[2] == ref[2], what


def _handle(cells_x, cells_v, k, basis):
    """A sheared 2x + 2v handle of the given basis and its oracle problem."""
    from oracle.dg import ConstantField, Problem
    from paper_2002_08110_gb300 import DG
    S = np.array([[1.0, 0.1], [0.0, 1.2]])
    a = [0.3, -0.2, 0.5, 0.1]
    kw = dict(x_lo=[0.0, 0.0], x_hi=[1.0, 1.0], v_lo=[-1.0, -2.0], v_hi=[1.0, 1.5])
    dg = DG(2, 2, k, cells_x, cells_v, field_kind=0, a_const=a, shear=S, basis=basis, **kw)
    p = Problem(2, 2, k, cells_x, cells_v, kw["x_lo"], kw["x_hi"], kw["v_lo"], kw["v_hi"],
                ConstantField(a), shear=S, basis={0: "gl", 1: "gllc"}[basis])
    return dg, p


@pytest.mark.parametrize("basis", [0, 1])
def test_noalloc_integrals_match_dg_integrals_and_oracle_twice(lib, basis):
    """Each covered basis: two calls in a row (the second input much smaller
    in magnitude, so stale partial sums of the first would show) against
    dg_integrals and the oracle's cell quadrature."""
    dg, p = _handle((5, 3), (4, 6), 3, basis)
    rng = np.random.default_rng(11 + basis)
    for scale in (1.0, 1e-3):
        un = scale * (1.0 + rng.standard_normal(p.n_dofs))
        u = torch.tensor(un, device="cuda")
        st, out = _noalloc(lib, u, dg)
        assert st == 0, lib.dg_last_error()
        _close(out, dg.integrals(u), f"basis {basis} vs dg_integrals")
        _close(out, p.integrals(un), f"basis {basis} vs oracle")
    dg.close()


def test_noalloc_integrals_many_blocks_then_fewer(lib):
    """A call over 2.5 chunks of 2^20 DoFs (three blocks, the last one partial),
    then a call over one partial chunk on the same device: both match
    dg_integrals, so the fold over several partial sums and the reuse of the
    shared array without clearing are exercised."""
    big, _ = _handle((10, 8), (16, 8), 3, 0)
    assert big.n_dofs == 2_621_440
    small, _ = _handle((3, 2), (4, 5), 3, 0)
    rng = np.random.default_rng(5)
    for dg, shift in ((big, 2.0), (small, -0.5), (big, 0.25)):
        u = torch.tensor(shift + rng.standard_normal(dg.n_dofs), device="cuda")
        st, out = _noalloc(lib, u, dg)
        assert st == 0, lib.dg_last_error()
        _close(out, dg.integrals(u), f"{dg.n_dofs} DoFs")
    big.close()
    small.close()


def test_noalloc_integrals_reject_what_they_do_not_cover(lib):
    x = torch.zeros(16, device="cuda", dtype=torch.float64)
    out = np.zeros(3)
    optr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(x.data_ptr()), 1 << 40, 6, 3, 0, 1.0, optr, None)
    assert st == 1
    assert b"exceeds" in lib.dg_last_error()
    # the Lobatto-node, Gauss-quadrature element needs a change of basis first
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(x.data_ptr()), 1, 2, 3, 2, 1.0, optr, None)
    assert st == 2
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(x.data_ptr()), 1, 2, 3, 7, 1.0, optr, None)
    assert st == 1
