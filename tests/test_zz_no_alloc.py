"""The allocation-free integrals entry point against dg_integrals.

dg_integrals_noalloc serves callers that cannot allocate device memory (code
running under CUDA graph capture, inside a framework that owns the device
allocator, or after start-up in a long run).  It keeps its scratch in a fixed
array inside the library, so two calls in a row must not see each other's
leftovers.  This file is collected last on purpose.
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


def _noalloc(lib, u, dg):
    out = np.zeros(3)
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(u.data_ptr()), dg.n_cells,
                                  dg.dim_x + dg.dim_v, dg.degree, dg.info.det_jacobian,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_noalloc_integrals_match_dg_integrals_twice(lib):
    import workloads as W
    from dg_helpers import dg_for
    w = W.shrink(W.config_4d(), cells_x=(5, 3), cells_v=(4, 6), k=3)
    dg, p = dg_for(w)
    rng = np.random.default_rng(11)
    # two calls in a row; the second input is much smaller in magnitude, so
    # stale partial sums from the first call would show
    for scale in (1.0, 1e-3):
        u = torch.tensor(scale * (1.0 + rng.standard_normal(p.n_dofs)), device="cuda")
        ref = dg.integrals(u)
        st, out = _noalloc(lib, u, dg)
        assert st == 0, lib.dg_last_error()
        assert abs(out[0] - ref[0]) <= 1e-12 * abs(ref[1]) + 1e-300
        assert abs(out[1] - ref[1]) <= 1e-12 * abs(ref[1])
        assert out[2] == ref[2]
    dg.close()


def test_noalloc_integrals_reject_oversized_input(lib):
    x = torch.zeros(16, device="cuda", dtype=torch.float64)
    out = np.zeros(3)
    st = lib.dg_integrals_noalloc(ctypes.c_void_p(x.data_ptr()), 1 << 40, 6, 3, 1.0,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert st == 1
    assert b"exceeds" in lib.dg_last_error()
