"""The C-ABI library builds, loads, exports every declared symbol, and rejects
bad arguments on the host (no GPU needed)."""
import ctypes

import numpy as np
import pytest

import __graft_entry__ as entry
from paper_2002_08110_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _lib.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_reference_nodes(lib):
    assert lib.dg_version() == 4
    for k in range(6):
        x = np.zeros(k + 1)
        w = np.zeros(k + 1)
        assert lib.dg_reference_nodes(k, x.ctypes.data_as(_lib.c_double_p),
                                      w.ctypes.data_as(_lib.c_double_p)) == 0
        xr, wr = np.polynomial.legendre.leggauss(k + 1)
        assert np.allclose(x, xr, atol=1e-15) and np.allclose(w, wr, atol=1e-15)
    assert lib.dg_reference_nodes(6, x.ctypes.data_as(_lib.c_double_p), None) == 1
    assert lib.dg_reference_nodes(2, None, None) == 1


def test_basis_nodes(lib):
    """Gauss-Lobatto nodes (endpoints and the roots of P'_{n-1}) and weights
    (exact for polynomials of degree 2n-3) of the library's host tables."""
    P = np.polynomial.legendre.Legendre
    for k in range(1, 6):
        n = k + 1
        a = [np.zeros(n) for _ in range(3)]
        ptrs = [x.ctypes.data_as(_lib.c_double_p) for x in a]
        assert lib.dg_basis_nodes(1, k, *ptrs) == 0
        nodes, qp, qw = a
        ref = np.concatenate([[-1.0], np.sort(P.basis(n - 1).deriv().roots().real), [1.0]])
        assert np.allclose(nodes, ref, atol=1e-14) and np.allclose(qp, ref, atol=1e-14)
        for m in range(2 * n - 2):        # exact up to degree 2n-3
            exact = 0.0 if m % 2 else 2.0 / (m + 1)
            assert abs(qw @ qp ** m - exact) <= 1e-14
        assert lib.dg_basis_nodes(2, k, *ptrs) == 0        # GLL nodes, Gauss quadrature
        xg, wg = np.polynomial.legendre.leggauss(n)
        assert np.allclose(a[0], ref, atol=1e-14)
        assert np.allclose(a[1], xg, atol=1e-15) and np.allclose(a[2], wg, atol=1e-15)
    x = np.zeros(6)
    px = x.ctypes.data_as(_lib.c_double_p)
    assert lib.dg_basis_nodes(3, 2, px, None, None) == 1     # unknown basis
    assert lib.dg_basis_nodes(1, 0, px, None, None) == 1     # Lobatto needs degree >= 1
    assert lib.dg_basis_nodes(0, 6, px, None, None) == 1


def _create(lib, dx, dv, k, cx, cv, kind=0):
    g = _lib.Geometry()
    for j in range(3):
        g.x_lo[j], g.x_hi[j], g.v_lo[j], g.v_hi[j] = 0.0, 1.0, 0.0, 1.0
    g.field_kind = kind
    h = ctypes.c_void_p()
    cxa = (ctypes.c_int * max(1, len(cx)))(*cx)
    cva = (ctypes.c_int * max(1, len(cv)))(*cv)
    st = lib.dg_create(dx, dv, k, cxa, cva, ctypes.byref(g), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("dx,dv,k,status", [
    (0, 1, 3, 2), (1, 0, 3, 2), (4, 1, 3, 2), (3, 4, 3, 2), (1, 1, 0, 2), (1, 1, 6, 2),
])
def test_create_rejects_unsupported(lib, dx, dv, k, status):
    st, h = _create(lib, dx, dv, k, [2] * max(dx, 1), [2] * max(dv, 1))
    assert st == status
    assert h.value is None
    assert len(lib.dg_last_error()) > 0


def test_create_rejects_bad_arguments(lib):
    st, _ = _create(lib, 1, 1, 2, [0], [2])
    assert st == 1
    st, _ = _create(lib, 2, 1, 2, [2, 2], [2], kind=1)   # phase space needs dv >= dx
    assert st == 2
    st, _ = _create(lib, 1, 1, 2, [2], [2], kind=7)
    assert st == 1
    g = _lib.Geometry()
    h = ctypes.c_void_p()
    c = (ctypes.c_int * 1)(2)
    assert lib.dg_create(1, 1, 2, c, c, ctypes.byref(g), ctypes.byref(h)) == 1  # empty box
    assert lib.dg_create(1, 1, 2, None, c, ctypes.byref(g), ctypes.byref(h)) == 1


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.dg_apply(None, None, None, 0, None) == 1
    assert lib.dg_apply_adjoint(None, None, None, 0, None) == 1
    assert lib.dg_rk_step(None, None, None, None, 0.1, 1, 0, 0, None) == 1
    assert lib.dg_rk_stage(None, None, None, None, 0, 0.1, 0, 0, None) == 1
    assert lib.dg_check(None, None) == 1
    assert lib.dg_vp_rk_step(None, None, None, None, 0.1, 1, 0, None) == 1
    assert lib.dg_vp_step_adjoint(None, None, None, 0.1, None) == 1
    assert lib.dg_destroy(None) == 0


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/dg.h compiles as strict C99 and a C program links against the
    library and calls its host-only entry points (no GPU needed)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use_dg.c"
    src.write_text(
        '#include <stdio.h>\n#include "dg.h"\n'
        "int main(void) {\n"
        "  double x[4], w[4], q[4], qw[4];\n"
        "  if (dg_version() != DG_ABI_VERSION) return 1;\n"
        "  if (dg_reference_nodes(3, x, w) != DG_OK) return 2;\n"
        "  if (dg_basis_nodes(DG_BASIS_GLL, 3, x, q, qw) != DG_OK) return 3;\n"
        "  if (dg_reference_nodes(9, x, w) != DG_ERR_INVALID_ARG) return 4;\n"
        '  printf("%.15f %.15f\\n", x[0], qw[0]);\n'
        "  return 0;\n}\n")
    exe = tmp_path / "use_dg"
    pkg = os.path.join(root, "paper_2002_08110_gb300")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(root, "include"), str(src), "-o", str(exe),
                    "-L", pkg, "-ldg", "-Wl,-rpath," + pkg], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert abs(float(out[0]) + 1.0) < 1e-15          # first Gauss-Lobatto node
    assert abs(float(out[1]) - 1.0 / 6.0) < 1e-15     # its weight for n = 4
