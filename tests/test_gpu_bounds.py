"""The small parity cases against the bounds-check build of the library
(libdg_bounds.so, compiled with -DDG_BOUNDS_CHECK): every cell, neighbour,
tile and slab index a kernel computes is checked before use, and a violation
would make dg_check report DG_ERR_BOUNDS instead of trapping.  The cases
(bounds_cases.py) run in a child process that loads that library: the
2D-6D generic kernels with one- and two-cell directions, the 6D kernels in
both their variants (operator, transpose and stage), the host-buffer stage
pipelined over v3 slabs, the delta-f stage, the Gauss-Lobatto face-layer
kernel, the 4D register kernel and the batched kernels."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_check_build_runs_the_parity_cases_clean():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2002_08110_gb300.build import build
    build(variant="bounds")
    env = dict(os.environ, DG_LIBRARY_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "cases passed" in r.stdout
