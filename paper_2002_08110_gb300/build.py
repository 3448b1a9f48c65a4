"""Build the CUDA library ``libdg.so`` in-tree for sm_103a.

Every translation unit under ``csrc/`` is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``), then linked into
``paper_2002_08110_gb300/libdg.so`` with the CUDA runtime linked statically.
Object files go to ``_build/`` at the repository root.  Rebuilds only what
changed (source or header newer than its object).

``build(variant="bounds")`` makes the bounds-check library
``libdg_bounds.so`` instead (``-DDG_BOUNDS_CHECK``: every computed cell,
neighbour, tile and slab index is checked on the device and a violation is
reported by dg_check as DG_ERR_BOUNDS), with its objects in ``_build_bounds/``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libdg.so")
VARIANTS = {"": (BUILD, LIB, []),
            "bounds": (os.path.join(ROOT, "_build_bounds"), os.path.join(PKG, "libdg_bounds.so"),
                       ["-DDG_BOUNDS_CHECK"])}
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libdg.so")
    return cand


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "dg.h"))
    return hs


def _compile(src, obj, nvcc, extra):
    if src.endswith(".cu"):
        cmd = [nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-Xptxas", "-warn-spills", "-c", src, "-o", obj] + extra
    else:
        cmd = [nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-c", src, "-o", obj] + extra
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, jobs=None, extra_flags=None, variant=""):
    """Compile and link; returns the path of the library (libdg.so, or
    libdg_bounds.so for variant="bounds")."""
    nvcc = _nvcc()
    BUILD, LIB, vflags = VARIANTS[variant]
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra_flags or []) + vflags
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))
    newest_header = max(os.path.getmtime(h) for h in _headers())
    todo = []
    objs = []
    for f in srcs:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if (not os.path.exists(obj) or os.path.getmtime(obj) < os.path.getmtime(src)
                or os.path.getmtime(obj) < newest_header):
            todo.append((src, obj))
    jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = [ex.submit(_compile, s, o, nvcc, extra) for s, o in todo]
            for fu in cf.as_completed(futs):
                obj, err = fu.result()
                if verbose and err.strip():
                    print(err, file=sys.stderr)
    need_link = (not os.path.exists(LIB) or bool(todo)
                 or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs))
    if need_link:
        tmp = LIB + ".tmp"
        cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
