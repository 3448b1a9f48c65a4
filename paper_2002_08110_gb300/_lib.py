"""ctypes loader of ``libdg.so`` and the C structs of ``include/dg.h``.

Argument marshalling only: every step of the method runs inside the CUDA
library.  Importing this module fails loudly if the library has not been
built (there is no fallback implementation).
"""
import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
# DG_LIBRARY_VARIANT=bounds selects the bounds-check build (libdg_bounds.so,
# every computed index checked on the device; see DG_ERR_BOUNDS)
_VARIANT = os.environ.get("DG_LIBRARY_VARIANT", "")
LIB_PATH = os.path.join(PKG, "libdg_bounds.so" if _VARIANT == "bounds" else "libdg.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "dg.h")

DG_OK = 0
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_INVALID_ARG", 2: "DG_ERR_UNSUPPORTED", 3: "DG_ERR_CUDA",
                4: "DG_ERR_OOM", 5: "DG_ERR_NONFINITE", 6: "DG_ERR_TIMEOUT", 7: "DG_ERR_BOUNDS"}
PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
BASIS_GL, BASIS_GLL, BASIS_GLL_GAUSS = 0, 1, 2

c_double_p = ctypes.POINTER(ctypes.c_double)


class Geometry(ctypes.Structure):
    """dg_geometry of include/dg.h (field, box, shear, basis, deformation)."""
    _fields_ = [("x_lo", ctypes.c_double * 3), ("x_hi", ctypes.c_double * 3),
                ("v_lo", ctypes.c_double * 3), ("v_hi", ctypes.c_double * 3),
                ("shear_x", ctypes.c_double * 9), ("field_kind", ctypes.c_int),
                ("a_const", ctypes.c_double * 6), ("e_nodes", c_double_p),
                ("basis", ctypes.c_int), ("deform", ctypes.c_double * 3)]


class Info(ctypes.Structure):
    """dg_info_t of include/dg.h (sizes and properties of a handle)."""
    _fields_ = [("n_dofs", ctypes.c_longlong), ("n_cells", ctypes.c_longlong),
                ("n_xcells", ctypes.c_longlong), ("n_vcells", ctypes.c_longlong),
                ("dofs_per_cell", ctypes.c_int), ("dim_x", ctypes.c_int), ("dim_v", ctypes.c_int),
                ("degree", ctypes.c_int), ("speed_sum", ctypes.c_double),
                ("det_jacobian", ctypes.c_double), ("h", ctypes.c_double * 6),
                ("uniform_sides", ctypes.c_int), ("basis", ctypes.c_int)]


class Launch(ctypes.Structure):
    """dg_launch of include/dg.h (cell-kernel launch configuration)."""
    _fields_ = [("threads", ctypes.c_int), ("cells_per_block", ctypes.c_int),
                ("order", ctypes.c_int * 6), ("variant", ctypes.c_int)]


class BatchLaunch(ctypes.Structure):
    """dg_batch_launch of include/dg.h (batched-kernel launch configuration)."""
    _fields_ = [("tile_dofs", ctypes.c_int), ("threads", ctypes.c_int),
                ("threads4", ctypes.c_int), ("order", ctypes.c_int), ("r4_max_n", ctypes.c_int)]


class BatchTrial(ctypes.Structure):
    """dg_batch_trial of include/dg.h (one configuration the autotuner timed)."""
    _fields_ = [("tile_dofs", ctypes.c_int), ("threads", ctypes.c_int),
                ("threads4", ctypes.c_int), ("order", ctypes.c_int), ("r4_max_n", ctypes.c_int),
                ("ms", ctypes.c_double)]


class DGError(RuntimeError):
    """A dg_status other than DG_OK, with the library's last error message."""
    def __init__(self, status, message):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


_lib = None


def load():
    """Load libdg.so (once).  Raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "dg_version": (i, []),
        "dg_last_error": (ctypes.c_char_p, []),
        "dg_reference_nodes": (i, [i, c_double_p, c_double_p]),
        "dg_create": (i, [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(Geometry),
                          ctypes.POINTER(vp)]),
        "dg_destroy": (i, [vp]),
        "dg_info": (i, [vp, ctypes.POINTER(Info)]),
        "dg_node_coordinates": (i, [vp, i, c_double_p]),
        "dg_set_field": (i, [vp, c_double_p, vp]),
        "dg_apply": (i, [vp, vp, vp, i, vp]),
        "dg_apply_adjoint": (i, [vp, vp, vp, i, vp]),
        "dg_rk_stage": (i, [vp, vp, vp, vp, i, d, i, i, vp]),
        "dg_rk_step": (i, [vp, vp, vp, vp, d, i, i, i, vp]),
        "dg_integrals": (i, [vp, vp, c_double_p, vp]),
        "dg_integrals_noalloc": (i, [vp, ll, i, i, i, d, c_double_p, vp]),
        "dg_check": (i, [vp, vp]),
        "dg_selftest_wait": (i, [vp, vp]),
        "dg_basis_nodes": (i, [i, i, vp, vp, vp]),
        "dg_set_reference": (i, [vp, vp, vp]),
        "dg_apply_df": (i, [vp, vp, vp, vp]),
        "dg_rk_step_df": (i, [vp, vp, vp, vp, ctypes.c_double, i, vp]),
        "dg_charge_density": (i, [vp, vp, i, vp, vp]),
        "dg_poisson_periodic_1d": (i, [vp, vp, vp, vp]),
        "dg_set_field_device": (i, [vp, vp, i, ctypes.c_double, vp]),
        "dg_vp_rk_step": (i, [vp, vp, vp, vp, ctypes.c_double, i, i, vp]),
        "dg_vp_step_adjoint": (i, [vp, vp, vp, ctypes.c_double, vp]),
        "dg_rk_stage_host": (i, [vp, vp, vp, vp, i, ctypes.c_double, i, vp]),
        "dg_get_launch": (i, [vp, i, ctypes.POINTER(Launch)]),
        "dg_set_launch": (i, [vp, i, ctypes.POINTER(Launch)]),
        "dg_autotune": (i, [vp, vp, vp, i, vp, c_double_p]),
        "dg_batch_create": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "dg_batch_destroy": (i, [vp]),
        "dg_batch_rk_step": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 c_double_p, i, i, vp]),
        "dg_batch_info": (i, [vp, ctypes.POINTER(ll), ctypes.POINTER(ll)]),
        "dg_batch_check": (i, [vp, vp]),
        "dg_batch_set_launch": (i, [vp, i, i]),
        "dg_batch_set_launch_ex": (i, [vp, ctypes.POINTER(BatchLaunch)]),
        "dg_batch_get_launch": (i, [vp, ctypes.POINTER(BatchLaunch)]),
        "dg_batch_autotune_record": (i, [vp, ctypes.POINTER(BatchTrial), i, ctypes.POINTER(i)]),
        "dg_batch_autotune": (i, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                  c_double_p, i, vp, c_double_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    """Raise DGError unless status is DG_OK."""
    if status != DG_OK:
        msg = load().dg_last_error()
        raise DGError(status, msg.decode() if msg else "")


def declared_functions():
    """Names of the functions declared in include/dg.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", text)))
