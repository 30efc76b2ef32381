"""ctypes binding of libaxhelm.so: loads the library and declares the
prototype of every symbol in include/axhelm.h.  Argument marshalling only.

The library must have been built (``paper_2506_20994_gb300.build.build()``);
loading fails loudly otherwise - there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libaxhelm.so")

c_int, c_double, c_float = ctypes.c_int, ctypes.c_double, ctypes.c_float
c_int64, c_void_p, c_char_p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_char_p
P = ctypes.c_void_p  # every array argument is passed as a raw address

# name -> (restype, argtypes); mirrors include/axhelm.h
PROTOTYPES = {
    "ax_strerror": (c_char_p, [c_int]),
    "ax_version": (c_char_p, []),
    "ax_helm": (c_int, [P] * 11 + [c_int, c_int, c_void_p]),
    "ax_helm_variant": (c_int, [c_int] + [P] * 11 + [c_int, c_int, c_int, c_void_p]),
    "ax_helm_f32": (c_int, [P] * 11 + [c_int, c_int, c_void_p]),
    "ax_helm_bf16": (c_int, [P] * 11 + [c_int, c_int, c_void_p]),
    "ax_gll": (c_int, [c_int, P, P]),
    "ax_dmat": (c_int, [c_int, P, P]),
    "ax_box_geometry": (c_int, [c_int, c_int, c_int, c_int, P] + [P] * 8),
    "ax_box_corners": (c_int, [c_int, c_int, c_int, P, P]),
    "ax_tune_save": (c_int, [ctypes.c_char_p]),
    "ax_tune_load": (c_int, [ctypes.c_char_p]),
    "ax_box_numbering": (c_int, [c_int, c_int, c_int, c_int, P]),
    "ax_box_mask": (c_int, [c_int, c_int, c_int, c_int, P, P]),
    "ax_poisson_rhs": (c_int, [c_void_p, P, P, P, c_void_p]),
    "ax_cg_solve_part": (c_int, [P] * 8 + [c_double, c_int, P, P, c_void_p]),
    "ax_cg_solve_part_poisson": (c_int, [c_void_p, P, P, P, P, c_double, c_int, P, P,
                                         c_void_p]),
    "ax_df64_roundtrip": (c_int, [P, P, P, P, c_int64]),
    "ax_gs_setup": (c_int, [P, P, c_int64, c_void_p]),
    "ax_gs_sum": (c_int, [c_void_p, P, c_void_p]),
    "ax_gs_sum_f32": (c_int, [c_void_p, P, c_void_p]),
    "ax_gs_info": (c_int, [c_void_p, P, P, P]),
    "ax_gs_inverse_multiplicity": (c_void_p, [c_void_p]),
    "ax_gs_free": (c_int, [c_void_p]),
    "ax_poisson_create": (c_int, [P, c_int, c_int] + [P] * 10 + [c_void_p, c_void_p]),
    "ax_poisson_destroy": (c_int, [c_void_p]),
    "ax_poisson_apply": (c_int, [c_void_p, P, P, c_void_p]),
    "ax_poisson_jacobi": (c_int, [c_void_p, P]),
    "ax_poisson_set_check_every": (c_int, [c_void_p, c_int]),
    "ax_cg_solve": (c_int, [c_void_p, P, P, c_double, c_int, P, P, c_void_p]),
    "ax_mpcg_solve": (c_int, [c_void_p, c_int, P, P, c_double, c_double, c_int, c_int, P, P, P,
                              c_void_p]),
    "ax_batch_create": (c_int, [P, c_int, c_int, P, c_int, c_void_p]),
    "ax_batch_launch": (c_int, [c_void_p, c_void_p]),
    "ax_batch_graph_launch": (c_int, [c_void_p, c_void_p]),
    "ax_batch_info": (c_int, [c_void_p, P, P, P, P, P]),
    "ax_batch_error": (c_int, [P, P]),
    "ax_batch_destroy": (c_int, [c_void_p]),
    "ax_tune_run": (c_int, [c_int, c_int, c_int] + [P] * 11 + [c_int, P, P, c_void_p]),
    "ax_tune_set": (c_int, [c_int, c_int, c_int]),
    "ax_tune_get": (c_int, [c_int, c_int, P]),
    "ax_jacobi_noalloc": (c_int, [P] * 10 + [c_void_p, c_int, c_int, c_void_p]),
    "ax_mlp_create": (c_int, [P, c_int, c_int]),
    "ax_mlp_create_ex": (c_int, [P, c_int, c_int, c_int]),
    "ax_helm_h2": (c_int, [P] * 13 + [c_int, c_int, P]),
    "ax_helm_xyz": (c_int, [P] * 15 + [c_int, c_int, P]),
    "ax_helm_trilinear_f32": (c_int, [P] * 8 + [c_int, c_int, P]),
    "ax_helm_host": (c_int, [P] * 11 + [c_int, c_int, c_int, P]),
    "ax_tune_variant_run": (c_int, [c_int, c_int] + [P] * 11 + [c_int, P, P, P]),
    "ax_tune_variant_set": (c_int, [c_int, c_int]),
    "ax_tune_variant_get": (c_int, [c_int, P]),
    "ax_mass_add": (c_int, [P, P, P, c_int64, P]),
    "ax_mass_add_f32": (c_int, [P, P, P, c_int64, P]),
    "ax_op_set_h2": (c_int, [P, P, P, P]),
    "ax_poisson_set_h2": (c_int, [P, P, P, P]),
    "ax_op_create": (c_int, [P, c_int, c_int] + [P] * 9 + [P]),
    "ax_op_apply": (c_int, [P, P, P, P]),
    "ax_op_set_h1": (c_int, [P, P, P]),
    "ax_op_info": (c_int, [P, P, P]),
    "ax_op_error": (c_int, [P, P]),
    "ax_op_inject_copy_loss": (c_int, [P, c_int64]),
    "ax_op_destroy": (c_int, [P]),
    "ax_poisson_diag": (c_int, [P, P, P]),
    "ax_poisson_set_diag": (c_int, [P, P, P]),
    "ax_dot_weighted": (c_int, [P, P, P, c_int64, P, P, P]),
    "ax_gather": (c_int, [P, P, P, c_int64, P]),
    "ax_scatter_add": (c_int, [P, P, P, P, c_int64, P]),
    "ax_mlp_destroy": (c_int, [c_void_p]),
    "ax_mlp_nparams": (c_int, [c_void_p, P]),
    "ax_mlp_set_params": (c_int, [c_void_p, P, c_int64, c_void_p]),
    "ax_mlp_get_params": (c_int, [c_void_p, P, c_int64, c_void_p]),
    "ax_mlp_loss_grad": (c_int, [c_void_p, P, P, c_int, P, P, c_void_p]),
    "ax_mlp_adam": (c_int, [c_void_p, c_float, c_float, c_float, c_float, c_void_p]),
    "ax_mlp_gather_pairs": (c_int, [c_void_p, P, P, P, P, c_int, P, P, c_void_p]),
    "ax_mlp_train": (c_int, [c_void_p, P, P, c_int, P, c_int, c_int, c_float, P, c_void_p]),
    "ax_mlp_forward": (c_int, [c_void_p, P, P, P, P, P, c_int, c_void_p]),
    "ax_axpby": (c_int, [P, c_double, P, c_double, c_int64, c_void_p]),
    "ax_mlp_train_energy": (c_int, [c_void_p, c_void_p, P, P, c_int, c_int, c_float, P,
                                    c_void_p]),
    "ax_precondition": (c_int, [c_void_p, c_void_p, P, P, c_void_p]),
    "ax_fcg_solve": (c_int, [c_void_p, c_void_p, P, P, c_double, c_int, P, P, P, c_void_p]),
    "ax_mpfcg_solve": (c_int, [c_void_p, c_void_p, c_int, P, P, c_double, c_double, c_int,
                               c_int, P, P, P, P, c_void_p]),
}


class BatchMesh(ctypes.Structure):
    """Mirror of ax_batch_mesh."""
    _fields_ = [("lx", c_int), ("nelv", c_int)] + [
        (n, c_void_p) for n in ("w", "u", "dx", "dxt", "h1", "g11", "g22", "g33", "g12", "g13",
                                "g23")]

# the callback tables of the partitioned solve (ax_part_ops, ax_part_comm)
APPLY_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_void_p, c_void_p)
DOT_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                          c_void_p)
AXPBY_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_double, c_void_p, c_double, c_void_p)
ZERO_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_void_p)
HALO_FN = ctypes.CFUNCTYPE(c_int, c_void_p, c_void_p, c_void_p)
ALLSUM_FN = ctypes.CFUNCTYPE(c_int, c_void_p, ctypes.POINTER(c_double), c_int)


class PartOps(ctypes.Structure):
    """Mirror of ax_part_ops."""
    _fields_ = [("ctx", c_void_p), ("apply", APPLY_FN), ("precond", APPLY_FN),
                ("dot", DOT_FN), ("axpby", AXPBY_FN), ("copy", APPLY_FN), ("zero", ZERO_FN)]


class PartComm(ctypes.Structure):
    """Mirror of ax_part_comm."""
    _fields_ = [("ctx", c_void_p), ("halo", HALO_FN), ("allsum", ALLSUM_FN)]


AX_OK = 0
AX_EINVAL = -1
AX_ELAUNCH = -3
AX_ENOMEM = -4
AX_ENOTCONV = -5
AX_EBREAKDOWN = -6
AX_EIO = -7
AX_VARIANT_AUTO = 0
AX_VARIANT_F64_NATIVE = 1
AX_VARIANT_F64_DF = 2
AX_VARIANT_F64_DF_EO = 3
AX_PREC_F32 = 1
AX_PREC_BF16 = 2
AX_BATCH_F64 = 1
AX_BATCH_F32 = 2
AX_MLP_TANH = 0
AX_MLP_SYM = 1
AX_DOT_WORK = 608

_lib = None
_lock = threading.Lock()


class AxError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        msg = lib().ax_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {msg} ({code})")


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            h = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def check(fn: str, code: int) -> None:
    if code != AX_OK:
        raise AxError(fn, code)
