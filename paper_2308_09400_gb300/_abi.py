"""ctypes view of the C ABI in include/gipc.h (argument marshalling only).

Loading fails loudly when the in-tree library has not been built: there is no
fallback implementation.
"""
import ctypes
import os

from .build import LIB

GIPC_OK = 0
STATUS_NAMES = {0: "GIPC_OK", -1: "GIPC_ERR_INVALID_ARG", -2: "GIPC_ERR_CUDA", -3: "GIPC_ERR_OOM",
                -4: "GIPC_ERR_NOT_CONVERGED", -5: "GIPC_ERR_NONFINITE", -6: "GIPC_ERR_TIMEOUT",
                -7: "GIPC_ERR_CAPACITY", -8: "GIPC_ERR_INDEFINITE"}

GIPC_FP64, GIPC_MIXED = 0, 1
GIPC_HESS_DENSE, GIPC_HESS_RANK1, GIPC_HESS_BLOCKS = 0, 1, 2
GIPC_PRODUCT_NATIVE, GIPC_PRODUCT_FLOAT_PAIR = 0, 1
GIPC_PCG_STOP_ON_INDEFINITE = 1

FLAG_ACTIVE, FLAG_FILTERED, FLAG_MOLLIFIED, FLAG_INVALID = 0x01, 0x02, 0x04, 0x80


class BarrierParams(ctypes.Structure):
    _fields_ = [("dhat", ctypes.c_double), ("kappa", ctypes.c_double), ("d_thr_ratio", ctypes.c_double)]


class Bsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnzb", ctypes.c_int64), ("capacity", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("prec", ctypes.c_int)]


class Elements(ctypes.Structure):
    _fields_ = [("idx", ctypes.c_void_p), ("count", ctypes.c_int64), ("hess_mode", ctypes.c_int),
                ("hess", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("grad", ctypes.c_void_p)]


class ElasticParams(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("lam", ctypes.c_double), ("scale", ctypes.c_double)]


class PcgParams(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("product", ctypes.c_int), ("flags", ctypes.c_int)]


class Surface(ctypes.Structure):
    _fields_ = [("tris", ctypes.c_void_p), ("ntri", ctypes.c_int64), ("edges", ctypes.c_void_p),
                ("nedge", ctypes.c_int64), ("verts", ctypes.c_void_p), ("nvert", ctypes.c_int64)]


class Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rest_x", ctypes.c_void_p), ("tets", ctypes.c_void_p),
                ("T", ctypes.c_int64), ("Dm_inv", ctypes.c_void_p), ("vol", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("fixed", ctypes.c_void_p), ("surface", Surface),
                ("l", ctypes.c_double)]


class SceneBatch(ctypes.Structure):
    _fields_ = [("all", Scene), ("nscenes", ctypes.c_int32), ("vert_off_h", ctypes.c_void_p), ("l_h", ctypes.c_void_p)]


class StepParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("elastic", ElasticParams),
                ("barrier", BarrierParams), ("eps_d", ctypes.c_double), ("pcg_tol", ctypes.c_double),
                ("max_pcg", ctypes.c_int), ("max_newton", ctypes.c_int), ("max_ls", ctypes.c_int),
                ("prec", ctypes.c_int), ("hess_mode", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("ls_trials", ctypes.c_int),
                ("converged", ctypes.c_int), ("contacts", ctypes.c_int64), ("energy", ctypes.c_double),
                ("last_alpha", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


SPMV_VARIANTS = 4


class SpmvTuning(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("size_class", ctypes.c_int), ("chosen", ctypes.c_int),
                ("U", ctypes.c_int * SPMV_VARIANTS), ("W", ctypes.c_int * SPMV_VARIANTS),
                ("NS", ctypes.c_int * SPMV_VARIANTS), ("samples", ctypes.c_int * SPMV_VARIANTS),
                ("mean_us", ctypes.c_double * SPMV_VARIANTS)]


SOLVER_PHASES = ("product", "barrier_a", "total_a", "vector", "barrier_b", "total_b", "direction", "barrier_c",
                 "iteration")

PROF_KINDS = {"pcg_spmv": 0, "pcg_update": 1, "pcg_direction": 2, "asm_pattern": 3, "asm_values": 4,
              "contacts": 5, "ccd": 6, "elements": 7, "energy": 8, "pcg_loop": 9}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "gipc_create": (_INT, [ctypes.POINTER(_P)]),
    "gipc_destroy": (_INT, [_P]),
    "gipc_last_error": (ctypes.c_char_p, []),
    "gipc_compute_eps_x": (_INT, [_P, _I64, _P, _I64, _P, _P]),
    "gipc_eval_stencils": (_INT, [_P, _I64, _P, _I64, _P, ctypes.POINTER(BarrierParams), _INT, _INT,
                                  _P, _P, _P, _P, _P, _P]),
    "gipc_snh_params": (_INT, [_D, _D, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gipc_tet_rest": (_INT, [_P, _P, _I64, _P, _I64, _D, _P, _P, _P, _P]),
    "gipc_eval_tets": (_INT, [_P, _I64, _P, _I64, _P, _P, ctypes.POINTER(ElasticParams), _INT, _INT, _P, _P, _P, _P]),
    "gipc_assemble_bsr": (_INT, [_P, _I64, ctypes.POINTER(Elements), ctypes.POINTER(Elements), _P, _P,
                                 ctypes.POINTER(Bsr), _P, _P]),
    "gipc_pcg": (_INT, [_P, ctypes.POINTER(Bsr), _P, _P, _P, ctypes.POINTER(PcgParams),
                        ctypes.POINTER(_INT), ctypes.POINTER(_D), _P]),
    "gipc_pcg_noalloc": (_INT, [ctypes.POINTER(Bsr), _P, _P, _P, ctypes.POINTER(PcgParams),
                                ctypes.POINTER(_INT), ctypes.POINTER(_D), _P]),
    "gipc_profile_solver_trace": (_INT, [_P, _INT]),
    "gipc_profile_solver_phases": (_INT, [_P, ctypes.POINTER(_D), ctypes.POINTER(_INT)]),
    "gipc_spmv_autotune": (_INT, [_P, _INT]),
    "gipc_pcg_batch_persistent": (_INT, [_P, _INT]),
    "gipc_spmv_tunings": (_INT, [_P, _P, _INT, ctypes.POINTER(_INT)]),
    "gipc_find_contacts": (_INT, [_P, _P, _P, _I64, ctypes.POINTER(Surface), _D, _P, _P, _I64,
                                  ctypes.POINTER(_I64), _P]),
    "gipc_ccd_max_step": (_INT, [_P, _P, _P, _I64, ctypes.POINTER(Surface), _D, ctypes.POINTER(_D), _P]),
    "gipc_newton_step": (_INT, [_P, ctypes.POINTER(Scene), _P, _P, ctypes.POINTER(StepParams),
                                ctypes.POINTER(StepStats), _P]),
    "gipc_newton_step_batch": (_INT, [_P, ctypes.POINTER(SceneBatch), _P, _P, ctypes.POINTER(StepParams), _P, _P]),
    "gipc_scatter_elements": (_INT, [_P, _I64, ctypes.POINTER(Elements), ctypes.POINTER(Elements), _P, _P, _P]),
    "gipc_potential_derivs": (_INT, [_P, ctypes.POINTER(Scene), _P, _P, _P, _P, _I64, ctypes.POINTER(BarrierParams),
                                     ctypes.POINTER(ElasticParams), _P, ctypes.POINTER(_D), _P, _P, _P]),
    "gipc_potential_hessian": (_INT, [_P, ctypes.POINTER(Scene), _P, _P, _P, _I64, ctypes.POINTER(BarrierParams),
                                      ctypes.POINTER(ElasticParams), ctypes.POINTER(Bsr), _P]),
    "gipc_adjoint_step": (_INT, [_P, ctypes.POINTER(Scene), _P, _P, _P, ctypes.POINTER(StepParams), _P, _P, _P, _P,
                                 ctypes.POINTER(_D), ctypes.POINTER(_INT), _P]),
    "gipc_newton_polish": (_INT, [_P, ctypes.POINTER(Scene), _P, _P, _P, _P, ctypes.POINTER(StepParams), ctypes.c_double,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), _P]),
    "gipc_profile_begin": (_INT, [_P]),
    "gipc_profile_sampling": (_INT, [_P, _INT, _INT]),
    "gipc_profile_read": (_INT, [_P, _INT, ctypes.POINTER(KernelTime)]),
    "gipc_profile_stop": (_INT, [_P]),
}

_lib = None


class GipcError(RuntimeError):
    def __init__(self, fn, status):
        msg = lib().gipc_last_error().decode(errors="replace")
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"GIPC CUDA library not built ({LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


GIPC_ERR_CAPACITY = -7
GIPC_ERR_INDEFINITE = -8
GIPC_ERR_NOT_CONVERGED = -4


def call_status(name, *args):
    """Call without raising; returns the status."""
    return getattr(lib(), name)(*args)


def call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != GIPC_OK:
        raise GipcError(name, st)
    return st
