"""ctypes binding of libmgmlmc.so (the C ABI of include/mgmlmc.h).

Only argument marshalling lives here.  The shared library is loaded from the
package directory (built in-tree by `paper_2303_11512_gb300.build`); there is
no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgmlmc.so")

MAX_LEVELS = 8
OK, ERR_INVALID_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_CUDA, ERR_TIMEOUT, ERR_NAN, ERR_NOT_POSDEF = 0, -1, -2, -3, -4, -5, -6, -7
FP64, FP32, MIXED, TF32, BF16, FP16 = 0, 1, 2, 3, 4, 5
ACCUMULATED, REDUCED = 0, 1
OPTIMAL, UNIFORM = 0, 1
PHASE_STOCH, PHASE_SKETCH, PHASE_TESTVEC, PHASE_HUTCH = 0, 1, 2, 3
NOISE_RADEMACHER, NOISE_Z4 = 0, 1
TRACE_PLAIN, TRACE_GAMMA5 = 0, 1


class MgParams(C.Structure):
    _fields_ = [("levels", C.c_int), ("agg", C.c_int), ("ntv", C.c_int), ("sap_block_fine", C.c_int),
                ("sap_block_coarse", C.c_int), ("setup_sweeps", C.c_int), ("pre_smooth", C.c_int),
                ("post_smooth", C.c_int), ("seed", C.c_uint64), ("bootstrap", C.c_int),
                ("bootstrap_its", C.c_int), ("kcycle_its", C.c_int), ("kcycle_tol", C.c_double),
                ("tensor_cores", C.c_int), ("graphs", C.c_int), ("autotune", C.c_int)]


class SolveParams(C.Structure):
    _fields_ = [("m", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("precond", C.c_int),
                ("prec", C.c_int), ("inner_tol", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("max_relres", C.c_double), ("converged", C.c_int),
                ("total_iters", C.c_int64)]


class EstParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("d", C.c_int * MAX_LEVELS), ("k", C.c_int), ("nrhs_max", C.c_int),
                ("nrhs_first", C.c_int), ("policy", C.c_int), ("form", C.c_int), ("seed", C.c_uint64),
                ("cost", C.c_double * MAX_LEVELS), ("cost_mode", C.c_int), ("min_samples", C.c_int),
                ("max_samples", C.c_int64), ("solve", SolveParams),
                ("sample_out", C.POINTER(C.c_double) * MAX_LEVELS), ("sample_cap", C.c_int64),
                ("noise", C.c_int), ("weight", C.c_int)]


class EstResult(C.Structure):
    _fields_ = [("tau", C.c_double * 2), ("sigma", C.c_double), ("tau_L", C.c_double * 2), ("nlev", C.c_int),
                ("N", C.c_int64 * MAX_LEVELS), ("computed", C.c_int64 * MAX_LEVELS),
                ("mean", (C.c_double * 2) * MAX_LEVELS), ("V", C.c_double * MAX_LEVELS),
                ("C", C.c_double * MAX_LEVELS), ("tau_lr", (C.c_double * 2) * MAX_LEVELS),
                ("solves", C.c_int64), ("inner_iters", C.c_int64), ("steps", C.c_int), ("flops", C.c_double)]


class HutchParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("nrhs_first", C.c_int), ("nrhs_max", C.c_int), ("seed", C.c_uint64),
                ("noise", C.c_int), ("weight", C.c_int), ("min_samples", C.c_int), ("max_samples", C.c_int64),
                ("solve", SolveParams), ("sample_out", C.POINTER(C.c_double)), ("sample_cap", C.c_int64),
                ("deflate", C.c_void_p)]


class HutchResult(C.Structure):
    _fields_ = [("tau", C.c_double * 2), ("sigma", C.c_double), ("N", C.c_int64), ("computed", C.c_int64),
                ("solves", C.c_int64), ("inner_iters", C.c_int64), ("tau_defl", C.c_double * 2)]


vp = C.c_void_p
ip = C.c_int
dp = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "mgmlmc_version": (ip, []),
    "mgmlmc_ctx_create": (ip, [vp, C.POINTER(vp)]),
    "mgmlmc_ctx_destroy": (None, [vp]),
    "mgmlmc_last_error": (C.c_char_p, [vp]),
    "mgmlmc_launch_count": (C.c_int64, [vp]),
    "mgmlmc_timing_enable": (ip, [vp, ip, C.c_char_p]),
    "mgmlmc_timing_report": (ip, [vp, C.c_char_p, C.c_int64]),
    "schwinger_apply": (ip, [vp, vp, ip, C.c_double, vp, vp, ip, ip]),
    "mgmlmc_rademacher": (ip, [vp, C.c_uint64, ip, ip, C.c_int64, C.c_int64, ip, vp]),
    "mgmlmc_noise": (ip, [vp, ip, C.c_uint64, ip, ip, C.c_int64, C.c_int64, ip, vp]),
    "mg_params_default": (ip, [C.POINTER(MgParams)]),
    "mg_setup": (ip, [vp, vp, ip, C.c_double, C.POINTER(MgParams), C.POINTER(vp)]),
    "mg_destroy": (None, [vp]),
    "mg_num_levels": (ip, [vp]),
    "mg_level_info": (ip, [vp, ip, C.POINTER(ip), C.POINTER(ip), C.POINTER(C.c_int64)]),
    "mg_coarsest_trace": (ip, [vp, dp]),
    "mg_apply": (ip, [vp, vp, ip, vp, vp, ip, ip]),
    "mg_restrict": (ip, [vp, vp, ip, vp, vp, ip, ip]),
    "mg_prolong": (ip, [vp, vp, ip, vp, vp, ip, ip]),
    "mg_get_prolongator": (ip, [vp, vp, ip, vp]),
    "mg_get_stencil": (ip, [vp, vp, ip, vp]),
    "mg_vcycle": (ip, [vp, vp, ip, vp, vp, ip, ip]),
    "mg_dense_inverse": (ip, [vp, vp, ip, ip, C.c_int64]),
    "hutchpp_cholqr2": (ip, [vp, vp, ip, C.c_int64]),
    "mg_smooth": (ip, [vp, vp, ip, vp, vp, ip, ip, ip]),
    "mg_tc_status": (ip, [vp, vp]),
    "mg_autotune": (ip, [vp, vp, C.POINTER(ip), ip, ip]),
    "mgmlmc_tune_report": (ip, [C.c_char_p, C.c_int64]),
    "mgmlmc_tune_set": (ip, [ip, ip, ip, ip, ip]),
    "mgmlmc_tune_clear": (ip, []),
    "solve_params_default": (ip, [C.POINTER(SolveParams)]),
    "fgmres_batched": (ip, [vp, vp, ip, vp, vp, ip, C.POINTER(SolveParams), C.POINTER(SolveStats), vp]),
    "mlmc_level_sample": (ip, [vp, vp, ip, ip, vp, vp, ip, C.POINTER(SolveParams), C.POINTER(SolveStats)]),
    "mg_restrict_to_level": (ip, [vp, vp, ip, vp, vp, ip]),
    "hutchpp_sketch_qr": (ip, [vp, vp, ip, ip, ip, C.c_uint64, ip, C.POINTER(SolveParams), C.POINTER(vp), dp]),
    "hutchpp_sketch_destroy": (None, [vp]),
    "hutchpp_sketch_get_q": (ip, [vp, vp, vp, C.POINTER(ip), C.POINTER(C.c_int64)]),
    "hutchpp_project": (ip, [vp, vp, vp, vp, C.c_int64, ip, dp]),
    "hutchpp_project_noalloc": (ip, [vp, vp, ip, vp, vp, C.c_int64, ip, vp]),
    "nn_create": (ip, [vp, vp, ip, ip, ip, C.c_uint64, C.POINTER(vp)]),
    "nn_destroy": (None, [vp]),
    "nn_num_params": (C.c_int64, [vp]),
    "nn_set_params": (ip, [vp, vp, vp]),
    "nn_get_params": (ip, [vp, vp, vp]),
    "nn_forward": (ip, [vp, vp, vp, vp, ip]),
    "nn_loss_grad": (ip, [vp, vp, vp, vp, ip, dp, vp]),
    "nn_train_step": (ip, [vp, vp, vp, vp, ip, C.c_double, dp]),
    "nn_set_format": (ip, [vp, vp, ip]),
    "nn_get_format": (ip, [vp]),
    "mgmlmc_alu_peak": (ip, [vp, ip, dp]),
    "nn_set_field": (ip, [vp, vp, vp, ip]),
    "nn_harvest_pairs": (ip, [vp, vp, C.c_uint64, C.c_int64, ip, C.c_double, vp, vp]),
    "mg_attach_nn": (ip, [vp, vp, vp]),
    "est_params_default": (ip, [C.POINTER(EstParams)]),
    "trace_estimate": (ip, [vp, vp, C.POINTER(EstParams), C.POINTER(EstResult)]),
    "hutch_params_default": (ip, [C.POINTER(HutchParams)]),
    "hutchinson_estimate": (ip, [vp, vp, C.POINTER(HutchParams), C.POINTER(HutchResult)]),
    "deflation_basis": (ip, [vp, vp, ip, ip, C.c_uint64, C.POINTER(SolveParams), C.POINTER(vp), dp, dp]),
    "mlmc_update_active": (ip, [ip, C.POINTER(ip), dp, C.POINTER(C.c_int64), dp, C.c_double, C.c_double, ip, ip]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmgmlmc.so not built: run `python -m paper_2303_11512_gb300.build` "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class MgmlmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("mgmlmc error %d: %s" % (code, msg))
        self.code = code


def check(rc: int, ctx=None):
    if rc != OK:
        msg = load().mgmlmc_last_error(ctx).decode() if ctx else ""
        raise MgmlmcError(rc, msg)
