"""ctypes declarations of libap.so (include/ap.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

from . import _build

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F64 = ctypes.c_double

AP_OK = 0
ERRORS = {1: "AP_ERR_ARG", 2: "AP_ERR_CUDA", 3: "AP_ERR_CAPACITY", 4: "AP_ERR_NONFINITE", 5: "AP_ERR_TIMEOUT",
          6: "AP_ERR_STATE", 7: "AP_ERR_RADICAND", 8: "AP_ERR_BOX", 9: "AP_ERR_SKIN"}
PREC_FP64 = 0
PREC_MIXED = 1
DETECT_CSP = 0
REBUILD_SKIN = -1
DETECT_SELECTOR = 1
EAM_ANALYTIC = 0
EAM_MISHIN = 1
SEL_NFEAT = 24
SEL_NPARAMS = 5825
F32 = ctypes.c_float


class ApBox(ctypes.Structure):
    _fields_ = [("lo", F64 * 3), ("hi", F64 * 3), ("periodic", I32 * 3)]


class ApConfig(ctypes.Structure):
    _fields_ = ([(k, F64) for k in ("eam_beta", "eam_alpha", "eam_A", "eam_D", "eam_rp", "eam_r0", "eam_rc", "eam_h")]
                + [("ace_W", F64 * 320), ("ace_c", F64 * 512), ("ace_nc", I32), ("ace_rc", F64), ("ace_n0", F64),
                   ("csp_lo", F64), ("csp_hi", F64), ("r_lo", F64), ("r_hi", F64), ("dlam_min", F64),
                   ("n_csp_avg", I32), ("n_lam_avg", I32), ("fcut_mode", I32), ("skin", F64), ("cap_eam", I32),
                   ("cap_ace", I32), ("precision", I32), ("dt", F64), ("lambda_every", I32), ("indenter_on", I32),
                   ("ind_c0", F64 * 3), ("ind_v", F64 * 3), ("ind_R", F64), ("ind_k", F64),
                   ("rebuild_every", I32), ("detector", I32), ("sel_p_lo", F64), ("sel_p_hi", F64),
                   ("thermostat_on", I32), ("ace_fs_on", I32), ("ace_fs_eps", F64), ("ace_c2", F64 * 512),
                   ("eam_type", I32), ("eam_mishin", F64 * 29), ("ace_deterministic", I32)])


class ApStepStats(ctypes.Structure):
    _fields_ = [("step", I64), ("n_precise", I64), ("n_detected", I64), ("rebuilds", I64), ("e_pot", F64),
                ("e_kin", F64), ("max_disp", F64), ("error_bits", I32), ("th_corrected", I64), ("th_refused", I64),
                ("th_energy", F64), ("kept", I64), ("ace_rebuilds", I64)]


class ApError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{ERRORS.get(status, status)}: {msg}")
        self.status = status


# (name, restype, argtypes) of every entry point declared in include/ap.h
SIGNATURES = [
    ("ap_create", I32, [P, P]),
    ("ap_destroy", None, [P]),
    ("ap_last_error", ctypes.c_char_p, [P]),
    ("ap_need", I64, [P]),
    ("ap_ace_nbasis", I32, [P]),
    ("ap_ace_basis_desc", I32, [P, P]),
    ("ap_ace_gaunt", I32, [P, P]),
    ("ap_build_neighbors", I32, [P, I64, P, P, P, P]),
    ("ap_build_neighbors_batch", I32, [P, I32, P, P, P, P, P]),
    ("ap_get_neighbors", I32, [P, I32, P, P, P, I64, P]),
    ("ap_neighbor_total", I32, [P, I32, P]),
    ("ap_spatial_order", I32, [P, P, P]),
    ("ap_classify", I32, [P, I64, P, P, I32, P, P, P, P]),
    ("ap_reset_lambda", I32, [P]),
    ("ap_precise_queue", I32, [P, I64, P, P, P, P]),
    ("ap_get_lambda_state", I32, [P, P, P, P, P, P, P]),
    ("ap_eval_eam", I32, [P, I64, P, P, P, P, P, P]),
    ("ap_eval_ace", I32, [P, I64, P, P, P, P, P, P, P]),
    ("ap_blend_forces", I32, [P, I64, P, P, P, P, P, P]),
    ("ap_step", I32, [P, I64, P, P, P, P, P, P, I64, P, P]),
    ("ap_eval_eam_static", I32, [P, I64, P, P, P, P, P, P]),
    ("ap_profile_enable", I32, [P, I32]),
    ("ap_profile_read", I32, [P, P, P, P, P, P]),
    ("ap_profile_mma", I32, [P, P]),
    ("ap_probe_peak", I32, [I32, I32, P, P, P]),
    ("ap_state_export", I32, [P, P, P]),
    ("ap_state_import", I32, [P, P, ctypes.c_size_t]),
    ("ap_sel_set_model", I32, [P, P, P, P]),
    ("ap_sel_get_model", I32, [P, P, P, P]),
    ("ap_sel_features", I32, [P, I64, P, P, P, P]),
    ("ap_sel_predict", I32, [P, I64, P, P, P, P]),
    ("ap_sel_train_step", I32, [P, I64, P, P, P, P, F32, F32, F32, F32, P, P]),
    ("ap_sel_get_grad", I32, [P, P, P]),
]

_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libap.so, compiling it first if it is missing or stale.  Raises if
    the CUDA library cannot be built or loaded: there is no other path."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libap.so not found at {path}")
        l = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(l, name)
            fn.restype = res
            fn.argtypes = args
        _lib = l
    return _lib
