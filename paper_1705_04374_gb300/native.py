"""ctypes binding of ``libofmlmc.so`` (the C ABI declared in include/ofmlmc.h).

Argument marshalling only: every computation runs in the library.  The
structures below mirror the header field by field; the functions keep the
header's names.  Loading fails with an ImportError if the library has not
been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libofmlmc.so")

OFM_OK, OFM_EINVAL, OFM_ENOMEM, OFM_ECUDA, OFM_ENUMERIC, OFM_ETIMEOUT = 0, -1, -2, -3, -4, -5
OFM_FP64, OFM_FP32 = 0, 1
OFM_BC_TRANSMISSIVE, OFM_BC_PERIODIC, OFM_BC_CHARACTERISTIC = 0, 1, 2
OFM_RADII_UNIFORM, OFM_RADII_LOGNORMAL = 0, 1
OFM_MODE_TOL, OFM_MODE_BUDGET = 0, 1
OFM_ST_NONFINITE, OFM_ST_NEGATIVE, OFM_ST_MAXSTEPS, OFM_ST_TIMEOUT = 1, 2, 4, 8
OFM_MAX_SENSORS, OFM_MAX_GROUPS, OFM_MAX_LEVELS = 8, 8, 16
OFM_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


class ofm_bubble(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("r", C.c_double)]


class ofm_cloud_params(C.Structure):
    _fields_ = [("n_bubbles", C.c_int), ("radius_law", C.c_int), ("cloud_radius", C.c_double),
                ("r_min", C.c_double), ("r_max", C.c_double), ("ln_mu", C.c_double),
                ("ln_sigma", C.c_double), ("domain_L", C.c_double)]


class ofm_solver_config(C.Structure):
    _fields_ = [("gamma", C.c_double * 2), ("pc", C.c_double * 2), ("rho0", C.c_double * 2),
                ("p_gas", C.c_double), ("p_liq", C.c_double), ("cfl", C.c_double),
                ("t_end", C.c_double), ("weno_eps", C.c_double), ("domain_L", C.c_double),
                ("precision", C.c_int), ("bc", C.c_int), ("max_steps", C.c_int),
                ("n_sensors", C.c_int), ("sensors", (C.c_double * 4) * OFM_MAX_SENSORS),
                ("n_out_times", C.c_int), ("p_cloud", C.c_double), ("ramp_radius", C.c_double),
                ("bc_penalty", C.c_double), ("weno_order", C.c_int)]


class ofm_qoi(C.Structure):
    _fields_ = [("p_peak", C.c_double), ("p_peak_xyz", C.c_double * 3), ("p_peak_t", C.c_double),
                ("p_peak_dist", C.c_double), ("peak_index", C.c_int64),
                ("sensor_peak", C.c_double * OFM_MAX_SENSORS), ("totals0", C.c_double * 6),
                ("totals_end", C.c_double * 6), ("t_final", C.c_double), ("n_steps", C.c_int),
                ("status", C.c_int), ("c_max", C.c_double), ("sensor_alpha0", C.c_double * OFM_MAX_SENSORS),
                ("sensor_alpha_min", C.c_double * OFM_MAX_SENSORS),
                ("sensor_alpha_min_t", C.c_double * OFM_MAX_SENSORS)]


class ofm_group(C.Structure):
    _fields_ = [("N", C.c_int), ("n_samples", C.c_int), ("sample_ids", C.POINTER(C.c_uint64)),
                ("seed", C.c_uint64), ("bubbles", C.POINTER(ofm_bubble)),
                ("qoi_out", C.POINTER(ofm_qoi)), ("sensor_hist", C.POINTER(C.c_double)),
                ("alpha_hist", C.POINTER(C.c_double))]


class ofm_level_moments(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean_f", C.c_double), ("mean_c", C.c_double), ("m2_f", C.c_double),
                ("m2_c", C.c_double), ("c_fc", C.c_double)]


class ofm_estimate_out(C.Structure):
    _fields_ = [("alpha", C.c_double * OFM_MAX_LEVELS), ("sigma2", C.c_double * OFM_MAX_LEVELS),
                ("cov", C.c_double * OFM_MAX_LEVELS), ("sigma_tilde2", C.c_double * OFM_MAX_LEVELS),
                ("mean", C.c_double), ("eps2", C.c_double)]


class ofm_run_config(C.Structure):
    _fields_ = [("L", C.c_int), ("N", C.c_int * OFM_MAX_LEVELS), ("mode", C.c_int), ("target", C.c_double),
                ("qoi", C.c_int), ("seed", C.c_uint64), ("max_iterations", C.c_int), ("min_samples", C.c_int),
                ("max_batch_bytes", C.c_size_t), ("max_cell_steps", C.c_double), ("fit_variances", C.c_int),
                ("surrogate", C.c_int), ("surrogate_min_pairs", C.c_int), ("surrogate_nearest", C.c_int),
                ("surrogate_steps", C.c_int), ("surrogate_hidden", C.c_int), ("surrogate_lr", C.c_double),
                ("surrogate_h_out", C.POINTER(C.c_double))]


class ofm_run_result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("M", C.c_int64 * OFM_MAX_LEVELS), ("W", C.c_double * OFM_MAX_LEVELS),
                ("gpu_seconds", C.c_double), ("cell_steps", C.c_double), ("failed", C.c_int64),
                ("capped", C.c_int), ("est", ofm_estimate_out), ("surrogate_used", C.c_int), ("beta", C.c_double),
                ("surrogate_seconds", C.c_double), ("eps2_plain", C.c_double),
                ("sigma_tilde2_plain", C.c_double * OFM_MAX_LEVELS)]


_vp = C.c_void_p
_P = C.POINTER

# name -> (restype, argtypes), in header order
SIGNATURES = {
    "ofm_last_error": (C.c_char_p, []),
    "ofm_version": (C.c_char_p, []),
    "ofm_sample_cloud": (C.c_int, [_P(ofm_cloud_params), C.c_uint64, C.c_uint64, _P(ofm_bubble)]),
    "ofm_solver_create": (C.c_int, [_P(_vp), _P(ofm_solver_config)]),
    "ofm_solver_destroy": (None, [_vp]),
    "ofm_batch_workspace_bytes": (C.c_int, [_vp, _P(ofm_cloud_params), _P(ofm_group), C.c_int,
                                            _P(C.c_size_t)]),
    "ofm_batch_create": (C.c_int, [_P(_vp), _vp, _P(ofm_cloud_params), _P(ofm_group), C.c_int, _vp,
                                   C.c_size_t, _vp]),
    "ofm_batch_init": (C.c_int, [_vp]),
    "ofm_batch_run": (C.c_int, [_vp, C.c_int, _P(C.c_int)]),
    "ofm_batch_qoi": (C.c_int, [_vp]),
    "ofm_batch_copy_state": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_size_t]),
    "ofm_batch_set_state": (C.c_int, [_vp, C.c_int, C.c_int, _vp, C.c_size_t]),
    "ofm_batch_cell_steps": (C.c_int, [_vp, _P(C.c_double)]),
    "ofm_batch_kernel_launches": (C.c_int, [_vp, _P(C.c_int64)]),
    "ofm_batch_set_profiling": (C.c_int, [_vp, C.c_int]),
    "ofm_batch_set_variant": (C.c_int, [_vp, C.c_int]),
    "ofm_batch_get_variant": (C.c_int, [_vp, _P(C.c_int), _P(C.c_float)]),
    "ofm_batch_stage_time": (C.c_int, [_vp, _P(C.c_double), _P(C.c_int64)]),
    "ofm_batch_transfer_bytes": (C.c_int, [_vp, _P(C.c_int64), _P(C.c_int64)]),
    "ofm_batch_destroy": (None, [_vp]),
    "ofm_solve_batch": (C.c_int, [_vp, _P(ofm_cloud_params), _P(ofm_group), C.c_int, _vp, C.c_size_t,
                                  _vp]),
    "ofm_solve_level": (C.c_int, [_vp, _P(ofm_cloud_params), C.c_int, C.c_int, _P(C.c_uint64),
                                  C.c_uint64, _P(ofm_qoi), _P(C.c_double), _vp, C.c_size_t, _vp]),
    "ofm_solve_level_static": (C.c_int, [_vp, _P(ofm_cloud_params), C.c_int, C.c_int, _P(C.c_uint64),
                                         C.c_uint64, _P(ofm_qoi), _P(C.c_double), _vp]),
    "ofm_run": (C.c_int, [_vp, _P(ofm_cloud_params), _P(ofm_run_config), _P(C.c_double), _P(C.c_uint64),
                          C.c_int64, _P(ofm_run_result), _vp]),
    "ofm_estimate_surrogate": (C.c_int, [C.c_int, _P(C.c_int64), _P(_P(C.c_double)), _P(C.c_double),
                                         _P(C.c_double), _P(C.c_double), C.c_double, _P(ofm_estimate_out),
                                         _P(C.c_double), _P(C.c_double)]),
    "ofm_sj_bandwidth": (C.c_int, [_P(C.c_double), C.c_int64, _P(C.c_double)]),
    "ofm_level_kde": (C.c_int, [C.c_int, _P(C.c_int64), _P(_P(C.c_double)), _P(C.c_double), _P(C.c_double),
                                C.c_int64, _P(C.c_double), _P(C.c_double)]),
    "ofm_surrogate_cv": (C.c_int, [_P(C.c_double), _P(C.c_double), C.c_int64, _P(C.c_double), C.c_int64,
                                   _P(C.c_double), _P(C.c_double), _P(C.c_double)]),
    "ofm_mlp_workspace_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P(C.c_size_t)]),
    "ofm_mlp_create": (C.c_int, [_P(_vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, C.c_size_t]),
    "ofm_mlp_destroy": (None, [_vp]),
    "ofm_mlp_param_count": (C.c_int, [_vp, _P(C.c_int64)]),
    "ofm_mlp_set_params": (C.c_int, [_vp, _P(C.c_float)]),
    "ofm_mlp_get_params": (C.c_int, [_vp, _P(C.c_float)]),
    "ofm_mlp_set_scaling": (C.c_int, [_vp, _P(C.c_float), _P(C.c_float), _P(C.c_float), _P(C.c_float)]),
    "ofm_mlp_forward": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp]),
    "ofm_mlp_gradients": (C.c_int, [_vp, _vp, _vp, C.c_int, _P(C.c_float), _P(C.c_float), _vp]),
    "ofm_mlp_train": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _P(C.c_float), _vp]),
    "ofm_column_moments": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp]),
    "ofm_cloud_features": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _vp, _vp]),
    "ofm_estimate": (C.c_int, [C.c_int, _P(C.c_int64), _P(_P(C.c_double)), _P(C.c_double),
                               _P(ofm_estimate_out)]),
    "ofm_estimate_fitted": (C.c_int, [C.c_int, _P(C.c_int64), _P(_P(C.c_double)), _P(C.c_double),
                                      _P(ofm_estimate_out), _P(C.c_double)]),
    "ofm_fit_level_variances": (C.c_int, [C.c_int, _P(C.c_int64), _P(C.c_double), _P(C.c_double),
                                          _P(C.c_double)]),
    "ofm_level_moments_of": (C.c_int, [_P(C.c_double), C.c_int64, _P(ofm_level_moments)]),
    "ofm_merge_moments": (C.c_int, [_P(ofm_level_moments), _P(ofm_level_moments), _P(ofm_level_moments)]),
    "ofm_estimate_moments": (C.c_int, [C.c_int, _P(ofm_level_moments), _P(C.c_double), _P(ofm_estimate_out)]),
    "ofm_estimate_moments_fitted": (C.c_int, [C.c_int, _P(ofm_level_moments), _P(C.c_double),
                                              _P(ofm_estimate_out), _P(C.c_double)]),
    "ofm_probe_fma_tflops": (C.c_int, [C.c_int, _P(C.c_double), _vp]),
    "ofm_optimal_samples": (C.c_int, [C.c_int, _P(C.c_double), _P(C.c_double), _P(C.c_int64),
                                      C.c_double, C.c_int, _P(C.c_int64)]),
    "ofm_warmup_samples": (C.c_int, [C.c_int, _P(C.c_double), _P(C.c_int64)]),
}

_lib = None


def lib() -> C.CDLL:
    """Load the library (once).  Raises ImportError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class OfmError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().ofm_last_error().decode(errors="replace")
        super().__init__(f"{where}: error {code}: {msg}")
        self.code = code


def check(code: int, where: str) -> int:
    if code != OFM_OK:
        raise OfmError(code, where)
    return code
