"""ctypes declarations of libcsc (include/csc.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcsc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "csc.h")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_uint32 = ctypes.c_uint32
c_uint64 = ctypes.c_uint64
c_double = ctypes.c_double
c_float = ctypes.c_float
c_void_p = ctypes.c_void_p
P = ctypes.POINTER

# status codes and flags (mirrors include/csc.h)
CSC_OK = 0
CSC_E_INVALID = 1
CSC_E_CSR = 2
CSC_E_OOM = 3
CSC_E_CUDA = 4
CSC_E_NOT_CONVERGED = 5
CSC_E_DEVICE_TIMEOUT = 6
CSC_E_NUMERIC = 7
CSC_E_UNSUPPORTED = 8

CSC_F32, CSC_BF16, CSC_F64 = 0, 1, 2
CSC_RCM, CSC_CHECK_SYM, CSC_DEVICE_INPUT, CSC_DEGREE_ORDER = 1, 2, 4, 8
CSC_NORMALIZE_ROWS, CSC_NO_JACKSON, CSC_CLENSHAW, CSC_HIGHPASS, CSC_VARDENSITY = 1, 2, 4, 8, 16
CSC_CHECK_FINITE = 32
CSC_MLP_IN, CSC_MLP_HIDDEN, CSC_MLP_OUT, CSC_MLP_PARAMS = 72, 256, 2, 84994
CSC_BRACKET_PROBES, CSC_BRACKET_MOMENTS = 8, 64
CSC_EIGENCOUNT_REFILTER = 1


class csc_lambda_info(ctypes.Structure):
    _fields_ = [("lambda_", c_double), ("count", c_double), ("iters", c_int32), ("hit", c_int32),
                ("n_probes", c_int32), ("m", c_int32), ("bracket_used", c_int32), ("moment_passes", c_int32)]


class csc_cg_info(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("converged", c_int32), ("max_rel_residual", c_double)]


class csc_params(ctypes.Structure):
    _fields_ = [("k", c_int32), ("m", c_int32), ("d", c_int32), ("d_pad", c_int32), ("n", c_int64),
                ("n_probes", c_int32), ("g_power", c_int32), ("gamma", c_double), ("cg_tol", c_double),
                ("cg_max_iter", c_int32), ("replicates", c_int32), ("km_max_iter", c_int32),
                ("storage", c_int32), ("seed", c_uint64), ("lambda_k", c_double), ("bracket", P(c_double)),
                ("flags", c_uint32), ("m_count", c_int32), ("m_interp", c_int32)]


class csc_batch_info(ctypes.Structure):
    _fields_ = [("cg", csc_cg_info), ("lambda_hits", c_int32), ("ms_lambda", c_float), ("ms_filter", c_float),
                ("ms_sample", c_float), ("ms_kmeans", c_float), ("ms_interp", c_float), ("ms_total", c_float)]


class csc_cluster_info(ctypes.Structure):
    _fields_ = [("lambda_", csc_lambda_info), ("cg", csc_cg_info), ("inertia", c_double),
                ("ms_lambda", c_float), ("ms_filter", c_float), ("ms_sample", c_float),
                ("ms_kmeans", c_float), ("ms_interp", c_float), ("ms_total", c_float)]


_SIGNATURES = {
    "csc_graph_create": [c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_uint32, c_void_p, P(c_void_p)],
    "csc_graph_create_batched": [c_int32, c_void_p, c_void_p, c_void_p, c_uint32, c_void_p, P(c_void_p)],
    "csc_graph_destroy": [c_void_p],
    "csc_graph_info": [c_void_p, P(c_int64), P(c_int64), P(c_int32)],
    "csc_graph_degrees": [c_void_p, c_void_p, c_void_p],
    "csc_graph_tuned_shape": [c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32), c_void_p],
    "csc_graph_pin_shape": [c_void_p, c_int32, c_int32, c_int32, c_void_p],
    "csc_chebyshev_coefficients": [c_double, c_int32, c_uint32, c_void_p],
    "csc_filter_random_signals": [c_void_p, c_double, c_int32, c_int32, c_int32, c_uint64, c_int32, c_void_p,
                                  c_void_p, c_uint32, c_void_p],
    "csc_kpm_moments": [c_void_p, c_int32, c_int32, c_uint64, c_int32, c_void_p, c_void_p],
    "csc_eigencount": [c_void_p, c_int32, c_double, c_uint32, P(c_double)],
    "csc_estimate_lambda_k": [c_void_p, c_int32, c_int32, c_int32, c_uint64, c_void_p, P(csc_lambda_info),
                              c_void_p],
    "csc_bracket_features": [c_void_p, c_int32, c_uint64, c_void_p, c_void_p, c_void_p],
    "csc_bracket_target": [c_void_p, c_int32, c_int32, c_void_p],
    "csc_mlp_init": [c_void_p, c_uint64, c_void_p],
    "csc_mlp_forward": [c_void_p, c_void_p, c_int32, c_void_p, c_void_p],
    "csc_mlp_loss_grad": [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p],
    "csc_mlp_adam_step": [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_float, c_void_p],
    "csc_mlp_train": [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_uint64, c_void_p,
                      c_void_p],
    "csc_bracket_fit": [c_void_p, c_void_p, c_int32, c_double, c_int32, c_int32, c_float, c_uint64, c_int32,
                        c_double, c_void_p, c_void_p, P(c_double), P(c_int32), c_void_p, c_void_p],
    "csc_bracket_predict": [c_void_p, c_void_p, c_double, c_void_p, c_int32, c_void_p, c_void_p, c_void_p],
    "csc_estimate_lambda_k_learned": [c_void_p, c_int32, c_int32, c_int32, c_uint64, c_void_p, c_void_p, c_double,
                                      c_uint32, P(csc_lambda_info), c_void_p, c_void_p],
    "csc_estimate_lambda_k_refilter": [c_void_p, c_int32, c_int32, c_int32, c_uint64, c_void_p,
                                       P(csc_lambda_info), c_void_p],
    "csc_kpm_moments_batched": [c_void_p, c_int32, c_int32, c_uint64, c_int32, c_void_p, c_void_p],
    "csc_estimate_lambda_k_batched": [c_void_p, c_void_p, c_int32, c_int32, c_uint64, c_void_p, c_void_p,
                                      c_void_p],
    "csc_filter_batched": [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_uint64, c_int32, c_void_p, c_void_p,
                           c_uint32, c_void_p],
    "csc_sample_batched": [c_void_p, c_void_p, c_uint64, c_void_p, c_void_p],
    "csc_kmeans_batched": [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_uint64,
                           c_void_p, c_void_p, c_void_p],
    "csc_interpolate_batched": [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_double, c_double,
                                c_int32, c_void_p, c_void_p, P(csc_cg_info), c_void_p],
    "csc_cluster_batched": [c_void_p, c_void_p, P(csc_params), c_void_p, c_void_p, P(csc_batch_info), c_void_p],
    "csc_interpolate_batched_highpass": [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int32, c_double,
                                         c_double, c_int32, c_void_p, c_void_p, P(csc_cg_info), c_void_p],
    "csc_interpolate_highpass": [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_double, c_int32, c_double,
                                 c_double, c_int32, c_void_p, c_void_p, P(csc_cg_info), c_void_p],
    "csc_sample": [c_int64, c_int64, c_uint64, c_void_p, c_void_p],
    "csc_coherence_scores": [c_void_p, c_int32, c_int64, c_int32, c_int32, c_int32, c_void_p, c_void_p],
    "csc_sample_weighted": [c_void_p, c_int64, c_int64, c_uint64, c_void_p, c_void_p, c_void_p],
    "csc_interpolate_weighted": [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_double,
                                 c_double, c_int32, c_void_p, c_void_p, P(csc_cg_info), c_void_p],
    "csc_sample_noalloc": [c_int64, c_int64, c_uint64, c_void_p, c_void_p],
    "csc_gather_rows": [c_void_p, c_int64, c_int32, c_void_p, c_int64, c_int32, c_void_p, c_int32, c_void_p],
    "csc_kmeans_reduced": [c_void_p, c_int64, c_int32, c_int32, c_int32, c_int32, c_int32, c_uint64, c_void_p,
                           P(c_double), c_void_p],
    "csc_interpolate": [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_double, c_double, c_int32,
                        c_void_p, c_void_p, P(csc_cg_info), c_void_p],
    "csc_cluster": [c_void_p, P(csc_params), c_void_p, P(csc_cluster_info), c_void_p],
    "csc_profile_enable": [c_int32],
    "csc_profile_reset": [],
    "csc_profile_launches": [P(c_int64)],
    "csc_profile_query": [c_int32, ctypes.c_char_p, c_int32, P(c_int64), P(c_double), P(c_double)],
    "csc_status_str": [c_int32],
    "csc_last_error": [],
    "csc_version": [],
}
_RESTYPE = {"csc_status_str": ctypes.c_char_p, "csc_last_error": ctypes.c_char_p, "csc_version": ctypes.c_char_p}

_lib = None


def header_symbols() -> list[str]:
    """Every entry point declared in include/csc.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"CSC_API\s+(?:csc_status|const char\*)\s+(csc_\w+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libcsc.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcsc.so not found at {LIB_PATH}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (CUDA toolkit required)")
    L = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, c_int32)
    _lib = L
    return L


class CscError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.csc_last_error().decode(errors="replace")
        name = L.csc_status_str(status).decode()
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str, allow=()) -> int:
    if status != CSC_OK and status not in allow:
        raise CscError(status, where)
    return status
