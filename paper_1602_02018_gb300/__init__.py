"""Compressive Spectral Clustering on GB300 (sm_103a).

The computation lives in the CUDA library libcsc (``csrc/``, ABI in
``include/csc.h``); this package only marshals arguments to it.  Build the
library with ``paper_1602_02018_gb300.build.build()``.
"""
from .api import (  # noqa: F401
    BF16,
    CHECK_SYM,
    DEVICE_INPUT,
    F32,
    F64,
    NO_JACKSON,
    NORMALIZE_ROWS,
    RCM,
    CgInfo,
    ClusterInfo,
    Graph,
    LambdaInfo,
    csc_chebyshev_coefficients,
    csc_cluster,
    csc_eigencount,
    csc_estimate_lambda_k,
    csc_filter_random_signals,
    csc_gather_rows,
    csc_graph_create,
    csc_graph_create_batched,
    csc_graph_degrees,
    csc_graph_pin_shape,
    csc_graph_tuned_shapes,
    csc_interpolate,
    csc_kmeans_reduced,
    csc_kpm_moments,
    csc_profile_enable,
    csc_profile_launches,
    csc_profile_query,
    csc_profile_reset,
    csc_sample,
    csc_sample_noalloc,
    default_sizes,
)
from ._native import CscError, header_symbols, lib  # noqa: F401
