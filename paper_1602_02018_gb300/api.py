"""Python binding of libcsc with the C ABI's names (argument marshalling only).

Device arrays are torch CUDA tensors, host arrays numpy arrays; every step
of the computation runs in the CUDA library.  Streams default to torch's
current stream on the current device.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _native as nat
from ._native import check, lib

F32, BF16, F64 = nat.CSC_F32, nat.CSC_BF16, nat.CSC_F64
RCM, CHECK_SYM, DEVICE_INPUT, DEGREE_ORDER = nat.CSC_RCM, nat.CSC_CHECK_SYM, nat.CSC_DEVICE_INPUT, nat.CSC_DEGREE_ORDER
NORMALIZE_ROWS, NO_JACKSON, CLENSHAW, HIGHPASS, VARDENSITY = (nat.CSC_NORMALIZE_ROWS, nat.CSC_NO_JACKSON,
                                                              nat.CSC_CLENSHAW, nat.CSC_HIGHPASS,
                                                              nat.CSC_VARDENSITY)
CHECK_FINITE = nat.CSC_CHECK_FINITE


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Graph:
    """Owner of a csc_graph handle (freed on close / garbage collection)."""

    def __init__(self, handle: ctypes.c_void_p, keep=None):
        self.handle = handle
        self._keep = keep
        n, nnz, ng = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(lib().csc_graph_info(handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(ng)), "csc_graph_info")
        self.N, self.nnz, self.n_graphs = n.value, nnz.value, ng.value

    def close(self):
        if self.handle:
            lib().csc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def csc_graph_create(row_ptr, col_idx, flags: int = 0, stream=None) -> Graph:
    """Create a graph from CSR arrays: numpy (host) or CUDA tensors (adds CSC_DEVICE_INPUT)."""
    out = ctypes.c_void_p()
    if isinstance(row_ptr, torch.Tensor):
        rp = row_ptr.to(torch.int64).contiguous()
        ci = col_idx.to(torch.int32).contiguous()
        n = rp.numel() - 1
        check(lib().csc_graph_create(n, ci.numel(), _dptr(rp), _dptr(ci), None, flags | DEVICE_INPUT,
                                     _stream(stream), ctypes.byref(out)), "csc_graph_create")
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        n = rp.size - 1
        check(lib().csc_graph_create(n, ci.size, _hptr(rp), _hptr(ci), None, flags, _stream(stream),
                                     ctypes.byref(out)), "csc_graph_create")
    return Graph(out)


def csc_graph_create_batched(graphs, flags: int = 0, stream=None) -> Graph:
    """Pack a list of (row_ptr, col_idx) host CSR graphs block-diagonally into one handle."""
    rps = [np.ascontiguousarray(r, dtype=np.int64) for r, _ in graphs]
    cis = [np.ascontiguousarray(c, dtype=np.int32) for _, c in graphs]
    G = len(rps)
    ns = np.array([r.size - 1 for r in rps], dtype=np.int64)
    rp_ptrs = (ctypes.c_void_p * G)(*[r.ctypes.data for r in rps])
    ci_ptrs = (ctypes.c_void_p * G)(*[c.ctypes.data if c.size else 0 for c in cis])
    out = ctypes.c_void_p()
    check(lib().csc_graph_create_batched(G, _hptr(ns), rp_ptrs, ci_ptrs, flags, _stream(stream), ctypes.byref(out)),
          "csc_graph_create_batched")
    return Graph(out, keep=(rps, cis))


def csc_graph_degrees(g: Graph, stream=None) -> np.ndarray:
    out = np.empty(g.N, dtype=np.int32)
    check(lib().csc_graph_degrees(g.handle, _hptr(out), _stream(stream)), "csc_graph_degrees")
    return out


def csc_graph_tuned_shapes(g: Graph) -> list:
    """Launch shapes chosen by the autotuner on this handle (kind, dtype bytes, columns, shape)."""
    out = []
    i = 0
    kinds = {1: "cheb_step", 2: "mom_step", 3: "cg", 4: "clenshaw"}
    while True:
        kind, db, cols = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        shape = (ctypes.c_int32 * 6)()
        if lib().csc_graph_tuned_shape(g.handle, i, ctypes.byref(kind), ctypes.byref(db), ctypes.byref(cols),
                                       shape) != nat.CSC_OK:
            break
        out.append(dict(kernel=kinds.get(kind.value, str(kind.value)), dtype_bytes=db.value, columns=cols.value,
                        G=shape[0], NT=shape[1], threads=shape[2], P=shape[3], tiles=shape[4],
                        global_index=shape[5] & 1, lean=(shape[5] >> 1) & 1))
        i += 1
    return out


def csc_graph_pin_shape(g: Graph, kernel: str, dtype_bytes: int, columns: int, G: int, NT: int, threads: int,
                        P: int, tiles: int, global_index: int = 0, lean: int = 0) -> None:
    """Fix a launch shape on this handle instead of tuning it (global_index = 1: the row-range
    kernels read column indices from global memory instead of staging them in shared memory;
    lean = 1: the lean form of the Clenshaw and CG kernels, NT = 1 and 256 threads)."""
    kind = {"cheb_step": 1, "mom_step": 2, "cg": 3, "clenshaw": 4}[kernel]
    shape = (ctypes.c_int32 * 6)(G, NT, threads, P, tiles, global_index + 2 * lean)  # checked by the library
    check(lib().csc_graph_pin_shape(g.handle, kind, dtype_bytes, columns, shape), "csc_graph_pin_shape")


def csc_chebyshev_coefficients(lambda_c: float, m: int, flags: int = 0) -> np.ndarray:
    out = np.empty(m + 1, dtype=np.float64)
    check(lib().csc_chebyshev_coefficients(lambda_c, m, flags, _hptr(out)), "csc_chebyshev_coefficients")
    return out


def csc_filter_random_signals(g: Graph, lambda_c: float, m: int, d: int, d_pad: Optional[int] = None,
                              seed: int = 0, storage: int = F32, R_in: Optional[torch.Tensor] = None,
                              Y_out: Optional[torch.Tensor] = None, flags: int = NORMALIZE_ROWS,
                              stream=None) -> torch.Tensor:
    d_pad = ((d + 7) // 8) * 8 if d_pad is None else d_pad
    ydt = torch.float64 if storage == F64 else torch.float32
    if Y_out is None:
        Y_out = torch.empty((g.N, d_pad), dtype=ydt, device="cuda")
    if R_in is not None and (R_in.dtype != torch.float32 or tuple(R_in.shape) != (g.N, d_pad)):
        raise ValueError("R_in must be float32 of shape (N, d_pad)")
    check(lib().csc_filter_random_signals(g.handle, lambda_c, m, d, d_pad, seed, storage, _dptr(R_in), _dptr(Y_out),
                                          flags, _stream(stream)), "csc_filter_random_signals")
    return Y_out


def csc_kpm_moments(g: Graph, n_moments: int, n_probes: int, seed: int = 0, storage: int = F32,
                    stream=None) -> np.ndarray:
    out = np.empty(n_moments, dtype=np.float64)
    check(lib().csc_kpm_moments(g.handle, n_moments, n_probes, seed, storage, _hptr(out), _stream(stream)),
          "csc_kpm_moments")
    return out


def csc_eigencount(mu: np.ndarray, lam: float, flags: int = 0) -> float:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = ctypes.c_double()
    check(lib().csc_eigencount(_hptr(mu), mu.size - 1, lam, flags, ctypes.byref(out)), "csc_eigencount")
    return out.value


@dataclass
class LambdaInfo:
    lam: float
    count: float
    iters: int
    hit: bool
    n_probes: int
    m: int
    bracket_used: bool
    moment_passes: int


def _lambda_info(x: nat.csc_lambda_info) -> LambdaInfo:
    return LambdaInfo(x.lambda_, x.count, x.iters, bool(x.hit), x.n_probes, x.m, bool(x.bracket_used),
                      x.moment_passes)


def csc_estimate_lambda_k(g: Graph, k: int, m: int = 50, n_probes: int = 0, seed: int = 0, bracket=None,
                          stream=None) -> LambdaInfo:
    info = nat.csc_lambda_info()
    br = None
    if bracket is not None:
        br_arr = np.ascontiguousarray(bracket, dtype=np.float64)
        br = _hptr(br_arr)
    check(lib().csc_estimate_lambda_k(g.handle, k, m, n_probes, seed, br, ctypes.byref(info), _stream(stream)),
          "csc_estimate_lambda_k")
    return _lambda_info(info)


# ------------------------------------------------------- learned lambda_k bracket

MLP_PARAMS = nat.CSC_MLP_PARAMS


def _f32_dev(t: torch.Tensor, shape, name: str) -> torch.Tensor:
    if t.dtype != torch.float32 or tuple(t.shape) != tuple(shape) or not t.is_cuda:
        raise ValueError(f"{name} must be a float32 CUDA tensor of shape {tuple(shape)}")
    return t


def csc_bracket_features(g: Graph, k: int, seed: int = 0, stream=None):
    """(features float32[72], raw 8-probe moments float64[64])."""
    feat = np.empty(nat.CSC_MLP_IN, dtype=np.float32)
    mu = np.empty(nat.CSC_BRACKET_MOMENTS, dtype=np.float64)
    check(lib().csc_bracket_features(g.handle, k, seed, _hptr(feat), _hptr(mu), _stream(stream)),
          "csc_bracket_features")
    return feat, mu


def csc_bracket_target(mu: np.ndarray, k: int) -> tuple:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = np.empty(2, dtype=np.float64)
    check(lib().csc_bracket_target(_hptr(mu), mu.size - 1, k, _hptr(out)), "csc_bracket_target")
    return float(out[0]), float(out[1])


def csc_mlp_init(seed: int = 0, params: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if params is None:
        params = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    _f32_dev(params, (MLP_PARAMS,), "params")
    check(lib().csc_mlp_init(_dptr(params), seed, _stream(stream)), "csc_mlp_init")
    return params


def csc_mlp_forward(params: torch.Tensor, X: torch.Tensor, Y: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    B = X.shape[0]
    _f32_dev(params, (MLP_PARAMS,), "params")
    _f32_dev(X, (B, nat.CSC_MLP_IN), "X")
    if Y is None:
        Y = torch.empty((B, nat.CSC_MLP_OUT), dtype=torch.float32, device="cuda")
    check(lib().csc_mlp_forward(_dptr(params), _dptr(X), B, _dptr(Y), _stream(stream)), "csc_mlp_forward")
    return Y


def csc_mlp_loss_grad(params: torch.Tensor, X: torch.Tensor, T: torch.Tensor, stream=None):
    """(loss, gradient float32[MLP_PARAMS])."""
    B = X.shape[0]
    _f32_dev(params, (MLP_PARAMS,), "params")
    _f32_dev(X, (B, nat.CSC_MLP_IN), "X")
    _f32_dev(T, (B, nat.CSC_MLP_OUT), "T")
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctypes.c_double()
    check(lib().csc_mlp_loss_grad(_dptr(params), _dptr(X), _dptr(T), B, _dptr(grad), ctypes.byref(loss),
                                  _stream(stream)), "csc_mlp_loss_grad")
    return loss.value, grad


def csc_mlp_adam_step(params: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, t: int,
                      lr: float, stream=None) -> None:
    for name, a in (("params", params), ("grad", grad), ("m", m), ("v", v)):
        _f32_dev(a, (MLP_PARAMS,), name)
    check(lib().csc_mlp_adam_step(_dptr(params), _dptr(grad), _dptr(m), _dptr(v), t, lr, _stream(stream)),
          "csc_mlp_adam_step")


def csc_mlp_train(params: torch.Tensor, X: torch.Tensor, T: torch.Tensor, epochs: int, batch: int, lr: float,
                  seed: int = 0, stream=None) -> np.ndarray:
    """Minibatch Adam in place on `params`; returns the mean loss of each epoch."""
    n = X.shape[0]
    _f32_dev(params, (MLP_PARAMS,), "params")
    _f32_dev(X, (n, nat.CSC_MLP_IN), "X")
    _f32_dev(T, (n, nat.CSC_MLP_OUT), "T")
    hist = np.zeros(max(epochs, 1), dtype=np.float64)
    check(lib().csc_mlp_train(_dptr(params), _dptr(X), _dptr(T), n, epochs, batch, lr, seed, _hptr(hist),
                              _stream(stream)), "csc_mlp_train")
    return hist[:epochs]


def csc_bracket_fit(feats: np.ndarray, brackets: np.ndarray, val_frac: float = 0.15, epochs: int = 300,
                    batch: int = 32, lr: float = 1e-3, seed: int = 0, widen_rule: int = 0, coverage: float = 0.9,
                    params: Optional[torch.Tensor] = None, stream=None):
    """(params device float[MLP_PARAMS], norm float32[148], widen, n_fit, epoch losses float64[epochs])."""
    feats = np.ascontiguousarray(feats, dtype=np.float32)
    brackets = np.ascontiguousarray(brackets, dtype=np.float64)
    n = feats.shape[0]
    if feats.shape != (n, nat.CSC_MLP_IN) or brackets.shape != (n, 2):
        raise ValueError("feats must be n x 72 and brackets n x 2")
    if params is None:
        params = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    _f32_dev(params, (MLP_PARAMS,), "params")
    norm = np.empty(2 * nat.CSC_MLP_IN + 2 * nat.CSC_MLP_OUT, dtype=np.float32)
    hist = np.zeros(max(epochs, 1), dtype=np.float64)
    widen = ctypes.c_double()
    n_fit = ctypes.c_int32()
    check(lib().csc_bracket_fit(_hptr(feats), _hptr(brackets), n, val_frac, epochs, batch, lr, seed, widen_rule,
                                coverage, _dptr(params), _hptr(norm), ctypes.byref(widen), ctypes.byref(n_fit),
                                _hptr(hist), _stream(stream)), "csc_bracket_fit")
    return params, norm, widen.value, n_fit.value, hist[:epochs]


def csc_bracket_predict(params: torch.Tensor, norm: np.ndarray, widen: float, feats: np.ndarray, stream=None):
    """(targets float64[n x 2] = (centre, ln half-width), brackets float64[n x 2])."""
    _f32_dev(params, (MLP_PARAMS,), "params")
    norm = np.ascontiguousarray(norm, dtype=np.float32)
    feats = np.ascontiguousarray(feats, dtype=np.float32)
    n = feats.shape[0]
    if feats.shape != (n, nat.CSC_MLP_IN) or norm.shape != (2 * nat.CSC_MLP_IN + 2 * nat.CSC_MLP_OUT,):
        raise ValueError("feats must be n x 72 and norm hold 148 floats")
    t = np.empty((n, 2), dtype=np.float64)
    b = np.empty((n, 2), dtype=np.float64)
    check(lib().csc_bracket_predict(_dptr(params), _hptr(norm), widen, _hptr(feats), n, _hptr(t), _hptr(b),
                                    _stream(stream)), "csc_bracket_predict")
    return t, b


def csc_estimate_lambda_k_learned(g: Graph, k: int, params: torch.Tensor, norm: np.ndarray, m: int = 50,
                                  n_probes: int = 0, seed: int = 0, widen: float = 1.0, refilter: bool = False,
                                  stream=None):
    """(LambdaInfo, predicted bracket (lo, hi))."""
    _f32_dev(params, (MLP_PARAMS,), "params")
    norm = np.ascontiguousarray(norm, dtype=np.float32)
    if norm.shape != (2 * nat.CSC_MLP_IN + 2 * nat.CSC_MLP_OUT,):
        raise ValueError("norm must hold feature mean, feature std, target mean, target std (148 floats)")
    info = nat.csc_lambda_info()
    br = np.zeros(2, dtype=np.float64)
    flags = nat.CSC_EIGENCOUNT_REFILTER if refilter else 0
    check(lib().csc_estimate_lambda_k_learned(g.handle, k, m, n_probes, seed, _dptr(params), _hptr(norm), widen,
                                              flags, ctypes.byref(info), _hptr(br), _stream(stream)),
          "csc_estimate_lambda_k_learned")
    return _lambda_info(info), (float(br[0]), float(br[1]))


def csc_estimate_lambda_k_refilter(g: Graph, k: int, m: int = 50, n_probes: int = 0, seed: int = 0, bracket=None,
                                   stream=None) -> LambdaInfo:
    """The paper-literal estimator: one filter pass over the probes per threshold."""
    info = nat.csc_lambda_info()
    br = None
    if bracket is not None:
        br_arr = np.ascontiguousarray(bracket, dtype=np.float64)
        br = _hptr(br_arr)
    check(lib().csc_estimate_lambda_k_refilter(g.handle, k, m, n_probes, seed, br, ctypes.byref(info),
                                               _stream(stream)), "csc_estimate_lambda_k_refilter")
    return _lambda_info(info)


def _check_index_out(out: torch.Tensor, n: int, name: str) -> None:
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.int64 or not out.is_contiguous():
        raise ValueError(f"{name}: out must be a contiguous int64 CUDA tensor")
    if out.numel() < n:
        raise ValueError(f"{name}: out holds {out.numel()} elements, n = {n} are written")


def csc_sample(N: int, n: int, seed: int = 0, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device="cuda")
    _check_index_out(out, n, "csc_sample")
    check(lib().csc_sample(N, n, seed, _dptr(out) if n else None, _stream(stream)), "csc_sample")
    return out


def csc_coherence_scores(Y: torch.Tensor, d: int, normalize: bool = False, out: Optional[torch.Tensor] = None,
                         stream=None) -> torch.Tensor:
    """s_i = ||Y_i||^2 (fp64) over the first d columns; optionally normalise Y's rows in place."""
    if Y.dtype not in (torch.float32, torch.float64):
        raise ValueError("Y must be float32 or float64")
    N, ld = Y.shape
    y_type = F64 if Y.dtype == torch.float64 else F32
    if out is None:
        out = torch.empty(N, dtype=torch.float64, device="cuda")
    check(lib().csc_coherence_scores(_dptr(Y), y_type, N, d, ld, 1 if normalize else 0, _dptr(out),
                                     _stream(stream)), "csc_coherence_scores")
    return out


def csc_sample_weighted(score: torch.Tensor, n: int, seed: int = 0, idx_out: Optional[torch.Tensor] = None,
                        w_out: Optional[torch.Tensor] = None, weights: bool = True, stream=None):
    """(idx int64[n] sorted with repeats, decoder weights float32[n] or None) of n variable-density draws."""
    if score.dtype != torch.float64:
        raise ValueError("score must be float64")
    N = score.numel()
    if idx_out is None:
        idx_out = torch.empty(n, dtype=torch.int64, device="cuda")
    if weights and w_out is None:
        w_out = torch.empty(n, dtype=torch.float32, device="cuda")
    check(lib().csc_sample_weighted(_dptr(score), N, n, seed, _dptr(idx_out) if n else None,
                                    _dptr(w_out) if (weights and n) else None, _stream(stream)),
          "csc_sample_weighted")
    return idx_out, (w_out if weights else None)


def csc_sample_noalloc(N: int, n: int, seed: int, out: torch.Tensor, stream=None) -> torch.Tensor:
    """csc_sample without any device allocation inside the library (the caller gives `out`)."""
    _check_index_out(out, n, "csc_sample_noalloc")
    check(lib().csc_sample_noalloc(N, n, seed, _dptr(out) if n else None, _stream(stream)), "csc_sample_noalloc")
    return out


def csc_gather_rows(X: torch.Tensor, idx: torch.Tensor, d: Optional[int] = None,
                    out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    N, ld = X.shape
    d = ld if d is None else d
    n = idx.numel()
    if out is None:
        out = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    check(lib().csc_gather_rows(_dptr(X), N, ld, _dptr(idx), n, d, _dptr(out), out.shape[1], _stream(stream)),
          "csc_gather_rows")
    return out


def csc_kmeans_reduced(X: torch.Tensor, d: int, k: int, replicates: int = 20, max_iter: int = 100, seed: int = 0,
                       labels_out: Optional[torch.Tensor] = None, stream=None):
    n, ld = X.shape
    if labels_out is None:
        labels_out = torch.empty(n, dtype=torch.int32, device="cuda")
    inertia = ctypes.c_double()
    check(lib().csc_kmeans_reduced(_dptr(X), n, d, ld, k, replicates, max_iter, seed, _dptr(labels_out),
                                   ctypes.byref(inertia), _stream(stream)), "csc_kmeans_reduced")
    return labels_out, inertia.value


@dataclass
class CgInfo:
    iters: int
    converged: bool
    max_rel_residual: float


def csc_interpolate(g: Graph, sample_idx: torch.Tensor, sample_labels: torch.Tensor, k: int, g_power: int = 4,
                    gamma: float = 1e-3, rel_tol: float = 1e-6, max_iter: int = 2000,
                    labels_out: Optional[torch.Tensor] = None, fuzzy: bool = False, stream=None):
    """Returns (labels int32[N], fuzzy float[N, k] or None, CgInfo); raises unless converged or NOT_CONVERGED."""
    if labels_out is None:
        labels_out = torch.empty(g.N, dtype=torch.int32, device="cuda")
    fz = torch.empty((g.N, k), dtype=torch.float32, device="cuda") if fuzzy else None
    info = nat.csc_cg_info()
    st = lib().csc_interpolate(g.handle, _dptr(sample_idx), _dptr(sample_labels), sample_idx.numel(), k, g_power,
                               gamma, rel_tol, max_iter, _dptr(labels_out), _dptr(fz), ctypes.byref(info),
                               _stream(stream))
    check(st, "csc_interpolate", allow=(nat.CSC_E_NOT_CONVERGED,))
    return labels_out, fz, CgInfo(info.iters, bool(info.converged), info.max_rel_residual)


def csc_interpolate_weighted(g: Graph, sample_idx: torch.Tensor, sample_labels: torch.Tensor,
                             sample_w: torch.Tensor, k: int, g_power: int = 4, gamma: float = 1e-3,
                             rel_tol: float = 1e-6, max_iter: int = 2000, labels_out: Optional[torch.Tensor] = None,
                             fuzzy: bool = False, stream=None):
    """Weighted decoder of variable-density draws: (labels, fuzzy or None, CgInfo)."""
    if sample_w.dtype != torch.float32 or sample_w.numel() != sample_idx.numel():
        raise ValueError("sample_w must be float32 with one weight per draw")
    if labels_out is None:
        labels_out = torch.empty(g.N, dtype=torch.int32, device="cuda")
    fz = torch.empty((g.N, k), dtype=torch.float32, device="cuda") if fuzzy else None
    info = nat.csc_cg_info()
    st = lib().csc_interpolate_weighted(g.handle, _dptr(sample_idx), _dptr(sample_labels), _dptr(sample_w),
                                        sample_idx.numel(), k, g_power, gamma, rel_tol, max_iter, _dptr(labels_out),
                                        _dptr(fz), ctypes.byref(info), _stream(stream))
    check(st, "csc_interpolate_weighted", allow=(nat.CSC_E_NOT_CONVERGED,))
    return labels_out, fz, CgInfo(info.iters, bool(info.converged), info.max_rel_residual)


def csc_interpolate_highpass(g: Graph, sample_idx: torch.Tensor, sample_labels: torch.Tensor, k: int,
                             lambda_c: float, m: int = 50, gamma: float = 1e-3, rel_tol: float = 1e-6,
                             max_iter: int = 2000, labels_out: Optional[torch.Tensor] = None, fuzzy: bool = False,
                             stream=None):
    """Eq. 5 with g = 1 - h~_{lambda_c}: (labels, fuzzy or None, CgInfo)."""
    if labels_out is None:
        labels_out = torch.empty(g.N, dtype=torch.int32, device="cuda")
    fz = torch.empty((g.N, k), dtype=torch.float32, device="cuda") if fuzzy else None
    info = nat.csc_cg_info()
    st = lib().csc_interpolate_highpass(g.handle, _dptr(sample_idx), _dptr(sample_labels), sample_idx.numel(), k,
                                        lambda_c, m, gamma, rel_tol, max_iter, _dptr(labels_out), _dptr(fz),
                                        ctypes.byref(info), _stream(stream))
    check(st, "csc_interpolate_highpass", allow=(nat.CSC_E_NOT_CONVERGED,))
    return labels_out, fz, CgInfo(info.iters, bool(info.converged), info.max_rel_residual)


@dataclass
class ClusterInfo:
    lam: LambdaInfo
    cg: CgInfo
    inertia: float
    ms: dict


def csc_cluster(g: Graph, k: int, m: int = 0, d: int = 0, d_pad: int = 0, n: int = 0, n_probes: int = 0,
                g_power: int = 0, gamma: float = 0.0, cg_tol: float = 0.0, cg_max_iter: int = 0,
                replicates: int = 0, km_max_iter: int = 0, storage: int = F32, seed: int = 0,
                lambda_k: float = 0.0, bracket=None, labels_out: Optional[torch.Tensor] = None, flags: int = 0,
                m_count: int = 0, m_interp: int = 0, stream=None):
    """Alg. 2 end to end; zero arguments take the library defaults.  Returns (labels, ClusterInfo)."""
    p = nat.csc_params()
    p.k, p.m, p.d, p.d_pad, p.n, p.n_probes, p.g_power = k, m, d, d_pad, n, n_probes, g_power
    p.gamma, p.cg_tol, p.cg_max_iter, p.replicates, p.km_max_iter = gamma, cg_tol, cg_max_iter, replicates, km_max_iter
    p.storage, p.seed, p.lambda_k, p.flags, p.m_count, p.m_interp = storage, seed, lambda_k, flags, m_count, m_interp
    br_arr = None
    if bracket is not None:
        br_arr = np.ascontiguousarray(bracket, dtype=np.float64)
        p.bracket = br_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if labels_out is None:
        labels_out = torch.empty(g.N, dtype=torch.int32, device="cuda")
    info = nat.csc_cluster_info()
    check(lib().csc_cluster(g.handle, ctypes.byref(p), _dptr(labels_out), ctypes.byref(info), _stream(stream)),
          "csc_cluster")
    ms = dict(lambda_k=info.ms_lambda, filter=info.ms_filter, sample=info.ms_sample, kmeans=info.ms_kmeans,
              interp=info.ms_interp, total=info.ms_total)
    return labels_out, ClusterInfo(_lambda_info(info.lambda_),
                                   CgInfo(info.cg.iters, bool(info.cg.converged), info.cg.max_rel_residual),
                                   info.inertia, ms)


# ----------------------------------------------------------------- batches

def graph_offsets(g: Graph, sizes) -> np.ndarray:
    """Packed row offsets of a batch from its graphs' node counts."""
    return np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))])


def csc_kpm_moments_batched(g: Graph, n_moments: int, n_probes: int, seed: int = 0, storage: int = F32,
                            stream=None) -> np.ndarray:
    out = np.empty((g.n_graphs, n_moments), dtype=np.float64)
    check(lib().csc_kpm_moments_batched(g.handle, n_moments, n_probes, seed, storage, _hptr(out), _stream(stream)),
          "csc_kpm_moments_batched")
    return out


def csc_estimate_lambda_k_batched(g: Graph, k, m: int = 50, n_probes: int = 0, seed: int = 0, stream=None):
    """(lambda float64[G], [LambdaInfo] per graph)."""
    kk = np.ascontiguousarray(k, dtype=np.int32)
    lam = np.empty(g.n_graphs, dtype=np.float64)
    infos = (nat.csc_lambda_info * g.n_graphs)()
    check(lib().csc_estimate_lambda_k_batched(g.handle, _hptr(kk), m, n_probes, seed, _hptr(lam), infos,
                                              _stream(stream)), "csc_estimate_lambda_k_batched")
    return lam, [_lambda_info(x) for x in infos]


def csc_filter_batched(g: Graph, lam, m: int, d: int, d_pad: Optional[int] = None, seed: int = 0,
                       storage: int = F32, R_in: Optional[torch.Tensor] = None, Y_out: Optional[torch.Tensor] = None,
                       flags: int = NORMALIZE_ROWS, stream=None) -> torch.Tensor:
    d_pad = ((d + 7) // 8) * 8 if d_pad is None else d_pad
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    ydt = torch.float64 if storage == F64 else torch.float32
    if Y_out is None:
        Y_out = torch.empty((g.N, d_pad), dtype=ydt, device="cuda")
    if R_in is not None and (R_in.dtype != torch.float32 or tuple(R_in.shape) != (g.N, d_pad)):
        raise ValueError("R_in must be float32 of shape (N, d_pad)")
    check(lib().csc_filter_batched(g.handle, _hptr(lam), m, d, d_pad, seed, storage, _dptr(R_in), _dptr(Y_out),
                                   flags, _stream(stream)), "csc_filter_batched")
    return Y_out


def csc_sample_batched(g: Graph, n, seed: int = 0, stream=None) -> torch.Tensor:
    nn = np.ascontiguousarray(n, dtype=np.int64)
    out = torch.empty(int(nn.sum()), dtype=torch.int64, device="cuda")
    check(lib().csc_sample_batched(g.handle, _hptr(nn), seed, _dptr(out), _stream(stream)), "csc_sample_batched")
    return out


def csc_kmeans_batched(X: torch.Tensor, n, k, d: Optional[int] = None, replicates: int = 20, max_iter: int = 100,
                       seed: int = 0, stream=None):
    """(labels int32[sum n] on the device, inertia float64[problems])."""
    nn = np.ascontiguousarray(n, dtype=np.int64)
    kk = np.ascontiguousarray(k, dtype=np.int32)
    ld = X.shape[1]
    d = ld if d is None else d
    labels = torch.empty(int(nn.sum()), dtype=torch.int32, device="cuda")
    inertia = np.empty(nn.size, dtype=np.float64)
    check(lib().csc_kmeans_batched(_dptr(X), nn.size, _hptr(nn), _hptr(kk), d, ld, replicates, max_iter, seed,
                                   _dptr(labels), _hptr(inertia), _stream(stream)), "csc_kmeans_batched")
    return labels, inertia


def csc_interpolate_batched(g: Graph, sample_idx: torch.Tensor, sample_labels: torch.Tensor, k, g_power: int = 4,
                            gamma: float = 1e-3, rel_tol: float = 1e-6, max_iter: int = 2000, fuzzy: bool = False,
                            stream=None):
    kk = np.ascontiguousarray(k, dtype=np.int32)
    labels = torch.empty(g.N, dtype=torch.int32, device="cuda")
    fz = torch.zeros((g.N, int(kk.max())), dtype=torch.float32, device="cuda") if fuzzy else None
    info = nat.csc_cg_info()
    check(lib().csc_interpolate_batched(g.handle, _dptr(sample_idx), _dptr(sample_labels), sample_idx.numel(),
                                        _hptr(kk), g_power, gamma, rel_tol, max_iter, _dptr(labels), _dptr(fz),
                                        ctypes.byref(info), _stream(stream)),
          "csc_interpolate_batched", allow=(nat.CSC_E_NOT_CONVERGED,))
    return labels, fz, CgInfo(info.iters, bool(info.converged), info.max_rel_residual)


def csc_interpolate_batched_highpass(g: Graph, sample_idx: torch.Tensor, sample_labels: torch.Tensor, k, lam,
                                     m: int = 50, gamma: float = 1e-3, rel_tol: float = 1e-6, max_iter: int = 2000,
                                     fuzzy: bool = False, stream=None):
    """Per-graph Eq. 5 with g = 1 - h~ at each graph's cut-off lam[i]: (labels, fuzzy or None, CgInfo)."""
    kk = np.ascontiguousarray(k, dtype=np.int32)
    ll = np.ascontiguousarray(lam, dtype=np.float64)
    labels = torch.empty(g.N, dtype=torch.int32, device="cuda")
    fz = torch.zeros((g.N, int(kk.max())), dtype=torch.float32, device="cuda") if fuzzy else None
    info = nat.csc_cg_info()
    check(lib().csc_interpolate_batched_highpass(g.handle, _dptr(sample_idx), _dptr(sample_labels),
                                                 sample_idx.numel(), _hptr(kk), _hptr(ll), m, gamma, rel_tol,
                                                 max_iter, _dptr(labels), _dptr(fz), ctypes.byref(info),
                                                 _stream(stream)),
          "csc_interpolate_batched_highpass", allow=(nat.CSC_E_NOT_CONVERGED,))
    return labels, fz, CgInfo(info.iters, bool(info.converged), info.max_rel_residual)


@dataclass
class BatchInfo:
    cg: CgInfo
    lambda_hits: int
    ms: dict


def csc_cluster_batched(g: Graph, k, m: int = 0, d: int = 0, d_pad: int = 0, n_probes: int = 0, g_power: int = 0,
                        gamma: float = 0.0, cg_tol: float = 0.0, cg_max_iter: int = 0, replicates: int = 0,
                        km_max_iter: int = 0, storage: int = F32, seed: int = 0,
                        labels_out: Optional[torch.Tensor] = None, flags: int = 0, m_count: int = 0,
                        m_interp: int = 0, stream=None):
    """Alg. 2 for every graph of a batched handle.  Returns (labels, lambda float64[G], BatchInfo)."""
    kk = np.ascontiguousarray(k, dtype=np.int32)
    p = nat.csc_params()
    p.k, p.m, p.d, p.d_pad, p.n, p.n_probes, p.g_power = 0, m, d, d_pad, 0, n_probes, g_power
    p.gamma, p.cg_tol, p.cg_max_iter, p.replicates, p.km_max_iter = gamma, cg_tol, cg_max_iter, replicates, km_max_iter
    p.storage, p.seed, p.lambda_k, p.flags, p.m_count, p.m_interp = storage, seed, 0.0, flags, m_count, m_interp
    if labels_out is None:
        labels_out = torch.empty(g.N, dtype=torch.int32, device="cuda")
    lam = np.empty(g.n_graphs, dtype=np.float64)
    info = nat.csc_batch_info()
    check(lib().csc_cluster_batched(g.handle, _hptr(kk), ctypes.byref(p), _dptr(labels_out), _hptr(lam),
                                    ctypes.byref(info), _stream(stream)), "csc_cluster_batched")
    ms = dict(lambda_k=info.ms_lambda, filter=info.ms_filter, sample=info.ms_sample, kmeans=info.ms_kmeans,
              interp=info.ms_interp, total=info.ms_total)
    return labels_out, lam, BatchInfo(CgInfo(info.cg.iters, bool(info.cg.converged), info.cg.max_rel_residual),
                                      info.lambda_hits, ms)


def csc_profile_enable(on: bool = True) -> None:
    check(lib().csc_profile_enable(1 if on else 0), "csc_profile_enable")


def csc_profile_reset() -> None:
    check(lib().csc_profile_reset(), "csc_profile_reset")


def csc_profile_launches() -> int:
    n = ctypes.c_int64()
    check(lib().csc_profile_launches(ctypes.byref(n)), "csc_profile_launches")
    return n.value


def csc_profile_query() -> dict:
    """{class name: dict(launches, ms, bytes)} for every kernel class seen since the last reset."""
    out = {}
    i = 0
    while True:
        name = ctypes.create_string_buffer(64)
        launches, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        st = lib().csc_profile_query(i, name, 64, ctypes.byref(launches), ctypes.byref(ms), ctypes.byref(by))
        if st != nat.CSC_OK:
            break
        out[name.value.decode()] = dict(launches=launches.value, ms=ms.value, bytes=by.value)
        i += 1
    return out


def default_sizes(N: int, k: int) -> dict:
    """The library's parameter defaults (d = ceil(4 ln N), n = ceil(2 k ln k), n_v = ceil(2 ln N))."""
    d = max(1, math.ceil(4 * math.log(N))) if N > 1 else 1
    n = min(N, max(k, math.ceil(2 * k * math.log(k)))) if k > 1 else 1
    nv = max(1, math.ceil(2 * math.log(N))) if N > 1 else 1
    return dict(d=d, d_pad=((d + 7) // 8) * 8, n=n, n_probes=nv)
