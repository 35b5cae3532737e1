"""Write the FP64 oracle's end-to-end result on the SBM with N = 1e5 nodes and k = 200
equal communities (mean degree 16, eps = eps_c / 4, seed 0; d = ceil(4 ln N) = 47,
m = 50, n = ceil(2 k ln k) = 2120, g(L) = L^4 with gamma = 1e-3) to
``csc_sbm_n1e5_k200_seed0.npz`` beside this script.

Alg. 2 is run by ``oracle.pipeline.csc`` only: the eigencount dichotomy of
Sec. 4.3, the Jackson-Chebyshev filter and row normalisation of step 4, uniform
sampling (Eq. 4), k-means with 20 replicates, the interpolation of Eq. 5 solved
to a relative residual of 1e-10, and the argmax rule of Sec. 4.1.  Nothing here
calls the CUDA path.  Stored: the labels, lambda_k, the ARI against the planted
communities, the k-means inertia and the CG iteration count, plus the CSR's
size and a hash of its arrays so a test can tell the graph generator has not
changed since.

Run:  python -m tests.golden.make_csc_sbm_n1e5_k200   (about ten minutes on one core)
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csc_sbm_n1e5_k200_seed0.npz")
N, K, SEED = 100_000, 200, 0


def csr_hash(row_ptr: np.ndarray, col_idx: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(row_ptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(col_idx, dtype=np.int32).tobytes())
    return h.hexdigest()


def main() -> None:
    import csc_inputs as ci
    from oracle import ari, pipeline

    g = ci.sbm(N, K, seed=SEED)
    t0 = time.perf_counter()
    tt: dict = {}
    res = pipeline.csc(g.row_ptr, g.col_idx, K, seed=SEED, timings=tt)
    a = ari.ari(res["labels"], g.labels)
    np.savez_compressed(
        OUT,
        labels=res["labels"].astype(np.uint8),
        lam=np.float64(res["lam"]),
        ari_vs_planted=np.float64(a),
        inertia=np.float64(res["inertia"]),
        cg_iters=np.int64(res["cg_iters"]),
        cg_res=np.float64(res["cg_res"]),
        n_nodes=np.int64(g.n),
        nnz=np.int64(g.nnz),
        csr_sha256=np.array(csr_hash(g.row_ptr, g.col_idx)),
    )
    print(f"lambda_k {res['lam']:.6f}  ARI {a:.4f}  inertia {res['inertia']:.6f}  CG {res['cg_iters']} iterations "
          f"(residual {res['cg_res']:.2e})  {time.perf_counter() - t0:.0f} s  stages {tt}")


if __name__ == "__main__":
    main()
