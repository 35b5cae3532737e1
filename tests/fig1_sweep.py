"""Recovery and lambda_k sweeps of Sec. 5.2 on synthetic SBMs, through the library.

* Fig. 1 a-d: ARI of CSC against the planted partition versus eps on the SBM
  N = 1e3, k = 20, s = 16, varying one of n, d, m (the paper's p) and gamma away
  from the defaults of Alg. 2, beside spectral clustering (Alg. 1, the oracle's
  dense implementation) on the same graphs;
* Fig. 1 e: the lambda_k estimate of Sec. 4.3 against the true lambda_k and
  lambda_{k+1} (dense eigendecomposition) versus eps;
* Fig. 1 f-g (CSC side): ARI and time versus N and k at eps = eps_c / 4, SC at
  N = 1e3 only;
* every CSC default run twice: with g(L) = L^4 and with the paper's g = 1 - h~
  (Fig. 1 f-g also with the eigencount filter at degree 200, four times m);
* the supplementary heterogeneous SBM (community sizes 5, 10, ..., 50, 50, ...,
  95; eps from 0 to 0.2), CSC beside SC.

CSC runs on the GPU (csc_cluster); SC and the eigenvalues run in a pool of
spawned CPU processes started before the first CUDA call.  The figures' plotted
values are not in the paper's text, so the tables are measurements, not parity
checks; tests/test_gpu_sweeps.py asserts the paper's stated findings on a
reduced sweep.

    python -m tests.fig1_sweep --figs a b c d e het fg --realisations 20 --out sweep.md
"""
from __future__ import annotations

import argparse
import math
import os
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np

K, N0, S = 20, 1000, 16.0
HET_SIZES = [5, 10, 15, 20, 25, 30, 35, 40, 45, 50, 50, 55, 60, 65, 70, 75, 80, 85, 90, 95]
EPS_GRID = [0.0, 0.02, 0.04, 0.06, 0.08, 0.10, 0.13]
HET_EPS = [0.0, 0.025, 0.05, 0.075, 0.10, 0.125, 0.15, 0.175, 0.20]


def defaults(n_nodes: int = N0, k: int = K) -> dict:
    """Alg. 2 defaults as read here: n = ceil(2 k ln k), d = ceil(4 ln N), m = 50, gamma = 1e-3."""
    return dict(n=math.ceil(2 * k * math.log(k)), d=math.ceil(4 * math.log(n_nodes)), m=50, gamma=1e-3)


def variants(n_nodes: int = N0, k: int = K) -> dict:
    """One parameter changed at a time (Fig. 1 a-d); the values are this sweep's choice."""
    lk = k * math.log(k)
    ln = math.log(n_nodes)
    return {
        "a": ("n", [k, math.ceil(lk), math.ceil(2 * lk), math.ceil(4 * lk)]),
        "b": ("d", [math.ceil(ln), math.ceil(2 * ln), math.ceil(4 * ln), math.ceil(8 * ln)]),
        "c": ("m", [10, 20, 50, 100]),
        "d": ("gamma", [1e-5, 1e-3, 1e-1, 1.0]),
    }


def make_graph(n_nodes: int, k: int, eps: float, seed: int, het: bool = False):
    import csc_inputs as ci

    return ci.sbm(n_nodes, k, s=S, eps=eps, seed=seed, sizes=HET_SIZES if het else None)


def sc_job(args):
    """Spawned worker: SC (Alg. 1) ARI, the eigenvalues lambda_k, lambda_{k+1} and SC seconds."""
    n_nodes, k, eps, seed, het = args
    from oracle import ari, sc

    g = make_graph(n_nodes, k, eps, seed, het)
    t0 = time.perf_counter()
    lab, ev = sc.spectral_clustering(g.row_ptr, g.col_idx, k, seed=seed)
    return dict(ari=ari.ari(lab, g.labels), lk=float(ev[k - 1]), lk1=float(ev[k]), sec=time.perf_counter() - t0)


def graph_job(args):
    n_nodes, k, eps, seed = args
    g = make_graph(n_nodes, k, eps, seed)
    return g.row_ptr, g.col_idx, g.labels


def _csc_runs(csc, h, g, seed: int, figs, n_nodes: int = N0, k: int = K):
    """ARI per (figure, value) and the default run's lambda_k estimate."""
    from oracle import ari

    base = defaults(n_nodes, k)
    out, lam = {}, None
    jobs = [("def", None, base), ("hp", None, base)]
    for f, (key, vals) in variants(n_nodes, k).items():
        if f in figs:
            for v in vals:
                p = dict(base)
                p[key] = v
                jobs.append((f, v, p))
    for f, v, p in jobs:
        d_pad = ((p["d"] + 7) // 8) * 8
        labels, info = csc.csc_cluster(h, k, m=p["m"], d=p["d"], d_pad=d_pad, n=p["n"], gamma=p["gamma"], seed=seed,
                                       flags=csc.HIGHPASS if f == "hp" else 0)
        out[(f, v)] = ari.ari(labels.cpu().numpy(), g.labels)
        if f == "def":
            lam = info.lam.lam
    return out, lam


def _mean(xs):
    return float(np.mean(xs)) if len(xs) else float("nan")


def run(figs, realisations: int, eps_grid=EPS_GRID, het_eps=HET_EPS, workers: int = 0,
        fg_sizes=((1_000, 20), (10_000, 20), (100_000, 20), (1_000_000, 20), (10_000, 200), (100_000, 200),
                  (1_000_000, 200)), fg_realisations: int = 3) -> dict:
    """Run the requested sweeps; returns nested dictionaries of means (see format_tables)."""
    import csc_inputs as ci

    workers = workers or max(1, min(14, (os.cpu_count() or 2) - 2))
    # one BLAS thread per worker process (the workers inherit the environment at spawn)
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({v: "1" for v in saved})
    pool = ProcessPoolExecutor(workers, mp_context=get_context("spawn"))  # before any CUDA call
    seeds = range(realisations)
    hom = any(f in figs for f in "abcde")
    sc_hom = {(e, s): pool.submit(sc_job, (N0, K, e, s, False)) for e in eps_grid for s in seeds} if hom else {}
    sc_het = {(e, s): pool.submit(sc_job, (N0, K, e, s, True)) for e in het_eps for s in seeds} \
        if "het" in figs else {}
    fg_graphs = {}
    if "fg" in figs:
        for n_nodes, k in fg_sizes:
            eps = 0.25 * ci.epsilon_c(S, k)
            for s in range(fg_realisations):
                fg_graphs[(n_nodes, k, s)] = pool.submit(graph_job, (n_nodes, k, eps, s))
        sc_fg = {s: pool.submit(sc_job, (N0, K, 0.25 * ci.epsilon_c(S, K), s, False)) for s in range(fg_realisations)}

    import torch

    import paper_1602_02018_gb300 as csc
    from oracle import ari

    res = {}
    if hom or "het" in figs:
        for tag, grid, het, scf in (("hom", eps_grid, False, sc_hom), ("het", het_eps, True, sc_het)):
            if (tag == "hom" and not hom) or (tag == "het" and "het" not in figs):
                continue
            rows = {}
            for e in grid:
                acc, lams = {}, []
                for s in seeds:
                    g = make_graph(N0, K, e, s, het)
                    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
                        a, lam = _csc_runs(csc, h, g, s, figs if tag == "hom" else (), N0, K)
                    for key, v in a.items():
                        acc.setdefault(key, []).append(v)
                    lams.append(lam)
                scr = [scf[(e, s)].result() for s in seeds]
                rows[e] = dict(csc={key: _mean(v) for key, v in acc.items()}, sc=_mean([r["ari"] for r in scr]),
                               lam_est=_mean(lams), lk=_mean([r["lk"] for r in scr]),
                               lk1=_mean([r["lk1"] for r in scr]),
                               est_in_gap=_mean([float(r["lk"] - 1e-12 <= l <= r["lk1"]) for r, l in zip(scr, lams)]))
            res[tag] = rows
    if "fg" in figs:
        rows = {}
        for n_nodes, k in fg_sizes:
            row = {}
            for tag, fl, mc in (("l4", 0, 0), ("hp", csc.HIGHPASS, 0), ("hp200", csc.HIGHPASS, 200)):
                a, ms, wall = [], [], []
                for s in range(fg_realisations):
                    rp, ci_, lab = fg_graphs[(n_nodes, k, s)].result()
                    with csc.csc_graph_create(rp, ci_) as h:
                        csc.csc_cluster(h, k, seed=s, flags=fl, m_count=mc)  # warm-up: tuning, graph capture
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        labels, info = csc.csc_cluster(h, k, seed=s, flags=fl, m_count=mc)
                        wall.append(time.perf_counter() - t0)
                    a.append(ari.ari(labels.cpu().numpy(), lab))
                    ms.append(info.ms["total"])
                row[tag] = dict(ari=_mean(a), ms=_mean(ms), wall_s=_mean(wall))
            rows[(n_nodes, k)] = row
        scr = [sc_fg[s].result() for s in range(fg_realisations)]
        res["fg"] = rows
        res["fg_sc"] = dict(ari=_mean([r["ari"] for r in scr]), sec=_mean([r["sec"] for r in scr]))
    pool.shutdown()
    for v, x in saved.items():
        if x is None:
            os.environ.pop(v, None)
        else:
            os.environ[v] = x
    return res


def format_tables(res: dict, realisations: int) -> str:
    out = []
    var = variants()
    if "hom" in res:
        rows = res["hom"]
        first = next(iter(rows.values()))["csc"]
        for f, (key, vals) in var.items():
            if (f, vals[0]) not in first:
                continue
            out.append(f"Fig. 1 {f}: ARI vs eps, SBM N = 1e3, k = 20, s = 16, {realisations} realisations, "
                       f"varying {key} (others at the defaults)\n")
            out.append("| eps | " + " | ".join(f"CSC {key} = {v:g}" for v in vals) + " | SC |")
            out.append("|---:|" + "---:|" * (len(vals) + 1))
            for e, r in rows.items():
                out.append(f"| {e:g} | " + " | ".join(f"{r['csc'][(f, v)]:.3f}" for v in vals) + f" | {r['sc']:.3f} |")
            out.append("")
        out.append(f"Fig. 1 e: lambda_k estimate (Sec. 4.3) vs the true lambda_k, lambda_(k+1), "
                   f"{realisations} realisations\n")
        out.append("| eps | estimate | lambda_k | lambda_(k+1) | share in [lambda_k, lambda_(k+1)] | CSC ARI, L^4 | "
                   "CSC ARI, 1 - h~ | SC ARI |")
        out.append("|---:|---:|---:|---:|---:|---:|---:|---:|")
        for e, r in rows.items():
            out.append(f"| {e:g} | {r['lam_est']:.4f} | {r['lk']:.4f} | {r['lk1']:.4f} | {r['est_in_gap']:.2f} | "
                       f"{r['csc'][('def', None)]:.3f} | {r['csc'][('hp', None)]:.3f} | {r['sc']:.3f} |")
        out.append("")
    if "het" in res:
        out.append(f"Heterogeneous SBM (sizes 5 ... 95, N = 1e3, k = 20): ARI vs eps, {realisations} realisations\n")
        out.append("| eps | CSC, L^4 | CSC, 1 - h~ | SC | lambda_k estimate | lambda_k | lambda_(k+1) |")
        out.append("|---:|---:|---:|---:|---:|---:|---:|")
        for e, r in res["het"].items():
            out.append(f"| {e:g} | {r['csc'][('def', None)]:.3f} | {r['csc'][('hp', None)]:.3f} | {r['sc']:.3f} | "
                       f"{r['lam_est']:.4f} | {r['lk']:.4f} | {r['lk1']:.4f} |")
        out.append("")
    if "fg" in res:
        out.append("Fig. 1 f-g (CSC on one GB300): ARI and time vs N and k at eps = eps_c/4\n")
        out.append("| N | k | ARI, L^4 | device ms, L^4 | ARI, 1 - h~ | device ms, 1 - h~ | "
                   "ARI, 1 - h~, eigencount degree 200 | device ms |")
        out.append("|---:|---:|---:|---:|---:|---:|---:|---:|")
        for (n_nodes, k), r in res["fg"].items():
            out.append(f"| {n_nodes:,} | {k} | {r['l4']['ari']:.3f} | {r['l4']['ms']:.1f} | {r['hp']['ari']:.3f} | "
                       f"{r['hp']['ms']:.1f} | {r['hp200']['ari']:.3f} | {r['hp200']['ms']:.1f} |")
        sc = res["fg_sc"]
        out.append(f"\nSC (Alg. 1, dense FP64 on the host, one process) at N = 1e3, k = 20: ARI {sc['ari']:.3f}, "
                   f"{sc['sec']:.2f} s per graph")
        out.append("")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--figs", nargs="+", default=["a", "b", "c", "d", "e", "het", "fg"])
    ap.add_argument("--realisations", type=int, default=20)
    ap.add_argument("--fg-realisations", type=int, default=3)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    t0 = time.perf_counter()
    res = run(set(args.figs), args.realisations, workers=args.workers, fg_realisations=args.fg_realisations)
    text = format_tables(res, args.realisations) + f"\n(sweep wall time {time.perf_counter() - t0:.0f} s)\n"
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
