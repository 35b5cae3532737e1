// batched.cu -- Alg. 2 on many graphs at once: the graphs of a batched handle are
// packed block-diagonally (graph i owns rows offsets[i] .. offsets[i+1]-1), so one
// sparse product serves all of them.  Every stage keeps the graphs apart:
//   * row ranges never straddle two graphs (get_partition), so per-graph sums are
//     sums over a graph's own ranges (moments, CG inner products);
//   * the filter reads c_j of the row's graph from a coefficient table;
//   * sampling, k-means and the CG systems run per graph inside single launches
//     (one CTA per graph, one problem per grid row, one set of columns per graph).
// Per-graph seeds: graph i samples and seeds k-means with seed + i; the signal and
// probe blocks are drawn once for the packed rows.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "device.cuh"

namespace csc {
namespace {

constexpr int kBsThreads = 1024;

// Uniform sampling of Eq. 4 per graph: graph g keeps the n_g nodes with the smallest
// keys SplitMix64_{seed+g}(i), i local, written in increasing i as packed indices at
// out[out_off[g] ..].  One CTA per graph: the n_g-th smallest key T is found by an
// eight-pass radix select (8 bits per pass, keys recomputed each pass; keys are
// distinct, so the sample is exactly {i : key_i <= T}), then an ordered compaction.
__global__ void __launch_bounds__(kBsThreads) batched_sample_kernel(const int64_t* __restrict__ offsets,
                                                                    const int64_t* __restrict__ n_per,
                                                                    const int64_t* __restrict__ out_off,
                                                                    uint64_t seed, int64_t* __restrict__ out) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ long long s_need;
    __shared__ int warp_cnt[kBsThreads / 32];
    const int gi = blockIdx.x;
    const int64_t base = offsets[gi], Ng = offsets[gi + 1] - base;
    const int64_t ng = n_per[gi];
    if (ng <= 0) return;
    const uint64_t sg = seed + (uint64_t)gi;
    const int T = threadIdx.x;
    if (T == 0) {
        s_prefix = 0ull;
        s_need = ng;
    }
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = T; b < 256; b += kBsThreads) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        for (int64_t i = T; i < Ng; i += kBsThreads) {
            const uint64_t key = splitmix64_at(sg, (uint64_t)i);
            if (pass == 0 || (key >> (shift + 8)) == (prefix >> (shift + 8)))
                atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (T == 0) {
            long long need = s_need, cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + (long long)hist[b] >= need) break;
                cum += hist[b];
            }
            s_need = need - cum;
            s_prefix = prefix | ((unsigned long long)b << shift);
        }
        __syncthreads();
    }
    const uint64_t thr = s_prefix;
    const int lane = T & 31, w = T >> 5;
    int64_t written = 0;
    int64_t* dst = out + out_off[gi];
    for (int64_t c0 = 0; c0 < Ng; c0 += kBsThreads) {
        const int64_t i = c0 + T;
        const bool f = i < Ng && splitmix64_at(sg, (uint64_t)i) <= thr;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_cnt[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int q = 0; q < kBsThreads / 32; ++q) {
            if (q < w) before += warp_cnt[q];
            total += warp_cnt[q];
        }
        if (f) {
            const int64_t pos = written + before + __popc(m & ((1u << lane) - 1u));
            if (pos < ng) dst[pos] = base + i;
        }
        written += total;
        __syncthreads();  // warp counts are rewritten next chunk
    }
}

int64_t default_samples(int k, int64_t Ng) {
    int64_t n = k > 1 ? (int64_t)ceil(2.0 * k * log((double)k)) : 1;
    if (n < k) n = k;
    if (n > Ng) n = Ng;
    return n;
}

csc_status check_batch(csc_graph g, const char* who) {
    if (!g) {
        set_error("%s: NULL graph", who);
        return CSC_E_INVALID;
    }
    if (g->poisoned) {
        set_error("%s: the handle saw a CUDA error earlier and must be destroyed", who);
        return CSC_E_CUDA;
    }
    return CSC_OK;
}

int batch_probes(const Graph* g) {
    int64_t nmax = 1;
    const int G = std::max(1, (int)g->n_graphs);
    for (int i = 0; i < G; ++i) nmax = std::max(nmax, g->offsets[i + 1] - g->offsets[i]);
    return nmax > 1 ? (int)ceil(2.0 * log((double)nmax)) : 1;
}

// run_sample per graph of the batch (one launch); idx_out: device int64[sum n].
csc_status run_sample_batched(Graph* g, const int64_t* n_per, uint64_t seed, int64_t* idx_out, cudaStream_t s) {
    const int G = std::max(1, (int)g->n_graphs);
    std::vector<int64_t> hn(G), hoff(G + 1, 0);
    for (int i = 0; i < G; ++i) {
        const int64_t Ng = g->offsets[i + 1] - g->offsets[i];
        if (n_per[i] < 0 || n_per[i] > Ng) {
            set_error("batched sampling: graph %d asks for %lld of %lld nodes", i, (long long)n_per[i],
                      (long long)Ng);
            return CSC_E_INVALID;
        }
        hn[i] = n_per[i];
        hoff[i + 1] = hoff[i] + hn[i];
    }
    void* ws = nullptr;
    CSC_TRY(ws_get(g, WS_SAMPLE, (size_t)(3 * G + 2) * sizeof(int64_t), &ws));
    int64_t* d_off = (int64_t*)ws;
    int64_t* d_n = d_off + (G + 1);
    int64_t* d_out = d_n + G;
    CSC_CUDA_TRY(cudaMemcpyAsync(d_off, g->offsets.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(d_n, hn.data(), G * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(d_out, hoff.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CSC_KLAUNCH("sample_batched", 8.0 * hoff[G], s,
                batched_sample_kernel<<<G, kBsThreads, 0, s>>>(d_off, d_n, d_out, seed, idx_out));
    // the host staging vectors die with this frame
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    return CSC_OK;
}

// lambda_k of every graph: per-graph moments once, then the Sec. 4.3 dichotomy per graph.
csc_status lambda_batched(Graph* g, const int32_t* k, int m, int n_probes, uint64_t seed, double* lam,
                          csc_lambda_info* infos, cudaStream_t s) {
    const int G = std::max(1, (int)g->n_graphs);
    if (n_probes == 0) n_probes = batch_probes(g);
    std::vector<double> mu((size_t)G * (m + 1));
    int passes = 0;
    CSC_TRY(run_moments(g, m + 1, n_probes, seed, CSC_F32, mu.data(), &passes, s, true));
    for (int i = 0; i < G; ++i) {
        csc_lambda_info info;
        memset(&info, 0, sizeof(info));
        info.n_probes = n_probes;
        info.m = m;
        info.moment_passes = passes;
        estimate_from_moments(mu.data() + (size_t)i * (m + 1), m, k[i], &info);
        lam[i] = info.lambda;
        if (infos) infos[i] = info;
    }
    return CSC_OK;
}

}  // namespace
}  // namespace csc

using namespace csc;

extern "C" {

csc_status csc_kpm_moments_batched(csc_graph g, int32_t n_moments, int32_t n_probes, uint64_t seed,
                                   csc_dtype storage, double* mu_out, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_kpm_moments_batched"));
    if (n_moments < 1 || n_probes < 1 || !mu_out) {
        set_error("csc_kpm_moments_batched: need n_moments >= 1, n_probes >= 1 and mu_out");
        return CSC_E_INVALID;
    }
    csc_status st = run_moments(g, n_moments, n_probes, seed, storage, mu_out, nullptr, (cudaStream_t)stream, true);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_estimate_lambda_k_batched(csc_graph g, const int32_t* k, int32_t m, int32_t n_probes, uint64_t seed,
                                         double* lambda_out, csc_lambda_info* info_out, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_estimate_lambda_k_batched"));
    const int G = std::max(1, (int)g->n_graphs);
    if (!k || !lambda_out || m < 1 || n_probes < 0) {
        set_error("csc_estimate_lambda_k_batched: invalid arguments");
        return CSC_E_INVALID;
    }
    for (int i = 0; i < G; ++i)
        if (k[i] < 1 || k[i] > g->offsets[i + 1] - g->offsets[i]) {
            set_error("csc_estimate_lambda_k_batched: graph %d has k = %d outside [1, N]", i, k[i]);
            return CSC_E_INVALID;
        }
    csc_status st = lambda_batched(g, k, m, n_probes, seed, lambda_out, info_out, (cudaStream_t)stream);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_filter_batched(csc_graph g, const double* lambda, int32_t m, int32_t d, int32_t d_pad, uint64_t seed,
                              csc_dtype storage, const float* R_in, void* Y_out, uint32_t flags, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_filter_batched"));
    const int G = std::max(1, (int)g->n_graphs);
    if (!lambda || !Y_out || m < 1 || d < 1 || d_pad < d || d_pad % 8) {
        set_error("csc_filter_batched: invalid arguments (m=%d d=%d d_pad=%d)", m, d, d_pad);
        return CSC_E_INVALID;
    }
    std::vector<double> c((size_t)G * (m + 1));
    for (int i = 0; i < G; ++i) {
        if (!(lambda[i] >= 0.0 && lambda[i] <= 2.0)) {
            set_error("csc_filter_batched: lambda of graph %d outside [0, 2]", i);
            return CSC_E_INVALID;
        }
        cheb_coefficients(lambda[i], m, (flags & CSC_NO_JACKSON) == 0, c.data() + (size_t)i * (m + 1));
    }
    if (G == 1) {
        csc_status st = run_filter(g, c.data(), m, d, d_pad, seed, storage, R_in, Y_out,
                                   (flags & CSC_NORMALIZE_ROWS) != 0, (cudaStream_t)stream,
                                   (flags & CSC_CLENSHAW) != 0);
        if (st == CSC_E_CUDA) g->poisoned = true;
        return st;
    }
    csc_status st = run_filter_batched(g, c.data(), m, d, d_pad, seed, storage, R_in, Y_out,
                                       (flags & CSC_NORMALIZE_ROWS) != 0, (cudaStream_t)stream,
                                       (flags & CSC_CLENSHAW) != 0);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_sample_batched(csc_graph g, const int64_t* n, uint64_t seed, int64_t* idx_out, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_sample_batched"));
    if (!n || !idx_out) {
        set_error("csc_sample_batched: need n and idx_out");
        return CSC_E_INVALID;
    }
    csc_status st = run_sample_batched(g, n, seed, idx_out, (cudaStream_t)stream);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_kmeans_batched(const float* X, int32_t n_problems, const int64_t* n, const int32_t* k, int32_t d,
                              int32_t ld, int32_t replicates, int32_t max_iter, uint64_t seed, int32_t* labels_out,
                              double* inertia_out, void* stream) {
    clear_error();
    if (!X || n_problems < 1 || !n || !k || d < 1 || ld < d || replicates < 1 || max_iter < 0 || !labels_out) {
        set_error("csc_kmeans_batched: invalid arguments");
        return CSC_E_INVALID;
    }
    std::vector<KmTask> tasks;
    int64_t off = 0;
    for (int i = 0; i < n_problems; ++i) {
        if (k[i] < 1 || n[i] < k[i] || n[i] >= (int64_t)INT32_MAX) {
            set_error("csc_kmeans_batched: problem %d needs 1 <= k <= n", i);
            return CSC_E_INVALID;
        }
        KmTask t;
        t.X = X + off * ld;
        t.n = (int)n[i];
        t.k = k[i];
        t.seed = seed + (uint64_t)i;
        t.labels_out = labels_out + off;
        tasks.push_back(t);
        off += n[i];
    }
    return run_kmeans_multi(tasks, d, ld, replicates, max_iter, inertia_out, nullptr, (cudaStream_t)stream);
}

csc_status csc_interpolate_batched(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                   int64_t n_total, const int32_t* k, int32_t g_power, double gamma, double rel_tol,
                                   int32_t max_iter, int32_t* labels_out, float* fuzzy_out, csc_cg_info* info,
                                   void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_interpolate_batched"));
    const int G = std::max(1, (int)g->n_graphs);
    if (!sample_idx || !sample_labels || n_total < 1 || !k || g_power < 1 || !(gamma > 0.0) || !(rel_tol > 0.0) ||
        max_iter < 1 || !labels_out) {
        set_error("csc_interpolate_batched: invalid arguments");
        return CSC_E_INVALID;
    }
    int kmax = 1;
    for (int i = 0; i < G; ++i) {
        if (k[i] < 1) {
            set_error("csc_interpolate_batched: graph %d has k < 1", i);
            return CSC_E_INVALID;
        }
        kmax = std::max(kmax, k[i]);
    }
    csc_status st = run_interpolate(g, sample_idx, sample_labels, n_total, kmax, g_power, gamma, rel_tol, max_iter,
                                    labels_out, fuzzy_out, info, (cudaStream_t)stream, G > 1 ? k : nullptr);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_interpolate_batched_highpass(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                            int64_t n_total, const int32_t* k, const double* lambda, int32_t m,
                                            double gamma, double rel_tol, int32_t max_iter, int32_t* labels_out,
                                            float* fuzzy_out, csc_cg_info* info, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_interpolate_batched_highpass"));
    const int G = std::max(1, (int)g->n_graphs);
    if (!sample_idx || !sample_labels || n_total < 1 || !k || !lambda || m < 1 || !(gamma > 0.0) ||
        !(rel_tol > 0.0) || max_iter < 1 || !labels_out) {
        set_error("csc_interpolate_batched_highpass: invalid arguments");
        return CSC_E_INVALID;
    }
    int kmax = 1;
    std::vector<double> c((size_t)G * (m + 1));
    for (int i = 0; i < G; ++i) {
        if (k[i] < 1 || !(lambda[i] >= 0.0 && lambda[i] <= 2.0)) {
            set_error("csc_interpolate_batched_highpass: graph %d has k < 1 or a cut-off outside [0, 2]", i);
            return CSC_E_INVALID;
        }
        kmax = std::max(kmax, k[i]);
        cheb_coefficients(lambda[i], m, true, c.data() + (size_t)i * (m + 1));
    }
    csc_status st = run_interpolate(g, sample_idx, sample_labels, n_total, kmax, 1, gamma, rel_tol, max_iter,
                                    labels_out, fuzzy_out, info, (cudaStream_t)stream, G > 1 ? k : nullptr, c.data(),
                                    m);
    if (st == CSC_E_CUDA) g->poisoned = true;
    return st;
}

csc_status csc_cluster_batched(csc_graph g, const int32_t* k, const csc_params* p, int32_t* labels_out,
                               double* lambda_out, csc_batch_info* info, void* stream) {
    clear_error();
    CSC_TRY(check_batch(g, "csc_cluster_batched"));
    const int G = std::max(1, (int)g->n_graphs);
    if (!k || !p || !labels_out) {
        set_error("csc_cluster_batched: invalid arguments");
        return CSC_E_INVALID;
    }
    if (p->flags & CSC_VARDENSITY) {
        set_error("csc_cluster_batched: CSC_VARDENSITY is a single-graph option (csc_cluster)");
        return CSC_E_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nmax = 1;
    std::vector<int64_t> n_per(G), soff(G + 1, 0);
    int kmax = 1;
    for (int i = 0; i < G; ++i) {
        const int64_t Ng = g->offsets[i + 1] - g->offsets[i];
        if (k[i] < 1 || k[i] > Ng) {
            set_error("csc_cluster_batched: graph %d has k = %d outside [1, N]", i, k[i]);
            return CSC_E_INVALID;
        }
        nmax = std::max(nmax, Ng);
        kmax = std::max(kmax, k[i]);
        n_per[i] = default_samples(k[i], Ng);
        soff[i + 1] = soff[i] + n_per[i];
    }
    const int64_t N = g->N, n_total = soff[G];
    const int m = p->m > 0 ? p->m : 50;
    const int d = p->d > 0 ? p->d : (nmax > 1 ? (int)ceil(4.0 * log((double)nmax)) : 1);
    const int d_pad = p->d_pad > 0 ? p->d_pad : ((d + 7) / 8) * 8;
    const int g_power = p->g_power > 0 ? p->g_power : 4;
    const double gamma = p->gamma > 0 ? p->gamma : 1e-3;
    const double cg_tol = p->cg_tol > 0 ? p->cg_tol : 1e-6;
    const int cg_max = p->cg_max_iter > 0 ? p->cg_max_iter : 2000;
    const int reps = p->replicates > 0 ? p->replicates : 20;
    const int km_iter = p->km_max_iter > 0 ? p->km_max_iter : 100;
    const csc_dtype storage = p->storage;
    if (d_pad < d || d_pad % 8 || (storage != CSC_F32 && storage != CSC_BF16 && storage != CSC_F64)) {
        set_error("csc_cluster_batched: invalid d_pad or storage");
        return CSC_E_INVALID;
    }
    csc_batch_info local;
    memset(&local, 0, sizeof(local));
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; ++i) CSC_CUDA_TRY(cudaEventCreate(&ev[i]));
    auto done = [&](csc_status r) {
        for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
        if (r == CSC_E_CUDA) g->poisoned = true;
        return r;
    };
    cudaEventRecord(ev[0], s);
    std::vector<double> lam(G);
    std::vector<csc_lambda_info> linfo(G);
    csc_status st = lambda_batched(g, k, p->m_count > 0 ? p->m_count : m, p->n_probes, p->seed, lam.data(),
                                   linfo.data(), s);
    if (st != CSC_OK) return done(st);
    for (int i = 0; i < G; ++i) local.lambda_hits += linfo[i].hit;
    cudaEventRecord(ev[1], s);
    // pipeline buffers: Y (N x d_pad), idx (n_total), Xr (n_total x d_pad fp32), sample labels
    const size_t ybytes = (size_t)N * d_pad * (storage == CSC_F64 ? 8 : 4);
    const size_t off_idx = (ybytes + 255) / 256 * 256;
    const size_t off_xr = off_idx + ((size_t)n_total * 8 + 255) / 256 * 256;
    const size_t off_lab = off_xr + ((size_t)n_total * d_pad * 4 + 255) / 256 * 256;
    const size_t total = off_lab + (size_t)n_total * 4 + 256;
    void* base = nullptr;
    st = ws_get(g, WS_PIPE, total, &base);
    if (st != CSC_OK) return done(st);
    char* b = (char*)base;
    void* Y = b;
    int64_t* idx = (int64_t*)(b + off_idx);
    float* Xr = (float*)(b + off_xr);
    int32_t* slab = (int32_t*)(b + off_lab);
    std::vector<double> c((size_t)G * (m + 1));
    for (int i = 0; i < G; ++i) cheb_coefficients(lam[i], m, true, c.data() + (size_t)i * (m + 1));
    const bool clen = (p->flags & CSC_CLENSHAW) != 0;
    st = G > 1 ? run_filter_batched(g, c.data(), m, d, d_pad, p->seed, storage, nullptr, Y, true, s, clen)
               : run_filter(g, c.data(), m, d, d_pad, p->seed, storage, nullptr, Y, true, s, clen);
    if (st != CSC_OK) return done(st);
    cudaEventRecord(ev[2], s);
    st = run_sample_batched(g, n_per.data(), p->seed, idx, s);
    if (st != CSC_OK) return done(st);
    st = storage == CSC_F64 ? run_gather_rows_f64((const double*)Y, N, d_pad, idx, n_total, d, Xr, d_pad, s)
                            : run_gather_rows((const float*)Y, N, d_pad, idx, n_total, d, Xr, d_pad, s);
    if (st != CSC_OK) return done(st);
    cudaEventRecord(ev[3], s);
    {
        std::vector<KmTask> tasks(G);
        for (int i = 0; i < G; ++i) {
            tasks[i].X = Xr + (size_t)soff[i] * d_pad;
            tasks[i].n = (int)n_per[i];
            tasks[i].k = k[i];
            tasks[i].seed = p->seed + (uint64_t)i;
            tasks[i].labels_out = slab + soff[i];
        }
        st = run_kmeans_multi(tasks, d, d_pad, reps, km_iter, nullptr, g, s);
        if (st != CSC_OK) return done(st);
    }
    cudaEventRecord(ev[4], s);
    // CSC_HIGHPASS: g = 1 - h~ with each graph's own cut-off, at degree m_interp (default m:
    // the filter's coefficients c)
    const bool hp = (p->flags & CSC_HIGHPASS) != 0;
    const int m_hp = p->m_interp > 0 ? p->m_interp : m;
    std::vector<double> chp;
    if (hp && m_hp != m) {
        chp.resize((size_t)G * (m_hp + 1));
        for (int i = 0; i < G; ++i) cheb_coefficients(lam[i], m_hp, true, chp.data() + (size_t)i * (m_hp + 1));
    }
    st = run_interpolate(g, idx, slab, n_total, kmax, hp ? 1 : g_power, gamma, cg_tol, cg_max, labels_out, nullptr,
                         &local.cg, s, G > 1 ? k : nullptr, hp ? (chp.empty() ? c.data() : chp.data()) : nullptr,
                         m_hp);
    if (st != CSC_OK && st != CSC_E_NOT_CONVERGED) return done(st);
    cudaEventRecord(ev[5], s);
    cudaError_t ce = cudaEventSynchronize(ev[5]);
    if (ce != cudaSuccess) {
        set_error("csc_cluster_batched: %s", cudaGetErrorString(ce));
        return done(CSC_E_CUDA);
    }
    cudaEventElapsedTime(&local.ms_lambda, ev[0], ev[1]);
    cudaEventElapsedTime(&local.ms_filter, ev[1], ev[2]);
    cudaEventElapsedTime(&local.ms_sample, ev[2], ev[3]);
    cudaEventElapsedTime(&local.ms_kmeans, ev[3], ev[4]);
    cudaEventElapsedTime(&local.ms_interp, ev[4], ev[5]);
    cudaEventElapsedTime(&local.ms_total, ev[0], ev[5]);
    if (lambda_out) memcpy(lambda_out, lam.data(), G * sizeof(double));
    if (info) *info = local;
    return done(st);
}

}  // extern "C"
