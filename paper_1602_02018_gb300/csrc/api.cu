// api.cu -- the C ABI of libcsc (include/csc.h): graph handles, host-side
// mathematics (Jackson-Chebyshev coefficients, the eigencount dichotomy,
// reverse Cuthill-McKee) and the Alg. 2 pipeline driver.
#include <math.h>
#include <stdint.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "common.cuh"

namespace csc {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

csc_status ws_get(Graph* g, WsSlot slot, size_t bytes, void** out) {
    Buffer& b = g->ws[slot];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.ptr) {
            CSC_CUDA_TRY(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.ptr = nullptr;
            set_error("cudaMalloc(%zu) for scratch slot %d: %s", bytes, (int)slot, cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        b.bytes = bytes;
    }
    *out = b.ptr;
    return CSC_OK;
}

namespace {
struct TuneKey {
    uint64_t key;
    int device;
    int64_t N, nnz;
    bool operator<(const TuneKey& o) const {
        if (key != o.key) return key < o.key;
        if (device != o.device) return device < o.device;
        if (N != o.N) return N < o.N;
        return nnz < o.nnz;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaunchCfg> g_tune_cache;
}  // namespace

bool tune_cache_get(const Graph* g, uint64_t key, LaunchCfg* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(TuneKey{key, g->device, g->N, g->nnz});
    if (it == g_tune_cache.end()) return false;
    *out = it->second;
    return true;
}

void tune_cache_put(const Graph* g, uint64_t key, const LaunchCfg& cfg) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[TuneKey{key, g->device, g->N, g->nnz}] = cfg;
}

// Row ranges [bounds[b], bounds[b+1]) of rows lo..hi-1 split q ways with equal cost,
// cost(r) = light edges before r + 2r (nondecreasing).
static void split_rows(const std::vector<int64_t>& rp, int64_t lo, int64_t hi, int q, int32_t* bounds) {
    const double c0 = (double)rp[lo] + 2.0 * (double)lo;
    const double total = (double)rp[hi] + 2.0 * (double)hi - c0;
    int64_t a0 = lo;
    for (int b = 1; b < q; ++b) {
        const double target = c0 + total * (double)b / (double)q;
        int64_t a = a0, z = hi;
        while (a < z) {
            const int64_t mid = (a + z) / 2;
            if ((double)rp[mid] + 2.0 * (double)mid >= target) z = mid;
            else a = mid + 1;
        }
        a0 = a;
        bounds[b] = (int32_t)a;
    }
}

csc_status get_partition(Graph* g, int P, const int32_t** out) {
    auto it = g->parts.find(P);
    if (it != g->parts.end()) {
        *out = it->second;
        return CSC_OK;
    }
    const int64_t N = g->N;
    const std::vector<int64_t>& rp = g->h_light;  // heavy rows' edges are swept elsewhere
    std::vector<int32_t> bounds(P + 1);
    bounds[0] = 0;
    bounds[P] = (int32_t)N;
    std::vector<int32_t> gblk;
    const int G = g->n_graphs;
    if (G <= 1) {
        split_rows(rp, 0, N, P, bounds.data());
        gblk = {0, P};
    } else {
        // batched handle: every range inside one graph (per-graph sums then need no
        // segmentation inside a CTA); graph i gets 1 + its cost share of the other P - G
        if (P < G) {
            set_error("a row partition of a batch of %d graphs needs at least %d ranges (got %d)", G, G, P);
            return CSC_E_INVALID;
        }
        std::vector<double> cost(G);
        double total = 0.0;
        for (int i = 0; i < G; ++i) {
            const int64_t a = g->offsets[i], b = g->offsets[i + 1];
            cost[i] = (double)(rp[b] - rp[a]) + 2.0 * (double)(b - a);
            total += cost[i];
        }
        std::vector<int> q(G);
        std::vector<std::pair<double, int>> frac(G);
        int used = 0;
        for (int i = 0; i < G; ++i) {
            const double share = total > 0 ? (double)(P - G) * cost[i] / total : 0.0;
            q[i] = 1 + (int)floor(share);
            frac[i] = {-(share - floor(share)), i};
            used += q[i];
        }
        std::sort(frac.begin(), frac.end());  // largest remainder first, ties to the lower graph
        for (int r = 0; used < P; ++r, ++used) ++q[frac[r % G].second];
        gblk.assign(G + 1, 0);
        int b = 0;
        for (int i = 0; i < G; ++i) {
            gblk[i] = b;
            bounds[b] = (int32_t)g->offsets[i];
            split_rows(rp, g->offsets[i], g->offsets[i + 1], q[i], bounds.data() + b);
            bounds[b] = (int32_t)g->offsets[i];
            b += q[i];
        }
        gblk[G] = P;
    }
    int32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (P + 1) * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc for a row partition: %s", cudaGetErrorString(e));
        return CSC_E_OOM;
    }
    CSC_CUDA_TRY(cudaMemcpy(d, bounds.data(), (P + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    g->parts[P] = d;
    g->h_parts[P] = bounds;
    {
        // the largest staged CSR slice: row pointers r0 .. r1 and the range's light edges
        int64_t most = 0;
        for (int x = 0; x < P; ++x) {
            const int64_t nr = (int64_t)bounds[x + 1] - bounds[x];
            if (nr > 0) most = std::max(most, nr + 1 + (rp[bounds[x + 1]] - rp[bounds[x]]));
        }
        g->part_smem[P] = (int)(most * 4);
    }
    int32_t* dg = nullptr;
    e = cudaMalloc(&dg, gblk.size() * sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc for partition segments: %s", cudaGetErrorString(e));
        return CSC_E_OOM;
    }
    CSC_CUDA_TRY(cudaMemcpy(dg, gblk.data(), gblk.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    g->part_gblk[P] = dg;
    *out = d;
    return CSC_OK;
}

int staged_smem(const Graph* g, int P) {
    auto it = g->part_smem.find(P);
    return it == g->part_smem.end() ? 0 : it->second;
}

csc_status check_staged_smem(int bytes) {
    if (bytes > kStagedSmemMax) {
        set_error("a row range's CSR slice needs %d bytes of shared memory (at most %d): use more row ranges",
                  bytes, kStagedSmemMax);
        return CSC_E_UNSUPPORTED;
    }
    return CSC_OK;
}

csc_status fit_staged_partition(Graph* g, int P, int64_t max_p, int* out) {
    for (;;) {
        const int32_t* pr = nullptr;
        CSC_TRY(get_partition(g, P, &pr));
        if (staged_smem(g, P) <= kStagedSmemMax || P >= max_p) break;
        P = (int)std::min<int64_t>(max_p, 2 * (int64_t)P);
    }
    *out = P;
    return CSC_OK;
}

csc_status get_segments(Graph* g, int P, const int32_t** gblk, const int32_t** ghvy) {
    const int32_t* part = nullptr;
    CSC_TRY(get_partition(g, P, &part));
    *gblk = g->part_gblk[P];
    if (!g->d_hvy_start) {
        // first heavy row of each graph (the heavy list is in increasing row order)
        const int G = g->n_graphs < 1 ? 1 : g->n_graphs;
        std::vector<int32_t> hs(G + 1, 0);
        std::vector<int32_t> heavy(g->n_heavy);
        if (g->n_heavy)
            CSC_CUDA_TRY(cudaMemcpy(heavy.data(), g->heavy, g->n_heavy * sizeof(int32_t), cudaMemcpyDeviceToHost));
        for (int i = 0; i <= G; ++i) {
            const int64_t off = G == 1 ? (i == 0 ? 0 : g->N) : g->offsets[i];
            hs[i] = (int32_t)(std::lower_bound(heavy.begin(), heavy.end(), (int32_t)std::min<int64_t>(off, INT32_MAX)) -
                              heavy.begin());
        }
        hs[G] = g->n_heavy;
        cudaError_t e = cudaMalloc(&g->d_hvy_start, (G + 1) * sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->d_hvy_start = nullptr;
            set_error("cudaMalloc for heavy-row segments: %s", cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        CSC_CUDA_TRY(cudaMemcpy(g->d_hvy_start, hs.data(), (G + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    *ghvy = g->d_hvy_start;
    return CSC_OK;
}


// ------------------------------------------------- Jackson-Chebyshev (Sec. 4.3)
// c_j = g_j gamma_j for the ideal low-pass of Eq. 1 on t = lambda - 1 in [-1, 1]:
//   gamma_0 = 1 - theta/pi, gamma_j = -2 sin(j theta)/(j pi), theta = arccos(lambda_c - 1),
//   g_j = [(1 - j/(m+2)) sin(a) cos(j a) + cos(a) sin(j a)/(m+2)] / sin(a), a = pi/(m+2).
void cheb_coefficients(double lambda_c, int m, bool jackson, double* c) {
    double t = lambda_c - 1.0;
    t = t < -1.0 ? -1.0 : (t > 1.0 ? 1.0 : t);
    const double theta = acos(t);
    const double a = M_PI / (double)(m + 2);
    const double sa = sin(a), ca = cos(a);
    for (int j = 0; j <= m; ++j) {
        const double gam = j == 0 ? 1.0 - theta / M_PI : -2.0 * sin(j * theta) / (j * M_PI);
        double damp = 1.0;
        if (jackson)
            damp = ((1.0 - (double)j / (m + 2)) * sa * cos(j * a) + ca * sin(j * a) / (m + 2)) / sa;
        c[j] = gam * damp;
    }
}

static double eigencount_host(const double* mu, int m, double lambda, bool jackson, std::vector<double>& c) {
    c.resize(m + 1);
    cheb_coefficients(lambda, m, jackson, c.data());
    double s = 0.0;
    for (int j = 0; j <= m; ++j) s += c[j] * mu[j];
    return s;
}

static long long round_half_away(double x) { return x >= 0 ? (long long)floor(x + 0.5) : -(long long)floor(-x + 0.5); }

// Sec. 4.3 dichotomy on [lo, hi]: stop when round(count) == k.  `count(lambda,
// &value)` evaluates the eigencount (host arithmetic on moments, or a filter
// pass for the paper-literal estimator) and returns a status.
template <typename CountFn>
static csc_status dichotomy_fn(CountFn&& count, int k, double lo, double hi, csc_lambda_info* out) {
    for (int it = 1; it <= 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        double cnt = 0.0;
        CSC_TRY(count(mid, &cnt));
        if (round_half_away(cnt) == k) {
            out->lambda = mid;
            out->count = cnt;
            out->iters = it;
            out->hit = 1;
            return CSC_OK;
        }
        if (cnt > (double)k) hi = mid;
        else lo = mid;
        if (hi - lo < 1e-12 || it == 60) {
            out->lambda = hi;
            CSC_TRY(count(hi, &out->count));
            out->iters = it;
            out->hit = 0;
            return CSC_OK;
        }
    }
    return CSC_OK;
}

// The Sec. 4.3 halving started from a predicted cut-off c with half-width hw:
// the count at c decides the side, the predicted end on that side (c - hw or
// c + hw, clipped to [0, 2]) is evaluated next; when it lies across k the
// halving continues inside the prediction, else on the remaining part of
// [0, 2].  *inside tells whether the answer came from within [c - hw, c + hw].
template <typename CountFn>
static csc_status guarded_dichotomy(CountFn&& count, int k, double c, double hw, csc_lambda_info* out,
                                    bool* inside) {
    c = std::min(2.0, std::max(0.0, c));
    double v = 0.0;
    CSC_TRY(count(c, &v));
    *inside = true;
    if (round_half_away(v) == k) {
        out->lambda = c;
        out->count = v;
        out->iters = 1;
        out->hit = 1;
        return CSC_OK;
    }
    const bool above = v > (double)k;  // answer below c
    const double e = above ? std::max(0.0, c - hw) : std::min(2.0, c + hw);
    double ve = 0.0;
    CSC_TRY(count(e, &ve));
    if (round_half_away(ve) == k) {
        out->lambda = e;
        out->count = ve;
        out->iters = 2;
        out->hit = 1;
        return CSC_OK;
    }
    double lo, hi;
    if (above) {
        if (ve < (double)k) lo = e, hi = c;
        else lo = 0.0, hi = e, *inside = false;
    } else {
        if (ve > (double)k) lo = c, hi = e;
        else lo = e, hi = 2.0, *inside = false;
    }
    CSC_TRY(dichotomy_fn(count, k, lo, hi, out));
    out->iters += 2;
    return CSC_OK;
}

static void dichotomy(const double* mu, int m, int k, double lo, double hi, csc_lambda_info* out) {
    std::vector<double> c;
    dichotomy_fn(
        [&](double lam, double* v) {
            *v = eigencount_host(mu, m, lam, true, c);
            return CSC_OK;
        },
        k, lo, hi, out);
}

void estimate_from_moments(const double* mu, int m, int k, csc_lambda_info* out) { dichotomy(mu, m, k, 0.0, 2.0, out); }

// ------------------------------------------------------- host row chunks
// body(r0, r1) over contiguous row chunks of about equal edge counts (rp: row starts,
// clamped to a nondecreasing sequence so that an unvalidated rp still gives a partition;
// NULL: rows of equal weight), eight chunks per thread taken in order from a shared
// counter by up to all host cores; the caller's thread works too.  Each row must be
// handled independently of the split.
template <typename F>
static void for_row_chunks(int64_t N, const int64_t* rp, F&& body) {
    auto start = [&](int64_t i) { return rp ? std::max<int64_t>(rp[i], 0) : 0; };
    const int64_t nnz = start(N);
    const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(),
                                                              (N + nnz) / 65536));
    if (nt <= 1) {
        body(0, N);
        return;
    }
    const int64_t nc = nt * 8;
    std::vector<int64_t> cut(nc + 1, N);
    cut[0] = 0;
    for (int64_t c = 1; c < nc; ++c) {
        // first row whose start reaches c/nc of the edges plus rows (rows weigh one edge)
        const int64_t target = (nnz + N) * c / nc;
        int64_t a = cut[c - 1], z = N;
        while (a < z) {
            const int64_t mid = (a + z) / 2;
            if (start(mid) + mid >= target) z = mid;
            else a = mid + 1;
        }
        cut[c] = a;
    }
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        for (int64_t c; (c = next.fetch_add(1)) < nc;)
            if (cut[c] < cut[c + 1]) body(cut[c], cut[c + 1]);
    };
    std::vector<std::thread> pool;
    try {
        for (int64_t t = 1; t < nt; ++t) pool.emplace_back(worker);
    } catch (const std::system_error&) {
        // fewer threads than asked for: the chunks are shared among those that started
    }
    worker();
    for (auto& th : pool) th.join();
}

// --------------------------------------------------------- reverse Cuthill-McKee
// Stable counting sort of ids by a small integer key (degrees): the same order as a stable
// comparison sort by that key, in O(N + max key) without per-call allocations.
static void stable_sort_by_key(std::vector<int32_t>& ids, const std::vector<int32_t>& key, bool decreasing) {
    int32_t kmax = 0;
    for (int32_t v : ids) kmax = std::max(kmax, key[v]);
    std::vector<int64_t> start((size_t)kmax + 2, 0);
    for (int32_t v : ids) ++start[(size_t)(decreasing ? kmax - key[v] : key[v]) + 1];
    for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
    std::vector<int32_t> out(ids.size());
    for (int32_t v : ids) out[(size_t)start[(size_t)(decreasing ? kmax - key[v] : key[v])]++] = v;
    ids.swap(out);
}

// Cuthill & McKee (1969), reversed (George 1971): BFS from a minimum-degree
// node of each component, visiting neighbours by increasing degree; the
// visit order reversed gives perm[new] = old (then sorted by degree within
// blocks of 128 rows, see below).
static void rcm_order(int64_t N, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                      std::vector<int32_t>& perm, bool block_degree_sort) {
    std::vector<int32_t> deg(N);
    for (int64_t i = 0; i < N; ++i) deg[i] = (int32_t)(rp[i + 1] - rp[i]);
    std::vector<int32_t> order(N);
    std::iota(order.begin(), order.end(), 0);
    stable_sort_by_key(order, deg, false);
    std::vector<char> seen(N, 0);
    std::vector<int32_t> visit;
    visit.reserve(N);
    std::vector<int32_t> nb;
    // neighbours by increasing degree, ties in index order (a stable sort); short lists by
    // insertion, which allocates nothing
    auto by_degree = [&](std::vector<int32_t>& l) {
        if (l.size() <= 32) {
            for (size_t i = 1; i < l.size(); ++i) {
                const int32_t v = l[i];
                size_t j = i;
                for (; j > 0 && deg[l[j - 1]] > deg[v]; --j) l[j] = l[j - 1];
                l[j] = v;
            }
        } else {
            std::stable_sort(l.begin(), l.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
        }
    };
    // A large level is expanded on all host cores with the same result: a node of the next
    // level belongs to the first node of this level (in visit order) adjacent to it, and
    // each node's own new neighbours follow in the order above, so the next level is its
    // nodes' neighbour lists concatenated in visit order.  owner[v] collects that first
    // position (an atomic minimum); owner is unset (INT32_MAX) for every other node.
    std::unique_ptr<std::atomic<int32_t>[]> owner;
    std::vector<int64_t> wsum, cnt;
    auto expand_parallel = [&](int64_t l0, int64_t l1) {
        if (!owner) {
            owner.reset(new std::atomic<int32_t>[N]);
            for (int64_t i = 0; i < N; ++i) owner[i].store(INT32_MAX, std::memory_order_relaxed);
        }
        const int64_t nl = l1 - l0;
        wsum.assign(nl + 1, 0);
        for (int64_t i = 0; i < nl; ++i) wsum[i + 1] = wsum[i] + deg[visit[l0 + i]];
        for_row_chunks(nl, wsum.data(), [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                const int32_t u = visit[l0 + i], pos = (int32_t)(l0 + i);
                for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                    const int32_t v = ci[e];
                    if (seen[v]) continue;
                    int32_t cur = owner[v].load(std::memory_order_relaxed);
                    while (pos < cur && !owner[v].compare_exchange_weak(cur, pos, std::memory_order_relaxed)) {
                    }
                }
            }
        });
        cnt.assign(nl + 1, 0);
        for_row_chunks(nl, wsum.data(), [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                const int32_t u = visit[l0 + i], pos = (int32_t)(l0 + i);
                int64_t c = 0;
                for (int64_t e = rp[u]; e < rp[u + 1]; ++e) c += owner[ci[e]].load(std::memory_order_relaxed) == pos;
                cnt[i + 1] = c;
            }
        });
        for (int64_t i = 0; i < nl; ++i) cnt[i + 1] += cnt[i];
        visit.resize((size_t)(l1 + cnt[nl]));
        for_row_chunks(nl, wsum.data(), [&](int64_t i0, int64_t i1) {
            std::vector<int32_t> kids;
            for (int64_t i = i0; i < i1; ++i) {
                const int32_t u = visit[l0 + i], pos = (int32_t)(l0 + i);
                kids.clear();
                for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
                    if (owner[ci[e]].load(std::memory_order_relaxed) == pos) kids.push_back(ci[e]);
                by_degree(kids);
                std::copy(kids.begin(), kids.end(), visit.begin() + l1 + cnt[i]);
            }
        });
        for_row_chunks(cnt[nl], nullptr, [&](int64_t j0, int64_t j1) {
            for (int64_t j = j0; j < j1; ++j) {
                const int32_t v = visit[l1 + j];
                seen[v] = 1;
                owner[v].store(INT32_MAX, std::memory_order_relaxed);
            }
        });
    };
    constexpr int64_t kParallelLevel = 1 << 17;  // edges + nodes of a level worth the threads
    for (int64_t s = 0; s < N; ++s) {
        const int32_t start = order[s];
        if (seen[start]) continue;
        int64_t l0 = (int64_t)visit.size();
        visit.push_back(start);
        seen[start] = 1;
        while (l0 < (int64_t)visit.size()) {  // one level [l0, l1) at a time
            const int64_t l1 = (int64_t)visit.size();
            int64_t work = l1 - l0;
            for (int64_t i = l0; i < l1 && work < kParallelLevel; ++i) work += deg[visit[i]];
            if (work >= kParallelLevel && std::thread::hardware_concurrency() > 1) {
                expand_parallel(l0, l1);
            } else {
                for (int64_t i = l0; i < l1; ++i) {
                    const int32_t u = visit[i];
                    nb.clear();
                    for (int64_t e = rp[u]; e < rp[u + 1]; ++e)
                        if (!seen[ci[e]]) {
                            seen[ci[e]] = 1;
                            nb.push_back(ci[e]);
                        }
                    by_degree(nb);
                    visit.insert(visit.end(), nb.begin(), nb.end());
                }
            }
            l0 = l1;
        }
    }
    perm.assign(visit.rbegin(), visit.rend());
    // a global stable sort by degree that follows leaves equal-degree rows in this order,
    // which the block sort below does not change: skipped then
    if (!block_degree_sort) return;
    // then, within blocks of kDegreeBlock consecutive rows, rows by decreasing degree: the two
    // lane groups of a warp sweep neighbouring rows, which then need about as many gather
    // batches each (power-law degrees otherwise leave one group idle while the other
    // finishes a long row); the block is far below a row range, so locality is kept
    constexpr int64_t kDegreeBlock = 128;
    for (int64_t b = 0; b < N; b += kDegreeBlock)
        std::stable_sort(perm.begin() + b, perm.begin() + std::min<int64_t>(N, b + kDegreeBlock),
                         [&](int32_t x, int32_t y) { return deg[x] > deg[y]; });
}

// ------------------------------------------------------------- graph create
struct HostCSR {
    int64_t N = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
};

// Validate a CSR (sorted rows, in range, optional symmetry) and drop self loops.
static csc_status validate_and_clean(int64_t N, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                     bool check_sym, HostCSR& out, int64_t node_base = 0) {
    if (row_ptr[0] != 0) {
        set_error("row_ptr[0] = %lld, expected 0", (long long)row_ptr[0]);
        return CSC_E_CSR;
    }
    if (row_ptr[N] != nnz) {
        set_error("row_ptr[N] = %lld differs from nnz = %lld", (long long)row_ptr[N], (long long)nnz);
        return CSC_E_CSR;
    }
    out.N = N;
    out.rp.assign(N + 1, 0);
    // first pass, rows in parallel: each row checked as a row-by-row scan would (its extent,
    // then its columns in order) and its kept (non-loop) entries counted into rp[i + 1]; a
    // chunk stops at its first bad row, and the lowest bad row of all chunks is reported,
    // so the message is the one a sequential scan gives
    struct Bad {
        int64_t row = -1, pos = 0, col = 0;
        int kind = 0;  // 1 extent, 2 column out of range, 3 not strictly increasing, 4 asymmetric
    };
    std::mutex mu;
    Bad first;
    auto note = [&](const Bad& b) {
        std::lock_guard<std::mutex> lk(mu);
        if (first.row < 0 || b.row < first.row || (b.row == first.row && b.pos < first.pos)) first = b;
    };
    for_row_chunks(N, row_ptr, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; ++i) {
            const int64_t b = row_ptr[i], e = row_ptr[i + 1];
            if (e < b || b < 0 || e > nnz) {
                note(Bad{i, 0, 0, 1});
                return;
            }
            int64_t prev = -1, kept = 0;
            for (int64_t p = b; p < e; ++p) {
                const int64_t c = col_idx[p];
                if (c < 0 || c >= N) {
                    note(Bad{i, p, c, 2});
                    return;
                }
                if (c <= prev) {
                    note(Bad{i, p, c, 3});
                    return;
                }
                prev = c;
                kept += c != i ? 1 : 0;
            }
            out.rp[i + 1] = kept;
        }
    });
    if (first.row >= 0) {
        if (first.kind == 1)
            set_error("row_ptr not nondecreasing at row %lld", (long long)(first.row + node_base));
        else if (first.kind == 2)
            set_error("col_idx[%lld] = %lld out of range [0, %lld)", (long long)first.pos, (long long)first.col,
                      (long long)N);
        else
            set_error("row %lld not strictly increasing (duplicate or unsorted column %lld)",
                      (long long)(first.row + node_base), (long long)first.col);
        return CSC_E_CSR;
    }
    for (int64_t i = 0; i < N; ++i) out.rp[i + 1] += out.rp[i];
    out.ci.resize((size_t)out.rp[N]);
    // second pass: the kept entries of each row copied to its new start
    for_row_chunks(N, row_ptr, [&](int64_t r0, int64_t r1) {
        for (int64_t i = r0; i < r1; ++i) {
            int64_t w = out.rp[i];
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                if (col_idx[p] != i) out.ci[w++] = col_idx[p];
        }
    });
    if (check_sym) {
        for_row_chunks(N, out.rp.data(), [&](int64_t r0, int64_t r1) {
            for (int64_t i = r0; i < r1; ++i)
                for (int64_t p = out.rp[i]; p < out.rp[i + 1]; ++p) {
                    const int32_t j = out.ci[p];
                    const int32_t* b = out.ci.data() + out.rp[j];
                    const int32_t* e = out.ci.data() + out.rp[j + 1];
                    if (!std::binary_search(b, e, (int32_t)i)) {
                        note(Bad{i, p, j, 4});
                        return;
                    }
                }
        });
        if (first.row >= 0) {
            set_error("matrix not symmetric: (%lld, %lld) present, (%lld, %lld) missing",
                      (long long)(first.row + node_base), (long long)first.col, (long long)first.col,
                      (long long)(first.row + node_base));
            return CSC_E_CSR;
        }
    }
    return CSC_OK;
}

static void permute_csr(const HostCSR& in, const std::vector<int32_t>& perm, HostCSR& out) {
    const int64_t N = in.N;
    std::vector<int32_t> iperm(N);
    for (int64_t p = 0; p < N; ++p) iperm[perm[p]] = (int32_t)p;
    out.N = N;
    out.rp.assign(N + 1, 0);
    out.ci.resize(in.ci.size());
    for (int64_t p = 0; p < N; ++p) {
        const int32_t o = perm[p];
        out.rp[p + 1] = out.rp[p] + (in.rp[o + 1] - in.rp[o]);
    }
    // rows relabelled and sorted independently, in chunks of about equal edge counts over
    // the host's cores (the hub rows, which the degree orders put first, do not all fall to
    // one thread; the result does not depend on the split)
    for_row_chunks(N, out.rp.data(), [&](int64_t p0, int64_t p1) {
        for (int64_t p = p0; p < p1; ++p) {
            const int32_t o = perm[p];
            int64_t w = out.rp[p];
            for (int64_t e = in.rp[o]; e < in.rp[o + 1]; ++e) out.ci[w++] = iperm[in.ci[e]];
            std::sort(out.ci.begin() + out.rp[p], out.ci.begin() + out.rp[p + 1]);
        }
    });
}

static void free_graph(Graph* g) {
    if (!g) return;
    cudaFree(g->row_ptr);
    cudaFree(g->col_idx);
    cudaFree(g->dinv);
    cudaFree(g->dinv64);
    cudaFree(g->deg);
    cudaFree(g->invdeg);
    cudaFree(g->sqdeg);
    cudaFree(g->invdeg64);
    cudaFree(g->sqdeg64);
    cudaFree(g->perm);
    cudaFree(g->iperm);
    cudaFree(g->d_offsets);
    cudaFree(g->graph_of_row);
    for (auto& b : g->ws) cudaFree(b.ptr);
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second.first);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->side_stream) cudaStreamDestroy(g->side_stream);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    for (auto& kv : g->parts) cudaFree(kv.second);
    for (auto& kv : g->part_gblk) cudaFree(kv.second);
    cudaFree(g->d_hvy_start);
    cudaFree(g->heavy);
    if (g->light_owned) {
        cudaFree(g->lrp);
        cudaFree(g->lci);
    }
    for (auto& e : g->ev)
        if (e) cudaEventDestroy(e);
    if (g->pinned) cudaFreeHost(g->pinned);
    delete g;
}

template <typename T>
static csc_status dev_alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc(%zu): %s", count * sizeof(T), cudaGetErrorString(e));
        return CSC_E_OOM;
    }
    return CSC_OK;
}

// Upload a cleaned CSR (already in internal order) and compute degrees.
static csc_status upload(Graph* g, const HostCSR& h, const std::vector<int32_t>* perm, cudaStream_t s) {
    const int64_t N = h.N;
    const int64_t nnz = (int64_t)h.ci.size();
    if (nnz >= (int64_t)INT32_MAX) {
        set_error("nnz = %lld exceeds the int32 row-pointer range of the library", (long long)nnz);
        return CSC_E_UNSUPPORTED;
    }
    g->N = N;
    g->nnz = nnz;
    CSC_CUDA_TRY(cudaGetDevice(&g->device));
    CSC_CUDA_TRY(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    {
        int l2 = 0;
        CSC_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device));
        g->l2_bytes = l2;
    }
    std::vector<int32_t>& rp32 = g->h_row_ptr;
    rp32.resize(N + 1);
    for (int64_t i = 0; i <= N; ++i) rp32[i] = (int32_t)h.rp[i];
    std::vector<int32_t> heavy;
    g->h_light.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) {
        const int64_t dg = h.rp[i + 1] - h.rp[i];
        if (dg > kHeavyRow) heavy.push_back((int32_t)i);
        g->h_light[i + 1] = g->h_light[i] + (dg > kHeavyRow ? 0 : dg);
    }
    g->n_heavy = (int)heavy.size();
    {
        // degree quantiles by counting sort (the sorted degree at index floor(p (N - 1)))
        int64_t max_deg = 0;
        for (int64_t i = 0; i < N; ++i) max_deg = std::max(max_deg, h.rp[i + 1] - h.rp[i]);
        std::vector<int64_t> cnt(max_deg + 2, 0);
        for (int64_t i = 0; i < N; ++i) ++cnt[h.rp[i + 1] - h.rp[i]];
        static const double kQ[6] = {0.0, 0.1, 0.25, 0.5, 0.75, 1.0};
        int64_t below = 0, dv = 0;
        for (int q = 0; q < 6; ++q) {
            const int64_t at = (int64_t)floor(kQ[q] * (double)(N - 1));
            while (below + cnt[dv] <= at) below += cnt[dv++];
            g->deg_quant[q] = (int32_t)dv;
        }
    }
    if (!heavy.empty()) {
        CSC_TRY(dev_alloc(&g->heavy, heavy.size()));
        CSC_CUDA_TRY(cudaMemcpy(g->heavy, heavy.data(), heavy.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    CSC_TRY(dev_alloc(&g->row_ptr, N + 1));
    CSC_TRY(dev_alloc(&g->col_idx, nnz));
    CSC_TRY(dev_alloc(&g->dinv, N));
    CSC_TRY(dev_alloc(&g->dinv64, N));
    CSC_TRY(dev_alloc(&g->deg, N));
    CSC_TRY(dev_alloc(&g->invdeg, N));
    CSC_TRY(dev_alloc(&g->sqdeg, N));
    CSC_TRY(dev_alloc(&g->invdeg64, N));
    CSC_TRY(dev_alloc(&g->sqdeg64, N));
    CSC_CUDA_TRY(cudaMemcpyAsync(g->row_ptr, rp32.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (nnz)
        CSC_CUDA_TRY(cudaMemcpyAsync(g->col_idx, h.ci.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (heavy.empty()) {
        g->lrp = g->row_ptr;  // no heavy rows: the CSR is its own light part
        g->lci = g->col_idx;
    } else {
        // compact light CSR: heavy rows keep no edges and are flagged in bit 31
        const int64_t nl = g->h_light[N];
        std::vector<int32_t> lrp(N + 1), lci((size_t)std::max<int64_t>(nl, 1));
        lrp[0] = 0;
        for (int64_t i = 0; i < N; ++i) {
            const int64_t a = h.rp[i], b = h.rp[i + 1];
            const bool hv = b - a > kHeavyRow;
            if (!hv) std::copy(h.ci.begin() + a, h.ci.begin() + b, lci.begin() + g->h_light[i]);
            lrp[i + 1] = (int32_t)g->h_light[i + 1] | (hv ? (int32_t)0x80000000u : 0);
        }
        g->light_owned = true;
        CSC_TRY(dev_alloc(&g->lrp, N + 1));
        CSC_TRY(dev_alloc(&g->lci, lci.size()));
        CSC_CUDA_TRY(cudaMemcpy(g->lrp, lrp.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
        CSC_CUDA_TRY(cudaMemcpy(g->lci, lci.data(), lci.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    if (perm) {
        std::vector<int32_t> iperm(N);
        for (int64_t p = 0; p < N; ++p) iperm[(*perm)[p]] = (int32_t)p;
        CSC_TRY(dev_alloc(&g->perm, N));
        CSC_TRY(dev_alloc(&g->iperm, N));
        CSC_CUDA_TRY(cudaMemcpyAsync(g->perm, perm->data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CSC_CUDA_TRY(cudaMemcpyAsync(g->iperm, iperm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    CSC_CUDA_TRY(cudaMallocHost((void**)&g->pinned, 4096 * sizeof(double)));
    for (auto& e : g->ev) CSC_CUDA_TRY(cudaEventCreate(&e));
    CSC_TRY(launch_degrees(g, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    return CSC_OK;
}

static csc_status check_graph(csc_graph g) {
    if (!g) {
        set_error("null graph handle");
        return CSC_E_INVALID;
    }
    if (g->poisoned) {
        set_error("graph handle unusable after an earlier CUDA error");
        return CSC_E_CUDA;
    }
    return CSC_OK;
}

static csc_status poison_on_cuda(Graph* g, csc_status st) {
    if (st == CSC_E_CUDA && g) g->poisoned = true;
    return st;
}

}  // namespace csc

using namespace csc;

extern "C" {

const char* csc_version(void) { return "csc-gb300 0.1 (sm_103a)"; }

const char* csc_status_str(csc_status s) {
    switch (s) {
        case CSC_OK: return "CSC_OK";
        case CSC_E_INVALID: return "CSC_E_INVALID";
        case CSC_E_CSR: return "CSC_E_CSR";
        case CSC_E_OOM: return "CSC_E_OOM";
        case CSC_E_CUDA: return "CSC_E_CUDA";
        case CSC_E_NOT_CONVERGED: return "CSC_E_NOT_CONVERGED";
        case CSC_E_DEVICE_TIMEOUT: return "CSC_E_DEVICE_TIMEOUT";
        case CSC_E_NUMERIC: return "CSC_E_NUMERIC";
        case CSC_E_UNSUPPORTED: return "CSC_E_UNSUPPORTED";
        default: return "CSC_E_UNKNOWN";
    }
}

const char* csc_last_error(void) { return g_last_error.c_str(); }

csc_status csc_graph_create(int64_t N, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                            const float* weights, uint32_t flags, void* stream, csc_graph* out) {
    clear_error();
    if (!out || !row_ptr || (nnz > 0 && !col_idx) || N < 1 || nnz < 0) {
        set_error("csc_graph_create: invalid arguments (N=%lld, nnz=%lld)", (long long)N, (long long)nnz);
        return CSC_E_INVALID;
    }
    *out = nullptr;
    if (weights) {
        set_error("weighted graphs are not supported: pass weights = NULL");
        return CSC_E_UNSUPPORTED;
    }
    if (N >= (int64_t)INT32_MAX || nnz >= (int64_t)INT32_MAX) {
        set_error("N and nnz must be below 2^31");
        return CSC_E_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> hrp;
    std::vector<int32_t> hci;
    const int64_t* rp = row_ptr;
    const int32_t* ci = col_idx;
    if (flags & CSC_DEVICE_INPUT) {
        hrp.resize(N + 1);
        hci.resize(nnz);
        CSC_CUDA_TRY(cudaMemcpyAsync(hrp.data(), row_ptr, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (nnz) CSC_CUDA_TRY(cudaMemcpyAsync(hci.data(), col_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        rp = hrp.data();
        ci = hci.data();
    }
    HostCSR clean;
    try {
        CSC_TRY(validate_and_clean(N, nnz, rp, ci, (flags & CSC_CHECK_SYM) != 0, clean));
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed while validating the CSR");
        return CSC_E_OOM;
    }
    csc_graph g = new (std::nothrow) csc_graph_s();
    if (!g) {
        set_error("host allocation failed");
        return CSC_E_OOM;
    }
    csc_status st;
    if (flags & (CSC_RCM | CSC_DEGREE_ORDER)) {
        std::vector<int32_t> perm;
        if (flags & CSC_RCM) {
            rcm_order(N, clean.rp, clean.ci, perm, (flags & CSC_DEGREE_ORDER) == 0);
        } else {
            perm.resize(N);
            std::iota(perm.begin(), perm.end(), 0);
        }
        if (flags & CSC_DEGREE_ORDER) {
            // decreasing degree: the rows most neighbours gather come first, back to back
            std::vector<int32_t> deg(N);
            for (int64_t i = 0; i < N; ++i) deg[i] = (int32_t)(clean.rp[i + 1] - clean.rp[i]);
            stable_sort_by_key(perm, deg, true);
        }
        HostCSR pc;
        permute_csr(clean, perm, pc);
        st = upload(g, pc, &perm, s);
    } else {
        st = upload(g, clean, nullptr, s);
    }
    if (st != CSC_OK) {
        free_graph(g);
        return st;
    }
    g->offsets = {0, N};
    *out = g;
    return CSC_OK;
}

csc_status csc_graph_create_batched(int32_t G, const int64_t* Ns, const int64_t* const* row_ptr,
                                    const int32_t* const* col_idx, uint32_t flags, void* stream, csc_graph* out) {
    clear_error();
    if (!out || G < 1 || !Ns || !row_ptr || !col_idx) {
        set_error("csc_graph_create_batched: invalid arguments");
        return CSC_E_INVALID;
    }
    *out = nullptr;
    if (flags & (CSC_DEVICE_INPUT | CSC_RCM | CSC_DEGREE_ORDER)) {
        set_error("csc_graph_create_batched: host input only, without reordering");
        return CSC_E_UNSUPPORTED;
    }
    HostCSR packed;
    std::vector<int64_t> offsets(G + 1, 0);
    for (int i = 0; i < G; ++i) {
        if (Ns[i] < 1 || !row_ptr[i]) {
            set_error("csc_graph_create_batched: graph %d has N < 1 or a null row_ptr", i);
            return CSC_E_INVALID;
        }
        offsets[i + 1] = offsets[i] + Ns[i];
    }
    const int64_t NT = offsets[G];
    if (NT >= (int64_t)INT32_MAX) {
        set_error("packed node count must be below 2^31");
        return CSC_E_UNSUPPORTED;
    }
    packed.N = NT;
    packed.rp.assign(NT + 1, 0);
    try {
        for (int i = 0; i < G; ++i) {
            HostCSR one;
            const int64_t nnz_i = row_ptr[i][Ns[i]];
            if (nnz_i > 0 && !col_idx[i]) {
                set_error("graph %d: col_idx is NULL", i);
                return CSC_E_INVALID;
            }
            CSC_TRY(validate_and_clean(Ns[i], nnz_i, row_ptr[i], col_idx[i], (flags & CSC_CHECK_SYM) != 0, one,
                                       offsets[i]));
            const int64_t base = (int64_t)packed.ci.size();
            for (int64_t r = 0; r < Ns[i]; ++r) packed.rp[offsets[i] + r + 1] = base + one.rp[r + 1];
            for (int32_t c : one.ci) packed.ci.push_back((int32_t)(c + offsets[i]));
        }
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed while packing graphs");
        return CSC_E_OOM;
    }
    csc_graph g = new (std::nothrow) csc_graph_s();
    if (!g) {
        set_error("host allocation failed");
        return CSC_E_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    csc_status st = upload(g, packed, nullptr, s);
    if (st == CSC_OK) {
        g->n_graphs = G;
        g->offsets = offsets;
        std::vector<int32_t> gid(NT);
        for (int i = 0; i < G; ++i)
            for (int64_t r = offsets[i]; r < offsets[i + 1]; ++r) gid[r] = i;
        st = dev_alloc(&g->d_offsets, G + 1);
        if (st == CSC_OK) st = dev_alloc(&g->graph_of_row, NT);
        if (st == CSC_OK && (cudaMemcpy(g->d_offsets, offsets.data(), (G + 1) * sizeof(int64_t),
                                        cudaMemcpyHostToDevice) != cudaSuccess ||
                             cudaMemcpy(g->graph_of_row, gid.data(), NT * sizeof(int32_t),
                                        cudaMemcpyHostToDevice) != cudaSuccess)) {
            set_error("copying batch tables failed");
            st = CSC_E_CUDA;
        }
    }
    if (st != CSC_OK) {
        free_graph(g);
        return st;
    }
    *out = g;
    return CSC_OK;
}

csc_status csc_graph_destroy(csc_graph g) {
    if (!g) return CSC_OK;
    free_graph(g);
    return CSC_OK;
}

csc_status csc_graph_info(csc_graph g, int64_t* N, int64_t* nnz, int32_t* n_graphs) {
    CSC_TRY(check_graph(g));
    if (N) *N = g->N;
    if (nnz) *nnz = g->nnz;
    if (n_graphs) *n_graphs = g->n_graphs;
    return CSC_OK;
}

csc_status csc_graph_tuned_shape(csc_graph g, int32_t i, int32_t* kind, int32_t* dtype_bytes, int32_t* columns,
                                 int32_t* shape) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (i < 0 || i >= (int32_t)g->tuned.size()) return CSC_E_INVALID;
    auto it = g->tuned.begin();
    std::advance(it, i);
    const uint64_t key = it->first;
    if (kind) *kind = (int32_t)(key >> 48);
    if (dtype_bytes) *dtype_bytes = (int32_t)((key >> 40) & 0xff);
    if (columns) *columns = (int32_t)(key & 0xffffffffu);
    if (shape) {
        shape[0] = it->second.G;
        shape[1] = it->second.NT;
        shape[2] = it->second.threads;
        shape[3] = it->second.P;
        shape[4] = it->second.tiles;
        shape[5] = (it->second.staged ? 0 : 1) | (it->second.lean ? 2 : 0);
    }
    return CSC_OK;
}

csc_status csc_graph_pin_shape(csc_graph g, int32_t kind, int32_t dtype_bytes, int32_t columns,
                               const int32_t* shape) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!shape || kind < 1 || kind > 4 || columns < 1 || shape[0] < 1 || shape[1] < 1 ||
        (shape[2] != 256 && shape[2] != 512) || shape[3] < 1 || shape[4] < 1 || shape[5] < 0 || shape[5] > 3) {
        set_error("csc_graph_pin_shape: invalid shape");
        return CSC_E_INVALID;
    }
    if ((shape[5] & 2) && ((kind != 3 && kind != 4) || shape[1] != 1 || shape[2] != 256)) {
        set_error("csc_graph_pin_shape: the lean form exists for the CG products and Clenshaw orders with NT = 1 "
                  "and 256 threads");
        return CSC_E_INVALID;
    }
    const int vec_bytes = 16;
    const int elem = kind == 3 ? 4 : dtype_bytes;
    if (elem != 2 && elem != 4 && elem != 8) {
        set_error("csc_graph_pin_shape: dtype_bytes must be 2, 4 or 8");
        return CSC_E_INVALID;
    }
    const int nv = (columns * elem + vec_bytes - 1) / vec_bytes;
    const int cap = shape[0] * shape[1];
    if ((nv + cap - 1) / cap != shape[4]) {
        set_error("csc_graph_pin_shape: %d column tiles do not match %d columns at G*NT = %d", shape[4], columns, cap);
        return CSC_E_INVALID;
    }
    LaunchCfg c;
    c.G = shape[0];
    c.NT = shape[1];
    c.threads = shape[2];
    c.P = shape[3];
    c.tiles = shape[4];
    c.staged = (shape[5] & 1) ? 0 : 1;
    c.lean = (shape[5] & 2) ? 1 : 0;
    const uint64_t key = kind == 3 ? ((3ull << 48) | (uint64_t)(uint32_t)columns)
                                   : (((uint64_t)kind << 48) | ((uint64_t)(dtype_bytes & 0xff) << 40) |
                                      (uint64_t)(uint32_t)columns);
    g->tuned[key] = c;
    return CSC_OK;
}

csc_status csc_graph_degrees(csc_graph g, int32_t* deg_out, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!deg_out) {
        set_error("deg_out is NULL");
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> d(g->N);
    cudaError_t e = cudaMemcpyAsync(d.data(), g->deg, g->N * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("copying degrees: %s", cudaGetErrorString(e));
        return poison_on_cuda(g, CSC_E_CUDA);
    }
    if (g->perm) {
        std::vector<int32_t> perm(g->N);
        e = cudaMemcpy(perm.data(), g->perm, g->N * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("copying permutation: %s", cudaGetErrorString(e));
            return poison_on_cuda(g, CSC_E_CUDA);
        }
        for (int64_t p = 0; p < g->N; ++p) deg_out[perm[p]] = d[p];
    } else {
        memcpy(deg_out, d.data(), g->N * sizeof(int32_t));
    }
    return CSC_OK;
}

csc_status csc_chebyshev_coefficients(double lambda_c, int32_t m, uint32_t flags, double* c_out) {
    clear_error();
    if (m < 0 || !c_out || !(lambda_c >= 0.0 && lambda_c <= 2.0)) {
        set_error("csc_chebyshev_coefficients: need m >= 0, lambda_c in [0, 2], c_out != NULL");
        return CSC_E_INVALID;
    }
    cheb_coefficients(lambda_c, m, (flags & CSC_NO_JACKSON) == 0, c_out);
    return CSC_OK;
}

csc_status csc_filter_random_signals(csc_graph g, double lambda_c, int32_t m, int32_t d, int32_t d_pad,
                                     uint64_t seed, csc_dtype storage, const float* R_in, void* Y_out,
                                     uint32_t flags, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (m < 0 || d < 1 || d_pad < d || d_pad % 8 != 0 || !Y_out || !(lambda_c >= 0.0 && lambda_c <= 2.0) ||
        (storage != CSC_F32 && storage != CSC_BF16 && storage != CSC_F64)) {
        set_error("csc_filter_random_signals: invalid arguments (m=%d d=%d d_pad=%d lambda_c=%g storage=%d)", m, d,
                  d_pad, lambda_c, (int)storage);
        return CSC_E_INVALID;
    }
    std::vector<double> c(m + 1);
    cheb_coefficients(lambda_c, m, (flags & CSC_NO_JACKSON) == 0, c.data());
    const bool check = (flags & CSC_CHECK_FINITE) != 0;
    if (check && R_in) {
        const csc_status sc = run_check_finite(g, R_in, false, g->N, d, d_pad, "R_in", (cudaStream_t)stream);
        if (sc != CSC_OK) return poison_on_cuda(g, sc);
    }
    csc_status st = run_filter(g, c.data(), m, d, d_pad, seed, storage, R_in, Y_out,
                               (flags & CSC_NORMALIZE_ROWS) != 0, (cudaStream_t)stream, (flags & CSC_CLENSHAW) != 0);
    if (st == CSC_OK && check)
        st = run_check_finite(g, Y_out, storage == CSC_F64, g->N, d, d_pad, "the filtered block Y",
                              (cudaStream_t)stream);
    return poison_on_cuda(g, st);
}

csc_status csc_kpm_moments(csc_graph g, int32_t n_moments, int32_t n_probes, uint64_t seed, csc_dtype storage,
                           double* mu_out, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (n_moments < 1 || n_probes < 0 || !mu_out || n_moments > 4096) {
        set_error("csc_kpm_moments: need 1 <= n_moments <= 4096, n_probes >= 0, mu_out != NULL");
        return CSC_E_INVALID;
    }
    if (n_probes == 0) n_probes = g->N > 1 ? (int)ceil(2.0 * log((double)g->N)) : 1;  // Sec. 4.3: 2 log N
    return poison_on_cuda(g, run_moments(g, n_moments, n_probes, seed, storage, mu_out, nullptr,
                                         (cudaStream_t)stream));
}

csc_status csc_eigencount(const double* mu, int32_t m, double lambda, uint32_t flags, double* count_out) {
    clear_error();
    if (!mu || !count_out || m < 0 || !(lambda >= 0.0 && lambda <= 2.0)) {
        set_error("csc_eigencount: invalid arguments");
        return CSC_E_INVALID;
    }
    std::vector<double> c;
    *count_out = eigencount_host(mu, m, lambda, (flags & CSC_NO_JACKSON) == 0, c);
    return CSC_OK;
}

csc_status csc_estimate_lambda_k(csc_graph g, int32_t k, int32_t m, int32_t n_probes, uint64_t seed,
                                 const double* bracket, csc_lambda_info* out, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (k < 1 || m < 1 || n_probes < 0 || !out ||
        (bracket && !(bracket[0] >= 0.0 && bracket[0] < bracket[1] && bracket[1] <= 2.0))) {
        set_error("csc_estimate_lambda_k: invalid arguments (k=%d m=%d n_probes=%d)", k, m, n_probes);
        return CSC_E_INVALID;
    }
    if (n_probes == 0) n_probes = g->N > 1 ? (int)ceil(2.0 * log((double)g->N)) : 1;
    std::vector<double> mu(m + 1);
    int passes = 0;
    csc_status st = run_moments(g, m + 1, n_probes, seed, CSC_F32, mu.data(), &passes, (cudaStream_t)stream);
    if (st != CSC_OK) return poison_on_cuda(g, st);
    memset(out, 0, sizeof(*out));
    out->n_probes = n_probes;
    out->m = m;
    out->moment_passes = passes;
    double lo = 0.0, hi = 2.0;
    if (bracket) {
        std::vector<double> c;
        const double clo = eigencount_host(mu.data(), m, bracket[0], true, c);
        const double chi = eigencount_host(mu.data(), m, bracket[1], true, c);
        if (round_half_away(clo) <= k && k <= round_half_away(chi)) {
            lo = bracket[0];
            hi = bracket[1];
            out->bracket_used = 1;
        }
    }
    dichotomy(mu.data(), m, k, lo, hi, out);
    return CSC_OK;
}

// ------------------------------------------------ learned lambda_k bracket

// Smallest lambda in [0, 2] (60 halvings) where count(lambda) reaches `level`;
// count is nondecreasing in lambda.
static double count_crossing(const double* mu, int m, double level) {
    std::vector<double> c;
    double lo = 0.0, hi = 2.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (eigencount_host(mu, m, mid, true, c) < level) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static csc_status bracket_features(Graph* g, int k, uint64_t seed, float* feat, double* mu, int* passes,
                                   cudaStream_t s) {
    CSC_TRY(run_moments(g, CSC_BRACKET_MOMENTS, CSC_BRACKET_PROBES, seed, CSC_F32, mu, passes, s));
    const int64_t N = g->N;
    for (int j = 0; j < CSC_BRACKET_MOMENTS; ++j) feat[j] = (float)(mu[j] / (double)N);
    feat[CSC_BRACKET_MOMENTS] = (float)log((double)N);
    feat[CSC_BRACKET_MOMENTS + 1] = (float)k;
    // degree quantiles (computed when the graph was created)
    for (int q = 0; q < 6; ++q) feat[CSC_BRACKET_MOMENTS + 2 + q] = (float)log1p((double)g->deg_quant[q]);
    return CSC_OK;
}

csc_status csc_bracket_features(csc_graph g, int32_t k, uint64_t seed, float* feat_out, double* mu_out,
                                void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (k < 1 || !feat_out) {
        set_error("csc_bracket_features: need k >= 1 and feat_out");
        return CSC_E_INVALID;
    }
    double mu[CSC_BRACKET_MOMENTS];
    int passes = 0;
    csc_status st = bracket_features(g, k, seed, feat_out, mu, &passes, (cudaStream_t)stream);
    if (st != CSC_OK) return poison_on_cuda(g, st);
    if (mu_out) memcpy(mu_out, mu, sizeof(mu));
    return CSC_OK;
}

csc_status csc_bracket_target(const double* mu, int32_t m, int32_t k, double* lo_hi_out) {
    clear_error();
    if (!mu || !lo_hi_out || m < 0 || k < 1) {
        set_error("csc_bracket_target: invalid arguments");
        return CSC_E_INVALID;
    }
    lo_hi_out[0] = count_crossing(mu, m, (double)k - 0.5);
    lo_hi_out[1] = count_crossing(mu, m, (double)k + 0.5);
    return CSC_OK;
}

// Paper-literal dichotomy: every threshold costs one filter pass over the probes.
// A caller bracket is checked by the counts at its two ends first.
static csc_status refilter_dichotomy(Graph* g, int k, int m, int n_probes, uint64_t seed, const double* bracket,
                                     csc_lambda_info* out, int* products, cudaStream_t s) {
    auto count = [&](double lam, double* v) -> csc_status {
        *products += m;
        return run_refilter_count(g, lam, m, n_probes, seed, v, s);
    };
    double lo = 0.0, hi = 2.0;
    if (bracket && bracket[0] < bracket[1]) {
        double clo = 0.0, chi = 0.0;
        CSC_TRY(count(bracket[0], &clo));
        CSC_TRY(count(bracket[1], &chi));
        if (round_half_away(clo) <= k && k <= round_half_away(chi)) {
            lo = bracket[0];
            hi = bracket[1];
            out->bracket_used = 1;
        }
    }
    return dichotomy_fn(count, k, lo, hi, out);
}

csc_status csc_estimate_lambda_k_refilter(csc_graph g, int32_t k, int32_t m, int32_t n_probes, uint64_t seed,
                                          const double* bracket, csc_lambda_info* out, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (k < 1 || m < 1 || n_probes < 0 || !out ||
        (bracket && !(bracket[0] >= 0.0 && bracket[0] < bracket[1] && bracket[1] <= 2.0))) {
        set_error("csc_estimate_lambda_k_refilter: invalid arguments (k=%d m=%d n_probes=%d)", k, m, n_probes);
        return CSC_E_INVALID;
    }
    if (n_probes == 0) n_probes = g->N > 1 ? (int)ceil(2.0 * log((double)g->N)) : 1;
    memset(out, 0, sizeof(*out));
    out->n_probes = n_probes;
    out->m = m;
    int products = 0;
    csc_status st = refilter_dichotomy(g, k, m, n_probes, seed, bracket, out, &products, (cudaStream_t)stream);
    out->moment_passes = products;
    return poison_on_cuda(g, st);
}

csc_status csc_estimate_lambda_k_learned(csc_graph g, int32_t k, int32_t m, int32_t n_probes, uint64_t seed,
                                         const float* params, const float* norm, double widen, uint32_t flags,
                                         csc_lambda_info* out, double* bracket_out, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (k < 1 || m < 1 || n_probes < 0 || !out || !params || !norm || !(widen > 0.0)) {
        set_error("csc_estimate_lambda_k_learned: invalid arguments (k=%d m=%d n_probes=%d)", k, m, n_probes);
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float feat[CSC_MLP_IN];
    double mu8[CSC_BRACKET_MOMENTS];
    int passes8 = 0;
    csc_status st = bracket_features(g, k, seed, feat, mu8, &passes8, s);
    if (st != CSC_OK) return poison_on_cuda(g, st);
    // standardise, run the network on the device, undo the target scaling
    float* io = (float*)g->pinned + 64;  // pinned host staging (past the CG flags)
    for (int i = 0; i < CSC_MLP_IN; ++i) {
        const float sd = norm[CSC_MLP_IN + i];
        io[i] = sd > 0.f ? (feat[i] - norm[i]) / sd : 0.f;
    }
    void* dbuf = nullptr;
    CSC_TRY(ws_get(g, WS_MLP, 512, &dbuf));
    float* dx = (float*)dbuf;
    float* dy = dx + 96;
    CSC_CUDA_TRY(cudaMemcpyAsync(dx, io, CSC_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, s));
    st = mlp_forward_device(params, dx, 1, dy, s);
    if (st != CSC_OK) return poison_on_cuda(g, st);
    CSC_CUDA_TRY(cudaMemcpyAsync(io + 96, dy, 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    const float* tm = norm + 2 * CSC_MLP_IN;
    const double centre = (double)io[96] * tm[2] + tm[0];
    const double lnhw = (double)io[97] * tm[3] + tm[1];
    const double hw = widen * exp(std::min(lnhw, 10.0));
    if (bracket_out) {
        bracket_out[0] = std::max(0.0, centre - hw);
        bracket_out[1] = std::min(2.0, centre + hw);
    }
    memset(out, 0, sizeof(*out));
    out->m = m;
    bool inside = false;
    if (flags & CSC_EIGENCOUNT_REFILTER) {
        // paper-literal estimator throughout, started from the prediction
        if (n_probes == 0) n_probes = g->N > 1 ? (int)ceil(2.0 * log((double)g->N)) : 1;
        out->n_probes = n_probes;
        int products = passes8;
        st = guarded_dichotomy(
            [&](double lam, double* v) -> csc_status {
                products += m;
                return run_refilter_count(g, lam, m, n_probes, seed, v, s);
            },
            k, centre, hw, out, &inside);
        out->moment_passes = products;
        out->bracket_used = inside ? 1 : 0;
        return poison_on_cuda(g, st);
    }
    if (m < CSC_BRACKET_MOMENTS) {
        // moments-once on the 8-probe moments; accepted when found inside the prediction
        std::vector<double> c;
        csc_lambda_info trial;
        memset(&trial, 0, sizeof(trial));
        guarded_dichotomy(
            [&](double lam, double* v) -> csc_status {
                *v = eigencount_host(mu8, m, lam, true, c);
                return CSC_OK;
            },
            k, centre, hw, &trial, &inside);
        if (inside && trial.hit) {
            *out = trial;
            out->m = m;
            out->n_probes = CSC_BRACKET_PROBES;
            out->moment_passes = passes8;
            out->bracket_used = 1;
            return CSC_OK;
        }
    }
    // the eigencount rejected the bracket: plain moments-once dichotomy
    if (n_probes == 0) n_probes = g->N > 1 ? (int)ceil(2.0 * log((double)g->N)) : 1;
    std::vector<double> mu(m + 1);
    int passes = 0;
    st = run_moments(g, m + 1, n_probes, seed, CSC_F32, mu.data(), &passes, s);
    if (st != CSC_OK) return poison_on_cuda(g, st);
    out->n_probes = n_probes;
    out->moment_passes = passes8 + passes;
    out->bracket_used = 0;
    dichotomy(mu.data(), m, k, 0.0, 2.0, out);
    return CSC_OK;
}

csc_status csc_sample(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out, void* stream) {
    clear_error();
    if (N < 1 || n < 0 || n > N || (n > 0 && !idx_out) || N >= (int64_t)INT32_MAX) {
        set_error("csc_sample: need 0 <= n <= N < 2^31 and idx_out != NULL");
        return CSC_E_INVALID;
    }
    if (n == 0) return CSC_OK;
    return run_sample(N, n, seed, idx_out, nullptr, (cudaStream_t)stream);
}

csc_status csc_coherence_scores(void* Y, csc_dtype y_type, int64_t N, int32_t d, int32_t ld, int32_t normalize,
                                double* score_out, void* stream) {
    clear_error();
    if (!Y || !score_out || N < 1 || N >= (int64_t)INT32_MAX || d < 1 || ld < d ||
        (y_type != CSC_F32 && y_type != CSC_BF16 && y_type != CSC_F64)) {
        set_error("csc_coherence_scores: invalid arguments (N=%lld d=%d ld=%d y_type=%d)", (long long)N, d, ld,
                  (int)y_type);
        return CSC_E_INVALID;
    }
    int dev = 0, sms = 0;
    CSC_CUDA_TRY(cudaGetDevice(&dev));
    CSC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return run_row_scores(Y, y_type == CSC_F64, N, d, ld, score_out, normalize != 0, sms, (cudaStream_t)stream);
}

csc_status csc_sample_weighted(const double* score, int64_t N, int64_t n, uint64_t seed, int64_t* idx_out,
                               float* w_out, void* stream) {
    clear_error();
    if (!score || N < 1 || N >= (int64_t)INT32_MAX || n < 0 || n >= (int64_t)INT32_MAX || (n > 0 && !idx_out)) {
        set_error("csc_sample_weighted: need 1 <= N < 2^31, 0 <= n < 2^31, score and idx_out != NULL");
        return CSC_E_INVALID;
    }
    if (n == 0) return CSC_OK;
    return run_sample_weighted(score, N, n, seed, idx_out, w_out, nullptr, (cudaStream_t)stream);
}

csc_status csc_gather_rows(const float* X, int64_t N, int32_t ld, const int64_t* idx, int64_t n, int32_t d,
                           float* out, int32_t ld_out, void* stream) {
    clear_error();
    if (!X || !idx || !out || N < 1 || n < 0 || d < 1 || ld < d || ld_out < d) {
        set_error("csc_gather_rows: invalid arguments");
        return CSC_E_INVALID;
    }
    if (n == 0) return CSC_OK;
    return run_gather_rows(X, N, ld, idx, n, d, out, ld_out, (cudaStream_t)stream);
}

csc_status csc_kmeans_reduced(const float* X, int64_t n, int32_t d, int32_t ld, int32_t k, int32_t replicates,
                              int32_t max_iter, uint64_t seed, int32_t* labels_out, double* inertia_out,
                              void* stream) {
    clear_error();
    if (!X || !labels_out || k < 1 || n < k || d < 1 || ld < d || replicates < 1 || max_iter < 0) {
        set_error("csc_kmeans_reduced: invalid arguments (n=%lld d=%d k=%d replicates=%d)", (long long)n, d, k,
                  replicates);
        return CSC_E_INVALID;
    }
    if (k > 1024 || d > 256) {
        set_error("csc_kmeans_reduced: k <= 1024 and d <= 256 in this library");
        return CSC_E_UNSUPPORTED;
    }
    return run_kmeans(X, n, d, ld, k, replicates, max_iter, seed, labels_out, inertia_out, nullptr,
                      (cudaStream_t)stream);
}

csc_status csc_interpolate(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels, int64_t n,
                           int32_t k, int32_t g_power, double gamma, double rel_tol, int32_t max_iter,
                           int32_t* labels_out, float* fuzzy_out, csc_cg_info* info, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!sample_idx || !sample_labels || !labels_out || n < 1 || n > g->N || k < 1 || g_power < 1 ||
        !(gamma > 0.0) || !(rel_tol > 0.0) || max_iter < 1) {
        set_error("csc_interpolate: invalid arguments (n=%lld k=%d g_power=%d gamma=%g rel_tol=%g)", (long long)n, k,
                  g_power, gamma, rel_tol);
        return CSC_E_INVALID;
    }
    csc_status st = run_interpolate(g, sample_idx, sample_labels, n, k, g_power, gamma, rel_tol, max_iter,
                                    labels_out, fuzzy_out, info, (cudaStream_t)stream);
    return poison_on_cuda(g, st);
}

csc_status csc_interpolate_highpass(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels, int64_t n,
                                    int32_t k, double lambda_c, int32_t m, double gamma, double rel_tol,
                                    int32_t max_iter, int32_t* labels_out, float* fuzzy_out, csc_cg_info* info,
                                    void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!sample_idx || !sample_labels || !labels_out || n < 1 || n > g->N || k < 1 || m < 1 ||
        !(lambda_c >= 0.0 && lambda_c <= 2.0) || !(gamma > 0.0) || !(rel_tol > 0.0) || max_iter < 1) {
        set_error("csc_interpolate_highpass: invalid arguments (n=%lld k=%d m=%d lambda_c=%g gamma=%g)", (long long)n,
                  k, m, lambda_c, gamma);
        return CSC_E_INVALID;
    }
    std::vector<double> c(m + 1);
    cheb_coefficients(lambda_c, m, true, c.data());
    csc_status st = run_interpolate(g, sample_idx, sample_labels, n, k, 1, gamma, rel_tol, max_iter, labels_out,
                                    fuzzy_out, info, (cudaStream_t)stream, nullptr, c.data(), m);
    return poison_on_cuda(g, st);
}

csc_status csc_interpolate_weighted(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                    const float* sample_w, int64_t n, int32_t k, int32_t g_power, double gamma,
                                    double rel_tol, int32_t max_iter, int32_t* labels_out, float* fuzzy_out,
                                    csc_cg_info* info, void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!sample_idx || !sample_labels || !sample_w || !labels_out || n < 1 || n >= (int64_t)INT32_MAX || k < 1 ||
        g_power < 1 || !(gamma > 0.0) || !(rel_tol > 0.0) || max_iter < 1) {
        set_error("csc_interpolate_weighted: invalid arguments (n=%lld k=%d g_power=%d gamma=%g rel_tol=%g)",
                  (long long)n, k, g_power, gamma, rel_tol);
        return CSC_E_INVALID;
    }
    csc_status st = run_interpolate(g, sample_idx, sample_labels, n, k, g_power, gamma, rel_tol, max_iter,
                                    labels_out, fuzzy_out, info, (cudaStream_t)stream, nullptr, nullptr, 0, sample_w);
    return poison_on_cuda(g, st);
}

csc_status csc_cluster(csc_graph g, const csc_params* p, int32_t* labels_out, csc_cluster_info* info,
                       void* stream) {
    clear_error();
    CSC_TRY(check_graph(g));
    if (!p || !labels_out || p->k < 1 || p->k > g->N) {
        set_error("csc_cluster: invalid arguments");
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = g->N;
    const int k = p->k;
    const int m = p->m > 0 ? p->m : 50;
    const int d = p->d > 0 ? p->d : (N > 1 ? (int)ceil(4.0 * log((double)N)) : 1);
    const int d_pad = p->d_pad > 0 ? p->d_pad : ((d + 7) / 8) * 8;
    int64_t n = p->n > 0 ? p->n : (k > 1 ? (int64_t)ceil(2.0 * k * log((double)k)) : 1);
    if (n < k) n = k;
    if (n > N) n = N;
    const int g_power = p->g_power > 0 ? p->g_power : 4;
    const double gamma = p->gamma > 0 ? p->gamma : 1e-3;
    const double cg_tol = p->cg_tol > 0 ? p->cg_tol : 1e-6;
    const int cg_max = p->cg_max_iter > 0 ? p->cg_max_iter : 2000;
    const int reps = p->replicates > 0 ? p->replicates : 20;
    const int km_iter = p->km_max_iter > 0 ? p->km_max_iter : 100;
    const csc_dtype storage = p->storage;
    if (d_pad < d || d_pad % 8 || (storage != CSC_F32 && storage != CSC_BF16 && storage != CSC_F64)) {
        set_error("csc_cluster: invalid d_pad or storage");
        return CSC_E_INVALID;
    }
    csc_cluster_info local;
    memset(&local, 0, sizeof(local));
    cudaEvent_t e0, e1, e2, e3, e4, e5;
    CSC_CUDA_TRY(cudaEventCreate(&e0));
    CSC_CUDA_TRY(cudaEventCreate(&e1));
    CSC_CUDA_TRY(cudaEventCreate(&e2));
    CSC_CUDA_TRY(cudaEventCreate(&e3));
    CSC_CUDA_TRY(cudaEventCreate(&e4));
    CSC_CUDA_TRY(cudaEventCreate(&e5));
    csc_status st = CSC_OK;
    auto done = [&](csc_status r) {
        cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
        cudaEventDestroy(e3); cudaEventDestroy(e4); cudaEventDestroy(e5);
        return poison_on_cuda(g, r);
    };
    cudaEventRecord(e0, s);
    double lam = p->lambda_k;
    if (!(lam > 0.0)) {
        st = csc_estimate_lambda_k(g, k, p->m_count > 0 ? p->m_count : m, p->n_probes, p->seed, p->bracket,
                                   &local.lambda, stream);
        if (st != CSC_OK) return done(st);
        lam = local.lambda.lambda;
    } else {
        local.lambda.lambda = lam;
    }
    cudaEventRecord(e1, s);
    // pipeline buffers: Y (N x d_pad, fp32 or fp64), idx (n), Xr (n x d_pad fp32), sample labels (n);
    // variable density adds the scores (N doubles) and the draw weights (n floats)
    const bool vd = (p->flags & CSC_VARDENSITY) != 0;
    const size_t ybytes = (size_t)N * d_pad * (storage == CSC_F64 ? 8 : 4);
    const size_t off_idx = (ybytes + 255) / 256 * 256;
    const size_t off_xr = off_idx + ((size_t)n * 8 + 255) / 256 * 256;
    const size_t off_lab = off_xr + ((size_t)n * d_pad * 4 + 255) / 256 * 256;
    const size_t off_w = off_lab + ((size_t)n * 4 + 255) / 256 * 256;
    const size_t off_sc = off_w + (vd ? ((size_t)n * 4 + 255) / 256 * 256 : 0);
    const size_t total = off_sc + (vd ? (size_t)N * 8 : 0) + 256;
    void* base = nullptr;
    st = ws_get(g, WS_PIPE, total, &base);
    if (st != CSC_OK) return done(st);
    char* b = (char*)base;
    void* Y = b;
    int64_t* idx = (int64_t*)(b + off_idx);
    float* Xr = (float*)(b + off_xr);
    int32_t* slab = (int32_t*)(b + off_lab);
    float* wdraw = vd ? (float*)(b + off_w) : nullptr;
    double* score = vd ? (double*)(b + off_sc) : nullptr;
    std::vector<double> c(m + 1);
    cheb_coefficients(lam, m, true, c.data());
    st = run_filter(g, c.data(), m, d, d_pad, p->seed, storage, nullptr, Y, !vd, s, (p->flags & CSC_CLENSHAW) != 0);
    if (st == CSC_OK && (p->flags & CSC_CHECK_FINITE))
        st = run_check_finite(g, Y, storage == CSC_F64, N, d, d_pad, "the filtered features", s);
    if (st != CSC_OK) return done(st);
    // variable density: scores ||Y_i||^2 of the unnormalised rows, then step 4's normalisation
    if (vd) st = run_row_scores(Y, storage == CSC_F64, N, d, d_pad, score, true, g->num_sms, s);
    if (st != CSC_OK) return done(st);
    cudaEventRecord(e2, s);
    st = vd ? run_sample_weighted(score, N, n, p->seed, idx, wdraw, g, s) : run_sample(N, n, p->seed, idx, g, s);
    if (st != CSC_OK) return done(st);
    if (storage == CSC_F64) {
        // fp64 feature rows are narrowed to fp32 for k-means
        st = run_gather_rows_f64((const double*)Y, N, d_pad, idx, n, d, Xr, d_pad, s);
    } else {
        st = run_gather_rows((const float*)Y, N, d_pad, idx, n, d, Xr, d_pad, s);
    }
    if (st != CSC_OK) return done(st);
    cudaEventRecord(e3, s);
    st = run_kmeans(Xr, n, d, d_pad, k, reps, km_iter, p->seed, slab, &local.inertia, g, s);
    if (st != CSC_OK) return done(st);
    cudaEventRecord(e4, s);
    std::vector<double> hpc;
    const int m_hp = p->m_interp > 0 ? p->m_interp : m;
    if (p->flags & CSC_HIGHPASS) {
        hpc.resize(m_hp + 1);
        cheb_coefficients(lam, m_hp, true, hpc.data());
    }
    st = run_interpolate(g, idx, slab, n, k, g_power, gamma, cg_tol, cg_max, labels_out, nullptr, &local.cg, s,
                         nullptr, hpc.empty() ? nullptr : hpc.data(), m_hp, wdraw);
    if (st != CSC_OK && st != CSC_E_NOT_CONVERGED) return done(st);
    cudaEventRecord(e5, s);
    cudaError_t ce = cudaEventSynchronize(e5);
    if (ce != cudaSuccess) {
        set_error("csc_cluster: %s", cudaGetErrorString(ce));
        return done(CSC_E_CUDA);
    }
    cudaEventElapsedTime(&local.ms_lambda, e0, e1);
    cudaEventElapsedTime(&local.ms_filter, e1, e2);
    cudaEventElapsedTime(&local.ms_sample, e2, e3);
    cudaEventElapsedTime(&local.ms_kmeans, e3, e4);
    cudaEventElapsedTime(&local.ms_interp, e4, e5);
    cudaEventElapsedTime(&local.ms_total, e0, e5);
    if (info) *info = local;
    return done(st);
}

}  // extern "C"
