// common.cuh -- internal declarations shared by the translation units of libcsc.
//
// Graph handle layout, error plumbing, workspace slots and the launchers each
// .cu file exports to the C-ABI layer (api.cu).  Nothing here is part of the
// public ABI (include/csc.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/csc.h"

namespace csc {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define CSC_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e__ = (expr);                                                       \
        if (e__ != cudaSuccess) {                                                       \
            ::csc::set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, \
                             __LINE__);                                                 \
            return CSC_E_CUDA;                                                          \
        }                                                                               \
    } while (0)

#define CSC_TRY(expr)                      \
    do {                                   \
        csc_status s__ = (expr);           \
        if (s__ != CSC_OK) return s__;     \
    } while (0)

#define CSC_LAUNCH_CHECK()                                                                  \
    do {                                                                                    \
        cudaError_t e__ = cudaGetLastError();                                               \
        if (e__ != cudaSuccess) {                                                           \
            ::csc::set_error("kernel launch: %s (%s:%d)", cudaGetErrorString(e__), __FILE__, \
                             __LINE__);                                                     \
            return CSC_E_CUDA;                                                              \
        }                                                                                   \
    } while (0)

// ------------------------------------------------------- launch accounting
// Every kernel launch goes through CSC_KLAUNCH(class name, algorithmic bytes,
// stream, kernel<<<...>>>(...)): it is counted, optionally bracketed by
// events on its stream (profile.cu), and checked.
extern bool g_prof_enabled;
int prof_begin(const char* name, double bytes, cudaStream_t s);
void prof_end(int slot, cudaStream_t s);
void count_launch();
void count_launches(int64_t n);

#define CSC_KLAUNCH(NAME, BYTES, STREAM, ...)                                                \
    do {                                                                                    \
        ::csc::count_launch();                                                              \
        const int slot__ = ::csc::g_prof_enabled ? ::csc::prof_begin(NAME, (double)(BYTES), STREAM) : -1; \
        __VA_ARGS__;                                                                        \
        if (slot__ >= 0) ::csc::prof_end(slot__, STREAM);                                   \
        CSC_LAUNCH_CHECK();                                                                 \
    } while (0)

// Rows with more edges than this ("heavy" rows: the hubs of power-law graphs) are
// not swept by one lane group of the row-range kernels; a second kernel gives each
// of them a CTA whose groups split its edge list.
constexpr int kHeavyRow = 256;

// ------------------------------------------------------------- workspace
// Scratch slots owned by a graph handle; each grows on demand (cudaMalloc)
// and lives until the handle is destroyed.
enum WsSlot {
    WS_XA = 0,      // signal block ping (X_j / X_{j-1})
    WS_XB,          // signal block pong
    WS_YACC,        // fp64 accumulator (F64 storage)
    WS_PARTIAL,     // per-block fp64 partial sums
    WS_MOMENTS,     // moment sums
    WS_CG,          // CG vectors
    WS_SAMPLE,      // sampling scratch
    WS_KMEANS,      // k-means scratch
    WS_MISC,
    WS_PIPE,        // pipeline buffers of csc_cluster
    WS_MLP,         // predictor input / output of the learned bracket
    WS_REFILTER,    // filtered probes and partials of the paper-literal eigencount
    WS_COEF,        // per-graph filter coefficients of a batch
    WS_COEF1,       // filter coefficients read by a captured CUDA graph
    WS_XR,          // s R, read by every order of the Clenshaw form
    WS_CHECK,       // flag word of the non-finite scan (CSC_CHECK_FINITE)
    WS_COUNT
};

struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Launch shape of a row-sweep SpMM kernel: G lanes per row, NT 16-byte vectors
// per lane (a column tile of G*NT vectors), `threads` per CTA, P row ranges
// (one CTA each per tile) and `tiles` column tiles.
struct LaunchCfg {
    int G = 0, NT = 0, threads = 0, P = 0, tiles = 1;
    int staged = 1;  // row-range kernels: indices staged in shared memory (0: read from global)
    // Clenshaw and CG row-range kernels, NT = 1 and 256 threads only: the lean form, with at
    // most 4 neighbour rows in flight per lane and a launch bound of 5 CTAs per SM (48
    // registers instead of 60), trading loads in flight per warp for resident warps
    int lean = 0;
};

struct Graph {
    int64_t N = 0;        // nodes (packed total for batched graphs)
    int64_t nnz = 0;      // stored entries after self-loop removal
    int32_t n_graphs = 1;
    int device = 0;
    int num_sms = 148;
    int64_t l2_bytes = 0;
    int32_t* row_ptr = nullptr;  // device int32[N+1], internal node order
    int32_t* col_idx = nullptr;  // device int32[nnz]
    float* dinv = nullptr;       // device float[N]: D^-1/2 (0 for isolated nodes)
    double* dinv64 = nullptr;    // device double[N]
    // Row factors of the pre-scaled form Z = s X with s = D^-1/2 (1 for isolated
    // nodes): invdeg = 1/deg (0 if isolated), sqdeg = 1/s = sqrt(deg) (1 if isolated)
    float* invdeg = nullptr;
    float* sqdeg = nullptr;
    double* invdeg64 = nullptr;
    double* sqdeg64 = nullptr;
    int32_t* deg = nullptr;      // device int32[N]
    int32_t* perm = nullptr;     // device int32[N]: internal row -> original id (nullptr: identity)
    int32_t* iperm = nullptr;    // device int32[N]: original id -> internal row
    // batched handles
    std::vector<int64_t> offsets;    // host, n_graphs+1 (packed node offsets)
    int64_t* d_offsets = nullptr;    // device copy
    int32_t* graph_of_row = nullptr; // device int32[N]
    Buffer ws[WS_COUNT];
    std::vector<int32_t> h_row_ptr;               // host copy of row_ptr (internal order)
    std::vector<int64_t> h_light;                 // prefix sums of the edges of non-heavy rows
    int32_t deg_quant[6] = {0, 0, 0, 0, 0, 0};    // degrees at p = 0, .1, .25, .5, .75, 1 (floor(p (N-1)))
    int32_t* heavy = nullptr;                     // device int32[n_heavy]: heavy rows
    int n_heavy = 0;
    // compact light CSR (device.cuh: stage_csr): lrp int32[N+1] = light edges before each
    // row, bit 31 of lrp[i+1] set for a heavy row i; lci = the light rows' indices.  Without
    // heavy rows they alias row_ptr / col_idx (light_owned = false).
    int32_t* lrp = nullptr;
    int32_t* lci = nullptr;
    bool light_owned = false;
    std::map<int, int32_t*> parts;                // P -> device int32[P+1] row-range bounds
    std::map<int, std::vector<int32_t>> h_parts;  // host copies of the bounds
    std::map<int, int> part_smem;                 // P -> shared-memory bytes of the largest staged range
    std::map<int, int32_t*> part_gblk;            // P -> device int32[G+1]: first range of each graph
    int32_t* d_hvy_start = nullptr;               // device int32[G+1]: first heavy row of each graph
    // captured CUDA graphs of fixed launch sequences (key -> executable, kernel launches)
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    // side stream and events of fork_join (heavy-row launches beside the row ranges)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::map<std::string, std::pair<cudaGraphExec_t, int64_t>> graphs;
    std::map<uint64_t, LaunchCfg> tuned;          // (kernel kind, dtype, columns) -> shape
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double* pinned = nullptr;  // small pinned host staging (4096 doubles)
    bool poisoned = false;
};

csc_status ws_get(Graph* g, WsSlot slot, size_t bytes, void** out);

// Tuned launch shapes shared by all handles of the process, keyed by the tuning key,
// device, N and nnz (graphs of the same size reuse a shape without re-tuning).
bool tune_cache_get(const Graph* g, uint64_t key, LaunchCfg* out);
void tune_cache_put(const Graph* g, uint64_t key, const LaunchCfg& cfg);

// Launch the sequence `record(stream)` issues, as a CUDA graph captured once per
// key on the handle's capture stream and replayed on s.  The recorded launches
// must not depend on anything but the key.  *launches: kernel launches per replay.
int64_t launch_count();
template <typename Rec>
csc_status replay_graph(Graph* g, const std::string& key, cudaStream_t s, int64_t* launches, Rec&& record) {
    auto it = g->graphs.find(key);
    if (it == g->graphs.end()) {
        if (!g->cap_stream) CSC_CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        if (g->graphs.size() >= 64) {  // bound the cache
            for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second.first);
            g->graphs.clear();
        }
        const int64_t before = launch_count();
        // relaxed: one-time host set-up inside `record` (a partition upload) runs eagerly
        CSC_CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
        const csc_status st = record(g->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        const int64_t n = launch_count() - before;
        count_launches(-n);  // captured, not run
        if (st != CSC_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (st == CSC_OK) set_error("CUDA graph capture: %s", cudaGetErrorString(e));
            return st != CSC_OK ? st : CSC_E_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            set_error("CUDA graph instantiation: %s", cudaGetErrorString(ei));
            return CSC_E_CUDA;
        }
        it = g->graphs.emplace(key, std::make_pair(exec, n)).first;
    }
    CSC_CUDA_TRY(cudaGraphLaunch(it->second.first, s));
    count_launches(it->second.second);
    *launches = it->second.second;
    return CSC_OK;
}

// Runs heavy(stream) on the handle's side stream alongside light(s) -- the heavy-row
// launch and the row-range launch of one product write disjoint rows -- and makes s wait
// for both; inside a capture this records two parallel branches.  With per-launch timing
// on, or without heavy rows, the launches run one after the other on s.
template <typename H, typename L>
csc_status fork_join(Graph* g, cudaStream_t s, bool has_heavy, H&& heavy, L&& light) {
    if (!has_heavy) return light(s);
    if (g_prof_enabled) {
        CSC_TRY(heavy(s));
        return light(s);
    }
    if (!g->side_stream) {
        CSC_CUDA_TRY(cudaStreamCreateWithFlags(&g->side_stream, cudaStreamNonBlocking));
        CSC_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
        CSC_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    }
    CSC_CUDA_TRY(cudaEventRecord(g->ev_fork, s));
    CSC_CUDA_TRY(cudaStreamWaitEvent(g->side_stream, g->ev_fork, 0));
    const csc_status hs = heavy(g->side_stream);
    CSC_CUDA_TRY(cudaEventRecord(g->ev_join, g->side_stream));
    const csc_status ls = light(s);
    CSC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_join, 0));
    return hs != CSC_OK ? hs : ls;
}

// P contiguous row ranges of about equal cost (edges + 2 per row); cached per P.
csc_status get_partition(Graph* g, int P, const int32_t** out);
// Shared-memory bytes a CTA needs to stage the CSR slice of the largest range of
// partition P (get_partition must have built it).
int staged_smem(const Graph* g, int P);
// Most shared memory a staged CSR slice may take (within the 48 KB a CTA gets without
// an opt-in, beside the kernels' own reduction arrays of up to 16 KB).
constexpr int kStagedSmemMax = 30 * 1024;
csc_status check_staged_smem(int bytes);
// The smallest row-range count >= P (doubling, at most max_p) whose staged slices fit
// kStagedSmemMax; builds the partitions it tries.
csc_status fit_staged_partition(Graph* g, int P, int64_t max_p, int* out);
// Per-graph segments of partition P: first range of each graph (device int32[G+1]; a
// batched handle's ranges never straddle graphs) and first heavy row of each graph.
csc_status get_segments(Graph* g, int P, const int32_t** gblk, const int32_t** ghvy);

// Start rows of the W-row windows (one per row range of partition P) that cover
// the most neighbour indices of each range; cached per (P, W).

// Device helpers exported by the kernel translation units -----------------

// spmm.cu: degrees and D^-1/2 from the CSR pattern (K4)
csc_status launch_degrees(Graph* g, cudaStream_t s);

// spmm.cu: the Jackson-Chebyshev filter (K3 + K1 + K5)
// h~(L) = sum_j c_j T_j(L - I) on an fp32 block in internal row order (Clenshaw form).
struct PolyOp {
    LaunchCfg cfg;
    const float* coef = nullptr;
    const int32_t* gid = nullptr;  // batched handle: graph of each row (coef holds one row of m + 1 per graph)
    const int32_t* gcols = nullptr;  // with gid: columns each graph carries (multiple of 4); NULL: all
    int m = 0, ld = 0;
    float *b0 = nullptr, *b1 = nullptr, *rs = nullptr;
};
// c: host double[n_coef x (m + 1)]; n_coef = 1, or the handle's graph count (graph i's
// polynomial is applied to graph i's rows).
csc_status poly_prepare(Graph* g, const double* c, int m, int ld, PolyOp* op, cudaStream_t s, int n_coef = 1);
csc_status poly_apply(Graph* g, const PolyOp& op, const float* X, float* Y, cudaStream_t s);

// Batched handle: c_graphs is host double[n_graphs x (m + 1)], graph i's coefficients.
csc_status run_filter_batched(Graph* g, const double* c_graphs, int m, int d, int d_pad, uint64_t seed,
                              csc_dtype storage, const float* R_in, void* Y_out, bool normalize, cudaStream_t s,
                              bool clenshaw = false);
csc_status run_filter(Graph* g, const double* coeffs, int m, int d, int d_pad, uint64_t seed,
                      csc_dtype storage, const float* R_in, void* Y_out, bool normalize,
                      cudaStream_t s, bool clenshaw = false);

// spmm.cu: eigencount moments (K2); mu_host receives n_moments values
// per_graph: one moment vector per graph of a batched handle (mu_host: n_graphs x n_moments)
csc_status run_moments(Graph* g, int n_moments, int n_probes, uint64_t seed, csc_dtype storage,
                       double* mu_host, int* passes, cudaStream_t s, bool per_graph = false);

// spmm.cu: paper-literal eigencount at one cut-off (m sparse products)
csc_status run_refilter_count(Graph* g, double lambda, int m, int n_probes, uint64_t seed, double* count,
                              cudaStream_t s);

// mlp.cu: Y = network(X) for B rows (device pointers)
csc_status mlp_forward_device(const float* params, const float* X, int B, float* Y, cudaStream_t s);

// sample.cu (K6)
csc_status run_sample_weighted(const double* score, int64_t N, int64_t n, uint64_t seed, int64_t* idx_out,
                               float* w_out, Graph* scratch_owner, cudaStream_t s);
csc_status run_row_scores(void* Y, bool y_f64, int64_t N, int d, int ld, double* score, bool normalize,
                          int num_sms, cudaStream_t s);
// spmm.cu: CSC_E_NUMERIC if any of the first `cols` entries of the `rows` rows (stride ld)
// of X (fp32, or fp64 when x_f64) is NaN or infinite; synchronizes s.  `what` names X.
csc_status run_check_finite(Graph* g, const void* X, bool x_f64, int64_t rows, int cols, int ld, const char* what,
                            cudaStream_t s);
csc_status run_sample(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out, Graph* scratch_owner,
                      cudaStream_t s);
csc_status run_gather_rows(const float* X, int64_t N, int ld, const int64_t* idx, int64_t n, int d,
                           float* out, int ld_out, cudaStream_t s);
csc_status run_gather_rows_f64(const double* X, int64_t N, int ld, const int64_t* idx, int64_t n, int d,
                               float* out, int ld_out, cudaStream_t s);

// kmeans.cu (K7)
// One k-means problem of run_kmeans_multi: n points at X (rows of stride ld), k
// clusters, the replicate seed, and the device output labels[n].
struct KmTask {
    const float* X = nullptr;
    int n = 0, k = 0;
    uint64_t seed = 0;
    int32_t* labels_out = nullptr;
};
// Several k-means problems in one launch (grid y = problem); inertia_out: NULL or
// host double[tasks.size()].  Synchronizes s.
csc_status run_kmeans_multi(const std::vector<KmTask>& tasks, int d, int ld, int reps, int max_iter,
                            double* inertia_out, Graph* owner, cudaStream_t s);
csc_status run_kmeans(const float* X, int64_t n, int d, int ld, int k, int replicates, int max_iter,
                      uint64_t seed, int32_t* labels_out, double* inertia_out, Graph* scratch_owner,
                      cudaStream_t s);

// cg.cu (K8 + K9).  k_graphs: NULL, or (batched handle) host int32[n_graphs], each
// graph's k (k = their maximum): one set of systems per graph.  hp_coef: NULL for
// g(L) = L^g_power, or host double[hp_m + 1], the coefficients of h~ for g = 1 - h~.
// With k_graphs, hp_coef holds one row of hp_m + 1 coefficients per graph.
// sample_w: NULL for Eq. 5's 0/1 mask, or device float[n] draw weights (weighted decoder).
csc_status run_interpolate(Graph* g, const int64_t* sample_idx, const int32_t* sample_labels,
                           int64_t n, int k, int g_power, double gamma, double rel_tol, int max_iter,
                           int32_t* labels_out, float* fuzzy_out, csc_cg_info* info, cudaStream_t s,
                           const int32_t* k_graphs = nullptr, const double* hp_coef = nullptr, int hp_m = 0,
                           const float* sample_w = nullptr);

// host math (api.cu)
void cheb_coefficients(double lambda_c, int m, bool jackson, double* c);
// The Sec. 4.3 dichotomy on [0, 2] from degree-m moments (fills lambda, count, iters, hit).
void estimate_from_moments(const double* mu, int m, int k, csc_lambda_info* out);

// Philox4x32-10 and SplitMix64 stream identifiers (the key's high word is
// xor-ed with these so that signals, probes and k-means draws are disjoint).
constexpr uint32_t STREAM_SIGNALS = 0x5349474Eu;
constexpr uint32_t STREAM_PROBES = 0x50524F42u;
constexpr uint32_t STREAM_KMEANS = 0x4B4D4541u;

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace csc

// The opaque handle of the C ABI is the internal graph record.
struct csc_graph_s : public csc::Graph {};

