// kmeans.cu -- k-means on the reduced feature set (Alg. 2 step 6).
//
// One thread-block cluster per replicate (the paper runs 20 replicates, Sec. 5):
// the C CTAs of a cluster split the n points into contiguous slices; every CTA
// keeps the whole k x d centre table in its shared memory, and CTA r owns the
// clusters j with j % C == r.  Centre sums are exact 64-bit fixed-point
// integers added with distributed-shared-memory atomics into the owner's
// shared memory, so they do not depend on the order of the additions; owners
// then write the new centres into every CTA of the cluster.
//
// Seeding is k-means++ with uniforms from Philox4x32-10 (key = (seed, "k-means"),
// counter = (replicate, draw)): the first centre is point floor(u n), centre
// t >= 1 the first point whose running sum of squared distances to the chosen
// centres reaches u * total.  Lloyd iterations assign each point to its
// nearest centre (ties to the lower index) and move each centre to the mean of
// its points; an empty cluster (in increasing index) takes the point farthest
// from its own centre, which moves to it.  The best replicate by inertia (ties
// to the first) wins.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "device.cuh"

namespace cg = cooperative_groups;

namespace csc {

constexpr int kKmThreads = 256;
constexpr int kKmLanesPerPoint = 8;  // lanes sharing one point in the assignment

__device__ __forceinline__ float sqdist(const float* __restrict__ x, const float* __restrict__ c, int d) {
    float s = 0.f;
    for (int q = 0; q < d; ++q) {
        const float t = x[q] - c[q];
        s = fmaf(t, t, s);
    }
    return s;
}

__device__ __forceinline__ double km_uniform(uint64_t seed, uint32_t rep, uint32_t t) {
    const Philox4 r = philox4x32_10(rep, 0u, t, 0u, (uint32_t)seed, (uint32_t)(seed >> 32) ^ STREAM_KMEANS);
    return (double)philox_uniform(r.x[0]);
}

// Per-CTA scalars; the other CTAs of the cluster read them through DSMEM.
struct KmShared {
    double part;                          // this CTA's share of a cluster-wide sum
    double scan_w[kKmThreads / 32];
    int pick;                             // chosen point (seeding / empty-cluster refill)
    int changed;
    float best_v;                         // this CTA's farthest point / local maximum
    int best_i;
    double scale;
    float shv[kKmThreads / 32];
    int shi[kKmThreads / 32];
};

// Dynamic shared memory of one CTA.
struct KmLayout {
    size_t cen, sums, counts, empty, d2, lab, nlab, xs, total;
    static __host__ __device__ size_t al(size_t x) { return (x + 15) / 16 * 16; }
    // stage_x: the CTA's points are copied into shared memory (rows of d floats)
    __host__ __device__ KmLayout(int k, int d, int own_k, int n_loc, bool stage_x) {
        cen = 0;
        sums = al(cen + (size_t)k * d * 4);
        counts = al(sums + (size_t)own_k * d * 8);
        empty = al(counts + (size_t)own_k * 4);
        d2 = al(empty + (size_t)k * 4);
        lab = al(d2 + (size_t)n_loc * 8);
        nlab = al(lab + (size_t)n_loc * 4);
        xs = al(nlab + (size_t)n_loc * 4);
        total = al(xs + (stage_x ? (size_t)n_loc * d * 4 : 0));
    }
};

// Block-wide exclusive scan of one double per thread (fixed order); the block
// total goes to *tot.
__device__ double km_block_scan(double v, double* warp_tot, double* tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int i = 0; i < kKmThreads / 32; ++i) {
            const double t = warp_tot[i];
            warp_tot[i] = acc;
            acc += t;
        }
        *tot = acc;
    }
    __syncthreads();
    return warp_tot[w] + x - v;
}

// One k-means problem of a launch (blockIdx.y): points X[0..n) (rows of stride ld),
// k clusters, its seed, and where its replicates' labels (reps x n) and inertias go.
struct KmProblem {
    const float* X;
    int n, k;
    uint64_t seed;
    int32_t* labels_all;
    double* inertia_all;
};

__global__ void __launch_bounds__(kKmThreads)
kmeans_cluster_kernel(const KmProblem* __restrict__ probs, int d, int ld, int max_iter, int stage_x) {
    const KmProblem pr = probs[blockIdx.y];
    const float* __restrict__ X = pr.X;
    const int n = pr.n, k = pr.k;
    const uint64_t seed = pr.seed;
    int32_t* __restrict__ labels_all = pr.labels_all;
    double* __restrict__ inertia_all = pr.inertia_all;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ KmShared S;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int rep = blockIdx.x / C;
    const int T = threadIdx.x;
    const int own_k = (k + C - 1) / C;
    const int n_loc = (n + C - 1) / C;
    const KmLayout L(k, d, own_k, n_loc, stage_x != 0);
    float* Cen = (float*)(smem + L.cen);
    unsigned long long* sums = (unsigned long long*)(smem + L.sums);
    int* counts = (int*)(smem + L.counts);
    int* empty = (int*)(smem + L.empty);
    double* d2 = (double*)(smem + L.d2);
    int* lab = (int*)(smem + L.lab);
    int* nlab = (int*)(smem + L.nlab);
    const int i0 = rank * n_loc;
    const int cnt = max(0, min(n, i0 + n_loc) - i0);  // this CTA's points: i0 .. i0+cnt-1
    // the CTA's points, read by every seeding draw and Lloyd step: staged into shared
    // memory (rows of d floats) when they fit, else read in place (rows of ld)
    const float* Xl = X + (int64_t)i0 * ld;
    int ldl = ld;
    if (stage_x) {
        float* xs = (float*)(smem + L.xs);
        for (int64_t t = T; t < (int64_t)cnt * d; t += kKmThreads) xs[t] = Xl[(t / d) * ld + t % d];
        Xl = xs;
        ldl = d;
        __syncthreads();
    }

    // fixed-point scale for exact centre sums: n * max|x| * scale < 2^62 (cluster-wide max)
    {
        float mx = 0.f;
        for (int64_t t = T; t < (int64_t)cnt * d; t += kKmThreads)
            mx = fmaxf(mx, fabsf(X[(int64_t)(i0 + t / d) * ld + t % d]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((T & 31) == 0) S.shv[T >> 5] = mx;
        __syncthreads();
        if (T == 0) {
            float m = 0.f;
            for (int i = 0; i < kKmThreads / 32; ++i) m = fmaxf(m, S.shv[i]);
            S.best_v = m;
        }
        cluster.sync();
        if (T == 0) {
            float m = 0.f;
            for (int r = 0; r < C; ++r) m = fmaxf(m, cluster.map_shared_rank(&S, r)->best_v);
            const int e = 61 - (int)ceil(log2((double)n + 1.0)) - (m > 0.f ? (int)ceil(log2((double)m)) : 0);
            S.scale = ldexp(1.0, e > 1000 ? 1000 : e);
        }
        cluster.sync();  // the maxima are read before best_v is reused
    }
    const double scale = S.scale;

    // ------------------------------------------------------- k-means++ seeding
    {
        const double u0 = km_uniform(seed, (uint32_t)rep, 0u);
        const int p0 = min((int)(u0 * (double)n), n - 1);
        for (int q = T; q < d; q += kKmThreads) Cen[q] = X[(int64_t)p0 * ld + q];
        __syncthreads();
        for (int i = T; i < cnt; i += kKmThreads) d2[i] = (double)sqdist(Xl + (int64_t)i * ldl, Cen, d);
        __syncthreads();
    }
    const int chunk = (cnt + kKmThreads - 1) / kKmThreads;
    for (int t = 1; t < k; ++t) {
        // per-thread contiguous chunks of this CTA's points; fixed-order scan of the chunk sums
        const int a0 = min(cnt, T * chunk), a1 = min(cnt, a0 + chunk);
        double mine = 0.0;
        for (int i = a0; i < a1; ++i) mine += d2[i];
        const double excl_t = km_block_scan(mine, S.scan_w, &S.part);
        if (T == 0) S.pick = n - 1;  // stays if rounding leaves the target past the end
        cluster.sync();
        // cluster-wide total and this CTA's offset, in rank order (identical in every CTA)
        double total = 0.0, my_off = 0.0;
        for (int r = 0; r < C; ++r) {
            const double pr = cluster.map_shared_rank(&S, r)->part;
            if (r == rank) my_off = total;
            total += pr;
        }
        const double u = km_uniform(seed, (uint32_t)rep, (uint32_t)t);
        if (total <= 0.0) {
            if (rank == 0 && T == 0) {
                const int p = min((int)(u * (double)n), n - 1);
                for (int r = 0; r < C; ++r) cluster.map_shared_rank(&S, r)->pick = p;
            }
        } else {
            const double target = u * total;
            const double lo = my_off + excl_t, hi = my_off + excl_t + mine;
            if (a0 < a1 && lo < target && target <= hi) {
                double acc = lo;
                int p = a1 - 1;
                for (int i = a0; i < a1; ++i) {
                    acc += d2[i];
                    if (acc >= target) {
                        p = i;
                        break;
                    }
                }
                for (int r = 0; r < C; ++r) cluster.map_shared_rank(&S, r)->pick = i0 + p;
            }
        }
        cluster.sync();
        const int p = S.pick;
        for (int q = T; q < d; q += kKmThreads) Cen[t * d + q] = X[(int64_t)p * ld + q];
        __syncthreads();
        for (int i = T; i < cnt; i += kKmThreads) {
            const double dd = (double)sqdist(Xl + (int64_t)i * ldl, Cen + t * d, d);
            if (dd < d2[i]) d2[i] = dd;
        }
        __syncthreads();
    }

    // ----------------------------------------------------------- Lloyd iterations
    // Assignment: kKmLanesPerPoint lanes per point split the centres, then a
    // min-reduction within the lane group (ties to the lower centre index).  The
    // loop count is uniform across the block so every shuffle has all lanes.
    constexpr int kGroups = kKmThreads / kKmLanesPerPoint;
    auto assign = [&](int* out, bool count_changes) {
        int changed = 0;
        const int sub = T % kKmLanesPerPoint;
        const int rounds = (cnt + kGroups - 1) / kGroups;
        for (int it = 0; it < rounds; ++it) {
            const int pt = it * kGroups + T / kKmLanesPerPoint;
            const bool valid = pt < cnt;
            float best = INFINITY;
            int bj = 0x7fffffff;
            if (valid) {
                const float* x = Xl + (int64_t)pt * ldl;
                for (int j = sub; j < k; j += kKmLanesPerPoint) {
                    const float dj = sqdist(x, Cen + j * d, d);
                    if (dj < best) {
                        best = dj;
                        bj = j;
                    }
                }
            }
#pragma unroll
            for (int o = kKmLanesPerPoint / 2; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, best, o, kKmLanesPerPoint);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o, kKmLanesPerPoint);
                if (ov < best || (ov == best && oj < bj)) {
                    best = ov;
                    bj = oj;
                }
            }
            if (valid && sub == 0) {
                if (count_changes && bj != lab[pt]) changed = 1;
                out[pt] = bj;
            }
        }
        return changed;
    };
    assign(lab, false);
    __syncthreads();
    for (int it = 1; it <= max_iter; ++it) {
        for (int q = T; q < own_k * d; q += kKmThreads) sums[q] = 0ull;
        for (int j = T; j < own_k; j += kKmThreads) counts[j] = 0;
        cluster.sync();  // every owner has zeroed before anyone adds
        for (int i = T; i < cnt; i += kKmThreads) {
            const int j = lab[i];
            const int owner = j % C, slot = j / C;
            unsigned long long* rs = cluster.map_shared_rank(sums, owner) + (size_t)slot * d;
            atomicAdd(cluster.map_shared_rank(counts, owner) + slot, 1);
            const float* x = Xl + (int64_t)i * ldl;
            for (int q = 0; q < d; ++q) {
                const long long v = llrint((double)x[q] * scale);
                atomicAdd(rs + q, (unsigned long long)v);
            }
        }
        cluster.sync();
        // owners: new centres of their clusters into every CTA; empty flags likewise
        for (int q = T; q < own_k * d; q += kKmThreads) {
            const int slot = q / d, j = slot * C + rank;
            if (j >= k) continue;
            const int c = counts[slot];
            if (c > 0) {
                const float v = (float)((double)(long long)sums[q] / scale / (double)c);
                for (int r = 0; r < C; ++r) cluster.map_shared_rank(Cen, r)[j * d + q % d] = v;
            }
        }
        for (int slot = T; slot < own_k; slot += kKmThreads) {
            const int j = slot * C + rank;
            if (j < k) {
                const int e = counts[slot] == 0 ? 1 : 0;
                for (int r = 0; r < C; ++r) cluster.map_shared_rank(empty, r)[j] = e;
            }
        }
        cluster.sync();
        // empty clusters in increasing index: the point farthest from its own centre moves there
        for (int j = 0; j < k; ++j) {
            if (!empty[j]) continue;  // the same list in every CTA
            float bv = -1.f;
            int bi = 0x7fffffff;
            for (int i = T; i < cnt; i += kKmThreads) {
                const float v = sqdist(Xl + (int64_t)i * ldl, Cen + lab[i] * d, d);
                if (v > bv) {
                    bv = v;
                    bi = i0 + i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if ((T & 31) == 0) {
                S.shv[T >> 5] = bv;
                S.shi[T >> 5] = bi;
            }
            __syncthreads();
            if (T == 0) {
                float v = S.shv[0];
                int ix = S.shi[0];
                for (int w = 1; w < kKmThreads / 32; ++w)
                    if (S.shv[w] > v || (S.shv[w] == v && S.shi[w] < ix)) {
                        v = S.shv[w];
                        ix = S.shi[w];
                    }
                S.best_v = v;
                S.best_i = ix;
            }
            cluster.sync();
            if (T == 0) {
                float v = -2.f;
                int ix = 0x7fffffff;
                for (int r = 0; r < C; ++r) {
                    const KmShared* o = cluster.map_shared_rank(&S, r);
                    if (o->best_v > v || (o->best_v == v && o->best_i < ix)) {
                        v = o->best_v;
                        ix = o->best_i;
                    }
                }
                S.pick = ix;
            }
            __syncthreads();
            const int p = S.pick;
            for (int q = T; q < d; q += kKmThreads) Cen[j * d + q] = X[(int64_t)p * ld + q];
            if (T == 0 && p >= i0 && p < i0 + cnt) lab[p - i0] = j;  // the donor keeps its centre
            cluster.sync();  // candidates read everywhere before the next empty cluster
        }
        if (T == 0) S.changed = 0;
        __syncthreads();
        if (assign(nlab, true)) S.changed = 1;
        __syncthreads();
        for (int i = T; i < cnt; i += kKmThreads) lab[i] = nlab[i];
        cluster.sync();
        int any = 0;
        for (int r = 0; r < C; ++r) any |= cluster.map_shared_rank(&S, r)->changed;
        cluster.sync();  // flags read before the next iteration resets them
        if (!any) break;
    }
    // inertia: fp32 distances, fp64 sums in a fixed order; labels
    double in = 0.0;
    for (int i = T; i < cnt; i += kKmThreads) in += (double)sqdist(Xl + (int64_t)i * ldl, Cen + lab[i] * d, d);
    in = warp_sum(in);
    if ((T & 31) == 0) S.scan_w[T >> 5] = in;
    __syncthreads();
    if (T == 0) {
        double t = 0.0;
        for (int w = 0; w < kKmThreads / 32; ++w) t += S.scan_w[w];
        S.part = t;
    }
    for (int i = T; i < cnt; i += kKmThreads) labels_all[(int64_t)rep * n + i0 + i] = lab[i];
    cluster.sync();
    if (rank == 0 && T == 0) {
        double t = 0.0;
        for (int r = 0; r < C; ++r) t += cluster.map_shared_rank(&S, r)->part;
        inertia_all[rep] = t;
    }
    cluster.sync();  // every CTA's shared memory stays alive until rank 0 has read it
}

// Best replicate of problem blockIdx.y (ties to the first): labels to out[y], inertia to inertia_out[y].
__global__ void kmeans_pick_kernel(const KmProblem* __restrict__ probs, int reps, int32_t* const* __restrict__ out,
                                   double* __restrict__ inertia_out_all) {
    const KmProblem pr = probs[blockIdx.y];
    const int32_t* __restrict__ labels_all = pr.labels_all;
    const double* __restrict__ inertia_all = pr.inertia_all;
    const int n = pr.n;
    int32_t* __restrict__ labels_out = out[blockIdx.y];
    double* __restrict__ inertia_out = inertia_out_all + blockIdx.y;
    __shared__ int best;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int r = 1; r < reps; ++r)
            if (inertia_all[r] < inertia_all[b]) b = r;
        best = b;
        *inertia_out = inertia_all[b];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) labels_out[i] = labels_all[(int64_t)best * n + i];
}

csc_status run_kmeans_multi(const std::vector<KmTask>& tasks, int d, int ld, int reps, int max_iter,
                            double* inertia_out, Graph* owner, cudaStream_t s) {
    const int NP = (int)tasks.size();
    if (NP == 0) return CSC_OK;
    int dev = 0, sms = 148;
    CSC_CUDA_TRY(cudaGetDevice(&dev));
    CSC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int n_max = 0, n_min = 1 << 30, k_max = 0;
    int64_t lab_total = 0;
    for (const KmTask& t : tasks) {
        n_max = std::max(n_max, t.n);
        n_min = std::min(n_min, t.n);
        k_max = std::max(k_max, t.k);
        lab_total += (int64_t)reps * t.n;
    }
    // cluster size: spread the replicates of all problems over the SMs, at most 8 CTAs
    // (the portable cluster size), and slices of at least 16 points
    int C = sms / (reps * NP);
    C = C < 1 ? 1 : (C > 8 ? 8 : C);
    while (C > 1 && (n_min + C - 1) / C < 16) --C;
    size_t smem = 0;
    for (;; --C) {
        const KmLayout L(k_max, d, (k_max + C - 1) / C, (n_max + C - 1) / C, false);
        smem = L.total;
        if (smem <= 200 * 1024 || C == 1) break;
    }
    // stage each CTA's points in shared memory when they fit beside the rest
    const KmLayout Ls(k_max, d, (k_max + C - 1) / C, (n_max + C - 1) / C, true);
    const int stage_x = Ls.total <= 200 * 1024 ? 1 : 0;
    if (stage_x) smem = Ls.total;
    if (smem > 200 * 1024) {
        set_error("k-means: k*d = %d with n = %d needs %zu bytes of shared memory per CTA", k_max * d, n_max, smem);
        return CSC_E_UNSUPPORTED;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_lab = take((size_t)lab_total * 4), o_in = take((size_t)reps * NP * 8),
                 o_best = take((size_t)NP * 8), o_prob = take((size_t)NP * sizeof(KmProblem)),
                 o_out = take((size_t)NP * sizeof(int32_t*));
    void* base = nullptr;
    bool async_alloc = false;
    if (owner) {
        CSC_TRY(ws_get(owner, WS_KMEANS, off, &base));
    } else {
        cudaError_t e = cudaMallocAsync(&base, off, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocAsync(%zu) for k-means scratch: %s", off, cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        async_alloc = true;
    }
    char* b = (char*)base;
    std::vector<KmProblem> probs(NP);
    std::vector<int32_t*> outs(NP);
    int64_t lab_off = 0;
    for (int p = 0; p < NP; ++p) {
        probs[p].X = tasks[p].X;
        probs[p].n = tasks[p].n;
        probs[p].k = tasks[p].k;
        probs[p].seed = tasks[p].seed;
        probs[p].labels_all = (int32_t*)(b + o_lab) + lab_off;
        probs[p].inertia_all = (double*)(b + o_in) + (size_t)p * reps;
        lab_off += (int64_t)reps * tasks[p].n;
        outs[p] = tasks[p].labels_out;
    }
    KmProblem* d_probs = (KmProblem*)(b + o_prob);
    int32_t** d_outs = (int32_t**)(b + o_out);
    double* d_best = (double*)(b + o_best);
    CSC_CUDA_TRY(cudaMemcpyAsync(d_probs, probs.data(), NP * sizeof(KmProblem), cudaMemcpyHostToDevice, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(d_outs, outs.data(), NP * sizeof(int32_t*), cudaMemcpyHostToDevice, s));
    CSC_CUDA_TRY(cudaFuncSetAttribute(kmeans_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(reps * C, NP, 1);
    cfg.blockDim = dim3(kKmThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    double pts = 0.0;
    for (const KmTask& t : tasks) pts += (double)t.n;
    CSC_KLAUNCH("kmeans", 4.0 * pts * d * reps, s,
                CSC_CUDA_TRY(cudaLaunchKernelEx(&cfg, kmeans_cluster_kernel, (const KmProblem*)d_probs, d, ld,
                                                max_iter, stage_x)));
    CSC_KLAUNCH("kmeans_pick", 8.0 * pts, s,
                kmeans_pick_kernel<<<dim3(1, NP), 256, 0, s>>>(d_probs, reps, d_outs, d_best));
    std::vector<double> hb;
    if (inertia_out) {
        hb.resize(NP);
        CSC_CUDA_TRY(cudaMemcpyAsync(hb.data(), d_best, NP * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    // the host descriptor arrays die with this frame
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    if (inertia_out) memcpy(inertia_out, hb.data(), NP * sizeof(double));
    if (async_alloc) CSC_CUDA_TRY(cudaFreeAsync(base, s));
    return CSC_OK;
}

csc_status run_kmeans(const float* X, int64_t n64, int d, int ld, int k, int reps, int max_iter, uint64_t seed,
                      int32_t* labels_out, double* inertia_out, Graph* owner, cudaStream_t s) {
    std::vector<KmTask> t(1);
    t[0].X = X;
    t[0].n = (int)n64;
    t[0].k = k;
    t[0].seed = seed;
    t[0].labels_out = labels_out;
    return run_kmeans_multi(t, d, ld, reps, max_iter, inertia_out, owner, s);
}

}  // namespace csc
