// kmeans.cu -- k-means on the reduced feature set (Alg. 2 step 6).
//
// One CTA per replicate (the paper runs 20 replicates, Sec. 5).  Seeding is
// k-means++ with uniforms from Philox4x32-10 (key = (seed, "k-means"),
// counter = (replicate, draw)): the first centre is point floor(u n), centre
// t >= 1 the first point whose running sum of squared distances to the chosen
// centres reaches u * total.  Lloyd iterations assign each point to its
// nearest centre (ties to the lower index) and move each centre to the mean
// of its points; an empty cluster (in increasing index) takes the point
// farthest from its own centre, which moves to it.  Centre sums are exact
// 64-bit fixed-point integers, so they do not depend on the order in which
// threads add them.  The best replicate by inertia (ties to the first) wins.
#include <math.h>

#include "common.cuh"
#include "device.cuh"

namespace csc {

constexpr int kKmThreads = 512;

__device__ __forceinline__ float sqdist(const float* __restrict__ x, const float* __restrict__ c, int d) {
    float s = 0.f;
    for (int q = 0; q < d; ++q) {
        const float t = x[q] - c[q];
        s = fmaf(t, t, s);
    }
    return s;
}

// block-wide reductions over kKmThreads threads
__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kKmThreads / 32; ++i) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// argmax of (value, -index): largest value, ties to the lowest index
__device__ void block_argmax(float v, int idx, float* shv, int* shi, float* out_v, int* out_i) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        shv[w] = v;
        shi[w] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bv = shv[0];
        int bi = shi[0];
        for (int i = 1; i < kKmThreads / 32; ++i)
            if (shv[i] > bv || (shv[i] == bv && shi[i] < bi)) {
                bv = shv[i];
                bi = shi[i];
            }
        *out_v = bv;
        *out_i = bi;
    }
    __syncthreads();
}

__device__ __forceinline__ double km_uniform(uint64_t seed, uint32_t rep, uint32_t t) {
    const Philox4 r = philox4x32_10(rep, 0u, t, 0u, (uint32_t)seed, (uint32_t)(seed >> 32) ^ STREAM_KMEANS);
    return (double)philox_uniform(r.x[0]);
}

__global__ void __launch_bounds__(kKmThreads)
kmeans_replicate_kernel(const float* __restrict__ X, int n, int d, int ld, int k, int max_iter, uint64_t seed,
                        int32_t* __restrict__ labels_all, double* __restrict__ inertia_all,
                        double* __restrict__ d2_all, unsigned long long* __restrict__ sums_all,
                        int* __restrict__ counts_all, int32_t* __restrict__ newlab_all) {
    extern __shared__ float C[];  // k x d centres
    __shared__ double shd[40];
    __shared__ float shv[32];
    __shared__ int shi[32];
    __shared__ int sh_pick;
    __shared__ float sh_best;
    __shared__ int sh_changed;
    __shared__ double sh_scale;
    const int rep = blockIdx.x;
    double* d2 = d2_all + (int64_t)rep * n;
    int32_t* lab = labels_all + (int64_t)rep * n;
    int32_t* nlab = newlab_all + (int64_t)rep * n;
    unsigned long long* sums = sums_all + (int64_t)rep * k * d;
    int* counts = counts_all + (int64_t)rep * k;
    const int T = threadIdx.x;

    // fixed-point scale for exact centre sums: n * max|x| * scale < 2^62
    {
        float mx = 0.f;
        for (int64_t t = T; t < (int64_t)n * d; t += kKmThreads) mx = fmaxf(mx, fabsf(X[(t / d) * ld + t % d]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((T & 31) == 0) shv[T >> 5] = mx;
        __syncthreads();
        if (T == 0) {
            float m = 0.f;
            for (int i = 0; i < kKmThreads / 32; ++i) m = fmaxf(m, shv[i]);
            int e = 61 - (int)ceil(log2((double)n + 1.0)) - (m > 0.f ? (int)ceil(log2((double)m)) : 0);
            sh_scale = ldexp(1.0, e > 1000 ? 1000 : e);
        }
        __syncthreads();
    }
    const double scale = sh_scale;

    // ---- k-means++ seeding
    if (T == 0) {
        const double u = km_uniform(seed, (uint32_t)rep, 0u);
        int p = (int)(u * (double)n);
        sh_pick = p < n - 1 ? p : n - 1;
    }
    __syncthreads();
    for (int q = T; q < d; q += kKmThreads) C[q] = X[(int64_t)sh_pick * ld + q];
    __syncthreads();
    for (int i = T; i < n; i += kKmThreads) d2[i] = (double)sqdist(X + (int64_t)i * ld, C, d);
    __syncthreads();
    const int chunk = (n + kKmThreads - 1) / kKmThreads;
    for (int t = 1; t < k; ++t) {
        // per-thread contiguous chunk sums, exclusive scan across threads
        const int i0 = T * chunk, i1 = min(n, i0 + chunk);
        double part = 0.0;
        for (int i = i0; i < i1; ++i) part += d2[i];
        // exclusive scan of `part` over the block (fp64, fixed order)
        __shared__ double scan_w[kKmThreads / 32];
        double incl = part;
        const int lane = T & 31, w = T >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) scan_w[w] = incl;
        __syncthreads();
        if (T == 0) {
            double acc = 0.0;
            for (int i = 0; i < kKmThreads / 32; ++i) {
                const double v = scan_w[i];
                scan_w[i] = acc;
                acc += v;
            }
            shd[33] = acc;  // total
            sh_pick = n;    // "not found yet"
        }
        __syncthreads();
        const double excl = scan_w[w] + incl - part;
        const double total = shd[33];
        const double u = km_uniform(seed, (uint32_t)rep, (uint32_t)t);
        if (total <= 0.0) {
            if (T == 0) {
                int p = (int)(u * (double)n);
                sh_pick = p < n - 1 ? p : n - 1;
            }
        } else {
            const double target = u * total;
            // first i with cumulative >= target lies in the chunk where excl < target <= excl + part
            if (i0 < i1 && excl < target && target <= excl + part) {
                double acc = excl;
                int p = i1 - 1;
                for (int i = i0; i < i1; ++i) {
                    acc += d2[i];
                    if (acc >= target) {
                        p = i;
                        break;
                    }
                }
                atomicMin(&sh_pick, p);
            }
        }
        __syncthreads();
        if (T == 0 && sh_pick >= n) sh_pick = n - 1;  // rounding left the target past the end
        __syncthreads();
        const int p = sh_pick;
        for (int q = T; q < d; q += kKmThreads) C[t * d + q] = X[(int64_t)p * ld + q];
        __syncthreads();
        for (int i = T; i < n; i += kKmThreads) {
            const double dd = (double)sqdist(X + (int64_t)i * ld, C + t * d, d);
            if (dd < d2[i]) d2[i] = dd;
        }
        __syncthreads();
    }

    // ---- Lloyd iterations
    auto assign = [&](int32_t* out) {
        int changed = 0;
        for (int i = T; i < n; i += kKmThreads) {
            const float* x = X + (int64_t)i * ld;
            float best = sqdist(x, C, d);
            int bj = 0;
            for (int j = 1; j < k; ++j) {
                const float dj = sqdist(x, C + j * d, d);
                if (dj < best) {
                    best = dj;
                    bj = j;
                }
            }
            if (out == nlab && bj != lab[i]) changed = 1;
            out[i] = bj;
        }
        return changed;
    };
    assign(lab);
    __syncthreads();
    for (int it = 1; it <= max_iter; ++it) {
        for (int q = T; q < k * d; q += kKmThreads) sums[q] = 0ull;
        for (int j = T; j < k; j += kKmThreads) counts[j] = 0;
        __syncthreads();
        for (int i = T; i < n; i += kKmThreads) {
            const int j = lab[i];
            atomicAdd(counts + j, 1);
            for (int q = 0; q < d; ++q) {
                const long long v = llrint((double)X[(int64_t)i * ld + q] * scale);
                atomicAdd(sums + (int64_t)j * d + q, (unsigned long long)v);
            }
        }
        __syncthreads();
        for (int q = T; q < k * d; q += kKmThreads) {
            const int j = q / d;
            if (counts[j] > 0) C[q] = (float)((double)(long long)sums[q] / scale / (double)counts[j]);
        }
        __syncthreads();
        for (int j = 0; j < k; ++j) {
            if (counts[j] > 0) continue;  // uniform across the block
            float bv = -1.f;
            int bi = 0x7fffffff;
            for (int i = T; i < n; i += kKmThreads) {
                const float v = sqdist(X + (int64_t)i * ld, C + lab[i] * d, d);
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
            block_argmax(bv, bi, shv, shi, &sh_best, &sh_pick);
            const int p = sh_pick;
            for (int q = T; q < d; q += kKmThreads) C[j * d + q] = X[(int64_t)p * ld + q];
            __syncthreads();
            if (T == 0) {
                // the donor cluster keeps its centre and is not revisited this update
                counts[j] = 1;
                lab[p] = j;
            }
            __syncthreads();
        }
        if (T == 0) sh_changed = 0;
        __syncthreads();
        const int ch = assign(nlab);
        if (ch) atomicOr(&sh_changed, 1);
        __syncthreads();
        for (int i = T; i < n; i += kKmThreads) lab[i] = nlab[i];
        __syncthreads();
        if (!sh_changed) break;
    }
    double in = 0.0;
    for (int i = T; i < n; i += kKmThreads) in += (double)sqdist(X + (int64_t)i * ld, C + lab[i] * d, d);
    in = block_sum_d(in, shd);
    if (T == 0) inertia_all[rep] = in;
}

__global__ void kmeans_pick_kernel(const int32_t* __restrict__ labels_all, const double* __restrict__ inertia_all,
                                   int reps, int n, int32_t* __restrict__ labels_out, double* __restrict__ inertia_out) {
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

csc_status run_kmeans(const float* X, int64_t n64, int d, int ld, int k, int reps, int max_iter, uint64_t seed,
                      int32_t* labels_out, double* inertia_out, Graph* owner, cudaStream_t s) {
    const int n = (int)n64;
    const size_t smem = (size_t)k * d * sizeof(float);
    if (smem > 200 * 1024) {
        set_error("k-means: k*d = %d exceeds the shared-memory centre table", k * d);
        return CSC_E_UNSUPPORTED;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_lab = take((size_t)reps * n * 4), o_nlab = take((size_t)reps * n * 4);
    const size_t o_in = take((size_t)reps * 8 + 8), o_d2 = take((size_t)reps * n * 8);
    const size_t o_sum = take((size_t)reps * k * d * 8), o_cnt = take((size_t)reps * k * 4);
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
    if (smem > 48 * 1024)
        CSC_CUDA_TRY(cudaFuncSetAttribute(kmeans_replicate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    double* inertia_all = (double*)(b + o_in);
    CSC_KLAUNCH("kmeans", 4.0 * n * d * reps, s,
                kmeans_replicate_kernel<<<reps, kKmThreads, smem, s>>>(
                    X, n, d, ld, k, max_iter, seed, (int32_t*)(b + o_lab), inertia_all, (double*)(b + o_d2),
                    (unsigned long long*)(b + o_sum), (int*)(b + o_cnt), (int32_t*)(b + o_nlab)));
    double* dev_inertia = inertia_all + reps;
    CSC_KLAUNCH("kmeans_pick", 8.0 * n, s,
                kmeans_pick_kernel<<<1, 256, 0, s>>>((int32_t*)(b + o_lab), inertia_all, reps, n, labels_out,
                                                     dev_inertia));
    if (inertia_out) {
        CSC_CUDA_TRY(cudaMemcpyAsync(inertia_out, dev_inertia, sizeof(double), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (async_alloc) CSC_CUDA_TRY(cudaFreeAsync(base, s));
    return CSC_OK;
}

}  // namespace csc
