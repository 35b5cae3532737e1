// sample.cu -- uniform sampling without replacement (Sec. 3.2, Eq. 4),
// variable-density sampling with replacement (Sec. 3.2.3 after Theorem 3.4)
// and the row gather of Alg. 2 step 5.
//
// Node i gets the key k_i = SplitMix64_seed(i) (output i of SplitMix64
// seeded with `seed`); the sample is the n nodes with the smallest (k_i, i),
// written in increasing node order.  Selection is a two-level radix select on
// the top 32 key bits (two 65536-bin histograms), a rank pass over the few
// keys that share the threshold prefix, and an order-preserving compaction of
// the selection flags.  Integer-only, so the result is bit-exact and
// independent of thread scheduling.
#include "common.cuh"
#include "device.cuh"

namespace csc {

constexpr int kBins = 65536;

__global__ void sample_hist1_kernel(int64_t N, uint64_t seed, uint32_t* __restrict__ h1) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = splitmix64_at(seed, (uint64_t)i);
        atomicAdd(h1 + (k >> 48), 1u);
    }
}

__global__ void sample_hist2_kernel(int64_t N, uint64_t seed, const uint32_t* __restrict__ sel,
                                    uint32_t* __restrict__ h2) {
    const uint32_t b1 = sel[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = splitmix64_at(seed, (uint64_t)i);
        if ((uint32_t)(k >> 48) == b1) atomicAdd(h2 + ((k >> 32) & 0xFFFFu), 1u);
    }
}

// One block of 1024 threads: find bin b with cum(< b) < need <= cum(<= b).
// sel[2*level] = b, sel[2*level+1] = cum(< b).  need = n - (earlier levels' counts).
__global__ void sample_find_kernel(const uint32_t* __restrict__ h, int64_t n, uint32_t* __restrict__ sel,
                                   int level) {
    __shared__ unsigned long long part[1024];
    __shared__ unsigned long long base[1024];
    const int t = threadIdx.x;
    const int per = kBins / 1024;  // 64 bins per thread
    int64_t need = n;
    if (level == 1) need = n - (int64_t)sel[1];
    unsigned long long s = 0;
    for (int i = 0; i < per; ++i) s += h[t * per + i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        unsigned long long acc = 0;
        for (int i = 0; i < 1024; ++i) {
            base[i] = acc;
            acc += part[i];
        }
    }
    __syncthreads();
    const unsigned long long lo = base[t], hi = base[t] + part[t];
    if ((int64_t)lo < need && need <= (int64_t)hi) {
        unsigned long long acc = lo;
        for (int i = 0; i < per; ++i) {
            const unsigned long long c = h[t * per + i];
            if ((int64_t)acc < need && need <= (int64_t)(acc + c)) {
                sel[2 * level] = (uint32_t)(t * per + i);
                sel[2 * level + 1] = (uint32_t)acc;
                break;
            }
            acc += c;
        }
    }
}

// flags[i] = 1 if the key's top 32 bits are below the threshold prefix; keys
// equal to it are appended to the candidate list.
__global__ void sample_mark_kernel(int64_t N, uint64_t seed, const uint32_t* __restrict__ sel,
                                   uint8_t* __restrict__ flags, unsigned long long* __restrict__ cand_key,
                                   int64_t* __restrict__ cand_idx, unsigned int* __restrict__ cand_count) {
    const uint32_t prefix = (sel[0] << 16) | sel[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = splitmix64_at(seed, (uint64_t)i);
        const uint32_t top = (uint32_t)(k >> 32);
        uint8_t f = top < prefix ? 1 : 0;
        if (top == prefix) {
            const unsigned int slot = atomicAdd(cand_count, 1u);
            cand_key[slot] = k;
            cand_idx[slot] = i;
        }
        flags[i] = f;
    }
}

// Candidates sharing the threshold prefix: keep those whose rank by (key, index)
// is below the remaining count.
__global__ void sample_resolve_kernel(int64_t n, const uint32_t* __restrict__ sel,
                                      const unsigned long long* __restrict__ cand_key,
                                      const int64_t* __restrict__ cand_idx, const unsigned int* __restrict__ cand_count,
                                      uint8_t* __restrict__ flags) {
    const int64_t need = n - (int64_t)sel[1] - (int64_t)sel[3];
    const unsigned int c = *cand_count;
    for (unsigned int a = threadIdx.x; a < c; a += blockDim.x) {
        const unsigned long long ka = cand_key[a];
        const int64_t ia = cand_idx[a];
        int64_t rank = 0;
        for (unsigned int b = 0; b < c; ++b) {
            const unsigned long long kb = cand_key[b];
            rank += (kb < ka || (kb == ka && cand_idx[b] < ia)) ? 1 : 0;
        }
        if (rank < need) flags[ia] = 1;
    }
}

constexpr int kChunk = 4096;  // flags per compaction block (1024 threads x 4)

template <typename T>
__device__ __forceinline__ T block_excl_scan_1024(T v, T* warp_tot, T* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = warp_tot[lane];
        T incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        warp_tot[lane] = incl - t;
        if (lane == 31) *total = incl;
    }
    __syncthreads();
    return warp_tot[w] + x - v;
}

// F: uint8 selection flags, or int32 draw counts (variable density)
template <typename F>
__global__ void compact_count_kernel(const F* __restrict__ flags, int64_t N, int* __restrict__ counts) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * 4;
    int v = 0;
    for (int q = 0; q < 4; ++q)
        if (base + q < N) v += (int)flags[base + q];
    block_excl_scan_1024<int>(v, warp_tot, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

__global__ void compact_scan_kernel(int* __restrict__ counts, int nblocks) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nblocks; ++b) {
            const int c = counts[b];
            counts[b] = acc;
            acc += c;
        }
    }
}

__global__ void compact_write_kernel(const uint8_t* __restrict__ flags, int64_t N, const int* __restrict__ offs,
                                     int64_t* __restrict__ out, int64_t n_out) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * 4;
    uint8_t f[4];
    int v = 0;
    for (int q = 0; q < 4; ++q) {
        f[q] = (base + q < N) ? flags[base + q] : 0;
        v += f[q];
    }
    int pos = offs[blockIdx.x] + block_excl_scan_1024<int>(v, warp_tot, &total);
    for (int q = 0; q < 4; ++q)
        if (f[q]) {
            if (pos < n_out) out[pos] = base + q;  // exactly n flags are set; the guard is insurance
            ++pos;
        }
}

csc_status run_sample(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out, Graph* owner, cudaStream_t s) {
    const int nblk = ceil_div(N, kChunk);
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_h1 = take(kBins * 4), o_h2 = take(kBins * 4), o_sel = take(64);
    const size_t o_cnt = take(16), o_ck = take((size_t)N * 8), o_ci = take((size_t)N * 8);
    const size_t o_fl = take((size_t)N), o_bc = take((size_t)nblk * 4);
    void* base = nullptr;
    bool async_alloc = false;
    if (owner) {
        CSC_TRY(ws_get(owner, WS_SAMPLE, off, &base));
    } else {
        cudaError_t e = cudaMallocAsync(&base, off, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocAsync(%zu) for sampling scratch: %s", off, cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        async_alloc = true;
    }
    char* b = (char*)base;
    uint32_t* h1 = (uint32_t*)(b + o_h1);
    uint32_t* h2 = (uint32_t*)(b + o_h2);
    uint32_t* sel = (uint32_t*)(b + o_sel);
    unsigned int* cnt = (unsigned int*)(b + o_cnt);
    unsigned long long* ck = (unsigned long long*)(b + o_ck);
    int64_t* cidx = (int64_t*)(b + o_ci);
    uint8_t* fl = (uint8_t*)(b + o_fl);
    int* bc = (int*)(b + o_bc);
    // histograms, selection words and the candidate counter start at zero
    CSC_CUDA_TRY(cudaMemsetAsync(b, 0, o_ck, s));
    int grid = ceil_div(N, 256);
    if (grid > 4096) grid = 4096;
    CSC_KLAUNCH("sample_hist", 4.0 * kBins, s, sample_hist1_kernel<<<grid, 256, 0, s>>>(N, seed, h1));
    CSC_KLAUNCH("sample_find", 4.0 * kBins, s, sample_find_kernel<<<1, 1024, 0, s>>>(h1, n, sel, 0));
    CSC_KLAUNCH("sample_hist", 4.0 * kBins, s, sample_hist2_kernel<<<grid, 256, 0, s>>>(N, seed, sel, h2));
    CSC_KLAUNCH("sample_find", 4.0 * kBins, s, sample_find_kernel<<<1, 1024, 0, s>>>(h2, n, sel, 1));
    CSC_KLAUNCH("sample_mark", (double)N, s,
                sample_mark_kernel<<<grid, 256, 0, s>>>(N, seed, sel, fl, ck, cidx, cnt));
    CSC_KLAUNCH("sample_resolve", 16.0, s, sample_resolve_kernel<<<1, 1024, 0, s>>>(n, sel, ck, cidx, cnt, fl));
    CSC_KLAUNCH("sample_compact", (double)N, s, compact_count_kernel<uint8_t><<<nblk, 1024, 0, s>>>(fl, N, bc));
    CSC_KLAUNCH("sample_compact", 8.0 * nblk, s, compact_scan_kernel<<<1, 32, 0, s>>>(bc, nblk));
    CSC_KLAUNCH("sample_compact", (double)N + 8.0 * n, s,
                compact_write_kernel<<<nblk, 1024, 0, s>>>(fl, N, bc, idx_out, n));
    if (async_alloc) CSC_CUDA_TRY(cudaFreeAsync(base, s));
    return CSC_OK;
}

// ---------------------------------------------------------------- variable density
// Variable-density sampling (Sec. 3.2.3 after Theorem 3.4; the coherence
// estimate of the remark closing Sec. 4.2).  Node i gets the integer weight
// q_i = floor(2^32 * (s_i / max s)) of its score s_i >= 0; draw t takes the word
// r_t = SplitMix64_seed(t), the point u_t = floor(r_t * Q / 2^64) (Q = sum q),
// and the node with the smallest inclusive prefix sum of q above u_t, so node i
// is drawn with probability q_i / Q.  The draws are i.i.d. (with replacement)
// and written sorted by node, each with the decoder weight Q / (N q_i).  Only
// the q / Q arithmetic touches floating point (one correctly rounded fp64
// division per node); the rest is integer, so the draws are bit-exact.

__device__ __forceinline__ uint64_t vd_weight(double s, double smax) {
    if (!(s > 0.0) || !(s <= smax)) return 0ull;  // zero, negative, NaN or past the maximum
    return (uint64_t)floor((s / smax) * 4294967296.0);
}

// maximum score (as the bits of a non-negative double, which order like the
// values) and a flag for scores that are negative, NaN or infinite
__global__ void vd_max_kernel(const double* __restrict__ score, int64_t N, unsigned long long* __restrict__ maxbits,
                              int* __restrict__ bad) {
    unsigned long long mb = 0ull;
    int b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = score[i];
        if (!(v >= 0.0) || isinf(v)) {
            b = 1;
        } else if (v > 0.0) {
            const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
            mb = vb > mb ? vb : mb;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = y > mb ? y : mb;
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mb) atomicMax(maxbits, mb);
        if (b) atomicOr(bad, 1);
    }
}

// per chunk of kChunk nodes: sum of q
__global__ void vd_chunk_sum_kernel(const double* __restrict__ score, int64_t N,
                                    const unsigned long long* __restrict__ maxbits,
                                    unsigned long long* __restrict__ csum) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long total;
    const double smax = __longlong_as_double((long long)*maxbits);
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * 4;
    unsigned long long v = 0ull;
    for (int q = 0; q < 4; ++q)
        if (base + q < N) v += vd_weight(score[base + q], smax);
    block_excl_scan_1024<unsigned long long>(v, warp_tot, &total);
    if (threadIdx.x == 0) csum[blockIdx.x] = total;
}

// exclusive scan of the chunk sums in place; csum[nblocks] = Q
__global__ void vd_chunk_scan_kernel(unsigned long long* __restrict__ csum, int nblocks) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long acc = 0ull;
        for (int b = 0; b < nblocks; ++b) {
            const unsigned long long c = csum[b];
            csum[b] = acc;
            acc += c;
        }
        csum[nblocks] = acc;
    }
}

// cum[i] = q_0 + ... + q_i
__global__ void vd_cum_kernel(const double* __restrict__ score, int64_t N, const unsigned long long* __restrict__ maxbits,
                              const unsigned long long* __restrict__ csum, unsigned long long* __restrict__ cum) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long total;
    const double smax = __longlong_as_double((long long)*maxbits);
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * 4;
    unsigned long long q[4], v = 0ull;
    for (int e = 0; e < 4; ++e) {
        q[e] = base + e < N ? vd_weight(score[base + e], smax) : 0ull;
        v += q[e];
    }
    unsigned long long acc = csum[blockIdx.x] + block_excl_scan_1024<unsigned long long>(v, warp_tot, &total);
    for (int e = 0; e < 4; ++e) {
        acc += q[e];
        if (base + e < N) cum[base + e] = acc;
    }
}

// one thread per draw: binary search of the inverse CDF, count the draws per node
__global__ void vd_draw_kernel(int64_t n, uint64_t seed, const unsigned long long* __restrict__ cum, int64_t N,
                               const unsigned long long* __restrict__ Qp, int* __restrict__ cnt) {
    const unsigned long long Q = *Qp;
    if (Q == 0ull) return;  // every score zero: reported by the host
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long u = __umul64hi(splitmix64_at(seed, (uint64_t)t), Q);  // u < Q = cum[N-1]
        int64_t lo = 0, hi = N - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid] > u) hi = mid;
            else lo = mid + 1;
        }
        atomicAdd(cnt + lo, 1);
    }
}

// node i repeated cnt[i] times, in node order, each copy with weight Q / (N q_i)
__global__ void vd_write_kernel(const int* __restrict__ cnt, const unsigned long long* __restrict__ cum, int64_t N,
                                const unsigned long long* __restrict__ Qp, const int* __restrict__ offs,
                                int64_t* __restrict__ idx_out, float* __restrict__ w_out, int64_t n_out) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const int64_t base = (int64_t)blockIdx.x * kChunk + threadIdx.x * 4;
    int c[4], v = 0;
    for (int e = 0; e < 4; ++e) {
        c[e] = (base + e < N) ? cnt[base + e] : 0;
        v += c[e];
    }
    int64_t pos = offs[blockIdx.x] + block_excl_scan_1024<int>(v, warp_tot, &total);
    const double Q = (double)*Qp;
    for (int e = 0; e < 4; ++e) {
        if (!c[e]) continue;
        const int64_t i = base + e;
        const unsigned long long qi = cum[i] - (i > 0 ? cum[i - 1] : 0ull);
        const float w = (float)(Q / ((double)N * (double)qi));
        for (int r = 0; r < c[e]; ++r, ++pos) {
            if (pos < n_out) {  // the counts add up to n_out; the guard is insurance
                idx_out[pos] = i;
                if (w_out) w_out[pos] = w;
            }
        }
    }
}

csc_status run_sample_weighted(const double* score, int64_t N, int64_t n, uint64_t seed, int64_t* idx_out,
                               float* w_out, Graph* owner, cudaStream_t s) {
    const int nblk = ceil_div(N, kChunk);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_hdr = take(64), o_cnt = take((size_t)N * 4), o_cs = take((size_t)(nblk + 1) * 8);
    const size_t o_cum = take((size_t)N * 8), o_bc = take((size_t)nblk * 4);
    void* base = nullptr;
    bool async_alloc = false;
    if (owner) {
        CSC_TRY(ws_get(owner, WS_SAMPLE, off, &base));
    } else {
        cudaError_t e = cudaMallocAsync(&base, off, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocAsync(%zu) for sampling scratch: %s", off, cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        async_alloc = true;
    }
    char* b = (char*)base;
    unsigned long long* maxbits = (unsigned long long*)(b + o_hdr);
    int* bad = (int*)(b + o_hdr + 8);
    int* cnt = (int*)(b + o_cnt);
    unsigned long long* cs = (unsigned long long*)(b + o_cs);
    unsigned long long* cum = (unsigned long long*)(b + o_cum);
    int* bc = (int*)(b + o_bc);
    // header (maximum, flag) and the per-node draw counts start at zero
    CSC_CUDA_TRY(cudaMemsetAsync(b, 0, o_cs, s));
    int grid = ceil_div(N, 256);
    if (grid > 4096) grid = 4096;
    CSC_KLAUNCH("vd_scan", 8.0 * N, s, vd_max_kernel<<<grid, 256, 0, s>>>(score, N, maxbits, bad));
    CSC_KLAUNCH("vd_scan", 8.0 * N, s, vd_chunk_sum_kernel<<<nblk, 1024, 0, s>>>(score, N, maxbits, cs));
    CSC_KLAUNCH("vd_scan", 16.0 * nblk, s, vd_chunk_scan_kernel<<<1, 32, 0, s>>>(cs, nblk));
    CSC_KLAUNCH("vd_scan", 16.0 * N, s, vd_cum_kernel<<<nblk, 1024, 0, s>>>(score, N, maxbits, cs, cum));
    int dgrid = (int)std::min<int64_t>(ceil_div(n, 256), 4096);
    CSC_KLAUNCH("vd_draw", 8.0 * n * 24, s, vd_draw_kernel<<<dgrid, 256, 0, s>>>(n, seed, cum, N, cs + nblk, cnt));
    CSC_KLAUNCH("sample_compact", 4.0 * N, s, compact_count_kernel<int><<<nblk, 1024, 0, s>>>(cnt, N, bc));
    CSC_KLAUNCH("sample_compact", 8.0 * nblk, s, compact_scan_kernel<<<1, 32, 0, s>>>(bc, nblk));
    CSC_KLAUNCH("sample_compact", 12.0 * N + 12.0 * n, s,
                vd_write_kernel<<<nblk, 1024, 0, s>>>(cnt, cum, N, cs + nblk, bc, idx_out, w_out, n));
    struct {
        unsigned long long maxbits;
        int bad;
    } h{};
    CSC_CUDA_TRY(cudaMemcpyAsync(&h.maxbits, maxbits, 8, cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(&h.bad, bad, 4, cudaMemcpyDeviceToHost, s));
    if (async_alloc) CSC_CUDA_TRY(cudaFreeAsync(base, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.bad) {
        set_error("variable-density sampling: scores must be finite and non-negative");
        return CSC_E_INVALID;
    }
    if (!h.maxbits) {
        set_error("variable-density sampling: every score is zero");
        return CSC_E_INVALID;
    }
    return CSC_OK;
}

// ---------------------------------------------------------------- gather
// Rows with an index outside [0, N) are written as zeros.
template <typename S>
__global__ void gather_rows_kernel(const S* __restrict__ X, int64_t N, int ld, const int64_t* __restrict__ idx,
                                   int64_t n, int d, float* __restrict__ out, int ld_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * d) return;
    const int64_t i = t / d;
    const int c = (int)(t % d);
    const int64_t r = idx[i];
    out[i * ld_out + c] = (r >= 0 && r < N) ? (float)X[r * ld + c] : 0.0f;
}

csc_status run_gather_rows(const float* X, int64_t N, int ld, const int64_t* idx, int64_t n, int d, float* out,
                           int ld_out, cudaStream_t s) {
    CSC_KLAUNCH("gather_rows", 8.0 * n * d + 8.0 * n, s,
                gather_rows_kernel<float><<<ceil_div(n * d, 256), 256, 0, s>>>(X, N, ld, idx, n, d, out, ld_out));
    return CSC_OK;
}

csc_status run_gather_rows_f64(const double* X, int64_t N, int ld, const int64_t* idx, int64_t n, int d,
                               float* out, int ld_out, cudaStream_t s) {
    CSC_KLAUNCH("gather_rows", 12.0 * n * d + 8.0 * n, s,
                gather_rows_kernel<double><<<ceil_div(n * d, 256), 256, 0, s>>>(X, N, ld, idx, n, d, out, ld_out));
    return CSC_OK;
}

}  // namespace csc
