// sample_noalloc.cu -- csc_sample_noalloc: the uniform sampling of csc_sample
// (same keys, same result) for callers that cannot allocate device memory.
//
// Who needs it: applications that hand all device memory to an allocator they
// own (a framework's caching pool, an arena sized at start-up), or that run
// with a fixed device-memory budget, or that sit on a latency-critical path
// where cudaMalloc / cudaFree may implicitly synchronize the device.  They
// still pass the output buffer; everything else lives in one fixed scratch
// array of this file, created when the library is loaded on a device and
// held by every device that loads the library until the process exits.
//
// Method: node i has the key SplitMix64_seed(i).  These keys are pairwise
// distinct (an odd-stride counter sequence through a bijective mixer), so the
// n smallest keys are determined by the n-th smallest key T alone.  T is found
// by a four-level radix select, 16 bits per level, each level a histogram of
// the keys that match the bits already fixed; the sample is then {i : key_i <= T}
// written in increasing i by a two-pass compaction that recomputes the keys.
// No per-node storage is needed, so the scratch size does not grow with N
// except for one int per 4096 nodes.
#include <mutex>

#include "common.cuh"
#include "device.cuh"

namespace csc {
namespace {

constexpr int kNaBins = 65536;                 // 16-bit histogram
constexpr int kNaChunk = 4096;                 // nodes per compaction block
constexpr int kNaMaxBlocks = 16384;            // -> at most 2^26 nodes
constexpr int64_t kNaMaxNodes = (int64_t)kNaChunk * kNaMaxBlocks;
constexpr size_t kNaHistOff = 0;
constexpr size_t kNaSelOff = kNaBins * 4;                  // 8 x uint32 selection words
constexpr size_t kNaBlkOff = kNaSelOff + 256;              // kNaMaxBlocks x int
constexpr size_t kNaScratchBytes = kNaBlkOff + (size_t)kNaMaxBlocks * 4;  // 327,936 bytes

// The scratch: one fixed array per device, shared by every call of
// csc_sample_noalloc on that device.
static __device__ __align__(256) unsigned char g_sample_noalloc_scratch[kNaScratchBytes];

// Host-side device addresses of the scratch, resolved once per device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};

// Keys matching the bits fixed by the previous levels add to the histogram of
// their next 16 bits.  sel[2*l] holds the bin chosen at level l.
__global__ void na_hist_kernel(int64_t N, uint64_t seed, int level, const uint32_t* __restrict__ sel,
                               uint32_t* __restrict__ hist) {
    uint64_t prefix = 0;
    for (int l = 0; l < level; ++l) prefix = (prefix << 16) | sel[2 * l];
    const int shift_fixed = 64 - 16 * level;  // bits above this are fixed
    const int shift_bin = 48 - 16 * level;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = splitmix64_at(seed, (uint64_t)i);
        if (level == 0 || (k >> shift_fixed) == prefix) atomicAdd(hist + ((k >> shift_bin) & 0xFFFFu), 1u);
    }
}

// One block of 1024 threads: the bin b holding the `need`-th key of this level,
// need = n - (keys below the chosen bins of earlier levels).
__global__ void na_find_kernel(const uint32_t* __restrict__ hist, int64_t n, int level, uint32_t* __restrict__ sel) {
    __shared__ unsigned long long part[1024];
    __shared__ unsigned long long base[1024];
    const int t = threadIdx.x;
    constexpr int per = kNaBins / 1024;
    int64_t need = n;
    for (int l = 0; l < level; ++l) need -= (int64_t)sel[2 * l + 1];
    unsigned long long s = 0;
    for (int i = 0; i < per; ++i) s += hist[t * per + i];
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
            const unsigned long long c = hist[t * per + i];
            if ((int64_t)acc < need && need <= (int64_t)(acc + c)) {
                sel[2 * level] = (uint32_t)(t * per + i);
                sel[2 * level + 1] = (uint32_t)acc;
                break;
            }
            acc += c;
        }
    }
}

__device__ __forceinline__ uint64_t na_threshold(const uint32_t* sel) {
    return ((uint64_t)sel[0] << 48) | ((uint64_t)sel[2] << 32) | ((uint64_t)sel[4] << 16) | (uint64_t)sel[6];
}

__device__ __forceinline__ int na_block_excl_scan(int v, int* warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        const int t = warp_tot[lane];
        int incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        warp_tot[lane] = incl - t;
    }
    __syncthreads();
    return warp_tot[w] + x - v;
}

// Selected nodes per 4096-node chunk (selection recomputed from the keys).
__global__ void na_count_kernel(int64_t N, uint64_t seed, const uint32_t* __restrict__ sel, int* __restrict__ counts) {
    __shared__ int warp_tot[32];
    const uint64_t T = na_threshold(sel);
    const int64_t base = (int64_t)blockIdx.x * kNaChunk + threadIdx.x * 4;
    int v = 0;
    for (int q = 0; q < 4; ++q)
        if (base + q < N && splitmix64_at(seed, (uint64_t)(base + q)) <= T) ++v;
    const int ex = na_block_excl_scan(v, warp_tot);
    if (threadIdx.x == blockDim.x - 1) counts[blockIdx.x] = ex + v;
}

__global__ void na_scan_kernel(int* __restrict__ counts, int nblocks) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nblocks; ++b) {
            const int c = counts[b];
            counts[b] = acc;
            acc += c;
        }
    }
}

__global__ void na_write_kernel(int64_t N, uint64_t seed, const uint32_t* __restrict__ sel,
                                const int* __restrict__ offs, int64_t* __restrict__ out, int64_t n_out) {
    __shared__ int warp_tot[32];
    const uint64_t T = na_threshold(sel);
    const int64_t base = (int64_t)blockIdx.x * kNaChunk + threadIdx.x * 4;
    bool f[4];
    int v = 0;
    for (int q = 0; q < 4; ++q) {
        f[q] = base + q < N && splitmix64_at(seed, (uint64_t)(base + q)) <= T;
        v += f[q] ? 1 : 0;
    }
    int pos = offs[blockIdx.x] + na_block_excl_scan(v, warp_tot);
    for (int q = 0; q < 4; ++q)
        if (f[q]) {
            if (pos < n_out) out[pos] = base + q;
            ++pos;
        }
}

// Device address of the scratch on the current device, resolved on the first
// call for that device (cudaGetSymbolAddress with the device current).
csc_status na_scratch(void** out) {
    int dev = 0;
    CSC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("csc_sample_noalloc: device ordinal %d beyond the %d supported", dev, kNaMaxDevices);
        return CSC_E_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sample_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("csc_sample_noalloc: cudaGetSymbolAddress of the scratch failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return CSC_E_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return CSC_OK;
}

}  // namespace
}  // namespace csc

using namespace csc;

extern "C" CSC_API csc_status csc_sample_noalloc(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out,
                                                 void* stream) {
    clear_error();
    if (N < 1 || n < 0 || n > N || (n > 0 && !idx_out)) {
        set_error("csc_sample_noalloc: need 0 <= n <= N, N >= 1 and idx_out != NULL");
        return CSC_E_INVALID;
    }
    if (N > kNaMaxNodes) {
        set_error("csc_sample_noalloc: N = %lld exceeds the fixed scratch limit of %lld nodes; use csc_sample",
                  (long long)N, (long long)kNaMaxNodes);
        return CSC_E_UNSUPPORTED;
    }
    if (n == 0) return CSC_OK;
    void* base = nullptr;
    CSC_TRY(na_scratch(&base));
    cudaStream_t s = (cudaStream_t)stream;
    char* b = (char*)base;
    uint32_t* hist = (uint32_t*)(b + kNaHistOff);
    uint32_t* sel = (uint32_t*)(b + kNaSelOff);
    int* blk = (int*)(b + kNaBlkOff);
    const int nblk = ceil_div(N, kNaChunk);
    int grid = ceil_div(N, 256);
    if (grid > 4096) grid = 4096;
    // the scratch keeps the previous call's contents: clear the selection words
    CSC_CUDA_TRY(cudaMemsetAsync(sel, 0, 8 * sizeof(uint32_t), s));
    for (int level = 0; level < 4; ++level) {
        CSC_CUDA_TRY(cudaMemsetAsync(hist, 0, kNaBins * sizeof(uint32_t), s));
        CSC_KLAUNCH("sample_noalloc", 4.0 * kNaBins, s, na_hist_kernel<<<grid, 256, 0, s>>>(N, seed, level, sel, hist));
        CSC_KLAUNCH("sample_noalloc", 4.0 * kNaBins, s, na_find_kernel<<<1, 1024, 0, s>>>(hist, n, level, sel));
    }
    CSC_KLAUNCH("sample_noalloc", 4.0 * nblk, s, na_count_kernel<<<nblk, 1024, 0, s>>>(N, seed, sel, blk));
    CSC_KLAUNCH("sample_noalloc", 8.0 * nblk, s, na_scan_kernel<<<1, 32, 0, s>>>(blk, nblk));
    CSC_KLAUNCH("sample_noalloc", 8.0 * n, s, na_write_kernel<<<nblk, 1024, 0, s>>>(N, seed, sel, blk, idx_out, n));
    return CSC_OK;
}
