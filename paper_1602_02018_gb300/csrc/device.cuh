// device.cuh -- device-side building blocks of the CSR SpMM kernels.
//
// * 16-byte row-vector loads/stores for the three storage types: fp32
//   (float4, 4 values), bf16 (uint4 holding 8 values, widened to fp32) and
//   fp64 (double2, 2 values).  Arithmetic is fp32 for fp32/bf16 storage and
//   fp64 for fp64 storage.
// * gather_row: the neighbour sum sum_{l in N(i)} dinv_l X[l, :] of one row
//   of S X with S = D^-1/2 W D^-1/2 (Sec. 2.1; the edge weight
//   1/sqrt(d_i d_l) is rebuilt from the degree vector, never stored).  A
//   group of G lanes owns one row; each lane owns NT 16-byte column vectors
//   spaced G vectors apart, so a group covers NT*G*VEC columns.
// * Philox4x32-10 (Salmon et al., SC'11) and SplitMix64 (Steele et al.,
//   OOPSLA'14) counter-based generators.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace csc {

template <typename T>
struct StoreTraits;

template <>
struct StoreTraits<float> {
    using acc_t = float;
    using raw_t = float4;  // one 16-byte vector as loaded (prefetched operands)
    static constexpr int VEC = 4;
    __device__ static inline raw_t ld_raw(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
    __device__ static inline raw_t ld_raw_cs(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
    __device__ static inline void unraw(const raw_t& q, float (&v)[4]) {
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static inline void load(const float* p, float (&v)[4]) {
        float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    // streaming load (data read once: X_{j-1}, Y)
    __device__ static inline void load_cs(const float* p, float (&v)[4]) {
        float4 q = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static inline void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    // streaming (evict-first) store: data not read again soon
    __device__ static inline void store_cs(float* p, const float (&v)[4]) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
    __device__ static inline float round(float v) { return v; }
};

template <>
struct StoreTraits<__nv_bfloat16> {
    using acc_t = float;
    using raw_t = uint4;
    static constexpr int VEC = 8;
    __device__ static inline raw_t ld_raw(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
    __device__ static inline raw_t ld_raw_cs(const __nv_bfloat16* p) {
        return __ldcs(reinterpret_cast<const uint4*>(p));
    }
    __device__ static inline void unpack(const uint4& q, float (&v)[8]) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static inline void unraw(const raw_t& q, float (&v)[8]) { unpack(q, v); }
    __device__ static inline void load(const __nv_bfloat16* p, float (&v)[8]) {
        uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
        unpack(q, v);
    }
    __device__ static inline void load_cs(const __nv_bfloat16* p, float (&v)[8]) {
        uint4 q = __ldcs(reinterpret_cast<const uint4*>(p));
        unpack(q, v);
    }
    __device__ static inline void store(__nv_bfloat16* p, const float (&v)[8]) {
        uint4 q;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        *reinterpret_cast<uint4*>(p) = q;
    }
    __device__ static inline void store_cs(__nv_bfloat16* p, const float (&v)[8]) {
        uint4 q;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        __stcs(reinterpret_cast<uint4*>(p), q);
    }
    // the value the recurrence continues with is the stored (rounded) one
    __device__ static inline float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

template <>
struct StoreTraits<double> {
    using acc_t = double;
    using raw_t = double2;
    static constexpr int VEC = 2;
    __device__ static inline raw_t ld_raw(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
    __device__ static inline raw_t ld_raw_cs(const double* p) { return __ldcs(reinterpret_cast<const double2*>(p)); }
    __device__ static inline void unraw(const raw_t& q, double (&v)[2]) {
        v[0] = q.x; v[1] = q.y;
    }
    __device__ static inline void load(const double* p, double (&v)[2]) {
        double2 q = __ldg(reinterpret_cast<const double2*>(p));
        v[0] = q.x; v[1] = q.y;
    }
    __device__ static inline void load_cs(const double* p, double (&v)[2]) {
        double2 q = __ldcs(reinterpret_cast<const double2*>(p));
        v[0] = q.x; v[1] = q.y;
    }
    __device__ static inline void store(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
    __device__ static inline void store_cs(double* p, const double (&v)[2]) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    }
    __device__ static inline double round(double v) { return v; }
};

// VEC accumulator values (fp32 or fp64) moved as 16-byte chunks; used for the
// fp32/fp64 accumulator Y whose row chunk matches one storage vector.
template <typename A, int VEC>
struct AccIO {
    static constexpr int PER = 16 / sizeof(A);
    static_assert(VEC % PER == 0, "accumulator chunk must be whole 16-byte vectors");
    __device__ static inline void load_cs(const A* p, A (&v)[VEC]) {
#pragma unroll
        for (int q = 0; q < VEC / PER; ++q) {
            A t[PER];
            StoreTraits<A>::load_cs(p + q * PER, t);
#pragma unroll
            for (int i = 0; i < PER; ++i) v[q * PER + i] = t[i];
        }
    }
    __device__ static inline void load(const A* p, A (&v)[VEC]) {
#pragma unroll
        for (int q = 0; q < VEC / PER; ++q) {
            A t[PER];
            StoreTraits<A>::load(p + q * PER, t);
#pragma unroll
            for (int i = 0; i < PER; ++i) v[q * PER + i] = t[i];
        }
    }
    __device__ static inline void store(A* p, const A (&v)[VEC]) {
#pragma unroll
        for (int q = 0; q < VEC / PER; ++q) {
            A t[PER];
#pragma unroll
            for (int i = 0; i < PER; ++i) t[i] = v[q * PER + i];
            StoreTraits<A>::store(p + q * PER, t);
        }
    }
    __device__ static inline void store_cs(A* p, const A (&v)[VEC]) {
#pragma unroll
        for (int q = 0; q < VEC / PER; ++q) {
            A t[PER];
#pragma unroll
            for (int i = 0; i < PER; ++i) t[i] = v[q * PER + i];
            StoreTraits<A>::store_cs(p + q * PER, t);
        }
    }
};

// Packed fp32 pair arithmetic (add.rn.f32x2 / fma.rn.f32x2, one instruction for
// two lanes' worth of values): halves the floating-point instructions of the gather.
__device__ __forceinline__ void add_f32x2(float& a0, float& a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
        "add.rn.f32x2 ra, ra, rb;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fma_f32x2(float& a0, float& a1, float w, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rw;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
        "mov.b64 rw, {%4, %4};\n\tfma.rn.f32x2 ra, rw, rb, ra;\n\tmov.b64 {%0, %1}, ra;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1), "f"(w));
}

// acc += w * x over one vector: packed pairs for fp32 accumulators, scalar fma for fp64.
template <bool WEIGHTED, int VEC>
__device__ __forceinline__ void acc_vec(float (&acc)[VEC], float w, const float (&x)[VEC]) {
#pragma unroll
    for (int v = 0; v < VEC; v += 2) {
        if (WEIGHTED) fma_f32x2(acc[v], acc[v + 1], w, x[v], x[v + 1]);
        else add_f32x2(acc[v], acc[v + 1], x[v], x[v + 1]);
    }
}
template <bool WEIGHTED, int VEC>
__device__ __forceinline__ void acc_vec(double (&acc)[VEC], double w, const double (&x)[VEC]) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = WEIGHTED ? fma(w, x[v], acc[v]) : acc[v] + x[v];
}

// The rows r0 + first, r0 + first + stride, ... below r1 of a CTA's row range, each
// passed to body(row, e0, e1) with its edge range [e0, e1) -- rows with more than
// kHeavyRow edges (common.cuh) are skipped.  The next row's extents are loaded before the current
// row is processed, so the row-pointer load is off the critical path of the gather.
template <typename Body>
__device__ __forceinline__ void for_each_row(const int32_t* __restrict__ rp, int r0, int r1, int stride, Body&& body) {
    int row = r0;
    int e0 = 0, e1 = 0;
    if (row < r1) {
        e0 = __ldg(rp + row);
        e1 = __ldg(rp + row + 1);
    }
    while (row < r1) {
        const int nrow = row + stride;
        int n0 = 0, n1 = 0;
        if (nrow < r1) {
            n0 = __ldg(rp + nrow);
            n1 = __ldg(rp + nrow + 1);
        }
        if (e1 - e0 <= kHeavyRow) body(row, e0, e1);
        row = nrow;
        e0 = n0;
        e1 = n1;
    }
}

// ------------------------------------------------ CSR slice staged in shared memory
// The light part of the CSR in a compact form: lrp[i] (i = 0..N) is the number of
// light-row edges before row i, with bit 31 of lrp[i + 1] set when row i is heavy
// (its edges, left to the one-CTA-per-row kernels, are not in lci); lci holds the
// light rows' column indices back to back.  A CTA whose rows are [r0, r1) copies
// lrp[r0 .. r1] and its rows' indices lci[lrp[r0] .. lrp[r1]) into shared memory with
// asynchronous copies, so that no index load is on the path of a row's gather.
constexpr int32_t kHeavyBit = (int32_t)0x80000000u;
constexpr int32_t kEdgeMask = 0x7fffffff;

__device__ __forceinline__ void cp_async4(int32_t* smem_dst, const int32_t* gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

struct StagedCsr {
    const int32_t* rp;  // shared: lrp[r0 .. r1] as loaded (bit 31 = the previous row is heavy)
    const int32_t* ci;  // shared: the range's light column indices
    int r0, nr, base;
};

// Copies the CSR slice of rows [r0, r1) into smem (which must hold (r1 - r0) + 1 +
// light edges of the range entries) and waits for it with the whole CTA.  Every thread
// of the CTA must call it.
__device__ __forceinline__ StagedCsr stage_csr(const int32_t* __restrict__ lrp, const int32_t* __restrict__ lci,
                                               int r0, int r1, int32_t* smem) {
    const int nr = r1 > r0 ? r1 - r0 : 0;
    const int base = nr ? (__ldg(lrp + r0) & kEdgeMask) : 0;
    const int ne = nr ? (__ldg(lrp + r1) & kEdgeMask) - base : 0;
    int32_t* s_rp = smem;
    int32_t* s_ci = smem + nr + 1;
    for (int i = threadIdx.x; i <= nr && nr; i += blockDim.x) cp_async4(s_rp + i, lrp + r0 + i);
    for (int k = threadIdx.x; k < ne; k += blockDim.x) cp_async4(s_ci + k, lci + base + k);
    cp_async_wait_all();
    __syncthreads();
    StagedCsr c;
    c.rp = s_rp;
    c.ci = s_ci;
    c.r0 = r0;
    c.nr = nr;
    c.base = base;
    return c;
}

// Rows first, first + stride, ... of a staged range, each passed to body(row, e0, e1)
// with its edge range [e0, e1) in c.ci; heavy rows are skipped.
template <typename Body>
__device__ __forceinline__ void for_each_staged_row(const StagedCsr& c, int first, int stride, Body&& body) {
    for (int i = first; i < c.nr; i += stride) {
        const int32_t v1 = c.rp[i + 1];
        if (v1 & kHeavyBit) continue;
        body(c.r0 + i, (c.rp[i] & kEdgeMask) - c.base, v1 - c.base);
    }
}

// One batch of gather_staged: edges e .. e + cnt - 1 (cnt <= BB) with BB load slots.
template <int BB, typename T, int G, int NT, bool WEIGHTED, typename W>
__device__ __forceinline__ void gather_batch(int e, int cnt, const int32_t* ci, const W* __restrict__ wv,
                                             const T* __restrict__ X, int64_t ld, int lane, const bool (&valid)[NT],
                                             typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    const T* rowp[BB];
    A w[BB];
#pragma unroll
    for (int u = 0; u < BB; ++u) {
        const int l = u < cnt ? ci[e + u] : 0;
        rowp[u] = X + (int64_t)l * ld + lane * VEC;
        if (WEIGHTED) w[u] = u < cnt ? A(__ldg(wv + l)) : A(0);
        else w[u] = A(1);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        if (!valid[t]) continue;
        if constexpr (sizeof(T) == 2) {
            // bf16: the loads stay packed (half the registers of their fp32 values) until added
            typename Tr::raw_t q[BB];
#pragma unroll
            for (int u = 0; u < BB; ++u) q[u] = u < cnt ? Tr::ld_raw(rowp[u] + t * G * VEC) : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < BB; ++u) {
                A x[VEC];
                Tr::unraw(q[u], x);
                acc_vec<WEIGHTED, VEC>(acc[t], w[u], x);
            }
        } else {
            A x[BB][VEC];
#pragma unroll
            for (int u = 0; u < BB; ++u) {
                if (u < cnt)
                    Tr::load(rowp[u] + t * G * VEC, x[u]);
                else
#pragma unroll
                    for (int v = 0; v < VEC; ++v) x[u][v] = A(0);
            }
#pragma unroll
            for (int u = 0; u < BB; ++u) acc_vec<WEIGHTED, VEC>(acc[t], w[u], x[u]);
        }
    }
}

// Neighbour sum of one row whose column indices ci[e .. end) are in shared memory
// (see gather_range for acc, G, NT and the weights): every lane of a group reads each
// index itself (one broadcast shared-memory word), so no shuffle or global index load
// precedes the neighbour-row loads.  Edges go in batches of up to B neighbour rows in
// flight; when every lane group of the warp has a short tail (most rows of a power-law
// graph have one to four edges) the batch has 2 or 4 slots, so fewer instructions go to
// empty slots.  The sum runs over the edges in order whatever the batching, so every
// batching gives the same bits.
template <typename T, int G, int NT, bool WEIGHTED, typename W, bool LEAN = false>
__device__ __forceinline__ void gather_staged(int e, const int end, const int32_t* ci, const W* __restrict__ wv,
                                              const T* __restrict__ X, int64_t ld, int lane, int ncols,
                                              typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    // edges in flight per lane: 8 one-vector rows, or 4 rows of NT >= 2 vectors (or in the
    // lean form, LaunchCfg::lean)
    constexpr int B = (NT == 1 && !LEAN) ? 8 : 4;
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[t][v] = A(0);
    bool valid[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) valid[t] = ((t * G + lane) * VEC) < ncols;
    for (; e < end; e += B) {
        const int cnt = min(B, end - e);
        // the batch size follows the largest count among the lanes here, so the lane groups
        // of a warp take the same branch and issue their loads together
        const int most = (int)__reduce_max_sync(__activemask(), (unsigned)cnt);
        if (most > B / 2)
            gather_batch<B, T, G, NT, WEIGHTED, W>(e, cnt, ci, wv, X, ld, lane, valid, acc);
        else if (B == 8 && most > 2)
            gather_batch<4, T, G, NT, WEIGHTED, W>(e, cnt, ci, wv, X, ld, lane, valid, acc);
        else
            gather_batch<2, T, G, NT, WEIGHTED, W>(e, cnt, ci, wv, X, ld, lane, valid, acc);
    }
}

// Neighbour sum of one row: acc[t][v] = sum_{e in row} w_e * X[col[e], c(t, v)] with
// c(t, v) = (t * G + lane) * VEC + v, where w_e = wv[col[e]] if WEIGHTED, else 1
// (the pre-scaled operand form, whose weights are folded into the rows of X).
// The G lanes of a group load a chunk of the row's column indices (and
// weights) with one coalesced access each, then broadcast them by shuffles
// within the group, so the neighbour-row loads of a chunk issue back to back
// without a dependent index load in front of each.  Columns >= ncols are
// skipped (their accumulators stay 0).
template <typename T, int G, int NT, bool WEIGHTED, typename W, bool LEAN = false>
__device__ __forceinline__ void gather_range(int e, const int end, const int32_t* __restrict__ ci,
                                             const W* __restrict__ wv, const T* __restrict__ X, int64_t ld,
                                             int lane, int ncols,
                                             typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    constexpr int J = G >= 16 ? 1 : 16 / G;  // index registers per lane
    constexpr int CH = G * J;                // edges per chunk
    const unsigned gmask =
        G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(G - 1)));
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[t][v] = A(0);
    bool valid[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) valid[t] = ((t * G + lane) * VEC) < ncols;
    for (; e < end; e += CH) {
        int li[J];
        A wi[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int idx = e + j * G + lane;
            const bool ok = idx < end;
            li[j] = ok ? __ldg(ci + idx) : 0;
            if (WEIGHTED) wi[j] = ok ? A(__ldg(wv + li[j])) : A(0);
        }
        const int cnt = min(CH, end - e);
        // edges in flight per lane: 8 one-vector rows, or 4 rows of NT >= 2 vectors (or in
        // the lean form, LaunchCfg::lean)
        constexpr int B = (NT == 1 && !LEAN) ? 8 : 4;
#pragma unroll
        for (int q0 = 0; q0 < CH; q0 += B) {
            if (q0 >= cnt) break;
            int l[B];
            A w[B];
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int q = q0 + u;
                l[u] = __shfl_sync(gmask, li[q / G], q % G, G);
                if (WEIGHTED) w[u] = __shfl_sync(gmask, wi[q / G], q % G, G);
                else w[u] = A(1);
            }
            // one address per neighbour row; the tiles of a lane are fixed offsets from it
            const T* rowp[B];
#pragma unroll
            for (int u = 0; u < B; ++u) rowp[u] = X + (int64_t)l[u] * ld + lane * VEC;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (!valid[t]) continue;
                A x[B][VEC];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    if (q0 + u < cnt)
                        Tr::load(rowp[u] + t * G * VEC, x[u]);
                    else
#pragma unroll
                        for (int v = 0; v < VEC; ++v) x[u][v] = A(0);
                }
#pragma unroll
                for (int u = 0; u < B; ++u) acc_vec<WEIGHTED, VEC>(acc[t], w[u], x[u]);
            }
        }
    }
}

// ------------------------------------------------ row sweeps with either index source
// A row-range kernel reads its rows' column indices either from the CTA's staged slice in
// shared memory (STAGED: one bulk copy at the start, no index load before a gather) or
// straight from global memory (the next row's extents prefetched); the autotuner times
// both, as the staging pays off on short rows (power-law graphs) and costs a start-up
// wait on short ranges.  sweep_rows calls body(row, e0, e1, idx) for the CTA's light rows
// [r0, r1) of lane group threadIdx.x / G, with the row's indices idx[e0 .. e1).
template <bool STAGED, int G, typename Body>
__device__ __forceinline__ void sweep_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                           const int32_t* __restrict__ lrp, const int32_t* __restrict__ lci, int r0,
                                           int r1, int32_t* smem, Body&& body) {
    if constexpr (STAGED) {
        const StagedCsr sc = stage_csr(lrp, lci, r0, r1, smem);
        for_each_staged_row(sc, (int)(threadIdx.x / G), (int)(blockDim.x / G),
                            [&](int row, int e0, int e1) { body(row, e0, e1, sc.ci); });
    } else {
        for_each_row(rp, r0 + (int)(threadIdx.x / G), r1, (int)(blockDim.x / G),
                     [&](int row, int e0, int e1) { body(row, e0, e1, ci); });
    }
}

// The neighbour sum of a whole row (see gather_range).
template <typename T, int G, int NT, bool WEIGHTED, typename W>
__device__ __forceinline__ void gather_row(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                           const W* __restrict__ wv, const T* __restrict__ X, int64_t ld, int row,
                                           int lane, int ncols,
                                           typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    gather_range<T, G, NT, WEIGHTED, W>(__ldg(rp + row), __ldg(rp + row + 1), ci, wv, X, ld, lane, ncols, acc);
}

// The neighbour sum of one light row with indices from either source (see sweep_rows).
template <bool STAGED, typename T, int G, int NT, bool WEIGHTED, typename W, bool LEAN = false>
__device__ __forceinline__ void gather_any(int e0, int e1, const int32_t* idx, const W* __restrict__ wv,
                                           const T* __restrict__ X, int64_t ld, int lane, int ncols,
                                           typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    if constexpr (STAGED) gather_staged<T, G, NT, WEIGHTED, W, LEAN>(e0, e1, idx, wv, X, ld, lane, ncols, acc);
    else gather_range<T, G, NT, WEIGHTED, W, LEAN>(e0, e1, idx, wv, X, ld, lane, ncols, acc);
}

// Neighbour sum of a heavy row (see kHeavyRow) by a whole CTA of kHeavyThreads
// threads: group q takes the q-th contiguous slice of the row's edges; the
// slices' sums are added in a fixed order (a shuffle tree across the groups of a
// warp, then the warps in order through shared memory), and group 0 returns the
// total for its lanes' columns in acc (other groups' acc is unspecified).
constexpr int kHeavyThreads = 256;

template <typename T, int G, int NT, bool WEIGHTED, typename W>
__device__ __forceinline__ void gather_heavy(int e0, int e1, const int32_t* __restrict__ ci, const W* __restrict__ wv,
                                             const T* __restrict__ X, int64_t ld, int lane, int ncols,
                                             typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC]) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    constexpr int WARPS = kHeavyThreads / 32;
    __shared__ A red[WARPS * TW];
    const int groups = kHeavyThreads / G;
    const int q = threadIdx.x / G;
    const int len = (e1 - e0 + groups - 1) / groups;
    const int a = min(e1, e0 + q * len), b = min(e1, a + len);
    gather_range<T, G, NT, WEIGHTED, W>(a, b, ci, wv, X, ld, lane, ncols, acc);
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < VEC; ++v)
#pragma unroll
            for (int o = G; o < 32; o <<= 1) acc[t][v] += __shfl_xor_sync(0xffffffffu, acc[t][v], o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) < G)
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int v = 0; v < VEC; ++v) red[w * TW + (t * G + lane) * VEC + v] = acc[t][v];
    __syncthreads();
    if (q == 0)
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                A s = A(0);
                for (int i = 0; i < WARPS; ++i) s += red[i * TW + (t * G + lane) * VEC + v];
                acc[t][v] = s;
            }
}

// ------------------------------------------------------------ generators
struct Philox4 {
    uint32_t x[4];
};

// Philox4x32-10: ten rounds of two 32x32->64 multiplies with Weyl key bumps.
__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    Philox4 out;
    out.x[0] = c0; out.x[1] = c1; out.x[2] = c2; out.x[3] = c3;
    return out;
}

// u = (x >> 9) * 2^-23 + 2^-24: 23 random bits, exact in fp32, strictly inside (0, 1).
__device__ __forceinline__ float philox_uniform(uint32_t x) {
    return __fmaf_rn((float)(x >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t t) {
    uint64_t z = seed + (t + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------ reductions
// fp64 instructions issue at a small fraction of the fp32 rate on this part, so sums
// that need more than fp32 accuracy run on fp32 pairs: per thread a compensated (Kahan)
// sum (its result carries about one fp32 rounding of its magnitude), between threads an
// unevaluated pair hi + lo added with Knuth's error-free two-sum (the pair additions keep
// about 48 significant bits), converted to fp64 once per block.
struct FF {
    float hi, lo;
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// (a.hi + a.lo) + (b.hi + b.lo): two-sum of the high parts, the low parts and the
// rounding error added to it, renormalised.  No products, so no FMA contraction applies.
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    const float err = (a.hi - (s - bv)) + (b.hi - bv);
    const float t = err + (a.lo + b.lo);
    const float h = s + t;
    return FF{h, t - (h - s)};
}

struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ FF pair() const { return FF{s, -c}; }
};

__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace csc
