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
    static constexpr int VEC = 4;
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
    static constexpr int VEC = 8;
    __device__ static inline void unpack(const uint4& q, float (&v)[8]) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
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
    static constexpr int VEC = 2;
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

// Neighbour sum of one row: acc[t][v] = sum_{e in row} w_e * X[col[e], c(t, v)] with
// c(t, v) = (t * G + lane) * VEC + v, where w_e = wv[col[e]] if WEIGHTED, else 1
// (the pre-scaled operand form, whose weights are folded into the rows of X).
// The G lanes of a group load a chunk of the row's column indices (and
// weights) with one coalesced access each, then broadcast them by shuffles
// within the group, so the neighbour-row loads of a chunk issue back to back
// without a dependent index load in front of each.  Columns >= ncols are
// skipped (their accumulators stay 0).
template <typename T, int G, int NT, bool WEIGHTED, typename W>
__device__ __forceinline__ void gather_row(const int32_t* __restrict__ rp,
                                           const int32_t* __restrict__ ci,
                                           const W* __restrict__ wv, const T* __restrict__ X,
                                           int64_t ld, int row, int lane, int ncols,
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
    int e = __ldg(rp + row);
    const int end = __ldg(rp + row + 1);
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
#pragma unroll
        for (int q0 = 0; q0 < CH; q0 += 4) {
            if (q0 >= cnt) break;
            int l[4];
            A w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u;
                l[u] = __shfl_sync(gmask, li[q / G], q % G, G);
                if (WEIGHTED) w[u] = __shfl_sync(gmask, wi[q / G], q % G, G);
                else w[u] = A(1);
            }
            // one address per neighbour row; the tiles of a lane are fixed offsets from it
            const T* rowp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) rowp[u] = X + (int64_t)l[u] * ld + lane * VEC;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (!valid[t]) continue;
                A x[4][VEC];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (q0 + u < cnt) Tr::load(rowp[u] + t * G * VEC, x[u]);
                    else
#pragma unroll
                        for (int v = 0; v < VEC; ++v) x[u][v] = A(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc_vec<WEIGHTED, VEC>(acc[t], w[u], x[u]);
            }
        }
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
