// spmm.cuh -- pieces shared by the sparse-product translation units (spmm.cu: the
// forward recurrence and the dispatch; spmm_clenshaw.cu: Clenshaw orders;
// spmm_moments.cu: eigencount moment steps): the row factor of the pre-scaled form,
// device coefficient tables, the signal entries from Philox, the compiled tile
// shapes, and the launchers each unit exports.  Each unit compiles its own kernels,
// so the three build in parallel.
#pragma once

#include <math.h>

#include "common.cuh"
#include "device.cuh"

namespace csc {

// s_i of the pre-scaled form: D^-1/2, or 1 for an isolated node
template <typename A>
__device__ __forceinline__ A row_scale(A dinv_i) {
    return dinv_i > A(0) ? dinv_i : A(1);
}

// Filter coefficients read from device memory: c[gid[row] * stride + j] is c_j of
// the row's graph in a batch; with gid == nullptr, c[j] for every row (the form
// replayed by a captured CUDA graph); c == nullptr: the scalar coefficients apply.
template <typename A>
struct CoefTab {
    const A* c = nullptr;
    const int32_t* gid = nullptr;
    int stride = 0;
    int j = 0;                        // index of c_next; c_0 at 0
    const int32_t* gcols = nullptr;   // with gid: columns each graph carries (the rest are not touched)
};

// Entries 4q..4q+3 of row `orig` (original order) of the signal block: Philox4x32-10
// with counter (orig, 0, q, 0) and key (seed_lo, seed_hi ^ stream), Box-Muller on
// the two uniform pairs, times sigma; columns >= d are 0.
__device__ __forceinline__ void gauss_quad(uint32_t orig, int q, int d, uint64_t seed, uint32_t stream, float sigma,
                                           float (&z)[4]) {
    z[0] = z[1] = z[2] = z[3] = 0.f;
    if (4 * q >= d) return;
    const Philox4 r = philox4x32_10(orig, 0u, (uint32_t)q, 0u, (uint32_t)seed, (uint32_t)(seed >> 32) ^ stream);
    const float u0 = philox_uniform(r.x[0]), u1 = philox_uniform(r.x[1]);
    const float u2 = philox_uniform(r.x[2]), u3 = philox_uniform(r.x[3]);
    const float r01 = sqrtf(-2.0f * logf(u0));
    const float r23 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    z[0] = r01 * c1; z[1] = r01 * s1; z[2] = r23 * c3; z[3] = r23 * s3;
#pragma unroll
    for (int v = 0; v < 4; ++v) z[v] = (4 * q + v < d) ? z[v] * sigma : 0.f;
}

// Working sets up to this share of L2 are loaded and stored without evict-first hints.
static const double kKeepL2Fraction = 0.75;

// (G, NT) pairs compiled for the SpMM kernels.
struct TileShape {
    int G, NT;
};
static const TileShape kShapes[] = {{2, 1}, {2, 2}, {2, 3}, {4, 1}, {4, 2}, {4, 3}, {8, 1},
                                    {8, 2}, {8, 3}, {16, 1}, {16, 2}, {32, 1}, {32, 2}};
static const int kThreadChoices[] = {256, 512};

enum KernelKind { KK_CHEB = 1, KK_MOM = 2, KK_CLEN = 4 };

// Expands BODY for the compiled (G, NT) equal to (cfg.G, cfg.NT), with GG / NN bound.
#define CSC_SHAPE_SWITCH(cfg, BODY)                                                       \
    do {                                                                                  \
        switch ((cfg).G * 8 + (cfg).NT) {                                                     \
            case 2 * 8 + 1: { constexpr int GG = 2, NN = 1; BODY; } break;                    \
            case 2 * 8 + 2: { constexpr int GG = 2, NN = 2; BODY; } break;                    \
            case 2 * 8 + 3: { constexpr int GG = 2, NN = 3; BODY; } break;                    \
            case 4 * 8 + 1: { constexpr int GG = 4, NN = 1; BODY; } break;                    \
            case 4 * 8 + 2: { constexpr int GG = 4, NN = 2; BODY; } break;                    \
            case 4 * 8 + 3: { constexpr int GG = 4, NN = 3; BODY; } break;                    \
            case 8 * 8 + 1: { constexpr int GG = 8, NN = 1; BODY; } break;                    \
            case 8 * 8 + 2: { constexpr int GG = 8, NN = 2; BODY; } break;                    \
            case 8 * 8 + 3: { constexpr int GG = 8, NN = 3; BODY; } break;                    \
            case 16 * 8 + 1: { constexpr int GG = 16, NN = 1; BODY; } break;                  \
            case 16 * 8 + 2: { constexpr int GG = 16, NN = 2; BODY; } break;                  \
            case 32 * 8 + 1: { constexpr int GG = 32, NN = 1; BODY; } break;                  \
            case 32 * 8 + 2: { constexpr int GG = 32, NN = 2; BODY; } break;                  \
            default:                                                                          \
                set_error("no compiled tile shape G=%d NT=%d", (cfg).G, (cfg).NT);            \
                return CSC_E_UNSUPPORTED;                                                     \
        }                                                                               \
    } while (0)

// Resident CTAs per SM for a kernel at a block size.
template <typename K>
inline int occupancy(K kernel, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n < 1 ? 1 : n;
}

// One Clenshaw order (spmm_clenshaw.cu); mode bits as in clenshaw_epilogue.  Defined
// for float, __nv_bfloat16 and double storage.
template <typename T>
csc_status launch_clenshaw_step(Graph* g, const LaunchCfg& cfg, const T* bnext, T* bpp,
                                typename StoreTraits<T>::acc_t* Y, int ncols, int64_t ld, double cj, int mode,
                                const T* rs, cudaStream_t s, CoefTab<typename StoreTraits<T>::acc_t> tab = {},
                                bool internal = false);
template <typename T>
int clenshaw_occupancy(const TileShape& sh, int threads, bool lean);

// One eigencount moment step (spmm_moments.cu); float and __nv_bfloat16 storage.
template <typename T>
csc_status launch_mom_step(Graph* g, const LaunchCfg& cfg, const T* xcur, T* xpn, int ncols, int64_t ld, int first,
                           double* partials, cudaStream_t s);
template <typename T>
int mom_occupancy(const TileShape& sh, int threads);

}  // namespace csc
