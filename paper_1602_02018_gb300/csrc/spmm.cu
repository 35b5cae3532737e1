// spmm.cu -- the Jackson-Chebyshev filtering path of Compressive Spectral Clustering.
//
// Kernels (one pass over the graph per polynomial order):
//   degrees_kernel      D_ii = #{j != i : W_ij = 1} and D^-1/2 (Sec. 2.1).
//   gauss_fill_kernel   R ~ N(0, sigma^2) from Philox4x32-10 + Box-Muller (Alg. 2 step 3).
//   cheb_step_kernel    X_{j+1} = 2 (L - I) X_j - X_{j-1} = -2 S X_j - X_{j-1}
//                       (X_1 = -S X_0) fused with Y += c_{j+1} X_{j+1}
//                       (Sec. 2.1 "Fast graph filtering", Alg. 2 step 4).
//   normalize_kernel    Y_i <- Y_i / ||Y_i|| (Alg. 2 step 4), fp64 norm.
//   mom_step_kernel     the same recurrence on probe vectors with fp64 block
//                       partials of <X_{j+1}, X_j> and <X_{j+1}, X_{j+1}>, from which
//                       the eigencount moments of Sec. 4.3 follow by
//                       T_2j = 2 T_j^2 - T_0 and T_2j+1 = 2 T_j+1 T_j - T_1.
//
// Layout: signal blocks are N x ld row-major (ld = padded column count, a
// multiple of the 16-byte vector width), ping-ponged between two scratch
// buffers; X_{j+1} overwrites X_{j-1} in place (each element is read and
// written by the same thread).  The accumulator Y is the caller's output
// buffer, addressed in original node order through `perm`.
#include <math.h>
#include <stdio.h>

#include "common.cuh"
#include "device.cuh"

namespace csc {

// ------------------------------------------------------------------- K4
__global__ void degrees_kernel(const int32_t* __restrict__ rp, int32_t N, int32_t* __restrict__ deg,
                               float* __restrict__ dinv, double* __restrict__ dinv64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int dg = rp[i + 1] - rp[i];
    deg[i] = dg;
    const double r = dg > 0 ? 1.0 / sqrt((double)dg) : 0.0;
    dinv64[i] = r;
    dinv[i] = (float)r;
}

csc_status launch_degrees(Graph* g, cudaStream_t s) {
    if (g->N == 0) return CSC_OK;
    CSC_KLAUNCH("degrees", 4.0 * (g->N + 1) + 16.0 * g->N, s,
                degrees_kernel<<<ceil_div(g->N, 256), 256, 0, s>>>(g->row_ptr, (int32_t)g->N, g->deg, g->dinv,
                                                                   g->dinv64));
    return CSC_OK;
}

// ------------------------------------------------------------------- K3
// One thread per (row, column quad): four normals from one Philox call.
template <typename T>
__global__ void gauss_fill_kernel(T* __restrict__ X, int32_t N, int d, int ld, uint64_t seed,
                                  uint32_t stream, float sigma, const int32_t* __restrict__ perm) {
    using Tr = StoreTraits<T>;
    const int quads = ld / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * quads) return;
    const int row = (int)(t / quads);
    const int q = (int)(t % quads);
    const uint32_t orig = perm ? (uint32_t)perm[row] : (uint32_t)row;
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * q < d) {
        const Philox4 r = philox4x32_10(orig, 0u, (uint32_t)q, 0u, (uint32_t)seed,
                                        (uint32_t)(seed >> 32) ^ stream);
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
    T* dst = X + (int64_t)row * ld + 4 * q;
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v] = (T)z[v];
}

// Copy a caller block R_in (original order, row stride ld_in, fp32) into X (internal order).
template <typename T>
__global__ void copy_in_kernel(T* __restrict__ X, const float* __restrict__ R, int32_t N, int d, int ld,
                               int ld_in, const int32_t* __restrict__ perm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * ld) return;
    const int row = (int)(t / ld);
    const int c = (int)(t % ld);
    const int64_t orig = perm ? perm[row] : row;
    X[t] = (T)(c < d ? R[orig * ld_in + c] : 0.0f);
}

// ------------------------------------------------------------------- K1
template <typename T, int G, int NT>
__global__ void __launch_bounds__(256)
cheb_step_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                 const typename StoreTraits<T>::acc_t* __restrict__ dinv, const T* __restrict__ xcur,
                 T* __restrict__ xprev_next, typename StoreTraits<T>::acc_t* __restrict__ Y,
                 const int32_t* __restrict__ perm, int32_t N, int ncols, int64_t ld,
                 typename StoreTraits<T>::acc_t c0, typename StoreTraits<T>::acc_t c_next, int first) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t r = group; r < N; r += ngroups) {
        const int row = (int)r;
        A acc[NT][VEC];
        gather_row<T, G, NT>(rp, ci, dinv, xcur, ld, row, lane, ncols, acc);
        const A di = dinv[row];
        const int64_t yrow = perm ? (int64_t)perm[row] : (int64_t)row;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * VEC;
            if (c >= ncols) continue;
            A xn[VEC], y[VEC];
            T* xp_ptr = xprev_next + (int64_t)row * ld + c;
            A* y_ptr = Y + yrow * ld + c;
            if (first) {
                A x0[VEC];
                Tr::load(xcur + (int64_t)row * ld + c, x0);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xn[v] = Tr::round(-di * acc[t][v]);
                Tr::store(xp_ptr, xn);
                // Y accumulates the stored (for bf16: rounded) values the recurrence continues with
#pragma unroll
                for (int v = 0; v < VEC; ++v) y[v] = c0 * x0[v] + c_next * xn[v];
            } else {
                A xp[VEC];
                Tr::load_cs(xp_ptr, xp);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xn[v] = Tr::round(A(-2) * di * acc[t][v] - xp[v]);
                Tr::store(xp_ptr, xn);
                AccIO<A, VEC>::load_cs(y_ptr, y);
#pragma unroll
                for (int v = 0; v < VEC; ++v) y[v] = fma(c_next, xn[v], y[v]);
            }
            AccIO<A, VEC>::store(y_ptr, y);
        }
    }
}

// Y = c0 * X0 (degree 0)
template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ X, typename StoreTraits<T>::acc_t* __restrict__ Y,
                                  const int32_t* __restrict__ perm, int32_t N, int ld,
                                  typename StoreTraits<T>::acc_t c0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * ld) return;
    const int row = (int)(t / ld);
    const int c = (int)(t % ld);
    const int64_t yrow = perm ? perm[row] : row;
    Y[yrow * ld + c] = c0 * (typename StoreTraits<T>::acc_t)X[t];
}

// ------------------------------------------------------------------- K5
// One warp per row: fp64 sum of squares of the first d columns, then scale.
template <typename A>
__global__ void normalize_kernel(A* __restrict__ Y, int32_t N, int d, int ld) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < N; row += nwarps) {
        A* y = Y + row * ld;
        double s = 0.0;
        for (int c = lane; c < d; c += 32) {
            const double v = (double)y[c];
            s += v * v;
        }
        s = warp_sum(s);
        if (s > 0.0) {
            const double inv = 1.0 / sqrt(s);
            for (int c = lane; c < d; c += 32) y[c] = (A)((double)y[c] * inv);
        }
    }
}

// ------------------------------------------------------------------- K2
// Moment step: like cheb_step without Y; block partials of three fp64 sums:
//   first: s0 = <X0,X0>, s1 = <X1,X0>, s2 = <X1,X1>
//   later: s1 = <X_{j+1},X_j>, s2 = <X_{j+1},X_{j+1}>
template <typename T, int G, int NT>
__global__ void __launch_bounds__(256)
mom_step_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                const float* __restrict__ dinv, const T* __restrict__ xcur, T* __restrict__ xprev_next,
                int32_t N, int ncols, int64_t ld, int first, double* __restrict__ partials) {
    using Tr = StoreTraits<T>;
    constexpr int VEC = Tr::VEC;
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t r = group; r < N; r += ngroups) {
        const int row = (int)r;
        float acc[NT][VEC];
        gather_row<T, G, NT>(rp, ci, dinv, xcur, ld, row, lane, ncols, acc);
        const float di = dinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * VEC;
            if (c >= ncols) continue;
            float xc[VEC], xn[VEC];
            Tr::load(xcur + (int64_t)row * ld + c, xc);
            T* xp_ptr = xprev_next + (int64_t)row * ld + c;
            if (first) {
#pragma unroll
                for (int v = 0; v < VEC; ++v) xn[v] = Tr::round(-di * acc[t][v]);
            } else {
                float xp[VEC];
                Tr::load_cs(xp_ptr, xp);
#pragma unroll
                for (int v = 0; v < VEC; ++v) xn[v] = Tr::round(-2.0f * di * acc[t][v] - xp[v]);
            }
            Tr::store(xp_ptr, xn);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                s0 += (double)xc[v] * (double)xc[v];
                s1 += (double)xn[v] * (double)xc[v];
                s2 += (double)xn[v] * (double)xn[v];
            }
        }
    }
    __shared__ double red[3][8];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = s0; red[1][w] = s1; red[2][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
        partials[(int64_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// Sum block partials in a fixed order: out[q] = sum_b partials[b*3+q].
__global__ void reduce_partials_kernel(const double* __restrict__ partials, int nblocks,
                                       double* __restrict__ out) {
    __shared__ double red[3][32];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int q = 0; q < 3; ++q) s[q] += partials[(int64_t)b * 3 + q];
    for (int q = 0; q < 3; ++q) s[q] = warp_sum(s[q]);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 3; ++q) red[q][w] = s[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
        out[threadIdx.x] = t;
    }
}

// ------------------------------------------------------------- dispatch
struct TileShape {
    int G, NT;
};

// (G, NT) pairs compiled for the SpMM kernels.
static const TileShape kShapes[] = {{2, 1}, {2, 2}, {2, 3}, {4, 1}, {4, 2}, {4, 3}, {8, 1},
                                    {8, 2}, {8, 3}, {16, 1}, {16, 2}, {32, 1}, {32, 2}};

// Pick the compiled shape covering nv 16-byte vectors per row with the least
// idle lanes; ties go to the group width closest to 8 lanes.
static TileShape choose_shape(int nv) {
    TileShape best{32, 2};
    int best_waste = 1 << 30, best_pref = 1 << 30;
    for (const TileShape& s : kShapes) {
        const int cap = s.G * s.NT;
        if (cap < nv) continue;
        const int waste = cap - nv;
        const int pref = s.G >= 8 ? s.G / 8 : 8 / s.G;
        if (waste < best_waste || (waste == best_waste && pref < best_pref)) {
            best = s;
            best_waste = waste;
            best_pref = pref;
        }
    }
    return best;
}

static int grid_for(Graph* g, int64_t rows, int G) {
    const int64_t groups_per_block = 256 / G;
    int64_t blocks = (rows + groups_per_block - 1) / groups_per_block;
    const int64_t cap = (int64_t)g->num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename T>
static csc_status launch_cheb_step(Graph* g, TileShape sh, const T* xcur, T* xpn,
                                   typename StoreTraits<T>::acc_t* Y, int ncols, int64_t ld,
                                   double c0, double cn, int first, cudaStream_t s) {
    using A = typename StoreTraits<T>::acc_t;
    const A* dv;
    if constexpr (sizeof(A) == 8) dv = g->dinv64; else dv = g->dinv;
    const int grid = grid_for(g, g->N, sh.G);
    // algorithmic bytes of one order: CSR + D^-1/2, X_j gathered once, X_{j-1} read and
    // X_{j+1} written (first order: X_0 read, X_1 written), Y written or read+written
    const double nx = (double)g->N * ncols;
    const double bytes = 4.0 * g->nnz + 4.0 * (g->N + 1) + (double)sizeof(A) * g->N +
                         (first ? 2.0 : 3.0) * nx * sizeof(T) + (first ? 1.0 : 2.0) * nx * sizeof(A);
#define CSC_CHEB_CASE(GG, NN)                                                                    \
    if (sh.G == GG && sh.NT == NN) {                                                             \
        CSC_KLAUNCH("cheb_step", bytes, s,                                                       \
                    cheb_step_kernel<T, GG, NN><<<grid, 256, 0, s>>>(g->row_ptr, g->col_idx, dv, xcur,  \
                                                                     xpn, Y, g->perm, (int32_t)g->N,    \
                                                                     ncols, ld, (A)c0, (A)cn, first));   \
        return CSC_OK;                                                                           \
    }
    CSC_CHEB_CASE(2, 1) CSC_CHEB_CASE(2, 2) CSC_CHEB_CASE(2, 3) CSC_CHEB_CASE(4, 1)
    CSC_CHEB_CASE(4, 2) CSC_CHEB_CASE(4, 3) CSC_CHEB_CASE(8, 1) CSC_CHEB_CASE(8, 2)
    CSC_CHEB_CASE(8, 3) CSC_CHEB_CASE(16, 1) CSC_CHEB_CASE(16, 2) CSC_CHEB_CASE(32, 1)
    CSC_CHEB_CASE(32, 2)
#undef CSC_CHEB_CASE
    set_error("no compiled tile shape G=%d NT=%d", sh.G, sh.NT);
    return CSC_E_UNSUPPORTED;
}

template <typename T>
static csc_status launch_mom_step(Graph* g, TileShape sh, const T* xcur, T* xpn, int ncols, int64_t ld,
                                  int first, double* partials, int grid, cudaStream_t s) {
    const double bytes = 4.0 * g->nnz + 8.0 * g->N + 4.0 + (first ? 2.0 : 3.0) * (double)g->N * ncols * sizeof(T);
#define CSC_MOM_CASE(GG, NN)                                                                     \
    if (sh.G == GG && sh.NT == NN) {                                                             \
        CSC_KLAUNCH("mom_step", bytes, s,                                                        \
                    mom_step_kernel<T, GG, NN><<<grid, 256, 0, s>>>(g->row_ptr, g->col_idx, g->dinv,    \
                                                                    xcur, xpn, (int32_t)g->N, ncols, ld, \
                                                                    first, partials));                   \
        return CSC_OK;                                                                           \
    }
    CSC_MOM_CASE(2, 1) CSC_MOM_CASE(2, 2) CSC_MOM_CASE(2, 3) CSC_MOM_CASE(4, 1)
    CSC_MOM_CASE(4, 2) CSC_MOM_CASE(4, 3) CSC_MOM_CASE(8, 1) CSC_MOM_CASE(8, 2)
    CSC_MOM_CASE(8, 3) CSC_MOM_CASE(16, 1) CSC_MOM_CASE(16, 2) CSC_MOM_CASE(32, 1)
    CSC_MOM_CASE(32, 2)
#undef CSC_MOM_CASE
    set_error("no compiled tile shape G=%d NT=%d", sh.G, sh.NT);
    return CSC_E_UNSUPPORTED;
}

template <typename T>
static csc_status fill_block(Graph* g, T* X, int d, int ld, uint64_t seed, uint32_t stream, float sigma,
                             const float* R_in, int ld_in, cudaStream_t s) {
    const int64_t N = g->N;
    if (R_in) {
        const int64_t tot = N * ld;
        CSC_KLAUNCH("copy_in", (double)tot * (4 + sizeof(T)), s,
                    copy_in_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X, R_in, (int32_t)N, d, ld, ld_in,
                                                                         g->perm));
    } else {
        const int64_t tot = N * (ld / 4);
        CSC_KLAUNCH("gauss_fill", (double)N * ld * sizeof(T), s,
                    gauss_fill_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X, (int32_t)N, d, ld, seed, stream,
                                                                            sigma, g->perm));
    }
    return CSC_OK;
}

template <typename T>
static csc_status filter_typed(Graph* g, const double* c, int m, int d, int d_pad, uint64_t seed,
                               const float* R_in, void* Y_out, bool normalize, cudaStream_t s) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    const int64_t N = g->N;
    const size_t bytes = (size_t)N * d_pad * sizeof(T);
    void *xa = nullptr, *xb = nullptr;
    CSC_TRY(ws_get(g, WS_XA, bytes, &xa));
    CSC_TRY(ws_get(g, WS_XB, bytes, &xb));
    T* X[2] = {(T*)xa, (T*)xb};
    A* Y = (A*)Y_out;
    const float sigma = d > 0 ? (float)(1.0 / sqrt((double)d)) : 1.0f;
    CSC_TRY(fill_block<T>(g, X[0], d, d_pad, seed, STREAM_SIGNALS, sigma, R_in, d_pad, s));
    if (m == 0) {
        const int64_t tot = N * d_pad;
        CSC_KLAUNCH("scale_copy", (double)tot * (sizeof(T) + sizeof(A)), s,
                    scale_copy_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X[0], Y, g->perm, (int32_t)N, d_pad,
                                                                            (A)c[0]));
    } else {
        const TileShape sh = choose_shape(d_pad / VEC);
        CSC_TRY(launch_cheb_step<T>(g, sh, X[0], X[1], Y, d_pad, d_pad, c[0], c[1], 1, s));
        for (int j = 1; j < m; ++j) {
            // X_j lives in X[j & 1]; X_{j-1} (overwritten by X_{j+1}) in the other buffer
            CSC_TRY(launch_cheb_step<T>(g, sh, X[j & 1], X[(j + 1) & 1], Y, d_pad, d_pad, 0.0, c[j + 1], 0, s));
        }
    }
    if (normalize) {
        const int grid = grid_for(g, N, 32);
        CSC_KLAUNCH("normalize", 2.0 * N * d_pad * sizeof(A), s,
                    normalize_kernel<A><<<grid, 256, 0, s>>>(Y, (int32_t)N, d, d_pad));
    }
    return CSC_OK;
}

csc_status run_filter(Graph* g, const double* coeffs, int m, int d, int d_pad, uint64_t seed,
                      csc_dtype storage, const float* R_in, void* Y_out, bool normalize,
                      cudaStream_t s) {
    switch (storage) {
        case CSC_F32:
            return filter_typed<float>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s);
        case CSC_BF16:
            return filter_typed<__nv_bfloat16>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s);
        case CSC_F64:
            return filter_typed<double>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s);
        default:
            set_error("unknown storage type %d", (int)storage);
            return CSC_E_INVALID;
    }
}

template <typename T>
static csc_status moments_typed(Graph* g, int n_moments, int n_probes, uint64_t seed, double* mu,
                                int* passes, cudaStream_t s) {
    constexpr int VEC = StoreTraits<T>::VEC;
    const int64_t N = g->N;
    const int ld = ((n_probes + 7) / 8) * 8;
    const size_t bytes = (size_t)N * ld * sizeof(T);
    void *xa = nullptr, *xb = nullptr, *part = nullptr, *sums = nullptr;
    CSC_TRY(ws_get(g, WS_XA, bytes, &xa));
    CSC_TRY(ws_get(g, WS_XB, bytes, &xb));
    T* X[2] = {(T*)xa, (T*)xb};
    const TileShape sh = choose_shape(ld / VEC);
    const int grid = grid_for(g, N, sh.G);
    // moments 0..M-1 need X_0..X_J with 2J >= M-1
    const int J = n_moments <= 2 ? 1 : n_moments / 2;
    CSC_TRY(ws_get(g, WS_PARTIAL, (size_t)grid * 3 * sizeof(double), &part));
    CSC_TRY(ws_get(g, WS_MOMENTS, (size_t)J * 3 * sizeof(double), &sums));
    double* P = (double*)part;
    double* S = (double*)sums;
    CSC_TRY(fill_block<T>(g, X[0], n_probes, ld, seed, STREAM_PROBES, 1.0f, nullptr, ld, s));
    for (int j = 0; j < J; ++j) {
        CSC_TRY(launch_mom_step<T>(g, sh, X[j & 1], X[(j + 1) & 1], ld, ld, j == 0 ? 1 : 0, P, grid, s));
        CSC_KLAUNCH("reduce", 24.0 * grid, s, reduce_partials_kernel<<<1, 256, 0, s>>>(P, grid, S + 3 * j));
    }
    double* host = g->pinned;
    const size_t nsum = (size_t)J * 3;
    if (nsum > 4096) {
        set_error("too many moments requested (%d)", n_moments);
        return CSC_E_UNSUPPORTED;
    }
    CSC_CUDA_TRY(cudaMemcpyAsync(host, S, nsum * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    const double nv = (double)n_probes;
    // step 0: s0 = <X0,X0>, s1 = <X1,X0>, s2 = <X1,X1>
    const double mu0 = host[0] / nv;
    const double mu1 = host[1] / nv;
    mu[0] = mu0;
    if (n_moments > 1) mu[1] = mu1;
    if (n_moments > 2) mu[2] = 2.0 * host[2] / nv - mu0;
    for (int j = 1; j < J; ++j) {
        const int odd = 2 * j + 1, even = 2 * j + 2;
        if (odd < n_moments) mu[odd] = 2.0 * host[3 * j + 1] / nv - mu1;
        if (even < n_moments) mu[even] = 2.0 * host[3 * j + 2] / nv - mu0;
    }
    if (passes) *passes = J;
    return CSC_OK;
}

csc_status run_moments(Graph* g, int n_moments, int n_probes, uint64_t seed, csc_dtype storage,
                       double* mu_host, int* passes, cudaStream_t s) {
    switch (storage) {
        case CSC_F32:
            return moments_typed<float>(g, n_moments, n_probes, seed, mu_host, passes, s);
        case CSC_BF16:
            return moments_typed<__nv_bfloat16>(g, n_moments, n_probes, seed, mu_host, passes, s);
        default:
            set_error("moments support CSC_F32 and CSC_BF16 storage");
            return CSC_E_UNSUPPORTED;
    }
}

}  // namespace csc
