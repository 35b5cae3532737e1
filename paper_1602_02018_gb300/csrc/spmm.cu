// spmm.cu -- the Jackson-Chebyshev filtering path of Compressive Spectral Clustering.
//
// Kernels here (one pass over the graph per polynomial order):
//   degrees_kernel      D_ii = #{j != i : W_ij = 1} and D^-1/2 (Sec. 2.1).
//   gauss_fill_kernel   R ~ N(0, sigma^2) from Philox4x32-10 + Box-Muller (Alg. 2 step 3).
//   cheb_step_kernel    X_{j+1} = 2 (L - I) X_j - X_{j-1} = -2 S X_j - X_{j-1}
//                       (X_1 = -S X_0) fused with Y += c_{j+1} X_{j+1}
//                       (Sec. 2.1 "Fast graph filtering", Alg. 2 step 4).
//   normalize_kernel    Y_i <- Y_i / ||Y_i|| (Alg. 2 step 4), fp64 norm.
// and the dispatch (launch shapes, autotuner, filter / moment / polynomial drivers).
// The Clenshaw orders live in spmm_clenshaw.cu, the eigencount moment steps
// (mom_step_kernel: the same recurrence on probe vectors with fp64 block partials of
// <X_{j+1}, X_j> and <X_{j+1}, X_{j+1}>, from which the moments of Sec. 4.3 follow by
// T_2j = 2 T_j^2 - T_0 and T_2j+1 = 2 T_j+1 T_j - T_1) in spmm_moments.cu.
//
// Pre-scaled form: the kernels carry Z_j = s X_j with s = D^-1/2 (s_i = 1 for
// an isolated node), for which the recurrence reads
//   Z_{j+1} = -2 D^-1 W Z_j - Z_{j-1},   Z_1 = -D^-1 W Z_0,   Z_0 = s R,
// so the neighbour sum is unweighted: the edge weight 1/sqrt(d_i d_l) is
// carried by the rows of Z and by the row factor 1/d_i, both from the degree
// vector, and no per-edge weight is loaded.  Y = D^1/2 sum_j c_j Z_j: the
// accumulator holds sum_j c_j Z_j until the last order multiplies by sqrt(d_i).
//
// Layout: signal blocks are N x ld row-major (ld = padded column count, a
// multiple of the 16-byte vector width), ping-ponged between two scratch
// buffers; Z_{j+1} overwrites Z_{j-1} in place (each element is read and
// written by the same thread).  The accumulator Y is the caller's output
// buffer, addressed in original node order through `perm`.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "spmm.cuh"

namespace csc {

// ------------------------------------------------------------------- K4
__global__ void degrees_kernel(const int32_t* __restrict__ rp, int32_t N, int32_t* __restrict__ deg,
                               float* __restrict__ dinv, double* __restrict__ dinv64, float* __restrict__ invdeg,
                               float* __restrict__ sqdeg, double* __restrict__ invdeg64,
                               double* __restrict__ sqdeg64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int dg = rp[i + 1] - rp[i];
    deg[i] = dg;
    const double r = dg > 0 ? 1.0 / sqrt((double)dg) : 0.0;
    dinv64[i] = r;
    dinv[i] = (float)r;
    const double id = dg > 0 ? 1.0 / (double)dg : 0.0;
    const double sq = dg > 0 ? sqrt((double)dg) : 1.0;
    invdeg64[i] = id;
    sqdeg64[i] = sq;
    invdeg[i] = (float)id;
    sqdeg[i] = (float)sq;
}

csc_status launch_degrees(Graph* g, cudaStream_t s) {
    if (g->N == 0) return CSC_OK;
    CSC_KLAUNCH("degrees", 4.0 * (g->N + 1) + 40.0 * g->N, s,
                degrees_kernel<<<ceil_div(g->N, 256), 256, 0, s>>>(g->row_ptr, (int32_t)g->N, g->deg, g->dinv,
                                                                   g->dinv64, g->invdeg, g->sqdeg, g->invdeg64,
                                                                   g->sqdeg64));
    return CSC_OK;
}

// ------------------------------------------------------------------- K3
// One thread per (row, column quad): four normals from one Philox call.
// Writes Z_0 = s R (row scale s of the pre-scaled form; `scale` = D^-1/2, NULL for none).
// Block partials of sum_i sum_c R[i, c] Y[i, c] with R regenerated from Philox
// (probe stream, sigma 1) -- the trace estimate of Sec. 4.3 read literally:
// count = (1/n_v) sum_l r_l^T h~(L) r_l.  Y is in original node order.
// partials[3 b] = block sum, partials[3 b + 1 .. 2] = 0 (reduce_partials format).
__global__ void __launch_bounds__(256) probe_trace_kernel(const float* __restrict__ Y, int32_t N, int d, int ld,
                                                          uint64_t seed, double* __restrict__ partials) {
    __shared__ double red[8];
    const int quads = ld / 4;
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * quads;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t / quads), q = (int)(t % quads);
        float z[4];
        gauss_quad((uint32_t)o, q, d, seed, STREAM_PROBES, 1.0f, z);
        const float4 y = *reinterpret_cast<const float4*>(Y + (int64_t)o * ld + 4 * q);
        acc += (double)z[0] * y.x + (double)z[1] * y.y + (double)z[2] * y.z + (double)z[3] * y.w;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        partials[3 * (int64_t)blockIdx.x] = t;
        partials[3 * (int64_t)blockIdx.x + 1] = 0.0;
        partials[3 * (int64_t)blockIdx.x + 2] = 0.0;
    }
}

template <typename T>
__global__ void gauss_fill_kernel(T* __restrict__ X, int32_t N, int d, int ld, uint64_t seed,
                                  uint32_t stream, float sigma, const int32_t* __restrict__ perm,
                                  const typename StoreTraits<T>::acc_t* __restrict__ scale,
                                  CoefTab<typename StoreTraits<T>::acc_t> ftab) {
    using Tr = StoreTraits<T>;
    const int quads = ld / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * quads) return;
    const int row = (int)(t / quads);
    const int q = (int)(t % quads);
    const uint32_t orig = perm ? (uint32_t)perm[row] : (uint32_t)row;
    float z[4];
    gauss_quad(orig, q, d, seed, stream, sigma, z);
    using A = typename Tr::acc_t;
    A sc = scale ? row_scale<A>(scale[row]) : A(1);
    if (ftab.c) sc *= (ftab.gid ? ftab.c + (int64_t)ftab.gid[row] * ftab.stride : ftab.c)[ftab.j];
    T* dst = X + (int64_t)row * ld + 4 * q;
#pragma unroll
    for (int v = 0; v < 4; ++v) dst[v] = (T)((A)z[v] * sc);
}

// Copy a caller block R_in (original order, row stride ld_in, fp32) into X (internal order).
template <typename T>
__global__ void copy_in_kernel(T* __restrict__ X, const float* __restrict__ R, int32_t N, int d, int ld,
                               int ld_in, const int32_t* __restrict__ perm,
                               const typename StoreTraits<T>::acc_t* __restrict__ scale,
                               CoefTab<typename StoreTraits<T>::acc_t> ftab) {
    using A = typename StoreTraits<T>::acc_t;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * ld) return;
    const int row = (int)(t / ld);
    const int c = (int)(t % ld);
    const int64_t orig = perm ? perm[row] : row;
    A sc = scale ? row_scale<A>(scale[row]) : A(1);
    if (ftab.c) sc *= (ftab.gid ? ftab.c + (int64_t)ftab.gid[row] * ftab.stride : ftab.c)[ftab.j];
    X[t] = (T)(c < d ? (A)R[orig * ld_in + c] * sc : A(0));
}

// ------------------------------------------------------------------- K1
// mode bit 1: first order (Z_1 = -D^-1 W Z_0, Y = c_0 Z_0 + c_1 Z_1)
// mode bit 2: last order (Y is brought back to X space: Y *= sqrt(d_i))
//
// Launch shape (all SpMM kernels): CTA x sweeps the contiguous row range
// [part[x], part[x+1]) in order, G lanes per row, so that rows close in the
// node order -- the neighbours in a community, or in a bandwidth-reduced (RCM)
// order -- are gathered by the same CTA while they are in its L1; CTA y covers
// the column tile [y*TW, (y+1)*TW) with TW = G*NT*VEC.  Rows with more than
// kHeavyRow edges are skipped here and done by the *_heavy kernels.

// Operands of one row of a forward order that do not depend on the gather: Z_0 (first
// order) or Z_{j-1}, and the accumulator row of Y (not on the first order); loaded
// before the neighbour sum so their latency overlaps it.
template <typename T, int G, int NT>
struct ChebOperands {
    using A = typename StoreTraits<T>::acc_t;
    typename StoreTraits<T>::raw_t z[NT];
    A y[NT][StoreTraits<T>::VEC];
    __device__ __forceinline__ void load(int row, int lane, int col0, int tcols, int mode, const T* __restrict__ zcur,
                                         const T* __restrict__ zprev, const A* __restrict__ Y,
                                         const int32_t* __restrict__ perm, int64_t ld) {
        using Tr = StoreTraits<T>;
        constexpr int VEC = Tr::VEC;
        const bool first = (mode & 1) != 0, keep = (mode & 4) != 0;
        const int64_t yrow = perm ? (int64_t)perm[row] : (int64_t)row;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * VEC;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            if (first) {
                z[t] = Tr::ld_raw(zcur + o);
            } else {
                z[t] = keep ? Tr::ld_raw(zprev + o) : Tr::ld_raw_cs(zprev + o);
                if (keep) AccIO<A, VEC>::load(Y + yrow * ld + col0 + cl, y[t]);
                else AccIO<A, VEC>::load_cs(Y + yrow * ld + col0 + cl, y[t]);
            }
        }
    }
};

// The per-row update of one order given the row's neighbour sum acc (column tile col0)
// and the row's prefetched operands op.
template <typename T, int G, int NT>
__device__ __forceinline__ void cheb_epilogue(int row, int lane, int col0, int tcols,
                                              typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC],
                                              const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                                              const typename StoreTraits<T>::acc_t* __restrict__ sqdeg,
                                              T* __restrict__ zprev_next,
                                              typename StoreTraits<T>::acc_t* __restrict__ Y,
                                              const int32_t* __restrict__ perm, int64_t ld,
                                              typename StoreTraits<T>::acc_t c0, typename StoreTraits<T>::acc_t c_next,
                                              int mode, const ChebOperands<T, G, NT>& op) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    const bool first = (mode & 1) != 0, last = (mode & 2) != 0;
    const bool keep = (mode & 4) != 0;  // working set fits L2: no evict-first hints
    const A f = (first ? A(-1) : A(-2)) * invdeg[row];
    const A back = last ? sqdeg[row] : A(1);
    const int64_t yrow = perm ? (int64_t)perm[row] : (int64_t)row;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * VEC;
        if (cl >= tcols) continue;
        const int c = col0 + cl;
        A zn[VEC], y[VEC];
        T* zp_ptr = zprev_next + (int64_t)row * ld + c;
        A* y_ptr = Y + yrow * ld + c;
        if (first) {
            A z0[VEC];
            Tr::unraw(op.z[t], z0);
#pragma unroll
            for (int v = 0; v < VEC; ++v) zn[v] = Tr::round(f * acc[t][v]);
            Tr::store(zp_ptr, zn);
            // Y accumulates the stored (for bf16: rounded) values the recurrence continues with
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = (c0 * z0[v] + c_next * zn[v]) * back;
        } else {
            A zp[VEC];
            Tr::unraw(op.z[t], zp);
#pragma unroll
            for (int v = 0; v < VEC; ++v) zn[v] = Tr::round(f * acc[t][v] - zp[v]);
            Tr::store(zp_ptr, zn);
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = fma(c_next, zn[v], op.y[t][v]) * back;
        }
        // Y is read again only by the next order: evict-first keeps Z_j resident in L2
        // (unless everything fits there)
        if (keep) AccIO<A, VEC>::store(y_ptr, y);
        else AccIO<A, VEC>::store_cs(y_ptr, y);
    }
}

template <typename T, int G, int NT, bool STAGED>
__global__ void __launch_bounds__(512)
cheb_step_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ lrp,
                 const int32_t* __restrict__ lci,
                 const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                 const typename StoreTraits<T>::acc_t* __restrict__ sqdeg, const T* __restrict__ zcur,
                 T* __restrict__ zprev_next, typename StoreTraits<T>::acc_t* __restrict__ Y,
                 const int32_t* __restrict__ perm, const int32_t* __restrict__ part, int ncols, int64_t ld,
                 typename StoreTraits<T>::acc_t c0, typename StoreTraits<T>::acc_t c_next, int mode,
                 CoefTab<typename StoreTraits<T>::acc_t> tab) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int tcols = min(TW, ncols - col0);
    const int r0 = part[blockIdx.x], r1 = part[blockIdx.x + 1];
    if (tab.c && r0 < r1) {  // a batch's row range lies inside one graph
        const A* cg = tab.gid ? tab.c + (int64_t)tab.gid[r0] * tab.stride : tab.c;
        c0 = cg[0];
        c_next = cg[tab.j];
    }
    extern __shared__ int32_t s_csr[];
    sweep_rows<STAGED, G>(rp, ci, lrp, lci, r0, r1, s_csr, [&](int row, int e0, int e1, const int32_t* idx) {
        ChebOperands<T, G, NT> op;
        op.load(row, lane, col0, tcols, mode, zcur, zprev_next, Y, perm, ld);
        A acc[NT][VEC];
        gather_any<STAGED, T, G, NT, false, A>(e0, e1, idx, nullptr, zcur + col0, ld, lane, tcols, acc);
        cheb_epilogue<T, G, NT>(row, lane, col0, tcols, acc, invdeg, sqdeg, zprev_next, Y, perm, ld, c0, c_next, mode,
                                op);
    });
}

// Heavy rows: one CTA (kHeavyThreads threads) per row, its groups splitting the edges.
template <typename T, int G, int NT>
__global__ void __launch_bounds__(kHeavyThreads)
cheb_step_heavy_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                       const typename StoreTraits<T>::acc_t* __restrict__ sqdeg, const T* __restrict__ zcur,
                       T* __restrict__ zprev_next, typename StoreTraits<T>::acc_t* __restrict__ Y,
                       const int32_t* __restrict__ perm, const int32_t* __restrict__ heavy, int ncols, int64_t ld,
                       typename StoreTraits<T>::acc_t c0, typename StoreTraits<T>::acc_t c_next, int mode,
                       CoefTab<typename StoreTraits<T>::acc_t> tab) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int tcols = min(TW, ncols - col0);
    const int row = heavy[blockIdx.x];
    if (tab.c) {
        const A* cg = tab.gid ? tab.c + (int64_t)tab.gid[row] * tab.stride : tab.c;
        c0 = cg[0];
        c_next = cg[tab.j];
    }
    A acc[NT][VEC];
    gather_heavy<T, G, NT, false, A>(__ldg(rp + row), __ldg(rp + row + 1), ci, nullptr, zcur + col0, ld, lane, tcols,
                                     acc);
    if (threadIdx.x < G) {
        ChebOperands<T, G, NT> op;
        op.load(row, lane, col0, tcols, mode, zcur, zprev_next, Y, perm, ld);
        cheb_epilogue<T, G, NT>(row, lane, col0, tcols, acc, invdeg, sqdeg, zprev_next, Y, perm, ld, c0, c_next, mode,
                                op);
    }
}

template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ X, typename StoreTraits<T>::acc_t* __restrict__ Y,
                                  const int32_t* __restrict__ perm, int32_t N, int ld,
                                  typename StoreTraits<T>::acc_t c0,
                                  const typename StoreTraits<T>::acc_t* __restrict__ sqdeg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * ld) return;
    const int row = (int)(t / ld);
    const int c = (int)(t % ld);
    const int64_t yrow = perm ? perm[row] : row;
    Y[yrow * ld + c] = c0 * (typename StoreTraits<T>::acc_t)X[t] * sqdeg[row];
}

// ------------------------------------------------------------------- K5
// One warp per row: fp64 sum of squares of the first d columns, then scale.
// score (optional) receives the sum of squares ||Y_i||^2, the coherence estimate
// of the remark closing Sec. 4.2; scale = 0 leaves Y as it is.
template <typename A>
__global__ void normalize_kernel(A* __restrict__ Y, int32_t N, int d, int ld, double* __restrict__ score, int scale) {
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
        if (score && lane == 0) score[row] = s;
        if (scale && s > 0.0) {
            const double inv = 1.0 / sqrt(s);
            for (int c = lane; c < d; c += 32) y[c] = (A)((double)y[c] * inv);
        }
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

// Per-graph sums of the block partials of one step, in a fixed order: block g adds,
// for each column tile, the slots of its graph's row ranges [gblk[g], gblk[g+1]) and
// then those of its heavy rows [ghvy[g], ghvy[g+1]) (slot layout of mom_step_kernel /
// mom_step_heavy_kernel).  nseg = 1 sums everything (gblk, ghvy unused).
// out[(g * J + j) * 3 + q].
__global__ void __launch_bounds__(256) segment_partials_kernel(const double* __restrict__ partials, int P, int tiles,
                                                               int H, const int32_t* __restrict__ gblk,
                                                               const int32_t* __restrict__ ghvy, int nseg, int j,
                                                               int J, double* __restrict__ out) {
    __shared__ double red[3][8];
    const int gi = blockIdx.x;
    const int b0 = nseg == 1 ? 0 : gblk[gi], b1 = nseg == 1 ? P : gblk[gi + 1];
    const int h0 = nseg == 1 ? 0 : ghvy[gi], h1 = nseg == 1 ? H : ghvy[gi + 1];
    const int nb = b1 - b0, nh = h1 - h0;
    const int per_tile = nb + nh;
    double a[3] = {0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < per_tile * tiles; t += blockDim.x) {
        const int y = t / per_tile, i = t % per_tile;
        const int64_t slot = i < nb ? (int64_t)y * P + b0 + i : (int64_t)P * tiles + (int64_t)y * H + h0 + (i - nb);
        for (int q = 0; q < 3; ++q) a[q] += partials[slot * 3 + q];
    }
    for (int q = 0; q < 3; ++q) a[q] = warp_sum(a[q]);
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 3; ++q) red[q][threadIdx.x >> 5] = a[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        out[((int64_t)gi * J + j) * 3 + threadIdx.x] = t;
    }
}

template <typename T>
static csc_status launch_cheb_step(Graph* g, const LaunchCfg& cfg, const T* xcur, T* xpn,
                                   typename StoreTraits<T>::acc_t* Y, int ncols, int64_t ld,
                                   double c0, double cn, int mode, cudaStream_t s,
                                   CoefTab<typename StoreTraits<T>::acc_t> tab = {}) {
    using A = typename StoreTraits<T>::acc_t;
    const A *idg, *sqd;
    if constexpr (sizeof(A) == 8) {
        idg = g->invdeg64;
        sqd = g->sqdeg64;
    } else {
        idg = g->invdeg;
        sqd = g->sqdeg;
    }
    const int first = mode & 1;
    // Z_j, Z_{j-1}, Y and the CSR within three quarters of L2: plain caching
    const double ws = (double)g->N * ld * (2.0 * sizeof(T) + sizeof(A)) + 4.0 * g->nnz + 8.0 * g->N;
    if (ws <= kKeepL2Fraction * (double)g->l2_bytes) mode |= 4;
    const int32_t* part = nullptr;
    CSC_TRY(get_partition(g, cfg.P, &part));
    const int smem = cfg.staged ? staged_smem(g, cfg.P) : 0;  // the CTA's CSR slice (stage_csr)
    CSC_TRY(check_staged_smem(smem));
    const dim3 grid(cfg.P, cfg.tiles);
    // algorithmic bytes of one order: CSR + row factors, Z_j gathered once, Z_{j-1} read and
    // Z_{j+1} written (first order: Z_0 read, Z_1 written), Y written or read+written;
    // split between the row-range launch and the heavy-row launch by their edges and rows
    const double nx = (double)g->N * ncols;
    const double all_bytes = 4.0 * g->nnz + 4.0 * (g->N + 1) + (double)sizeof(A) * g->N * (mode & 2 ? 2 : 1) +
                             (first ? 2.0 : 3.0) * nx * sizeof(T) + (first ? 1.0 : 2.0) * nx * sizeof(A);
    const double heavy_edges = (double)g->nnz - (double)g->h_light[g->N];
    const double heavy_frac = g->n_heavy ? (heavy_edges + g->n_heavy) / ((double)g->nnz + g->N) : 0.0;
    const double bytes = all_bytes * (1.0 - heavy_frac);
    const dim3 hgrid(g->n_heavy > 0 ? g->n_heavy : 1, cfg.tiles);
    auto heavy = [&](cudaStream_t st) -> csc_status {
        CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("cheb_step_heavy", all_bytes * heavy_frac, st,
                                          cheb_step_heavy_kernel<T, GG, NN><<<hgrid, kHeavyThreads, 0, st>>>(
                                              g->row_ptr, g->col_idx, idg, sqd, xcur, xpn, Y, g->perm, g->heavy,
                                              ncols, ld, (A)c0, (A)cn, mode, tab)));
        return CSC_OK;
    };
    auto light = [&](cudaStream_t st) -> csc_status {
        if (cfg.staged)
            CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("cheb_step", bytes, st,
                                              cheb_step_kernel<T, GG, NN, true><<<grid, cfg.threads, smem, st>>>(
                                                  g->row_ptr, g->col_idx, g->lrp, g->lci, idg, sqd, xcur, xpn, Y,
                                                  g->perm, part, ncols, ld, (A)c0, (A)cn, mode, tab)));
        else
            CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("cheb_step", bytes, st,
                                              cheb_step_kernel<T, GG, NN, false><<<grid, cfg.threads, 0, st>>>(
                                                  g->row_ptr, g->col_idx, g->lrp, g->lci, idg, sqd, xcur, xpn, Y,
                                                  g->perm, part, ncols, ld, (A)c0, (A)cn, mode, tab)));
        return CSC_OK;
    };
    return fork_join(g, s, g->n_heavy > 0, heavy, light);
}

template <typename T>
static int kernel_occupancy(int kind, const TileShape& sh, int threads, bool lean = false) {
    if (kind == KK_CLEN) return clenshaw_occupancy<T>(sh, threads, lean);
    if (kind == KK_MOM) {
        if constexpr (sizeof(T) <= 4) return mom_occupancy<T>(sh, threads);
        return 1;
    }
    int occ = 1;
#define CSC_OCC_CASE(GG, NN) \
    if (sh.G == GG && sh.NT == NN) occ = occupancy(cheb_step_kernel<T, GG, NN, true>, threads);
    CSC_OCC_CASE(2, 1) CSC_OCC_CASE(2, 2) CSC_OCC_CASE(2, 3) CSC_OCC_CASE(4, 1) CSC_OCC_CASE(4, 2)
    CSC_OCC_CASE(4, 3) CSC_OCC_CASE(8, 1) CSC_OCC_CASE(8, 2) CSC_OCC_CASE(8, 3) CSC_OCC_CASE(16, 1)
    CSC_OCC_CASE(16, 2) CSC_OCC_CASE(32, 1) CSC_OCC_CASE(32, 2)
#undef CSC_OCC_CASE
    return occ;
}


// Candidate launch shapes for nv 16-byte vectors per row: every compiled (G, NT)
// whose column tiles leave at most a third of their lanes idle, at each block size,
// with one CTA per row range and tile for every resident CTA slot of the GPU.
template <typename T>
static std::vector<LaunchCfg> candidates(Graph* g, int kind, int nv) {
    std::vector<LaunchCfg> out;
    // narrow rows (a few vectors) cannot fill any group: then the least-waste shapes are kept
    int min_waste = 1 << 30;
    for (const TileShape& sh : kShapes) {
        const int cap = sh.G * sh.NT;
        const int tiles = (nv + cap - 1) / cap;
        if (tiles <= 16) min_waste = std::min(min_waste, tiles * cap - nv);
    }
    for (const TileShape& sh : kShapes) {
        const int cap = sh.G * sh.NT;
        const int tiles = (nv + cap - 1) / cap;
        if (tiles > 16) continue;
        const int waste = tiles * cap - nv;
        if (3 * waste > tiles * cap && waste > min_waste) continue;
        for (int th : kThreadChoices) {
            // the lean form (LaunchCfg::lean) exists for the Clenshaw orders, NT = 1, 256 threads
            for (int lean = 0; lean <= 1; ++lean) {
                if (lean && !(kind == KK_CLEN && sh.NT == 1 && th == 256)) continue;
                LaunchCfg c;
                c.G = sh.G;
                c.NT = sh.NT;
                c.threads = th;
                c.tiles = tiles;
                c.lean = lean;
                const int occ = kernel_occupancy<T>(kind, sh, th, lean != 0);
                const int64_t max_p = (g->N + (th / sh.G) - 1) / (th / sh.G);  // at least one row per group
                // one to eight waves of resident CTAs: more, shorter row ranges balance SMs that
                // run at different speeds (distance to the memory holding their rows)
                for (int waves = 1; waves <= 8; waves *= 2) {
                    int P = (g->num_sms * occ * waves + tiles - 1) / tiles;
                    if (P > max_p) P = (int)max_p;
                    if (P < g->n_graphs) P = g->n_graphs;  // a batch needs a range per graph
                    P = P < 1 ? 1 : P;
                    // the CTA's staged CSR slice must fit shared memory: more, shorter ranges if not
                    if (fit_staged_partition(g, P, std::max<int64_t>(max_p, g->n_graphs), &P) != CSC_OK ||
                        staged_smem(g, P) > kStagedSmemMax)
                        continue;
                    c.P = P;
                    if (!out.empty() && out.back().G == c.G && out.back().NT == c.NT &&
                        out.back().threads == th && out.back().lean == lean && out.back().P == c.P)
                        continue;
                    // both index sources (sweep_rows): the staged slice, and global loads
                    c.staged = 1;
                    out.push_back(c);
                    c.staged = 0;
                    out.push_back(c);
                }
            }
        }
    }
    return out;
}

// Time each candidate (3 launches after one warm-up) and keep the fastest.  `run`
// launches one candidate on scratch data of the real problem.
template <typename RunFn>
static csc_status autotune(Graph* g, uint64_t key, const std::vector<LaunchCfg>& cands, cudaStream_t s,
                           RunFn run, LaunchCfg* out) {
    auto it = g->tuned.find(key);
    if (it != g->tuned.end()) {
        *out = it->second;
        return CSC_OK;
    }
    if (tune_cache_get(g, key, out)) {
        g->tuned[key] = *out;
        return CSC_OK;
    }
    if (cands.empty()) {
        set_error("autotune: no launch shape fits");
        return CSC_E_UNSUPPORTED;
    }
    const bool prof = g_prof_enabled;
    g_prof_enabled = false;  // tuning launches are not part of the measured work
    cudaEvent_t a = g->ev[0], b = g->ev[1];
    float best_ms = 1e30f;
    LaunchCfg best = cands[0];
    csc_status st = CSC_OK;
    for (const LaunchCfg& c : cands) {
        st = run(c);
        if (st != CSC_OK) break;
        cudaEventRecord(a, s);
        for (int r = 0; r < 3 && st == CSC_OK; ++r) st = run(c);
        cudaEventRecord(b, s);
        if (st != CSC_OK) break;
        if (cudaEventSynchronize(b) != cudaSuccess) {
            st = CSC_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    g_prof_enabled = prof;
    if (st != CSC_OK) return st;
    g->tuned[key] = best;
    tune_cache_put(g, key, best);
    *out = best;
    return CSC_OK;
}

static uint64_t tune_key(int kind, int dtype, int ncols) {
    return ((uint64_t)kind << 48) | ((uint64_t)(dtype & 0xff) << 40) | (uint64_t)(uint32_t)ncols;
}

template <typename T>
static csc_status fill_block(Graph* g, T* X, int d, int ld, uint64_t seed, uint32_t stream, float sigma,
                             const float* R_in, int ld_in, cudaStream_t s,
                             CoefTab<typename StoreTraits<T>::acc_t> ftab = {}) {
    using A = typename StoreTraits<T>::acc_t;
    const int64_t N = g->N;
    const A* scale;  // Z_0 = D^-1/2 R (row factor 1 for isolated nodes)
    if constexpr (sizeof(A) == 8) scale = g->dinv64; else scale = g->dinv;
    if (R_in) {
        const int64_t tot = N * ld;
        CSC_KLAUNCH("copy_in", (double)tot * (4 + sizeof(T)), s,
                    copy_in_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X, R_in, (int32_t)N, d, ld, ld_in,
                                                                         g->perm, scale, ftab));
    } else {
        const int64_t tot = N * (ld / 4);
        CSC_KLAUNCH("gauss_fill", (double)N * ld * sizeof(T), s,
                    gauss_fill_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X, (int32_t)N, d, ld, seed, stream,
                                                                            sigma, g->perm, scale, ftab));
    }
    return CSC_OK;
}

template <typename T>
static csc_status filter_typed(Graph* g, const double* c, int m, int d, int d_pad, uint64_t seed,
                               const float* R_in, void* Y_out, bool normalize, cudaStream_t s,
                               uint32_t rng_stream = STREAM_SIGNALS, float sigma_override = 0.f,
                               const double* c_graphs = nullptr, bool clenshaw = false) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    const int64_t N = g->N;
    const size_t bytes = (size_t)N * d_pad * sizeof(T);
    void *xa = nullptr, *xb = nullptr;
    CSC_TRY(ws_get(g, WS_XA, bytes, &xa));
    CSC_TRY(ws_get(g, WS_XB, bytes, &xb));
    T* X[2] = {(T*)xa, (T*)xb};
    A* Y = (A*)Y_out;
    const float sigma = sigma_override > 0.f ? sigma_override : d > 0 ? (float)(1.0 / sqrt((double)d)) : 1.0f;
    CoefTab<A> tab;
    if (c_graphs) {
        // per-graph coefficients, G x (m + 1), in the accumulator type
        const int G = g->n_graphs;
        if (m == 0 || !g->graph_of_row) {
            set_error("per-graph filter coefficients need m >= 1 and a batched handle");
            return CSC_E_UNSUPPORTED;
        }
        std::vector<A> h((size_t)G * (m + 1));
        for (size_t i = 0; i < h.size(); ++i) h[i] = (A)c_graphs[i];
        void* dc = nullptr;
        CSC_TRY(ws_get(g, WS_COEF, h.size() * sizeof(A), &dc));
        CSC_CUDA_TRY(cudaMemcpyAsync(dc, h.data(), h.size() * sizeof(A), cudaMemcpyHostToDevice, s));
        // the host copy dies with this frame: wait for the copy
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        tab.c = (const A*)dc;
        tab.gid = g->graph_of_row;
        tab.stride = m + 1;
    }
    const bool graphs = !g_prof_enabled && m >= 2 && g->use_graphs;
    if (m == 0) {
        CSC_TRY(fill_block<T>(g, X[0], d, d_pad, seed, rng_stream, sigma, R_in, d_pad, s));
        const int64_t tot = N * d_pad;
        const A* sqd;
        if constexpr (sizeof(A) == 8) sqd = g->sqdeg64; else sqd = g->sqdeg;
        CSC_KLAUNCH("scale_copy", (double)tot * (sizeof(T) + sizeof(A)), s,
                    scale_copy_kernel<T><<<ceil_div(tot, 256), 256, 0, s>>>(X[0], Y, g->perm, (int32_t)N, d_pad,
                                                                            (A)c[0], sqd));
    } else if (!clenshaw) {
        CSC_TRY(fill_block<T>(g, X[0], d, d_pad, seed, rng_stream, sigma, R_in, d_pad, s));
        // launch shape tuned once per handle on this graph: trial orders read Z_0 and write
        // scratch (the Z_1 buffer and Y are overwritten by the first real order)
        LaunchCfg cfg;
        CSC_TRY(autotune(g, tune_key(KK_CHEB, (int)sizeof(T), d_pad), candidates<T>(g, KK_CHEB, d_pad / VEC), s,
                         [&](const LaunchCfg& c) {
                             return launch_cheb_step<T>(g, c, X[0], X[1], Y, d_pad, d_pad, 0.0, 0.0, 0, s);
                         },
                         &cfg));
        // the m orders; replayed from a captured CUDA graph when no per-launch timing is
        // asked for (one launch instead of m, no launch gaps between orders)
        auto orders = [&](cudaStream_t st, CoefTab<A> tb) -> csc_status {
            tb.j = 1;
            CSC_TRY(launch_cheb_step<T>(g, cfg, X[0], X[1], Y, d_pad, d_pad, c ? c[0] : 0.0, c ? c[1] : 0.0,
                                        1 | (m == 1 ? 2 : 0), st, tb));
            for (int j = 1; j < m; ++j) {
                // Z_j lives in X[j & 1]; Z_{j-1} (overwritten by Z_{j+1}) in the other buffer
                tb.j = j + 1;
                CSC_TRY(launch_cheb_step<T>(g, cfg, X[j & 1], X[(j + 1) & 1], Y, d_pad, d_pad, 0.0,
                                            c ? c[j + 1] : 0.0, j == m - 1 ? 2 : 0, st, tb));
            }
            return CSC_OK;
        };
        if (!tab.c && graphs) {
            // coefficients to a device array the graph reads (stream-ordered before the replay)
            std::vector<A> hc(m + 1);
            for (int j = 0; j <= m; ++j) hc[j] = (A)c[j];
            void* dc = nullptr;
            CSC_TRY(ws_get(g, WS_COEF1, (m + 1) * sizeof(A), &dc));
            CSC_CUDA_TRY(cudaMemcpyAsync(dc, hc.data(), (m + 1) * sizeof(A), cudaMemcpyHostToDevice, s));
            CoefTab<A> gt;
            gt.c = (const A*)dc;
            char key[256];
            snprintf(key, sizeof(key), "cheb:%zu:%d:%d:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p", sizeof(T), d_pad, m, cfg.G,
                     cfg.NT, cfg.threads, cfg.P, cfg.tiles, cfg.staged, (void*)X[0], (void*)X[1], (void*)Y, dc);
            int64_t launches = 0;
            const int32_t* pr = nullptr;
            CSC_TRY(get_partition(g, cfg.P, &pr));  // before the capture
            CSC_TRY(replay_graph(g, key, s, &launches, [&](cudaStream_t cap) { return orders(cap, gt); }));
            (void)launches;
        } else {
            CSC_TRY(orders(s, tab));
        }
    } else {
        // Clenshaw form: coefficients always from device memory (per graph in a batch)
        if (!tab.c) {
            std::vector<A> hc(m + 1);
            for (int j = 0; j <= m; ++j) hc[j] = (A)c[j];
            void* dc = nullptr;
            CSC_TRY(ws_get(g, WS_COEF1, (m + 1) * sizeof(A), &dc));
            CSC_CUDA_TRY(cudaMemcpyAsync(dc, hc.data(), (m + 1) * sizeof(A), cudaMemcpyHostToDevice, s));
            tab.c = (const A*)dc;
        }
        // B_m = c_m s R, and s R itself in a third buffer that every order reads (recomputing
        // it from Philox inside every order instead was slower: 39.6 against 28.3 ms for the
        // filter of the power-law workload)
        CoefTab<A> ft = tab;
        ft.j = m;
        CSC_TRY(fill_block<T>(g, X[0], d, d_pad, seed, rng_stream, sigma, R_in, d_pad, s, ft));
        void* xr = nullptr;
        CSC_TRY(ws_get(g, WS_XR, bytes, &xr));
        T* RS = (T*)xr;
        CSC_TRY(fill_block<T>(g, RS, d, d_pad, seed, rng_stream, sigma, R_in, d_pad, s));
        LaunchCfg cfg;
        // timed on a middle order (B_{j+2} read, B_j written in place); the contents of the
        // scratch blocks do not matter for the timing, and B_m in X[0] is only read
        CSC_TRY(autotune(g, tune_key(KK_CLEN, (int)sizeof(T), d_pad), candidates<T>(g, KK_CLEN, d_pad / VEC), s,
                         [&](const LaunchCfg& c) {
                             return launch_clenshaw_step<T>(g, c, X[0], X[1], Y, d_pad, d_pad, 0.0, 0, RS, s);
                         },
                         &cfg));
        const bool fused_norm = normalize && cfg.tiles == 1;
        auto orders = [&](cudaStream_t st) -> csc_status {
            CoefTab<A> tb = tab;
            // B_j lives in X[(m - j) & 1]; B_{j+2} (overwritten by B_j) in the same buffer
            for (int j = m - 1; j >= 1; --j) {
                tb.j = j;
                CSC_TRY(launch_clenshaw_step<T>(g, cfg, X[(m - j - 1) & 1], X[(m - j) & 1], Y, d_pad, d_pad, 0.0,
                                                j == m - 1 ? 1 : 0, RS, st, tb));
            }
            tb.j = 0;
            return launch_clenshaw_step<T>(g, cfg, X[(m - 1) & 1], X[m & 1], Y, d_pad, d_pad, 0.0,
                                           2 | (m == 1 ? 1 : 0) | (fused_norm ? 8 : 0), RS, st, tb);
        };
        if (graphs) {
            char key[320];
            snprintf(key, sizeof(key), "clen:%zu:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p", sizeof(T), d_pad, m,
                     d, (int)fused_norm, cfg.G, cfg.NT, cfg.threads, cfg.P, cfg.tiles, cfg.staged, cfg.lean,
                     (const void*)RS, (void*)X[0], (void*)X[1], (void*)Y, (const void*)tab.c);
            int64_t launches = 0;
            const int32_t* pr = nullptr;
            CSC_TRY(get_partition(g, cfg.P, &pr));  // before the capture
            CSC_TRY(replay_graph(g, key, s, &launches, orders));
        } else {
            CSC_TRY(orders(s));
        }
        if (fused_norm) return CSC_OK;
    }
    if (normalize) {
        int grid = ceil_div(N, 8);
        if (grid > g->num_sms * 8) grid = g->num_sms * 8;
        CSC_KLAUNCH("normalize", 2.0 * N * d_pad * sizeof(A), s,
                    normalize_kernel<A><<<grid, 256, 0, s>>>(Y, (int32_t)N, d, d_pad, nullptr, 1));
    }
    return CSC_OK;
}

csc_status run_filter_batched(Graph* g, const double* c_graphs, int m, int d, int d_pad, uint64_t seed,
                              csc_dtype storage, const float* R_in, void* Y_out, bool normalize, cudaStream_t s,
                              bool clenshaw) {
    switch (storage) {
        case CSC_F32:
            return filter_typed<float>(g, nullptr, m, d, d_pad, seed, R_in, Y_out, normalize, s, STREAM_SIGNALS, 0.f,
                                       c_graphs, clenshaw);
        case CSC_BF16:
            return filter_typed<__nv_bfloat16>(g, nullptr, m, d, d_pad, seed, R_in, Y_out, normalize, s,
                                               STREAM_SIGNALS, 0.f, c_graphs, clenshaw);
        case CSC_F64:
            return filter_typed<double>(g, nullptr, m, d, d_pad, seed, R_in, Y_out, normalize, s, STREAM_SIGNALS,
                                        0.f, c_graphs, clenshaw);
        default:
            set_error("unknown storage type %d", (int)storage);
            return CSC_E_INVALID;
    }
}

// ---------------------------------------------- h~(L) on a block in internal order
// Used by the interpolation with g = 1 - h~: Y = sum_j c_j T_j(L - I) X for an fp32
// block X already in internal row order (stride ld, all ld columns), Y likewise, by
// the Clenshaw form.  poly_prepare uploads the coefficients and settles the launch
// shape (it may synchronize); poly_apply only launches, so it can be captured.
csc_status poly_prepare(Graph* g, const double* c, int m, int ld, PolyOp* op, cudaStream_t s, int n_coef) {
    if (m < 1 || ld % 4 || n_coef < 1 || (n_coef > 1 && n_coef != g->n_graphs)) {
        set_error("polynomial operator: need m >= 1, ld a multiple of 4 and one coefficient row or one per graph");
        return CSC_E_INVALID;
    }
    const size_t bytes = (size_t)g->N * ld * sizeof(float);
    void *a = nullptr, *b = nullptr, *r = nullptr, *dc = nullptr;
    CSC_TRY(ws_get(g, WS_XA, bytes, &a));
    CSC_TRY(ws_get(g, WS_XB, bytes, &b));
    CSC_TRY(ws_get(g, WS_XR, bytes, &r));
    const size_t nc = (size_t)n_coef * (m + 1);
    CSC_TRY(ws_get(g, WS_COEF1, nc * sizeof(float), &dc));
    std::vector<float> hc(nc);
    for (size_t j = 0; j < nc; ++j) hc[j] = (float)c[j];
    CSC_CUDA_TRY(cudaMemcpyAsync(dc, hc.data(), nc * sizeof(float), cudaMemcpyHostToDevice, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    op->b0 = (float*)a;
    op->b1 = (float*)b;
    op->rs = (float*)r;
    op->coef = (const float*)dc;
    op->gid = n_coef > 1 ? g->graph_of_row : nullptr;
    op->m = m;
    op->ld = ld;
    // launch shape: the Clenshaw order's tuned shape for this column count
    CSC_TRY(autotune(g, tune_key(KK_CLEN, (int)sizeof(float), ld), candidates<float>(g, KK_CLEN, ld / 4), s,
                     [&](const LaunchCfg& cf) {
                         return launch_clenshaw_step<float>(g, cf, op->b0, op->b1, nullptr, ld, ld, 0.0, 1, op->rs, s,
                                                            {}, true);
                     },
                     &op->cfg));
    const int32_t* pr = nullptr;
    return get_partition(g, op->cfg.P, &pr);
}

csc_status poly_apply(Graph* g, const PolyOp& op, const float* X, float* Y, cudaStream_t s) {
    const int64_t N = g->N;
    const int ld = op.ld, m = op.m;
    const int64_t tot = N * ld;
    CoefTab<float> tab;
    tab.c = op.coef;
    tab.gid = op.gid;
    tab.stride = m + 1;
    tab.gcols = op.gid ? op.gcols : nullptr;
    CoefTab<float> ft = tab;
    ft.j = m;
    // s X and B_m = c_m s X (internal order: no permutation)
    CSC_KLAUNCH("copy_in", (double)tot * 8, s,
                copy_in_kernel<float><<<ceil_div(tot, 256), 256, 0, s>>>(op.rs, X, (int32_t)N, ld, ld, ld, nullptr,
                                                                        g->dinv, CoefTab<float>()));
    CSC_KLAUNCH("copy_in", (double)tot * 8, s,
                copy_in_kernel<float><<<ceil_div(tot, 256), 256, 0, s>>>(op.b0, X, (int32_t)N, ld, ld, ld, nullptr,
                                                                        g->dinv, ft));
    float* B[2] = {op.b0, op.b1};
    for (int j = m - 1; j >= 1; --j) {
        tab.j = j;
        CSC_TRY(launch_clenshaw_step<float>(g, op.cfg, B[(m - j - 1) & 1], B[(m - j) & 1], Y, ld, ld, 0.0,
                                            j == m - 1 ? 1 : 0, op.rs, s, tab, true));
    }
    tab.j = 0;
    return launch_clenshaw_step<float>(g, op.cfg, B[(m - 1) & 1], B[m & 1], Y, ld, ld, 0.0, 2 | (m == 1 ? 1 : 0),
                                       op.rs, s, tab, true);
}

csc_status run_filter(Graph* g, const double* coeffs, int m, int d, int d_pad, uint64_t seed,
                      csc_dtype storage, const float* R_in, void* Y_out, bool normalize,
                      cudaStream_t s, bool clenshaw) {
    switch (storage) {
        case CSC_F32:
            return filter_typed<float>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s, STREAM_SIGNALS, 0.f,
                                       nullptr, clenshaw);
        case CSC_BF16:
            return filter_typed<__nv_bfloat16>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s,
                                               STREAM_SIGNALS, 0.f, nullptr, clenshaw);
        case CSC_F64:
            return filter_typed<double>(g, coeffs, m, d, d_pad, seed, R_in, Y_out, normalize, s, STREAM_SIGNALS, 0.f,
                                        nullptr, clenshaw);
        default:
            set_error("unknown storage type %d", (int)storage);
            return CSC_E_INVALID;
    }
}

// s_i = ||Y_i||^2 over the first d columns (fp64), then optionally Y_i / ||Y_i||.
// Y is the filter's output: float for fp32 and bf16 storage, double for fp64.
csc_status run_row_scores(void* Y, bool y_f64, int64_t N, int d, int ld, double* score, bool normalize,
                          int num_sms, cudaStream_t s) {
    int grid = ceil_div(N, 8);
    if (grid > num_sms * 8) grid = num_sms * 8;
    const double bytes = (normalize ? 2.0 : 1.0) * N * d * (y_f64 ? 8.0 : 4.0) + 8.0 * N;
    if (y_f64) {
        CSC_KLAUNCH("normalize", bytes, s,
                    normalize_kernel<double><<<grid, 256, 0, s>>>((double*)Y, (int32_t)N, d, ld, score,
                                                                  normalize ? 1 : 0));
    } else {
        CSC_KLAUNCH("normalize", bytes, s,
                    normalize_kernel<float><<<grid, 256, 0, s>>>((float*)Y, (int32_t)N, d, ld, score,
                                                                 normalize ? 1 : 0));
    }
    return CSC_OK;
}

// Non-finite scan: *flag = 1 when any of the first `cols` entries of a row is NaN or
// infinite (every writer stores the same value).
template <typename A>
__global__ void finite_scan_kernel(const A* __restrict__ X, int64_t rows, int cols, int ld, int* __restrict__ flag) {
    const int64_t total = rows * (int64_t)cols;
    int bad = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols;
        const int c = (int)(t - r * cols);
        if (!isfinite(X[r * ld + c])) bad = 1;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

csc_status run_check_finite(Graph* g, const void* X, bool x_f64, int64_t rows, int cols, int ld, const char* what,
                            cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return CSC_OK;
    void* fw = nullptr;
    CSC_TRY(ws_get(g, WS_CHECK, sizeof(int), &fw));
    int* flag = (int*)fw;
    CSC_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    int grid = (int)std::min<int64_t>(ceil_div(rows * cols, 256), (int64_t)g->num_sms * 8);
    const double bytes = (double)rows * cols * (x_f64 ? 8.0 : 4.0);
    if (x_f64)
        CSC_KLAUNCH("check_finite", bytes, s,
                    finite_scan_kernel<double><<<grid, 256, 0, s>>>((const double*)X, rows, cols, ld, flag));
    else
        CSC_KLAUNCH("check_finite", bytes, s,
                    finite_scan_kernel<float><<<grid, 256, 0, s>>>((const float*)X, rows, cols, ld, flag));
    int* h = (int*)g->pinned;
    CSC_CUDA_TRY(cudaMemcpyAsync(h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    if (*h) {
        set_error("non-finite values (NaN or infinity) in %s", what);
        return CSC_E_NUMERIC;
    }
    return CSC_OK;
}

// Paper-literal eigencount at one cut-off: filter n_probes N(0, 1) probes (the
// probe stream of csc_kpm_moments) with the degree-m Jackson-Chebyshev step at
// lambda, then count = (1/n_probes) sum_l r_l^T Y_l.  m sparse products.
csc_status run_refilter_count(Graph* g, double lambda, int m, int n_probes, uint64_t seed, double* count,
                              cudaStream_t s) {
    const int64_t N = g->N;
    const int ld = ((n_probes + 7) / 8) * 8;
    std::vector<double> c(m + 1);
    cheb_coefficients(lambda, m, true, c.data());
    const int nblk = std::min(ceil_div(N * (ld / 4), 256), g->num_sms * 8);
    void *yb = nullptr, *pb = nullptr;
    CSC_TRY(ws_get(g, WS_REFILTER, (size_t)N * ld * sizeof(float) + 256 + ((size_t)nblk * 3 + 3) * 8, &yb));
    float* Y = (float*)yb;
    pb = (char*)yb + (((size_t)N * ld * sizeof(float) + 255) / 256) * 256;
    double* part = (double*)pb;
    double* sum = part + (size_t)nblk * 3;
    CSC_TRY(filter_typed<float>(g, c.data(), m, n_probes, ld, seed, nullptr, Y, false, s, STREAM_PROBES, 1.0f));
    CSC_KLAUNCH("probe_trace", 4.0 * N * ld, s,
                probe_trace_kernel<<<nblk, 256, 0, s>>>(Y, (int32_t)N, n_probes, ld, seed, part));
    CSC_KLAUNCH("reduce", 24.0 * nblk, s, reduce_partials_kernel<<<1, 256, 0, s>>>(part, nblk, sum));
    double* host = g->pinned;
    CSC_CUDA_TRY(cudaMemcpyAsync(host, sum, sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    *count = host[0] / (double)n_probes;
    return CSC_OK;
}

template <typename T>
static csc_status moments_typed(Graph* g, int n_moments, int n_probes, uint64_t seed, double* mu,
                                int* passes, cudaStream_t s, bool per_graph) {
    constexpr int VEC = StoreTraits<T>::VEC;
    const int64_t N = g->N;
    const int ld = ((n_probes + 7) / 8) * 8;
    const size_t bytes = (size_t)N * ld * sizeof(T);
    void *xa = nullptr, *xb = nullptr, *part = nullptr, *sums = nullptr;
    CSC_TRY(ws_get(g, WS_XA, bytes, &xa));
    CSC_TRY(ws_get(g, WS_XB, bytes, &xb));
    T* X[2] = {(T*)xa, (T*)xb};
    // moments 0..M-1 need X_0..X_J with 2J >= M-1
    const int J = n_moments <= 2 ? 1 : n_moments / 2;
    const std::vector<LaunchCfg> cands = candidates<T>(g, KK_MOM, ld / VEC);
    int max_blocks = 1;
    for (const LaunchCfg& c : cands) max_blocks = std::max(max_blocks, (c.P + g->n_heavy) * c.tiles);
    {
        // a shape pinned on the handle or tuned earlier sizes the block partials too
        const uint64_t key = tune_key(KK_MOM, (int)sizeof(T), ld);
        LaunchCfg known;
        auto it = g->tuned.find(key);
        if (it != g->tuned.end()) max_blocks = std::max(max_blocks, (it->second.P + g->n_heavy) * it->second.tiles);
        else if (tune_cache_get(g, key, &known))
            max_blocks = std::max(max_blocks, (known.P + g->n_heavy) * known.tiles);
    }
    const int nseg = per_graph ? std::max(1, (int)g->n_graphs) : 1;
    CSC_TRY(ws_get(g, WS_PARTIAL, (size_t)max_blocks * 3 * sizeof(double), &part));
    CSC_TRY(ws_get(g, WS_MOMENTS, (size_t)nseg * J * 3 * sizeof(double), &sums));
    double* P = (double*)part;
    double* S = (double*)sums;
    CSC_TRY(fill_block<T>(g, X[0], n_probes, ld, seed, STREAM_PROBES, 1.0f, nullptr, ld, s));
    LaunchCfg cfg;
    CSC_TRY(autotune(g, tune_key(KK_MOM, (int)sizeof(T), ld), cands, s,
                     [&](const LaunchCfg& c) { return launch_mom_step<T>(g, c, X[0], X[1], ld, ld, 0, P, s); },
                     &cfg));
    const int grid = (cfg.P + g->n_heavy) * cfg.tiles;  // block partial slots per step
    const int32_t *gblk = nullptr, *ghvy = nullptr;
    if (nseg > 1) CSC_TRY(get_segments(g, cfg.P, &gblk, &ghvy));
    auto steps = [&](cudaStream_t st) -> csc_status {
        for (int j = 0; j < J; ++j) {
            CSC_TRY(launch_mom_step<T>(g, cfg, X[j & 1], X[(j + 1) & 1], ld, ld, j == 0 ? 1 : 0, P, st));
            CSC_KLAUNCH("reduce", 24.0 * grid, st,
                        segment_partials_kernel<<<nseg, 256, 0, st>>>(P, cfg.P, cfg.tiles, g->n_heavy, gblk, ghvy,
                                                                     nseg, j, J, S));
        }
        return CSC_OK;
    };
    if (!g_prof_enabled && g->use_graphs && J >= 2) {
        // the J steps replay as one captured CUDA graph
        const int32_t* pr = nullptr;
        CSC_TRY(get_partition(g, cfg.P, &pr));
        char key[256];
        snprintf(key, sizeof(key), "mom:%zu:%d:%d:%d:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p", sizeof(T), ld, J, nseg, cfg.G,
                 cfg.NT, cfg.threads, cfg.P, cfg.tiles, cfg.staged, (void*)X[0], (void*)X[1], (void*)P, (void*)S);
        int64_t launches = 0;
        CSC_TRY(replay_graph(g, key, s, &launches, steps));
    } else {
        CSC_TRY(steps(s));
    }
    const size_t nsum = (size_t)nseg * J * 3;
    std::vector<double> hbuf;
    double* host = g->pinned;
    if (nsum > 4096) {
        hbuf.resize(nsum);
        host = hbuf.data();
    }
    CSC_CUDA_TRY(cudaMemcpyAsync(host, S, nsum * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    const double nv = (double)n_probes;
    for (int gi = 0; gi < nseg; ++gi) {
        const double* h = host + (size_t)gi * J * 3;
        double* m = mu + (size_t)gi * n_moments;
        // step 0: s0 = <X0,X0>, s1 = <X1,X0>, s2 = <X1,X1>
        const double mu0 = h[0] / nv;
        const double mu1 = h[1] / nv;
        m[0] = mu0;
        if (n_moments > 1) m[1] = mu1;
        if (n_moments > 2) m[2] = 2.0 * h[2] / nv - mu0;
        for (int j = 1; j < J; ++j) {
            const int odd = 2 * j + 1, even = 2 * j + 2;
            if (odd < n_moments) m[odd] = 2.0 * h[3 * j + 1] / nv - mu1;
            if (even < n_moments) m[even] = 2.0 * h[3 * j + 2] / nv - mu0;
        }
    }
    if (passes) *passes = J;
    return CSC_OK;
}

csc_status run_moments(Graph* g, int n_moments, int n_probes, uint64_t seed, csc_dtype storage,
                       double* mu_host, int* passes, cudaStream_t s, bool per_graph) {
    switch (storage) {
        case CSC_F32:
            return moments_typed<float>(g, n_moments, n_probes, seed, mu_host, passes, s, per_graph);
        case CSC_BF16:
            return moments_typed<__nv_bfloat16>(g, n_moments, n_probes, seed, mu_host, passes, s, per_graph);
        default:
            set_error("moments support CSC_F32 and CSC_BF16 storage");
            return CSC_E_UNSUPPORTED;
    }
}

}  // namespace csc
