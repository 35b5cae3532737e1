// cg.cu -- label interpolation (Alg. 2 step 7, Eq. 5) and the partition rule of Sec. 4.1.
//
// For every cluster j the minimiser of ||M x - c_j^r||^2 + gamma x^T L^p x solves
// (M^T M + gamma L^p) x_j = M^T c_j^r.  All k systems are solved together by
// Jacobi-preconditioned conjugate gradients on an N x k row-major fp32 block
// (one independent CG per column; per-column inner products summed in
// compensated fp32 per thread, as error-free fp32 pairs across the threads of a
// block and in fp64 across blocks, in a fixed order).  A p = mask * p + gamma L^p p is computed with p sparse
// passes, the last one fused with the mask term and the <p, A p> partials.
// The products by L run in the pre-scaled form v = D^-1/2 t, so only the
// first of them loads per-edge weights (see lap_kernel).
// Preconditioner: diag(M^T M) + gamma (diag(L) = 1).
// Labels: node i -> argmax_j x_j(i) / ||x_j|| (ties to the lowest j).
// Columns whose CG has converged leave the iteration: the blocks are rewritten as
// dense blocks of the columns still iterating (column compaction, run_interpolate).
//
// Launch shape (every kernel of one solve): CTA x sweeps the contiguous row
// range [part[x], part[x+1]) with G lanes per row; CTA y covers the column tile
// [y*TW, (y+1)*TW), TW = 4*G*NT.  The shape is tuned once per graph and k; each
// compacted width takes lane groups of its own width (one column tile) with a row-range
// count, thread count and kernel form tuned for that width.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "device.cuh"

namespace csc {

constexpr int kCgMaxThreads = 512;

// Per-block, per-column partial sums of NS quantities, written as fp64 to
// partials[(q * nslots + slot) * ldp + col0 + c]: the lane groups of a warp (lanes of
// equal lane % G) are added by a shuffle butterfly, then the warps' sums in warp order,
// so the work per column does not grow with the number of row groups (narrow tiles have
// up to 256 of them).  Both stages add float pairs (FF), so no thread issues an fp64
// instruction; one fp64 value per column leaves the block.  Every thread of the block
// must call it.
template <int G, int NT, int NS>
__device__ __forceinline__ void block_column_partials(KSum (&acc)[NS][NT][4], int lane, int col0, int tcols,
                                                      int64_t ldp, double* __restrict__ partials, int64_t slot,
                                                      int64_t nslots) {
    constexpr int MAXWARPS = kCgMaxThreads / 32;
    constexpr int COLS = G * NT * 4;
    __shared__ float2 red[MAXWARPS * COLS];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    for (int q = 0; q < NS; ++q) {
        FF v[NT][4];
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int u = 0; u < 4; ++u) v[t][u] = acc[q][t][u].pair();
#pragma unroll
        for (int o = G; o < 32; o <<= 1)
#pragma unroll
            for (int t = 0; t < NT; ++t)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float bh = __shfl_xor_sync(0xffffffffu, v[t][u].hi, o);
                    const float bl = __shfl_xor_sync(0xffffffffu, v[t][u].lo, o);
                    v[t][u] = ff_add(v[t][u], FF{bh, bl});
                }
        __syncthreads();
        if ((threadIdx.x & 31) < G)
#pragma unroll
            for (int t = 0; t < NT; ++t)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    red[w * COLS + (t * G + lane) * 4 + u] = make_float2(v[t][u].hi, v[t][u].lo);
        __syncthreads();
        for (int c = threadIdx.x; c < COLS && c < tcols; c += blockDim.x) {
            FF sum{0.f, 0.f};
            for (int i = 0; i < warps; ++i) {
                const float2 e = red[i * COLS + c];
                sum = ff_add(sum, FF{e.x, e.y});
            }
            partials[((int64_t)q * nslots + slot) * ldp + col0 + c] = sum.value();
        }
    }
}

// The fp64 per-column scalars (alpha, beta) of this CTA's column tile as fp32, each
// converted once per CTA into shared memory.  Every thread of the block must call it.
template <int G, int NT>
__device__ __forceinline__ void tile_scalars(const double* __restrict__ src, int tcols, float (&out)[NT][4],
                                             int lane) {
    constexpr int COLS = G * NT * 4;
    __shared__ float s_col[COLS];
    for (int c = threadIdx.x; c < COLS; c += blockDim.x) s_col[c] = (src && c < tcols) ? (float)src[c] : 0.f;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) out[t][v] = s_col[(t * G + lane) * 4 + v];
}

// Batch view of the CG kernels (all members NULL for one graph): gid = graph of
// each row, gk4 = each graph's k rounded up to a multiple of 4 (the columns its
// rows carry; the rest stay zero), gact = each graph's columns still iterating
// (a graph with none left is skipped: its x, r and p no longer change).
struct CgBatch {
    const int32_t* gid = nullptr;
    const int32_t* gk4 = nullptr;
    const int* gact = nullptr;
    __device__ __forceinline__ int cols(int row, int ncols) const {
        if (!gid) return ncols;
        const int gr = gid[row];
        if (gact && gact[gr] == 0) return 0;
        return min(ncols, gk4[gr]);
    }
};

// Column tile of this CTA; a CTA whose graph needs no column of the tile (or has
// converged) leaves at once -- uniformly, before any barrier.
#define CG_TILE(G, NT)                                                          \
    const int lane = threadIdx.x % (G);                                         \
    const int col0 = blockIdx.y * ((G) * (NT) * 4);                             \
    const int r1 = part[blockIdx.x + 1];                                        \
    const int ncols_b = part[blockIdx.x] < r1 ? bt.cols(part[blockIdx.x], ncols) : ncols; \
    const int tcols = min((G) * (NT) * 4, ncols_b - col0);                      \
    if (tcols <= 0) return;
#define CG_ROWS(G) \
    for (int row = part[blockIdx.x] + (int)(threadIdx.x / (G)); row < r1; row += (int)(blockDim.x / (G)))

// The L-chain in pre-scaled form v = s t (s = D^-1/2, 1 for isolated nodes):
//   WIN (first product, unscaled input p):  v = s (p - D^-1/2 W D^-1/2 p)
//   !WIN (middle products, scaled input v): v' = v - D^-1 W v
// so only the first product loads per-edge weights.
// The row's own entries of a block (this CTA's column tile), loaded before the
// neighbour sum so their latency overlaps it.
template <int G, int NT>
struct RowVecs {
    float4 v[NT];
    __device__ __forceinline__ void load(const float* __restrict__ blk, int row, int lane, int col0, int tcols,
                                         int64_t ld) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl < tcols) v[t] = __ldg(reinterpret_cast<const float4*>(blk + (int64_t)row * ld + col0 + cl));
        }
    }
    __device__ __forceinline__ void get(int t, float (&x)[4]) const { StoreTraits<float>::unraw(v[t], x); }
};

template <int G, int NT, bool WIN>
__device__ __forceinline__ void lap_epilogue(int row, int lane, int col0, int tcols, float (&acc)[NT][4],
                                             const float* __restrict__ dinv, const float* __restrict__ invdeg,
                                             const RowVecs<G, NT>& in, float* __restrict__ out, int64_t ld) {
    const float di = dinv[row];
    const float sc = di > 0.f ? di : 1.f;
    const float f = WIN ? di : invdeg[row];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * 4;
        if (cl >= tcols) continue;
        const int64_t o = (int64_t)row * ld + col0 + cl;
        float x[4];
        in.get(t, x);
#pragma unroll
        for (int v = 0; v < 4; ++v) x[v] = WIN ? sc * (x[v] - f * acc[t][v]) : x[v] - f * acc[t][v];
        StoreTraits<float>::store(out + o, x);
    }
}

// Rows of degree > kHeavyRow are left to lap_heavy_kernel.
template <int G, int NT, bool WIN, bool STAGED, bool LEAN>
__global__ void __launch_bounds__(LEAN ? 256 : kCgMaxThreads, LEAN ? 5 : 0)
lap_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ lrp,
           const int32_t* __restrict__ lci, const float* __restrict__ dinv,
           const float* __restrict__ invdeg, const float* __restrict__ in, float* __restrict__ out,
           const int32_t* __restrict__ part, int ncols, int64_t ld, CgBatch bt) {
    CG_TILE(G, NT)
    extern __shared__ int32_t s_csr[];
    sweep_rows<STAGED, G>(rp, ci, lrp, lci, part[blockIdx.x], r1, s_csr, [&](int row, int e0, int e1,
                                                                            const int32_t* idx) {
        RowVecs<G, NT> x;
        x.load(in, row, lane, col0, tcols, ld);
        float acc[NT][4];
        gather_any<STAGED, float, G, NT, WIN, float, LEAN>(e0, e1, idx, dinv, in + col0, ld, lane, tcols, acc);
        lap_epilogue<G, NT, WIN>(row, lane, col0, tcols, acc, dinv, invdeg, x, out, ld);
    });
}

// Heavy rows: one CTA of kHeavyThreads per row (CTA x = heavy row, CTA y = column tile).
template <int G, int NT, bool WIN>
__global__ void __launch_bounds__(kHeavyThreads)
lap_heavy_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const float* __restrict__ dinv,
                 const float* __restrict__ invdeg, const float* __restrict__ in, float* __restrict__ out,
                 const int32_t* __restrict__ heavy, int ncols, int64_t ld, CgBatch bt) {
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * (G * NT * 4);
    const int row = heavy[blockIdx.x];
    const int tcols = min(G * NT * 4, bt.cols(row, ncols) - col0);
    if (tcols <= 0) return;
    float acc[NT][4];
    gather_heavy<float, G, NT, WIN, float>(__ldg(rp + row), __ldg(rp + row + 1), ci, dinv, in + col0, ld, lane, tcols,
                                           acc);
    if (threadIdx.x < G) {
        RowVecs<G, NT> x;
        x.load(in, row, lane, col0, tcols, ld);
        lap_epilogue<G, NT, WIN>(row, lane, col0, tcols, acc, dinv, invdeg, x, out, ld);
    }
}

// Ap = mask * p + gamma L t with per-column partials of <p, Ap>; the last product of
// the chain.  WIN: t = p itself (g(L) = L); else tin = s t from the chain.
template <int G, int NT, bool WIN>
__device__ __forceinline__ void lap_ax_epilogue(int row, int lane, int col0, int tcols, float (&acc)[NT][4],
                                                const float* __restrict__ dinv, const float* __restrict__ sqdeg,
                                                const RowVecs<G, NT>& tin, const RowVecs<G, NT>& p,
                                                const float* __restrict__ mask, float gamma, float* __restrict__ Ap,
                                                int64_t ld, KSum (&dot)[1][NT][4]) {
    const float di = dinv[row];
    const float back = WIN ? 1.f : sqdeg[row];
    const float mk = mask[row];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * 4;
        if (cl >= tcols) continue;
        const int64_t o = (int64_t)row * ld + col0 + cl;
        float tt[4], pp[4], a[4];
        tin.get(t, tt);
        p.get(t, pp);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            a[v] = mk * pp[v] + gamma * (tt[v] * back - di * acc[t][v]);
            dot[0][t][v].add(pp[v] * a[v]);
        }
        StoreTraits<float>::store(Ap + o, a);
    }
}

// <p, A p> partial slots: [0, gridDim.x) for the row ranges, then one per heavy
// row (lap_ax_heavy_kernel); nslots counts both.
template <int G, int NT, bool WIN, bool STAGED, bool LEAN>
__global__ void __launch_bounds__(LEAN ? 256 : kCgMaxThreads, LEAN ? 5 : 0)
lap_ax_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ lrp,
              const int32_t* __restrict__ lci, const float* __restrict__ dinv,
              const float* __restrict__ sqdeg, const float* __restrict__ tin, const float* __restrict__ p,
              const float* __restrict__ mask, float gamma, float* __restrict__ Ap, const int32_t* __restrict__ part,
              int ncols, int64_t ld, double* __restrict__ partials, int nslots, CgBatch bt) {
    CG_TILE(G, NT)
    KSum dot[1][NT][4];
    extern __shared__ int32_t s_csr[];
    sweep_rows<STAGED, G>(rp, ci, lrp, lci, part[blockIdx.x], r1, s_csr, [&](int row, int e0, int e1,
                                                                            const int32_t* idx) {
        RowVecs<G, NT> tv, pv;
        tv.load(tin, row, lane, col0, tcols, ld);
        pv.load(p, row, lane, col0, tcols, ld);
        float acc[NT][4];
        gather_any<STAGED, float, G, NT, WIN, float, LEAN>(e0, e1, idx, dinv, tin + col0, ld, lane, tcols, acc);
        lap_ax_epilogue<G, NT, WIN>(row, lane, col0, tcols, acc, dinv, sqdeg, tv, pv, mask, gamma, Ap, ld, dot);
    });
    block_column_partials<G, NT, 1>(dot, lane, col0, tcols, ld, partials, blockIdx.x, nslots);
}

template <int G, int NT, bool WIN>
__global__ void __launch_bounds__(kHeavyThreads)
lap_ax_heavy_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const float* __restrict__ dinv,
                    const float* __restrict__ sqdeg, const float* __restrict__ tin, const float* __restrict__ p,
                    const float* __restrict__ mask, float gamma, float* __restrict__ Ap,
                    const int32_t* __restrict__ heavy, int ncols, int64_t ld, double* __restrict__ partials,
                    int slot_base, int nslots, CgBatch bt) {
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * (G * NT * 4);
    const int row = heavy[blockIdx.x];
    const int tcols = min(G * NT * 4, bt.cols(row, ncols) - col0);
    if (tcols <= 0) return;
    float acc[NT][4];
    gather_heavy<float, G, NT, WIN, float>(__ldg(rp + row), __ldg(rp + row + 1), ci, dinv, tin + col0, ld, lane,
                                           tcols, acc);
    KSum dot[1][NT][4];
    if (threadIdx.x < G) {
        RowVecs<G, NT> tv, pv;
        tv.load(tin, row, lane, col0, tcols, ld);
        pv.load(p, row, lane, col0, tcols, ld);
        lap_ax_epilogue<G, NT, WIN>(row, lane, col0, tcols, acc, dinv, sqdeg, tv, pv, mask, gamma, Ap, ld, dot);
    }
    block_column_partials<G, NT, 1>(dot, lane, col0, tcols, ld, partials, slot_base + blockIdx.x, nslots);
}

// High-pass form of A p (g = 1 - h~): Ap = mask p + gamma (p - h~(L) p), with
// hp = h~(L) p computed by the Clenshaw operator; partials of <p, Ap> in slots
// [0, gridDim.x).
template <int G, int NT>
__global__ void __launch_bounds__(kCgMaxThreads)
hp_ax_kernel(const float* __restrict__ p, const float* __restrict__ hp, const float* __restrict__ mask, float gamma,
             float* __restrict__ Ap, const int32_t* __restrict__ part, int ncols, int64_t ld,
             double* __restrict__ partials, CgBatch bt) {
    CG_TILE(G, NT)
    KSum dot[1][NT][4];
    CG_ROWS(G) {
        const float mk = mask[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            float x[4], h[4], a[4];
            StoreTraits<float>::load(p + o, x);
            StoreTraits<float>::load(hp + o, h);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                a[v] = mk * x[v] + gamma * (x[v] - h[v]);
                dot[0][t][v].add(x[v] * a[v]);
            }
            StoreTraits<float>::store(Ap + o, a);
        }
    }
    block_column_partials<G, NT, 1>(dot, lane, col0, tcols, ld, partials, blockIdx.x, gridDim.x);
}

// x += alpha p; r -= alpha Ap; partials of <r, r/P> and <r, r>.  alpha == nullptr: no update.
template <int G, int NT>
__global__ void __launch_bounds__(kCgMaxThreads)
cg_update_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                 const float* __restrict__ Ap, const double* __restrict__ alpha, const int32_t* __restrict__ gid,
                 const float* __restrict__ pinv, const int32_t* __restrict__ part, int ncols, int64_t ld,
                 double* __restrict__ partials, CgBatch bt) {
    CG_TILE(G, NT)
    KSum dots[2][NT][4];
    float al[NT][4];
    // the columns' scalars of this range's graph (a batch's ranges lie inside one graph)
    const int64_t sg = (gid && part[blockIdx.x] < r1) ? (int64_t)gid[part[blockIdx.x]] * ld : 0;
    tile_scalars<G, NT>(alpha ? alpha + sg + col0 : nullptr, tcols, al, lane);
    CG_ROWS(G) {
        const float pi = pinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            float rv[4];
            StoreTraits<float>::load(r + o, rv);
            if (alpha) {
                float xv[4], pv[4], av[4];
                StoreTraits<float>::load_cs(x + o, xv);
                StoreTraits<float>::load(p + o, pv);
                StoreTraits<float>::load_cs(Ap + o, av);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    xv[v] = fmaf(al[t][v], pv[v], xv[v]);
                    rv[v] = fmaf(-al[t][v], av[v], rv[v]);
                }
                // x is not read again until the next update: evict-first
                StoreTraits<float>::store_cs(x + o, xv);
                StoreTraits<float>::store(r + o, rv);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                dots[0][t][v].add(rv[v] * (rv[v] * pi));
                dots[1][t][v].add(rv[v] * rv[v]);
            }
        }
    }
    block_column_partials<G, NT, 2>(dots, lane, col0, tcols, ld, partials, blockIdx.x, gridDim.x);
}

// p = r/P + beta p
template <int G, int NT>
__global__ void __launch_bounds__(kCgMaxThreads)
cg_pupdate_kernel(const float* __restrict__ r, float* __restrict__ p, const double* __restrict__ beta,
                  const int32_t* __restrict__ gid, const float* __restrict__ pinv, const int32_t* __restrict__ part,
                  int ncols, int64_t ld, CgBatch bt) {
    CG_TILE(G, NT)
    float be[NT][4];
    const int64_t sg = (gid && part[blockIdx.x] < r1) ? (int64_t)gid[part[blockIdx.x]] * ld : 0;
    tile_scalars<G, NT>(beta + sg + col0, tcols, be, lane);
    CG_ROWS(G) {
        const float pi = pinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            float rv[4], pv[4];
            StoreTraits<float>::load(r + o, rv);
            StoreTraits<float>::load(p + o, pv);
#pragma unroll
            for (int v = 0; v < 4; ++v) pv[v] = fmaf(be[t][v], pv[v], rv[v] * pi);
            StoreTraits<float>::store(p + o, pv);
        }
    }
}

// ||b - A x||^2 per column: partials.  b is rebuilt from the sample labels, or
// read from bfull (weighted decoder) when that is not NULL.
template <int G, int NT>
__global__ void __launch_bounds__(kCgMaxThreads)
residual_kernel(const float* __restrict__ Ax, const int32_t* __restrict__ slab, const float* __restrict__ bfull,
                const int32_t* __restrict__ part, int ncols, int64_t ld, double* __restrict__ partials, CgBatch bt) {
    CG_TILE(G, NT)
    KSum acc[1][NT][4];
    CG_ROWS(G) {
        const int lab = slab[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl >= tcols) continue;
            const int c = col0 + cl;
            float a[4], bv[4];
            StoreTraits<float>::load(Ax + (int64_t)row * ld + c, a);
            if (bfull) {
                StoreTraits<float>::load(bfull + (int64_t)row * ld + c, bv);
            } else {
#pragma unroll
                for (int v = 0; v < 4; ++v) bv[v] = c + v == lab ? 1.0f : 0.0f;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float e = bv[v] - a[v];
                acc[0][t][v].add(e * e);
            }
        }
    }
    block_column_partials<G, NT, 1>(acc, lane, col0, tcols, ld, partials, blockIdx.x, gridDim.x);
}

// column norms^2 of x (partials)
template <int G, int NT>
__global__ void __launch_bounds__(kCgMaxThreads)
colnorm_kernel(const float* __restrict__ x, const int32_t* __restrict__ part, int ncols, int64_t ld,
               double* __restrict__ partials, CgBatch bt) {
    CG_TILE(G, NT)
    KSum acc[1][NT][4];
    CG_ROWS(G) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * 4;
            if (cl >= tcols) continue;
            float a[4];
            StoreTraits<float>::load(x + (int64_t)row * ld + col0 + cl, a);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[0][t][v].add(a[v] * a[v]);
        }
    }
    block_column_partials<G, NT, 1>(acc, lane, col0, tcols, ld, partials, blockIdx.x, gridDim.x);
}

// Column state (fp64, length k each): rz, bnorm2, alpha, beta, active flags.
struct CgState {
    double* rz;
    double* bn2;
    double* alpha;
    double* beta;
    double* rr;
    int* active;
    int* n_active;
};

// Which partial slots belong to graph blockIdx.y of a batch: row ranges
// [gblk[y], gblk[y+1]) and heavy rows [ghvy[y], ghvy[y+1]) (slots P + h); with
// gblk == nullptr there is one graph: ranges [0, P), heavy rows [0, H).
struct Segs {
    const int32_t* gblk = nullptr;
    const int32_t* ghvy = nullptr;
    const int32_t* gk = nullptr;  // each graph's k (columns at or past it are not iterated)
    int* gact = nullptr;          // each graph's count of columns still iterating
    int P = 0, H = 0;
    __device__ __forceinline__ int kg(int g, int k) const { return gk ? gk[g] : k; }
    __device__ __forceinline__ void get(int g, int& b0, int& b1, int& h0, int& h1) const {
        b0 = gblk ? gblk[g] : 0;
        b1 = gblk ? gblk[g + 1] : P;
        h0 = ghvy ? ghvy[g] : 0;
        h1 = ghvy ? ghvy[g + 1] : H;
    }
};

// Column sums of block partials of one graph in a fixed order.  The graph's slots (its
// row ranges, then with heavy = true its heavy rows) are cut into gridDim.z slices of
// consecutive slots; a 32 x 32 thread block covers 32 columns of one slice: thread row y
// sums slots y, y+32, ... of the slice into four interleaved running sums (slot i of its
// sequence into sum i mod 4, so four loads are in flight) added in order, then the 32
// row sums are added in order.  The slices' sums go to lvl2; the block that completes a
// column chunk last (an atomic count per chunk; no block waits for another) adds them
// in slice order and returns true with the totals in out (threads with y == 0).  The
// result does not depend on which block is last.  nslots: the stride between the NS
// quantities' slot arrays.
constexpr int kReduceRows = 32;
constexpr int kSliceSlots = 256;  // slots per slice (8 per thread row)

template <int NS>
__device__ __forceinline__ bool reduce_columns(const double* __restrict__ partials, int nslots, const Segs& sg,
                                               bool heavy, int64_t ldp, int j, double* __restrict__ lvl2,
                                               int* __restrict__ counters, double (&out)[NS]) {
    __shared__ double red[NS][kReduceRows][33];
    __shared__ int s_last;
    const int x = threadIdx.x, y = threadIdx.y;
    int b0, b1, h0, h1;
    sg.get(blockIdx.y, b0, b1, h0, h1);
    const int nb = b1 - b0, total = nb + (heavy ? h1 - h0 : 0);
    const int z = blockIdx.z, S = gridDim.z;
    const int l0 = (int)((int64_t)total * z / S), l1 = (int)((int64_t)total * (z + 1) / S);
    // list position l -> slot: row ranges first, then heavy rows (slots P + h)
    auto slot = [&](int l) { return l < nb ? b0 + l : sg.P + h0 + (l - nb); };
    double s[NS][4];
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) s[q][u] = 0.0;
    int l = l0 + y;
    for (; l + 3 * kReduceRows < l1; l += 4 * kReduceRows)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < NS; ++q)
                s[q][u] += partials[((int64_t)q * nslots + slot(l + u * kReduceRows)) * ldp + j];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        const int ll = l + u * kReduceRows;
        if (ll < l1)
#pragma unroll
            for (int q = 0; q < NS; ++q) s[q][u] += partials[((int64_t)q * nslots + slot(ll)) * ldp + j];
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) red[q][y][x] = ((s[q][0] + s[q][1]) + s[q][2]) + s[q][3];
    __syncthreads();
    const int64_t chunk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (y == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            double t = 0.0;
            for (int i = 0; i < kReduceRows; ++i) t += red[q][i][x];
            lvl2[((chunk * S + z) * NS + q) * 32 + x] = t;
        }
    }
    __threadfence();
    __syncthreads();
    if (x == 0 && y == 0) s_last = atomicAdd(counters + chunk, 1) == S - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    if (y == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            double t = 0.0;
            for (int zz = 0; zz < S; ++zz) t += __ldcg(lvl2 + ((chunk * S + zz) * NS + q) * 32 + x);
            out[q] = t;
        }
        if (x == 0) counters[chunk] = 0;  // ready for the next launch
    }
    return true;
}

// pAp_j = sum of partials (row ranges and heavy rows); alpha_j = rz_j / pAp_j for
// active columns.  Graph blockIdx.y's column j lives at state index y * ldp + j.
__global__ void __launch_bounds__(1024) cg_alpha_kernel(const double* __restrict__ partials, int nslots, Segs sg,
                                                       int k, int64_t ldp, CgState st, double* __restrict__ lvl2,
                                                       int* __restrict__ counters) {
    const int jc = blockIdx.x * 32 + threadIdx.x;
    double s[1];
    if (!reduce_columns<1>(partials, nslots, sg, true, ldp, jc < k ? jc : 0, lvl2, counters, s)) return;
    if (threadIdx.y != 0 || jc >= sg.kg(blockIdx.y, k)) return;
    const int64_t j = (int64_t)blockIdx.y * ldp + jc;
    st.alpha[j] = (st.active[j] && s[0] != 0.0) ? st.rz[j] / s[0] : 0.0;
}

// After an update: rz_new, rr; convergence; beta.  init != 0: first call (sets bn2, active).
__global__ void __launch_bounds__(1024) cg_beta_kernel(const double* __restrict__ partials, int nslots, Segs sg,
                                                      int k, int64_t ldp, CgState st, double tol2, int init,
                                                      double* __restrict__ lvl2, int* __restrict__ counters) {
    const int jc = blockIdx.x * 32 + threadIdx.x;
    double s2[2];
    if (!reduce_columns<2>(partials, nslots, sg, false, ldp, jc < k ? jc : 0, lvl2, counters, s2)) return;
    if (threadIdx.y != 0 || jc >= sg.kg(blockIdx.y, k)) return;
    const int64_t j = (int64_t)blockIdx.y * ldp + jc;
    int act = st.active[j];
    if (!init && !act) return;  // a finished column keeps its state (its graph may be skipped)
    const double rz = s2[0], rr = s2[1];
    st.rr[j] = rr;
    if (init) {
        st.bn2[j] = rr;
        st.rz[j] = rz;
        st.beta[j] = 0.0;
        act = rr > 0.0 ? 1 : 0;
    } else {
        if (rr <= tol2 * st.bn2[j]) act = 0;
        st.beta[j] = (act && st.rz[j] != 0.0) ? rz / st.rz[j] : 0.0;
        st.rz[j] = rz;
    }
    st.active[j] = act;
    if (act) {
        atomicAdd(st.n_active, 1);
        if (sg.gact) atomicAdd(sg.gact + blockIdx.y, 1);
    }
}

__global__ void __launch_bounds__(1024) column_sum_kernel(const double* __restrict__ partials, int nslots, Segs sg,
                                                         int k, int64_t ldp, double* __restrict__ out,
                                                         double* __restrict__ lvl2, int* __restrict__ counters) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    double s[1];
    if (!reduce_columns<1>(partials, nslots, sg, false, ldp, j < k ? j : 0, lvl2, counters, s)) return;
    if (threadIdx.y == 0 && j < sg.kg(blockIdx.y, k)) out[(int64_t)blockIdx.y * ldp + j] = s[0];
}

// gk / gid (batched handle): a sample's label must be below its graph's k.
// w (weighted decoder of variable-density draws): NULL for the 0/1 mask of Eq. 5,
// else each draw adds its weight to the mask and to the right-hand side (a node
// drawn twice counts twice); weights must be finite and positive.
__global__ void cg_setup_kernel(const int64_t* __restrict__ sample_idx, const int32_t* __restrict__ sample_labels,
                                const float* __restrict__ w, int64_t n, int64_t N, const int32_t* __restrict__ iperm,
                                float* __restrict__ r, float* __restrict__ mask, int32_t* __restrict__ slab,
                                int64_t ld, int k, const int32_t* __restrict__ gk, const int32_t* __restrict__ gid,
                                int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t node = sample_idx[i];
    const int lab = sample_labels[i];
    if (node < 0 || node >= N) {
        atomicOr(bad, 1);
        return;
    }
    const int64_t row = iperm ? iperm[node] : node;
    const int kk = gk ? gk[gid[row]] : k;
    if (lab < 0 || lab >= kk) {
        atomicOr(bad, 1);
        return;
    }
    if (w) {
        const float wt = w[i];
        if (!(wt > 0.0f) || isinf(wt)) {
            atomicOr(bad, 1);
            return;
        }
        atomicAdd(r + row * ld + lab, wt);
        atomicAdd(mask + row, wt);
    } else {
        r[row * ld + lab] = 1.0f;
        mask[row] = 1.0f;
    }
    slab[row] = lab;
}

__global__ void precond_kernel(const float* __restrict__ mask, float gamma, float* __restrict__ pinv, int32_t N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) pinv[i] = 1.0f / (mask[i] + gamma);
}

// ||x_j|| (fp64) and 1/||x_j|| rounded to fp32 of every (graph, column); 0 and 0
// for a zero column.
__global__ void label_scale_kernel(const double* __restrict__ norm2, int64_t n, double* __restrict__ nrm,
                                   float* __restrict__ rnrm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double q = norm2[i];
    const double r = q > 0.0 ? sqrt(q) : 0.0;
    nrm[i] = r;
    rnrm[i] = q > 0.0 ? (float)(1.0 / r) : 0.f;
}

// label(i) = argmax_j x_ij / ||x_j|| with the quotient rounded in fp64 (ties to the
// lowest j; a zero column scores 0), one warp per row.  FP64 is slow on this part,
// so the quotients are first approximated in fp32, x times the fp32 reciprocal
// (within 2^-22 relative of the fp64 quotient); only columns within 2^-20 relative
// of the largest approximation, which always include the winner, get the fp64
// division.  The decision therefore equals dividing every entry in fp64.  A row
// whose approximations are not all finite, or whose largest one lies below 2^-100,
// takes the fp64 division everywhere.
__global__ void label_argmax_kernel(const float* __restrict__ x, const double* __restrict__ nrm_all,
                                    const float* __restrict__ rnrm_all, int32_t N, int k_all, int64_t ld,
                                    const int32_t* __restrict__ gk, const int32_t* __restrict__ gid,
                                    const int32_t* __restrict__ perm, int32_t* __restrict__ labels,
                                    float* __restrict__ fuzzy) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < N; row += nw) {
        const int gr = gid ? gid[row] : 0;
        const int k = gk ? gk[gr] : k_all;
        const double* nrm = nrm_all + (int64_t)gr * ld;
        const float* rnrm = rnrm_all + (int64_t)gr * ld;
        const float* xr = x + row * ld;
        float am = -INFINITY;
        int finite = 1;
        for (int j = lane; j < k; j += 32) {
            const float a = xr[j] * rnrm[j];
            finite &= isfinite(a) ? 1 : 0;
            am = fmaxf(am, a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        // non-finite approximations, or a maximum so small that fp32 loses relative
        // precision (subnormal range): fp64 division everywhere
        const bool all = __all_sync(0xffffffffu, finite) == 0 || fabsf(am) < 0x1p-100f;
        const float thr = am - fabsf(am) * 0x1p-20f;
        double bv = -INFINITY;
        int best = 0x7fffffff;
        for (int j = lane; j < k; j += 32) {
            if (all || xr[j] * rnrm[j] >= thr) {
                const double nj = nrm[j];
                const double v = nj > 0.0 ? (double)xr[j] / nj : 0.0;
                if (v > bv || (v == bv && j < best)) {
                    bv = v;
                    best = j;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            if (ov > bv || (ov == bv && ob < best)) {
                bv = ov;
                best = ob;
            }
        }
        const int64_t orig = perm ? perm[row] : row;
        if (lane == 0) labels[orig] = best < k ? best : 0;
        if (fuzzy)
            for (int j = lane; j < k; j += 32) fuzzy[orig * k_all + j] = xr[j];
    }
}

// Column compaction of the CG blocks, into dense blocks of the new width: for every row,
// slot s < nw of the new x, r, p (row stride ln) takes slot src[s] of the old ones (row
// stride lo), and the x of each column leaving the iteration (old slot lv_slot[q]) goes to
// column lv_col[q] of xf, the solution in column order (row stride ldf).  One warp per row;
// out of place.
__global__ void compact_columns_kernel(const float* __restrict__ ox, const float* __restrict__ orr,
                                       const float* __restrict__ op, int lo, float* __restrict__ nx,
                                       float* __restrict__ nr, float* __restrict__ np, int ln,
                                       const int32_t* __restrict__ src, int nw, const int32_t* __restrict__ lv_slot,
                                       const int32_t* __restrict__ lv_col, int nlv, float* __restrict__ xf, int ldf,
                                       int32_t N) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < N; row += nwarps) {
        const int64_t o = row * lo, n = row * ln;
        for (int j = lane; j < nw; j += 32) {
            const int sj = src[j];
            nx[n + j] = ox[o + sj];
            nr[n + j] = orr[o + sj];
            np[n + j] = op[o + sj];
        }
        for (int q = lane; q < nlv; q += 32) xf[row * ldf + lv_col[q]] = ox[o + lv_slot[q]];
    }
}

// ------------------------------------------------------------- dispatch
static const int kCgShapes[][2] = {{2, 1}, {4, 1}, {8, 1}, {16, 1}, {16, 2}, {32, 1}, {32, 2}};
static const int kCgThreadChoices[] = {256, 512};

#define CG_SWITCH(cfg, ...)                                                                        \
    do {                                                                                           \
        switch ((cfg).G * 8 + (cfg).NT) {                                                          \
            case 2 * 8 + 1: { constexpr int G_ = 2, NT_ = 1; __VA_ARGS__; } break;                 \
            case 4 * 8 + 1: { constexpr int G_ = 4, NT_ = 1; __VA_ARGS__; } break;                 \
            case 8 * 8 + 1: { constexpr int G_ = 8, NT_ = 1; __VA_ARGS__; } break;                 \
            case 16 * 8 + 1: { constexpr int G_ = 16, NT_ = 1; __VA_ARGS__; } break;               \
            case 16 * 8 + 2: { constexpr int G_ = 16, NT_ = 2; __VA_ARGS__; } break;               \
            case 32 * 8 + 1: { constexpr int G_ = 32, NT_ = 1; __VA_ARGS__; } break;               \
            case 32 * 8 + 2: { constexpr int G_ = 32, NT_ = 2; __VA_ARGS__; } break;               \
            default:                                                                               \
                set_error("no compiled CG shape G=%d NT=%d", (cfg).G, (cfg).NT);                   \
                return CSC_E_UNSUPPORTED;                                                          \
        }                                                                                          \
    } while (0)

template <int G, int NT>
static int cg_occupancy_of(int threads, bool lean) {
    // the solve's most register-hungry kernel bounds the residency of all of them (the lean
    // form: its products, which take most of the time)
    int a = 1, b = 1;
    cudaError_t e;
    if constexpr (NT == 1) {
        if (lean) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, lap_kernel<G, NT, false, true, true>, threads, 0);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return 1;
            }
            return a < 1 ? 1 : a;
        }
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, lap_kernel<G, NT, false, true, false>, threads, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cg_update_kernel<G, NT>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const int n = std::min(a, b);
    return n < 1 ? 1 : n;
}

// Row-range launches of one product of the L-chain and of the last product, in the shape's
// index source and form (LaunchCfg::staged, LaunchCfg::lean; the lean form has NT = 1).
template <int G, int NT, bool WIN>
static void lap_rows(const LaunchCfg& c, dim3 grid, int smem, cudaStream_t s, const Graph* g, const float* in,
                     float* out, const int32_t* part, int ncols, int64_t ld, const CgBatch& bt) {
    if constexpr (NT == 1) {
        if (c.lean) {
            if (c.staged)
                lap_kernel<G, NT, WIN, true, true><<<grid, c.threads, smem, s>>>(
                    g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->invdeg, in, out, part, ncols, ld, bt);
            else
                lap_kernel<G, NT, WIN, false, true><<<grid, c.threads, 0, s>>>(
                    g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->invdeg, in, out, part, ncols, ld, bt);
            return;
        }
    }
    if (c.staged)
        lap_kernel<G, NT, WIN, true, false><<<grid, c.threads, smem, s>>>(
            g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->invdeg, in, out, part, ncols, ld, bt);
    else
        lap_kernel<G, NT, WIN, false, false><<<grid, c.threads, 0, s>>>(
            g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->invdeg, in, out, part, ncols, ld, bt);
}

template <int G, int NT, bool WIN>
static void lap_ax_rows(const LaunchCfg& c, dim3 grid, int smem, cudaStream_t s, const Graph* g, const float* tin,
                        const float* p, const float* mask, float gamma, float* Ap, const int32_t* part, int ncols,
                        int64_t ld, double* partials, int nslots, const CgBatch& bt) {
    if constexpr (NT == 1) {
        if (c.lean) {
            if (c.staged)
                lap_ax_kernel<G, NT, WIN, true, true><<<grid, c.threads, smem, s>>>(
                    g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->sqdeg, tin, p, mask, gamma, Ap, part, ncols,
                    ld, partials, nslots, bt);
            else
                lap_ax_kernel<G, NT, WIN, false, true><<<grid, c.threads, 0, s>>>(
                    g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->sqdeg, tin, p, mask, gamma, Ap, part, ncols,
                    ld, partials, nslots, bt);
            return;
        }
    }
    if (c.staged)
        lap_ax_kernel<G, NT, WIN, true, false><<<grid, c.threads, smem, s>>>(
            g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->sqdeg, tin, p, mask, gamma, Ap, part, ncols, ld,
            partials, nslots, bt);
    else
        lap_ax_kernel<G, NT, WIN, false, false><<<grid, c.threads, 0, s>>>(
            g->row_ptr, g->col_idx, g->lrp, g->lci, g->dinv, g->sqdeg, tin, p, mask, gamma, Ap, part, ncols, ld,
            partials, nslots, bt);
}

// Dynamic shared memory a staged launch of the shape may add to the solve's kernels' own
// arrays (the fused product's column partials take 16 KB per vector per lane).
template <int G, int NT>
static int cg_staged_room() {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, lap_ax_kernel<G, NT, false, true, false>) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int)a.maxDynamicSharedSizeBytes;
}

static csc_status cg_occupancy(const LaunchCfg& c, int* out) {
    CG_SWITCH(c, *out = cg_occupancy_of<G_, NT_>(c.threads, c.lean != 0));
    return CSC_OK;
}

// Candidate launch shapes of the CG kernels for nv 16-byte vectors per row: column tiles
// of 4*G*NT floats with at most a third idle (only_G > 0: lane groups of only_G, NT = 1),
// one to eight waves of resident CTAs (at most p_cap row ranges when p_cap > 0); *max_p
// grows to the largest row-range count.
static csc_status cg_candidates(Graph* g, int64_t N, int nv, int p_cap, int only_G, std::vector<LaunchCfg>* out,
                                int* max_p) {
    int min_waste = 1 << 30;  // narrow blocks (k <= 4) keep the least-waste shapes
    for (const auto& sh : kCgShapes) {
        const int cap = sh[0] * sh[1];
        const int tiles = (nv + cap - 1) / cap;
        if (tiles <= 64) min_waste = std::min(min_waste, tiles * cap - nv);
    }
    for (const auto& sh : kCgShapes) {
        const int cap = sh[0] * sh[1];
        const int tiles = (nv + cap - 1) / cap;
        const int waste = tiles * cap - nv;
        if (only_G > 0 ? (sh[0] != only_G || sh[1] != 1)
                       : (tiles > 64 || (3 * waste > tiles * cap && waste > min_waste)))
            continue;
        for (int th : kCgThreadChoices)
            for (int lean = 0; lean <= 1; ++lean) {
                if (lean && (sh[1] != 1 || th != 256)) continue;  // the lean form: NT = 1, 256 threads
                LaunchCfg c;
                c.G = sh[0];
                c.NT = sh[1];
                c.threads = th;
                c.tiles = tiles;
                c.lean = lean;
                int occ = 1;
                CSC_TRY(cg_occupancy(c, &occ));
                const int64_t lim = (N + (th / c.G) - 1) / (th / c.G);
                // one to eight waves of resident CTAs (shorter row ranges balance uneven SMs)
                for (int waves = 1; waves <= 8; waves *= 2) {
                    int P = (g->num_sms * occ * waves + tiles - 1) / tiles;
                    if (P > lim) P = (int)lim;
                    if (P < g->n_graphs) P = g->n_graphs;  // a batch needs a range per graph
                    P = P < 1 ? 1 : P;
                    // the CTA's staged CSR slice must fit shared memory: more, shorter ranges if not
                    CSC_TRY(fit_staged_partition(g, P, std::max<int64_t>(lim, g->n_graphs), &P));
                    if (staged_smem(g, P) > kStagedSmemMax || (p_cap > 0 && P > p_cap)) continue;
                    c.P = P;
                    if (!out->empty() && out->back().G == c.G && out->back().NT == c.NT &&
                        out->back().threads == th && out->back().lean == lean && out->back().P == c.P)
                        continue;
                    *max_p = std::max(*max_p, c.P);
                    int room = 0;
                    CG_SWITCH(c, room = cg_staged_room<G_, NT_>());
                    c.staged = 1;  // both index sources (sweep_rows), the staged one where it fits
                    if (staged_smem(g, c.P) <= std::min(room, kStagedSmemMax)) out->push_back(c);
                    c.staged = 0;
                    out->push_back(c);
                }
            }
    }
    return CSC_OK;
}

csc_status run_interpolate(Graph* g, const int64_t* sample_idx, const int32_t* sample_labels, int64_t n, int k,
                           int g_power, double gamma, double rel_tol, int max_iter, int32_t* labels_out,
                           float* fuzzy_out, csc_cg_info* info, cudaStream_t s, const int32_t* k_graphs,
                           const double* hp_coef, int hp_m, const float* sample_w) {
    const int32_t N = (int32_t)g->N;
    // one independent set of k systems per graph of a batch (k_graphs: each graph's k)
    const int nseg = (k_graphs && g->n_graphs > 1) ? g->n_graphs : 1;
    const bool hp = hp_coef != nullptr;  // g = 1 - h~ instead of L^p (per graph for a batch)
    const int ld = ((k + 3) / 4) * 4;
    const int nv = ld / 4;
    std::vector<LaunchCfg> cands;
    int max_p = 1;
    CSC_TRY(cg_candidates(g, N, nv, 0, 0, &cands, &max_p));
    if (cands.empty()) {
        set_error("csc_interpolate: no launch shape for k = %d", k);
        return CSC_E_UNSUPPORTED;
    }
    // a shape pinned on the handle or tuned earlier is used as is: its row-range count
    // sizes the per-block partials too
    const uint64_t tkey = (3ull << 48) | (uint64_t)(uint32_t)ld;
    LaunchCfg known;
    bool have_known = false;
    {
        auto it = g->tuned.find(tkey);
        if (it != g->tuned.end()) {
            known = it->second;
            have_known = true;
        } else if (tune_cache_get(g, tkey, &known)) {
            g->tuned[tkey] = known;
            have_known = true;
        }
        if (have_known) max_p = std::max(max_p, known.P);
    }
    const size_t blk = (size_t)N * ld * sizeof(float);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_x = take(blk), o_r = take(blk), o_p = take(blk), o_ap = take(blk), o_t1 = take(blk),
                 o_t2 = take(blk);
    const size_t o_mask = take((size_t)N * 4), o_pinv = take((size_t)N * 4), o_slab = take((size_t)N * 4);
    const size_t o_b = take(sample_w ? blk : 0);  // weighted right-hand side, kept for the residual
    // two quantities per row-range block; <p, A p> also has one slot per heavy row
    const size_t o_part = take((size_t)2 * (max_p + g->n_heavy) * ld * 8);
    const size_t sl = (size_t)nseg * ld;  // per-(graph, column) state length
    const size_t o_state = take(sl * 8 * 8 + sl * 4 + 64);
    const size_t o_gk = take((size_t)nseg * 4 * 3);
    // sliced column reductions (reduce_columns): per column chunk, slice sums and a count
    const int nchunks = ceil_div(k, 32) * nseg;
    const int max_slices = std::max(1, ceil_div(max_p + (int)g->n_heavy, kSliceSlots));
    const size_t o_lvl2 = take((size_t)nchunks * max_slices * 2 * 32 * 8);
    const size_t o_cnt = take((size_t)nchunks * 4);
    const size_t o_src = take((size_t)3 * ld * 4);  // slot maps of a compaction
    const bool compact = !hp && nseg == 1 && ld <= 1024;  // column compaction (see below)
    const size_t o_xf = take(compact ? blk : 0);          // the solution in column order
    void* base = nullptr;
    CSC_TRY(ws_get(g, WS_CG, off, &base));
    char* b = (char*)base;
    float* x = (float*)(b + o_x);
    float* r = (float*)(b + o_r);
    float* p = (float*)(b + o_p);
    float* Ap = (float*)(b + o_ap);
    float* t1 = (float*)(b + o_t1);
    float* t2 = (float*)(b + o_t2);
    float* mask = (float*)(b + o_mask);
    float* pinv = (float*)(b + o_pinv);
    int32_t* slab = (int32_t*)(b + o_slab);
    float* bfull = sample_w ? (float*)(b + o_b) : nullptr;
    double* part = (double*)(b + o_part);
    double* sd = (double*)(b + o_state);
    CgState st;
    st.rz = sd;
    st.bn2 = sd + sl;
    st.alpha = sd + 2 * sl;
    st.beta = sd + 3 * sl;
    st.rr = sd + 4 * sl;
    double* norm2 = sd + 5 * sl;
    double* nrm = sd + 6 * sl;   // column norms ||x_j|| (label rule)
    float* rnrm = (float*)(sd + 7 * sl);  // their reciprocals (fp32)
    st.active = (int*)(sd + 8 * sl);
    st.n_active = st.active + sl;
    int* bad = st.n_active + 1;
    double* lvl2 = (double*)(b + o_lvl2);
    int* red_cnt = (int*)(b + o_cnt);
    int32_t* d_src = (int32_t*)(b + o_src);
    float* xf = compact ? (float*)(b + o_xf) : nullptr;
    int32_t* d_gk = nullptr;
    const int32_t* gid = nullptr;
    CgBatch bt, bt_all;  // bt also skips finished graphs; bt_all only narrows the columns
    std::vector<int32_t> hk;
    if (nseg > 1) {
        d_gk = (int32_t*)(b + o_gk);
        int32_t* d_gk4 = d_gk + nseg;
        int* d_gact = (int*)(d_gk4 + nseg);
        hk.assign(k_graphs, k_graphs + nseg);
        for (int q = 0; q < nseg; ++q) hk.push_back((k_graphs[q] + 3) / 4 * 4);
        CSC_CUDA_TRY(cudaMemcpyAsync(d_gk, hk.data(), (size_t)2 * nseg * 4, cudaMemcpyHostToDevice, s));
        CSC_CUDA_TRY(cudaMemsetAsync(d_gact, 0, (size_t)nseg * 4, s));
        gid = g->graph_of_row;
        bt.gid = bt_all.gid = gid;
        bt.gk4 = bt_all.gk4 = d_gk4;
        bt.gact = d_gact;
        // columns past a graph's k are never written: keep them zero
        CSC_CUDA_TRY(cudaMemsetAsync(p, 0, blk, s));
        CSC_CUDA_TRY(cudaMemsetAsync(Ap, 0, blk, s));
    }
    CSC_CUDA_TRY(cudaMemsetAsync(sd, 0, sl * 8 * 8 + sl * 4, s));
    CSC_CUDA_TRY(cudaMemsetAsync(red_cnt, 0, (size_t)nchunks * 4, s));

    // zero x, r, mask; slab = -1
    CSC_CUDA_TRY(cudaMemsetAsync(x, 0, blk, s));
    CSC_CUDA_TRY(cudaMemsetAsync(r, 0, blk, s));
    CSC_CUDA_TRY(cudaMemsetAsync(mask, 0, (size_t)N * 4, s));
    CSC_CUDA_TRY(cudaMemsetAsync(slab, 0xff, (size_t)N * 4, s));
    CSC_CUDA_TRY(cudaMemsetAsync(st.n_active, 0, 2 * sizeof(int), s));
    CSC_KLAUNCH("cg_setup", 24.0 * n, s,
                cg_setup_kernel<<<ceil_div(n, 256), 256, 0, s>>>(sample_idx, sample_labels, sample_w, n,
                                                                 (int64_t)N, g->iperm, r, mask, slab, ld, k, d_gk,
                                                                 gid, bad));
    if (bfull) CSC_CUDA_TRY(cudaMemcpyAsync(bfull, r, blk, cudaMemcpyDeviceToDevice, s));
    CSC_KLAUNCH("cg_setup", 8.0 * N, s, precond_kernel<<<ceil_div(N, 256), 256, 0, s>>>(mask, (float)gamma, pinv, N));

    // launch shapes are tuned on one iteration's row-range work at `cols` columns (row
    // stride cols): three products of the chain, the last product with the mask term and
    // <., .> partials, and the update's partials (alpha = NULL: nothing is updated).  It
    // reads r, p, x and writes only t1, t2, Ap and the partials, which hold nothing between
    // iterations, so a compacted solve can tune its new width in place.
    auto tune = [&](const std::vector<LaunchCfg>& cs, int cols, LaunchCfg* best) -> csc_status {
        struct ProfOff {  // tuning launches are not part of the measured work
            bool prev = g_prof_enabled;
            ProfOff() { g_prof_enabled = false; }
            ~ProfOff() { g_prof_enabled = prev; }
        } off;
        float best_ms = 1e30f;
        *best = cs[0];
        for (const LaunchCfg& c : cs) {
            const int32_t* pr = nullptr;
            CSC_TRY(get_partition(g, c.P, &pr));
            const dim3 grid(c.P, c.tiles);
            float ms = 0.f;
            const int sm = c.staged ? staged_smem(g, c.P) : 0;
            for (int rep = 0; rep < 3; ++rep) {
                if (rep == 1) cudaEventRecord(g->ev[0], s);
                const float* src[3] = {r, t1, t2};
                float* dst[3] = {t1, t2, t1};
                for (int q = 0; q < 3; ++q)
                    CG_SWITCH(c, lap_rows<G_, NT_, false>(c, grid, sm, s, g, src[q], dst[q], pr, cols, cols,
                                                          CgBatch()));
                CG_SWITCH(c, lap_ax_rows<G_, NT_, false>(c, grid, sm, s, g, t1, p, mask, (float)gamma, Ap, pr, cols,
                                                         cols, part, c.P, CgBatch()));
                CG_SWITCH(c, cg_update_kernel<G_, NT_><<<grid, c.threads, 0, s>>>(x, r, p, Ap, nullptr, nullptr, pinv,
                                                                                   pr, cols, cols, part, CgBatch()));
            }
            cudaEventRecord(g->ev[1], s);
            CSC_CUDA_TRY(cudaEventSynchronize(g->ev[1]));
            CSC_CUDA_TRY(cudaGetLastError());
            cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]);
            if (ms < best_ms) {
                best_ms = ms;
                *best = c;
            }
        }
        return CSC_OK;
    };
    LaunchCfg cfg;
    if (have_known) {
        cfg = known;
    } else {
        CSC_TRY(tune(cands, ld, &cfg));
        g->tuned[tkey] = cfg;
        tune_cache_put(g, tkey, cfg);
    }
    const int32_t* rpart = nullptr;
    CSC_TRY(get_partition(g, cfg.P, &rpart));
    const int csmem = cfg.staged ? staged_smem(g, cfg.P) : 0;  // the CTA's CSR slice (stage_csr)
    CSC_TRY(check_staged_smem(csmem));
    {
        int room = 0;
        CG_SWITCH(cfg, room = cg_staged_room<G_, NT_>());
        if (csmem > room) {
            set_error("csc_interpolate: a row range's CSR slice (%d bytes) does not fit beside the CG kernels' "
                      "shared arrays (%d bytes free): use more row ranges or the global index source", csmem, room);
            return CSC_E_UNSUPPORTED;
        }
    }
    const dim3 grid(cfg.P, cfg.tiles);
    const int th = cfg.threads;
    const int P = cfg.P;
    const int H = hp ? 0 : (int)g->n_heavy;  // the high-pass A p has no heavy-row slots
    const int PH = P + H;  // <p, A p> partial slots
    PolyOp op;
    if (hp) {
        CSC_TRY(poly_prepare(g, hp_coef, hp_m, ld, &op, s, nseg));
        // a batch's graphs carry only their own k columns (rounded up to 4) through h~
        if (nseg > 1) op.gcols = d_gk + nseg;
    }
    const dim3 hgrid(H > 0 ? H : 1, cfg.tiles);
    Segs sg;
    sg.P = P;
    sg.H = H;
    if (nseg > 1) {
        CSC_TRY(get_segments(g, P, &sg.gblk, &sg.ghvy));
        sg.gk = d_gk;
        sg.gact = (int*)bt.gact;
    }
    auto reset_active = [&](cudaStream_t s) -> csc_status {
        CSC_CUDA_TRY(cudaMemsetAsync(st.n_active, 0, sizeof(int), s));
        if (sg.gact) CSC_CUDA_TRY(cudaMemsetAsync(sg.gact, 0, (size_t)nseg * sizeof(int), s));
        return CSC_OK;
    };

    // algorithmic bytes per launch of each CG kernel (fp32 N x ld blocks)
    double blkb = (double)N * ld * 4.0;
    const double csr_b = 4.0 * g->nnz + 4.0 * (N + 1) + 4.0 * N;
    double scal_b = 8.0 * P * ld;
    double scal_ax = 8.0 * PH * ld;
    // share of the sparse bytes that falls on heavy rows (launched separately)
    const double heavy_frac = g->nnz > 0 ? (double)(g->nnz - g->h_light.back()) / (double)g->nnz : 0.0;
    // reductions over P slots (updates, residual, norms) and P + H slots (<p, A p>)
    dim3 kb(ceil_div(k, 32), nseg, std::max(1, ceil_div(P, kSliceSlots)));
    dim3 kb_ax(ceil_div(k, 32), nseg, std::max(1, ceil_div(PH, kSliceSlots)));
    const dim3 rb(32, kReduceRows);
    CG_SWITCH(cfg, CSC_KLAUNCH("cg_update", blkb + 4.0 * N, s,
                               cg_update_kernel<G_, NT_><<<grid, th, 0, s>>>(x, r, p, Ap, nullptr, gid, pinv, rpart, ld,
                                                                             ld, part, bt_all)));
    CSC_KLAUNCH("cg_scalar", 2 * scal_b, s,
                cg_beta_kernel<<<kb, rb, 0, s>>>(part, P, sg, k, ld, st, rel_tol * rel_tol, 1, lvl2, red_cnt));
    CG_SWITCH(cfg, CSC_KLAUNCH("cg_pupdate", 3 * blkb + 4.0 * N, s,
                               cg_pupdate_kernel<G_, NT_><<<grid, th, 0, s>>>(r, p, st.beta, gid, pinv, rpart, ld,
                                                                              ld, bt)));
    int* h_active = (int*)g->pinned;
    CSC_CUDA_TRY(cudaMemcpyAsync(h_active, st.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_active[1]) {
        set_error("csc_interpolate: a sample label is outside [0, k), a sample index outside [0, N) or a sample "
                  "weight not finite and positive");
        return CSC_E_INVALID;
    }
    // Column compaction (one graph, g = L^p): a column whose CG has converged keeps its x
    // and leaves the iteration.  At a convergence check that finds at least 4 slots idle
    // (one 16-byte vector per row), x, r and p are rewritten as dense blocks of the columns still
    // iterating (row stride kw: the rows stay contiguous in memory), the x of the columns
    // leaving goes to xf in column order, their scalars follow on the host, and every kernel
    // of the following iterations covers the kw slots only, with a launch shape narrowed to
    // that width; slot_col[s] is the column held in slot s.  Each column's arithmetic is
    // unchanged by its slot.
    int kw = ld;          // slots the iterations cover
    int lw = ld;          // row stride of the iteration blocks (kw once compacted)
    bool compacted = false;
    std::vector<double> bn2_col(ld, 0.0);  // ||b_j||^2 by column, kept on the host
    int kcols = k;        // columns the scalar kernels cover (slots past them are idle)
    LaunchCfg wcfg = cfg; // launch shape of the iterations at width kw
    dim3 wgrid = grid, whgrid = hgrid;
    int wP = P, wPH = PH, wcsmem = csmem;  // its row ranges, partial slots and staged slice
    const int32_t* wpart = rpart;
    Segs wsg = sg;  // the scalar kernels' slot layout at that shape
    std::vector<int> slot_col(ld);
    for (int j = 0; j < ld; ++j) slot_col[j] = j;
    auto set_width = [&](int w) -> csc_status {
        kw = w;
        kcols = w < ld ? w : k;
        wcfg = cfg;
        const int nvw = ceil_div(w, 4);
        // lane groups of the next power of two of the width's vectors (NT = 1, one column
        // tile up to 128 columns)
        int G2 = 2;
        while (G2 < nvw && G2 < 32) G2 *= 2;
        if (w < ld) {
            // row ranges, threads and kernel form of a compacted width: pinned or tuned
            // earlier, else tuned now on the compacted blocks with those lane groups and at
            // most max_p row ranges (the partials are sized for them); their cost per
            // iteration grows with the row-range count as the width shrinks
            const uint64_t wkey = (3ull << 48) | (uint64_t)(uint32_t)w;
            LaunchCfg c;
            bool have = false;
            auto it = g->tuned.find(wkey);
            if (it != g->tuned.end()) {
                c = it->second;
                have = true;
            } else if (tune_cache_get(g, wkey, &c)) {
                // tuned on another handle of the same size: its staged slices must fit here
                have = true;
                if (c.staged) {
                    const int32_t* pr = nullptr;
                    CSC_TRY(get_partition(g, c.P, &pr));
                    int room = 0;
                    CG_SWITCH(c, room = cg_staged_room<G_, NT_>());
                    if (staged_smem(g, c.P) > std::min(room, kStagedSmemMax)) have = false;
                }
            }
            if (have && c.P > max_p) have = false;
            if (!have) {
                std::vector<LaunchCfg> wc;
                int wmax = 1;
                CSC_TRY(cg_candidates(g, N, nvw, max_p, G2, &wc, &wmax));
                if (!wc.empty()) {
                    CSC_TRY(tune(wc, w, &c));
                    have = true;
                }
            }
            if (have) {
                g->tuned[wkey] = c;
                tune_cache_put(g, wkey, c);
                wcfg = c;
            } else if (2 * nvw <= cfg.G * cfg.NT) {  // no candidate: narrower lane groups of the tuned shape
                wcfg.G = G2;
                wcfg.NT = 1;
            }
        }
        wcfg.tiles = ceil_div(nvw, wcfg.G * wcfg.NT);
        wP = wcfg.P;
        wPH = wP + H;
        wsg.P = wP;
        CSC_TRY(get_partition(g, wP, &wpart));
        wcsmem = wcfg.staged ? staged_smem(g, wP) : 0;
        CSC_TRY(check_staged_smem(wcsmem));
        int room = 0;
        CG_SWITCH(wcfg, room = cg_staged_room<G_, NT_>());
        if (wcsmem > room) {
            set_error("csc_interpolate: a row range's CSR slice (%d bytes) does not fit beside the CG kernels' "
                      "shared arrays (%d bytes free) at %d columns", wcsmem, room, w);
            return CSC_E_UNSUPPORTED;
        }
        wgrid = dim3(wP, wcfg.tiles);
        whgrid = dim3(H > 0 ? H : 1, wcfg.tiles);
        blkb = (double)N * w * 4.0;
        scal_b = 8.0 * wP * w;
        scal_ax = 8.0 * wPH * w;
        kb.x = kb_ax.x = ceil_div(kcols, 32);
        kb.z = std::max(1, ceil_div(wP, kSliceSlots));
        kb_ax.z = std::max(1, ceil_div(wPH, kSliceSlots));
        return CSC_OK;
    };
    auto apply_A = [&](const float* in, const CgBatch& bb, cudaStream_t s) -> csc_status {
        if (hp) {
            CSC_TRY(poly_apply(g, op, in, t1, s));
            CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_ax", 4.0 * N + 3 * blkb + scal_b, s,
                                       hp_ax_kernel<G_, NT_><<<wgrid, wcfg.threads, 0, s>>>(
                                           in, t1, mask, (float)gamma, Ap, wpart, kw, lw, part, bb)));
            return CSC_OK;
        }
        // t = L^(p-1) in, then Ap = mask*in + gamma * L t with <in, Ap> partials; each product's
        // heavy-row launch runs beside its row-range launch (fork_join)
        const float* cur = in;
        float* bufs[2] = {t1, t2};
        for (int q = 0; q < g_power - 1; ++q) {
            float* o = bufs[q & 1];
            // CSR + row factors, the input block gathered once, the output block written;
            // heavy rows (if any) in their own launch, bytes split by their edge share
            const double lb = csr_b + 2 * blkb;
            const bool win = q == 0;
            auto heavy = [&](cudaStream_t st) -> csc_status {
                if (win)
                    CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_heavy", lb * heavy_frac, st,
                                               lap_heavy_kernel<G_, NT_, true><<<whgrid, kHeavyThreads, 0, st>>>(
                                                   g->row_ptr, g->col_idx, g->dinv, g->invdeg, cur, o, g->heavy, kw,
                                                   lw, bb)));
                else
                    CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_heavy", lb * heavy_frac, st,
                                               lap_heavy_kernel<G_, NT_, false><<<whgrid, kHeavyThreads, 0, st>>>(
                                                   g->row_ptr, g->col_idx, g->dinv, g->invdeg, cur, o, g->heavy, kw,
                                                   lw, bb)));
                return CSC_OK;
            };
            auto light = [&](cudaStream_t st) -> csc_status {
                const double by = lb * (1.0 - heavy_frac);
                if (win)
                    CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap", by, st,
                                                lap_rows<G_, NT_, true>(wcfg, wgrid, wcsmem, st, g, cur, o, wpart, kw,
                                                                        lw, bb)));
                else
                    CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap", by, st,
                                                lap_rows<G_, NT_, false>(wcfg, wgrid, wcsmem, st, g, cur, o, wpart, kw,
                                                                         lw, bb)));
                return CSC_OK;
            };
            CSC_TRY(fork_join(g, s, H > 0, heavy, light));
            cur = o;
        }
        // CSR + row factors + mask, t gathered once, p read, Ap written
        const double ab = csr_b + 4.0 * N + 3 * blkb + scal_ax;
        const bool win = g_power == 1;
        auto heavy = [&](cudaStream_t st) -> csc_status {
            if (win)
                CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_ax_heavy", ab * heavy_frac, st,
                                           lap_ax_heavy_kernel<G_, NT_, true><<<whgrid, kHeavyThreads, 0, st>>>(
                                               g->row_ptr, g->col_idx, g->dinv, g->sqdeg, cur, in, mask, (float)gamma,
                                               Ap, g->heavy, kw, lw, part, wP, wPH, bb)));
            else
                CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_ax_heavy", ab * heavy_frac, st,
                                           lap_ax_heavy_kernel<G_, NT_, false><<<whgrid, kHeavyThreads, 0, st>>>(
                                               g->row_ptr, g->col_idx, g->dinv, g->sqdeg, cur, in, mask, (float)gamma,
                                               Ap, g->heavy, kw, lw, part, wP, wPH, bb)));
            return CSC_OK;
        };
        auto light = [&](cudaStream_t st) -> csc_status {
            const double by = ab * (1.0 - heavy_frac);
            if (win)
                CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_ax", by, st,
                                            lap_ax_rows<G_, NT_, true>(wcfg, wgrid, wcsmem, st, g, cur, in, mask,
                                                                       (float)gamma, Ap, wpart, kw, lw, part, wPH,
                                                                       bb)));
            else
                CG_SWITCH(wcfg, CSC_KLAUNCH("cg_lap_ax", by, st,
                                            lap_ax_rows<G_, NT_, false>(wcfg, wgrid, wcsmem, st, g, cur, in, mask,
                                                                        (float)gamma, Ap, wpart, kw, lw, part, wPH,
                                                                        bb)));
            return CSC_OK;
        };
        return fork_join(g, s, H > 0, heavy, light);
    };
    // `count` CG iterations; between convergence checks they replay as one CUDA graph
    // when no per-launch timing is asked for
    auto iterations = [&](cudaStream_t s, int count) -> csc_status {
        for (int q = 0; q < count; ++q) {
            CSC_TRY(apply_A(p, bt, s));
            CSC_KLAUNCH("cg_scalar", scal_ax, s,
                        cg_alpha_kernel<<<kb_ax, rb, 0, s>>>(part, wPH, wsg, kcols, lw, st, lvl2, red_cnt));
            // x, r, p, Ap read; x, r written
            CG_SWITCH(wcfg, CSC_KLAUNCH("cg_update", 6 * blkb + 4.0 * N + 2 * scal_b, s,
                                       cg_update_kernel<G_, NT_><<<wgrid, wcfg.threads, 0, s>>>(
                                           x, r, p, Ap, st.alpha, gid, pinv, wpart, kw, lw, part, bt)));
            CSC_TRY(reset_active(s));
            CSC_KLAUNCH("cg_scalar", 2 * scal_b, s,
                        cg_beta_kernel<<<kb, rb, 0, s>>>(part, wP, wsg, kcols, lw, st, rel_tol * rel_tol, 0, lvl2,
                                                         red_cnt));
            CG_SWITCH(wcfg, CSC_KLAUNCH("cg_pupdate", 3 * blkb + 4.0 * N, s,
                                       cg_pupdate_kernel<G_, NT_><<<wgrid, wcfg.threads, 0, s>>>(
                                           r, p, st.beta, gid, pinv, wpart, kw, lw, bt)));
        }
        return CSC_OK;
    };
    int it = 0;
    const int check_every = 8;
    bool converged = h_active[0] == 0;
    while (!converged && it < max_iter) {
        const int batch = std::min(check_every, max_iter - it);
        if (!g_prof_enabled && g->use_graphs) {
            char key[320];
            snprintf(key, sizeof(key), "cg:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%d:%.17g:%.17g:%p:%p:%p:%p:%p:%p",
                     batch, ld, k, kw, nseg, g_power, hp ? hp_m : -1, wcfg.G, wcfg.NT, wcfg.threads, wcfg.P, wcfg.tiles,
                     wcfg.staged * 2 + wcfg.lean, gamma, rel_tol,
                     (void*)x, (void*)sd, (void*)part, (void*)d_gk, (const void*)sg.gblk, (const void*)op.coef);
            int64_t launches = 0;
            CSC_TRY(replay_graph(g, key, s, &launches, [&](cudaStream_t cap) { return iterations(cap, batch); }));
        } else {
            CSC_TRY(iterations(s, batch));
        }
        it += batch;
        CSC_CUDA_TRY(cudaMemcpyAsync(h_active, st.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        converged = h_active[0] == 0;
        const int want = ((h_active[0] + 3) / 4) * 4;
        if (compact && !converged && it < max_iter && want <= kw - 4) {
            // new slots: the active ones in slot order, then idle ones up to the width `want`
            // (they stay frozen); the other idle slots leave, their x going to xf
            std::vector<int> act(kw);
            std::vector<double> sc((size_t)5 * kw);
            double* cols[5] = {st.rz, st.bn2, st.alpha, st.beta, st.rr};
            CSC_CUDA_TRY(cudaMemcpyAsync(act.data(), st.active, (size_t)kw * sizeof(int), cudaMemcpyDeviceToHost, s));
            for (int q = 0; q < 5; ++q)
                CSC_CUDA_TRY(cudaMemcpyAsync(sc.data() + (size_t)q * kw, cols[q], (size_t)kw * sizeof(double),
                                             cudaMemcpyDeviceToHost, s));
            CSC_CUDA_TRY(cudaStreamSynchronize(s));
            for (int j = 0; j < kw; ++j) bn2_col[slot_col[j]] = sc[(size_t)kw + j];
            int n_act = 0;
            for (int j = 0; j < kw; ++j) n_act += act[j] ? 1 : 0;
            const int want_w = std::max(want, ((n_act + 3) / 4) * 4);  // every active slot is kept
            std::vector<int32_t> maps;  // [src (want_w) | leaving slots | their columns]
            maps.reserve((size_t)2 * kw);
            for (int j = 0; j < kw; ++j)
                if (act[j]) maps.push_back(j);
            std::vector<int32_t> leave;
            for (int j = 0; j < kw; ++j)
                if (!act[j]) {
                    if ((int)maps.size() < want_w) maps.push_back(j);
                    else leave.push_back(j);
                }
            const int nlv = (int)leave.size();
            std::vector<int> col2(want_w), act2(want_w);
            std::vector<double> sc2((size_t)5 * want_w);
            for (int j = 0; j < want_w; ++j) {
                col2[j] = slot_col[maps[j]];
                act2[j] = act[maps[j]];
                for (int q = 0; q < 5; ++q) sc2[(size_t)q * want_w + j] = sc[(size_t)q * kw + maps[j]];
            }
            for (int q = 0; q < nlv; ++q) maps.push_back(leave[q]);
            for (int q = 0; q < nlv; ++q) maps.push_back(slot_col[leave[q]]);
            std::copy(col2.begin(), col2.end(), slot_col.begin());
            CSC_CUDA_TRY(cudaMemcpyAsync(d_src, maps.data(), maps.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            CSC_CUDA_TRY(
                cudaMemcpyAsync(st.active, act2.data(), (size_t)want_w * sizeof(int), cudaMemcpyHostToDevice, s));
            for (int q = 0; q < 5; ++q)
                CSC_CUDA_TRY(cudaMemcpyAsync(cols[q], sc2.data() + (size_t)q * want_w,
                                             (size_t)want_w * sizeof(double), cudaMemcpyHostToDevice, s));
            // t1, t2 and Ap hold nothing between iterations: they take the dense blocks, and the
            // old x, r, p become the scratch
            CSC_KLAUNCH("cg_compact", 4.0 * N * (3.0 * kw + 3.0 * want_w + 2.0 * nlv), s,
                        compact_columns_kernel<<<(int)std::min<int64_t>(ceil_div(N, 8), g->num_sms * 16), 256, 0,
                                                 s>>>(x, r, p, lw, t1, t2, Ap, want_w, d_src, want_w, d_src + want_w,
                                                      d_src + want_w + nlv, nlv, xf, ld, N));
            std::swap(x, t1);
            std::swap(r, t2);
            std::swap(p, Ap);
            // the host vectors above are released when this scope ends: wait for the copies
            CSC_CUDA_TRY(cudaStreamSynchronize(s));
            compacted = true;
            lw = want_w;
            CSC_TRY(set_width(want_w));
        }
    }
    if (compacted) {
        // the columns still in slots go to xf too, which then holds every column's x; the
        // final residual and the labels run on it at full width
        std::vector<double> sc(kw);
        CSC_CUDA_TRY(cudaMemcpyAsync(sc.data(), st.bn2, (size_t)kw * sizeof(double), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        for (int j = 0; j < kw; ++j) bn2_col[slot_col[j]] = sc[j];
        std::vector<int32_t> maps((size_t)2 * kw);
        for (int j = 0; j < kw; ++j) {
            maps[j] = j;
            maps[(size_t)kw + j] = slot_col[j];
        }
        CSC_CUDA_TRY(cudaMemcpyAsync(d_src, maps.data(), maps.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        CSC_CUDA_TRY(cudaMemcpyAsync(st.bn2, bn2_col.data(), (size_t)ld * sizeof(double), cudaMemcpyHostToDevice, s));
        CSC_KLAUNCH("cg_compact", 8.0 * N * kw, s,
                    compact_columns_kernel<<<(int)std::min<int64_t>(ceil_div(N, 8), g->num_sms * 16), 256, 0, s>>>(
                        x, r, p, lw, t1, t2, Ap, 0, d_src, 0, d_src, d_src + kw, kw, xf, ld, N));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        x = xf;
        lw = ld;
        for (int j = 0; j < ld; ++j) slot_col[j] = j;
    }
    if (compact) CSC_TRY(set_width(ld));
    // true residual ||b - A x|| / ||b|| per column
    CSC_TRY(apply_A(x, bt_all, s));
    CG_SWITCH(cfg, CSC_KLAUNCH("cg_residual", blkb + 4.0 * N, s,
                               residual_kernel<G_, NT_><<<grid, th, 0, s>>>(Ap, slab, bfull, rpart, ld, ld, part,
                                                                            bt_all)));
    CSC_KLAUNCH("cg_scalar", scal_b, s,
                column_sum_kernel<<<kb, rb, 0, s>>>(part, P, sg, k, ld, st.rr, lvl2, red_cnt));
    // labels
    CG_SWITCH(cfg, CSC_KLAUNCH("label_norms", blkb, s,
                               colnorm_kernel<G_, NT_><<<grid, th, 0, s>>>(x, rpart, ld, ld, part, bt_all)));
    CSC_KLAUNCH("cg_scalar", scal_b, s,
                column_sum_kernel<<<kb, rb, 0, s>>>(part, P, sg, k, ld, norm2, lvl2, red_cnt));
    CSC_KLAUNCH("label_argmax", 24.0 * sl, s,
                label_scale_kernel<<<ceil_div((int64_t)sl, 256), 256, 0, s>>>(norm2, (int64_t)sl, nrm, rnrm));
    {
        int lgrid = ceil_div(N, 8);  // a warp per row, 8 per CTA
        if (lgrid > g->num_sms * 16) lgrid = g->num_sms * 16;
        CSC_KLAUNCH("label_argmax", blkb + 4.0 * N + (fuzzy_out ? (double)N * k * 4 : 0.0), s,
                    label_argmax_kernel<<<lgrid, 256, 0, s>>>(x, nrm, rnrm, N, k, ld, d_gk, gid, g->perm,
                                                              labels_out, fuzzy_out));
    }
    std::vector<double> rr(sl), bn(sl);
    CSC_CUDA_TRY(cudaMemcpyAsync(rr.data(), st.rr, sl * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(bn.data(), st.bn2, sl * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int q = 0; q < nseg; ++q)
        for (int j = 0; j < k; ++j) {
            const size_t i = (size_t)q * ld + j;
            if (bn[i] > 0) worst = std::max(worst, sqrt(rr[i] / bn[i]));
        }
    if (info) {
        info->iters = it;
        info->converged = converged ? 1 : 0;
        info->max_rel_residual = worst;
    }
    if (!converged) {
        set_error("csc_interpolate: CG reached max_iter = %d (max relative residual %.3g)", max_iter, worst);
        return CSC_E_NOT_CONVERGED;
    }
    return CSC_OK;
}

}  // namespace csc
