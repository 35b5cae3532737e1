// spmm_clenshaw.cu -- the Chebyshev filter evaluated by Clenshaw's backward recurrence
// (one launch per order; the row-range kernel and the heavy-row kernel).
#include "spmm.cuh"

namespace csc {

// ------------------------------------------------------- K4 (Clenshaw form)
// The same Y = sum_j c_j T_j(L - I) R evaluated by Clenshaw's backward recurrence
// (Clenshaw 1955): b_j = c_j R + 2 (L - I) b_{j+1} - b_{j+2} for j = m-1 .. 1 from
// b_m = c_m R, b_{m+1} = 0, and Y = c_0 R + (L - I) b_1 - b_2.  In the pre-scaled form
// B_j = s b_j:  B_j = c_j s R - 2 D^-1 W B_{j+1} - B_{j+2},  Y = D^1/2 (c_0 s R -
// D^-1 W B_1 - B_2).  Each order gathers B_{j+1}, reads B_{j+2} and overwrites it
// with B_j; the block s R is stored once in the storage type and read back every
// order instead of accumulating Y in memory, so an order moves 4 N d stored values
// plus the CSR instead of 3 N d stored plus 2 N d accumulator values.  The last
// order writes Y (optionally normalised per row when one column tile holds the
// whole row).

// Operands of one row of a Clenshaw order that do not depend on the gather: s R and
// B_{j+2} (none on the first order, j = m-1), loaded before the neighbour sum so their
// latency overlaps it.  mode bits as in clenshaw_epilogue.
template <typename T, int G, int NT>
struct ClenOperands {
    typename StoreTraits<T>::raw_t r[NT], b2[NT];
    typename StoreTraits<T>::acc_t inv;  // 1 / d_i (0 for an isolated node)
    __device__ __forceinline__ void load(int row, int lane, int col0, int tcols, int mode, const T* __restrict__ rs,
                                         const T* __restrict__ bpp, int64_t ld,
                                         const typename StoreTraits<T>::acc_t* __restrict__ invdeg) {
        using Tr = StoreTraits<T>;
        constexpr int VEC = Tr::VEC;
        const bool first = (mode & 1) != 0, keep = (mode & 4) != 0;
        inv = invdeg[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * VEC;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            // s R and B_{j+2} are dead after this order: evict-first unless all fits L2, so
            // the gathered B_{j+1} and the B_j written here (gathered next) stay resident
            r[t] = keep ? Tr::ld_raw(rs + o) : Tr::ld_raw_cs(rs + o);
            if (!first) b2[t] = keep ? Tr::ld_raw(bpp + o) : Tr::ld_raw_cs(bpp + o);
        }
    }
};

// Row epilogue of one Clenshaw order.  mode: 1 = no B_{j+2} (j = m-1), 2 = last
// order (write Y), 4 = plain caching (working set fits L2), 8 = normalise Y rows
// (the group's lanes hold the whole row; gmask = the group's lanes).
// op: the row's s R (the block stored in T, internal row order) and B_{j+2}.  LAST:
// the order j = 0 (writes Y); a separate instantiation so the other orders carry no Y
// state.
template <typename T, int G, int NT, bool LAST>
__device__ __forceinline__ void clenshaw_epilogue(int row, int lane, int col0, int tcols,
                                                  typename StoreTraits<T>::acc_t (&acc)[NT][StoreTraits<T>::VEC],
                                                  const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                                                  const typename StoreTraits<T>::acc_t* __restrict__ sqdeg,
                                                  T* __restrict__ bpp, typename StoreTraits<T>::acc_t* __restrict__ Y,
                                                  const int32_t* __restrict__ perm, int64_t ld,
                                                  typename StoreTraits<T>::acc_t cj, int mode,
                                                  const ClenOperands<T, G, NT>& op, unsigned gmask) {
    using Tr = StoreTraits<T>;
    using A = typename Tr::acc_t;
    constexpr int VEC = Tr::VEC;
    const bool first = (mode & 1) != 0;
    constexpr bool last = LAST;
    const A f = (last ? A(-1) : A(-2)) * op.inv;
    A out[LAST ? NT : 1][VEC];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * VEC;
        if (cl >= tcols) continue;
        const int c = col0 + cl;
        const int to = LAST ? t : 0;
        A r[VEC], b2[VEC];
        Tr::unraw(op.r[t], r);
        if (first) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) b2[v] = A(0);
        } else {
            Tr::unraw(op.b2[t], b2);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) out[to][v] = cj * r[v] + f * acc[t][v] - b2[v];
        if constexpr (!LAST) {
            A bn[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) bn[v] = Tr::round(out[0][v]);
            Tr::store(bpp + (int64_t)row * ld + c, bn);
        }
    }
    if constexpr (!LAST) return;
    else {
    // the row norm in the accumulator type (fp32 for fp32 and bf16 storage: fp64
    // instructions issue at a small fraction of the fp32 rate on this part)
    const A back = sqdeg[row];
    A inv = A(1);
    if (mode & 8) {
        A ss = A(0);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * VEC;
            if (cl >= tcols) continue;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const A y = out[t][v] * back;
                ss += y * y;
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(gmask, ss, o, G);
        if (ss > A(0)) inv = A(1) / sqrt(ss);
    }
    const int64_t yrow = perm ? (int64_t)perm[row] : (int64_t)row;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * VEC;
        if (cl >= tcols) continue;
        A y[VEC];
        if (mode & 8) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = (out[t][v] * back) * inv;
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) y[v] = out[t][v] * back;
        }
        AccIO<A, VEC>::store(Y + yrow * ld + col0 + cl, y);
    }
    }
}

template <typename T, int G, int NT, bool LAST, bool STAGED, bool LEAN>
__global__ void __launch_bounds__(LEAN ? 256 : 512, LEAN ? 5 : 0)
clenshaw_step_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ lrp,
                     const int32_t* __restrict__ lci,
                     const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                     const typename StoreTraits<T>::acc_t* __restrict__ sqdeg,
                     const T* __restrict__ bnext, T* __restrict__ bpp, typename StoreTraits<T>::acc_t* __restrict__ Y,
                     const int32_t* __restrict__ perm, const int32_t* __restrict__ part, int ncols, int64_t ld,
                     typename StoreTraits<T>::acc_t cj, int mode, CoefTab<typename StoreTraits<T>::acc_t> tab,
                     const T* __restrict__ rs) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int r0 = part[blockIdx.x], r1 = part[blockIdx.x + 1];
    // a batch whose graphs carry fewer columns than the block: only the range's graph's
    const int ncols_b = (tab.gcols && r0 < r1) ? min(ncols, tab.gcols[tab.gid[r0]]) : ncols;
    const int tcols = min(TW, ncols_b - col0);
    if (tcols <= 0) return;
    if (tab.c && r0 < r1) cj = (tab.gid ? tab.c + (int64_t)tab.gid[r0] * tab.stride : tab.c)[tab.j];
    const unsigned gmask =
        G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(G - 1)));
    extern __shared__ int32_t s_csr[];
    sweep_rows<STAGED, G>(rp, ci, lrp, lci, r0, r1, s_csr, [&](int row, int e0, int e1, const int32_t* idx) {
        ClenOperands<T, G, NT> op;
        op.load(row, lane, col0, tcols, mode, rs, bpp, ld, invdeg);
        A acc[NT][VEC];
        gather_any<STAGED, T, G, NT, false, A, LEAN>(e0, e1, idx, nullptr, bnext + col0, ld, lane, tcols, acc);
        clenshaw_epilogue<T, G, NT, LAST>(row, lane, col0, tcols, acc, invdeg, sqdeg, bpp, Y, perm, ld, cj, mode, op,
                                          gmask);
    });
}

template <typename T, int G, int NT>
__global__ void __launch_bounds__(kHeavyThreads)
clenshaw_step_heavy_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const typename StoreTraits<T>::acc_t* __restrict__ invdeg,
                           const typename StoreTraits<T>::acc_t* __restrict__ sqdeg,
                           const T* __restrict__ bnext, T* __restrict__ bpp,
                           typename StoreTraits<T>::acc_t* __restrict__ Y, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ heavy, int ncols, int64_t ld, typename StoreTraits<T>::acc_t cj,
                           int mode, CoefTab<typename StoreTraits<T>::acc_t> tab, const T* __restrict__ rs) {
    using A = typename StoreTraits<T>::acc_t;
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int row = heavy[blockIdx.x];
    const int tcols = min(TW, (tab.gcols ? min(ncols, tab.gcols[tab.gid[row]]) : ncols) - col0);
    if (tcols <= 0) return;
    if (tab.c) cj = (tab.gid ? tab.c + (int64_t)tab.gid[row] * tab.stride : tab.c)[tab.j];
    A acc[NT][VEC];
    gather_heavy<T, G, NT, false, A>(__ldg(rp + row), __ldg(rp + row + 1), ci, nullptr, bnext + col0, ld, lane, tcols,
                                     acc);
    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    if (threadIdx.x < G) {
        ClenOperands<T, G, NT> op;
        op.load(row, lane, col0, tcols, mode, rs, bpp, ld, invdeg);
        if (mode & 2)
            clenshaw_epilogue<T, G, NT, true>(row, lane, col0, tcols, acc, invdeg, sqdeg, bpp, Y, perm, ld, cj, mode,
                                              op, gmask);
        else
            clenshaw_epilogue<T, G, NT, false>(row, lane, col0, tcols, acc, invdeg, sqdeg, bpp, Y, perm, ld, cj, mode,
                                               op, gmask);
    }
}

// One Clenshaw order (see clenshaw_step_kernel): the heavy rows beside the row ranges.
template <typename T>
csc_status launch_clenshaw_step(Graph* g, const LaunchCfg& cfg, const T* bnext, T* bpp,
                                       typename StoreTraits<T>::acc_t* Y, int ncols, int64_t ld, double cj, int mode,
                                       const T* rs, cudaStream_t s, CoefTab<typename StoreTraits<T>::acc_t> tab,
                                       bool internal) {
    const int32_t* perm = internal ? nullptr : g->perm;  // internal: Y rows in internal order
    using A = typename StoreTraits<T>::acc_t;
    const A *idg, *sqd;
    if constexpr (sizeof(A) == 8) {
        idg = g->invdeg64;
        sqd = g->sqdeg64;
    } else {
        idg = g->invdeg;
        sqd = g->sqdeg;
    }
    const double ws = (double)g->N * ld * 3.0 * sizeof(T) + 4.0 * g->nnz + 8.0 * g->N;
    if (ws <= kKeepL2Fraction * (double)g->l2_bytes) mode |= 4;
    const int32_t* part = nullptr;
    CSC_TRY(get_partition(g, cfg.P, &part));
    const int smem = cfg.staged ? staged_smem(g, cfg.P) : 0;  // the CTA's CSR slice (stage_csr)
    CSC_TRY(check_staged_smem(smem));
    const dim3 grid(cfg.P, cfg.tiles);
    // algorithmic bytes of one order: CSR + row factors, B_{j+1} gathered once, B_{j+2} read
    // (not on the first order), B_j written (not on the last), Y written (last), s R read
    const double nx = (double)g->N * ncols;
    const bool first = mode & 1, last = mode & 2;
    const double all_bytes = 4.0 * g->nnz + 4.0 * (g->N + 1) + (double)sizeof(A) * g->N * (last ? 2 : 1) +
                             nx * sizeof(T) * (2.0 + (first ? 0.0 : 1.0) + (last ? 0.0 : 1.0)) +
                             (last ? nx * sizeof(A) : 0.0);
    const double heavy_edges = (double)g->nnz - (double)g->h_light[g->N];
    const double heavy_frac = g->n_heavy ? (heavy_edges + g->n_heavy) / ((double)g->nnz + g->N) : 0.0;
    const dim3 hgrid(g->n_heavy > 0 ? g->n_heavy : 1, cfg.tiles);
    auto heavy = [&](cudaStream_t st) -> csc_status {
        CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("cheb_step_heavy", all_bytes * heavy_frac, st,
                                          clenshaw_step_heavy_kernel<T, GG, NN><<<hgrid, kHeavyThreads, 0, st>>>(
                                              g->row_ptr, g->col_idx, idg, sqd, bnext, bpp, Y, perm, g->heavy,
                                              ncols, ld, (A)cj, mode, tab, rs)));
        return CSC_OK;
    };
    auto light = [&](cudaStream_t st) -> csc_status {
        const double lb = all_bytes * (1.0 - heavy_frac);
        // the lean form is compiled for NT = 1 only (LaunchCfg::lean)
#define CSC_CLEN(LASTV, STG, LN)                                                                              \
    CSC_SHAPE_SWITCH(cfg, if constexpr (!(LN) || NN == 1) {                                                   \
        CSC_KLAUNCH("cheb_step", lb, st,                                                                      \
                    (clenshaw_step_kernel<T, GG, NN, LASTV, STG, LN><<<grid, cfg.threads, (STG) ? smem : 0, st>>>( \
                        g->row_ptr, g->col_idx, g->lrp, g->lci, idg, sqd, bnext, bpp, Y, perm, part, ncols, ld,    \
                        (A)cj, mode, tab, rs)));                                                              \
    } else {                                                                                                  \
        set_error("the lean Clenshaw kernel needs NT = 1");                                                   \
        return CSC_E_UNSUPPORTED;                                                                             \
    })
        if (cfg.lean) {
            if (last && cfg.staged) CSC_CLEN(true, true, true);
            else if (last) CSC_CLEN(true, false, true);
            else if (cfg.staged) CSC_CLEN(false, true, true);
            else CSC_CLEN(false, false, true);
        } else {
            if (last && cfg.staged) CSC_CLEN(true, true, false);
            else if (last) CSC_CLEN(true, false, false);
            else if (cfg.staged) CSC_CLEN(false, true, false);
            else CSC_CLEN(false, false, false);
        }
#undef CSC_CLEN
        return CSC_OK;
    };
    return fork_join(g, s, g->n_heavy > 0, heavy, light);
}

template <typename T>
int clenshaw_occupancy(const TileShape& sh, int threads, bool lean) {
    int occ = 1;
    if (lean) {
        if (sh.NT != 1) return 1;
#define CSC_OCC_LEAN(GG) \
    if (sh.G == GG) occ = occupancy(clenshaw_step_kernel<T, GG, 1, false, true, true>, threads);
        CSC_OCC_LEAN(2) CSC_OCC_LEAN(4) CSC_OCC_LEAN(8) CSC_OCC_LEAN(16) CSC_OCC_LEAN(32)
#undef CSC_OCC_LEAN
        return occ;
    }
#define CSC_OCC_CASE(GG, NN) \
    if (sh.G == GG && sh.NT == NN) occ = occupancy(clenshaw_step_kernel<T, GG, NN, false, true, false>, threads);
    CSC_OCC_CASE(2, 1) CSC_OCC_CASE(2, 2) CSC_OCC_CASE(2, 3) CSC_OCC_CASE(4, 1) CSC_OCC_CASE(4, 2)
    CSC_OCC_CASE(4, 3) CSC_OCC_CASE(8, 1) CSC_OCC_CASE(8, 2) CSC_OCC_CASE(8, 3) CSC_OCC_CASE(16, 1)
    CSC_OCC_CASE(16, 2) CSC_OCC_CASE(32, 1) CSC_OCC_CASE(32, 2)
#undef CSC_OCC_CASE
    return occ;
}

#define CSC_INST(T)                                                                                             \
    template csc_status launch_clenshaw_step<T>(Graph*, const LaunchCfg&, const T*, T*,                        \
                                                typename StoreTraits<T>::acc_t*, int, int64_t, double, int,     \
                                                const T*, cudaStream_t, CoefTab<typename StoreTraits<T>::acc_t>, \
                                                bool);                                                          \
    template int clenshaw_occupancy<T>(const TileShape&, int, bool);
CSC_INST(float)
CSC_INST(__nv_bfloat16)
CSC_INST(double)
#undef CSC_INST

}  // namespace csc
