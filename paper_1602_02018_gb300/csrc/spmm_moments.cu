// spmm_moments.cu -- the eigencount moment steps of Sec. 4.3: the three-term
// recurrence on the probe block with fp64 block partials of the inner products.
#include "spmm.cuh"

namespace csc {

// ------------------------------------------------------------------- K2
// Moment step on the pre-scaled probes Z = s X: like cheb_step without Y; block
// partials of three fp64 sums of X-space inner products, <X_a, X_b> =
// sum_i d_i <Z_a, Z_b>_i (d_i -> 1 for an isolated node):
//   first: s0 = <X0,X0>, s1 = <X1,X0>, s2 = <X1,X1>
//   later: s1 = <X_{j+1},X_j>, s2 = <X_{j+1},X_{j+1}>
// The row's Z_j and Z_{j-1} (not on the first step), loaded before the neighbour sum.
template <typename T, int NT>
struct MomOperands {
    typename StoreTraits<T>::raw_t zc[NT], zp[NT];
    __device__ __forceinline__ void load(int row, int lane, int G, int col0, int tcols, int first,
                                         const T* __restrict__ zcur, const T* __restrict__ zprev, int64_t ld) {
        using Tr = StoreTraits<T>;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int cl = (t * G + lane) * Tr::VEC;
            if (cl >= tcols) continue;
            const int64_t o = (int64_t)row * ld + col0 + cl;
            zc[t] = Tr::ld_raw(zcur + o);
            if (!first) zp[t] = Tr::ld_raw_cs(zprev + o);
        }
    }
};

// One row of the moment step: Z_{j+1} of the row's columns of this tile, and the
// row's fp32 products <z_c, z_c>, <z_n, z_c>, <z_n, z_n> summed over them.
template <typename T, int G, int NT>
__device__ __forceinline__ void mom_epilogue(int row, int lane, int col0, int tcols, float (&acc)[NT][StoreTraits<T>::VEC],
                                             const float* __restrict__ invdeg, T* __restrict__ zprev_next, int64_t ld,
                                             int first, const MomOperands<T, NT>& op, float& p0, float& p1,
                                             float& p2) {
    using Tr = StoreTraits<T>;
    constexpr int VEC = Tr::VEC;
    const float f = (first ? -1.0f : -2.0f) * invdeg[row];
    p0 = p1 = p2 = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int cl = (t * G + lane) * VEC;
        if (cl >= tcols) continue;
        const int c = col0 + cl;
        float zc[VEC], zn[VEC];
        Tr::unraw(op.zc[t], zc);
        T* zp_ptr = zprev_next + (int64_t)row * ld + c;
        if (first) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) zn[v] = Tr::round(f * acc[t][v]);
        } else {
            float zp[VEC];
            Tr::unraw(op.zp[t], zp);
#pragma unroll
            for (int v = 0; v < VEC; ++v) zn[v] = Tr::round(f * acc[t][v] - zp[v]);
        }
        Tr::store(zp_ptr, zn);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            p0 = fmaf(zc[v], zc[v], p0);
            p1 = fmaf(zn[v], zc[v], p1);
            p2 = fmaf(zn[v], zn[v], p2);
        }
    }
}

// Block partials of the three sums -> partials[slot * 3 + q]: the threads' compensated
// fp32 sums added as fp32 pairs across the block (no fp64 instruction per thread) and
// converted to fp64 once.
__device__ __forceinline__ void mom_block_partials(const KSum (&s)[3], int64_t slot, double* __restrict__ partials) {
    __shared__ float2 red[3][32];
    FF v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = warp_sum_ff(s[q].pair());
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) red[q][w] = make_float2(v[q].hi, v[q].lo);
    __syncthreads();
    if (threadIdx.x < 3) {
        FF t{0.f, 0.f};
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            const float2 e = red[threadIdx.x][i];
            t = ff_add(t, FF{e.x, e.y});
        }
        partials[slot * 3 + threadIdx.x] = t.value();
    }
}

template <typename T, int G, int NT, bool STAGED>
__global__ void __launch_bounds__(512)
mom_step_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const int32_t* __restrict__ lrp,
                const int32_t* __restrict__ lci, const float* __restrict__ invdeg,
                const int32_t* __restrict__ deg, const T* __restrict__ zcur, T* __restrict__ zprev_next,
                const int32_t* __restrict__ part, int ncols, int64_t ld, int first, double* __restrict__ partials) {
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int tcols = min(TW, ncols - col0);
    const int r1 = part[blockIdx.x + 1];
    KSum sums[3];
    extern __shared__ int32_t s_csr[];
    sweep_rows<STAGED, G>(rp, ci, lrp, lci, part[blockIdx.x], r1, s_csr, [&](int row, int e0, int e1,
                                                                            const int32_t* idx) {
        MomOperands<T, NT> op;
        op.load(row, lane, G, col0, tcols, first, zcur, zprev_next, ld);
        float acc[NT][VEC];
        gather_any<STAGED, T, G, NT, false, float>(e0, e1, idx, nullptr, zcur + col0, ld, lane, tcols, acc);
        float p0, p1, p2;
        mom_epilogue<T, G, NT>(row, lane, col0, tcols, acc, invdeg, zprev_next, ld, first, op, p0, p1, p2);
        // the row's degree (d_i of the X-space inner product) is its edge count (exact in fp32)
        const float wr = e1 > e0 ? (float)(e1 - e0) : 1.f;
        sums[0].add(wr * p0);
        sums[1].add(wr * p1);
        sums[2].add(wr * p2);
    });
    mom_block_partials(sums, (int64_t)blockIdx.y * gridDim.x + blockIdx.x, partials);
}

// Heavy rows: one CTA per row; partial slots after the regular blocks' (slot_base).
template <typename T, int G, int NT>
__global__ void __launch_bounds__(kHeavyThreads)
mom_step_heavy_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                      const float* __restrict__ invdeg, const int32_t* __restrict__ deg, const T* __restrict__ zcur,
                      T* __restrict__ zprev_next, const int32_t* __restrict__ heavy, int ncols, int64_t ld, int first,
                      double* __restrict__ partials, int64_t slot_base) {
    constexpr int VEC = StoreTraits<T>::VEC;
    constexpr int TW = G * NT * VEC;
    const int lane = threadIdx.x % G;
    const int col0 = blockIdx.y * TW;
    const int tcols = min(TW, ncols - col0);
    const int row = heavy[blockIdx.x];
    float acc[NT][VEC];
    gather_heavy<T, G, NT, false, float>(__ldg(rp + row), __ldg(rp + row + 1), ci, nullptr, zcur + col0, ld, lane,
                                         tcols, acc);
    KSum sums[3];
    if (threadIdx.x < G) {
        MomOperands<T, NT> op;
        op.load(row, lane, G, col0, tcols, first, zcur, zprev_next, ld);
        float p0, p1, p2;
        mom_epilogue<T, G, NT>(row, lane, col0, tcols, acc, invdeg, zprev_next, ld, first, op, p0, p1, p2);
        const float wr = (float)deg[row];
        sums[0].add(wr * p0);
        sums[1].add(wr * p1);
        sums[2].add(wr * p2);
    }
    mom_block_partials(sums, slot_base + (int64_t)blockIdx.y * gridDim.x + blockIdx.x, partials);
}

template <typename T>
csc_status launch_mom_step(Graph* g, const LaunchCfg& cfg, const T* xcur, T* xpn, int ncols, int64_t ld,
                                  int first, double* partials, cudaStream_t s) {
    const double bytes = 4.0 * g->nnz + 8.0 * g->N + 4.0 + (first ? 2.0 : 3.0) * (double)g->N * ncols * sizeof(T);
    const int32_t* part = nullptr;
    CSC_TRY(get_partition(g, cfg.P, &part));
    const int smem = cfg.staged ? staged_smem(g, cfg.P) : 0;  // the CTA's CSR slice (stage_csr)
    CSC_TRY(check_staged_smem(smem));
    const dim3 grid(cfg.P, cfg.tiles);
    // heavy rows' partial sums go to the slots after the row-range blocks'
    const dim3 hgrid(g->n_heavy > 0 ? g->n_heavy : 1, cfg.tiles);
    auto heavy = [&](cudaStream_t st) -> csc_status {
        CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("mom_step_heavy", 0.0, st,
                                          mom_step_heavy_kernel<T, GG, NN><<<hgrid, kHeavyThreads, 0, st>>>(
                                              g->row_ptr, g->col_idx, g->invdeg, g->deg, xcur, xpn, g->heavy, ncols,
                                              ld, first, partials, (int64_t)cfg.P * cfg.tiles)));
        return CSC_OK;
    };
    auto light = [&](cudaStream_t st) -> csc_status {
        if (cfg.staged)
            CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("mom_step", bytes, st,
                                              mom_step_kernel<T, GG, NN, true><<<grid, cfg.threads, smem, st>>>(
                                                  g->row_ptr, g->col_idx, g->lrp, g->lci, g->invdeg, g->deg, xcur,
                                                  xpn, part, ncols, ld, first, partials)));
        else
            CSC_SHAPE_SWITCH(cfg, CSC_KLAUNCH("mom_step", bytes, st,
                                              mom_step_kernel<T, GG, NN, false><<<grid, cfg.threads, 0, st>>>(
                                                  g->row_ptr, g->col_idx, g->lrp, g->lci, g->invdeg, g->deg, xcur,
                                                  xpn, part, ncols, ld, first, partials)));
        return CSC_OK;
    };
    return fork_join(g, s, g->n_heavy > 0, heavy, light);
}

template <typename T>
int mom_occupancy(const TileShape& sh, int threads) {
    int occ = 1;
#define CSC_OCC_CASE(GG, NN) \
    if (sh.G == GG && sh.NT == NN) occ = occupancy(mom_step_kernel<T, GG, NN, true>, threads);
    CSC_OCC_CASE(2, 1) CSC_OCC_CASE(2, 2) CSC_OCC_CASE(2, 3) CSC_OCC_CASE(4, 1) CSC_OCC_CASE(4, 2)
    CSC_OCC_CASE(4, 3) CSC_OCC_CASE(8, 1) CSC_OCC_CASE(8, 2) CSC_OCC_CASE(8, 3) CSC_OCC_CASE(16, 1)
    CSC_OCC_CASE(16, 2) CSC_OCC_CASE(32, 1) CSC_OCC_CASE(32, 2)
#undef CSC_OCC_CASE
    return occ;
}

#define CSC_INST(T)                                                                                          \
    template csc_status launch_mom_step<T>(Graph*, const LaunchCfg&, const T*, T*, int, int64_t, int, double*, \
                                           cudaStream_t);                                                    \
    template int mom_occupancy<T>(const TileShape&, int);
CSC_INST(float)
CSC_INST(__nv_bfloat16)
#undef CSC_INST

}  // namespace csc
