// cg.cu -- label interpolation (Alg. 2 step 7, Eq. 5) and the partition rule of Sec. 4.1.
//
// For every cluster j the minimiser of ||M x - c_j^r||^2 + gamma x^T L^p x solves
// (M^T M + gamma L^p) x_j = M^T c_j^r.  All k systems are solved together by
// Jacobi-preconditioned conjugate gradients on an N x k row-major fp32 block
// (one independent CG per column; per-column inner products in fp64 with
// fixed-order reductions).  A p = mask * p + gamma L^p p is computed with p
// sparse passes L t = t - S t (S = D^-1/2 W D^-1/2 rebuilt from the degree
// vector), the last one fused with the mask term and the <p, A p> partials.
// Preconditioner: diag(M^T M) + gamma (diag(L) = 1).
// Labels: node i -> argmax_j x_j(i) / ||x_j|| (ties to the lowest j).
#include <math.h>

#include <vector>

#include "common.cuh"
#include "device.cuh"

namespace csc {

constexpr int kCgThreads = 256;

// Per-block, per-column fp64 partial sums: every thread holds sums for its
// NT*4 columns; threads of equal lane across the block's groups are summed
// in group order, then written to partials[block * ld + col].
template <int G, int NT, int NS>
__device__ __forceinline__ void block_column_partials(double (&acc)[NS][NT][4], int lane, int ncols, int64_t ldp,
                                                      double* __restrict__ partials) {
    constexpr int GROUPS = kCgThreads / G;
    constexpr int COLS = G * NT * 4;
    __shared__ double red[GROUPS * COLS];
    const int grp = threadIdx.x / G;
    for (int s = 0; s < NS; ++s) {
        __syncthreads();
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int v = 0; v < 4; ++v) red[grp * COLS + (t * G + lane) * 4 + v] = acc[s][t][v];
        __syncthreads();
        for (int c = threadIdx.x; c < COLS && c < ncols; c += kCgThreads) {
            double sum = 0.0;
            for (int q = 0; q < GROUPS; ++q) sum += red[q * COLS + c];
            partials[((int64_t)s * gridDim.x + blockIdx.x) * ldp + c] = sum;
        }
    }
}

// out = in - S in   (L applied to every column)
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
lap_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const float* __restrict__ dinv,
           const float* __restrict__ in, float* __restrict__ out, int32_t N, int ncols, int64_t ld) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t r = group; r < N; r += ngroups) {
        const int row = (int)r;
        float acc[NT][4];
        gather_row<float, G, NT>(rp, ci, dinv, in, ld, row, lane, ncols, acc);
        const float di = dinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            float x[4];
            StoreTraits<float>::load(in + (int64_t)row * ld + c, x);
#pragma unroll
            for (int v = 0; v < 4; ++v) x[v] = x[v] - di * acc[t][v];
            StoreTraits<float>::store(out + (int64_t)row * ld + c, x);
        }
    }
}

// Ap = mask * p + gamma (t - S t), with per-column partials of <p, Ap>.
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
lap_ax_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const float* __restrict__ dinv,
              const float* __restrict__ tin, const float* __restrict__ p, const float* __restrict__ mask, float gamma,
              float* __restrict__ Ap, int32_t N, int ncols, int64_t ld, double* __restrict__ partials) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    double dot[1][NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) dot[0][t][v] = 0.0;
    for (int64_t r = group; r < N; r += ngroups) {
        const int row = (int)r;
        float acc[NT][4];
        gather_row<float, G, NT>(rp, ci, dinv, tin, ld, row, lane, ncols, acc);
        const float di = dinv[row];
        const float mk = mask[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            float tt[4], pp[4], a[4];
            StoreTraits<float>::load(tin + (int64_t)row * ld + c, tt);
            StoreTraits<float>::load(p + (int64_t)row * ld + c, pp);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                a[v] = mk * pp[v] + gamma * (tt[v] - di * acc[t][v]);
                dot[0][t][v] += (double)pp[v] * (double)a[v];
            }
            StoreTraits<float>::store(Ap + (int64_t)row * ld + c, a);
        }
    }
    block_column_partials<G, NT, 1>(dot, lane, ncols, ld, partials);
}

// x += alpha p; r -= alpha Ap; partials of <r, r/P> and <r, r>.  alpha == nullptr: no update.
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
cg_update_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                 const float* __restrict__ Ap, const double* __restrict__ alpha, const float* __restrict__ pinv,
                 int32_t N, int ncols, int64_t ld, double* __restrict__ partials) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    double dots[2][NT][4];
    float al[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            dots[0][t][v] = 0.0;
            dots[1][t][v] = 0.0;
            const int c = (t * G + lane) * 4 + v;
            al[t][v] = (alpha && c < ncols) ? (float)alpha[c] : 0.f;
        }
    for (int64_t rr = group; rr < N; rr += ngroups) {
        const int row = (int)rr;
        const float pi = pinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            const int64_t o = (int64_t)row * ld + c;
            float rv[4];
            StoreTraits<float>::load(r + o, rv);
            if (alpha) {
                float xv[4], pv[4], av[4];
                StoreTraits<float>::load(x + o, xv);
                StoreTraits<float>::load(p + o, pv);
                StoreTraits<float>::load(Ap + o, av);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    xv[v] = fmaf(al[t][v], pv[v], xv[v]);
                    rv[v] = fmaf(-al[t][v], av[v], rv[v]);
                }
                StoreTraits<float>::store(x + o, xv);
                StoreTraits<float>::store(r + o, rv);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double rd = (double)rv[v];
                dots[0][t][v] += rd * (double)(rv[v] * pi);
                dots[1][t][v] += rd * rd;
            }
        }
    }
    block_column_partials<G, NT, 2>(dots, lane, ncols, ld, partials);
}

// p = r/P + beta p
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
cg_pupdate_kernel(const float* __restrict__ r, float* __restrict__ p, const double* __restrict__ beta,
                  const float* __restrict__ pinv, int32_t N, int ncols, int64_t ld) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    float be[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = (t * G + lane) * 4 + v;
            be[t][v] = c < ncols ? (float)beta[c] : 0.f;
        }
    for (int64_t rr = group; rr < N; rr += ngroups) {
        const int row = (int)rr;
        const float pi = pinv[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            const int64_t o = (int64_t)row * ld + c;
            float rv[4], pv[4];
            StoreTraits<float>::load(r + o, rv);
            StoreTraits<float>::load(p + o, pv);
#pragma unroll
            for (int v = 0; v < 4; ++v) pv[v] = fmaf(be[t][v], pv[v], rv[v] * pi);
            StoreTraits<float>::store(p + o, pv);
        }
    }
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

// pAp_j = sum of partials; alpha_j = rz_j / pAp_j for active columns.
__global__ void cg_alpha_kernel(const double* __restrict__ partials, int nblocks, int k, int64_t ldp, CgState st) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * ldp + j];
    st.alpha[j] = (st.active[j] && s != 0.0) ? st.rz[j] / s : 0.0;
}

// After an update: rz_new, rr; convergence; beta.  init != 0: first call (sets bn2, active).
__global__ void cg_beta_kernel(const double* __restrict__ partials, int nblocks, int k, int64_t ldp, CgState st,
                               double tol2, int init) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double rz = 0.0, rr = 0.0;
    for (int b = 0; b < nblocks; ++b) rz += partials[(int64_t)b * ldp + j];
    for (int b = 0; b < nblocks; ++b) rr += partials[((int64_t)nblocks + b) * ldp + j];
    st.rr[j] = rr;
    if (init) {
        st.bn2[j] = rr;
        st.rz[j] = rz;
        st.beta[j] = 0.0;
        const int act = rr > 0.0 ? 1 : 0;
        st.active[j] = act;
        if (act) atomicAdd(st.n_active, 1);
        return;
    }
    int act = st.active[j];
    if (act && rr <= tol2 * st.bn2[j]) act = 0;
    st.beta[j] = (act && st.rz[j] != 0.0) ? rz / st.rz[j] : 0.0;
    st.rz[j] = rz;
    st.active[j] = act;
    if (act) atomicAdd(st.n_active, 1);
}

__global__ void cg_setup_kernel(const int64_t* __restrict__ sample_idx, const int32_t* __restrict__ sample_labels,
                                int64_t n, int64_t N, const int32_t* __restrict__ iperm, float* __restrict__ r,
                                float* __restrict__ mask, int32_t* __restrict__ slab, int64_t ld, int k,
                                int* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t node = sample_idx[i];
    const int lab = sample_labels[i];
    if (lab < 0 || lab >= k || node < 0 || node >= N) {
        atomicOr(bad, 1);
        return;
    }
    const int64_t row = iperm ? iperm[node] : node;
    r[row * ld + lab] = 1.0f;
    mask[row] = 1.0f;
    slab[row] = lab;
}

__global__ void precond_kernel(const float* __restrict__ mask, float gamma, float* __restrict__ pinv, int32_t N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) pinv[i] = 1.0f / (mask[i] + gamma);
}

// ||b - A x||^2 per column, b rebuilt from the sample labels: partials
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
residual_kernel(const float* __restrict__ Ax, const int32_t* __restrict__ slab, int32_t N, int ncols, int64_t ld,
                double* __restrict__ partials) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    double acc[1][NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[0][t][v] = 0.0;
    for (int64_t rr = group; rr < N; rr += ngroups) {
        const int row = (int)rr;
        const int lab = slab[row];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            float a[4];
            StoreTraits<float>::load(Ax + (int64_t)row * ld + c, a);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double e = (c + v == lab ? 1.0 : 0.0) - (double)a[v];
                acc[0][t][v] += e * e;
            }
        }
    }
    block_column_partials<G, NT, 1>(acc, lane, ncols, ld, partials);
}

__global__ void column_sum_kernel(const double* __restrict__ partials, int nblocks, int k, int64_t ldp,
                                  double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * ldp + j];
    out[j] = s;
}

// column norms^2 of x (partials) -- reuse residual-free layout
template <int G, int NT>
__global__ void __launch_bounds__(kCgThreads)
colnorm_kernel(const float* __restrict__ x, int32_t N, int ncols, int64_t ld, double* __restrict__ partials) {
    const int lane = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
    double acc[1][NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[0][t][v] = 0.0;
    for (int64_t rr = group; rr < N; rr += ngroups) {
        const int row = (int)rr;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = (t * G + lane) * 4;
            if (c >= ncols) continue;
            float a[4];
            StoreTraits<float>::load(x + (int64_t)row * ld + c, a);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[0][t][v] += (double)a[v] * (double)a[v];
        }
    }
    block_column_partials<G, NT, 1>(acc, lane, ncols, ld, partials);
}

// label(i) = argmax_j x_ij / ||x_j|| (fp64 comparison, ties to the lowest j); one thread per row.
__global__ void label_argmax_kernel(const float* __restrict__ x, const double* __restrict__ norm2, int32_t N, int k,
                                    int64_t ld, const int32_t* __restrict__ perm, int32_t* __restrict__ labels,
                                    float* __restrict__ fuzzy) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    const float* xr = x + (int64_t)row * ld;
    int best = 0;
    double bv = -INFINITY;
    for (int j = 0; j < k; ++j) {
        const double nj = norm2[j];
        const double v = nj > 0.0 ? (double)xr[j] / sqrt(nj) : 0.0;
        if (v > bv) {
            bv = v;
            best = j;
        }
    }
    const int64_t orig = perm ? perm[row] : row;
    labels[orig] = best;
    if (fuzzy)
        for (int j = 0; j < k; ++j) fuzzy[orig * k + j] = xr[j];
}

// ------------------------------------------------------------- dispatch
struct Shape {
    int G, NT;
};
static Shape cg_shape(int nv) {
    static const Shape s[] = {{2, 1}, {4, 1}, {8, 1}, {16, 1}, {32, 1}, {32, 2}};
    for (const Shape& x : s)
        if (x.G * x.NT >= nv) return x;
    return {0, 0};
}

#define CG_DISPATCH(SH, ...)                                                            \
    do {                                                                                \
        if (SH.G == 2 && SH.NT == 1) { constexpr int G_ = 2, NT_ = 1; __VA_ARGS__; }          \
        else if (SH.G == 4) { constexpr int G_ = 4, NT_ = 1; __VA_ARGS__; }                   \
        else if (SH.G == 8) { constexpr int G_ = 8, NT_ = 1; __VA_ARGS__; }                   \
        else if (SH.G == 16) { constexpr int G_ = 16, NT_ = 1; __VA_ARGS__; }                 \
        else if (SH.G == 32 && SH.NT == 1) { constexpr int G_ = 32, NT_ = 1; __VA_ARGS__; }   \
        else { constexpr int G_ = 32, NT_ = 2; __VA_ARGS__; }                                 \
    } while (0)

csc_status run_interpolate(Graph* g, const int64_t* sample_idx, const int32_t* sample_labels, int64_t n, int k,
                           int g_power, double gamma, double rel_tol, int max_iter, int32_t* labels_out,
                           float* fuzzy_out, csc_cg_info* info, cudaStream_t s) {
    const int32_t N = (int32_t)g->N;
    // process columns in chunks of at most 256 (the widest compiled shape)
    if (k > 256) {
        set_error("csc_interpolate: k <= 256 in this build");
        return CSC_E_UNSUPPORTED;
    }
    const int ld = ((k + 3) / 4) * 4;
    const Shape sh = cg_shape(ld / 4);
    const int64_t rows_per_block = kCgThreads / sh.G;
    int grid = (int)((N + rows_per_block - 1) / rows_per_block);
    if (grid > g->num_sms * 8) grid = g->num_sms * 8;
    if (grid < 1) grid = 1;
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
    const size_t o_part = take((size_t)2 * grid * ld * 8);
    const size_t o_state = take((size_t)ld * 8 * 6 + (size_t)ld * 4 + 64);
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
    double* part = (double*)(b + o_part);
    double* sd = (double*)(b + o_state);
    CgState st;
    st.rz = sd;
    st.bn2 = sd + ld;
    st.alpha = sd + 2 * ld;
    st.beta = sd + 3 * ld;
    st.rr = sd + 4 * ld;
    double* norm2 = sd + 5 * ld;
    st.active = (int*)(sd + 6 * ld);
    st.n_active = st.active + ld;
    int* bad = st.n_active + 1;

    // zero x, r, mask; slab = -1
    CSC_CUDA_TRY(cudaMemsetAsync(x, 0, blk, s));
    CSC_CUDA_TRY(cudaMemsetAsync(r, 0, blk, s));
    CSC_CUDA_TRY(cudaMemsetAsync(mask, 0, (size_t)N * 4, s));
    CSC_CUDA_TRY(cudaMemsetAsync(slab, 0xff, (size_t)N * 4, s));
    CSC_CUDA_TRY(cudaMemsetAsync(st.n_active, 0, 2 * sizeof(int), s));
    // algorithmic bytes per launch of each CG kernel (fp32 N x ld blocks)
    const double blkb = (double)N * ld * 4.0;
    const double csr_b = 4.0 * g->nnz + 4.0 * (N + 1) + 4.0 * N;
    const double scal_b = 8.0 * grid * ld;
    CSC_KLAUNCH("cg_setup", 12.0 * n + 12.0 * n, s,
                cg_setup_kernel<<<ceil_div(n, 256), 256, 0, s>>>(sample_idx, sample_labels, n, (int64_t)N, g->iperm,
                                                                 r, mask, slab, ld, k, bad));
    CSC_KLAUNCH("cg_setup", 8.0 * N, s, precond_kernel<<<ceil_div(N, 256), 256, 0, s>>>(mask, (float)gamma, pinv, N));
    const int kb = ceil_div(k, 128);
    CG_DISPATCH(sh, CSC_KLAUNCH("cg_update", blkb + 4.0 * N, s,
                                cg_update_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(x, r, p, Ap, nullptr, pinv, N, ld,
                                                                                      ld, part)));
    CSC_KLAUNCH("cg_scalar", 2 * scal_b, s, cg_beta_kernel<<<kb, 128, 0, s>>>(part, grid, k, ld, st, rel_tol * rel_tol, 1));
    CG_DISPATCH(sh, CSC_KLAUNCH("cg_pupdate", 3 * blkb + 4.0 * N, s,
                                cg_pupdate_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(r, p, st.beta, pinv, N, ld, ld)));
    int* h_active = (int*)g->pinned;
    CSC_CUDA_TRY(cudaMemcpyAsync(h_active, st.n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_active[1]) {
        set_error("csc_interpolate: a sample label is outside [0, k) or a sample index outside [0, N)");
        return CSC_E_INVALID;
    }
    auto apply_A = [&](const float* in) -> csc_status {
        // t = L^(p-1) in, then Ap = mask*in + gamma * L t with <in, Ap> partials
        const float* cur = in;
        float* bufs[2] = {t1, t2};
        for (int q = 0; q < g_power - 1; ++q) {
            float* o = bufs[q & 1];
            // CSR + D^-1/2, the input block gathered once, the output block written
            CG_DISPATCH(sh, CSC_KLAUNCH("cg_lap", csr_b + 2 * blkb, s,
                                        lap_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(g->row_ptr, g->col_idx, g->dinv,
                                                                                        cur, o, N, ld, ld)));
            cur = o;
        }
        // CSR + D^-1/2 + mask, t gathered once, p read, Ap written
        CG_DISPATCH(sh, CSC_KLAUNCH("cg_lap_ax", csr_b + 4.0 * N + 3 * blkb + scal_b, s,
                                    lap_ax_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(g->row_ptr, g->col_idx, g->dinv,
                                                                                       cur, in, mask, (float)gamma, Ap,
                                                                                       N, ld, ld, part)));
        return CSC_OK;
    };
    int it = 0;
    const int check_every = 8;
    bool converged = h_active[0] == 0;
    while (!converged && it < max_iter) {
        const int batch = std::min(check_every, max_iter - it);
        for (int q = 0; q < batch; ++q) {
            CSC_TRY(apply_A(p));
            CSC_KLAUNCH("cg_scalar", scal_b, s, cg_alpha_kernel<<<kb, 128, 0, s>>>(part, grid, k, ld, st));
            // x, r, p, Ap read; x, r written
            CG_DISPATCH(sh, CSC_KLAUNCH("cg_update", 6 * blkb + 4.0 * N + 2 * scal_b, s,
                                        cg_update_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(x, r, p, Ap, st.alpha, pinv,
                                                                                              N, ld, ld, part)));
            CSC_CUDA_TRY(cudaMemsetAsync(st.n_active, 0, sizeof(int), s));
            CSC_KLAUNCH("cg_scalar", 2 * scal_b, s,
                        cg_beta_kernel<<<kb, 128, 0, s>>>(part, grid, k, ld, st, rel_tol * rel_tol, 0));
            CG_DISPATCH(sh, CSC_KLAUNCH("cg_pupdate", 3 * blkb + 4.0 * N, s,
                                        cg_pupdate_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(r, p, st.beta, pinv, N, ld,
                                                                                               ld)));
        }
        it += batch;
        CSC_CUDA_TRY(cudaMemcpyAsync(h_active, st.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
        converged = h_active[0] == 0;
    }
    // true residual ||b - A x|| / ||b|| per column
    CSC_TRY(apply_A(x));
    CG_DISPATCH(sh, CSC_KLAUNCH("cg_residual", blkb + 4.0 * N, s,
                                residual_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(Ap, slab, N, ld, ld, part)));
    CSC_KLAUNCH("cg_scalar", scal_b, s, column_sum_kernel<<<kb, 128, 0, s>>>(part, grid, k, ld, st.rr));
    // labels
    CG_DISPATCH(sh, CSC_KLAUNCH("label_norms", blkb, s,
                                colnorm_kernel<G_, NT_><<<grid, kCgThreads, 0, s>>>(x, N, ld, ld, part)));
    CSC_KLAUNCH("cg_scalar", scal_b, s, column_sum_kernel<<<kb, 128, 0, s>>>(part, grid, k, ld, norm2));
    CSC_KLAUNCH("label_argmax", blkb + 4.0 * N + (fuzzy_out ? (double)N * k * 4 : 0.0), s,
                label_argmax_kernel<<<ceil_div(N, 256), 256, 0, s>>>(x, norm2, N, k, ld, g->perm, labels_out,
                                                                     fuzzy_out));
    std::vector<double> rr(k), bn(k);
    CSC_CUDA_TRY(cudaMemcpyAsync(rr.data(), st.rr, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaMemcpyAsync(bn.data(), st.bn2, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    CSC_CUDA_TRY(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int j = 0; j < k; ++j)
        if (bn[j] > 0) worst = std::max(worst, sqrt(rr[j] / bn[j]));
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
