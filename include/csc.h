/*
 * csc.h -- C ABI of the GB300 (sm_103a) Compressive Spectral Clustering library.
 *
 * Compressive Spectral Clustering (Tremblay, Puy, Gribonval, Vandergheynst,
 * ICML 2016) replaces the partial eigendecomposition of spectral clustering by
 * polynomial filtering of a few random signals with the normalized Laplacian
 * L = I - D^-1/2 W D^-1/2 (Sec. 2.1), clusters a random subset of the nodes
 * and interpolates the labels back (Alg. 2).  This header declares every
 * entry point of the library.
 *
 * Conventions (all entry points):
 *  - Every function returns csc_status; CSC_OK (0) on success.  Nothing
 *    throws or aborts across this boundary.  On failure csc_last_error()
 *    returns a thread-local message describing the last error of the
 *    calling thread.
 *  - The caller owns every buffer it passes in.  The library owns only the
 *    opaque csc_graph (it copies the graph in and keeps its own device
 *    scratch space in it) and frees everything in csc_graph_destroy.
 *  - "device" pointers are CUDA device (or managed) memory on the current
 *    device; "host" pointers are ordinary host memory.  Large arrays are
 *    device pointers, scalars and short arrays are host pointers; each
 *    argument says which.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are stream-ordered and asynchronous unless they return
 *    a host value, in which case they synchronize `stream` before returning.
 *  - Node indices at this boundary are always in the caller's original node
 *    order; any internal reordering (CSC_RCM) is invisible.
 *  - A csc_graph is used by one host thread at a time; calls on one handle
 *    that overlap on the GPU (different streams without ordering) race on
 *    the handle's scratch space.
 *  - Matrices are dense, row-major, with an explicit leading dimension
 *    (row stride in elements) where stated.
 */
#ifndef CSC_H
#define CSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CSC_API __attribute__((visibility("default")))
#else
#define CSC_API
#endif

/* ------------------------------------------------------------------ status */
typedef int32_t csc_status;
#define CSC_OK                 0
#define CSC_E_INVALID          1  /* invalid argument; no side effects            */
#define CSC_E_CSR              2  /* malformed CSR input                          */
#define CSC_E_OOM              3  /* device or host allocation failed             */
#define CSC_E_CUDA             4  /* a CUDA runtime call failed (handle poisoned) */
#define CSC_E_NOT_CONVERGED    5  /* iterative solver hit max_iter; outputs valid */
#define CSC_E_DEVICE_TIMEOUT   6  /* reserved: no entry point waits on the device  */
#define CSC_E_NUMERIC          7  /* non-finite values detected (CSC_CHECK_FINITE) */
#define CSC_E_UNSUPPORTED      8  /* valid but outside what the library supports  */

/* storage type of the signal blocks */
typedef int32_t csc_dtype;
#define CSC_F32   0
#define CSC_BF16  1
#define CSC_F64   2

/* csc_graph_create flags */
#define CSC_RCM            1u  /* reorder nodes by reverse Cuthill-McKee internally
                                  (then by decreasing degree within blocks of 128) */
#define CSC_CHECK_SYM      2u  /* verify W is symmetric (O(nnz log) host check)        */
#define CSC_DEVICE_INPUT   4u  /* row_ptr / col_idx are device pointers                */
#define CSC_DEGREE_ORDER   8u  /* reorder nodes by decreasing degree internally (ties
                                  in the CSC_RCM order when given, else by index)    */

/* csc_filter_random_signals flags */
#define CSC_NORMALIZE_ROWS 1u  /* Alg. 2 step 4: divide every row by its l2 norm      */
#define CSC_NO_JACKSON     2u  /* truncated Chebyshev (no Jackson damping)            */
#define CSC_CLENSHAW       4u  /* evaluate the same polynomial by Clenshaw's backward
                                  recurrence, s R stored and re-read per order       */
#define CSC_HIGHPASS       8u  /* csc_cluster: interpolate with g = 1 - h~ (Sec. 4.4)  */
#define CSC_VARDENSITY    16u  /* csc_cluster: variable-density draws (scores ||Y_i||^2)
                                  and the weighted decoder (Sec. 3.2.3, Theorem 3.4)  */
#define CSC_CHECK_FINITE  32u  /* csc_filter_random_signals: scan R_in (when given)
                                  before and Y after the filter; csc_cluster: scan the
                                  filtered features; CSC_E_NUMERIC on NaN or infinity
                                  (one synchronizing pass per scan)                   */

typedef struct csc_graph_s* csc_graph;

/* Result of csc_estimate_lambda_k. */
typedef struct {
    double  lambda;       /* estimate of lambda_k                                     */
    double  count;        /* eigencount at lambda (sum_j c_j(lambda) mu_j)            */
    int32_t iters;        /* dichotomy halvings performed                             */
    int32_t hit;          /* 1 if round(count) == k was reached, 0 if the bracket collapsed */
    int32_t n_probes;     /* probe vectors used                                       */
    int32_t m;            /* polynomial degree used                                   */
    int32_t bracket_used; /* 1 if a caller bracket was given and contained the answer */
    int32_t moment_passes;/* sparse block products spent on eigencounts                */
} csc_lambda_info;

/* Result of csc_interpolate. */
typedef struct {
    int32_t iters;            /* CG iterations performed (max over clusters)          */
    int32_t converged;        /* 1 if every cluster reached rel_tol                   */
    double  max_rel_residual; /* max_j ||b_j - A x_j|| / ||b_j|| at exit (FP64)       */
} csc_cg_info;

/* Parameters of the whole pipeline (csc_cluster).  Zero means "default". */
typedef struct {
    int32_t  k;            /* number of clusters (required, >= 1)                     */
    int32_t  m;            /* Jackson-Chebyshev degree; default 50 (Alg. 2)           */
    int32_t  d;            /* random signals; default ceil(4 ln N)                    */
    int32_t  d_pad;        /* padded columns (multiple of 8); default round up of d   */
    int64_t  n;            /* sampled nodes; default ceil(2 k ln k) (at least k)      */
    int32_t  n_probes;     /* eigencount probes; default ceil(2 ln N)                 */
    int32_t  g_power;      /* interpolation g(L) = L^g_power; default 4               */
    double   gamma;        /* Eq. 5 regularisation; default 1e-3                      */
    double   cg_tol;       /* relative residual target; default 1e-6                  */
    int32_t  cg_max_iter;  /* default 2000                                            */
    int32_t  replicates;   /* k-means replicates; default 20                          */
    int32_t  km_max_iter;  /* k-means iterations; default 100                         */
    csc_dtype storage;     /* signal-block storage; default CSC_F32                   */
    uint64_t seed;
    double   lambda_k;     /* > 0: skip step 1 and use this cut-off                   */
    const double* bracket; /* NULL or host {lo, hi}: learned bracket for step 1       */
    uint32_t flags;        /* CSC_CLENSHAW: filter by Clenshaw's recurrence; CSC_HIGHPASS:
                              interpolate with g = 1 - h~ at lambda_k (degree m_interp);
                              CSC_VARDENSITY: csc_coherence_scores, csc_sample_weighted
                              and the weighted decoder in place of uniform sampling     */
    int32_t  m_count;      /* degree of the eigencount filter of step 1 (Sec. 4.3 does
                              not fix it); default m.  The damped step leaks a little of
                              every eigenvalue above the cut-off into the count, which on
                              graphs of ~1e6 nodes can alone reach k: a higher degree
                              (e.g. 4 m) sharpens it for a few extra moment passes      */
    int32_t  m_interp;     /* CSC_HIGHPASS: degree of h~ inside g = 1 - h~; default m.
                              Each CG iteration costs m_interp sparse products          */
} csc_params;

/* Per-stage results and timings of csc_cluster. */
typedef struct {
    csc_lambda_info lambda;
    csc_cg_info     cg;
    double          inertia;      /* best reduced k-means inertia (FP64)             */
    float           ms_lambda, ms_filter, ms_sample, ms_kmeans, ms_interp, ms_total;
} csc_cluster_info;

/* Results and stage timings of csc_cluster_batched. */
typedef struct {
    csc_cg_info cg;               /* CG over all graphs' systems (max iterations / residual) */
    int32_t     lambda_hits;      /* graphs whose dichotomy reached round(count) == k        */
    float       ms_lambda, ms_filter, ms_sample, ms_kmeans, ms_interp, ms_total;
} csc_batch_info;

/* ---------------------------------------------------------------- graphs */

/* csc_graph_create -- copy an undirected graph in CSR form into a new handle.
 * Defines W of Sec. 2.1; degrees D_ii = sum_{j != i} W_ij are computed on the
 * device (self loops are dropped, so they count neither in W nor in D).
 *   N        nodes (>= 1; N < 2^31).
 *   nnz      stored entries (row_ptr[N]); < 2^31.
 *   row_ptr  int64[N+1], nondecreasing, row_ptr[0] = 0, row_ptr[N] = nnz.
 *   col_idx  int32[nnz], each row strictly increasing (sorted, no duplicates),
 *            values in [0, N).  The matrix must be symmetric (checked only with
 *            CSC_CHECK_SYM).
 *   weights  must be NULL: the graphs of this library are unweighted
 *            (W_ij in {0,1}); non-NULL returns CSC_E_UNSUPPORTED.
 *   flags    CSC_RCM | CSC_DEGREE_ORDER | CSC_CHECK_SYM | CSC_DEVICE_INPUT.  Without
 *            CSC_DEVICE_INPUT the arrays are host memory; with it they are
 *            device memory, copied to the host first.  Either way the CSR is
 *            validated on the host and every flag applies.
 *   out      receives the handle.
 * Errors: CSC_E_INVALID (null pointers, N < 1, nnz < 0), CSC_E_CSR (any
 * violation above), CSC_E_OOM, CSC_E_CUDA.  Synchronizes `stream`. */
CSC_API csc_status csc_graph_create(int64_t N, int64_t nnz, const int64_t* row_ptr,
                            const int32_t* col_idx, const float* weights,
                            uint32_t flags, void* stream, csc_graph* out);

/* csc_graph_create_batched -- G independent graphs packed block-diagonally
 * into one handle (graph g occupies node ids offsets[g] .. offsets[g+1]-1 of
 * the packed graph, each with its own CSR whose column ids are local to g).
 * Host arrays only.  Same validation as csc_graph_create per graph. */
CSC_API csc_status csc_graph_create_batched(int32_t G, const int64_t* N, const int64_t* const* row_ptr,
                                    const int32_t* const* col_idx, uint32_t flags,
                                    void* stream, csc_graph* out);

/* csc_graph_destroy -- free the handle and all its device memory.  NULL is a no-op. */
CSC_API csc_status csc_graph_destroy(csc_graph g);

/* csc_graph_info -- sizes: N, nnz (after self-loop removal), number of packed
 * graphs (1 unless batched).  Any output pointer may be NULL.  Host outputs. */
CSC_API csc_status csc_graph_info(csc_graph g, int64_t* N, int64_t* nnz, int32_t* n_graphs);

/* csc_graph_tuned_shape -- the launch shapes the autotuner chose on this handle
 * (not a step of the paper's method).  Shapes are tuned on first use per kernel
 * kind (1 = Chebyshev step, 2 = moment step, 3 = CG products, 4 = Clenshaw step),
 * storage width and column count, by timing every compiled shape on the handle's
 * graph; a CG solve that compacts its columns (csc_interpolate) also tunes each
 * narrower width it reaches, with lane groups of that width and one column tile,
 * and reports it as a kind-3 entry of that column count.  Entry i
 * (0-based) is written to kind, dtype_bytes (4 fp32, 2 bf16, 8 fp64), columns and
 * shape[6] = {lanes per row G, vectors per lane NT, threads per CTA, row ranges P,
 * column tiles, variant}: variant bit 0 = the index source (0: each CTA stages its
 * rows' column indices in shared memory, 1: the indices are read from global memory),
 * bit 1 = the lean form of the Clenshaw orders and CG products (NT = 1, 256 threads:
 * at most 4 neighbour rows in flight per lane, 5 CTAs per SM instead of 4).  Host
 * outputs (any may be NULL).  CSC_E_INVALID when i is out of range. */
CSC_API csc_status csc_graph_tuned_shape(csc_graph g, int32_t i, int32_t* kind, int32_t* dtype_bytes,
                                         int32_t* columns, int32_t* shape);

/* csc_graph_pin_shape -- fix the launch shape of one kernel kind on this handle
 * instead of tuning it (reproducible timings; tests of every compiled shape).
 * kind, dtype_bytes, columns and shape[6] as in csc_graph_tuned_shape (host).
 * (G, NT) must be a compiled pair, threads 256 or 512, tiles = ceil(vectors per
 * row / (G NT)), variant 0 .. 3 (the lean bit only for kinds 3 and 4 with NT = 1 and
 * 256 threads).
 * Errors: CSC_E_INVALID (no side effects); an uncompiled (G, NT) surfaces as
 * CSC_E_UNSUPPORTED at the next launch. */
CSC_API csc_status csc_graph_pin_shape(csc_graph g, int32_t kind, int32_t dtype_bytes, int32_t columns,
                                       const int32_t* shape);

/* csc_graph_degrees -- D_ii of Sec. 2.1 (integer edge counts, bit-exact) in
 * original node order.  deg_out: host int32[N].  Synchronizes `stream`. */
CSC_API csc_status csc_graph_degrees(csc_graph g, int32_t* deg_out, void* stream);

/* ------------------------------------------------------- the Chebyshev path */

/* csc_chebyshev_coefficients -- c_j = g_j gamma_j (j = 0..m) of the
 * Jackson-Chebyshev approximation of the ideal low-pass h_{lambda_c} of Eq. 1
 * on the variable t = lambda - 1 (Sec. 4.3, Jackson damping after Di Napoli,
 * Polizzi and Saad): gamma_0 = 1 - theta_c/pi, gamma_j = -2 sin(j theta_c)/(j pi),
 * theta_c = arccos(lambda_c - 1), g_j the Jackson factors with alpha = pi/(m+2).
 * With CSC_NO_JACKSON in flags, g_j = 1.  c_out: host double[m+1].
 * Errors: CSC_E_INVALID if m < 0, lambda_c outside [0, 2] or c_out NULL. */
CSC_API csc_status csc_chebyshev_coefficients(double lambda_c, int32_t m, uint32_t flags, double* c_out);

/* csc_filter_random_signals -- Alg. 2 steps 2-4: Y = h~_{lambda_c}(L) R with
 * h~ the degree-m Jackson-Chebyshev polynomial, computed by the three-term
 * recurrence X_0 = R, X_1 = (L - I) R, X_{j+1} = 2 (L - I) X_j - X_{j-1}
 * (Sec. 2.1 "Fast graph filtering"); optionally rows normalised (step 4).
 *   lambda_c  cut-off in [0, 2].
 *   m         degree >= 0 (m = 0 gives Y = c_0 R).
 *   d, d_pad  signal count and row stride (d_pad >= d, d_pad % 8 == 0).
 *   seed      R is drawn as N(0, 1/d) by Philox4x32-10 (counter = (node id,
 *             column/4), key = (seed, stream "signals")) with Box-Muller, unless R_in
 *             is given.
 *   storage   CSC_F32 / CSC_BF16 (X_j stored in bf16, arithmetic and Y in fp32)
 *             / CSC_F64 (X_j, arithmetic and Y in fp64).
 *   R_in      NULL, or device float[N * d_pad] row-major in original node order
 *             (padding columns are ignored and treated as zero).
 *   Y_out     device, N * d_pad row-major in original node order: float for
 *             CSC_F32/CSC_BF16, double for CSC_F64.  Padding columns are zero.
 *   flags     CSC_NORMALIZE_ROWS, CSC_NO_JACKSON, CSC_CLENSHAW, CSC_CHECK_FINITE.  Without
 *             CSC_CLENSHAW the orders run the three-term forward recurrence
 *             X_{j+1} = 2 (L - I) X_j - X_{j-1} accumulating Y (Sec. 2.1); with it
 *             Clenshaw's recurrence b_j = c_j R + 2 (L - I) b_{j+1} - b_{j+2},
 *             Y = c_0 R + (L - I) b_1 - b_2 (Clenshaw 1955), which needs no Y
 *             traffic until the last order; both give Y up to rounding.
 * Errors: CSC_E_INVALID (no side effects), CSC_E_OOM, CSC_E_CUDA; with
 * CSC_CHECK_FINITE, CSC_E_NUMERIC when R_in (nothing is filtered then) or Y holds a
 * NaN or infinity.  Asynchronous, except that each CSC_CHECK_FINITE scan synchronizes. */
CSC_API csc_status csc_filter_random_signals(csc_graph g, double lambda_c, int32_t m, int32_t d,
                                     int32_t d_pad, uint64_t seed, csc_dtype storage,
                                     const float* R_in, void* Y_out, uint32_t flags,
                                     void* stream);

/* csc_kpm_moments -- eigencount moments of Sec. 4.3:
 * mu_j = (1/n_probes) sum_l r_l^T T_j(L - I) r_l, j = 0..n_moments-1, with
 * r_l ~ N(0, 1) drawn by Philox (key = (seed, stream "probes")), computed with
 * ceil((n_moments-1)/2) sparse block products using T_2j = 2 T_j^2 - T_0 and
 * T_2j+1 = 2 T_j+1 T_j - T_1, reductions in fp64.
 *   n_probes 0 -> ceil(2 ln N) (Sec. 4.3).
 *   storage  CSC_F32 or CSC_BF16 for the probe block.
 *   mu_out   host double[n_moments].  Synchronizes `stream`.
 * Errors: CSC_E_INVALID (n_moments < 1, n_probes < 0). */
CSC_API csc_status csc_kpm_moments(csc_graph g, int32_t n_moments, int32_t n_probes, uint64_t seed,
                           csc_dtype storage, double* mu_out, void* stream);

/* csc_eigencount -- count(lambda) = sum_j c_j(lambda) mu_j for given moments
 * (host, O(m)).  mu: host double[m+1].  count_out: host double. */
CSC_API csc_status csc_eigencount(const double* mu, int32_t m, double lambda, uint32_t flags,
                          double* count_out);

/* csc_estimate_lambda_k -- Alg. 2 step 1 (Sec. 4.3): moments computed once on
 * the device, then a dichotomy on [0, 2] evaluated on the host from them: at
 * mid = (lo+hi)/2 stop if round(count(mid)) == k (half away from zero), else
 * hi = mid if count(mid) > k, lo = mid otherwise; after 60 halvings or when
 * hi - lo < 1e-12 the upper end is returned with hit = 0.
 *   k         clusters (>= 1).   m  degree (>= 1).
 *   n_probes  0 -> ceil(2 ln N).
 *   bracket   NULL, or host double[2] {lo, hi} with 0 <= lo < hi <= 2 (e.g. from
 *             the learned predictor): the dichotomy starts from it when
 *             round(count(lo)) <= k <= round(count(hi)), else from [0, 2].
 *   out       host.  Synchronizes `stream`. */
CSC_API csc_status csc_estimate_lambda_k(csc_graph g, int32_t k, int32_t m, int32_t n_probes,
                                 uint64_t seed, const double* bracket, csc_lambda_info* out,
                                 void* stream);

/* csc_estimate_lambda_k_refilter -- the Sec. 4.3 estimator read literally: every
 * dichotomy threshold lambda filters the n_probes N(0, 1) probes (the probes of
 * csc_kpm_moments) with the degree-m Jackson-Chebyshev step at lambda (m sparse
 * block products) and takes count = (1/n_probes) sum_l r_l^T h~_lambda(L) r_l,
 * reduced on the device in fp64.  The dichotomy rule is that of
 * csc_estimate_lambda_k.  In exact arithmetic the counts equal the
 * moments-once counts; this entry point exists to measure what the paper's
 * form costs.  bracket: NULL or host {lo, hi}, checked by the counts at both
 * ends (two passes) and used when round(count(lo)) <= k <= round(count(hi)).
 * out->moment_passes counts the sparse products.  Synchronizes `stream`. */
CSC_API csc_status csc_estimate_lambda_k_refilter(csc_graph g, int32_t k, int32_t m, int32_t n_probes,
                                          uint64_t seed, const double* bracket, csc_lambda_info* out,
                                          void* stream);

/* ------------------------------------------- learned lambda_k bracket
 * The paper is silent on learning lambda_k; these calls add a predictor of a
 * bracket for the Sec. 4.3 dichotomy, and the eigencount still decides:
 * a bracket is used only when the eigencount confirms it, otherwise the
 * plain dichotomy runs.  The predictor is a 72 -> 256 -> 256 -> 2 ReLU
 * perceptron (smooth-L1 loss, Adam) trained on the device by the calls below.
 * Parameters are one device float[CSC_MLP_PARAMS] in the order W1 [72 x 256]
 * (row = input, row-major), b1 [256], W2 [256 x 256], b2, W3 [256 x 2], b3 [2].
 * All device buffers are owned by the caller. */
#define CSC_MLP_IN 72
#define CSC_MLP_HIDDEN 256
#define CSC_MLP_OUT 2
#define CSC_MLP_PARAMS 84994
#define CSC_BRACKET_PROBES 8
#define CSC_BRACKET_MOMENTS 64
/* flags of csc_estimate_lambda_k_learned */
#define CSC_EIGENCOUNT_REFILTER 1u /* check the bracket with the paper-literal estimator */

/* csc_bracket_features -- the 72 predictor inputs of one graph (host float[72]):
 * [0, 64) eigencount moments mu_j / N of CSC_BRACKET_PROBES N(0, 1) probes
 * (the Sec. 4.3 estimator, j = 0..63, one device moment pass); 64: ln N;
 * 65: k; 66..71: ln(1 + q) for the degree quantiles q at 0, 0.1, 0.25, 0.5,
 * 0.75, 1 (sorted degree at index floor(p (N - 1))).  mu_out: NULL or host
 * double[64], the raw moments.  Synchronizes `stream`. */
CSC_API csc_status csc_bracket_features(csc_graph g, int32_t k, uint64_t seed, float* feat_out,
                                        double* mu_out, void* stream);

/* csc_bracket_target -- host: the cut-offs where count(lambda) = sum_j c_j(lambda)
 * mu_j (Sec. 4.3, degree m, mu: host double[m+1]) crosses k - 1/2 and k + 1/2,
 * each by 60 bisection halvings on [0, 2]; every lambda between them rounds to
 * count k.  lo_hi_out: host double[2]. */
CSC_API csc_status csc_bracket_target(const double* mu, int32_t m, int32_t k, double* lo_hi_out);

/* csc_mlp_init -- He-uniform weights U(-a, a), a = sqrt(6 / fan_in), from Philox
 * (counter = parameter index, key = seed), zero biases.  params: device. */
CSC_API csc_status csc_mlp_init(float* params, uint64_t seed, void* stream);

/* csc_mlp_forward -- Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3 for B rows.
 * X: device float[B x 72]; Y: device float[B x 2]; 1 <= B <= 65536. */
CSC_API csc_status csc_mlp_forward(const float* params, const float* X, int32_t B, float* Y, void* stream);

/* csc_mlp_loss_grad -- smooth-L1 (beta = 1) loss averaged over the B x 2 outputs
 * against targets T (device float[B x 2]) and its gradient (device
 * float[CSC_MLP_PARAMS], overwritten).  loss: NULL or host double (then the
 * call synchronizes `stream`). */
CSC_API csc_status csc_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t B,
                                     float* grad, double* loss, void* stream);

/* csc_mlp_adam_step -- one Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected at step t >= 1).  m, v: device float[CSC_MLP_PARAMS] moment
 * estimates (zero before the first step). */
CSC_API csc_status csc_mlp_adam_step(float* params, const float* grad, float* m, float* v, int32_t t,
                                     float lr, void* stream);

/* csc_mlp_train -- `epochs` passes of minibatch Adam over n samples (X: device
 * float[n x 72], T: device float[n x 2]), batches of `batch` rows in an order
 * shuffled per epoch by SplitMix64(seed).  Adam state starts at zero.
 * epoch_loss: NULL or host double[epochs], the mean batch loss of each
 * epoch.  Synchronizes `stream`. */
CSC_API csc_status csc_mlp_train(float* params, const float* X, const float* T, int32_t n, int32_t epochs,
                                 int32_t batch, float lr, uint64_t seed, double* epoch_loss, void* stream);

/* csc_bracket_fit -- fits the bracket predictor that csc_estimate_lambda_k_learned
 * uses (the paper has no learned component; this is the training side of that add-on):
 *   1. targets (centre, ln half-width) = ((lo + hi) / 2, ln max((hi - lo) / 2, 1e-12))
 *      of each sample's target bracket (from csc_bracket_target);
 *   2. the last round(val_frac * n) samples (ties to even; none when n < 10) are held
 *      back, the others fitted: norm_out = their feature mean [72] and standard
 *      deviation [72] (population), target mean [2] and standard deviation [2] (a zero
 *      spread taken as 1), as fp32;
 *   3. the standardised fitted features (as at inference: (x - mean) / std in fp32, 0
 *      for a zero-spread feature) and targets train a network from csc_mlp_init(seed)
 *      by csc_mlp_train(epochs, batch, lr, seed);
 *   4. widen_out = the half-width factor calibrated on the held-back samples (on the
 *      fitted ones when none is held back): widen_rule 0 -> the factor 0.25 * 2^(j/4),
 *      j = 0..56, whose started halving (see csc_estimate_lambda_k_learned) takes the
 *      fewest eigencount evaluations on average when the accepted cut-offs are
 *      exactly the target bracket (first one on ties); widen_rule 1 -> the smallest
 *      factor with which a `coverage` share of the predicted intervals meet their
 *      target brackets (linear interpolation between order statistics), at least 1.
 * feats: host float[n x 72] (csc_bracket_features); brackets: host double[n x 2] with
 * lo <= hi.  params: device float[CSC_MLP_PARAMS] (overwritten).  norm_out: host
 * float[148].  n_fit_out, epoch_loss (host double[epochs]): NULL or outputs.
 * Errors: CSC_E_INVALID (no side effects), CSC_E_OOM, CSC_E_CUDA.  Synchronizes
 * `stream`. */
CSC_API csc_status csc_bracket_fit(const float* feats, const double* brackets, int32_t n, double val_frac,
                                   int32_t epochs, int32_t batch, float lr, uint64_t seed, int32_t widen_rule,
                                   double coverage, float* params, float* norm_out, double* widen_out,
                                   int32_t* n_fit_out, double* epoch_loss, void* stream);

/* csc_bracket_predict -- the predictor on n feature rows (host float[n x 72]):
 * targets_out (host double[n x 2] or NULL) = (centre, ln half-width) as the network
 * gives them after the standardisation of norm; brackets_out (host double[n x 2] or
 * NULL) = centre -+ widen * exp(min(ln half-width, 10)) clipped to [0, 2], the
 * bracket csc_estimate_lambda_k_learned starts from.  params: device.  norm: host
 * float[148] from csc_bracket_fit.  Synchronizes `stream`. */
CSC_API csc_status csc_bracket_predict(const float* params, const float* norm, double widen, const float* feats,
                                       int32_t n, double* targets_out, double* brackets_out, void* stream);

/* csc_estimate_lambda_k_learned -- Alg. 2 step 1 with a predicted bracket:
 *   1. csc_bracket_features (one moment pass over 8 probes, 64 moments);
 *   2. z = (features - mean) / std, y = network(z), (centre, ln half-width) =
 *      y * target_std + target_mean, bracket = centre -+ widen * exp(ln half-width)
 *      clipped to [0, 2];
 *   3. the Sec. 4.3 halving started from the prediction: the count at the
 *      centre c decides the side, the predicted end on that side (c -+ hw) is
 *      evaluated next, and the halving continues inside [c - hw, c + hw] when
 *      that end lies across k, else on the rest of [0, 2]; it stops as soon
 *      as round(count) == k, like csc_estimate_lambda_k;
 *   4. moments-once (flags = 0): step 3 runs on the 8-probe moments (m <= 63);
 *      an answer found inside the prediction is returned (bracket_used = 1,
 *      n_probes = 8); otherwise the plain path runs: n_probes probes
 *      (0 -> ceil(2 ln N)) and the dichotomy on [0, 2] (bracket_used = 0).
 *      With flags & CSC_EIGENCOUNT_REFILTER, step 3 evaluates every count
 *      with the paper-literal estimator of csc_estimate_lambda_k_refilter
 *      (n_probes probes); bracket_used tells whether the answer lay inside
 *      the prediction.
 * params: device float[CSC_MLP_PARAMS].  norm: host float[148] = feature mean
 * [72], feature std [72], target mean [2], target std [2].  widen > 0.
 * bracket_out: NULL or host double[2], the predicted bracket.  moment_passes
 * counts the sparse products of both moment passes.  Synchronizes `stream`. */
CSC_API csc_status csc_estimate_lambda_k_learned(csc_graph g, int32_t k, int32_t m, int32_t n_probes,
                                                 uint64_t seed, const float* params, const float* norm,
                                                 double widen, uint32_t flags, csc_lambda_info* out,
                                                 double* bracket_out, void* stream);

/* ------------------------------------------------- sampling and k-means */

/* csc_sample -- Sec. 3.2 / Eq. 4: n of N nodes uniformly without replacement.
 * Node i gets the 64-bit key SplitMix64_seed(i) (output i of SplitMix64 seeded
 * with `seed`); the n nodes with the smallest (key, i) are returned sorted
 * ascending.  Bit-exact and deterministic.
 *   idx_out  device int64[n].  0 <= n <= N.  Asynchronous.
 * Errors: CSC_E_INVALID. */
CSC_API csc_status csc_sample(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out, void* stream);

/* csc_sample_noalloc -- the same sample as csc_sample (bit for bit), for callers
 * that cannot allocate device memory: applications whose device memory is all
 * owned by their own allocator (a framework's caching pool, an arena sized at
 * start-up), applications with a fixed device-memory budget, and latency-critical
 * code where cudaMalloc / cudaFree may implicitly synchronize the device.  The
 * paper has no counterpart.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch is one
 * fixed array of 327,936 bytes inside the library, present on every device that
 * loads the library until the process exits.
 *   N         1 <= N <= 2^26 (67,108,864); larger N returns CSC_E_UNSUPPORTED
 *             with a message (use csc_sample).
 *   idx_out   device int64[n], sorted ascending.  Asynchronous on `stream`.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  Every call on a device shares the one scratch array, which
 * keeps the previous call's contents (each call clears what must start at zero):
 * calls that overlap on the GPU (different streams, or different host threads
 * using the same device) race and give wrong results. */
CSC_API csc_status csc_sample_noalloc(int64_t N, int64_t n, uint64_t seed, int64_t* idx_out, void* stream);

/* csc_coherence_scores -- s_i = ||Y_i||^2 over the first d columns (FP64 sum) of
 * an UNnormalised filtered block Y = h~(L) R.  With R's N(0, 1/d) entries its
 * expectation is ||h~(L) delta_i||^2, the estimate of the squared local cumulative
 * coherence v_k(i)^2 given in the remark closing Sec. 4.2.  With normalize != 0
 * the rows are then divided by their norms in place (Alg. 2 step 4; zero rows are
 * left as they are).
 *   Y          device, N x ld row-major (ld >= d): float when y_type is CSC_F32 or
 *              CSC_BF16 (the filter's output for those storages), double for CSC_F64.
 *   score_out  device double[N].  Asynchronous.
 * Errors: CSC_E_INVALID. */
CSC_API csc_status csc_coherence_scores(void* Y, csc_dtype y_type, int64_t N, int32_t d, int32_t ld,
                                        int32_t normalize, double* score_out, void* stream);

/* csc_sample_weighted -- variable-density sampling (Sec. 3.2.3 after Theorem 3.4):
 * n draws i.i.d. WITH replacement, node i with probability q_i / Q, where
 * q_i = floor(2^32 * (s_i / max_j s_j)) (one correctly rounded FP64 division) and
 * Q = sum_i q_i.  Draw t takes the word r_t = SplitMix64_seed(t), the point
 * u_t = floor(r_t * Q / 2^64) and the node with the smallest inclusive prefix
 * sum of q above u_t (exact integer inverse CDF: bit-exact and deterministic).
 *   score    device double[N]: finite, >= 0, at least one > 0 (for example
 *            csc_coherence_scores, the distribution p_i ~ v_k(i)^2 of the cited
 *            sampling theory).
 *   idx_out  device int64[n], sorted ascending, repeated draws adjacent.
 *   w_out    NULL or device float[n]: each draw's decoder weight Q / (N q_i)
 *            (FP64, rounded to float): 1 for a flat profile.
 *   1 <= N < 2^31, 0 <= n < 2^31.  Synchronizes `stream` (the scores are checked
 *   on the device and the outcome read back).
 * Errors: CSC_E_INVALID (arguments; a negative, NaN or infinite score; every score
 * zero), CSC_E_OOM. */
CSC_API csc_status csc_sample_weighted(const double* score, int64_t N, int64_t n, uint64_t seed, int64_t* idx_out,
                                       float* w_out, void* stream);

/* csc_gather_rows -- out[i, :] = X[idx[i], :] for i < n (Alg. 2 step 5).
 *   X    device float[N * ld];  idx  device int64[n] (values in [0, N));
 *   out  device float[n * ld_out], columns 0..d-1 written.  Asynchronous. */
CSC_API csc_status csc_gather_rows(const float* X, int64_t N, int32_t ld, const int64_t* idx, int64_t n,
                           int32_t d, float* out, int32_t ld_out, void* stream);

/* csc_kmeans_reduced -- Alg. 2 step 6: k-means on n points of dimension d.
 * k-means++ seeding from Philox draws (key = (seed, stream "k-means"),
 * counter = (replicate, draw)), Lloyd iterations (ties to the lowest centre,
 * an empty cluster takes the point farthest from its centre), at most
 * max_iter updates, best of `replicates` runs by inertia (ties to the first).
 *   X           device float[n * ld], ld >= d.
 *   labels_out  device int32[n].   inertia_out  host double (may be NULL).
 * Errors: CSC_E_INVALID (k < 1, n < k, d < 1, replicates < 1), CSC_E_UNSUPPORTED
 * (k > 1024 or d > 256).  Synchronizes `stream` when inertia_out != NULL. */
CSC_API csc_status csc_kmeans_reduced(const float* X, int64_t n, int32_t d, int32_t ld, int32_t k,
                              int32_t replicates, int32_t max_iter, uint64_t seed,
                              int32_t* labels_out, double* inertia_out, void* stream);

/* ------------------------------------------------------- interpolation */

/* csc_interpolate -- Alg. 2 step 7: for every cluster j solve Eq. 5,
 * (M^T M + gamma L^g_power) x_j = M^T c_j^r, by Jacobi-preconditioned
 * conjugate gradients (fp32 vectors; inner products compensated in fp32 within a
 * block and summed in fp64 across blocks; one CG per column, a column stopping at
 * ||r_j|| <= rel_tol ||b_j||), then label node i with argmax_j x_j(i) / ||x_j||
 * (Sec. 4.1; ties to the lowest j).  Columns that have converged leave the
 * iteration (the others are compacted into narrower dense blocks); the first solve
 * that reaches a width tunes a launch shape for it (csc_graph_tuned_shape).
 *   sample_idx     device int64[n]: sampled node ids (distinct).
 *   sample_labels  device int32[n]: their clusters in [0, k).
 *   g_power        >= 1.   gamma > 0.   rel_tol > 0.   max_iter >= 1.
 *   labels_out     device int32[N].
 *   fuzzy_out      NULL or device float[N * k]: the x_j (column j), Sec. 4.1's
 *                  fuzzy memberships.
 *   info           host (may be NULL).
 * Returns CSC_E_NOT_CONVERGED when max_iter was reached first (outputs are
 * still written).  Synchronizes `stream` (convergence checks). */
CSC_API csc_status csc_interpolate(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                           int64_t n, int32_t k, int32_t g_power, double gamma, double rel_tol,
                           int32_t max_iter, int32_t* labels_out, float* fuzzy_out,
                           csc_cg_info* info, void* stream);

/* csc_interpolate_highpass -- Eq. 5 with the paper's preferred high-pass
 * regulariser g = 1 - h~_{lambda_c} (the discussion after Eq. 5, Sec. 4.4): h~ the
 * Jackson-Chebyshev low-pass of degree m at lambda_c (the filter of Alg. 2 step 4),
 * so every CG iteration applies h~(L) to the k columns (m sparse products, Clenshaw
 * form) and A p = mask p + gamma (p - h~(L) p).  Arguments as csc_interpolate,
 * with lambda_c in [0, 2] and m >= 1 instead of g_power.  On a batched handle
 * the packed graph is one graph here (one cut-off, one set of k systems); per-graph
 * systems are csc_interpolate_batched_highpass. */
CSC_API csc_status csc_interpolate_highpass(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                            int64_t n, int32_t k, double lambda_c, int32_t m, double gamma,
                                            double rel_tol, int32_t max_iter, int32_t* labels_out,
                                            float* fuzzy_out, csc_cg_info* info, void* stream);

/* csc_interpolate_weighted -- the decoder of variable-density draws: Eq. 5 with
 * the fidelity term weighted per draw (the P^{-1/2} weighting of the sampling
 * theory cited after Theorem 3.4),
 *   x_j = argmin_x sum_t w_t (x(omega_t) - [label_t == j])^2 + gamma x^T L^g_power x,
 * the sum over draws t, so a node drawn twice counts twice.  The normal equations
 * (M^T W M + gamma L^p) x = M^T W c_j are solved by the CG of csc_interpolate
 * (preconditioner 1 / (sum of the node's weights + gamma)); the residual is
 * measured against the weighted right-hand side, kept in an extra N x k block.
 * Arguments as csc_interpolate plus
 *   sample_w  device float[n], finite and > 0 (csc_sample_weighted's w_out).
 *   n         >= 1 draws; repeats allowed (n may exceed N).
 * Weights of repeated draws are summed in an unspecified order (bit-reproducible
 * when a node's draws carry equal weights, as csc_sample_weighted's do).
 * Unit weights on distinct draws give csc_interpolate's systems.
 * Errors: as csc_interpolate; a weight not finite and positive is CSC_E_INVALID. */
CSC_API csc_status csc_interpolate_weighted(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                            const float* sample_w, int64_t n, int32_t k, int32_t g_power,
                                            double gamma, double rel_tol, int32_t max_iter, int32_t* labels_out,
                                            float* fuzzy_out, csc_cg_info* info, void* stream);

/* --------------------------------------------------------- whole pipeline */

/* csc_cluster -- Alg. 2 end to end on one graph with the parameters above.
 *   labels_out  device int32[N] in original node order.
 *   info        host (may be NULL).  Synchronizes `stream`.
 * With CSC_CHECK_FINITE in params->flags the filtered features are scanned before
 * sampling and a NaN or infinity stops the call with CSC_E_NUMERIC.
 * For a batched handle use csc_cluster_batched. */
CSC_API csc_status csc_cluster(csc_graph g, const csc_params* params, int32_t* labels_out,
                       csc_cluster_info* info, void* stream);

/* ------------------------------------------------------------ batches
 * Alg. 2 on the G graphs of a handle made by csc_graph_create_batched: graph i
 * owns the packed rows offsets[i] .. offsets[i+1]-1 (block-diagonal W), and
 * every sparse product serves all graphs at once.  Graph i's results are those
 * of the single-graph calls on graph i alone, except that the signal and probe
 * blocks are drawn for the packed rows, and graph i samples and seeds k-means
 * with seed + i.  Host arrays of per-graph values have G entries.  Node
 * indices and labels are packed (graph i's node j is offsets[i] + j); labels
 * are per-graph cluster numbers in [0, k_i). */

/* csc_kpm_moments_batched -- the moments of csc_kpm_moments for each graph (the
 * trace runs over the graph's own rows).  mu_out: host double[G x n_moments]. */
CSC_API csc_status csc_kpm_moments_batched(csc_graph g, int32_t n_moments, int32_t n_probes, uint64_t seed,
                                           csc_dtype storage, double* mu_out, void* stream);

/* csc_estimate_lambda_k_batched -- csc_estimate_lambda_k per graph from one
 * moment pass over the packed graph.  k: host int32[G] (1 <= k_i <= N_i).
 * n_probes: 0 -> ceil(2 ln max_i N_i) for every graph.  lambda_out: host
 * double[G]; info_out: NULL or host csc_lambda_info[G].  Synchronizes. */
CSC_API csc_status csc_estimate_lambda_k_batched(csc_graph g, const int32_t* k, int32_t m, int32_t n_probes,
                                                 uint64_t seed, double* lambda_out, csc_lambda_info* info_out,
                                                 void* stream);

/* csc_filter_batched -- csc_filter_random_signals with graph i's rows filtered at
 * cut-off lambda[i] (host double[G], each in [0, 2]); m >= 1.  Y_out: device
 * N x d_pad (packed rows), as for the single-graph call. */
CSC_API csc_status csc_filter_batched(csc_graph g, const double* lambda, int32_t m, int32_t d, int32_t d_pad,
                                      uint64_t seed, csc_dtype storage, const float* R_in, void* Y_out,
                                      uint32_t flags, void* stream);

/* csc_sample_batched -- csc_sample(N_i, n[i], seed + i) for every graph in one
 * launch (one CTA per graph): idx_out (device int64[sum n]) holds graph 0's
 * packed indices in increasing order, then graph 1's, ...  n: host int64[G],
 * 0 <= n[i] <= N_i.  Synchronizes. */
CSC_API csc_status csc_sample_batched(csc_graph g, const int64_t* n, uint64_t seed, int64_t* idx_out, void* stream);

/* csc_kmeans_batched -- csc_kmeans_reduced on n_problems point sets in one launch:
 * problem i has n[i] rows of X (device, stride ld) after those of problems < i,
 * k[i] clusters and seed + i; labels_out: device int32[sum n], same row order.
 * inertia_out: NULL or host double[n_problems].  Synchronizes. */
CSC_API csc_status csc_kmeans_batched(const float* X, int32_t n_problems, const int64_t* n, const int32_t* k,
                                      int32_t d, int32_t ld, int32_t replicates, int32_t max_iter, uint64_t seed,
                                      int32_t* labels_out, double* inertia_out, void* stream);

/* csc_interpolate_batched -- csc_interpolate per graph (Eq. 5): graph i solves
 * its k[i] systems on its own rows; all systems share every sparse product and
 * CG step, each with its own scalars and stopping test.  sample_idx: device
 * int64[n_total] packed node indices; sample_labels: device int32[n_total],
 * each below its graph's k.  labels_out: device int32[N]; fuzzy_out: NULL or
 * device float[N x max_i k_i] (columns >= k_i untouched). */
CSC_API csc_status csc_interpolate_batched(csc_graph g, const int64_t* sample_idx, const int32_t* sample_labels,
                                           int64_t n_total, const int32_t* k, int32_t g_power, double gamma,
                                           double rel_tol, int32_t max_iter, int32_t* labels_out, float* fuzzy_out,
                                           csc_cg_info* info, void* stream);

/* csc_interpolate_batched_highpass -- csc_interpolate_highpass per graph: graph i's
 * systems use g = 1 - h~ with its own cut-off lambda[i] (host double[G], each in
 * [0, 2]) and the common degree m >= 1; the Clenshaw products of every CG iteration
 * serve all graphs at once (each row range takes its graph's coefficients).  Other
 * arguments as csc_interpolate_batched. */
CSC_API csc_status csc_interpolate_batched_highpass(csc_graph g, const int64_t* sample_idx,
                                                    const int32_t* sample_labels, int64_t n_total, const int32_t* k,
                                                    const double* lambda, int32_t m, double gamma, double rel_tol,
                                                    int32_t max_iter, int32_t* labels_out, float* fuzzy_out,
                                                    csc_cg_info* info, void* stream);

/* csc_cluster_batched -- Alg. 2 for every graph: csc_estimate_lambda_k_batched,
 * csc_filter_batched (rows normalised), csc_sample_batched with n_i =
 * ceil(2 k_i ln k_i), row gather, csc_kmeans_batched, csc_interpolate_batched.
 * p: the shared parameters of csc_cluster (p->k, p->n, p->lambda_k and
 * p->bracket are ignored; d defaults to ceil(4 ln max_i N_i); p->flags may
 * hold CSC_CLENSHAW and CSC_HIGHPASS (each graph interpolated with g = 1 - h~ at
 * its own lambda_k, as csc_interpolate_batched_highpass), while CSC_VARDENSITY
 * gives CSC_E_UNSUPPORTED).  k: host int32[G].  labels_out: device int32[N].
 * lambda_out: NULL or host double[G].  info: NULL or host.  Synchronizes. */
CSC_API csc_status csc_cluster_batched(csc_graph g, const int32_t* k, const csc_params* p, int32_t* labels_out,
                                       double* lambda_out, csc_batch_info* info, void* stream);

/* ------------------------------------------------------ instrumentation
 * Launch accounting (not a step of the paper's method): every kernel launch
 * of the library is counted; while profiling is enabled each launch is also
 * bracketed by CUDA events recorded on its own stream and tagged with a
 * kernel-class name and its algorithmic bytes (the minimum bytes the
 * operation must move).  Process-wide state; not thread-safe against
 * concurrent enable/reset. */

/* csc_profile_enable -- on != 0 starts event timing of subsequent launches. */
CSC_API csc_status csc_profile_enable(int32_t on);
/* csc_profile_reset -- forget all classes and zero the launch counter. */
CSC_API csc_status csc_profile_reset(void);
/* csc_profile_launches -- kernel launches since the last reset (host int64 out). */
CSC_API csc_status csc_profile_launches(int64_t* n);
/* csc_profile_query -- class i (0-based): its name (NUL-terminated, truncated to
 * name_len), launches, summed event time in ms and summed algorithmic bytes.
 * Waits for the recorded events.  CSC_E_INVALID when i is out of range. */
CSC_API csc_status csc_profile_query(int32_t i, char* name, int32_t name_len, int64_t* launches,
                                     double* total_ms, double* bytes);

/* --------------------------------------------------------------- errors */
CSC_API const char* csc_status_str(csc_status s);
CSC_API const char* csc_last_error(void);
/* Library version string. */
CSC_API const char* csc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CSC_H */
