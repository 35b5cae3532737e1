// mlp.cu -- the lambda_k bracket regressor: a 72 -> 256 -> 256 -> 2 ReLU
// perceptron with smooth-L1 loss and Adam, trained and run on the device.
//
// The paper finds lambda_k by a dichotomy on an eigencount (Sec. 4.3); this
// network proposes a bracket for that dichotomy and the eigencount checks it.
// Parameters are one flat fp32 vector: W1 [72 x 256] (row = input), b1, W2
// [256 x 256], b2, W3 [256 x 2], b3 (84,994 values).  Activations are B x width
// row-major.  Every reduction runs in a fixed order (weight gradients loop over
// the batch in sample order; the loss is summed by one block), so results do
// not depend on scheduling.  The layers are a few hundred kFLOP per graph:
// these kernels are latency-bound by design and use plain FMA pipes.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "device.cuh"

namespace csc {
namespace {

constexpr int kIn = CSC_MLP_IN, kH = CSC_MLP_HIDDEN, kOut = CSC_MLP_OUT;
constexpr int64_t oW1 = 0, ob1 = oW1 + kIn * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
                  ob3 = oW3 + kH * kOut, kParams = ob3 + kOut;
static_assert(kParams == CSC_MLP_PARAMS, "parameter layout");
constexpr uint32_t STREAM_MLP = 0x4D4C5049u;
constexpr int kMaxBatch = 1 << 16;

// He-uniform weights U(-a, a), a = sqrt(6 / fan_in), from Philox (counter =
// parameter index); biases 0.
__global__ void mlp_init_kernel(float* __restrict__ p, uint64_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    int fan_in = 0;
    if (i < ob1) fan_in = kIn;
    else if (i >= oW2 && i < ob2) fan_in = kH;
    else if (i >= oW3 && i < ob3) fan_in = kH;
    if (fan_in == 0) {
        p[i] = 0.f;
        return;
    }
    const Philox4 r = philox4x32_10((uint32_t)i, 0u, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32) ^ STREAM_MLP);
    const float u = philox_uniform(r.x[0]);
    p[i] = (2.f * u - 1.f) * sqrtf(6.f / (float)fan_in);
}

// out[b, o] = act(bias[o] + sum_i in[b, i] W[i, o]); one block row per sample.
template <bool RELU>
__global__ void __launch_bounds__(256) dense_fwd_kernel(const float* __restrict__ in, int din,
                                                        const float* __restrict__ W, const float* __restrict__ bias,
                                                        int dout, float* __restrict__ out) {
    __shared__ float xs[kH];
    const int b = blockIdx.y;
    for (int i = threadIdx.x; i < din; i += blockDim.x) xs[i] = in[(int64_t)b * din + i];
    __syncthreads();
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= dout) return;
    float acc = bias[o];
    for (int i = 0; i < din; ++i) acc = fmaf(xs[i], W[(int64_t)i * dout + o], acc);
    out[(int64_t)b * dout + o] = RELU ? fmaxf(acc, 0.f) : acc;
}

// Smooth-L1 (beta = 1) over the B x 2 outputs: dY = clip(Y - T, -1, 1) / (2B),
// loss = mean of the elementwise loss, summed in fp64 by one block in a fixed order.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                                        int n, float* __restrict__ dY, double* __restrict__ loss) {
    __shared__ double red[256];
    double s = 0.0;
    const float inv = 1.f / (float)n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float e = Y[i] - T[i];
        const float a = fabsf(e);
        s += a < 1.f ? 0.5 * (double)e * (double)e : (double)a - 0.5;
        dY[i] = fminf(fmaxf(e, -1.f), 1.f) * inv;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (double)n;
}

// dIn[b, i] = [act[b, i] > 0] * sum_o dOut[b, o] W[i, o]
__global__ void __launch_bounds__(256) dense_bwd_kernel(const float* __restrict__ dOut, int dout,
                                                        const float* __restrict__ W, const float* __restrict__ act,
                                                        int din, float* __restrict__ dIn) {
    __shared__ float gs[kH];
    const int b = blockIdx.y;
    for (int o = threadIdx.x; o < dout; o += blockDim.x) gs[o] = dOut[(int64_t)b * dout + o];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= din) return;
    float acc = 0.f;
    const float* wr = W + (int64_t)i * dout;
    for (int o = 0; o < dout; ++o) acc = fmaf(gs[o], wr[o], acc);
    dIn[(int64_t)b * din + i] = act[(int64_t)b * din + i] > 0.f ? acc : 0.f;
}

// gW[i, o] = sum_b in[b, i] dOut[b, o]; gb[o] = sum_b dOut[b, o] (thread row din).
__global__ void __launch_bounds__(256) wgrad_kernel(const float* __restrict__ in, int din,
                                                    const float* __restrict__ dOut, int dout, int B,
                                                    float* __restrict__ gW, float* __restrict__ gb) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)(din + 1) * dout) return;
    const int i = (int)(t / dout), o = (int)(t % dout);
    float acc = 0.f;
    if (i < din) {
        for (int b = 0; b < B; ++b) acc = fmaf(in[(int64_t)b * din + i], dOut[(int64_t)b * dout + o], acc);
        gW[(int64_t)i * dout + o] = acc;
    } else {
        for (int b = 0; b < B; ++b) acc += dOut[(int64_t)b * dout + o];
        gb[o] = acc;
    }
}

// Adam with bias correction (Kingma & Ba 2015); bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float bc1, float bc2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

__global__ void gather_batch_kernel(const float* __restrict__ X, const float* __restrict__ T,
                                    const int32_t* __restrict__ idx, int B, float* __restrict__ Xb,
                                    float* __restrict__ Tb) {
    const int b = blockIdx.x;
    const int64_t r = idx[b];
    for (int i = threadIdx.x; i < kIn; i += blockDim.x) Xb[(int64_t)b * kIn + i] = X[r * kIn + i];
    if (threadIdx.x < kOut) Tb[(int64_t)b * kOut + threadIdx.x] = T[r * kOut + threadIdx.x];
}

// Activation scratch for a batch of B: H1, H2, Y, dY, dH2, dH1 (+ Xb, Tb, index).
struct MlpScratch {
    float* base = nullptr;
    size_t cap = 0;
};
std::mutex g_mlp_mu;
MlpScratch g_mlp_scratch[64];

csc_status mlp_scratch(int B, float** out) {
    // activations (carve order), 256-byte alignment pad, grad / m / v, fp64 loss slot
    const size_t need = (size_t)B * (4 * kH + 3 * kOut + kIn) + 64 + kParams * 3 + 64;
    int dev = 0;
    CSC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return CSC_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    MlpScratch& sc = g_mlp_scratch[dev];
    if (sc.cap < need) {
        if (sc.base) {
            CSC_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(sc.base);
            sc.base = nullptr;
            sc.cap = 0;
        }
        cudaError_t e = cudaMalloc(&sc.base, need * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("mlp scratch: cudaMalloc(%zu): %s", need * sizeof(float), cudaGetErrorString(e));
            return CSC_E_OOM;
        }
        sc.cap = need;
    }
    *out = sc.base;
    return CSC_OK;
}

struct Acts {
    float *h1, *h2, *y, *dy, *dh2, *dh1, *xb, *tb, *gm, *gv, *grad;
};

Acts carve(float* base, int B) {
    Acts a;
    float* p = base;
    a.h1 = p, p += (size_t)B * kH;
    a.h2 = p, p += (size_t)B * kH;
    a.dh2 = p, p += (size_t)B * kH;
    a.dh1 = p, p += (size_t)B * kH;
    a.y = p, p += (size_t)B * kOut;
    a.dy = p, p += (size_t)B * kOut;
    a.xb = p, p += (size_t)B * kIn;
    a.tb = p, p += (size_t)B * kOut;
    p = (float*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    a.grad = p, p += kParams;
    a.gm = p, p += kParams;
    a.gv = p;
    return a;
}

csc_status forward(const float* P, const float* X, int B, const Acts& a, float* Y, cudaStream_t s) {
    const dim3 g1(1, B), g3(1, B);
    CSC_KLAUNCH("mlp", 4.0 * B * (kIn + kH), s,
                dense_fwd_kernel<true><<<g1, 256, 0, s>>>(X, kIn, P + oW1, P + ob1, kH, a.h1));
    CSC_KLAUNCH("mlp", 8.0 * B * kH, s, dense_fwd_kernel<true><<<g1, 256, 0, s>>>(a.h1, kH, P + oW2, P + ob2, kH, a.h2));
    CSC_KLAUNCH("mlp", 4.0 * B * (kH + kOut), s,
                dense_fwd_kernel<false><<<g3, 32, 0, s>>>(a.h2, kH, P + oW3, P + ob3, kOut, Y));
    return CSC_OK;
}

csc_status backward(const float* P, const float* X, int B, const Acts& a, double* loss, const float* T,
                    float* grad, cudaStream_t s) {
    CSC_KLAUNCH("mlp", 12.0 * B * kOut, s, loss_grad_kernel<<<1, 256, 0, s>>>(a.y, T, B * kOut, a.dy, loss));
    const dim3 gb(1, B);
    CSC_KLAUNCH("mlp", 8.0 * B * kH, s, dense_bwd_kernel<<<gb, 256, 0, s>>>(a.dy, kOut, P + oW3, a.h2, kH, a.dh2));
    CSC_KLAUNCH("mlp", 8.0 * B * kH, s, dense_bwd_kernel<<<gb, 256, 0, s>>>(a.dh2, kH, P + oW2, a.h1, kH, a.dh1));
    auto wg = [&](const float* in, int din, const float* dout_, int dout, float* gW, float* gbias) -> csc_status {
        const int64_t n = (int64_t)(din + 1) * dout;
        CSC_KLAUNCH("mlp", 4.0 * (double)B * (din + dout) + 4.0 * n, s,
                    wgrad_kernel<<<ceil_div(n, 256), 256, 0, s>>>(in, din, dout_, dout, B, gW, gbias));
        return CSC_OK;
    };
    CSC_TRY(wg(a.h2, kH, a.dy, kOut, grad + oW3, grad + ob3));
    CSC_TRY(wg(a.h1, kH, a.dh2, kH, grad + oW2, grad + ob2));
    return wg(X, kIn, a.dh1, kH, grad + oW1, grad + ob1);
}

// one minibatch: gather, forward, backward, Adam at step t
csc_status train_step(float* params, const float* X, const float* T, const int32_t* idx, int bs, const Acts& a,
                      double* loss, int t, float lr, cudaStream_t s) {
    CSC_KLAUNCH("mlp", 4.0 * bs * (kIn + kOut) * 2, s,
                gather_batch_kernel<<<bs, 128, 0, s>>>(X, T, idx, bs, a.xb, a.tb));
    CSC_TRY(forward(params, a.xb, bs, a, a.y, s));
    CSC_TRY(backward(params, a.xb, bs, a, loss, a.tb, a.grad, s));
    const float bc1 = (float)(1.0 - pow(0.9, t)), bc2 = (float)(1.0 - pow(0.999, t));
    CSC_KLAUNCH("mlp", 24.0 * kParams, s,
                adam_kernel<<<ceil_div(kParams, 256), 256, 0, s>>>(params, a.grad, a.gm, a.gv, lr, bc1, bc2));
    return CSC_OK;
}

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

csc_status mlp_forward_device(const float* params, const float* X, int B, float* Y, cudaStream_t s) {
    float* base = nullptr;
    CSC_TRY(mlp_scratch(B, &base));
    const Acts a = carve(base, B);
    return forward(params, X, B, a, Y, s);
}

}  // namespace csc

using namespace csc;

extern "C" CSC_API csc_status csc_mlp_init(float* params, uint64_t seed, void* stream) {
    clear_error();
    if (!params) {
        set_error("csc_mlp_init: params is NULL");
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CSC_KLAUNCH("mlp", 4.0 * kParams, s, mlp_init_kernel<<<ceil_div(kParams, 256), 256, 0, s>>>(params, seed));
    CSC_CUDA_TRY(cudaGetLastError());
    return CSC_OK;
}

extern "C" CSC_API csc_status csc_mlp_forward(const float* params, const float* X, int32_t B, float* Y,
                                              void* stream) {
    clear_error();
    if (!params || !X || !Y || B < 1 || B > kMaxBatch) {
        set_error("csc_mlp_forward: need params, X, Y and 1 <= B <= %d", kMaxBatch);
        return CSC_E_INVALID;
    }
    return mlp_forward_device(params, X, B, Y, (cudaStream_t)stream);
}

extern "C" CSC_API csc_status csc_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t B,
                                                float* grad, double* loss, void* stream) {
    clear_error();
    if (!params || !X || !T || !grad || B < 1 || B > kMaxBatch) {
        set_error("csc_mlp_loss_grad: need params, X, T, grad and 1 <= B <= %d", kMaxBatch);
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* base = nullptr;
    CSC_TRY(mlp_scratch(B, &base));
    const Acts a = carve(base, B);
    double* dloss = (double*)(a.gv + kParams);  // 64 floats reserved past the Adam moments
    CSC_TRY(forward(params, X, B, a, a.y, s));
    CSC_TRY(backward(params, X, B, a, dloss, T, grad, s));
    if (loss) {
        CSC_CUDA_TRY(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CSC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return CSC_OK;
}

extern "C" CSC_API csc_status csc_mlp_adam_step(float* params, const float* grad, float* m, float* v, int32_t t,
                                                float lr, void* stream) {
    clear_error();
    if (!params || !grad || !m || !v || t < 1 || !(lr > 0.f)) {
        set_error("csc_mlp_adam_step: need params, grad, m, v, t >= 1 and lr > 0");
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float bc1 = (float)(1.0 - pow(0.9, t)), bc2 = (float)(1.0 - pow(0.999, t));
    CSC_KLAUNCH("mlp", 24.0 * kParams, s,
                adam_kernel<<<ceil_div(kParams, 256), 256, 0, s>>>(params, grad, m, v, lr, bc1, bc2));
    CSC_CUDA_TRY(cudaGetLastError());
    return CSC_OK;
}

extern "C" CSC_API csc_status csc_mlp_train(float* params, const float* X, const float* T, int32_t n,
                                            int32_t epochs, int32_t batch, float lr, uint64_t seed,
                                            double* epoch_loss, void* stream) {
    clear_error();
    if (!params || !X || !T || n < 1 || epochs < 0 || batch < 1 || batch > kMaxBatch || !(lr > 0.f)) {
        set_error("csc_mlp_train: invalid arguments (n=%d epochs=%d batch=%d)", n, epochs, batch);
        return CSC_E_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int B = std::min(batch, n);
    float* base = nullptr;
    CSC_TRY(mlp_scratch(B, &base));
    const Acts a = carve(base, B);
    const int nb = (n + B - 1) / B;
    int32_t* d_idx = nullptr;
    double* d_loss = nullptr;
    CSC_CUDA_TRY(cudaMalloc(&d_idx, (size_t)n * sizeof(int32_t)));
    cudaError_t e = cudaMalloc(&d_loss, (size_t)std::max(1, epochs * nb) * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_idx);
        set_error("csc_mlp_train: cudaMalloc: %s", cudaGetErrorString(e));
        return CSC_E_OOM;
    }
    csc_status st = CSC_OK;
    std::vector<int32_t> perm(n);
    CSC_CUDA_TRY(cudaMemsetAsync(a.gm, 0, kParams * sizeof(float), s));
    CSC_CUDA_TRY(cudaMemsetAsync(a.gv, 0, kParams * sizeof(float), s));
    int t = 0;
    for (int ep = 0; ep < epochs && st == CSC_OK; ++ep) {
        // Fisher-Yates shuffle driven by SplitMix64 on (seed, epoch, position)
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) {
            const uint64_t r = mix64(seed + 0x9E3779B97F4A7C15ull * ((uint64_t)ep * (uint64_t)n + (uint64_t)i + 1));
            std::swap(perm[i], perm[(int)(r % (uint64_t)(i + 1))]);
        }
        if (cudaMemcpyAsync(d_idx, perm.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            st = CSC_E_CUDA;
            break;
        }
        // the host array is rewritten next epoch: wait for the copy
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = CSC_E_CUDA;
            break;
        }
        for (int b = 0; b < nb && st == CSC_OK; ++b) {
            const int b0 = b * B, bs = std::min(B, n - b0);
            ++t;
            st = train_step(params, X, T, d_idx + b0, bs, a, d_loss + (size_t)ep * nb + b, t, lr, s);
        }
        if (cudaGetLastError() != cudaSuccess) st = CSC_E_CUDA;
    }
    if (st == CSC_OK && epoch_loss && epochs > 0) {
        std::vector<double> h((size_t)epochs * nb);
        if (cudaMemcpyAsync(h.data(), d_loss, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = CSC_E_CUDA;
        } else {
            // mean batch loss weighted by batch size
            for (int ep = 0; ep < epochs; ++ep) {
                double acc = 0.0;
                for (int b = 0; b < nb; ++b) acc += h[(size_t)ep * nb + b] * std::min(B, n - b * B);
                epoch_loss[ep] = acc / n;
            }
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(d_idx);
    cudaFree(d_loss);
    if (st != CSC_OK) set_error("csc_mlp_train: CUDA error during training");
    return st;
}

// ------------------------------------------------------------ bracket predictor fit
// The training-set arithmetic of the learned lambda_k bracket (an add-on the paper does
// not have): targets (centre, ln half-width) of the target brackets, standardisation
// constants of the fitted samples, the network's training, and the calibration of the
// half-width factor on the held-back samples.
namespace csc {
namespace {

// the network input of one feature row: the standardisation csc_estimate_lambda_k_learned
// applies at inference (fp32, a feature of zero spread maps to 0)
void standardise_row(const float* f, const float* norm, float* out) {
    for (int i = 0; i < CSC_MLP_IN; ++i) {
        const float sd = norm[CSC_MLP_IN + i];
        out[i] = sd > 0.f ? (f[i] - norm[i]) / sd : 0.f;
    }
}

// Eigencount evaluations that the halving started from a prediction (centre c, half-width
// hw) spends when the accepted cut-offs are exactly [lo, hi] (the count rounds to k inside,
// exceeds it above, falls short below): the centre decides the side, the predicted end on
// that side comes next, then halving inside the prediction or on the rest of [0, 2], as
// csc_estimate_lambda_k_learned searches.
int search_evaluations(double c, double hw, double lo, double hi) {
    auto side = [&](double x) { return (lo <= x && x <= hi) ? 0 : (x > hi ? 1 : -1); };
    auto halve = [&](double a, double b, int n) {
        for (int it = 1; it <= 60; ++it) {
            const double mid = 0.5 * (a + b);
            const int sd = side(mid);
            if (sd == 0) return n + it;
            if (sd > 0) b = mid; else a = mid;
            if (b - a < 1e-12 || it == 60) return n + it + 1;
        }
        return n + 60;
    };
    c = std::min(2.0, std::max(0.0, c));
    const int sc = side(c);
    if (sc == 0) return 1;
    const double e = sc > 0 ? std::max(0.0, c - hw) : std::min(2.0, c + hw);
    const int se = side(e);
    if (se == 0) return 2;
    if (sc > 0) return se < 0 ? halve(e, c, 2) : halve(0.0, e, 2);
    return se > 0 ? halve(c, e, 2) : halve(e, 2.0, 2);
}

// (centre, ln half-width) of n feature rows through the network, kMaxBatch rows at a time
csc_status predict_targets(const float* params, const float* norm, const float* feats, int n, double* t,
                           cudaStream_t s) {
    const int cb = std::min(n, kMaxBatch);
    std::vector<float> x((size_t)cb * CSC_MLP_IN), y((size_t)cb * CSC_MLP_OUT);
    float *dx = nullptr, *dy = nullptr;
    CSC_CUDA_TRY(cudaMalloc(&dx, x.size() * sizeof(float)));
    if (cudaMalloc(&dy, y.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dx);
        set_error("bracket prediction: cudaMalloc failed");
        return CSC_E_OOM;
    }
    csc_status st = CSC_OK;
    const float* tm = norm + 2 * CSC_MLP_IN;  // target mean [2], target std [2]
    for (int b0 = 0; b0 < n && st == CSC_OK; b0 += cb) {
        const int b = std::min(cb, n - b0);
        for (int i = 0; i < b; ++i)
            standardise_row(feats + (size_t)(b0 + i) * CSC_MLP_IN, norm, x.data() + (size_t)i * CSC_MLP_IN);
        if (cudaMemcpyAsync(dx, x.data(), (size_t)b * CSC_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
            st = CSC_E_CUDA;
            break;
        }
        st = mlp_forward_device(params, dx, b, dy, s);
        if (st != CSC_OK) break;
        if (cudaMemcpyAsync(y.data(), dy, (size_t)b * CSC_MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = CSC_E_CUDA;
            break;
        }
        for (int i = 0; i < b; ++i) {
            t[2 * (size_t)(b0 + i)] = (double)y[2 * (size_t)i] * tm[2] + tm[0];
            t[2 * (size_t)(b0 + i) + 1] = (double)y[2 * (size_t)i + 1] * tm[3] + tm[1];
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(dx);
    cudaFree(dy);
    if (st == CSC_E_CUDA) set_error("bracket prediction: CUDA error");
    return st;
}

}  // namespace
}  // namespace csc

extern "C" CSC_API csc_status csc_bracket_fit(const float* feats, const double* brackets, int32_t n,
                                              double val_frac, int32_t epochs, int32_t batch, float lr,
                                              uint64_t seed, int32_t widen_rule, double coverage, float* params,
                                              float* norm_out, double* widen_out, int32_t* n_fit_out,
                                              double* epoch_loss, void* stream) {
    clear_error();
    if (!feats || !brackets || n < 2 || !(val_frac >= 0.0 && val_frac < 1.0) || epochs < 0 || batch < 1 ||
        batch > kMaxBatch || !(lr > 0.f) || (widen_rule != 0 && widen_rule != 1) ||
        !(coverage > 0.0 && coverage <= 1.0) || !params || !norm_out || !widen_out) {
        set_error("csc_bracket_fit: invalid arguments (n=%d epochs=%d batch=%d rule=%d)", n, epochs, batch,
                  widen_rule);
        return CSC_E_INVALID;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!(brackets[2 * i] <= brackets[2 * i + 1])) {
            set_error("csc_bracket_fit: bracket %lld has lo > hi", (long long)i);
            return CSC_E_INVALID;
        }
    cudaStream_t s = (cudaStream_t)stream;
    // held-back share rounded half to even; none below 10 samples
    const int n_val = n >= 10 ? (int)nearbyint(val_frac * n) : 0;
    const int n_fit = n - n_val;
    if (n_fit < 1) {
        set_error("csc_bracket_fit: no sample left to fit");
        return CSC_E_INVALID;
    }
    // targets (centre, ln half-width) and the standardisation of the fitted samples
    std::vector<double> t((size_t)2 * n);
    for (int i = 0; i < n; ++i) {
        const double lo = brackets[2 * (size_t)i], hi = brackets[2 * (size_t)i + 1];
        t[2 * (size_t)i] = 0.5 * (lo + hi);
        t[2 * (size_t)i + 1] = log(std::max(0.5 * (hi - lo), 1e-12));
    }
    std::vector<double> fm(CSC_MLP_IN, 0.0), fs(CSC_MLP_IN, 0.0), tmean(2, 0.0), tstd(2, 0.0);
    for (int i = 0; i < n_fit; ++i) {
        for (int j = 0; j < CSC_MLP_IN; ++j) fm[j] += feats[(size_t)i * CSC_MLP_IN + j];
        for (int j = 0; j < 2; ++j) tmean[j] += t[2 * (size_t)i + j];
    }
    for (int j = 0; j < CSC_MLP_IN; ++j) fm[j] /= n_fit;
    for (int j = 0; j < 2; ++j) tmean[j] /= n_fit;
    for (int i = 0; i < n_fit; ++i) {
        for (int j = 0; j < CSC_MLP_IN; ++j) {
            const double v = feats[(size_t)i * CSC_MLP_IN + j] - fm[j];
            fs[j] += v * v;
        }
        for (int j = 0; j < 2; ++j) {
            const double v = t[2 * (size_t)i + j] - tmean[j];
            tstd[j] += v * v;
        }
    }
    for (int j = 0; j < CSC_MLP_IN; ++j) fs[j] = sqrt(fs[j] / n_fit);
    for (int j = 0; j < 2; ++j) {
        tstd[j] = sqrt(tstd[j] / n_fit);
        if (!(tstd[j] > 0.0)) tstd[j] = 1.0;
    }
    for (int j = 0; j < CSC_MLP_IN; ++j) {
        norm_out[j] = (float)fm[j];
        norm_out[CSC_MLP_IN + j] = (float)fs[j];
    }
    for (int j = 0; j < 2; ++j) {
        norm_out[2 * CSC_MLP_IN + j] = (float)tmean[j];
        norm_out[2 * CSC_MLP_IN + 2 + j] = (float)tstd[j];
    }
    // standardised training arrays on the device, then minibatch Adam from a fresh network
    std::vector<float> x((size_t)n_fit * CSC_MLP_IN), y((size_t)n_fit * 2);
    for (int i = 0; i < n_fit; ++i) {
        standardise_row(feats + (size_t)i * CSC_MLP_IN, norm_out, x.data() + (size_t)i * CSC_MLP_IN);
        for (int j = 0; j < 2; ++j) y[2 * (size_t)i + j] = (float)((t[2 * (size_t)i + j] - tmean[j]) / tstd[j]);
    }
    float *dx = nullptr, *dy = nullptr;
    CSC_CUDA_TRY(cudaMalloc(&dx, x.size() * sizeof(float)));
    if (cudaMalloc(&dy, y.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dx);
        set_error("csc_bracket_fit: cudaMalloc failed");
        return CSC_E_OOM;
    }
    csc_status st = CSC_OK;
    if (cudaMemcpyAsync(dx, x.data(), x.size() * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dy, y.data(), y.size() * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = CSC_E_CUDA;
    if (st == CSC_OK) st = csc_mlp_init(params, seed, stream);
    if (st == CSC_OK) st = csc_mlp_train(params, dx, dy, n_fit, epochs, batch, lr, seed, epoch_loss, stream);
    cudaStreamSynchronize(s);
    cudaFree(dx);
    cudaFree(dy);
    if (st != CSC_OK) return st;
    // the half-width factor, calibrated on the held-back samples (the fitted ones if none)
    const int c0 = n_val ? n_fit : 0, nc = n_val ? n_val : n_fit;
    std::vector<double> pt((size_t)2 * nc);
    CSC_TRY(predict_targets(params, norm_out, feats + (size_t)c0 * CSC_MLP_IN, nc, pt.data(), s));
    const double* br = brackets + 2 * (size_t)c0;
    double widen = 1.0;
    if (widen_rule == 1) {
        // the smallest factor at which a `coverage` share of the predictions meet their brackets
        std::vector<double> need(nc);
        for (int i = 0; i < nc; ++i) {
            const double c = pt[2 * (size_t)i], hw = exp(pt[2 * (size_t)i + 1]);
            const double lo = br[2 * (size_t)i], hi = br[2 * (size_t)i + 1];
            const double dist = c < lo ? lo - c : (c > hi ? c - hi : 0.0);
            need[i] = dist / hw;
        }
        std::sort(need.begin(), need.end());
        const double pos = coverage * (nc - 1);
        const int i0 = (int)floor(pos), i1 = std::min(nc - 1, i0 + 1);
        const double q = need[i0] + (pos - i0) * (need[i1] - need[i0]);
        widen = std::max(1.0, q);
    } else {
        // the factor on the grid 0.25 * 2^(j/4), j = 0..56, with the fewest mean evaluations
        double best = 1e300;
        for (int j = 0; j <= 56; ++j) {
            const double w = 0.25 * exp2(j / 4.0);
            double cost = 0.0;
            for (int i = 0; i < nc; ++i)
                cost += search_evaluations(pt[2 * (size_t)i], w * exp(std::min(pt[2 * (size_t)i + 1], 10.0)),
                                           br[2 * (size_t)i], br[2 * (size_t)i + 1]);
            cost /= nc;
            if (cost < best) {
                best = cost;
                widen = w;
            }
        }
    }
    *widen_out = widen;
    if (n_fit_out) *n_fit_out = n_fit;
    return CSC_OK;
}

extern "C" CSC_API csc_status csc_bracket_predict(const float* params, const float* norm, double widen,
                                                  const float* feats, int32_t n, double* targets_out,
                                                  double* brackets_out, void* stream) {
    clear_error();
    if (!params || !norm || !feats || n < 1 || !(widen > 0.0) || (!targets_out && !brackets_out)) {
        set_error("csc_bracket_predict: invalid arguments (n=%d)", n);
        return CSC_E_INVALID;
    }
    std::vector<double> t((size_t)2 * n);
    CSC_TRY(predict_targets(params, norm, feats, n, t.data(), (cudaStream_t)stream));
    for (int i = 0; i < n; ++i) {
        const double c = t[2 * (size_t)i], lnhw = t[2 * (size_t)i + 1];
        if (targets_out) {
            targets_out[2 * (size_t)i] = c;
            targets_out[2 * (size_t)i + 1] = lnhw;
        }
        if (brackets_out) {
            // as csc_estimate_lambda_k_learned: widen * exp(ln half-width), clipped to [0, 2]
            const double hw = widen * exp(std::min(lnhw, 10.0));
            brackets_out[2 * (size_t)i] = std::max(0.0, c - hw);
            brackets_out[2 * (size_t)i + 1] = std::min(2.0, c + hw);
        }
    }
    return CSC_OK;
}
