// ft_mlp.cu -- the learned detection-probability surrogate: a 4-layer perceptron
// d_in -> W -> W -> W -> 1 (ReLU between layers, sigmoid output) trained with binary cross
// entropy and Adam, entirely by the kernels below; FP32 training, BF16 inference.
//
// The detection probability it models is the paper's p_det (Sec. V, Eqs. (pdet_abstract),
// (simple_eq)): the fraction of a signal population that the search detects.  Training
// labels are outcomes of injection-recovery runs (ft_run_injections + the rule z > tau).
//
// Parameters, FP32, one contiguous vector in this order:
//   W1[W][d_in] b1[W] W2[W][W] b2[W] W3[W][W] b3[W] W4[1][W] b4[1].
// Determinism: every reduction (over the batch for weight gradients, over a row for a
// layer output) runs in a fixed order, so a training run is bit-reproducible.
#include "ft_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

struct ft_mlp {
    ft_ctx *ctx = nullptr;
    int d_in = 0, width = 0;
    long long n_params = 0;
    float *d_theta = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    __nv_bfloat16 *d_theta_bf16 = nullptr;
    bool bf16_stale = true;
    long long adam_t = 0;
    // workspace for a batch: activations (pre-activation kept for ReLU masks)
    float *d_act = nullptr;
    size_t act_floats = 0;
    float *d_loss = nullptr;
    float *d_xb = nullptr, *d_yb = nullptr;
    size_t batch_cap = 0;
    int *d_idx = nullptr;
};

namespace {

constexpr int kT = 16;  // GEMM tile

struct Layout {
    long long W1, b1, W2, b2, W3, b3, W4, b4, n;
};

Layout layout(int d, int w)
{
    Layout L;
    long long o = 0;
    L.W1 = o;
    o += static_cast<long long>(w) * d;
    L.b1 = o;
    o += w;
    L.W2 = o;
    o += static_cast<long long>(w) * w;
    L.b2 = o;
    o += w;
    L.W3 = o;
    o += static_cast<long long>(w) * w;
    L.b3 = o;
    o += w;
    L.W4 = o;
    o += w;
    L.b4 = o;
    o += 1;
    L.n = o;
    return L;
}

// Y[m][n] = act(sum_k X[m][k] Wt[n][k] + b[n]); act = ReLU if relu.  Fixed-order k loop.
__global__ void k_linear_fwd(const float *X, const float *Wt, const float *b, float *Y, int M,
                             int N, int K, int relu)
{
    __shared__ float xs[kT][kT + 1], ws[kT][kT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * kT + ty, n = blockIdx.x * kT + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += kT) {
        xs[ty][tx] = (m < M && k0 + tx < K) ? X[static_cast<long long>(m) * K + k0 + tx] : 0.f;
        ws[ty][tx] = (blockIdx.x * kT + ty < N && k0 + tx < K)
                         ? Wt[static_cast<long long>(blockIdx.x * kT + ty) * K + k0 + tx]
                         : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kT; ++k)
            acc = __fmaf_rn(xs[ty][k], ws[tx][k], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        float y = __fadd_rn(acc, b[n]);
        if (relu)
            y = y > 0.f ? y : 0.f;
        Y[static_cast<long long>(m) * N + n] = y;
    }
}

// dX[m][k] = (sum_n dY[m][n] Wt[n][k]) * (X[m][k] > 0 if mask)  (X = the layer's input,
// which is a ReLU output for hidden layers, so X > 0 is the ReLU derivative).
__global__ void k_linear_bwd_data(const float *dY, const float *Wt, const float *X, float *dX, int M,
                                  int N, int K, int mask)
{
    __shared__ float ds[kT][kT + 1], ws[kT][kT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * kT + ty, k = blockIdx.x * kT + tx;
    float acc = 0.f;
    for (int n0 = 0; n0 < N; n0 += kT) {
        ds[ty][tx] = (m < M && n0 + tx < N) ? dY[static_cast<long long>(m) * N + n0 + tx] : 0.f;
        ws[ty][tx] = (n0 + ty < N && k < K) ? Wt[static_cast<long long>(n0 + ty) * K + k] : 0.f;
        __syncthreads();
#pragma unroll
        for (int n = 0; n < kT; ++n)
            acc = __fmaf_rn(ds[ty][n], ws[n][tx], acc);
        __syncthreads();
    }
    if (m < M && k < K) {
        if (mask && !(X[static_cast<long long>(m) * K + k] > 0.f))
            acc = 0.f;
        dX[static_cast<long long>(m) * K + k] = acc;
    }
}

// dW[n][k] = sum_m dY[m][n] X[m][k] (m ascending), db[n] = sum_m dY[m][n].
__global__ void k_linear_bwd_weight(const float *dY, const float *X, float *dW, float *db, int M,
                                    int N, int K)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long tot = static_cast<long long>(N) * (K + 1);
    if (i >= tot)
        return;
    const int n = static_cast<int>(i / (K + 1)), k = static_cast<int>(i % (K + 1));
    float acc = 0.f;
    if (k < K) {
        for (int m = 0; m < M; ++m)
            acc = __fmaf_rn(dY[static_cast<long long>(m) * N + n], X[static_cast<long long>(m) * K + k], acc);
        dW[static_cast<long long>(n) * K + k] = acc;
    } else {
        for (int m = 0; m < M; ++m)
            acc = __fadd_rn(acc, dY[static_cast<long long>(m) * N + n]);
        db[n] = acc;
    }
}

// Output layer: logit z = Y3 . W4 + b4 per sample was formed by k_linear_fwd (N = 1);
// d loss / d z for mean binary cross entropy with logits = (sigmoid(z) - y) / B.  The loss
// is summed in sample order by one thread.
__global__ void k_bce(const float *z, const float *y, int B, float *dz, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) {
        const float s = 1.f / (1.f + expf(-z[i]));
        dz[i] = (s - y[i]) / static_cast<float>(B);
    }
    if (i == 0) {
        double L = 0.0;
        for (int j = 0; j < B; ++j) {
            const double zz = z[j], yy = y[j];
            L += fmax(zz, 0.0) - zz * yy + log1p(exp(-fabs(zz)));
        }
        *loss = static_cast<float>(L / B);
    }
}

__global__ void k_sigmoid(float *z, long long n)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < n)
        z[i] = 1.f / (1.f + expf(-z[i]));
}

__global__ void k_adam(float *theta, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_gather_rows(const float *X, const float *y, const int *idx, int B, int d,
                              float *xb, float *yb)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < static_cast<long long>(B) * d) {
        const int r = static_cast<int>(i / d), c = static_cast<int>(i % d);
        xb[i] = X[static_cast<long long>(idx[r]) * d + c];
    }
    if (i < B)
        yb[i] = y[idx[i]];
}

__global__ void k_to_bf16(const float *a, __nv_bfloat16 *b, long long n)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i < n)
        b[i] = __float2bfloat16_rn(a[i]);
}

// BF16 inference: one warp per sample; weights and activations in BF16, FP32 accumulation;
// p = sigmoid(logit).  Hidden widths up to 256.
__global__ void k_infer_bf16(const float *X, long long n, int d, int w, const __nv_bfloat16 *th,
                             long long oW1, long long ob1, long long oW2, long long ob2, long long oW3,
                             long long ob3, long long oW4, long long ob4, float *p)
{
    extern __shared__ __nv_bfloat16 sact[];  // [warps][2][w]
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long s = blockIdx.x * static_cast<long long>(blockDim.x >> 5) + wp;
    __nv_bfloat16 *a0 = sact + static_cast<size_t>(wp) * 2 * w, *a1 = a0 + w;
    if (s < n) {
        // layer 1 from the FP32 features (rounded to BF16)
        for (int o = lane; o < w; o += 32) {
            float acc = __bfloat162float(th[ob1 + o]);
            for (int k = 0; k < d; ++k)
                acc = __fmaf_rn(__bfloat162float(th[oW1 + static_cast<long long>(o) * d + k]),
                                __bfloat162float(__float2bfloat16_rn(X[s * d + k])), acc);
            a0[o] = __float2bfloat16_rn(acc > 0.f ? acc : 0.f);
        }
        __syncwarp();
        const long long oW[2] = {oW2, oW3}, ob[2] = {ob2, ob3};
        for (int l = 0; l < 2; ++l) {
            __nv_bfloat16 *in = l == 0 ? a0 : a1, *out = l == 0 ? a1 : a0;
            for (int o = lane; o < w; o += 32) {
                float acc = __bfloat162float(th[ob[l] + o]);
                for (int k = 0; k < w; ++k)
                    acc = __fmaf_rn(__bfloat162float(th[oW[l] + static_cast<long long>(o) * w + k]),
                                    __bfloat162float(in[k]), acc);
                out[o] = __float2bfloat16_rn(acc > 0.f ? acc : 0.f);
            }
            __syncwarp();
        }
        float acc = 0.f;
        for (int k = lane; k < w; k += 32)
            acc = __fmaf_rn(__bfloat162float(th[oW4 + k]), __bfloat162float(a0[k]), acc);
        for (int off = 16; off > 0; off >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0)
            p[s] = 1.f / (1.f + expf(-(acc + __bfloat162float(th[ob4]))));
    }
}

dim3 gemm_grid(int M, int N)
{
    return dim3((N + kT - 1) / kT, (M + kT - 1) / kT);
}

int ensure_batch(ft_mlp *m, size_t B)
{
    if (B <= m->batch_cap)
        return FT_OK;
    cudaFree(m->d_act);
    cudaFree(m->d_xb);
    cudaFree(m->d_yb);
    cudaFree(m->d_idx);
    m->d_act = m->d_xb = m->d_yb = nullptr;
    m->d_idx = nullptr;
    // activations: Y1, Y2, Y3 [B][W], z [B]; gradients dY1..dY3 [B][W], dz [B]
    m->act_floats = B * (6 * static_cast<size_t>(m->width) + 2);
    FT_CUDA(cudaMalloc(&m->d_act, m->act_floats * 4));
    FT_CUDA(cudaMalloc(&m->d_xb, B * m->d_in * 4));
    FT_CUDA(cudaMalloc(&m->d_yb, B * 4));
    FT_CUDA(cudaMalloc(&m->d_idx, B * 4));
    m->batch_cap = B;
    return FT_OK;
}

// forward + backward of one batch already on the device; gradient into d_grad
int loss_grad_dev(ft_mlp *m, const float *X, const float *y, int B, cudaStream_t st)
{
    const int d = m->d_in, w = m->width;
    const Layout L = layout(d, w);
    float *th = m->d_theta, *g = m->d_grad;
    float *Y1 = m->d_act, *Y2 = Y1 + static_cast<size_t>(B) * w, *Y3 = Y2 + static_cast<size_t>(B) * w;
    float *z = Y3 + static_cast<size_t>(B) * w;
    float *dY1 = z + B, *dY2 = dY1 + static_cast<size_t>(B) * w, *dY3 = dY2 + static_cast<size_t>(B) * w;
    float *dz = dY3 + static_cast<size_t>(B) * w;
    const dim3 blk(kT, kT);
    k_linear_fwd<<<gemm_grid(B, w), blk, 0, st>>>(X, th + L.W1, th + L.b1, Y1, B, w, d, 1);
    k_linear_fwd<<<gemm_grid(B, w), blk, 0, st>>>(Y1, th + L.W2, th + L.b2, Y2, B, w, w, 1);
    k_linear_fwd<<<gemm_grid(B, w), blk, 0, st>>>(Y2, th + L.W3, th + L.b3, Y3, B, w, w, 1);
    k_linear_fwd<<<gemm_grid(B, 1), blk, 0, st>>>(Y3, th + L.W4, th + L.b4, z, B, 1, w, 0);
    k_bce<<<(B + 255) / 256, 256, 0, st>>>(z, y, B, dz, m->d_loss);
    auto wgrid = [](long long tot) { return static_cast<unsigned>((tot + 255) / 256); };
    k_linear_bwd_weight<<<wgrid(1ll * (w + 1)), 256, 0, st>>>(dz, Y3, g + L.W4, g + L.b4, B, 1, w);
    k_linear_bwd_data<<<gemm_grid(B, w), blk, 0, st>>>(dz, th + L.W4, Y3, dY3, B, 1, w, 1);
    k_linear_bwd_weight<<<wgrid(1ll * w * (w + 1)), 256, 0, st>>>(dY3, Y2, g + L.W3, g + L.b3, B, w, w);
    k_linear_bwd_data<<<gemm_grid(B, w), blk, 0, st>>>(dY3, th + L.W3, Y2, dY2, B, w, w, 1);
    k_linear_bwd_weight<<<wgrid(1ll * w * (w + 1)), 256, 0, st>>>(dY2, Y1, g + L.W2, g + L.b2, B, w, w);
    k_linear_bwd_data<<<gemm_grid(B, w), blk, 0, st>>>(dY2, th + L.W2, Y1, dY1, B, w, w, 1);
    k_linear_bwd_weight<<<wgrid(1ll * w * (d + 1)), 256, 0, st>>>(dY1, X, g + L.W1, g + L.b1, B, w, d);
    FT_CUDA(cudaGetLastError());
    m->bf16_stale = true;
    return FT_OK;
}

int adam_dev(ft_mlp *m, float lr, float b1, float b2, float eps, cudaStream_t st)
{
    m->adam_t += 1;
    const float c1 = static_cast<float>(1.0 - std::pow(static_cast<double>(b1), static_cast<double>(m->adam_t)));
    const float c2 = static_cast<float>(1.0 - std::pow(static_cast<double>(b2), static_cast<double>(m->adam_t)));
    k_adam<<<static_cast<unsigned>((m->n_params + 255) / 256), 256, 0, st>>>(
        m->d_theta, m->d_grad, m->d_m, m->d_v, m->n_params, lr, b1, b2, eps, c1, c2);
    FT_CUDA(cudaGetLastError());
    m->bf16_stale = true;
    return FT_OK;
}

}  // namespace

extern "C" {

int ft_mlp_create(ft_ctx *ctx, int d_in, int width, uint64_t seed, ft_mlp **out)
{
    if (!ctx || !out)
        FT_FAIL(FT_ERR_ARG, "mlp_create: null argument");
    if (d_in < 1 || d_in > 256 || width < 1 || width > 256)
        FT_FAIL(FT_ERR_RANGE, "mlp_create: d_in and width must be in [1, 256]");
    ft_mlp *m = new ft_mlp;
    m->ctx = ctx;
    (void)cudaGetLastError();
    m->d_in = d_in;
    m->width = width;
    const Layout L = layout(d_in, width);
    m->n_params = L.n;
    // He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from a seeded host generator
    std::vector<float> th(L.n, 0.f);
    std::mt19937_64 gen(seed);
    auto fill = [&](long long off, long long cnt, int fan_in) {
        std::uniform_real_distribution<double> U(-std::sqrt(6.0 / fan_in), std::sqrt(6.0 / fan_in));
        for (long long i = 0; i < cnt; ++i)
            th[off + i] = static_cast<float>(U(gen));
    };
    fill(L.W1, 1ll * width * d_in, d_in);
    fill(L.W2, 1ll * width * width, width);
    fill(L.W3, 1ll * width * width, width);
    fill(L.W4, width, width);
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_theta, L.n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_grad, L.n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_m, L.n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_v, L.n * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_theta_bf16, L.n * 2)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_loss, 4)) != cudaSuccess) {
        ft_mlp_destroy(m);
        FT_FAIL(FT_ERR_OOM, "mlp_create: allocation failed");
    }
    cudaMemcpy(m->d_theta, th.data(), L.n * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->d_grad, 0, L.n * 4);
    cudaMemset(m->d_m, 0, L.n * 4);
    cudaMemset(m->d_v, 0, L.n * 4);
    *out = m;
    return FT_OK;
}

void ft_mlp_destroy(ft_mlp *m)
{
    if (!m)
        return;
    cudaFree(m->d_theta);
    cudaFree(m->d_grad);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_theta_bf16);
    cudaFree(m->d_act);
    cudaFree(m->d_loss);
    cudaFree(m->d_xb);
    cudaFree(m->d_yb);
    cudaFree(m->d_idx);
    delete m;
}

int ft_mlp_n_params(const ft_mlp *m, int64_t *n)
{
    if (!m || !n)
        FT_FAIL(FT_ERR_ARG, "mlp_n_params: null argument");
    *n = m->n_params;
    return FT_OK;
}

int ft_mlp_get_params(ft_mlp *m, float *host)
{
    if (!m || !host)
        FT_FAIL(FT_ERR_ARG, "mlp_get_params: null argument");
    FT_CUDA(cudaMemcpy(host, m->d_theta, m->n_params * 4, cudaMemcpyDeviceToHost));
    return FT_OK;
}

int ft_mlp_set_params(ft_mlp *m, const float *host)
{
    if (!m || !host)
        FT_FAIL(FT_ERR_ARG, "mlp_set_params: null argument");
    FT_CUDA(cudaMemcpy(m->d_theta, host, m->n_params * 4, cudaMemcpyHostToDevice));
    FT_CUDA(cudaMemset(m->d_m, 0, m->n_params * 4));
    FT_CUDA(cudaMemset(m->d_v, 0, m->n_params * 4));
    m->adam_t = 0;
    m->bf16_stale = true;
    return FT_OK;
}

int ft_mlp_get_state(ft_mlp *m, float *state, int64_t *adam_t)
{
    if (!m || !state || !adam_t)
        FT_FAIL(FT_ERR_ARG, "mlp_get_state: null argument");
    const size_t nb = static_cast<size_t>(m->n_params) * 4;
    FT_CUDA(cudaMemcpy(state, m->d_theta, nb, cudaMemcpyDeviceToHost));
    FT_CUDA(cudaMemcpy(state + m->n_params, m->d_m, nb, cudaMemcpyDeviceToHost));
    FT_CUDA(cudaMemcpy(state + 2 * m->n_params, m->d_v, nb, cudaMemcpyDeviceToHost));
    *adam_t = m->adam_t;
    return FT_OK;
}

int ft_mlp_set_state(ft_mlp *m, const float *state, int64_t adam_t)
{
    if (!m || !state || adam_t < 0)
        FT_FAIL(FT_ERR_ARG, "mlp_set_state: bad arguments");
    const size_t nb = static_cast<size_t>(m->n_params) * 4;
    FT_CUDA(cudaMemcpy(m->d_theta, state, nb, cudaMemcpyHostToDevice));
    FT_CUDA(cudaMemcpy(m->d_m, state + m->n_params, nb, cudaMemcpyHostToDevice));
    FT_CUDA(cudaMemcpy(m->d_v, state + 2 * m->n_params, nb, cudaMemcpyHostToDevice));
    m->adam_t = adam_t;
    m->bf16_stale = true;
    return FT_OK;
}

int ft_mlp_loss_grad(ft_mlp *m, const float *X, const float *y, int B, float *loss, float *grad)
{
    if (!m || !X || !y || B < 1)
        FT_FAIL(FT_ERR_ARG, "mlp_loss_grad: bad arguments");
    FT_TRY(ensure_batch(m, B));
    FT_CUDA(cudaMemcpy(m->d_xb, X, static_cast<size_t>(B) * m->d_in * 4, cudaMemcpyHostToDevice));
    FT_CUDA(cudaMemcpy(m->d_yb, y, static_cast<size_t>(B) * 4, cudaMemcpyHostToDevice));
    FT_TRY(loss_grad_dev(m, m->d_xb, m->d_yb, B, nullptr));
    FT_CUDA(cudaDeviceSynchronize());
    if (loss)
        FT_CUDA(cudaMemcpy(loss, m->d_loss, 4, cudaMemcpyDeviceToHost));
    if (grad)
        FT_CUDA(cudaMemcpy(grad, m->d_grad, m->n_params * 4, cudaMemcpyDeviceToHost));
    return FT_OK;
}

int ft_mlp_adam_step(ft_mlp *m, float lr, float beta1, float beta2, float eps)
{
    if (!m)
        FT_FAIL(FT_ERR_ARG, "mlp_adam_step: null mlp");
    FT_TRY(adam_dev(m, lr, beta1, beta2, eps, nullptr));
    FT_CUDA(cudaDeviceSynchronize());
    return FT_OK;
}

int ft_mlp_train(ft_mlp *m, const float *X, const float *y, int64_t n, int batch, int epochs, float lr,
                 uint64_t seed, float *loss_history)
{
    if (!m || !X || !y || n < 1 || batch < 1 || epochs < 0 || !(lr > 0))
        FT_FAIL(FT_ERR_ARG, "mlp_train: bad arguments");
    const int B = static_cast<int>(std::min<int64_t>(batch, n));
    FT_TRY(ensure_batch(m, B));
    float *dX = nullptr, *dy = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&dX, n * m->d_in * 4)) != cudaSuccess || (e = cudaMalloc(&dy, n * 4)) != cudaSuccess) {
        cudaFree(dX);
        FT_FAIL(FT_ERR_OOM, "mlp_train: allocation failed");
    }
    struct Free {
        float *a, *b;
        ~Free()
        {
            cudaFree(a);
            cudaFree(b);
        }
    } fr{dX, dy};
    FT_CUDA(cudaMemcpy(dX, X, n * m->d_in * 4, cudaMemcpyHostToDevice));
    FT_CUDA(cudaMemcpy(dy, y, n * 4, cudaMemcpyHostToDevice));
    std::vector<int> perm(n);
    std::mt19937_64 gen(seed);
    const int nb = static_cast<int>((n + B - 1) / B);
    for (int ep = 0; ep < epochs; ++ep) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), gen);
        double sum = 0.0;
        for (int bi = 0; bi < nb; ++bi) {
            const int off = bi * B;
            const int b = static_cast<int>(std::min<int64_t>(B, n - off));
            FT_CUDA(cudaMemcpy(m->d_idx, perm.data() + off, b * 4, cudaMemcpyHostToDevice));
            k_gather_rows<<<static_cast<unsigned>((1ll * b * m->d_in + 255) / 256), 256>>>(
                dX, dy, m->d_idx, b, m->d_in, m->d_xb, m->d_yb);
            FT_TRY(loss_grad_dev(m, m->d_xb, m->d_yb, b, nullptr));
            FT_TRY(adam_dev(m, lr, 0.9f, 0.999f, 1e-8f, nullptr));
            if (loss_history) {
                float l = 0.f;
                FT_CUDA(cudaMemcpy(&l, m->d_loss, 4, cudaMemcpyDeviceToHost));
                sum += static_cast<double>(l) * b;
            }
        }
        if (loss_history)
            loss_history[ep] = static_cast<float>(sum / n);
    }
    FT_CUDA(cudaDeviceSynchronize());
    return FT_OK;
}

int ft_mlp_predict(ft_mlp *m, const float *X, int64_t n, float *p, int bf16, int on_device, void *stream)
{
    if (!m || !X || !p || n < 0)
        FT_FAIL(FT_ERR_ARG, "mlp_predict: bad arguments");
    if (n == 0)
        return FT_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *dX = X;
    float *dp = p;
    float *tmpX = nullptr, *tmpP = nullptr;
    if (!on_device) {
        FT_CUDA(cudaMalloc(&tmpX, n * m->d_in * 4));
        if (cudaMalloc(&tmpP, n * 4) != cudaSuccess) {
            cudaFree(tmpX);
            FT_FAIL(FT_ERR_OOM, "mlp_predict: allocation failed");
        }
        cudaMemcpyAsync(tmpX, X, n * m->d_in * 4, cudaMemcpyHostToDevice, st);
        dX = tmpX;
        dp = tmpP;
    }
    const Layout L = layout(m->d_in, m->width);
    int rc = FT_OK;
    if (bf16) {
        if (m->bf16_stale) {
            k_to_bf16<<<static_cast<unsigned>((m->n_params + 255) / 256), 256, 0, st>>>(m->d_theta, m->d_theta_bf16,
                                                                                          m->n_params);
            m->bf16_stale = false;
        }
        const int warps = 8;
        k_infer_bf16<<<static_cast<unsigned>((n + warps - 1) / warps), 32 * warps,
                       warps * 2 * m->width * sizeof(__nv_bfloat16), st>>>(
            dX, n, m->d_in, m->width, m->d_theta_bf16, L.W1, L.b1, L.W2, L.b2, L.W3, L.b3, L.W4, L.b4, dp);
    } else {
        // FP32 forward in chunks through the training kernels
        const int chunk = 4096;
        rc = ensure_batch(m, chunk);
        if (rc == FT_OK) {
            const int d = m->d_in, w = m->width;
            float *Y1 = m->d_act, *Y2 = Y1 + static_cast<size_t>(chunk) * w, *Y3 = Y2 + static_cast<size_t>(chunk) * w;
            const dim3 blk(kT, kT);
            for (int64_t o = 0; o < n; o += chunk) {
                const int b = static_cast<int>(std::min<int64_t>(chunk, n - o));
                const float *xo = dX + o * d;
                k_linear_fwd<<<gemm_grid(b, w), blk, 0, st>>>(xo, m->d_theta + L.W1, m->d_theta + L.b1, Y1, b, w, d, 1);
                k_linear_fwd<<<gemm_grid(b, w), blk, 0, st>>>(Y1, m->d_theta + L.W2, m->d_theta + L.b2, Y2, b, w, w, 1);
                k_linear_fwd<<<gemm_grid(b, w), blk, 0, st>>>(Y2, m->d_theta + L.W3, m->d_theta + L.b3, Y3, b, w, w, 1);
                k_linear_fwd<<<gemm_grid(b, 1), blk, 0, st>>>(Y3, m->d_theta + L.W4, m->d_theta + L.b4, dp + o, b, 1, w, 0);
            }
            // logits -> probabilities
            k_sigmoid<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(dp, n);
        }
    }
    if (rc == FT_OK && cudaGetLastError() != cudaSuccess)
        rc = FT_ERR_CUDA;
    if (!on_device) {
        if (rc == FT_OK)
            cudaMemcpyAsync(p, tmpP, n * 4, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        cudaFree(tmpX);
        cudaFree(tmpP);
    }
    if (rc != FT_OK)
        FT_FAIL(rc, "mlp_predict: launch failed");
    return FT_OK;
}

}  // extern "C"
