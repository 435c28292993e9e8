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
#include "ft_ptx.cuh"

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

// ------------------------------------------------------------------ BF16 inference on
// the tensor cores
//
// One persistent CTA per SM keeps the weights in shared memory and runs four groups of 128
// threads, each inferring its own tiles of 128 samples, so that four tiles are in flight per
// SM and one group's products overlap the others' epilogues.  Each layer of a tile is one
// M = 128 matrix product D[m][n] = sum_k A[m][k] W[n][k] by tcgen05.mma (kind::f16, BF16
// operands from shared memory, FP32 accumulators in the group's tensor-memory columns),
// issued by one thread of the group and tracked by the group's mbarrier; the products
// accumulate onto the layer's bias, stored into those columns beforehand.  Sample m's row of
// D sits in tensor-memory lane m, read by thread m of the group, which applies the ReLU with
// the rounding to BF16 (one conversion per pair) and writes the activations back to the
// group's shared-memory A for the next layer.  The last layer (width -> 1) and the sigmoid
// run on the CUDA cores in FP32.  The groups synchronise with named barriers only.
// Numerics match the SIMT BF16 path: BF16 inputs, weights and activations, FP32 sums.
//
// Shared-memory operands use the no-swizzle K-major layout of the tcgen05 matrix
// descriptors: an R x K BF16 matrix (K a multiple of 16) is a grid of 8 x 8-element core
// matrices of 128 contiguous bytes, element (r, k) at byte
//     (r / 8) (16 K) + (k / 8) 128 + (r % 8) 16 + (k % 8) 2,
// so core matrices adjacent in K are 128 bytes apart (the descriptor's leading-dimension
// offset) and adjacent 8-row groups 16 K bytes apart (its stride-dimension offset); the
// product over k in [16 i, 16 i + 16) starts 256 i bytes into each operand.

constexpr int kTcM = 128;       // samples per tile (the MMA's M)
constexpr int kTcGroups = 4;    // tiles in flight per CTA (one group of kTcM threads each)
constexpr int kTcThreads = kTcM * kTcGroups;
constexpr int kTcMaxW = 128;    // hidden widths 16 .. 128 (multiples of 16)
constexpr int kTcMaxK = 64;     // padded inputs 16 .. 64

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ int kmaj_off(int r, int k, int K)
{
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-
// dimension byte offset >> 4 (bits 16-29), stride-dimension byte offset >> 4 (bits 32-45),
// the fixed value 1 at bits 46-48, no base offset, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, int K)
{
    return static_cast<unsigned long long>((addr & 0x3FFFFu) >> 4) |
           (static_cast<unsigned long long>(128 >> 4) << 16) |
           (static_cast<unsigned long long>((K * 16) >> 4) << 32) | (1ull << 46);
}

// tcgen05 instruction descriptor, kind::f16: FP32 D (bits 4-5 = 1), BF16 A (bits 7-9 = 1)
// and B (bits 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at
// bits 24-28
__host__ __device__ constexpr unsigned tc_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<unsigned>(N >> 3) << 17) |
           (static_cast<unsigned>(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                       unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor cores' reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane, as raw bits; the values
// are usable after tc_wait_ld()
__device__ __forceinline__ void tc_ld8(unsigned taddr, unsigned *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's tensor-memory lane from shared memory (bias
// values); complete after tc_wait_st()
__device__ __forceinline__ void tc_st8(unsigned taddr, const float *v)
{
    const float4 a = *reinterpret_cast<const float4 *>(v), b = *reinterpret_cast<const float4 *>(v + 4);
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)),
                 "r"(__float_as_uint(a.w)), "r"(__float_as_uint(b.x)), "r"(__float_as_uint(b.y)),
                 "r"(__float_as_uint(b.z)), "r"(__float_as_uint(b.w))
                 : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the kTcM threads of group g (named barrier g + 1; barrier 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kTcM) : "memory");
}

// group_sync that also returns whether v holds on every thread of the group
__device__ __forceinline__ bool group_all(int g, bool v)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(g + 1), "r"(kTcM)
        : "memory");
    return r != 0;
}

// bf16(max(a, 0)) in the low half and bf16(max(b, 0)) in the high half, round to nearest
__device__ __forceinline__ unsigned relu_bf16x2(float a, float b)
{
    unsigned d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

struct TcSmem {
    size_t w1, w2, w3, act, act_bytes, bias, bar, tm, total;
};

__host__ __device__ inline TcSmem tc_layout(int K1, int W)
{
    TcSmem L;
    size_t o = 0;
    L.w1 = o;
    o += static_cast<size_t>(W) * K1 * 2;
    L.w2 = o;
    o += static_cast<size_t>(W) * W * 2;
    L.w3 = o;
    o += static_cast<size_t>(W) * W * 2;
    L.act = o;  // one A operand per group
    L.act_bytes = static_cast<size_t>(kTcM) * (K1 > W ? K1 : W) * 2;
    o += kTcGroups * L.act_bytes;
    L.bias = o;  // b1, b2, b3, W4 as FP32 [4][W], then b4
    o += (4 * static_cast<size_t>(W) + 4) * 4;
    o = (o + 15) / 16 * 16;
    L.bar = o;  // one mbarrier per group
    o += 8 * kTcGroups;
    L.tm = o;
    o += 16;
    L.total = o;
    return L;
}

// rows [0, R) x k in [0, K) of a BF16 matrix into the K-major operand layout, zero past
// (rows_valid, k_valid); the source row r starts at src + r * ld
__device__ void tc_stage_bf16(unsigned char *dst, const __nv_bfloat16 *src, long long ld, int R, int K,
                              int rows_valid, int k_valid)
{
    for (int i = threadIdx.x; i < R * (K / 8); i += blockDim.x) {
        const int r = i / (K / 8), k0 = (i - r * (K / 8)) * 8;
        __align__(16) __nv_bfloat16 e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            e[j] = (r < rows_valid && k0 + j < k_valid) ? src[r * ld + k0 + j] : __float2bfloat16_rn(0.f);
        *reinterpret_cast<uint4 *>(dst + kmaj_off(r, k0, K)) = *reinterpret_cast<const uint4 *>(e);
    }
}

// One layer's products: D (tensor-memory columns col..col+W) += A (128 x K) x W^T (W x K),
// onto the bias already stored in those columns.
__device__ __forceinline__ void tc_layer(unsigned tm, int col, const unsigned char *A, const unsigned char *Wt, int K,
                                         int W, unsigned long long *bar)
{
    const unsigned a0 = smem_u32(A), b0 = smem_u32(Wt), idesc = tc_idesc_bf16(kTcM, W);
    for (int i = 0; i < K / 16; ++i)
        tc_mma(tm + static_cast<unsigned>(col), tc_desc(a0 + 256u * i, K), tc_desc(b0 + 256u * i, K), idesc, 1);
    tc_commit(bar);
}

template <int W>
__global__ void __launch_bounds__(kTcThreads, 1) k_infer_tc(const float *X, long long n, int d, int K1,
                                                           const __nv_bfloat16 *th, long long oW1, long long ob1,
                                                           long long oW2, long long ob2, long long oW3, long long ob3,
                                                           long long oW4, long long ob4, float *p, unsigned *status)
{
    // tensor-memory columns per group (a power of two, so that the allocation is one)
    constexpr int Wc = W <= 32 ? 32 : W <= 64 ? 64 : 128;
    constexpr unsigned ncols = kTcGroups * Wc;
    extern __shared__ __align__(128) unsigned char tsm[];
    const TcSmem L = tc_layout(K1, W);
    const int g = threadIdx.x / kTcM, m = threadIdx.x % kTcM;  // group; sample row and lane
    const int warp = threadIdx.x >> 5;
    unsigned char *sW1 = tsm + L.w1, *sW2 = tsm + L.w2, *sW3 = tsm + L.w3;
    unsigned char *sA = tsm + L.act + g * L.act_bytes;
    float *sb = reinterpret_cast<float *>(tsm + L.bias);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(tsm + L.bar) + g;
    unsigned *s_tm = reinterpret_cast<unsigned *>(tsm + L.tm);
    const long long n_tiles = (n + kTcM - 1) / kTcM;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcGroups; ++i)
            ftp::mbar_init(reinterpret_cast<unsigned long long *>(tsm + L.bar) + i, 1);
        ftp::fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tm)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the weights, once per CTA (persistent over sample tiles); biases and W4 in FP32
    tc_stage_bf16(sW1, th + oW1, d, W, K1, W, d);
    tc_stage_bf16(sW2, th + oW2, W, W, W, W, W);
    tc_stage_bf16(sW3, th + oW3, W, W, W, W, W);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        sb[i] = __bfloat162float(th[ob1 + i]);
        sb[W + i] = __bfloat162float(th[ob2 + i]);
        sb[2 * W + i] = __bfloat162float(th[ob3 + i]);
        sb[3 * W + i] = __bfloat162float(th[oW4 + i]);
    }
    if (threadIdx.x == 0)
        sb[4 * W] = __bfloat162float(th[ob4]);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the group's accumulator columns; this thread's lane m (warp w reads lanes 32 (w % 4) ..)
    const unsigned tg = *s_tm + static_cast<unsigned>(g * Wc);
    const unsigned trow = tg + (static_cast<unsigned>((warp & 3) * 32) << 16);
    // layer 1's bias into this row's accumulator columns
#pragma unroll
    for (int c = 0; c < W; c += 8)
        tc_st8(trow + static_cast<unsigned>(c), sb + c);
    tc_wait_st();
    bool ok = true;
    unsigned phase = 0;  // parity of the group's barrier's next completion
    const long long stride = static_cast<long long>(gridDim.x) * kTcGroups;
    for (long long tile = static_cast<long long>(blockIdx.x) * kTcGroups + g; tile < n_tiles && ok;
         tile += stride) {
        const long long s0 = tile * kTcM;
        const int rows = static_cast<int>(min(static_cast<long long>(kTcM), n - s0));
        // this tile's features rounded to BF16 (the previous tile's last product has read A)
        for (int i = m; i < kTcM * (K1 / 8); i += kTcM) {
            const int r = i / (K1 / 8), k0 = (i - r * (K1 / 8)) * 8;
            __align__(16) __nv_bfloat16 e[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                e[j] = __float2bfloat16_rn(r < rows && k0 + j < d ? X[(s0 + r) * d + k0 + j] : 0.f);
            *reinterpret_cast<uint4 *>(sA + kmaj_off(r, k0, K1)) = *reinterpret_cast<const uint4 *>(e);
        }
        fence_async_smem();
        tc_fence_before();
        group_sync(g);
        tc_fence_after();
        float logit = 0.f;
        for (int l = 0; l < 3; ++l) {
            if (m == 0)
                tc_layer(tg, 0, sA, l == 0 ? sW1 : l == 1 ? sW2 : sW3, l == 0 ? K1 : W, W, bar);
            ok = group_all(g, ftp::mbar_wait_bounded(bar, phase));
            phase ^= 1u;
            if (!ok)
                break;
            tc_fence_after();
            // 32 columns at a time: ReLU and BF16, layers 1-2 back to shared memory as the
            // next A, layer 3 into the last layer's dot product; then the next product's bias
            // into the columns just read (layer l + 1's, or layer 1's of the next tile)
            const float *nb = sb + (l == 2 ? 0 : l + 1) * W;
#pragma unroll
            for (int c0 = 0; c0 < W; c0 += 32) {
                constexpr int kC = W < 32 ? W : 32;
                unsigned raw[kC];
#pragma unroll
                for (int c = 0; c < kC; c += 8)
                    tc_ld8(trow + static_cast<unsigned>(c0 + c), raw + c);
                tc_wait_ld();
#pragma unroll
                for (int c = 0; c < kC && c0 + c < W; c += 8) {
                    uint4 e;
                    e.x = relu_bf16x2(__uint_as_float(raw[c]), __uint_as_float(raw[c + 1]));
                    e.y = relu_bf16x2(__uint_as_float(raw[c + 2]), __uint_as_float(raw[c + 3]));
                    e.z = relu_bf16x2(__uint_as_float(raw[c + 4]), __uint_as_float(raw[c + 5]));
                    e.w = relu_bf16x2(__uint_as_float(raw[c + 6]), __uint_as_float(raw[c + 7]));
                    if (l < 2) {
                        *reinterpret_cast<uint4 *>(sA + kmaj_off(m, c0 + c, W)) = e;
                    } else {
                        const float *w4 = sb + 3 * W + c0 + c;
                        const unsigned u[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            logit = __fmaf_rn(w4[2 * i], __uint_as_float(u[i] << 16), logit);
                            logit = __fmaf_rn(w4[2 * i + 1], __uint_as_float(u[i] & 0xffff0000u), logit);
                        }
                    }
                    tc_st8(trow + static_cast<unsigned>(c0 + c), nb + c0 + c);
                }
            }
            tc_wait_st();
            fence_async_smem();
            tc_fence_before();
            group_sync(g);
            tc_fence_after();
        }
        if (ok && m < rows)
            p[s0 + m] = 1.f / (1.f + expf(-(logit + sb[4 * W])));
    }
    if (!ok && m == 0) {
        atomicOr(status, FT_STATUS_TIMEOUT);
        // a product still in flight finishes (bounded) before its tensor memory is freed
        (void)ftp::mbar_wait_bounded(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tm), "r"(ncols) : "memory");
    }
}

// the tensor-core inference for hidden width W (a multiple of 16, at most kTcMaxW)
template <int W>
cudaError_t tc_launch(const float *X, long long n, int d, int K1, const __nv_bfloat16 *th, const Layout &L,
                      float *p, unsigned *status, int sms, size_t smem_optin, cudaStream_t st)
{
    const size_t smem = tc_layout(K1, W).total;
    if (smem > smem_optin)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_infer_tc<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    const long long grid =
        std::min<long long>(((n + kTcM - 1) / kTcM + kTcGroups - 1) / kTcGroups, std::max(sms, 1));
    k_infer_tc<W><<<static_cast<unsigned>(grid), kTcThreads, smem, st>>>(X, n, d, K1, th, L.W1, L.b1,
                                                                          L.W2, L.b2, L.W3, L.b3, L.W4, L.b4, p,
                                                                          status);
    return cudaGetLastError();
}

cudaError_t tc_dispatch(int W, const float *X, long long n, int d, int K1, const __nv_bfloat16 *th,
                        const Layout &L, float *p, unsigned *status, int sms, size_t smem_optin,
                        cudaStream_t st)
{
    switch (W) {
    case 16: return tc_launch<16>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 32: return tc_launch<32>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 48: return tc_launch<48>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 64: return tc_launch<64>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 80: return tc_launch<80>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 96: return tc_launch<96>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 112: return tc_launch<112>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    case 128: return tc_launch<128>(X, n, d, K1, th, L, p, status, sms, smem_optin, st);
    default: return cudaErrorInvalidValue;
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
    if (cudaMalloc(&m->d_theta, L.n * 4) != cudaSuccess || cudaMalloc(&m->d_grad, L.n * 4) != cudaSuccess ||
        cudaMalloc(&m->d_m, L.n * 4) != cudaSuccess || cudaMalloc(&m->d_v, L.n * 4) != cudaSuccess ||
        cudaMalloc(&m->d_theta_bf16, L.n * 2) != cudaSuccess || cudaMalloc(&m->d_loss, 4) != cudaSuccess) {
        ft_mlp_destroy(m);
        FT_FAIL(FT_ERR_OOM, "mlp_create: allocation failed");
    }
    if (cudaMemcpy(m->d_theta, th.data(), L.n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->d_grad, 0, L.n * 4) != cudaSuccess || cudaMemset(m->d_m, 0, L.n * 4) != cudaSuccess ||
        cudaMemset(m->d_v, 0, L.n * 4) != cudaSuccess) {
        ft_mlp_destroy(m);
        FT_FAIL(FT_ERR_CUDA, "mlp_create: initialisation failed");
    }
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
    if (cudaMalloc(&dX, n * m->d_in * 4) != cudaSuccess || cudaMalloc(&dy, n * 4) != cudaSuccess) {
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
        const int W = m->width, K1 = (m->d_in + 15) / 16 * 16;
        const bool tc = bf16 != 2 && W % 16 == 0 && W <= kTcMaxW && K1 <= kTcMaxK;
        if (tc) {
            // tensor cores: 128 samples per CTA
            if (tc_dispatch(W, dX, n, m->d_in, K1, m->d_theta_bf16, L, dp, m->ctx->d_status, m->ctx->sm_count,
                            m->ctx->smem_optin, st) != cudaSuccess)
                rc = FT_ERR_CUDA;
        } else {
            // CUDA cores: one warp per sample
            const int warps = 8;
            k_infer_bf16<<<static_cast<unsigned>((n + warps - 1) / warps), 32 * warps,
                           warps * 2 * m->width * sizeof(__nv_bfloat16), st>>>(
                dX, n, m->d_in, m->width, m->d_theta_bf16, L.W1, L.b1, L.W2, L.b2, L.W3, L.b3, L.W4, L.b4, dp);
        }
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
