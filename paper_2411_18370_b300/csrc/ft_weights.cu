// ft_weights.cu -- the kernels behind the all-sky weights and the number count (Sec. II.B,
// Eq. (number_count)): the per-SFT FP32 records of D / sqrt(S_n) the evaluation kernels form
// their weights from, each sky point's normalisation and noise moments, and the binarised
// spectrogram of the number count.
#include "ft_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cmath>

// ------------------------------------------------------------------ all-sky weight norms

namespace {

__global__ void k_rowd(const double *D, const double *sn, long long N, long long n_pad, float4 *out)
{
    const long long a = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (a >= n_pad)
        return;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (a < N) {
        const double g = 1.0 / sqrt(sn[a]);
        const double *d = D + 6 * a;
        const double e0 = d[0] * g, e1 = d[1] * g, e2 = d[2] * g, e3 = d[3] * g, e4 = d[4] * g, e5 = d[5] * g;
        const double dd = e0 * e0 + e3 * e3 + e5 * e5 + 2.0 * (e1 * e1 + e2 * e2 + e4 * e4);
        r0 = make_float4(static_cast<float>(e0), static_cast<float>(e1), static_cast<float>(e2), static_cast<float>(e3));
        r1 = make_float4(static_cast<float>(e4), static_cast<float>(e5), static_cast<float>(dd),
                         static_cast<float>(e0 + e3 + e5));
    }
    out[2 * a] = r0;
    out[2 * a + 1] = r1;
}

constexpr int kNormThreads = 256;

__global__ void __launch_bounds__(kNormThreads)
    k_sky_norms(long long N, const float4 *rowd, const double *sky, double m1, double sd1, double *inv,
                double *mu, double *sig)
{
    __shared__ double s1[kNormThreads], s2[kNormThreads];
    const double *n = sky + 3 * blockIdx.x;
    const float n0 = static_cast<float>(n[0]), n1 = static_cast<float>(n[1]), n2 = static_cast<float>(n[2]);
    double a1 = 0.0, a2 = 0.0;
    for (long long a = threadIdx.x; a < N; a += kNormThreads) {
        // the same FP32 value of (a^2 + b^2) / S_n as the evaluation kernels' weights, so
        // that the weights of a sky point sum to 1 up to the FP32 rounding of the product
        const double r = ft_sky_r32(rowd[2 * a], rowd[2 * a + 1], n0, n1, n2);
        a1 += r;
        a2 += r * r;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int off = kNormThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s1[threadIdx.x] += s1[threadIdx.x + off];
            s2[threadIdx.x] += s2[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // w = r / sum r: sum w = 1, so the noise mean is m1 and the variance v1 sum w^2
        inv[blockIdx.x] = 1.0 / s1[0];
        mu[blockIdx.x] = m1;
        sig[blockIdx.x] = sd1 * sqrt(s2[0]) / s1[0];
    }
}

}  // namespace

int ft_launch_rowd(const double *D, const double *sn, long long N, long long n_pad, float4 *out,
                   cudaStream_t st)
{
    if (n_pad <= 0)
        return FT_OK;
    k_rowd<<<static_cast<unsigned>((n_pad + 255) / 256), 256, 0, st>>>(D, sn, N, n_pad, out);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int ft_launch_sky_norms(const ft_band *band, const ft_bank *bank, cudaStream_t st)
{
    if (bank->n_sky > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "sky weights: too many sky points");
    if (!band->d_rowd)
        FT_FAIL(FT_ERR_ARG, "sky weights: the band has no weight records");
    k_sky_norms<<<static_cast<unsigned>(bank->n_sky), kNormThreads, 0, st>>>(
        static_cast<long long>(band->N), band->d_rowd, bank->d_sky, band->m1, std::sqrt(band->v1),
        bank->d_sky_inv, bank->d_sky_mu, bank->d_sky_sig);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

// ------------------------------------------------------------------ number count
//
// The binarised spectrogram of Eq. (number_count): every stored element (both copies of a
// 16-bit pair row, and the zero padding, which stays 0 for a threshold >= 0) becomes 1 when
// its value exceeds the threshold.  Grid-stride over 16-byte vectors.

namespace {

template <typename T>
__device__ __forceinline__ T bin_of(T x, double thr);
template <>
__device__ __forceinline__ float bin_of<float>(float x, double thr)
{
    return static_cast<double>(x) > thr ? 1.f : 0.f;
}
template <>
__device__ __forceinline__ __half bin_of<__half>(__half x, double thr)
{
    return __ushort_as_half(static_cast<double>(__half2float(x)) > thr ? 0x3C00 : 0);
}
template <>
__device__ __forceinline__ __nv_bfloat16 bin_of<__nv_bfloat16>(__nv_bfloat16 x, double thr)
{
    return __ushort_as_bfloat16(static_cast<double>(__bfloat162float(x)) > thr ? 0x3F80 : 0);
}

template <typename T>
__global__ void k_binarize(const uint4 *src, uint4 *dst, long long n_vec, double thr)
{
    constexpr int E = 16 / sizeof(T);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n_vec;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        uint4 u = src[i];
        T *e = reinterpret_cast<T *>(&u);
#pragma unroll
        for (int q = 0; q < E; ++q)
            e[q] = bin_of<T>(e[q], thr);
        dst[i] = u;
    }
}

}  // namespace

int ft_launch_binarize(const ft_band *src, ft_band *dst, double threshold, cudaStream_t st)
{
    const long long bytes = static_cast<long long>(src->N) * src->Wp * 4;
    const long long n_vec = bytes / 16;  // Wp is a multiple of 32 elements: rows are whole vectors
    const int threads = 256;
    const long long want = (n_vec + threads - 1) / threads;
    const unsigned grid = static_cast<unsigned>(std::max(1ll, std::min(want, 148ll * 8)));
    const uint4 *s = static_cast<const uint4 *>(src->d_power);
    uint4 *d = static_cast<uint4 *>(dst->d_power);
    switch (src->dtype) {
    case FT_F32: k_binarize<float><<<grid, threads, 0, st>>>(s, d, n_vec, threshold); break;
    case FT_F16: k_binarize<__half><<<grid, threads, 0, st>>>(s, d, n_vec, threshold); break;
    case FT_BF16: k_binarize<__nv_bfloat16><<<grid, threads, 0, st>>>(s, d, n_vec, threshold); break;
    default: FT_FAIL(FT_ERR_ARG, "number count: unknown storage type");
    }
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
