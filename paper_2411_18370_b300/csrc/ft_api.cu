// ft_api.cu -- host side of the fasttracks C ABI (include/fasttracks.h).
#include "ft_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <limits>
#include <type_traits>

namespace {

thread_local std::string g_err;

cudaStream_t as_stream(void *s)
{
    return static_cast<cudaStream_t>(s);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
        // errors of earlier, unrelated runtime calls on this thread are not ours to report
        (void)cudaGetLastError();
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

int read_status(ft_ctx *ctx, cudaStream_t st)
{
    unsigned int h = 0;
    FT_CUDA(cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, st));
    FT_CUDA(cudaStreamSynchronize(st));
    if (h != 0) {
        FT_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), st));
        FT_CUDA(cudaStreamSynchronize(st));
        if (h & FT_STATUS_TIMEOUT)
            FT_FAIL(FT_ERR_TIMEOUT, "a device-side bounded wait ran out (kernel abandoned its tile)");
        if (h & FT_STATUS_NONFINITE)
            FT_FAIL(FT_ERR_ARG, "non-finite value in the SFT power");
        if (h & FT_STATUS_WINDOW)
            FT_FAIL(FT_ERR_RANGE, "a track window exceeded its shared-memory bound");
        FT_FAIL(FT_ERR_CUDA, "unknown device status");
    }
    return FT_OK;
}

int grow(void **p, size_t *have, size_t need)
{
    if (need <= *have)
        return FT_OK;
    if (*p)
        FT_CUDA(cudaFree(*p));
    *p = nullptr;
    *have = 0;
    size_t sz = std::max(need, static_cast<size_t>(1) << 20);
    FT_CUDA(cudaMalloc(p, sz));
    *have = sz;
    return FT_OK;
}

template <typename T>
int dev_upload(T **dst, const T *src, size_t n, cudaStream_t st)
{
    FT_CUDA(cudaMalloc(reinterpret_cast<void **>(dst), std::max<size_t>(n, 1) * sizeof(T)));
    if (n)
        FT_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
    return FT_OK;
}

bool finite_all(const double *p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i]))
            return false;
    return true;
}

// Conservative global-bin extent of every track of a bank over a band's SFTs, using
// |v.n| <= |v| (Eq. (track), a_p = 0, plus f1).  Returns FT_OK and kmin/kmax.
int track_extent(int64_t k0, int n_f0, const double *f1, int n_f1, const std::vector<double> &tau,
                 const std::vector<double> &vabs, int64_t *kmin, int64_t *kmax)
{
    double f1lo = f1[0], f1hi = f1[0];
    for (int i = 1; i < n_f1; ++i) {
        f1lo = std::min(f1lo, f1[i]);
        f1hi = std::max(f1hi, f1[i]);
    }
    double xmin = std::numeric_limits<double>::infinity(), xmax = -xmin;
    for (size_t a = 0; a < tau.size(); ++a) {
        const double d1 = f1lo * tau[a], d2 = f1hi * tau[a];
        if (std::fabs(d1) >= 1048576.0 || std::fabs(d2) >= 1048576.0)
            FT_FAIL(FT_ERR_RANGE, "|f1 (t - t0) T_SFT| must stay below 2^20 bins");
        const double lo_f = static_cast<double>(k0) + std::min(d1, d2);
        const double hi_f = static_cast<double>(k0) + (n_f0 - 1) + std::max(d1, d2);
        if (lo_f <= 0.0)
            FT_FAIL(FT_ERR_ARG, "track frequency must stay positive");
        xmin = std::min(xmin, lo_f * (1.0 - vabs[a]));
        xmax = std::max(xmax, hi_f * (1.0 + vabs[a]));
    }
    *kmin = static_cast<int64_t>(std::floor(xmin + 0.5)) - 1;
    *kmax = static_cast<int64_t>(std::floor(xmax + 0.5)) + 1;
    return FT_OK;
}

int check_bank_desc(const ft_bank_desc *d)
{
    if (!d || !d->f1 || !d->sky)
        FT_FAIL(FT_ERR_ARG, "bank: null descriptor or array");
    if (d->n_f0 < 1 || d->n_f0 > (1 << 24))
        FT_FAIL(FT_ERR_RANGE, "bank: n_f0 must be in [1, 2^24]");
    if (d->n_f1 < 1 || d->n_f1 > 65535)
        FT_FAIL(FT_ERR_RANGE, "bank: n_f1 must be in [1, 65535]");
    if (d->n_sky < 1)
        FT_FAIL(FT_ERR_ARG, "bank: n_sky must be >= 1");
    if (d->subband_bins < 1)
        FT_FAIL(FT_ERR_ARG, "bank: subband_bins must be >= 1");
    if (!finite_all(d->f1, d->n_f1) || !finite_all(d->sky, 3 * static_cast<size_t>(d->n_sky)))
        FT_FAIL(FT_ERR_ARG, "bank: non-finite f1 or sky value");
    for (int64_t i = 0; i < d->n_sky; ++i) {
        const double *n = d->sky + 3 * i;
        const double r2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        if (std::fabs(r2 - 1.0) > 1e-9)
            FT_FAIL(FT_ERR_ARG, "bank: sky vectors must be unit vectors");
    }
    return FT_OK;
}

}  // namespace

void ft_set_error(const std::string &msg)
{
    g_err = msg;
}

int ft_ctx_scratch(ft_ctx *ctx, size_t bytes, void **p)
{
    FT_TRY(grow(&ctx->scratch, &ctx->scratch_bytes, bytes));
    *p = ctx->scratch;
    return FT_OK;
}

int ft_ctx_outbuf(ft_ctx *ctx, size_t bytes, void **p)
{
    FT_TRY(grow(&ctx->outbuf, &ctx->outbuf_bytes, bytes));
    *p = ctx->outbuf;
    return FT_OK;
}

int ft_read_status(ft_ctx *ctx, cudaStream_t st)
{
    return read_status(ctx, st);
}

extern "C" {

const char *ft_last_error(void)
{
    return g_err.c_str();
}

int ft_abi_version(void)
{
    return FT_ABI_VERSION;
}

int ft_create(ft_ctx **out, int device)
{
    if (!out)
        FT_FAIL(FT_ERR_ARG, "ft_create: null out");
    *out = nullptr;
    int n = 0;
    FT_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n)
        FT_FAIL(FT_ERR_ARG, "ft_create: no such device");
    cudaDeviceProp prop;
    FT_CUDA(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3))
        FT_FAIL(FT_ERR_UNSUPPORTED, "ft_create: kernels are built for sm_103a (B300); device is sm_" +
                                        std::to_string(prop.major) + std::to_string(prop.minor));
    DeviceGuard g(device);
    ft_ctx *c = new ft_ctx;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMalloc(&c->d_status, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(unsigned int)) != cudaSuccess) {
        delete c;
        FT_FAIL(FT_ERR_OOM, "ft_create: status word allocation failed");
    }
    *out = c;
    return FT_OK;
}

void ft_destroy(ft_ctx *ctx)
{
    if (!ctx)
        return;
    DeviceGuard g(ctx->device);
    cudaFree(ctx->d_status);
    cudaFree(ctx->scratch);
    cudaFree(ctx->outbuf);
    delete ctx;
}

int ft_set_tune(ft_ctx *ctx, const ft_tune *tune)
{
    if (!ctx)
        FT_FAIL(FT_ERR_ARG, "set_tune: null ctx");
    if (!tune) {
        ctx->tune = ft_tune{0, 0, 0};
        return FT_OK;
    }
    if (tune->rows_per_stage < 0 || tune->rows_per_stage > 64 || tune->stages < 0 ||
        tune->stages > 4 || tune->tile_f0 < 0 || tune->tile_f0 > 256)
        FT_FAIL(FT_ERR_RANGE, "set_tune: field out of range");
    ctx->tune = *tune;
    return FT_OK;
}

int ft_gather_roof(ft_ctx *ctx, int dtype, double *evals_per_s, double *evals_per_clk_sm)
{
    if (!ctx || !evals_per_s || !evals_per_clk_sm)
        FT_FAIL(FT_ERR_ARG, "gather_roof: null argument");
    DeviceGuard g(ctx->device);
    return ft_run_gather_roof(dtype, ctx->sm_count, evals_per_s, evals_per_clk_sm);
}

int ft_ctx_memory(const ft_ctx *ctx, size_t *scratch_bytes, size_t *staging_bytes)
{
    if (!ctx)
        FT_FAIL(FT_ERR_ARG, "ft_ctx_memory: null ctx");
    if (scratch_bytes)
        *scratch_bytes = ctx->scratch_bytes;
    if (staging_bytes)
        *staging_bytes = ctx->outbuf_bytes;
    return FT_OK;
}

int ft_check_status(ft_ctx *ctx, void *stream)
{
    if (!ctx)
        FT_FAIL(FT_ERR_ARG, "ft_check_status: null ctx");
    DeviceGuard g(ctx->device);
    return read_status(ctx, as_stream(stream));
}

int ft_load_sfts(ft_ctx *ctx, const ft_band_desc *d, const void *power, int power_dtype,
                 int64_t row_stride, int power_on_device, const double *t_mid,
                 const double *v_over_c, const float *w, const double *s_n, void *stream,
                 ft_band **out)
{
    if (!ctx || !d || !power || !t_mid || !v_over_c || !out || !d->n_sft)
        FT_FAIL(FT_ERR_ARG, "load_sfts: null argument");
    *out = nullptr;
    if (d->n_det < 1)
        FT_FAIL(FT_ERR_ARG, "load_sfts: n_det must be >= 1");
    if (d->dtype != FT_F32 && d->dtype != FT_F16 && d->dtype != FT_BF16)
        FT_FAIL(FT_ERR_ARG, "load_sfts: storage dtype must be FT_F32, FT_F16 or FT_BF16");
    if (power_dtype != FT_F32 && power_dtype != FT_F64)
        FT_FAIL(FT_ERR_ARG, "load_sfts: input power must be FT_F32 or FT_F64");
    if (d->n_bins < 1 || d->n_bins > (1 << 20))
        FT_FAIL(FT_ERR_RANGE, "load_sfts: n_bins must be in [1, 2^20]");
    if (row_stride < d->n_bins)
        FT_FAIL(FT_ERR_ARG, "load_sfts: row_stride < n_bins");
    if (!(d->t_sft > 0) || !std::isfinite(d->t_sft) || !std::isfinite(d->t0))
        FT_FAIL(FT_ERR_ARG, "load_sfts: bad t_sft / t0");
    int64_t N = 0;
    for (int x = 0; x < d->n_det; ++x) {
        if (d->n_sft[x] < 0)
            FT_FAIL(FT_ERR_ARG, "load_sfts: negative SFT count");
        N += d->n_sft[x];
    }
    if (N < 1)
        FT_FAIL(FT_ERR_ARG, "load_sfts: no SFTs");
    if (N > INT32_MAX)
        FT_FAIL(FT_ERR_RANGE, "load_sfts: too many SFT rows");
    if (!finite_all(t_mid, N) || !finite_all(v_over_c, 3 * N))
        FT_FAIL(FT_ERR_ARG, "load_sfts: non-finite t_mid or velocity");
    if (s_n && !finite_all(s_n, N))
        FT_FAIL(FT_ERR_ARG, "load_sfts: non-finite S_n");
    for (int64_t a = 0; s_n && a < N; ++a)
        if (!(s_n[a] > 0.0))
            FT_FAIL(FT_ERR_ARG, "load_sfts: S_n must be > 0");
    std::vector<float> wv(N, 1.0f);
    bool weighted = false;
    if (w) {
        for (int64_t a = 0; a < N; ++a) {
            if (!std::isfinite(w[a]) || w[a] < 0)
                FT_FAIL(FT_ERR_ARG, "load_sfts: weights must be finite and >= 0");
            wv[a] = w[a];
            weighted = weighted || w[a] != 1.0f;
        }
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    ft_band *b = new ft_band;
    b->ctx = ctx;
    b->device = ctx->device;
    b->n_det = d->n_det;
    b->n_sft.assign(d->n_sft, d->n_sft + d->n_det);
    b->N = N;
    b->W = d->n_bins;
    b->Wp = d->dtype == FT_F32 ? (d->n_bins + 31) / 32 * 32 : (d->n_bins + 63) / 64 * 64;
    b->k_lo = d->k_lo;
    b->t_sft = d->t_sft;
    b->t0 = d->t0;
    b->dtype = d->dtype;
    b->weighted = weighted;
    b->h_tau.resize(N);
    b->h_vabs.resize(N);
    b->h_dt.resize(N);
    double sw = 0, sw2 = 0;
    for (int64_t a = 0; a < N; ++a) {
        b->h_dt[a] = t_mid[a] - d->t0;
        b->h_tau[a] = (t_mid[a] - d->t0) * d->t_sft;
        const double *v = v_over_c + 3 * a;
        b->h_vabs[a] = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        sw += wv[a];
        sw2 += static_cast<double>(wv[a]) * wv[a];
        b->tau_absmax = std::max(b->tau_absmax, std::fabs(b->h_tau[a]));
        b->vmax = std::max(b->vmax, b->h_vabs[a]);
    }
    b->mu = 2.0 * sw;
    b->sigma = std::sqrt(4.0 * sw2);
    for (int64_t a = 0; a < N; ++a) {
        if (b->h_vabs[a] >= 1e-3) {
            delete b;
            FT_FAIL(FT_ERR_RANGE, "load_sfts: |v/c| must be < 1e-3");
        }
    }
    if (!(b->sigma > 0)) {
        delete b;
        FT_FAIL(FT_ERR_ARG, "load_sfts: all weights are zero");
    }
    auto fail = [&](int rc) {
        ft_band_destroy(b);
        return rc;
    };
    if (cudaMalloc(&b->d_power, static_cast<size_t>(N) * b->Wp * 4) != cudaSuccess) {
        b->d_power = nullptr;
        ft_set_error("load_sfts: power allocation failed");
        return fail(FT_ERR_OOM);
    }
    int rc;
    if ((rc = dev_upload(&b->d_tau, b->h_tau.data(), N, st)) != FT_OK ||
        (rc = dev_upload(&b->d_v, v_over_c, 3 * N, st)) != FT_OK ||
        (rc = dev_upload(&b->d_w, wv.data(), N, st)) != FT_OK)
        return fail(rc);
    if (s_n && (rc = dev_upload(&b->d_sn, s_n, N, st)) != FT_OK)
        return fail(rc);
    const void *src = power;
    if (!power_on_device) {
        const size_t sbytes = static_cast<size_t>(N) * row_stride * (power_dtype == FT_F64 ? 8 : 4);
        void *stage = nullptr;
        if ((rc = ft_ctx_outbuf(ctx, sbytes, &stage)) != FT_OK)
            return fail(rc);
        if (cudaMemcpyAsync(stage, power, sbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            ft_set_error("load_sfts: host-to-device copy failed");
            return fail(FT_ERR_CUDA);
        }
        src = stage;
    }
    if ((rc = ft_launch_convert(src, power_dtype, row_stride, b->d_power, d->dtype, N, b->W, b->Wp,
                                ctx->d_status, st)) != FT_OK)
        return fail(rc);
    if ((rc = read_status(ctx, st)) != FT_OK)
        return fail(rc);
    *out = b;
    return FT_OK;
}

void ft_band_destroy(ft_band *b)
{
    if (!b)
        return;
    DeviceGuard g(b->device);
    cudaFree(b->d_power);
    cudaFree(b->d_tau);
    cudaFree(b->d_v);
    cudaFree(b->d_w);
    cudaFree(b->d_sn);
    cudaFree(b->d_D);
    cudaFree(b->d_rowd);
    delete b;
}

int ft_band_set_sky_weights(ft_band *band, const double *det_tensor, void *stream)
{
    if (!band)
        FT_FAIL(FT_ERR_ARG, "band_set_sky_weights: null band");
    DeviceGuard g(band->device);
    cudaStream_t st = as_stream(stream);
    if (!det_tensor) {
        cudaFree(band->d_D);
        cudaFree(band->d_rowd);
        band->d_D = nullptr;
        band->d_rowd = nullptr;
        return FT_OK;
    }
    if (!band->d_sn)
        FT_FAIL(FT_ERR_ARG, "band_set_sky_weights: the band was loaded without S_n");
    const size_t n6 = static_cast<size_t>(band->N) * 6;
    if (!finite_all(det_tensor, n6))
        FT_FAIL(FT_ERR_ARG, "band_set_sky_weights: non-finite detector tensor");
    if (!band->d_D)
        FT_CUDA(cudaMalloc(&band->d_D, n6 * sizeof(double)));
    if (!band->d_rowd)
        FT_CUDA(cudaMalloc(&band->d_rowd, static_cast<size_t>(band->N) * 2 * sizeof(float4)));
    FT_CUDA(cudaMemcpyAsync(band->d_D, det_tensor, n6 * sizeof(double), cudaMemcpyHostToDevice, st));
    FT_TRY(ft_launch_rowd(band->d_D, band->d_sn, band->N, band->N, band->d_rowd, st));
    FT_CUDA(cudaStreamSynchronize(st));
    return FT_OK;
}

int ft_number_count_band(ft_ctx *ctx, const ft_band *band, double threshold, void *stream,
                         ft_band **out)
{
    if (!ctx || !band || !out)
        FT_FAIL(FT_ERR_ARG, "number_count_band: null argument");
    if (band->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "number_count_band: band belongs to another context");
    if (band->number_count)
        FT_FAIL(FT_ERR_ARG, "number_count_band: the band is already a number count");
    if (!(threshold >= 0.0) || !std::isfinite(threshold))
        FT_FAIL(FT_ERR_ARG, "number_count_band: threshold must be finite and >= 0");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    const size_t N = static_cast<size_t>(band->N);
    ft_band *b = new ft_band(*band);  // metadata; device buffers are replaced below
    b->d_power = nullptr;
    b->d_tau = nullptr;
    b->d_v = nullptr;
    b->d_w = nullptr;
    b->d_sn = nullptr;
    b->d_D = nullptr;
    b->d_rowd = nullptr;
    auto fail = [&](int rc) {
        ft_band_destroy(b);
        return rc;
    };
    auto dup = [&](auto **dst, const auto *src, size_t n) -> int {
        if (!src)
            return FT_OK;
        using T = std::remove_cv_t<std::remove_reference_t<decltype(*src)>>;
        if (cudaMalloc(dst, n * sizeof(T)) != cudaSuccess) {
            *dst = nullptr;
            ft_set_error("number_count_band: allocation failed");
            return FT_ERR_OOM;
        }
        if (cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            ft_set_error("number_count_band: device copy failed");
            return FT_ERR_CUDA;
        }
        return FT_OK;
    };
    int rc;
    if ((rc = dup(&b->d_tau, band->d_tau, N)) != FT_OK || (rc = dup(&b->d_v, band->d_v, 3 * N)) != FT_OK ||
        (rc = dup(&b->d_w, band->d_w, N)) != FT_OK || (rc = dup(&b->d_sn, band->d_sn, N)) != FT_OK ||
        (rc = dup(&b->d_D, band->d_D, 6 * N)) != FT_OK || (rc = dup(&b->d_rowd, band->d_rowd, 2 * N)) != FT_OK)
        return fail(rc);
    if (cudaMalloc(&b->d_power, N * band->Wp * 4) != cudaSuccess) {
        b->d_power = nullptr;
        ft_set_error("number_count_band: power allocation failed");
        return fail(FT_ERR_OOM);
    }
    if ((rc = ft_launch_binarize(band, b, threshold, st)) != FT_OK)
        return fail(rc);
    // P is exponential with mean 2 in Gaussian noise: P(P > x) = exp(-x / 2)
    const double pr = std::exp(-0.5 * threshold);
    const double sw = band->mu / band->m1, sw2 = band->sigma * band->sigma / band->v1;
    b->number_count = true;
    b->m1 = pr;
    b->v1 = pr * (1.0 - pr);
    b->mu = pr * sw;
    b->sigma = std::sqrt(b->v1 * sw2);
    if (!(b->sigma > 0)) {
        ft_set_error("number_count_band: threshold leaves no noise variance");
        return fail(FT_ERR_ARG);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        ft_set_error("number_count_band: stream failed");
        return fail(FT_ERR_CUDA);
    }
    *out = b;
    return FT_OK;
}

int ft_band_info(const ft_band *b, int64_t *n, int *n_bins, int *stride, int *dtype, double *mu,
                 double *sigma)
{
    if (!b)
        FT_FAIL(FT_ERR_ARG, "band_info: null band");
    if (n)
        *n = b->N;
    if (n_bins)
        *n_bins = b->W;
    if (stride)
        *stride = b->Wp;
    if (dtype)
        *dtype = b->dtype;
    if (mu)
        *mu = b->mu;
    if (sigma)
        *sigma = b->sigma;
    return FT_OK;
}

// Position of cell (x, y) along the Hilbert curve that fills a 2^bits x 2^bits grid: the
// curve visits the four quadrants of every square in turn (each reflected so that it starts
// next to where the last one ended), so cells close along the curve are close in the grid.
static uint64_t hilbert_position(uint32_t x, uint32_t y, int bits)
{
    uint64_t d = 0;
    for (uint32_t s = 1u << (bits - 1); s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += static_cast<uint64_t>(s) * s * ((3u * rx) ^ ry);
        // bring the quadrant into the curve's base orientation for the next level
        x &= s - 1;
        y &= s - 1;
        if (ry == 0) {
            if (rx == 1) {
                x = s - 1 - x;
                y = s - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

// Sky points ordered along a Hilbert curve over the equal-area map ((z + 1)/2, (phi + pi)/2pi)
// of the sphere, so that any run of consecutive points is a compact patch of sky: a CTA's
// group of P points, a sky box, and the few hundred groups the resident CTAs of a launch
// work on at once (whose rows' windows then overlap in L2).  dmax[P] is the largest distance
// between two points of one run g*P .. g*P + P - 1 of the order.
static void sky_proximity_order(const double *sky, int64_t n, std::vector<int> &order,
                                double dmax[kMaxSkyGroup + 1])
{
    constexpr int bits = 16;
    constexpr double kPi = 3.14159265358979323846;
    const double cells = static_cast<double>(1u << bits);
    auto cell = [&](double u) {
        return static_cast<uint32_t>(std::min(std::max(u * cells, 0.0), cells - 1.0));
    };
    std::vector<std::pair<uint64_t, int>> key(n);
    for (int64_t i = 0; i < n; ++i) {
        const double x = sky[3 * i], y = sky[3 * i + 1], z = sky[3 * i + 2];
        const double u = (z + 1.0) * 0.5, v = (std::atan2(y, x) + kPi) / (2.0 * kPi);
        key[i] = {hilbert_position(cell(u), cell(v), bits), static_cast<int>(i)};
    }
    std::sort(key.begin(), key.end());
    order.resize(n);
    for (int64_t i = 0; i < n; ++i)
        order[i] = key[i].second;
    dmax[0] = dmax[1] = 0.0;
    for (int P = 2; P <= kMaxSkyGroup; ++P) {
        double m = 0.0;
        for (int64_t g0 = 0; g0 < n; g0 += P)
            for (int64_t a = g0; a < std::min<int64_t>(g0 + P, n); ++a)
                for (int64_t b = a + 1; b < std::min<int64_t>(g0 + P, n); ++b) {
                    const double *u = sky + 3 * static_cast<int64_t>(order[a]);
                    const double *w = sky + 3 * static_cast<int64_t>(order[b]);
                    const double dx = u[0] - w[0], dy = u[1] - w[1], dz = u[2] - w[2];
                    m = std::max(m, std::sqrt(dx * dx + dy * dy + dz * dz));
                }
        dmax[P] = m;
    }
}

int ft_make_bank(ft_ctx *ctx, const ft_band *band, const ft_bank_desc *d, void *stream,
                 ft_bank **out)
{
    if (!ctx || !band || !out)
        FT_FAIL(FT_ERR_ARG, "make_bank: null argument");
    *out = nullptr;
    if (band->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "make_bank: band belongs to another context");
    FT_TRY(check_bank_desc(d));
    int64_t kmin, kmax;
    FT_TRY(track_extent(d->k0, d->n_f0, d->f1, d->n_f1, band->h_tau, band->h_vabs, &kmin, &kmax));
    const long long gsz = static_cast<long long>(band->N) * d->n_f1;
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    ft_bank *b = new ft_bank;
    b->ctx = ctx;
    b->device = ctx->device;
    b->band = band;
    b->k0 = d->k0;
    b->n_f0 = d->n_f0;
    b->n_f1 = d->n_f1;
    b->n_sky = d->n_sky;
    b->sub = d->subband_bins;
    b->n_sub = (d->n_f0 + d->subband_bins - 1) / d->subband_bins;
    b->window_safe = kmin >= band->k_lo && kmax <= band->k_lo + band->W - 1;
    b->f1_lo = *std::min_element(d->f1, d->f1 + d->n_f1);
    b->f1_hi = *std::max_element(d->f1, d->f1 + d->n_f1);
    std::vector<int> order;
    sky_proximity_order(d->sky, d->n_sky, order, b->sky_dmax);
    int rc;
    if ((rc = dev_upload(&b->d_f1, d->f1, d->n_f1, st)) != FT_OK ||
        (rc = dev_upload(&b->d_sky, d->sky, 3 * static_cast<size_t>(d->n_sky), st)) != FT_OK ||
        (rc = dev_upload(&b->d_sky_order, order.data(), order.size(), st)) != FT_OK) {
        ft_bank_destroy(b);
        return rc;
    }
    if (cudaMalloc(&b->d_G, gsz * sizeof(long long)) != cudaSuccess) {
        b->d_G = nullptr;
        ft_bank_destroy(b);
        FT_FAIL(FT_ERR_OOM, "make_bank: track table allocation failed");
    }
    if ((rc = ft_launch_gtable(b->d_f1, b->n_f1, band->d_tau, band->N, b->d_G, st)) != FT_OK) {
        ft_bank_destroy(b);
        return rc;
    }
    if (band->d_D) {
        // all-sky weights: per sky point the normalisation and mu_G, sigma_G
        const size_t ns = static_cast<size_t>(b->n_sky) * sizeof(double);
        if (cudaMalloc(&b->d_sky_inv, ns) != cudaSuccess || cudaMalloc(&b->d_sky_mu, ns) != cudaSuccess ||
            cudaMalloc(&b->d_sky_sig, ns) != cudaSuccess) {
            ft_bank_destroy(b);
            FT_FAIL(FT_ERR_OOM, "make_bank: sky-weight table allocation failed");
        }
        if ((rc = ft_launch_sky_norms(band, b, st)) != FT_OK) {
            ft_bank_destroy(b);
            return rc;
        }
    }
    *out = b;
    return FT_OK;
}

void ft_bank_destroy(ft_bank *b)
{
    if (!b)
        return;
    DeviceGuard g(b->device);
    cudaFree(b->d_f1);
    cudaFree(b->d_sky);
    cudaFree(b->d_sky_order);
    cudaFree(b->d_sky_inv);
    cudaFree(b->d_sky_mu);
    cudaFree(b->d_sky_sig);
    cudaFree(b->d_G);
    delete b;
}

int ft_bank_info(const ft_bank *b, int64_t *n_templates, int *n_sub, int *window_safe)
{
    if (!b)
        FT_FAIL(FT_ERR_ARG, "bank_info: null bank");
    if (n_templates)
        *n_templates = b->n_sky * b->n_f1 * static_cast<int64_t>(b->n_f0);
    if (n_sub)
        *n_sub = b->n_sub;
    if (window_safe)
        *window_safe = b->window_safe ? 1 : 0;
    return FT_OK;
}

int ft_required_wings(const ft_band_desc *d, const double *t_mid, const double *v_over_c,
                      const ft_bank_desc *bank, int *lo, int *hi)
{
    if (!d || !t_mid || !v_over_c || !lo || !hi || !d->n_sft)
        FT_FAIL(FT_ERR_ARG, "required_wings: null argument");
    FT_TRY(check_bank_desc(bank));
    int64_t N = 0;
    for (int x = 0; x < d->n_det; ++x)
        N += d->n_sft[x];
    if (N < 1)
        FT_FAIL(FT_ERR_ARG, "required_wings: no SFTs");
    std::vector<double> tau(N), vabs(N);
    for (int64_t a = 0; a < N; ++a) {
        tau[a] = (t_mid[a] - d->t0) * d->t_sft;
        const double *v = v_over_c + 3 * a;
        vabs[a] = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
    int64_t kmin, kmax;
    FT_TRY(track_extent(bank->k0, bank->n_f0, bank->f1, bank->n_f1, tau, vabs, &kmin, &kmax));
    *lo = static_cast<int>(std::max<int64_t>(0, bank->k0 - kmin));
    *hi = static_cast<int>(std::max<int64_t>(0, kmax - (bank->k0 + bank->n_f0 - 1)));
    return FT_OK;
}

static EvalParams base_params(const ft_band *band, const ft_bank *bank)
{
    return ft_eval_base_params(band, bank);
}

static int check_pair(ft_ctx *ctx, const ft_band *band, const ft_bank *bank)
{
    if (!ctx || !band || !bank)
        FT_FAIL(FT_ERR_ARG, "null ctx/band/bank");
    if (band->ctx != ctx || bank->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "band/bank belong to another context");
    if (bank->band != band)
        FT_FAIL(FT_ERR_ARG, "bank was made for another band");
    return FT_OK;
}

int ft_eval_statistic(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, float *s_out,
                      float *z_out, int32_t *n_oob_out, int out_on_device, void *stream)
{
    FT_TRY(check_pair(ctx, band, bank));
    if (!s_out)
        FT_FAIL(FT_ERR_ARG, "eval_statistic: s_out is required");
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    const size_t nt = static_cast<size_t>(bank->n_sky) * bank->n_f1 * bank->n_f0;
    EvalParams p = base_params(band, bank);
    const EvalShape sh = ft_default_shape(ctx, band, bank);
    float *ds = s_out, *dz = z_out;
    int *doob = reinterpret_cast<int *>(n_oob_out);
    if (!out_on_device) {
        const size_t need = nt * (4 + (z_out ? 4 : 0) + (n_oob_out ? 4 : 0));
        void *buf = nullptr;
        FT_TRY(ft_ctx_outbuf(ctx, need, &buf));
        char *c = static_cast<char *>(buf);
        ds = reinterpret_cast<float *>(c);
        c += nt * 4;
        dz = z_out ? reinterpret_cast<float *>(c) : nullptr;
        c += z_out ? nt * 4 : 0;
        doob = n_oob_out ? reinterpret_cast<int *>(c) : nullptr;
    }
    p.s_out = ds;
    p.z_out = dz;
    p.oob_out = doob;
    FT_TRY(ft_launch_eval(band, bank, sh, p, st));
    if (!out_on_device) {
        FT_CUDA(cudaMemcpyAsync(s_out, ds, nt * 4, cudaMemcpyDeviceToHost, st));
        if (z_out)
            FT_CUDA(cudaMemcpyAsync(z_out, dz, nt * 4, cudaMemcpyDeviceToHost, st));
        if (n_oob_out)
            FT_CUDA(cudaMemcpyAsync(n_oob_out, doob, nt * 4, cudaMemcpyDeviceToHost, st));
        return read_status(ctx, st);
    }
    return FT_OK;
}

static int topk_impl(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k, const float *gate,
                     float gate_min, ft_candidate *out, int out_on_device, void *stream, int sky_box = 0,
                     int f1_box = 0)
{
    FT_TRY(check_pair(ctx, band, bank));
    if (!out)
        FT_FAIL(FT_ERR_ARG, "topk_per_band: null out");
    if (k < 1 || k > 32)
        FT_FAIL(FT_ERR_RANGE, "topk_per_band: k must be in [1, 32]");
    if (sky_box < 0 || sky_box > INT_MAX / 2)
        FT_FAIL(FT_ERR_ARG, "topk_per_skybox: bad sky box size");
    if (f1_box < 0)
        FT_FAIL(FT_ERR_ARG, "topk_per_box: bad f1 box size");
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    const EvalShape sh = ft_default_shape(ctx, band, bank, sky_box, f1_box);
    const int J = sh.J;
    const long long n_cta = ft_grid_ctas(bank, sh);
    const int lsub_max = std::min(bank->n_sub, (J + bank->sub - 1) / bank->sub + 1);
    const size_t cand_bytes = static_cast<size_t>(n_cta) * lsub_max * k * sizeof(ft_candidate);
    const long long n_boxes = (sky_box > 0 ? (bank->n_sky + sky_box - 1) / sky_box : 1) *
                              (f1_box > 0 ? (bank->n_f1 + f1_box - 1) / f1_box : 1);
    const size_t out_bytes = static_cast<size_t>(n_boxes) * bank->n_sub * k * sizeof(ft_candidate);
    void *scr = nullptr;
    FT_TRY(ft_ctx_scratch(ctx, cand_bytes, &scr));
    ft_candidate *dout = out;
    if (!out_on_device) {
        void *ob = nullptr;
        FT_TRY(ft_ctx_outbuf(ctx, out_bytes, &ob));
        dout = static_cast<ft_candidate *>(ob);
    }
    EvalParams p = base_params(band, bank);
    p.gate = gate;
    p.gate_min = gate_min;
    p.cand = static_cast<FtCand *>(scr);
    p.k = k;
    p.sub = bank->sub;
    p.lsub_max = lsub_max;
    FT_TRY(ft_launch_eval(band, bank, sh, p, st));
    FT_TRY(ft_launch_merge(bank, sh, p.cand, k, lsub_max, dout, st, sky_box, f1_box));
    if (!out_on_device) {
        FT_CUDA(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, st));
        return read_status(ctx, st);
    }
    return FT_OK;
}

int ft_topk_per_skybox(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box, int k,
                       ft_candidate *out, int out_on_device, void *stream)
{
    if (sky_box < 1)
        FT_FAIL(FT_ERR_ARG, "topk_per_skybox: sky_box must be >= 1");
    return topk_impl(ctx, band, bank, k, nullptr, 0.f, out, out_on_device, stream, sky_box);
}

static int check_gate(const float *gate, float gate_min, const char *who)
{
    if (!gate)
        FT_FAIL(FT_ERR_ARG, std::string(who) + ": null gate");
    if (std::isnan(gate_min))
        FT_FAIL(FT_ERR_ARG, std::string(who) + ": gate_min is NaN");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, gate) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        FT_FAIL(FT_ERR_ARG, std::string(who) + ": gate must be device memory");
    }
    return FT_OK;
}

int ft_topk_per_box(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box, int f1_box,
                    int k, const float *gate, float gate_min, ft_candidate *out, int out_on_device,
                    void *stream)
{
    if (!bank)
        FT_FAIL(FT_ERR_ARG, "topk_per_box: null bank");
    if (sky_box < 1 || f1_box < 1)
        FT_FAIL(FT_ERR_ARG, "topk_per_box: sky_box and f1_box must be >= 1");
    if (gate)
        FT_TRY(check_gate(gate, gate_min, "topk_per_box"));
    // a box as wide as the dimension is the whole dimension (one box, the fastest shape)
    return topk_impl(ctx, band, bank, k, gate, gate_min, out, out_on_device, stream,
                     sky_box >= bank->n_sky ? 0 : sky_box, f1_box >= bank->n_f1 ? 0 : f1_box);
}

int ft_bank_sky_order(const ft_bank *bank, int32_t *order)
{
    if (!bank || !order)
        FT_FAIL(FT_ERR_ARG, "bank_sky_order: null argument");
    DeviceGuard g(bank->device);
    FT_CUDA(cudaMemcpy(order, bank->d_sky_order, static_cast<size_t>(bank->n_sky) * sizeof(int),
                       cudaMemcpyDeviceToHost));
    return FT_OK;
}

int ft_topk_per_band(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k,
                     ft_candidate *out, int out_on_device, void *stream)
{
    return topk_impl(ctx, band, bank, k, nullptr, 0.f, out, out_on_device, stream);
}

int ft_topk_per_band_gated(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k,
                           const float *gate, float gate_min, ft_candidate *out, int out_on_device,
                           void *stream)
{
    FT_TRY(check_gate(gate, gate_min, "topk_per_band_gated"));
    return topk_impl(ctx, band, bank, k, gate, gate_min, out, out_on_device, stream);
}

int ft_track_bins(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, const int64_t *templates,
                  int64_t n, int32_t *bins, int on_device, void *stream)
{
    FT_TRY(check_pair(ctx, band, bank));
    if (n < 0 || (n > 0 && (!templates || !bins)))
        FT_FAIL(FT_ERR_ARG, "track_bins: bad arguments");
    if (n == 0)
        return FT_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = as_stream(stream);
    const long long *dt = reinterpret_cast<const long long *>(templates);
    int *db = reinterpret_cast<int *>(bins);
    const size_t nb = static_cast<size_t>(n) * band->N * 4;
    if (!on_device) {
        void *buf = nullptr;
        // the int64 template indices after the bins, at an aligned offset
        const size_t off = (nb + 255) / 256 * 256;
        FT_TRY(ft_ctx_outbuf(ctx, off + n * 8, &buf));
        db = static_cast<int *>(buf);
        long long *tt = reinterpret_cast<long long *>(static_cast<char *>(buf) + off);
        FT_CUDA(cudaMemcpyAsync(tt, templates, n * 8, cudaMemcpyHostToDevice, st));
        dt = tt;
    }
    FT_TRY(ft_launch_track_bins(band, bank, dt, n, db, st));
    if (!on_device) {
        FT_CUDA(cudaMemcpyAsync(bins, db, nb, cudaMemcpyDeviceToHost, st));
        return read_status(ctx, st);
    }
    return FT_OK;
}

}  // extern "C"
