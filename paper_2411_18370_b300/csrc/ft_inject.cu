// ft_inject.cu -- injection-recovery runs (the Monte-Carlo estimate of p_det).
//
// arXiv 2411.18370, Sec. V, Eq. (sampling): p_det is the fraction of simulated signals that
// the search detects, each run giving one sample z^(i) of the detection statistic that the
// rule R(z; tau) of Sec. V.B scores.  One run here:
//   * signal (Sec. II.B.2): in SFT alpha the normalised power rho^2 = 4|h~|^2/(T S_n),
//     |h~| = 0.7737 (T/2) h0 |Q|, |Q|^2 = (F+ (1+cos^2 i)/2)^2 + (Fx cos i)^2 (polarisations
//     in quadrature), F+ = a cos2psi + b sin2psi, Fx = b cos2psi - a sin2psi, a = D:e+,
//     b = D:ex from the detector tensor D and the wave frame of n, placed in the bin
//     nearest f(t_alpha) T (FP64);
//   * data, generated in shared memory row by row and never stored: bins k_sig +- H with
//     complex unit Gaussian noise (Sec. II.B.1) plus the signal amplitude sqrt(rho^2) in
//     bin k_sig, i.e. P = -2 ln u1 off the signal and P = r^2 + rho^2 + 2 r sqrt(rho^2)
//     cos(2 pi u2) on it; u1, u2 are 24-bit uniforms from Philox4x32-10 (Salmon et al.,
//     SC'11) at counter (absolute bin, alpha, run id) and key = seed;
//   * local bank: f0 bins around the source's, every f1, the K bank sky points nearest to
//     n (chosen on the host); each template's statistic is Eq. (short_coh_general) with the
//     canonical exact track bins of the search kernels, z by Eq. (critical_ratio);
//   * output: max z over the local bank, its template, and the count of reads outside the
//     generated window (0 when H covers the bank).
#include "ft_internal.cuh"
#include "ft_ptx.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

constexpr double kTwo32 = 4294967296.0;
constexpr int kInjThreads = 256;
constexpr int kInjSlots = 16;  // local templates per thread
constexpr int kInjMaxK = 128;
constexpr int kInjMaxF1 = 64;

struct InjRun {
    double h0, cosi, psi, f0, f1, n[3];
};

// float count rounded up to a multiple of 4 (16 bytes)
__host__ __device__ constexpr int align16f(int n)
{
    return (n + 3) & ~3;
}

struct InjParams {
    long long N, k_lo, K0;
    int n_f0, n_f1, K, half_f0, H;
    double t0, t_sft, mu, sigma, noise_scale;
    const double *tau, *v, *sn, *D, *sky;
    const float *w;
    const long long *G;          // [n_f1][N]
    const InjRun *runs;          // [n_runs]
    const int *sky_idx;          // [n_runs][K] indices into the bank's sky points
    const int *sky_cidx;         // [n_runs][K] indices into the E / C tables
    const int *Etab;             // [n_used][N] E of the used sky points
    const long long *Ctab;       // [n_used][N] C of the used sky points
    const long long *ksig_rows;  // [n_runs][N] signal bin of each run and row (window centre)
    const float *amp_rows;       // [n_runs][N] signal amplitude sqrt(rho^2)
    unsigned long long seed, first_id;
    double *max_z;
    long long *argmax, *oob;
};

// The first two words of Philox4x32-10 at counter (c0..c3), key (k0, k1).
__device__ __forceinline__ void philox4x32_10(unsigned c0, unsigned c1, unsigned c2, unsigned c3,
                                              unsigned k0, unsigned k1, unsigned &o0, unsigned &o1)
{
    unsigned o[4];
    ftp::philox4x32_10(c0, c1, c2, c3, k0, k1, o);
    o0 = o[0];
    o1 = o[1];
}

__device__ __forceinline__ float uniform24(unsigned x)
{
    return static_cast<float>((x >> 8) + 1u) * (1.0f / 16777216.0f);
}

__device__ void antenna_ab(const double *D, const double *n, double &a, double &b)
{
    const double rho = sqrt(n[0] * n[0] + n[1] * n[1]);
    double X[3], Y[3];
    if (rho > 0) {
        X[0] = -n[1] / rho;
        X[1] = n[0] / rho;
        X[2] = 0.0;
    } else {
        X[0] = 1.0;
        X[1] = 0.0;
        X[2] = 0.0;
    }
    Y[0] = n[1] * X[2] - n[2] * X[1];
    Y[1] = n[2] * X[0] - n[0] * X[2];
    Y[2] = n[0] * X[1] - n[1] * X[0];
    const double M[3][3] = {{D[0], D[1], D[2]}, {D[1], D[3], D[4]}, {D[2], D[4], D[5]}};
    double sp = 0.0, sx = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            sp += M[i][j] * (X[i] * X[j] - Y[i] * Y[j]);
            sx += M[i][j] * (X[i] * Y[j] + Y[i] * X[j]);
        }
    a = sp;
    b = sx;
}

__device__ __forceinline__ void track_ec_inj(const double *v, const double *n, long long K0,
                                             long long k_lo, int &E, long long &C)
{
    const double eps = __fma_rn(v[2], n[2], __fma_rn(v[1], n[1], __dmul_rn(v[0], n[0])));
    E = static_cast<int>(__double2ll_rn(__dmul_rn(eps, kTwo32)));
    C = __double2ll_rn(
        __dmul_rn(__fma_rn(static_cast<double>(K0), eps, static_cast<double>(K0 - k_lo)), kTwo32));
}

__device__ __forceinline__ long long cross_q32_inj(long long G, int E)
{
    const int Gh = static_cast<int>(G >> 32);
    const unsigned Gl = static_cast<unsigned>(G);
    const long long lo = static_cast<long long>(static_cast<unsigned long long>(Gl) *
                                                static_cast<unsigned long long>(static_cast<long long>(E)));
    return static_cast<long long>(Gh) * E + (lo >> 32);
}

// E and C (Q32 track terms, FP64 as in the search kernels) of the used sky points in every
// row: [n_used][N].
__global__ void k_inj_ec(long long N, int n_used, const int *used, const double *v, const double *sky,
                         long long K0, long long k_lo, int *Etab, long long *Ctab)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= N * n_used)
        return;
    const long long u = i / N, a = i - u * N;
    int E;
    long long C;
    track_ec_inj(v + 3 * a, sky + 3 * used[u], K0, k_lo, E, C);
    Etab[i] = E;
    Ctab[i] = C;
}

// The signal bin and amplitude of every (run, row): [n_runs][N].
__global__ void k_inj_rows(const InjParams p, long long n_runs, long long *ksig_rows, float *amp_rows)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n_runs * p.N)
        return;
    const long long run = i / p.N, a = i - run * p.N;
    const InjRun inj = p.runs[run];
    const double *v = p.v + 3 * a;
    const double eps = __fma_rn(v[2], inj.n[2], __fma_rn(v[1], inj.n[1], __dmul_rn(v[0], inj.n[0])));
    const double x = __dsub_rn(__dmul_rn(__fma_rn(inj.f0, p.t_sft, __dmul_rn(inj.f1, p.tau[a])),
                                         __dadd_rn(1.0, eps)),
                               static_cast<double>(p.k_lo));
    ksig_rows[i] = __double2ll_rd(__dadd_rn(x, 0.5));
    double amp = 0.0;
    if (inj.h0 > 0.0) {
        double aa, bb;
        antenna_ab(p.D + 6 * a, inj.n, aa, bb);
        const double c2 = cos(2.0 * inj.psi), s2 = sin(2.0 * inj.psi);
        const double fp = aa * c2 + bb * s2, fx = bb * c2 - aa * s2;
        const double ap = 0.5 * (1.0 + inj.cosi * inj.cosi), ax = inj.cosi;
        const double q2 = fp * fp * ap * ap + fx * fx * ax * ax;
        const double h = 0.7737 * 0.5 * p.t_sft * inj.h0;
        amp = sqrt(4.0 * h * h * q2 / (p.t_sft * p.sn[a]));
    }
    amp_rows[i] = static_cast<float>(amp);
}

// One CTA per run.  Per row: E, C of the run's K sky points from the tables, the track
// origins of every (sky, f1), the generated window, then each thread's local templates.
// A template slot's (f1 row r, sky ks, f0 offset) is decoded once, before the row loop;
// the compensated sums live in shared memory between folds.
__global__ void __launch_bounds__(kInjThreads, 4) k_injections(const InjParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.K;
    double *skyv = reinterpret_cast<double *>(smem);                       // [K][3] (unused)
    long long *X0 = reinterpret_cast<long long *>(skyv + 3 * K);           // [K][n_f1]
    int *Et = reinterpret_cast<int *>(X0 + static_cast<size_t>(K) * p.n_f1);  // [K]
    long long *Ct = reinterpret_cast<long long *>(smem) +                   // [K] (8-aligned)
                    (3 * K + K * p.n_f1) + (K + 1) / 2;
    float *Pw = reinterpret_cast<float *>(Ct + K);                          // [2H + 1]
    float *s_hi = Pw + align16f(2 * p.H + 1);                               // [kInjSlots][threads]
    float *s_lo = s_hi + kInjSlots * kInjThreads;
    __shared__ double s_best_z[kInjThreads / 32];
    __shared__ long long s_best_t[kInjThreads / 32];

    const long long run = blockIdx.x;
    const InjRun inj = p.runs[run];
    const unsigned long long rid = p.first_id + static_cast<unsigned long long>(run);
    const int tid = threadIdx.x;
    const long long jc = __double2ll_rd(__dadd_rn(__dmul_rn(inj.f0, p.t_sft), 0.5)) - p.K0;
    const int j_lo = static_cast<int>(max(0ll, jc - p.half_f0));
    const int j_hi = static_cast<int>(min(static_cast<long long>(p.n_f0 - 1), jc + p.half_f0));
    const int nf0 = j_hi - j_lo + 1;
    const int nt = nf0 * p.n_f1 * K;
    // local template slot i of this thread: t = tid + i * blockDim.x -> f1 row r = t / nf0
    // (= ks n_f1 + f), sky ks, f0 offset t % nf0; packed as r | ks << 13 | offset << 20,
    // or ~0 past the local bank
    unsigned slot[kInjSlots];
    float part[kInjSlots];
    int oobc = 0;
#pragma unroll
    for (int i = 0; i < kInjSlots; ++i) {
        const int t = tid + i * kInjThreads;
        const int r = t / nf0;
        slot[i] = t < nt ? static_cast<unsigned>(r) | static_cast<unsigned>(r / p.n_f1) << 13 |
                               static_cast<unsigned>(t - r * nf0) << 20
                         : ~0u;
        part[i] = 0.f;
        s_hi[i * kInjThreads + tid] = 0.f;
        s_lo[i * kInjThreads + tid] = 0.f;
    }
    // (sky, f1) entries of this thread in the per-row origin loop, stepped without division
    const int nkf = K * p.n_f1;
    const int ks_first = tid / p.n_f1, f_first = tid - ks_first * p.n_f1;
    const int dks = kInjThreads / p.n_f1, df = kInjThreads - dks * p.n_f1;
    const int *cidx = p.sky_cidx + run * K;
    const long long *ksig_row = p.ksig_rows + run * p.N;
    const float *amp_row = p.amp_rows + run * p.N;
    const unsigned key0 = static_cast<unsigned>(p.seed), key1 = static_cast<unsigned>(p.seed >> 32);
    const int W = 2 * p.H + 1;
    int rows = 0;
    for (long long a = 0; a < p.N; ++a) {
        __syncthreads();  // previous row fully consumed
        if (tid < K) {
            const long long o = static_cast<long long>(cidx[tid]) * p.N + a;
            Et[tid] = p.Etab[o];
            Ct[tid] = p.Ctab[o];
        }
        __syncthreads();
        // track origins of (sky, f1) for this row
        for (int i = tid, ks = ks_first, f = f_first; i < nkf; i += kInjThreads) {
            const long long G = p.G[static_cast<long long>(f) * p.N + a];
            const int E = Et[ks];
            X0[i] = Ct[ks] + G + cross_q32_inj(G, E) + (1ll << 31);
            ks += dks;
            f += df;
            if (f >= p.n_f1) {
                f -= p.n_f1;
                ++ks;
            }
        }
        // the generated window of this row
        const long long ksig = ksig_row[a];
        const float amp = amp_row[a];
        for (int q = tid; q < W; q += blockDim.x) {
            const long long kabs = ksig + (q - p.H) + p.k_lo;
            unsigned o0, o1;
            philox4x32_10(static_cast<unsigned>(kabs), static_cast<unsigned>(a),
                          static_cast<unsigned>(rid), static_cast<unsigned>(rid >> 32), key0, key1, o0, o1);
            const float r2 = -2.0f * logf(uniform24(o0));
            float P;
            if (q == p.H && amp > 0.f) {
                const float r = static_cast<float>(p.noise_scale) * sqrtf(r2);
                P = r * r + amp * amp + 2.0f * amp * r * cospif(2.0f * uniform24(o1));
            } else {
                const float s = static_cast<float>(p.noise_scale);
                P = s * s * r2;
            }
            Pw[q] = P;
        }
        __syncthreads();
        const float wa = p.w[a];
#pragma unroll
        for (int i = 0; i < kInjSlots; ++i) {
            const unsigned sl = slot[i];
            if (sl != ~0u) {
                const int r = static_cast<int>(sl & 0x1FFFu);
                const int jj = j_lo + static_cast<int>(sl >> 20);
                const long long acc = X0[r] + static_cast<long long>(jj) * Et[(sl >> 13) & 0x7Fu];
                const long long k = jj + (acc >> 32);
                const long long q = k - ksig + p.H;
                if (q >= 0 && q < W)
                    part[i] = __fmaf_rn(wa, Pw[q], part[i]);
                else
                    ++oobc;
            }
        }
        if (++rows == 128 || a == p.N - 1) {
#pragma unroll
            for (int i = 0; i < kInjSlots; ++i) {
                float &hi = s_hi[i * kInjThreads + tid];
                float &lo = s_lo[i * kInjThreads + tid];
                const float s = __fadd_rn(hi, part[i]);
                const float bp = __fsub_rn(s, hi);
                const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(part[i], bp));
                lo = __fadd_rn(lo, e);
                hi = s;
                part[i] = 0.f;
            }
            rows = 0;
        }
    }
    // arg-max of z over the local bank: (z desc, global template index asc)
    double bz = -INFINITY;
    long long bt = LLONG_MAX;
#pragma unroll
    for (int i = 0; i < kInjSlots; ++i) {
        const unsigned sl = slot[i];
        if (sl != ~0u) {
            const int jj = j_lo + static_cast<int>(sl >> 20);
            const int r = static_cast<int>(sl & 0x1FFFu);
            const int ks = static_cast<int>((sl >> 13) & 0x7Fu), f = r - ks * p.n_f1;
            const long long tg =
                (static_cast<long long>(p.sky_idx[run * K + ks]) * p.n_f1 + f) * p.n_f0 + jj;
            const double z = (static_cast<double>(s_hi[i * kInjThreads + tid]) +
                              static_cast<double>(s_lo[i * kInjThreads + tid]) - p.mu) /
                             p.sigma;
            if (z > bz || (z == bz && tg < bt)) {
                bz = z;
                bt = tg;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double oz = __shfl_xor_sync(0xffffffffu, bz, off);
        const long long ot = __shfl_xor_sync(0xffffffffu, bt, off);
        if (oz > bz || (oz == bz && ot < bt)) {
            bz = oz;
            bt = ot;
        }
    }
    int oobw = oobc;
    for (int off = 16; off > 0; off >>= 1)
        oobw += __shfl_xor_sync(0xffffffffu, oobw, off);
    __shared__ long long s_oob;
    if (tid == 0)
        s_oob = 0;
    __syncthreads();
    if ((tid & 31) == 0) {
        s_best_z[tid >> 5] = bz;
        s_best_t[tid >> 5] = bt;
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_oob), static_cast<unsigned long long>(oobw));
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kInjThreads / 32; ++w)
            if (s_best_z[w] > bz || (s_best_z[w] == bz && s_best_t[w] < bt)) {
                bz = s_best_z[w];
                bt = s_best_t[w];
            }
        p.max_z[run] = bz;
        p.argmax[run] = bt;
        p.oob[run] = s_oob;
    }
}

size_t inj_smem(int K, int n_f1, int H)
{
    size_t words8 = 3 * K + static_cast<size_t>(K) * n_f1 + (K + 1) / 2 + K;  // 8-byte words
    return words8 * 8 + static_cast<size_t>(align16f(2 * H + 1)) * 4 +
           2 * static_cast<size_t>(kInjSlots) * kInjThreads * 4 + 16;
}

}  // namespace

extern "C" int ft_run_injections(ft_ctx *ctx, const ft_band *band, const ft_bank *bank,
                                 const double *det_tensor, const ft_inj_desc *desc, int64_t n,
                                 const ft_injection *inj, ft_inj_result *out, void *stream)
{
    if (!ctx || !band || !bank || !det_tensor || !desc || (n > 0 && (!inj || !out)))
        FT_FAIL(FT_ERR_ARG, "run_injections: null argument");
    if (band->ctx != ctx || bank->ctx != ctx || bank->band != band)
        FT_FAIL(FT_ERR_ARG, "run_injections: band/bank do not belong together or to ctx");
    if (!band->d_sn)
        FT_FAIL(FT_ERR_ARG, "run_injections: the band was loaded without S_n");
    const int K = desc->k_sky;
    if (K < 1 || K > kInjMaxK || K > bank->n_sky)
        FT_FAIL(FT_ERR_RANGE, "run_injections: k_sky must be in [1, min(128, n_sky)]");
    if (desc->half_f0 < 0 || desc->half_f0 > 7 || desc->half_window < 1 || desc->half_window > 1024)
        FT_FAIL(FT_ERR_RANGE, "run_injections: half_f0 in [0, 7], half_window in [1, 1024]");
    if (bank->n_f1 > kInjMaxF1)
        FT_FAIL(FT_ERR_RANGE, "run_injections: at most 64 f1 values");
    const long long max_nt = static_cast<long long>(2 * desc->half_f0 + 1) * bank->n_f1 * K;
    if (max_nt > static_cast<long long>(kInjThreads) * kInjSlots)
        FT_FAIL(FT_ERR_RANGE, "run_injections: local bank larger than 4096 templates");
    if (!(desc->noise_scale >= 0.0))
        FT_FAIL(FT_ERR_ARG, "run_injections: noise_scale must be >= 0");
    if (n == 0)
        return FT_OK;
    for (int64_t i = 0; i < n; ++i) {
        const double *nn = inj[i].n;
        const double r2 = nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2];
        if (!(std::fabs(r2 - 1.0) < 1e-9) || !std::isfinite(inj[i].h0) || inj[i].h0 < 0 ||
            !std::isfinite(inj[i].f0) || !std::isfinite(inj[i].f1) || !std::isfinite(inj[i].cosi) ||
            !std::isfinite(inj[i].psi))
            FT_FAIL(FT_ERR_ARG, "run_injections: bad injection parameters at index " + std::to_string(i));
    }
    int prev = -1;
    FT_CUDA(cudaGetDevice(&prev));
    if (prev != ctx->device)
        FT_CUDA(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();  // drop errors left by earlier, unrelated runtime calls
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0)
                cudaSetDevice(d);
        }
    } restore{prev != ctx->device ? prev : -1};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // local sky banks: the K bank sky points nearest to each source (largest dot product in
    // FP64, fma(n2, m2, fma(n1, m1, n0 m0)), ties by index)
    std::vector<double> sky(static_cast<size_t>(3 * bank->n_sky));
    FT_CUDA(cudaMemcpy(sky.data(), bank->d_sky, sky.size() * 8, cudaMemcpyDeviceToHost));
    std::vector<int> sidx(static_cast<size_t>(n) * K);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t r = 0; r < n; ++r) {
        std::vector<std::pair<double, int>> d(bank->n_sky);
        const double *m = inj[r].n;
        for (int64_t i = 0; i < bank->n_sky; ++i) {
            const double *s = &sky[3 * i];
            d[i] = {std::fma(m[2], s[2], std::fma(m[1], s[1], m[0] * s[0])), static_cast<int>(i)};
        }
        std::partial_sort(d.begin(), d.begin() + K, d.end(), [](const auto &x, const auto &y) {
            return x.first > y.first || (x.first == y.first && x.second < y.second);
        });
        for (int k = 0; k < K; ++k)
            sidx[r * K + k] = d[k].second;
    }

    // the sky points any run uses, compacted: their E / C tables are computed once
    std::vector<int> cpos(static_cast<size_t>(bank->n_sky), -1), used, cidx(sidx.size());
    for (size_t i = 0; i < sidx.size(); ++i) {
        int &c = cpos[sidx[i]];
        if (c < 0) {
            c = static_cast<int>(used.size());
            used.push_back(sidx[i]);
        }
        cidx[i] = c;
    }
    const size_t N = band->N;
    const size_t n_used = used.size();
    // runs per launch: the per-(run, row) signal bins and amplitudes of one chunk take at
    // most about 1 GB
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (1ll << 30) / (12 * static_cast<long long>(N))));
    double *dD = nullptr;
    InjRun *druns = nullptr;
    int *dsidx = nullptr, *dcidx = nullptr, *dused = nullptr, *dE = nullptr;
    long long *dC = nullptr, *dks = nullptr;
    float *damp = nullptr;
    double *dz = nullptr;
    long long *darg = nullptr, *doob = nullptr;
    auto release = [&]() {
        cudaFree(dD);
        cudaFree(druns);
        cudaFree(dsidx);
        cudaFree(dcidx);
        cudaFree(dused);
        cudaFree(dE);
        cudaFree(dC);
        cudaFree(dks);
        cudaFree(damp);
        cudaFree(dz);
        cudaFree(darg);
        cudaFree(doob);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&dD, N * 6 * 8)) != cudaSuccess ||
        (e = cudaMalloc(&druns, n * sizeof(InjRun))) != cudaSuccess ||
        (e = cudaMalloc(&dsidx, sidx.size() * 4)) != cudaSuccess ||
        (e = cudaMalloc(&dcidx, cidx.size() * 4)) != cudaSuccess ||
        (e = cudaMalloc(&dused, n_used * 4)) != cudaSuccess ||
        (e = cudaMalloc(&dE, n_used * N * 4)) != cudaSuccess ||
        (e = cudaMalloc(&dC, n_used * N * 8)) != cudaSuccess ||
        (e = cudaMalloc(&dks, static_cast<size_t>(chunk) * N * 8)) != cudaSuccess ||
        (e = cudaMalloc(&damp, static_cast<size_t>(chunk) * N * 4)) != cudaSuccess ||
        (e = cudaMalloc(&dz, n * 8)) != cudaSuccess || (e = cudaMalloc(&darg, n * 8)) != cudaSuccess ||
        (e = cudaMalloc(&doob, n * 8)) != cudaSuccess) {
        release();
        FT_FAIL(FT_ERR_OOM, std::string("run_injections: ") + cudaGetErrorString(e));
    }
    static_assert(sizeof(InjRun) == sizeof(ft_injection), "injection record layout");
    bool okc = cudaMemcpyAsync(dD, det_tensor, N * 6 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(druns, inj, n * sizeof(InjRun), cudaMemcpyHostToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(dsidx, sidx.data(), sidx.size() * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(dcidx, cidx.data(), cidx.size() * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
               cudaMemcpyAsync(dused, used.data(), n_used * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (!okc) {
        release();
        FT_FAIL(FT_ERR_CUDA, "run_injections: upload failed");
    }
    InjParams p;
    std::memset(&p, 0, sizeof(p));
    p.N = band->N;
    p.k_lo = band->k_lo;
    p.K0 = bank->k0;
    p.n_f0 = bank->n_f0;
    p.n_f1 = bank->n_f1;
    p.K = K;
    p.half_f0 = desc->half_f0;
    p.H = desc->half_window;
    p.t0 = band->t0;
    p.t_sft = band->t_sft;
    p.mu = band->mu;
    p.sigma = band->sigma;
    p.noise_scale = desc->noise_scale;
    p.tau = band->d_tau;
    p.v = band->d_v;
    p.sn = band->d_sn;
    p.D = dD;
    p.sky = bank->d_sky;
    p.w = band->d_w;
    p.G = bank->d_G;
    p.runs = druns;
    p.sky_idx = dsidx;
    p.sky_cidx = dcidx;
    p.Etab = dE;
    p.Ctab = dC;
    p.ksig_rows = dks;
    p.amp_rows = damp;
    p.seed = desc->seed;
    p.first_id = desc->first_run_id;
    p.max_z = dz;
    p.argmax = darg;
    p.oob = doob;
    const size_t smem = inj_smem(K, bank->n_f1, desc->half_window);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_injections, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) != cudaSuccess) {
            release();
            FT_FAIL(FT_ERR_RANGE, "run_injections: shared memory for this local bank too large");
        }
    }
    {
        const long long tot = static_cast<long long>(n_used) * static_cast<long long>(N);
        k_inj_ec<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(
            static_cast<long long>(N), static_cast<int>(n_used), dused, band->d_v, bank->d_sky, bank->k0,
            band->k_lo, dE, dC);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            release();
            FT_FAIL(FT_ERR_CUDA, std::string("run_injections: launch: ") + cudaGetErrorString(e));
        }
    }
    for (int64_t done = 0; done < n;) {
        const int64_t m = std::min<int64_t>(n - done, chunk);
        InjParams q = p;
        q.runs = druns + done;
        q.sky_idx = dsidx + done * K;
        q.sky_cidx = dcidx + done * K;
        q.first_id = desc->first_run_id + done;
        q.max_z = dz + done;
        q.argmax = darg + done;
        q.oob = doob + done;
        const long long rows = static_cast<long long>(m) * static_cast<long long>(N);
        k_inj_rows<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, st>>>(q, m, dks, damp);
        k_injections<<<static_cast<unsigned>(m), kInjThreads, smem, st>>>(q);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            release();
            FT_FAIL(FT_ERR_CUDA, std::string("run_injections: launch: ") + cudaGetErrorString(e));
        }
        done += m;
    }
    std::vector<double> hz(n);
    std::vector<long long> ha(n), ho(n);
    okc = cudaMemcpyAsync(hz.data(), dz, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaMemcpyAsync(ha.data(), darg, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaMemcpyAsync(ho.data(), doob, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess;
    release();
    if (!okc)
        FT_FAIL(FT_ERR_CUDA, "run_injections: result copy failed");
    for (int64_t i = 0; i < n; ++i) {
        out[i].max_z = hz[i];
        out[i].template_idx = ha[i];
        out[i].n_out_of_window = ho[i];
    }
    return FT_OK;
}

// ------------------------------------------------------------------ semi-analytic q (Sec. V.A)
//
// One CTA per population draw: every thread sums w rho^2 and w^2 rho^2 (h0 = 1) over a
// strided set of SFTs in FP64, then a fixed-order tree over the CTA.

namespace {

constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads) k_pdet_q(long long N, double t_sft, const double *sn,
                                                      const double *D, const float *w,
                                                      const InjRun *pop, double *rho1, double *rho2)
{
    __shared__ double s1[kQThreads], s2[kQThreads];
    const InjRun r = pop[blockIdx.x];
    const double c2 = cos(2.0 * r.psi), sn2 = sin(2.0 * r.psi);
    const double ap = 0.5 * (1.0 + r.cosi * r.cosi), ax = r.cosi;
    const double h = 0.7737 * 0.5 * t_sft;  // |h~| per unit h0 and |Q|
    double a1 = 0.0, a2 = 0.0;
    for (long long a = threadIdx.x; a < N; a += kQThreads) {
        double aa, bb;
        antenna_ab(D + 6 * a, r.n, aa, bb);
        const double fp = aa * c2 + bb * sn2, fx = bb * c2 - aa * sn2;
        const double q2 = fp * fp * ap * ap + fx * fx * ax * ax;
        const double rho = 4.0 * h * h * q2 / (t_sft * sn[a]);
        const double wa = w != nullptr ? static_cast<double>(w[a]) : 1.0;
        a1 += wa * rho;
        a2 += wa * wa * rho;
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int off = kQThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s1[threadIdx.x] += s1[threadIdx.x + off];
            s2[threadIdx.x] += s2[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rho1[blockIdx.x] = s1[0];
        rho2[blockIdx.x] = s2[0];
    }
}

}  // namespace

extern "C" int ft_pdet_q(ft_ctx *ctx, const ft_band *band, const double *det_tensor, int64_t n,
                         const ft_injection *pop, double *rho1, double *rho2, void *stream)
{
    if (!ctx || !band || !det_tensor || (n > 0 && (!pop || !rho1 || !rho2)))
        FT_FAIL(FT_ERR_ARG, "pdet_q: null argument");
    if (band->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "pdet_q: band belongs to another context");
    if (!band->d_sn)
        FT_FAIL(FT_ERR_ARG, "pdet_q: the band was loaded without S_n");
    if (n < 0)
        FT_FAIL(FT_ERR_ARG, "pdet_q: negative count");
    if (n == 0)
        return FT_OK;
    for (int64_t i = 0; i < n; ++i) {
        const double *nn = pop[i].n;
        const double r2 = nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2];
        if (!(std::fabs(r2 - 1.0) < 1e-9) || !std::isfinite(pop[i].cosi) || !std::isfinite(pop[i].psi))
            FT_FAIL(FT_ERR_ARG, "pdet_q: bad draw at index " + std::to_string(i));
    }
    int prev = -1;
    FT_CUDA(cudaGetDevice(&prev));
    if (prev != ctx->device)
        FT_CUDA(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();  // drop errors left by earlier, unrelated runtime calls
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0)
                cudaSetDevice(d);
        }
    } restore{prev != ctx->device ? prev : -1};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t N = band->N;
    double *dD = nullptr, *d1 = nullptr, *d2 = nullptr;
    InjRun *dpop = nullptr;
    auto release = [&]() {
        cudaFree(dD);
        cudaFree(dpop);
        cudaFree(d1);
        cudaFree(d2);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&dD, N * 6 * 8)) != cudaSuccess ||
        (e = cudaMalloc(&dpop, n * sizeof(InjRun))) != cudaSuccess ||
        (e = cudaMalloc(&d1, n * 8)) != cudaSuccess || (e = cudaMalloc(&d2, n * 8)) != cudaSuccess) {
        release();
        FT_FAIL(FT_ERR_OOM, std::string("pdet_q: ") + cudaGetErrorString(e));
    }
    bool ok = cudaMemcpyAsync(dD, det_tensor, N * 6 * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(dpop, pop, n * sizeof(InjRun), cudaMemcpyHostToDevice, st) == cudaSuccess;
    for (int64_t done = 0; ok && done < n;) {
        const int64_t m = std::min<int64_t>(n - done, 1 << 30);
        k_pdet_q<<<static_cast<unsigned>(m), kQThreads, 0, st>>>(static_cast<long long>(N), band->t_sft,
                                                                 band->d_sn, dD, band->d_w, dpop + done,
                                                                 d1 + done, d2 + done);
        ok = cudaGetLastError() == cudaSuccess;
        done += m;
    }
    ok = ok && cudaMemcpyAsync(rho1, d1, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaMemcpyAsync(rho2, d2, n * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
    release();
    if (!ok)
        FT_FAIL(FT_ERR_CUDA, "pdet_q: device work failed");
    return FT_OK;
}
