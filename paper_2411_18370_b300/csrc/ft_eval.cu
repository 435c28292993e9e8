// ft_eval.cu -- device kernels of the brute-force short-coherence statistic.
//
// Statistic (arXiv 2411.18370, Sec. II.B, Eq. (short_coh_general)):
//     s(lambda) = sum_alpha w_alpha P[alpha][k_alpha(lambda)]
// Track bin (Sec. II.A, Eq. (track) with a_p = 0 plus an f1 term), exact integer form:
//     eps = fma(vz, nz, fma(vy, ny, vx*nx))            FP64, pinned order
//     E   = rint(eps 2^32)                              (|E| < 2^22 since |v/c| < 1e-3)
//     C   = rint(fma(K0, eps, K0 - k_lo) 2^32)
//     G   = rint((f1 tau) 2^32), tau = (t_mid - t0) T_SFT   (per (f1, SFT), built once per bank)
//     X0  = C + G + floor(G E / 2^32)
//     k_j = j + floor((X0 + 2^31 + j E) / 2^32)
//
// Work decomposition (one CTA = one sky point x F consecutive f1 values x 32R consecutive
// f0 indices; warp w <-> f1 value, lane <-> f0 index j0 + lane + 32 r, r < R):
//   * SFT rows are streamed through shared memory in stages of S rows, each stage one
//     contiguous cp.async.bulk (TMA) copy completing on an mbarrier, double-buffered.
//   * per stage the CTA computes E, C per SFT (FP64, one thread per row) and X0 per
//     (f1, SFT) (integer), so the per-evaluation work is one IMAD.WIDE, one shared-memory
//     load and one FFMA; lanes of a warp read consecutive bins (conflict-free).
//   * FP32 partial sums per stage are folded into a compensated (2Sum) FP32 pair.
//   * epilogue: either write s (and z, out-of-window counts) or select, per sub-band, the
//     k loudest templates of the CTA into a candidate list (merged by k_topk_merge).
#include "ft_internal.cuh"

#include <climits>
#include <cmath>

namespace {

constexpr double kTwo32 = 4294967296.0;
constexpr int kNbuf = 2;

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase, giving up after about one second of wall time.
__device__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_ns() - t0 > 1000000000ull)
            return false;
    }
}

// ------------------------------------------------------------------ track arithmetic

// E and C of one (sky, SFT) pair.  v is v/c (3 doubles), n the sky unit vector.
__device__ __forceinline__ void track_ec(const double *v, double n0, double n1, double n2,
                                         long long K0, long long k_lo, int &E, long long &C)
{
    const double eps = __fma_rn(v[2], n2, __fma_rn(v[1], n1, __dmul_rn(v[0], n0)));
    E = static_cast<int>(__double2ll_rn(__dmul_rn(eps, kTwo32)));
    C = __double2ll_rn(
        __dmul_rn(__fma_rn(static_cast<double>(K0), eps, static_cast<double>(K0 - k_lo)), kTwo32));
}

// X0 = C + G + floor(G E / 2^32), with the product formed exactly in 128 bits.
__device__ __forceinline__ long long track_x0(long long C, long long G, int E)
{
    const unsigned long long lo =
        static_cast<unsigned long long>(G) * static_cast<unsigned long long>(static_cast<long long>(E));
    const long long hi = __mul64hi(G, static_cast<long long>(E));
    const long long q = static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | (lo >> 32));
    return C + G + q;
}

// k_j = j + floor((X0p + j E) / 2^32), X0p = X0 + 2^31.
__device__ __forceinline__ int track_bin(long long X0p, int E, int j)
{
    const long long acc = X0p + static_cast<long long>(j) * static_cast<long long>(E);
    return j + static_cast<int>(acc >> 32);
}

template <typename T>
__device__ __forceinline__ float to_float(T x);
template <>
__device__ __forceinline__ float to_float<float>(float x)
{
    return x;
}
template <>
__device__ __forceinline__ float to_float<__half>(__half x)
{
    return __half2float(x);
}
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 x)
{
    return __bfloat162float(x);
}

// ------------------------------------------------------------------ shared-memory layout

struct SmemLayout {
    size_t bars, tabE, tabW, tabC, tabX, buf, total, buf_bytes;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a)
{
    return (x + a - 1) / a * a;
}

__host__ __device__ inline SmemLayout smem_layout(int S, int F, int Wp, int esize, int R, bool topk)
{
    SmemLayout L;
    size_t o = 0;
    L.bars = o;
    o += 128;
    L.tabE = o;
    o = align_up(o + 2 * S * sizeof(int), 16);
    L.tabW = o;
    o = align_up(o + 2 * S * sizeof(float), 16);
    L.tabC = o;
    o = align_up(o + 2 * S * sizeof(long long), 16);
    L.tabX = o;
    o = align_up(o + 2 * (size_t)F * S * sizeof(long long), 128);
    L.buf = o;
    size_t stage_bytes = (size_t)kNbuf * S * Wp * esize;
    size_t topk_bytes = topk ? (size_t)F * 32 * R * 2 * sizeof(float) : 0;
    L.buf_bytes = stage_bytes > topk_bytes ? stage_bytes : topk_bytes;
    o += L.buf_bytes;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ evaluation kernel

template <typename T, int R, bool CHECKED>
__global__ void __launch_bounds__(1024, 1) k_eval(const EvalParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int F = blockDim.x >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = p.S;
    const SmemLayout L = smem_layout(S, F, p.Wp, sizeof(T), R, p.cand != nullptr);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + L.bars);
    int *tabE = reinterpret_cast<int *>(smem + L.tabE);
    float *tabW = reinterpret_cast<float *>(smem + L.tabW);
    long long *tabC = reinterpret_cast<long long *>(smem + L.tabC);
    long long *tabX = reinterpret_cast<long long *>(smem + L.tabX);
    T *buf = reinterpret_cast<T *>(smem + L.buf);

    const long long cta = blockIdx.x;
    const int f0t = static_cast<int>(cta % p.n_f0t);
    const long long rest = cta / p.n_f0t;
    const int f1g = static_cast<int>(rest % p.n_f1g);
    const long long sky = rest / p.n_f1g;
    const int j0 = f0t * 32 * R;
    const int f = f1g * F + warp;
    const bool f_ok = f < p.n_f1;
    const double n0 = p.sky[3 * sky], n1 = p.sky[3 * sky + 1], n2 = p.sky[3 * sky + 2];

    int jr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = j0 + lane + 32 * r;
        jr[r] = j < p.n_f0 ? j : p.n_f0 - 1;
    }

    const size_t stage_elems = static_cast<size_t>(S) * p.Wp;
    const long long N = p.N;
    const int n_stages = p.n_stages;

    auto rows_in_stage = [&](int st) -> int {
        const long long left = N - static_cast<long long>(st) * S;
        return static_cast<int>(left < S ? left : S);
    };
    auto issue = [&](int st) {
        const int nb = st % kNbuf;
        const unsigned bytes = static_cast<unsigned>(rows_in_stage(st)) * p.Wp * sizeof(T);
        mbar_arrive_expect_tx(&bars[nb], bytes);
        bulk_copy_g2s(buf + nb * stage_elems,
                      static_cast<const T *>(p.power) + static_cast<size_t>(st) * stage_elems, bytes,
                      &bars[nb]);
    };
    // per-SFT terms of stage st: E, w, C
    auto table_a = [&](int st) {
        const int tb = st & 1;
        const int nr = rows_in_stage(st);
        for (int a = tid; a < nr; a += blockDim.x) {
            const long long alpha = static_cast<long long>(st) * S + a;
            int E;
            long long C;
            track_ec(p.v + 3 * alpha, n0, n1, n2, p.K0, p.k_lo, E, C);
            tabE[tb * S + a] = E;
            tabC[tb * S + a] = C;
            tabW[tb * S + a] = p.w[alpha];
        }
    };
    // per-(f1, SFT) origins of stage st: X0 + 2^31
    auto table_b = [&](int st) {
        const int tb = st & 1;
        const int nr = rows_in_stage(st);
        for (int i = tid; i < F * nr; i += blockDim.x) {
            const int fl = i / nr, a = i - fl * nr;
            int fg = f1g * F + fl;
            fg = fg < p.n_f1 ? fg : p.n_f1 - 1;
            const long long alpha = static_cast<long long>(st) * S + a;
            const long long G = p.G[static_cast<long long>(fg) * N + alpha];
            tabX[(static_cast<size_t>(tb) * F + fl) * S + a] =
                track_x0(tabC[tb * S + a], G, tabE[tb * S + a]) + (1ll << 31);
        }
    };

    if (tid == 0) {
        for (int b = 0; b < kNbuf; ++b)
            mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int st = 0; st < kNbuf && st < n_stages; ++st)
            issue(st);
    }
    table_a(0);
    __syncthreads();
    table_b(0);

    float part[R], hi[R], lo[R];
    int oob[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        part[r] = 0.f;
        hi[r] = 0.f;
        lo[r] = 0.f;
        oob[r] = 0;
    }

    bool ok = true;
    int st = 0;
    for (; st < n_stages; ++st) {
        const int tb = st & 1;
        if (st + 1 < n_stages)
            table_a(st + 1);
        const bool got = mbar_wait_bounded(&bars[st % kNbuf], (st / kNbuf) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        const T *rows = buf + (st % kNbuf) * stage_elems;
        const int nr = rows_in_stage(st);
        const int *tE = tabE + tb * S;
        const float *tW = tabW + tb * S;
        const long long *tX = tabX + (static_cast<size_t>(tb) * F + warp) * S;
#pragma unroll 2
        for (int a = 0; a < nr; ++a) {
            const T *row = rows + static_cast<size_t>(a) * p.Wp;
            const int E = tE[a];
            const float wa = tW[a];
            const long long X = tX[a];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = track_bin(X, E, jr[r]);
                float val;
                if (CHECKED) {
                    const bool in = static_cast<unsigned>(k) < static_cast<unsigned>(p.W);
                    const int kc = min(max(k, 0), p.W - 1);
                    val = in ? to_float<T>(row[kc]) : 0.f;
                    oob[r] += in ? 0 : 1;
                } else {
                    val = to_float<T>(row[k]);
                }
                part[r] = __fmaf_rn(wa, val, part[r]);
            }
        }
        // fold the stage partial into the compensated pair (2Sum)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float s = __fadd_rn(hi[r], part[r]);
            const float bp = __fsub_rn(s, hi[r]);
            const float e = __fadd_rn(__fsub_rn(hi[r], __fsub_rn(s, bp)), __fsub_rn(part[r], bp));
            lo[r] = __fadd_rn(lo[r], e);
            hi[r] = s;
            part[r] = 0.f;
        }
        if (st + 1 < n_stages)
            table_b(st + 1);
        __syncthreads();
        if (tid == 0 && st + kNbuf < n_stages)
            issue(st + kNbuf);
    }

    if (!ok) {
        if (tid == 0) {
            atomicOr(p.status, FT_STATUS_TIMEOUT);
            // let copies still in flight land before the CTA's shared memory is released
            for (int s2 = st; s2 < n_stages && s2 < st + kNbuf; ++s2)
                (void)mbar_wait_bounded(&bars[s2 % kNbuf], (s2 / kNbuf) & 1);
        }
        return;
    }

    // ---------------------------------------------------------------- epilogue
    const long long trow = (sky * p.n_f1 + f) * static_cast<long long>(p.n_f0);
    float sv[R], zv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        sv[r] = __fadd_rn(hi[r], lo[r]);
        zv[r] = static_cast<float>(
            (static_cast<double>(hi[r]) + static_cast<double>(lo[r]) - p.mu) / p.sigma);
    }
    if (p.s_out != nullptr && f_ok) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + lane + 32 * r;
            if (j < p.n_f0) {
                p.s_out[trow + j] = sv[r];
                if (p.z_out)
                    p.z_out[trow + j] = zv[r];
                if (p.oob_out)
                    p.oob_out[trow + j] = oob[r];
            }
        }
    }
    if (p.cand == nullptr)
        return;

    // fused candidate selection: per sub-band, the k loudest templates of this CTA
    const int J = 32 * R;
    float *vs = reinterpret_cast<float *>(buf);
    float *vz = vs + F * J;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        vs[warp * J + lane + 32 * r] = sv[r];
        vz[warp * J + lane + 32 * r] = zv[r];
    }
    __syncthreads();
    const int jhi = min(j0 + J, p.n_f0);
    const int lb0 = j0 / p.sub, lb1 = (jhi - 1) / p.sub;
    const int nf = min(F, p.n_f1 - f1g * F);
    for (int lb = lb0 + warp; lb <= lb1; lb += F) {
        const int ja = max(j0, lb * p.sub), jb = min(jhi, (lb + 1) * p.sub);
        const int width = jb - ja;
        const int count = nf * width;
        float last_s = INFINITY;
        long long last_t = -1;
        ft_candidate *out = reinterpret_cast<ft_candidate *>(p.cand) +
                            (cta * p.lsub_max + (lb - lb0)) * p.k;
        for (int i = 0; i < p.k; ++i) {
            bool have = false;
            float bs = -INFINITY, bz = 0.f;
            long long bt = LLONG_MAX;
            for (int c = lane; c < count; c += 32) {
                const int fl = c / width, jj = ja + (c - fl * width);
                const float s = vs[fl * J + (jj - j0)];
                const long long t = (sky * p.n_f1 + f1g * F + fl) * static_cast<long long>(p.n_f0) + jj;
                const bool elig = (s < last_s) || (s == last_s && t > last_t);
                const bool better = !have || (s > bs) || (s == bs && t < bt);
                if (elig && better) {
                    have = true;
                    bs = s;
                    bt = t;
                    bz = vz[fl * J + (jj - j0)];
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, bs, off);
                const float oz = __shfl_xor_sync(0xffffffffu, bz, off);
                const long long ot = __shfl_xor_sync(0xffffffffu, bt, off);
                const bool oh = __shfl_xor_sync(0xffffffffu, have ? 1 : 0, off) != 0;
                if (oh && (!have || os > bs || (os == bs && ot < bt))) {
                    have = true;
                    bs = os;
                    bt = ot;
                    bz = oz;
                }
            }
            if (lane == 0) {
                ft_candidate c;
                c.template_idx = have ? bt : -1;
                c.s = have ? bs : -INFINITY;
                c.z = have ? bz : 0.f;
                out[i] = c;
            }
            last_s = bs;
            last_t = bt;
        }
    }
}

// ------------------------------------------------------------------ candidate merge

__device__ __forceinline__ bool cand_better(const ft_candidate &a, const ft_candidate &b)
{
    return a.s > b.s || (a.s == b.s && a.template_idx < b.template_idx);
}

constexpr int kKmax = 32;
constexpr int kMergeThreads = 256;

// One CTA per sub-band: gathers the per-CTA lists of every evaluation CTA whose f0 tile
// meets the sub-band and keeps the k best by (s desc, template index asc).
__global__ void __launch_bounds__(kMergeThreads) k_topk_merge(const ft_candidate *cand, int k,
                                                              int lsub_max, long long n_sky,
                                                              int n_f1g, int n_f0t, int J, int sub,
                                                              int n_f0, ft_candidate *out)
{
    __shared__ ft_candidate wl[kMergeThreads / 32][kKmax];
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ft_lo = (b * sub) / J;
    const int ft_hi = (min((b + 1) * sub, n_f0) - 1) / J;
    const int nft = ft_hi - ft_lo + 1;
    const long long total = n_sky * n_f1g * static_cast<long long>(nft) * k;

    ft_candidate Lst[kKmax];
    int n = 0;
    for (long long c = tid; c < total; c += blockDim.x) {
        const long long q = c / k;
        const int i = static_cast<int>(c - q * k);
        const int ftl = static_cast<int>(q % nft);
        const long long sg = q / nft;
        const int ft = ft_lo + ftl;
        const long long cta = sg * n_f0t + ft;
        const int lb = b - (ft * J) / sub;
        const ft_candidate x = cand[(cta * lsub_max + lb) * k + i];
        if (x.template_idx < 0)
            continue;
        if (n < k || cand_better(x, Lst[n - 1])) {
            int pos = n < k ? n : k - 1;
            while (pos > 0 && cand_better(x, Lst[pos - 1])) {
                Lst[pos] = Lst[pos - 1];
                --pos;
            }
            Lst[pos] = x;
            if (n < k)
                ++n;
        }
    }
    // warp-level merge of the lanes' sorted lists
    int h = 0;
    for (int i = 0; i < k; ++i) {
        ft_candidate c;
        bool have = h < n;
        if (have)
            c = Lst[h];
        else {
            c.template_idx = LLONG_MAX;
            c.s = -INFINITY;
            c.z = 0.f;
        }
        int src = lane;
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, c.s, off);
            const long long ot = __shfl_xor_sync(0xffffffffu, c.template_idx, off);
            const int osrc = __shfl_xor_sync(0xffffffffu, src, off);
            const bool oh = __shfl_xor_sync(0xffffffffu, have ? 1 : 0, off) != 0;
            if (oh && (!have || os > c.s || (os == c.s && ot < c.template_idx))) {
                have = true;
                c.s = os;
                c.template_idx = ot;
                src = osrc;
            }
        }
        c.z = __shfl_sync(0xffffffffu, (h < n) ? Lst[h].z : 0.f, src);
        if (have && lane == src)
            ++h;
        if (lane == 0) {
            if (!have) {
                c.template_idx = -1;
                c.s = -INFINITY;
                c.z = 0.f;
            }
            wl[warp][i] = c;
        }
    }
    __syncthreads();
    if (warp != 0)
        return;
    // block-level merge of the warps' lists (lane w < n_warps holds list w)
    const int nw = blockDim.x >> 5;
    h = 0;
    for (int i = 0; i < k; ++i) {
        ft_candidate c;
        bool have = lane < nw && h < k && wl[lane][h].template_idx >= 0;
        if (have)
            c = wl[lane][h];
        else {
            c.template_idx = LLONG_MAX;
            c.s = -INFINITY;
            c.z = 0.f;
        }
        int src = lane;
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, c.s, off);
            const float oz = __shfl_xor_sync(0xffffffffu, c.z, off);
            const long long ot = __shfl_xor_sync(0xffffffffu, c.template_idx, off);
            const int osrc = __shfl_xor_sync(0xffffffffu, src, off);
            const bool oh = __shfl_xor_sync(0xffffffffu, have ? 1 : 0, off) != 0;
            if (oh && (!have || os > c.s || (os == c.s && ot < c.template_idx))) {
                have = true;
                c.s = os;
                c.z = oz;
                c.template_idx = ot;
                src = osrc;
            }
        }
        if (have && lane == src)
            ++h;
        if (lane == 0) {
            if (!have) {
                c.template_idx = -1;
                c.s = -INFINITY;
                c.z = 0.f;
            }
            out[static_cast<long long>(b) * k + i] = c;
        }
    }
}

// ------------------------------------------------------------------ helpers

__global__ void k_convert(const void *src, int sdt, long long sstride, void *dst, int ddt,
                          long long N, int W, int Wp, unsigned int *status)
{
    const long long total = N * Wp;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long row = i / Wp;
        const int col = static_cast<int>(i - row * Wp);
        double x = 0.0;
        if (col < W) {
            x = (sdt == FT_F64) ? static_cast<const double *>(src)[row * sstride + col]
                                : static_cast<double>(static_cast<const float *>(src)[row * sstride + col]);
            if (!isfinite(x))
                atomicOr(status, FT_STATUS_NONFINITE);
        }
        if (ddt == FT_F32)
            static_cast<float *>(dst)[i] = __double2float_rn(x);
        else if (ddt == FT_F16)
            static_cast<__half *>(dst)[i] = __double2half(x);
        else
            static_cast<__nv_bfloat16 *>(dst)[i] = __double2bfloat16(x);
    }
}

__global__ void k_gtable(const double *f1, int n_f1, const double *tau, long long N, long long *G)
{
    const long long total = N * n_f1;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long f = i / N, a = i - f * N;
        G[i] = __double2ll_rn(__dmul_rn(__dmul_rn(f1[f], tau[a]), kTwo32));
    }
}

__global__ void k_track_bins(const double *v, const double *sky, const long long *G,
                             long long N, long long K0, long long k_lo, int n_f0, int n_f1,
                             long long n_templates, const long long *tmpl, long long n, int *bins)
{
    const long long total = n * N;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long r = i / N, a = i - r * N;
        const long long t = tmpl[r];
        if (t < 0 || t >= n_templates) {
            bins[i] = INT_MIN;
            continue;
        }
        const int j = static_cast<int>(t % n_f0);
        const long long q = t / n_f0;
        const int f = static_cast<int>(q % n_f1);
        const long long s = q / n_f1;
        int E;
        long long C;
        track_ec(v + 3 * a, sky[3 * s], sky[3 * s + 1], sky[3 * s + 2], K0, k_lo, E, C);
        const long long X0 = track_x0(C, G[f * N + a], E);
        bins[i] = track_bin(X0 + (1ll << 31), E, j);
    }
}

int grid_for(long long total, int threads)
{
    long long g = (total + threads - 1) / threads;
    if (g > 148 * 32)
        g = 148 * 32;
    return static_cast<int>(g < 1 ? 1 : g);
}

template <typename T, int R, bool CHECKED>
int launch_eval_t(const EvalShape &sh, const EvalParams &p, long long n_cta, size_t smem,
                  cudaStream_t st)
{
    static size_t configured = 0;
    auto fn = k_eval<T, R, CHECKED>;
    if (smem > configured) {
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
        configured = smem;
    }
    fn<<<static_cast<unsigned>(n_cta), 32 * sh.F, smem, st>>>(p);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

template <typename T, bool CHECKED>
int launch_eval_r(const EvalShape &sh, const EvalParams &p, long long n_cta, size_t smem,
                  cudaStream_t st)
{
    switch (sh.R) {
    case 1: return launch_eval_t<T, 1, CHECKED>(sh, p, n_cta, smem, st);
    case 2: return launch_eval_t<T, 2, CHECKED>(sh, p, n_cta, smem, st);
    case 3: return launch_eval_t<T, 3, CHECKED>(sh, p, n_cta, smem, st);
    case 4: return launch_eval_t<T, 4, CHECKED>(sh, p, n_cta, smem, st);
    case 5: return launch_eval_t<T, 5, CHECKED>(sh, p, n_cta, smem, st);
    case 6: return launch_eval_t<T, 6, CHECKED>(sh, p, n_cta, smem, st);
    case 7: return launch_eval_t<T, 7, CHECKED>(sh, p, n_cta, smem, st);
    case 8: return launch_eval_t<T, 8, CHECKED>(sh, p, n_cta, smem, st);
    default: FT_FAIL(FT_ERR_ARG, "eval: unsupported tile width R");
    }
}

template <typename T>
int launch_eval_c(bool checked, const EvalShape &sh, const EvalParams &p, long long n_cta,
                  size_t smem, cudaStream_t st)
{
    return checked ? launch_eval_r<T, true>(sh, p, n_cta, smem, st)
                   : launch_eval_r<T, false>(sh, p, n_cta, smem, st);
}

int esize_of(int dtype)
{
    return dtype == FT_F32 ? 4 : 2;
}

}  // namespace

// ------------------------------------------------------------------ host launchers

size_t ft_eval_smem_bytes(const ft_band *band, const EvalShape &sh, int k)
{
    return smem_layout(sh.S, sh.F, band->Wp, esize_of(band->dtype), sh.R, k > 0).total;
}

EvalShape ft_default_shape(const ft_ctx *ctx, const ft_band *band, const ft_bank *bank)
{
    EvalShape sh;
    const int groups = (bank->n_f1 + 31) / 32;
    sh.F = (bank->n_f1 + groups - 1) / groups;
    // f0 slots per lane: fewest wasted lanes, then the widest tile
    int best_r = 1;
    long long best_waste = LLONG_MAX;
    for (int r = 1; r <= 8; ++r) {
        const long long J = 32ll * r;
        const long long tiles = (bank->n_f0 + J - 1) / J;
        const long long waste = tiles * J - bank->n_f0;
        if (waste < best_waste || (waste == best_waste && r > best_r)) {
            best_waste = waste;
            best_r = r;
        }
    }
    sh.R = best_r;
    sh.nbuf = kNbuf;
    const size_t row_bytes = static_cast<size_t>(band->Wp) * esize_of(band->dtype);
    int S = static_cast<int>((96 * 1024) / (kNbuf * row_bytes));
    S = S > 64 ? 64 : S;
    S = S < 1 ? 1 : S;
    if (S >= 8)
        S &= ~7;
    sh.S = S;
    (void)ctx;
    return sh;
}

int ft_launch_eval(const ft_band *band, const ft_bank *bank, const EvalShape &sh, EvalParams p,
                   cudaStream_t st)
{
    const int J = 32 * sh.R;
    p.n_f0t = (bank->n_f0 + J - 1) / J;
    p.n_f1g = (bank->n_f1 + sh.F - 1) / sh.F;
    p.S = sh.S;
    p.n_stages = static_cast<int>((band->N + sh.S - 1) / sh.S);
    const long long n_cta = bank->n_sky * p.n_f1g * static_cast<long long>(p.n_f0t);
    if (n_cta <= 0 || n_cta > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "eval: grid too large (n_sky * f1 groups * f0 tiles >= 2^31)");
    const size_t smem = ft_eval_smem_bytes(band, sh, p.cand ? p.k : 0);
    if (smem > band->ctx->smem_optin)
        FT_FAIL(FT_ERR_RANGE, "eval: tile needs more shared memory than the device offers");
    const bool checked = !bank->window_safe;
    switch (band->dtype) {
    case FT_F32: return launch_eval_c<float>(checked, sh, p, n_cta, smem, st);
    case FT_F16: return launch_eval_c<__half>(checked, sh, p, n_cta, smem, st);
    case FT_BF16: return launch_eval_c<__nv_bfloat16>(checked, sh, p, n_cta, smem, st);
    default: FT_FAIL(FT_ERR_ARG, "eval: bad dtype");
    }
}

int ft_launch_merge(const ft_bank *bank, const EvalShape &sh, const FtCand *cand, int k,
                    int lsub_max, ft_candidate *out, cudaStream_t st)
{
    const int J = 32 * sh.R;
    const int n_f0t = (bank->n_f0 + J - 1) / J;
    const int n_f1g = (bank->n_f1 + sh.F - 1) / sh.F;
    k_topk_merge<<<bank->n_sub, kMergeThreads, 0, st>>>(
        reinterpret_cast<const ft_candidate *>(cand), k, lsub_max, bank->n_sky, n_f1g, n_f0t, J,
        bank->sub, bank->n_f0, out);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int ft_launch_convert(const void *src, int src_dtype, long long src_stride, void *dst,
                      int dst_dtype, long long N, int W, int Wp, unsigned int *status,
                      cudaStream_t st)
{
    k_convert<<<grid_for(N * Wp, 256), 256, 0, st>>>(src, src_dtype, src_stride, dst, dst_dtype,
                                                      N, W, Wp, status);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int ft_launch_gtable(const double *f1, int n_f1, const double *tau, long long N, long long *G,
                     cudaStream_t st)
{
    k_gtable<<<grid_for(N * n_f1, 256), 256, 0, st>>>(f1, n_f1, tau, N, G);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int ft_launch_track_bins(const ft_band *band, const ft_bank *bank, const long long *tmpl,
                         long long n, int *bins, cudaStream_t st)
{
    const long long n_templates = bank->n_sky * bank->n_f1 * static_cast<long long>(bank->n_f0);
    k_track_bins<<<grid_for(n * band->N, 256), 256, 0, st>>>(
        band->d_v, bank->d_sky, bank->d_G, band->N, bank->k0, band->k_lo, bank->n_f0, bank->n_f1,
        n_templates, tmpl, n, bins);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}
