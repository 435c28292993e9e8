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
// Work decomposition: one CTA = one sky point x F consecutive f1 values (one warp each) x
// a tile of J consecutive f0 indices.  SFT rows stream through shared memory in stages of S
// rows, each stage one contiguous cp.async.bulk (TMA) copy completing on an mbarrier,
// double-buffered.  Per stage the CTA computes E, C per SFT (FP64) and each warp the track
// origin of its f1 value per SFT (integer).  Two kernels:
//   * k_eval_fast (tracks provably inside the window): shifted-row sums, see below;
//   * k_eval_checked (otherwise): the full bin per (template, SFT) with a bounds check.
// FP32 partial sums per stage are folded into a compensated (2Sum) FP32 pair.  The
// epilogue writes s (and z, out-of-window counts) or selects, per sub-band, the k loudest
// templates of the CTA into a candidate list that k_topk_merge reduces.
#include "ft_internal.cuh"
#include "ft_ptx.cuh"

#include <cudaTypedefs.h>
#include <cstring>
#include <mutex>

#include <algorithm>
#include <climits>
#include <cmath>

namespace {

constexpr double kTwo32 = 4294967296.0;
constexpr int kNbuf = 2;

// ------------------------------------------------------------------ PTX helpers

using ftp::bulk_g2s;
using ftp::fence_mbar_init;
using ftp::global_ns;
using ftp::mbar_arrive;
using ftp::mbar_arrive_expect_tx;
using ftp::mbar_init;
using ftp::mbar_try_wait;
using ftp::mbar_wait_bounded;
using ftp::smem_addr;
using ftp::tensor_copy_3d;
using ftp::tensor_copy_4d;

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

__host__ __device__ inline size_t align_up(size_t x, size_t a)
{
    return (x + a - 1) / a * a;
}

// Offsets (bytes) of the per-CTA shared-memory regions.  Stage tables are double-buffered
// (index tb = stage & 1); power stages use kNbuf buffers of S rows x row_bytes each, plus a
// guard tail so that lanes past the end of the f0 range may read (and discard) past the
// last row without leaving the allocation.
struct SmemLayout {
    size_t bars, tabE, tabW, tabC, tabX, evA, evK, evN, buf, total, stage_bytes;
};

__host__ __device__ inline SmemLayout smem_layout(int S, int F, int row_bytes, int J, bool fast,
                                                  bool topk)
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
    L.tabX = o;  // checked kernel: X0 [2][F][S] int64; fast kernel: word offsets [2][F][S] int
    o = align_up(o + 2 * (size_t)F * S * (fast ? sizeof(int) : sizeof(long long)), 16);
    L.evA = o;
    o = align_up(o + (fast ? 2 * (size_t)F * S * sizeof(int) : 0), 16);
    L.evK = o;
    o = align_up(o + (fast ? 2 * (size_t)F * S * sizeof(int) : 0), 16);
    L.evN = o;
    o = align_up(o + (fast ? 2 * (size_t)F * sizeof(int) : 0), 128);
    L.buf = o;
    L.stage_bytes = (size_t)S * row_bytes;
    const size_t pipe = kNbuf * L.stage_bytes + (size_t)(J + 64) * 4;
    const size_t tk = topk ? (size_t)F * J * 2 * sizeof(float) + (size_t)F * sizeof(long long) : 0;
    o += pipe > tk ? pipe : tk;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ pieces shared by kernels

struct CtaTile {
    long long cta, skyg, sky;  // sky group, and its first sky point
    int f0t, f1g, j0;
    double n0, n1, n2;         // unit vector of that sky point
};

// Sky index of member q of sky group g (P consecutive points of the bank's sky order), or
// -1 past the last sky point.
__device__ __forceinline__ long long sky_of(const EvalParams &p, long long g, int q)
{
    const long long i = g * p.P + q;
    if (i >= p.n_sky)
        return -1;
    return p.sky_order != nullptr ? static_cast<long long>(p.sky_order[i]) : i;
}

// Template index base (sky, f1) * n_f0 of evaluating warp w of the tile, or -1 when the
// warp has no template (past the last sky point or f1 value, or beyond P * F1 warps).
__device__ __forceinline__ long long warp_template_base(const EvalParams &p, long long skyg,
                                                        int f1g, int w)
{
    const int q = w / p.F1, f = f1g * p.F1 + (w - q * p.F1);
    if (q >= p.P || f >= p.n_f1)
        return -1;
    const long long sk = sky_of(p, skyg, q);
    return sk < 0 ? -1 : (sk * p.n_f1 + f) * static_cast<long long>(p.n_f0);
}

__device__ __forceinline__ CtaTile decode_tile(const EvalParams &p, int J, long long tile)
{
    CtaTile c;
    c.cta = tile;
    c.f0t = static_cast<int>(c.cta % p.n_f0t);
    const long long rest = c.cta / p.n_f0t;
    c.f1g = static_cast<int>(rest % p.n_f1g);
    c.skyg = rest / p.n_f1g;
    c.sky = sky_of(p, c.skyg, 0);
    c.j0 = c.f0t * J;
    c.n0 = p.sky[3 * c.sky];
    c.n1 = p.sky[3 * c.sky + 1];
    c.n2 = p.sky[3 * c.sky + 2];
    return c;
}

__device__ __forceinline__ int rows_in_stage(const EvalParams &p, int st)
{
    const long long left = p.N - static_cast<long long>(st) * p.S;
    return static_cast<int>(left < p.S ? left : p.S);
}

// Thread 0: expect the stage's bytes on its buffer's mbarrier and start the bulk copy.
__device__ __forceinline__ void issue_stage(const EvalParams &p, unsigned char *buf,
                                            unsigned long long *bars, size_t stage_bytes, int st)
{
    const int nb = st % kNbuf;
    const unsigned bytes = static_cast<unsigned>(rows_in_stage(p, st)) * p.row_bytes;
    mbar_arrive_expect_tx(&bars[nb], bytes);
    bulk_g2s(buf + nb * stage_bytes,
                  static_cast<const unsigned char *>(p.power) + static_cast<size_t>(st) * stage_bytes,
                  bytes, &bars[nb]);
}

// Per-SFT terms of stage st for this CTA's sky point: E, C (track arithmetic) and w.
__device__ __forceinline__ void stage_table_a(const EvalParams &p, const CtaTile &c, int st,
                                              int *tabE, long long *tabC, float *tabW)
{
    const int tb = st & 1;
    const int nr = rows_in_stage(p, st);
    for (int a = threadIdx.x; a < nr; a += blockDim.x) {
        const long long alpha = static_cast<long long>(st) * p.S + a;
        int E;
        long long C;
        track_ec(p.v + 3 * alpha, c.n0, c.n1, c.n2, p.K0, p.k_lo, E, C);
        tabE[tb * p.S + a] = E;
        tabC[tb * p.S + a] = C;
        tabW[tb * p.S + a] =
            p.D != nullptr ? ft_sky_r32(p.rowd[2 * alpha], p.rowd[2 * alpha + 1], static_cast<float>(c.n0),
                                        static_cast<float>(c.n1), static_cast<float>(c.n2)) *
                                 static_cast<float>(p.sky_inv[c.sky])
                           : p.w[alpha];
    }
}

// Thread 0 after a failed wait: record the timeout and let copies still in flight land
// before the CTA's shared memory is released.
__device__ void abandon_tile(const EvalParams &p, unsigned long long *bars, int st)
{
    if (threadIdx.x == 0) {
        atomicOr(p.status, FT_STATUS_TIMEOUT);
        for (int s2 = st; s2 < p.n_stages && s2 < st + kNbuf; ++s2)
            (void)mbar_wait_bounded(&bars[s2 % kNbuf], (s2 / kNbuf) & 1);
    }
}

// Fused candidate selection: vs/vz hold [F][J] values of this CTA's templates (index
// = warp * J + j - j0) and wt[w] the template base of warp w (-1: no templates).  Per
// sub-band, one warp extracts the k best by (s desc, t asc) in k rounds of a warp arg-max
// restricted to keys ranked after the previous pick.
__device__ void cta_topk(const EvalParams &p, const CtaTile &c, int F, int J, const float *vs,
                         const float *vz, const long long *wt, ft_candidate *dst)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int jhi = min(c.j0 + J, p.n_f0);
    const int lb0 = c.j0 / p.sub, lb1 = (jhi - 1) / p.sub;
    for (int lb = lb0 + warp; lb <= lb1; lb += F) {
        const int ja = max(c.j0, lb * p.sub), jb = min(jhi, (lb + 1) * p.sub);
        const int width = jb - ja;
        const int count = F * width;
        float last_s = INFINITY;
        long long last_t = -1;
        ft_candidate *out = dst + (lb - lb0) * p.k;
        for (int i = 0; i < p.k; ++i) {
            bool have = false;
            float bs = -INFINITY, bz = 0.f;
            long long bt = LLONG_MAX;
            for (int q = lane; q < count; q += 32) {
                const int fl = q / width, jj = ja + (q - fl * width);
                const long long tb = wt[fl];
                if (tb < 0)
                    continue;
                const float s = vs[fl * J + (jj - c.j0)];
                if (s == -INFINITY)
                    continue;  // gated out
                const long long t = tb + jj;
                const bool elig = (s < last_s) || (s == last_s && t > last_t);
                const bool better = !have || (s > bs) || (s == bs && t < bt);
                if (elig && better) {
                    have = true;
                    bs = s;
                    bt = t;
                    bz = vz[fl * J + (jj - c.j0)];
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
                ft_candidate cd;
                cd.template_idx = have ? bt : -1;
                cd.s = have ? bs : -INFINITY;
                cd.z = have ? bz : 0.f;
                out[i] = cd;
            }
            last_s = bs;
            last_t = bt;
        }
    }
}

// Fold a stage's FP32 partial into the compensated pair (hi, lo) with 2Sum.
__device__ __forceinline__ void fold2sum(float &hi, float &lo, float &part)
{
    const float s = __fadd_rn(hi, part);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(part, bp));
    lo = __fadd_rn(lo, e);
    hi = s;
    part = 0.f;
}

// Epilogue shared by both kernels: s = hi + lo, z in FP64; write and/or select.  F is
// the number of evaluating warps (warps >= F only take part in the barrier).
template <int NS, bool WEIGHTED>
__device__ __forceinline__ void finish_tile(const EvalParams &p, const CtaTile &c, int F, int J,
                                            const int (&jrel)[NS], const float (&hi)[NS],
                                            const float (&lo)[NS], const int (&oob)[NS],
                                            unsigned char *buf, ft_candidate *dst)
{
    const int warp = threadIdx.x >> 5;
    const bool active = warp < F;
    const long long trow = active ? warp_template_base(p, c.skyg, c.f1g, warp) : -1;
    const bool f_ok = trow >= 0;
    double mu = p.mu, sigma = p.sigma;
    if (WEIGHTED && p.sky_sig != nullptr && f_ok) {
        const long long sk = trow / (static_cast<long long>(p.n_f1) * p.n_f0);
        mu = p.sky_mu[sk];
        sigma = p.sky_sig[sk];
    }
    float sv[NS], zv[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        sv[r] = __fadd_rn(hi[r], lo[r]);
        zv[r] = static_cast<float>(
            (static_cast<double>(hi[r]) + static_cast<double>(lo[r]) - mu) / sigma);
    }
    if (p.s_out != nullptr && f_ok) {
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            const int j = c.j0 + jrel[r];
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
    float *vs = reinterpret_cast<float *>(buf);
    float *vz = vs + F * J;
    long long *wt = reinterpret_cast<long long *>(vz + F * J);
    if (active) {
#pragma unroll
        for (int r = 0; r < NS; ++r) {
            float sel = sv[r];
            if (p.gate != nullptr && f_ok) {
                // gated out: -inf never enters the selection
                const int j = c.j0 + jrel[r];
                if (j < p.n_f0 && !(p.gate[trow + j] >= p.gate_min))
                    sel = -INFINITY;
            }
            vs[warp * J + jrel[r]] = sel;
            vz[warp * J + jrel[r]] = zv[r];
        }
        if ((threadIdx.x & 31) == 0)
            wt[warp] = trow;
    }
    __syncthreads();
    if (active) {
        if (dst == nullptr)
            dst = reinterpret_cast<ft_candidate *>(p.cand) + c.cta * p.lsub_max * p.k;
        cta_topk(p, c, F, J, vs, vz, wt, dst);
    }
}

// ------------------------------------------------------------------ checked kernel
//
// General evaluation kernel: per (template, SFT) the full Q32 bin with a bounds check.
// Used when the bank's tracks may leave the band's window (reads outside contribute 0 and
// are counted).  Power rows hold plain elements of T at p.row_elems elements per row.

template <typename T, int R>
__global__ void __launch_bounds__(1024, 1) k_eval_checked(const EvalParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int J = 32 * R;
    const int F = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = p.S;
    const SmemLayout L = smem_layout(S, F, p.row_bytes, J, false, p.cand != nullptr);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + L.bars);
    int *tabE = reinterpret_cast<int *>(smem + L.tabE);
    float *tabW = reinterpret_cast<float *>(smem + L.tabW);
    long long *tabC = reinterpret_cast<long long *>(smem + L.tabC);
    long long *tabX = reinterpret_cast<long long *>(smem + L.tabX);
    unsigned char *buf = smem + L.buf;
    const CtaTile c = decode_tile(p, J, blockIdx.x);

    int jrel[R], jr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        jrel[r] = lane + 32 * r;
        const int j = c.j0 + jrel[r];
        jr[r] = j < p.n_f0 ? j : p.n_f0 - 1;
    }
    auto table_b = [&](int st) {
        const int tb = st & 1;
        const int nr = rows_in_stage(p, st);
        for (int i = threadIdx.x; i < F * nr; i += blockDim.x) {
            const int fl = i / nr, a = i - fl * nr;
            int fg = c.f1g * F + fl;
            fg = fg < p.n_f1 ? fg : p.n_f1 - 1;
            const long long alpha = static_cast<long long>(st) * S + a;
            const long long G = p.G[static_cast<long long>(fg) * p.N + alpha];
            tabX[(static_cast<size_t>(tb) * F + fl) * S + a] =
                track_x0(tabC[tb * S + a], G, tabE[tb * S + a]) + (1ll << 31);
        }
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < kNbuf; ++b)
            mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int st = 0; st < kNbuf && st < p.n_stages; ++st)
            issue_stage(p, buf, bars, L.stage_bytes, st);
    stage_table_a(p, c, 0, tabE, tabC, tabW);
    __syncthreads();
    table_b(0);

    float part[R], hi[R], lo[R];
    int oob[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        part[r] = hi[r] = lo[r] = 0.f;
        oob[r] = 0;
    }
    for (int st = 0; st < p.n_stages; ++st) {
        const int tb = st & 1;
        if (st + 1 < p.n_stages)
            stage_table_a(p, c, st + 1, tabE, tabC, tabW);
        const bool got = mbar_wait_bounded(&bars[st % kNbuf], (st / kNbuf) & 1);
        if (!__syncthreads_and(got)) {
            abandon_tile(p, bars, st);
            return;
        }
        const T *rows = reinterpret_cast<const T *>(buf + (st % kNbuf) * L.stage_bytes);
        const int nr = rows_in_stage(p, st);
        const int *tE = tabE + tb * S;
        const float *tW = tabW + tb * S;
        const long long *tX = tabX + (static_cast<size_t>(tb) * F + warp) * S;
        for (int a = 0; a < nr; ++a) {
            const T *row = rows + static_cast<size_t>(a) * p.row_elems;
            const int E = tE[a];
            const float wa = tW[a];
            const long long X = tX[a];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = track_bin(X, E, jr[r]);
                const bool in = static_cast<unsigned>(k) < static_cast<unsigned>(p.W);
                const int kc = min(max(k, 0), p.W - 1);
                const float val = in ? to_float<T>(row[kc]) : 0.f;
                oob[r] += in ? 0 : 1;
                part[r] = __fmaf_rn(wa, val, part[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            fold2sum(hi[r], lo[r], part[r]);
        if (st + 1 < p.n_stages)
            table_b(st + 1);
        __syncthreads();
        if (threadIdx.x == 0 && st + kNbuf < p.n_stages)
            issue_stage(p, buf, bars, L.stage_bytes, st + kNbuf);
    }
    finish_tile<R, true>(p, c, F, J, jrel, hi, lo, oob, buf, nullptr);
}

// ------------------------------------------------------------------ fast kernel
//
// For a fixed (sky, f1, SFT) the bins of a tile's f0 values are k(j0 + u) = base + u,
// plus at most one step of sign(E) from some u = jc on, because the tile is narrower than
// 1/|eps| bins (J |E| < 2^32).  Per stage, each warp derives for its own f1 value and
// every SFT row the word offset of `base` in shared memory and, for the rare rows whose
// step falls inside the tile, an entry in its correction list.  The main loop is then a
// plain shifted-row sum: one shared load (lanes on consecutive words) and one FMA per
// evaluation; the corrections add w (P[k + s] - P[k]) for the affected f0 afterwards.
//
// MODE_F32: rows of FP32, lane <-> f0 offset lane + 32 r.
// MODE_F16 / MODE_BF16: each row is stored twice as 32-bit pairs, even-aligned
// (P[2m], P[2m+1]) and odd-aligned (P[2m+1], P[2m+2]); the copy matching the parity of
// `base` gives every lane the pair of bins (base + 2 lane + 64 r, +1) in one aligned,
// conflict-free 32-bit load.  Without weights the pair is accumulated by two
// mixed-precision FMAs (16-bit input, FP32 accumulator), i.e. with no conversion step.

enum { MODE_F32 = 0, MODE_F16 = 1, MODE_BF16 = 2 };
constexpr int kFastMaxWarps = 20;

template <int MODE>
__device__ __forceinline__ float lo_to_float(unsigned u)
{
    if (MODE == MODE_F16)
        return __half2float(__ushort_as_half(static_cast<unsigned short>(u & 0xffffu)));
    return __uint_as_float(u << 16);
}

template <int MODE>
__device__ __forceinline__ float hi_to_float(unsigned u)
{
    if (MODE == MODE_F16)
        return __half2float(__ushort_as_half(static_cast<unsigned short>(u >> 16)));
    return __uint_as_float(u & 0xffff0000u);
}

// a0 += lo(u), a1 += hi(u) with 16-bit inputs and FP32 accumulators (exact products by 1).
template <int MODE>
__device__ __forceinline__ void acc_pair(float &a0, float &a1, unsigned u)
{
    if (MODE == MODE_F16) {
        asm("{\n\t.reg .b16 l, h, one;\n\t"
            "mov.b32 {l, h}, %2;\n\t"
            "mov.b16 one, 0x3C00;\n\t"
            "fma.rn.f32.f16 %0, l, one, %0;\n\t"
            "fma.rn.f32.f16 %1, h, one, %1;\n\t}"
            : "+f"(a0), "+f"(a1)
            : "r"(u));
    } else {
        asm("{\n\t.reg .b16 l, h, one;\n\t"
            "mov.b32 {l, h}, %2;\n\t"
            "mov.b16 one, 0x3F80;\n\t"
            "fma.rn.f32.bf16 %0, l, one, %0;\n\t"
            "fma.rn.f32.bf16 %1, h, one, %1;\n\t}"
            : "+f"(a0), "+f"(a1)
            : "r"(u));
    }
}

// a += sg (hi(u) - lo(u)), sg = +-1, with 16-bit inputs and an FP32 accumulator.
template <int MODE>
__device__ __forceinline__ void acc_diff(float &a, unsigned u, int sg)
{
    const unsigned short one = MODE == MODE_F16 ? 0x3C00 : 0x3F80;  // +1 in the storage type
    const unsigned short sign = 0x8000;
    const unsigned short mh = sg < 0 ? static_cast<unsigned short>(one | sign) : one;
    const unsigned short ml = static_cast<unsigned short>(mh ^ sign);
    if (MODE == MODE_F16) {
        asm("{\n\t.reg .b16 l, h;\n\t"
            "mov.b32 {l, h}, %1;\n\t"
            "fma.rn.f32.f16 %0, h, %2, %0;\n\t"
            "fma.rn.f32.f16 %0, l, %3, %0;\n\t}"
            : "+f"(a)
            : "r"(u), "h"(mh), "h"(ml));
    } else {
        asm("{\n\t.reg .b16 l, h;\n\t"
            "mov.b32 {l, h}, %1;\n\t"
            "fma.rn.f32.bf16 %0, h, %2, %0;\n\t"
            "fma.rn.f32.bf16 %0, l, %3, %0;\n\t}"
            : "+f"(a)
            : "r"(u), "h"(mh), "h"(ml));
    }
}

template <int MODE>
__device__ __forceinline__ float read_bin(const unsigned char *rows, int row_words, int a, int k)
{
    if (MODE == MODE_F32)
        return reinterpret_cast<const float *>(rows)[static_cast<size_t>(a) * row_words + k];
    const unsigned u =
        reinterpret_cast<const unsigned *>(rows)[static_cast<size_t>(a) * row_words + (k >> 1)];
    return (k & 1) ? hi_to_float<MODE>(u) : lo_to_float<MODE>(u);
}

// Shared-memory layout of the fast kernel: nst pipeline slots, each with S <= 32 rows of
// power and one 24-byte record per row (the track terms C, E and span, the weight and
// the window start);
// per evaluating warp its own row offsets and correction list for the slot it works on.
constexpr int kMaxStages = 4;
constexpr int kFoldRows = 512;  // FP32 partials cover at most this many SFT rows

// ------------------------------------------------------------------ tensor memory
//
// Between folds the compensated sums (hi, lo) of every evaluating warp are parked in the
// SM's tensor memory instead of registers: 16 columns per warp in the warp's lane quarter
// (warp w reaches lanes 32 (w mod 4) .. + 31), hi in the first 8 columns and lo in the
// next 8, column base 16 (w div 4).  Warp 0 allocates the columns for the CTA and frees
// them when the CTA ends.

__host__ __device__ constexpr unsigned tm_cols_for(int F)
{
    return ((F + 3) / 4) * 16 <= 32 ? 32u : ((F + 3) / 4) * 16 <= 64 ? 64u : 128u;
}

__device__ __forceinline__ void tm_alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tm_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tm_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Eight consecutive columns of this thread's lane into v (valid after tm_wait_ld).
__device__ __forceinline__ void tm_ld8(unsigned taddr, float (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr)
                 : "memory");
}

// Wait for this thread's tensor-memory loads; a and b are the registers they fill, tied to
// the wait so that no use moves above it.
__device__ __forceinline__ void tm_wait_ld(float (&a)[8], float (&b)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(a[4]), "+f"(a[5]),
                   "+f"(a[6]), "+f"(a[7]), "+f"(b[0]), "+f"(b[1]), "+f"(b[2]), "+f"(b[3]),
                   "+f"(b[4]), "+f"(b[5]), "+f"(b[6]), "+f"(b[7])
                 :
                 : "memory");
}

__device__ __forceinline__ void tm_st8(unsigned taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                     taddr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]),
                 "f"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// One row's track terms for one sky point of the tile (16 bytes: one shared load per lane).
struct __align__(16) RowRec {
    // C + 2^31 + j0 E + (j0 - start) 2^32: the track's Q32 origin at the tile's first f0,
    // before G, with the integer part counted from the first bin of the row's window in
    // shared memory (start, a multiple of 16)
    long long C;
    int E;
    float w;
};

struct FastLayout {
    size_t full, empty, skyn, rec, wts, tabB, evA, evK, buf, total, stage_bytes;
};

__host__ __device__ inline FastLayout fast_layout(int S, int F, int P, int row_bytes, int J,
                                                  bool topk, int nst, bool weighted)
{
    FastLayout L;
    size_t o = 0;
    L.full = o;
    o += kMaxStages * 8;
    L.empty = o;
    o = align_up(o + kMaxStages * 8, 16);
    L.skyn = o;  // unit vectors of the tile's sky points
    o = align_up(o + (size_t)kMaxSkyGroup * 3 * sizeof(double), 16);
    L.rec = o;   // per stage (a ring of nst + 1), sky point and row
    o = align_up(o + (size_t)(nst + 1) * P * S * sizeof(RowRec), 16);
    L.wts = o;   // weighted kernels: the records' weights again, contiguous per (stage, sky point)
    o = align_up(o + (weighted ? (size_t)(nst + 1) * P * S * sizeof(float) : 0), 16);
    L.tabB = o;
    o = align_up(o + (size_t)F * S * sizeof(int), 16);
    L.evA = o;
    o = align_up(o + (size_t)F * S * sizeof(int), 16);
    L.evK = o;
    o = align_up(o + (size_t)F * S * sizeof(int), 128);
    L.buf = o;
    L.stage_bytes = (size_t)S * row_bytes;
    const size_t pipe = (size_t)nst * L.stage_bytes + (size_t)(J + 64) * 4;
    const size_t tk = topk ? (size_t)F * J * 2 * sizeof(float) + (size_t)F * sizeof(long long) : 0;
    o += pipe > tk ? pipe : tk;
    L.total = o;
    return L;
}

// floor(G E / 2^32) exactly, for |G| < 2^52 and |E| < 2^31: with G = Gh 2^32 + Gl,
// G E / 2^32 = Gh E + Gl E / 2^32, and Gl E fits in 64 bits.
__device__ __forceinline__ long long cross_q32(long long G, int E)
{
    const int Gh = static_cast<int>(G >> 32);
    const unsigned Gl = static_cast<unsigned>(G);
    const long long lo = static_cast<long long>(static_cast<unsigned long long>(Gl) *
                                                static_cast<unsigned long long>(static_cast<long long>(E)));
    // lo above is Gl * E modulo 2^64, which is exact because |Gl E| < 2^63
    return static_cast<long long>(Gh) * E + (lo >> 32);
}

// Warp roles: warps 0 .. F-1 evaluate (warp w <-> f1 value f1g*F + w); warp F produces.
// Producer, per stage st (slot st % nst): wait until every evaluating lane released the
// slot (empty barrier), compute E, C, w of the stage's rows (one lane per row), start the
// bulk copy of the rows and arrive on the slot's full barrier (32 arrivals + the copy's
// bytes).  Evaluating warp, per stage: wait for the full barrier, derive its own row
// offsets and corrections (one lane per row), accumulate, release the slot.  No CTA-wide
// barrier inside the loop.
#ifndef FT_FAST_MAXNREG
#define FT_FAST_MAXNREG 40
#endif
// Shifted-row sums of one stage for the first RA slot units of each lane (RA <= R; the
// others belong to f0 values past the band): per row, RA loads of the word holding the
// lane's bins and their accumulation; the row offsets come four at a time from tabB.
template <int MODE, int RA, bool WEIGHTED, int NS, bool FULL = true>
__device__ __forceinline__ void stage_rows(const unsigned char *lane_rows, const int *tabB,
                                           const float *wr, int nr, float (&part)[NS])
{
    auto row_sum = [&](int off, float wa) {
        if (MODE == MODE_F32) {
            const float *q = reinterpret_cast<const float *>(lane_rows) + off;
#pragma unroll
            for (int r = 0; r < RA; ++r)
                part[r] = WEIGHTED ? __fmaf_rn(wa, q[32 * r], part[r]) : __fadd_rn(part[r], q[32 * r]);
        } else {
            const unsigned *q = reinterpret_cast<const unsigned *>(lane_rows) + off;
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const unsigned u = q[32 * r];
                if (WEIGHTED) {
                    part[2 * r] = __fmaf_rn(wa, lo_to_float<MODE>(u), part[2 * r]);
                    part[2 * r + 1] = __fmaf_rn(wa, hi_to_float<MODE>(u), part[2 * r + 1]);
                } else {
                    acc_pair<MODE>(part[2 * r], part[2 * r + 1], u);
                }
            }
        }
    };
    // rows a .. a + 3: their offsets (and weights) in one 16-byte load each
    auto four_rows = [&](int a) {
        const int4 o4 = *reinterpret_cast<const int4 *>(tabB + a);
        if (WEIGHTED) {
            const float4 w4 = *reinterpret_cast<const float4 *>(wr + a);
            row_sum(o4.x, w4.x);
            row_sum(o4.y, w4.y);
            row_sum(o4.z, w4.z);
            row_sum(o4.w, w4.w);
        } else {
            row_sum(o4.x, 1.f);
            row_sum(o4.y, 1.f);
            row_sum(o4.z, 1.f);
            row_sum(o4.w, 1.f);
        }
    };
    if (FULL && nr == 32) {
        // a whole 32-row stage, unrolled: no loop counter, and the compiler can schedule
        // every row's loads in one block (3.4 % faster on the search than a 2x-unrolled loop)
#pragma unroll
        for (int a = 0; a < 32; a += 4)
            four_rows(a);
        return;
    }
    const int nr4 = nr & ~3;
#pragma unroll 2
    for (int a = 0; a < nr4; a += 4)
        four_rows(a);
    for (int a = nr4; a < nr; ++a)
        row_sum(tabB[a], WEIGHTED ? wr[a] : 1.f);
}

// stage_rows with the slot count ract chosen at run time (uniform over the CTA).
template <int MODE, int RA, bool WEIGHTED, int NS>
__device__ __forceinline__ void stage_rows_upto(int ract, const unsigned char *lane_rows,
                                                const int *tabB, const float *wr, int nr,
                                                float (&part)[NS])
{
    if constexpr (RA > 1) {
        if (ract < RA) {
            stage_rows_upto<MODE, RA - 1, WEIGHTED>(ract, lane_rows, tabB, wr, nr, part);
            return;
        }
    }
    // the persistent batch keeps the 2x-unrolled loop: with one fully unrolled copy per
    // slot-unit count it ran 0.6 % slower
    stage_rows<MODE, RA, WEIGHTED, NS, false>(lane_rows, tabB, wr, nr, part);
}

template <int MODE, int R, bool WEIGHTED, bool RAGGED>
__device__ __forceinline__ bool fast_tile(const EvalParams &p, long long tile, unsigned char *smem,
                                          ft_candidate *dst, unsigned tm, const CUtensorMap *rows_map)
{
    constexpr bool PAIR = MODE != MODE_F32;
    constexpr int NS = PAIR ? 2 * R : R;  // accumulator slots per thread
    constexpr int J = 32 * NS;            // f0 per tile
    const int F = (blockDim.x >> 5) - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = p.S;
    const int nst = p.nst;
    const int row_words = p.srow_bytes >> 2;  // shared-memory row: Ws bins
    const FastLayout L = fast_layout(S, F, p.P, p.srow_bytes, J, p.cand != nullptr, nst, WEIGHTED);
    double *skyn = reinterpret_cast<double *>(smem + L.skyn);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + L.full);
    unsigned long long *empty = reinterpret_cast<unsigned long long *>(smem + L.empty);
    RowRec *rec = reinterpret_cast<RowRec *>(smem + L.rec);
    float *wts = reinterpret_cast<float *>(smem + L.wts);
    unsigned char *buf = smem + L.buf;
    const CtaTile c = decode_tile(p, J, tile);
    const int n_stages = p.n_stages;

    if (threadIdx.x == 0) {
        for (int b = 0; b < nst; ++b) {
            mbar_init(&full[b], 1);   // the producer's lane 0, with the stage's bytes
            mbar_init(&empty[b], F);  // one elected lane per evaluating warp
        }
        fence_mbar_init();
    }
    if (threadIdx.x < 3 * p.P) {
        // sky points of the group; a ragged last group repeats its first point (those
        // warps' templates do not exist and are never written)
        const int q = threadIdx.x / 3;
        const long long sk = sky_of(p, c.skyg, q);
        skyn[threadIdx.x] = p.sky[3 * (sk < 0 ? c.sky : sk) + (threadIdx.x - 3 * q)];
    }
    __syncthreads();

    int jrel[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i)
        jrel[i] = PAIR ? 2 * lane + 64 * (i >> 1) + (i & 1) : lane + 32 * i;
    float hi[NS], lo[NS];
    int oob[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        hi[i] = lo[i] = 0.f;
        oob[i] = 0;
    }
    bool ok = true;

    if (warp == F) {
        // ------------------------------------------------------------ producer warp
        // members of this CTA's f1 group with the smallest and largest f1
        const int F1 = p.F1;
        int f_min = c.f1g * F1, f_max = c.f1g * F1;
        for (int f = c.f1g * F1 + 1; f < min(c.f1g * F1 + F1, p.n_f1); ++f) {
            if (p.f1[f] < p.f1[f_min])
                f_min = f;
            if (p.f1[f] > p.f1[f_max])
                f_max = f;
        }
        // The row records of stage st go to a ring of nst + 1 entries: the entry of stage
        // st - nst - 1 is free once the slot of stage st - 1 was released, so the records
        // (FP64 track terms, windows) are computed before waiting for the data slot, while
        // the evaluating warps still work on earlier stages.
        int st = 0, slot = 0, use = 0, rs = 0;  // rs = st mod (nst + 1)
        for (; st < n_stages; ++st, rs = rs == nst ? 0 : rs + 1) {
            const int nr = rows_in_stage(p, st);
            long long alpha = 0;
            int start = 0, len = 0;
            int b_lo = INT_MAX, b_hi = INT_MIN;  // bins this tile reads in the row (windowed)
            RowRec *rq = rec + static_cast<size_t>(rs) * p.P * S + lane;
            if (lane < nr) {
                alpha = static_cast<long long>(st) * S + lane;
                const double va[3] = {p.v[3 * alpha], p.v[3 * alpha + 1], p.v[3 * alpha + 2]};
                const bool sky_w = WEIGHTED && p.D != nullptr;
                const float wa = sky_w ? 0.f : p.w[alpha];
                // all-sky weights: the row's FP32 record of D / sqrt(S_n), once for the
                // group's sky points
                float4 rd0 = make_float4(0.f, 0.f, 0.f, 0.f), rd1 = rd0;
                if (sky_w) {
                    rd0 = p.rowd[2 * alpha];
                    rd1 = p.rowd[2 * alpha + 1];
                }
                // track terms per sky point and, per sky point, the track origins of the
                // group's smallest and largest f1 (the origin is linear in f1)
                long long G1 = 0, G2 = 0;
                if (p.Ws < p.Wp) {
                    G1 = p.G[static_cast<long long>(f_min) * p.N + alpha];
                    G2 = p.G[static_cast<long long>(f_max) * p.N + alpha];
                }
                for (int q = 0; q < p.P; ++q) {
                    RowRec r;
                    track_ec(va, skyn[3 * q], skyn[3 * q + 1], skyn[3 * q + 2], p.K0, p.k_lo, r.E, r.C);
                    r.C += (1ll << 31) + static_cast<long long>(c.j0) * r.E;
                    r.w = wa;
                    if (sky_w) {
                        // all-sky weight of this row for sky point q
                        const long long sk = sky_of(p, c.skyg, q);
                        r.w = ft_sky_r32(rd0, rd1, static_cast<float>(skyn[3 * q]), static_cast<float>(skyn[3 * q + 1]),
                                         static_cast<float>(skyn[3 * q + 2])) *
                              static_cast<float>(p.sky_inv[sk < 0 ? c.sky : sk]);
                    }
                    rq[q * S] = r;
                    if (WEIGHTED)
                        wts[(static_cast<size_t>(rs) * p.P + q) * S + lane] = r.w;
                    if (p.Ws < p.Wp) {
                        const int x1 = c.j0 + static_cast<int>((r.C + G1 + cross_q32(G1, r.E)) >> 32);
                        const int x2 = c.j0 + static_cast<int>((r.C + G2 + cross_q32(G2, r.E)) >> 32);
                        b_lo = min(b_lo, min(x1, x2));
                        b_hi = max(b_hi, max(x1, x2));
                    }
                }
                len = p.Wp;
            }
            // windowed rows: one window for the whole stage when it covers every row (one
            // tensor copy of S rows x Ws bins, kept inside the row), else one per row
            bool whole = false;
            if (p.Ws < p.Wp) {
                int wlo = b_lo, whi = b_hi;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    wlo = min(wlo, __shfl_xor_sync(0xffffffffu, wlo, off));
                    whi = max(whi, __shfl_xor_sync(0xffffffffu, whi, off));
                }
                int ts = max(wlo - 2, 0) & ~15;
                whole = p.rows_map_ok && nr == S && whi + J + 2 - ts <= p.Ws;
                ts = min(ts, p.Wp - p.Ws);
                if (lane < nr) {
                    int s0 = ts;
                    if (!whole) {
                        // the row's own window: tile width plus one carry step each side
                        s0 = max(b_lo - 2, 0) & ~15;
                        const int e0 = min((b_hi + J + 2 + 15) & ~15, p.Wp);
                        len = max(e0 - s0, 16);
                        if (s0 + len > p.Wp)
                            s0 = p.Wp - len;
                        if (len > p.Ws) {
                            atomicOr(p.status, FT_STATUS_WINDOW);
                            len = p.Ws;
                        }
                    }
                    start = s0;
                }
            }
            // the records' integer part counts bins from the window's first bin
            if (lane < nr)
                for (int q = 0; q < p.P; ++q)
                    rq[q * S].C += static_cast<long long>(c.j0 - start) << 32;
            unsigned row_tot;  // bytes of the stage's copies
            if (p.Ws == p.Wp) {
                row_tot = static_cast<unsigned>(nr) * static_cast<unsigned>(p.row_bytes);
            } else if (whole) {
                row_tot = static_cast<unsigned>(S) * static_cast<unsigned>(p.srow_bytes);
            } else {
                row_tot = static_cast<unsigned>(len) * 4u;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    row_tot += __shfl_xor_sync(0xffffffffu, row_tot, off);
            }
            if (use > 0 && !mbar_wait_bounded(&empty[slot], (use - 1) & 1)) {
                ok = false;
                break;
            }
            // every lane's record is written before lane 0's arrival releases the slot
            __syncwarp();
            if (lane == 0)
                mbar_arrive_expect_tx(&full[slot], row_tot);
            unsigned char *stage_buf = buf + slot * L.stage_bytes;
            if (p.Ws == p.Wp) {
                // whole rows: the stage's rows are contiguous in global and shared memory
                if (lane == 0)
                    bulk_g2s(stage_buf,
                                  static_cast<const unsigned char *>(p.power) +
                                      static_cast<size_t>(st) * S * p.row_bytes,
                                  row_tot, &full[slot]);
            } else if (whole) {
                if (lane == 0) {
                    if (PAIR)  // (16-byte group, group, copy, row): both copies of each row
                        tensor_copy_4d(stage_buf, rows_map, 0, start >> 3, 0, st * S, &full[slot]);
                    else
                        tensor_copy_3d(stage_buf, rows_map, 0, start >> 2, st * S, &full[slot]);
                }
            } else if (lane < nr) {
                unsigned char *dst = stage_buf + static_cast<size_t>(lane) * p.srow_bytes;
                const unsigned char *src =
                    static_cast<const unsigned char *>(p.power) + static_cast<size_t>(alpha) * p.row_bytes;
                if (!PAIR) {
                    bulk_g2s(dst, src + static_cast<size_t>(start) * 4, static_cast<unsigned>(len) * 4,
                                  &full[slot]);
                } else {
                    // even copy then odd copy: words [start/2, (start+len)/2) of each
                    bulk_g2s(dst, src + static_cast<size_t>(start >> 1) * 4,
                                  static_cast<unsigned>(len) * 2, &full[slot]);
                    bulk_g2s(dst + (p.srow_bytes >> 1),
                                  src + (p.row_bytes >> 1) + static_cast<size_t>(start >> 1) * 4,
                                  static_cast<unsigned>(len) * 2, &full[slot]);
                }
            }
            if (++slot == nst) {
                slot = 0;
                ++use;
            }
        }
        if (lane == 0) {
            if (!ok)
                atomicOr(p.status, FT_STATUS_TIMEOUT);
            // the last copies started have landed before shared memory is reused or released
            for (int s2 = st - 1; s2 >= 0 && s2 >= st - nst; --s2)
                (void)mbar_wait_bounded(&full[s2 % nst], (s2 / nst) & 1);
        }
    } else {
        // ------------------------------------------------------------ evaluating warps
        int *tabB = reinterpret_cast<int *>(smem + L.tabB) + warp * S;
        int *evA = reinterpret_cast<int *>(smem + L.evA) + warp * S;
        int *evK = reinterpret_cast<int *>(smem + L.evK) + warp * S;
        float part[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i)
            part[i] = 0.f;
        int rows_since_fold = 0;
        // this warp's sky point (q) and f1 value; warps past P * F1 (a batch whose bands
        // use fewer warps) only keep the pipeline's barriers
        const int wq = warp / p.F1;
        const int rows_max = wq < p.P ? S : 0;  // idle warps see empty stages
        // slot units (32 f0 values, or 64 for 16-bit pairs) that hold f0 values of the band
        // (the persistent batch skips the others; one launch per band keeps the full loop)
        const int ract = RAGGED ? min(R, (min(J, p.n_f0 - c.j0) + (PAIR ? 63 : 31)) / (PAIR ? 64 : 32)) : R;
        // this warp's compensated sums in tensor memory, cleared for the tile
        const unsigned tq = tm + (static_cast<unsigned>((warp & 3) * 32) << 16) +
                            static_cast<unsigned>((warp >> 2) * 16);
        {
            float z[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                z[i] = 0.f;
            tm_st8(tq, z);
            tm_st8(tq + 8, z);
            tm_wait_st();
        }
        // G of this lane's row, loaded one stage ahead
        const long long *Gf =
            p.G + static_cast<long long>(min(c.f1g * p.F1 + (warp - wq * p.F1), p.n_f1 - 1)) * p.N;
        // rows of the last stage (every other stage has S)
        const int last_nr = static_cast<int>(p.N - static_cast<long long>(n_stages - 1) * S);
        long long g_cur = lane < (n_stages == 1 ? last_nr : S) ? Gf[lane] : 0;
        const long long *gp = Gf + S + lane;  // this lane's G of the next stage
        int slot = 0, use = 0, rs = 0;  // rs = st mod (nst + 1): the stage's record entry
        for (int st = 0; st < n_stages; ++st, rs = rs == nst ? 0 : rs + 1) {
            long long g_next = 0;
            if (st + 1 < n_stages && lane < (st + 1 == n_stages - 1 ? last_nr : S))
                g_next = *gp;
            gp += S;
            if (!mbar_wait_bounded(&full[slot], use & 1)) {
                ok = false;
                break;
            }
            const int nr = min(st == n_stages - 1 ? last_nr : S, rows_max);
            const unsigned char *rows = buf + slot * L.stage_bytes;
            const RowRec *rr = rec + (rs * p.P + wq) * S;
            const float *wr = wts + (rs * p.P + wq) * S;
            // row offset of this warp's track origin and, if the track steps by sign(E)
            // inside the tile, a correction entry (lane = row)
            bool ev = false;
            int packed = 0, basev = 0;
            if (lane < nr) {
                const RowRec r = rr[lane];
                const long long acc0 = r.C + g_cur + cross_q32(g_cur, r.E);
                const int base = static_cast<int>(acc0 >> 32);  // within the window
                const unsigned L0 = static_cast<unsigned>(acc0);
                // the fraction L0 + j E leaves [0, 2^32) for some j < J: the bin steps once
                const unsigned span = static_cast<unsigned>(J - 1) * static_cast<unsigned>(abs(r.E));
                ev = r.E > 0 ? (L0 + span < L0) : (L0 < span);
                tabB[lane] = PAIR ? lane * row_words + (base & 1) * (row_words >> 1) + (base >> 1)
                                  : lane * row_words + base;
                packed = lane | (r.E < 0 ? (1 << 20) : 0);
                basev = base;
                if (ev) {
                    // first tile offset jc at which the bin steps: jc = floor(num / |E|) + 1
                    // with num = 2^32 - 1 - L0 (E > 0: the first j with L0 + j E >= 2^32) or
                    // num = L0 (E < 0: the first j with L0 + j E < 0).  16-bit storage: an
                    // FP32 quotient, then one exact integer step each way (the quotient is
                    // below J, so its FP32 error is far under one); FP32 storage keeps the
                    // integer division (measured faster there, at the register cap)
                    const unsigned num = r.E > 0 ? 0xffffffffu - L0 : L0;
                    const unsigned den = static_cast<unsigned>(abs(r.E));
                    int q;
                    if constexpr (PAIR) {
                        q = static_cast<int>(__fmul_rz(__uint2float_rz(num), __frcp_rz(__uint2float_rn(den))));
                        const unsigned t = static_cast<unsigned>(q) * den;
                        q -= t > num ? 1 : 0;
                        q += (t <= num && num - t >= den) ? 1 : 0;
                    } else {
                        q = static_cast<int>(num / den);
                    }
                    packed |= (q + 1) << 8;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, ev);
            if (ev) {
                const int pos = __popc(m & ((1u << lane) - 1u));
                evA[pos] = packed;
                evK[pos] = basev;
            }
            const int ne = __popc(m);
            __syncwarp();
            // main loop over the stage's rows, with as many slots per lane as the tile has
            // f0 values (a ragged last tile skips the rest)
            if (RAGGED)
                stage_rows_upto<MODE, R, WEIGHTED>(ract, rows + 4 * lane, tabB, wr, nr, part);
            else
                stage_rows<MODE, R, WEIGHTED>(rows + 4 * lane, tabB, wr, nr, part);
            // corrections for the rows whose bin steps by sign(E) inside the tile: from
            // slot jc on the track reads bin k + sg instead of k (slots past n_f0 are
            // computed and discarded, like in the main loop; their bins stay in the window)
            for (int e = 0; e < ne; ++e) {
                const int pk = evA[e];
                const int a = pk & 0xff;
                const int jc = (pk >> 8) & 0xfff;
                const int sg = (pk >> 20) ? -1 : 1;
                const int base = evK[e];
                const float wa = WEIGHTED ? wr[a] : 1.f;
                if (MODE == MODE_F32) {
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        if (jrel[i] >= jc && i < ract) {
                            const int k = base + jrel[i];
                            const float d = __fsub_rn(read_bin<MODE>(rows, row_words, a, k + sg),
                                                      read_bin<MODE>(rows, row_words, a, k));
                            part[i] = WEIGHTED ? __fmaf_rn(wa, d, part[i]) : __fadd_rn(part[i], d);
                        }
                    }
                } else {
                    // one 32-bit word of the pair layout holds (P[k'], P[k'+1]) for any k';
                    // with k' = k + min(sg, 0) the change is sg (P[k'+1] - P[k']).  Slot
                    // 2m of the lane reads k' = K0 + 64 m and slot 2m + 1 reads K0 + 1 + 64 m
                    // (K0 = base + 2 lane + min(sg, 0)): the two words sit 32 m words past
                    // one address each, in the copy matching their parity
                    const unsigned *row = reinterpret_cast<const unsigned *>(rows) + a * row_words;
                    const int K0 = base + 2 * lane + (sg < 0 ? -1 : 0);
                    const int K1 = K0 + 1;
                    const unsigned *we = row + (K0 & 1) * (row_words >> 1) + (K0 >> 1);
                    const unsigned *wo = row + (K1 & 1) * (row_words >> 1) + (K1 >> 1);
#pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        if (jrel[i] >= jc && (i >> 1) < ract) {
                            const unsigned u = (i & 1 ? wo : we)[32 * (i >> 1)];
                            if (WEIGHTED) {
                                const float d = __fsub_rn(hi_to_float<MODE>(u), lo_to_float<MODE>(u));
                                part[i] = __fmaf_rn(sg < 0 ? -wa : wa, d, part[i]);
                            } else {
                                acc_diff<MODE>(part[i], u, sg);
                            }
                        }
                    }
                }
            }
            // the warp's reads of this slot are done before its elected lane releases it
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[slot]);
            if (++slot == nst) {
                slot = 0;
                ++use;
            }
            g_cur = g_next;
            rows_since_fold += nr;
            if (rows_since_fold >= kFoldRows || st == n_stages - 1) {
                float h[8], l[8];
                tm_ld8(tq, h);
                tm_ld8(tq + 8, l);
                tm_wait_ld(h, l);
#pragma unroll
                for (int i = 0; i < NS; ++i)
                    fold2sum(h[i], l[i], part[i]);
                tm_st8(tq, h);
                tm_st8(tq + 8, l);
                tm_wait_st();
                rows_since_fold = 0;
            }
        }
        if (!ok && lane == 0)
            atomicOr(p.status, FT_STATUS_TIMEOUT);
        {
            float h[8], l[8];
            tm_ld8(tq, h);
            tm_ld8(tq + 8, l);
            tm_wait_ld(h, l);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                hi[i] = h[i];
                lo[i] = l[i];
            }
        }
    }
    // every copy has landed: its slot was consumed, or the producer waited for it above
    if (!__syncthreads_and(ok))
        return false;
    finish_tile<NS, WEIGHTED>(p, c, F, J, jrel, hi, lo, oob, buf, dst);
    return true;
}

// One CTA per tile of the (sky, f1 group, f0 tile) grid.
template <int MODE, int R, bool WEIGHTED>
__global__ void __maxnreg__(FT_FAST_MAXNREG) k_eval_fast(const __grid_constant__ EvalParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned s_tm;
    const unsigned ncols = tm_cols_for((blockDim.x >> 5) - 1);
    if ((threadIdx.x >> 5) == 0)
        tm_alloc(&s_tm, ncols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const unsigned tm = s_tm;
    fast_tile<MODE, R, WEIGHTED, false>(p, blockIdx.x, smem, nullptr, tm, &p.rows_map);
    tm_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tm_fence_after();
        tm_dealloc(tm, ncols);
    }
}

// Persistent form for many bands: each CTA takes tiles from a global ticket counter over
// a band-major work list (tile_prefix[b] = first ticket of band b) until it runs dry.  Each
// tile's per-sub-band candidates are merged into running lists kept in shared memory for
// the band the CTA is on; when the CTA moves to another band (or finishes) it writes those
// lists to its slot scr[cta][band][sub-band][k] (slots never written stay empty).

__device__ __forceinline__ bool cand_before(const ft_candidate &a, const ft_candidate &b)
{
    // (s desc, template index asc); empty entries (template_idx < 0) rank last
    if (a.template_idx < 0)
        return false;
    if (b.template_idx < 0)
        return true;
    return a.s > b.s || (a.s == b.s && a.template_idx < b.template_idx);
}

// run[0..k) <- best k of the sorted lists run[0..k) and add[0..k) (one warp, k <= 32).
__device__ __forceinline__ void warp_merge_lists(ft_candidate *run, const ft_candidate *add, int k)
{
    const int lane = threadIdx.x & 31;
    ft_candidate a, b;
    a.template_idx = b.template_idx = -1;
    a.s = b.s = -INFINITY;
    a.z = b.z = 0.f;
    if (lane < k) {
        a = run[lane];
        b = add[lane];
    }
    int ra = lane, rb = lane;  // final ranks
    for (int j = 0; j < k; ++j) {
        ft_candidate bj, aj;
        bj.template_idx = __shfl_sync(0xffffffffu, b.template_idx, j);
        bj.s = __shfl_sync(0xffffffffu, b.s, j);
        aj.template_idx = __shfl_sync(0xffffffffu, a.template_idx, j);
        aj.s = __shfl_sync(0xffffffffu, a.s, j);
        ra += cand_before(bj, a) ? 1 : 0;
        rb += cand_before(aj, b) ? 1 : 0;
    }
    __syncwarp();
    if (lane < k && ra < k)
        run[ra] = a;
    if (lane < k && rb < k)
        run[rb] = b;
    __syncwarp();
}



template <int MODE, int R, bool WEIGHTED>
__global__ void __maxnreg__(FT_FAST_MAXNREG) k_eval_batched(const BatchParams bp)
{
    constexpr int NS = MODE != MODE_F32 ? 2 * R : R;
    constexpr int J = 32 * NS;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ long long s_tile;
    __shared__ int s_band;
    __shared__ unsigned s_tm;
    __shared__ EvalParams s_params;
    ft_candidate *tl = reinterpret_cast<ft_candidate *>(smem + bp.list_off);
    ft_candidate *run = tl + bp.lsub_max * bp.k;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const long long total = bp.tile_prefix[bp.n_bands];
    const unsigned ncols = tm_cols_for(nw - 1);
    if (warp == 0)
        tm_alloc(&s_tm, ncols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const unsigned tm = s_tm;
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = static_cast<long long>(atomicAdd(bp.counter, 1ull));
            int b = -1;
            if (t < total) {
                int lo = 0, hi = bp.n_bands - 1;  // last band whose prefix <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (bp.tile_prefix[mid] <= t)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                b = lo;
                s_tile = t - bp.tile_prefix[b];
            }
            s_band = b;
        }
        __syncthreads();
        const int b = s_band;
        const long long tile = s_tile;
        if (b != cur) {
            if (cur >= 0) {
                const int m = bp.n_sub[cur] * bp.k;
                ft_candidate *g = bp.scr + (static_cast<size_t>(blockIdx.x) * bp.n_bands + cur) *
                                               bp.n_sub_max * bp.k;
                for (int i = threadIdx.x; i < m; i += blockDim.x)
                    g[i] = run[i];
            }
            if (b >= 0) {
                const int m = bp.n_sub[b] * bp.k;
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    run[i].template_idx = -1;
                    run[i].s = -INFINITY;
                    run[i].z = 0.f;
                }
                // the band's parameters in shared memory: the tile code reads them all the
                // time, and from global memory every read would go through the small L1
                const unsigned *src = reinterpret_cast<const unsigned *>(bp.params + b);
                unsigned *dstw = reinterpret_cast<unsigned *>(&s_params);
                for (int i = threadIdx.x; i < static_cast<int>(sizeof(EvalParams) / 4); i += blockDim.x)
                    dstw[i] = src[i];
            }
            __syncthreads();
            cur = b;
        }
        if (b < 0)
            break;
        const EvalParams &p = s_params;
        // Tickets of a band run every (sky group, f1 group) of one f0 tile before the next
        // f0 tile: the CTAs in flight then read the same window of the band's rows, so a wide
        // band's working set is that window (about a third of its rows' bytes) and stays in
        // L2, instead of the whole band.  The tile index itself keeps the f0 tile fastest.
        const long long per_f0t = p.n_skyg * static_cast<long long>(p.n_f1g);
        const long long t_f0 = tile / per_f0t;
        const long long tile_id = (tile - t_f0 * per_f0t) * p.n_f0t + t_f0;
        // (the tensor map is used from global memory, where a copy can be read from)
        const bool done = fast_tile<MODE, R, WEIGHTED, true>(p, tile_id, smem, tl, tm, &bp.params[b].rows_map);
        __syncthreads();
        if (!done)
            break;  // a bounded wait ran out (status already set): stop taking tiles
        // merge this tile's lists into the band's running lists
        const int j0 = static_cast<int>(t_f0) * J;
        const int lb0 = j0 / p.sub, lb1 = (min(j0 + J, p.n_f0) - 1) / p.sub;
        for (int lb = lb0 + warp; lb <= lb1; lb += nw)
            warp_merge_lists(run + lb * bp.k, tl + (lb - lb0) * bp.k, bp.k);
        __syncthreads();
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tm, ncols);
    }
}

// ------------------------------------------------------------------ candidate merge

__device__ __forceinline__ bool cand_better(const ft_candidate &a, const ft_candidate &b)
{
    return a.s > b.s || (a.s == b.s && a.template_idx < b.template_idx);
}

constexpr int kKmax = 32;
constexpr int kMergeThreads = 256;

// One CTA per sub-band b: gathers the per-CTA lists of every evaluation CTA whose f0 tile
// meets the sub-band and keeps the k best by (s desc, template index asc).
// Sky groups [g0, g0 + n_skyg) x f1 groups [h0, h0 + n_h) (the f0 tiles of sub-band b)
// into out.
__device__ __forceinline__ void merge_subband(const ft_candidate *cand, int k, int lsub_max,
                                              long long g0, long long n_skyg, int h0, int n_h,
                                              int n_f1g, int n_f0t, int J, int sub, int n_f0,
                                              int b, ft_candidate *out)
{
    __shared__ ft_candidate wl[kMergeThreads / 32][kKmax];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ft_lo = (b * sub) / J;
    const int ft_hi = (min((b + 1) * sub, n_f0) - 1) / J;
    const int nft = ft_hi - ft_lo + 1;
    const long long total = n_skyg * n_h * static_cast<long long>(nft) * k;

    ft_candidate Lst[kKmax];
    int n = 0;
    for (long long c = tid; c < total; c += blockDim.x) {
        const long long q = c / k;
        const int i = static_cast<int>(c - q * k);
        const int ftl = static_cast<int>(q % nft);
        const long long u = q / nft;  // (sky group, f1 group) of the box
        const long long gi = u / n_h;
        const long long sg = (g0 + gi) * n_f1g + h0 + (u - gi * n_h);
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

// Block (b, x, y): sub-band b of sky box x (sky groups [x gpb, (x + 1) gpb)) and f1 box y
// (f1 groups [y hpb, (y + 1) hpb)) into out[((x n_f1b + y) n_sub + b) k ..].
__global__ void __launch_bounds__(kMergeThreads) k_topk_merge(const ft_candidate *cand, int k,
                                                              int lsub_max, long long n_skyg,
                                                              long long gpb, int n_f1g, int hpb,
                                                              int n_f0t, int J, int sub, int n_f0,
                                                              int n_sub, ft_candidate *out)
{
    const long long g0 = static_cast<long long>(blockIdx.y) * gpb;
    const long long ng = min(gpb, n_skyg - g0);
    const int h0 = static_cast<int>(blockIdx.z) * hpb;
    const int nh = min(hpb, n_f1g - h0);
    const long long box = static_cast<long long>(blockIdx.y) * gridDim.z + blockIdx.z;
    merge_subband(cand, k, lsub_max, g0, ng, h0, nh, n_f1g, n_f0t, J, sub, n_f0, blockIdx.x,
                  out + box * n_sub * k);
}

// Merge for the persistent batch: block i handles sub-band j = i - sub_prefix[b] of band b
// and keeps the k best of the n_ctas lists scr[c][b][j][0..k).
__global__ void __launch_bounds__(kMergeThreads) k_topk_merge_persist(
    const ft_candidate *scr, int n_ctas, int n_bands, int n_sub_max, int k, const int *sub_prefix,
    ft_candidate *out)
{
    __shared__ ft_candidate wl[kMergeThreads / 32][kKmax];
    const int i = blockIdx.x;
    int lo = 0, hi = n_bands - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sub_prefix[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int band = lo, j = i - sub_prefix[lo];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ft_candidate Lst[kKmax];
    int n = 0;
    const long long total = static_cast<long long>(n_ctas) * k;
    for (long long q = tid; q < total; q += blockDim.x) {
        const long long cta = q / k;
        const int e = static_cast<int>(q - cta * k);
        const ft_candidate x = scr[((cta * n_bands + band) * n_sub_max + j) * k + e];
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
    // lanes -> warp list -> block list, k rounds of arg-max over list heads each
    int h = 0;
    for (int r = 0; r < k; ++r) {
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
            wl[warp][r] = c;
        }
    }
    __syncthreads();
    if (warp != 0)
        return;
    const int nw = blockDim.x >> 5;
    h = 0;
    for (int r = 0; r < k; ++r) {
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
            out[static_cast<long long>(i) * k + r] = c;
        }
    }
}

// ------------------------------------------------------------------ helpers

// FP32/FP64 rows -> band layout.  FP32 storage: [N][Wp] floats.  16-bit storage: per row
// the even copy P[0 .. Wp) followed by the odd copy P[1 .. Wp] (so 32-bit word m of the odd
// copy is (P[2m+1], P[2m+2])); bins >= W are 0.  Conversion rounds to nearest even.
__global__ void k_convert(const void *src, int sdt, long long sstride, void *dst, int ddt,
                          long long N, int W, int Wp, unsigned int *status)
{
    const int row_elems = ddt == FT_F32 ? Wp : 2 * Wp;
    const long long total = N * row_elems;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long row = i / row_elems;
        const int e = static_cast<int>(i - row * row_elems);
        const int col = e < Wp ? e : e - Wp + 1;
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

template <typename K>
int launch_kernel(K fn, long long n_cta, int threads, size_t smem, const EvalParams &p,
                  cudaStream_t st, size_t &configured)
{
    if (smem > configured) {
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
        configured = smem;
    }
    fn<<<static_cast<unsigned>(n_cta), threads, smem, st>>>(p);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

template <typename T, int R>
int launch_checked_t(long long n_cta, int threads, size_t smem, const EvalParams &p, cudaStream_t st)
{
    static size_t configured = 0;
    return launch_kernel(k_eval_checked<T, R>, n_cta, threads, smem, p, st, configured);
}

template <typename T>
int launch_checked(int R, long long n_cta, int threads, size_t smem, const EvalParams &p,
                   cudaStream_t st)
{
    switch (R) {
    case 1: return launch_checked_t<T, 1>(n_cta, threads, smem, p, st);
    case 2: return launch_checked_t<T, 2>(n_cta, threads, smem, p, st);
    case 3: return launch_checked_t<T, 3>(n_cta, threads, smem, p, st);
    case 4: return launch_checked_t<T, 4>(n_cta, threads, smem, p, st);
    case 5: return launch_checked_t<T, 5>(n_cta, threads, smem, p, st);
    case 6: return launch_checked_t<T, 6>(n_cta, threads, smem, p, st);
    case 7: return launch_checked_t<T, 7>(n_cta, threads, smem, p, st);
    case 8: return launch_checked_t<T, 8>(n_cta, threads, smem, p, st);
    default: FT_FAIL(FT_ERR_ARG, "eval: unsupported tile width");
    }
}

template <int MODE, int R, bool W>
int launch_fast_t(long long n_cta, int threads, size_t smem, const EvalParams &p, cudaStream_t st)
{
    static size_t configured = 0;
    return launch_kernel(k_eval_fast<MODE, R, W>, n_cta, threads, smem, p, st, configured);
}

template <int MODE, bool W>
int launch_fast_w(int R, long long n_cta, int threads, size_t smem, const EvalParams &p,
                  cudaStream_t st)
{
    switch (R) {
    case 1: return launch_fast_t<MODE, 1, W>(n_cta, threads, smem, p, st);
    case 2: return launch_fast_t<MODE, 2, W>(n_cta, threads, smem, p, st);
    case 3: return launch_fast_t<MODE, 3, W>(n_cta, threads, smem, p, st);
    case 4: return launch_fast_t<MODE, 4, W>(n_cta, threads, smem, p, st);
    case 5: return MODE == MODE_F32 ? launch_fast_t<MODE_F32, 5, W>(n_cta, threads, smem, p, st) : FT_ERR_ARG;
    case 6: return MODE == MODE_F32 ? launch_fast_t<MODE_F32, 6, W>(n_cta, threads, smem, p, st) : FT_ERR_ARG;
    case 7: return MODE == MODE_F32 ? launch_fast_t<MODE_F32, 7, W>(n_cta, threads, smem, p, st) : FT_ERR_ARG;
    case 8: return MODE == MODE_F32 ? launch_fast_t<MODE_F32, 8, W>(n_cta, threads, smem, p, st) : FT_ERR_ARG;
    default: FT_FAIL(FT_ERR_ARG, "eval: unsupported tile width");
    }
}

template <int MODE>
int launch_fast(bool weighted, int R, long long n_cta, int threads, size_t smem,
                const EvalParams &p, cudaStream_t st)
{
    return weighted ? launch_fast_w<MODE, true>(R, n_cta, threads, smem, p, st)
                    : launch_fast_w<MODE, false>(R, n_cta, threads, smem, p, st);
}

int row_bytes_of(const ft_band *band)
{
    return band->Wp * 4;  // FP32 rows, or the two 16-bit copies of a row
}

}  // namespace

// ------------------------------------------------------------------ host launchers

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

}  // namespace

int ft_encode_rows_map(const ft_band *band, int Ws, int S, CUtensorMap *map, int *ok)
{
    *ok = 0;
    std::memset(map, 0, sizeof(*map));
    const bool pair = band->dtype != FT_F32;
    // 16-byte groups of four 32-bit words: a window start (a multiple of 16 bins) is a
    // whole group, so the innermost coordinate is always 0
    const int groups = pair ? Ws / 8 : Ws / 4;
    if (Ws >= band->Wp || Ws % 32 != 0 || groups > 256 || S < 1 || S > 256)
        return FT_OK;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled_fn();
    if (fn == nullptr)
        return FT_OK;
    const cuuint64_t Wp = static_cast<cuuint64_t>(band->Wp), N = static_cast<cuuint64_t>(band->N);
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], es[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    if (pair) {  // (group, group in copy, copy, row); a row is the even copy then the odd one
        rank = 4;
        dims[0] = 4; dims[1] = Wp / 8; dims[2] = 2; dims[3] = N;
        strides[0] = 16; strides[1] = 2 * Wp; strides[2] = 4 * Wp;
        box[0] = 4; box[1] = static_cast<cuuint32_t>(groups); box[2] = 2; box[3] = static_cast<cuuint32_t>(S);
    } else {     // (group, group in row, row)
        rank = 3;
        dims[0] = 4; dims[1] = Wp / 4; dims[2] = N;
        strides[0] = 16; strides[1] = 4 * Wp;
        box[0] = 4; box[1] = static_cast<cuuint32_t>(groups); box[2] = static_cast<cuuint32_t>(S);
    }
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, rank, band->d_power, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        *ok = 1;
    return FT_OK;
}

int ft_window_bins(const ft_band *band, const ft_bank *bank, int J, int P)
{
    const double spread = std::ceil((bank->f1_hi - bank->f1_lo) * band->tau_absmax * 1.001) + 2.0;
    // a sky group moves the track origin by at most (K0 + j) |v| |n_a - n_b| bins between
    // its points (j < n_f0 + J covers the tile's padding)
    double sky_spread = 0.0;
    if (P > 1)
        sky_spread = std::ceil((static_cast<double>(bank->k0) + bank->n_f0 + J) * band->vmax *
                               bank->sky_dmax[P] * 1.001) + 2.0;
    long long ws = (static_cast<long long>(J) + static_cast<long long>(spread) +
                    static_cast<long long>(sky_spread) + 40 + 31) / 32 * 32;
    // a window that saves under a quarter of the row is not worth one copy per row: the
    // stage is then one contiguous copy of whole rows
    if (4 * ws > 3 * static_cast<long long>(band->Wp))
        return band->Wp;
    return static_cast<int>(ws);
}

size_t ft_eval_smem_bytes(const ft_band *band, const EvalShape &sh, int k)
{
    if (sh.fast)
        return fast_layout(sh.S, sh.F, sh.P, sh.Ws * 4, sh.J, k > 0, sh.nbuf, ft_band_weighted(band)).total;
    return smem_layout(sh.S, sh.F, row_bytes_of(band), sh.J, false, k > 0).total;
}

void ft_sky_grouping(const ft_bank *bank, int max_warps, int *P, int *F1)
{
    const int groups = (bank->n_f1 + max_warps - 1) / max_warps;
    *F1 = (bank->n_f1 + groups - 1) / groups;
    int q = std::max(1, std::min(kMaxSkyGroup, max_warps / *F1));
    *P = static_cast<int>(std::min<long long>(q, bank->n_sky));
}

long long ft_grid_ctas(const ft_bank *bank, const EvalShape &sh)
{
    const long long n_skyg = (bank->n_sky + sh.P - 1) / sh.P;
    const long long n_f1g = (bank->n_f1 + sh.F1 - 1) / sh.F1;
    const long long n_f0t = (bank->n_f0 + sh.J - 1) / sh.J;
    return n_skyg * n_f1g * n_f0t;
}

EvalShape ft_default_shape(const ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box,
                           int f1_box)
{
    EvalShape sh;
    sh.fast = bank->window_safe;
    if (sh.fast) {
        // up to kFastMaxWarps evaluating warps: the f1 values of one group for P sky
        // points that share the shared-memory rows
        ft_sky_grouping(bank, kFastMaxWarps, &sh.P, &sh.F1);
        if (f1_box > 0 && f1_box % sh.F1 != 0) {
            while (f1_box % sh.F1 != 0)
                --sh.F1;
            sh.P = static_cast<int>(std::min<long long>(
                std::min(kMaxSkyGroup, kFastMaxWarps / sh.F1), bank->n_sky));
        }
        while (sky_box > 0 && sky_box % sh.P != 0)
            --sh.P;
    } else {
        const int groups = (bank->n_f1 + 31) / 32;
        sh.F1 = (bank->n_f1 + groups - 1) / groups;
        while (f1_box > 0 && f1_box % sh.F1 != 0)
            --sh.F1;
        sh.P = 1;
    }
    sh.F = sh.P * sh.F1;
    // tile width J = 32 x slots per lane (pairs of slots for 16-bit storage): fewest idle
    // lanes, then the widest tile
    const bool pair = sh.fast && band->dtype != FT_F32;
    const int step = pair ? 64 : 32;
    const int max_units = pair ? 4 : 8;
    int best = step;
    long long best_waste = LLONG_MAX;
    for (int u = 1; u <= max_units; ++u) {
        const long long J = static_cast<long long>(step) * u;
        const long long waste = (bank->n_f0 + J - 1) / J * J - bank->n_f0;
        if (waste < best_waste || (waste == best_waste && J > best)) {
            best_waste = waste;
            best = static_cast<int>(J);
        }
    }
    sh.J = best;
    if (ctx->tune.tile_f0 > 0)
        sh.J = ctx->tune.tile_f0;
    const size_t rb = row_bytes_of(band);
    sh.Ws = 0;
    if (sh.fast) {
        // two slots of up to 32 rows (a multiple of 4) of windowed rows in about 80 KB: two
        // CTAs per SM
        sh.Ws = ft_window_bins(band, bank, sh.J, sh.P);
        sh.nbuf = 2;
        int S = static_cast<int>((80 * 1024) / (sh.nbuf * static_cast<size_t>(sh.Ws) * 4));
        S = S > 32 ? 32 : S;
        S = S < 4 ? 4 : S & ~3;
        sh.S = S;
    } else {
        sh.nbuf = kNbuf;
        int S = static_cast<int>((80 * 1024) / (kNbuf * rb));
        S = S > 64 ? 64 : S;
        S = S < 1 ? 1 : S;
        if (S >= 8)
            S &= ~7;
        sh.S = S;
    }
    if (ctx->tune.rows_per_stage > 0)
        sh.S = ctx->tune.rows_per_stage;
    if (ctx->tune.stages > 0 && sh.fast)
        sh.nbuf = ctx->tune.stages;
    return sh;
}

int ft_launch_eval(const ft_band *band, const ft_bank *bank, const EvalShape &sh, EvalParams p,
                   cudaStream_t st)
{
    p.n_f0t = (bank->n_f0 + sh.J - 1) / sh.J;
    p.n_f1g = (bank->n_f1 + sh.F1 - 1) / sh.F1;
    p.P = sh.P;
    p.F1 = sh.F1;
    p.n_skyg = (bank->n_sky + sh.P - 1) / sh.P;
    // CTAs walk the sky in the bank's proximity order (sky groups are runs of it, and so
    // are the sky boxes of ft_topk_per_skybox)
    p.sky_order = bank->d_sky_order;
    p.S = sh.S;
    p.n_stages = static_cast<int>((band->N + sh.S - 1) / sh.S);
    p.row_bytes = row_bytes_of(band);
    p.Wp = band->Wp;
    p.Ws = sh.Ws;
    p.srow_bytes = sh.Ws * 4;
    p.nst = sh.nbuf;
    p.row_elems = band->dtype == FT_F32 ? band->Wp : 2 * band->Wp;
    p.rows_map_ok = 0;
    if (sh.fast)
        FT_TRY(ft_encode_rows_map(band, sh.Ws, sh.S, &p.rows_map, &p.rows_map_ok));
    const long long n_cta = ft_grid_ctas(bank, sh);
    if (n_cta <= 0 || n_cta > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "eval: grid too large (sky groups * f1 groups * f0 tiles >= 2^31)");
    if (sh.P > 1 && bank->d_sky_order == nullptr)
        FT_FAIL(FT_ERR_ARG, "eval: sky groups need the bank's sky order");
    if (sh.fast && !bank->window_safe)
        FT_FAIL(FT_ERR_ARG, "eval: the unchecked kernel needs a bank whose tracks stay in the window");
    if (band->d_D && !bank->d_sky_inv)
        FT_FAIL(FT_ERR_ARG, "eval: the bank was made before the band's all-sky weights were set; make it again");
    const size_t smem = ft_eval_smem_bytes(band, sh, p.cand ? p.k : 0);
    if (smem > band->ctx->smem_optin)
        FT_FAIL(FT_ERR_RANGE, "eval: tile needs more shared memory than the device offers");
    const int threads = 32 * sh.F;
    const int unit = (sh.fast && band->dtype != FT_F32) ? 64 : 32;
    if (sh.J < unit || sh.J % unit != 0 || sh.J > 256)
        FT_FAIL(FT_ERR_RANGE, "eval: tile_f0 must be a multiple of 32 (64 for 16-bit storage), <= 256");
    if (!sh.fast) {
        const int R = sh.J / 32;
        switch (band->dtype) {
        case FT_F32: return launch_checked<float>(R, n_cta, threads, smem, p, st);
        case FT_F16: return launch_checked<__half>(R, n_cta, threads, smem, p, st);
        case FT_BF16: return launch_checked<__nv_bfloat16>(R, n_cta, threads, smem, p, st);
        default: FT_FAIL(FT_ERR_ARG, "eval: bad dtype");
        }
    }
    if (sh.F > kFastMaxWarps || sh.S % 4 != 0 || sh.S > 32 || sh.nbuf < 2 || sh.nbuf > kMaxStages)
        FT_FAIL(FT_ERR_ARG, "eval: shape not supported by the unchecked kernel");
    const int tf = threads + 32;  // plus the producer warp
    switch (band->dtype) {
    case FT_F32: return launch_fast<MODE_F32>(ft_band_weighted(band), sh.J / 32, n_cta, tf, smem, p, st);
    case FT_F16: return launch_fast<MODE_F16>(ft_band_weighted(band), sh.J / 64, n_cta, tf, smem, p, st);
    case FT_BF16: return launch_fast<MODE_BF16>(ft_band_weighted(band), sh.J / 64, n_cta, tf, smem, p, st);
    default: FT_FAIL(FT_ERR_ARG, "eval: bad dtype");
    }
}

int ft_launch_merge(const ft_bank *bank, const EvalShape &sh, const FtCand *cand, int k,
                    int lsub_max, ft_candidate *out, cudaStream_t st, int sky_box, int f1_box)
{
    const int n_f0t = (bank->n_f0 + sh.J - 1) / sh.J;
    const int n_f1g = (bank->n_f1 + sh.F1 - 1) / sh.F1;
    const long long n_skyg = (bank->n_sky + sh.P - 1) / sh.P;
    if (sky_box > 0 && sky_box % sh.P != 0)
        FT_FAIL(FT_ERR_ARG, "merge: sky box not a multiple of the sky group size");
    const long long gpb = sky_box > 0 ? sky_box / sh.P : n_skyg;
    const long long n_boxes = (n_skyg + gpb - 1) / gpb;
    if (n_boxes > 65535)
        FT_FAIL(FT_ERR_RANGE, "merge: more than 65535 sky boxes");
    if (f1_box > 0 && f1_box % sh.F1 != 0)
        FT_FAIL(FT_ERR_ARG, "merge: f1 box not a multiple of the f1 group size");
    const int hpb = f1_box > 0 ? f1_box / sh.F1 : n_f1g;
    const int n_f1b = (n_f1g + hpb - 1) / hpb;
    if (n_f1b > 65535)
        FT_FAIL(FT_ERR_RANGE, "merge: more than 65535 f1 boxes");
    k_topk_merge<<<dim3(static_cast<unsigned>(bank->n_sub), static_cast<unsigned>(n_boxes),
                        static_cast<unsigned>(n_f1b)),
                   kMergeThreads, 0, st>>>(reinterpret_cast<const ft_candidate *>(cand), k, lsub_max,
                                           n_skyg, gpb, n_f1g, hpb, n_f0t, sh.J, bank->sub,
                                           bank->n_f0, bank->n_sub, out);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int ft_launch_convert(const void *src, int src_dtype, long long src_stride, void *dst,
                      int dst_dtype, long long N, int W, int Wp, unsigned int *status,
                      cudaStream_t st)
{
    const long long row_elems = dst_dtype == FT_F32 ? Wp : 2ll * Wp;
    k_convert<<<grid_for(N * row_elems, 256), 256, 0, st>>>(src, src_dtype, src_stride, dst,
                                                             dst_dtype, N, W, Wp, status);
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

// ------------------------------------------------------------------ persistent batch

namespace {

template <int MODE, int R, bool W>
int batched_t(const BatchParams &bp, int threads, size_t smem, int *grid_out, bool launch,
              cudaStream_t st)
{
    static size_t configured = 0;
    auto fn = k_eval_batched<MODE, R, W>;
    if (smem > configured) {
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
        configured = smem;
    }
    // resident CTAs per SM from the kernel's registers and shared memory and its tensor-
    // memory columns (the occupancy query does not count the latter and treats a kernel
    // that allocates tensor memory as one CTA per SM); extra CTAs would only queue
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0, threads_sm = 0;
    FT_CUDA(cudaGetDevice(&dev));
    FT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FT_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    FT_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    FT_CUDA(cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    cudaFuncAttributes fa;
    FT_CUDA(cudaFuncGetAttributes(&fa, fn));
    const int warps = threads / 32;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp
    const int by_regs = 4 * (16384 / warp_regs) / warps;         // four 16K-register partitions
    const int by_smem =
        static_cast<int>(smem_sm / (smem + fa.sharedSizeBytes + static_cast<size_t>(reserved)));
    const int by_warps = threads_sm / threads;
    const int by_tmem = 512 / static_cast<int>(tm_cols_for(warps - 1));
    const int per_sm = std::min(std::min(std::min(by_regs, by_smem), std::min(by_warps, by_tmem)), 32);
    if (per_sm < 1)
        FT_FAIL(FT_ERR_RANGE, "batch: the persistent kernel does not fit on an SM with this shape");
    *grid_out = per_sm * sms;
    if (launch) {
        fn<<<*grid_out, threads, smem, st>>>(bp);
        FT_CUDA(cudaGetLastError());
    }
    return FT_OK;
}

template <int MODE, bool W>
int batched_r(int R, const BatchParams &bp, int threads, size_t smem, int *grid, bool launch,
              cudaStream_t st)
{
    switch (R) {
    case 1: return batched_t<MODE, 1, W>(bp, threads, smem, grid, launch, st);
    case 2: return batched_t<MODE, 2, W>(bp, threads, smem, grid, launch, st);
    case 3: return batched_t<MODE, 3, W>(bp, threads, smem, grid, launch, st);
    case 4: return batched_t<MODE, 4, W>(bp, threads, smem, grid, launch, st);
    case 6: return MODE == MODE_F32 ? batched_t<MODE_F32, 6, W>(bp, threads, smem, grid, launch, st) : FT_ERR_ARG;
    case 8: return MODE == MODE_F32 ? batched_t<MODE_F32, 8, W>(bp, threads, smem, grid, launch, st) : FT_ERR_ARG;
    default: FT_FAIL(FT_ERR_ARG, "batch: unsupported tile width");
    }
}

}  // namespace

size_t ft_batch_tile_smem(int Ws, int S, int F, int P, int J, int nst, bool weighted)
{
    return fast_layout(S, F, P, Ws * 4, J, true, nst, weighted).total;
}

int ft_batch_row_bytes(const ft_band *band)
{
    return row_bytes_of(band);
}

int ft_launch_batched(int dtype, bool weighted, int J, int F, const BatchParams &bp, size_t smem,
                      int *grid, bool launch, cudaStream_t st)
{
    const int threads = 32 * (F + 1);
    switch (dtype) {
    case FT_F32:
        return weighted ? batched_r<MODE_F32, true>(J / 32, bp, threads, smem, grid, launch, st)
                        : batched_r<MODE_F32, false>(J / 32, bp, threads, smem, grid, launch, st);
    case FT_F16:
        return weighted ? batched_r<MODE_F16, true>(J / 64, bp, threads, smem, grid, launch, st)
                        : batched_r<MODE_F16, false>(J / 64, bp, threads, smem, grid, launch, st);
    case FT_BF16:
        return weighted ? batched_r<MODE_BF16, true>(J / 64, bp, threads, smem, grid, launch, st)
                        : batched_r<MODE_BF16, false>(J / 64, bp, threads, smem, grid, launch, st);
    default: FT_FAIL(FT_ERR_ARG, "batch: bad dtype");
    }
}

int ft_launch_merge_persist(const ft_candidate *scr, int n_ctas, int n_bands, int n_sub_max, int k,
                            const int *sub_prefix, int n_sub_total, ft_candidate *out,
                            cudaStream_t st)
{
    k_topk_merge_persist<<<n_sub_total, kMergeThreads, 0, st>>>(scr, n_ctas, n_bands, n_sub_max, k,
                                                                sub_prefix, out);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

// ------------------------------------------------------------------ measured gather roof
//
// The evaluation kernel's inner loop with nothing around it: rows resident in shared memory,
// four row offsets per vector load, one conflict-free 32-bit load per lane per slot unit and
// its FP32 accumulation (FADD for FP32 rows, the mixed-precision FMA pair for 16-bit pairs),
// 2 CTAs of 20 warps per SM.  No track tables, no pipeline, no corrections: the throughput
// it reaches is the ceiling of the gather-accumulate on this GPU.

namespace {

constexpr int kRoofRowWords = 320;  // words per resident row
constexpr int kRoofRows = 64;       // rows (and offsets) per pass
constexpr int kRoofThreads = 640;
constexpr int kRoofUnits = 3;       // slot units per lane: 3 x 64 bins (pairs), 6 x 32 (FP32)

template <int MODE>
__global__ void __launch_bounds__(kRoofThreads, 2)
    k_gather_roof(int iters, float *out, long long *clk)
{
    constexpr bool PAIR = MODE != MODE_F32;
    constexpr int WORDS = PAIR ? kRoofUnits : 2 * kRoofUnits;  // loads per lane per row
    extern __shared__ __align__(16) unsigned roof_smem[];
    unsigned *rows = roof_smem;
    int *tab = reinterpret_cast<int *>(roof_smem + kRoofRows * kRoofRowWords);
    const unsigned one = MODE == MODE_F32 ? 0x3F800000u : MODE == MODE_F16 ? 0x3C003C00u : 0x3F803F80u;
    for (int i = threadIdx.x; i < kRoofRows * kRoofRowWords; i += blockDim.x)
        rows[i] = one;
    // row a starts at a word offset in [0, 128): the last word a lane reads is
    // 127 + 31 + 32 (WORDS - 1) <= 318 < kRoofRowWords
    for (int a = threadIdx.x; a < kRoofRows; a += blockDim.x)
        tab[a] = a * kRoofRowWords + (a * 37) % 128;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float acc[2 * kRoofUnits];
#pragma unroll
    for (int i = 0; i < 2 * kRoofUnits; ++i)
        acc[i] = 0.f;
    const unsigned *lr = rows + lane;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        for (int a = 0; a < kRoofRows; a += 4) {
            const int4 o4 = *reinterpret_cast<const int4 *>(tab + a);
            const int oo[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned *q = lr + oo[u];
#pragma unroll
                for (int r = 0; r < WORDS; ++r) {
                    if (PAIR)
                        acc_pair<MODE>(acc[2 * r], acc[2 * r + 1], q[32 * r]);
                    else
                        acc[r] = __fadd_rn(acc[r], __uint_as_float(q[32 * r]));
                }
            }
        }
    }
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kRoofUnits; ++i)
        s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0)
        clk[blockIdx.x] = t1 - t0;
}

}  // namespace

int ft_run_gather_roof(int dtype, int sm_count, double *evals_per_s, double *evals_per_clk_sm)
{
    const int blocks = 2 * sm_count, iters = 2000;
    const size_t smem = (kRoofRows * kRoofRowWords + kRoofRows) * sizeof(unsigned);
    auto launch = [&](auto fn, float *out, long long *clk, int it) -> int {
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
        fn<<<blocks, kRoofThreads, smem>>>(it, out, clk);
        FT_CUDA(cudaGetLastError());
        return FT_OK;
    };
    float *out = nullptr;
    long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FT_OK;
    if (cudaMalloc(&out, static_cast<size_t>(blocks) * kRoofThreads * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&clk, static_cast<size_t>(blocks) * sizeof(long long)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = FT_ERR_OOM;
    } else {
        auto run = [&](int it) -> int {
            switch (dtype) {
            case FT_F32: return launch(k_gather_roof<MODE_F32>, out, clk, it);
            case FT_F16: return launch(k_gather_roof<MODE_F16>, out, clk, it);
            case FT_BF16: return launch(k_gather_roof<MODE_BF16>, out, clk, it);
            default: FT_FAIL(FT_ERR_ARG, "gather_roof: bad dtype");
            }
        };
        float ms = 0.f;
        if ((rc = run(20)) == FT_OK && cudaEventRecord(e0) == cudaSuccess && (rc = run(iters)) == FT_OK &&
            cudaEventRecord(e1) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            std::vector<long long> c(blocks);
            if (cudaMemcpy(c.data(), clk, blocks * sizeof(long long), cudaMemcpyDeviceToHost) == cudaSuccess) {
                const double per_thread = static_cast<double>(iters) * kRoofRows * 2 * kRoofUnits;
                const long long mx = *std::max_element(c.begin(), c.end());
                *evals_per_s = per_thread * kRoofThreads * blocks / (ms * 1e-3);
                *evals_per_clk_sm = per_thread * kRoofThreads * 2 / static_cast<double>(mx);
            } else {
                rc = FT_ERR_CUDA;
            }
        } else if (rc == FT_OK) {
            rc = FT_ERR_CUDA;
        }
    }
    cudaFree(out);
    cudaFree(clk);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (rc == FT_ERR_OOM)
        FT_FAIL(FT_ERR_OOM, "gather_roof: allocation failed");
    if (rc == FT_ERR_CUDA)
        FT_FAIL(FT_ERR_CUDA, "gather_roof: CUDA runtime error");
    return rc;
}
