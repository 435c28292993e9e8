// ft_binary.cu -- the binary-orbit track (Eq. (track) with the orbit term) over a random
// template bank in uniform coordinates (Sec. IV.A, App. A), cut into hyperboxes (Sec. IV.B).
//
// Templates are never stored: every thread derives its templates (kBtTPT of them, sharing
// each row's records) from Philox counters and keeps the per-template terms of the canonical
// bin rule in registers.  Each CTA evaluates up to kBtThreads templates of one box over all
// SFTs; stages of S SFT rows (power row, FP32 velocity + weight, fixed-point time) are brought
// into shared memory by bulk copies on two mbarrier-tracked buffers.  Per (template, SFT) the
// work is integer phase arithmetic, a table cosine, the bin, one shared-memory read and one
// add: the kernel is bound by instruction issue and shared-memory reads, not by HBM.  Every floating-point operation of the rule is an
// explicit round-to-nearest intrinsic so that the compiler cannot contract or reorder it.

#include "ft_internal.cuh"
#include "ft_ptx.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

struct ft_binary_bank {
    ft_ctx *ctx = nullptr;
    int device = 0;
    const ft_band *band = nullptr;
    ft_binary_bank_desc desc{};
    long long n_templates = 0, n_boxes = 0;
    double xlo[6] = {}, step[6] = {};
    int n_pad = 0;                 // rows of d_rowv / d_tq (N rounded up to kBtRowPad)
    float4 *d_rowv = nullptr;      // [n_pad] (v/c as FP32, weight); zero beyond N
    long long *d_tq = nullptr;     // [n_pad] round((t_mid - t0) 2^10)
    float2 *d_costab = nullptr;    // [kBtTab + 1] full-turn cosine table (value, difference)
    // all-sky weights (band with detector tensors): per SFT D / sqrt(S_n) in FP32 as
    // (D00, D01, D02, D11), (D12, D22, |D|^2, tr D); zero beyond N
    float4 *d_rowd = nullptr;      // [n_pad][2]
};

namespace {

constexpr int kBtThreads = 512;              // templates per CTA
constexpr int kBtTPT = 4;                    // templates per thread (they share each row's records)
constexpr int kBtBlock = kBtThreads / kBtTPT;  // threads per CTA
constexpr int kBtRowPad = 64;
constexpr int kBtTab = 1024;  // intervals of the full-turn cosine table

struct BtParams {
    double xlo[6], step[6];
    double hi0sq, hi3;             // Newton starting points (top of the f0^2 and a_p ranges)
    int n_div[6];
    long long n_per_box;
    unsigned key0, key1;
    double t_sft;
    long long k_lo;
    const unsigned char *power;    // row alpha starts at power + alpha * row_pitch
    long long row_pitch;           // bytes between consecutive rows
    int row_bytes;                 // bytes copied per row (Wp elements of the storage type)
    int W, N, S, n_stages;
    const float4 *rowv;
    const long long *tq;
    const float2 *costab;          // (cos(i (pi/2) / 1024) in FP32, next minus this)
    const float4 *rowd;            // null, or the all-sky weight records [n_pad][2]
    double mu, sigma;
    double m1, sd1;                // one SFT's noise mean and deviation (2, 2 for power)
    // eval mode (box_mode == 0): templates [first, first + count), CTA c takes kBtThreads of them
    long long first, count;
    float *s_out, *z_out;
    int *oob_out;
    // box mode: CTA c is tile c % tiles_per_box of box c / tiles_per_box
    int box_mode, tiles_per_box, k;
    ft_candidate *cand;            // [n_ctas][k]
    const float *gate;             // null, or [n_templates]: only gate[t] >= gate_min compete
    float gate_min;
    unsigned *status;
};

// ------------------------------------------------------------------ canonical rule
//
// Every step below is the canonical bin rule (header: the binary section): the same
// operations in the same precision and order as its statement, so that the bins are a
// function of (seed, template, SFT) alone.

__device__ __forceinline__ double bt_u53(unsigned a, unsigned b)
{
    const double hi = static_cast<double>(a >> 5), lo = static_cast<double>(b >> 6);
    return __ddiv_rn(__dadd_rn(__dmul_rn(hi, 67108864.0), lo), 9007199254740992.0);
}

__device__ __forceinline__ double bt_cbrt(double x, double y0)
{
    if (!(x > 0.0))
        return 0.0;
    double y = y0;
    for (int it = 0; it < 24; ++it) {
        const double y2 = __dmul_rn(y, y);
        const double y3 = __dmul_rn(y2, y);
        const double num = __dsub_rn(y3, x);
        const double den = __dmul_rn(3.0, y2);
        y = __dsub_rn(y, __ddiv_rn(num, den));
    }
    return y;
}

__device__ void bt_lambda(const BtParams &p, long long i, double lam[6])
{
    double u[6];
#pragma unroll
    for (unsigned c = 0; c < 3; ++c) {
        unsigned w[4];
        ftp::philox4x32_10(static_cast<unsigned>(i), static_cast<unsigned>(static_cast<unsigned long long>(i) >> 32),
                           c, 0x62696e61u, p.key0, p.key1, w);
        u[2 * c] = bt_u53(w[0], w[1]);
        u[2 * c + 1] = bt_u53(w[2], w[3]);
    }
    long long box = i / p.n_per_box;
    long long bk[6];
#pragma unroll
    for (int d = 5; d >= 0; --d) {
        bk[d] = box % p.n_div[d];
        box /= p.n_div[d];
    }
    double xi[6];
#pragma unroll
    for (int d = 0; d < 6; ++d)
        xi[d] = __dadd_rn(p.xlo[d], __dmul_rn(__dadd_rn(static_cast<double>(bk[d]), u[d]), p.step[d]));
    lam[0] = __dsqrt_rn(bt_cbrt(xi[0], p.hi0sq));
    lam[1] = xi[1];
    lam[2] = xi[2];
    lam[3] = bt_cbrt(xi[3], p.hi3);
    lam[4] = __dsqrt_rn(__dsqrt_rn(xi[4]));
    lam[5] = xi[5];
    const double below1 = 0x1.fffffffffffffp-1;
    if (lam[1] >= 1.0)
        lam[1] = below1;
    if (lam[5] >= 1.0)
        lam[5] = below1;
    lam[2] = fmin(fmax(lam[2], -1.0), 1.0);
}

// cos(2 pi theta / 2^32): linear interpolation between entry theta >> 22 of the full-turn
// table and the next, at the fraction given by the low 22 bits
__device__ __forceinline__ float bt_cos_q32(unsigned theta, const float2 *tab)
{
    const float f = __fmul_rn(__uint2float_rn(theta & 0x3FFFFFu), 0x1p-22f);
    const float2 e = tab[theta >> 22];
    return __fmaf_rn(f, e.y, e.x);
}

struct BtTmpl {
    int K;
    float phi, F, nx, ny, nz, D;
    float wx, wy;  // the sky vector's x and y to FP32 accuracy, for the all-sky weights
    unsigned long long nu_q, psi_q;
};

__device__ void bt_derive(const BtParams &p, const double lam[6], const float2 *tab, BtTmpl &t)
{
    const double F = __dmul_rn(lam[0], p.t_sft);
    const double Fl = floor(F);
    t.K = static_cast<int>(__double2ll_rz(Fl) - p.k_lo);
    t.phi = __double2float_rn(__dsub_rn(F, Fl));
    t.F = __double2float_rn(F);
    const double c2 = __dsub_rn(1.0, __dmul_rn(lam[2], lam[2]));
    const float cd = __double2float_rn(__dsqrt_rn(c2 > 0.0 ? c2 : 0.0));
    const unsigned ta = __double2uint_rz(__dmul_rn(lam[1], 4294967296.0));
    t.nx = __fmul_rn(cd, bt_cos_q32(ta, tab));
    t.ny = __fmul_rn(cd, bt_cos_q32(ta - 0x40000000u, tab));
    // the weights follow the template's true direction, not the track's table cosine
    double sa, ca;
    sincospi(__dmul_rn(2.0, lam[1]), &sa, &ca);
    const double cd64 = sqrt(c2 > 0.0 ? c2 : 0.0);
    t.wx = __double2float_rn(cd64 * ca);
    t.wy = __double2float_rn(cd64 * sa);
    t.nz = __double2float_rn(lam[2]);
    t.D = __double2float_rn(__dmul_rn(__dmul_rn(F, lam[3]), lam[4]));
    const double nu = __ddiv_rn(lam[4], 6.283185307179586);
    t.nu_q = __double2ull_rz(floor(__dadd_rn(__dmul_rn(nu, 18014398509481984.0), 0.5)));
    t.psi_q = __double2ull_rz(__dmul_rn(lam[5], 18446744073709551616.0));
}

__device__ __forceinline__ int bt_bin(const BtTmpl &t, float4 v, long long tq, const float2 *tab)
{
    const unsigned long long ph = t.nu_q * static_cast<unsigned long long>(tq) - t.psi_q;
    const float c = bt_cos_q32(static_cast<unsigned>(ph >> 32), tab);
    const float a = __fmul_rn(v.z, t.nz);
    const float b = __fmaf_rn(v.y, t.ny, a);
    const float vn = __fmaf_rn(v.x, t.nx, b);
    const float dop = __fmul_rn(t.F, vn);
    const float m = __fmul_rn(t.D, c);
    const float X = __fsub_rn(__fadd_rn(t.phi, dop), m);
    return t.K + static_cast<int>(floorf(__fadd_rn(X, 0.5f)));
}

template <typename T>
__device__ __forceinline__ float bt_load(const unsigned char *row, int k);
template <>
__device__ __forceinline__ float bt_load<float>(const unsigned char *row, int k)
{
    return reinterpret_cast<const float *>(row)[k];
}
template <>
__device__ __forceinline__ float bt_load<__half>(const unsigned char *row, int k)
{
    return __half2float(reinterpret_cast<const __half *>(row)[k]);
}
template <>
__device__ __forceinline__ float bt_load<__nv_bfloat16>(const unsigned char *row, int k)
{
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(row)[k]);
}

// ------------------------------------------------------------------ kernels

// One stage: S power rows (each its own bulk copy), S velocity records, S times.
__device__ __forceinline__ void bt_issue(const BtParams &p, int st, unsigned char *rows,
                                         float4 *sv, long long *stq, float4 *sd, unsigned long long *bar)
{
    const int lane = threadIdx.x & 31;
    const int nr = min(p.S, p.N - st * p.S);
    if (lane == 0)
        ftp::mbar_arrive_expect_tx(bar, static_cast<unsigned>(nr * p.row_bytes + p.S * 24 +
                                                              (p.rowd != nullptr ? p.S * 32 : 0)));
    __syncwarp();
    for (int r = lane; r < nr; r += 32)
        ftp::bulk_g2s(rows + static_cast<size_t>(r) * p.row_bytes,
                      p.power + (static_cast<long long>(st) * p.S + r) * p.row_pitch,
                      static_cast<unsigned>(p.row_bytes), bar);
    if (lane == 0) {
        ftp::bulk_g2s(sv, p.rowv + static_cast<long long>(st) * p.S, static_cast<unsigned>(p.S * 16), bar);
        ftp::bulk_g2s(stq, p.tq + static_cast<long long>(st) * p.S, static_cast<unsigned>(p.S * 8), bar);
        if (p.rowd != nullptr)
            ftp::bulk_g2s(sd, p.rowd + 2ll * st * p.S, static_cast<unsigned>(p.S * 32), bar);
    }
}

// (a^2 + b^2)(D, n) / S_n for the FP32 record of D / sqrt(S_n): with u = D n and c = n.u,
// a^2 + b^2 = 2 |TT(D)|^2 = 2 |D|^2 - 4 |u|^2 + 2 c^2 - (tr D - c)^2 for a unit n (the
// transverse-traceless projection; no wave frame needed).
__device__ __forceinline__ float bt_sky_r(float4 d0, float4 d1, float nx, float ny, float nz)
{
    const float u0 = d0.x * nx + d0.y * ny + d0.z * nz;
    const float u1 = d0.y * nx + d0.w * ny + d1.x * nz;
    const float u2 = d0.z * nx + d1.x * ny + d1.y * nz;
    const float c = nx * u0 + ny * u1 + nz * u2;
    const float uu = u0 * u0 + u1 * u1 + u2 * u2;
    const float tc = d1.w - c;
    return 2.f * d1.z - 4.f * uu + 2.f * c * c - tc * tc;
}

__device__ __forceinline__ void fold2(float &hi, float &lo, float part)
{
    const float s = __fadd_rn(hi, part);
    const float bp = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(part, bp)));
    hi = s;
}

template <typename T, bool WEIGHTED, bool SKY>
__global__ void __launch_bounds__(kBtBlock) k_bt_eval(const BtParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t rows_bytes = static_cast<size_t>(p.S) * p.row_bytes;
    unsigned char *rows[2] = {smem, smem + rows_bytes};
    float4 *sv[2] = {reinterpret_cast<float4 *>(smem + 2 * rows_bytes),
                     reinterpret_cast<float4 *>(smem + 2 * rows_bytes) + p.S};
    long long *stq[2] = {reinterpret_cast<long long *>(sv[1] + p.S),
                         reinterpret_cast<long long *>(sv[1] + p.S) + p.S};
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(stq[1] + p.S);
    float2 *tab = reinterpret_cast<float2 *>(bars + 2);
    float4 *sd[2] = {reinterpret_cast<float4 *>(tab + kBtTab + 1 + 1), nullptr};  // 16-byte aligned
    sd[1] = sd[0] + 2 * p.S;

    // this CTA's templates
    long long t_begin, t_end;
    if (p.box_mode) {
        const long long box = blockIdx.x / p.tiles_per_box;
        const long long tile = blockIdx.x % p.tiles_per_box;
        t_begin = box * p.n_per_box + tile * kBtThreads;
        t_end = min(t_begin + kBtThreads, (box + 1) * p.n_per_box);
    } else {
        t_begin = p.first + static_cast<long long>(blockIdx.x) * kBtThreads;
        t_end = min(t_begin + kBtThreads, p.first + p.count);
    }
    // this thread's templates: t_begin + threadIdx.x + u kBtBlock
    long long ti[kBtTPT];
    bool valid[kBtTPT];
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        ti[u] = t_begin + threadIdx.x + u * kBtBlock;
        valid[u] = ti[u] < t_end;
    }

    if (threadIdx.x == 0) {
        ftp::mbar_init(&bars[0], 1);
        ftp::mbar_init(&bars[1], 1);
        ftp::fence_mbar_init();
    }
    for (int i = threadIdx.x; i <= kBtTab; i += kBtBlock)
        tab[i] = p.costab[i];
    __syncthreads();
    if (threadIdx.x < 32) {
        bt_issue(p, 0, rows[0], sv[0], stq[0], sd[0], &bars[0]);
        if (p.n_stages > 1)
            bt_issue(p, 1, rows[1], sv[1], stq[1], sd[1], &bars[1]);
    }

    BtTmpl t[kBtTPT];
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        double lam[6];
        bt_lambda(p, valid[u] ? ti[u] : t_begin, lam);
        bt_derive(p, lam, tab, t[u]);
    }

    float hi[kBtTPT], lo[kBtTPT];
    // all-sky weights: sum r, sum r^2 (r = (a^2 + b^2) / S_n), compensated like the sum
    float hiB[kBtTPT], loB[kBtTPT], hiC[kBtTPT], loC[kBtTPT];
    int oob[kBtTPT];
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        hi[u] = lo[u] = hiB[u] = loB[u] = hiC[u] = loC[u] = 0.f;
        oob[u] = 0;
    }
    bool failed = false;
    for (int st = 0; st < p.n_stages; ++st) {
        const int b = st & 1;
        const bool ok = ftp::mbar_wait_bounded(&bars[b], (st >> 1) & 1);
        const int nr = min(p.S, p.N - st * p.S);
        float part[kBtTPT], partB[kBtTPT], partC[kBtTPT];
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u)
            part[u] = partB[u] = partC[u] = 0.f;
        if (ok) {
            const unsigned char *rb = rows[b];
#pragma unroll 2
            for (int r = 0; r < nr; ++r) {
                const float4 v = sv[b][r];
                const long long tq = stq[b][r];
                const unsigned char *row = rb + static_cast<size_t>(r) * p.row_bytes;
#pragma unroll
                for (int u = 0; u < kBtTPT; ++u) {
                    const int k = bt_bin(t[u], v, tq, tab);
                    const bool in = static_cast<unsigned>(k) < static_cast<unsigned>(p.W);
                    const float val = in ? bt_load<T>(row, k) : 0.f;
                    oob[u] += in ? 0 : 1;
                    if (SKY) {
                        const float rw = bt_sky_r(sd[b][2 * r], sd[b][2 * r + 1], t[u].wx, t[u].wy, t[u].nz);
                        part[u] = __fmaf_rn(rw, val, part[u]);
                        partB[u] = __fadd_rn(partB[u], rw);
                        partC[u] = __fmaf_rn(rw, rw, partC[u]);
                    } else {
                        part[u] = WEIGHTED ? __fmaf_rn(v.w, val, part[u]) : __fadd_rn(part[u], val);
                    }
                }
            }
        }
        // compensated folds of the stage's partials (2Sum)
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u) {
            fold2(hi[u], lo[u], part[u]);
            if (SKY) {
                fold2(hiB[u], loB[u], partB[u]);
                fold2(hiC[u], loC[u], partC[u]);
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (threadIdx.x < 32 && st + 2 < p.n_stages)
            bt_issue(p, st + 2, rows[b], sv[b], stq[b], sd[b], &bars[b]);
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(p.status, FT_STATUS_TIMEOUT);
            // let copies still in flight land before the shared memory is released
            (void)ftp::mbar_wait_bounded(&bars[0], 0);
            (void)ftp::mbar_wait_bounded(&bars[1], 0);
        }
        __syncthreads();
        return;
    }

    // s and z: the plain sum, or under all-sky weights sum r P / sum r with mu_G = m1 and
    // sigma_G = sd1 sqrt(sum r^2) / sum r of this template's sky direction (m1 = sd1 = 2 for
    // normalised power; p and sqrt(p (1 - p)) for a number-count band)
    float *vs = reinterpret_cast<float *>(smem);
    float *vz = vs + kBtThreads;
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        double s64 = static_cast<double>(hi[u]) + static_cast<double>(lo[u]);
        double z64 = (s64 - p.mu) / p.sigma;
        if (SKY) {
            const double B = static_cast<double>(hiB[u]) + static_cast<double>(loB[u]);
            const double C = static_cast<double>(hiC[u]) + static_cast<double>(loC[u]);
            s64 /= B;
            z64 = (s64 - p.m1) / (p.sd1 * sqrt(C) / B);
        }
        const float sv_ = SKY ? static_cast<float>(s64) : __fadd_rn(hi[u], lo[u]);
        if (!p.box_mode) {
            if (valid[u]) {
                const long long o = ti[u] - p.first;
                p.s_out[o] = sv_;
                if (p.z_out)
                    p.z_out[o] = static_cast<float>(z64);
                if (p.oob_out)
                    p.oob_out[o] = oob[u];
            }
            continue;
        }
        // candidates of the per-CTA selection; -inf: not a candidate
        const bool pass = valid[u] && (p.gate == nullptr || p.gate[ti[u]] >= p.gate_min);
        vs[threadIdx.x + u * kBtBlock] = pass ? sv_ : -INFINITY;
        vz[threadIdx.x + u * kBtBlock] = static_cast<float>(z64);
    }
    if (!p.box_mode)
        return;

    // per-CTA top-k by (s desc, index asc): warp 0 extracts k rounds of the arg-max among
    // keys ranked after the previous pick
    __syncthreads();
    if (threadIdx.x >= 32)
        return;
    const int lane = threadIdx.x;
    const int n_here = static_cast<int>(t_end - t_begin);
    float last_s = INFINITY;
    long long last_t = -1;
    ft_candidate *out = p.cand + static_cast<long long>(blockIdx.x) * p.k;
    for (int j = 0; j < p.k; ++j) {
        bool have = false;
        float bs = -INFINITY, bz = 0.f;
        long long bt = LLONG_MAX;
        for (int q = lane; q < n_here; q += 32) {
            const float s = vs[q];
            if (s == -INFINITY)
                continue;
            const long long tt = t_begin + q;
            const bool elig = (s < last_s) || (s == last_s && tt > last_t);
            if (elig && (!have || s > bs || (s == bs && tt < bt))) {
                have = true;
                bs = s;
                bt = tt;
                bz = vz[q];
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
            out[j] = cd;
        }
        last_s = bs;
        last_t = bt;
    }
}

// One CTA per box: k rounds of a block-wide arg-max over the box's tile lists.
__global__ void __launch_bounds__(256) k_bt_merge(const ft_candidate *cand, int tiles_per_box, int k,
                                                   ft_candidate *out)
{
    __shared__ float rs[8];
    __shared__ long long rt[8];
    __shared__ float rz[8];
    __shared__ int rh[8];
    const long long box = blockIdx.x;
    const ft_candidate *c = cand + box * tiles_per_box * k;
    const int n = tiles_per_box * k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float last_s = INFINITY;
    long long last_t = -1;
    for (int j = 0; j < k; ++j) {
        bool have = false;
        float bs = -INFINITY, bz = 0.f;
        long long bt = LLONG_MAX;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const ft_candidate e = c[q];
            if (e.template_idx < 0)
                continue;
            const bool elig = (e.s < last_s) || (e.s == last_s && e.template_idx > last_t);
            if (elig && (!have || e.s > bs || (e.s == bs && e.template_idx < bt))) {
                have = true;
                bs = e.s;
                bt = e.template_idx;
                bz = e.z;
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
            rs[warp] = bs;
            rt[warp] = bt;
            rz[warp] = bz;
            rh[warp] = have ? 1 : 0;
        }
        __syncthreads();
        have = false;
        bs = -INFINITY;
        bt = LLONG_MAX;
        bz = 0.f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
            if (rh[w] && (!have || rs[w] > bs || (rs[w] == bs && rt[w] < bt))) {
                have = true;
                bs = rs[w];
                bt = rt[w];
                bz = rz[w];
            }
        }
        if (threadIdx.x == 0) {
            ft_candidate cd;
            cd.template_idx = have ? bt : -1;
            cd.s = have ? bs : -INFINITY;
            cd.z = have ? bz : 0.f;
            out[box * k + j] = cd;
        }
        last_s = bs;
        last_t = bt;
        __syncthreads();
    }
}

__global__ void k_bt_templates(const BtParams p, long long first, long long n, double *lam_out)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n)
        return;
    double lam[6];
    bt_lambda(p, first + i, lam);
    for (int d = 0; d < 6; ++d)
        lam_out[6 * i + d] = lam[d];
}

__global__ void k_bt_bins(const BtParams p, const long long *tmpl, long long n, int *bins)
{
    const long long i = blockIdx.x;
    if (i >= n)
        return;
    double lam[6];
    bt_lambda(p, tmpl[i], lam);
    BtTmpl t;
    bt_derive(p, lam, p.costab, t);
    for (int a = threadIdx.x; a < p.N; a += blockDim.x)
        bins[i * p.N + a] = bt_bin(t, p.rowv[a], p.tq[a], p.costab);
}

__global__ void k_bt_rowv(const double *v, const float *w, int N, int n_pad, float4 *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_pad)
        return;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < N)
        r = make_float4(__double2float_rn(v[3 * a]), __double2float_rn(v[3 * a + 1]),
                        __double2float_rn(v[3 * a + 2]), w[a]);
    out[a] = r;
}

__global__ void k_bt_rowd(const double *D, const double *sn, int N, int n_pad, float4 *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
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

// ------------------------------------------------------------------ host side

struct Guard {
    int prev = -1, dev;
    explicit Guard(int d) : dev(d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
        (void)cudaGetLastError();
    }
    ~Guard()
    {
        if (prev >= 0 && prev != dev)
            cudaSetDevice(prev);
    }
};

double xi_of(int d, double lam)
{
    switch (d) {
    case 0: {
        const double x2 = lam * lam;
        const double x3 = x2 * lam;
        return x3 * x3;
    }
    case 3: {
        const double x2 = lam * lam;
        return x2 * lam;
    }
    case 4: {
        const double x2 = lam * lam;
        return x2 * x2;
    }
    default: return lam;
    }
}

int elem_bytes(int dtype)
{
    return dtype == FT_F32 ? 4 : 2;
}

BtParams base_params(const ft_band *band, const ft_binary_bank *bk)
{
    BtParams p;
    std::memset(&p, 0, sizeof(p));
    for (int d = 0; d < 6; ++d) {
        p.xlo[d] = bk->xlo[d];
        p.step[d] = bk->step[d];
        p.n_div[d] = bk->desc.n_div[d];
    }
    p.hi0sq = bk->desc.hi[0] * bk->desc.hi[0];
    p.hi3 = bk->desc.hi[3];
    p.n_per_box = bk->desc.n_per_box;
    p.key0 = static_cast<unsigned>(bk->desc.seed);
    p.key1 = static_cast<unsigned>(bk->desc.seed >> 32);
    p.t_sft = band->t_sft;
    p.k_lo = band->k_lo;
    p.power = static_cast<const unsigned char *>(band->d_power);
    const int eb = elem_bytes(band->dtype);
    // FP32 rows are [N][Wp]; 16-bit rows [N][2][Wp] (the first copy holds the plain row)
    p.row_pitch = static_cast<long long>(band->Wp) * eb * (band->dtype == FT_F32 ? 1 : 2);
    p.row_bytes = band->Wp * eb;
    p.W = band->W;
    p.N = static_cast<int>(band->N);
    p.rowv = bk->d_rowv;
    p.tq = bk->d_tq;
    p.costab = bk->d_costab;
    p.rowd = band->d_D != nullptr ? bk->d_rowd : nullptr;
    p.mu = band->mu;
    p.m1 = band->m1;
    p.sd1 = std::sqrt(band->v1);
    p.sigma = band->sigma;
    p.status = band->ctx->d_status;
    return p;
}

int stage_rows(const ft_band *band)
{
    // at most 16 KB of rows per stage, 8..64 rows (a divisor of kBtRowPad): two stages and
    // the cosine table leave room for 4 CTAs per SM, as many as the registers allow
    const int rb = band->Wp * elem_bytes(band->dtype);
    int S = 64;
    while (S > 8 && S * rb > 16 * 1024)
        S >>= 1;
    return S;
}

size_t eval_smem(const BtParams &p)
{
    return 2 * (static_cast<size_t>(p.S) * p.row_bytes + p.S * 24) + 16 + (kBtTab + 2) * sizeof(float2) +
           (p.rowd != nullptr ? 2 * static_cast<size_t>(p.S) * 32 : 0);
}

template <typename T, bool Wt>
int launch_t(long long n_cta, size_t smem, const BtParams &p, cudaStream_t st)
{
    auto fn = p.rowd != nullptr ? k_bt_eval<T, false, true> : k_bt_eval<T, Wt, false>;
    FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    fn<<<static_cast<unsigned>(n_cta), kBtBlock, smem, st>>>(p);
    FT_CUDA(cudaGetLastError());
    return FT_OK;
}

int launch_eval(const ft_band *band, long long n_cta, BtParams p, cudaStream_t st)
{
    p.S = stage_rows(band);
    p.n_stages = static_cast<int>((band->N + p.S - 1) / p.S);
    const size_t smem = std::max(eval_smem(p), static_cast<size_t>(2 * kBtThreads * 4));
    if (smem > band->ctx->smem_optin)
        FT_FAIL(FT_ERR_RANGE, "binary: band rows too wide for the shared-memory stages");
    if (n_cta <= 0)
        return FT_OK;
    if (n_cta > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "binary: too many CTAs for one launch");
    const bool w = band->weighted;
    switch (band->dtype) {
    case FT_F32: return w ? launch_t<float, true>(n_cta, smem, p, st) : launch_t<float, false>(n_cta, smem, p, st);
    case FT_F16: return w ? launch_t<__half, true>(n_cta, smem, p, st) : launch_t<__half, false>(n_cta, smem, p, st);
    case FT_BF16:
        return w ? launch_t<__nv_bfloat16, true>(n_cta, smem, p, st)
                 : launch_t<__nv_bfloat16, false>(n_cta, smem, p, st);
    default: FT_FAIL(FT_ERR_ARG, "binary: unknown storage type");
    }
}

int check(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank)
{
    if (!ctx || !band || !bank)
        FT_FAIL(FT_ERR_ARG, "binary: null ctx/band/bank");
    if (band->ctx != ctx || bank->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "binary: band/bank belong to another context");
    if (bank->band != band)
        FT_FAIL(FT_ERR_ARG, "binary: bank was made for another band");
    if (band->d_D && !bank->d_rowd)
        FT_FAIL(FT_ERR_ARG, "binary: the bank was made before the band's all-sky weights were set; make it again");
    return FT_OK;
}

}  // namespace

int ft_make_binary_bank(ft_ctx *ctx, const ft_band *band, const ft_binary_bank_desc *desc,
                        ft_binary_bank **out)
{
    if (!ctx || !band || !desc || !out)
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: null argument");
    if (band->ctx != ctx)
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: band belongs to another context");
    *out = nullptr;
    const ft_binary_bank_desc &d = *desc;
    for (int k = 0; k < 6; ++k) {
        if (!std::isfinite(d.lo[k]) || !std::isfinite(d.hi[k]) || !(d.lo[k] <= d.hi[k]))
            FT_FAIL(FT_ERR_ARG, "make_binary_bank: each range needs finite lo <= hi");
        if (d.n_div[k] < 1)
            FT_FAIL(FT_ERR_ARG, "make_binary_bank: n_div must be >= 1");
    }
    for (int k : {0, 3, 4}) {
        const bool isolated = k == 3 && d.lo[k] == 0.0 && d.hi[k] == 0.0;
        if (!isolated && !(d.lo[k] > 0.0 && d.hi[k] <= 16.0 * d.lo[k]))
            FT_FAIL(FT_ERR_ARG, "make_binary_bank: f0, a_p and Omega need 0 < lo <= hi <= 16 lo "
                                "(a_p may be 0..0)");
    }
    if (d.lo[1] < 0.0 || d.hi[1] > 1.0 || d.lo[5] < 0.0 || d.hi[5] > 1.0)
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: alpha and phi_b are turns within [0, 1]");
    if (d.lo[2] < -1.0 || d.hi[2] > 1.0)
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: sin(delta) must lie within [-1, 1]");
    if (d.n_per_box < 1)
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: n_per_box must be >= 1");
    double nb = 1.0;
    long long n_boxes = 1;
    for (int k = 0; k < 6; ++k) {
        nb *= d.n_div[k];
        n_boxes *= d.n_div[k];
        if (nb > 1e12)
            FT_FAIL(FT_ERR_RANGE, "make_binary_bank: too many boxes");
    }
    if (nb * static_cast<double>(d.n_per_box) >= 1099511627776.0)
        FT_FAIL(FT_ERR_RANGE, "make_binary_bank: n_templates must be below 2^40");
    if (d.hi[0] * band->t_sft - static_cast<double>(band->k_lo) > 2e9 ||
        d.lo[0] * band->t_sft - static_cast<double>(band->k_lo) < -2e9)
        FT_FAIL(FT_ERR_RANGE, "make_binary_bank: f0 range far outside the band");
    if (band->N > INT_MAX - kBtRowPad)
        FT_FAIL(FT_ERR_RANGE, "make_binary_bank: too many SFTs");
    if (band->h_dt.size() != static_cast<size_t>(band->N))
        FT_FAIL(FT_ERR_ARG, "make_binary_bank: band has no SFT times");

    Guard g(ctx->device);
    ft_binary_bank *b = new ft_binary_bank;
    b->ctx = ctx;
    b->device = ctx->device;
    b->band = band;
    b->desc = d;
    b->n_boxes = n_boxes;
    b->n_templates = n_boxes * d.n_per_box;
    for (int k = 0; k < 6; ++k) {
        b->xlo[k] = xi_of(k, d.lo[k]);
        b->step[k] = (xi_of(k, d.hi[k]) - b->xlo[k]) / static_cast<double>(d.n_div[k]);
    }
    const int N = static_cast<int>(band->N);
    b->n_pad = (N + kBtRowPad - 1) / kBtRowPad * kBtRowPad;
    std::vector<long long> tq(b->n_pad, 0);
    for (int a = 0; a < N; ++a)
        tq[a] = static_cast<long long>(std::floor(band->h_dt[a] * 1024.0 + 0.5));
    auto fail = [&](int rc) {
        ft_binary_bank_destroy(b);
        return rc;
    };
    // full-turn cosine table: cos(i 2 pi / 1024) from the host's libm in FP64, rounded
    // to FP32, with the FP32 difference to the next entry (0 after the last)
    float tc[kBtTab + 1];
    for (int i = 0; i <= kBtTab; ++i)
        tc[i] = static_cast<float>(std::cos(static_cast<double>(i) * 6.135923151542565e-03));
    std::vector<float2> tab(kBtTab + 1);
    for (int i = 0; i <= kBtTab; ++i)
        tab[i] = make_float2(tc[i], i < kBtTab ? tc[i + 1] - tc[i] : 0.0f);
    if (cudaMalloc(&b->d_rowv, static_cast<size_t>(b->n_pad) * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&b->d_tq, static_cast<size_t>(b->n_pad) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_costab, tab.size() * sizeof(float2)) != cudaSuccess) {
        ft_set_error("make_binary_bank: allocation failed");
        return fail(FT_ERR_OOM);
    }
    if (cudaMemcpy(b->d_tq, tq.data(), tq.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_costab, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        ft_set_error("make_binary_bank: copy failed");
        return fail(FT_ERR_CUDA);
    }
    k_bt_rowv<<<(b->n_pad + 255) / 256, 256>>>(band->d_v, band->d_w, N, b->n_pad, b->d_rowv);
    if (band->d_D) {
        if (cudaMalloc(&b->d_rowd, static_cast<size_t>(b->n_pad) * 2 * sizeof(float4)) != cudaSuccess) {
            b->d_rowd = nullptr;
            ft_set_error("make_binary_bank: allocation failed");
            return fail(FT_ERR_OOM);
        }
        k_bt_rowd<<<(b->n_pad + 255) / 256, 256>>>(band->d_D, band->d_sn, N, b->n_pad, b->d_rowd);
    }
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        ft_set_error("make_binary_bank: set-up kernel failed");
        return fail(FT_ERR_CUDA);
    }
    *out = b;
    return FT_OK;
}

void ft_binary_bank_destroy(ft_binary_bank *b)
{
    if (!b)
        return;
    Guard g(b->device);
    cudaFree(b->d_rowv);
    cudaFree(b->d_tq);
    cudaFree(b->d_costab);
    cudaFree(b->d_rowd);
    delete b;
}

int ft_binary_bank_info(const ft_binary_bank *b, int64_t *n_templates, int64_t *n_boxes)
{
    if (!b)
        FT_FAIL(FT_ERR_ARG, "binary_bank_info: null bank");
    if (n_templates)
        *n_templates = b->n_templates;
    if (n_boxes)
        *n_boxes = b->n_boxes;
    return FT_OK;
}

int ft_binary_templates(ft_ctx *ctx, const ft_binary_bank *bank, int64_t first, int64_t n,
                        double *lambda_out, void *stream)
{
    if (!ctx || !bank || bank->ctx != ctx || n < 0 || (n > 0 && !lambda_out) || first < 0 ||
        first + n > bank->n_templates)
        FT_FAIL(FT_ERR_ARG, "binary_templates: bad arguments");
    if (n == 0)
        return FT_OK;
    Guard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BtParams p = base_params(bank->band, bank);
    void *buf = nullptr;
    FT_TRY(ft_ctx_outbuf(ctx, static_cast<size_t>(n) * 48, &buf));
    k_bt_templates<<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(p, first, n, static_cast<double *>(buf));
    FT_CUDA(cudaGetLastError());
    FT_CUDA(cudaMemcpyAsync(lambda_out, buf, static_cast<size_t>(n) * 48, cudaMemcpyDeviceToHost, st));
    FT_CUDA(cudaStreamSynchronize(st));
    return FT_OK;
}

int ft_binary_track_bins(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank,
                         const int64_t *templates, int64_t n, int32_t *bins, int on_device,
                         void *stream)
{
    FT_TRY(check(ctx, band, bank));
    if (n < 0 || (n > 0 && (!templates || !bins)))
        FT_FAIL(FT_ERR_ARG, "binary_track_bins: bad arguments");
    if (n == 0)
        return FT_OK;
    if (n > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "binary_track_bins: too many templates");
    Guard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nb = static_cast<size_t>(n) * band->N * 4;
    const long long *dt = reinterpret_cast<const long long *>(templates);
    int *db = reinterpret_cast<int *>(bins);
    if (!on_device) {
        void *buf = nullptr;
        FT_TRY(ft_ctx_outbuf(ctx, nb + static_cast<size_t>(n) * 8, &buf));
        db = static_cast<int *>(buf);
        long long *t = reinterpret_cast<long long *>(static_cast<char *>(buf) + nb);
        FT_CUDA(cudaMemcpyAsync(t, templates, static_cast<size_t>(n) * 8, cudaMemcpyHostToDevice, st));
        dt = t;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!on_device && (templates[i] < 0 || templates[i] >= bank->n_templates))
            FT_FAIL(FT_ERR_ARG, "binary_track_bins: template index out of range");
    BtParams p = base_params(band, bank);
    k_bt_bins<<<static_cast<unsigned>(n), 256, 0, st>>>(p, dt, n, db);
    FT_CUDA(cudaGetLastError());
    if (!on_device) {
        FT_CUDA(cudaMemcpyAsync(bins, db, nb, cudaMemcpyDeviceToHost, st));
        FT_CUDA(cudaStreamSynchronize(st));
    }
    return FT_OK;
}

int ft_binary_eval(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank, int64_t first,
                   int64_t n, float *s_out, float *z_out, int32_t *n_oob_out, int out_on_device,
                   void *stream)
{
    FT_TRY(check(ctx, band, bank));
    if (!s_out || n < 0 || first < 0 || first + n > bank->n_templates)
        FT_FAIL(FT_ERR_ARG, "binary_eval: bad arguments");
    if (n == 0)
        return FT_OK;
    Guard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *ds = s_out, *dz = z_out;
    int *doob = reinterpret_cast<int *>(n_oob_out);
    const size_t nn = static_cast<size_t>(n);
    if (!out_on_device) {
        void *buf = nullptr;
        FT_TRY(ft_ctx_outbuf(ctx, nn * 12, &buf));
        ds = static_cast<float *>(buf);
        dz = z_out ? ds + nn : nullptr;
        doob = n_oob_out ? reinterpret_cast<int *>(ds + 2 * nn) : nullptr;
    }
    BtParams p = base_params(band, bank);
    p.first = first;
    p.count = n;
    p.s_out = ds;
    p.z_out = dz;
    p.oob_out = doob;
    FT_TRY(launch_eval(band, (n + kBtThreads - 1) / kBtThreads, p, st));
    if (!out_on_device) {
        FT_CUDA(cudaMemcpyAsync(s_out, ds, nn * 4, cudaMemcpyDeviceToHost, st));
        if (z_out)
            FT_CUDA(cudaMemcpyAsync(z_out, dz, nn * 4, cudaMemcpyDeviceToHost, st));
        if (n_oob_out)
            FT_CUDA(cudaMemcpyAsync(n_oob_out, doob, nn * 4, cudaMemcpyDeviceToHost, st));
        return ft_read_status(ctx, st);
    }
    return FT_OK;
}

namespace {

int binary_topk(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank, int k, const float *gate,
                float gate_min, ft_candidate *out, int out_on_device, void *stream)
{
    FT_TRY(check(ctx, band, bank));
    if (!out)
        FT_FAIL(FT_ERR_ARG, "binary_topk_per_box: null out");
    if (k < 1 || k > 32)
        FT_FAIL(FT_ERR_RANGE, "binary_topk_per_box: k must be in [1, 32]");
    if (bank->n_boxes > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "binary_topk_per_box: too many boxes for one launch");
    Guard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long tiles = (bank->desc.n_per_box + kBtThreads - 1) / kBtThreads;
    const long long n_cta = tiles * bank->n_boxes;
    if (tiles * k > INT_MAX)
        FT_FAIL(FT_ERR_RANGE, "binary_topk_per_box: boxes too large");
    const size_t cand_bytes = static_cast<size_t>(n_cta) * k * sizeof(ft_candidate);
    const size_t out_bytes = static_cast<size_t>(bank->n_boxes) * k * sizeof(ft_candidate);
    void *scr = nullptr;
    FT_TRY(ft_ctx_scratch(ctx, cand_bytes, &scr));
    ft_candidate *dout = out;
    if (!out_on_device) {
        void *ob = nullptr;
        FT_TRY(ft_ctx_outbuf(ctx, out_bytes, &ob));
        dout = static_cast<ft_candidate *>(ob);
    }
    BtParams p = base_params(band, bank);
    p.box_mode = 1;
    p.gate = gate;
    p.gate_min = gate_min;
    p.tiles_per_box = static_cast<int>(tiles);
    p.k = k;
    p.cand = static_cast<ft_candidate *>(scr);
    FT_TRY(launch_eval(band, n_cta, p, st));
    k_bt_merge<<<static_cast<unsigned>(bank->n_boxes), 256, 0, st>>>(p.cand, p.tiles_per_box, k, dout);
    FT_CUDA(cudaGetLastError());
    if (!out_on_device) {
        FT_CUDA(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, st));
        return ft_read_status(ctx, st);
    }
    return FT_OK;
}

}  // namespace

int ft_binary_topk_per_box(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank, int k,
                           ft_candidate *out, int out_on_device, void *stream)
{
    return binary_topk(ctx, band, bank, k, nullptr, 0.f, out, out_on_device, stream);
}

int ft_binary_topk_per_box_gated(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank, int k,
                                 const float *gate, float gate_min, ft_candidate *out,
                                 int out_on_device, void *stream)
{
    if (!gate)
        FT_FAIL(FT_ERR_ARG, "binary_topk_per_box_gated: null gate");
    if (std::isnan(gate_min))
        FT_FAIL(FT_ERR_ARG, "binary_topk_per_box_gated: gate_min is NaN");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, gate) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        FT_FAIL(FT_ERR_ARG, "binary_topk_per_box_gated: gate must be device memory");
    }
    return binary_topk(ctx, band, bank, k, gate, gate_min, out, out_on_device, stream);
}
