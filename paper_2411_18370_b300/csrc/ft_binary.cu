// ft_binary.cu -- the binary-orbit track (Eq. (track) with the orbit term) over a random
// template bank in uniform coordinates (Sec. IV.A, App. A), cut into hyperboxes (Sec. IV.B).
//
// Templates are never stored: every thread derives its templates (kBtTPT of them, sharing
// each row's records) from Philox counters and keeps the per-template terms of the track in
// registers.  Each CTA evaluates up to kBtThreads templates of one box over all SFTs; stages
// of S SFT rows (power row, FP32 velocity + weight, fixed-point time) are brought into shared
// memory by bulk copies on two mbarrier-tracked buffers.
//
// The bin is the FP64 bin of Eq. (track), X = f0 (1 + v.n - a_p Omega cos(Omega t - phi_b))
// T_SFT - k_lo rounded half up.  Per (template, SFT) the kernel first evaluates X in FP32
// (integer orbit phase, the special-function unit's cosine, FMA chain) with a derived error
// bound delta; only when that value lies within delta of a rounding boundary (a fraction of about
// 2 delta of all evaluations) is X recomputed in FP64 from the template's FP64 terms and the
// SFT's FP64 velocity and time, so every bin equals the FP64 bin.  Then one shared-memory
// read and one add: the kernel is bound by instruction issue, not by HBM.

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
    double *d_t64 = nullptr;       // [n_pad] t_mid - t0 (s), FP64
    // all-sky weights (band with detector tensors): per SFT D / sqrt(S_n) in FP32 as
    // (D00, D01, D02, D11), (D12, D22, |D|^2, tr D); zero beyond N
    float4 *d_rowd = nullptr;      // [n_pad][2]
    unsigned long long *d_n64 = nullptr;  // running count of FP64 decisions
    double delta = 0;              // screening bound of the last launch (bins)
};

namespace {

constexpr int kBtThreads = 512;              // templates per CTA
constexpr int kBtTPT = 4;                    // templates per thread (they share each row's records)
constexpr int kBtBlock = kBtThreads / kBtTPT;  // threads per CTA
constexpr int kBtRowPad = 64;
constexpr int kBtRowGroup = 2;  // SFT rows whose screens run before one branch to the FP64 decisions
constexpr int kBtSlow = 7;    // FP64 terms per template for the FP64 decisions
// The screen's cosine: the orbit phase ph (2^-32 turns, read as a signed angle in [-pi, pi))
// is converted to FP32 radians and passed to the special-function unit's cosine (__cosf).
// Its error against cos(2 pi ph / 2^32) is at most kBtCosErr: the conversion of ph rounds by
// at most 2^7 units (2 pi 2^-25 rad), the FP32 scale 2 pi / 2^32 and the product add at most
// 2 u pi (u = 2^-24), and __cosf is documented to within 2^-21.19 for arguments in
// [-pi, pi] (taken here as 2^-21).  ft_binary_cos_screen_check measures the whole step over
// all 2^32 phases against this bound.
constexpr float kBtPhRad = 1.46291807926715968e-9f;  // 2 pi / 2^32
constexpr double kBtCosErr = 6.283185307179586 * 0x1p-25 + 3.141592653589793 * 0x1p-23 + 0x1p-21;
constexpr float kMagic = 12582912.0f;  // 1.5 2^23: t + kMagic rounds t to an integer in its low bits

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
    const double *v64;             // [N][3] v / c, FP64
    const double *t64;             // [N] t_mid - t0, FP64
    const float4 *rowd;            // null, or the all-sky weight records [n_pad][2]
    float half_delta;              // screen: FP64 decision when |t - rint(t)| > 1/2 - delta
    double vmax;                   // largest |v| / c of the band (window proof per CTA)
    double mu, sigma;
    double m1, sd1;                // one SFT's noise mean and deviation (2, 2 for power)
    long long cta_base;            // CTA index of this launch's first CTA (launches are chunked)
    double *slow;                  // [CTAs of the launch][kBtSlow][kBtThreads] FP64 terms
    unsigned long long *n64;       // running count of FP64 decisions
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

// ------------------------------------------------------------------ templates
//
// The templates are a pure function of (seed, index): every FP64 step of their derivation
// is an explicit round-to-nearest intrinsic, so that the compiler cannot contract or reorder
// it and the host oracle derives the same lambda bit for bit.

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

// ------------------------------------------------------------------ the track
//
// Per template (FP64 once, then rounded): F = f0 T_SFT, K = floor(F) - k_lo,
// t0 = F - floor(F), a = F n, A = F a_p Omega; the orbit frequency Omega / 2 pi in units
// of 2^-54 turns/s (64-bit nu) and minus the top word of phi_b 2^64 (npsi).  Per SFT: the
// 64-bit time t_q = round((t_mid - t0) 2^10).
//
// FP32 screen per (template, SFT), t = X - K:
//   phase  ph = top word of (nu t_q) mod 2^64 + npsi, in 2^-32 turns, from three 32-bit
//          multiplies (the low word's borrow is dropped: |error| < 1 unit);
//   cosine __cosf of ph as a signed FP32 angle (bt_cos, error below kBtCosErr);
//   t      = t0 + a.v - A cos (one FMA chain);
//   bin    = K + rint(t) by the 1.5 2^23 rounding trick, and d = t - rint(t).
// Its error against the exact real value is below the launch's delta (host: bt_delta); when
// |d| > 1/2 - delta the FP64 decision replaces it (exact half-integers included).

struct BtTmpl {
    int K;
    float t0, ax, ay, az, A;
    unsigned nlo, nhi, npsi;
    float wx, wy, wz;  // the unit sky vector in FP32, for the all-sky weights
};

// FP64 terms of the decision, slot q of the CTA: F - k_lo, F n (3), F a_p Omega, Omega,
// 2 pi phi_b.  Returns whether every bin the track can reach (|v.n| <= vmax) lies in [0, W).
__device__ bool bt_derive(const BtParams &p, const double lam[6], BtTmpl &t, double *sl, int q)
{
    const double F = lam[0] * p.t_sft;
    const double Fl = floor(F);
    t.K = static_cast<int>(static_cast<long long>(Fl) - p.k_lo);
    t.t0 = __double2float_rn(F - Fl);
    double sa, ca;
    sincospi(2.0 * lam[1], &sa, &ca);
    const double c2 = 1.0 - lam[2] * lam[2];
    const double cd = sqrt(c2 > 0.0 ? c2 : 0.0);
    const double n0 = cd * ca, n1 = cd * sa, n2 = lam[2];
    const double A = F * lam[3] * lam[4];
    t.ax = __double2float_rn(F * n0);
    t.ay = __double2float_rn(F * n1);
    t.az = __double2float_rn(F * n2);
    t.A = __double2float_rn(A);
    t.wx = __double2float_rn(n0);
    t.wy = __double2float_rn(n1);
    t.wz = __double2float_rn(n2);
    const double nu = lam[4] * 0.15915494309189533577;  // Omega / 2 pi
    const unsigned long long nu_q = __double2ull_rn(nu * 18014398509481984.0);
    t.nlo = static_cast<unsigned>(nu_q);
    t.nhi = static_cast<unsigned>(nu_q >> 32);
    const unsigned long long psi_q = __double2ull_rz(lam[5] * 18446744073709551616.0);
    t.npsi = 0u - static_cast<unsigned>(psi_q >> 32);
    if (sl != nullptr) {
        sl[0 * kBtThreads + q] = F - static_cast<double>(p.k_lo);
        sl[1 * kBtThreads + q] = F * n0;
        sl[2 * kBtThreads + q] = F * n1;
        sl[3 * kBtThreads + q] = F * n2;
        sl[4 * kBtThreads + q] = A;
        sl[5 * kBtThreads + q] = lam[4];
        sl[6 * kBtThreads + q] = 6.283185307179586476925286766559 * lam[5];
    }
    const double x = F - static_cast<double>(p.k_lo), reach = F * p.vmax + fabs(A) + 1e-3;
    return floor(x - reach + 0.5) >= 0.0 && floor(x + reach + 0.5) <= static_cast<double>(p.W - 1);
}

// cos(2 pi ph / 2^32) of the screen, within kBtCosErr
__device__ __forceinline__ float bt_cos(unsigned ph)
{
    return __cosf(__fmul_rn(__int2float_rn(static_cast<int>(ph)), kBtPhRad));
}

// t = X - K of the FP32 screen (see above)
__device__ __forceinline__ float bt_t(const BtTmpl &t, float4 v, uint2 tq)
{
    const unsigned ph = __umulhi(t.nlo, tq.x) + t.nlo * tq.y + t.nhi * tq.x + t.npsi;
    const float base = __fmaf_rn(v.x, t.ax, __fmaf_rn(v.y, t.ay, __fmaf_rn(v.z, t.az, t.t0)));
    return __fmaf_rn(-t.A, bt_cos(ph), base);
}

// rint(t) as an integer (|t| < 2^22) and whether t is within delta of a rounding boundary
__device__ __forceinline__ int bt_round(float tv, float half_delta, bool &near)
{
    const float r = __fadd_rn(tv, kMagic);
    const float d = __fsub_rn(tv, __fsub_rn(r, kMagic));
    near = fabsf(d) > half_delta;
    return __float_as_int(r) - __float_as_int(kMagic);
}

// The FP64 bin (band column) of one (template, SFT): Eq. (track) from the template's FP64
// terms sl[0..6] (stride `st`) and the SFT's FP64 velocity and time.
__device__ __noinline__ int bt_bin64(const double *sl, int st, const double *v, double t)
{
    const double vn = sl[st] * v[0] + sl[2 * st] * v[1] + sl[3 * st] * v[2];
    const double X = (sl[0] + vn) - sl[4 * st] * cos(sl[5 * st] * t - sl[6 * st]);
    return static_cast<int>(floor(X + 0.5));
}

// Bin of one (template, SFT): the screen, or the FP64 decision near a rounding boundary.
__device__ __forceinline__ int bt_bin(const BtParams &p, const BtTmpl &t, const double *sl, int st,
                                      int a, float4 v, uint2 tq, bool &dec)
{
    const int kr = bt_round(bt_t(t, v, tq), p.half_delta, dec);
    if (dec)
        return bt_bin64(sl, st, p.v64 + 3ll * a, p.t64[a]);
    return t.K + kr;
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

// acc += P[k] (0 outside the band) with an FP32 accumulator; 16-bit values go straight into
// a mixed-precision FMA against 1 (exact product), with no conversion step.
template <typename T>
__device__ __forceinline__ void bt_add(float &acc, const unsigned char *row, int k, bool in);
template <>
__device__ __forceinline__ void bt_add<float>(float &acc, const unsigned char *row, int k, bool in)
{
    acc = __fadd_rn(acc, in ? reinterpret_cast<const float *>(row)[k] : 0.f);
}
template <>
__device__ __forceinline__ void bt_add<__half>(float &acc, const unsigned char *row, int k, bool in)
{
    const unsigned short h = in ? reinterpret_cast<const unsigned short *>(row)[k] : 0;
    asm("{\n\t.reg .b16 one;\n\tmov.b16 one, 0x3C00;\n\tfma.rn.f32.f16 %0, %1, one, %0;\n\t}"
        : "+f"(acc)
        : "h"(h));
}
template <>
__device__ __forceinline__ void bt_add<__nv_bfloat16>(float &acc, const unsigned char *row, int k, bool in)
{
    const unsigned short h = in ? reinterpret_cast<const unsigned short *>(row)[k] : 0;
    asm("{\n\t.reg .b16 one;\n\tmov.b16 one, 0x3F80;\n\tfma.rn.f32.bf16 %0, %1, one, %0;\n\t}"
        : "+f"(acc)
        : "h"(h));
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

__device__ __forceinline__ void fold2(float &hi, float &lo, float part)
{
    const float s = __fadd_rn(hi, part);
    const float bp = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(part, bp)));
    hi = s;
}

// The rows of one stage for this thread's templates.  CHECK: bins may leave [0, W) (then
// they add 0 and are counted); without it every track of the CTA is proven inside.
// Rows r0 .. r0 + RG - 1 of one stage for this thread's templates: the screen of all RG x
// kBtTPT (template, SFT) pairs first, one branch to the FP64 decisions for any of them, then
// the reads and adds.  CHECK: bins may leave [0, W) (then they add 0 and are counted);
// without it every track of the CTA is proven inside.
template <typename T, bool WEIGHTED, bool SKY, bool CHECK, int RG>
__device__ __forceinline__ void bt_row_group(const BtParams &p, const BtTmpl (&t)[kBtTPT], const bool (&valid)[kBtTPT],
                                             const double *sl, int a0, int r0, const float4 *svb, const uint2 *tqs,
                                             const unsigned char *rb, const float4 *sdb,
                                             float (&part)[kBtTPT], float (&partB)[kBtTPT], float (&partC)[kBtTPT],
                                             int (&oob)[kBtTPT], unsigned &n64)
{
    int k[RG][kBtTPT];
    bool dec[RG][kBtTPT];
    bool any = false;
#pragma unroll
    for (int g = 0; g < RG; ++g) {
        const float4 v = svb[r0 + g];
        const uint2 tq = tqs[r0 + g];
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u) {
            k[g][u] = t[u].K + bt_round(bt_t(t[u], v, tq), p.half_delta, dec[g][u]);
            any |= dec[g][u];
        }
    }
    if (any) {
        // near a rounding boundary: the FP64 bin decides
#pragma unroll
        for (int g = 0; g < RG; ++g) {
            const int a = a0 + r0 + g;
#pragma unroll
            for (int u = 0; u < kBtTPT; ++u)
                if (dec[g][u]) {
                    k[g][u] = bt_bin64(sl + threadIdx.x + u * kBtBlock, kBtThreads, p.v64 + 3ll * a, p.t64[a]);
                    n64 += valid[u] ? 1u : 0u;
                }
        }
    }
#pragma unroll
    for (int g = 0; g < RG; ++g) {
        const int r = r0 + g;
        const unsigned char *row = rb + static_cast<size_t>(r) * p.row_bytes;
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u) {
            const bool in = !CHECK || static_cast<unsigned>(k[g][u]) < static_cast<unsigned>(p.W);
            if (CHECK)
                oob[u] += in ? 0 : 1;
            if (SKY) {
                const float val = in ? bt_load<T>(row, k[g][u]) : 0.f;
                const float rw = ft_sky_r32(sdb[2 * r], sdb[2 * r + 1], t[u].wx, t[u].wy, t[u].wz);
                part[u] = __fmaf_rn(rw, val, part[u]);
                partB[u] = __fadd_rn(partB[u], rw);
                partC[u] = __fmaf_rn(rw, rw, partC[u]);
            } else if (WEIGHTED) {
                const float val = in ? bt_load<T>(row, k[g][u]) : 0.f;
                part[u] = __fmaf_rn(svb[r].w, val, part[u]);
            } else {
                bt_add<T>(part[u], row, k[g][u], in);
            }
        }
    }
}

// The rows of one stage for this thread's templates, kBtRowGroup at a time.
template <typename T, bool WEIGHTED, bool SKY, bool CHECK>
__device__ __forceinline__ void bt_rows(const BtParams &p, const BtTmpl (&t)[kBtTPT], const bool (&valid)[kBtTPT],
                                        const double *sl, int a0, int nr, const float4 *svb, const uint2 *tqs,
                                        const unsigned char *rb, const float4 *sdb,
                                        float (&part)[kBtTPT], float (&partB)[kBtTPT], float (&partC)[kBtTPT],
                                        int (&oob)[kBtTPT], unsigned &n64)
{
    // (the all-sky weighted loop keeps one row per group: its weight terms need the registers)
    constexpr int RG = SKY ? 1 : kBtRowGroup;
    int r = 0;
    for (; r + RG <= nr; r += RG)
        bt_row_group<T, WEIGHTED, SKY, CHECK, RG>(p, t, valid, sl, a0, r, svb, tqs, rb, sdb, part, partB,
                                                           partC, oob, n64);
    for (; r < nr; ++r)
        bt_row_group<T, WEIGHTED, SKY, CHECK, 1>(p, t, valid, sl, a0, r, svb, tqs, rb, sdb, part, partB, partC,
                                                 oob, n64);
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
    float4 *sd[2] = {reinterpret_cast<float4 *>(bars + 2), nullptr};  // 16-byte aligned
    sd[1] = sd[0] + 2 * p.S;

    // this CTA's templates
    const long long cta = p.cta_base + blockIdx.x;
    long long t_begin, t_end;
    if (p.box_mode) {
        const long long box = cta / p.tiles_per_box;
        const long long tile = cta % p.tiles_per_box;
        t_begin = box * p.n_per_box + tile * kBtThreads;
        t_end = min(t_begin + kBtThreads, (box + 1) * p.n_per_box);
    } else {
        t_begin = p.first + cta * kBtThreads;
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

    __shared__ unsigned s_done[2];
    __shared__ int s_issued[2];  // the last stage copied into each buffer (-1: none)
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        ftp::mbar_init(&bars[0], 1);
        ftp::mbar_init(&bars[1], 1);
        ftp::fence_mbar_init();
        s_done[0] = s_done[1] = 0;
        s_issued[0] = 0;
        s_issued[1] = p.n_stages > 1 ? 1 : -1;
        s_abort = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        bt_issue(p, 0, rows[0], sv[0], stq[0], sd[0], &bars[0]);
        if (p.n_stages > 1)
            bt_issue(p, 1, rows[1], sv[1], stq[1], sd[1], &bars[1]);
    }

    // the templates' FP32 screen terms in registers, their FP64 terms in this CTA's slot of
    // the launch scratch (read back by this thread only, for the FP64 decisions)
    double *sl = p.slow + static_cast<size_t>(blockIdx.x) * (kBtSlow * kBtThreads);
    BtTmpl t[kBtTPT];
    bool inside = true;
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        double lam[6];
        bt_lambda(p, valid[u] ? ti[u] : t_begin, lam);
        inside &= bt_derive(p, lam, t[u], sl, threadIdx.x + u * kBtBlock);
    }
    // one loop for the whole CTA: unchecked only when every track stays inside the band
    inside = __syncthreads_and(inside) != 0;

    float hi[kBtTPT], lo[kBtTPT];
    // all-sky weights: sum r, sum r^2 (r = (a^2 + b^2) / S_n), compensated like the sum
    float hiB[kBtTPT], loB[kBtTPT], hiC[kBtTPT], loC[kBtTPT];
    int oob[kBtTPT];
#pragma unroll
    for (int u = 0; u < kBtTPT; ++u) {
        hi[u] = lo[u] = hiB[u] = loB[u] = hiC[u] = loC[u] = 0.f;
        oob[u] = 0;
    }
    unsigned n64 = 0;
    // No CTA barrier per stage: each warp releases a buffer when it is done with it, and the
    // last warp to release it refills it with the stage after next, so a warp slowed down by
    // FP64 decisions holds the others back only when they are a whole stage ahead.
    // s_done[b] counts releases of buffer b: stage st is its (st / 2)-th use.
    const int lane = threadIdx.x & 31;
    constexpr unsigned kWarps = kBtBlock / 32;
    for (int st = 0; st < p.n_stages; ++st) {
        const int b = st & 1;
        if (*reinterpret_cast<volatile int *>(&s_abort) != 0)
            break;
        const bool ok = __all_sync(0xffffffffu, ftp::mbar_wait_bounded(&bars[b], (st >> 1) & 1));
        if (!ok) {
            if (lane == 0)
                atomicExch(&s_abort, 1);
            break;
        }
        const int nr = min(p.S, p.N - st * p.S);
        float part[kBtTPT], partB[kBtTPT], partC[kBtTPT];
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u)
            part[u] = partB[u] = partC[u] = 0.f;
        const uint2 *tqs = reinterpret_cast<const uint2 *>(stq[b]);
        if (inside)
            bt_rows<T, WEIGHTED, SKY, false>(p, t, valid, sl, st * p.S, nr, sv[b], tqs, rows[b], sd[b],
                                             part, partB, partC, oob, n64);
        else
            bt_rows<T, WEIGHTED, SKY, true>(p, t, valid, sl, st * p.S, nr, sv[b], tqs, rows[b], sd[b],
                                            part, partB, partC, oob, n64);
        // compensated folds of the stage's partials (2Sum)
#pragma unroll
        for (int u = 0; u < kBtTPT; ++u) {
            fold2(hi[u], lo[u], part[u]);
            if (SKY) {
                fold2(hiB[u], loB[u], partB[u]);
                fold2(hiC[u], loC[u], partC[u]);
            }
        }
        // release buffer b: the warp's reads of it are done before lane 0 counts the release
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&s_done[b], 1u) + 1u == kWarps * static_cast<unsigned>((st >> 1) + 1) ? 1u : 0u;
        }
        if (__shfl_sync(0xffffffffu, last, 0) != 0 && st + 2 < p.n_stages) {
            // every warp's reads of the buffer come before the copies that overwrite it
            __threadfence_block();
            ftp::fence_proxy_async_smem();
            bt_issue(p, st + 2, rows[b], sv[b], stq[b], sd[b], &bars[b]);
            if (lane == 0)
                s_issued[b] = st + 2;
        }
    }
    if (p.n64 != nullptr) {
        const unsigned w64 = __reduce_add_sync(0xffffffffu, n64);
        if (lane == 0 && w64 != 0)
            atomicAdd(p.n64, static_cast<unsigned long long>(w64));
    }
    // every warp is past its last read of the stage buffers (the epilogue reuses them)
    __syncthreads();
    if (s_abort != 0) {
        if (threadIdx.x == 0) {
            atomicOr(p.status, FT_STATUS_TIMEOUT);
            // let the last copies issued into each buffer land before the shared memory is
            // released (stage s is phase s / 2 of its buffer's barrier)
            for (int b2 = 0; b2 < 2; ++b2)
                if (s_issued[b2] >= 0)
                    (void)ftp::mbar_wait_bounded(&bars[b2], (s_issued[b2] >> 1) & 1);
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
    const int n_here = static_cast<int>(t_end - t_begin);
    float last_s = INFINITY;
    long long last_t = -1;
    ft_candidate *out = p.cand + cta * p.k;
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

// Bins of templates tmpl[0..n) in every SFT: one CTA per template, the same screen and
// FP64 decisions as the evaluation kernel.
__global__ void __launch_bounds__(256) k_bt_bins(const BtParams p, const long long *tmpl, long long n, int *bins)
{
    __shared__ BtTmpl ts;
    __shared__ double sl[kBtSlow * kBtThreads];
    const long long i = blockIdx.x;
    if (i >= n)
        return;
    if (threadIdx.x == 0) {
        double lam[6];
        bt_lambda(p, tmpl[i], lam);
        BtTmpl t;
        bt_derive(p, lam, t, sl, 0);
        ts = t;
    }
    __syncthreads();
    const BtTmpl t = ts;
    for (int a = threadIdx.x; a < p.N; a += blockDim.x) {
        const long long tq = p.tq[a];
        bool dec;
        bins[i * p.N + a] = bt_bin(p, t, sl, kBtThreads, a, p.rowv[a],
                                   make_uint2(static_cast<unsigned>(tq), static_cast<unsigned>(
                                                  static_cast<unsigned long long>(tq) >> 32)),
                                   dec);
    }
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

// Largest |bt_cos(ph) - cos(2 pi ph / 2^32)| over every 32-bit phase: thread i of the grid
// takes ph = i, i + stride, ... (stride = grid size, a power of two), the reference is the
// FP64 cospi of the exact argument ph 2^-31 (ph read as a signed angle).  The non-negative
// maximum is kept as the bit pattern of a double, whose integer order is its numeric order.
__global__ void __launch_bounds__(256) k_bt_cos_check(unsigned long long *max_bits)
{
    const unsigned stride = gridDim.x * blockDim.x;
    double m = 0.0;
    for (unsigned long long ph = blockIdx.x * blockDim.x + threadIdx.x; ph < (1ull << 32); ph += stride) {
        const unsigned u = static_cast<unsigned>(ph);
        const double ref = cospi(static_cast<double>(static_cast<int>(u)) * 0x1p-31);
        m = fmax(m, fabs(static_cast<double>(bt_cos(u)) - ref));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(max_bits, static_cast<unsigned long long>(__double_as_longlong(m)));
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

// The FP32 screen's error bound (bins) for this band and bank, against the exact real
// t* = X - K (all terms below are bounds; u = 2^-24 is the FP32 unit roundoff):
//   t0 = FP32(frac F) in [0, 1): u;
//   a.v with a = FP32(F n), v = FP32(v / c): inputs 2u |a| |v| = 2u F|v| (Cauchy-Schwarz),
//     three FMA roundings 3u (1 + F|v|) (every partial sum is below 1 + F|v|);
//   A = FP32(F a_p Omega): u A;  the final FMA: u (1 + F|v| + A);
//   the cosine of the integer phase: kBtCosErr (conversion, scale and __cosf), times A;
//   the orbit phase: the dropped borrow (2^-32 turn), nu rounded to 2^-55 turn/s times the
//     largest |t|, t rounded to 2^-11 s times the largest nu: times 2 pi A.
// So delta = u (5 + 6 F|v| + 2 A) + A (kBtCosErr + e_phase), taken with a 1.5 safety factor
// and the FP64 decision's own rounding (1e-9) added.  F, |v|, A and nu are the largest over
// the bank and band.
double bt_delta(const ft_band *band, const ft_binary_bank *bk)
{
    const double u = 0x1p-24;
    const double F = std::fabs(bk->desc.hi[0]) * band->t_sft;
    const double Fv = F * band->vmax;
    const double A = F * std::fabs(bk->desc.hi[3]) * std::fabs(bk->desc.hi[4]);
    double tmax = 0.0;
    for (double t : band->h_dt)
        tmax = std::max(tmax, std::fabs(t));
    const double nu = std::fabs(bk->desc.hi[4]) / 6.283185307179586;
    const double e_ph = 6.283185307179586 * (0x1p-32 + 0x1p-55 * tmax + 0x1p-11 * nu);
    const double e = u * (5.0 + 6.0 * Fv + 2.0 * A) + A * (kBtCosErr + e_ph);
    return 1.5 * e + 1e-9;
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
    p.v64 = band->d_v;
    p.t64 = bk->d_t64;
    p.n64 = bk->d_n64;
    p.half_delta = std::nextafter(static_cast<float>(0.5 - bk->delta), 0.0f);
    p.vmax = band->vmax;
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
    // at most 16 KB of rows per stage, 8..64 rows (a divisor of kBtRowPad): two stages
    // leave room for 4 CTAs per SM, as many as the registers allow
    const int rb = band->Wp * elem_bytes(band->dtype);
    int S = 64;
    while (S > 8 && S * rb > 16 * 1024)
        S >>= 1;
    return S;
}

size_t eval_smem(const BtParams &p)
{
    return 2 * (static_cast<size_t>(p.S) * p.row_bytes + p.S * 24) + 16 +
           (p.rowd != nullptr ? 2 * static_cast<size_t>(p.S) * 32 : 0);
}

// Launches n_cta CTAs in chunks of at most 8 waves: every chunk's CTAs keep their FP64
// template terms in one scratch slot each (kBtSlow x kBtThreads doubles), reused by the next
// chunk.  With cand_bytes > 0 the per-CTA candidate lists come first in the same scratch
// (*cand set to them).
template <typename T, bool Wt>
int launch_t(ft_ctx *ctx, long long n_cta, size_t smem, BtParams p, size_t cand_bytes,
             ft_candidate **cand, cudaStream_t st)
{
    auto fn = p.rowd != nullptr ? k_bt_eval<T, false, true> : k_bt_eval<T, Wt, false>;
    FT_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    FT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBtBlock, smem));
    const long long chunk = std::min<long long>(n_cta, 8ll * std::max(per_sm, 1) * std::max(ctx->sm_count, 1));
    const size_t off = (cand_bytes + 255) / 256 * 256;
    void *scr = nullptr;
    FT_TRY(ft_ctx_scratch(ctx, off + static_cast<size_t>(chunk) * kBtSlow * kBtThreads * sizeof(double), &scr));
    if (cand != nullptr)
        *cand = static_cast<ft_candidate *>(scr);
    p.cand = static_cast<ft_candidate *>(scr);
    p.slow = reinterpret_cast<double *>(static_cast<char *>(scr) + off);
    for (long long c0 = 0; c0 < n_cta; c0 += chunk) {
        p.cta_base = c0;
        fn<<<static_cast<unsigned>(std::min(chunk, n_cta - c0)), kBtBlock, smem, st>>>(p);
        FT_CUDA(cudaGetLastError());
    }
    return FT_OK;
}

int launch_eval(const ft_band *band, long long n_cta, BtParams p, size_t cand_bytes, ft_candidate **cand,
                cudaStream_t st)
{
    p.S = stage_rows(band);
    p.n_stages = static_cast<int>((band->N + p.S - 1) / p.S);
    const size_t smem = std::max(eval_smem(p), static_cast<size_t>(2 * kBtThreads * 4));
    if (smem > band->ctx->smem_optin)
        FT_FAIL(FT_ERR_RANGE, "binary: band rows too wide for the shared-memory stages");
    if (n_cta <= 0)
        return FT_OK;
    ft_ctx *ctx = band->ctx;
    const bool w = band->weighted;
    switch (band->dtype) {
    case FT_F32:
        return w ? launch_t<float, true>(ctx, n_cta, smem, p, cand_bytes, cand, st)
                 : launch_t<float, false>(ctx, n_cta, smem, p, cand_bytes, cand, st);
    case FT_F16:
        return w ? launch_t<__half, true>(ctx, n_cta, smem, p, cand_bytes, cand, st)
                 : launch_t<__half, false>(ctx, n_cta, smem, p, cand_bytes, cand, st);
    case FT_BF16:
        return w ? launch_t<__nv_bfloat16, true>(ctx, n_cta, smem, p, cand_bytes, cand, st)
                 : launch_t<__nv_bfloat16, false>(ctx, n_cta, smem, p, cand_bytes, cand, st);
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
    std::vector<double> t64(b->n_pad, 0.0);
    for (int a = 0; a < N; ++a)
        t64[a] = band->h_dt[a];
    if (cudaMalloc(&b->d_rowv, static_cast<size_t>(b->n_pad) * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&b->d_tq, static_cast<size_t>(b->n_pad) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_t64, static_cast<size_t>(b->n_pad) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_n64, sizeof(unsigned long long)) != cudaSuccess) {
        ft_set_error("make_binary_bank: allocation failed");
        return fail(FT_ERR_OOM);
    }
    if (cudaMemcpy(b->d_tq, tq.data(), tq.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_t64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_n64, 0, sizeof(unsigned long long)) != cudaSuccess) {
        ft_set_error("make_binary_bank: copy failed");
        return fail(FT_ERR_CUDA);
    }
    b->delta = bt_delta(band, b);
    k_bt_rowv<<<(b->n_pad + 255) / 256, 256>>>(band->d_v, band->d_w, N, b->n_pad, b->d_rowv);
    if (band->d_D) {
        if (cudaMalloc(&b->d_rowd, static_cast<size_t>(b->n_pad) * 2 * sizeof(float4)) != cudaSuccess) {
            b->d_rowd = nullptr;
            ft_set_error("make_binary_bank: allocation failed");
            return fail(FT_ERR_OOM);
        }
        if (ft_launch_rowd(band->d_D, band->d_sn, N, b->n_pad, b->d_rowd, 0) != FT_OK)
            return fail(FT_ERR_CUDA);
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
    cudaFree(b->d_t64);
    cudaFree(b->d_n64);
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

int ft_binary_decisions(ft_binary_bank *bank, uint64_t *n_fp64, double *delta)
{
    if (!bank)
        FT_FAIL(FT_ERR_ARG, "binary_decisions: null bank");
    Guard g(bank->device);
    unsigned long long h = 0;
    FT_CUDA(cudaDeviceSynchronize());
    FT_CUDA(cudaMemcpy(&h, bank->d_n64, sizeof(h), cudaMemcpyDeviceToHost));
    FT_CUDA(cudaMemset(bank->d_n64, 0, sizeof(unsigned long long)));
    if (n_fp64)
        *n_fp64 = h;
    if (delta)
        *delta = bank->delta;
    return FT_OK;
}

int ft_binary_cos_screen_check(ft_ctx *ctx, double *max_abs_err, double *bound)
{
    if (!ctx || !max_abs_err)
        FT_FAIL(FT_ERR_ARG, "binary_cos_screen_check: null argument");
    Guard g(ctx->device);
    void *scr = nullptr;
    FT_TRY(ft_ctx_scratch(ctx, sizeof(unsigned long long), &scr));
    auto *d = static_cast<unsigned long long *>(scr);
    FT_CUDA(cudaMemset(d, 0, sizeof(unsigned long long)));
    // 2^18 threads of 2^14 phases each
    k_bt_cos_check<<<1024, 256>>>(d);
    FT_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    FT_CUDA(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost));
    double m;
    std::memcpy(&m, &h, sizeof(m));
    *max_abs_err = m;
    if (bound)
        *bound = kBtCosErr;
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
        // the int64 template indices after the bins, at an aligned offset
        const size_t off = (nb + 255) / 256 * 256;
        FT_TRY(ft_ctx_outbuf(ctx, off + static_cast<size_t>(n) * 8, &buf));
        db = static_cast<int *>(buf);
        long long *t = reinterpret_cast<long long *>(static_cast<char *>(buf) + off);
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
    FT_TRY(launch_eval(band, (n + kBtThreads - 1) / kBtThreads, p, 0, nullptr, st));
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
    ft_candidate *cand = nullptr;
    FT_TRY(launch_eval(band, n_cta, p, cand_bytes, &cand, st));
    k_bt_merge<<<static_cast<unsigned>(bank->n_boxes), 256, 0, st>>>(cand, p.tiles_per_box, k, dout);
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
