// ft_internal.cuh -- shared internals of the fasttracks CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/fasttracks.h"

// ------------------------------------------------------------------ host error plumbing

void ft_set_error(const std::string &msg);

#define FT_FAIL(code, msg)              \
    do {                                \
        ft_set_error(msg);              \
        return (code);                  \
    } while (0)

#define FT_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ft_set_error(std::string(#call) + ": " + cudaGetErrorString(e_));              \
            return (e_ == cudaErrorMemoryAllocation) ? FT_ERR_OOM : FT_ERR_CUDA;           \
        }                                                                                  \
    } while (0)

#define FT_TRY(call)            \
    do {                        \
        int rc_ = (call);       \
        if (rc_ != FT_OK)       \
            return rc_;         \
    } while (0)

// device status word bits
#define FT_STATUS_TIMEOUT 1u
#define FT_STATUS_NONFINITE 2u
#define FT_STATUS_WINDOW 4u

// ------------------------------------------------------------------ handles

struct ft_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    unsigned int *d_status = nullptr;  // device status word (FT_STATUS_*)
    void *scratch = nullptr;           // grown on demand; candidate lists etc.
    size_t scratch_bytes = 0;
    void *outbuf = nullptr;            // device staging for host outputs
    size_t outbuf_bytes = 0;
    ft_tune tune = {0, 0, 0};          // launch-shape override (zeros: built-in choice)
};

struct ft_band {
    ft_ctx *ctx = nullptr;
    int device = 0;  // kept so that destruction never needs the context
    int n_det = 0;
    std::vector<int> n_sft;
    int64_t N = 0;        // total rows
    int W = 0;            // bins per row
    int Wp = 0;           // padded bins per row copy (FP32: one copy; 16-bit: even + odd copies)
    int64_t k_lo = 0;
    double t_sft = 0, t0 = 0;
    int dtype = FT_F32;
    void *d_power = nullptr;  // [N][Wp] FP32, or [N][2][Wp] 16-bit (even / odd-shifted copies)
    double *d_tau = nullptr;  // [N] (t_mid - t0) * T_SFT
    double *d_v = nullptr;    // [N][3]
    float *d_w = nullptr;     // [N]
    double *d_sn = nullptr;   // [N] or null
    double mu = 0, sigma = 0;
    bool weighted = false;
    std::vector<double> h_tau, h_vabs;
    std::vector<double> h_dt;  // t_mid - t0 (s), FP64 as given
    double tau_absmax = 0;
    double vmax = 0;  // largest |v| / c over the SFTs
    double *d_D = nullptr;  // [N][6] detector tensors when the all-sky weights are on
    // [N][2] their FP32 records for the kernels: D / sqrt(S_n) as (D00, D01, D02, D11),
    // (D12, D22, |D|^2, tr D), so that (a^2 + b^2) / S_n = ft_sky_r32(record, n)
    float4 *d_rowd = nullptr;
    // mean and variance of one SFT's value in Gaussian noise: 2 and 4 for normalised power
    // (exponential with mean 2); p and p (1 - p) for a number-count band, p = exp(-threshold / 2)
    double m1 = 2.0, v1 = 4.0;
    bool number_count = false;
};

struct ft_bank {
    ft_ctx *ctx = nullptr;
    int device = 0;
    const ft_band *band = nullptr;
    int64_t k0 = 0;
    int n_f0 = 0, n_f1 = 0;
    int64_t n_sky = 0;
    int sub = 1;
    int n_sub = 0;
    double *d_f1 = nullptr;    // [n_f1]
    double *d_sky = nullptr;   // [n_sky][3]
    // the sky points in an order that keeps neighbours on the sky together, so that a CTA
    // can search P consecutive ones over the same shared-memory rows; sky_dmax[P] is the
    // largest distance between two points of one such group of P (P <= kMaxSkyGroup)
    int *d_sky_order = nullptr;
    double sky_dmax[5] = {};
    // all-sky weights (band with detector tensors): per sky point 1 / sum_alpha (a^2+b^2)/S_n,
    // and mu_G, sigma_G of the normalised weights
    double *d_sky_inv = nullptr, *d_sky_mu = nullptr, *d_sky_sig = nullptr;
    long long *d_G = nullptr;  // [n_f1][N] Q32 f1*tau
    bool window_safe = false;
    double f1_lo = 0, f1_hi = 0;
};

int ft_ctx_scratch(ft_ctx *ctx, size_t bytes, void **p);

// The evaluation kernels weight the rows: per-SFT weights other than 1, or all-sky weights.
inline bool ft_band_weighted(const ft_band *b)
{
    return b->weighted || b->d_D != nullptr;
}
int ft_ctx_outbuf(ft_ctx *ctx, size_t bytes, void **p);
// Synchronise `st`, report and clear the device status word (FT_ERR_TIMEOUT etc.).
int ft_read_status(ft_ctx *ctx, cudaStream_t st);

// ------------------------------------------------------------------ kernel parameters

struct FtCand {
    float s;
    float z;
    long long t;
};

struct EvalParams {
    // tiled view of the power rows for one-instruction window copies of a whole stage:
    // 16-byte groups x groups per row copy (x 2 copies for 16-bit storage) x rows, box
    // (S rows, Ws bins); rows_map_ok = 0 when the launch shape has no such view
    CUtensorMap rows_map;
    int rows_map_ok;
    const void *power;
    int row_bytes;  // bytes per stored row (FP32 row, or the two 16-bit copies)
    int Wp;         // bins per stored row copy
    int Ws;         // bins per shared-memory row window (fast kernels)
    int srow_bytes; // bytes per shared-memory row (Ws bins, FP32 or the two 16-bit copies)
    int row_elems;  // storage elements per stored row
    int W;
    long long N;
    const double *tau;
    const double *v;
    const float *w;
    // all-sky weights (null: per-SFT w): w_alpha(n) = (a^2 + b^2)(D_alpha, n) / S_n,alpha
    // times sky_inv[n]; z uses sky_mu[n], sky_sig[n]
    const double *D, *sn, *sky_inv, *sky_mu, *sky_sig;
    const float4 *rowd;  // [N][2] FP32 records of D / sqrt(S_n) (see ft_band::d_rowd)
    // candidate gate (null: none): template t takes part in the selection only when
    // gate[t] >= gate_min (e.g. its weighted number count)
    const float *gate;
    float gate_min;
    const double *sky;
    const int *sky_order;  // [n_sky] CTA sky groups are runs of P in this order (null: identity)
    const long long *G;  // [n_f1][N]
    const double *f1;    // [n_f1]
    long long K0, k_lo;
    int n_f0, n_f1;
    long long n_sky;
    int n_f1g, n_f0t;  // f1 groups (F1 f1 values each) and f0 tiles (32*R each)
    int P, F1;         // sky points per CTA and f1 values per sky point: warps = P * F1
    long long n_skyg;  // sky groups: ceil(n_sky / P)
    int S, n_stages;   // SFT rows per stage
    int nst;           // pipeline slots (fast kernel)
    double mu, sigma;
    float *s_out;
    float *z_out;
    int *oob_out;
    FtCand *cand;  // per-CTA candidate lists [n_cta][lsub_max][k]
    int k, sub, lsub_max;
    unsigned int *status;
};

// The evaluation parameters every search of (band, bank) shares: data, bank, weights,
// noise moments and the status word; the launch shape and the outputs are left zero.
inline EvalParams ft_eval_base_params(const ft_band *band, const ft_bank *bank)
{
    EvalParams p;
    memset(&p, 0, sizeof(p));
    p.power = band->d_power;
    p.W = band->W;
    p.N = band->N;
    p.tau = band->d_tau;
    p.v = band->d_v;
    p.w = band->d_w;
    if (band->d_D) {
        p.D = band->d_D;
        p.sn = band->d_sn;
        p.rowd = band->d_rowd;
        p.sky_inv = bank->d_sky_inv;
        p.sky_mu = bank->d_sky_mu;
        p.sky_sig = bank->d_sky_sig;
    }
    p.sky = bank->d_sky;
    p.G = bank->d_G;
    p.f1 = bank->d_f1;
    p.K0 = bank->k0;
    p.k_lo = band->k_lo;
    p.n_f0 = bank->n_f0;
    p.n_f1 = bank->n_f1;
    p.n_sky = bank->n_sky;
    p.mu = band->mu;
    p.sigma = band->sigma;
    p.status = band->ctx->d_status;
    return p;
}

// Persistent multi-band launch: band-major work list of tiles, running candidate lists.
struct BatchParams {
    const EvalParams *params;      // [n_bands], device
    const long long *tile_prefix;  // [n_bands + 1], device
    const int *n_sub;              // [n_bands] sub-bands per band
    int n_bands;
    int k;
    int n_sub_max;                 // max sub-bands over the bands
    int lsub_max;                  // max sub-bands met by one tile
    size_t list_off;               // shared-memory offset of the candidate lists
    unsigned long long *counter;   // zeroed before the launch
    ft_candidate *scr;             // [gridDim.x][n_bands][n_sub_max][k], pre-filled empty
};

// launch helpers implemented in ft_eval.cu
struct EvalShape {
    int J;       // f0 values per CTA tile (32 x slots per lane)
    int F;       // evaluating warps per CTA: P sky points x F1 f1 values
    int P;       // sky points per CTA
    int F1;      // f1 values per CTA
    int S;       // SFT rows per stage
    int nbuf;    // stage buffers
    bool fast;   // shifted-row kernel (bank tracks provably inside the window)
    int Ws;      // fast kernel: bins per shared-memory row window
};

// Bins per shared-memory row window of the fast kernels for tile width J and P sky points
// per CTA: the tile, the spread of the track origins over the bank's f1 range and over a
// sky group, carry and alignment slack.
int ft_window_bins(const ft_band *band, const ft_bank *bank, int J, int P);

// Sky points per CTA and f1 values per CTA for a bank whose f1 values are split into groups
// of at most max_warps: P * F1 <= max_warps, P <= kMaxSkyGroup.
void ft_sky_grouping(const ft_bank *bank, int max_warps, int *P, int *F1);
constexpr int kMaxSkyGroup = 4;

// Tiled tensor-map view of the band's power rows with a (S rows, Ws bins) box; returns 0
// and sets *ok = 0 when the shape cannot be expressed (box larger than the hardware allows).
int ft_encode_rows_map(const ft_band *band, int Ws, int S, CUtensorMap *map, int *ok);

// (a^2 + b^2) / S_n in FP32 (Sec. II.B), where a = D : e+ and b = D : ex in any wave frame
// perpendicular to the unit direction n, from an SFT's record d0 = (e00, e01, e02, e11),
// d1 = (e12, e22, |e|^2, tr e) of e = D / sqrt(S_n) (D = xx, xy, xz, yy, yz, zz).  a^2 + b^2
// is twice the squared norm of the transverse-traceless part of D, so
//     (a^2 + b^2) / S_n = 2 |e|^2 - 4 |u|^2 + 2 c^2 - (tr e - c)^2,   u = e n, c = n . u,
// which needs no frame (no square root or division; exact algebraically).  The terms are
// O(1 / S_n), so the result is good to a few FP32 ulps of 1 / S_n in absolute terms: the
// weights it makes are stored in FP32 anyway.
__device__ __forceinline__ float ft_sky_r32(float4 d0, float4 d1, float nx, float ny, float nz)
{
    const float u0 = d0.x * nx + d0.y * ny + d0.z * nz;
    const float u1 = d0.y * nx + d0.w * ny + d1.x * nz;
    const float u2 = d0.z * nx + d1.x * ny + d1.y * nz;
    const float c = nx * u0 + ny * u1 + nz * u2;
    const float uu = u0 * u0 + u1 * u1 + u2 * u2;
    const float tc = d1.w - c;
    return 2.f * d1.z - 4.f * uu + 2.f * c * c - tc * tc;
}

// The FP32 records of D / sqrt(S_n) for rows [0, N) of D [N][6], zeros for rows [N, n_pad);
// out [n_pad][2].
int ft_launch_rowd(const double *D, const double *sn, long long N, long long n_pad, float4 *out,
                   cudaStream_t st);

// Per sky point of the bank: 1 / sum (a^2+b^2)/S_n and mu_G, sigma_G of the normalised
// all-sky weights (one CTA per sky point; the band must carry detector tensors).
int ft_launch_sky_norms(const ft_band *band, const ft_bank *bank, cudaStream_t st);
// dst power = 1[src power > threshold] element by element (same layout and storage type;
// the stored value is compared in FP64)
int ft_launch_binarize(const ft_band *src, ft_band *dst, double threshold, cudaStream_t st);

// Runs the gather-roof microbenchmark on the current device (see ft_gather_roof).
int ft_run_gather_roof(int dtype, int sm_count, double *evals_per_s, double *evals_per_clk_sm);

// CTAs of the evaluation grid: sky groups x f1 groups x f0 tiles.
long long ft_grid_ctas(const ft_bank *bank, const EvalShape &sh);

size_t ft_eval_smem_bytes(const ft_band *band, const EvalShape &sh, int k);
// sky_box > 0: the sky group size P is reduced to a divisor of sky_box, so that no CTA's sky
// points straddle two sky boxes (runs of sky_box points of the bank's sky order); f1_box > 0:
// likewise the f1 group size F1 to a divisor of f1_box (runs of f1_box values of the f1 list)
EvalShape ft_default_shape(const ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box = 0,
                           int f1_box = 0);
int ft_launch_eval(const ft_band *band, const ft_bank *bank, const EvalShape &sh, EvalParams p,
                   cudaStream_t st);
// Merge of the per-CTA lists: per sub-band (sky_box = f1_box = 0), or per (sky box, f1 box,
// sub-band) into out [n_sky_boxes][n_f1_boxes][n_sub][k] (sky_box a multiple of sh.P, f1_box
// of sh.F1; 0 = one box over that dimension).
int ft_launch_merge(const ft_bank *bank, const EvalShape &sh, const FtCand *cand, int k,
                    int lsub_max, ft_candidate *out, cudaStream_t st, int sky_box = 0,
                    int f1_box = 0);
int ft_launch_convert(const void *src, int src_dtype, long long src_stride, void *dst,
                      int dst_dtype, long long N, int W, int Wp, unsigned int *status,
                      cudaStream_t st);
int ft_launch_gtable(const double *f1, int n_f1, const double *tau, long long N,
                     long long *G, cudaStream_t st);
int ft_launch_track_bins(const ft_band *band, const ft_bank *bank, const long long *tmpl,
                         long long n, int *bins, cudaStream_t st);

size_t ft_batch_tile_smem(int Ws, int S, int F, int P, int J, int nst, bool weighted);
int ft_batch_row_bytes(const ft_band *band);
int ft_launch_batched(int dtype, bool weighted, int J, int F, const BatchParams &bp, size_t smem,
                      int *grid, bool launch, cudaStream_t st);
int ft_launch_merge_persist(const ft_candidate *scr, int n_ctas, int n_bands, int n_sub_max, int k,
                            const int *sub_prefix, int n_sub_total, ft_candidate *out,
                            cudaStream_t st);
