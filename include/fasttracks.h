/*
 * fasttracks.h -- C ABI of the B300 (sm_103a) short-coherence search engine.
 *
 * The engine evaluates, by brute force, the short-coherence detection statistic of
 * arXiv 2411.18370 over a regular template bank and reduces it to per-sub-band candidates:
 *
 *   s(lambda) = sum_{X,alpha} w_{X alpha} P_X[alpha][k_{X alpha}(lambda)]      Sec. II.B, Eq. (short_coh_general)
 *   k = round-half-up of f(t_alpha) T_SFT - k_lo,
 *   f(t) = (f0 + f1 (t - t0)) (1 + v(t).n / c)                                 Sec. II.A, Eq. (track), a_p = 0
 *   z = (s - mu_G) / sigma_G, mu_G = 2 sum w, sigma_G^2 = 4 sum w^2            Sec. II.B.1, Eq. (critical_ratio)
 *   candidates: the k loudest templates of each disjoint f0 sub-band           Sec. IV.B (ahead-of-time boxes)
 *
 * Track bins are computed exactly: per (sky, SFT) eps = v.n in FP64 with a pinned operation
 * order, then integer Q32 fixed-point arithmetic (see ft_track_bins below for the rule).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns FT_OK (0) or a negative FT_ERR_* code; ft_last_error() gives a
 *   human-readable message for the calling thread's last failure.
 * - Handles (ft_ctx, ft_band, ft_bank) are opaque and owned by the library; release them
 *   with the matching *_destroy.  A band or bank is bound to the context (device) that
 *   created it.
 * - Input arrays passed as host pointers are copied before the call returns; the caller
 *   keeps ownership.
 * - Output buffers are caller-owned.  `out_on_device` = 1 means the pointers are device
 *   pointers on the context's device: the call is asynchronous on `stream`.  0 means host
 *   pointers: the call copies the results back and synchronises `stream` before returning.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 * - Device-side failures (a bounded wait that ran out) are reported as FT_ERR_TIMEOUT by
 *   the next synchronising call or by ft_check_status().
 * - Sizes: template indices are int64; at most 2^31-1 SFT rows, 2^20 bins per row,
 *   |v/c| < 1e-3, |f1 (t - t0) T_SFT| < 2^20 bins.
 */
#ifndef FASTTRACKS_H
#define FASTTRACKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FT_API __attribute__((visibility("default")))
#else
#define FT_API
#endif

#define FT_ABI_VERSION 1

#define FT_OK 0
#define FT_ERR_ARG (-1)         /* invalid argument / descriptor / NaN input          */
#define FT_ERR_CUDA (-2)        /* a CUDA runtime call failed                           */
#define FT_ERR_OOM (-3)         /* device allocation failed                             */
#define FT_ERR_TIMEOUT (-4)     /* a device-side bounded wait ran out                   */
#define FT_ERR_RANGE (-5)       /* sizes or values beyond the documented limits         */
#define FT_ERR_UNSUPPORTED (-6) /* feature not available (e.g. no sm_103 device)       */

/* element types */
#define FT_F32 0
#define FT_F16 1
#define FT_BF16 2
#define FT_F64 3

typedef struct ft_ctx ft_ctx;
typedef struct ft_band ft_band;
typedef struct ft_bank ft_bank;

/* Message of the calling thread's most recent error ("" if none).  Valid until the
 * thread's next failing call. */
FT_API const char *ft_last_error(void);

/* FT_ABI_VERSION of the loaded library. */
FT_API int ft_abi_version(void);

/* Create a context on CUDA device `device`.  Fails with FT_ERR_UNSUPPORTED when the
 * device is not compute capability 10.3 (the kernels are built for sm_103a only). */
FT_API int ft_create(ft_ctx **ctx, int device);
FT_API void ft_destroy(ft_ctx *ctx);

/* Synchronise `stream` and report any device-side failure recorded since the last check
 * (FT_ERR_TIMEOUT), then clear it. */
FT_API int ft_check_status(ft_ctx *ctx, void *stream);

/* Device bytes the context holds for scratch (per-CTA candidate lists and the like, grown on
 * demand by the searches) and for staging host outputs (nullable pointers).  A diagnostic:
 * the paper has no counterpart.  Errors: FT_ERR_ARG (null ctx). */
FT_API int ft_ctx_memory(const ft_ctx *ctx, size_t *scratch_bytes, size_t *staging_bytes);

/* ----------------------------------------------------------------------------- SFTs --
 * A narrow band of normalised SFT power, P = 4|x~|^2/(T_SFT S_n) (Sec. II.B, Eq. (s_tf)),
 * for n_det detectors.  Rows are detector-major: detector 0's n_sft[0] SFTs, then
 * detector 1's, ...; row alpha holds bins k_lo .. k_lo + n_bins - 1 (bin = f T_SFT).
 */
typedef struct {
    int n_det;          /* number of detectors X (>= 1)                                */
    const int *n_sft;   /* host [n_det]: SFTs per detector (>= 0 each, total >= 1)      */
    int n_bins;         /* W: bins per row (1 .. 2^20)                                  */
    int64_t k_lo;       /* global bin index of column 0                                 */
    double t_sft;       /* SFT duration T_SFT (s)                                       */
    double t0;          /* reference time at which f0 is defined (s)                    */
    int dtype;          /* storage type of the power on the device: FT_F32/F16/BF16     */
} ft_band_desc;

/* Copy one band of SFT power to the device, converting to desc->dtype (round to nearest
 * even) into a padded row-major layout.
 *   power            [N_SFT][row_stride] elements of power_dtype (FT_F32 or FT_F64), host
 *                    or device (power_on_device); only the first n_bins of each row are read.
 *   t_mid            host [N_SFT] SFT mid-times (s).
 *   v_over_c         host [N_SFT][3] detector velocity / c at t_mid (equatorial frame).
 *   w                host [N_SFT] per-SFT weights w_alpha >= 0, or NULL for w = 1
 *                    (Sec. II.B: weights are defined up to a constant).
 *   s_n              host [N_SFT] PSD levels (finite, > 0), or NULL (needed by injections,
 *                    the semi-analytic numbers and the all-sky weights).
 * Errors: FT_ERR_ARG on an inconsistent descriptor or non-finite power/metadata,
 * FT_ERR_RANGE beyond the size/velocity limits, FT_ERR_OOM.  Synchronises `stream`. */
FT_API int ft_load_sfts(ft_ctx *ctx, const ft_band_desc *desc, const void *power, int power_dtype,
                 int64_t row_stride, int power_on_device, const double *t_mid,
                 const double *v_over_c, const float *w, const double *s_n, void *stream,
                 ft_band **out);
FT_API void ft_band_destroy(ft_band *band);

/* Band facts: total SFT rows, bins, padded row stride (elements), storage dtype,
 * mu_G = 2 sum w and sigma_G = sqrt(4 sum w^2) (Sec. II.B.1).  Any pointer may be NULL. */
FT_API int ft_band_info(const ft_band *band, int64_t *n_sft_total, int *n_bins, int *row_stride,
                 int *dtype, double *mu_g, double *sigma_g);

/* All-sky weights (Sec. II.B): for a template at sky point n the weight of SFT alpha becomes
 *     w_alpha(n) = r_alpha(n) / sum_beta r_beta(n),   r_alpha(n) = (a_alpha(n)^2 + b_alpha(n)^2) / S_n,alpha
 * with a = D:e+, b = D:ex the antenna-pattern amplitudes of detector tensor D_alpha for
 * direction n (the frame of ft_run_injections), so that each sky point's weights sum to 1;
 * the statistic is then s = sum_alpha w_alpha(n) P_alpha(bin), and z uses that sky point's
 * mu_G = 2 and sigma_G = sqrt(4 sum_alpha w_alpha(n)^2).  Candidates
 * of a sub-band are still ranked by s (every sky point has the same noise mean).
 *   det_tensor  host [N_SFT][6] (Dxx, Dxy, Dxz, Dyy, Dyz, Dzz), or NULL to turn the weights
 *               off again (the per-SFT weights of ft_load_sfts apply once more).
 * The per-sky sums are computed by ft_make_bank: banks made before this call keep none and
 * are refused by the evaluation calls while the weights are on.  Binary banks made after this
 * call weight every (template, SFT) by its template's own sky direction (the sums per
 * template are formed in the evaluation kernel).  The injection and
 * semi-analytic calls keep the per-SFT weights.  Errors: FT_ERR_ARG (null band, band loaded
 * without S_n, non-finite tensor), FT_ERR_OOM.  Synchronises `stream`. */
FT_API int ft_band_set_sky_weights(ft_band *band, const double *det_tensor, void *stream);

/* Number count (Sec. II.B, Eq. (number_count)): a new band whose value in SFT alpha, bin k is
 * nc = 1 if P > threshold else 0 (the paper's threshold is 3.2), with the source band's
 * metadata, per-SFT weights, S_n and all-sky weights copied, so that ft_eval_statistic /
 * ft_topk_per_band on it (with its own bank, same bank description) give the weighted
 * number count sum_alpha w_alpha nc_alpha along each track.  The comparison takes the
 * stored value (after the source band's FP16/BF16 rounding) in FP64.  Its mu_G and sigma_G
 * (ft_band_info, and z) are the weighted count's Gaussian-noise mean and deviation:
 * p sum w and sqrt(p (1 - p) sum w^2), p = exp(-threshold / 2) (P is exponential with mean
 * 2); with all-sky weights p and sqrt(p (1 - p) sum w(n)^2) per sky point.  The source band
 * is not changed.  Errors: FT_ERR_ARG (null, foreign or number-count band, threshold
 * negative or not finite), FT_ERR_OOM.  Synchronises `stream`. */
FT_API int ft_number_count_band(ft_ctx *ctx, const ft_band *band, double threshold, void *stream,
                                ft_band **out);

/* ----------------------------------------------------------------------------- bank --
 * Regular bank: f0_j = (k0 + j)/T_SFT, j < n_f0 (delta f0 = 1/T_SFT, App. A); a list of
 * f1 values; a list of sky unit vectors n.  Template index
 *     t = (i_sky * n_f1 + i_f1) * n_f0 + j       (f0 fastest).
 * Candidate sub-band of a template: j / subband_bins (the 1-D ahead-of-time boxes).
 */
typedef struct {
    int64_t k0;          /* global bin of f0 index 0                                    */
    int n_f0;            /* 1 .. 2^24                                                   */
    int n_f1;            /* 1 .. 65535                                                  */
    const double *f1;    /* host [n_f1] spindown values (Hz/s)                          */
    int64_t n_sky;       /* >= 1                                                        */
    const double *sky;   /* host [n_sky][3] unit vectors (equatorial)                   */
    int subband_bins;    /* >= 1                                                        */
} ft_bank_desc;

/* Upload a bank for use with `band` (it precomputes per-(f1, SFT) integer track terms).
 * The bank stays valid while `band` lives.  It records whether every track provably stays
 * inside the band's window (then the fast unchecked kernel runs); otherwise reads outside
 * the window contribute 0 and are counted (see ft_eval_statistic).
 * Errors: FT_ERR_ARG (bad descriptor, non-unit sky vector), FT_ERR_RANGE, FT_ERR_OOM. */
FT_API int ft_make_bank(ft_ctx *ctx, const ft_band *band, const ft_bank_desc *desc, void *stream,
                 ft_bank **out);
FT_API void ft_bank_destroy(ft_bank *bank);

/* Bank facts: template count, sub-band count, and whether every track stays inside the
 * window (1) or the bounds-checked kernel is used (0).  Any pointer may be NULL. */
FT_API int ft_bank_info(const ft_bank *bank, int64_t *n_templates, int *n_subbands, int *window_safe);

/* Wings needed so that every track of the bank stays inside the window: the number of
 * bins required below bin k0 (lo) and above bin k0 + n_f0 - 1 (hi), from the conservative
 * bound |v.n| <= |v|.  desc->k_lo and desc->n_bins are ignored.  Host-only computation. */
FT_API int ft_required_wings(const ft_band_desc *desc, const double *t_mid, const double *v_over_c,
                      const ft_bank_desc *bank, int *lo, int *hi);

/* ----------------------------------------------------------------------------- statistic --
 * Evaluate s for every template of `bank` (Eq. (short_coh_general)) and optionally
 * z = (s - mu_G)/sigma_G (Eq. (critical_ratio)) and the per-template count of SFTs whose
 * track bin falls outside the window (those contribute 0).
 *   s_out     [n_templates] float, required
 *   z_out     [n_templates] float or NULL
 *   n_oob_out [n_templates] int32 or NULL
 * Accumulation: FP32 partial sums over stages of SFTs, combined with a compensated (2Sum)
 * FP32 pair; z is formed in FP64 from that pair. */
FT_API int ft_eval_statistic(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, float *s_out,
                      float *z_out, int32_t *n_oob_out, int out_on_device, void *stream);

/* One candidate: template index (-1 for an empty slot), its s and z. */
typedef struct {
    int64_t template_idx;
    float s;
    float z;
} ft_candidate;

/* Per sub-band b (templates with j / subband_bins == b), the k loudest templates ordered
 * by s descending, ties by smaller template index (Sec. IV.B: loudest per disjoint box).
 * out: [n_subbands][k] ft_candidate; slots beyond a sub-band's population have
 * template_idx = -1, s = -inf.  1 <= k <= 32.  The statistic is not written to memory: the
 * selection is fused into the evaluation kernel, followed by one merge kernel. */
FT_API int ft_topk_per_band(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k,
                     ft_candidate *out, int out_on_device, void *stream);

/* ft_topk_per_band restricted to templates whose gate[t] >= gate_min: the loudest s among
 * templates that also pass a second statistic (Sec. VI.B: the loudest normalised power
 * whose weighted number count is at least its Gaussian-noise mean + 3 sigma; there gate is
 * the s_out of ft_eval_statistic on the ft_number_count_band of the same data and bank
 * shape, and gate_min = mu + 3 sigma of that band's ft_band_info).  A sub-band with fewer
 * than k passing templates fills the rest with empty slots.
 *   gate  device [n_templates] float (template index order of `bank`)
 * Errors: FT_ERR_ARG (host or null gate, NaN gate_min), else as ft_topk_per_band. */
FT_API int ft_topk_per_band_gated(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k,
                                  const float *gate, float gate_min, ft_candidate *out,
                                  int out_on_device, void *stream);

/* Ahead-of-time boxes across the sky (Sec. IV.B) for the regular bank: box (x, b) holds the
 * templates of sub-band b whose sky point is among positions x sky_box .. (x + 1) sky_box - 1
 * of the bank's sky order (ft_bank_sky_order: a Hilbert curve over the equal-area map
 * ((z + 1)/2, (longitude + pi)/2pi) of the sphere, so a box is a compact patch of
 * neighbouring sky points), every f1 value.  out: [n_sky_boxes][n_subbands][k]
 * ft_candidate with n_sky_boxes = ceil(n_sky / sky_box), each list as in ft_topk_per_band.
 * The launch shape keeps every CTA's sky points inside one box.  Errors: FT_ERR_ARG
 * (sky_box < 1), FT_ERR_RANGE (more than 65535 sky boxes, k), else as ft_topk_per_band. */
FT_API int ft_topk_per_skybox(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box,
                              int k, ft_candidate *out, int out_on_device, void *stream);

/* Ahead-of-time boxes over all three dimensions of the regular bank (Sec. IV.B: disjoint
 * boxes of neighbouring templates, the loudest kept per box): box (x, y, b) holds the templates
 * of sub-band b whose sky point is at positions x sky_box .. (x + 1) sky_box - 1 of the bank's
 * sky order (as in ft_topk_per_skybox) and whose f1 index is in y f1_box .. (y + 1) f1_box - 1
 * of the bank's f1 list.  out: [n_sky_boxes][n_f1_boxes][n_subbands][k] ft_candidate with
 * n_sky_boxes = ceil(n_sky / sky_box), n_f1_boxes = ceil(n_f1 / f1_box), each list as in
 * ft_topk_per_band.  gate: NULL for the plain loudest, else as in ft_topk_per_band_gated (the
 * count-gated loudest per box of Sec. VI.B).  The launch shape keeps every CTA's sky points and
 * f1 values inside one box; small f1 boxes shrink the CTAs' f1 groups and cost speed.
 * sky_box >= n_sky (f1_box >= n_f1) makes one box over that dimension.
 * Errors: FT_ERR_ARG (sky_box or f1_box < 1; a gate as in ft_topk_per_band_gated),
 * FT_ERR_RANGE (more than 65535 boxes along either dimension, k), else as ft_topk_per_band. */
FT_API int ft_topk_per_box(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int sky_box,
                           int f1_box, int k, const float *gate, float gate_min,
                           ft_candidate *out, int out_on_device, void *stream);

/* The bank's sky order (the Hilbert-curve order described at ft_topk_per_skybox): order[i] =
 * index (in the bank's sky list) of the sky point at position i; host [n_sky] int32. */
FT_API int ft_bank_sky_order(const ft_bank *bank, int32_t *order);

/* Same search and same output as ft_topk_per_band, for callers that cannot let the library
 * allocate device memory during the call: processes whose device memory is owned by another
 * allocator (a framework's caching allocator or a budget fixed at start-up, where a new
 * cudaMalloc may fail or fragment the device) and latency-critical loops that cannot take
 * an allocation's implicit synchronisation.  There is no counterpart in the paper: this is
 * purely a memory-management variant.
 * - The candidate scratch lives in one file-scope device array of FT_NOALLOC_SCRATCH_BYTES
 *   (16 MiB) that every device loading the library holds until the process exits.  A bank
 *   needing more (n_sky x f1 groups x f0 tiles x sub-bands per tile x k x 16 bytes, plus the
 *   output when out is on the host) is rejected with FT_ERR_RANGE; the search-shaped band
 *   (1e4 sky x 20 f1 x 180 f0, k = 10) fits.
 * - The call makes no cudaMalloc / cudaFree and calls no allocating library routine.  The
 *   band, bank and context were allocated when they were created.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current; make that first call before any stream capture.
 * - Every call shares the one array and the array keeps the last call's contents; calls
 *   that overlap on the GPU (different streams, or different contexts on the same device)
 *   race on it and must be serialised by the caller.  Nothing needs clearing between calls:
 *   each call writes every slot it reads.
 * Arguments, output layout and errors are those of ft_topk_per_band. */
#define FT_NOALLOC_SCRATCH_BYTES (16u << 20)
FT_API int ft_topk_per_band_noalloc(ft_ctx *ctx, const ft_band *band, const ft_bank *bank, int k,
                                    ft_candidate *out, int out_on_device, void *stream);

/* ----------------------------------------------------------------------------- injections --
 * Injection-recovery runs: the Monte-Carlo estimate of the detection probability
 * (Sec. V, Eq. (sampling)).  Each run simulates one signal in Gaussian noise and returns
 * the loudest critical ratio z of a local bank around it; the caller applies the
 * detection rule z > tau (Sec. V.B) and fits p_det(h0).
 *   Signal (Sec. II.B.2): in SFT alpha the normalised power
 *     rho^2 = 4 |h~|^2 / (T_SFT S_n),  |h~| = 0.7737 (T_SFT/2) h0 |Q|,
 *     |Q|^2 = (F+ (1 + cos^2 iota)/2)^2 + (Fx cos iota)^2   (polarisations in quadrature),
 *     F+ = a cos 2psi + b sin 2psi, Fx = b cos 2psi - a sin 2psi, a = D : e+, b = D : ex,
 *     with D the detector tensor at the SFT and e+, ex built on X = z x n/|z x n|, Y = n x X;
 *   placed in the bin nearest (f0 T_SFT + f1 tau)(1 + v.n) (FP64, tau = (t_mid - t0) T_SFT).
 *   Data: per SFT the bins k_sig - H .. k_sig + H, generated on the device and never
 *   stored: complex unit Gaussian noise (scaled by noise_scale) plus sqrt(rho^2) in k_sig,
 *   i.e. P = -2 ln u1, or |r e^{i 2 pi u2} + sqrt(rho^2)|^2 with r^2 = -2 ln u1 in k_sig;
 *   u1, u2 = ((x >> 8) + 1) / 2^24 from Philox4x32-10 (Salmon et al., SC'11) with counter
 *   (absolute bin, SFT index, run id low, run id high) and key (seed low, seed high).
 *   Local bank: the k_sky bank sky points nearest to n, every bank f1, and the bank f0 bins
 *   within half_f0 of round(f0 T_SFT); each template's statistic is that of
 *   ft_eval_statistic (same track bins and weights), reads outside the generated window
 *   contribute 0 and are counted.
 * The band supplies times, velocities, weights and S_n (it must be loaded with s_n); its
 * stored power is not used.  det_tensor: host [N_SFT][6] (xx, xy, xz, yy, yz, zz).
 * inj/out: host arrays of n runs; run i uses run id desc->first_run_id + i.
 * Limits: k_sky <= 128, half_f0 <= 7, 1 <= half_window <= 1024, n_f1 <= 64 and at most 4096
 * local templates.  Allocates device memory for the call; synchronises `stream`. */
typedef struct {
    double h0;    /* amplitude, in the units of sqrt(S_n T_SFT) of the band's power       */
    double cosi;  /* cos(inclination)                                                        */
    double psi;   /* polarisation angle (rad)                                               */
    double f0;    /* frequency at t0 (Hz)                                                    */
    double f1;    /* spindown (Hz/s)                                                         */
    double n[3];  /* source direction, unit vector (equatorial)                              */
} ft_injection;

typedef struct {
    int k_sky;
    int half_f0;
    int half_window;
    double noise_scale; /* 1: Gaussian noise; 0: noise-free data (checking)                  */
    uint64_t seed;
    uint64_t first_run_id;
} ft_inj_desc;

typedef struct {
    double max_z;            /* loudest critical ratio over the local bank                   */
    int64_t template_idx;    /* the template attaining it (ties: smaller index)              */
    int64_t n_out_of_window; /* local-bank reads outside the generated window                */
} ft_inj_result;

FT_API int ft_run_injections(ft_ctx *ctx, const ft_band *band, const ft_bank *bank,
                             const double *det_tensor, const ft_inj_desc *desc, int64_t n,
                             const ft_injection *inj, ft_inj_result *out, void *stream);

/* Semi-analytic sensitivity inputs (Sec. V.A): the signal-dependent two of the four numbers
 * q = {mu_G, sigma_G, rho^2_1, rho^2_2} that fix the distribution of s for a population
 * draw.  For draw i of pop (direction n, cos iota, psi; h0 and f0, f1 ignored):
 *   rho1[i] = sum_alpha w_alpha rho^2_alpha(h0 = 1),  rho2[i] = sum_alpha w_alpha^2 rho^2_alpha(h0 = 1),
 * with rho^2_alpha the per-SFT normalised signal power of ft_run_injections (same antenna
 * patterns, polarisations in quadrature, the band's S_n and weights); for amplitude h0 both
 * scale by h0^2.  mu_G and sigma_G are the band's (ft_band_info).  det_tensor: host
 * [N_SFT][6]; pop, rho1, rho2: host arrays of n.  Sums in FP64 in a fixed order (one CTA
 * per draw).  Synchronises `stream`.  Errors: FT_ERR_ARG (null pointer, band without S_n,
 * bad draw), FT_ERR_OOM, FT_ERR_CUDA. */
FT_API int ft_pdet_q(ft_ctx *ctx, const ft_band *band, const double *det_tensor, int64_t n,
                     const ft_injection *pop, double *rho1, double *rho2, void *stream);

/* ----------------------------------------------------------------------------- binary --
 * Sources in circular binary orbits (Eq. (track) with the orbit term, no spindown):
 *     f(t) = f0 [1 + v(t).n - a_p Omega cos(Omega t - phi_b)],   t = t_mid - t0,
 * searched with a random template bank (Sec. IV.A): templates uniform in the coordinates
 * xi = {f0^6, alpha, sin(delta), a_p^3, Omega^4, phi_b} in which the template density of
 * App. A (rho ~ f0^5 a_p^2 Omega^3) is constant (Eq. (xi_of_lambda), Eq. (unif_transform);
 * constant factors dropped), cut ahead of time into regular hyperboxes of n_per_box templates
 * each (Sec. IV.B).  Templates are pure functions of (seed, index) and are never stored: the
 * kernels derive each one from a Philox4x32-10 counter.
 *
 * Templates (the same on every path, and in the oracle):
 *   - template i is in box i / n_per_box (box index row-major over BINARY dims, f0 slowest);
 *     u_0..u_5 are 53-bit uniforms ((a >> 5) 2^26 + (b >> 6)) / 2^53 from Philox4x32-10 at
 *     counter (i lo, i hi, c, 0x62696e61), key (seed lo, seed hi), c = 0, 1, 2 (words 0,1 and
 *     2,3 of each call); xi_d = xi_lo + (box_d + u_d) (xi_hi - xi_lo) / n_div_d; f0 =
 *     sqrt(cbrt(xi_0)), a_p = cbrt(xi_3) (24 Newton steps y -= (y^3 - x) / (3 y^2) from the
 *     range's top), Omega = sqrt(sqrt(xi_4)); alpha and phi_b stay below 1 turn.
 * Bins: the FP64 bin of Eq. (track), bin = floor(X + 1/2) with
 *     X = f0 (1 + v.n - a_p Omega cos(Omega t - 2 pi phi_b)) T_SFT - k_lo,
 *     n = (cos delta cos 2 pi alpha, cos delta sin 2 pi alpha, sin delta), t = t_mid - t0.
 *   The kernels evaluate X first in FP32 (64-bit integer orbit phase, the special-function
 *   unit's cosine of that phase, one FMA chain) with an error below a bound delta derived
 *   from the bank's largest f0 T_SFT |v|, f0 T_SFT a_p Omega and orbit frequency (about 3e-5
 *   bins for the paper's search ranges); where that value lies within delta of a rounding
 *   boundary they recompute X in FP64 from the template's FP64 terms and the SFT's FP64 v
 *   and t, and that decides.  So every bin is the FP64 bin, except where the FP64 value
 *   itself is within its own rounding (about 1e-10 bins) of the boundary.
 *   Bins outside the band contribute 0 and are counted, as for the isolated bank.
 */
typedef struct ft_binary_bank ft_binary_bank;

typedef struct {
    /* ranges per dimension, order: f0 (Hz), alpha (right ascension, turns in [0, 1]),
     * sin(delta) (in [-1, 1]), a_p (light-seconds), Omega (rad/s), phi_b (turns in [0, 1]).
     * For f0, a_p and Omega: 0 < lo <= hi <= 16 lo, or (a_p only) lo = hi = 0 for an
     * isolated source. */
    double lo[6], hi[6];
    int32_t n_div[6];    /* boxes per dimension (>= 1 each) */
    int64_t n_per_box;   /* templates per box (>= 1); n_templates = prod(n_div) n_per_box < 2^40 */
    uint64_t seed;
} ft_binary_bank_desc;

/* Set up a binary bank for `band` (uses its SFT times, velocities and weights: the per-SFT
 * weights, or, when ft_band_set_sky_weights was called before, the all-sky weights
 * (a^2 + b^2)/S_n of each template's own sky direction (to FP32 accuracy), normalised per
 * template; then s =
 * sum r P / sum r and z uses mu_G = m and sigma_G = d sqrt(sum r^2) / sum r, with one SFT's
 * noise mean m and deviation d: 2 and 2 for normalised power, p and sqrt(p (1 - p)) for a
 * number-count band).  Errors: FT_ERR_ARG (ranges, counts), FT_ERR_OOM. */
FT_API int ft_make_binary_bank(ft_ctx *ctx, const ft_band *band, const ft_binary_bank_desc *desc,
                               ft_binary_bank **out);
FT_API void ft_binary_bank_destroy(ft_binary_bank *bank);
FT_API int ft_binary_bank_info(const ft_binary_bank *bank, int64_t *n_templates, int64_t *n_boxes);

/* lambda of templates first .. first + n - 1: host [n][6] in the order of ft_binary_bank_desc
 * (alpha and phi_b in turns), as the kernels derive them. */
FT_API int ft_binary_templates(ft_ctx *ctx, const ft_binary_bank *bank, int64_t first, int64_t n,
                               double *lambda_out, void *stream);

/* Running count of the FP64 decisions the binary kernels took on this bank (evaluations
 * whose FP32 screen fell within delta of a rounding boundary) since the last call, and the
 * bank's delta in bins (either pointer nullable).  Resets the count; synchronises the
 * device.  Errors: FT_ERR_ARG (null bank), FT_ERR_CUDA. */
FT_API int ft_binary_decisions(ft_binary_bank *bank, uint64_t *n_fp64, double *delta);

/* The FP32 screen's cosine step (the orbit phase ph in 2^-32 turns as a signed FP32 angle,
 * then the special-function unit's cosine) against cos(2 pi ph / 2^32), over all 2^32 phases
 * on the context's device: the largest absolute error, and the bound the screen's delta
 * assumes for it (bound nullable).  This checks the one step of the screen whose error comes
 * from hardware rather than from FP32 rounding (Sec. II.A Eq. (track): its cosine term).
 * Synchronises the device; about a second.  Errors: FT_ERR_ARG (null ctx or max_abs_err),
 * FT_ERR_OOM, FT_ERR_CUDA. */
FT_API int ft_binary_cos_screen_check(ft_ctx *ctx, double *max_abs_err, double *bound);

/* Bins of templates[0..n) in every SFT (the kernels' rule above): bins [n][N_SFT] int32 columns of the band
 * (may lie outside [0, n_bins)).  templates / bins both host or both device (on_device). */
FT_API int ft_binary_track_bins(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank,
                                const int64_t *templates, int64_t n, int32_t *bins, int on_device,
                                void *stream);

/* s (Eq. (short_coh_general) along the binary track), z = (s - mu_G) / sigma_G and the
 * out-of-window count of templates first .. first + n - 1 into s_out[n] (required), z_out,
 * n_oob_out (nullable).  FP32 partial sums per stage of SFTs folded into a compensated FP32
 * pair.  Synchronises `stream` for host outputs. */
FT_API int ft_binary_eval(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank,
                          int64_t first, int64_t n, float *s_out, float *z_out,
                          int32_t *n_oob_out, int out_on_device, void *stream);

/* The k loudest templates of every hyperbox (Sec. IV.B: the loudest per box), ordered by s
 * descending, ties by smaller index: out [n_boxes][k] (empty slots: index -1, s = -inf).
 * 1 <= k <= 32.  The statistic is not written to memory. */
FT_API int ft_binary_topk_per_box(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank,
                                  int k, ft_candidate *out, int out_on_device, void *stream);

/* ft_binary_topk_per_box among templates with gate[t] >= gate_min only (Sec. VI.B: the
 * loudest normalised power whose weighted number count reaches its noise mean + 3 sigma;
 * gate = s_out of ft_binary_eval on the ft_number_count_band of the same data, with a bank
 * of the same description).  gate: device [n_templates] float.  Errors: FT_ERR_ARG (host or
 * null gate, NaN gate_min), else as ft_binary_topk_per_box. */
FT_API int ft_binary_topk_per_box_gated(ft_ctx *ctx, const ft_band *band, const ft_binary_bank *bank,
                                        int k, const float *gate, float gate_min, ft_candidate *out,
                                        int out_on_device, void *stream);

/* ----------------------------------------------------------------------------- surrogate --
 * A learned model of the detection probability p_det (Sec. V, Eqs. (pdet_abstract),
 * (simple_eq)) trained on injection-recovery outcomes: a 4-layer perceptron
 * d_in -> width -> width -> width -> 1 with ReLU and a sigmoid output, binary cross entropy
 * (mean over the batch) and Adam, all in this library's CUDA kernels.  FP32 training;
 * inference in FP32 or BF16 (weights and activations rounded to BF16, FP32 accumulation).
 * Parameter vector (FP32, this order): W1[width][d_in] b1 W2[width][width] b2 W3 b3
 * W4[1][width] b4[1].  Reductions run in a fixed order: training is bit-reproducible.
 * The model is bound to the context's device; host arrays unless stated. */
typedef struct ft_mlp ft_mlp;
/* He-uniform weights (bound sqrt(6/fan_in)) and zero biases from `seed`; 1 <= d_in, width <= 256. */
FT_API int ft_mlp_create(ft_ctx *ctx, int d_in, int width, uint64_t seed, ft_mlp **out);
FT_API void ft_mlp_destroy(ft_mlp *mlp);
FT_API int ft_mlp_n_params(const ft_mlp *mlp, int64_t *n);
FT_API int ft_mlp_get_params(ft_mlp *mlp, float *params);
/* Sets the parameters and resets the optimiser state. */
FT_API int ft_mlp_set_params(ft_mlp *mlp, const float *params);
/* The whole training state, for checkpoints: state [3][n_params] = parameters, Adam's first
 * and second moments; adam_t = the optimiser's step count (bias correction).  Setting it
 * restores training exactly where it was taken. */
FT_API int ft_mlp_get_state(ft_mlp *mlp, float *state, int64_t *adam_t);
FT_API int ft_mlp_set_state(ft_mlp *mlp, const float *state, int64_t adam_t);
/* Loss and gradient of one batch X [B][d_in], labels y [B] in {0, 1} (loss, grad nullable;
 * grad [n_params]).  The gradient stays on the device for ft_mlp_adam_step. */
FT_API int ft_mlp_loss_grad(ft_mlp *mlp, const float *X, const float *y, int B, float *loss,
                            float *grad);
/* One Adam update with the last gradient (bias-corrected moments). */
FT_API int ft_mlp_adam_step(ft_mlp *mlp, float lr, float beta1, float beta2, float eps);
/* Mini-batch training on n samples for `epochs` passes (shuffled by `seed`; Adam with
 * beta1 0.9, beta2 0.999, eps 1e-8); loss_history [epochs] (nullable) gets each pass's mean
 * batch loss. */
FT_API int ft_mlp_train(ft_mlp *mlp, const float *X, const float *y, int64_t n, int batch,
                        int epochs, float lr, uint64_t seed, float *loss_history);
/* p = sigmoid(network(X)) for n samples; X and p both host (on_device 0) or both device (1,
 * asynchronous on `stream`).  bf16: 0 = FP32 forward; 1 = BF16 inference (BF16 inputs,
 * weights and activations, FP32 sums) on the tensor cores -- each hidden layer one
 * tcgen05.mma product of 128 samples, FP32 accumulators in tensor memory -- when the width
 * is a multiple of 16 up to 128 and d_in is at most 64, else on the CUDA cores; 2 = the same
 * BF16 inference on the CUDA cores (one warp per sample).  Errors: FT_ERR_ARG, FT_ERR_OOM,
 * FT_ERR_CUDA. */
FT_API int ft_mlp_predict(ft_mlp *mlp, const float *X, int64_t n, float *p, int bf16,
                          int on_device, void *stream);

/* ----------------------------------------------------------------------------- tuning --
 * Launch shape of the evaluation kernels.  Zero fields keep the built-in choice.
 *   rows_per_stage  SFT rows per shared-memory stage (fast kernel: multiple of 4, <= 32)
 *   stages          pipeline stages in flight (fast kernel: 2 .. 4)
 *   tile_f0         f0 values per CTA tile (multiple of 32; 16-bit storage: of 64; <= 256)
 * A shape that does not fit the band (shared memory) makes the evaluation calls fail with
 * FT_ERR_RANGE; nothing else about the results depends on it. */
typedef struct {
    int rows_per_stage;
    int stages;
    int tile_f0;
} ft_tune;

/* Set (tune != NULL) or clear (NULL) the context-wide launch-shape override. */
FT_API int ft_set_tune(ft_ctx *ctx, const ft_tune *tune);

/* Measured ceiling of the gather-accumulate (a benchmark aid, not part of the search): the
 * evaluation kernel's inner loop alone, with rows resident in shared memory, four row
 * offsets per vector load and one conflict-free 32-bit load per lane per 32 (FP32, dtype
 * FT_F32) or 64 (16-bit pairs, FT_F16 / FT_BF16) f0 values, accumulated in FP32; 2 CTAs of
 * 640 threads per SM, about 1.5e11 evaluations.  Writes evaluations per second (CUDA events)
 * and per clock per SM (clock64 of the slowest CTA).  Synchronises the device.  Errors:
 * FT_ERR_ARG (null pointer, bad dtype), FT_ERR_OOM, FT_ERR_CUDA. */
FT_API int ft_gather_roof(ft_ctx *ctx, int dtype, double *evals_per_s, double *evals_per_clk_sm);

/* Failure-detection self-test: one CTA waits on an mbarrier that no thread ever arrives at,
 * with the same bounded wait (about 1 s of %globaltimer) as the search kernels, records
 * FT_STATUS_TIMEOUT in the context's status word and returns.  The call synchronises
 * `stream` and returns FT_ERR_TIMEOUT as a search that ran out would; the status word is
 * then clear and the context usable.  *waited_s (nullable) gets the device-measured wait. */
FT_API int ft_selftest_bounded_wait(ft_ctx *ctx, double *waited_s, void *stream);

/* ----------------------------------------------------------------------------- batches --
 * Many bands of uneven width and sky density searched by one persistent launch (the
 * batching pattern; each band's statistic and candidates are those of ft_topk_per_band).
 * The tiles of all bands form one band-major work list that resident CTAs consume through a
 * global ticket counter; each CTA merges its tiles' candidates into per-sub-band lists in
 * shared memory.  The launch sequence (clear, persistent kernel, merge) is captured once in
 * a CUDA graph at creation and replayed by ft_batch_run.
 *   bands/banks  n_bands pairs; all bands share the storage type and weighting and every
 *                bank's tracks must stay inside its band's window (FT_ERR_ARG otherwise)
 *   tune         tile_f0 and stages of the persistent kernel; NULL or zero fields run the
 *                autotuner, which times candidate shapes on a subset of every band's tiles
 *                (cached per storage type, weighting, k, rows, f1 count and window widths)
 *   out          [sum over bands of n_subbands][k] candidates, band after band
 * Creation allocates device memory and synchronises `stream`; runs do not allocate. */
typedef struct ft_batch ft_batch;
FT_API int ft_batch_create(ft_ctx *ctx, int n_bands, const ft_band *const *bands,
                           const ft_bank *const *banks, int k, const ft_tune *tune, void *stream,
                           ft_batch **out);
FT_API int ft_batch_run(ft_batch *batch, ft_candidate *out, int out_on_device, void *stream);
/* Total candidate slots, evaluations per run, the launch shape in use, resident CTAs. */
FT_API int ft_batch_info(const ft_batch *batch, int64_t *n_candidates, int64_t *evals,
                         ft_tune *chosen, int *n_ctas);
FT_API void ft_batch_destroy(ft_batch *batch);
/* One-shot create + run + destroy; synchronises `stream` before returning. */
FT_API int ft_eval_batched(ft_ctx *ctx, int n_bands, const ft_band *const *bands,
                           const ft_bank *const *banks, int k, ft_candidate *out, int out_on_device,
                           const ft_tune *tune, void *stream);

/* Track bins used by the evaluation kernels, for a list of templates (a checking aid):
 * bins[i][alpha] = k_{alpha}(templates[i]) relative to column 0 (may lie outside
 * [0, n_bins)).  The rule (Eq. (track), a_p = 0, exact integer form):
 *   eps = fma(vz, nz, fma(vy, ny, vx*nx)); E = rint(eps 2^32); C = rint(fma(k0, eps, k0-k_lo) 2^32)
 *   G = rint((f1 tau) 2^32), tau = (t_mid - t0) T_SFT; X0 = C + G + floor(G E / 2^32)
 *   k_j = j + floor((X0 + j E + 2^31) / 2^32)
 * templates and bins are both host or both device pointers (on_device). */
FT_API int ft_track_bins(ft_ctx *ctx, const ft_band *band, const ft_bank *bank,
                  const int64_t *templates, int64_t n, int32_t *bins, int on_device,
                  void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTTRACKS_H */
