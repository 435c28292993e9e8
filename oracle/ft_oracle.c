/*
 * ft_oracle.c -- plain CPU FP64 oracle for the short-coherence statistic.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path in paper_2411_18370_b300/csrc/.
 *
 * What it computes (arXiv 2411.18370):
 *   s(lambda) = sum_{X,alpha} w_{X alpha} * P[t_{X alpha}; f(t_{X alpha}; lambda)]
 *       -- Sec. II.B, Eq. (short_coh_general), with P the normalised power of Eq. (s_tf).
 *   f(t; lambda) = (f0 + f1 (t - t0)) * (1 + v(t).n / c)
 *       -- Sec. II.A, Eq. (track) with a_p = 0 (isolated source); the f1 spindown term is
 *          the reading used for this workload (the paper neglects spindown).
 *   Bin of a frequency f in SFT alpha: round-half-up of f * T_SFT (the frequency grid of
 *   an SFT has spacing 1/T_SFT, App. A "delta f0 = 1/T_SFT"), taken relative to the
 *   window's first column k_lo.
 *
 * Two bin routines are provided:
 *   or_bin_fp64   the direct FP64 evaluation floor((K0 + j + f1 tau)(1 + eps) - k_lo + 1/2)
 *                 with tau = (t - t0) T_SFT;
 *   or_bin_q32    the canonical exact-integer evaluation (Q32 fixed point, below), which
 *                 the statistic uses.  The two agree except where the real-valued track
 *                 lies within ~1e-7 bin of a half-integer; tests pin that.
 *
 * Canonical Q32 bin (the reading the whole project uses; every quantity below is a
 * correctly-rounded IEEE double operation in the order written, then an exact integer):
 *   eps = fma(vz, nz, fma(vy, ny, vx * nx))                 (v already divided by c)
 *   E   = llrint(eps * 2^32)
 *   C   = llrint(fma(K0, eps, K0 - k_lo) * 2^32)
 *   G   = llrint((f1 * tau) * 2^32)
 *   X0  = C + G + floor(G * E / 2^32)                       (128-bit product)
 *   k_j = j + floor((X0 + j * E + 2^31) / 2^32)
 * i.e. x(j) = (K0 - k_lo) + K0 eps + f1 tau + f1 tau eps + j + j eps in 32.32 fixed point,
 * rounded half-up.
 *
 * Out-of-window tracks (k < 0 or k >= W) contribute 0 and are counted per template.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define TWO32 4294967296.0

static double or_eps(const double *v, const double *n)
{
    return fma(v[2], n[2], fma(v[1], n[1], v[0] * n[0]));
}

static int64_t floor_div_2_32(__int128 x)
{
    /* floor(x / 2^32): gcc's signed right shift is arithmetic (sign-extending). */
    return (int64_t)(x >> 32);
}

/* Canonical Q32 track bin of template (K0 + j, f1, n) in an SFT with mid-time offset
 * tau = (t_alpha - t0) * T_SFT and velocity v (units of c).  Eq. (track), a_p = 0. */
int64_t or_bin_q32(int64_t K0, int64_t k_lo, int64_t j, double f1, double tau,
                   const double *v, const double *n)
{
    double eps = or_eps(v, n);
    int64_t E = llrint(eps * TWO32);
    int64_t C = llrint(fma((double)K0, eps, (double)(K0 - k_lo)) * TWO32);
    int64_t G = llrint((f1 * tau) * TWO32);
    int64_t X0 = C + G + floor_div_2_32((__int128)G * (__int128)E);
    __int128 acc = (__int128)X0 + (__int128)j * (__int128)E + ((__int128)1 << 31);
    return j + floor_div_2_32(acc);
}

/* Direct FP64 track bin, Eq. (track): floor(f(t) T_SFT - k_lo + 1/2).  Also returns the
 * signed distance of the real-valued position from the nearest rounding boundary. */
int64_t or_bin_fp64(int64_t K0, int64_t k_lo, int64_t j, double f1, double tau,
                    const double *v, const double *n, double *dist_to_tie)
{
    double eps = or_eps(v, n);
    double x = ((double)(K0 + j) + f1 * tau) * (1.0 + eps) - (double)k_lo;
    double k = floor(x + 0.5);
    if (dist_to_tie) {
        double frac = x + 0.5 - k; /* in [0, 1) */
        *dist_to_tie = frac < 0.5 ? frac : frac - 1.0;
    }
    return (int64_t)k;
}

typedef struct {
    const double *power; /* [n_sft][W] normalised power */
    int64_t n_sft;
    int64_t W;
    int64_t k_lo;
    const double *t_mid; /* [n_sft] */
    const double *v;     /* [n_sft][3] v/c */
    const double *w;     /* [n_sft] or NULL (=> 1) */
    double t0;
    double t_sft;
    int64_t K0;
    int64_t n_f0;
    int64_t n_f1;
    const double *f1;  /* [n_f1] */
    int64_t n_sky;
    const double *sky; /* [n_sky][3] */
    const double *wsky; /* [n_sky][n_sft] sky-dependent weights, or NULL (then w) */
} or_problem;

/* Offset of SFT alpha's mid-time from the reference time, times T_SFT: tau = (t - t0) T. */
static double or_tau(const or_problem *p, int64_t a)
{
    return (p->t_mid[a] - p->t0) * p->t_sft;
}

static void split_template(const or_problem *p, int64_t t, int64_t *isky, int64_t *if1,
                           int64_t *j)
{
    *j = t % p->n_f0;
    int64_t r = t / p->n_f0;
    *if1 = r % p->n_f1;
    *isky = r / p->n_f1;
}

/* s(lambda) for a list of templates (template index t = (i_sky n_f1 + i_f1) n_f0 + j),
 * Eq. (short_coh_general): FP64 sum over SFTs in row order.  templates == NULL means all
 * templates 0..n_out-1.  n_oob (nullable) receives the count of out-of-window reads. */
void or_statistic(const or_problem *p, const int64_t *templates, int64_t n_out,
                  double *s_out, int32_t *n_oob)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_out; i++) {
        int64_t t = templates ? templates[i] : i;
        int64_t isky, if1, j;
        split_template(p, t, &isky, &if1, &j);
        const double *n = p->sky + 3 * isky;
        double f1 = p->f1[if1];
        double s = 0.0;
        int32_t oob = 0;
        for (int64_t a = 0; a < p->n_sft; a++) {
            int64_t k = or_bin_q32(p->K0, p->k_lo, j, f1, or_tau(p, a), p->v + 3 * a, n);
            if (k < 0 || k >= p->W) {
                oob++;
                continue;
            }
            double w = p->wsky ? p->wsky[isky * p->n_sft + a] : (p->w ? p->w[a] : 1.0);
            s += w * p->power[a * p->W + k];
        }
        s_out[i] = s;
        if (n_oob)
            n_oob[i] = oob;
    }
}

/* Track bins of a list of templates: bins[i][alpha] (canonical Q32), and optionally the
 * direct FP64 bins and their distance to the rounding boundary. */
void or_bins(const or_problem *p, const int64_t *templates, int64_t n_out, int64_t *bins,
             int64_t *bins_fp64, double *dist)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_out; i++) {
        int64_t isky, if1, j;
        split_template(p, templates[i], &isky, &if1, &j);
        const double *n = p->sky + 3 * isky;
        double f1 = p->f1[if1];
        for (int64_t a = 0; a < p->n_sft; a++) {
            double tau = or_tau(p, a);
            bins[i * p->n_sft + a] = or_bin_q32(p->K0, p->k_lo, j, f1, tau, p->v + 3 * a, n);
            if (bins_fp64)
                bins_fp64[i * p->n_sft + a] = or_bin_fp64(
                    p->K0, p->k_lo, j, f1, tau, p->v + 3 * a, n, dist ? dist + i * p->n_sft + a : NULL);
        }
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
