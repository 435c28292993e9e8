/* CPU oracle for the binary-orbit track and the random template bank (arXiv 2411.18370).
 *
 * TEST INFRASTRUCTURE ONLY: called by tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline; shares no code with the CUDA library.
 *
 * What it follows:
 *   Eq. (track)            f(t) = f0 [1 + v(t).n - a_p Omega cos(Omega t - phi_b)] (no spindown)
 *   Eq. (xi_of_lambda) and App. A, Eq. (unif_transform): the uniform-density coordinates
 *                          xi = {f0^6, alpha, sin(delta), a_p^3, Omega^4, phi_b}; overall
 *                          constants are dropped (they only rescale xi).
 *   Sec. IV.A              a random bank is uniform in xi, mapped back to lambda.
 *   Sec. IV.B              the xi hyperbox is cut into regular boxes of n_per_box templates.
 *   Eq. (short_coh_general) the weighted sum of normalised power along the track.
 *
 * The track is the plain definition, in FP64 with libm's trigonometric functions:
 *   n  = (cos(delta) cos(2 pi alpha), cos(delta) sin(2 pi alpha), sin(delta)), alpha in turns;
 *   t  = t_mid - t0 (the SFT's mid-time from the start of the observation, where f0 is
 *        defined);
 *   X  = f0 (1 + v.n - a_p Omega cos(Omega t - 2 pi phi_b)) T_SFT - k_lo, phi_b in turns;
 *   bin = floor(X + 1/2)  (round half up to a column of the band).
 * Random numbers are inputs of the method, drawn the same way on both sides:
 *   Philox4x32-10 (or_philox4x32_10) at counter (i lo, i hi, c, 0x62696e61) with key
 *   (seed lo, seed hi), c = 0, 1, 2, two 53-bit uniforms per call; template i lies in box
 *   i / n_per_box (f0 slowest, phi_b fastest) and its xi is uniform in the box; the roots use
 *   sqrt (correctly rounded) and a fixed 24-step Newton cube root, so lambda is a pure
 *   function of (seed, i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

typedef struct {
    double lo[6], hi[6]; /* f0 (Hz), alpha (turns), sin(delta), a_p (light-s), Omega (rad/s), phi_b (turns) */
    int32_t n_div[6];    /* boxes per dimension */
    int64_t n_per_box;
    uint64_t seed;
} or_bdesc;

static const double TWO_PI = 6.283185307179586476925286766559;

static double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) / 9007199254740992.0;
}

/* cube root by Newton's method from y0 >= the root: 24 steps, operations as written */
static double cbrt_newton(double x, double y0)
{
    if (!(x > 0.0))
        return 0.0;
    double y = y0;
    for (int it = 0; it < 24; it++) {
        double y2 = y * y;
        double y3 = y2 * y;
        double num = y3 - x;
        double den = 3.0 * y2;
        y = y - num / den;
    }
    return y;
}

static double xi_of(int d, double lam)
{
    switch (d) {
    case 0: {
        double x2 = lam * lam;
        double x3 = x2 * lam;
        return x3 * x3;
    }
    case 3: {
        double x2 = lam * lam;
        return x2 * lam;
    }
    case 4: {
        double x2 = lam * lam;
        return x2 * x2;
    }
    default: return lam;
    }
}

static double lam_of(int d, double xi, const or_bdesc *b)
{
    switch (d) {
    case 0: return sqrt(cbrt_newton(xi, b->hi[0] * b->hi[0]));
    case 3: return cbrt_newton(xi, b->hi[3]);
    case 4: return sqrt(sqrt(xi));
    default: return xi;
    }
}

/* lam[6] of template i */
void or_bt_lambda(const or_bdesc *b, int64_t i, double lam[6])
{
    uint32_t key[2] = {(uint32_t)b->seed, (uint32_t)(b->seed >> 32)};
    double u[6];
    for (uint32_t c = 0; c < 3; c++) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), c, 0x62696e61u};
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        u[2 * c] = u53(w[0], w[1]);
        u[2 * c + 1] = u53(w[2], w[3]);
    }
    int64_t box = i / b->n_per_box;
    int64_t bk[6];
    for (int d = 5; d >= 0; d--) {
        bk[d] = box % b->n_div[d];
        box /= b->n_div[d];
    }
    for (int d = 0; d < 6; d++) {
        double xlo = xi_of(d, b->lo[d]), xhi = xi_of(d, b->hi[d]);
        double step = (xhi - xlo) / (double)b->n_div[d];
        double t = (double)bk[d] + u[d];
        double xi = xlo + t * step;
        lam[d] = lam_of(d, xi, b);
    }
    const double below1 = 0x1.fffffffffffffp-1;
    if (lam[1] >= 1.0)
        lam[1] = below1;
    if (lam[5] >= 1.0)
        lam[5] = below1;
    if (lam[2] > 1.0)
        lam[2] = 1.0;
    if (lam[2] < -1.0)
        lam[2] = -1.0;
}

/* the unit sky vector of (alpha in turns, sin(delta)) */
void or_bt_sky(const double lam[6], double n[3])
{
    double cd = sqrt(fmax(0.0, 1.0 - lam[2] * lam[2]));
    n[0] = cd * cos(TWO_PI * lam[1]);
    n[1] = cd * sin(TWO_PI * lam[1]);
    n[2] = lam[2];
}

/* Eq. (track) times T_SFT, as a column of the band: X = f(t) T_SFT - k_lo */
double or_bt_position(const double lam[6], const double n[3], const double v[3], double t,
                      double t_sft, int64_t k_lo)
{
    double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    double orbit = lam[3] * lam[4] * cos(lam[4] * t - TWO_PI * lam[5]);
    double f = lam[0] * (1.0 + vn - orbit);
    return f * t_sft - (double)k_lo;
}

/* t of SFT a: its mid-time from the start of the observation */
static double sft_t(const double *t_mid, int64_t a, double t0)
{
    return t_mid[a] - t0;
}

/* round half up, and |X - the nearest rounding boundary (a half-integer)| */
static int64_t bin_of(double X, double *dist)
{
    double k = floor(X + 0.5);
    if (dist) {
        double lo = X - (k - 0.5), hi = (k + 0.5) - X;
        *dist = lo < hi ? lo : hi;
    }
    return (int64_t)k;
}

/* bins[n][N] (columns of the band) of templates tmpl[0..n) over SFTs 0..N-1, and optionally
 * the distance of each real-valued position from its rounding boundary */
void or_bt_bins(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, const double *t_mid,
                const double *v, double t0, double t_sft, int64_t k_lo, int64_t *bins, double *dist)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6], nn[3];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl[i], lam);
        or_bt_sky(lam, nn);
        for (int64_t a = 0; a < N; a++) {
            double X = or_bt_position(lam, nn, v + 3 * a, sft_t(t_mid, a, t0), t_sft, k_lo);
            bins[i * N + a] = bin_of(X, dist ? dist + i * N + a : NULL);
        }
    }
}

/* s = sum_alpha w_alpha P[alpha][bin] (FP64, alpha order); bins outside [0, W) add 0 and
 * are counted. */
void or_bt_statistic(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, int64_t W,
                     const double *power, const double *w, const double *t_mid, const double *v,
                     double t0, double t_sft, int64_t k_lo, double *s, int32_t *oob)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6], nn[3];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl ? tmpl[i] : i, lam);
        or_bt_sky(lam, nn);
        double acc = 0.0;
        int32_t out = 0;
        for (int64_t a = 0; a < N; a++) {
            int64_t k = bin_of(or_bt_position(lam, nn, v + 3 * a, sft_t(t_mid, a, t0), t_sft, k_lo), NULL);
            if (k < 0 || k >= W) {
                out++;
                continue;
            }
            acc += (w ? w[a] : 1.0) * power[a * W + k];
        }
        s[i] = acc;
        oob[i] = out;
    }
}

/* lambda [n][6] of templates tmpl[0..n) */
void or_bt_templates(const or_bdesc *b, const int64_t *tmpl, int64_t n, double *lam)
{
    for (int64_t i = 0; i < n; i++)
        or_bt_lambda(b, tmpl[i], lam + 6 * i);
}

void or_antenna_ab(const double *D, const double *n, double *a, double *b);

/* The statistic under the all-sky weights of Sec. II.B for the binary bank: per template the
 * weights are w_alpha = r_alpha / sum r, r_alpha = (a^2 + b^2)(D_alpha, n) / S_n,alpha, with
 * n the template's unit sky vector; s = sum w P along the track's bins, and
 * sigma_G = 2 sqrt(sum w^2) (mu_G = 2). */
void or_bt_statistic_sky(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, int64_t W,
                         const double *power, const double *D, const double *s_n, const double *t_mid,
                         const double *v, double t0, double t_sft, int64_t k_lo, double *s,
                         double *sigma, int32_t *oob)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6], nn[3];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl ? tmpl[i] : i, lam);
        or_bt_sky(lam, nn);
        double acc = 0.0, sr = 0.0, sr2 = 0.0;
        int32_t out = 0;
        for (int64_t a = 0; a < N; a++) {
            double aa, bb;
            or_antenna_ab(D + 6 * a, nn, &aa, &bb);
            double r = (aa * aa + bb * bb) / s_n[a];
            sr += r;
            sr2 += r * r;
            int64_t k = bin_of(or_bt_position(lam, nn, v + 3 * a, sft_t(t_mid, a, t0), t_sft, k_lo), NULL);
            if (k < 0 || k >= W) {
                out++;
                continue;
            }
            acc += r * power[a * W + k];
        }
        s[i] = acc / sr;
        sigma[i] = 2.0 * sqrt(sr2) / sr;
        oob[i] = out;
    }
}
