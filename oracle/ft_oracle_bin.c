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
 * Canonical evaluation (the kernels evaluate the same rule in the same precision):
 *   - random numbers: Philox4x32-10 (or_philox4x32_10) at counter (i lo, i hi, c, 0x62696e61)
 *     with key (seed lo, seed hi), c = 0, 1, 2, two 53-bit uniforms per call;
 *   - template i lies in box i / n_per_box (f0 slowest, phi_b fastest); its xi is uniform in
 *     the box; the roots use sqrt (correctly rounded) and a fixed 24-step Newton cube root;
 *   - per template: F = f0 T_SFT split into K = floor(F) - k_lo and the FP32 fraction phi;
 *     the sky vector and the orbit amplitude D = F a_p Omega in FP32; the orbit frequency and
 *     phase as 64-bit fixed point (turns);
 *   - per SFT: the orbit phase of (t_mid - t0) in exact 64-bit integer arithmetic, its cosine
 *     by linear interpolation in a full-turn table of 1024 intervals (entries: libm's
 *     cos rounded to FP32, differences in FP32), and
 *         X = (phi + F v.n) - D cos,  bin = K + floor(X + 1/2)   (FP32, operations as written).
 *   or_bt_bins also returns the FP64 bin of Eq. (track) with libm's cos and its distance from
 *   the rounding boundary, which pins the canonical rule to the plain definition.
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

typedef struct {
    int64_t K;     /* floor(f0 T_SFT) - k_lo */
    float phi;     /* f0 T_SFT - floor(f0 T_SFT) */
    float F;       /* f0 T_SFT */
    float nx, ny, nz;
    float D;       /* f0 T_SFT a_p Omega */
    uint64_t nu_q; /* Omega / 2 pi in turns per second, units of 2^-54 */
    uint64_t psi_q; /* phi_b in turns, units of 2^-64 */
} or_bder;

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

/* full-turn table: C[i] = cos(i 2 pi / 1024) (libm, FP64, rounded to FP32), D[i] =
 * C[i+1] - C[i] in FP32, D[1024] = 0 */
static float tab_c[1025], tab_d[1025];
static int tab_ready;

void or_bt_init(void)
{
    if (tab_ready)
        return;
    for (int i = 0; i <= 1024; i++)
        tab_c[i] = (float)cos((double)i * 6.135923151542565e-03);
    for (int i = 0; i < 1024; i++)
        tab_d[i] = tab_c[i + 1] - tab_c[i];
    tab_d[1024] = 0.0f;
    tab_ready = 1;
}

/* cos(2 pi theta / 2^32): the turn theta / 2^32 falls in table interval theta >> 22 at
 * fraction (theta mod 2^22) / 2^22; linear interpolation between that entry and the next */
float or_cos_q32(uint32_t theta)
{
    or_bt_init();
    uint32_t i = theta >> 22;
    float f = (float)(theta & 0x3FFFFFu) * 0x1p-22f;
    return fmaf(f, tab_d[i], tab_c[i]);
}

void or_bt_derived(const double lam[6], double t_sft, int64_t k_lo, or_bder *o)
{
    double F = lam[0] * t_sft;
    double Fl = floor(F);
    o->K = (int64_t)Fl - k_lo;
    o->phi = (float)(F - Fl);
    o->F = (float)F;
    double s = lam[2];
    double c2 = 1.0 - s * s;
    float cd = (float)sqrt(c2 > 0.0 ? c2 : 0.0);
    uint32_t ta = (uint32_t)(lam[1] * 4294967296.0);
    float ca = or_cos_q32(ta), sa = or_cos_q32(ta - 0x40000000u);
    o->nx = cd * ca;
    o->ny = cd * sa;
    o->nz = (float)s;
    o->D = (float)((F * lam[3]) * lam[4]);
    double nu = lam[4] / 6.283185307179586;
    o->nu_q = (uint64_t)floor(nu * 18014398509481984.0 + 0.5);
    o->psi_q = (uint64_t)(lam[5] * 18446744073709551616.0);
}

int64_t or_bt_tq(double t_mid, double t0)
{
    return (int64_t)floor((t_mid - t0) * 1024.0 + 0.5);
}

static int64_t canonical_bin(const or_bder *d, int64_t tq, const float v[3])
{
    uint64_t ph = d->nu_q * (uint64_t)tq - d->psi_q;
    float c = or_cos_q32((uint32_t)(ph >> 32));
    float a = v[2] * d->nz;
    float b = fmaf(v[1], d->ny, a);
    float vn = fmaf(v[0], d->nx, b);
    float dop = d->F * vn;
    float m = d->D * c;
    float X = (d->phi + dop) - m;
    return d->K + (int64_t)floorf(X + 0.5f);
}

/* bins[n][N] (columns of the band); optionally the FP64 bins of Eq. (track) with libm cos
 * for the same lambda and sky vector, and the distance of that real-valued track from the
 * rounding boundary. */
void or_bt_bins(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, const double *t_mid,
                 const double *v, double t0, double t_sft, int64_t k_lo, int64_t *bins,
                 int64_t *bins64, double *dist)
{
    or_bt_init();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl[i], lam);
        or_bder d;
        or_bt_derived(lam, t_sft, k_lo, &d);
        for (int64_t a = 0; a < N; a++) {
            float v32[3] = {(float)v[3 * a], (float)v[3 * a + 1], (float)v[3 * a + 2]};
            bins[i * N + a] = canonical_bin(&d, or_bt_tq(t_mid[a], t0), v32);
            if (bins64) {
                double vn = v[3 * a] * (double)d.nx + v[3 * a + 1] * (double)d.ny + v[3 * a + 2] * (double)d.nz;
                double t = t_mid[a] - t0;
                double f = lam[0] * (1.0 + vn - lam[3] * lam[4] * cos(lam[4] * t - 6.283185307179586 * lam[5]));
                double X = f * t_sft - (double)k_lo;
                double k = floor(X + 0.5);
                bins64[i * N + a] = (int64_t)k;
                dist[i * N + a] = fabs(X - k - 0.5) < fabs(X - k + 0.5) ? fabs(X - k - 0.5) : fabs(X - k + 0.5);
            }
        }
    }
}

/* s = sum_alpha w_alpha P[alpha][bin] (FP64, alpha order); bins outside [0, W) add 0 and
 * are counted. */
void or_bt_statistic(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, int64_t W,
                      const double *power, const double *w, const double *t_mid, const double *v,
                      double t0, double t_sft, int64_t k_lo, double *s, int32_t *oob)
{
    or_bt_init();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl ? tmpl[i] : i, lam);
        or_bder d;
        or_bt_derived(lam, t_sft, k_lo, &d);
        double acc = 0.0;
        int32_t out = 0;
        for (int64_t a = 0; a < N; a++) {
            float v32[3] = {(float)v[3 * a], (float)v[3 * a + 1], (float)v[3 * a + 2]};
            int64_t k = canonical_bin(&d, or_bt_tq(t_mid[a], t0), v32);
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

/* lambda [n][6] and the derived per-template quantities of templates tmpl[0..n) */
void or_bt_templates(const or_bdesc *b, const int64_t *tmpl, int64_t n, double t_sft, int64_t k_lo,
                      double *lam, or_bder *der)
{
    for (int64_t i = 0; i < n; i++) {
        or_bt_lambda(b, tmpl[i], lam + 6 * i);
        if (der)
            or_bt_derived(lam + 6 * i, t_sft, k_lo, der + i);
    }
}

void or_antenna_ab(const double *D, const double *n, double *a, double *b);

/* The statistic under the all-sky weights of Sec. II.B for the binary bank: per template the
 * weights are w_alpha = r_alpha / sum r, r_alpha = (a^2 + b^2)(D_alpha, n) / S_n,alpha, with
 * n the template's unit sky vector (FP64, libm cos / sin of alpha); s = sum w P along the
 * canonical bins, and sigma_G = 2 sqrt(sum w^2) (mu_G = 2). */
void or_bt_statistic_sky(const or_bdesc *b, const int64_t *tmpl, int64_t n, int64_t N, int64_t W,
                         const double *power, const double *D, const double *s_n, const double *t_mid,
                         const double *v, double t0, double t_sft, int64_t k_lo, double *s,
                         double *sigma, int32_t *oob)
{
    or_bt_init();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double lam[6];
        or_bdesc bd = *b;
        or_bt_lambda(&bd, tmpl ? tmpl[i] : i, lam);
        or_bder d;
        or_bt_derived(lam, t_sft, k_lo, &d);
        double cdl = sqrt(fmax(0.0, 1.0 - lam[2] * lam[2]));
        double nn[3] = {cdl * cos(6.283185307179586 * lam[1]), cdl * sin(6.283185307179586 * lam[1]), lam[2]};
        double acc = 0.0, sr = 0.0, sr2 = 0.0;
        int32_t out = 0;
        for (int64_t a = 0; a < N; a++) {
            double aa, bb;
            or_antenna_ab(D + 6 * a, nn, &aa, &bb);
            double r = (aa * aa + bb * bb) / s_n[a];
            sr += r;
            sr2 += r * r;
            float v32[3] = {(float)v[3 * a], (float)v[3 * a + 1], (float)v[3 * a + 2]};
            int64_t k = canonical_bin(&d, or_bt_tq(t_mid[a], t0), v32);
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
