/*
 * ft_oracle_inj.c -- plain CPU FP64 oracle of one injection-recovery run.
 *
 * TEST INFRASTRUCTURE ONLY (see ft_oracle.c).  Shares no code with the CUDA path.
 *
 * One run (arXiv 2411.18370, Sec. V, Eq. (sampling): one sample z^(i) of the detection
 * statistic for a software-simulated signal, scored by the rule R(z; tau) of Sec. V.B):
 *  1. Signal model (Sec. II.B.2, "Distribution under the signal hypothesis"): in SFT alpha
 *     the signal sits in the bin nearest f(t_alpha) T_SFT with normalised power
 *         rho^2 = 4 |h~|^2 / (T_SFT S_n),  |h~| = 0.7737 (T_SFT / 2) h0 |Q|,
 *         |Q|^2 = (F+ (1 + cos^2 iota)/2)^2 + (Fx cos iota)^2
 *     (reading: the two polarisations are in quadrature, so their amplitudes add in
 *     squares), F+ = a cos 2psi + b sin 2psi, Fx = b cos 2psi - a sin 2psi, with
 *     a = D : e+, b = D : ex for the detector tensor D and the wave-frame tensors of the
 *     source direction n (X = z x n / |z x n|, Y = n x X, e+ = XX - YY, ex = XY + YX).
 *  2. Data: in every SFT, the bins k_sig - H .. k_sig + H around the signal bin.  The
 *     complex bin is noise g (Re, Im ~ N(0, 1), Sec. II.B.1) plus, in the signal bin, an
 *     amplitude a = sqrt(rho^2), so P = |g + a|^2 = r^2 + a^2 + 2 a r cos(theta) with
 *     r^2 = -2 ln u1, theta = 2 pi u2 (Box-Muller), and P = -2 ln u1 elsewhere.  u1, u2 are
 *     24-bit uniforms in (0, 1] from Philox4x32-10 (Salmon et al., SC'11) at counter
 *     (absolute bin, alpha, run id lo, run id hi) and key (seed lo, seed hi).
 *  3. Local bank: f0 bins j_c - half_f0 .. j_c + half_f0 (j_c = nearest grid bin to f0),
 *     every f1 of the bank, and the K sky points of the bank nearest to n (largest n.n_i,
 *     ties by index).  The statistic of every local template is Eq. (short_coh_general)
 *     with the canonical track bins of ft_oracle.c; reads outside the generated window
 *     are counted and contribute 0.
 *  4. Output: the largest critical ratio z (Eq. (critical_ratio)) over the local bank and
 *     the template that attains it (ties by the smaller template index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TWO32 4294967296.0

/* ---------------------------------------------------------------- Philox4x32-10 */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: round multipliers 0xD2511F53 and 0xCD9E8D57, key schedule
 * Weyl increments 0x9E3779B9 and 0xBB67AE85 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, x0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* 24-bit uniform in (0, 1]: ((x >> 8) + 1) / 2^24 (exact in single and double precision). */
double or_uniform24(uint32_t x)
{
    return ((double)(x >> 8) + 1.0) / 16777216.0;
}

/* ---------------------------------------------------------------- antenna patterns */

/* a = D : e+, b = D : ex for source direction n; D given as (xx, xy, xz, yy, yz, zz). */
void or_antenna_ab(const double *D, const double *n, double *a, double *b)
{
    double rho = sqrt(n[0] * n[0] + n[1] * n[1]);
    double X[3], Y[3];
    if (rho > 0) {
        X[0] = -n[1] / rho;
        X[1] = n[0] / rho;
        X[2] = 0.0;
    } else { /* source at a pole: any X perpendicular to n */
        X[0] = 1.0;
        X[1] = 0.0;
        X[2] = 0.0;
    }
    Y[0] = n[1] * X[2] - n[2] * X[1];
    Y[1] = n[2] * X[0] - n[0] * X[2];
    Y[2] = n[0] * X[1] - n[1] * X[0];
    double M[3][3] = {{D[0], D[1], D[2]}, {D[1], D[3], D[4]}, {D[2], D[4], D[5]}};
    double sp = 0.0, sx = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            sp += M[i][j] * (X[i] * X[j] - Y[i] * Y[j]);
            sx += M[i][j] * (X[i] * Y[j] + Y[i] * X[j]);
        }
    *a = sp;
    *b = sx;
}

/* rho^2 of one SFT (step 1 above). */
double or_rho2(const double *D, const double *n, double h0, double cosi, double psi, double t_sft,
               double s_n)
{
    double a, b;
    or_antenna_ab(D, n, &a, &b);
    double c2 = cos(2.0 * psi), s2 = sin(2.0 * psi);
    double fp = a * c2 + b * s2, fx = b * c2 - a * s2;
    double ap = 0.5 * (1.0 + cosi * cosi), ax = cosi;
    double q2 = fp * fp * ap * ap + fx * fx * ax * ax;
    double h = 0.7737 * 0.5 * t_sft * h0;
    return 4.0 * h * h * q2 / (t_sft * s_n);
}

/* ---------------------------------------------------------------- one run */

typedef struct {
    int64_t n_sft;
    int64_t k_lo;
    const double *t_mid; /* [n_sft] */
    const double *v;     /* [n_sft][3] */
    const double *w;     /* [n_sft] or NULL */
    const double *s_n;   /* [n_sft] */
    const double *D;     /* [n_sft][6] detector tensors */
    double t0, t_sft;
    int64_t K0, n_f0, n_f1;
    const double *f1;    /* [n_f1] */
    int64_t n_sky;
    const double *sky;   /* [n_sky][3] */
} or_inj_problem;

typedef struct {
    double h0, cosi, psi, f0, f1, n[3];
} or_inj;

/* canonical bin (ft_oracle.c) */
int64_t or_bin_q32(int64_t K0, int64_t k_lo, int64_t j, double f1, double tau, const double *v,
                   const double *n);

typedef struct {
    double d;
    int64_t i;
} dot_idx;

static int cmp_dot(const void *pa, const void *pb)
{
    const dot_idx *a = pa, *b = pb;
    if (a->d > b->d)
        return -1;
    if (a->d < b->d)
        return 1;
    return (a->i < b->i) ? -1 : (a->i > b->i);
}

/* The K bank sky points nearest to n (largest dot product, ties by index), ascending by
 * rank.  Dot products in FP64: fma(n2, m2, fma(n1, m1, n0 m0)). */
void or_nearest_sky(const or_inj_problem *p, const double *n, int K, int64_t *out)
{
    dot_idx *d = malloc(sizeof(dot_idx) * p->n_sky);
    for (int64_t i = 0; i < p->n_sky; i++) {
        const double *m = p->sky + 3 * i;
        d[i].d = fma(n[2], m[2], fma(n[1], m[1], n[0] * m[0]));
        d[i].i = i;
    }
    qsort(d, p->n_sky, sizeof(dot_idx), cmp_dot);
    for (int k = 0; k < K && k < p->n_sky; k++)
        out[k] = d[k].i;
    free(d);
}

/* Signal bin of SFT a relative to k_lo: floor((f0 T + f1 tau)(1 + eps) - k_lo + 1/2) with
 * tau = (t - t0) T and eps = fma(vz, nz, fma(vy, ny, vx nx)); FP64 in this order. */
int64_t or_signal_bin(const or_inj_problem *p, const or_inj *inj, int64_t a)
{
    const double *v = p->v + 3 * a;
    double eps = fma(v[2], inj->n[2], fma(v[1], inj->n[1], v[0] * inj->n[0]));
    double tau = (p->t_mid[a] - p->t0) * p->t_sft;
    double x = fma(inj->f0, p->t_sft, inj->f1 * tau) * (1.0 + eps) - (double)p->k_lo;
    return (int64_t)floor(x + 0.5);
}

/* Normalised power of absolute bin kabs in SFT a of run (run_id, seed) (step 2). */
double or_inj_power(int64_t kabs, int64_t a, uint64_t run_id, uint64_t seed, double amp,
                    double noise_scale)
{
    uint32_t ctr[4] = {(uint32_t)kabs, (uint32_t)a, (uint32_t)run_id, (uint32_t)(run_id >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    double r2 = -2.0 * log(or_uniform24(o[0]));
    if (amp == 0.0)
        return noise_scale * noise_scale * r2;
    double r = noise_scale * sqrt(r2);
    return r * r + amp * amp + 2.0 * amp * r * cos(2.0 * M_PI * or_uniform24(o[1]));
}

/* One run: returns max z over the local bank, the argmax template index, the number of
 * reads outside the generated window and (second_z, nullable) the second largest z of the
 * local bank, so that a caller can tell near-ties of the loudest template apart.  h0 is in the
 * units of sqrt(S_n T_SFT) of the data; half_f0 and H set the local f0 span and the window
 * half-width. */
void or_injection(const or_inj_problem *p, const or_inj *inj_in, uint64_t run_id, uint64_t seed,
                  int K, int half_f0, int H, double noise_scale, double *max_z, int64_t *argmax,
                  int64_t *oob_out, double *second_z)
{
    or_inj inj = *inj_in;
    int64_t *sky = malloc(sizeof(int64_t) * K);
    if (K > p->n_sky)
        K = (int)p->n_sky;
    or_nearest_sky(p, inj.n, K, sky);
    int64_t jc = (int64_t)floor(inj.f0 * p->t_sft + 0.5) - p->K0;
    int64_t j_lo = jc - half_f0, j_hi = jc + half_f0;
    if (j_lo < 0)
        j_lo = 0;
    if (j_hi > p->n_f0 - 1)
        j_hi = p->n_f0 - 1;
    double sw = 0.0, sw2 = 0.0;
    for (int64_t a = 0; a < p->n_sft; a++) {
        double w = p->w ? p->w[a] : 1.0;
        sw += w;
        sw2 += w * w;
    }
    double mu = 2.0 * sw, sigma = sqrt(4.0 * sw2);
    double best = -INFINITY;
    int64_t best_t = -1, oob = 0;
    int64_t nf0 = j_hi - j_lo + 1;
    int64_t ntl = nf0 * p->n_f1 * K;
    double *s = calloc(ntl, sizeof(double));
    double *P = malloc(sizeof(double) * (2 * H + 1));
    for (int64_t a = 0; a < p->n_sft; a++) {
        int64_t ks = or_signal_bin(p, &inj, a);
        double amp = inj.h0 > 0 ? sqrt(or_rho2(p->D + 6 * a, inj.n, inj.h0, inj.cosi, inj.psi,
                                                p->t_sft, p->s_n[a]))
                                : 0.0;
        for (int64_t q = -H; q <= H; q++)
            P[q + H] = or_inj_power(ks + q + p->k_lo, a, run_id, seed, q == 0 ? amp : 0.0,
                                    noise_scale);
        double w = p->w ? p->w[a] : 1.0;
        double tau = (p->t_mid[a] - p->t0) * p->t_sft;
        for (int64_t t = 0; t < ntl; t++) {
            int64_t jj = j_lo + t % nf0;
            int64_t r = t / nf0;
            int64_t if1 = r % p->n_f1, ks_i = r / p->n_f1;
            int64_t k = or_bin_q32(p->K0, p->k_lo, jj, p->f1[if1], tau, p->v + 3 * a,
                                   p->sky + 3 * sky[ks_i]);
            int64_t q = k - ks;
            if (q < -H || q > H) {
                oob++;
                continue;
            }
            s[t] += w * P[q + H];
        }
    }
    double second = -INFINITY;
    for (int64_t t = 0; t < ntl; t++) {
        int64_t jj = j_lo + t % nf0;
        int64_t r = t / nf0;
        int64_t if1 = r % p->n_f1, ks_i = r / p->n_f1;
        int64_t tg = (sky[ks_i] * p->n_f1 + if1) * p->n_f0 + jj;
        double z = (s[t] - mu) / sigma;
        if (z > best || (z == best && tg < best_t)) {
            second = best;
            best = z;
            best_t = tg;
        } else if (z > second) {
            second = z;
        }
    }
    *max_z = best;
    *argmax = best_t;
    *oob_out = oob;
    if (second_z)
        *second_z = second;
    free(s);
    free(P);
    free(sky);
}

/* Many independent runs (OpenMP over runs): run r uses run id first_id + r. */
void or_injections(const or_inj_problem *p, const or_inj *inj, int64_t n, uint64_t first_id,
                   uint64_t seed, int K, int half_f0, int H, double noise_scale, double *max_z,
                   int64_t *argmax, int64_t *oob, double *second_z)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n; r++)
        or_injection(p, inj + r, first_id + (uint64_t)r, seed, K, half_f0, H, noise_scale,
                     max_z + r, argmax + r, oob + r, second_z ? second_z + r : NULL);
}

/* ---------------------------------------------------------------- semi-analytic q */

/* Sec. V.A ("Simulating detection statistics"): for each population draw the two
 * signal-dependent numbers of q, rho1 = sum_alpha w_alpha rho^2_alpha and
 * rho2 = sum_alpha w_alpha^2 rho^2_alpha, with rho^2 of one SFT at h0 = 1 (or_rho2).
 * draws: [n][5] = (cos iota, psi, n_x, n_y, n_z); w may be NULL (all 1). */
void or_pdet_q(int64_t n_sft, double t_sft, const double *s_n, const double *D, const double *w,
               int64_t n, const double *draws, double *rho1, double *rho2)
{
    for (int64_t i = 0; i < n; i++) {
        const double *d = draws + 5 * i;
        double s1 = 0.0, s2 = 0.0;
        for (int64_t a = 0; a < n_sft; a++) {
            double r = or_rho2(D + 6 * a, d + 2, 1.0, d[0], d[1], t_sft, s_n[a]);
            double wa = w ? w[a] : 1.0;
            s1 += wa * r;
            s2 += wa * wa * r;
        }
        rho1[i] = s1;
        rho2[i] = s2;
    }
}

/* ---------------------------------------------------------------- sky-dependent weights */

/* Sec. II.B: the all-sky weights w_alpha(n) proportional to (a^2 + b^2) / S_n, with a, b
 * the detector response of SFT alpha to direction n (or_antenna_ab), normalised so that
 * sum_alpha w_alpha(n) = 1 for every sky point.  wsky: [n_sky][n_sft]. */
void or_sky_weights(int64_t n_sft, const double *D, const double *s_n, int64_t n_sky,
                    const double *sky, double *wsky)
{
    for (int64_t i = 0; i < n_sky; i++) {
        double *wi = wsky + i * n_sft;
        double tot = 0.0;
        for (int64_t a = 0; a < n_sft; a++) {
            double aa, bb;
            or_antenna_ab(D + 6 * a, sky + 3 * i, &aa, &bb);
            wi[a] = (aa * aa + bb * bb) / s_n[a];
            tot += wi[a];
        }
        for (int64_t a = 0; a < n_sft; a++)
            wi[a] /= tot;
    }
}
