/*
 * FP64 CPU oracle of the all-sky F-statistic search -- test infrastructure only.
 * Used by the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg; never by the product path.  See fstat_oracle.h for the steps and the
 * passages they follow.  Everything here is double precision and deliberately
 * plain: no blocking, no fusion, one step after the other in the order of the
 * flow diagram (Fig. 1).
 */
#include "fstat_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559
#define PI_D 3.1415926535897932384626433832795
/* Earth's sidereal rotation rate, rad/s (one turn per 86164.0905 s). */
#define OMEGA_R (TWO_PI / 86164.0905)

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* Kahan-compensated accumulator. */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double v) {
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* ============================================================== transforms === */

/* Iterative radix-2 decimation-in-time FFT, in place, natural order in and out.
   Twiddles e^{sign 2 pi i k / n} are each evaluated directly with cos/sin. */
int orc_fft_pow2(double *z, int64_t n, int sign) {
    if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
    if (n == 1) return 0;
    double *tw = (double *)malloc(sizeof(double) * (size_t)n);  /* n/2 complex */
    if (!tw) return -2;
    for (int64_t k = 0; k < n / 2; ++k) {
        double ang = sign * TWO_PI * (double)k / (double)n;
        tw[2 * k] = cos(ang);
        tw[2 * k + 1] = sin(ang);
    }
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = z[2 * i], ti = z[2 * i + 1];
            z[2 * i] = z[2 * j]; z[2 * i + 1] = z[2 * j + 1];
            z[2 * j] = tr; z[2 * j + 1] = ti;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1, step = n / len;
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < half; ++k) {
                double wr = tw[2 * k * step], wi = tw[2 * k * step + 1];
                double *p = z + 2 * (i + k), *q = z + 2 * (i + k + half);
                double vr = q[0] * wr - q[1] * wi;
                double vi = q[0] * wi + q[1] * wr;
                q[0] = p[0] - vr; q[1] = p[1] - vi;
                p[0] += vr; p[1] += vi;
            }
        }
    }
    free(tw);
    return 0;
}

/* The definition: out_k = sum_j z_j e^{sign 2 pi i jk/n}, O(n^2).  The exponent
   index jk is reduced mod n in integer arithmetic before the angle is formed. */
int orc_dft_brute(const double *z, double *out, int64_t n, int sign) {
    if (n <= 0 || (sign != 1 && sign != -1)) return -1;
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t m = (int64_t)(((__int128)j * k) % n);
            double ang = sign * TWO_PI * (double)m / (double)n;
            double c = cos(ang), s = sin(ang);
            sr += z[2 * j] * c - z[2 * j + 1] * s;
            si += z[2 * j] * s + z[2 * j + 1] * c;
        }
        out[2 * k] = sr;
        out[2 * k + 1] = si;
    }
    return 0;
}

/* Any length: radix-2 for powers of two, else Bluestein's chirp-z identity
   jk = (j^2 + k^2 - (k-j)^2)/2, which turns the DFT into a convolution that is
   evaluated with power-of-two FFTs of length M >= 2n - 1. */
int orc_fft_any(double *z, int64_t n, int sign) {
    if (n <= 0 || (sign != 1 && sign != -1)) return -1;
    if (is_pow2(n)) return orc_fft_pow2(z, n, sign);
    int64_t M = 1;
    while (M < 2 * n - 1) M <<= 1;
    double *c = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double *A = (double *)calloc(2 * (size_t)M, sizeof(double));
    double *B = (double *)calloc(2 * (size_t)M, sizeof(double));
    if (!c || !A || !B) { free(c); free(A); free(B); return -2; }
    for (int64_t m = 0; m < n; ++m) {
        /* c_m = e^{sign i pi m^2 / n}; m^2 mod 2n keeps the angle small */
        int64_t q = (int64_t)(((__int128)m * m) % (2 * n));
        double ang = sign * PI_D * (double)q / (double)n;
        c[2 * m] = cos(ang);
        c[2 * m + 1] = sin(ang);
    }
    for (int64_t j = 0; j < n; ++j) {           /* A_j = z_j c_j */
        A[2 * j] = z[2 * j] * c[2 * j] - z[2 * j + 1] * c[2 * j + 1];
        A[2 * j + 1] = z[2 * j] * c[2 * j + 1] + z[2 * j + 1] * c[2 * j];
    }
    for (int64_t m = 0; m < n; ++m) {           /* B_m = conj(c_m), wrapped for m < 0 */
        B[2 * m] = c[2 * m];
        B[2 * m + 1] = -c[2 * m + 1];
        if (m > 0) {
            B[2 * (M - m)] = c[2 * m];
            B[2 * (M - m) + 1] = -c[2 * m + 1];
        }
    }
    int rc = orc_fft_pow2(A, M, -1);
    if (!rc) rc = orc_fft_pow2(B, M, -1);
    if (!rc) {
        for (int64_t k = 0; k < M; ++k) {
            double ar = A[2 * k], ai = A[2 * k + 1], br = B[2 * k], bi = B[2 * k + 1];
            A[2 * k] = ar * br - ai * bi;
            A[2 * k + 1] = ar * bi + ai * br;
        }
        rc = orc_fft_pow2(A, M, +1);
    }
    if (!rc) {
        for (int64_t k = 0; k < n; ++k) {       /* X_k = c_k (A*B)_k / M */
            double vr = A[2 * k] / (double)M, vi = A[2 * k + 1] / (double)M;
            z[2 * k] = vr * c[2 * k] - vi * c[2 * k + 1];
            z[2 * k + 1] = vr * c[2 * k + 1] + vi * c[2 * k];
        }
    }
    free(c); free(A); free(B);
    return rc;
}

/* ============================================================ per band === */

double orc_sigma2(const double *x, int64_t n) {
    ksum k = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) kadd(&k, x[i] * x[i]);
    return k.s / (double)n;
}

/* U-fold trigonometric interpolation: the length-N spectrum is placed in a
   length-UN spectrum (positive frequencies low, negative high, the Nyquist bin
   of an even N split in half between +N/2 and -N/2), and transformed back, so
   that xu[U k] = x[k] and xu is the band-limited interpolant in between. */
int orc_upsample(const double *x, int64_t n, int U, double *xu) {
    if (n < 2 || U < 1) return -1;
    if (U == 1) { memcpy(xu, x, sizeof(double) * (size_t)n); return 0; }
    int64_t M = (int64_t)U * n;
    double *X = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double *Y = (double *)calloc(2 * (size_t)M, sizeof(double));
    if (!X || !Y) { free(X); free(Y); return -2; }
    for (int64_t k = 0; k < n; ++k) { X[2 * k] = x[k]; X[2 * k + 1] = 0.0; }
    int rc = orc_fft_any(X, n, -1);
    if (!rc) {
        int64_t npos = (n % 2 == 0) ? n / 2 : (n + 1) / 2;   /* bins 0 .. npos-1 */
        for (int64_t m = 0; m < npos; ++m) { Y[2 * m] = X[2 * m]; Y[2 * m + 1] = X[2 * m + 1]; }
        int64_t neg0 = (n % 2 == 0) ? n / 2 + 1 : (n + 1) / 2;
        for (int64_t m = neg0; m < n; ++m) {
            Y[2 * (M - n + m)] = X[2 * m];
            Y[2 * (M - n + m) + 1] = X[2 * m + 1];
        }
        if (n % 2 == 0) {
            int64_t h = n / 2;
            Y[2 * h] = 0.5 * X[2 * h];           Y[2 * h + 1] = 0.5 * X[2 * h + 1];
            Y[2 * (M - h)] = 0.5 * X[2 * h];     Y[2 * (M - h) + 1] = 0.5 * X[2 * h + 1];
        }
        rc = orc_fft_any(Y, M, +1);
    }
    if (!rc)
        for (int64_t j = 0; j < M; ++j) xu[j] = Y[2 * j] / (double)n;
    free(X); free(Y);
    return rc;
}

/* Keys cubic convolution with a = -1/2 (the Catmull-Rom spline) at real position
   p on a series of period m: four samples i-1 .. i+2 around i = floor(p). */
double orc_keys(const double *xu, int64_t m, double p) {
    double fl = floor(p);
    double mu = p - fl;
    int64_t i = (int64_t)fl;
    double w[4];
    w[0] = ((-0.5 * mu + 1.0) * mu - 0.5) * mu;
    w[1] = (1.5 * mu - 2.5) * mu * mu + 1.0;
    w[2] = ((-1.5 * mu + 2.0) * mu + 0.5) * mu;
    w[3] = (0.5 * mu - 0.5) * mu * mu;
    double v = 0.0;
    for (int j = 0; j < 4; ++j) {
        int64_t idx = (i - 1 + j) % m;
        if (idx < 0) idx += m;
        v += w[j] * xu[idx];
    }
    return v;
}

/* ============================================================= per sky === */

/* Amplitude modulation functions of a right-angle interferometer at latitude
   lat with arm bisector at gamma (counter-clockwise from East), for a source at
   (alpha, delta) when the local sidereal time is lst (Jaranowski, Krolak &
   Schutz 1998, the a(t) and b(t) of the F-statistic). */
void orc_ab(double lat, double gamma, double alpha, double delta, double lst,
            double *a, double *b) {
    double h = alpha - lst;
    double s2g = sin(2 * gamma), c2g = cos(2 * gamma);
    double sl = sin(lat), cl = cos(lat), s2l = sin(2 * lat), c2l = cos(2 * lat);
    double sd = sin(delta), cd = cos(delta), s2d = sin(2 * delta), c2d = cos(2 * delta);
    *a = (1.0 / 16.0) * s2g * (3.0 - c2l) * (3.0 - c2d) * cos(2 * h)
       - 0.25 * c2g * sl * (3.0 - c2d) * sin(2 * h)
       + 0.25 * s2g * s2l * s2d * cos(h)
       - 0.5 * c2g * cl * s2d * sin(h)
       + 0.75 * s2g * cl * cl * cd * cd;
    *b = c2g * sl * sd * cos(2 * h)
       + 0.25 * s2g * (3.0 - c2l) * sd * sin(2 * h)
       + c2g * cl * cd * cos(h)
       + 0.5 * s2g * s2l * cd * sin(h);
}

/* Delay at fractional sample position u by linear interpolation between the two
   neighbouring samples (the end segments extend linearly beyond the data). */
double orc_delay_lin(const double *dk, int64_t n, double u) {
    double fl = floor(u);
    int64_t j = (int64_t)fl;
    if (j < 0) j = 0;
    if (j > n - 2) j = n - 2;
    double f = u - (double)j;
    return dk[j] + f * (dk[j + 1] - dk[j]);
}

int orc_sky_prepare(const orc_band *band, const orc_params *p, const double *xu,
                    double alpha, double delta, double *y, double *a, double *b,
                    uint8_t *mask, double *u_out, double *S) {
    int64_t n = band->n;
    double dt = band->dt;
    if (n < 2 || dt <= 0.0 || p->upsample < 1) return -1;
    int64_t M = (int64_t)p->upsample * n;
    double nh[3] = {cos(delta) * cos(alpha), cos(delta) * sin(alpha), sin(delta)};
    double *dk = (double *)malloc(sizeof(double) * (size_t)n);
    if (!dk) return -2;
    for (int64_t k = 0; k < n; ++k)   /* Roemer delay nhat . r_k, seconds */
        dk[k] = nh[0] * band->r[3 * k] + nh[1] * band->r[3 * k + 1] + nh[2] * band->r[3 * k + 2];
    ksum saa = {0, 0}, sbb = {0, 0}, sab = {0, 0};
    for (int64_t k = 0; k < n; ++k) {
        /* detector time t of the k-th barycentric sample, as a sample position u */
        double u0 = (double)k - dk[k] / dt;
        double d1 = orc_delay_lin(dk, n, u0);
        double u = (double)k - d1 / dt;
        double d2 = orc_delay_lin(dk, n, u);
        int valid = (u >= 0.0) && (u <= (double)(n - 1));
        double t = u * dt;
        double av, bv;
        if (p->amp_mode == 1) { av = 1.0; bv = 0.0; }
        else orc_ab(p->lat, p->gamma, alpha, delta, band->phi0 + OMEGA_R * t, &av, &bv);
        double yr = 0.0, yi = 0.0;
        if (valid) {
            double v = orc_keys(xu, M, (double)p->upsample * u);
            double cyc = band->f_off * d2;            /* residual phase, cycles */
            double fr = cyc - floor(cyc);
            yr = v * cos(TWO_PI * fr);
            yi = -v * sin(TWO_PI * fr);
            kadd(&saa, av * av);
            kadd(&sbb, bv * bv);
            kadd(&sab, av * bv);
        }
        if (y) { y[2 * k] = yr; y[2 * k + 1] = yi; }
        if (a) a[k] = av;
        if (b) b[k] = bv;
        if (mask) mask[k] = (uint8_t)valid;
        if (u_out) u_out[k] = u;
    }
    if (S) { S[0] = saa.s; S[1] = sbb.s; S[2] = sab.s; }
    free(dk);
    return 0;
}

/* ============================================================ per cell === */

static double fstat_combine(const orc_params *p, const double *S, double sigma2,
                            double far, double fai, double fbr, double fbi) {
    double pa = far * far + fai * fai, pb = fbr * fbr + fbi * fbi;
    if (p->full_form) {
        double D = S[0] * S[1] - S[2] * S[2];
        double cr = far * fbr + fai * fbi;     /* Re(F_a conj(F_b)) */
        return (S[1] * pa + S[0] * pb - 2.0 * S[2] * cr) / (sigma2 * D);
    }
    double F = 0.0;
    if (S[0] > 0.0) F += pa / (sigma2 * S[0]);
    if (S[1] > 0.0) F += pb / (sigma2 * S[1]);
    return F;
}

int orc_cell_F(const orc_band *band, const orc_params *p, const double *y, const double *a,
               const double *b, const double *S, double sigma2, double fdot,
               int64_t bin_lo, int64_t bin_hi, double *F, double *work) {
    int64_t n = band->n, nf = band->n_fft;
    if (!is_pow2(nf) || nf < 2 * n || bin_lo < 0 || bin_hi >= nf || bin_lo > bin_hi) return -1;
    double *za = work ? work : (double *)malloc(sizeof(double) * 4 * (size_t)nf);
    if (!za) return -2;
    double *zb = za + 2 * nf;
    memset(za, 0, sizeof(double) * 4 * (size_t)nf);
    for (int64_t k = 0; k < n; ++k) {
        double tk = (double)k * band->dt;
        double cyc = 0.5 * fdot * tk * tk;        /* spindown phase, cycles */
        double fr = cyc - floor(cyc);
        double c = cos(TWO_PI * fr), s = -sin(TWO_PI * fr);
        double wr = y[2 * k] * c - y[2 * k + 1] * s;
        double wi = y[2 * k] * s + y[2 * k + 1] * c;
        za[2 * k] = a[k] * wr; za[2 * k + 1] = a[k] * wi;
        zb[2 * k] = b[k] * wr; zb[2 * k + 1] = b[k] * wi;
    }
    if (p->interbin) {
        /* interbinning: a transform of half the length (still >= n), even output
           bins taken as they are, odd bins from the difference of the two
           neighbours scaled by pi/4 (the value a tone half-way between two
           Fourier frequencies has there) */
        const int64_t m = nf / 2;
        int rc = orc_fft_pow2(za, m, -1);
        if (!rc) rc = orc_fft_pow2(zb, m, -1);
        if (!rc)
            for (int64_t l = bin_lo; l <= bin_hi; ++l) {
                const int64_t k = l / 2, k1 = (k + 1) % m;
                double ar = za[2 * k], ai = za[2 * k + 1], br = zb[2 * k], bi = zb[2 * k + 1];
                if (l % 2) {
                    const double q = 0.25 * PI_D;
                    ar = q * (ar - za[2 * k1]); ai = q * (ai - za[2 * k1 + 1]);
                    br = q * (br - zb[2 * k1]); bi = q * (bi - zb[2 * k1 + 1]);
                }
                F[l - bin_lo] = fstat_combine(p, S, sigma2, ar, ai, br, bi);
            }
        if (!work) free(za);
        return rc;
    }
    int rc = orc_fft_pow2(za, nf, -1);
    if (!rc) rc = orc_fft_pow2(zb, nf, -1);
    if (!rc)
        for (int64_t l = bin_lo; l <= bin_hi; ++l)
            F[l - bin_lo] = fstat_combine(p, S, sigma2, za[2 * l], za[2 * l + 1], zb[2 * l],
                                          zb[2 * l + 1]);
    if (!work) free(za);
    return rc;
}

int orc_exact_F(const orc_band *band, const orc_params *p, double alpha, double delta,
                double fdot, double sigma2, const int64_t *bins, int64_t n_bins, double *F) {
    int64_t n = band->n;
    double dt = band->dt;
    double nh[3] = {cos(delta) * cos(alpha), cos(delta) * sin(alpha), sin(delta)};
    double *av = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    if (!av) return -2;
    double *bv = av + n, *tau = av + 2 * n, *dd = av + 3 * n;
    ksum saa = {0, 0}, sbb = {0, 0}, sab = {0, 0};
    for (int64_t k = 0; k < n; ++k) {
        double t = (double)k * dt;
        dd[k] = nh[0] * band->r[3 * k] + nh[1] * band->r[3 * k + 1] + nh[2] * band->r[3 * k + 2];
        tau[k] = t + dd[k];
        if (p->amp_mode == 1) { av[k] = 1.0; bv[k] = 0.0; }
        else orc_ab(p->lat, p->gamma, alpha, delta, band->phi0 + OMEGA_R * t, &av[k], &bv[k]);
        /* only samples whose barycentric time falls in the resampled window
           [0, (n-1) dt] enter, as in the resampled search */
        if (tau[k] < 0.0 || tau[k] > (double)(n - 1) * dt) { av[k] = 0.0; bv[k] = 0.0; }
        kadd(&saa, av[k] * av[k]); kadd(&sbb, bv[k] * bv[k]); kadd(&sab, av[k] * bv[k]);
    }
    double S[3] = {saa.s, sbb.s, sab.s};
    for (int64_t i = 0; i < n_bins; ++i) {
        double f = (double)bins[i] / ((double)band->n_fft * dt);
        double far = 0, fai = 0, fbr = 0, fbi = 0;
        for (int64_t k = 0; k < n; ++k) {
            double cyc = f * tau[k] + 0.5 * fdot * tau[k] * tau[k] + band->f_off * dd[k];
            double fr = cyc - floor(cyc);
            double c = cos(TWO_PI * fr), s = -sin(TWO_PI * fr);
            double xv = band->x[k];
            far += xv * av[k] * c; fai += xv * av[k] * s;
            fbr += xv * bv[k] * c; fbi += xv * bv[k] * s;
        }
        F[i] = fstat_combine(p, S, sigma2, far, fai, fbr, fbi);
    }
    free(av);
    return 0;
}

/* ========================================================== whole search === */

typedef struct {
    orc_candidate *v;
    int64_t n, cap;
} cand_vec;

static int cv_push(cand_vec *cv, orc_candidate c) {
    if (cv->n == cv->cap) {
        int64_t nc = cv->cap ? 2 * cv->cap : 1024;
        orc_candidate *nv = (orc_candidate *)realloc(cv->v, sizeof(orc_candidate) * (size_t)nc);
        if (!nv) return -2;
        cv->v = nv; cv->cap = nc;
    }
    cv->v[cv->n++] = c;
    return 0;
}

typedef struct {
    const orc_band *band;
    int band_idx;
    const orc_params *p;
    const double *xu;
    double sigma2;
    int64_t n_sky, n_spin;
    const double *alpha, *delta, *fdot;
    double thr;
    int64_t lo, hi;
    int tid, nthreads;
    cand_vec out;
    int rc;
    /* cell-list mode */
    const int64_t *cells_sky, *cells_spin;
    int64_t n_cells;
    double *F_all;
} worker_arg;

static void *search_worker(void *argp) {
    worker_arg *w = (worker_arg *)argp;
    int64_t n = w->band->n, nf = w->band->n_fft, nb = w->hi - w->lo + 1;
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    double *work = (double *)malloc(sizeof(double) * 4 * (size_t)nf);
    double *F = (double *)malloc(sizeof(double) * (size_t)nb);
    w->rc = 0;
    if (!y || !a || !b || !work || !F) { w->rc = -2; goto done; }
    double S[3];
    if (w->cells_sky) {
        /* contiguous chunks, so that a caller grouping cells by sky prepares each
           sky once per thread */
        int64_t chunk = (w->n_cells + w->nthreads - 1) / w->nthreads;
        int64_t c0 = (int64_t)w->tid * chunk, c1 = c0 + chunk;
        if (c1 > w->n_cells) c1 = w->n_cells;
        int64_t prev_sky = -1;
        for (int64_t c = c0; c < c1; ++c) {
            int64_t s = w->cells_sky[c], j = w->cells_spin[c];
            if (s != prev_sky) {
                w->rc = orc_sky_prepare(w->band, w->p, w->xu, w->alpha[s], w->delta[s], y, a, b,
                                        NULL, NULL, S);
                if (w->rc) goto done;
                prev_sky = s;
            }
            w->rc = orc_cell_F(w->band, w->p, y, a, b, S, w->sigma2, w->fdot[j], w->lo, w->hi,
                               w->F_all + c * nb, work);
            if (w->rc) goto done;
        }
        goto done;
    }
    for (int64_t s = w->tid; s < w->n_sky; s += w->nthreads) {   /* round-robin sky loop */
        w->rc = orc_sky_prepare(w->band, w->p, w->xu, w->alpha[s], w->delta[s], y, a, b, NULL,
                                NULL, S);
        if (w->rc) goto done;
        for (int64_t j = 0; j < w->n_spin; ++j) {                /* spindown loop */
            w->rc = orc_cell_F(w->band, w->p, y, a, b, S, w->sigma2, w->fdot[j], w->lo, w->hi,
                               F, work);
            if (w->rc) goto done;
            for (int64_t l = 0; l < nb; ++l) {
                if (2.0 * F[l] > w->thr) {
                    orc_candidate c = {w->band_idx, 0, s, j, w->lo + l, F[l]};
                    if (cv_push(&w->out, c)) { w->rc = -2; goto done; }
                }
            }
        }
    }
done:
    free(y); free(a); free(b); free(work); free(F);
    return NULL;
}

static int cand_cmp(const void *pa, const void *pb) {
    const orc_candidate *x = (const orc_candidate *)pa, *y = (const orc_candidate *)pb;
    if (x->band != y->band) return x->band < y->band ? -1 : 1;
    if (x->sky != y->sky) return x->sky < y->sky ? -1 : 1;
    if (x->spin != y->spin) return x->spin < y->spin ? -1 : 1;
    if (x->bin != y->bin) return x->bin < y->bin ? -1 : 1;
    return 0;
}

static int band_setup(const orc_band *band, const orc_params *p, double **xu, double *sigma2,
                      int64_t *lo, int64_t *hi, int64_t bin_lo, int64_t bin_hi) {
    if (band->n < 2 || !is_pow2(band->n_fft) || band->n_fft < 2 * band->n) return -1;
    *lo = bin_lo; *hi = bin_hi;
    if (bin_lo == 0 && bin_hi == 0) { *lo = 1; *hi = band->n_fft / 2 - 1; }
    if (*lo < 0 || *hi >= band->n_fft || *lo > *hi) return -1;
    *sigma2 = p->sigma2 > 0.0 ? p->sigma2 : orc_sigma2(band->x, band->n);
    *xu = (double *)malloc(sizeof(double) * (size_t)p->upsample * (size_t)band->n);
    if (!*xu) return -2;
    int rc = orc_upsample(band->x, band->n, p->upsample, *xu);
    if (rc) { free(*xu); *xu = NULL; }
    return rc;
}

static orc_band band_resolved(const orc_band *b) {
    orc_band r = *b;
    if (r.n_fft == 0) { r.n_fft = 1; while (r.n_fft < 2 * r.n) r.n_fft <<= 1; }
    return r;
}

int64_t orc_search(const orc_band *bands, int n_bands, const orc_params *p,
                   int64_t n_sky, const double *alpha, const double *delta,
                   int64_t n_spin, const double *fdot, double thr_2F,
                   int64_t bin_lo, int64_t bin_hi, int nthreads,
                   orc_candidate *out, int64_t cap, int64_t *n_total) {
    if (nthreads < 1) nthreads = 1;
    cand_vec all = {NULL, 0, 0};
    int64_t rcall = 0;
    for (int bi = 0; bi < n_bands && !rcall; ++bi) {
        orc_band band = band_resolved(&bands[bi]);
        double *xu = NULL, sigma2;
        int64_t lo, hi;
        int rc = band_setup(&band, p, &xu, &sigma2, &lo, &hi, bin_lo, bin_hi);
        if (rc) { rcall = rc; break; }
        worker_arg *wa = (worker_arg *)calloc((size_t)nthreads, sizeof(worker_arg));
        pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
        if (!wa || !th) { free(wa); free(th); free(xu); rcall = -2; break; }
        for (int t = 0; t < nthreads; ++t) {
            wa[t] = (worker_arg){&band, bi, p, xu, sigma2, n_sky, n_spin, alpha, delta, fdot,
                                 thr_2F, lo, hi, t, nthreads, {NULL, 0, 0}, 0,
                                 NULL, NULL, 0, NULL};
            pthread_create(&th[t], NULL, search_worker, &wa[t]);
        }
        for (int t = 0; t < nthreads; ++t) {
            pthread_join(th[t], NULL);
            if (wa[t].rc) rcall = wa[t].rc;
            for (int64_t i = 0; i < wa[t].out.n && !rcall; ++i)
                if (cv_push(&all, wa[t].out.v[i])) rcall = -2;
            free(wa[t].out.v);
        }
        free(wa); free(th); free(xu);
    }
    if (rcall) { free(all.v); return rcall; }
    qsort(all.v, (size_t)all.n, sizeof(orc_candidate), cand_cmp);
    int64_t nw = all.n < cap ? all.n : cap;
    if (nw > 0 && out) memcpy(out, all.v, sizeof(orc_candidate) * (size_t)nw);
    if (n_total) *n_total = all.n;
    free(all.v);
    return nw;
}

int orc_cells_F(const orc_band *band_in, const orc_params *p, const double *alpha,
                const double *delta, const double *fdot, const int64_t *cells_sky,
                const int64_t *cells_spin, int64_t n_cells, int64_t bin_lo,
                int64_t bin_hi, int nthreads, double *F) {
    if (nthreads < 1) nthreads = 1;
    orc_band band = band_resolved(band_in);
    double *xu = NULL, sigma2;
    int64_t lo, hi;
    int rc = band_setup(&band, p, &xu, &sigma2, &lo, &hi, bin_lo, bin_hi);
    if (rc) return rc;
    worker_arg *wa = (worker_arg *)calloc((size_t)nthreads, sizeof(worker_arg));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!wa || !th) { free(wa); free(th); free(xu); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        wa[t] = (worker_arg){&band, 0, p, xu, sigma2, 0, 0, alpha, delta, fdot, 0.0, lo, hi,
                             t, nthreads, {NULL, 0, 0}, 0, cells_sky, cells_spin, n_cells, F};
        pthread_create(&th[t], NULL, search_worker, &wa[t]);
    }
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (wa[t].rc) rc = wa[t].rc;
    }
    free(wa); free(th); free(xu);
    return rc;
}

/* ---- grid from the generating matrix (Sect. 2, grid.bin) ------------------- */
/* The paper: the rows of the 4 x 4 matrix M span the 4-D parameter space and the
   integer multiples of the rows are the grid points; a sky position is a pair of
   integers (n, m), a spindown an integer s.  Coordinates of the space (a reading:
   the reference that defines them is not available):
     w0 = f dt                 frequency, cycles per sample (the FFT's own grid)
     w1 = fdot dt^2 / 2        spindown, cycles per sample^2 (the phase w1 k^2)
     w2 = f_ref tau_E beta1    sky: the ecliptic-plane components (beta1, beta2)
     w3 = f_ref tau_E beta2    of the unit vector towards the source, in cycles of
                               the orbital Roemer phase at the reference frequency
   with tau_E = 1 AU / c.  Grid point (s, n, m) = s M[1] + n M[2] + m M[3]
   (rows 0..3 = frequency, spindown, sky n, sky m).  A sky point lies on the
   sphere when beta1^2 + beta2^2 <= 1; the ecliptic latitude's sign is the
   hemisphere (points on the ecliptic belong to the north one). */
#define TAU_E_S 499.00478383615643   /* 1 AU / c, s */

int orc_lattice_spin(const double *M, double dt, int64_t s_lo, int64_t s_hi, double *fdot) {
    if (!M || !fdot || !(dt > 0) || s_hi < s_lo) return -1;
    for (int64_t s = s_lo; s <= s_hi; ++s) {
        const double w1 = (double)s * M[4 + 1];
        fdot[s - s_lo] = 2.0 * w1 / (dt * dt);
    }
    return 0;
}

/* Equatorial (alpha, delta) of the unit vector with ecliptic components
   (beta1, beta2, h sqrt(1 - beta1^2 - beta2^2)). */
static void ecl_to_equ(double b1, double b2, double h, double eps, double *alpha, double *delta) {
    double q = 1.0 - b1 * b1 - b2 * b2;
    if (q < 0.0) q = 0.0;
    const double ze = h * sqrt(q);
    const double x = b1;
    const double y = b2 * cos(eps) - ze * sin(eps);
    const double z = b2 * sin(eps) + ze * cos(eps);
    double a = atan2(y, x);
    if (a < 0.0) a += TWO_PI;
    *alpha = a;
    *delta = asin(z > 1.0 ? 1.0 : (z < -1.0 ? -1.0 : z));
}

int orc_lattice_sky(const double *M, double f_ref, double eps, int64_t n_lo, int64_t n_hi,
                    int64_t m_lo, int64_t m_hi, int hemispheres, double *alpha, double *delta,
                    int64_t *nm, int64_t cap, int64_t *count) {
    if (!M || !count || !(f_ref > 0) || n_hi < n_lo || m_hi < m_lo ||
        (hemispheres != 1 && hemispheres != 2))
        return -1;
    const double scale = f_ref * TAU_E_S;
    int64_t c = 0;
    for (int hs = 0; hs < hemispheres; ++hs) {
        const double h = hs == 0 ? 1.0 : -1.0;
        for (int64_t n = n_lo; n <= n_hi; ++n)
            for (int64_t m = m_lo; m <= m_hi; ++m) {
                const double w2 = (double)n * M[8 + 2] + (double)m * M[12 + 2];
                const double w3 = (double)n * M[8 + 3] + (double)m * M[12 + 3];
                const double b1 = w2 / scale, b2 = w3 / scale;
                const double r2 = b1 * b1 + b2 * b2;
                if (hs == 0 ? !(r2 <= 1.0) : !(r2 < 1.0)) continue;
                if (c < cap) {
                    if (alpha && delta) ecl_to_equ(b1, b2, h, eps, &alpha[c], &delta[c]);
                    if (nm) { nm[3 * c] = hs; nm[3 * c + 1] = n; nm[3 * c + 2] = m; }
                }
                ++c;
            }
    }
    *count = c;
    return 0;
}
