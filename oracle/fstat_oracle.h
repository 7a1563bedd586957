/*
 * FP64 CPU oracle of the all-sky F-statistic search (test infrastructure).
 *
 * This is a plain, slow restatement of what the search computes, used only to
 * check the CUDA path: by the tests, by the package's smoke check and by the
 * benchmark's CPU-baseline leg.  Nothing in the product links it, and it shares
 * no code, header or table with the CUDA path.
 *
 * The paper (Sect. 1.1, Sect. 2 and its Fig. 1) fixes the order of the steps but
 * prints no formula; the formulas below are the textbook F-statistic readings:
 *
 *   per band   sigma^2 = (1/N) sum x_k^2; x upsampled U-fold by a zero-padded FFT
 *              ("resampling using the FFT and splines", Sect. 2)
 *   per sky    delay d_k = nhat . r_k (Sect. 2, ephemeris); detector time of the
 *              k-th barycentric sample by a two-step fixed point
 *              t = k dt - d(k dt - d(k dt)), d linearly interpolated; a(t), b(t)
 *              amplitude modulations; y_k = Keys-cubic interpolant of the
 *              upsampled series at t, times exp(-2 pi i f_off d(t))
 *              ("amplitude and phase demodulation", "resampling", Fig. 1)
 *   per cell   z_k = y_k {a_k, b_k} exp(-i pi fdot (k dt)^2) ("spindown
 *              demodulation"), zero-padded to n_fft >= 2N ("Fourier transform
 *              twice as long"), two FFTs F_a, F_b, then
 *              F = |F_a|^2/(sigma^2 S_aa) + |F_b|^2/(sigma^2 S_bb)
 *              (or the full form with S_ab), and 2F > threshold registers a
 *              candidate (sky, frequency, spindown, F).
 *
 * Every function returns 0 on success and a negative value on a bad argument or
 * a failed allocation.
 */
#ifndef FSTAT_ORACLE_H
#define FSTAT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t n;          /* samples in the band */
    double dt;          /* sampling interval, s */
    double f_off;       /* lower band edge, Hz */
    const double *x;    /* x[n], real */
    const double *r;    /* r[3n], detector->SSB vector per sample, light-seconds, (x,y,z) */
    double phi0;        /* sidereal phase at the first sample, rad */
    double eps;         /* obliquity of the ecliptic, rad (carried; r is equatorial) */
    int64_t n_fft;      /* transform length, a power of two >= 2n (0: smallest such) */
} orc_band;

typedef struct {
    double lat;         /* detector latitude, rad */
    double gamma;       /* arm-bisector orientation, counter-clockwise from East, rad */
    int upsample;       /* U >= 1 */
    double sigma2;      /* noise variance; <= 0: estimate from x */
    int full_form;      /* 0: F with S_aa, S_bb only; 1: full form with S_ab */
    int amp_mode;       /* 0: JKS a(t), b(t); 1: diagnostic a = 1, b = 0 */
    int interbin;       /* 0: exact zero-padded transform of length n_fft;
                           1: the paper's "Fourier transform interpolation" (Sect. 2)
                           read as interbinning: a transform of length M = n_fft/2,
                           even bins 2k = X(k), odd bins 2k+1 = (pi/4)(X(k) - X(k+1)),
                           X(M) = X(0) */
} orc_params;

typedef struct {
    int32_t band;
    int32_t pad_;
    int64_t sky, spin, bin;
    double F;
} orc_candidate;

/* ---- transforms ------------------------------------------------------------ */
/* z: n complex numbers interleaved (re, im).  sign = -1: sum z_j e^{-2 pi i jk/n};
   sign = +1: e^{+...}.  No scaling. */
int orc_fft_pow2(double *z, int64_t n, int sign);
int orc_fft_any(double *z, int64_t n, int sign);   /* Bluestein when n is not 2^p */
int orc_dft_brute(const double *z, double *out, int64_t n, int sign);

/* ---- per-band steps -------------------------------------------------------- */
double orc_sigma2(const double *x, int64_t n);
int orc_upsample(const double *x, int64_t n, int U, double *xu /* [U n] */);
double orc_keys(const double *xu, int64_t m, double p);

/* ---- per-sky steps --------------------------------------------------------- */
void orc_ab(double lat, double gamma, double alpha, double delta, double lst,
            double *a, double *b);
double orc_delay_lin(const double *dk, int64_t n, double u);
/* Geometry, resampling and phase demodulation for one sky position.
   Outputs (any may be NULL): y[2n] complex, a[n], b[n], mask[n],
   u[n] (detector time / dt of each barycentric sample), S[3] = S_aa, S_bb, S_ab. */
int orc_sky_prepare(const orc_band *band, const orc_params *p, const double *xu,
                    double alpha, double delta, double *y, double *a, double *b,
                    uint8_t *mask, double *u, double *S);

/* ---- per-cell steps -------------------------------------------------------- */
/* F over bins [bin_lo, bin_hi] of one (sky, spindown) cell.  work: 4*n_fft doubles
   or NULL. */
int orc_cell_F(const orc_band *band, const orc_params *p, const double *y, const double *a,
               const double *b, const double *S, double sigma2, double fdot,
               int64_t bin_lo, int64_t bin_hi, double *F, double *work);

/* Brute-force demodulated DFT without resampling, at detector samples t_n = n dt:
   F^a(l) = sum_n x_n a(t_n) exp(-i[2 pi f_l tau_n + pi fdot tau_n^2 + 2 pi f_off d_n])
   with tau_n = t_n + d_n and f_l = l/(n_fft dt), over the samples whose tau_n lies
   in the resampled window [0, (n-1) dt] (S sums over the same samples); same F
   combination. */
int orc_exact_F(const orc_band *band, const orc_params *p, double alpha, double delta,
                double fdot, double sigma2, const int64_t *bins, int64_t n_bins, double *F);

/* ---- whole search ---------------------------------------------------------- */
/* All cells (or the listed (sky, spin) pairs of band `only_band` when cells != NULL),
   threaded over sky positions round-robin.  Candidates: 2F > thr_2F, sorted by
   (band, sky, spin, bin).  bin_lo = bin_hi = 0 selects [1, n_fft/2 - 1].
   Returns the number written (<= cap); *n_total receives the full count. */
int64_t orc_search(const orc_band *bands, int n_bands, const orc_params *p,
                   int64_t n_sky, const double *alpha, const double *delta,
                   int64_t n_spin, const double *fdot, double thr_2F,
                   int64_t bin_lo, int64_t bin_hi, int nthreads,
                   orc_candidate *out, int64_t cap, int64_t *n_total);

/* F for every bin of the listed cells of one band: F[c * nb + (l - lo)],
   nb = hi - lo + 1.  cells_sky / cells_spin index the grids. */
int orc_cells_F(const orc_band *band, const orc_params *p, const double *alpha,
                const double *delta, const double *fdot, const int64_t *cells_sky,
                const int64_t *cells_spin, int64_t n_cells, int64_t bin_lo,
                int64_t bin_hi, int nthreads, double *F);

/* ---- grid from the generating matrix M (Sect. 2, grid.bin) ---------------- */
/* M: 4 x 4 row-major, rows = frequency, spindown, sky n, sky m directions in the
   coordinates (f dt, fdot dt^2/2, f_ref tau_E beta1, f_ref tau_E beta2), beta the
   ecliptic-plane components of the unit vector towards the source, tau_E = 1 AU/c.
   orc_lattice_spin: fdot[s - s_lo] of the spindown integers s_lo..s_hi from the
   spindown row alone.  orc_lattice_sky: the sky points (n, m) of [n_lo, n_hi] x
   [m_lo, m_hi] that lie on the sphere, north ecliptic hemisphere first (then the
   south one when hemispheres = 2), n then m ascending; alpha, delta (rad) and
   nm[3 c .. 3 c + 2] = (hemisphere 0/1, n, m) of the first cap points; *count =
   all points. */
int orc_lattice_spin(const double *M, double dt, int64_t s_lo, int64_t s_hi, double *fdot);
int orc_lattice_sky(const double *M, double f_ref, double eps, int64_t n_lo, int64_t n_hi,
                    int64_t m_lo, int64_t m_hi, int hemispheres, double *alpha, double *delta,
                    int64_t *nm, int64_t cap, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
