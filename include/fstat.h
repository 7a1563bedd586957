/*
 * fstat.h -- C ABI of libfstat.so: the all-sky F-statistic search hot path on one
 * GB300 GPU (sm_103a), after Poghosyan et al., "Architecture, implementation and
 * parallelization of the software to search for periodic gravitational wave
 * signals" (CPC; arXiv:1410.3677).
 *
 * The problem statement follows the paper's Sect. 2: per (band, frame) the code
 * reads a narrow-band real time series sampled at dt, the detector-to-SSB vector
 * for every sample plus the sidereal phase phi0 at the first sample and the
 * obliquity eps, and a grid of sky positions and spindowns.  For every
 * (sky, spindown) cell it evaluates the F-statistic at every frequency bin of a
 * zero-padded FFT and registers the grid points where the statistic crosses a
 * threshold (Sect. 2 and Fig. 1: sky loop -> amplitude and phase demodulation
 * -> resampling -> spindown loop -> spindown demodulation -> FFT -> Fourier
 * transform interpolation -> F-statistic -> threshold).  A candidate carries the
 * sky position, frequency, spindown and the value of F (Sect. 2).
 *
 * Readings of what the paper leaves unstated (it prints no formula):
 *   F = |F_a|^2/(sigma^2 S_aa) + |F_b|^2/(sigma^2 S_bb), with F_a, F_b the
 *   FFTs of the resampled series weighted by the amplitude modulations a(t),
 *   b(t) of a right-angle interferometer (Jaranowski-Krolak-Schutz), S_aa, S_bb
 *   their sums of squares over the resampled window and sigma^2 = (1/N) sum x^2
 *   unless given; delay d = nhat . r in seconds (r in light-seconds, equatorial);
 *   detector time of barycentric sample k by the two-step fixed point
 *   t = k dt - d(k dt - d(k dt)) with d interpolated linearly; resampling by a
 *   U-fold FFT upsample then Keys cubic (a = -1/2) interpolation, samples whose
 *   detector time falls outside [0, (n-1) dt] set to zero; band-offset phase
 *   exp(-2 pi i f_off d(t)); spindown phase exp(-i pi fdot (k dt)^2); the "twice
 *   as long" transform as exact zero padding to n_fft >= 2n; strict 2F > thr.
 *
 * Conventions for every entry point:
 *   - returns an fstat_status; nothing throws across the ABI;
 *   - calls are synchronous with respect to the host (they return after the GPU
 *     work they queue has finished); a plan is not thread-safe, but different
 *     plans (each on its own stream) may be used from different host threads at
 *     the same time (their graph captures are thread-local);
 *   - the caller owns every array it passes and may free it after the call that
 *     received it returns; the plan owns all device memory it allocates;
 *   - after FSTAT_ERR_CUDA or FSTAT_ERR_TIMEOUT a plan is poisoned: later calls
 *     other than fstat_plan_destroy / fstat_plan_error return FSTAT_ERR_STATE.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FSTAT_OK = 0,
    FSTAT_ERR_ARG = 1,       /* invalid argument: nothing was done */
    FSTAT_ERR_OOM = 2,       /* a device or host allocation failed; nothing leaked */
    FSTAT_ERR_CUDA = 3,      /* a CUDA call failed; the plan is poisoned */
    FSTAT_ERR_OVERFLOW = 4,  /* more candidates than capacity; totals stay exact */
    FSTAT_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out; plan poisoned */
    FSTAT_ERR_STATE = 6,     /* plan poisoned by an earlier error, or misuse */
    FSTAT_ERR_INTERNAL = 7   /* an internal consistency check failed */
} fstat_status;

typedef enum {
    FSTAT_FP64_PLAIN = 0,    /* every step in FP64, one cell at a time */
    FSTAT_FP32_BATCHED = 1   /* FP32 resample/FFT/|F|^2; the delay in double-float
                                (~48-bit) and the spindown phase in 64-bit fixed point,
                                both reduced before any FP32 use; compensated sums;
                                many cells per launch */
} fstat_form;

/* One narrow band of one frame (Sect. 2: xdat_d_b.bin + DetSSB.bin). */
typedef struct {
    int64_t n;           /* samples, >= 16 */
    double dt;           /* sampling interval, s, > 0 */
    double f_off;        /* lower band edge, Hz (Eq. 1); enters the band-offset phase */
    const double *x;     /* x[n] float64, or NULL when x32 is given */
    const float *x32;    /* x[n] float32, or NULL when x is given (exactly one) */
    const double *r;     /* r[3n]: detector->SSB vector per sample, light-seconds,
                            equatorial, row-major (x, y, z) */
    double phi0;         /* sidereal phase of the detector at the first sample, rad */
    double eps;          /* obliquity of the ecliptic, rad; carried with the
                            ephemeris as in the paper, not used (r is equatorial) */
    int64_t n_fft;       /* transform length: 0 = smallest power of two >= 2n;
                            else a power of two >= 2n, 256 <= n_fft <= 2^20 */
} fstat_band;

/* The statistic evaluated per bin.  FSTAT_F_SIMPLE: F = |F_a|^2/(sigma^2 S_aa) +
   |F_b|^2/(sigma^2 S_bb) (the amplitude cross term S_ab neglected).  FSTAT_F_FULL:
   the Jaranowski-Krolak-Schutz form
     F = (S_bb |F_a|^2 + S_aa |F_b|^2 - 2 S_ab Re(F_a conj(F_b))) / (sigma^2 D),
     D = S_aa S_bb - S_ab^2,
   whose 2F follows a chi-square law with 4 degrees of freedom in Gaussian noise.
   S_aa, S_bb, S_ab are the sums of a^2, b^2, a b over the resampled window. */
typedef enum { FSTAT_F_SIMPLE = 0, FSTAT_F_FULL = 1 } fstat_statistic;

/* How the transform "twice as long" of Sect. 2 is formed.  FSTAT_INTERP_ZEROPAD:
   exact zero-padded transforms of length n_fft.  FSTAT_INTERP_INTERBIN: the
   paper's interpolation read as interbinning -- transforms of length n_fft / 2
   (still >= n), output bin 2k = X(k), bin 2k+1 = (pi/4)(X(k) - X(k+1)), X(n_fft/2)
   = X(0); the bins keep the n_fft grid.  About half the transform work; the odd
   bins are an approximation (exact for a tone half-way between Fourier
   frequencies, and a noise level of pi^2/4 per transform instead of 2).
   FSTAT_FP32_BATCHED only, n_fft in 2^13 .. 2^20. */
typedef enum { FSTAT_INTERP_ZEROPAD = 0, FSTAT_INTERP_INTERBIN = 1 } fstat_interpolation;

typedef struct {
    int n_bands;                 /* >= 1 */
    const fstat_band *bands;     /* [n_bands] */
    int64_t n_sky;               /* >= 1 */
    const double *alpha;         /* [n_sky] right ascension, rad */
    const double *delta;         /* [n_sky] declination, rad */
    int64_t n_spin;              /* >= 1 */
    const double *fdot;          /* [n_spin] spindown, Hz/s */
    double thr_2F;               /* register a candidate when 2F > thr_2F */
    int64_t bin_lo, bin_hi;      /* searched bins, inclusive; 0,0 = [1, n_fft/2 - 1]
                                    per band; else 0 <= lo <= hi < n_fft of every band */
    double lat;                  /* detector latitude, rad */
    double gamma;                /* arm-bisector orientation, counter-clockwise from
                                    local East, rad */
    int upsample;                /* U of the FFT upsample, 1..8 (2 recommended) */
    int statistic;               /* FSTAT_F_SIMPLE (0) or FSTAT_F_FULL (1), see below */
    double sigma2;               /* noise variance; <= 0: (1/N) sum x^2 per band */
    fstat_form form;
    int interpolation;           /* FSTAT_INTERP_ZEROPAD (0) or FSTAT_INTERP_INTERBIN (1) */
    int64_t cand_capacity;       /* device candidate records kept per search, >= 1 */
    void *cuda_stream;           /* cudaStream_t to run on, or NULL (the plan's own) */
    int inputs_on_device;        /* 0: x/x32/r/alpha/delta/fdot are host pointers;
                                    1: they are device pointers (copied device->device) */
} fstat_plan_desc;

/* One registered candidate (Sect. 2: sky position, frequency, spindown, F),
   plus the integer grid indices that identify it exactly. */
typedef struct {
    double alpha, delta;   /* sky position, rad */
    double freq;           /* f_off + bin / (n_fft dt), Hz */
    double fdot;           /* Hz/s */
    double F;              /* the F-statistic (not 2F) */
    int32_t band;
    int32_t reserved;
    int64_t sky, spin, bin;
} fstat_candidate;

typedef struct {
    int64_t n_cells;         /* n_bands * n_sky * n_spin */
    int64_t f_evals;         /* cells x searched bins, summed over bands */
    int64_t device_bytes;    /* device memory the plan holds */
    int64_t kernel_launches; /* kernels launched by the plan so far (graph nodes count) */
    int64_t n_fft_max;
} fstat_plan_info;

typedef struct fstat_plan fstat_plan;

/* Validate the description, allocate device memory, copy the inputs and prepare
   the launch configuration.  On success *out receives a plan; on failure *out is
   NULL and nothing is leaked.  Errors: FSTAT_ERR_ARG (any field out of range,
   NULL where a pointer is required, x and x32 both or neither given, more than
   2^32 - 1 cells), FSTAT_ERR_OOM, FSTAT_ERR_CUDA. */
fstat_status fstat_plan_create(fstat_plan **out, const fstat_plan_desc *desc);

/* Replace the data of band `band` (0-based) by the next segment of the same
   shape (Sect. 2: the search runs over many frames of one band): n, dt and n_fft
   must equal the plan's band; x or x32, r, f_off, phi0 and eps are taken.  The
   arrays are read from host or device memory as desc->inputs_on_device said and
   are copied before the call returns; the next fstat_search recomputes the
   noise variance and the upsample from them.  Device memory is reused: a
   stream of segments pays the allocation of fstat_plan_create once.  Earlier
   candidates stay readable until the next search.  Errors: FSTAT_ERR_ARG (band
   out of range, another shape, non-finite f_off or phi0, not exactly one of
   x, x32, r NULL), FSTAT_ERR_OOM (the float32 staging buffer), FSTAT_ERR_CUDA,
   FSTAT_ERR_STATE (poisoned plan). */
fstat_status fstat_plan_set_band(fstat_plan *plan, int band, const fstat_band *data);

/* Search cells [cell_begin, cell_end) in the order cell = (band * n_sky + sky)
   * n_spin + spin (cell_end = -1: to the last cell), replacing the candidates of
   the previous call.  Runs the whole hot path from the raw series: per band the
   noise variance and the FFT upsample; per sky the delay, a(t), b(t), the
   resampled and phase-demodulated series and S_aa, S_bb; per cell the spindown
   demodulation, the two zero-padded FFTs, F per bin, the threshold and the
   compaction of candidates into device memory.  Returns FSTAT_ERR_OVERFLOW when
   more than cand_capacity candidates were found (the first cand_capacity found
   are kept; the total stays exact). */
fstat_status fstat_search(fstat_plan *plan, int64_t cell_begin, int64_t cell_end);

/* Copy the candidates of the last search into buf[0 .. cap), sorted by
   (band, sky, spin, bin).  *n_written = min(kept, cap); *n_total = every
   candidate found, including those beyond the device capacity.  Returns
   FSTAT_ERR_OVERFLOW when *n_total > *n_written.  buf may be NULL when cap = 0.
   More than 65 536 records are sorted on the device (once per search, in a
   second device buffer the plan allocates on first use: FSTAT_ERR_OOM if it
   cannot) and read back through pinned host staging that the plan keeps. */
fstat_status fstat_candidates_get(fstat_plan *plan, fstat_candidate *buf, int64_t cap,
                                  int64_t *n_written, int64_t *n_total);

/* Diagnostics of the per-sky stage (geometry, resampling, phase demodulation)
   for one (band, sky) of the plan's inputs, as the search computes it: y[2n]
   interleaved complex resampled series, a[n], b[n], mask[n] (1 inside the
   resampled window), S[3] = {S_aa, S_bb, S_ab}.  Host pointers; any may be NULL.
   FP32_BATCHED plans report their FP32 values widened to double. */
fstat_status fstat_debug_sky(fstat_plan *plan, int band, int64_t sky, double *y, double *a,
                             double *b, uint8_t *mask, double *S);

fstat_status fstat_plan_get_info(const fstat_plan *plan, fstat_plan_info *info);

/* Per-kernel timing, measured with CUDA events on the plan's stream while it
   searches.  With sample_every = k > 0, every k-th launch of each timed kernel
   class is bracketed by events (the others run untouched), so the averages
   describe the launches of a normal search; k = 0 switches timing off.
   fstat_plan_kernel_stats fills up to cap entries (one per kernel class seen
   since timing was switched on) and returns their number in *n. */
typedef struct {
    char name[32];
    int64_t launches;        /* launches of this class since timing was switched on */
    int64_t timed_launches;  /* of which bracketed by events */
    double timed_ms;         /* summed duration of the timed launches */
    double flops_per_launch; /* algorithmic FP32/FP64 operations of one launch (mean) */
    double bytes_per_launch; /* algorithmic DRAM bytes of one launch (mean) */
} fstat_kernel_stat;

fstat_status fstat_plan_set_timing(fstat_plan *plan, int sample_every);
fstat_status fstat_plan_kernel_stats(const fstat_plan *plan, fstat_kernel_stat *out, int cap,
                                     int *n);

/* Launch-shape autotuner of an FSTAT_FP32_BATCHED plan (the paper's farm has no
   counterpart; it picks the GPU-side shapes the search runs with).  It times
   whole searches over the cells [0, sample_cells) (clamped to the grid) with
   CUDA events, changing one choice at a time -- FFT engine (two-stage radix
   32x16 / radix-8 Stockham), pass-2 tile (128 or 256 threads; one or four rows
   per CTA for the paired 512-point rows) and loader (bulk
   copies or per-thread loads with L2 prefetch), cells per launch pair, one fused
   ticket-ordered launch or two launches, and at N_fft = 2^18 the passes in
   paired FP32 instructions (two values per instruction: none, pass 2 only, or
   both passes) -- keeps a change only when it is at
   least 1 % faster, and leaves the plan configured with the best found.  The
   candidates of the tuning searches are discarded (fstat_candidates_get then
   reports none until the next fstat_search).  *chosen (may be NULL) receives the
   configuration and the measured milliseconds per sampled cell.  Results never
   depend on the choice beyond FP32 rounding (every shape computes the same
   transforms).  FSTAT_ERR_ARG for an FP64_PLAIN plan or sample_cells < 1. */
typedef struct {
    int32_t engine;          /* 2: two-stage engine, 1: radix-8 engine; 3: two-stage with
                                pass 2 in paired FP32 instructions at N_fft = 2^18, 4: with
                                both passes paired */
    int32_t pass2_threads;   /* threads per pass-2 CTA: 32 (one row) or 128 for the paired
                                512-point rows, 128 or 256 for the scalar pass 2 */
    int32_t pass2_bulk_copy; /* 1: bulk-copy staging, 0: per-thread loads */
    int32_t fused;           /* 1: one ticket-ordered launch per batch */
    int64_t cells_per_launch;
    double ms_per_cell;      /* of the chosen configuration on the sample */
} fstat_tuning;

fstat_status fstat_plan_autotune(fstat_plan *plan, int64_t sample_cells, fstat_tuning *chosen);

/* The search grid from a lattice generating matrix (Sect. 2: the file grid.bin
   holds a 4 x 4 matrix M whose rows span the 4-D parameter space; the integer
   multiples of the rows are the grid points; a sky position is a pair of
   integers (n, m), a spindown an integer s).  The coordinates of the space are a
   reading (the paper defers them to a reference not available here), row by row
   of M: frequency f dt (the FFT's own grid), spindown fdot dt^2 / 2, and the
   ecliptic-plane components (beta1, beta2) of the unit vector towards the source
   times f_ref tau_E (tau_E = 1 AU / c = 499.00478 s): the sky point (n, m) is
   n M[2] + m M[3], it lies on the sphere when beta1^2 + beta2^2 <= 1 (< 1 in the
   south hemisphere, so points on the ecliptic appear once), and its ecliptic
   latitude has the hemisphere's sign; spindown s is fdot = 2 s M[1][1] / dt^2.
   The grid is the product of the sky points and the spindowns, so M must have
   M[1][2] = M[1][3] = M[2][1] = M[3][1] = 0 (FSTAT_ERR_ARG otherwise). */
typedef struct {
    double M[16];               /* row-major; rows: frequency, spindown, sky n, sky m */
    double dt;                  /* sampling interval, s (> 0) */
    double f_ref;               /* reference frequency of the sky coordinates, Hz (> 0) */
    double eps;                 /* obliquity of the ecliptic, rad */
    int64_t s_lo, s_hi;         /* spindown integers, inclusive */
    int64_t n_lo, n_hi;         /* sky integers, inclusive (at most 2^20 values each) */
    int64_t m_lo, m_hi;
    int32_t hemispheres;        /* 1: north ecliptic hemisphere; 2: north, then south */
    int32_t reserved_;
} fstat_lattice;

/* Fills device arrays with the grid of a lattice, ordered by hemisphere, then n,
   then m (sky) and by s (spindown):
     alpha, delta  device pointers, cap_sky doubles each (rad, alpha in [0, 2 pi));
     nm            device pointer to 3 cap_sky int64 (hemisphere 0/1, n, m), or NULL;
     fdot          device pointer, cap_spin doubles (Hz/s).
   *n_sky and *n_spin (host) receive the full counts; cap_sky = cap_spin = 0 is a
   count-only query (the array pointers may then be NULL).  The arrays are ready to
   pass to fstat_plan_create with inputs_on_device = 1.  Synchronous with respect
   to the host; allocates and frees a small device buffer of per-block counts.
   Errors: FSTAT_ERR_ARG (NULL pointer where one is needed, non-finite entry,
   ranges empty or too large, coupled spindown and sky rows), FSTAT_ERR_OOM,
   FSTAT_ERR_CUDA, FSTAT_ERR_OVERFLOW (a count exceeds its capacity: the first
   cap entries are written, the counts stay exact). */
fstat_status fstat_lattice_grid(const fstat_lattice *lattice, double *alpha, double *delta,
                                int64_t *nm, int64_t cap_sky, int64_t *n_sky, double *fdot,
                                int64_t cap_spin, int64_t *n_spin, void *cuda_stream);

/* Allocation-free F of one cell (the paper has no counterpart: this entry point
   exists for callers that cannot allocate device memory -- for example a host
   application that reserves the whole device memory budget up front and hands
   libraries only views of it, or code that must not pay for an allocation while it
   runs).  It evaluates, without any cudaMalloc, the FP32 zero-padded transforms and
   F = |F_a|^2 norm_a + |F_b|^2 norm_b for every bin in [bin_lo, bin_hi] of one
   (sky, spindown) cell, from the resampled, phase-demodulated series of that sky:
     w      device pointer, 16-byte aligned, w[4 k .. 4 k + 3] = (Re y_k a_k,
            Im y_k a_k, Re y_k b_k, Im y_k b_k), k < n (the FP32 form's per-sky
            series; zero outside the resampled window);
     n_fft  power of two, 2^12 <= n_fft <= 2^18 (the maximum), n_fft >= 2 n;
     chirp_rate  fdot dt^2 / 2 (cycles per sample^2), |chirp_rate| < 1/4;
     norm_a, norm_b  1/(sigma^2 S_aa), 1/(sigma^2 S_bb), >= 0;
     F_out  device pointer to bin_hi - bin_lo + 1 floats, 4-byte aligned;
     cuda_stream  cudaStream_t or NULL.
   The transforms' intermediate lives in a file-scope device array of
   2 x 2^18 complex floats (4 MiB) and twiddle tables in another (about 20 KiB);
   every GPU that loads the library holds them until the process exits.  On its
   first call on a device (and on the first call for each transform length) the
   entry point resolves the arrays' device addresses and fills the twiddle table
   with a short kernel followed by a device synchronisation, so make that first
   call before any stream capture.  Every call shares the arrays and nothing in
   them has to start at zero (each call writes the whole intermediate it reads);
   calls that overlap on the GPU (other streams, other host threads) race on them.
   Every call ends by synchronising cuda_stream with the host, so no call may be
   made while a stream capture is active on cuda_stream.  The addresses and
   the filled-table flags are cached per device for the life of the process: after
   a cudaDeviceReset of a device the cache is stale, and this entry point must not
   be called on that device again.  Returns FSTAT_ERR_ARG for a NULL or misaligned
   pointer, a length beyond the maximum or any other invalid argument (nothing is
   launched), FSTAT_ERR_CUDA if a CUDA call fails. */
fstat_status fstat_cell_F_noalloc(const float *w, int64_t n, int64_t n_fft, double chirp_rate,
                                  double norm_a, double norm_b, int64_t bin_lo, int64_t bin_hi,
                                  float *F_out, void *cuda_stream);

/* Roofline denominators measured on the current device (not part of the
   method; the search path is bounded by its FFT FLOP on the CUDA cores and by
   its inter-pass scratch bytes).  fstat_measure_fp32_fma: the FP32 rate of
   independent FFMA chains in every lane (8 CTAs of 256 threads per SM), in
   TFLOP/s at 2 FLOP per FMA.  fstat_measure_l2_copy: the read + write bandwidth,
   in GB/s, of a copy of bytes/2 to another bytes/2 repeated through L2 only
   (ld/st.global.cg), so that a working set smaller than L2 is served from it.
   Each runs once untimed and once timed with CUDA events on cuda_stream (NULL:
   the legacy default stream), a few milliseconds; device memory is allocated
   and freed inside.  Errors: FSTAT_ERR_ARG (NULL output, bytes < 1 MiB),
   FSTAT_ERR_OOM, FSTAT_ERR_CUDA. */
fstat_status fstat_measure_fp32_fma(double *tflops, void *cuda_stream);
fstat_status fstat_measure_l2_copy(int64_t bytes, double *gbs, void *cuda_stream);

/* Release everything the plan holds.  NULL is accepted. */
void fstat_plan_destroy(fstat_plan *plan);

/* Static description of a status code. */
const char *fstat_status_string(fstat_status s);

/* Last error message of this plan ("" when none); valid until the next call. */
const char *fstat_plan_error(const fstat_plan *plan);

#ifdef __cplusplus
}
#endif
#endif
