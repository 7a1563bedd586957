// Internal declarations shared by the host orchestration (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fstat.h"

namespace fstat {

constexpr int kMinLogN = 8;    // n_fft >= 256
// Fused FP32 launch: scratch slots in its ring, and how many cells pass 2 trails
// pass 1 by (defaults).
constexpr int kFusedSlots = 16;
constexpr int kFusedAhead = 6;
constexpr int kMaxLogN = 20;   // n_fft <= 2^20

// Split of a power-of-two transform length N = N1 * N2 into the two passes of
// the four-step FFT: pass 1 transforms the N1 strided columns (length N2), pass
// 2 the N2 rows (length N1).
inline int log_n1(int logn) { return logn / 2; }
inline int log_n2(int logn) { return logn - logn / 2; }

// Twiddle tables of one transform length, forward direction e^{-2 pi i k / M}.
struct TwiddleSet {
    int logn = 0;
    // device pointers, interleaved (re, im); float and double copies
    const double *in1_d = nullptr, *in2_d = nullptr, *lo_d = nullptr, *hi_d = nullptr;
    const float *in1_f = nullptr, *in2_f = nullptr, *lo_f = nullptr, *hi_f = nullptr;
    // second engine: stage-1 twiddles W_M^{r j} laid out [r][j], r < R1, j < R0
    // (float), for the rows (M = N1 = R0 R1, pass 2) and the columns (M = N2, pass 1)
    const float *s1_f = nullptr, *s2_f = nullptr;
    // packed passes (512-point rows, N_fft = 2^18 and 2^19): stage-1 twiddles of a
    // 512-point pass as pairs,
    // [r][k] = (cos a_2k, cos a_2k+1, -sin a_2k, -sin a_2k+1), a_j = 2 pi r j / 512
    const float4 *p512_f = nullptr;
};

// Per-sky normaliser record: na, nb, nab, 0 in FP64 (doubles 0..3), then the
// same four as floats (doubles 4..5), padded to 8 doubles.
constexpr int kNormStride = 8;

// Device record of one candidate: global cell index, bin and F.
struct CandRecord {
    uint32_t cell;
    uint32_t bin;
    double F;
};

// Per-sky constants computed once per plan: unit vector and the coefficients of
// a(h) = A0 cos2h + A1 sin2h + A2 cosh + A3 sinh + A4 and
//       b(h) = B0 cos2h + B1 sin2h + B2 cosh + B3 sinh, h = alpha - LST.
struct SkyConst {
    double nx, ny, nz, alpha;
    double A[5];
    double B[4];
    float nf[6];   // nx, ny, nz as double-float pairs (hi, lo) for the FP32 delay
};

// Band data resident on the device.
struct BandDev {
    int64_t n = 0;
    double dt = 0, f_off = 0, phi0 = 0, eps = 0;
    int64_t n_fft = 0;
    int logn = 0;
    int64_t lo = 0, hi = 0;
    double *x = nullptr;      // [n] float64 (converted from float32 when needed)
    float *x32 = nullptr;     // [n] staging of a float32 series (allocated on first use)
    double *r = nullptr;      // [3n]
    void *r2 = nullptr;       // FP32 form: r as double-float pairs (DF[3n]), redone per search
    double *sigma2 = nullptr; // device scalar
    void *xu = nullptr;       // [U n]: double (FP64 form) or float (FP32 form)
};

struct Plan {
    fstat_plan_desc desc{};
    std::vector<BandDev> bands;
    std::vector<fstat_band> host_bands;
    int64_t n_cells = 0, f_evals = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool poisoned = false;
    std::string err;
    int64_t launches = 0;
    int64_t device_bytes = 0;
    std::vector<void *> allocs;

    // grids (device, and host copies for candidate retrieval)
    double *alpha = nullptr, *delta = nullptr, *fdot = nullptr;
    std::vector<double> h_alpha, h_delta, h_fdot;
    int64_t n_fft_max = 0;
    SkyConst *sky = nullptr;
    uint64_t *chirp_fx = nullptr;  // per (band, spin): frac(fdot dt^2 / 2) in 2^-64 cycles
    double *chirp_d = nullptr;     // per (band, spin): fdot dt^2 / 2 (FP64 form)

    // per sky batch (w and norm double-buffered by sky-batch parity so that the
    // geometry of the next sky batch can overlap the transforms of this one)
    int64_t sky_batch = 0;
    void *wbuf[2] = {nullptr, nullptr};   // FP32: float4 [sky_batch][w_stride]; FP64: {y a, y b} double2 pairs
    double *dbuf = nullptr;       // [sky_batch][n_max] per-sample delays
    double *partials = nullptr;   // [sky_batch][n_blocks_max][3]
    double *S = nullptr;          // [sky_batch][3]
    double *normbuf[2] = {nullptr, nullptr};   // [sky_batch][2]: 1/(sigma^2 S_aa), 1/(sigma^2 S_bb)
    int64_t n_max = 0;

    // FFT scratch (cell slots)
    int64_t cell_batch = 0;
    void *scratch = nullptr;
    int64_t w_stride = 0;          // per-sky stride of w, >= every band's n rounded up to N1

    // persistent FP32 search: cells per batch, scratch ring slots, queue counters
    int64_t pbatch = 2, pslots = 8;
    uint32_t *queue = nullptr;     // [head | done1[nb] | done2[nb]]
    uint32_t *qerr = nullptr;      // error word (bit 0: a bounded wait ran out)
    int64_t withhold_item = -1;    // test hook (FSTAT_TEST_WITHHOLD_ITEM): the persistent kernel's queue
                                   // item, or the cell whose pass 1 never reports in the fused launch
    bool use_persistent = false;   // FSTAT_PERSISTENT=1: one queue-fed launch per sky batch
    // worker streams of the batched FP32 passes, each with its own scratch slot
    int n_workers = 1;
    std::vector<cudaStream_t> workers, own_workers;
    cudaEvent_t ev_geo[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_done[2];
    std::vector<cudaEvent_t> ev_join;
    int elems_per_thread = 16;     // FP32 batched passes: 16 or 8 complex elements per thread
    int engine = 2;                // FP32 batched passes, 2^12 .. 2^19: 2 = two-stage engine, 1 = radix-8 engine
    bool fused = false;            // two-stage engine: both passes in one ticket-ordered launch
    bool interbin = false;         // FSTAT_INTERP_INTERBIN: half-length transforms + interbinning
    uint32_t *fctl = nullptr;      // per worker: 1 + 2 * cell_batch counters of the fused launch
    size_t slot_cells = 0;         // cells of scratch per worker (>= cell_batch, >= the fused ring)
    int fused_slots = kFusedSlots, fused_ahead = kFusedAhead;
    int packed = 1;                // N_fft = 2^18 in paired FP32 arithmetic (passes3.cuh): 0 neither
                                   // pass, 1 pass 2, 2 both passes, 3 pass 2 and the second
                                   // stage of pass 1
    int fused_tpi = 1;             // tiles per ticket of the fused launch (power of two)
    int64_t fused_batch = 1;       // cells per fused launch (a sky batch)
    int64_t pf_dist = 0;           // two-stage pass 2: L2 prefetch distance in CTAs (0: off)
    int64_t pf_dist_pk = 0;        // the same for the paired pass 2 (measured best off)
    bool share_chirp = true;       // pass 1: spindown phase shared by the lanes of a column
    int p2_ts = 32;                // paired pass 2: CTA size (32, 64 or 128: one warp per row)
    bool p2_rows = true;           // 256-point rows (2^16, 2^17): two rows per warp, packed
    bool tma = true;               // two-stage pass 2: rows staged by bulk copies
    int p2_threads = 128;          // two-stage pass 2 with bulk copies: CTA size 256 or 128

    // Bluestein / generic-FFT work buffers (double2)
    double *bw = nullptr;
    int64_t bw_elems = 0;

    // twiddles, one set per transform length used
    std::vector<TwiddleSet> tw;
    void *tw_pool = nullptr;

    // candidates
    CandRecord *cand = nullptr;
    unsigned long long *cand_count = nullptr;
    int64_t cand_capacity = 0;
    // pinned host staging of the candidate records (read back and sorted there),
    // grown on demand and reused by later calls
    CandRecord *h_rec = nullptr;           // pinned staging of the read-back
    std::vector<CandRecord> h_tmp;         // work array of the host sort (few records)
    int64_t h_rec_cap = 0;
    // device sort of the records before the read-back: the other ping-pong buffer,
    // the digit counts, the cell range of the records and the sorted buffer (null
    // until the first read-back after a search)
    CandRecord *cand_tmp = nullptr;
    uint32_t *sort_hist = nullptr;
    int64_t sort_cap = 0;
    int64_t cand_begin = 0, cand_end = 0;
    const CandRecord *cand_sorted = nullptr;
    int64_t last_total = 0;
    bool searched = false;

    // sampled per-kernel timing (fstat_plan_set_timing)
    struct KStat {
        std::string name;
        int64_t launches = 0, timed = 0;
        double ms = 0.0, flops = 0.0, bytes = 0.0;
    };
    struct Pending {
        int stat;
        cudaEvent_t a, b;
    };
    int timing_every = 0;
    int64_t timing_tick = 0;
    std::vector<KStat> kstats;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool, ev_all;

    // CUDA graph of the last search's launch sequence, replayed while the cell
    // range and the timing rate stay the same; with it the host-side counters
    // and the timing events its replay produces
    bool use_graph = true;
    int64_t prev_begin = -1, prev_end = -1;
    int prev_timing = -1;
    struct GraphRun {
        cudaGraphExec_t exec = nullptr;
        int64_t begin = -1, end = -1;
        int timing_every = 0;
        int64_t launches = 0;                    // kernels per replay
        std::vector<KStat> dk;                   // counter increments per replay
        std::vector<Pending> pending;            // events recorded by the graph (owned by it)
    } graph;

    const TwiddleSet *twiddles(int logn) const {
        for (auto &t : tw)
            if (t.logn == logn) return &t;
        return nullptr;
    }
};

// Buffers one launch pair works on.
struct CellBufs {
    const void *w;
    const double *norm;
    void *scratch;
    uint32_t *ctl = nullptr;   // fused launch: ticket + per-cell counters (1 + 2 * cell_batch), zeroed
};

// ---------------------------------------------------------------- launchers
// Each returns the number of kernels it launched (for the plan's counter).

// sigma^2 = (1/n) sum x^2, compensated, into *out (device); user_sigma2 > 0 overrides.
// partials: >= 256 doubles.
// FP32 form, per band and search: the ephemeris as double-float pairs (b.r2).
int launch_split_r(const BandDev &b, cudaStream_t s);
int launch_sigma2(const double *x, int64_t n, double user_sigma2, double *partials, double *out,
                  cudaStream_t s);

// Generic two-pass power-of-two FFT of `pairs` * 2 transforms of length 2^logn,
// in[t] -> out[t] (t over 2*pairs contiguous transforms, interleaved complex).
// dir = -1 forward, +1 inverse (unscaled).  FP64 or FP32 arithmetic.
int launch_fft_generic(const TwiddleSet &tw, bool fp64, int dir, const void *in, void *out,
                       int64_t n_transforms, void *scratch, cudaStream_t s);

// Bluestein DFT of arbitrary length n (double2 in/out), using the generic FFT of
// length M = 2^logm >= 2n - 1.  work holds 3*M double2.
int launch_bluestein(const TwiddleSet &twm, int dir, const double *in, double *out, int64_t n,
                     double *work, void *scratch, cudaStream_t s);

// U-fold FFT upsample of x[n] (double) into xu[U n] (double or float).
int launch_upsample(const Plan &p, const BandDev &b, int U, void *xu, bool xu_fp32,
                    cudaStream_t s);

// Geometry + resampling + phase demodulation for skies [s0, s0+ns) of band b.
// FP32 form writes w as float4 (y a, y b); FP64 form writes double2 wa, wb.
// Optional diagnostics (nullptr to skip): y (double2), a, b (double), mask (uint8).
int launch_geometry(const Plan &p, const BandDev &b, int64_t s0, int64_t ns, bool fp32,
                    void *w, double *dbg_y, double *dbg_a, double *dbg_b, uint8_t *dbg_mask,
                    cudaStream_t s);

// Per-sky S sums and normalisations for the ns skies of the last geometry launch.
int launch_reduce_norms(const Plan &p, const BandDev &b, int64_t ns, double *norm, cudaStream_t s);
// Stable device sort of n candidate records by (cell - cell0, bin), bins < 2^bin_bits,
// cells in [cell0, cell0 + cell_span); a and b ping-pong, hist holds 256 (ceil(n / 4096) + 1)
// counts; returns the buffer with the sorted records.
CandRecord *launch_cand_sort(CandRecord *a, CandRecord *b, uint32_t *hist, int64_t n, uint32_t cell0,
                             uint64_t cell_span, int bin_bits, cudaStream_t s, int64_t *launches);

// The two FFT passes of the search for cells [c0, c0 + nc) of band `band_idx`
// (cells of this band: c = sky * n_spin + spin, skies relative to sky base s0).
// Persistent FP32 search of band-local cells [c_lo, c_hi) of one sky batch
// (skies from s0): both passes in one launch fed by a device work queue.
bool persistent_supported(int logn);
int persistent_tiles_per_cell(int logn);
int launch_search_persistent(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                             int64_t c_lo, int64_t c_hi, cudaStream_t s, const CellBufs &cb);

// Records a timing event on s, as an external event node while s is being
// captured into a graph (so that the event stays readable after replays).
inline cudaError_t record_timing_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t r = cudaStreamIsCapturing(s, &cs);
    if (r != cudaSuccess) return r;
    return cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                               : cudaEventRecordDefault);
}
// Whether a band of transform length 2^logn (the n_fft bin grid) can run in the
// interbinning form (a half-length transform of 2^12 .. 2^19).
bool interbin_supported(int logn);
// Whether the FP32 cells of a band of length 2^logn run as one fused launch.
bool fused_supported(const Plan &p, int logn);
// `mid` (may be null) is recorded between the two passes.
int launch_search_cells_f32(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                            int64_t c0, int64_t nc, cudaStream_t s, cudaEvent_t mid,
                            const CellBufs &cb);
int launch_search_cells_f64(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                            int64_t c0, int64_t nc, cudaStream_t s, cudaEvent_t mid,
                            const CellBufs &cb);

}  // namespace fstat
