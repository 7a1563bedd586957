// Host side of libfstat.so: argument validation, device memory, the order of
// launches of one search, candidate retrieval.  See include/fstat.h.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "fft_engine2.cuh"
#include "fstat_internal.h"

struct fstat_plan : public fstat::Plan {};

namespace fstat {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

struct CudaError {
    cudaError_t e;
    const char *what;
};

// Test hook: FSTAT_TEST_FAIL_ALLOC=k makes the k-th device allocation of a plan
// (1-based) report failure, to exercise the out-of-memory path on the host.
int alloc_fail_at() {
    const char *v = getenv("FSTAT_TEST_FAIL_ALLOC");
    return v ? atoi(v) : 0;
}

void check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw CudaError{e, what};
}

struct OomError {};
struct TimeoutError {};

template <typename T>
T *dalloc(Plan &p, size_t count, int &n_alloc) {
    ++n_alloc;
    const int fail = alloc_fail_at();
    if (fail > 0 && n_alloc == fail) throw OomError{};
    void *ptr = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw OomError{};
    }
    check(e, "cudaMalloc");
    p.allocs.push_back(ptr);
    p.device_bytes += (int64_t)bytes;
    return reinterpret_cast<T *>(ptr);
}

int ilog2_exact(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return ((int64_t(1) << l) == v) ? l : -1;
}

bool is_finite(double v) { return isfinite(v) != 0; }

// Fixed-point 2^-64 cycles of frac(rate): exact wrap-around arithmetic on device.
uint64_t to_fixed64(double rate) {
    if (fabs(rate) < 0.25)                   // the usual case: keep the rate's full precision
        return (uint64_t)(int64_t)llround(ldexp(rate, 64));
    double fr = rate - floor(rate);          // [0, 1)
    double hi = floor(fr * 4294967296.0);    // top 32 bits
    double lo = (fr * 4294967296.0 - hi) * 4294967296.0;
    uint64_t h = (uint64_t)hi, l = (uint64_t)llround(lo);
    return (h << 32) + l;                    // l may round to 2^32: carries into h
}

// Unit vector towards (alpha, delta) and the coefficients of the amplitude
// modulations a(h), b(h) of a right-angle interferometer (Jaranowski, Krolak &
// Schutz 1998) in cos 2h, sin 2h, cos h, sin h (h = alpha - local sidereal time),
// evaluated on the host in FP64.
SkyConst sky_const(double al, double de, double lat, double gamma) {
    const double sd = sin(de), cd = cos(de);
    const double s2g = sin(2.0 * gamma), c2g = cos(2.0 * gamma);
    const double sl = sin(lat), cl = cos(lat), s2l = sin(2.0 * lat), c2l = cos(2.0 * lat);
    const double s2d = sin(2.0 * de), c2d = cos(2.0 * de);
    SkyConst c;
    c.nx = cd * cos(al);
    c.ny = cd * sin(al);
    c.nz = sd;
    c.alpha = al;
    const double nv[3] = {c.nx, c.ny, c.nz};
    for (int i = 0; i < 3; ++i) {
        const DF d = df_from_double(nv[i]);
        c.nf[2 * i] = d.hi;
        c.nf[2 * i + 1] = d.lo;
    }
    c.A[0] = (1.0 / 16.0) * s2g * (3.0 - c2l) * (3.0 - c2d);   // cos 2h
    c.A[1] = -0.25 * c2g * sl * (3.0 - c2d);                   // sin 2h
    c.A[2] = 0.25 * s2g * s2l * s2d;                           // cos h
    c.A[3] = -0.5 * c2g * cl * s2d;                            // sin h
    c.A[4] = 0.75 * s2g * cl * cl * cd * cd;                   // constant
    c.B[0] = c2g * sl * sd;                                    // cos 2h
    c.B[1] = 0.25 * s2g * (3.0 - c2l) * sd;                    // sin 2h
    c.B[2] = c2g * cl * cd;                                    // cos h
    c.B[3] = 0.5 * s2g * s2l * cd;                             // sin h
    return c;
}

std::string band_err(int i, const char *m) { return "band " + std::to_string(i) + ": " + m; }

fstat_status validate(const fstat_plan_desc *d, std::string &err) {
    if (!d) { err = "desc is NULL"; return FSTAT_ERR_ARG; }
    if (d->n_bands < 1 || !d->bands) { err = "need n_bands >= 1 and bands"; return FSTAT_ERR_ARG; }
    if (d->n_sky < 1 || !d->alpha || !d->delta) { err = "need n_sky >= 1, alpha, delta"; return FSTAT_ERR_ARG; }
    if (d->n_spin < 1 || !d->fdot) { err = "need n_spin >= 1 and fdot"; return FSTAT_ERR_ARG; }
    if (d->form != FSTAT_FP64_PLAIN && d->form != FSTAT_FP32_BATCHED) { err = "unknown form"; return FSTAT_ERR_ARG; }
    if (d->statistic != FSTAT_F_SIMPLE && d->statistic != FSTAT_F_FULL) { err = "unknown statistic"; return FSTAT_ERR_ARG; }
    if (d->interpolation != FSTAT_INTERP_ZEROPAD && d->interpolation != FSTAT_INTERP_INTERBIN) {
        err = "unknown interpolation"; return FSTAT_ERR_ARG;
    }
    if (d->interpolation == FSTAT_INTERP_INTERBIN && d->form != FSTAT_FP32_BATCHED) {
        err = "interbinning needs the FP32 batched form"; return FSTAT_ERR_ARG;
    }
    if (d->upsample < 1 || d->upsample > 8) { err = "upsample must be 1..8"; return FSTAT_ERR_ARG; }
    if (d->cand_capacity < 1 || d->cand_capacity > (int64_t(1) << 34)) { err = "cand_capacity out of range"; return FSTAT_ERR_ARG; }
    if (!is_finite(d->thr_2F) || !is_finite(d->lat) || !is_finite(d->gamma) || !is_finite(d->sigma2)) {
        err = "non-finite scalar"; return FSTAT_ERR_ARG;
    }
    if (d->inputs_on_device != 0 && d->inputs_on_device != 1) { err = "inputs_on_device must be 0 or 1"; return FSTAT_ERR_ARG; }
    const int64_t cells = (int64_t)d->n_bands * d->n_sky * d->n_spin;
    if (d->n_sky > (int64_t(1) << 31) || d->n_spin > (int64_t(1) << 31) || cells >= (int64_t(1) << 32)) {
        err = "more than 2^32 - 1 cells"; return FSTAT_ERR_ARG;
    }
    for (int i = 0; i < d->n_bands; ++i) {
        const fstat_band &b = d->bands[i];
        if (b.n < 16 || b.n > (int64_t(1) << 19)) { err = band_err(i, "n must be 16 .. 2^19"); return FSTAT_ERR_ARG; }
        if (!(b.dt > 0) || !is_finite(b.dt) || !is_finite(b.f_off) || !is_finite(b.phi0)) { err = band_err(i, "bad dt/f_off/phi0"); return FSTAT_ERR_ARG; }
        if ((b.x == nullptr) == (b.x32 == nullptr)) { err = band_err(i, "give exactly one of x, x32"); return FSTAT_ERR_ARG; }
        if (!b.r) { err = band_err(i, "r is NULL"); return FSTAT_ERR_ARG; }
        int64_t nf = b.n_fft;
        if (nf == 0) { nf = 1; while (nf < 2 * b.n) nf <<= 1; }
        const int lg = ilog2_exact(nf);
        if (lg < kMinLogN || lg > kMaxLogN || nf < 2 * b.n) { err = band_err(i, "n_fft must be a power of two >= 2n in [256, 2^20]"); return FSTAT_ERR_ARG; }
        if (d->interpolation == FSTAT_INTERP_INTERBIN && !interbin_supported(lg)) {
            err = band_err(i, "interbinning needs n_fft in [2^13, 2^20]"); return FSTAT_ERR_ARG;
        }
        if (d->bin_lo != 0 || d->bin_hi != 0) {
            if (d->bin_lo < 0 || d->bin_hi < d->bin_lo || d->bin_hi >= nf) { err = band_err(i, "bin range outside [0, n_fft)"); return FSTAT_ERR_ARG; }
        }
    }
    return FSTAT_OK;
}

void host_twiddles(int logn, std::vector<double> &in1, std::vector<double> &in2,
                   std::vector<double> &lo, std::vector<double> &hi) {
    const int64_t N = int64_t(1) << logn;
    const int64_t N1 = int64_t(1) << log_n1(logn), N2 = int64_t(1) << log_n2(logn);
    auto w = [](int64_t k, int64_t M, double *o) {
        // e^{-2 pi i k / M} with k reduced to the first octant-free form
        const double a = -kTwoPi * (double)k / (double)M;
        o[0] = cos(a);
        o[1] = sin(a);
    };
    in1.resize(2 * N1); in2.resize(2 * N2); lo.resize(2 * N1); hi.resize(2 * N2);
    for (int64_t k = 0; k < N1; ++k) w(k, N1, &in1[2 * k]);
    for (int64_t k = 0; k < N2; ++k) w(k, N2, &in2[2 * k]);
    for (int64_t k = 0; k < N1; ++k) w(k, N, &lo[2 * k]);
    for (int64_t k = 0; k < N2; ++k) w(k * N1, N, &hi[2 * k]);
}

// Stage-1 twiddles of the second engine: W_M^{r j}, [r][j], for a pass length M
// (N1 of the rows, N2 of the columns) split as R0 R1 by the engine's plan.
void stage1_twiddles(int logm, std::vector<double> &o) {
    const int64_t M = int64_t(1) << logm;
    const int64_t R0 = eng2::radix0((int)M), R1 = eng2::radix1((int)M);
    o.assign((size_t)(2 * R0 * R1), 0.0);
    for (int64_t r = 0; r < R1; ++r)
        for (int64_t j = 0; j < R0; ++j) {
            const double a = -kTwoPi * (double)((r * j) % M) / (double)M;
            o[(size_t)(2 * (r * R0 + j))] = cos(a);
            o[(size_t)(2 * (r * R0 + j) + 1)] = sin(a);
        }
}

// Stage-1 twiddles of a 512-point pass (radix 32 then 16) as packed pairs of
// jobs (2k, 2k + 1): [r][k] = (cos a_2k, cos a_2k+1, -sin a_2k, -sin a_2k+1),
// a_j = 2 pi (r j mod 512) / 512, r < 16, k < 16.
void packed512_twiddles(std::vector<double> &o) {
    o.assign(16 * 16 * 4, 0.0);
    for (int r = 0; r < 16; ++r)
        for (int k = 0; k < 16; ++k)
            for (int e = 0; e < 2; ++e) {
                const double a = kTwoPi * (double)((r * (2 * k + e)) % 512) / 512.0;
                o[(size_t)(4 * (r * 16 + k) + e)] = cos(a);
                o[(size_t)(4 * (r * 16 + k) + 2 + e)] = -sin(a);
            }
}

void build_twiddles(Plan &p, const std::vector<int> &logs, int &n_alloc) {
    std::vector<double> hd;
    std::vector<size_t> offs;
    constexpr int kSets = 7;
    for (int lg : logs) {
        std::vector<double> a, b, c, d, e, f, g;
        host_twiddles(lg, a, b, c, d);
        stage1_twiddles(log_n1(lg), e);
        stage1_twiddles(log_n2(lg), f);
        if (log_n1(lg) == 9) packed512_twiddles(g);   // 512-point rows: N_fft = 2^18, 2^19
        for (auto *v : {&a, &b, &c, &d, &e, &f, &g}) {
            while (hd.size() % 4) hd.push_back(0.0);   // 16-byte aligned float tables
            offs.push_back(hd.size());
            hd.insert(hd.end(), v->begin(), v->end());
        }
    }
    double *dd = dalloc<double>(p, hd.size(), n_alloc);
    float *df = dalloc<float>(p, hd.size(), n_alloc);
    std::vector<float> hf(hd.begin(), hd.end());
    check(cudaMemcpy(dd, hd.data(), hd.size() * sizeof(double), cudaMemcpyHostToDevice), "twiddles");
    check(cudaMemcpy(df, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice), "twiddles");
    for (size_t i = 0; i < logs.size(); ++i) {
        TwiddleSet t;
        const size_t *o = &offs[kSets * i];
        t.logn = logs[i];
        t.in1_d = dd + o[0]; t.in2_d = dd + o[1];
        t.lo_d = dd + o[2]; t.hi_d = dd + o[3];
        t.in1_f = df + o[0]; t.in2_f = df + o[1];
        t.lo_f = df + o[2]; t.hi_f = df + o[3];
        t.s1_f = df + o[4]; t.s2_f = df + o[5];
        if (log_n1(logs[i]) == 9) t.p512_f = reinterpret_cast<const float4 *>(df + o[6]);
        p.tw.push_back(t);
    }
}

__global__ void k_f32_to_f64(const float *__restrict__ in, int64_t n, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

void copy_in(void *dst, const void *src, size_t bytes, bool on_device, cudaStream_t s) {
    check(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
          "input copy");
}

void create_impl(Plan &p, const fstat_plan_desc *d) {
    int n_alloc = 0;
    p.desc = *d;
    const bool dev = d->inputs_on_device == 1;
    const bool fp32 = d->form == FSTAT_FP32_BATCHED;
    p.interbin = d->interpolation == FSTAT_INTERP_INTERBIN;
    if (d->cuda_stream) {
        p.stream = (cudaStream_t)d->cuda_stream;
    } else {
        check(cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking), "cudaStreamCreate");
        p.own_stream = true;
    }
    cudaStream_t s = p.stream;
    const int U = d->upsample;

    // grids (host copies kept for candidate retrieval and the chirp tables)
    p.h_alpha.resize(d->n_sky); p.h_delta.resize(d->n_sky); p.h_fdot.resize(d->n_spin);
    const cudaMemcpyKind k2h = dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    check(cudaMemcpy(p.h_alpha.data(), d->alpha, d->n_sky * sizeof(double), k2h), "alpha");
    check(cudaMemcpy(p.h_delta.data(), d->delta, d->n_sky * sizeof(double), k2h), "delta");
    check(cudaMemcpy(p.h_fdot.data(), d->fdot, d->n_spin * sizeof(double), k2h), "fdot");
    for (int64_t i = 0; i < d->n_sky; ++i)
        if (!is_finite(p.h_alpha[i]) || !is_finite(p.h_delta[i])) throw std::string("non-finite sky position");
    for (int64_t j = 0; j < d->n_spin; ++j)
        if (!is_finite(p.h_fdot[j])) throw std::string("non-finite spindown");

    std::vector<int> logs;
    auto need = [&](int lg) { if (std::find(logs.begin(), logs.end(), lg) == logs.end()) logs.push_back(lg); };
    int64_t max_m = 0, max_nfft = 0;
    p.n_max = 0;
    for (int i = 0; i < d->n_bands; ++i) {
        const fstat_band &hb = d->bands[i];
        BandDev b;
        b.n = hb.n; b.dt = hb.dt; b.f_off = hb.f_off; b.phi0 = hb.phi0; b.eps = hb.eps;
        b.n_fft = hb.n_fft;
        if (b.n_fft == 0) { b.n_fft = 1; while (b.n_fft < 2 * b.n) b.n_fft <<= 1; }
        b.logn = ilog2_exact(b.n_fft);
        need(b.logn);
        if (d->interpolation == FSTAT_INTERP_INTERBIN) need(b.logn - 1);
        if (d->bin_lo == 0 && d->bin_hi == 0) { b.lo = 1; b.hi = b.n_fft / 2 - 1; }
        else { b.lo = d->bin_lo; b.hi = d->bin_hi; }
        // upsample transforms: a power of two >= 256 directly, else Bluestein
        if (U > 1) {
            const int lgn = ilog2_exact(b.n);
            if (lgn >= kMinLogN && lgn <= kMaxLogN) need(lgn);
            else {
                int lm = kMinLogN;
                while ((int64_t(1) << lm) < 2 * b.n - 1) ++lm;
                need(lm);
                max_m = std::max<int64_t>(max_m, int64_t(1) << lm);
            }
        }
        max_nfft = std::max(max_nfft, b.n_fft);
        p.n_max = std::max(p.n_max, b.n);
        b.x = dalloc<double>(p, b.n, n_alloc);
        b.r = dalloc<double>(p, 3 * b.n, n_alloc);
        if (fp32) b.r2 = dalloc<DF>(p, 3 * b.n, n_alloc);
        b.sigma2 = dalloc<double>(p, 1, n_alloc);
        b.xu = fp32 ? (void *)dalloc<float>(p, (size_t)U * b.n, n_alloc)
                    : (void *)dalloc<double>(p, (size_t)U * b.n, n_alloc);
        if (hb.x) {
            copy_in(b.x, hb.x, b.n * sizeof(double), dev, s);
        } else {
            b.x32 = dalloc<float>(p, b.n, n_alloc);
            copy_in(b.x32, hb.x32, b.n * sizeof(float), dev, s);
            k_f32_to_f64<<<(unsigned)((b.n + 255) / 256), 256, 0, s>>>(b.x32, b.n, b.x);
            ++p.launches;
        }
        copy_in(b.r, hb.r, 3 * b.n * sizeof(double), dev, s);
        p.bands.push_back(b);
        p.n_cells += d->n_sky * d->n_spin;
        p.f_evals += d->n_sky * d->n_spin * (b.hi - b.lo + 1);
    }
    p.n_fft_max = max_nfft;
    build_twiddles(p, logs, n_alloc);

    p.alpha = dalloc<double>(p, d->n_sky, n_alloc);
    p.delta = dalloc<double>(p, d->n_sky, n_alloc);
    p.fdot = dalloc<double>(p, d->n_spin, n_alloc);
    check(cudaMemcpyAsync(p.alpha, p.h_alpha.data(), d->n_sky * sizeof(double), cudaMemcpyHostToDevice, s), "alpha");
    check(cudaMemcpyAsync(p.delta, p.h_delta.data(), d->n_sky * sizeof(double), cudaMemcpyHostToDevice, s), "delta");
    check(cudaMemcpyAsync(p.fdot, p.h_fdot.data(), d->n_spin * sizeof(double), cudaMemcpyHostToDevice, s), "fdot");
    p.sky = dalloc<SkyConst>(p, d->n_sky, n_alloc);
    {
        std::vector<SkyConst> hs((size_t)d->n_sky);
        for (int64_t i = 0; i < d->n_sky; ++i) hs[(size_t)i] = sky_const(p.h_alpha[i], p.h_delta[i], d->lat, d->gamma);
        check(cudaMemcpy(p.sky, hs.data(), hs.size() * sizeof(SkyConst), cudaMemcpyHostToDevice), "sky");
    }

    // spindown phase rates per (band, spin): fdot dt^2 / 2 cycles per k^2
    std::vector<uint64_t> cfx((size_t)d->n_bands * d->n_spin);
    std::vector<double> cd((size_t)d->n_bands * d->n_spin);
    for (int i = 0; i < d->n_bands; ++i)
        for (int64_t j = 0; j < d->n_spin; ++j) {
            const double rate = 0.5 * p.h_fdot[j] * d->bands[i].dt * d->bands[i].dt;
            cd[(size_t)i * d->n_spin + j] = rate;
            cfx[(size_t)i * d->n_spin + j] = to_fixed64(rate);
        }
    p.chirp_fx = dalloc<uint64_t>(p, cfx.size(), n_alloc);
    p.chirp_d = dalloc<double>(p, cd.size(), n_alloc);
    check(cudaMemcpy(p.chirp_fx, cfx.data(), cfx.size() * sizeof(uint64_t), cudaMemcpyHostToDevice), "chirp");
    check(cudaMemcpy(p.chirp_d, cd.data(), cd.size() * sizeof(double), cudaMemcpyHostToDevice), "chirp");

    // per-sky-batch buffers; w rows padded to a multiple of each band's N1 so that
    // column tiles of the first FFT pass never read past a sky's stretch
    p.w_stride = p.n_max;
    for (auto &b : p.bands) {
        const int64_t n1 = int64_t(1) << log_n1(b.logn);
        p.w_stride = std::max<int64_t>(p.w_stride, (b.n + n1 - 1) / n1 * n1);
    }
    const int64_t nblk = (p.n_max + 255) / 256;
    // sky positions per batch: 64, or up to 256 when the spindowns are few, so that a
    // batch holds the 4096 cells of a launch pair
    p.sky_batch = fp32 ? std::min<int64_t>(d->n_sky, std::max<int64_t>(64, std::min<int64_t>(256, (4096 + d->n_spin - 1) / d->n_spin)))
                       : 1;
    if (fp32)
        if (const char *v = getenv("FSTAT_SKY_BATCH")) p.sky_batch = std::max<int64_t>(1, std::min<int64_t>(d->n_sky, atoll(v)));
    const size_t w_elem = fp32 ? 16 : 32;
    for (int q = 0; q < 2; ++q) {
        p.wbuf[q] = dalloc<unsigned char>(p, (size_t)p.sky_batch * p.w_stride * w_elem, n_alloc);
        check(cudaMemsetAsync(p.wbuf[q], 0, (size_t)p.sky_batch * p.w_stride * w_elem, s), "memset");
    }
    // per-sample delays (FP64 form) or 16-byte shift records (FP32 form)
    p.dbuf = dalloc<double>(p, (size_t)p.sky_batch * p.n_max * (fp32 ? 2 : 1), n_alloc);
    p.partials = dalloc<double>(p, std::max<int64_t>((int64_t)p.sky_batch * nblk * 3, 256), n_alloc);
    p.S = dalloc<double>(p, 3 * p.sky_batch, n_alloc);
    for (int q = 0; q < 2; ++q) p.normbuf[q] = dalloc<double>(p, kNormStride * p.sky_batch, n_alloc);

    // FFT scratch: cell slots of 2 transforms; also hosts the generic FFT of the upsample
    const size_t tsz = fp32 ? sizeof(float2) : sizeof(double2);
    if (fp32) {
        // several worker streams, each running launch pairs of a batch of cells on its
        // own scratch slot: one stream's partial last wave overlaps the next grids
        // one stream with large launches is as fast as several overlapping streams
        // and keeps the per-launch event timings free of overlap
        p.n_workers = 1;
        if (const char *v = getenv("FSTAT_STREAMS")) p.n_workers = std::max(1, std::min(8, atoi(v)));
        const int64_t budget = int64_t(16) << 30;    // per worker slot (a sky batch of 2^18 cells)
        p.cell_batch = std::max<int64_t>(1, std::min<int64_t>(4096, budget / (2 * max_nfft * (int64_t)tsz)));
        p.cell_batch = std::min<int64_t>(p.cell_batch, p.sky_batch * d->n_spin);
        if (const char *v = getenv("FSTAT_CELL_BATCH")) p.cell_batch = std::max(1, std::min(65535, atoi(v)));
    } else {
        p.n_workers = 1;
        p.cell_batch = 1;
    }
    // a worker's slot holds a launch's cells, or the ring of the fused launch
    if (fp32) {
        if (const char *v = getenv("FSTAT_FUSED")) p.fused = atoi(v) != 0;
        if (const char *v = getenv("FSTAT_GRAPH")) p.use_graph = atoi(v) != 0;
        {   // pass-2 prefetch distance: one CTA per resident slot (3 per SM) ahead
            int dev = 0, sms = 0;
            check(cudaGetDevice(&dev), "cudaGetDevice");
            check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
            p.pf_dist = 3 * (int64_t)sms;
        }
        if (const char *v = getenv("FSTAT_PF_DIST")) p.pf_dist = std::max(0, atoi(v));
        if (const char *v = getenv("FSTAT_PF_DIST_PAIRED")) p.pf_dist_pk = std::max(0, atoi(v));
        if (const char *v = getenv("FSTAT_SHARE_CHIRP")) p.share_chirp = atoi(v) != 0;
        if (const char *v = getenv("FSTAT_P2_ROWS")) p.p2_rows = atoi(v) != 0;
        if (const char *v = getenv("FSTAT_P2_TS")) {
            const int ts = atoi(v);
            p.p2_ts = ts == 64 || ts == 128 ? ts : 32;
        }
        if (const char *v = getenv("FSTAT_TMA")) p.tma = atoi(v) != 0;
        if (const char *v = getenv("FSTAT_PACKED")) p.packed = std::max(0, std::min(3, atoi(v)));
        if (const char *v = getenv("FSTAT_P2_THREADS")) p.p2_threads = atoi(v) == 128 ? 128 : 256;
        if (const char *v = getenv("FSTAT_FUSED_SLOTS")) p.fused_slots = std::max(2, std::min(256, atoi(v)));
        if (const char *v = getenv("FSTAT_FUSED_AHEAD")) p.fused_ahead = std::max(1, atoi(v));
        p.fused_ahead = std::min(p.fused_ahead, p.fused_slots - 1);
        if (const char *v = getenv("FSTAT_FUSED_TPI")) {
            int t = 1;
            while (2 * t <= std::min(64, atoi(v))) t *= 2;
            p.fused_tpi = t;
        }
        // the fused launch needs no scratch per cell (a ring of slots): one launch
        // per sky batch
        p.fused_batch = std::max<int64_t>(1, std::min<int64_t>(65535, p.sky_batch * d->n_spin));
        if (const char *v = getenv("FSTAT_FUSED_BATCH")) p.fused_batch = std::max(1, std::min(65535, atoi(v)));
    }
    p.slot_cells = (size_t)std::max<int64_t>(p.cell_batch, fp32 ? p.fused_slots : 1);
    size_t scratch_bytes = std::max<size_t>((size_t)p.n_workers * p.slot_cells * 2 * max_nfft * tsz,
                                            (size_t)2 * std::max<int64_t>(max_m, p.n_max) * sizeof(double2) * 2);
    if (fp32) {
        if (const char *v = getenv("FSTAT_PERSIST_BATCH")) p.pbatch = std::max(1, atoi(v));
        if (const char *v = getenv("FSTAT_PERSIST_SLOTS")) p.pslots = std::max(2, atoi(v));
        scratch_bytes = std::max<size_t>(scratch_bytes, (size_t)p.pslots * p.pbatch * 2 * max_nfft * sizeof(float2));
        const int64_t nb_max = (p.sky_batch * d->n_spin + p.pbatch - 1) / p.pbatch + 1;
        p.queue = dalloc<uint32_t>(p, (size_t)(1 + 2 * nb_max), n_alloc);
        p.qerr = dalloc<uint32_t>(p, 1, n_alloc);
        check(cudaMemsetAsync(p.qerr, 0, sizeof(uint32_t), s), "memset");
        if (const char *v = getenv("FSTAT_TEST_WITHHOLD_ITEM")) p.withhold_item = atoll(v);
        if (const char *v = getenv("FSTAT_PERSISTENT")) p.use_persistent = atoi(v) != 0;
        if (const char *v = getenv("FSTAT_ELEMS_PER_THREAD")) p.elems_per_thread = atoi(v) == 8 ? 8 : 16;
        if (const char *v = getenv("FSTAT_ENGINE")) p.engine = atoi(v) == 1 ? 1 : 2;
        p.fctl = dalloc<uint32_t>(p, (size_t)p.n_workers * (1 + 2 * (size_t)std::max(p.cell_batch, p.fused_batch)),
                                  n_alloc);
    }
    p.scratch = dalloc<unsigned char>(p, scratch_bytes, n_alloc);
    p.bw_elems = 2 * p.n_max + 2 * max_m;
    p.bw = dalloc<double>(p, 2 * (size_t)std::max<int64_t>(p.bw_elems, 1), n_alloc);

    // worker streams (the FP64 plain form runs on the plan's stream alone)
    for (int q = 0; q < 2; ++q) {
        check(cudaEventCreateWithFlags(&p.ev_geo[q], cudaEventDisableTiming), "event");
        p.ev_all.push_back(p.ev_geo[q]);
    }
    for (int i = 0; i < p.n_workers; ++i) {
        cudaStream_t ws = s;
        if (p.n_workers > 1) {
            check(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking), "cudaStreamCreate");
            p.own_workers.push_back(ws);
        }
        p.workers.push_back(ws);
        for (int q = 0; q < 2; ++q) {
            cudaEvent_t e;
            check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            p.ev_all.push_back(e);
            p.ev_done[q].push_back(e);
        }
        cudaEvent_t e;
        check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        p.ev_all.push_back(e);
        p.ev_join.push_back(e);
    }

    p.cand_capacity = d->cand_capacity;
    p.cand = dalloc<CandRecord>(p, (size_t)p.cand_capacity, n_alloc);
    p.cand_count = dalloc<unsigned long long>(p, 1, n_alloc);
    check(cudaMemsetAsync(p.cand_count, 0, sizeof(unsigned long long), s), "memset");
    check(cudaStreamSynchronize(s), "plan setup");
    check(cudaGetLastError(), "plan setup launch");
}

void free_all(Plan &p) {
    if (p.graph.exec) cudaGraphExecDestroy(p.graph.exec);
    p.graph.exec = nullptr;
    if (!p.allocs.empty() || p.own_stream) cudaDeviceSynchronize();
    for (void *ptr : p.allocs) cudaFree(ptr);
    p.allocs.clear();
    for (cudaEvent_t e : p.ev_all) cudaEventDestroy(e);
    p.ev_all.clear();
    for (cudaStream_t w : p.own_workers) cudaStreamDestroy(w);
    p.own_workers.clear();
    p.workers.clear();
    p.ev_pool.clear();
    p.pending.clear();
    if (p.own_stream && p.stream) cudaStreamDestroy(p.stream);
    p.stream = nullptr;
    p.own_stream = false;
    if (p.h_rec) cudaFreeHost(p.h_rec);
    p.h_rec = nullptr;
    p.h_rec_cap = 0;
    p.h_tmp.clear();
    p.h_tmp.shrink_to_fit();
    if (p.cand_tmp) cudaFree(p.cand_tmp);
    if (p.sort_hist) cudaFree(p.sort_hist);
    p.cand_tmp = nullptr;
    p.sort_hist = nullptr;
    p.sort_cap = 0;
    p.cand_sorted = nullptr;
}

// ---------------------------------------------------------------- sampled timing
int stat_index(Plan &p, const char *name) {
    for (size_t i = 0; i < p.kstats.size(); ++i)
        if (p.kstats[i].name == name) return (int)i;
    Plan::KStat k;
    k.name = name;
    p.kstats.push_back(k);
    return (int)p.kstats.size() - 1;
}

void rec_timing(cudaEvent_t e, cudaStream_t s) { check(record_timing_event(e, s), "event"); }

cudaEvent_t ev_get(Plan &p) {
    if (!p.ev_pool.empty()) {
        cudaEvent_t e = p.ev_pool.back();
        p.ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    check(cudaEventCreate(&e), "cudaEventCreate");
    p.ev_all.push_back(e);
    return e;
}

// Counts one launch of class `name` with its algorithmic work; returns whether
// this launch is one of the sampled ones.
bool stat_launch(Plan &p, int idx, double flops, double bytes) {
    auto &k = p.kstats[(size_t)idx];
    k.launches += 1;
    k.flops += flops;
    k.bytes += bytes;
    return p.timing_every > 0 && (k.launches - 1) % p.timing_every == 0;
}

void collect_timing(Plan &p, bool recycle = true) {
    std::vector<cudaEvent_t> used;
    for (auto &pe : p.pending) {
        float ms = 0.f;
        check(cudaEventElapsedTime(&ms, pe.a, pe.b), "cudaEventElapsedTime");
        p.kstats[(size_t)pe.stat].timed += 1;
        p.kstats[(size_t)pe.stat].ms += ms;
        used.push_back(pe.a);
        used.push_back(pe.b);
    }
    // an event may close one interval and open the next: return each once
    std::sort(used.begin(), used.end());
    used.erase(std::unique(used.begin(), used.end()), used.end());
    if (recycle)
        for (cudaEvent_t e : used) p.ev_pool.push_back(e);
    p.pending.clear();
}

// Per-band prologue: sigma^2 and the FFT upsample.
void band_prologue(Plan &p, BandDev &b) {
    const bool fp32 = p.desc.form == FSTAT_FP32_BATCHED;
    const int idx = stat_index(p, "band_prologue");
    const bool t = stat_launch(p, idx, 0.0, (double)b.n * 8.0 * (1 + p.desc.upsample));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (t) { e0 = ev_get(p); e1 = ev_get(p); rec_timing(e0, p.stream); }
    p.launches += launch_sigma2(b.x, b.n, p.desc.sigma2, p.partials, b.sigma2, p.stream);
    p.launches += launch_upsample(p, b, p.desc.upsample, b.xu, fp32, p.stream);
    if (fp32) p.launches += launch_split_r(b, p.stream);
    if (t) { rec_timing(e1, p.stream); p.pending.push_back({idx, e0, e1}); }
}

void enqueue_search(Plan &p, int64_t begin, int64_t end) {
    p.cand_begin = begin;
    p.cand_end = end;
    const fstat_plan_desc &d = p.desc;
    const bool fp32 = d.form == FSTAT_FP32_BATCHED;
    cudaStream_t s = p.stream;
    check(cudaMemsetAsync(p.cand_count, 0, sizeof(unsigned long long), s), "memset");
    if (p.qerr) check(cudaMemsetAsync(p.qerr, 0, sizeof(uint32_t), s), "memset");
    const int64_t per_band = d.n_sky * d.n_spin;
    const int NW = (int)p.workers.size();
    const size_t slot_bytes = p.slot_cells * 2 * (size_t)p.n_fft_max * (fp32 ? 8 : 16);
    const size_t ctl_words = 1 + 2 * (size_t)std::max(p.cell_batch, p.fused_batch);
    // the plan's stream waits for every worker stream
    auto join_workers = [&]() {
        if (NW < 2) return;
        for (int i = 0; i < NW; ++i) {
            check(cudaEventRecord(p.ev_join[i], p.workers[i]), "event");
            check(cudaStreamWaitEvent(s, p.ev_join[i], 0), "stream wait");
        }
    };
    // the worker streams start after everything queued so far on the plan's stream
    {
        check(cudaEventRecord(p.ev_geo[0], s), "event");
        for (int i = 0; i < NW; ++i)
            if (p.workers[i] != s) check(cudaStreamWaitEvent(p.workers[i], p.ev_geo[0], 0), "stream wait");
    }
    int64_t q = 0;        // sky batches so far (parity selects the w / norm buffers)
    int64_t cbi = 0;      // cell batches so far (round-robin over the workers)
    for (int bi = 0; bi < d.n_bands; ++bi) {
        const int64_t b0 = (int64_t)bi * per_band;
        const int64_t lc0 = std::max<int64_t>(begin, b0) - b0;
        const int64_t lc1 = std::min<int64_t>(end, b0 + per_band) - b0;
        if (lc1 <= lc0) continue;
        BandDev &b = p.bands[bi];
        join_workers();   // the prologue's transforms use the scratch area
        band_prologue(p, b);
        const int64_t s_first = lc0 / d.n_spin, s_last = (lc1 - 1) / d.n_spin;
        // transform length of the search (half of n_fft when interbinning)
        const int tlog = p.interbin ? b.logn - 1 : b.logn;
        const double nfft = (double)(int64_t(1) << tlog);
        const double lg1 = (double)log_n1(tlog), lg2 = (double)log_n2(tlog);
        const int i_geo = stat_index(p, "geometry_resample");
        const int i_p1 = stat_index(p, fp32 ? "fft_pass1_f32" : "fft_pass1_f64");
        const int i_p2 = stat_index(p, fp32 ? "fft_pass2_fstat_f32" : "fft_pass2_fstat_f64");
        const int i_pp = stat_index(p, "fft_fstat_persistent_f32");
        const int i_fu = stat_index(p, "fft_fused_f32");
        const double welem = fp32 ? 16.0 : 32.0;
        for (int64_t sb = s_first; sb <= s_last; sb += p.sky_batch, ++q) {
            const int par = (int)(q & 1);
            const int64_t ns = std::min<int64_t>(p.sky_batch, s_last + 1 - sb);
            // the buffers of parity `par` were last read by the transforms of sky batch q - 2
            if (q >= 2 && NW > 1)
                for (int i = 0; i < NW; ++i)
                    check(cudaStreamWaitEvent(s, p.ev_done[par][i], 0), "stream wait");
            // algorithmic bytes: ephemeris + upsampled series read, w written per sky
            const bool tg = stat_launch(p, i_geo, 0.0,
                                        (double)b.n * (24.0 + welem * ns) + (double)p.desc.upsample * b.n * (fp32 ? 4 : 8));
            cudaEvent_t g0 = nullptr, g1 = nullptr;
            if (tg) { g0 = ev_get(p); g1 = ev_get(p); rec_timing(g0, s); }
            p.launches += launch_geometry(p, b, sb, ns, fp32, p.wbuf[par], nullptr, nullptr, nullptr, nullptr, s);
            p.launches += launch_reduce_norms(p, b, ns, p.normbuf[par], s);
            if (tg) { rec_timing(g1, s); p.pending.push_back({i_geo, g0, g1}); }
            const int64_t c_lo = std::max<int64_t>(lc0, sb * d.n_spin);
            const int64_t c_hi = std::min<int64_t>(lc1, (sb + ns) * d.n_spin);
            if (fp32 && p.use_persistent && !p.interbin && persistent_supported(b.logn)) {
                join_workers();
                const bool tp = stat_launch(p, i_pp, 2.0 * (c_hi - c_lo) * 5.0 * nfft * (lg1 + lg2),
                                            (double)ns * b.n * welem);
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (tp) { e0 = ev_get(p); e1 = ev_get(p); rec_timing(e0, s); }
                const CellBufs cbuf{p.wbuf[par], p.normbuf[par], p.scratch};
                p.launches += launch_search_persistent(p, bi, b, sb, c_lo, c_hi, s, cbuf);
                if (tp) { rec_timing(e1, s); p.pending.push_back({i_pp, e0, e1}); }
                if (NW > 1)
                    for (int i = 0; i < NW; ++i) check(cudaEventRecord(p.ev_done[par][i], s), "event");
                continue;
            }
            if (NW > 1) {
                check(cudaEventRecord(p.ev_geo[par], s), "event");
                for (int i = 0; i < NW; ++i)
                    check(cudaStreamWaitEvent(p.workers[i], p.ev_geo[par], 0), "stream wait");
            }
            const bool fused = fp32 && fused_supported(p, b.logn);
            const int64_t batch = fused ? p.fused_batch : p.cell_batch;
            for (int64_t c = c_lo; c < c_hi; c += batch, ++cbi) {
                const int wi = (int)(cbi % NW);
                cudaStream_t ws = p.workers[wi];
                const int64_t nc = std::min<int64_t>(batch, c_hi - c);
                CellBufs cbuf{p.wbuf[par], p.normbuf[par],
                              static_cast<unsigned char *>(p.scratch) + wi * slot_bytes};
                if (fused) {
                    cbuf.ctl = p.fctl + wi * ctl_words;
                    check(cudaMemsetAsync(cbuf.ctl, 0, (1 + 2 * (size_t)nc) * sizeof(uint32_t), ws), "memset");
                    const int64_t sky_a = c / d.n_spin, sky_b = (c + nc - 1) / d.n_spin;
                    const bool tf = stat_launch(p, i_fu, 2.0 * nc * 5.0 * nfft * (lg1 + lg2),
                                                (double)(sky_b - sky_a + 1) * b.n * welem);
                    cudaEvent_t e0 = nullptr, e1 = nullptr;
                    if (tf) { e0 = ev_get(p); e1 = ev_get(p); rec_timing(e0, ws); }
                    const int L = launch_search_cells_f32(p, bi, b, sb, c, nc, ws, nullptr, cbuf);
                    if (L < 0) throw std::string("unsupported transform length");
                    p.launches += L;
                    if (tf) { rec_timing(e1, ws); p.pending.push_back({i_fu, e0, e1}); }
                    continue;
                }
                // 5 N log2 N per complex transform, split between the passes; two
                // transforms per cell.  Pass 1 reads w once per distinct sky.
                const int64_t sky_a = c / d.n_spin, sky_b = (c + nc - 1) / d.n_spin;
                const bool t1 = stat_launch(p, i_p1, 2.0 * nc * 5.0 * nfft * lg2,
                                            (double)(sky_b - sky_a + 1) * b.n * welem);
                stat_launch(p, i_p2, 2.0 * nc * 5.0 * nfft * lg1, 0.0);
                cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
                if (t1) {
                    e0 = ev_get(p); e1 = ev_get(p); e2 = ev_get(p);
                    rec_timing(e0, ws);
                }
                const int L = fp32 ? launch_search_cells_f32(p, bi, b, sb, c, nc, ws, e1, cbuf)
                                   : launch_search_cells_f64(p, bi, b, sb, c, nc, ws, e1, cbuf);
                if (L < 0) throw std::string("unsupported transform length");
                p.launches += L;
                if (t1) {
                    rec_timing(e2, ws);
                    p.pending.push_back({i_p1, e0, e1});
                    p.pending.push_back({i_p2, e1, e2});
                }
            }
            if (NW > 1)
                for (int i = 0; i < NW; ++i) check(cudaEventRecord(p.ev_done[par][i], p.workers[i]), "event");
        }
    }
    join_workers();
    check(cudaGetLastError(), "search launch");
}

// Waits for the search, reads the error word and the candidate count.
void finish_search(Plan &p, bool recycle_events) {
    check(cudaStreamSynchronize(p.stream), "search");
    collect_timing(p, recycle_events);
    if (p.qerr) {
        uint32_t e = 0;
        check(cudaMemcpy(&e, p.qerr, sizeof(e), cudaMemcpyDeviceToHost), "queue status");
        if (e) throw TimeoutError{};
    }
    unsigned long long cnt = 0;
    check(cudaMemcpy(&cnt, p.cand_count, sizeof(cnt), cudaMemcpyDeviceToHost), "count");
    p.last_total = (int64_t)cnt;
    p.searched = true;
    p.cand_sorted = nullptr;
}

void drop_graph(Plan &p) {
    if (p.graph.exec) cudaGraphExecDestroy(p.graph.exec);
    // its events go back to the pool
    for (auto &pe : p.graph.pending) { p.ev_pool.push_back(pe.a); p.ev_pool.push_back(pe.b); }
    std::sort(p.ev_pool.begin(), p.ev_pool.end());
    p.ev_pool.erase(std::unique(p.ev_pool.begin(), p.ev_pool.end()), p.ev_pool.end());
    p.graph = Plan::GraphRun{};
}

// One search: the launch sequence is captured into a CUDA graph the first time
// a cell range is searched (at the current timing rate) and replayed after
// that, so a repeated search costs one graph launch on the host.
void search_impl(Plan &p, int64_t begin, int64_t end) {
    auto &g = p.graph;
    const bool hit = g.exec && g.begin == begin && g.end == end && g.timing_every == p.timing_every;
    // capture only a search that repeats the previous one (a plan searched once
    // never pays for the capture)
    const bool repeat = p.prev_begin == begin && p.prev_end == end && p.prev_timing == p.timing_every;
    p.prev_begin = begin;
    p.prev_end = end;
    p.prev_timing = p.timing_every;
    if (!p.use_graph || (!hit && !repeat)) {
        enqueue_search(p, begin, end);
        finish_search(p, true);
        return;
    }
    if (!hit) {
        drop_graph(p);
        const std::vector<Plan::KStat> before = p.kstats;
        const int64_t launches0 = p.launches;
        cudaGraph_t graph = nullptr;
        check(cudaStreamBeginCapture(p.stream, cudaStreamCaptureModeThreadLocal), "graph capture");
        try {
            enqueue_search(p, begin, end);
        } catch (...) {
            cudaStreamEndCapture(p.stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        check(cudaStreamEndCapture(p.stream, &graph), "graph capture");
        const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        check(ie, "graph instantiate");
        g.begin = begin;
        g.end = end;
        g.timing_every = p.timing_every;
        g.launches = p.launches - launches0;
        g.dk = p.kstats;
        for (size_t i = 0; i < g.dk.size(); ++i) {
            const Plan::KStat b0 = i < before.size() ? before[i] : Plan::KStat{};
            g.dk[i].launches -= b0.launches;
            g.dk[i].flops -= b0.flops;
            g.dk[i].bytes -= b0.bytes;
        }
        g.pending = p.pending;   // the capture's host counters stand for this first run
    } else {
        for (const auto &k : g.dk) {   // by name: the statistics may have been reset since
            if (k.launches == 0) continue;
            auto &t = p.kstats[(size_t)stat_index(p, k.name.c_str())];
            t.launches += k.launches;
            t.flops += k.flops;
            t.bytes += k.bytes;
        }
        p.launches += g.launches;
        p.pending = g.pending;
        for (auto &pe : p.pending) pe.stat = stat_index(p, g.dk[(size_t)pe.stat].name.c_str());
    }
    check(cudaGraphLaunch(g.exec, p.stream), "graph launch");
    finish_search(p, false);
}

template <class F>
fstat_status guarded(fstat_plan *p, F &&f) {
    if (!p) return FSTAT_ERR_ARG;
    if (p->poisoned) return FSTAT_ERR_STATE;
    p->err.clear();
    try {
        return f();
    } catch (const CudaError &e) {
        p->err = std::string(e.what) + ": " + cudaGetErrorString(e.e);
        p->poisoned = true;
        return FSTAT_ERR_CUDA;
    } catch (const OomError &) {
        p->err = "out of device memory";
        return FSTAT_ERR_OOM;
    } catch (const TimeoutError &) {
        p->err = "a bounded device-side wait of the work queue ran out";
        p->poisoned = true;
        return FSTAT_ERR_TIMEOUT;
    } catch (const std::bad_alloc &) {
        p->err = "out of host memory";
        return FSTAT_ERR_OOM;
    } catch (const std::string &m) {
        p->err = m;
        return FSTAT_ERR_ARG;
    }
}

}  // namespace
}  // namespace fstat

using namespace fstat;

namespace {

inline uint64_t cand_key(const fstat::CandRecord &r) { return ((uint64_t)r.cell << 32) | r.bin; }
constexpr int64_t kDeviceSortMin = 1 << 16;   // fewer records are sorted on the host
constexpr int64_t kTileSlack = 4096;          // device positions are 32-bit

// Runs f(t) for t in [0, nt) on nt threads (the calling thread takes t = 0).
template <class Fn>
void parallel_for_threads(int nt, Fn f) {
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(f, t);
    f(0);
    for (auto &x : th) x.join();
}

// Sorts the records by (cell, bin): a bucket pass over the cell range into tmp,
// then the buckets side by side, each by a counting sort over its cells back
// into rec and a sort of each cell's records by bin.  rec and tmp hold n
// records; the result is in the returned pointer (one of the two).
fstat::CandRecord *sort_records(fstat::CandRecord *rec, fstat::CandRecord *tmp, int64_t n) {
    using fstat::CandRecord;
    auto less = [](const CandRecord &a, const CandRecord &b) { return cand_key(a) < cand_key(b); };
    const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<int64_t>(std::min(hc, 64u), std::max<int64_t>(1, n >> 16));
    if (nt <= 1) {
        std::sort(rec, rec + n, less);
        return rec;
    }
    const int nb = 8 * nt;   // buckets
    std::vector<uint32_t> lo_t(nt, UINT32_MAX), hi_t(nt, 0);
    auto chunk = [&](int t, int64_t &a, int64_t &b) { a = n * t / nt; b = n * (t + 1) / nt; };
    parallel_for_threads(nt, [&](int t) {
        int64_t a, b;
        chunk(t, a, b);
        for (int64_t i = a; i < b; ++i) {
            lo_t[t] = std::min(lo_t[t], rec[i].cell);
            hi_t[t] = std::max(hi_t[t], rec[i].cell);
        }
    });
    const uint64_t lo = *std::min_element(lo_t.begin(), lo_t.end());
    const uint64_t span = *std::max_element(hi_t.begin(), hi_t.end()) - lo + 1;
    auto bucket = [&](const CandRecord &r) { return (int)((r.cell - lo) * (uint64_t)nb / span); };
    std::vector<int64_t> hist((size_t)nt * nb, 0);
    parallel_for_threads(nt, [&](int t) {
        int64_t a, b;
        chunk(t, a, b);
        int64_t *h = &hist[(size_t)t * nb];
        for (int64_t i = a; i < b; ++i) ++h[bucket(rec[i])];
    });
    std::vector<int64_t> start(nb + 1, 0), off((size_t)nt * nb);
    int64_t acc = 0;
    for (int k = 0; k < nb; ++k) {
        start[k] = acc;
        for (int t = 0; t < nt; ++t) {
            off[(size_t)t * nb + k] = acc;
            acc += hist[(size_t)t * nb + k];
        }
    }
    start[nb] = acc;
    parallel_for_threads(nt, [&](int t) {
        int64_t a, b;
        chunk(t, a, b);
        int64_t *o = &off[(size_t)t * nb];
        for (int64_t i = a; i < b; ++i) tmp[o[bucket(rec[i])]++] = rec[i];
    });
    // each bucket: counting sort by cell back into rec, then every cell's few
    // records (tens at a typical threshold) by bin
    std::atomic<int> next{0};
    parallel_for_threads(nt, [&](int) {
        std::vector<int64_t> cnt;
        for (int k; (k = next.fetch_add(1)) < nb;) {
            const int64_t a = start[k], b = start[k + 1];
            if (b - a < 64) {
                std::copy(tmp + a, tmp + b, rec + a);
                std::sort(rec + a, rec + b, less);
                continue;
            }
            uint32_t cmin = UINT32_MAX, cmax = 0;
            for (int64_t i = a; i < b; ++i) {
                cmin = std::min(cmin, tmp[i].cell);
                cmax = std::max(cmax, tmp[i].cell);
            }
            const size_t nc = (size_t)(cmax - cmin) + 1;
            cnt.assign(nc + 1, 0);
            for (int64_t i = a; i < b; ++i) ++cnt[tmp[i].cell - cmin + 1];
            for (size_t c = 1; c <= nc; ++c) cnt[c] += cnt[c - 1];
            for (int64_t i = a; i < b; ++i) rec[a + cnt[tmp[i].cell - cmin]++] = tmp[i];
            // cnt[c] is now the end of cell c's run
            int64_t lo_i = a;
            for (size_t c = 0; c < nc; ++c) {
                const int64_t hi_i = a + cnt[c];
                if (hi_i - lo_i > 1) {
                    if (hi_i - lo_i <= 32) {        // insertion sort by bin
                        for (int64_t i = lo_i + 1; i < hi_i; ++i) {
                            const CandRecord v = rec[i];
                            int64_t j = i - 1;
                            while (j >= lo_i && rec[j].bin > v.bin) { rec[j + 1] = rec[j]; --j; }
                            rec[j + 1] = v;
                        }
                    } else {
                        std::sort(rec + lo_i, rec + hi_i, less);
                    }
                }
                lo_i = hi_i;
            }
        }
    });
    return rec;
}

}  // namespace

extern "C" {

fstat_status fstat_plan_create(fstat_plan **out, const fstat_plan_desc *desc) {
    if (!out) return FSTAT_ERR_ARG;
    *out = nullptr;
    std::string err;
    fstat_status st = validate(desc, err);
    if (st != FSTAT_OK) {
        if (getenv("FSTAT_LOG")) fprintf(stderr, "fstat_plan_create: %s\n", err.c_str());
        return st;
    }
    fstat_plan *p = new (std::nothrow) fstat_plan();
    if (!p) return FSTAT_ERR_OOM;
    try {
        create_impl(*p, desc);
    } catch (const CudaError &e) {
        if (getenv("FSTAT_LOG")) fprintf(stderr, "fstat_plan_create: %s: %s\n", e.what, cudaGetErrorString(e.e));
        free_all(*p);
        delete p;
        return FSTAT_ERR_CUDA;
    } catch (const OomError &) {
        free_all(*p);
        delete p;
        return FSTAT_ERR_OOM;
    } catch (const std::bad_alloc &) {
        free_all(*p);
        delete p;
        return FSTAT_ERR_OOM;
    } catch (const std::string &m) {
        if (getenv("FSTAT_LOG")) fprintf(stderr, "fstat_plan_create: %s\n", m.c_str());
        free_all(*p);
        delete p;
        return FSTAT_ERR_ARG;
    }
    *out = p;
    return FSTAT_OK;
}

fstat_status fstat_search(fstat_plan *p, int64_t cell_begin, int64_t cell_end) {
    return guarded(p, [&]() -> fstat_status {
        if (cell_end < 0) cell_end = p->n_cells;
        if (cell_begin < 0 || cell_begin > cell_end || cell_end > p->n_cells) {
            p->err = "cell range outside [0, n_cells]";
            return FSTAT_ERR_ARG;
        }
        search_impl(*p, cell_begin, cell_end);
        return p->last_total > p->cand_capacity ? FSTAT_ERR_OVERFLOW : FSTAT_OK;
    });
}

fstat_status fstat_candidates_get(fstat_plan *p, fstat_candidate *buf, int64_t cap,
                                  int64_t *n_written, int64_t *n_total) {
    return guarded(p, [&]() -> fstat_status {
        if (cap < 0 || (cap > 0 && !buf)) { p->err = "bad buffer"; return FSTAT_ERR_ARG; }
        if (n_written) *n_written = 0;
        if (n_total) *n_total = 0;
        if (!p->searched) return FSTAT_OK;
        if (n_total) *n_total = p->last_total;
        if (cap == 0) return p->last_total > 0 ? FSTAT_ERR_OVERFLOW : FSTAT_OK;   // count only
        const int64_t kept = std::min<int64_t>(p->last_total, p->cand_capacity);
        if (kept > p->h_rec_cap) {   // pinned staging, reused: no page faults, full-rate copies
            if (p->h_rec) cudaFreeHost(p->h_rec);
            p->h_rec = nullptr;
            p->h_rec_cap = 0;
            const int64_t want = std::max<int64_t>(kept, kept + kept / 4);
            if (cudaHostAlloc((void **)&p->h_rec, want * sizeof(CandRecord), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                p->h_rec = nullptr;
                throw std::bad_alloc();
            }
            p->h_rec_cap = want;
        }
        CandRecord *rec = p->h_rec;
        // many records: sorted on the device once per search, then read back in order
        const bool dev_sort = kept >= kDeviceSortMin && kept < (int64_t(1) << 32) - kTileSlack;
        // a few records: sorted on the host, with a pageable work array (no pinning)
        if (!dev_sort && (int64_t)p->h_tmp.size() < kept) p->h_tmp.resize((size_t)kept);
        CandRecord *tmp = p->h_tmp.data();
        if (dev_sort && !p->cand_sorted) {
            if (kept > p->sort_cap) {
                if (p->cand_tmp) cudaFree(p->cand_tmp);
                if (p->sort_hist) cudaFree(p->sort_hist);
                p->cand_tmp = nullptr;
                p->sort_hist = nullptr;
                p->sort_cap = 0;
                const int64_t want = std::min<int64_t>(p->cand_capacity, kept + kept / 4);
                const int64_t nblk = (want + 4095) / 4096;
                if (cudaMalloc((void **)&p->cand_tmp, want * sizeof(CandRecord)) != cudaSuccess ||
                    cudaMalloc((void **)&p->sort_hist, 256 * (nblk + 1) * sizeof(uint32_t)) != cudaSuccess) {
                    cudaGetLastError();
                    if (p->cand_tmp) cudaFree(p->cand_tmp);
                    p->cand_tmp = nullptr;
                    throw OomError{};
                }
                p->sort_cap = want;
            }
            int bin_bits = 0;
            while ((int64_t(1) << bin_bits) < p->n_fft_max) ++bin_bits;
            p->cand_sorted = launch_cand_sort(p->cand, p->cand_tmp, p->sort_hist, kept, (uint32_t)p->cand_begin,
                                              (uint64_t)(p->cand_end - p->cand_begin), bin_bits, p->stream,
                                              &p->launches);
            check(cudaGetLastError(), "candidate sort");
        }
        if (kept > 0) {
            check(cudaMemcpyAsync(rec, dev_sort ? p->cand_sorted : p->cand, kept * sizeof(CandRecord),
                                  cudaMemcpyDeviceToHost, p->stream),
                  "candidates");
            check(cudaStreamSynchronize(p->stream), "candidates");
        }
        const CandRecord *sorted = kept > 0 && !dev_sort ? sort_records(rec, tmp, kept) : rec;
        const int64_t nw = std::min<int64_t>(kept, cap);
        const fstat_plan_desc &d = p->desc;
        const int64_t per_band = d.n_sky * d.n_spin;
        const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
        const int nt = (int)std::min<int64_t>(std::min(hc, 64u), std::max<int64_t>(1, nw >> 16));
        parallel_for_threads(nt, [&](int t) {
            for (int64_t i = nw * t / nt; i < nw * (t + 1) / nt; ++i) {
                const CandRecord &r = sorted[i];
                const int band = (int)(r.cell / per_band);
                const int64_t rem = r.cell - (int64_t)band * per_band;
                fstat_candidate &c = buf[i];
                c.band = band;
                c.reserved = 0;
                c.sky = rem / d.n_spin;
                c.spin = rem % d.n_spin;
                c.bin = r.bin;
                c.alpha = p->h_alpha[(size_t)c.sky];
                c.delta = p->h_delta[(size_t)c.sky];
                c.fdot = p->h_fdot[(size_t)c.spin];
                const BandDev &b = p->bands[(size_t)band];
                c.freq = b.f_off + (double)r.bin / ((double)b.n_fft * b.dt);
                c.F = r.F;
            }
        });
        if (n_written) *n_written = nw;
        return p->last_total > nw ? FSTAT_ERR_OVERFLOW : FSTAT_OK;
    });
}

fstat_status fstat_plan_set_band(fstat_plan *p, int band, const fstat_band *nb) {
    return guarded(p, [&]() -> fstat_status {
        if (!nb || band < 0 || band >= p->desc.n_bands) {
            p->err = "band out of range";
            return FSTAT_ERR_ARG;
        }
        BandDev &b = p->bands[(size_t)band];
        int64_t nf = nb->n_fft;
        if (nf == 0) { nf = 1; while (nf < 2 * nb->n) nf <<= 1; }
        if (nb->n != b.n || nb->dt != b.dt || nf != b.n_fft) {
            p->err = "n, dt and n_fft must equal those of the plan's band";
            return FSTAT_ERR_ARG;
        }
        if (!is_finite(nb->f_off) || !is_finite(nb->phi0) || (nb->x == nullptr) == (nb->x32 == nullptr) || !nb->r) {
            p->err = "bad f_off/phi0, or not exactly one of x, x32, or r is NULL";
            return FSTAT_ERR_ARG;
        }
        const bool dev = p->desc.inputs_on_device == 1;
        cudaStream_t s = p->stream;
        if (nb->x) {
            copy_in(b.x, nb->x, b.n * sizeof(double), dev, s);
        } else {
            if (!b.x32) {
                int n_alloc = 0;
                b.x32 = dalloc<float>(*p, b.n, n_alloc);
            }
            copy_in(b.x32, nb->x32, b.n * sizeof(float), dev, s);
            k_f32_to_f64<<<(unsigned)((b.n + 255) / 256), 256, 0, s>>>(b.x32, b.n, b.x);
            check(cudaGetLastError(), "launch");
            ++p->launches;
        }
        copy_in(b.r, nb->r, 3 * b.n * sizeof(double), dev, s);
        // scalars are kernel arguments of a captured search: a change forces a recapture
        if (nb->f_off != b.f_off || nb->phi0 != b.phi0 || nb->eps != b.eps) {
            b.f_off = nb->f_off;
            b.phi0 = nb->phi0;
            b.eps = nb->eps;
            drop_graph(*p);
        }
        check(cudaStreamSynchronize(s), "band copy");
        return FSTAT_OK;
    });
}

fstat_status fstat_debug_sky(fstat_plan *p, int band, int64_t sky, double *y, double *a,
                             double *b, uint8_t *mask, double *S) {
    return guarded(p, [&]() -> fstat_status {
        if (band < 0 || band >= p->desc.n_bands || sky < 0 || sky >= p->desc.n_sky) {
            p->err = "band or sky out of range";
            return FSTAT_ERR_ARG;
        }
        BandDev &bd = p->bands[(size_t)band];
        const int64_t n = bd.n;
        double *dy = nullptr, *da = nullptr, *db = nullptr;
        uint8_t *dm = nullptr;
        int n_alloc = 0;
        const size_t before = p->allocs.size();
        const int64_t bytes_before = p->device_bytes;
        try {
            dy = dalloc<double>(*p, 2 * n, n_alloc);
            da = dalloc<double>(*p, n, n_alloc);
            db = dalloc<double>(*p, n, n_alloc);
            dm = dalloc<uint8_t>(*p, n, n_alloc);
        } catch (...) {
            for (size_t i = before; i < p->allocs.size(); ++i) cudaFree(p->allocs[i]);
            p->allocs.resize(before);
            p->device_bytes = bytes_before;
            throw;
        }
        const bool fp32 = p->desc.form == FSTAT_FP32_BATCHED;
        band_prologue(*p, bd);
        p->launches += launch_geometry(*p, bd, sky, 1, fp32, p->wbuf[0], dy, da, db, dm, p->stream);
        p->launches += launch_reduce_norms(*p, bd, 1, p->normbuf[0], p->stream);
        check(cudaStreamSynchronize(p->stream), "debug sky");
        if (y) check(cudaMemcpy(y, dy, 2 * n * sizeof(double), cudaMemcpyDeviceToHost), "y");
        if (a) check(cudaMemcpy(a, da, n * sizeof(double), cudaMemcpyDeviceToHost), "a");
        if (b) check(cudaMemcpy(b, db, n * sizeof(double), cudaMemcpyDeviceToHost), "b");
        if (mask) check(cudaMemcpy(mask, dm, n, cudaMemcpyDeviceToHost), "mask");
        if (S) check(cudaMemcpy(S, p->S, 3 * sizeof(double), cudaMemcpyDeviceToHost), "S");
        for (size_t i = before; i < p->allocs.size(); ++i) cudaFree(p->allocs[i]);
        p->allocs.resize(before);
        p->device_bytes = bytes_before;
        return FSTAT_OK;
    });
}

fstat_status fstat_plan_autotune(fstat_plan *p, int64_t sample_cells, fstat_tuning *chosen) {
    return guarded(p, [&]() -> fstat_status {
        if (p->desc.form != FSTAT_FP32_BATCHED || sample_cells < 1) {
            p->err = "autotune needs an FP32_BATCHED plan and sample_cells >= 1";
            return FSTAT_ERR_ARG;
        }
        const int64_t nc = std::min<int64_t>(sample_cells, p->n_cells);
        const int timing = p->timing_every;
        const bool graph = p->use_graph;
        p->timing_every = 0;
        p->use_graph = false;
        drop_graph(*p);
        cudaEvent_t e0 = ev_get(*p), e1 = ev_get(*p);
        auto time_once = [&]() -> double {
            check(cudaEventRecord(e0, p->stream), "event");
            enqueue_search(*p, 0, nc);
            check(cudaEventRecord(e1, p->stream), "event");
            finish_search(*p, true);
            float ms = 0.f;
            check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            return ms;
        };
        auto measure = [&]() -> double {   // best of two after one untimed run
            time_once();
            return std::min(time_once(), time_once());
        };
        double best = measure();
        // one choice at a time; a change stays when it is >= 1 % faster
        auto try_set = [&](auto set, auto undo) {
            set();
            const double t = measure();
            if (t < 0.99 * best) best = t;
            else undo();
        };
        const int64_t cb0 = p->cell_batch;
        for (int64_t cb : {int64_t(256), int64_t(512)}) {
            if (cb >= p->cell_batch) continue;
            const int64_t old = p->cell_batch;
            try_set([&] { p->cell_batch = cb; }, [&] { p->cell_batch = old; });
        }
        (void)cb0;
        { const int old = p->p2_threads;
          try_set([&] { p->p2_threads = old == 128 ? 256 : 128; }, [&] { p->p2_threads = old; }); }
        { const int old = p->p2_ts;   // the paired rows: one or four rows per CTA
          try_set([&] { p->p2_ts = old == 32 ? 128 : 32; }, [&] { p->p2_ts = old; }); }
        { const bool old = p->tma;
          try_set([&] { p->tma = !old; }, [&] { p->tma = old; }); }
        { const bool old = p->fused;
          try_set([&] { p->fused = !old; }, [&] { p->fused = old; }); }
        { const int old = p->engine;
          try_set([&] { p->engine = old == 2 ? 1 : 2; }, [&] { p->engine = old; }); }
        for (int pkv : {0, 2}) {   // paired arithmetic in neither pass, or in both
            const int old = p->packed;
            if (pkv == old) continue;
            try_set([&] { p->packed = pkv; }, [&] { p->packed = old; });
        }
        p->ev_pool.push_back(e0);
        p->ev_pool.push_back(e1);
        p->timing_every = timing;
        p->use_graph = graph;
        p->kstats.clear();
        p->searched = false;
        p->prev_begin = p->prev_end = -1;
        if (chosen) {
            // the paired pass 2 (512-point rows) runs whenever packed >= 1 with the
            // bulk-copy loader and 128-thread scalar tiles
            const bool paired2 = p->packed >= 1 && p->tma && p->p2_threads == 128;
            chosen->engine = p->engine == 2 && paired2 ? 2 + p->packed : p->engine;
            chosen->pass2_threads = paired2 ? p->p2_ts : p->p2_threads;
            chosen->pass2_bulk_copy = p->tma ? 1 : 0;
            chosen->fused = p->fused ? 1 : 0;
            chosen->cells_per_launch = p->cell_batch;
            chosen->ms_per_cell = best / (double)nc;
        }
        return FSTAT_OK;
    });
}

fstat_status fstat_plan_set_timing(fstat_plan *p, int sample_every) {
    return guarded(p, [&]() -> fstat_status {
        if (sample_every < 0) { p->err = "sample_every must be >= 0"; return FSTAT_ERR_ARG; }
        p->timing_every = sample_every;
        p->kstats.clear();
        return FSTAT_OK;
    });
}

fstat_status fstat_plan_kernel_stats(const fstat_plan *p, fstat_kernel_stat *out, int cap, int *n) {
    if (!p || !n || cap < 0 || (cap > 0 && !out)) return FSTAT_ERR_ARG;
    const int m = std::min<int>(cap, (int)p->kstats.size());
    for (int i = 0; i < m; ++i) {
        const auto &k = p->kstats[(size_t)i];
        memset(&out[i], 0, sizeof(fstat_kernel_stat));
        strncpy(out[i].name, k.name.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = k.launches;
        out[i].timed_launches = k.timed;
        out[i].timed_ms = k.ms;
        out[i].flops_per_launch = k.launches ? k.flops / (double)k.launches : 0.0;
        out[i].bytes_per_launch = k.launches ? k.bytes / (double)k.launches : 0.0;
    }
    *n = (int)p->kstats.size();
    return FSTAT_OK;
}

fstat_status fstat_plan_get_info(const fstat_plan *p, fstat_plan_info *info) {
    if (!p || !info) return FSTAT_ERR_ARG;
    info->n_cells = p->n_cells;
    info->f_evals = p->f_evals;
    info->device_bytes = p->device_bytes;
    info->kernel_launches = p->launches;
    info->n_fft_max = p->n_fft_max;
    return FSTAT_OK;
}

void fstat_plan_destroy(fstat_plan *p) {
    if (!p) return;
    free_all(*p);
    delete p;
}

const char *fstat_status_string(fstat_status s) {
    switch (s) {
        case FSTAT_OK: return "ok";
        case FSTAT_ERR_ARG: return "invalid argument";
        case FSTAT_ERR_OOM: return "out of memory";
        case FSTAT_ERR_CUDA: return "CUDA error";
        case FSTAT_ERR_OVERFLOW: return "candidate capacity exceeded";
        case FSTAT_ERR_TIMEOUT: return "device wait timed out";
        case FSTAT_ERR_STATE: return "plan poisoned by an earlier error";
        case FSTAT_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *fstat_plan_error(const fstat_plan *p) { return p ? p->err.c_str() : ""; }

}  // extern "C"
