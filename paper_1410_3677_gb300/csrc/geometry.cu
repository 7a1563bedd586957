// Per-band and per-sky steps of the search (Sect. 2, Fig. 1):
//   per band: noise variance, U-fold FFT upsample of the narrow-band series
//             ("resampling ... using the FFT and splines");
//   per sky:  Roemer delay nhat . r, detector time of every barycentric sample,
//             amplitude modulations a(t), b(t), Keys-cubic resampling and the
//             band-offset phase demodulation ("amplitude and phase
//             demodulation", "resampling", done once per sky position), and the
//             FP64 compensated sums S_aa, S_bb, S_ab.
#include <math.h>

#include "dfloat.cuh"
#include "fstat_internal.h"

namespace fstat {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kOmegaR = kTwoPi / 86164.0905;   // sidereal rotation rate, rad/s

struct KahanD {
    double s = 0.0, c = 0.0;
    __device__ void add(double v) {
        double y = v - c;
        double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over a 256-thread block into thread 0's return value.
__device__ double block_sum256(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// The FP32 form's three S terms at once: each warp adds its 32 terms of each in
// FP32 (relative error ~1e-7), one barrier, then three threads add the block's
// warp sums in FP64 and write the block's partials (blockDim.x = 256); the
// blocks' partials are then added with compensation.  The S sums thus keep FP64
// accumulation where the term count is large, and spend no FP64 instructions per
// sample.
__device__ void block_sum3_f(float a, float b, float c, double *sh, double *out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[w] = (double)a;
        sh[8 + w] = (double)b;
        sh[16 + w] = (double)c;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += sh[8 * threadIdx.x + i];
        out[threadIdx.x] = t;
    }
}

// ------------------------------------------------------------------ sigma^2
__global__ void __launch_bounds__(256) k_sumsq(const double *__restrict__ x, int64_t n,
                                               double *__restrict__ partials) {
    __shared__ double sh[8];
    KahanD k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        k.add(x[i] * x[i]);
    const double s = block_sum256(k.s - k.c, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_sigma2_final(const double *__restrict__ partials, int nblk, int64_t n,
                               double user_sigma2, double *__restrict__ out) {
    KahanD k;
    for (int i = threadIdx.x; i < nblk; i += 32) k.add(partials[i]);
    double s = warp_sum(k.s - k.c);
    if (threadIdx.x == 0) *out = user_sigma2 > 0.0 ? user_sigma2 : s / (double)n;
}

// ------------------------------------------------------------------ geometry
// FP32 form: the delay of sample j reduced once, in double-float arithmetic
// (FP64 runs at 1/64 of the FP32 rate on GB300), to the sample shift
// d_j / dt = I + phi (integer part exact, fraction in FP32) and to the
// band-offset phase f_off d_j mod 1 with its increment f_off (d_{j+1} - d_j), so
// that the detector-time inversion and the phase interpolation run in integer
// and FP32 arithmetic (positions and phases to ~1e-7 samples and cycles).
struct DelayRec {
    int I;
    float phi, psi, dpsi;
};

struct GeoArgs {
    const double *r;
    const double *d;          // per-sample delays of the sky batch, [sky][stride]
    const DelayRec *dr;       // FP32 form: the same as shift records
    int64_t d_stride;
    const void *xu;
    int64_t m_up;
    int U;
    int64_t n;
    double dt, inv_dt, f_off, phi0;
    const SkyConst *sky;
    int64_t s0;
    void *w;
    int64_t w_stride;
    double *partials;
    int nblk;
    double *dbg_y, *dbg_a, *dbg_b;
    uint8_t *dbg_mask;
};

// The delay chain is evaluated with explicitly rounded operations (no fused
// multiply-add): the band-offset phase 2 pi f_off d reaches ~1e5 rad, so the
// rounding of d decides the FP64 agreement of F at the 1e-10 level.
__device__ __forceinline__ double delay_at(const double *__restrict__ r, const SkyConst &sc,
                                           int64_t j) {
    return __dadd_rn(__dadd_rn(__dmul_rn(sc.nx, r[3 * j]), __dmul_rn(sc.ny, r[3 * j + 1])),
                     __dmul_rn(sc.nz, r[3 * j + 2]));
}

// Linear interpolation of the delay at fractional sample u from the per-sample
// delays dk; the end segments extend beyond the data.
__device__ __forceinline__ double delay_lin(const double *__restrict__ dk, int64_t n, double u) {
    int64_t j = (int64_t)floor(u);
    j = j < 0 ? 0 : (j > n - 2 ? n - 2 : j);
    const double f = __dsub_rn(u, (double)j);
    const double d0 = dk[j], d1 = dk[j + 1];
    return __dadd_rn(d0, __dmul_rn(f, __dsub_rn(d1, d0)));
}

// Roemer delay nhat . r_k of every sample of skies [s0, s0 + gridDim.y).
__global__ void __launch_bounds__(256) k_delays(const double *__restrict__ r,
                                                const SkyConst *__restrict__ sky, int64_t s0,
                                                int64_t n, int64_t stride,
                                                double *__restrict__ d) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int sl = blockIdx.y;
    if (k < n) d[(int64_t)sl * stride + k] = delay_at(r, sky[s0 + sl], k);
}

// The ephemeris of a band as double-float pairs (once per search of the band).
__global__ void k_split_r(const double *__restrict__ r, int64_t m, DF *__restrict__ r2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) r2[i] = df_from_double(r[i]);
}

// Shift records of every sample of skies [s0, s0 + gridDim.y): the delay
// nhat . r_k and its reductions in double-float arithmetic (about 2^-46
// relative: 1e-11 samples and 1e-9 cycles at the delays and offsets of a
// search, against the 6e-8 of the FP32 results); d_{k+1} of the phase
// increment comes from the next thread (the block's first thread evaluates
// the one past the block).  The increment of the last sample is never used
// (the interpolation segment index is <= n - 2).
__global__ void __launch_bounds__(256) k_delays_split(const DF *__restrict__ r2,
                                                      const SkyConst *__restrict__ sky, int64_t s0,
                                                      int64_t n, int64_t stride, DF inv_dt, DF f_off,
                                                      int phase, DelayRec *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int sl = blockIdx.y;
    __shared__ DF dsh[257];
    const float *nf = sky[s0 + sl].nf;
    const DF nx{nf[0], nf[1]}, ny{nf[2], nf[3]}, nz{nf[4], nf[5]};
    auto delay = [&](int64_t j) {
        const DF *rj = r2 + 3 * j;
        return df_add(df_add(df_mul(nx, rj[0]), df_mul(ny, rj[1])), df_mul(nz, rj[2]));
    };
    const DF dk = k < n ? delay(k) : DF{0.f, 0.f};
    DelayRec o;
    float phi;
    o.I = (int)df_split_floor(df_mul(dk, inv_dt), &phi);
    o.phi = phi;
    o.psi = 0.f;
    o.dpsi = 0.f;
    if (phase) {   // uniform: no phase records for a band at zero offset
        dsh[threadIdx.x] = dk;
        if (threadIdx.x == 0) {
            const int64_t kn = k + blockDim.x;
            dsh[blockDim.x] = kn < n ? delay(kn) : DF{0.f, 0.f};
        }
        __syncthreads();
        float psi;
        df_split_floor(df_mul(f_off, dk), &psi);
        o.psi = psi;
        if (k + 1 < n) {
            const DF dd = df_add(dsh[threadIdx.x + 1], df_neg(dk));
            o.dpsi = (f_off.hi + f_off.lo) * (dd.hi + dd.lo);
        }
    }
    if (k < n) out[(int64_t)sl * stride + k] = o;
}

template <bool FP32>
__global__ void __launch_bounds__(256) k_geometry(GeoArgs g) {
    __shared__ double sh[24];
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int sl = blockIdx.y;
    double saa = 0.0, sbb = 0.0, sab = 0.0;    // FP64 form
    float saa_f = 0.f, sbb_f = 0.f, sab_f = 0.f;   // FP32 form
    if constexpr (FP32) {
        // the sky's constants in FP32, converted once per block
        __shared__ float cf[12];
        if (threadIdx.x < 12) {
            const SkyConst &sc = g.sky[g.s0 + sl];
            const int i = threadIdx.x;
            cf[i] = i < 5 ? (float)sc.A[i] : i < 9 ? (float)sc.B[i - 5]
                  : i == 9 ? (float)(sc.alpha - g.phi0) : i == 10 ? (float)g.dt : 0.f;
        }
        __syncthreads();
        if (k < g.n) {
            // detector time t of barycentric sample k, t = k dt - d(k dt - d(k dt)),
            // as u = t / dt = A - F1: A an exact integer, F1 an FP32 fraction
            const int n = (int)g.n, kk = (int)k;
            const DelayRec *dr = g.dr + (int64_t)sl * g.d_stride;
            const DelayRec rk = dr[kk];
            const int a0 = kk - rk.I;                       // u0 = a0 - phi_k
            const int j0 = min(max(a0 - 1, 0), n - 2);
            const float f0 = (float)(a0 - j0) - rk.phi;     // u0 - j0
            const DelayRec p0 = dr[j0], p1 = dr[j0 + 1];
            const float F1 = p0.phi + f0 * ((float)(p1.I - p0.I) + (p1.phi - p0.phi));
            const int A = kk - p0.I;
            const float fl1 = floorf(-F1);
            int j = A + (int)fl1;
            float f = -F1 - fl1;                            // u - j in [0, 1)
            const int jc = min(max(j, 0), n - 2);
            f += (float)(j - jc);
            j = jc;
            const bool valid = F1 <= (float)A && F1 >= (float)(A - (n - 1));
            // band-offset phase at t, cycles: psi_j + f dpsi_j (mod 1)
            const DelayRec q0 = dr[j];
            const float cyc = q0.psi + f * q0.dpsi;
            const float frs = cyc - rintf(cyc);
            // hour angle h = alpha - phi0 - Omega_r t (|h| < 20 rad, error ~1e-6 rad
            // from t rounded to FP32)
            const float uf = (float)A - F1;
            const float hr = cf[9] - (float)kOmegaR * (uf * cf[10]);
            float s1, c1;
            sincosf(hr, &s1, &c1);
            const float c2 = c1 * c1 - s1 * s1, s2 = 2.f * s1 * c1;
            const float av = cf[0] * c2 + cf[1] * s2 + cf[2] * c1 + cf[3] * s1 + cf[4];
            const float bv = cf[5] * c2 + cf[6] * s2 + cf[7] * c1 + cf[8] * s1;
            float yr = 0.f, yi = 0.f;
            if (valid) {
                // Keys cubic (a = -1/2) at p = U u = U A - U F1 on the upsampled series,
                // periodic indexing (only tap -1 and taps >= U n wrap, a single step)
                const float up = -(float)g.U * F1;
                const float upf = floorf(up);
                const float mu = up - upf;
                const int64_t i0 = (int64_t)g.U * A + (int64_t)upf - 1;
                const float w0 = ((-0.5f * mu + 1.f) * mu - 0.5f) * mu;
                const float w1 = (1.5f * mu - 2.5f) * mu * mu + 1.f;
                const float w2 = ((-1.5f * mu + 2.f) * mu + 0.5f) * mu;
                const float w3 = (0.5f * mu - 0.5f) * mu * mu;
                const float *xu = (const float *)g.xu;
                float x4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t v = i0 + q;
                    x4[q] = xu[v < 0 ? v + g.m_up : (v >= g.m_up ? v - g.m_up : v)];
                }
                const float v = w0 * x4[0] + w1 * x4[1] + w2 * x4[2] + w3 * x4[3];
                float sp, cp;
                sincospif(2.f * frs, &sp, &cp);
                yr = v * cp;
                yi = -v * sp;
                saa_f = av * av;
                sbb_f = bv * bv;
                sab_f = av * bv;
            }
            float4 *w = (float4 *)g.w + (int64_t)sl * g.w_stride;
            w[k] = make_float4(yr * av, yi * av, yr * bv, yi * bv);
            if (g.dbg_y) {
                g.dbg_y[2 * k] = yr; g.dbg_y[2 * k + 1] = yi;
                g.dbg_a[k] = av; g.dbg_b[k] = bv; g.dbg_mask[k] = valid;
            }
        }
    } else if (k < g.n) {
        const SkyConst sc = g.sky[g.s0 + sl];
        // detector time t of barycentric sample k: t = k dt - d(k dt - d(k dt)),
        // in the oracle's rounding sequence, for 1e-10 agreement of F
        const double *dd = g.d + (int64_t)sl * g.d_stride;
        const double dk = dd[k];
        const double u0 = __dsub_rn((double)k, __ddiv_rn(dk, g.dt));
        const double d1 = delay_lin(dd, g.n, u0);
        const double u = __dsub_rn((double)k, __ddiv_rn(d1, g.dt));
        const double d2 = delay_lin(dd, g.n, u);
        const bool valid = (u >= 0.0) && (u <= (double)(g.n - 1));
        // Keys cubic (a = -1/2) on the upsampled series, periodic indexing
        const double p = (double)g.U * u;
        const double pf = floor(p);
        // taps i0 .. i0 + 3 around floor(p), periodic: inside the window p lies in
        // [0, U (n - 1)], so only i0 = -1 and indices >= U n wrap (a single step)
        int64_t idx[4];
        if (valid) {
            const int64_t i0 = (int64_t)pf - 1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t v = i0 + q;
                idx[q] = v < 0 ? v + g.m_up : (v >= g.m_up ? v - g.m_up : v);
            }
        }
        // band-offset phase, cycles, reduced in FP64
        const double cyc = __dmul_rn(g.f_off, d2);
        const double fr = __dsub_rn(cyc, floor(cyc));
        {
            const double h = sc.alpha - (g.phi0 + kOmegaR * (u * g.dt));
            double s1, c1;
            sincos(h, &s1, &c1);
            const double c2 = c1 * c1 - s1 * s1, s2 = 2.0 * s1 * c1;
            const double av = sc.A[0] * c2 + sc.A[1] * s2 + sc.A[2] * c1 + sc.A[3] * s1 + sc.A[4];
            const double bv = sc.B[0] * c2 + sc.B[1] * s2 + sc.B[2] * c1 + sc.B[3] * s1;
            double yr = 0.0, yi = 0.0;
            if (valid) {
                const double mu = p - pf;
                const double w0 = ((-0.5 * mu + 1.0) * mu - 0.5) * mu;
                const double w1 = (1.5 * mu - 2.5) * mu * mu + 1.0;
                const double w2 = ((-1.5 * mu + 2.0) * mu + 0.5) * mu;
                const double w3 = (0.5 * mu - 0.5) * mu * mu;
                const double *xu = (const double *)g.xu;
                const double v = w0 * xu[idx[0]] + w1 * xu[idx[1]] + w2 * xu[idx[2]] + w3 * xu[idx[3]];
                double sp, cp;
                sincospi(2.0 * fr, &sp, &cp);
                yr = v * cp;
                yi = -v * sp;
                saa = av * av;
                sbb = bv * bv;
                sab = av * bv;
            }
            // {y a, y b} as two double2 (32 bytes per sample)
            double2 *w = (double2 *)g.w + 2 * ((int64_t)sl * g.w_stride + k);
            w[0] = make_double2(yr * av, yi * av);
            w[1] = make_double2(yr * bv, yi * bv);
            if (g.dbg_y) {
                g.dbg_y[2 * k] = yr; g.dbg_y[2 * k + 1] = yi;
                g.dbg_a[k] = av; g.dbg_b[k] = bv; g.dbg_mask[k] = valid;
            }
        }
    }
    double *o = g.partials + ((int64_t)sl * g.nblk + blockIdx.x) * 3;
    if constexpr (FP32) {
        block_sum3_f(saa_f, sbb_f, sab_f, sh, o);
    } else {
        const double ta = block_sum256(saa, sh);
        const double tb = block_sum256(sbb, sh);
        const double tab = block_sum256(sab, sh);
        if (threadIdx.x == 0) {
            o[0] = ta; o[1] = tb; o[2] = tab;
        }
    }
}

// S sums per sky (Kahan over the block partials) and the normalisations
// 1/(sigma^2 S_aa), 1/(sigma^2 S_bb).
__global__ void k_reduce_norms(const double *__restrict__ partials, int nblk,
                               const double *__restrict__ sigma2, double *__restrict__ S,
                               double *__restrict__ norm, int full) {
    const int sl = blockIdx.x;
    double out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        KahanD k;
        for (int i = threadIdx.x; i < nblk; i += 32) k.add(partials[((int64_t)sl * nblk + i) * 3 + c]);
        out[c] = warp_sum(k.s - k.c);
    }
    if (threadIdx.x == 0) {
        const double s2 = *sigma2;
        S[3 * sl] = out[0];
        S[3 * sl + 1] = out[1];
        S[3 * sl + 2] = out[2];
        // F = na |F_a|^2 + nb |F_b|^2 + nab Re(F_a conj F_b)
        double na = 0.0, nb = 0.0, nab = 0.0;
        if (full) {
            const double D = out[0] * out[1] - out[2] * out[2];
            if (D > 0.0) {
                na = out[1] / (s2 * D);
                nb = out[0] / (s2 * D);
                nab = -2.0 * out[2] / (s2 * D);
            }
        } else {
            na = out[0] > 0.0 ? 1.0 / (s2 * out[0]) : 0.0;
            nb = out[1] > 0.0 ? 1.0 / (s2 * out[1]) : 0.0;
        }
        norm[kNormStride * sl] = na;
        norm[kNormStride * sl + 1] = nb;
        norm[kNormStride * sl + 2] = nab;
        norm[kNormStride * sl + 3] = 0.0;
        // FP32 copies for the FP32 epilogues (no conversion in every CTA)
        float *nf = reinterpret_cast<float *>(norm + kNormStride * sl + 4);
        nf[0] = (float)na;
        nf[1] = (float)nb;
        nf[2] = (float)nab;
        nf[3] = 0.f;
    }
}

// ------------------------------------------------------------------ FFT upsample
__global__ void k_real_to_cplx(const double *__restrict__ x, int64_t n, double2 *__restrict__ z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = make_double2(x[i], 0.0);
}

// Bluestein: c_m = e^{dir i pi (m^2 mod 2n)/n}; A = in * c (zero beyond n);
// B = conj(c) wrapped around M so that the circular convolution is linear.
__global__ void k_blue_prep(const double2 *__restrict__ in, int64_t n, int64_t M, int dir,
                            double2 *__restrict__ A, double2 *__restrict__ B) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    int64_t mm = -1;
    if (m < n) mm = m;
    else if (m > M - n) mm = M - m;
    if (mm >= 0) {
        const int64_t q = (mm * mm) % (2 * n);
        double s, c;
        sincospi((double)dir * (double)q / (double)n, &s, &c);
        b = make_double2(c, -s);
        if (m < n) {
            const double2 v = in[m];
            a = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
        }
    }
    A[m] = a;
    B[m] = b;
}

__global__ void k_cmul_inplace(double2 *__restrict__ A, const double2 *__restrict__ B, int64_t M) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double2 a = A[m], b = B[m];
    A[m] = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_blue_post(const double2 *__restrict__ A, int64_t n, int64_t M, int dir,
                            double2 *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t q = (k * k) % (2 * n);
    double s, c;
    sincospi((double)dir * (double)q / (double)n, &s, &c);
    const double2 v = A[k];
    const double inv = 1.0 / (double)M;
    out[k] = make_double2((v.x * c - v.y * s) * inv, (v.x * s + v.y * c) * inv);
}

// Spectrum of the s-th sub-phase of the U-fold interpolant: Y_m = X_m e^{2 pi i m s/(U n)}
// over signed frequencies; the Nyquist bin of an even n contributes X cos(pi s / U).
__global__ void k_shift_spectrum(const double2 *__restrict__ X, int64_t n, int s, int U,
                                 double2 *__restrict__ Y) {
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double2 v = X[m];
    if ((n % 2 == 0) && m == n / 2) {
        double c = cospi((double)s / (double)U);
        Y[m] = make_double2(v.x * c, v.y * c);
        return;
    }
    const int64_t ms = (2 * m < n) ? m : m - n;
    const int64_t un = (int64_t)U * n;
    int64_t q = (ms * s) % un;
    if (q < 0) q += un;
    double sn, cs;
    sincospi(2.0 * (double)q / (double)un, &sn, &cs);
    Y[m] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

template <typename TO>
__global__ void k_scatter_sub(const double2 *__restrict__ z, const double *__restrict__ x, int64_t n,
                              int U, int s, TO *__restrict__ xu) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    xu[(int64_t)U * k + s] = (TO)(s == 0 ? x[k] : z[k].x / (double)n);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ================================================================== launchers
int launch_split_r(const BandDev &b, cudaStream_t s) {
    const int64_t m = 3 * b.n;
    k_split_r<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(b.r, m, static_cast<DF *>(b.r2));
    return 1;
}

int launch_sigma2(const double *x, int64_t n, double user_sigma2, double *partials,
                  double *out, cudaStream_t s) {
    constexpr int nblk = 256;
    k_sumsq<<<nblk, 256, 0, s>>>(x, n, partials);
    k_sigma2_final<<<1, 32, 0, s>>>(partials, nblk, n, user_sigma2, out);
    return 2;
}

int launch_bluestein(const TwiddleSet &twm, int dir, const double *in, double *out, int64_t n,
                     double *work, void *scratch, cudaStream_t s) {
    const int64_t M = (int64_t)1 << twm.logn;
    double2 *A = reinterpret_cast<double2 *>(work);
    double2 *B = A + M;
    int L = 0;
    k_blue_prep<<<blocks(M, 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(in), n, M, dir,
                                                A, B);
    ++L;
    L += launch_fft_generic(twm, true, -1, A, A, 2, scratch, s);
    k_cmul_inplace<<<blocks(M, 256), 256, 0, s>>>(A, B, M);
    ++L;
    L += launch_fft_generic(twm, true, +1, A, A, 1, scratch, s);
    k_blue_post<<<blocks(n, 256), 256, 0, s>>>(A, n, M, dir, reinterpret_cast<double2 *>(out));
    ++L;
    return L;
}

static int dft_any(const Plan &p, int64_t n, int dir, double2 *z, double *work, cudaStream_t s) {
    const bool pow2 = (n & (n - 1)) == 0 && n >= (1 << kMinLogN);
    if (pow2) {
        int lg = 0;
        while ((int64_t(1) << lg) < n) ++lg;
        return launch_fft_generic(*p.twiddles(lg), true, dir, z, z, 1, p.scratch, s);
    }
    int lm = kMinLogN;
    while ((int64_t(1) << lm) < 2 * n - 1) ++lm;
    return launch_bluestein(*p.twiddles(lm), dir, reinterpret_cast<double *>(z),
                            reinterpret_cast<double *>(z), n, work, p.scratch, s);
}

int launch_upsample(const Plan &p, const BandDev &b, int U, void *xu, bool xu_fp32,
                    cudaStream_t s) {
    const int64_t n = b.n;
    int L = 0;
    if (U == 1) {
        if (xu_fp32) k_scatter_sub<float><<<blocks(n, 256), 256, 0, s>>>(nullptr, b.x, n, 1, 0, (float *)xu);
        else k_scatter_sub<double><<<blocks(n, 256), 256, 0, s>>>(nullptr, b.x, n, 1, 0, (double *)xu);
        return 1;
    }
    double2 *X = reinterpret_cast<double2 *>(p.bw);
    double2 *Y = X + p.n_max;
    double *work = reinterpret_cast<double *>(Y + p.n_max);
    k_real_to_cplx<<<blocks(n, 256), 256, 0, s>>>(b.x, n, X);
    ++L;
    L += dft_any(p, n, -1, X, work, s);
    for (int sub = 0; sub < U; ++sub) {
        if (sub > 0) {
            k_shift_spectrum<<<blocks(n, 256), 256, 0, s>>>(X, n, sub, U, Y);
            ++L;
            L += dft_any(p, n, +1, Y, work, s);
        }
        if (xu_fp32)
            k_scatter_sub<float><<<blocks(n, 256), 256, 0, s>>>(Y, b.x, n, U, sub, (float *)xu);
        else
            k_scatter_sub<double><<<blocks(n, 256), 256, 0, s>>>(Y, b.x, n, U, sub, (double *)xu);
        ++L;
    }
    return L;
}

int launch_geometry(const Plan &p, const BandDev &b, int64_t s0, int64_t ns, bool fp32,
                    void *w, double *dbg_y, double *dbg_a, double *dbg_b, uint8_t *dbg_mask,
                    cudaStream_t s) {
    GeoArgs g;
    g.r = b.r;
    g.d = p.dbuf;
    g.dr = reinterpret_cast<const DelayRec *>(p.dbuf);
    g.d_stride = p.n_max;
    g.xu = b.xu;
    g.U = p.desc.upsample;
    g.m_up = (int64_t)g.U * b.n;
    g.n = b.n;
    g.dt = b.dt;
    g.inv_dt = 1.0 / b.dt;
    g.f_off = b.f_off;
    g.phi0 = b.phi0;
    g.sky = p.sky;
    g.s0 = s0;
    g.w = w;
    g.w_stride = p.w_stride;
    g.partials = p.partials;
    g.nblk = (int)blocks(b.n, 256);
    g.dbg_y = dbg_y;
    g.dbg_a = dbg_a;
    g.dbg_b = dbg_b;
    g.dbg_mask = dbg_mask;
    dim3 grid(g.nblk, (unsigned)ns);
    if (fp32) {
        k_delays_split<<<grid, 256, 0, s>>>(static_cast<const DF *>(b.r2), p.sky, s0, b.n, p.n_max,
                                            df_from_double(g.inv_dt), df_from_double(b.f_off),
                                            b.f_off != 0.0 ? 1 : 0, reinterpret_cast<DelayRec *>(p.dbuf));
        k_geometry<true><<<grid, 256, 0, s>>>(g);
    } else {
        k_delays<<<grid, 256, 0, s>>>(b.r, p.sky, s0, b.n, p.n_max, p.dbuf);
        k_geometry<false><<<grid, 256, 0, s>>>(g);
    }
    return 2;
}

int launch_reduce_norms(const Plan &p, const BandDev &b, int64_t ns, double *norm, cudaStream_t s) {
    k_reduce_norms<<<(unsigned)ns, 32, 0, s>>>(p.partials, (int)blocks(b.n, 256), b.sigma2, p.S,
                                               norm, p.desc.statistic == FSTAT_F_FULL ? 1 : 0);
    return 1;
}

}  // namespace fstat
