// The two FP32 search passes on the second FFT engine (one transform per thread
// group, 32 elements per thread, two register stages per pass).  Same four-step
// split and scratch layout as the first engine's passes: pass 1 transforms the
// columns k1 (length N2) of the demodulated series and writes them, twiddled by
// W_N^{k1 l2} and transposed, to scratch; pass 2 transforms the rows l2 (length
// N1) and evaluates F on every bin it produces.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine2.cuh"
#include "fstat_internal.h"

namespace fstat {

template <int LOGN, int PASS>
struct Cfg2 {
    static constexpr int LOGN1 = LOGN / 2;
    static constexpr int LOGN2 = LOGN - LOGN / 2;
    static constexpr int N1 = 1 << LOGN1;
    static constexpr int N2 = 1 << LOGN2;
    static constexpr int N = 1 << LOGN;
    static constexpr int M = PASS == 1 ? N2 : N1;        // length of this pass's FFTs
    static constexpr int OTHER = PASS == 1 ? N1 : N2;    // number of such FFTs per transform
    static constexpr int EH = 32;
    static constexpr int TPF = M / EH;
    static constexpr int SEQ0 = 256 / TPF;
    static constexpr int SEQ = SEQ0 < 2 * OTHER ? SEQ0 : 2 * OTHER;   // sequences per tile
    static constexpr int F = SEQ / 2;                    // columns / rows per tile
    static constexpr int THREADS = SEQ * TPF;
    static constexpr int TILES = OTHER / F;
    static constexpr size_t SMEM = eng2::smem_bytes<float, M, SEQ>();
    static_assert(M >= 64 && THREADS == 256, "tile shape");
};

// Pass 1 input: w[k] = (y a, y b) of one sky as float4, read as the float2 half
// t; z = w e^{-2 pi i phi_k}, phi_k = frac(fdot dt^2 k^2 / 2) from a 64-bit
// fixed-point product, zero for k >= n.
template <class C>
struct SearchLoad2 {
    const float4 *w;
    int64_t w_stride;
    int n;
    const uint64_t *chirp;
    int n_spin;
    int64_t c0, s0;
    const float2 *ws;
    uint64_t afx;
    int k1_0;
    __device__ void init() {
        const int64_t c = c0 + blockIdx.y;
        const int64_t sky = c / n_spin;
        ws = reinterpret_cast<const float2 *>(w + (sky - s0) * w_stride);
        afx = chirp[c - sky * n_spin];
        k1_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        const int kb = k1_0 + q.f + C::N1 * q.j;
#pragma unroll
        for (int r = 0; r < R; ++r) {      // loads first: all in flight together
            const int k = kb + C::N1 * JPF * r;
            float2 v = make_float2(0.f, 0.f);
            if (k < n) v = __ldg(ws + 2 * k + q.t);
            re[r] = v.x; im[r] = v.y;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t k = (uint32_t)(kb + C::N1 * JPF * r);
            if (k < (uint32_t)n) {        // the zero padding needs no phase
                const uint64_t kk = (uint64_t)k * (uint64_t)k;
                const int32_t top = (int32_t)((afx * kk) >> 32);          // cycles in [-1/2, 1/2)
                const float ph = (float)top * 1.4629180792671596e-09f;    // 2 pi / 2^32
                float s, c;
                __sincosf(ph, &s, &c);
                const float x = re[r], y = im[r];
                re[r] = x * c + y * s;
                im[r] = y * c - x * s;
            }
        }
    }
};

// Pass 1 output: twiddle W_N^{k1 l2}, l2 = j + r JPF, as W^{k1 j} (W^{k1 JPF})^r
// (two lookups W_N^m = hi[m >> log N1] lo[m & (N1 - 1)] per job), then the
// transposed store A_t[l2][k1] into scratch slot blockIdx.y.
template <class C>
struct ScratchStore2 {
    float2 *scratch;
    const float *lo, *hi;
    float2 *base;
    int k1_0;
    __device__ void init() {
        base = scratch + (int64_t)blockIdx.y * 2 * C::N;
        k1_0 = blockIdx.x * C::F;
    }
    __device__ __forceinline__ float2 wn(int m) const {
        const float2 th = __ldg(reinterpret_cast<const float2 *>(hi) + (m >> C::LOGN1));
        const float2 tl = __ldg(reinterpret_cast<const float2 *>(lo) + (m & (C::N1 - 1)));
        return float2{th.x * tl.x - th.y * tl.y, th.x * tl.y + th.y * tl.x};
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(const eng2::Job &q, float *re, float *im) const {
        const int k1 = k1_0 + q.f;
        float2 w = wn(k1 * q.j);
        const float2 st = wn(k1 * JPF);
        float2 *dst = base + (int64_t)q.t * C::N + (int64_t)q.j * C::N1 + k1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float xr = re[r], xi = im[r];
            dst[(int64_t)r * JPF * C::N1] = float2{xr * w.x - xi * w.y, xr * w.y + xi * w.x};
            if (r + 1 < R) w = float2{w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x};
        }
    }
};

// Pass 2 input: row l2 of transform t from scratch slot blockIdx.y.
template <class C>
struct ScratchLoad2 {
    const float2 *scratch;
    const float2 *base;
    int l2_0;
    __device__ void init() {
        base = scratch + (int64_t)blockIdx.y * 2 * C::N;
        l2_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        const float2 *row = base + (int64_t)q.t * C::N + (int64_t)(l2_0 + q.f) * C::N1 + q.j;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 v = row[r * JPF];
            re[r] = v.x; im[r] = v.y;
        }
    }
};

// Pass 2 output: F = |F_a|^2/(sigma^2 S_aa) + |F_b|^2/(sigma^2 S_bb) per bin
// (Fig. 1, "F-statistics calculation"), strict 2F > thr, appended with one
// atomic per warp and output slot.  Lanes l (F_a) and l ^ 16 (F_b) hold the same
// bins; each forms |.|^2 of its own values and trades half of them with its
// partner, so the a lane evaluates F on the first half of the outputs and the b
// lane on the second.  LOWER: the bin range lies below N/2, so only the outputs
// l1 < N1/2 (r < R/2) are used and the rest of the last DFT is never computed.
template <class C, bool LOWER>
struct SearchEpi2 {
    const double *norm;      // [sky_local][2]
    int n_spin;
    int64_t c0, s0;
    uint32_t cell_base;      // first global cell index of this band
    int64_t bin_lo, bin_hi;
    float thr;
    CandRecord *out;
    unsigned long long *count;
    unsigned long long cap;
    float na, nb, thr_half;
    uint32_t cell;
    int l2_0;
    __device__ void init() {
        const int64_t c = c0 + blockIdx.y;
        const int64_t sky = c / n_spin;
        na = (float)norm[2 * (sky - s0)];
        nb = (float)norm[2 * (sky - s0) + 1];
        cell = cell_base + (uint32_t)c;
        l2_0 = blockIdx.x * C::F;
        thr_half = 0.5f * thr;   // 2F > thr  <=>  F > thr / 2, both sides exact
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(const eng2::Job &q, float *re, float *im) const {
        constexpr int H = (LOWER ? R / 2 : R) / 2;   // values per lane
        const int lane = threadIdx.x & 31;
        float Fv[H];
        bool pr[H];
        bool any = false;
        // bins < 2^19: 32-bit arithmetic; lo <= bin <= hi as one unsigned compare
        const int bin0 = C::N2 * (q.j + q.t * H * JPF) + l2_0 + q.f;
        const int lo = (int)bin_lo;
        const unsigned span = (unsigned)(bin_hi - bin_lo);
#pragma unroll
        for (int r = 0; r < H; ++r) {
            // this lane's |x|^2 at outputs r (a lane's bins) and r + H (b lane's)
            const float p_lo = re[r] * re[r] + im[r] * im[r];
            const float p_hi = re[r + H] * re[r + H] + im[r + H] * im[r + H];
            const float other = __shfl_xor_sync(0xffffffffu, q.t == 0 ? p_hi : p_lo, 16);
            Fv[r] = q.t == 0 ? p_lo * na + other * nb : other * na + p_hi * nb;
            const unsigned off = (unsigned)(bin0 + r * C::N2 * JPF - lo);
            pr[r] = (off <= span) && (Fv[r] > thr_half);
            any |= pr[r];
        }
        if (!__any_sync(0xffffffffu, any)) return;
#pragma unroll
        for (int r = 0; r < H; ++r) {
            const unsigned m = __ballot_sync(0xffffffffu, pr[r]);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b0 = 0;
                if (lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(m));
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (pr[r]) {
                    const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
                    if (idx < cap) out[idx] = CandRecord{cell, (uint32_t)(bin0 + r * C::N2 * JPF), (double)Fv[r]};
                }
            }
        }
    }
};

// Pass 2 holds fewer live values (no demodulation, no twiddle powers) and fits
// three CTAs per SM (<= 85 registers, 3 x 68 KB of shared memory); pass 1 two.
template <int LOGN, int PASS, int MAPM, class LD, class ST>
__global__ void __launch_bounds__(256, PASS == 2 ? 3 : 2) k_pass2(LD ld, ST st, const float *__restrict__ tw) {
    using C = Cfg2<LOGN, PASS>;
    ld.init();
    st.init();
    eng2::run_pass<float, C::M, C::SEQ, C::EH, -1, MAPM>(ld, st, tw);
}

}  // namespace fstat
