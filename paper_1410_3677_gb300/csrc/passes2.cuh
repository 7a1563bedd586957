// The two FP32 search passes on the second FFT engine (one transform per thread
// group, 32 elements per thread, two register stages per pass).  Same four-step
// split and scratch layout as the first engine's passes: pass 1 transforms the
// columns k1 (length N2) of the demodulated series and writes them transposed to
// scratch; pass 2 twiddles the rows l2 by W_N^{k1 l2}, transforms them (length
// N1) and evaluates F on every bin it produces.  Scratch holds the two
// transforms interleaved, A[l2][k1][t] (t = 0: F_a, 1: F_b), so a warp's store
// of 8 columns of both transforms is one 128-byte run and a pass-2 tile of rows
// is one contiguous block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine2.cuh"
#include "fstat_internal.h"
#include "sync_ptx.cuh"

namespace fstat {

template <int LOGN, int PASS, int TS = 256>
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
    static constexpr int SEQ0 = TS / TPF;
    static constexpr int SEQ = SEQ0 < 2 * OTHER ? SEQ0 : 2 * OTHER;   // sequences per tile
    static constexpr int F = SEQ / 2;                    // columns / rows per tile
    static constexpr int THREADS = SEQ * TPF;
    static constexpr int TILES = OTHER / F;
    static constexpr size_t SMEM = eng2::smem_bytes<float, M, SEQ, PASS == 1 && eng2::x16_layout(M, EH)>();
    static constexpr int MINB = 768 / TS;                // CTAs per SM (24 warps)
    static_assert(M >= 64 && THREADS == TS, "tile shape");
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
    // tile: column block; cell: cell of the launch; slot: scratch slot
    __device__ void init(int tile, int64_t cell, int64_t) {
        const int64_t c = c0 + cell;
        const int64_t sky = (int64_t)((uint32_t)c / (uint32_t)n_spin);   // cells < 2^32: 32-bit divide
        ws = reinterpret_cast<const float2 *>(w + (sky - s0) * w_stride);
        afx = chirp[c - sky * n_spin];
        k1_0 = tile * C::F;
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

// The same input with the spindown phase shared by the two lanes of a column
// (column mapping: lanes 2f and 2f + 1 hold the a and b halves of the same
// samples): each lane evaluates the phase of every other element, r = 2 i + t,
// and both read each element's (cos, sin) from the lane that evaluated it.
template <class C>
struct SearchLoad2S : SearchLoad2<C> {
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        static_assert(R % 2 == 0, "elements in pairs");
        const int kb = this->k1_0 + q.f + C::N1 * q.j;
#pragma unroll
        for (int r = 0; r < R; ++r) {      // loads first: all in flight together
            const int k = kb + C::N1 * JPF * r;
            float2 v = make_float2(0.f, 0.f);
            if (k < this->n) v = __ldg(this->ws + 2 * k + q.t);
            re[r] = v.x; im[r] = v.y;
        }
        float cs[R / 2], sn[R / 2];
        const int kt = kb + C::N1 * JPF * q.t;
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {   // this lane's half of the phases
            const uint32_t k = (uint32_t)(kt + C::N1 * JPF * 2 * i);
            const uint64_t kk = (uint64_t)k * (uint64_t)k;
            const int32_t top = (int32_t)((this->afx * kk) >> 32);   // cycles in [-1/2, 1/2)
            __sincosf((float)top * 1.4629180792671596e-09f, &sn[i], &cs[i]);   // 2 pi / 2^32
        }
        const int lane = (int)threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int src = (lane & ~1) | (r & 1);   // the lane that evaluated element r
            const float c = __shfl_sync(0xffffffffu, cs[r / 2], src);
            const float sv = __shfl_sync(0xffffffffu, sn[r / 2], src);
            const uint32_t k = (uint32_t)(kb + C::N1 * JPF * r);
            if (k < (uint32_t)this->n) {
                const float x = re[r], y = im[r];
                re[r] = x * c + y * sv;
                im[r] = y * c - x * sv;
            }
        }
    }
};

// The four-step twiddle W_N^{k1 l2} between the passes, applied by the pass-2
// loaders to the elements k1 = j + r JPF of row l2 as W^{l2 j} (W^{l2 JPF})^r,
// the two factors from the tables W_N^m = hi[m >> log N1] lo[m & (N1 - 1)].
// Pass 1 is bound by instruction issue and pass 2 by its DRAM reads, so the
// multiplies sit in the pass that has issue slots to spare.
template <int LOGN1>
struct InterTw {
    const float *lo, *hi;
    __device__ __forceinline__ float2 wn(int m) const {
        const float2 th = __ldg(reinterpret_cast<const float2 *>(hi) + (m >> LOGN1));
        const float2 tl = __ldg(reinterpret_cast<const float2 *>(lo) + (m & ((1 << LOGN1) - 1)));
        return float2{th.x * tl.x - th.y * tl.y, th.x * tl.y + th.y * tl.x};
    }
    template <int R, int JPF>
    __device__ __forceinline__ void apply(int l2, int j, float *re, float *im) const {
        apply<R>(wn(l2 * j), wn(l2 * JPF), re, im);
    }
    // the same with the two factors W^{l2 j}, W^{l2 JPF} fetched beforehand
    template <int R>
    __device__ __forceinline__ void apply(float2 w, const float2 st, float *re, float *im) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float xr = re[r], xi = im[r];
            re[r] = xr * w.x - xi * w.y;
            im[r] = xr * w.y + xi * w.x;
            if (r + 1 < R) w = float2{w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x};
        }
    }
};

// Pass 1 output: the transposed store A_t[l2][k1], l2 = j + r JPF, into the
// cell's scratch slot.  Scratch is written and read through L2 only
// (st.global.cg / ld.global.cg): it is streamed once each way, and a slot reused
// within one launch never meets a stale L1 line.
template <class C>
struct ScratchStore2 {
    static constexpr bool kStoreEarly = true;
    float2 *scratch;
    float2 *base;
    int k1_0;
    __device__ void init(int tile, int64_t, int64_t slot) {
        base = scratch + slot * 2 * C::N;
        k1_0 = tile * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(const eng2::Job &q, float *re, float *im) const {
        float2 *dst = base + 2 * ((int64_t)q.j * C::N1 + k1_0 + q.f) + q.t;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            __stcg(dst, float2{re[r], im[r]});
            dst += 2 * JPF * C::N1;
        }
    }
};

// Pass 2 input: row l2 of transform t from the cell's scratch slot.
template <class C>
struct ScratchLoad2 {
    const float2 *scratch;
    int64_t pf_dist;     // two-launch form: prefetch the tile this many CTAs ahead (0: off)
    InterTw<C::LOGN1> tw;
    const float2 *base;
    int l2_0;
    __device__ void init(int tile, int64_t, int64_t slot) {
        base = scratch + slot * 2 * C::N;
        l2_0 = tile * C::F;
    }
    // The rows of the tile `pf_dist` CTAs further in launch order go to L2 ahead of
    // their CTA (one contiguous run of F rows of both transforms), so the DRAM
    // reads of pass 2 run behind its computation instead of at the start of
    // every CTA.
    __device__ void prefetch_ahead() const {
        if (pf_dist <= 0 || threadIdx.x != 0) return;
        const int64_t b = blockIdx.x + (int64_t)gridDim.x * blockIdx.y + pf_dist;
        const int64_t total = (int64_t)gridDim.x * gridDim.y;
        if (b >= total) return;
        const int64_t slot = (uint32_t)b / gridDim.x;   // b < 2^32
        const int tile = (int)((uint32_t)b - (uint32_t)slot * gridDim.x);
        const float2 *rows = scratch + slot * 2 * C::N + 2 * (int64_t)tile * C::F * C::N1;
        ptx::bulk_prefetch_l2(rows, (uint32_t)(2 * C::F * C::N1 * sizeof(float2)));
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        const float2 *row = base + 2 * ((int64_t)(l2_0 + q.f) * C::N1 + q.j) + q.t;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 v = __ldcg(row + 2 * r * JPF);
            re[r] = v.x; im[r] = v.y;
        }
        tw.template apply<R, JPF>(l2_0 + q.f, q.j, re, im);
    }
};

// Pass 2 input staged by the TMA unit: the tile's rows are one contiguous run of
// 2 F N1 complex floats in scratch (both transforms interleaved); one thread
// copies it into the CTA's exchange area with a bulk copy completing on an
// mbarrier, and the threads then read their butterflies' elements from shared
// memory (a warp reads 32 consecutive elements, F_a and F_b alternating:
// conflict-free).
// The run_pass of a staged loader synchronises the CTA before the first scatter
// overwrites the staged rows.
template <class C>
struct ScratchLoadTMA {
    static constexpr bool kStaged = true;
    const float2 *scratch;
    int64_t pf_dist;        // see ScratchLoad2::prefetch_ahead
    uint32_t *err;          // set when the copy does not complete within 1 s
    InterTw<C::LOGN1> tw;
    int l2_0;
    const float2 *src;
    const float2 *rows;     // staged rows in shared memory: [f][N1][t]
    uint64_t *bar;
    __device__ void init(int tile, int64_t, int64_t slot) {
        src = scratch + slot * 2 * C::N + 2 * (int64_t)tile * C::F * C::N1;
        l2_0 = tile * C::F;
        unsigned char *sm = eng2::dyn_smem();
        rows = reinterpret_cast<const float2 *>(sm);
        bar = reinterpret_cast<uint64_t *>(sm + C::SMEM);
    }
    __device__ void prefetch_ahead() const {
        if (pf_dist <= 0 || threadIdx.x != 0) return;
        const int64_t b = blockIdx.x + (int64_t)gridDim.x * blockIdx.y + pf_dist;
        const int64_t total = (int64_t)gridDim.x * gridDim.y;
        if (b >= total) return;
        const int64_t slot = (uint32_t)b / gridDim.x;   // b < 2^32
        const int tile = (int)((uint32_t)b - (uint32_t)slot * gridDim.x);
        const float2 *r = scratch + slot * 2 * C::N + 2 * (int64_t)tile * C::F * C::N1;
        ptx::bulk_prefetch_l2(r, (uint32_t)(2 * C::F * C::N1 * sizeof(float2)));
    }
    // issue the copy (the whole CTA calls this once, before run_pass)
    __device__ void stage() const {
        constexpr uint32_t bytes = (uint32_t)(2 * C::F * C::N1 * sizeof(float2));
        static_assert(bytes <= eng2::exch_bytes<float, C::M, C::SEQ>(), "staged rows fit the exchange area");
        if (threadIdx.x == 0) {
            ptx::mbar_init(bar, 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ptx::mbar_arrive_expect_tx(bar, bytes);
            ptx::bulk_g2s(const_cast<float2 *>(rows), src, bytes, bar);
        }
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        // the twiddle factors load while the bulk copies are in flight
        const int l2 = l2_0 + q.f;
        const float2 w0 = tw.wn(l2 * q.j), st = tw.wn(l2 * JPF);
        if (!ptx::mbar_try_wait(bar, 0)) {
            const uint64_t t0 = ptx::globaltimer_ns();
            bool late = false;
            while (!ptx::mbar_try_wait(bar, 0)) {
                const uint64_t dt = ptx::globaltimer_ns() - t0;
                if (!late && dt > 1000000000ull) { atomicExch(err, 1u); late = true; }
                if (dt > 2000000000ull) break;   // reported above; results are discarded
            }
        }
        const float2 *row = rows + 2 * (q.f * C::N1 + q.j) + q.t;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 v = row[2 * r * JPF];
            re[r] = v.x; im[r] = v.y;
        }
        tw.template apply<R>(w0, st, re, im);
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
    const double *norm;      // per local sky (stride kNormStride): na, nb, nab (F = na|F_a|^2 + nb|F_b|^2
                             // + nab Re F_a F_b*) in FP64, then the same as floats
    int n_spin;
    int64_t c0, s0;
    uint32_t cell_base;      // first global cell index of this band
    int64_t bin_lo, bin_hi;
    float thr;
    CandRecord *out;
    unsigned long long *count;
    unsigned long long cap;
    float na, nb, nab, thr_half;
    uint32_t cell;
    int l2_0;
    __device__ void init(int tile, int64_t cl, int64_t) {
        const int64_t c = c0 + cl;
        const int64_t sky = (int64_t)((uint32_t)c / (uint32_t)n_spin);   // cells < 2^32: 32-bit divide
        const float *nf = reinterpret_cast<const float *>(norm + kNormStride * (sky - s0) + 4);
        na = nf[0];
        nb = nf[1];
        nab = nf[2];
        cell = cell_base + (uint32_t)c;
        l2_0 = tile * C::F;
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
        const bool full = nab != 0.f;   // the same for the whole grid
#pragma unroll
        for (int r = 0; r < H; ++r) {
            if (full) {   // the partner's complex value: the cross term needs it
                const float sr = q.t == 0 ? re[r + H] : re[r], si = q.t == 0 ? im[r + H] : im[r];
                const float orr = __shfl_xor_sync(0xffffffffu, sr, 16);
                const float oi = __shfl_xor_sync(0xffffffffu, si, 16);
                const float ar = q.t == 0 ? re[r] : orr, ai = q.t == 0 ? im[r] : oi;
                const float br = q.t == 0 ? orr : re[r + H], bi = q.t == 0 ? oi : im[r + H];
                Fv[r] = (ar * ar + ai * ai) * na + (br * br + bi * bi) * nb + (ar * br + ai * bi) * nab;
            } else {
                // this lane's |x|^2 at outputs r (a lane's bins) and r + H (b lane's)
                const float p_lo = re[r] * re[r] + im[r] * im[r];
                const float p_hi = re[r + H] * re[r + H] + im[r + H] * im[r + H];
                const float other = __shfl_xor_sync(0xffffffffu, q.t == 0 ? p_hi : p_lo, 16);
                Fv[r] = q.t == 0 ? p_lo * na + other * nb : other * na + p_hi * nb;
            }
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

// Pass 1: three CTAs of 256 threads per SM (<= 85 registers, about 70 KB of
// shared memory each); pass 2: six CTAs of 128 threads.
// Z1: eighths of each pass-1 column that can be non-zero.  Pass 1 of a search
// transform (N_fft >= 2n) reads only the first half of each column (Z1 = 4):
// elements k2 >= N2/2 lie at k >= N/2 >= n, in the zero padding; with
// n <= 3N/8 and a radix-32 first stage only the first three eighths (Z1 = 3);
// Z1 = 8: a transform only as long as the series allows (the half-length
// transform of the interbinning form, N >= n but not N >= 2n).
template <int LOGN, int PASS, int MAPM, class LD, class ST, int TS = 256, int Z1 = 4>
__global__ void __launch_bounds__(TS, 768 / TS) k_pass2(LD ld, ST st, const float *__restrict__ tw) {
    using C = Cfg2<LOGN, PASS, TS>;
    if constexpr (PASS == 2) ld.prefetch_ahead();
    ld.init(blockIdx.x, blockIdx.y, blockIdx.y);
    st.init(blockIdx.x, blockIdx.y, blockIdx.y);
    if constexpr (eng2::LoaderStaged<LD>::value) ld.stage();
    eng2::run_pass<float, C::M, C::SEQ, C::EH, -1, MAPM, LD, ST, PASS == 1 ? Z1 : 8, true>(ld, st, tw);
}

// ------------------------------------------------------------------ interbinning
// The paper's Fourier-transform interpolation to a transform twice as long
// (Sect. 2) as interbinning: the search transform has length N = n_fft / 2 and
// output bin 2k of the n_fft grid is X(k), bin 2k + 1 is (pi/4)(X(k) - X(k + 1)),
// X(N) = X(0).  With k = N2 l1 + l2, X(k + 1) sits in row l2 + 1 (or, for the
// last row, in row 0 at l1 + 1), so a pass-2 tile of F rows starts F - 1 rows
// after the previous one: its last row only serves as the neighbour of the row
// before it.  Rows past N2 are rows of the next l1 (wrapped).

// Pass 2 input of the interbinning form: row (l2_0 + f) mod N2 of transform t.
template <class C>
struct ScratchLoadIB {
    const float2 *scratch;
    InterTw<C::LOGN1> tw;
    const float2 *base;
    int l2_0;
    __device__ void init(int tile, int64_t, int64_t slot) {
        base = scratch + slot * 2 * C::N;
        l2_0 = tile * (C::F - 1);
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        const int l2 = (l2_0 + q.f) & (C::N2 - 1);
        const float2 *row = base + 2 * ((int64_t)l2 * C::N1 + q.j) + q.t;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 v = __ldcg(row + 2 * r * JPF);
            re[r] = v.x; im[r] = v.y;
        }
        tw.template apply<R, JPF>(l2, q.j, re, im);
    }
};

// The same rows staged by the TMA unit: one bulk copy of the rows l2_0 .. N2 - 1
// that the tile holds (both transforms, interleaved) and, for the last tile, one
// of the rows it wraps to from row 0; the tile F - 1 rows ahead is prefetched
// into L2.
template <class C>
struct ScratchLoadIBTMA {
    static constexpr bool kStaged = true;
    const float2 *scratch;
    int64_t pf_dist;
    uint32_t *err;
    InterTw<C::LOGN1> tw;
    const float2 *base;
    const float2 *rows;
    uint64_t *bar;
    int l2_0;
    __device__ void init(int tile, int64_t, int64_t slot) {
        base = scratch + slot * 2 * C::N;
        l2_0 = tile * (C::F - 1);
        unsigned char *sm = eng2::dyn_smem();
        rows = reinterpret_cast<const float2 *>(sm);
        bar = reinterpret_cast<uint64_t *>(sm + C::SMEM);
    }
    __device__ void prefetch_ahead() const {
        if (pf_dist <= 0 || threadIdx.x != 0) return;
        const int64_t b = blockIdx.x + (int64_t)gridDim.x * blockIdx.y + pf_dist;
        const int64_t total = (int64_t)gridDim.x * gridDim.y;
        if (b >= total) return;
        const int64_t slot = (uint32_t)b / gridDim.x;   // b < 2^32
        const int l2 = (int)((uint32_t)b - (uint32_t)slot * gridDim.x) * (C::F - 1);
        const int nr = C::N2 - l2 < C::F ? C::N2 - l2 : C::F;
        const float2 *r = scratch + slot * 2 * C::N + 2 * (int64_t)l2 * C::N1;
        ptx::bulk_prefetch_l2(r, (uint32_t)(2 * nr * C::N1 * sizeof(float2)));
    }
    __device__ void stage() const {
        static_assert(2 * C::F * C::N1 * sizeof(float2) <= eng2::exch_bytes<float, C::M, C::SEQ>(),
                      "staged rows fit the exchange area");
        if (threadIdx.x == 0) {
            ptx::mbar_init(bar, 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int na = C::N2 - l2_0 < C::F ? C::N2 - l2_0 : C::F;   // rows before the wrap
            const uint32_t row_bytes = (uint32_t)(2 * C::N1 * sizeof(float2));   // both transforms
            float2 *dst = const_cast<float2 *>(rows);
            ptx::mbar_arrive_expect_tx(bar, C::F * row_bytes);
            ptx::bulk_g2s(dst, base + 2 * (int64_t)l2_0 * C::N1, na * row_bytes, bar);
            if (na < C::F) ptx::bulk_g2s(dst + 2 * na * C::N1, base, (C::F - na) * row_bytes, bar);
        }
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(const eng2::Job &q, float *re, float *im) const {
        const int l2 = (l2_0 + q.f) & (C::N2 - 1);
        const float2 w0 = tw.wn(l2 * q.j), st = tw.wn(l2 * JPF);
        if (!ptx::mbar_try_wait(bar, 0)) {
            const uint64_t t0 = ptx::globaltimer_ns();
            bool late = false;
            while (!ptx::mbar_try_wait(bar, 0)) {
                const uint64_t dt = ptx::globaltimer_ns() - t0;
                if (!late && dt > 1000000000ull) { atomicExch(err, 1u); late = true; }
                if (dt > 2000000000ull) break;   // reported above; results are discarded
            }
        }
        const float2 *row = rows + 2 * (q.f * C::N1 + q.j) + q.t;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 v = row[2 * r * JPF];
            re[r] = v.x; im[r] = v.y;
        }
        tw.template apply<R>(w0, st, re, im);
    }
};

// Keeps each row's outputs X(l1) in the warp's own exchange row (free once the
// warp has gathered its stage-1 inputs; rows of the warp mapping belong to one
// warp), element l1 at pad(l1).
template <class C>
struct StoreRowsSmem {
    __device__ void init(int, int64_t, int64_t) {}
    template <int R, int JPF>
    __device__ __forceinline__ void store(const eng2::Job &q, float *re, float *im) const {
        __syncwarp();
        float2 *row = reinterpret_cast<float2 *>(eng2::dyn_smem()) + q.s * eng2::row_ld(C::M);
#pragma unroll
        for (int r = 0; r < R; ++r) row[eng2::pad(q.j + r * JPF)] = float2{re[r], im[r]};
    }
};

template <int LOGN, int TS = 256>
struct IBGeom {
    using C = Cfg2<LOGN, 2, TS>;
    static constexpr int STEP = C::F - 1;                    // rows emitted per tile
    static constexpr int TILES = (C::N2 + STEP - 1) / STEP;
};

template <int LOGN, int TS, class LD>
__global__ void __launch_bounds__(TS, 768 / TS)
k_pass2_ib(LD ld, SearchEpi2<Cfg2<LOGN, 2, TS>, false> ep, const float *__restrict__ tw) {
    using C = Cfg2<LOGN, 2, TS>;
    if constexpr (eng2::LoaderStaged<LD>::value) ld.prefetch_ahead();
    ld.init(blockIdx.x, blockIdx.y, blockIdx.y);
    ep.init(0, blockIdx.y, blockIdx.y);
    if constexpr (eng2::LoaderStaged<LD>::value) ld.stage();
    StoreRowsSmem<C> st;
    // stage-1 twiddles from the shared power-of-two rows: the full table through
    // L1 costs this kernel registers (spills) and time
    eng2::run_pass<float, C::M, C::SEQ, C::EH, -1, eng2::kMapW, LD, StoreRowsSmem<C>, 8, false>(ld, st, tw);
    __syncthreads();
    const float2 *X = reinterpret_cast<const float2 *>(eng2::dyn_smem());
    constexpr int RL = eng2::row_ld(C::M);
    constexpr int F = C::F, N1 = C::N1, N2 = C::N2;
    // bins below n_fft / 2 = N only need l1 < N1 / 2 (bin 2k + 1 with k < N / 2 reads
    // X(k + 1) <= X(N / 2), which the transform still produced)
    const int lg1 = ep.bin_hi < (int64_t)C::N ? C::LOGN1 - 1 : C::LOGN1;
    const int PAIRS = (F - 1) << lg1;
    constexpr float Q = 0.78539816339744831f;   // pi / 4
    const int l2_0 = blockIdx.x * (F - 1);
    const int lane = threadIdx.x & 31;
    const bool full = ep.nab != 0.f;
    const int lo = (int)ep.bin_lo;
    const unsigned span = (unsigned)(ep.bin_hi - ep.bin_lo);
#pragma unroll 1
    for (int p0 = 0; p0 < PAIRS; p0 += C::THREADS) {
        const int pr = p0 + (int)threadIdx.x;
        const int f = pr >> lg1, l1 = pr & ((1 << lg1) - 1);
        const int l2 = l2_0 + f;
        const bool own = pr < PAIRS && l2 < N2;
        float Fe = 0.f, Fo = 0.f;
        int k = 0;
        if (own) {
            // neighbour X(k + 1): row f + 1 at l1, or row 0 of l1 + 1 past the last row
            const int l1n = (l2 + 1 == N2) ? ((l1 + 1) & (N1 - 1)) : l1;
            const float2 a0 = X[f * RL + eng2::pad(l1)], b0 = X[(F + f) * RL + eng2::pad(l1)];
            const float2 a1 = X[(f + 1) * RL + eng2::pad(l1n)], b1 = X[(F + f + 1) * RL + eng2::pad(l1n)];
            const float ar = Q * (a0.x - a1.x), ai = Q * (a0.y - a1.y);
            const float br = Q * (b0.x - b1.x), bi = Q * (b0.y - b1.y);
            Fe = (a0.x * a0.x + a0.y * a0.y) * ep.na + (b0.x * b0.x + b0.y * b0.y) * ep.nb;
            Fo = (ar * ar + ai * ai) * ep.na + (br * br + bi * bi) * ep.nb;
            if (full) {
                Fe += (a0.x * b0.x + a0.y * b0.y) * ep.nab;
                Fo += (ar * br + ai * bi) * ep.nab;
            }
            k = N2 * l1 + l2;
        }
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int bin = 2 * k + o;
            const float Fv = o ? Fo : Fe;
            const bool hit = own && (unsigned)(bin - lo) <= span && Fv > ep.thr_half;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b0v = 0;
                if (lane == leader) b0v = atomicAdd(ep.count, (unsigned long long)__popc(m));
                b0v = __shfl_sync(0xffffffffu, b0v, leader);
                if (hit) {
                    const unsigned long long idx = b0v + __popc(m & ((1u << lane) - 1u));
                    if (idx < ep.cap) ep.out[idx] = CandRecord{ep.cell, (uint32_t)bin, (double)Fv};
                }
            }
        }
    }
}

// ------------------------------------------------------------------ fused launch
// Both passes of a batch of cells in one persistent launch fed by a device work
// queue (a ticket counter).  Items run in the order
//   step s: the I1 pass-1 items of cell s, then the I2 pass-2 items of cell s - A
// (A = ahead; an item is tpi tiles), so pass 2 of a cell starts A cells after its
// pass 1 and the cell's intermediate is still in L2.  Cells use a ring of S > A
// scratch slots (4 MiB each at N = 2^18, resident in L2).  Pass 2 of cell c needs
// the T1 pass-1 tiles of c; pass 1 of cell c reuses the slot of cell c - S and
// needs the T2 pass-2 tiles of that cell.  Every waited-on item carries a smaller
// ticket than the waiter, so it belongs to a CTA that is already running whatever
// order the hardware starts CTAs in, and every wait ends; waits are still bounded
// (1 s of global time), and one that runs out sets the error flag, which makes
// every later wait give up at once.
//
// The per-item protocol keeps the CTA's warps computing:
//  - thread 0 claims the next ticket when an item starts and reads the answer
//    when it ends, so the atomic's round trip runs under the item;
//  - at the end of an item thread 0 looks once (acquire load) at the next
//    item's dependency and hands the ticket to the CTA through shared memory at
//    the one CTA barrier per item;
//  - an item's completion is published (release fence, counter increment by
//    thread 0, covering the whole CTA's stores through that barrier) only after
//    the next item's loads are issued, where the fence's wait for the stores
//    overlaps the wait for those loads;
//  - when the look finds the dependency unmet (rare), thread 0 first publishes
//    the item it still holds (a waiter must never hold an unpublished item that
//    its own wait needs), then waits, behind one more barrier.
struct FusedCtl {
    uint32_t *ticket;   // next item
    uint32_t *done1;    // [nc] pass-1 tiles finished per cell
    uint32_t *done2;    // [nc] pass-2 tiles finished per cell
    uint32_t *err;      // non-zero after a wait ran out
    int64_t nc;         // cells in the launch
    int slots, ahead;   // ring slots S > ahead A
    int tpi;            // tiles per item (a power of two dividing both passes' tile counts)
    int64_t withhold;   // test hook: this cell's pass 1 never reports completion (-1: none)
};

__device__ __forceinline__ bool fused_wait(const uint32_t *cnt, uint32_t target, uint32_t *err) {
    if (ptx::ld_acquire(cnt) >= target) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    for (;;) {
        if (*reinterpret_cast<volatile uint32_t *>(err)) return false;
        if (ptx::ld_acquire(cnt) >= target) return true;
        if (ptx::globaltimer_ns() - t0 > 1000000000ull) {
            atomicExch(err, 1u);
            return false;
        }
        __nanosleep(100);
    }
}

// Release of one finished item: the CTA barrier before this call orders every
// thread's stores of the item before thread 0's fence.
__device__ __forceinline__ void fused_publish(uint32_t *cnt, uint32_t add) {
    __threadfence();
    atomicAdd(cnt, add);
}

// thread 0's hook inside run_pass, once its loads of the current item are
// issued (the waits below then overlap the wait for those loads): publishes the
// previous item and claims the ticket of the next one.
struct PublishHook {
    uint32_t *cnt;      // nullptr: nothing held
    uint32_t add;
    uint32_t *ticket;   // nullptr: no claim here
    uint32_t *next;     // shared-memory word that receives the claimed ticket
    __device__ __forceinline__ void after_loads() const {
        if (cnt) fused_publish(cnt, add);
        if (ticket) *next = atomicAdd(ticket, 1u);
    }
};

// An item's cell, pass and tile, and the counter it waits for (nullptr: none).
struct FusedItem {
    int64_t cell, slot;
    int tile;           // first tile of the item within its pass
    bool p1, valid;
    const uint32_t *dep;
    uint32_t target;
};

template <int T1, int T2>
__device__ __forceinline__ FusedItem fused_decode(uint32_t item, const FusedCtl &ctl) {
    const uint32_t I1 = (uint32_t)(T1 / ctl.tpi), I2 = (uint32_t)(T2 / ctl.tpi);
    const uint32_t step = item / (I1 + I2);
    const uint32_t r = item - step * (I1 + I2);
    FusedItem f;
    f.p1 = r < I1;
    f.cell = f.p1 ? (int64_t)step : (int64_t)step - ctl.ahead;
    f.valid = f.cell >= 0 && f.cell < ctl.nc;
    f.slot = f.valid ? (int64_t)((uint32_t)f.cell % (uint32_t)ctl.slots) : 0;
    f.tile = (int)(f.p1 ? r : r - I1) * ctl.tpi;
    f.dep = nullptr;
    f.target = 0;
    if (f.valid) {
        if (!f.p1) { f.dep = ctl.done1 + f.cell; f.target = T1; }
        else if (f.cell >= ctl.slots) { f.dep = ctl.done2 + (f.cell - ctl.slots); f.target = T2; }
    }
    return f;
}

// One tile of each pass, kept out of line: the persistent loop's own state then
// costs the passes no registers (inlined, the two passes and the loop spill).
template <int LOGN, int Z1>
__device__ __noinline__ void fused_tile1(const SearchLoad2<Cfg2<LOGN, 1>> *pl, const ScratchStore2<Cfg2<LOGN, 1>> *po,
                                         const float *__restrict__ tw, int tile, int64_t cell, int64_t slot,
                                         PublishHook hk) {
    using C1 = Cfg2<LOGN, 1>;
    SearchLoad2<C1> l = *pl;
    ScratchStore2<C1> o = *po;
    l.init(tile, cell, slot);
    o.init(tile, cell, slot);
    eng2::run_pass<float, C1::M, C1::SEQ, C1::EH, -1, eng2::kMapFJ, SearchLoad2<C1>, ScratchStore2<C1>, Z1, true,
                   PublishHook>(l, o, tw, hk);
}

template <int LOGN, bool LOWER>
__device__ __noinline__ void fused_tile2(const ScratchLoad2<Cfg2<LOGN, 2>> *pl,
                                         const SearchEpi2<Cfg2<LOGN, 2>, LOWER> *po, const float *__restrict__ tw,
                                         int tile, int64_t cell, int64_t slot, PublishHook hk) {
    using C2 = Cfg2<LOGN, 2>;
    ScratchLoad2<C2> l = *pl;
    SearchEpi2<C2, LOWER> o = *po;
    l.init(tile, cell, slot);
    o.init(tile, cell, slot);
    eng2::run_pass<float, C2::M, C2::SEQ, C2::EH, -1, eng2::kMapW, ScratchLoad2<C2>, SearchEpi2<C2, LOWER>, 8, true,
                   PublishHook>(l, o, tw, hk);
}

// Persistent: the grid holds as many CTAs as fit on the GPU at once.  The loop's
// state lives in shared memory and is re-read after each tile, so nothing but
// the item counter is live across the out-of-line tiles.
template <int LOGN, bool LOWER, int Z1>
__global__ void __launch_bounds__(256, 3)
k_search_fused(const __grid_constant__ SearchLoad2<Cfg2<LOGN, 1>> ld1,
               const __grid_constant__ ScratchStore2<Cfg2<LOGN, 1>> st1,
               const __grid_constant__ ScratchLoad2<Cfg2<LOGN, 2>> ld2,
               const __grid_constant__ SearchEpi2<Cfg2<LOGN, 2>, LOWER> st2,
               const float *__restrict__ tw_s1, const float *__restrict__ tw_s2, const FusedCtl ctl) {
    using C1 = Cfg2<LOGN, 1>;
    using C2 = Cfg2<LOGN, 2>;
    constexpr int T1 = C1::TILES, T2 = C2::TILES;
    __shared__ uint32_t s_item[2];
    __shared__ int s_wait[2];
    __shared__ int s_fail;
    __shared__ uint32_t *s_held;         // thread 0: counter of the finished, unpublished item
    __shared__ uint32_t s_nxt;           // thread 0: the ticket claimed while the item runs
    const bool t0 = threadIdx.x == 0;
    auto total = [&]() {                 // < 2^32: checked by the host
        return (uint32_t)(ctl.nc + ctl.ahead) * (uint32_t)(T1 / ctl.tpi + T2 / ctl.tpi);
    };
    if (t0) {
        s_item[0] = atomicAdd(ctl.ticket, 1u);
        s_wait[0] = 1;                   // the first item's dependency: waited for below
        s_fail = 0;
        s_held = nullptr;
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        {
            const uint32_t item = s_item[k & 1];
            if (item >= total()) break;  // the same for the whole CTA
            if (s_wait[k & 1]) {         // publish what is held, then wait
                if (t0) {
                    if (s_held) fused_publish(s_held, (uint32_t)ctl.tpi);
                    s_held = nullptr;
                    const FusedItem f = fused_decode<T1, T2>(item, ctl);
                    if (f.dep && !fused_wait(f.dep, f.target, ctl.err)) s_fail = 1;
                }
                __syncthreads();
                if (s_fail) return;
            }
        }
        for (int u = 0; u < ctl.tpi; ++u) {
            const FusedItem f = fused_decode<T1, T2>(s_item[k & 1], ctl);
            if (!f.valid) break;
            if (u) __syncthreads();      // the previous tile's exchange has been read
            const bool first = t0 && u == 0;
            const PublishHook h{first ? s_held : nullptr, (uint32_t)ctl.tpi, first ? ctl.ticket : nullptr,
                                &s_nxt};
            if (f.p1) fused_tile1<LOGN, Z1>(&ld1, &st1, tw_s2, f.tile + u, f.cell, f.slot, h);
            else fused_tile2<LOGN, LOWER>(&ld2, &st2, tw_s1, f.tile + u, f.cell, f.slot, h);
            if (first) s_held = nullptr;
        }
        if (t0) {
            const FusedItem f = fused_decode<T1, T2>(s_item[k & 1], ctl);
            if (!f.valid) {              // an empty item ran no hook
                if (s_held) fused_publish(s_held, (uint32_t)ctl.tpi);
                s_nxt = atomicAdd(ctl.ticket, 1u);
            }
            s_held = f.valid && !(f.p1 && f.cell == ctl.withhold) ? (f.p1 ? ctl.done1 : ctl.done2) + f.cell
                                                                  : nullptr;
            const uint32_t nxt = s_nxt;
            int wait = 0;
            if (nxt < total()) {         // one look at the next item's dependency
                const FusedItem g = fused_decode<T1, T2>(nxt, ctl);
                if (g.dep && ptx::ld_acquire(g.dep) < g.target) wait = 1;
            }
            s_item[(k + 1) & 1] = nxt;
            s_wait[(k + 1) & 1] = wait;
        }
        __syncthreads();                 // every thread's stores of the item; the next ticket
    }
    if (t0 && s_held) fused_publish(s_held, (uint32_t)ctl.tpi);
}

}  // namespace fstat
