// The two passes of the four-step transform N = N1 * N2 with their loaders and
// storers.  With k = k1 + N1 k2 and l = N2 l1 + l2:
//   pass 1, per column k1:  A[k1][l2] = W_N^{k1 l2} sum_k2 z[k1 + N1 k2] W_N2^{k2 l2}
//   pass 2, per row l2:     X[N2 l1 + l2] = sum_k1 A[k1][l2] W_N1^{k1 l1}
// Pass 1 writes A transposed (row l2 contiguous in k1) to an L2-resident scratch
// slot; pass 2 reads whole rows.  The search instantiations fuse the spindown
// demodulation into the pass-1 loader (Sect. 2, "for each s value ... we
// perform the demodulation") and the F-statistic, threshold and candidate
// compaction into the pass-2 storer (Fig. 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"
#include "fstat_internal.h"

namespace fstat {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Elements per thread per transform: 16 complex floats or 8 complex doubles
// (both 32 registers of payload per transform).
template <typename T> constexpr int elems_per_thread() { return sizeof(T) == 4 ? 16 : 8; }

// TS: target threads per CTA (tile shape); EHT: complex elements per thread per
// transform (0: the default for T).  Fewer elements per thread mean fewer
// registers and more resident warps.
template <typename T, int LOGN, int PASS, int TS = 256, int EHT = 0>
struct Cfg {
    static constexpr int LOGN1 = LOGN / 2;
    static constexpr int LOGN2 = LOGN - LOGN / 2;
    static constexpr int N1 = 1 << LOGN1;
    static constexpr int N2 = 1 << LOGN2;
    static constexpr int N = 1 << LOGN;
    static constexpr int M = PASS == 1 ? N2 : N1;         // length of this pass's FFTs
    static constexpr int OTHER = PASS == 1 ? N1 : N2;     // number of such FFTs
    static constexpr int EH = EHT > 0 ? EHT : elems_per_thread<T>();
    static constexpr int F0 = TS * EH / M;
    static constexpr int F = F0 < OTHER ? (F0 > 0 ? F0 : 1) : OTHER;   // sequences per tile
    static constexpr int THREADS = F * M / EH;
    static constexpr int TILES = OTHER / F;
    static constexpr size_t SMEM = eng::smem_bytes<T, M, F>();
    // resident threads per SM: 512 at 16 (FP32) / 8 (FP64) elements per thread
    // (<= 128 registers), 1024 at 8 FP32 elements (<= 64 registers)
    static constexpr int RES = (EH * (int)sizeof(T) <= 32) ? 1024 : 512;
    static constexpr int MIN_BLOCKS = THREADS >= 64 ? (RES / THREADS < 8 ? RES / THREADS : 8) : 1;
    static_assert(THREADS >= 1 && THREADS <= 256, "tile shape");
};

template <typename T>
__device__ __forceinline__ void cmul_tw(T &xr, T &xi, T wr, T wi) {
    T r = xr * wr - xi * wi;
    xi = xr * wi + xi * wr;
    xr = r;
}

// ------------------------------------------------------------------ pass 1 loaders
// Generic: n_tr transforms of length N stored back to back; pair = blockIdx.y.
template <typename T, class C>
struct GenericLoad {
    using V = typename Vec2<T>::type;
    const V *in;
    int64_t n_tr;
    const V *a, *b;
    bool has_b;
    int k1_0;
    __device__ void init() {
        const int64_t p = blockIdx.y;
        a = in + (2 * p) * (int64_t)C::N;
        has_b = 2 * p + 1 < n_tr;
        b = a + C::N;
        k1_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = k1_0 + f + C::N1 * (j + r * JPF);
            V va = a[k];
            ra[r] = va.x; ia[r] = va.y;
            if (has_b) { V vb = b[k]; rb[r] = vb.x; ib[r] = vb.y; }
            else { rb[r] = T(0); ib[r] = T(0); }
        }
    }
};

// Search, FP32: w[k] = (y_k a_k, y_k b_k) as float4 for one sky; z = w e^{-2 pi i phi_k},
// phi_k = frac(fdot dt^2 k^2 / 2) from a 64-bit fixed-point product (exact mod 1
// up to the rounding of the rate), zero for k >= n (the zero padding).
template <class C>
struct SearchLoadF32 {
    const float4 *w;
    int64_t w_stride;
    int n;
    const uint64_t *chirp;
    int n_spin;
    int64_t c0, s0;
    const float4 *ws;
    uint64_t afx;
    int k1_0;
    __device__ void init() {
        const int64_t c = c0 + blockIdx.y;
        const int64_t sky = c / n_spin;
        ws = w + (sky - s0) * w_stride;
        afx = chirp[c - sky * n_spin];
        k1_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, float *ra, float *ia, float *rb,
                                         float *ib) const {
        float4 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {      // loads first: all in flight together
            const int k = k1_0 + f + C::N1 * (j + r * JPF);
            v[r] = k < n ? __ldg(ws + k) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t k = (uint32_t)(k1_0 + f + C::N1 * (j + r * JPF));
            if (k < (uint32_t)n) {        // the zero padding needs no phase
                const uint64_t kk = (uint64_t)k * (uint64_t)k;
                const int32_t top = (int32_t)((afx * kk) >> 32);          // cycles in [-1/2, 1/2)
                const float ph = (float)top * 1.4629180792671596e-09f;    // 2 pi / 2^32
                float s, c;
                __sincosf(ph, &s, &c);
                ra[r] = v[r].x * c + v[r].y * s; ia[r] = v[r].y * c - v[r].x * s;
                rb[r] = v[r].z * c + v[r].w * s; ib[r] = v[r].w * c - v[r].z * s;
            } else {
                ra[r] = 0.f; ia[r] = 0.f; rb[r] = 0.f; ib[r] = 0.f;
            }
        }
    }
};

// Search, FP64: w[k] = {y a, y b} as two double2; phi_k = frac(rate k^2) in FP64.
struct alignas(16) W64 {
    double ar, ai, br, bi;
};

template <class C>
struct SearchLoadF64 {
    const W64 *w;
    int64_t w_stride;
    int n;
    const double *chirp;
    int n_spin;
    int64_t c0, s0;
    const W64 *ws;
    double rate;
    int k1_0;
    __device__ void init() {
        const int64_t c = c0 + blockIdx.y;
        const int64_t sky = c / n_spin;
        ws = w + (sky - s0) * w_stride;
        rate = chirp[c - sky * n_spin];
        k1_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, double *ra, double *ia, double *rb,
                                         double *ib) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = k1_0 + f + C::N1 * (j + r * JPF);
            if (k < n) {
                const W64 v = ws[k];
                const double kd = (double)k;
                const double cyc = rate * (kd * kd);
                const double fr = cyc - floor(cyc);
                double s, c;
                sincospi(2.0 * fr, &s, &c);
                ra[r] = v.ar * c + v.ai * s; ia[r] = v.ai * c - v.ar * s;
                rb[r] = v.br * c + v.bi * s; ib[r] = v.bi * c - v.br * s;
            } else {
                ra[r] = 0.0; ia[r] = 0.0; rb[r] = 0.0; ib[r] = 0.0;
            }
        }
    }
};

// ------------------------------------------------------------------ pass 1 storer
// Applies the inter-pass twiddle W_N^{k1 l2} and writes the transposed tile into
// scratch slot blockIdx.y.  A job's outputs sit at l2 = j + r JPF, so its
// twiddles are W^{k1 j} (W^{k1 JPF})^r: two table lookups per job, then complex
// powers, instead of a scattered lookup per element.  A lookup of W_N^m, m < N,
// is hi[m >> log N1] lo[m & (N1 - 1)].
template <typename T, class C, int DIR>
struct ScratchStore {
    using V = typename Vec2<T>::type;
    V *scratch;
    const T *lo, *hi;
    int64_t n_tr;   // generic: number of transforms (the odd one out has no b); search: 2*pairs
    V *base;
    bool has_b;
    int k1_0;
    __device__ void init() {
        const int64_t p = blockIdx.y;
        base = scratch + p * 2 * (int64_t)C::N;
        has_b = 2 * p + 1 < n_tr;
        k1_0 = blockIdx.x * C::F;
    }
    __device__ __forceinline__ V wn(int m) const {
        const V th = __ldg(reinterpret_cast<const V *>(hi) + (m >> C::LOGN1));
        const V tl = __ldg(reinterpret_cast<const V *>(lo) + (m & (C::N1 - 1)));
        return V{th.x * tl.x - th.y * tl.y, th.x * tl.y + th.y * tl.x};
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
        const int k1 = k1_0 + f;
        V w = wn(k1 * j);
        const V st = wn(k1 * JPF);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int l2 = j + r * JPF;
            const T wr = w.x, wi = (DIR > 0) ? -w.y : w.y;
            T xr = ra[r], xi = ia[r];
            cmul_tw(xr, xi, wr, wi);
            base[(int64_t)l2 * C::N1 + k1] = V{xr, xi};
            if (has_b) {
                xr = rb[r]; xi = ib[r];
                cmul_tw(xr, xi, wr, wi);
                base[C::N + (int64_t)l2 * C::N1 + k1] = V{xr, xi};
            }
            if (r + 1 < R) w = V{w.x * st.x - w.y * st.y, w.x * st.y + w.y * st.x};
        }
    }
};

// ------------------------------------------------------------------ pass 2 loader
template <typename T, class C>
struct ScratchLoad {
    using V = typename Vec2<T>::type;
    const V *scratch;
    const V *base;
    int l2_0;
    __device__ void init() {
        base = scratch + (int64_t)blockIdx.y * 2 * C::N;
        l2_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
        const V *row = base + (int64_t)(l2_0 + f) * C::N1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k1 = j + r * JPF;
            const V va = row[k1], vb = row[C::N + k1];
            ra[r] = va.x; ia[r] = va.y; rb[r] = vb.x; ib[r] = vb.y;
        }
    }
};

// ------------------------------------------------------------------ pass 2 storers
template <typename T, class C>
struct GenericStore {
    using V = typename Vec2<T>::type;
    V *out;
    int64_t n_tr;
    V *a, *b;
    bool has_b;
    int l2_0;
    __device__ void init() {
        const int64_t p = blockIdx.y;
        a = out + 2 * p * (int64_t)C::N;
        b = a + C::N;
        has_b = 2 * p + 1 < n_tr;
        l2_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
        const int l2 = l2_0 + f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int l = C::N2 * (j + r * JPF) + l2;
            a[l] = V{ra[r], ia[r]};
            if (has_b) b[l] = V{rb[r], ib[r]};
        }
    }
};

// F = |F_a|^2/(sigma^2 S_aa) + |F_b|^2/(sigma^2 S_bb) per bin (Fig. 1,
// "F-statistics calculation"), strict 2F > thr ("signals above the threshold
// registered"), appended with one atomic per warp: the same offset arithmetic as
// the paper's count-exchange before the collective write (Sect. 3.2), inside one
// GPU.
template <typename T, class C>
struct SearchEpi {
    const double *norm;      // [sky_local][4]: na, nb, nab (F = na|F_a|^2 + nb|F_b|^2 + nab Re F_a F_b*)
    int n_spin;
    int64_t c0, s0;
    uint32_t cell_base;      // first global cell index of this band
    int64_t bin_lo, bin_hi;
    T thr;
    CandRecord *out;
    unsigned long long *count;
    unsigned long long cap;
    T na, nb, nab;
    uint32_t cell;
    int l2_0;
    __device__ void init() {
        const int64_t c = c0 + blockIdx.y;
        const int64_t sky = c / n_spin;
        na = (T)norm[kNormStride * (sky - s0)];
        nb = (T)norm[kNormStride * (sky - s0) + 1];
        nab = (T)norm[kNormStride * (sky - s0) + 2];
        cell = cell_base + (uint32_t)c;
        l2_0 = blockIdx.x * C::F;
    }
    template <int R, int JPF>
    __device__ __forceinline__ void store(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
        constexpr unsigned FULL = C::THREADS >= 32 ? 0xffffffffu : ((1u << C::THREADS) - 1u);
        const int l2 = l2_0 + f;
        T Fv[R];
        bool any = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Fv[r] = (ra[r] * ra[r] + ia[r] * ia[r]) * na + (rb[r] * rb[r] + ib[r] * ib[r]) * nb;
            if (nab != T(0)) Fv[r] += (ra[r] * rb[r] + ia[r] * ib[r]) * nab;   // full form
            const int64_t bin = (int64_t)C::N2 * (j + r * JPF) + l2;
            const bool p = (bin >= bin_lo) && (bin <= bin_hi) && (T(2) * Fv[r] > thr);
            any |= p;
        }
        if (!__any_sync(FULL, any)) return;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t bin = (int64_t)C::N2 * (j + r * JPF) + l2;
            const bool p = (bin >= bin_lo) && (bin <= bin_hi) && (T(2) * Fv[r] > thr);
            const unsigned m = __ballot_sync(FULL, p);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b0 = 0;
                if (lane == leader) b0 = atomicAdd(count, (unsigned long long)__popc(m));
                b0 = __shfl_sync(FULL, b0, leader);
                if (p) {
                    const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
                    if (idx < cap) out[idx] = CandRecord{cell, (uint32_t)bin, (double)Fv[r]};
                }
            }
        }
    }
};

// ------------------------------------------------------------------ kernels
template <typename T, int LOGN, int PASS, int DIR, int MAPM, class LD, class ST, int TS = 256,
          int EHT = 0>
__global__ void __launch_bounds__(Cfg<T, LOGN, PASS, TS, EHT>::THREADS,
                                  Cfg<T, LOGN, PASS, TS, EHT>::MIN_BLOCKS)
k_pass(LD ld, ST st, const T *__restrict__ tw) {
    using C = Cfg<T, LOGN, PASS, TS, EHT>;
    ld.init();
    st.init();
    eng::run_pass<T, C::M, C::F, C::EH, DIR, MAPM>(ld, st, tw);
}

// Pass-1 output parked in the exchange area, in natural order, one row per
// sequence (the group that transformed a column writes only its own row).
template <typename T, class C>
struct RowParkStore {
    using V = typename Vec2<T>::type;
    V *sd;
    template <int R, int JPF>
    __device__ __forceinline__ void store(int f, int j, T *ra, T *ia, T *rb, T *ib) const {
        constexpr int RL = eng::row_ld(C::M);
        V *pa = sd + f * RL, *pb = sd + (C::F + f) * RL;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int l2 = j + r * JPF;
            pa[eng::pad(l2)] = V{ra[r], ia[r]};
            pb[eng::pad(l2)] = V{rb[r], ib[r]};
        }
    }
};

// Search pass 1 with one sequence per thread group: each group gathers its
// column, demodulates and transforms it with group-local synchronisation only,
// parks the result in its shared-memory row; then the CTA writes the tile to
// scratch row by row (coalesced), applying the inter-pass twiddle
// W_N^{k1 l2} = hi[m >> log N1] lo[m & (N1 - 1)], m = k1 l2.
template <typename T, int LOGN, int TS, class LD>
__global__ void __launch_bounds__(Cfg<T, LOGN, 1, TS>::THREADS, Cfg<T, LOGN, 1, TS>::MIN_BLOCKS)
k_search_pass1(LD ld, typename Vec2<T>::type *scratch, const T *__restrict__ lo,
               const T *__restrict__ hi, const T *__restrict__ tw) {
    using C = Cfg<T, LOGN, 1, TS>;
    using V = typename Vec2<T>::type;
    constexpr int RL = eng::row_ld(C::M);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sd = reinterpret_cast<V *>(smem_raw);
    ld.init();
    RowParkStore<T, C> st{sd};
    eng::run_pass<T, C::M, C::F, C::EH, -1, eng::kMapW>(ld, st, tw);
    __syncthreads();
    V *base = scratch + (int64_t)blockIdx.y * 2 * C::N;
    const int k1_0 = blockIdx.x * C::F;
    for (int idx = threadIdx.x; idx < C::F * C::M; idx += C::THREADS) {
        const int l2 = idx / C::F, f = idx - l2 * C::F;
        const int k1 = k1_0 + f;
        const int m = k1 * l2;
        const V th = __ldg(reinterpret_cast<const V *>(hi) + (m >> C::LOGN1));
        const V tl = __ldg(reinterpret_cast<const V *>(lo) + (m & (C::N1 - 1)));
        const T wr = th.x * tl.x - th.y * tl.y, wi = th.x * tl.y + th.y * tl.x;
        const V a = sd[f * RL + eng::pad(l2)], b = sd[(C::F + f) * RL + eng::pad(l2)];
        base[(int64_t)l2 * C::N1 + k1] = V{a.x * wr - a.y * wi, a.x * wi + a.y * wr};
        base[C::N + (int64_t)l2 * C::N1 + k1] = V{b.x * wr - b.y * wi, b.x * wi + b.y * wr};
    }
}

template <class KernelPtr>
inline void set_smem(KernelPtr k, size_t bytes) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace fstat
