// Register/shared-memory Stockham FFT engine for one pass of a four-step
// (two-pass) power-of-two transform.
//
// A CTA transforms a tile of F independent length-M sequences for each of two
// transforms (the pair F_a, F_b of the F-statistic, Sect. 2: "two Fourier
// transforms, each for one amplitude demodulation").  Each thread holds EH
// complex values of each transform; every stage is a radix-R Stockham
// autosort step (R = 8, the last stage 4 or 2 when log2 M is not a multiple of
// 3): gather R values, twiddle, R-point DFT in registers, scatter to shared
// memory.  The first stage reads through a Loader (global memory, or values
// generated on the fly) and the last stage hands its outputs to a Storer
// (global memory, or a fused epilogue), so the data crosses shared memory
// (stages - 1) times.  Shared memory holds complex elements (float2/double2)
// in rows of LD elements; element i of a row sits at pad(i) = i + i/16 + i/128,
// which spreads the radix-strided accesses of a warp over the banks and makes
// pad(j + r s) = pad(j) + pad(r s) for every stride s the stages use, so each
// thread forms one row address per job and reaches the R elements with
// immediate offsets.  The twiddles of each stage sit in their own table, in the
// order a warp reads them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace fstat {
namespace eng {

template <typename T> struct Vec2T;
template <> struct Vec2T<float> { using type = float2; };
template <> struct Vec2T<double> { using type = double2; };

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int n_main(int M) { return ilog2c(M) / 3; }
__host__ __device__ constexpr int rem_radix(int M) { return M >> (3 * n_main(M)); }
__host__ __device__ constexpr int n_stages(int M) { return n_main(M) + (rem_radix(M) > 1 ? 1 : 0); }
__host__ __device__ constexpr int stage_radix(int M, int s) { return s < n_main(M) ? 8 : rem_radix(M); }
__host__ __device__ constexpr int stage_ns(int M, int s) { return s < n_main(M) ? (1 << (3 * s)) : M / rem_radix(M); }
// words of the per-stage twiddle tables: sum over stages s >= 1 of (R_s - 1) NS_s (< M)
__host__ __device__ constexpr int tw_words(int M, int s = 1) {
    return s >= n_stages(M) ? 0 : (stage_radix(M, s) - 1) * stage_ns(M, s) + tw_words(M, s + 1);
}
__host__ __device__ constexpr int tw_offset(int M, int s) {
    return s <= 1 ? 0 : tw_offset(M, s - 1) + (stage_radix(M, s - 1) - 1) * stage_ns(M, s - 1);
}

__host__ __device__ constexpr int pad(int i) { return i + (i >> 4) + (i >> 7); }
// row length in elements: odd, so that rows of different sequences start in
// different banks
__host__ __device__ constexpr int row_ld(int M) { return (pad(M - 1) + 1) | 1; }
__host__ __device__ constexpr int tw_entries(int M) { return tw_words(M) > 0 ? tw_words(M) : 1; }

// bytes of the exchange area of a tile (2 transforms x F rows) and of a whole
// non-persistent pass (exchange + twiddle table)
template <typename T, int M, int F>
__host__ __device__ constexpr size_t exch_bytes() { return 2 * sizeof(T) * (size_t)(2 * F * row_ld(M)); }
template <typename T, int M, int F>
__host__ __device__ constexpr size_t smem_bytes() { return exch_bytes<T, M, F>() + 2 * sizeof(T) * (size_t)tw_entries(M); }

// ------------------------------------------------------------------ small DFTs
// Natural order in and out; DIR = -1 computes sum_j v_j e^{-2 pi i jk/R}.
template <int DIR, typename T>
__device__ __forceinline__ void dft2(T *re, T *im) {
    T tr = re[0] - re[1], ti = im[0] - im[1];
    re[0] += re[1];
    im[0] += im[1];
    re[1] = tr;
    im[1] = ti;
}

template <int DIR, typename T>
__device__ __forceinline__ void dft4(T &r0, T &i0, T &r1, T &i1, T &r2, T &i2, T &r3, T &i3) {
    T t0r = r0 + r2, t0i = i0 + i2;
    T t1r = r0 - r2, t1i = i0 - i2;
    T t2r = r1 + r3, t2i = i1 + i3;
    T t3r = r1 - r3, t3i = i1 - i3;
    // (DIR i) * t3
    T ur = (DIR < 0) ? t3i : -t3i;
    T ui = (DIR < 0) ? -t3r : t3r;
    r0 = t0r + t2r; i0 = t0i + t2i;
    r2 = t0r - t2r; i2 = t0i - t2i;
    r1 = t1r + ur;  i1 = t1i + ui;
    r3 = t1r - ur;  i3 = t1i - ui;
}

template <int DIR, typename T>
__device__ __forceinline__ void dft8(T *re, T *im) {
    const T h = T(0.70710678118654752440084436210485);
    T er0 = re[0], ei0 = im[0], er1 = re[2], ei1 = im[2], er2 = re[4], ei2 = im[4], er3 = re[6], ei3 = im[6];
    T or0 = re[1], oi0 = im[1], or1 = re[3], oi1 = im[3], or2 = re[5], oi2 = im[5], or3 = re[7], oi3 = im[7];
    dft4<DIR>(er0, ei0, er1, ei1, er2, ei2, er3, ei3);
    dft4<DIR>(or0, oi0, or1, oi1, or2, oi2, or3, oi3);
    // O_k *= W8^k, W8 = (1 + DIR i)/sqrt(2)
    T wr, wi;
    wr = (DIR < 0) ? (or1 + oi1) : (or1 - oi1);
    wi = (DIR < 0) ? (oi1 - or1) : (oi1 + or1);
    or1 = wr * h; oi1 = wi * h;
    wr = (DIR < 0) ? oi2 : -oi2;
    wi = (DIR < 0) ? -or2 : or2;
    or2 = wr; oi2 = wi;
    wr = (DIR < 0) ? (oi3 - or3) : (-or3 - oi3);
    wi = (DIR < 0) ? (-oi3 - or3) : (or3 - oi3);
    or3 = wr * h; oi3 = wi * h;
    re[0] = er0 + or0; im[0] = ei0 + oi0; re[4] = er0 - or0; im[4] = ei0 - oi0;
    re[1] = er1 + or1; im[1] = ei1 + oi1; re[5] = er1 - or1; im[5] = ei1 - oi1;
    re[2] = er2 + or2; im[2] = ei2 + oi2; re[6] = er2 - or2; im[6] = ei2 - oi2;
    re[3] = er3 + or3; im[3] = ei3 + oi3; re[7] = er3 - or3; im[7] = ei3 - oi3;
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(T *re, T *im) {
    if constexpr (R == 8) dft8<DIR>(re, im);
    else if constexpr (R == 4) dft4<DIR>(re[0], im[0], re[1], im[1], re[2], im[2], re[3], im[3]);
    else if constexpr (R == 2) dft2<DIR>(re, im);
}

// ------------------------------------------------------------------ barriers
// The whole CTA, or only the NT consumer threads of a warp-specialised CTA
// (named barrier 1; thread indices 0 .. NT-1).
struct CtaBarrier {
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};
template <int NT>
struct NamedBarrier {
    __device__ __forceinline__ static void sync() {
        asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    }
};

// Synchronises the TPF threads that share one sequence in the per-warp mapping:
// the warp when TPF <= 32, else a named barrier per group (ids 1 ..).
template <int TPF>
struct GroupBarrier {
    __device__ __forceinline__ static void sync() {
        if constexpr (TPF <= 32) {
            __syncwarp();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / TPF), "n"(TPF) : "memory");
        }
    }
};

// Job mappings (which sequence f and butterfly j a thread's i-th job of a stage is):
//   kMapJ   consecutive threads take consecutive butterflies, sequences interleave
//           across warps (CTA-wide barriers);
//   kMapFJ  as kMapJ, but the first and last stage take consecutive sequences
//           (columns of a strided tile, for coalesced global access);
//   kMapW   the TPF = M/EH threads of a group own one sequence for all stages, so
//           only the group synchronises (warps run out of phase).
constexpr int kMapJ = 0, kMapFJ = 1, kMapW = 2;

template <int MAPM, int S, int NST, int F, int JPF, int TPF, int THREADS>
__device__ __forceinline__ void job_fj(int i, int &f, int &j) {
    if constexpr (MAPM == kMapW) {
        f = (int)threadIdx.x / TPF;
        j = (int)threadIdx.x % TPF + TPF * i;
    } else {
        const int q = (int)threadIdx.x + i * THREADS;
        constexpr bool ffast = MAPM == kMapFJ && (S == 0 || S == NST - 1);
        f = ffast ? (q % F) : (q / JPF);
        j = ffast ? (q / F) : (q % JPF);
    }
}

// ------------------------------------------------------------------ the pass
// INPLACE: the Loader reads shared memory that the stage-0 scatter overwrites,
// so the scatter waits for every thread's gather.
template <typename T, int M, int F, int EH, int DIR, int MAPM, int S, class LD, class ST,
          class BAR = CtaBarrier, bool INPLACE = false>
__device__ __forceinline__ void run_stage(T (&re)[2][EH], T (&im)[2][EH],
                                          typename Vec2T<T>::type *sd,
                                          const typename Vec2T<T>::type *tw, LD &ld, ST &st) {
    using V = typename Vec2T<T>::type;
    constexpr int NST = n_stages(M);
    constexpr int R = stage_radix(M, S);
    constexpr int NS = stage_ns(M, S);
    constexpr int NJ = EH / R;
    constexpr int JPF = M / R;
    constexpr int THREADS = F * M / EH;
    constexpr int RL = row_ld(M);
    constexpr int TPF = M / EH;
    using SB = std::conditional_t<MAPM == kMapW, GroupBarrier<TPF>, BAR>;
    static_assert(EH % R == 0, "elements per thread must be a multiple of the radix");

    if constexpr (S == 0) {
        // every load of the tile is issued before any arithmetic
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            int f, j;
            job_fj<MAPM, S, NST, F, JPF, TPF, THREADS>(i, f, j);
            ld.template load<R, JPF>(f, j, &re[0][i * R], &im[0][i * R], &re[1][i * R],
                                     &im[1][i * R]);
        }
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            dft<R, DIR>(&re[0][i * R], &im[0][i * R]);
            dft<R, DIR>(&re[1][i * R], &im[1][i * R]);
        }
    } else {
        const V *tws = tw + tw_offset(M, S);
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            int f, j;
            job_fj<MAPM, S, NST, F, JPF, TPF, THREADS>(i, f, j);
            T *ra = &re[0][i * R], *ia = &im[0][i * R], *rb = &re[1][i * R], *ib = &im[1][i * R];
            const V *pa = sd + f * RL + pad(j);
            const V *pb = pa + F * RL;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const V va = pa[pad(r * JPF)], vb = pb[pad(r * JPF)];
                ra[r] = va.x; ia[r] = va.y;
                rb[r] = vb.x; ib[r] = vb.y;
            }
            // W_{NS R}^{r k}, k = j mod NS, from this stage's table [(r-1) NS + k]
            const V *tk = tws + (j % NS);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const V w = tk[(r - 1) * NS];
                const T wr = w.x, wi = (DIR < 0) ? w.y : -w.y;
                T xr = ra[r] * wr - ia[r] * wi, xi = ra[r] * wi + ia[r] * wr;
                ra[r] = xr; ia[r] = xi;
                xr = rb[r] * wr - ib[r] * wi; xi = rb[r] * wi + ib[r] * wr;
                rb[r] = xr; ib[r] = xi;
            }
            dft<R, DIR>(ra, ia);
            dft<R, DIR>(rb, ib);
        }
    }

    if constexpr (S == NST - 1) {
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            int f, j;
            job_fj<MAPM, S, NST, F, JPF, TPF, THREADS>(i, f, j);
            st.template store<R, JPF>(f, j, &re[0][i * R], &im[0][i * R], &re[1][i * R],
                                      &im[1][i * R]);
        }
    } else {
        if constexpr (S > 0 || INPLACE) SB::sync();   // every read of this stage is done
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            int f, j;
            job_fj<MAPM, S, NST, F, JPF, TPF, THREADS>(i, f, j);
            const int ob = (j / NS) * NS * R + (j % NS);
            V *pa = sd + f * RL + pad(ob);
            V *pb = pa + F * RL;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                pa[pad(r * NS)] = V{re[0][i * R + r], im[0][i * R + r]};
                pb[pad(r * NS)] = V{re[1][i * R + r], im[1][i * R + r]};
            }
        }
        SB::sync();
        run_stage<T, M, F, EH, DIR, MAPM, S + 1, LD, ST, BAR, INPLACE>(re, im, sd, tw, ld, st);
    }
}

// Fills the per-stage twiddle tables from the forward table e^{-2 pi i k/M}:
// stage s, entry (r-1) NS + k holds W_{NS R}^{r k} = W_M^{r k M/(NS R)}.
template <typename T, int M, int THREADS, int S>
__device__ __forceinline__ void fill_twiddles(typename Vec2T<T>::type *tws, const T *__restrict__ tw) {
    if constexpr (S < n_stages(M)) {
        constexpr int R = stage_radix(M, S), NS = stage_ns(M, S);
        constexpr int n = (R - 1) * NS, off = tw_offset(M, S), step = M / (NS * R);
        for (int e = (int)threadIdx.x; e < n; e += THREADS) {
            const int r = e / NS + 1, k = e % NS;
            const int m = r * k * step;
            tws[off + e] = typename Vec2T<T>::type{tw[2 * m], tw[2 * m + 1]};
        }
        fill_twiddles<T, M, THREADS, S + 1>(tws, tw);
    }
}

// One tile whose input the Loader reads from shared memory that is then reused
// in place for the stage exchanges (persistent kernels); twiddle tables filled.
template <typename T, int M, int F, int EH, int DIR, int MAPM, class BAR, class LD, class ST>
__device__ __forceinline__ void run_tile_inplace(LD &ld, ST &st, typename Vec2T<T>::type *buf,
                                                 const typename Vec2T<T>::type *tw) {
    T re[2][EH], im[2][EH];
    run_stage<T, M, F, EH, DIR, MAPM, 0, LD, ST, BAR, true>(re, im, buf, tw, ld, st);
}

// One pass over a tile.  tw: forward twiddles e^{-2 pi i k/M}, k < M, interleaved.
template <typename T, int M, int F, int EH, int DIR, int MAPM, class LD, class ST>
__device__ __forceinline__ void run_pass(LD &ld, ST &st, const T *__restrict__ tw) {
    using V = typename Vec2T<T>::type;
    constexpr int THREADS = F * M / EH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sd = reinterpret_cast<V *>(smem_raw);
    V *tws = reinterpret_cast<V *>(smem_raw + exch_bytes<T, M, F>());
    fill_twiddles<T, M, THREADS, 1>(tws, tw);
    // with CTA-wide stage barriers the first one publishes the tables; groups that
    // synchronise only among themselves need a CTA barrier here
    if constexpr (MAPM == kMapW && n_stages(M) > 1) __syncthreads();
    T re[2][EH], im[2][EH];
    run_stage<T, M, F, EH, DIR, MAPM, 0>(re, im, sd, tws, ld, st);
}

}  // namespace eng
}  // namespace fstat
