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
// (stages - 1) times.  Shared memory holds real and imaginary parts in separate
// arrays with one pad word per 32, which keeps both the unit-stride and the
// radix-strided accesses of a warp free of bank conflicts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fstat {
namespace eng {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int n_main(int M) { return ilog2c(M) / 3; }
__host__ __device__ constexpr int rem_radix(int M) { return M >> (3 * n_main(M)); }
__host__ __device__ constexpr int n_stages(int M) { return n_main(M) + (rem_radix(M) > 1 ? 1 : 0); }
__host__ __device__ constexpr int stage_radix(int M, int s) { return s < n_main(M) ? 8 : rem_radix(M); }
__host__ __device__ constexpr int stage_ns(int M, int s) { return s < n_main(M) ? (1 << (3 * s)) : M / rem_radix(M); }
__host__ __device__ constexpr int row_ld(int M) { return ((M + M / 32 + 1) % 2 == 0) ? (M + M / 32 + 2) : (M + M / 32 + 1); }

template <typename T, int M, int F>
constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(4 * F * row_ld(M) + 2 * M);
}

__device__ __forceinline__ int padi(int i) { return i + (i >> 5); }

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

// ------------------------------------------------------------------ the pass
// MAPF: first and last stage map consecutive threads to consecutive sequences
// (f fastest) -- used where the Loader/Storer walk a strided column tile, so that
// a warp's global accesses cover contiguous columns.  Middle stages always map
// consecutive threads to consecutive butterflies of one sequence.
template <typename T, int M, int F, int EH, int DIR, bool MAPF, int S, class LD, class ST>
__device__ __forceinline__ void run_stage(T (&re)[2][EH], T (&im)[2][EH], T *sre, T *sim,
                                          const T *twr, const T *twi, LD &ld, ST &st) {
    constexpr int NST = n_stages(M);
    constexpr int R = stage_radix(M, S);
    constexpr int NS = stage_ns(M, S);
    constexpr int NJ = EH / R;
    constexpr int JPF = M / R;
    constexpr int THREADS = F * M / EH;
    constexpr int RLD = row_ld(M);
    constexpr bool ffast = MAPF && (S == 0 || S == NST - 1);
    static_assert(EH % R == 0, "elements per thread must be a multiple of the radix");

#pragma unroll
    for (int i = 0; i < NJ; ++i) {
        const int q = threadIdx.x + i * THREADS;
        const int f = ffast ? (q % F) : (q / JPF);
        const int j = ffast ? (q / F) : (q % JPF);
        T *ra = &re[0][i * R], *ia = &im[0][i * R], *rb = &re[1][i * R], *ib = &im[1][i * R];
        if constexpr (S == 0) {
            ld.template load<R, JPF>(f, j, ra, ia, rb, ib);
        } else {
            const T *pa_r = sre + f * RLD, *pa_i = sim + f * RLD;
            const T *pb_r = sre + (F + f) * RLD, *pb_i = sim + (F + f) * RLD;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int idx = padi(j + r * JPF);
                ra[r] = pa_r[idx]; ia[r] = pa_i[idx];
                rb[r] = pb_r[idx]; ib[r] = pb_i[idx];
            }
            const int base = (j % NS) * (M / (NS * R));
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int e = r * base;
                const T wr = twr[e];
                const T wi = (DIR < 0) ? twi[e] : -twi[e];
                T xr = ra[r] * wr - ia[r] * wi, xi = ra[r] * wi + ia[r] * wr;
                ra[r] = xr; ia[r] = xi;
                xr = rb[r] * wr - ib[r] * wi; xi = rb[r] * wi + ib[r] * wr;
                rb[r] = xr; ib[r] = xi;
            }
        }
        dft<R, DIR>(ra, ia);
        dft<R, DIR>(rb, ib);
    }

    if constexpr (S == NST - 1) {
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int q = threadIdx.x + i * THREADS;
            const int f = ffast ? (q % F) : (q / JPF);
            const int j = ffast ? (q / F) : (q % JPF);
            st.template store<R, JPF>(f, j, &re[0][i * R], &im[0][i * R], &re[1][i * R],
                                      &im[1][i * R]);
        }
    } else {
        if constexpr (S > 0) __syncthreads();   // every read of this stage is done
#pragma unroll
        for (int i = 0; i < NJ; ++i) {
            const int q = threadIdx.x + i * THREADS;
            const int f = ffast ? (q % F) : (q / JPF);
            const int j = ffast ? (q / F) : (q % JPF);
            const int ob = (j / NS) * NS * R + (j % NS);
            T *pa_r = sre + f * RLD, *pa_i = sim + f * RLD;
            T *pb_r = sre + (F + f) * RLD, *pb_i = sim + (F + f) * RLD;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int idx = padi(ob + r * NS);
                pa_r[idx] = re[0][i * R + r]; pa_i[idx] = im[0][i * R + r];
                pb_r[idx] = re[1][i * R + r]; pb_i[idx] = im[1][i * R + r];
            }
        }
        __syncthreads();
        run_stage<T, M, F, EH, DIR, MAPF, S + 1>(re, im, sre, sim, twr, twi, ld, st);
    }
}

// One pass over a tile.  tw: forward twiddles e^{-2 pi i k/M}, k < M, interleaved.
template <typename T, int M, int F, int EH, int DIR, bool MAPF, class LD, class ST>
__device__ __forceinline__ void run_pass(LD &ld, ST &st, const T *__restrict__ tw) {
    constexpr int THREADS = F * M / EH;
    constexpr int RLD = row_ld(M);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sre = reinterpret_cast<T *>(smem_raw);
    T *sim = sre + 2 * F * RLD;
    T *twr = sim + 2 * F * RLD;
    T *twi = twr + M;
    if constexpr (n_stages(M) > 1) {
        for (int i = threadIdx.x; i < M; i += THREADS) {
            twr[i] = tw[2 * i];
            twi[i] = tw[2 * i + 1];
        }
        // made visible by the barrier that precedes the first shared-memory read
    }
    T re[2][EH], im[2][EH];
    run_stage<T, M, F, EH, DIR, MAPF, 0>(re, im, sre, sim, twr, twi, ld, st);
}

}  // namespace eng
}  // namespace fstat
