// Second FFT engine: one transform per thread group, 32 complex elements per
// thread, and every pass length M <= 1024 split into at most two register
// stages (M = R0 R1 with R0, R1 <= 32), so the data crosses shared memory once
// per pass instead of twice.
//
// A CTA transforms SEQ independent length-M sequences (for the F-statistic the
// F_a and F_b sequences of F tiles: s = t F + f, t = 0 for a, 1 for b).  Stage 0
// is a radix-R0 DFT of the elements j + r M/R0 of one sequence; stage 1 twiddles
// by W_M^{r j} and takes radix-R1 DFTs; outputs land at j + r R0.  Shared memory
// holds complex elements (float2) in rows of LD elements with element i at
// i + i/32, which makes both scatter and gather of the two-stage plan free of
// bank conflicts for M = 512 and leaves every radix offset an immediate; the
// column passes with two stage-1 jobs per thread use i + 2 (i/32) instead and
// exchange pairs of elements in 16-byte accesses (x16_layout below).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"

namespace fstat {
namespace eng2 {

using eng::Vec2T;

// ------------------------------------------------------------------ constants
// e^{-2 pi i k/32} from the first-octant values cos(pi m/16), sin(pi m/16).
__host__ __device__ constexpr double oct_cos(int m) {
    return m == 0 ? 1.0 : m == 1 ? 0.98078528040323044913 : m == 2 ? 0.92387953251128675613
         : m == 3 ? 0.83146961230254523708 : m == 4 ? 0.70710678118654752440
         : m == 5 ? 0.55557023301960222474 : m == 6 ? 0.38268343236508977173
         : m == 7 ? 0.19509032201612826785 : 0.0;
}
__host__ __device__ constexpr double oct_sin(int m) { return oct_cos(8 - m); }
__host__ __device__ constexpr double w32_re(int k) {
    return (k / 8) % 4 == 0 ? oct_cos(k % 8) : (k / 8) % 4 == 1 ? -oct_sin(k % 8)
         : (k / 8) % 4 == 2 ? -oct_cos(k % 8) : oct_sin(k % 8);
}
__host__ __device__ constexpr double w32_im(int k) {   // -sin(2 pi k / 32)
    return (k / 8) % 4 == 0 ? -oct_sin(k % 8) : (k / 8) % 4 == 1 ? -oct_cos(k % 8)
         : (k / 8) % 4 == 2 ? oct_sin(k % 8) : oct_cos(k % 8);
}

// ------------------------------------------------------------------ register DFTs
// Natural order in and out; DIR = -1 is the forward transform.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(T *re, T *im);

// x <- x W_32^e (DIR = -1) or x conj(W_32^e), e known at compile time once the
// callers' loops are unrolled: the quarter turns are swaps and negations, so
// no multiplication by 0 or 1 is left for the compiler to keep.
template <int DIR, typename T>
__device__ __forceinline__ void mul_w32(int e, T &xr, T &xi) {
    e &= 31;
    if (e == 0) return;
    if (e == 16) { xr = -xr; xi = -xi; return; }
    if (e == 8 || e == 24) {   // W = -i (e = 8) or +i (e = 24); conjugated for DIR > 0
        const bool minus_i = (e == 8) == (DIR < 0);
        const T r = xr;
        xr = minus_i ? xi : -xi;
        xi = minus_i ? -r : r;
        return;
    }
    const T wr = (T)w32_re(e);
    const T wi = DIR < 0 ? (T)w32_im(e) : -(T)w32_im(e);
    const T r = xr * wr - xi * wi;
    xi = xr * wi + xi * wr;
    xr = r;
}

// Radix-4 decimation in time: 4 sub-DFTs of length R/4 over x[4m + q], then for
// each k < R/4 the twiddles W_R^{q k} and a 4-point DFT across q.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft_r4(T *re, T *im) {
    constexpr int n = R / 4;
    T sr[4][n], si[4][n];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int m = 0; m < n; ++m) { sr[q][m] = re[4 * m + q]; si[q][m] = im[4 * m + q]; }
#pragma unroll
    for (int q = 0; q < 4; ++q) dft<n, DIR>(sr[q], si[q]);
#pragma unroll
    for (int k = 0; k < n; ++k) {
        T zr[4], zi[4];
        zr[0] = sr[0][k]; zi[0] = si[0][k];
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            zr[q] = sr[q][k];
            zi[q] = si[q][k];
            mul_w32<DIR>((32 / R) * q * k, zr[q], zi[q]);   // W_R^{q k} = W_32^{(32/R) q k}
        }
        eng::dft4<DIR>(zr[0], zi[0], zr[1], zi[1], zr[2], zi[2], zr[3], zi[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) { re[k + n * p] = zr[p]; im[k + n * p] = zi[p]; }
    }
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(T *re, T *im) {
    if constexpr (R == 32 || R == 16) dft_r4<R, DIR>(re, im);
    else eng::dft<R, DIR>(re, im);
}

// 4-point DFT whose inputs from index NZ on are known to be zero: the terms
// with a zero partner are left out (the compiler may not drop x + 0 itself,
// since -0 + 0 = +0 under IEEE rules).
template <int DIR, int NZ, typename T>
__device__ __forceinline__ void dft4z(T &r0, T &i0, T &r1, T &i1, T &r2, T &i2, T &r3, T &i3) {
    static_assert(NZ >= 1 && NZ <= 4, "non-zero inputs");
    if constexpr (NZ == 4) {
        eng::dft4<DIR>(r0, i0, r1, i1, r2, i2, r3, i3);
    } else {
        // t0 = x0 + x2, t1 = x0 - x2, t2 = t3 = x1 (x3 = 0); u = (DIR i) x1
        const T t0r = NZ >= 3 ? r0 + r2 : r0, t0i = NZ >= 3 ? i0 + i2 : i0;
        const T t1r = NZ >= 3 ? r0 - r2 : r0, t1i = NZ >= 3 ? i0 - i2 : i0;
        if constexpr (NZ == 1) {
            r1 = r2 = r3 = r0;
            i1 = i2 = i3 = i0;
        } else {
            const T ur = DIR < 0 ? i1 : -i1, ui = DIR < 0 ? -r1 : r1;
            const T x1r = r1, x1i = i1;
            r0 = t0r + x1r; i0 = t0i + x1i;
            r2 = t0r - x1r; i2 = t0i - x1i;
            r1 = t1r + ur;  i1 = t1i + ui;
            r3 = t1r - ur;  i3 = t1i - ui;
        }
    }
}

// 16-point DFT (radix-4 decimation in time, as dft_r4) of x[0 .. NZ) with
// x[NZ .. 16) = 0: the sub-DFT over x[4m + q] keeps its ceil((NZ - q)/4)
// non-zero inputs; the elements from NZ on are not read.
template <int DIR, int NZ, typename T>
__device__ __forceinline__ void dft16z(T *re, T *im) {
    static_assert(NZ >= 4 && NZ <= 16, "each sub-DFT keeps an input");
    T sr[4][4], si[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (4 * m + q < NZ) { sr[q][m] = re[4 * m + q]; si[q][m] = im[4 * m + q]; }
            else { sr[q][m] = T(0); si[q][m] = T(0); }   // never read below
    dft4z<DIR, (NZ + 3) / 4>(sr[0][0], si[0][0], sr[0][1], si[0][1], sr[0][2], si[0][2], sr[0][3], si[0][3]);
    dft4z<DIR, (NZ + 2) / 4>(sr[1][0], si[1][0], sr[1][1], si[1][1], sr[1][2], si[1][2], sr[1][3], si[1][3]);
    dft4z<DIR, (NZ + 1) / 4>(sr[2][0], si[2][0], sr[2][1], si[2][1], sr[2][2], si[2][2], sr[2][3], si[2][3]);
    dft4z<DIR, NZ / 4>(sr[3][0], si[3][0], sr[3][1], si[3][1], sr[3][2], si[3][2], sr[3][3], si[3][3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T zr[4], zi[4];
        zr[0] = sr[0][k]; zi[0] = si[0][k];
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            zr[q] = sr[q][k];
            zi[q] = si[q][k];
            mul_w32<DIR>(2 * q * k, zr[q], zi[q]);   // W_16^{q k} = W_32^{2 q k}
        }
        eng::dft4<DIR>(zr[0], zi[0], zr[1], zi[1], zr[2], zi[2], zr[3], zi[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) { re[k + 4 * p] = zr[p]; im[k + 4 * p] = zi[p]; }
    }
}

// R-point DFT of x[0 .. NZ) with x[NZ .. R) = 0, NZ <= R/2: the even outputs are
// the R/2-point DFT of x, the odd ones that of x_r W_R^r (the first radix-2
// layer of a decimation in frequency, whose partners are all zero); below R/2
// non-zero inputs the half-length DFTs skip their zero inputs too (R = 32).
template <int R, int DIR, int NZ = R / 2, typename T>
__device__ __forceinline__ void dft_half_zero(T *re, T *im) {
    constexpr int H = R / 2;
    static_assert(NZ <= H && (NZ == H || H == 16), "pruned half-length DFTs are 16-point");
    T er[H], ei[H], orr[H], oi[H];
#pragma unroll
    for (int r = 0; r < NZ; ++r) {
        er[r] = re[r]; ei[r] = im[r];
        orr[r] = re[r]; oi[r] = im[r];
        mul_w32<DIR>((32 / R) * r, orr[r], oi[r]);
    }
    if constexpr (NZ < H) {
        dft16z<DIR, NZ>(er, ei);
        dft16z<DIR, NZ>(orr, oi);
    } else if constexpr (H > 1) {
        dft<H, DIR>(er, ei);
        dft<H, DIR>(orr, oi);
    }
#pragma unroll
    for (int p = 0; p < H; ++p) {
        re[2 * p] = er[p]; im[2 * p] = ei[p];
        re[2 * p + 1] = orr[p]; im[2 * p + 1] = oi[p];
    }
}

// ------------------------------------------------------------------ plan
__host__ __device__ constexpr int radix0(int M) { return M <= 32 ? M : (M >= 512 ? 32 : (M >= 128 ? 16 : 8)); }
__host__ __device__ constexpr int radix1(int M) { return M <= 32 ? 1 : M / radix0(M); }
__host__ __device__ constexpr int pad(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int row_ld(int M) { return (pad(M - 1) + 1) | 1; }
// 16-byte exchange layout of the column passes (two stage-1 jobs per thread):
// two padding elements per 32 keep pairs (2i, 2i + 1) together and 16-byte
// aligned, and a row length of 2 mod 4 elements spreads the 8 lanes of a
// quarter-warp (consecutive sequences) over all eight 16-byte bank groups.
__host__ __device__ constexpr bool x16_layout(int M, int EH) { return M > 32 && EH == 2 * radix1(M) && radix0(M) % 2 == 0; }
__host__ __device__ constexpr int pad16(int i) { return i + 2 * (i >> 5); }
__host__ __device__ constexpr int row_ld16(int M) { return (pad16(M - 1) + 1) + ((6 - (pad16(M - 1) + 1) % 4) % 4); }
// stage-1 twiddles: rows b < log2 R1 of W_M^{2^b j}, j < R0
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int tw_entries(int M) { return M <= 32 ? 1 : ilog2c(radix1(M)) * radix0(M); }

template <typename T, int M, int SEQ, bool X16 = false>
__host__ __device__ constexpr size_t exch_bytes() { return 2 * sizeof(T) * (size_t)SEQ * (X16 ? row_ld16(M) : row_ld(M)); }
template <typename T, int M, int SEQ, bool X16 = false>
__host__ __device__ constexpr size_t smem_bytes() {
    return exch_bytes<T, M, SEQ, X16>() + 2 * sizeof(T) * (size_t)tw_entries(M);
}

// Mappings of a thread's i-th job of a stage to (sequence s, butterfly j) and of
// s to (transform t, tile column or row f):
//   kMapFJ  consecutive threads take consecutive sequences, s = 2 f + t (the a
//           and b halves of one float4 input side by side: coalesced access to a
//           strided tile of columns), CTA-wide barriers;
//   kMapW   s = t SEQ/2 + f; a warp holds F_a and F_b of the same tile rows in
//           its two halves (lanes l and l ^ 16 share j and f), warp-level
//           synchronisation only.
constexpr int kMapFJ = 1, kMapW = 2;

struct Job {
    int s, t, f, j;
};

template <int MAPM, int SEQ, int TPF, int THREADS>
__device__ __forceinline__ Job job(int i) {
    Job q;
    if constexpr (MAPM == kMapW) {
        constexpr int G = 32 / TPF;          // groups per warp, G/2 tile rows
        const int w = (int)threadIdx.x >> 5, l = (int)threadIdx.x & 31;
        const int gi = l / TPF;
        q.t = gi < G / 2 ? 0 : 1;
        q.f = w * (G / 2) + (gi % (G / 2));
        q.s = q.t * (SEQ / 2) + q.f;
        q.j = l % TPF + TPF * i;
    } else {
        const int x = (int)threadIdx.x + i * THREADS;
        q.s = x % SEQ;
        q.j = x / SEQ;
        q.t = q.s & 1;
        q.f = q.s >> 1;
    }
    return q;
}

// Fills the stage-1 twiddle table, entry b R0 + j = W_M^{2^b j}, from the forward
// table tw[m] = e^{-2 pi i m / M}.
template <typename T, int M, int THREADS>
__device__ __forceinline__ void fill_twiddles(typename Vec2T<T>::type *tws, const T *__restrict__ tw) {
    if constexpr (M > 32) {
        constexpr int R0 = radix0(M), n = tw_entries(M);
        for (int e = (int)threadIdx.x; e < n; e += THREADS) {
            const int m = (e % R0) << (e / R0);
            tws[e] = typename Vec2T<T>::type{tw[2 * m], tw[2 * m + 1]};
        }
    }
}

// One pass over a tile.  LD::load<R0, M/R0>(job, re, im) yields the elements
// j + r M/R0 of sequence (t, f); ST::store<R, JPF>(job, re, im) receives outputs
// j + r JPF (R = R1, JPF = R0 after two stages; R = M, JPF = 1 after one).
// The CTA's dynamic shared memory (exchange area, then the twiddle table).
__device__ __forceinline__ unsigned char *dyn_smem() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return smem_raw;
}

template <class ST, class = void>
struct StoreEarly { static constexpr bool value = false; };
template <class ST>
struct StoreEarly<ST, decltype(void(ST::kStoreEarly))> { static constexpr bool value = ST::kStoreEarly; };

template <class LD, class = void>
struct LoaderStaged { static constexpr bool value = false; };
template <class LD>
struct LoaderStaged<LD, decltype(void(LD::kStaged))> { static constexpr bool value = LD::kStaged; };

// Called by run_pass once this thread has issued the loads of its stage-0 inputs
// (work that may wait on memory, placed where the thread waits for its loads anyway).
struct NoHook {
    __device__ __forceinline__ void after_loads() const {}
};

// ZQ: the stage-0 inputs r >= R0 ZQ/8 (sequence elements >= M ZQ/8) are known
// to be zero (the zero padding of a transform at least 8/ZQ times the series):
// the loader is asked for R0 ZQ/8 elements and the first DFT skips the zeros
// (ZQ = 8: none known; 4: the upper half known zero; 3: the upper five eighths
// known zero, R0 = 32 only).
// TWFULL: tw is the full stage-1 table W_M^{r j} laid out [r][j] (r < R1, j < R0)
// and the twiddles are read from it through L1 (one 8-byte load per element, a
// half-warp reading 16 consecutive j); else tw is the table W_M^m, m < M, from
// which the power-of-two rows are staged in shared memory.
template <typename T, int M, int SEQ, int EH, int DIR, int MAPM, class LD, class ST, int ZQ = 8,
          bool TWFULL = false, class HK = NoHook>
__device__ __forceinline__ void run_pass(LD &ld, ST &st, const T *__restrict__ tw, const HK &hk = HK{}) {
    using V = typename Vec2T<T>::type;
    constexpr int R0 = radix0(M), R1 = radix1(M);
    constexpr int TPF = M / EH;
    constexpr int THREADS = SEQ * TPF;
    // column mapping with two stage-1 jobs per thread: 16-byte exchange, the
    // thread's stage-1 jobs being the neighbours j and j + 1
    constexpr bool X16 = MAPM == kMapFJ && x16_layout(M, EH) && sizeof(T) == 4;
    constexpr int RL = X16 ? row_ld16(M) : row_ld(M);
    constexpr int JPF0 = M / R0, NJ0 = EH / R0;
    static_assert(EH % R0 == 0 && (R1 == 1 || EH % R1 == 0), "elements per thread vs radix");
    static_assert(MAPM != kMapW || (TPF <= 16 && 32 % TPF == 0), "warp mapping needs <= 16 threads per sequence");
    unsigned char *smem_raw = dyn_smem();
    V *sd = reinterpret_cast<V *>(smem_raw);
    V *tws = reinterpret_cast<V *>(smem_raw + exch_bytes<T, M, SEQ, X16>());
    auto job1 = [](int i) -> Job {   // stage-1 job i of this thread
        if constexpr (X16) {
            Job q;
            q.s = (int)threadIdx.x % SEQ;
            q.j = 2 * ((int)threadIdx.x / SEQ) + i;
            q.t = q.s & 1;
            q.f = q.s >> 1;
            return q;
        } else {
            return job<MAPM, SEQ, TPF, THREADS>(i);
        }
    };
    if constexpr (!TWFULL) {
        fill_twiddles<T, M, THREADS>(tws, tw);
        if constexpr (R1 > 1) __syncthreads();
    }

    T re[EH], im[EH];
    static_assert(ZQ == 8 || ZQ == 4 || (ZQ == 3 && R0 == 32), "known-zero fraction of the first stage");
    constexpr int RL0 = R0 * ZQ / 8;   // stage-0 inputs that can be non-zero
#pragma unroll
    for (int i = 0; i < NJ0; ++i) ld.template load<RL0, JPF0>(job<MAPM, SEQ, TPF, THREADS>(i), &re[i * R0], &im[i * R0]);
    hk.after_loads();
#pragma unroll
    for (int i = 0; i < NJ0; ++i) {
        if constexpr (ZQ < 8) dft_half_zero<R0, DIR, RL0>(&re[i * R0], &im[i * R0]);
        else dft<R0, DIR>(&re[i * R0], &im[i * R0]);
    }
    if constexpr (R1 == 1) {
#pragma unroll
        for (int i = 0; i < NJ0; ++i) st.template store<R0, JPF0>(job<MAPM, SEQ, TPF, THREADS>(i), &re[i * R0], &im[i * R0]);
    } else {
        // a loader that staged its input in the exchange area has been read out by
        // every thread before the first scatter overwrites it
        if constexpr (LoaderStaged<LD>::value) __syncthreads();
        // scatter: stage-0 output r of butterfly j goes to j R0 + r
#pragma unroll
        for (int i = 0; i < NJ0; ++i) {
            const Job q = job<MAPM, SEQ, TPF, THREADS>(i);
            if constexpr (X16) {   // outputs r, r + 1 side by side (j R0 + r stays in one 32-block)
                float4 *p4 = reinterpret_cast<float4 *>(sd + q.s * RL + pad16(q.j * R0));
#pragma unroll
                for (int r = 0; r < R0; r += 2)
                    p4[r / 2] = make_float4(re[i * R0 + r], im[i * R0 + r], re[i * R0 + r + 1], im[i * R0 + r + 1]);
            } else {
                V *p = sd + q.s * RL + pad(q.j * R0);
#pragma unroll
                for (int r = 0; r < R0; ++r) p[pad(r)] = V{re[i * R0 + r], im[i * R0 + r]};
            }
        }
        if constexpr (MAPM == kMapW) __syncwarp(); else __syncthreads();
        constexpr int NJ1 = EH / R1;
        constexpr int LR1 = ilog2c(R1);
#pragma unroll
        for (int i = 0; i < NJ1; ++i) {
            const Job q = job1(i);   // q.j < R0
            T *xr = &re[i * R1], *xi = &im[i * R1];
            if constexpr (X16) {
                if (i == 0) {   // one 16-byte load per r serves both jobs (j even, j + 1)
                    const float4 *p4 = reinterpret_cast<const float4 *>(sd + q.s * RL + q.j);
#pragma unroll
                    for (int r = 0; r < R1; ++r) {
                        const float4 v = p4[pad16(r * R0) / 2];
                        re[r] = v.x; im[r] = v.y;
                        re[R1 + r] = v.z; im[R1 + r] = v.w;
                    }
                }
            } else {
                const V *p = sd + q.s * RL + pad(q.j);
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const V v = p[pad(r * R0)];
                    xr[r] = v.x; xi[r] = v.y;
                }
            }
            // W_M^{r j}: powers of two from the table, the rest as products
            // W^{r j} = W^{h j} W^{(r - h) j}, h the top bit of r (<= LR1 - 1 products deep)
            T wr[R1], wi[R1];
            if constexpr (TWFULL) {
                const V *row = reinterpret_cast<const V *>(tw) + q.j;
#pragma unroll
                for (int r = 1; r < R1; ++r) {
                    const V w = __ldg(row + r * R0);
                    wr[r] = w.x;
                    wi[r] = DIR < 0 ? w.y : -w.y;
                }
            } else {
#pragma unroll
                for (int b = 0; b < LR1; ++b) {
                    const V w = tws[b * R0 + q.j];
                    wr[1 << b] = w.x;
                    wi[1 << b] = DIR < 0 ? w.y : -w.y;
                }
#pragma unroll
                for (int r = 3; r < R1; ++r) {
                    int h = r;   // top bit of r (folds to a constant once unrolled)
                    h |= h >> 1; h |= h >> 2; h |= h >> 4;
                    h = (h + 1) >> 1;
                    if (h != r) {
                        wr[r] = wr[h] * wr[r - h] - wi[h] * wi[r - h];
                        wi[r] = wr[h] * wi[r - h] + wi[h] * wr[r - h];
                    }
                }
            }
#pragma unroll
            for (int r = 1; r < R1; ++r) {
                const T a = xr[r] * wr[r] - xi[r] * wi[r], b = xr[r] * wi[r] + xi[r] * wr[r];
                xr[r] = a; xi[r] = b;
            }
            dft<R1, DIR>(xr, xi);
            // a store that touches no shared memory can take each job as it is done
            if constexpr (StoreEarly<ST>::value) st.template store<R1, R0>(q, xr, xi);
        }
        if constexpr (!StoreEarly<ST>::value) {
#pragma unroll
            for (int i = 0; i < NJ1; ++i) st.template store<R1, R0>(job1(i), &re[i * R1], &im[i * R1]);
        }
    }
}

}  // namespace eng2
}  // namespace fstat
