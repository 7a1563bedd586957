// Packed FP32 arithmetic for the search passes: two independent complex values
// per "PC" (their real parts in one float2, their imaginary parts in another),
// computed with the paired single-precision instructions of sm_100-class GPUs
// (add/sub/mul/fma .f32x2).  A paired instruction occupies the FP32 pipe for
// as long as two scalar ones but takes one issue slot, and the FFT passes are
// bound by instruction issue, so two transforms of the same shape (two jobs of
// a stage, or the two halves of a decimation-in-frequency split) run for the
// issue cost of one.
//
// The DFT codelets below are the forward transform only (e^{-2 pi i jk/R}),
// natural order in and out, on arrays of PC.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fstat {
namespace pk {

__device__ __forceinline__ unsigned long long as_u64(float2 a) {
    return *reinterpret_cast<unsigned long long *>(&a);
}
__device__ __forceinline__ float2 as_f2(unsigned long long u) { return *reinterpret_cast<float2 *>(&u); }

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
    return as_f2(r);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

struct PC {
    float2 re, im;
};

__device__ __forceinline__ PC add(const PC &a, const PC &b) { return {padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ PC sub(const PC &a, const PC &b) { return {psub(a.re, b.re), psub(a.im, b.im)}; }
// a + i^K b (K mod 4): a quarter turn costs no instruction, only a choice of
// add or subtract per component
template <int K>
__device__ __forceinline__ PC add_rot(const PC &a, const PC &b) {
    constexpr int k = ((K % 4) + 4) % 4;
    if constexpr (k == 0) return add(a, b);
    else if constexpr (k == 2) return sub(a, b);
    else if constexpr (k == 1) return {psub(a.re, b.im), padd(a.im, b.re)};
    else return {padd(a.re, b.im), psub(a.im, b.re)};
}

// x (c + i s) for compile-time c, s (the negated s is a constant too)
__device__ __forceinline__ PC cmul_c(const PC &x, float c, float s) {
    return {pfma(x.re, bc(c), pmul(x.im, bc(-s))), pfma(x.re, bc(s), pmul(x.im, bc(c)))};
}
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
// x w for run-time twiddles w (one per lane of the pair); the negation is an
// operand modifier of the paired multiply, not an instruction
__device__ __forceinline__ PC cmul(const PC &x, const PC &w) {
    return {pfma(x.re, w.re, pmul(x.im, pneg(w.im))), pfma(x.re, w.im, pmul(x.im, w.re))};
}

// e^{-2 pi i e / 16}
__host__ __device__ constexpr float w16c(int e) {
    constexpr float t[16] = {1.f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                             0.f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f,
                             -1.f, -0.92387953251128675613f, -0.70710678118654752440f, -0.38268343236508977173f,
                             0.f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f};
    return t[e & 15];
}
__host__ __device__ constexpr float w16s(int e) { return -w16c((e + 12) & 15); }   // -sin(2 pi e / 16)

// x W16^e: a multiple of 4 is a quarter turn, folded by the caller through
// add_rot; other exponents multiply
__device__ __forceinline__ PC mul_w16(const PC &x, int e) {
    e &= 15;
    return cmul_c(x, w16c(e), w16s(e));
}

// 4-point DFT; input 2 carries a pending factor i^K2 (a quarter turn from the
// caller's twiddle, applied here through the choice of add or subtract).
// Outputs y_p = sum_q x_q (-i)^{qp}.  HALF: only y_0 and y_1.
template <int K2 = 0, bool HALF = false>
__device__ __forceinline__ void dft4(PC &x0, PC &x1, PC &x2, PC &x3) {
    const PC t0 = add_rot<K2>(x0, x2), t1 = add_rot<K2 + 2>(x0, x2);
    const PC t2 = add(x1, x3), t3 = sub(x1, x3);
    x0 = add(t0, t2);
    x1 = add_rot<3>(t1, t3);        // t1 - i t3
    if constexpr (!HALF) {
        x2 = sub(t0, t2);
        x3 = add_rot<1>(t1, t3);    // t1 + i t3
    }
}

// 16-point DFT by radix 4: sub-DFTs over x[4m + q], twiddles W16^{qk}, 4-point
// DFTs across q.  NZ: inputs from NZ on are zero (not read).  LOWER: only the
// outputs 0 .. 7.
template <int NZ = 16, bool LOWER = false>
__device__ __forceinline__ void dft16(PC *x) {
    static_assert(NZ >= 4 && NZ <= 16, "each sub-DFT keeps a non-zero input");
    PC s[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // inputs 4m + q, m < 4, of which those below NZ are non-zero
        const int nz = (NZ - q + 3) / 4;   // non-zero inputs of this sub-DFT (compile time once unrolled)
#pragma unroll
        for (int m = 0; m < 4; ++m) s[q][m] = x[4 * m + q < NZ ? 4 * m + q : 0];
        if (nz >= 4) {
            dft4(s[q][0], s[q][1], s[q][2], s[q][3]);
        } else if (nz == 3) {   // x3 = 0
            const PC a = s[q][0], b = s[q][1], c = s[q][2];
            const PC t0 = add(a, c), t1 = sub(a, c);
            s[q][0] = add(t0, b);
            s[q][2] = sub(t0, b);
            s[q][1] = add_rot<3>(t1, b);
            s[q][3] = add_rot<1>(t1, b);
        } else if (nz == 2) {   // x2 = x3 = 0
            const PC a = s[q][0], b = s[q][1];
            s[q][0] = add(a, b);
            s[q][2] = sub(a, b);
            s[q][1] = add_rot<3>(a, b);
            s[q][3] = add_rot<1>(a, b);
        } else {                // only x0
            s[q][1] = s[q][2] = s[q][3] = s[q][0];
        }
    }
    // twiddles W16^{qk}: exponents 0 (k or q = 0), quarter turns at qk = 4, else a multiply
#pragma unroll
    for (int q = 1; q < 4; ++q)
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if ((q * k) % 4 != 0) s[q][k] = mul_w16(s[q][k], q * k);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        PC a = s[0][k], b = s[1][k], c = s[2][k], d = s[3][k];
        // q = 2, k = 2: W16^4 = -i = i^3, pending on input 2
        if (k == 2) dft4<3, LOWER>(a, b, c, d);
        else dft4<0, LOWER>(a, b, c, d);
        x[k] = a;
        x[k + 4] = b;
        if constexpr (!LOWER) {
            x[k + 8] = c;
            x[k + 12] = d;
        }
    }
}

}  // namespace pk
}  // namespace fstat
