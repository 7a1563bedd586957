// Double-float arithmetic: a value held as the unevaluated sum hi + lo of two
// floats (about 48 significant bits), built from Knuth's two-sum and the exact
// product of two floats by a fused multiply-add (Dekker's two-product in its
// FMA form).  The per-sample Roemer delay of the FP32 form is evaluated this
// way on the FP32 pipes instead of in FP64, which GB300 runs at 1/64 of the
// FP32 rate.  The error-free transforms need every sum and product rounded on
// its own, so on the device they use the explicitly rounded intrinsics, which
// the compiler never contracts into fused multiply-adds (a host build compiles
// with contraction off).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace fstat {

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#endif

struct DF {
    float hi, lo;
};

// a + b exactly, as s + e
__host__ __device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    const float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
    return DF{s, e};
}

// the same when |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    return DF{s, DF_SUB(b, DF_SUB(s, a))};
}

__host__ __device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, DF_ADD(s.lo, DF_ADD(a.lo, b.lo)));
}

__host__ __device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// a b to about 2^-46 relative (the lo x lo term is left out)
__host__ __device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = DF_MUL(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);   // exact low part of hi x hi
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ DF df_from_double(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}

// x = I + f with I an integer (returned as float, exact) and f in [0, 1)
// rounded to float
__host__ __device__ __forceinline__ float df_split_floor(DF x, float *frac) {
    float fl = floorf(x.hi);
    float f = DF_ADD(DF_SUB(x.hi, fl), x.lo);   // x.hi - fl is exact for |x.hi| < 2^23
    if (f < 0.f) { f += 1.f; fl -= 1.f; }
    if (f >= 1.f) { f -= 1.f; fl += 1.f; }   // also a tiny negative f that rounded to 1
    *frac = f;
    return fl;
}

#undef DF_ADD
#undef DF_SUB
#undef DF_MUL

}  // namespace fstat
