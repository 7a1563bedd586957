// Generic power-of-two transforms on the two-pass engine: pairs of contiguous
// sequences in global memory, natural order in and out.  Used for the per-band
// FFT upsample (directly, or inside Bluestein's algorithm for lengths that are
// not powers of two) and by the diagnostic transform entry point.
#include "passes.cuh"

namespace fstat {

namespace {

template <typename T, int LOGN, int DIR>
int generic_t(const TwiddleSet &tw, const void *in, void *out, int64_t ntr, void *scratch,
              cudaStream_t s) {
    using C1 = Cfg<T, LOGN, 1>;
    using C2 = Cfg<T, LOGN, 2>;
    using V = typename Vec2<T>::type;
    const T *tin1, *tin2, *tlo, *thi;
    if constexpr (sizeof(T) == 4) { tin1 = tw.in1_f; tin2 = tw.in2_f; tlo = tw.lo_f; thi = tw.hi_f; }
    else { tin1 = tw.in1_d; tin2 = tw.in2_d; tlo = tw.lo_d; thi = tw.hi_d; }
    const unsigned pairs = (unsigned)((ntr + 1) / 2);

    GenericLoad<T, C1> ld1{};
    ld1.in = reinterpret_cast<const V *>(in);
    ld1.n_tr = ntr;
    ScratchStore<T, C1, DIR> st1{};
    st1.scratch = reinterpret_cast<V *>(scratch);
    st1.lo = tlo;
    st1.hi = thi;
    st1.n_tr = ntr;
    auto k1 = k_pass<T, LOGN, 1, DIR, eng::kMapFJ, GenericLoad<T, C1>, ScratchStore<T, C1, DIR>>;
    static bool a1 = false;
    if (!a1) { set_smem(k1, C1::SMEM); a1 = true; }
    k1<<<dim3(C1::TILES, pairs), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tin2);

    ScratchLoad<T, C2> ld2{};
    ld2.scratch = reinterpret_cast<const V *>(scratch);
    GenericStore<T, C2> st2{};
    st2.out = reinterpret_cast<V *>(out);
    st2.n_tr = ntr;
    auto k2 = k_pass<T, LOGN, 2, DIR, eng::kMapJ, ScratchLoad<T, C2>, GenericStore<T, C2>>;
    static bool a2 = false;
    if (!a2) { set_smem(k2, C2::SMEM); a2 = true; }
    k2<<<dim3(C2::TILES, pairs), C2::THREADS, C2::SMEM, s>>>(ld2, st2, tin1);
    return 2;
}

template <typename T, int DIR>
int generic_dispatch(const TwiddleSet &tw, const void *in, void *out, int64_t ntr, void *scratch,
                     cudaStream_t s) {
    switch (tw.logn) {
        case 8: return generic_t<T, 8, DIR>(tw, in, out, ntr, scratch, s);
        case 9: return generic_t<T, 9, DIR>(tw, in, out, ntr, scratch, s);
        case 10: return generic_t<T, 10, DIR>(tw, in, out, ntr, scratch, s);
        case 11: return generic_t<T, 11, DIR>(tw, in, out, ntr, scratch, s);
        case 12: return generic_t<T, 12, DIR>(tw, in, out, ntr, scratch, s);
        case 13: return generic_t<T, 13, DIR>(tw, in, out, ntr, scratch, s);
        case 14: return generic_t<T, 14, DIR>(tw, in, out, ntr, scratch, s);
        case 15: return generic_t<T, 15, DIR>(tw, in, out, ntr, scratch, s);
        case 16: return generic_t<T, 16, DIR>(tw, in, out, ntr, scratch, s);
        case 17: return generic_t<T, 17, DIR>(tw, in, out, ntr, scratch, s);
        case 18: return generic_t<T, 18, DIR>(tw, in, out, ntr, scratch, s);
        case 19: return generic_t<T, 19, DIR>(tw, in, out, ntr, scratch, s);
        case 20: return generic_t<T, 20, DIR>(tw, in, out, ntr, scratch, s);
        default: return -1;
    }
}

}  // namespace

int launch_fft_generic(const TwiddleSet &tw, bool fp64, int dir, const void *in, void *out,
                       int64_t n_transforms, void *scratch, cudaStream_t s) {
    if (fp64) {
        return dir < 0 ? generic_dispatch<double, -1>(tw, in, out, n_transforms, scratch, s)
                       : generic_dispatch<double, 1>(tw, in, out, n_transforms, scratch, s);
    }
    return dir < 0 ? generic_dispatch<float, -1>(tw, in, out, n_transforms, scratch, s)
                   : generic_dispatch<float, 1>(tw, in, out, n_transforms, scratch, s);
}

}  // namespace fstat
