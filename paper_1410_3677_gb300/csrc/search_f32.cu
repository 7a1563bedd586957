// FP32 instantiations of the search passes (FSTAT_FP32_BATCHED): the two-stage
// engine for transform lengths 2^12 .. 2^19, the radix-8 engine otherwise (and
// whenever the plan selects it).
#include "passes2.cuh"
#include "search_launch.cuh"

namespace fstat {
namespace {

template <int LOGN, bool LOWER>
void launch_pass2(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0, int64_t nc,
                  cudaStream_t s, const CellBufs &cb, const ScratchLoad2<Cfg2<LOGN, 2>> &ld2,
                  const float *tw_in1) {
    using C2 = Cfg2<LOGN, 2>;
    SearchEpi2<C2, LOWER> st2{};
    st2.norm = cb.norm;
    st2.n_spin = (int)p.desc.n_spin;
    st2.c0 = c0;
    st2.s0 = s0;
    st2.cell_base = (uint32_t)((int64_t)band_idx * p.desc.n_sky * p.desc.n_spin);
    st2.bin_lo = b.lo;
    st2.bin_hi = b.hi;
    st2.thr = (float)p.desc.thr_2F;
    st2.out = p.cand;
    st2.count = p.cand_count;
    st2.cap = (unsigned long long)p.cand_capacity;
    auto k2 = k_pass2<LOGN, 2, eng2::kMapW, ScratchLoad2<C2>, SearchEpi2<C2, LOWER>>;
    static bool attr2 = false;
    if (!attr2) { set_smem(k2, C2::SMEM); attr2 = true; }
    k2<<<dim3(C2::TILES, (unsigned)nc), C2::THREADS, C2::SMEM, s>>>(ld2, st2, tw_in1);
}

template <int LOGN>
int launch_search2(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0,
                   int64_t nc, cudaStream_t s, cudaEvent_t mid, const CellBufs &cb) {
    using C1 = Cfg2<LOGN, 1>;
    using C2 = Cfg2<LOGN, 2>;
    const TwiddleSet *tw = p.twiddles(LOGN);
    const int n_spin = (int)p.desc.n_spin;

    SearchLoad2<C1> ld1{};
    ld1.w = reinterpret_cast<const float4 *>(cb.w);
    ld1.w_stride = p.w_stride;
    ld1.n = (int)b.n;
    ld1.chirp = p.chirp_fx + (int64_t)band_idx * n_spin;
    ld1.n_spin = n_spin;
    ld1.c0 = c0;
    ld1.s0 = s0;
    ScratchStore2<C1> st1{};
    st1.scratch = reinterpret_cast<float2 *>(cb.scratch);
    st1.lo = tw->lo_f;
    st1.hi = tw->hi_f;
    auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2<C1>, ScratchStore2<C1>>;
    static bool attr1 = false;
    if (!attr1) { set_smem(k1, C1::SMEM); attr1 = true; }
    k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw->in2_f);
    if (mid) cudaEventRecord(mid, s);

    ScratchLoad2<C2> ld2{};
    ld2.scratch = reinterpret_cast<const float2 *>(cb.scratch);
    if (b.hi < (int64_t)C2::N / 2) launch_pass2<LOGN, true>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw->in1_f);
    else launch_pass2<LOGN, false>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw->in1_f);
    return 2;
}

}  // namespace

int launch_search_cells_f32(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                            int64_t c0, int64_t nc, cudaStream_t s, cudaEvent_t mid,
                            const CellBufs &cb) {
    if (p.engine == 2) {
        switch (b.logn) {
            case 12: return launch_search2<12>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 13: return launch_search2<13>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 14: return launch_search2<14>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 15: return launch_search2<15>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 16: return launch_search2<16>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 17: return launch_search2<17>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 18: return launch_search2<18>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 19: return launch_search2<19>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            default: break;
        }
    }
    return launch_search_dispatch<float>(p, band_idx, b, s0, c0, nc, s, mid, cb);
}
}  // namespace fstat
