// FP32 instantiations of the search passes (FSTAT_FP32_BATCHED): the two-stage
// engine for transform lengths 2^12 .. 2^19 (both passes in one ticket-ordered
// launch, or as two launches), the radix-8 engine otherwise (and whenever the
// plan selects it).
#include <algorithm>

#include "passes2.cuh"
#include "passes3.cuh"
#include "search_launch.cuh"

namespace fstat {
namespace {

template <int LOGN, bool LOWER, int TS = 256>
SearchEpi2<Cfg2<LOGN, 2, TS>, LOWER> make_epi(const Plan &p, int band_idx, const BandDev &b, int64_t c0,
                                              int64_t s0, const CellBufs &cb) {
    SearchEpi2<Cfg2<LOGN, 2, TS>, LOWER> st2{};
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
    return st2;
}

template <int LOGN, bool LOWER, int TS, class LD2>
void launch_pass2(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0, int64_t nc,
                  cudaStream_t s, const CellBufs &cb, const LD2 &ld2, const TwiddleSet *tw, size_t extra) {
    using C2 = Cfg2<LOGN, 2, TS>;
    const auto st2 = make_epi<LOGN, LOWER, TS>(p, band_idx, b, c0, s0, cb);
    auto k2 = k_pass2<LOGN, 2, eng2::kMapW, LD2, SearchEpi2<C2, LOWER>, TS>;
    static bool attr2 = false;
    if (!attr2) { set_smem(k2, C2::SMEM + extra); attr2 = true; }
    k2<<<dim3(C2::TILES, (unsigned)nc), C2::THREADS, C2::SMEM + extra, s>>>(ld2, st2, tw->s1_f);
}

// The paired pass 2 (512-point rows) in CTAs of TS / 32 rows, one warp per row.
template <int LOGN, bool LOWER, int TS>
void launch_pass2p(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0, int64_t nc,
                   cudaStream_t s, const CellBufs &cb, const ScratchLoad2<Cfg2<LOGN, 2>> &ld2,
                   const TwiddleSet *tw) {
    using D2 = Cfg2<LOGN, 2, TS>;
    ScratchLoadTMA<D2> lt{};
    lt.scratch = ld2.scratch;
    lt.tw = ld2.tw;
    lt.pf_dist = p.pf_dist_pk;   // the paired pass gains nothing from L2 prefetch ahead
    lt.err = p.qerr;
    const auto ep = make_epi<LOGN, LOWER, TS>(p, band_idx, b, c0, s0, cb);
    auto k2 = p3::k_pass2p<LOGN, LOWER, TS>;
    constexpr size_t smem2 = p3::pass2p_smem<D2>() + 16;   // staged tile + mbarrier
    static bool attr2p = false;
    if (!attr2p) { set_smem(k2, smem2); attr2p = true; }
    k2<<<dim3(D2::TILES, (unsigned)nc), D2::THREADS, smem2, s>>>(lt, ep, tw->p512_f);
}

template <int LOGN, bool LOWER>
int launch_two(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0, int64_t nc,
               cudaStream_t s, cudaEvent_t mid, const CellBufs &cb, const SearchLoad2<Cfg2<LOGN, 1>> &ld1,
               const ScratchStore2<Cfg2<LOGN, 1>> &st1, const ScratchLoad2<Cfg2<LOGN, 2>> &ld2,
               const TwiddleSet *tw) {
    using C1 = Cfg2<LOGN, 1>;
    using C2 = Cfg2<LOGN, 2>;
    // 512-point rows (N_fft = 2^18, 2^19): pass 2 in paired FP32 arithmetic; at 2^18
    // (512-point columns) also pass 1 with packed = 2 or 3
    const bool pk2 = (LOGN == 18 || LOGN == 19) && p.packed >= 1 && p.tma && p.p2_threads == 128 && tw->p512_f;
    const bool pk1 = pk2 && LOGN == 18 && p.packed >= 2;
    if constexpr (LOGN == 18) {
        if (pk1) {   // packed = 2: both stages paired; 3: scalar first stage, paired second
            const bool z3 = 8 * b.n <= 3 * (int64_t)C1::N;
            const bool hy = p.packed == 3;
            auto k1 = hy ? (z3 ? p3::k_pass1h<LOGN, 3> : p3::k_pass1h<LOGN, 4>)
                         : (z3 ? p3::k_pass1p<LOGN, 3> : p3::k_pass1p<LOGN, 4>);
            static bool attr1p[4] = {false, false, false, false};
            const int ai = (hy ? 2 : 0) + (z3 ? 1 : 0);
            if (!attr1p[ai]) { set_smem(k1, C1::SMEM); attr1p[ai] = true; }
            k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw->p512_f);
        }
    }
    // columns known zero beyond 3/8 of their length (radix-32 first stage) or 1/2
    bool launched = pk1;
    if constexpr (eng2::radix0(C1::M) == 32) {
        if (!launched && 8 * b.n <= 3 * (int64_t)C1::N && p.share_chirp) {
            SearchLoad2S<C1> l1s{};
            static_cast<SearchLoad2<C1> &>(l1s) = ld1;
            auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2S<C1>, ScratchStore2<C1>, 256, 3>;
            static bool attr3s = false;
            if (!attr3s) { set_smem(k1, C1::SMEM); attr3s = true; }
            k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(l1s, st1, tw->s2_f);
            launched = true;
        }
        if (!launched && 8 * b.n <= 3 * (int64_t)C1::N) {
            auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2<C1>, ScratchStore2<C1>, 256, 3>;
            static bool attr3 = false;
            if (!attr3) { set_smem(k1, C1::SMEM); attr3 = true; }
            k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw->s2_f);
            launched = true;
        }
    }
    if (!launched && p.share_chirp) {
        SearchLoad2S<C1> l1s{};
        static_cast<SearchLoad2<C1> &>(l1s) = ld1;
        auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2S<C1>, ScratchStore2<C1>, 256, 4>;
        static bool attr1s = false;
        if (!attr1s) { set_smem(k1, C1::SMEM); attr1s = true; }
        k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(l1s, st1, tw->s2_f);
        launched = true;
    }
    if (!launched) {
        auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2<C1>, ScratchStore2<C1>, 256, 4>;
        static bool attr1 = false;
        if (!attr1) { set_smem(k1, C1::SMEM); attr1 = true; }
        k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw->s2_f);
    }
    if (mid) record_timing_event(mid, s);
    if constexpr (LOGN == 16 || LOGN == 17) {   // 256-point rows: two per warp, packed
        if (p.packed >= 1 && p.tma && p.p2_threads != 256 && p.p2_rows) {
            using D2 = Cfg2<LOGN, 2, 32>;
            ScratchLoadTMA<D2> lt{};
            lt.scratch = ld2.scratch;
            lt.tw = ld2.tw;
            lt.pf_dist = 0;
            lt.err = p.qerr;
            const auto ep = make_epi<LOGN, LOWER, 32>(p, band_idx, b, c0, s0, cb);
            auto k2 = p3::k_pass2r<LOGN, LOWER>;
            constexpr size_t smem2 = (size_t)2 * D2::F * D2::N1 * sizeof(float2) + 16;   // staged rows + mbarrier
            static bool attr2r = false;
            if (!attr2r) { set_smem(k2, smem2); attr2r = true; }
            k2<<<dim3(D2::TILES, (unsigned)nc), D2::THREADS, smem2, s>>>(
                lt, ep, reinterpret_cast<const float2 *>(tw->in1_f));
            return 2;
        }
    }
    if constexpr (LOGN == 18 || LOGN == 19) {
        if (pk2) {
            if (p.p2_ts == 32) launch_pass2p<LOGN, LOWER, 32>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw);
            else if (p.p2_ts == 64) launch_pass2p<LOGN, LOWER, 64>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw);
            else launch_pass2p<LOGN, LOWER, 128>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw);
            return 2;
        }
    }
    if (p.tma && p.p2_threads == 128) {   // smaller tiles, six CTAs per SM
        ScratchLoadTMA<Cfg2<LOGN, 2, 128>> lt{};
        lt.scratch = ld2.scratch;
        lt.tw = ld2.tw;
        lt.pf_dist = 2 * ld2.pf_dist;
        lt.err = p.qerr;
        launch_pass2<LOGN, LOWER, 128>(p, band_idx, b, s0, c0, nc, s, cb, lt, tw, 16);
    } else if (p.tma) {   // rows staged by bulk copies; an 8-byte mbarrier after the shared memory
        ScratchLoadTMA<C2> lt{};
        lt.scratch = ld2.scratch;
        lt.tw = ld2.tw;
        lt.pf_dist = ld2.pf_dist;
        lt.err = p.qerr;
        launch_pass2<LOGN, LOWER, 256>(p, band_idx, b, s0, c0, nc, s, cb, lt, tw, 16);
    } else {
        launch_pass2<LOGN, LOWER, 256>(p, band_idx, b, s0, c0, nc, s, cb, ld2, tw, 0);
    }
    return 2;
}

template <int LOGN, bool LOWER>
int launch_fused(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0, int64_t nc,
                 cudaStream_t s, const CellBufs &cb, const SearchLoad2<Cfg2<LOGN, 1>> &ld1,
                 const ScratchStore2<Cfg2<LOGN, 1>> &st1, const ScratchLoad2<Cfg2<LOGN, 2>> &ld2,
                 const TwiddleSet *tw) {
    using C1 = Cfg2<LOGN, 1>;
    using C2 = Cfg2<LOGN, 2>;
    const auto st2 = make_epi<LOGN, LOWER>(p, band_idx, b, c0, s0, cb);
    // counters zeroed by the caller; the test hook names a plan-wide item (cell)
    const int64_t wh = p.withhold_item >= c0 && p.withhold_item < c0 + nc ? p.withhold_item - c0 : -1;
    const int tpi = std::min(p.fused_tpi, std::min(C1::TILES, C2::TILES));
    FusedCtl ctl{cb.ctl, cb.ctl + 1, cb.ctl + 1 + nc, p.qerr, nc, p.fused_slots, p.fused_ahead, tpi, wh};
    constexpr size_t smem = C1::SMEM > C2::SMEM ? C1::SMEM : C2::SMEM;
    // pass-1 columns known zero beyond 3/8 of their length (radix-32 first stage) or 1/2
    const bool z3 = eng2::radix0(C1::M) == 32 && 8 * b.n <= 3 * (int64_t)C1::N;
    auto k = z3 ? k_search_fused<LOGN, LOWER, eng2::radix0(C1::M) == 32 ? 3 : 4>
                : k_search_fused<LOGN, LOWER, 4>;
    static int resident[2] = {0, 0};   // CTAs of each variant that fit on the device at once
    int &res = resident[z3 ? 1 : 0];
    if (!res) {
        set_smem(k, smem);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
        res = std::max(1, sms * std::max(per_sm, 1));
    }
    const int64_t items = (nc + p.fused_ahead) * (int64_t)(C1::TILES / tpi + C2::TILES / tpi);
    const unsigned grid = (unsigned)std::min<int64_t>(items, res);
    k<<<grid, 256, smem, s>>>(ld1, st1, ld2, st2, tw->s1_f, tw->s2_f, ctl);
    return 1;
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
    ScratchLoad2<C2> ld2{};
    ld2.scratch = reinterpret_cast<const float2 *>(cb.scratch);
    ld2.tw = {tw->lo_f, tw->hi_f};
    ld2.pf_dist = p.pf_dist;
    const bool lower = b.hi < (int64_t)C2::N / 2;
    if (fused_supported(p, LOGN) && cb.ctl) {
        return lower ? launch_fused<LOGN, true>(p, band_idx, b, s0, c0, nc, s, cb, ld1, st1, ld2, tw)
                     : launch_fused<LOGN, false>(p, band_idx, b, s0, c0, nc, s, cb, ld1, st1, ld2, tw);
    }
    return lower ? launch_two<LOGN, true>(p, band_idx, b, s0, c0, nc, s, mid, cb, ld1, st1, ld2, tw)
                 : launch_two<LOGN, false>(p, band_idx, b, s0, c0, nc, s, mid, cb, ld1, st1, ld2, tw);
}

// Interbinning form: both passes at length 2^LOGN = n_fft / 2 (pass 1 without
// the zero-half assumption), pass 2 in overlapping row tiles.
template <int LOGN>
int launch_interbin(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0,
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
    auto k1 = k_pass2<LOGN, 1, eng2::kMapFJ, SearchLoad2<C1>, ScratchStore2<C1>, 256, 8>;
    static bool attr1 = false;
    if (!attr1) { set_smem(k1, C1::SMEM); attr1 = true; }
    k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw->s2_f);
    if (mid) record_timing_event(mid, s);
    if (p.tma) {   // 128-thread row tiles staged by bulk copies (8-byte mbarrier after the smem)
        using D2 = Cfg2<LOGN, 2, 128>;
        ScratchLoadIBTMA<D2> ld2{};
        ld2.scratch = reinterpret_cast<const float2 *>(cb.scratch);
        ld2.tw = {tw->lo_f, tw->hi_f};
        ld2.pf_dist = 2 * p.pf_dist;
        ld2.err = p.qerr;
        const auto ep = make_epi<LOGN, false, 128>(p, band_idx, b, c0, s0, cb);
        auto k2 = k_pass2_ib<LOGN, 128, ScratchLoadIBTMA<D2>>;
        static bool attr2t = false;
        if (!attr2t) { set_smem(k2, D2::SMEM + 16); attr2t = true; }
        k2<<<dim3(IBGeom<LOGN, 128>::TILES, (unsigned)nc), D2::THREADS, D2::SMEM + 16, s>>>(ld2, ep, tw->in1_f);
        return 2;
    }
    ScratchLoadIB<C2> ld2{};
    ld2.scratch = reinterpret_cast<const float2 *>(cb.scratch);
    ld2.tw = {tw->lo_f, tw->hi_f};
    const auto ep = make_epi<LOGN, false>(p, band_idx, b, c0, s0, cb);
    auto k2 = k_pass2_ib<LOGN, 256, ScratchLoadIB<C2>>;
    static bool attr2 = false;
    if (!attr2) { set_smem(k2, C2::SMEM); attr2 = true; }
    k2<<<dim3(IBGeom<LOGN>::TILES, (unsigned)nc), C2::THREADS, C2::SMEM, s>>>(ld2, ep, tw->in1_f);
    return 2;
}

}  // namespace

bool interbin_supported(int logn) { return logn - 1 >= 12 && logn - 1 <= 19; }

bool fused_supported(const Plan &p, int logn) {
    return p.engine == 2 && p.fused && !p.interbin && logn >= 12 && logn <= 19;
}

int launch_search_cells_f32(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                            int64_t c0, int64_t nc, cudaStream_t s, cudaEvent_t mid,
                            const CellBufs &cb) {
    if (p.interbin) {
        switch (b.logn - 1) {
            case 12: return launch_interbin<12>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 13: return launch_interbin<13>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 14: return launch_interbin<14>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 15: return launch_interbin<15>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 16: return launch_interbin<16>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 17: return launch_interbin<17>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 18: return launch_interbin<18>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            case 19: return launch_interbin<19>(p, band_idx, b, s0, c0, nc, s, mid, cb);
            default: return -1;
        }
    }
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
