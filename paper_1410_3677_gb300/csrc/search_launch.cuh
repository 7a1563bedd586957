// Launch helpers for the two search passes, instantiated per transform length
// by search_f32.cu and search_f64.cu.
#pragma once

#include <type_traits>

#include "passes.cuh"

namespace fstat {

template <typename T, int LOGN, int TS, int EHT>
int launch_search_t(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0,
                    int64_t nc, cudaStream_t s, cudaEvent_t mid, const CellBufs &cb) {
    using C1 = Cfg<T, LOGN, 1, TS, EHT>;
    using C2 = Cfg<T, LOGN, 2, TS, EHT>;
    using V = typename Vec2<T>::type;
    const TwiddleSet *tw = p.twiddles(LOGN);
    const T *tin1, *tin2, *tlo, *thi;
    if constexpr (sizeof(T) == 4) { tin1 = tw->in1_f; tin2 = tw->in2_f; tlo = tw->lo_f; thi = tw->hi_f; }
    else { tin1 = tw->in1_d; tin2 = tw->in2_d; tlo = tw->lo_d; thi = tw->hi_d; }
    const int n_spin = (int)p.desc.n_spin;

    using LD1 = std::conditional_t<sizeof(T) == 4, SearchLoadF32<C1>, SearchLoadF64<C1>>;
    LD1 ld1{};
    if constexpr (sizeof(T) == 4) {
        ld1.w = reinterpret_cast<const float4 *>(cb.w);
        ld1.chirp = p.chirp_fx + (int64_t)band_idx * n_spin;
    } else {
        ld1.w = reinterpret_cast<const W64 *>(cb.w);
        ld1.chirp = p.chirp_d + (int64_t)band_idx * n_spin;
    }
    ld1.w_stride = p.w_stride;
    ld1.n = (int)b.n;
    ld1.n_spin = n_spin;
    ld1.c0 = c0;
    ld1.s0 = s0;
    using ST1 = ScratchStore<T, C1, -1>;
    ST1 st1{};
    st1.scratch = reinterpret_cast<V *>(cb.scratch);
    st1.lo = tlo;
    st1.hi = thi;
    st1.n_tr = 2 * nc;
    auto k1 = k_pass<T, LOGN, 1, -1, eng::kMapFJ, LD1, ST1, TS, EHT>;
    static bool attr1 = false;
    if (!attr1) { set_smem(k1, C1::SMEM); attr1 = true; }
    k1<<<dim3(C1::TILES, (unsigned)nc), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tin2);
    if (mid) record_timing_event(mid, s);

    using LD2 = ScratchLoad<T, C2>;
    using ST2 = SearchEpi<T, C2>;
    LD2 ld2{};
    ld2.scratch = reinterpret_cast<const V *>(cb.scratch);
    ST2 st2{};
    st2.norm = cb.norm;
    st2.n_spin = n_spin;
    st2.c0 = c0;
    st2.s0 = s0;
    st2.cell_base = (uint32_t)((int64_t)band_idx * p.desc.n_sky * p.desc.n_spin);
    st2.bin_lo = b.lo;
    st2.bin_hi = b.hi;
    st2.thr = (T)p.desc.thr_2F;
    st2.out = p.cand;
    st2.count = p.cand_count;
    st2.cap = (unsigned long long)p.cand_capacity;
    auto k2 = k_pass<T, LOGN, 2, -1, eng::kMapW, LD2, ST2, TS, EHT>;
    static bool attr2 = false;
    if (!attr2) { set_smem(k2, C2::SMEM); attr2 = true; }
    k2<<<dim3(C2::TILES, (unsigned)nc), C2::THREADS, C2::SMEM, s>>>(ld2, st2, tin1);
    return 2;
}

template <typename T>
int launch_search_dispatch(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c0,
                           int64_t nc, cudaStream_t s, cudaEvent_t mid, const CellBufs &cb) {
    switch (b.logn) {
        case 8: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 8, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 8, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 9: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 9, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 9, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 10: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 10, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 10, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 11: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 11, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 11, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 12: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 12, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 12, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 13: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 13, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 13, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 14: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 14, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 14, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 15: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 15, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 15, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 16: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 16, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 16, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 17: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 17, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 17, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 18: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 18, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 18, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 19: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 19, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 19, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        case 20: return p.elems_per_thread == 8 && sizeof(T) == 4 ? launch_search_t<T, 20, 256, 8>(p, band_idx, b, s0, c0, nc, s, mid, cb) : launch_search_t<T, 20, 256, 0>(p, band_idx, b, s0, c0, nc, s, mid, cb);
        default: return -1;
    }
}

}  // namespace fstat
