// Persistent FP32 search kernel: one launch per sky batch runs both FFT passes
// of every cell, fed by a device-side work queue -- the GPU counterpart of the
// paper's task farm (Sect. 3, 3.1), where independent sky positions and
// spindowns are handed to whichever worker is free.
//
// Work items are tiles of one pass of one batch of B cells, in the order
//   P1(0), P1(1), P2(0), P1(2), P2(1), ..., P1(nb-1), P2(nb-2), P2(nb-1)
// (pass-2 tiles of a batch follow the pass-1 tiles of the next batch).  A
// pass-2 tile of batch b needs every pass-1 tile of b; a pass-1 tile of batch b
// reuses scratch slot b mod S and needs every pass-2 tile of b - S.  Both
// dependencies point to items dequeued earlier, so the queue cannot deadlock;
// every wait is bounded (1 s) and sets an error word that the host reports as
// FSTAT_ERR_TIMEOUT.
//
// Each CTA is warp-specialised: one producer warp dequeues the next item, waits
// for its dependency and copies its input tile into a free shared-memory
// buffer with bulk copies (cp.async.bulk, completion on an mbarrier); four
// consumer warps transform the previous tile in place in the other buffer.
#include <algorithm>

#include "passes.cuh"
#include "sync_ptx.cuh"

namespace fstat {

namespace {

constexpr int kEH = 16;                    // complex elements per thread per transform
constexpr int kETile = 2048;               // complex elements of one transform per tile
constexpr int kNC = kETile / kEH;          // consumer threads (4 warps)
constexpr int kThreads = kNC + 32;         // + one producer warp
// a staged tile (two transforms of complex float) or its padded exchange layout
constexpr int kStageBytes = 2 * kETile * 8;
constexpr uint64_t kWaitNs = 1000000000ull;

template <int LOGN>
struct PC {
    static constexpr int LOGN1 = LOGN / 2;
    static constexpr int N1 = 1 << LOGN1, N2 = 1 << (LOGN - LOGN1), N = 1 << LOGN;
    static constexpr int F1 = kETile / N2;   // columns per pass-1 tile
    static constexpr int F2 = kETile / N1;   // rows per pass-2 tile
    static constexpr int T = N / kETile;     // tiles per cell and pass
    static constexpr int TW1 = eng::tw_entries(N2);
    static constexpr int TW2 = eng::tw_entries(N1);
    static constexpr int E1 = (int)eng::exch_bytes<float, N2, F1>();
    static constexpr int E2 = (int)eng::exch_bytes<float, N1, F2>();
    static constexpr int BUF = ((kStageBytes > E1 ? (kStageBytes > E2 ? kStageBytes : E2)
                                                   : (E1 > E2 ? E1 : E2)) + 127) / 128 * 128;
    static constexpr size_t SMEM = 2 * (size_t)BUF + 8 * (size_t)(TW1 + TW2) + 64;
    static_assert(F1 >= 1 && F2 >= 1 && F1 <= N1 && F2 <= N2, "tile shape");
    // Cfg-compatible views for the loaders/storers of passes.cuh
    struct C1 {
        static constexpr int LOGN1 = PC::LOGN1, N1 = PC::N1, N2 = PC::N2, N = PC::N, F = F1,
                             THREADS = kNC;
    };
    struct C2 {
        static constexpr int LOGN1 = PC::LOGN1, N1 = PC::N1, N2 = PC::N2, N = PC::N, F = F2,
                             THREADS = kNC;
    };
};

struct PArgs {
    const float4 *w;
    int64_t w_stride;
    int n, rows;             // samples; rows of w a column tile spans (ceil(n / N1))
    int64_t s0;
    int n_spin;
    const uint64_t *chirp;   // this band's spindown rates
    int64_t c_lo, c_hi;      // band-local cells of this launch
    int B, S, nb;            // cells per batch, scratch slots, batches
    float2 *scratch;
    const float *tw1, *tw2;  // forward twiddles of the pass-1 (N2) and pass-2 (N1) FFTs
    const float *lo, *hi;    // inter-pass twiddles
    const double *norm;
    uint32_t cell_base;
    int64_t bin_lo, bin_hi;
    float thr;
    CandRecord *out;
    unsigned long long *count;
    unsigned long long cap;
    uint32_t *head, *done1, *done2, *err;
    int64_t withhold;        // test hook: this item does not publish its completion (-1: none)
};

struct ItemInfo {
    int kind;   // 0 stop, 1 pass 1, 2 pass 2
    int batch;
    int tile;
    int item;
};

__device__ __forceinline__ void decode(int item, int T, int B, int nb, int &kind, int &batch,
                                       int &tile) {
    const int GB = T * B;
    const int g = item / GB;
    tile = item - g * GB;
    if (g == 0) { kind = 1; batch = 0; }
    else if (g & 1) {
        const int m = (g + 1) / 2;
        if (m < nb) { kind = 1; batch = m; }
        else { kind = 2; batch = nb - 1; }
    } else { kind = 2; batch = g / 2 - 1; }
}

// Bounded wait for a counter to reach target; false on timeout or a raised error.
__device__ __forceinline__ bool wait_count(const uint32_t *cnt, uint32_t target,
                                           const uint32_t *err) {
    if (ptx::ld_acquire(cnt) >= target) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        __nanosleep(128);
        if (ptx::ld_acquire(cnt) >= target) return true;
        if (*(volatile const uint32_t *)err) return false;
        if (ptx::globaltimer_ns() - t0 > kWaitNs) return false;
    }
}

// Bounded mbarrier wait.  err == nullptr: only the deadline ends the wait (a
// consumer waiting for bulk copies must not leave while they may be in flight).
__device__ __forceinline__ bool wait_mbar(uint64_t *bar, uint32_t parity, const uint32_t *err) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (err && *(volatile const uint32_t *)err) return false;
        if (ptx::globaltimer_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// Pass-1 input from the staged rows of w: stage[k2 * F + f] = w[k1_0 + f + N1 k2],
// times the spindown phase; zero beyond the data (the zero padding).
template <class C>
struct StageLoadP1 {
    const float4 *stg;
    int rows, n, k1_0;
    uint64_t afx;
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, float *ra, float *ia, float *rb,
                                         float *ib) const {
        float4 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k2 = j + r * JPF;
            const int k = k1_0 + f + C::N1 * k2;
            v[r] = (k2 < rows && k < n) ? stg[k2 * C::F + f] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t k = (uint32_t)(k1_0 + f + C::N1 * (j + r * JPF));
            const uint64_t kk = (uint64_t)k * (uint64_t)k;
            const int32_t top = (int32_t)((afx * kk) >> 32);
            const float ph = (float)top * 1.4629180792671596e-09f;   // 2 pi / 2^32
            float s, c;
            __sincosf(ph, &s, &c);
            ra[r] = v[r].x * c + v[r].y * s; ia[r] = v[r].y * c - v[r].x * s;
            rb[r] = v[r].z * c + v[r].w * s; ib[r] = v[r].w * c - v[r].z * s;
        }
    }
};

// Pass-2 input from the staged scratch rows: stage[(t F + f) N1 + k1].
template <class C>
struct StageLoadP2 {
    const float2 *stg;
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, float *ra, float *ia, float *rb,
                                         float *ib) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k1 = j + r * JPF;
            const float2 a = stg[f * C::N1 + k1], b = stg[(C::F + f) * C::N1 + k1];
            ra[r] = a.x; ia[r] = a.y; rb[r] = b.x; ib[r] = b.y;
        }
    }
};

template <int LOGN>
__global__ void __launch_bounds__(kThreads, 3) k_search_persistent(PArgs a) {
    using P = PC<LOGN>;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs = smem;
    float2 *tw1 = reinterpret_cast<float2 *>(smem + 2 * P::BUF);
    float2 *tw2 = tw1 + P::TW1;
    uint64_t *full = reinterpret_cast<uint64_t *>(tw2 + P::TW2);
    uint64_t *empty = full + 2;
    ItemInfo *info = reinterpret_cast<ItemInfo *>(empty + 2);

    eng::fill_twiddles<float, P::N2, kThreads, 1>(tw1, a.tw1);
    eng::fill_twiddles<float, P::N1, kThreads, 1>(tw2, a.tw2);
    if (threadIdx.x == 0) {
        ptx::mbar_init(&full[0], 1);
        ptx::mbar_init(&full[1], 1);
        ptx::mbar_init(&empty[0], 1);
        ptx::mbar_init(&empty[1], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();

    const int total = 2 * a.nb * P::T * a.B;
    const int tid = threadIdx.x;

    if (tid >= kNC) {
        // ------------------------------------------------------------ producer warp
        const int lane = tid - kNC;
        for (int it = 0;; ++it) {
            const int buf = it & 1;
            const uint32_t par = (uint32_t)((it >> 1) & 1);
            bool ok = true;
            if (lane == 0) ok = wait_mbar(&empty[buf], par ^ 1u, a.err);
            int item = 0;
            if (lane == 0 && ok) item = (int)atomicAdd(a.head, 1u);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (!ok || item >= total || *(volatile uint32_t *)a.err) {
                if (lane == 0) {
                    if (!ok) atomicOr(a.err, 1u);
                    if (ok) {     // the buffer is ours: hand the consumers a stop item
                        info[buf] = ItemInfo{0, 0, 0, -1};
                        ptx::mbar_arrive(&full[buf]);
                    }
                }
                break;
            }
            int kind, batch, tile;
            decode(item, P::T, a.B, a.nb, kind, batch, tile);
            if (lane == 0) {
                const uint32_t GB = (uint32_t)(P::T * a.B);
                if (kind == 2) ok = wait_count(a.done1 + batch, GB, a.err);
                else if (batch >= a.S) ok = wait_count(a.done2 + batch - a.S, GB, a.err);
                if (!ok) atomicOr(a.err, 1u);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    info[buf] = ItemInfo{0, 0, 0, -1};
                    ptx::mbar_arrive(&full[buf]);
                }
                break;
            }
            ptx::fence_proxy_async();
            const int cib = tile / P::T, tic = tile - cib * P::T;
            const int64_t cell = a.c_lo + (int64_t)batch * a.B + cib;
            const bool valid = cell < a.c_hi;
            uint32_t bytes = 0;
            if (valid) bytes = kind == 1 ? (uint32_t)(a.rows * P::F1 * 16) : (uint32_t)kStageBytes;
            unsigned char *dst = bufs + buf * P::BUF;
            if (lane == 0) {
                info[buf] = ItemInfo{kind, batch, tile, item};
                ptx::mbar_arrive_expect_tx(&full[buf], bytes);
            }
            __syncwarp();
            if (valid) {
                if (kind == 1) {
                    const int64_t sky = cell / a.n_spin;
                    const float4 *src = a.w + (sky - a.s0) * a.w_stride + tic * P::F1;
                    for (int k2 = lane; k2 < a.rows; k2 += 32)
                        ptx::bulk_g2s(dst + k2 * P::F1 * 16, src + (int64_t)P::N1 * k2, P::F1 * 16,
                                      &full[buf]);
                } else {
                    const float2 *slot = a.scratch + ((int64_t)(batch % a.S) * a.B + cib) * 2 * P::N;
                    for (int q = lane; q < 2 * P::F2; q += 32) {
                        const int t = q / P::F2, f = q - t * P::F2;
                        ptx::bulk_g2s(dst + (int64_t)q * P::N1 * 8,
                                      slot + (int64_t)t * P::N + (int64_t)(tic * P::F2 + f) * P::N1,
                                      P::N1 * 8, &full[buf]);
                    }
                }
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    for (int it = 0;; ++it) {
        const int buf = it & 1;
        const uint32_t par = (uint32_t)((it >> 1) & 1);
        if (!wait_mbar(&full[buf], par, nullptr)) {
            if (tid == 0) atomicOr(a.err, 1u);
            break;
        }
        const ItemInfo inf = info[buf];
        if (inf.kind == 0) break;
        const int cib = inf.tile / P::T, tic = inf.tile - cib * P::T;
        const int64_t cell = a.c_lo + (int64_t)inf.batch * a.B + cib;
        float2 *bp = reinterpret_cast<float2 *>(bufs + buf * P::BUF);
        if (cell < a.c_hi) {
            const int64_t sky = cell / a.n_spin;
            if (inf.kind == 1) {
                using C = typename P::C1;
                StageLoadP1<C> ld;
                ld.stg = reinterpret_cast<const float4 *>(bp);
                ld.rows = a.rows;
                ld.n = a.n;
                ld.k1_0 = tic * P::F1;
                ld.afx = a.chirp[cell - sky * a.n_spin];
                ScratchStore<float, C, -1> st;
                st.scratch = a.scratch;
                st.lo = a.lo;
                st.hi = a.hi;
                st.n_tr = 2;
                st.base = a.scratch + ((int64_t)(inf.batch % a.S) * a.B + cib) * 2 * P::N;
                st.has_b = true;
                st.k1_0 = tic * P::F1;
                eng::run_tile_inplace<float, P::N2, P::F1, kEH, -1, eng::kMapFJ, eng::NamedBarrier<kNC>>(
                    ld, st, bp, tw1);
            } else {
                using C = typename P::C2;
                StageLoadP2<C> ld;
                ld.stg = reinterpret_cast<const float2 *>(bp);
                SearchEpi<float, C> st;
                st.na = (float)a.norm[kNormStride * (sky - a.s0)];
                st.nb = (float)a.norm[kNormStride * (sky - a.s0) + 1];
                st.nab = (float)a.norm[kNormStride * (sky - a.s0) + 2];
                st.cell = a.cell_base + (uint32_t)cell;
                st.l2_0 = tic * P::F2;
                st.bin_lo = a.bin_lo;
                st.bin_hi = a.bin_hi;
                st.thr = a.thr;
                st.out = a.out;
                st.count = a.count;
                st.cap = a.cap;
                eng::run_tile_inplace<float, P::N1, P::F2, kEH, -1, eng::kMapJ, eng::NamedBarrier<kNC>>(
                    ld, st, bp, tw2);
            }
        }
        eng::NamedBarrier<kNC>::sync();   // the buffer is read, every store issued
        if (tid == 0) {
            if ((int64_t)inf.item != a.withhold) {
                __threadfence();
                ptx::red_release_add((inf.kind == 1 ? a.done1 : a.done2) + inf.batch, 1u);
            }
            ptx::mbar_arrive(&empty[buf]);
        }
    }
}

template <int LOGN>
int launch_t(const Plan &p, int band_idx, const BandDev &b, int64_t s0, int64_t c_lo,
             int64_t c_hi, cudaStream_t s, const CellBufs &cb) {
    using P = PC<LOGN>;
    static int grid = 0;
    auto k = k_search_persistent<LOGN>;
    if (grid == 0) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
        int per_sm = 0, dev = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, P::SMEM);
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = std::max(1, per_sm) * std::max(1, sms);
    }
    const TwiddleSet *tw = p.twiddles(LOGN);
    PArgs a;
    a.w = reinterpret_cast<const float4 *>(cb.w);
    a.w_stride = p.w_stride;
    a.n = (int)b.n;
    a.rows = (int)((b.n + P::N1 - 1) / P::N1);
    a.s0 = s0;
    a.n_spin = (int)p.desc.n_spin;
    a.chirp = p.chirp_fx + (int64_t)band_idx * p.desc.n_spin;
    a.c_lo = c_lo;
    a.c_hi = c_hi;
    a.B = (int)p.pbatch;
    a.S = (int)p.pslots;
    a.nb = (int)((c_hi - c_lo + a.B - 1) / a.B);
    a.scratch = reinterpret_cast<float2 *>(cb.scratch);
    a.tw1 = tw->in2_f;
    a.tw2 = tw->in1_f;
    a.lo = tw->lo_f;
    a.hi = tw->hi_f;
    a.norm = cb.norm;
    a.cell_base = (uint32_t)((int64_t)band_idx * p.desc.n_sky * p.desc.n_spin);
    a.bin_lo = b.lo;
    a.bin_hi = b.hi;
    a.thr = (float)p.desc.thr_2F;
    a.out = p.cand;
    a.count = p.cand_count;
    a.cap = (unsigned long long)p.cand_capacity;
    a.head = p.queue;
    a.done1 = p.queue + 1;
    a.done2 = p.queue + 1 + a.nb;
    a.err = p.qerr;
    a.withhold = p.withhold_item;
    cudaMemsetAsync(p.queue, 0, sizeof(uint32_t) * (1 + 2 * (size_t)a.nb), s);
    k<<<grid, kThreads, P::SMEM, s>>>(a);
    return 1;
}

}  // namespace

bool persistent_supported(int logn) { return logn >= 12 && logn <= 20; }

int persistent_tiles_per_cell(int logn) { return (1 << logn) / kETile; }

int launch_search_persistent(const Plan &p, int band_idx, const BandDev &b, int64_t s0,
                             int64_t c_lo, int64_t c_hi, cudaStream_t s, const CellBufs &cb) {
    switch (b.logn) {
        case 12: return launch_t<12>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 13: return launch_t<13>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 14: return launch_t<14>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 15: return launch_t<15>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 16: return launch_t<16>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 17: return launch_t<17>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 18: return launch_t<18>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 19: return launch_t<19>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        case 20: return launch_t<20>(p, band_idx, b, s0, c_lo, c_hi, s, cb);
        default: return -1;
    }
}

}  // namespace fstat
