// fstat_cell_F_noalloc: the F-statistic of every bin of one cell from an
// already resampled and demodulated series, with no device allocation.  The two
// FFT passes use the same kernels as the FP32 search; the intermediate between
// them lives in a file-scope device array instead of plan-owned memory.
#include <mutex>

#include "passes.cuh"

namespace fstat {

namespace {

constexpr int kNoallocMaxLogN = 18;
constexpr int64_t kNoallocScratch = int64_t(2) << kNoallocMaxLogN;   // float2: two transforms

// Twiddle tables per transform length 2^L, L = 12 .. 18: W_N1^k (N1 entries),
// W_N2^k (N2), W_N^k (k < N1), W_N^{k N1} (k < N2), interleaved complex; the
// region of length L starts at tw_off(L).
constexpr int tw_len(int L) { return 2 * 2 * ((1 << (L / 2)) + (1 << (L - L / 2))); }
constexpr int tw_off(int L) { return L <= 12 ? 0 : tw_off(L - 1) + tw_len(L - 1); }
constexpr int kNoallocTw = tw_off(kNoallocMaxLogN + 1);

// Shared by every call in the process (on each device that loads the library).
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratch];
static __device__ __align__(256) float g_noalloc_tw[kNoallocTw];

// Device addresses of the two arrays, resolved once per device with that device
// current (in host code the symbol names are only host-side stand-ins), and which
// twiddle lengths have been filled on that device.
constexpr int kMaxDevices = 64;
struct DevState {
    float2 *scratch = nullptr;
    float *tw = nullptr;
    bool tw_ready[kNoallocMaxLogN + 1] = {};
};
DevState g_dev[kMaxDevices];
std::mutex g_dev_mu;

__global__ void k_noalloc_twiddles(float *tw, int L) {
    const int n1 = 1 << (L / 2), n2 = 1 << (L - L / 2);
    const int64_t N = int64_t(1) << L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // e^{-2 pi i k / M} = (cospi(2k/M), -sinpi(2k/M)), evaluated in FP64
    auto put = [&](int slot, int64_t k, int64_t M) {
        double s, c;
        sincospi(2.0 * (double)k / (double)M, &s, &c);
        tw[2 * slot] = (float)c;
        tw[2 * slot + 1] = (float)-s;
    };
    if (i < n1) put(i, i, n1);
    else if (i < n1 + n2) put(i, i - n1, n2);
    else if (i < 2 * n1 + n2) put(i, i - n1 - n2, N);
    else if (i < 2 * n1 + 2 * n2) put(i, (int64_t)(i - 2 * n1 - n2) * n1, N);
}

// Resolves the arrays' addresses and fills the twiddles of length 2^L on first
// use on the current device.  Returns false on a CUDA error.
bool setup_current_device(int L, DevState **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevState &d = g_dev[dev];
    if (!d.scratch) {
        void *a = nullptr, *b = nullptr;
        if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess) return false;
        if (cudaGetSymbolAddress(&b, g_noalloc_tw) != cudaSuccess) return false;
        d.scratch = static_cast<float2 *>(a);
        d.tw = static_cast<float *>(b);
    }
    if (!d.tw_ready[L]) {
        const int n = tw_len(L) / 2;
        k_noalloc_twiddles<<<(n + 255) / 256, 256>>>(d.tw + tw_off(L), L);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return false;
        d.tw_ready[L] = true;
    }
    *out = &d;
    return true;
}

// Pass-1 input: w[k] = (y a, y b) of one sky, times the spindown phase.
template <class C>
struct CellLoad {
    const float4 *w;
    int n;
    uint64_t afx;
    int k1_0;
    __device__ void init() { k1_0 = blockIdx.x * C::F; }
    template <int R, int JPF>
    __device__ __forceinline__ void load(int f, int j, float *ra, float *ia, float *rb,
                                         float *ib) const {
        float4 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = k1_0 + f + C::N1 * (j + r * JPF);
            v[r] = k < n ? __ldg(w + k) : make_float4(0.f, 0.f, 0.f, 0.f);
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

// Pass-2 output: F of every bin in [lo, hi] into out[bin - lo].
template <class C>
struct CellFOut {
    float *out;
    float na, nb;
    int64_t lo, hi;
    int l2_0;
    __device__ void init() { l2_0 = blockIdx.x * C::F; }
    template <int R, int JPF>
    __device__ __forceinline__ void store(int f, int j, float *ra, float *ia, float *rb,
                                          float *ib) const {
        const int l2 = l2_0 + f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t bin = (int64_t)C::N2 * (j + r * JPF) + l2;
            if (bin >= lo && bin <= hi)
                out[bin - lo] = (ra[r] * ra[r] + ia[r] * ia[r]) * na + (rb[r] * rb[r] + ib[r] * ib[r]) * nb;
        }
    }
};

template <int LOGN>
fstat_status run_cell(const float4 *w, int n, uint64_t afx, float na, float nb, int64_t lo,
                      int64_t hi, float *out, float2 *scratch, const float *tw_in1,
                      const float *tw_in2, const float *tw_lo, const float *tw_hi,
                      cudaStream_t s) {
    using C1 = Cfg<float, LOGN, 1>;
    using C2 = Cfg<float, LOGN, 2>;
    CellLoad<C1> ld1{w, n, afx, 0};
    ScratchStore<float, C1, -1> st1{};
    st1.scratch = scratch;
    st1.lo = tw_lo;
    st1.hi = tw_hi;
    st1.n_tr = 2;
    auto k1 = k_pass<float, LOGN, 1, -1, eng::kMapFJ, CellLoad<C1>, ScratchStore<float, C1, -1>>;
    auto k2 = k_pass<float, LOGN, 2, -1, eng::kMapW, ScratchLoad<float, C2>, CellFOut<C2>>;
    if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C1::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C2::SMEM) != cudaSuccess)
        return FSTAT_ERR_CUDA;
    k1<<<dim3(C1::TILES, 1), C1::THREADS, C1::SMEM, s>>>(ld1, st1, tw_in2);
    ScratchLoad<float, C2> ld2{};
    ld2.scratch = scratch;
    CellFOut<C2> st2{out, na, nb, lo, hi, 0};
    k2<<<dim3(C2::TILES, 1), C2::THREADS, C2::SMEM, s>>>(ld2, st2, tw_in1);
    return cudaGetLastError() == cudaSuccess ? FSTAT_OK : FSTAT_ERR_CUDA;
}

}  // namespace

}  // namespace fstat

extern "C" fstat_status fstat_cell_F_noalloc(const float *w, int64_t n, int64_t n_fft,
                                             double chirp_rate, double norm_a, double norm_b,
                                             int64_t bin_lo, int64_t bin_hi, float *F_out,
                                             void *cuda_stream) {
    using namespace fstat;
    int lg = 0;
    while ((int64_t(1) << lg) < n_fft) ++lg;
    // w is read as float4 (16-byte loads) and F_out written as floats: a view that
    // starts off those boundaries is refused here instead of faulting on the GPU
    if (!w || !F_out || (reinterpret_cast<uintptr_t>(w) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(F_out) & 3) != 0 || n < 1 || (int64_t(1) << lg) != n_fft || lg < 12 ||
        lg > kNoallocMaxLogN || 2 * n > n_fft || bin_lo < 0 || bin_hi < bin_lo || bin_hi >= n_fft ||
        !(norm_a >= 0.0) || !(norm_b >= 0.0))
        return FSTAT_ERR_ARG;
    DevState *d = nullptr;
    if (!setup_current_device(lg, &d)) return FSTAT_ERR_CUDA;
    float2 *scratch = d->scratch;
    const int64_t n1 = int64_t(1) << log_n1(lg), n2 = int64_t(1) << log_n2(lg);
    const float *tw_in1 = d->tw + tw_off(lg), *tw_in2 = tw_in1 + 2 * n1, *tw_lo = tw_in2 + 2 * n2,
                *tw_hi = tw_lo + 2 * n1;
    // frac(rate) in 2^-64 cycles (the rate is |fdot| dt^2 / 2 << 1/4)
    if (!(fabs(chirp_rate) < 0.25)) return FSTAT_ERR_ARG;
    const uint64_t afx = (uint64_t)(int64_t)llround(ldexp(chirp_rate, 64));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const float4 *w4 = reinterpret_cast<const float4 *>(w);
    fstat_status st = FSTAT_ERR_ARG;
#define FSTAT_NOALLOC_CASE(L)                                                                   \
    case L:                                                                                     \
        st = run_cell<L>(w4, (int)n, afx, (float)norm_a, (float)norm_b, bin_lo, bin_hi, F_out, \
                         scratch, tw_in1, tw_in2, tw_lo, tw_hi, s);                             \
        break;
    switch (lg) {
        FSTAT_NOALLOC_CASE(12)
        FSTAT_NOALLOC_CASE(13)
        FSTAT_NOALLOC_CASE(14)
        FSTAT_NOALLOC_CASE(15)
        FSTAT_NOALLOC_CASE(16)
        FSTAT_NOALLOC_CASE(17)
        FSTAT_NOALLOC_CASE(18)
        default: return FSTAT_ERR_ARG;
    }
#undef FSTAT_NOALLOC_CASE
    if (st != FSTAT_OK) return st;
    return cudaStreamSynchronize(s) == cudaSuccess ? FSTAT_OK : FSTAT_ERR_CUDA;
}
