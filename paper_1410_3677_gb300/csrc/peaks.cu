// Roofline denominators measured on the device the library runs on (not part
// of the method): the FP32 FMA rate of independent FFMA chains in every lane,
// and the bandwidth of a copy whose source and destination stay in L2.  The
// roofline of the search path is the slower of its FFT FLOP at the first and
// its inter-pass scratch bytes at the second (or at the HBM copy rate when the
// scratch reaches DRAM).
#include <cuda_runtime.h>

#include "fstat_internal.h"

namespace fstat {

namespace {

constexpr int kChains = 16;

// kChains independent a = a b + c chains per thread; the result is stored only
// under a condition the values never meet, so nothing is dropped.
__global__ void __launch_bounds__(256) k_fma_chains(float *out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1e-3f * (float)threadIdx.x + (float)i;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.25f) out[blockIdx.x] = s;
}

// reps copies of n4 float4 through L2 only (ld.global.cg / st.global.cg), so a
// working set that fits in L2 is served from it and not from L1.
__global__ void __launch_bounds__(256) k_l2_copy(const float4 *src, float4 *dst, int64_t n4, int reps) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride)
            __stcg(dst + i, __ldcg(src + i));
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Milliseconds of the work `run` queues on s, after one untimed run.
template <class F>
bool time_ms(cudaStream_t s, F run, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return false;
    }
    run();
    cudaEventRecord(e0, s);
    run();
    cudaEventRecord(e1, s);
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
                    cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok;
}

}  // namespace

}  // namespace fstat

extern "C" fstat_status fstat_measure_fp32_fma(double *tflops, void *cuda_stream) {
    using namespace fstat;
    if (!tflops) return FSTAT_ERR_ARG;
    *tflops = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float *out = nullptr;
    if (cudaMalloc(&out, 65536 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return FSTAT_ERR_OOM;
    }
    const int blocks = sm_count() * 8;   // 2048 threads per SM
    const int iters = 20000;
    float ms = 0.f;
    const bool ok = time_ms(s, [&] { k_fma_chains<<<blocks, 256, 0, s>>>(out, iters, 0.9999f, 1e-4f); }, &ms);
    cudaFree(out);
    if (!ok || ms <= 0.f) return FSTAT_ERR_CUDA;
    const double fmas = (double)blocks * 256 * iters * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return FSTAT_OK;
}

extern "C" fstat_status fstat_measure_l2_copy(int64_t bytes, double *gbs, void *cuda_stream) {
    using namespace fstat;
    if (!gbs || bytes < (int64_t)(1 << 20)) return FSTAT_ERR_ARG;
    *gbs = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t n4 = bytes / 2 / (int64_t)sizeof(float4);   // source and destination halves
    float4 *buf = nullptr;
    if (cudaMalloc(&buf, 2 * n4 * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return FSTAT_ERR_OOM;
    }
    cudaMemsetAsync(buf, 0, 2 * n4 * sizeof(float4), s);
    const int blocks = sm_count() * 8;
    const int reps = 256;
    float ms = 0.f;
    const bool ok = time_ms(s, [&] { k_l2_copy<<<blocks, 256, 0, s>>>(buf, buf + n4, n4, reps); }, &ms);
    cudaFree(buf);
    if (!ok || ms <= 0.f) return FSTAT_ERR_CUDA;
    *gbs = 2.0 * (double)n4 * sizeof(float4) * reps / (ms * 1e-3) / 1e9;
    return FSTAT_OK;
}
