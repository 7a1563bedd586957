// Candidate records put in (cell, bin) order on the device before they are read
// back: a stable least-significant-digit radix sort, 8-bit digits, over the key
// (cell - cell0) << bin_bits | bin of the searched range.  One pass is a digit
// histogram per tile of 4096 records, an exclusive scan of the histograms in
// digit-major order (the tile's first slot for each digit), and a scatter that
// ranks each record among the equal digits before it in its tile (warp match,
// per-warp counts in shared memory), so records with equal digits keep their
// order and the passes compose.  The scan runs per digit row (one CTA each) and
// the scatter adds the totals of the smaller digits.  The candidate set of
// Sect. 2 has no order of its own; the plan returns it sorted by (band, sky,
// spin, bin).
#include "fstat_internal.h"

namespace fstat {

namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 16;
constexpr int kTile = kThreads * kRounds;

__device__ __forceinline__ uint32_t digit_of(const CandRecord &r, uint32_t cell0, int bin_bits, int shift) {
    const uint64_t key = ((uint64_t)(r.cell - cell0) << bin_bits) | r.bin;
    return (uint32_t)(key >> shift) & 255u;
}

__global__ void __launch_bounds__(kThreads) k_digit_hist(const CandRecord *__restrict__ in, int64_t n,
                                                         uint32_t cell0, int bin_bits, int shift,
                                                         uint32_t *__restrict__ hist, int64_t nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kRounds; ++i) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[digit_of(in[idx], cell0, bin_bits, shift)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of each digit's row of tile counts in place, one CTA of 1024
// threads per digit (coalesced chunks of 1024 counts, warp-shuffle scans); the
// row total goes to tot[digit].
__global__ void __launch_bounds__(1024) k_scan_rows(uint32_t *__restrict__ h, int64_t nblk,
                                                    uint32_t *__restrict__ tot) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    uint32_t *row = h + (int64_t)blockIdx.x * nblk;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nblk; c0 += 1024) {
        const int64_t i = c0 + t;
        const uint32_t v = i < nblk ? row[i] : 0u;
        uint32_t x = v;   // inclusive scan within the warp
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (l >= d) x += y;
        }
        if (l == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t z = wsum[l];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, d);
                if (l >= d) z += y;
            }
            wsum[l] = z;   // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = carry + (w > 0 ? wsum[w - 1] : 0u) + x - v;
        if (i < nblk) row[i] = before;
        __syncthreads();
        if (t == 0) carry += wsum[31];
        __syncthreads();
    }
    if (t == 0) tot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads) k_digit_scatter(const CandRecord *__restrict__ in,
                                                            CandRecord *__restrict__ out, int64_t n,
                                                            uint32_t cell0, int bin_bits, int shift,
                                                            const uint32_t *__restrict__ off, int64_t nblk,
                                                            const uint32_t *__restrict__ tot) {
    __shared__ uint32_t run[256];             // slots of each digit used by earlier rounds
    __shared__ uint32_t wc[kThreads / 32][256];   // this round's count of each digit per warp
    __shared__ uint32_t wt[kThreads / 32];
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const unsigned below = (1u << l) - 1u;
    // first slot of digit t: the records of all smaller digits (an exclusive scan
    // of the 256 row totals) plus this tile's offset within the row of digit t
    const uint32_t v = tot[t];
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (l >= d) x += y;
    }
    if (l == 31) wt[w] = x;
    __syncthreads();
    uint32_t smaller = x - v;
    for (int q = 0; q < w; ++q) smaller += wt[q];
    run[t] = smaller + off[(int64_t)t * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int i = 0; i < kRounds; ++i) {
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) wc[q][t] = 0;
        __syncthreads();
        const int64_t idx = base + i * kThreads + t;
        const bool ok = idx < n;
        CandRecord r{};
        uint32_t d = 256;   // past the end: a digit no record has
        if (ok) {
            r = in[idx];
            d = digit_of(r, cell0, bin_bits, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & below);
        if (ok && rank == 0) wc[w][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = run[d] + (uint32_t)rank;
            for (int q = 0; q < w; ++q) pos += wc[q][d];
            out[pos] = r;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) add += wc[q][t];
        run[t] += add;
    }
}

}  // namespace

int sort_bits(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

// Sorts n records of `a` (using b as the other buffer of the ping-pong and hist
// for 256 ceil(n / 4096) counts plus 256 totals); returns the buffer that holds
// the result.
// cell0 and the cell span are those of the searched range, bins < 2^bin_bits.
CandRecord *launch_cand_sort(CandRecord *a, CandRecord *b, uint32_t *hist, int64_t n, uint32_t cell0,
                             uint64_t cell_span, int bin_bits, cudaStream_t s, int64_t *launches) {
    const int key_bits = sort_bits(cell_span > 0 ? cell_span - 1 : 0) + bin_bits;
    const int passes = (key_bits + 7) / 8;
    const int64_t nblk = (n + kTile - 1) / kTile;
    CandRecord *src = a, *dst = b;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_digit_hist<<<(unsigned)nblk, kThreads, 0, s>>>(src, n, cell0, bin_bits, shift, hist, nblk);
        k_scan_rows<<<256, 1024, 0, s>>>(hist, nblk, hist + 256 * nblk);
        k_digit_scatter<<<(unsigned)nblk, kThreads, 0, s>>>(src, dst, n, cell0, bin_bits, shift, hist, nblk,
                                                             hist + 256 * nblk);
        *launches += 3;
        CandRecord *x = src;
        src = dst;
        dst = x;
    }
    return src;
}

}  // namespace fstat
