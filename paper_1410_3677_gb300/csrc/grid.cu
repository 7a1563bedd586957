// The search grid from the generating matrix M (Sect. 2: the rows of M span the
// 4-D parameter space and their integer multiples are the grid points; a sky
// position is a pair of integers (n, m), a spindown an integer s).  Coordinates
// of the space, row by row of M: frequency f dt, spindown fdot dt^2 / 2, and the
// ecliptic-plane components (beta1, beta2) of the unit vector towards the source
// in units of the orbital Roemer phase at the reference frequency, f_ref tau_E
// beta (tau_E = 1 AU / c).  Sky point (n, m) = n M[2] + m M[3]; it lies on the
// sphere when beta1^2 + beta2^2 <= 1, and the hemisphere sets the sign of the
// ecliptic latitude.  The grid is a product (each sky position takes every
// spindown) when the spindown row has no sky components and the sky rows no
// spindown component; the frequency components are the FFT's own grid.
//
// The decision whether a point lies on the sphere is taken in FP64 with every
// product and sum rounded explicitly in a fixed order, so it is reproducible;
// the angles then come from atan2 and asin.
#include <math.h>

#include <algorithm>

#include "fstat_internal.h"

namespace fstat {
namespace {

constexpr double kTauE = 499.00478383615643;   // 1 AU / c, s
constexpr double kTwoPiD = 6.283185307179586476925286766559;

struct LatticeDev {
    double m22, m23, m32, m33;   // the sky block of M
    double scale;                // f_ref tau_E
    double ce, se;               // cos eps, sin eps (host libm)
    int64_t n_lo, m_lo, nn, nm;  // ranges: nn values of n, nm of m
    int64_t per_hemi;            // nn * nm
    int64_t total;               // per_hemi * hemispheres
};

// Ecliptic components of point i (hemisphere, n, m in that order of nesting) and
// whether it lies on the sphere.
__device__ __forceinline__ bool lattice_point(const LatticeDev &L, int64_t i, int &hs, int64_t &n,
                                              int64_t &m, double &b1, double &b2) {
    hs = (int)(i / L.per_hemi);
    const int64_t r = i - (int64_t)hs * L.per_hemi;
    n = L.n_lo + r / L.nm;
    m = L.m_lo + r % L.nm;
    const double dn = (double)n, dm = (double)m;
    const double w2 = __dadd_rn(__dmul_rn(dn, L.m22), __dmul_rn(dm, L.m32));
    const double w3 = __dadd_rn(__dmul_rn(dn, L.m23), __dmul_rn(dm, L.m33));
    b1 = w2 / L.scale;   // IEEE division
    b2 = w3 / L.scale;
    const double r2 = __dadd_rn(__dmul_rn(b1, b1), __dmul_rn(b2, b2));
    return hs == 0 ? (r2 <= 1.0) : (r2 < 1.0);   // the ecliptic belongs to the north
}

__global__ void k_lattice_count(LatticeDev L, int64_t *counts) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool on = false;
    if (i < L.total) {
        int hs;
        int64_t n, m;
        double b1, b2;
        on = lattice_point(L, i, hs, n, m, b1, b2);
    }
    const int c = __syncthreads_count(on);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of the per-block counts in place (one CTA, chunks of its size);
// counts[nb] receives the total.
__global__ void k_lattice_scan(int64_t *counts, int64_t nb) {
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? counts[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (unsigned o = 1; o < blockDim.x; o <<= 1) {   // inclusive Hillis-Steele scan
            const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) counts[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[nb] = carry;
}

__global__ void k_lattice_write(LatticeDev L, const int64_t *offsets, int64_t cap, double *alpha,
                                double *delta, int64_t *nm_out) {
    __shared__ int warp_base[32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int hs = 0;
    int64_t n = 0, m = 0;
    double b1 = 0.0, b2 = 0.0;
    const bool on = i < L.total && lattice_point(L, i, hs, n, m, b1, b2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) warp_base[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive scan over the block's warps
        int acc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int c = warp_base[w];
            warp_base[w] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (!on) return;
    const int64_t k = offsets[blockIdx.x] + warp_base[wid] + __popc(bal & ((1u << lane) - 1u));
    if (k >= cap) return;
    // unit vector: ecliptic (b1, b2, h sqrt(1 - b1^2 - b2^2)) rotated to equatorial
    double q = __dsub_rn(__dsub_rn(1.0, __dmul_rn(b1, b1)), __dmul_rn(b2, b2));
    if (q < 0.0) q = 0.0;
    const double ze = hs == 0 ? sqrt(q) : -sqrt(q);
    const double y = __dsub_rn(__dmul_rn(b2, L.ce), __dmul_rn(ze, L.se));
    const double z = __dadd_rn(__dmul_rn(b2, L.se), __dmul_rn(ze, L.ce));
    double a = atan2(y, b1);
    if (a < 0.0) a += kTwoPiD;
    alpha[k] = a;
    delta[k] = asin(z > 1.0 ? 1.0 : (z < -1.0 ? -1.0 : z));
    if (nm_out) {
        nm_out[3 * k] = hs;
        nm_out[3 * k + 1] = n;
        nm_out[3 * k + 2] = m;
    }
}

__global__ void k_lattice_spin(double m11, double dt2, int64_t s_lo, int64_t ns, int64_t cap,
                               double *fdot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns || i >= cap) return;
    const double w1 = __dmul_rn((double)(s_lo + i), m11);
    fdot[i] = __dmul_rn(2.0, w1) / dt2;
}

}  // namespace
}  // namespace fstat

extern "C" fstat_status fstat_lattice_grid(const fstat_lattice *Lh, double *alpha, double *delta,
                                           int64_t *nm, int64_t cap_sky, int64_t *n_sky, double *fdot,
                                           int64_t cap_spin, int64_t *n_spin, void *cuda_stream) {
    using namespace fstat;
    if (!Lh || !n_sky || !n_spin || cap_sky < 0 || cap_spin < 0) return FSTAT_ERR_ARG;
    const fstat_lattice &L = *Lh;
    const double *M = L.M;
    for (int i = 0; i < 16; ++i)
        if (!isfinite(M[i])) return FSTAT_ERR_ARG;
    if (!(L.dt > 0) || !isfinite(L.dt) || !(L.f_ref > 0) || !isfinite(L.f_ref) || !isfinite(L.eps) ||
        L.s_hi < L.s_lo || L.n_hi < L.n_lo || L.m_hi < L.m_lo || (L.hemispheres != 1 && L.hemispheres != 2))
        return FSTAT_ERR_ARG;
    // a product grid: no spindown component in the sky rows, no sky component in
    // the spindown row
    if (M[4 + 2] != 0.0 || M[4 + 3] != 0.0 || M[8 + 1] != 0.0 || M[12 + 1] != 0.0) return FSTAT_ERR_ARG;
    const int64_t nn = L.n_hi - L.n_lo + 1, nmr = L.m_hi - L.m_lo + 1, ns = L.s_hi - L.s_lo + 1;
    if (nn > (int64_t(1) << 20) || nmr > (int64_t(1) << 20) || ns > (int64_t(1) << 31) ||
        nn * nmr * L.hemispheres > (int64_t(1) << 31))
        return FSTAT_ERR_ARG;
    if ((cap_sky > 0 && (!alpha || !delta)) || (cap_spin > 0 && !fdot)) return FSTAT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    LatticeDev d;
    d.m22 = M[8 + 2];
    d.m23 = M[8 + 3];
    d.m32 = M[12 + 2];
    d.m33 = M[12 + 3];
    d.scale = L.f_ref * kTauE;
    d.ce = cos(L.eps);
    d.se = sin(L.eps);
    d.n_lo = L.n_lo;
    d.m_lo = L.m_lo;
    d.nn = nn;
    d.nm = nmr;
    d.per_hemi = nn * nmr;
    d.total = d.per_hemi * L.hemispheres;
    constexpr int kThreads = 256;
    const int64_t nb = (d.total + kThreads - 1) / kThreads;
    int64_t *offs = nullptr;
    if (cudaMalloc(&offs, (size_t)(nb + 1) * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return FSTAT_ERR_OOM;
    }
    fstat_status st = FSTAT_OK;
    int64_t total = 0;
    k_lattice_count<<<(unsigned)nb, kThreads, 0, s>>>(d, offs);
    k_lattice_scan<<<1, 1024, 0, s>>>(offs, nb);
    if (cap_sky > 0) k_lattice_write<<<(unsigned)nb, kThreads, 0, s>>>(d, offs, cap_sky, alpha, delta, nm);
    if (cap_spin > 0)
        k_lattice_spin<<<(unsigned)((std::min(ns, cap_spin) + 255) / 256), 256, 0, s>>>(
            M[4 + 1], L.dt * L.dt, L.s_lo, ns, cap_spin, fdot);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&total, offs + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        st = FSTAT_ERR_CUDA;
    cudaFree(offs);
    if (st != FSTAT_OK) return st;
    *n_sky = total;
    *n_spin = ns;
    if ((cap_sky > 0 && total > cap_sky) || (cap_spin > 0 && ns > cap_spin)) return FSTAT_ERR_OVERFLOW;
    return FSTAT_OK;
}
