// fld_anderson.cu -- Anderson mixing of blocks of sweeps (not in the paper).
//
// One block of red-black sweeps (Algorithm 1) is a fixed-point map
// G: phi -> phi' whose fixed point is the solution of Eq. 31.  Anderson
// mixing keeps the last m images g_i = G(x_i) and residuals f_i = g_i - x_i
// and starts the next block from x = sum_i a_i g_i, with the weights a
// (summing to 1) that minimise |sum_i a_i f_i|.  The weights come from the
// Gram matrix <f_i, f_j>, reduced here in FP64 and solved on the host.
//
// Per element of a padded field (both colours, ghosts and row padding
// included -- there f is 0 and every g_i is the same value):
//   k_and_collect: g = phi (hi + lo, or FP64), f = g - x_cur, stores g in its
//                  slot (FP64) and f (FP32), and accumulates <f, f_j> for
//                  every occupied slot j;
//   k_and_reduce:  sums the per-CTA partials in a fixed order;
//   k_and_mix:     x = g_s + sum_{j != s} a_j (g_j - g_s), written back as
//                  phi (hi/lo, float, or FP64) and as the next x_cur.
// The difference form leaves ghosts and padding exactly unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fld_internal.h"

namespace fld {
namespace {

constexpr int kAndThreads = 256;

struct SlotPtrs {
    const double *g[kAndersonMax];
    const float *f[kAndersonMax];
};

struct Coef {
    double a[kAndersonMax];
};

__device__ __forceinline__ double state_at(const float *hi, const float *lo, const double *p64, long long e) {
    if (p64) return p64[e];
    return lo ? (double)hi[e] + (double)lo[e] : (double)hi[e];
}

__global__ void __launch_bounds__(kAndThreads) k_and_capture(int n, const float *__restrict__ hi,
                                                              const float *__restrict__ lo,
                                                              const double *__restrict__ p64,
                                                              double *__restrict__ x_cur) {
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        x_cur[e] = state_at(hi, lo, p64, e);
}

__global__ void __launch_bounds__(kAndThreads) k_and_collect(int n, const float *__restrict__ hi,
                                                              const float *__restrict__ lo,
                                                              const double *__restrict__ p64,
                                                              const double *__restrict__ x_cur, SlotPtrs sl,
                                                              double *__restrict__ g_out, float *__restrict__ f_out,
                                                              int w, int s, double *__restrict__ part) {
    double acc[kAndersonMax];
#pragma unroll
    for (int j = 0; j < kAndersonMax; ++j) acc[j] = 0.0;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double g = state_at(hi, lo, p64, e);
        const float f = (float)(g - x_cur[e]);
        g_out[e] = g;
        f_out[e] = f;
        const double fd = (double)f;
#pragma unroll
        for (int j = 0; j < kAndersonMax; ++j) {
            if (j < w) acc[j] += fd * (double)(j == s ? f : sl.f[j][e]);
        }
    }
    // block reduction of every accumulator: warp shuffles, then one value
    // per warp in shared memory, summed by the first warp in warp order
    __shared__ double red[kAndThreads / 32][kAndersonMax];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kAndersonMax; ++j) {
        double v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < kAndersonMax) {
        double v = 0.0;
        for (int q = 0; q < kAndThreads / 32; ++q) v += red[q][threadIdx.x];
        part[(size_t)blockIdx.x * kAndersonMax + threadIdx.x] = v;
    }
}

__global__ void k_and_reduce(const double *__restrict__ part, int nblocks, double *__restrict__ out) {
    const int j = threadIdx.x;
    if (j >= kAndersonMax) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += part[(size_t)b * kAndersonMax + j];
    out[j] = v;
}

__global__ void __launch_bounds__(kAndThreads) k_and_mix(int n, SlotPtrs sl, int w, int s, Coef c,
                                                          float *__restrict__ hi, float *__restrict__ lo,
                                                          double *__restrict__ p64, double *__restrict__ x_cur) {
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double gs = sl.g[s][e];
        double x = gs;
#pragma unroll
        for (int j = 0; j < kAndersonMax; ++j) {
            if (j < w && j != s) x += c.a[j] * (sl.g[j][e] - gs);
        }
        if (p64) {
            p64[e] = x;
            x_cur[e] = x;
        } else {
            const float h = (float)x;
            if (lo) {
                const float l = (float)(x - (double)h);
                hi[e] = h;
                lo[e] = l;
                x_cur[e] = (double)h + (double)l;
            } else {
                hi[e] = h;
                x_cur[e] = (double)h;
            }
        }
    }
}

int and_grid(int n, int nsm) {
    const int want = (n + kAndThreads - 1) / kAndThreads;
    const int cap = 4 * nsm;
    return want < cap ? (want > 0 ? want : 1) : cap;
}

SlotPtrs slot_ptrs(const AndersonBuffers &b, int n, int w) {
    SlotPtrs sl;
    for (int j = 0; j < kAndersonMax; ++j) {
        sl.g[j] = j < w ? b.g + (size_t)j * n : nullptr;
        sl.f[j] = j < w ? b.f + (size_t)j * n : nullptr;
    }
    return sl;
}

}  // namespace

cudaError_t launch_anderson_capture(const AndersonBuffers &b, int n, const float *hi, const float *lo,
                                    const double *p64, int nsm, cudaStream_t s) {
    k_and_capture<<<and_grid(n, nsm), kAndThreads, 0, s>>>(n, hi, lo, p64, b.x);
    return cudaGetLastError();
}

cudaError_t launch_anderson_collect(const AndersonBuffers &b, int n, const float *hi, const float *lo,
                                    const double *p64, int slot, int w, int nsm, cudaStream_t s) {
    const int nb = and_grid(n, nsm);
    const SlotPtrs sl = slot_ptrs(b, n, w);
    k_and_collect<<<nb, kAndThreads, 0, s>>>(n, hi, lo, p64, b.x, sl, b.g + (size_t)slot * n,
                                             b.f + (size_t)slot * n, w, slot, b.part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_and_reduce<<<1, 32, 0, s>>>(b.part, nb, b.dots);
    return cudaGetLastError();
}

cudaError_t launch_anderson_mix(const AndersonBuffers &b, int n, int slot, int w, const double *a, float *hi,
                                float *lo, double *p64, int nsm, cudaStream_t s) {
    Coef c;
    for (int j = 0; j < kAndersonMax; ++j) c.a[j] = j < w ? a[j] : 0.0;
    k_and_mix<<<and_grid(n, nsm), kAndThreads, 0, s>>>(n, slot_ptrs(b, n, w), w, slot, c, hi, lo, p64, b.x);
    return cudaGetLastError();
}

}  // namespace fld
