// fld_anderson.cu -- Anderson mixing of blocks of sweeps (not in the paper).
//
// One block of red-black sweeps (Algorithm 1) is a fixed-point map
// G: phi -> phi' whose fixed point is the solution of Eq. 31.  Anderson
// mixing keeps the last m images g_i = G(x_i) and residuals f_i = g_i - x_i
// and starts the next block from x = sum_i a_i g_i, with the weights a
// (summing to 1) that minimise |sum_i a_i f_i|.  The weights come from the
// Gram matrix <f_i, f_j>, reduced here and solved on the host.
//
// Per element of a padded field (both colours, ghosts and row padding
// included -- there f is 0 and every g_i is the same value):
//   k_and_collect: g = phi (hi/lo pair, or FP64 split into one), f = g - x_cur
//                  rounded to float, stores g in its slot (float-float) and f
//                  (FP32), and accumulates <f, f_j> for every occupied slot j
//                  (exact products, float-float sums per thread and warp, FP64
//                  across warps and CTAs);
//   k_and_reduce:  sums the per-CTA partials in a fixed order (one warp per
//                  slot, strided lanes, then a fixed shuffle tree);
//   k_and_mix:     x = g_s + sum_{j != s} a_j (g_j - g_s) in float-float,
//                  written back as phi (hi/lo, float, or FP64) and as the next
//                  x_cur.
// All per-element arithmetic runs on the FP32 pipes as float-float (about 48
// bits): GB300 issues FP64 at a small fraction of its FP32 rate, and in FP64
// these passes cost a third of an Anderson-mixed solve.  The difference form
// leaves ghosts and padding exactly unchanged (every g_j - g_s is 0 there).
#include <cuda_runtime.h>
#include <stdint.h>

#include "fld_internal.h"

namespace fld {
namespace {

constexpr int kAndThreads = 256;

struct SlotPtrs {
    const float2 *g[kAndersonMax];
    const float *f[kAndersonMax];
};

// the mixing weights split into float-float pairs (on the host)
struct Coef {
    float hi[kAndersonMax], lo[kAndersonMax];
};

__device__ __forceinline__ ff ld_ff(const float2 *p, long long e) {
    const float2 v = p[e];
    return ff{v.x, v.y};
}

// The state at element e as a float-float pair: hi/lo (lo null: float), or
// FP64 split (FP64 sweeps only).
__device__ __forceinline__ ff state_at(const float *hi, const float *lo, const double *p64, long long e) {
    if (p64) {
        const double d = p64[e];
        const float h = (float)d;
        return ff{h, (float)(d - (double)h)};
    }
    return ff{hi[e], lo ? lo[e] : 0.0f};
}

__global__ void __launch_bounds__(kAndThreads) k_and_capture(int n, const float *__restrict__ hi,
                                                              const float *__restrict__ lo,
                                                              const double *__restrict__ p64,
                                                              float2 *__restrict__ x_cur) {
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const ff v = state_at(hi, lo, p64, e);
        x_cur[e] = make_float2(v.hi, v.lo);
    }
}

__global__ void __launch_bounds__(kAndThreads) k_and_collect(int n, const float *__restrict__ hi,
                                                              const float *__restrict__ lo,
                                                              const double *__restrict__ p64,
                                                              const float2 *__restrict__ x_cur, SlotPtrs sl,
                                                              float2 *__restrict__ g_out, float *__restrict__ f_out,
                                                              int w, int s, double *__restrict__ part) {
    ff acc[kAndersonMax];
#pragma unroll
    for (int j = 0; j < kAndersonMax; ++j) acc[j] = ff{0.0f, 0.0f};
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const ff g = state_at(hi, lo, p64, e);
        const ff d = ff_sub(g, ld_ff(x_cur, e));
        const float f = __fadd_rn(d.hi, d.lo);
        g_out[e] = make_float2(g.hi, g.lo);
        f_out[e] = f;
#pragma unroll
        for (int j = 0; j < kAndersonMax; ++j) {
            if (j < w) acc[j] = ff_add(acc[j], two_prod(f, j == s ? f : sl.f[j][e]));
        }
    }
    // block reduction of every accumulator: float-float warp shuffles, then
    // one FP64 value per warp in shared memory, summed by the first threads
    // in warp order
    __shared__ double red[kAndThreads / 32][kAndersonMax];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kAndersonMax; ++j) {
        if (j >= w) break;
        ff v = acc[j];
        for (int o = 16; o > 0; o >>= 1) {
            const ff u{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
            v = ff_add(v, u);
        }
        if (lane == 0) red[wid][j] = (double)v.hi + (double)v.lo;
    }
    __syncthreads();
    if (threadIdx.x < kAndersonMax) {
        double v = 0.0;
        if (threadIdx.x < w)
            for (int q = 0; q < kAndThreads / 32; ++q) v += red[q][threadIdx.x];
        part[(size_t)blockIdx.x * kAndersonMax + threadIdx.x] = v;
    }
}

// one warp per slot j: lane l sums partials l, l + 32, ... in order, then a
// fixed shuffle tree; the same order for the same number of CTAs
__global__ void __launch_bounds__(32 * kAndersonMax) k_and_reduce(const double *__restrict__ part, int nblocks,
                                                                  double *__restrict__ out) {
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += part[(size_t)b * kAndersonMax + j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[j] = v;
}

__global__ void __launch_bounds__(kAndThreads) k_and_mix(int n, SlotPtrs sl, int w, int s, Coef c,
                                                          float *__restrict__ hi, float *__restrict__ lo,
                                                          double *__restrict__ p64, float2 *__restrict__ x_cur) {
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const ff gs = ld_ff(sl.g[s], e);
        ff acc{0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < kAndersonMax; ++j) {
            if (j < w && j != s) acc = ff_add(acc, ff_mul(ff{c.hi[j], c.lo[j]}, ff_sub(ld_ff(sl.g[j], e), gs)));
        }
        ff x = ff_add(gs, acc);
        if (p64) {
            p64[e] = (double)x.hi + (double)x.lo;
        } else if (lo) {
            hi[e] = x.hi;
            lo[e] = x.lo;
        } else {
            hi[e] = x.hi;
            x.lo = 0.0f;
        }
        x_cur[e] = make_float2(x.hi, x.lo);
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
    k_and_reduce<<<1, 32 * kAndersonMax, 0, s>>>(b.part, nb, b.dots);
    return cudaGetLastError();
}

cudaError_t launch_anderson_mix(const AndersonBuffers &b, int n, int slot, int w, const double *a, float *hi,
                                float *lo, double *p64, int nsm, cudaStream_t s) {
    Coef c;
    for (int j = 0; j < kAndersonMax; ++j) {
        const double v = j < w ? a[j] : 0.0;
        c.hi[j] = (float)v;
        c.lo[j] = (float)(v - (double)c.hi[j]);
    }
    k_and_mix<<<and_grid(n, nsm), kAndThreads, 0, s>>>(n, slot_ptrs(b, n, w), w, slot, c, hi, lo, p64, b.x);
    return cudaGetLastError();
}

}  // namespace fld
