// fld_noalloc.cu -- an allocation-free variant of the residual evaluation.
//
// fld_residual (fld_capi.cu) works on a grid object and reduces through
// device buffers the grid allocated.  Some callers cannot allocate device
// memory at the point they need the residual: a renderer that embeds the
// solver in its frame loop (where cudaMalloc / cudaFree are banned after
// start-up because they synchronise the device and stall the frame), or a
// host application that owns all device memory through its own pool and
// hands the library only the buffers it is allowed to touch.  For them,
// fld_residual_noalloc takes every input and output from the caller and keeps
// its only scratch -- one pair of partial sums per thread block and a few
// result slots -- in the file-scope array below.
//
// The array lives in every GPU that loads this library until the process
// exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress (host code must not use the array's name as a device
// pointer: on the host it names a stand-in, not device memory).  Every call
// shares the array, so calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.  Nothing in it has to start at zero: each call writes every
// slot it later reads.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/fld.h"
#include "fld_device.cuh"
#include "fld_internal.h"

namespace {

using fld::knudsen_D_d;

constexpr int kMaxBlocks = FLD_NOALLOC_MAX_BLOCKS;   // partial-sum slots
constexpr int kSlots = 2 * kMaxBlocks + 8;           // + result slots
constexpr int kMaxDevices = 64;

// 2*kMaxBlocks + 8 doubles = 1 MiB + 64 bytes per device.
static __device__ __align__(256) double g_noalloc_scratch[kSlots];

std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Sum over the block, valid in thread 0.
__device__ __forceinline__ double na_block_sum(double v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < (nthr + 31) / 32) ? sh[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// Fixed-order sum of `nblocks` partial pairs into out[0], out[1].
__global__ void __launch_bounds__(256) k_na_finalize(const double *__restrict__ partials, int nblocks,
                                                     double *__restrict__ out) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = na_block_sum(a, sh);
    __syncthreads();
    b = na_block_sum(b, sh);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// Block partials of sum j^2 (first) over the unpadded source.
__global__ void __launch_bounds__(256) k_na_sumsq(int nx, int ny, const float *__restrict__ j,
                                                  double *__restrict__ partials) {
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int jj = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double a = 0.0;
    if (i < nx && jj < ny) {
        const double v = (double)j[((long long)k * ny + jj) * nx + i];
        a = v * v;
    }
    a = na_block_sum(a, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[2 * b] = a;
        partials[2 * b + 1] = 0.0;
    }
}

struct NaArgs {
    int nx, ny, nz, margin, lim;
    double h2, inv2h, sigma_eps, eps, larsen_n;
};

// D (Eq. 33-35) at unknown (i, j, k) from the packed padded phi.
__device__ __forceinline__ double na_D(const NaArgs &a, const float *__restrict__ st, const double *__restrict__ phi,
                                       int i, int j, int k, double floor_) {
    const long long px = a.nx + 2, plane = px * (a.ny + 2);
    const long long q = (long long)(k + 1) * plane + (long long)(j + 1) * px + (i + 1);
    const double sp = fmax((double)st[((long long)k * a.ny + j) * a.nx + i], a.sigma_eps);
    return knudsen_D_d(phi[q + 1] - phi[q - 1], phi[q + px] - phi[q - px], phi[q + plane] - phi[q - plane], a.inv2h,
                       sp, phi[q], floor_, a.lim, a.larsen_n);
}

// Residual of Eq. 37 with D recomputed from phi at the voxel and at its six
// neighbours (ghost neighbours keep the caller's ghost D); per-block partial
// sums of (R h^2)^2 over the margin set and of (j h^2)^2.
__global__ void __launch_bounds__(256) k_na_residual(NaArgs a, const float *__restrict__ st,
                                                     const float *__restrict__ alb, const float *__restrict__ js,
                                                     const double *__restrict__ phi, const double *__restrict__ D,
                                                     const double *__restrict__ jsum, double *__restrict__ partials) {
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const double nvox = (double)a.nx * a.ny * a.nz;
    const double jbar = sqrt(jsum[0] / nvox);
    const double floor_ = jbar > 0.0 ? a.eps * jbar : 1e-30;
    double r2 = 0.0, j2 = 0.0;
    if (i < a.nx && j < a.ny) {
        const long long px = a.nx + 2, plane = px * (a.ny + 2);
        const long long q = (long long)(k + 1) * plane + (long long)(j + 1) * px + (i + 1);
        const long long v = ((long long)k * a.ny + j) * a.nx + i;
        const double s = fmax((double)st[v], a.sigma_eps);
        const double ah = __dmul_rn(__dmul_rn(1.0 - (double)alb[v], s), a.h2);
        const double jh = __dmul_rn((double)js[v], a.h2);
        const double p0 = phi[q];
        const double Dp = na_D(a, st, phi, i, j, k, floor_);
        const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
        const long long nb[6] = {q - 1, q + 1, q - px, q + px, q - plane, q + plane};
        double A = 0.0, B = 0.0;
#pragma unroll
        for (int s6 = 0; s6 < 6; ++s6) {
            const int ii = i + di[s6], jn = j + dj[s6], kn = k + dk[s6];
            const bool ghost = ii < 0 || ii >= a.nx || jn < 0 || jn >= a.ny || kn < 0 || kn >= a.nz;
            const double Dn = ghost ? D[nb[s6]] : na_D(a, st, phi, ii, jn, kn, floor_);
            const double d = phi[nb[s6]] - p0;
            A += d;
            B = fma(Dn, d, B);
        }
        const double S = fma(0.5 * Dp, A, fma(0.5, B, fma(-ah, p0, jh)));
        const bool in = i >= a.margin && i < a.nx - a.margin && j >= a.margin && j < a.ny - a.margin &&
                        k >= a.margin && k < a.nz - a.margin;
        r2 = in ? S * S : 0.0;
        j2 = jh * jh;
    }
    r2 = na_block_sum(r2, sh);
    __syncthreads();
    j2 = na_block_sum(j2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[2 * b] = r2;
        partials[2 * b + 1] = j2;
    }
}

// Failures are reported through fld_last_error(), like every other entry point.
fld_status na_fail(fld_status s, const char *msg) {
    fld::set_error_text(msg);
    return s;
}

// Device address of the scratch array on the current device (looked up once).
fld_status scratch_address(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(FLD_ERR_NO_DEVICE, "no current CUDA device");
    }
    if (dev < 0 || dev >= kMaxDevices) return na_fail(FLD_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return na_fail(FLD_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return FLD_OK;
}

}  // namespace

extern "C" fld_status fld_residual_noalloc(int nx, int ny, int nz, double h, const fld_solve_params *p,
                                           const float *sigma_t, const float *albedo, const float *j,
                                           const double *phi, const double *D, double *rel, void *stream) {
    if (nx < 1 || ny < 1 || nz < 1) return na_fail(FLD_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (!(h > 0.0) || !isfinite(h)) return na_fail(FLD_ERR_INVALID_ARG, "h must be a positive finite number");
    if (!p || !sigma_t || !albedo || !j || !phi || !D || !rel)
        return na_fail(FLD_ERR_INVALID_ARG, "a required pointer is NULL");
    if (const char *bad = fld::check_limiter_margin(p->limiter, p->larsen_n, p->residual_margin))
        return na_fail(FLD_ERR_INVALID_ARG, bad);
    const dim3 blk(32, 8, 1);
    const dim3 grd((nx + 31) / 32, (ny + 7) / 8, nz);
    const long long nblocks = (long long)grd.x * grd.y * grd.z;
    if (nz > 65535 || nblocks > kMaxBlocks)
        return na_fail(FLD_ERR_INVALID_ARG,
                       "grid too large for the fixed scratch: ceil(nx/32)*ceil(ny/8)*nz must be <= "
                       "FLD_NOALLOC_MAX_BLOCKS (65536), e.g. 256^3");
    double *scratch = nullptr;
    fld_status st = scratch_address(&scratch);
    if (st != FLD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = scratch;                        // 2 * kMaxBlocks
    double *jsum = scratch + 2 * kMaxBlocks;           // [0] = sum j^2
    double *rsum = scratch + 2 * kMaxBlocks + 2;       // [0] = sum (R h^2)^2, [1] = sum (j h^2)^2

    int n = nx;
    if (ny > n) n = ny;
    if (nz > n) n = nz;
    NaArgs a;
    a.nx = nx; a.ny = ny; a.nz = nz; a.margin = p->residual_margin; a.lim = p->limiter;
    a.h2 = h * h;
    a.inv2h = 1.0 / (2.0 * h);
    a.sigma_eps = p->sigma_eps > 0.0 ? p->sigma_eps : 1e-3 / ((double)n * h);
    a.eps = p->eps > 0.0 ? p->eps : 1e-20;
    a.larsen_n = p->larsen_n;

    k_na_sumsq<<<grd, blk, 0, s>>>(nx, ny, j, partials);
    k_na_finalize<<<1, 256, 0, s>>>(partials, (int)nblocks, jsum);
    k_na_residual<<<grd, blk, 0, s>>>(a, sigma_t, albedo, j, phi, D, jsum, partials);
    k_na_finalize<<<1, 256, 0, s>>>(partials, (int)nblocks, rsum);
    cudaError_t e = cudaGetLastError();
    double r[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, rsum, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return na_fail(FLD_ERR_CUDA, cudaGetErrorString(e));
    }
    *rel = fld::rel_residual_from_sums(nx, ny, nz, h, a.margin, r[0], r[1]);
    return FLD_OK;
}
