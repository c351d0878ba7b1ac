// fld_kernels.cu -- CUDA kernels of the GB300 FLD solver (sm_103a).
//
// Koerner et al., "Flux-Limited Diffusion for Multiple Scattering in
// Participating Media", CGF 33(2) 2014:
//   * medium preparation and initialisation (Algorithm 1, first steps);
//   * one colour pass of the red-black SOR relaxation (Algorithm 1) with the
//     Knudsen number (Eq. 35), D update (Eq. 33), face coefficients
//     D_ps = (D_p + D_s)/2, local update (Eq. 32) and SOR blend (Eq. 36);
//   * the residual of Eq. 37 with D recomputed from phi, reduced on the
//     device (warp shuffles, block tree, deterministic second pass);
//   * the single-scatter source q_ri = L sigma_s T (Sec. 3 after Eq. 6) by
//     a transmittance march (Eq. 3).
//
// The stencil is memory-bound: no tensor-core formulation applies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "fld_cell.cuh"
#include "fld_device.cuh"
#include "fld_internal.h"

namespace fld {

namespace {

using namespace cell;

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block; valid in thread 0.  blockDim <= 1024.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < (nthr + 31) / 32) ? sh[tid] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Sum over the block of a float-float value per thread, valid in thread 0:
// float-float shuffles within each warp, then the warps' sums in FP64 in
// warp order (GB300's FP64 rate is a small fraction of its FP32 rate, so the
// per-element sums stay on the FP32 pipes).
__device__ __forceinline__ double block_sum_ff(ff v, double *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ff u{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, u);
    }
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = ff_to_d(v);
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < (nthr + 31) / 32) ? sh[tid] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Second pass: fixed-order sum of the per-block partial pairs.
__global__ void __launch_bounds__(kRedThreads) k_finalize(const double *__restrict__ partials, int nblocks,
                                                         double *__restrict__ result) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = block_sum(a, sh);
    __syncthreads();
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        result[0] = a;
        result[1] = b;
    }
}

// ---------------------------------------------------------------------------
// Preparation
// ---------------------------------------------------------------------------
// sigma' = max(sigma_t, sigma_eps) and sigma_a' = (1 - albedo) sigma' in
// single precision; with BF both are rounded to bfloat16 (nearest, ties to
// even), the bit patterns kept for the sweeps that read bfloat16 and the
// rounded values, upcast exactly, stored in sp / ah2 for all other kernels.
template <bool BF>
__global__ void k_prep_f(Layout L, const float *__restrict__ st, const float *__restrict__ alb,
                         const float *__restrict__ js, float *__restrict__ sp, float *__restrict__ ah2,
                         float *__restrict__ jh2, uint16_t *__restrict__ spb, uint16_t *__restrict__ sab, float seps,
                         float h2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const long long v = ((long long)k * L.ny + j) * L.nx + i;
    const int q = L.at(i, j, k);
    float s = fmaxf(st[v], seps);                                 // Algorithm 1: sigma floor
    float a = __fmul_rn(__fsub_rn(1.0f, alb[v]), s);              // (1 - albedo) sigma'
    if (BF) {
        const uint16_t sb = __bfloat16_as_ushort(__float2bfloat16_rn(s));
        const uint16_t ab = __bfloat16_as_ushort(__float2bfloat16_rn(a));
        spb[q] = sb;
        sab[q] = ab;
        s = bf16_bits_to_f(sb);
        a = bf16_bits_to_f(ab);
    }
    sp[q] = s;
    ah2[q] = __fmul_rn(a, h2);                                    // sigma_a' dl^2
    jh2[q] = __fmul_rn(js[v], h2);
}

template <bool BF>
__global__ void k_prep_d(Layout L, const float *__restrict__ st, const float *__restrict__ alb,
                         const float *__restrict__ js, double *__restrict__ sp, double *__restrict__ ah2,
                         double *__restrict__ jh2, double seps, double h2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const long long v = ((long long)k * L.ny + j) * L.nx + i;
    const int q = L.at(i, j, k);
    double s, a;
    if (BF) {   // the rounded medium of k_prep_f<true>, exactly
        const float s32 = fmaxf(st[v], (float)seps);
        const float a32 = __fmul_rn(__fsub_rn(1.0f, alb[v]), s32);
        s = (double)bf16_bits_to_f(__bfloat16_as_ushort(__float2bfloat16_rn(s32)));
        a = (double)bf16_bits_to_f(__bfloat16_as_ushort(__float2bfloat16_rn(a32)));
    } else {
        s = fmax((double)st[v], seps);
        a = __dmul_rn(1.0 - (double)alb[v], s);
    }
    sp[q] = s;
    ah2[q] = __dmul_rn(a, h2);
    jh2[q] = __dmul_rn((double)js[v], h2);
}

// Every element of both colour arrays: unknowns get (phi0, D0), the ghost
// layer (phi_b, D_b), the alignment slack of each half row 0.
template <typename T>
__global__ void k_init(Layout L, T *__restrict__ phi, float *__restrict__ phlo, T *__restrict__ D, T phi0, T D0,
                       T phi_b, T D_b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.total) return;
    const int c = e >= L.cs ? 1 : 0;
    const int r = e - c * L.cs;
    const int K = r / (L.hpx * L.py);
    const int w = r - K * (L.hpx * L.py);
    const int J = w / L.hpx;
    const int pos = w - J * L.hpx - kXoff;            // = (I + 1) >> 1 for a cell
    const int par = (J + K + 1 + c) & 1;               // I & 1 of this row's cells
    const int I = par ? 2 * pos - 1 : 2 * pos;
    T p = T(0), d = T(0);
    if (pos >= 0 && I >= 0 && I <= L.nx + 1) {
        const bool ghost = I == 0 || J == 0 || K == 0 || I == L.nx + 1 || J == L.ny + 1 || K == L.nz + 1;
        p = ghost ? phi_b : phi0;
        d = ghost ? D_b : D0;
    }
    phi[e] = p;
    D[e] = d;
    if (phlo) phlo[e] = 0.0f;
}

// Packed (nx+2)(ny+2)(nz+2) <-> device layout.
__global__ void k_unpack_to_f(Layout L, const double *__restrict__ src, float *__restrict__ hi,
                              float *__restrict__ lo) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    const int K = blockIdx.z;
    if (I > L.nx + 1) return;
    const double x = src[((long long)K * (L.ny + 2) + J) * (L.nx + 2) + I];
    const int q = L.at(I - 1, J - 1, K - 1);
    const float h = (float)x;
    hi[q] = h;
    if (lo) lo[q] = (float)(x - (double)h);
}

__global__ void k_unpack_to_d(Layout L, const double *__restrict__ src, double *__restrict__ dst) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    const int K = blockIdx.z;
    if (I > L.nx + 1) return;
    dst[L.at(I - 1, J - 1, K - 1)] = src[((long long)K * (L.ny + 2) + J) * (L.nx + 2) + I];
}

__global__ void k_pack_from_f(Layout L, const float *__restrict__ hi, const float *__restrict__ lo,
                              double *__restrict__ dst) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    const int K = blockIdx.z;
    if (I > L.nx + 1) return;
    const int q = L.at(I - 1, J - 1, K - 1);
    dst[((long long)K * (L.ny + 2) + J) * (L.nx + 2) + I] = (double)hi[q] + (lo ? (double)lo[q] : 0.0);
}

__global__ void k_pack_from_d(Layout L, const double *__restrict__ src, double *__restrict__ dst) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    const int K = blockIdx.z;
    if (I > L.nx + 1) return;
    dst[((long long)K * (L.ny + 2) + J) * (L.nx + 2) + I] = src[L.at(I - 1, J - 1, K - 1)];
}

__global__ void k_f_to_d(long long n, const float *__restrict__ hi, const float *__restrict__ lo,
                         double *__restrict__ dst) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) dst[e] = (double)hi[e] + (lo ? (double)lo[e] : 0.0);
}

__global__ void k_d_to_f(long long n, const double *__restrict__ src, float *__restrict__ hi,
                         float *__restrict__ lo) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double x = src[e];
    const float h = (float)x;
    hi[e] = h;
    if (lo) lo[e] = (float)(x - (double)h);
}

// ---------------------------------------------------------------------------
// Red-black pass.
//
// Thread (t, J, K) of colour c updates the t-th unknown of colour c in row
// (J, K) (padded I = 2t + 2 - ((J + K + 1 + c) & 1)) if the row has one.  All six neighbours have the other colour, so a pass is
// free of races and its result does not depend on thread order.  Within a
// warp every access is a run of consecutive elements of one colour array.
//
// Update in residual form: with d_s = phi_s - phi_p and D_ps = (D_p + D_s)/2,
//   S(D_p)   = j dl^2 - sigma_a' dl^2 phi_p + sum_s D_ps d_s
//            = jh2 - ah2 phi_p + (D_p/2) sum_s d_s + (1/2) sum_s D_s d_s
//   den(D_p) = ah2 + sum_s D_ps = ah2 + 3 D_p + (1/2) sum_s D_s
// and Eq. 32 reads phi' = phi_p + S/den (num/den of the paper with num - phi_p
// den = S).  Each local round recomputes D_p (Eq. 35, 33) at the current
// point value phi_p + delta and sets delta = S(D_p)/den(D_p); the SOR blend
// (Eq. 36) is phi_p + omega * delta.  One round is Algorithm 1 as printed.
// ---------------------------------------------------------------------------

struct Nbrs {
    int own, nb[6];
};

// Offsets of the t-th unknown of colour c in row (J, K) and of its
// neighbours (x-, x+, y-, y+, z-, z+); false if the row has fewer unknowns
// of that colour.  The row's unknowns of colour c are I = 2t + 2 - par,
// par = (J + K + 1 + c) & 1, i.e. every other I starting at 1 or 2.
__device__ __forceinline__ bool pass_cell(const Layout &L, int c, int t, int J, int K, Nbrs &o) {
    const int par = (J + K + 1 + c) & 1;
    const int I = 2 * t + 2 - par;
    if (I > L.nx) return false;
    const int row = L.row(J, K);
    const int ob = (1 - c) * L.cs;
    const int h = I >> 1;
    const int pos = (I + 1) >> 1;
    o.own = c * L.cs + row + pos;
    o.nb[0] = ob + row + h;
    o.nb[1] = ob + row + h + 1;
    o.nb[2] = ob + row - L.hpx + pos;
    o.nb[3] = ob + row + L.hpx + pos;
    o.nb[4] = ob + row - L.hpx * L.py + pos;
    o.nb[5] = ob + row + L.hpx * L.py + pos;
    return true;
}

// Terms of the residual-form update that do not depend on D_p, shared by the
// sweep and the residual kernel so both evaluate the same discrete equation
// bit for bit:  A = sum_s d_s,  B = sum_s D_s d_s,  C = sum_s D_s,
// base = jh2 - ah2 phi_p + B/2, and the central differences.  A and B are
// compensated sums (Ogita-Rump-Oishi style): each difference d_s =
// phi_s - phi_p is formed exactly as a pair (TwoSum of the high words plus
// the low words), each product D_s d_s exactly by TwoProd, and the running
// sums carry their rounding errors in a separate low word.
struct FFTerms {
    ff A, base;
    float C, gx, gy, gz;
};

__device__ __forceinline__ FFTerms ff_terms(float p0, float p0lo, const float ps[6], const float ls[6],
                                            const float Ds[6], float ah, float jj) {
    FFTerms t;
    t.gx = __fadd_rn(__fsub_rn(ps[1], ps[0]), __fsub_rn(ls[1], ls[0]));
    t.gy = __fadd_rn(__fsub_rn(ps[3], ps[2]), __fsub_rn(ls[3], ls[2]));
    t.gz = __fadd_rn(__fsub_rn(ps[5], ps[4]), __fsub_rn(ls[5], ls[4]));
    float Ah = 0.0f, Al = 0.0f, Bh = 0.0f, Bl = 0.0f, C = 0.0f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const ff dh = two_sum(ps[s], -p0);                                  // exact high part
        const float dl = __fadd_rn(__fsub_rn(ls[s], p0lo), dh.lo);          // low part
        const ff a = two_sum(Ah, dh.hi);
        Ah = a.hi;
        Al = __fadd_rn(Al, __fadd_rn(dl, a.lo));
        const ff pr = two_prod(Ds[s], dh.hi);
        const float pe = fmaf(Ds[s], dl, pr.lo);
        const ff b = two_sum(Bh, pr.hi);
        Bh = b.hi;
        Bl = __fadd_rn(Bl, __fadd_rn(pe, b.lo));
        C = __fadd_rn(C, Ds[s]);
    }
    const ff B = fast_two_sum(Bh, Bl);
    ff base = ff_add_f(ff_mul_f(ff{p0, p0lo}, -ah), jj);
    t.base = ff_add(base, ff{0.5f * B.hi, 0.5f * B.lo});
    t.A = fast_two_sum(Ah, Al);
    t.C = C;
    return t;
}

// S(D_p) = base + (D_p / 2) A  and  den(D_p) = ah2 + 3 D_p + C / 2.
__device__ __forceinline__ ff ff_S(const FFTerms &t, float Dp) { return ff_add(t.base, ff_mul_f(t.A, 0.5f * Dp)); }
__device__ __forceinline__ float ff_den(const FFTerms &t, float ah, float Dp) {
    return __fadd_rn(__fadd_rn(ah, 3.0f * Dp), 0.5f * t.C);
}

// Two adjacent unknowns t, t+1 (t even) of one colour in row (J, K) per
// thread: in the colour-split layout they are one aligned float2 of every
// field, their x-neighbours three consecutive elements of the other colour's
// row and their y/z-neighbours a float2 one row/plane away.
struct Pair {
    int own, xv, ym, yp, zm, zp;              // offsets of the float2s (own colour at own, the other at the rest)
    bool first, second;                       // which of the two cells are unknowns
    bool left;                                // x-neighbours at xv-1, xv, xv+1 (else xv, xv+1, xv+2)
};

__device__ __forceinline__ void pair_cells(const Layout &L, int c, int t, int J, int K, Pair &q) {
    const int par = (J + K + 1 + c) & 1;
    const int I0 = 2 * t + 2 - par;                 // padded I of cell t
    q.first = I0 <= L.nx;
    q.second = I0 + 2 <= L.nx;
    const int row = (K * L.py + J) * L.hpx + kXoff + 1;   // element of the row's first unknown
    const int ob = (1 - c) * L.cs;
    q.own = c * L.cs + row + t;
    q.left = par == 1;                              // x-neighbours of cell t: (I0 - 1) and (I0 + 1)
    q.xv = ob + row + t;
    q.ym = ob + row - L.hpx + t;
    q.yp = ob + row + L.hpx + t;
    q.zm = ob + row - L.hpx * L.py + t;
    q.zp = ob + row + L.hpx * L.py + t;
}

__device__ __forceinline__ float2 ld2(const float *__restrict__ p, int off) {
    return *reinterpret_cast<const float2 *>(p + off);
}


// Gather the six neighbours of the two cells of a pair from one field.
__device__ __forceinline__ void gather_pair(const float *f, const Pair &q, float v0[6], float v1[6]) {
    const float2 xv = ld2(f, q.xv);
    const float xe = q.left ? f[q.xv - 1] : f[q.xv + 2];
    if (q.left) {
        v0[0] = xe; v0[1] = xv.x; v1[0] = xv.x; v1[1] = xv.y;
    } else {
        v0[0] = xv.x; v0[1] = xv.y; v1[0] = xv.y; v1[1] = xe;
    }
    const float2 ym = ld2(f, q.ym), yp = ld2(f, q.yp), zm = ld2(f, q.zm), zp = ld2(f, q.zp);
    v0[2] = ym.x; v0[3] = yp.x; v0[4] = zm.x; v0[5] = zp.x;
    v1[2] = ym.y; v1[3] = yp.y; v1[4] = zm.y; v1[5] = zp.y;
}

// sigma' and sigma_a' h^2 of the two cells of a pair: the single-precision
// fields, or the bfloat16 copies (one 32-bit load each; the first cell is the
// low half) with sigma_a' scaled by h^2 as k_prep_f scales it.
template <bool BF>
__device__ __forceinline__ void medium_pair(const float *__restrict__ sp, const float *__restrict__ ah2,
                                            const uint16_t *__restrict__ spb, const uint16_t *__restrict__ sab,
                                            float h2, int off, float2 &s2, float2 &a2) {
    if (BF) {
        const uint32_t us = *reinterpret_cast<const uint32_t *>(spb + off);
        const uint32_t ua = *reinterpret_cast<const uint32_t *>(sab + off);
        s2 = make_float2(__uint_as_float(us << 16), __uint_as_float(us & 0xFFFF0000u));
        a2 = make_float2(__fmul_rn(__uint_as_float(ua << 16), h2), __fmul_rn(__uint_as_float(ua & 0xFFFF0000u), h2));
    } else {
        s2 = ld2(sp, off);
        a2 = ld2(ah2, off);
    }
}

// Single-precision pass (the bulk sweeps), two unknowns per thread: the pair
// (t, t+1) of row (J, K); waits for the preceding grid (pdl_wait) before
// reading phi / D.
template <int LIM, int ROUNDS, bool BF>
__device__ __forceinline__ void tile_f32(const Layout &L, const float *__restrict__ sp,
                                         const float *__restrict__ ah2, const float *__restrict__ jh2,
                                         const uint16_t *__restrict__ spb, const uint16_t *__restrict__ sab, float h2,
                                         float *phi, float *D, int colour, int lim_rt, float larsen_n, float omega,
                                         float inv2h, float floor_, int rounds_rt, int t, int J, int K) {
    if (J > L.ny) return;
    Pair q;
    pair_cells(L, colour, t, J, K, q);
    if (!q.first) return;
    float2 s2, a2;
    medium_pair<BF>(sp, ah2, spb, sab, h2, q.own, s2, a2);
    const float2 j2 = ld2(jh2, q.own);
    pdl_wait();
    float ps0[6], ps1[6], Ds0[6], Ds1[6];
    gather_pair(phi, q, ps0, ps1);
    gather_pair(D, q, Ds0, Ds1);
    const float2 p0 = ld2(phi, q.own);
    float pn0, dn0, pn1, dn1;
    cell_f32<LIM, ROUNDS>(p0.x, ps0, Ds0, s2.x, a2.x, j2.x, lim_rt, larsen_n, omega, inv2h, floor_, rounds_rt, pn0,
                          dn0);
    if (q.second) {
        cell_f32<LIM, ROUNDS>(p0.y, ps1, Ds1, s2.y, a2.y, j2.y, lim_rt, larsen_n, omega, inv2h, floor_, rounds_rt,
                              pn1, dn1);
        *reinterpret_cast<float2 *>(phi + q.own) = make_float2(pn0, pn1);
        *reinterpret_cast<float2 *>(D + q.own) = make_float2(dn0, dn1);
    } else {
        phi[q.own] = pn0;          // the element after the last unknown is a ghost: left untouched
        D[q.own] = dn0;
    }
}

// The launched FP32 pass.  Registers are left to hold all of a thread's
// loads in flight (48, five CTAs per SM): measured faster than capping them
// for occupancy (six CTAs at 40 registers: 8.0 against 7.8 us per 128^3 pass).
template <int LIM, int ROUNDS, bool BF>
__global__ void __launch_bounds__(256, 4) k_pass2_f32(Layout L, const float *__restrict__ sp,
                                                   const float *__restrict__ ah2, const float *__restrict__ jh2,
                                                   const uint16_t *__restrict__ spb,
                                                   const uint16_t *__restrict__ sab, float h2,
                                                   float *__restrict__ phi, float *__restrict__ D, int colour,
                                                   int lim_rt, float larsen_n, float omega, float inv2h,
                                                   float floor_, int rounds_rt) {
    pdl_launch_dependents();
    tile_f32<LIM, ROUNDS, BF>(L, sp, ah2, jh2, spb, sab, h2, phi, D, colour, lim_rt, larsen_n, omega,
                                           inv2h, floor_, rounds_rt, 2 * (blockIdx.x * blockDim.x + threadIdx.x),
                                           blockIdx.y * blockDim.y + threadIdx.y + 1, blockIdx.z + 1);
}

// Middle pass (phi as a hi/lo pair, FP32-summed update, cell::cell_fh):
// tile_fh is the arithmetic of a pair of unknowns; k_pass2_fh launches it.
template <int LIM, int ROUNDS, bool BF>
__device__ __forceinline__ void tile_fh(const Layout &L, const float *__restrict__ sp,
                                        const float *__restrict__ ah2, const float *__restrict__ jh2,
                                        const uint16_t *__restrict__ spb, const uint16_t *__restrict__ sab, float h2,
                                        float *phi, float *phlo, float *D, int colour, int lim_rt, float larsen_n,
                                        float omega, float inv2h, float floor_, int rounds_rt, int t, int J, int K) {
    if (J > L.ny) return;
    Pair q;
    pair_cells(L, colour, t, J, K, q);
    if (!q.first) return;
    float2 s2, a2;
    medium_pair<BF>(sp, ah2, spb, sab, h2, q.own, s2, a2);
    const float2 j2 = ld2(jh2, q.own);
    pdl_wait();
    float ps0[6], ps1[6], ls0[6], ls1[6], Ds0[6], Ds1[6];
    gather_pair(phi, q, ps0, ps1);
    gather_pair(phlo, q, ls0, ls1);
    gather_pair(D, q, Ds0, Ds1);
    const float2 p0 = ld2(phi, q.own), l0 = ld2(phlo, q.own);
    float h0, lo0, d0, h1, lo1, d1;
    cell_fh<LIM, ROUNDS>(p0.x, l0.x, ps0, ls0, Ds0, s2.x, a2.x, j2.x, lim_rt, larsen_n, omega, inv2h, floor_,
                         rounds_rt, h0, lo0, d0);
    if (q.second) {
        cell_fh<LIM, ROUNDS>(p0.y, l0.y, ps1, ls1, Ds1, s2.y, a2.y, j2.y, lim_rt, larsen_n, omega, inv2h, floor_,
                             rounds_rt, h1, lo1, d1);
        *reinterpret_cast<float2 *>(phi + q.own) = make_float2(h0, h1);
        *reinterpret_cast<float2 *>(phlo + q.own) = make_float2(lo0, lo1);
        *reinterpret_cast<float2 *>(D + q.own) = make_float2(d0, d1);
    } else {
        phi[q.own] = h0;
        phlo[q.own] = lo0;
        D[q.own] = d0;
    }
}

// The launched hi/lo pass (64 registers, four CTAs per SM, no spills; at
// five CTAs per SM it spilled and ran 15 % slower at 256^3).
template <int LIM, int ROUNDS, bool BF>
__global__ void __launch_bounds__(256, 4) k_pass2_fh(Layout L, const float *__restrict__ sp,
                                                  const float *__restrict__ ah2, const float *__restrict__ jh2,
                                                  const uint16_t *__restrict__ spb,
                                                  const uint16_t *__restrict__ sab, float h2,
                                                  float *__restrict__ phi, float *__restrict__ phlo,
                                                  float *__restrict__ D, int colour, int lim_rt, float larsen_n,
                                                  float omega, float inv2h, float floor_, int rounds_rt) {
    pdl_launch_dependents();
    tile_fh<LIM, ROUNDS, BF>(L, sp, ah2, jh2, spb, sab, h2, phi, phlo, D, colour, lim_rt, larsen_n,
                                          omega, inv2h, floor_, rounds_rt,
                                          2 * (blockIdx.x * blockDim.x + threadIdx.x),
                                          blockIdx.y * blockDim.y + threadIdx.y + 1, blockIdx.z + 1);
}

// Four adjacent unknowns t .. t+3 (t a multiple of 4) of one colour in row
// (J, K) per thread: one aligned 128-bit load per own field and per y/z
// neighbour row/plane, the x-neighbours five consecutive elements of the other
// colour's row (a 128-bit load and one scalar).  Same per-cell arithmetic as
// the pair passes (cell::cell_f32 / cell::cell_fh), so the results agree bit
// for bit; more independent cells per thread, fewer loads and address
// computations per cell.
struct Quad {
    int own, xv, ym, yp, zm, zp;              // offsets of the float4s (own colour at own, the other at the rest)
    int n;                                    // unknowns among the four (1 .. 4)
    bool left;                                // x-neighbours at xv-1 .. xv+3 (else xv .. xv+4)
};

__device__ __forceinline__ bool quad_cells(const Layout &L, int c, int t, int J, int K, Quad &q) {
    const int par = (J + K + 1 + c) & 1;
    const int I0 = 2 * t + 2 - par;                 // padded I of cell t
    if (I0 > L.nx) return false;
    q.n = min(4, (L.nx - I0) / 2 + 1);
    const int row = (K * L.py + J) * L.hpx + kXoff + 1;   // element of the row's first unknown
    const int ob = (1 - c) * L.cs;
    q.own = c * L.cs + row + t;
    q.left = par == 1;
    q.xv = ob + row + t;
    q.ym = ob + row - L.hpx + t;
    q.yp = ob + row + L.hpx + t;
    q.zm = ob + row - L.hpx * L.py + t;
    q.zp = ob + row + L.hpx * L.py + t;
    return true;
}

__device__ __forceinline__ float4 ld4(const float *__restrict__ p, int off) {
    return *reinterpret_cast<const float4 *>(p + off);
}

__device__ __forceinline__ float f4_at(const float4 &v, int m) {
    return m == 0 ? v.x : m == 1 ? v.y : m == 2 ? v.z : v.w;
}

// The six neighbours of the four cells of a quad from one field: v[m][s].
__device__ __forceinline__ void gather_quad(const float *f, const Quad &q, float v[4][6]) {
    const float4 xv = ld4(f, q.xv);
    const float xe = q.left ? f[q.xv - 1] : f[q.xv + 4];
    const float x5[5] = {q.left ? xe : xv.x, q.left ? xv.x : xv.y, q.left ? xv.y : xv.z, q.left ? xv.z : xv.w,
                         q.left ? xv.w : xe};
    const float4 ym = ld4(f, q.ym), yp = ld4(f, q.yp), zm = ld4(f, q.zm), zp = ld4(f, q.zp);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[m][0] = x5[m];
        v[m][1] = x5[m + 1];
        v[m][2] = f4_at(ym, m);
        v[m][3] = f4_at(yp, m);
        v[m][4] = f4_at(zm, m);
        v[m][5] = f4_at(zp, m);
    }
}

template <bool BF>
__device__ __forceinline__ void medium_quad(const float *__restrict__ sp, const float *__restrict__ ah2,
                                            const uint16_t *__restrict__ spb, const uint16_t *__restrict__ sab,
                                            float h2, int off, float s4[4], float a4[4]) {
    if (BF) {
        const uint2 us = *reinterpret_cast<const uint2 *>(spb + off);
        const uint2 ua = *reinterpret_cast<const uint2 *>(sab + off);
        const uint32_t w[4] = {us.x << 16, us.x & 0xFFFF0000u, us.y << 16, us.y & 0xFFFF0000u};
        const uint32_t z[4] = {ua.x << 16, ua.x & 0xFFFF0000u, ua.y << 16, ua.y & 0xFFFF0000u};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            s4[m] = __uint_as_float(w[m]);
            a4[m] = __fmul_rn(__uint_as_float(z[m]), h2);
        }
    } else {
        const float4 s = ld4(sp, off), a = ld4(ah2, off);
        s4[0] = s.x; s4[1] = s.y; s4[2] = s.z; s4[3] = s.w;
        a4[0] = a.x; a4[1] = a.y; a4[2] = a.z; a4[3] = a.w;
    }
}

__device__ __forceinline__ void store_quad(float *p, const Quad &q, const float v[4]) {
    if (q.n == 4) {
        *reinterpret_cast<float4 *>(p + q.own) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        // the element after the last unknown is a ghost: left untouched
        for (int m = 0; m < q.n; ++m) p[q.own + m] = v[m];
    }
}

// Four unknowns per thread, single precision (k_pass4_f32) or hi/lo (HL,
// k_pass4_fh).
template <int LIM, int ROUNDS, bool BF, bool HL>
__device__ __forceinline__ void tile4(const Layout &L, const float *__restrict__ sp, const float *__restrict__ ah2,
                                      const float *__restrict__ jh2, const uint16_t *__restrict__ spb,
                                      const uint16_t *__restrict__ sab, float h2, float *phi, float *phlo, float *D,
                                      int colour, int lim_rt, float larsen_n, float omega, float inv2h, float floor_,
                                      int rounds_rt, int t, int J, int K) {
    if (J > L.ny) return;
    Quad q;
    if (!quad_cells(L, colour, t, J, K, q)) return;
    float s4[4], a4[4];
    medium_quad<BF>(sp, ah2, spb, sab, h2, q.own, s4, a4);
    const float4 j4 = ld4(jh2, q.own);
    const float jj[4] = {j4.x, j4.y, j4.z, j4.w};
    pdl_wait();
    float ps[4][6], Ds[4][6];
    gather_quad(phi, q, ps);
    gather_quad(D, q, Ds);
    const float4 p4 = ld4(phi, q.own);
    const float p0[4] = {p4.x, p4.y, p4.z, p4.w};
    float pn[4], dn[4], ln[4];
    if (HL) {
        float ls[4][6];
        gather_quad(phlo, q, ls);
        const float4 l4 = ld4(phlo, q.own);
        const float l0[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int m = 0; m < 4; ++m)
            cell_fh<LIM, ROUNDS>(p0[m], l0[m], ps[m], ls[m], Ds[m], s4[m], a4[m], jj[m], lim_rt, larsen_n, omega,
                                 inv2h, floor_, rounds_rt, pn[m], ln[m], dn[m]);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m)
            cell_f32<LIM, ROUNDS>(p0[m], ps[m], Ds[m], s4[m], a4[m], jj[m], lim_rt, larsen_n, omega, inv2h, floor_,
                                  rounds_rt, pn[m], dn[m]);
    }
    store_quad(phi, q, pn);
    store_quad(D, q, dn);
    if (HL) store_quad(phlo, q, ln);
}

template <int LIM, int ROUNDS, bool BF, bool HL>
__global__ void __launch_bounds__(128) k_pass4(Layout L, const float *__restrict__ sp, const float *__restrict__ ah2,
                                               const float *__restrict__ jh2, const uint16_t *__restrict__ spb,
                                               const uint16_t *__restrict__ sab, float h2, float *__restrict__ phi,
                                               float *__restrict__ phlo, float *__restrict__ D, int colour,
                                               int lim_rt, float larsen_n, float omega, float inv2h, float floor_,
                                               int rounds_rt) {
    pdl_launch_dependents();
    tile4<LIM, ROUNDS, BF, HL>(L, sp, ah2, jh2, spb, sab, h2, phi, phlo, D, colour, lim_rt, larsen_n, omega, inv2h,
                               floor_, rounds_rt, 4 * (blockIdx.x * blockDim.x + threadIdx.x),
                               blockIdx.y * blockDim.y + threadIdx.y + 1, blockIdx.z + 1);
}

// Multi-grid colour pass: one launch updates one colour of every grid in a
// table of SweepDescs.  The CTAs are persistent (all resident) and walk the
// work items of all grids with a grid-wide stride; item i belongs to the last
// grid whose first item is <= i (binary search over the firsts, staged in
// shared memory).  An item is what a CTA of the solo pair pass covers and its
// unknowns go through tile_f32 / tile_fh with the grid's own parameters, so
// every grid gets the bits of its solo passes.  The table and both counts
// are read on the device: one captured graph of these launches serves any
// set of grids.
__device__ __forceinline__ SweepDesc load_sweep_desc(const SweepDesc *__restrict__ p) {
    SweepDesc d;
    const int4 *src = reinterpret_cast<const int4 *>(p);
    int4 *dst = reinterpret_cast<int4 *>(&d);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(SweepDesc) / 16); ++i) dst[i] = __ldg(src + i);
    return d;
}

constexpr int kMultiThreadsX = 32, kMultiThreadsY = 8;

// One instantiation per limiter fast path, medium and family (a table holds
// grids of one family; limiter and medium are the batch's own).
template <int LIM, int ROUNDS, bool BF, bool HL>
__global__ void __launch_bounds__(kMultiThreadsX * kMultiThreadsY, 4)
    k_pass2_multi(const SweepDesc *__restrict__ descs, const int *__restrict__ counts, int colour) {
    __shared__ int first[kMultiMaxGrids];
    pdl_launch_dependents();
    const int ng = min(__ldg(counts), kMultiMaxGrids), total = __ldg(counts + 1);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int g = tid; g < ng; g += blockDim.x * blockDim.y) first[g] = __ldg(&descs[g].first);
    __syncthreads();
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = ng - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const SweepDesc d = load_sweep_desc(descs + lo);
        const int local = item - d.first;
        const int bx = local % d.bx, rest = local / d.bx;
        const int by = rest % d.by, bz = rest / d.by;
        if (bz >= d.L.nz) continue;
        const int t = 2 * (bx * kMultiThreadsX + threadIdx.x);
        const int J = by * kMultiThreadsY + threadIdx.y + 1;
        if (HL)
            tile_fh<LIM, ROUNDS, BF>(d.L, d.sp, d.ah2, d.jh2, d.spb, d.sab, d.h2, d.phi, d.phlo, d.D, colour, d.lim,
                                     d.larsen_n, d.omega, d.inv2h, d.floor_, d.local_iters, t, J, bz + 1);
        else
            tile_f32<LIM, ROUNDS, BF>(d.L, d.sp, d.ah2, d.jh2, d.spb, d.sab, d.h2, d.phi, d.D, colour, d.lim,
                                      d.larsen_n, d.omega, d.inv2h, d.floor_, d.local_iters, t, J, bz + 1);
    }
}

template <bool BF, bool HL>
auto multi_kernel(int lim, int local_iters) {
    if (local_iters == 2 && lim == LIM_LP) return k_pass2_multi<LIM_LP, 2, BF, HL>;
    return k_pass2_multi<-1, 0, BF, HL>;
}

// Float-float correction pass: phi kept as a hi/lo pair, S summed so the
// update is accurate to the pair's precision; correctly rounded D (the same
// function the residual kernel evaluates).
template <int LIM, int ROUNDS>
__device__ __forceinline__ void pass_ff_body(const Layout &L, const float *__restrict__ sp,
                                             const float *__restrict__ ah2, const float *__restrict__ jh2,
                                             float *__restrict__ phi, float *__restrict__ phlo,
                                             float *__restrict__ D, int colour, int t, int J, int K, int lim_rt,
                                             float larsen_n, float omega, float inv2h, float floor_,
                                             int rounds_rt) {
    const int lim = LIM >= 0 ? LIM : lim_rt;
    const int local_iters = ROUNDS > 0 ? ROUNDS : rounds_rt;
    Nbrs o;
    if (J > L.ny || !pass_cell(L, colour, t, J, K, o)) return;
    const float s_ = sp[o.own], ah = ah2[o.own], jj = jh2[o.own];
    pdl_wait();
    const float p0 = phi[o.own], p0lo = phlo[o.own];
    float ps[6], ls[6], Ds[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        ps[s] = phi[o.nb[s]];
        ls[s] = phlo[o.nb[s]];
        Ds[s] = D[o.nb[s]];
    }
    const FFTerms T = ff_terms(p0, p0lo, ps, ls, Ds, ah, jj);
    const float gmax = grad_floor_f(T.gx, T.gy, T.gz, inv2h, floor_);
    float delta = 0.0f, Dp = 0.0f;
#pragma unroll
    for (int r = 0; r < (ROUNDS > 0 ? ROUNDS : 64); ++r) {
        if (ROUNDS == 0 && r >= local_iters) break;
        Dp = D_of_f(gmax, s_, __fadd_rn(p0, delta), floor_, lim, larsen_n);
        const ff S = ff_S(T, Dp);
        // delta is a correction: its rounding does not move the fixed point
        delta = __fdividef(__fadd_rn(S.hi, S.lo), ff_den(T, ah, Dp));
    }
    const ff nw = ff_add_f(ff{p0, p0lo}, __fmul_rn(omega, delta));
    phi[o.own] = nw.hi;
    phlo[o.own] = nw.lo;
    D[o.own] = Dp;
}

template <int LIM, int ROUNDS>
__global__ void __launch_bounds__(256) k_pass_ff(Layout L, const float *__restrict__ sp,
                                                 const float *__restrict__ ah2, const float *__restrict__ jh2,
                                                 float *__restrict__ phi, float *__restrict__ phlo,
                                                 float *__restrict__ D, int colour, int lim_rt, float larsen_n,
                                                 float omega, float inv2h, float floor_, int rounds_rt) {
    pdl_launch_dependents();
    pass_ff_body<LIM, ROUNDS>(L, sp, ah2, jh2, phi, phlo, D, colour, blockIdx.x * blockDim.x + threadIdx.x,
                              blockIdx.y * blockDim.y + threadIdx.y + 1, blockIdx.z + 1, lim_rt, larsen_n, omega,
                              inv2h, floor_, rounds_rt);
}

// Jacobi variant: phi^{k+1} at every unknown (both colours) from phi^k
// (src) and D^k (written by the preceding fresh-D pass), into dst.  The update
// is the residual form of Eq. 32 damped by omega (Eq. 36): phi' = phi_p +
// omega S / den, S = j h^2 - sigma_a' h^2 phi_p + 1/2 (D_p sum d + sum D_s d),
// den = sigma_a' h^2 + 3 D_p + 1/2 sum D_s, d = phi_s - phi_p.
template <typename T>
__global__ void __launch_bounds__(256) k_jacobi(Layout L, const T *__restrict__ ah2, const T *__restrict__ jh2,
                                                const T *__restrict__ src, const T *__restrict__ D,
                                                T *__restrict__ dst, T omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const int q = L.at(i, j, k);
    const int nb[6] = {L.at(i - 1, j, k), L.at(i + 1, j, k), L.at(i, j - 1, k),
                       L.at(i, j + 1, k), L.at(i, j, k - 1), L.at(i, j, k + 1)};
    const T p0 = src[q], Dp = D[q], ah = ah2[q];
    T A = 0, B = 0, C = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const T d = src[nb[s]] - p0;
        const T Ds = D[nb[s]];
        A += d;
        B += Ds * d;
        C += Ds;
    }
    const T S = jh2[q] - ah * p0 + T(0.5) * (Dp * A + B);
    const T den = ah + T(3) * Dp + T(0.5) * C;
    dst[q] = p0 + omega * (S / den);
}

// Descriptor of a batched grid, read by every thread with uniform 16-byte
// loads (one transaction per warp, no shared-memory staging or barrier).
__device__ __forceinline__ BatchDesc load_desc(const BatchDesc *__restrict__ p) {
    BatchDesc d;
    const int4 *src = reinterpret_cast<const int4 *>(p);
    int4 *dst = reinterpret_cast<int4 *>(&d);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(BatchDesc) / 16); ++i) dst[i] = __ldg(src + i);
    return d;
}

__global__ void __launch_bounds__(256) k_pass_d(Layout L, const double *__restrict__ sp,
                                                const double *__restrict__ ah2, const double *__restrict__ jh2,
                                                double *__restrict__ phi, double *__restrict__ D, int colour,
                                                int lim, double larsen_n, double omega, double inv2h,
                                                double floor_, int local_iters) {
    Nbrs o;
    if (!pass_cell(L, colour, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y + 1,
                   blockIdx.z + 1, o) ||
        blockIdx.y * blockDim.y + threadIdx.y >= L.ny)
        return;
    const double p0 = phi[o.own];
    double ps[6], Ds[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        ps[s] = phi[o.nb[s]];
        Ds[s] = D[o.nb[s]];
    }
    const double s_ = sp[o.own], ah = ah2[o.own], jj = jh2[o.own];
    const double gx = ps[1] - ps[0], gy = ps[3] - ps[2], gz = ps[5] - ps[4];
    double A = 0.0, B = 0.0, C = 0.0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const double d = ps[s] - p0;
        A += d;
        B = fma(Ds[s], d, B);
        C += Ds[s];
    }
    const double base = fma(0.5, B, fma(-ah, p0, jj));
    double delta = 0.0, Dp = 0.0;
    for (int r = 0; r < local_iters; ++r) {
        Dp = knudsen_D_d(gx, gy, gz, inv2h, s_, p0 + delta, floor_, lim, larsen_n);
        const double S = fma(0.5 * Dp, A, base);
        const double den = (ah + 3.0 * Dp) + 0.5 * C;
        delta = S / den;
    }
    phi[o.own] = fma(omega, delta, p0);
    D[o.own] = Dp;
}

// ---------------------------------------------------------------------------
// Residual (Eq. 37) with D recomputed from the current phi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fresh_D_f_body(const Layout &L, const float *__restrict__ sp,
                                               const float *__restrict__ phi, const float *__restrict__ phlo,
                                               float *__restrict__ Df, int lim, float larsen_n, float inv2h,
                                               float floor_, int i, int j, int k) {
    if (i >= L.nx || j >= L.ny) return;
    const int q = L.at(i, j, k);
    const int xm = L.at(i - 1, j, k), xp = L.at(i + 1, j, k), ym = L.at(i, j - 1, k), yp = L.at(i, j + 1, k);
    const int zm = L.at(i, j, k - 1), zp = L.at(i, j, k + 1);
    float lxm = 0, lxp = 0, lym = 0, lyp = 0, lzm = 0, lzp = 0;
    if (phlo) {
        lxm = phlo[xm]; lxp = phlo[xp]; lym = phlo[ym]; lyp = phlo[yp];
        lzm = phlo[zm]; lzp = phlo[zp];
    }
    const float gx = __fadd_rn(__fsub_rn(phi[xp], phi[xm]), __fsub_rn(lxp, lxm));
    const float gy = __fadd_rn(__fsub_rn(phi[yp], phi[ym]), __fsub_rn(lyp, lym));
    const float gz = __fadd_rn(__fsub_rn(phi[zp], phi[zm]), __fsub_rn(lzp, lzm));
    Df[q] = knudsen_D_f(gx, gy, gz, inv2h, sp[q], phi[q], floor_, lim, larsen_n);
}

__global__ void k_fresh_D_f(Layout L, const float *__restrict__ sp, const float *__restrict__ phi,
                            const float *__restrict__ phlo, float *__restrict__ Df, int lim, float larsen_n,
                            float inv2h, float floor_) {
    fresh_D_f_body(L, sp, phi, phlo, Df, lim, larsen_n, inv2h, floor_, blockIdx.x * blockDim.x + threadIdx.x,
                   blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z);
}

__global__ void k_fresh_D_d(Layout L, const double *__restrict__ sp, const double *__restrict__ phi,
                            double *__restrict__ Df, int lim, double larsen_n, double inv2h, double floor_) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const int q = L.at(i, j, k);
    Df[q] = knudsen_D_d(phi[L.at(i + 1, j, k)] - phi[L.at(i - 1, j, k)],
                        phi[L.at(i, j + 1, k)] - phi[L.at(i, j - 1, k)],
                        phi[L.at(i, j, k + 1)] - phi[L.at(i, j, k - 1)], inv2h, sp[q], phi[q], floor_, lim, larsen_n);
}

// Per-voxel residual R_p dl^2 = jh2 - ah2 phi_p + sum_s D_ps (phi_s - phi_p)
// in float-float; its square (over the margin set) and the source square in
// double.
__device__ __forceinline__ void residual_f_terms(const Layout &L, const float *__restrict__ ah2,
                                                 const float *__restrict__ jh2, const float *__restrict__ phi,
                                                 const float *__restrict__ phlo, const float *__restrict__ Df,
                                                 const float *__restrict__ Dghost, int margin, int i, int j, int k,
                                                 ff &r2, ff &j2) {
    r2 = ff{0.0f, 0.0f};
    j2 = ff{0.0f, 0.0f};
    if (i >= L.nx || j >= L.ny) return;
    const int q = L.at(i, j, k);
    const int nb[6] = {L.at(i - 1, j, k), L.at(i + 1, j, k), L.at(i, j - 1, k),
                       L.at(i, j + 1, k), L.at(i, j, k - 1), L.at(i, j, k + 1)};
    const bool onface[6] = {i == 0, i == L.nx - 1, j == 0, j == L.ny - 1, k == 0, k == L.nz - 1};
    float ps[6], ls[6], Ds[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        ps[s] = phi[nb[s]];
        ls[s] = phlo ? phlo[nb[s]] : 0.0f;
        // ghost neighbours keep their Dirichlet D (never recomputed)
        Ds[s] = onface[s] ? Dghost[nb[s]] : Df[nb[s]];
    }
    const float ah = ah2[q];
    const FFTerms T = ff_terms(phi[q], phlo ? phlo[q] : 0.0f, ps, ls, Ds, ah, jh2[q]);
    const ff S = ff_S(T, Df[q]);
    const bool in = i >= margin && i < L.nx - margin && j >= margin && j < L.ny - margin && k >= margin &&
                    k < L.nz - margin;
    if (in) r2 = ff_mul(S, S);
    j2 = two_prod(jh2[q], jh2[q]);
}

__global__ void __launch_bounds__(256) k_residual_f(Layout L, const float *__restrict__ ah2,
                                                    const float *__restrict__ jh2, const float *__restrict__ phi,
                                                    const float *__restrict__ phlo, const float *__restrict__ Df,
                                                    const float *__restrict__ Dghost, int margin,
                                                    double *__restrict__ partials) {
    __shared__ double sh[32];
    ff r2f, j2f;
    residual_f_terms(L, ah2, jh2, phi, phlo, Df, Dghost, margin, blockIdx.x * blockDim.x + threadIdx.x,
                     blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z, r2f, j2f);
    const double r2 = block_sum_ff(r2f, sh);
    __syncthreads();
    const double j2 = block_sum_ff(j2f, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[2 * b] = r2;
        partials[2 * b + 1] = j2;
    }
}

// Batched fresh D / residual / finalize: CTA b works on grid cta_grid[b] with
// the same block decomposition as the solo launch, writes its partial sums to
// the grid's own slots, and one block per grid sums them in the solo order.
__global__ void __launch_bounds__(256) k_fresh_D_batch(const BatchDesc *__restrict__ descs,
                                                       const int *__restrict__ cta_grid, int lim) {
    const BatchDesc d = load_desc(descs + __ldg(cta_grid + blockIdx.x));
    if (!d.active) return;
    const int local = blockIdx.x - d.res_first;
    const int bx = local % d.res_bx, rest = local / d.res_bx;
    const int by = rest % d.res_by, bz = rest / d.res_by;
    fresh_D_f_body(d.L, d.sp, d.phi, d.mode ? d.phlo : nullptr, d.Df, lim, d.larsen_n, d.inv2h, d.floor_,
                   bx * blockDim.x + threadIdx.x, by * blockDim.y + threadIdx.y, bz);
}

__global__ void __launch_bounds__(256) k_residual_batch(const BatchDesc *__restrict__ descs,
                                                        const int *__restrict__ cta_grid, int margin,
                                                        double *__restrict__ partials) {
    __shared__ double sh[32];
    const BatchDesc d = load_desc(descs + __ldg(cta_grid + blockIdx.x));
    if (!d.active) return;
    const int local = blockIdx.x - d.res_first;
    const int bx = local % d.res_bx, rest = local / d.res_bx;
    const int by = rest % d.res_by, bz = rest / d.res_by;
    ff r2f, j2f;
    residual_f_terms(d.L, d.ah2, d.jh2, d.phi, d.mode ? d.phlo : nullptr, d.Df, d.D, margin,
                     bx * blockDim.x + threadIdx.x, by * blockDim.y + threadIdx.y, bz, r2f, j2f);
    const double r2 = block_sum_ff(r2f, sh);
    __syncthreads();
    const double j2 = block_sum_ff(j2f, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        partials[2 * (d.res_slot + local)] = r2;
        partials[2 * (d.res_slot + local) + 1] = j2;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_finalize_batch(const BatchDesc *__restrict__ descs,
                                                                const int *__restrict__ res_count,
                                                                const double *__restrict__ partials,
                                                                double *__restrict__ result) {
    __shared__ double sh[32];
    const BatchDesc &d = descs[blockIdx.x];
    if (!d.active) return;
    const int n = res_count[blockIdx.x];
    const double *p = partials + 2 * (long long)d.res_slot;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += p[2 * i];
        b += p[2 * i + 1];
    }
    a = block_sum(a, sh);
    __syncthreads();
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        result[2 * blockIdx.x] = a;
        result[2 * blockIdx.x + 1] = b;
    }
}

__global__ void __launch_bounds__(256) k_residual_d(Layout L, const double *__restrict__ ah2,
                                                    const double *__restrict__ jh2, const double *__restrict__ phi,
                                                    const double *__restrict__ Df, const double *__restrict__ Dghost,
                                                    int margin, double *__restrict__ partials) {
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double r2 = 0.0, j2 = 0.0;
    if (i < L.nx && j < L.ny) {
        const int q = L.at(i, j, k);
        const int nb[6] = {L.at(i - 1, j, k), L.at(i + 1, j, k), L.at(i, j - 1, k),
                           L.at(i, j + 1, k), L.at(i, j, k - 1), L.at(i, j, k + 1)};
        const bool onface[6] = {i == 0, i == L.nx - 1, j == 0, j == L.ny - 1, k == 0, k == L.nz - 1};
        const double p0 = phi[q], Dp = Df[q];
        double A = 0.0, B = 0.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            const double Dn = onface[s] ? Dghost[nb[s]] : Df[nb[s]];
            const double d = phi[nb[s]] - p0;
            A += d;
            B = fma(Dn, d, B);
        }
        const double S = fma(0.5 * Dp, A, fma(0.5, B, fma(-ah2[q], p0, jh2[q])));
        const bool in = i >= margin && i < L.nx - margin && j >= margin && j < L.ny - margin && k >= margin &&
                        k < L.nz - margin;
        r2 = in ? S * S : 0.0;
        j2 = jh2[q] * jh2[q];
    }
    r2 = block_sum(r2, sh);
    __syncthreads();
    j2 = block_sum(j2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[2 * b] = r2;
        partials[2 * b + 1] = j2;
    }
}

__global__ void __launch_bounds__(256) k_sumsq(long long n, const float *__restrict__ x,
                                               double *__restrict__ partials) {
    __shared__ double sh[32];
    double a = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double v = (double)x[e];
        a += v * v;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

// Input validation counters: [0] bad sigma (NaN/neg/inf), [1] bad albedo, [2] bad j.
__global__ void __launch_bounds__(256) k_validate(long long n, const float *__restrict__ st,
                                                  const float *__restrict__ alb, const float *__restrict__ js,
                                                  double *__restrict__ partials) {
    __shared__ double sh[32];
    double bs = 0.0, ba = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        if (st) {
            const float s = st[e];
            bs += !(s >= 0.0f && s <= 3.0e38f) ? 1.0 : 0.0;
        }
        if (alb) {
            const float a = alb[e];
            ba += !(a >= 0.0f && a <= 1.0f) ? 1.0 : 0.0;
        }
        if (js) {
            const float v = js[e];
            bs += !(v >= 0.0f && v <= 3.0e38f) ? 1.0 : 0.0;
        }
    }
    bs = block_sum(bs, sh);
    __syncthreads();
    ba = block_sum(ba, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = bs;
        partials[2 * blockIdx.x + 1] = ba;
    }
}

// ---------------------------------------------------------------------------
// Single-scatter source.
// ---------------------------------------------------------------------------

// exp(-(t.hi + t.lo)) for an optical depth held as a float-float pair
// (|t.lo| <= ulp(t.hi)/2, so exp(-t.lo) = 1 - t.lo to single precision)
__device__ __forceinline__ float transmittance(ff t) { return expf(-t.hi) * (1.0f - t.lo); }

// Light along -z with step h/2: the samples at quarter-voxel offsets blend the
// two nearest centres 3:1 and 1:3, so the optical depth above voxel k is the
// trapezoid sum over the centres above it plus half a voxel of the top
// centre -- an exclusive scan down each column.  Each trapezoid term
// (h/2)(s + s_above) is formed exactly as a float-float pair (TwoSum, then
// TwoProd by h/2) and summed in float-float, so the depth is as accurate as
// a double-precision sum without double-precision arithmetic.
__global__ void k_bake_scan_negz(Layout L, const float *__restrict__ st, const float *__restrict__ alb,
                                 float *__restrict__ js, float h, float radiance, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= L.nx || j >= L.ny) return;
    const long long col = (long long)j * L.nx + i;
    const long long sk = (long long)L.nx * L.ny;
    const float hh = 0.5f * h;
    ff tau = {0.0f, 0.0f};
    float above = 0.0f;
    for (int k = L.nz - 1; k >= 0; --k) {
        const long long v = col + (long long)k * sk;
        const float s = st[v];
        const ff sum = (k == L.nz - 1) ? ff{s, 0.0f} : two_sum(s, above);
        const ff p = two_prod(sum.hi, hh);
        tau = ff_add(tau, fast_two_sum(p.hi, fmaf(sum.lo, hh, p.lo)));
        above = s;
        const float q = radiance * (alb[v] * s) * transmittance(tau);
        js[v] = accumulate ? js[v] + q : q;
    }
}

__device__ __forceinline__ float sigma_trilinear(const Layout &L, const float *__restrict__ st, float h, float x,
                                                 float y, float z) {
    float u[3] = {x / h - 0.5f, y / h - 0.5f, z / h - 0.5f};
    const int n[3] = {L.nx, L.ny, L.nz};
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float w = fminf(fmaxf(u[a], 0.0f), (float)(n[a] - 1));
        int b = (int)floorf(w);
        b = min(max(b, 0), max(n[a] - 2, 0));
        i0[a] = b;
        f[a] = (n[a] == 1) ? 0.0f : w - (float)b;
    }
    const int i1 = min(i0[0] + 1, L.nx - 1), j1 = min(i0[1] + 1, L.ny - 1), k1 = min(i0[2] + 1, L.nz - 1);
    const long long sy = L.nx, sz = (long long)L.nx * L.ny;
    const long long b00 = i0[2] * sz + i0[1] * sy, b01 = i0[2] * sz + j1 * sy;
    const long long b10 = k1 * sz + i0[1] * sy, b11 = k1 * sz + j1 * sy;
    const float c00 = __ldg(st + b00 + i0[0]) * (1.0f - f[0]) + __ldg(st + b00 + i1) * f[0];
    const float c01 = __ldg(st + b01 + i0[0]) * (1.0f - f[0]) + __ldg(st + b01 + i1) * f[0];
    const float c10 = __ldg(st + b10 + i0[0]) * (1.0f - f[0]) + __ldg(st + b10 + i1) * f[0];
    const float c11 = __ldg(st + b11 + i0[0]) * (1.0f - f[0]) + __ldg(st + b11 + i1) * f[0];
    const float c0 = c00 * (1.0f - f[1]) + c01 * f[1];
    const float c1 = c10 * (1.0f - f[1]) + c11 * f[1];
    return c0 * (1.0f - f[2]) + c1 * f[2];
}

// General march: from the voxel centre towards the light, samples at the
// midpoints of steps of length `step`, the last step shortened to end at the
// grid boundary (or at a point light inside the grid).
__global__ void __launch_bounds__(256) k_bake_march(Layout L, const float *__restrict__ st,
                                                    const float *__restrict__ alb, float *__restrict__ js, float h,
                                                    float wx, float wy, float wz, float px, float py, float pz,
                                                    int point, float value, float step, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const long long v = ((long long)k * L.ny + j) * L.nx + i;
    const float x[3] = {(i + 0.5f) * h, (j + 0.5f) * h, (k + 0.5f) * h};
    float w[3] = {wx, wy, wz};
    float r = 0.0f;
    if (point) {
        const float d[3] = {px - x[0], py - x[1], pz - x[2]};
        r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r > 0.0f) {
            w[0] = d[0] / r; w[1] = d[1] / r; w[2] = d[2] / r;
        }
    }
    const float ext[3] = {L.nx * h, L.ny * h, L.nz * h};
    float len = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (w[a] > 0.0f) len = fminf(len, (ext[a] - x[a]) / w[a]);
        else if (w[a] < 0.0f) len = fminf(len, (0.0f - x[a]) / w[a]);
    }
    if (point) len = (r > 0.0f) ? fminf(len, r) : 0.0f;
    // optical depth: the single-precision samples sigma * step summed in
    // float-float (TwoSum), as accurate as a double-precision sum
    ff tau = {0.0f, 0.0f};
    const int m_full = (int)floorf(len / step);
    for (int m = 0; m < m_full; ++m) {
        const float t = ((float)m + 0.5f) * step;
        tau = ff_add_f(tau, sigma_trilinear(L, st, h, x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]) * step);
    }
    const float rem = len - (float)m_full * step;
    if (rem > 1e-6f * step) {
        const float t = (float)m_full * step + 0.5f * rem;
        tau = ff_add_f(tau, sigma_trilinear(L, st, h, x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]) * rem);
    }
    float q = value * (alb[v] * st[v]) * transmittance(tau);
    if (point) {
        const float rr = fmaxf(r, 0.5f * h);
        q = q / (4.0f * 3.14159265358979f * rr * rr);
    }
    js[v] = accumulate ? js[v] + q : q;
}

// One thread per unknown of the colour in a row (ceil(nx/2) of them), one
// y-row per thread row, one z-plane per block z.
inline dim3 pass_grid(const Layout &L, dim3 blk) {
    const int half = (L.nx + 1) / 2;
    return dim3((half + blk.x - 1) / blk.x, (L.ny + blk.y - 1) / blk.y, L.nz);
}

// two unknowns per thread (k_pass2_*): ceil(half / 2) threads per half row
inline dim3 pass2_grid(const Layout &L, dim3 blk) {
    const int pairs = ((L.nx + 1) / 2 + 1) / 2;
    return dim3((pairs + blk.x - 1) / blk.x, (L.ny + blk.y - 1) / blk.y, L.nz);
}

// four unknowns per thread (k_pass4): ceil(half / 4) threads per half row
inline dim3 pass4_grid(const Layout &L, dim3 blk) {
    const int quads = ((L.nx + 1) / 2 + 3) / 4;
    return dim3((quads + blk.x - 1) / blk.x, (L.ny + blk.y - 1) / blk.y, L.nz);
}

inline dim3 vox_block() { return dim3(32, 8, 1); }
inline dim3 vox_grid(const Layout &L) {
    return dim3((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_prep_f(const Layout &L, const Fields &f, float sigma_eps, float h2, bool bf16, cudaStream_t s) {
    auto k = bf16 ? k_prep_f<true> : k_prep_f<false>;
    k<<<vox_grid(L), vox_block(), 0, s>>>(L, f.sigma_t, f.albedo, f.jsrc, f.sp, f.ah2, f.jh2, f.spb, f.sab, sigma_eps,
                                          h2);
    return cudaGetLastError();
}

cudaError_t launch_prep_d(const Layout &L, const Fields &f, double sigma_eps, double h2, bool bf16,
                          cudaStream_t s) {
    auto k = bf16 ? k_prep_d<true> : k_prep_d<false>;
    k<<<vox_grid(L), vox_block(), 0, s>>>(L, f.sigma_t, f.albedo, f.jsrc, f.sp64, f.ah264, f.jh264, sigma_eps, h2);
    return cudaGetLastError();
}

cudaError_t launch_init_f(const Layout &L, float *phi, float *phlo, float *D, double phi0, double D0, double phi_b,
                          double D_b, cudaStream_t s) {
    const int blk = 256;
    const int nb = (L.total + blk - 1) / blk;
    k_init<float><<<nb, blk, 0, s>>>(L, phi, phlo, D, (float)phi0, (float)D0, (float)phi_b, (float)D_b);
    return cudaGetLastError();
}

cudaError_t launch_init_d(const Layout &L, double *phi, double *D, double phi0, double D0, double phi_b, double D_b,
                          cudaStream_t s) {
    const int blk = 256;
    const int nb = (L.total + blk - 1) / blk;
    k_init<double><<<nb, blk, 0, s>>>(L, phi, nullptr, D, phi0, D0, phi_b, D_b);
    return cudaGetLastError();
}

static dim3 packed_grid(const Layout &L) { return dim3((L.nx + 2 + 127) / 128, L.ny + 2, L.nz + 2); }

cudaError_t launch_unpack_to_f(const Layout &L, const double *src, float *hi, float *lo, cudaStream_t s) {
    k_unpack_to_f<<<packed_grid(L), 128, 0, s>>>(L, src, hi, lo);
    return cudaGetLastError();
}
cudaError_t launch_unpack_to_d(const Layout &L, const double *src, double *dst, cudaStream_t s) {
    k_unpack_to_d<<<packed_grid(L), 128, 0, s>>>(L, src, dst);
    return cudaGetLastError();
}
cudaError_t launch_pack_from_f(const Layout &L, const float *hi, const float *lo, double *dst, cudaStream_t s) {
    k_pack_from_f<<<packed_grid(L), 128, 0, s>>>(L, hi, lo, dst);
    return cudaGetLastError();
}
cudaError_t launch_pack_from_d(const Layout &L, const double *src, double *dst, cudaStream_t s) {
    k_pack_from_d<<<packed_grid(L), 128, 0, s>>>(L, src, dst);
    return cudaGetLastError();
}
cudaError_t launch_f_to_d(const Layout &L, const float *hi, const float *lo, double *dst, cudaStream_t s) {
    k_f_to_d<<<(L.total + 255) / 256, 256, 0, s>>>(L.total, hi, lo, dst);
    return cudaGetLastError();
}
cudaError_t launch_d_to_f(const Layout &L, const double *src, float *hi, float *lo, cudaStream_t s) {
    k_d_to_f<<<(L.total + 255) / 256, 256, 0, s>>>(L.total, src, hi, lo);
    return cudaGetLastError();
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the preceding grid in the stream finishes (see pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grd, dim3 blk, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = blk;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

cudaError_t launch_pass(Family fam, const Layout &L, const Fields &f, const PassParams &p, int colour,
                        cudaStream_t s) {
    const dim3 blk(32, 8, 1);
    const dim3 grd = pass_grid(L, blk);
    const dim3 grd2 = pass2_grid(L, blk);
    switch (fam) {
    case FAM_F32:
    case FAM_FH:
        if (fam == FAM_F32 ? p.quad_f32 : p.quad_fh) {
            const dim3 blk4(32, 4, 1);
            const dim3 grd4 = pass4_grid(L, blk4);
            auto pick4 = [&](auto bf, auto hl) {
                constexpr bool B = decltype(bf)::value, H = decltype(hl)::value;
                auto k = k_pass4<-1, 0, B, H>;
                if (p.local_iters == 2 && p.lim == LIM_LP) k = k_pass4<LIM_LP, 2, B, H>;
                return launch_pdl(k, grd4, blk4, s, L, f.sp, f.ah2, f.jh2, f.spb, f.sab, (float)p.h2, f.phi, f.phlo,
                                  f.D, colour, p.lim, (float)p.larsen_n, (float)p.omega, (float)p.inv2h,
                                  (float)p.floor_, p.local_iters);
            };
            if (fam == FAM_FH)
                return p.bf16 ? pick4(std::true_type{}, std::true_type{}) : pick4(std::false_type{}, std::true_type{});
            return p.bf16 ? pick4(std::true_type{}, std::false_type{}) : pick4(std::false_type{}, std::false_type{});
        }
        if (fam == FAM_FH) break;
        {
        auto pick = [&](auto bf) {
            constexpr bool B = decltype(bf)::value;
            auto k = k_pass2_f32<-1, 0, B>;
            if (p.local_iters == 2 && p.lim == LIM_LP) k = k_pass2_f32<LIM_LP, 2, B>;
            else if (p.local_iters == 2 && p.lim == LIM_KERSHAW) k = k_pass2_f32<LIM_KERSHAW, 2, B>;
            else if (p.local_iters == 2 && p.lim == LIM_LARSEN) k = k_pass2_f32<LIM_LARSEN, 2, B>;
            return launch_pdl(k, grd2, blk, s, L, f.sp, f.ah2, f.jh2, f.spb, f.sab, (float)p.h2, f.phi, f.D, colour,
                              p.lim, (float)p.larsen_n, (float)p.omega, (float)p.inv2h, (float)p.floor_,
                              p.local_iters);
        };
        return p.bf16 ? pick(std::true_type{}) : pick(std::false_type{});
        }
    default:
        break;
    }
    switch (fam) {
    case FAM_FF: {
        auto k = k_pass_ff<-1, 0>;
        if (p.local_iters == 2 && p.lim == LIM_LP) k = k_pass_ff<LIM_LP, 2>;
        else if (p.local_iters == 2 && p.lim == LIM_KERSHAW) k = k_pass_ff<LIM_KERSHAW, 2>;
        else if (p.local_iters == 2 && p.lim == LIM_LARSEN) k = k_pass_ff<LIM_LARSEN, 2>;
        return launch_pdl(k, grd, blk, s, L, f.sp, f.ah2, f.jh2, f.phi, f.phlo, f.D, colour, p.lim,
                          (float)p.larsen_n, (float)p.omega, (float)p.inv2h, (float)p.floor_, p.local_iters);
    }
    case FAM_FH: {
        auto pick = [&](auto bf) {
            constexpr bool B = decltype(bf)::value;
            auto k = k_pass2_fh<-1, 0, B>;
            if (p.local_iters == 2 && p.lim == LIM_LP) k = k_pass2_fh<LIM_LP, 2, B>;
            else if (p.local_iters == 2 && p.lim == LIM_KERSHAW) k = k_pass2_fh<LIM_KERSHAW, 2, B>;
            else if (p.local_iters == 2 && p.lim == LIM_LARSEN) k = k_pass2_fh<LIM_LARSEN, 2, B>;
            return launch_pdl(k, grd2, blk, s, L, f.sp, f.ah2, f.jh2, f.spb, f.sab, (float)p.h2, f.phi, f.phlo,
                              f.D, colour, p.lim, (float)p.larsen_n, (float)p.omega, (float)p.inv2h,
                              (float)p.floor_, p.local_iters);
        };
        return p.bf16 ? pick(std::true_type{}) : pick(std::false_type{});
    }
    case FAM_F64:
        k_pass_d<<<grd, blk, 0, s>>>(L, f.sp64, f.ah264, f.jh264, f.phi64, f.D64, colour, p.lim, p.larsen_n,
                                    p.omega, p.inv2h, p.floor_, p.local_iters);
        break;
    }
    return cudaGetLastError();
}

void residual_dims(const Layout &L, int *bx, int *by) {
    const dim3 g = vox_grid(L);
    *bx = (int)g.x;
    *by = (int)g.y;
}

cudaError_t launch_residual_batch(const BatchDesc *descs, const int *cta_grid, int nctas, int ngrids,
                                  const int *res_count, double *partials, double *result, int lim, int margin,
                                  cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    k_fresh_D_batch<<<nctas, vox_block(), 0, s>>>(descs, cta_grid, lim);
    k_residual_batch<<<nctas, vox_block(), 0, s>>>(descs, cta_grid, margin, partials);
    k_finalize_batch<<<ngrids, kRedThreads, 0, s>>>(descs, res_count, partials, result);
    return cudaGetLastError();
}

void multi_dims(const Layout &L, int *bx, int *by) {
    const dim3 g = pass2_grid(L, dim3(kMultiThreadsX, kMultiThreadsY, 1));
    *bx = (int)g.x;
    *by = (int)g.y;
}

int multi_ctas(int nsm, int hl, int bf16, int lim, int local_iters) {
    auto k = hl ? (bf16 ? multi_kernel<true, true>(lim, local_iters) : multi_kernel<false, true>(lim, local_iters))
                : (bf16 ? multi_kernel<true, false>(lim, local_iters) : multi_kernel<false, false>(lim, local_iters));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMultiThreadsX * kMultiThreadsY, 0) !=
            cudaSuccess ||
        per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * (nsm > 0 ? nsm : 1);
}

cudaError_t launch_pass_multi(const SweepDesc *descs, const int *counts, int hl, int bf16, int lim, int local_iters,
                              int colour, int nctas, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    auto k = hl ? (bf16 ? multi_kernel<true, true>(lim, local_iters) : multi_kernel<false, true>(lim, local_iters))
                : (bf16 ? multi_kernel<true, false>(lim, local_iters) : multi_kernel<false, false>(lim, local_iters));
    return launch_pdl(k, dim3(nctas), dim3(kMultiThreadsX, kMultiThreadsY, 1), s, descs, counts, colour);
}

int reduction_blocks(const Layout &L) {
    const dim3 g = vox_grid(L);
    const long long n = (long long)g.x * g.y * g.z;
    return (int)(n > 4096 ? n : 4096);
}

cudaError_t launch_fresh_D_into(const Layout &L, Fields &f, const PassParams &p, cudaStream_t s) {
    k_fresh_D_f<<<vox_grid(L), vox_block(), 0, s>>>(L, f.sp, f.phi, nullptr, f.D, p.lim, (float)p.larsen_n,
                                                    (float)p.inv2h, (float)p.floor_);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(Family fam, const Layout &L, const Fields &f, const PassParams &p, int to_second,
                          cudaStream_t s) {
    const dim3 grd = vox_grid(L), blk = vox_block();
    if (fam == FAM_F64) {
        const double *src = to_second ? f.phi64 : f.phi642;
        double *dst = to_second ? f.phi642 : f.phi64;
        k_fresh_D_d<<<grd, blk, 0, s>>>(L, f.sp64, src, f.D64, p.lim, p.larsen_n, p.inv2h, p.floor_);
        k_jacobi<double><<<grd, blk, 0, s>>>(L, f.ah264, f.jh264, src, f.D64, dst, p.omega);
    } else {
        const float *src = to_second ? f.phi : f.phi2;
        float *dst = to_second ? f.phi2 : f.phi;
        k_fresh_D_f<<<grd, blk, 0, s>>>(L, f.sp, src, nullptr, f.D, p.lim, (float)p.larsen_n, (float)p.inv2h,
                                        (float)p.floor_);
        k_jacobi<float><<<grd, blk, 0, s>>>(L, f.ah2, f.jh2, src, f.D, dst, (float)p.omega);
    }
    return cudaGetLastError();
}

cudaError_t launch_residual(Family fam, const Layout &L, const Fields &f, const PassParams &p, int margin,
                            cudaStream_t s) {
    const dim3 grd = vox_grid(L), blk = vox_block();
    const int nblocks = (int)(grd.x * grd.y * grd.z);
    if (nblocks > f.partial_cap) return cudaErrorInvalidValue;
    if (fam == FAM_F64) {
        k_fresh_D_d<<<grd, blk, 0, s>>>(L, f.sp64, f.phi64, f.Df64, p.lim, p.larsen_n, p.inv2h, p.floor_);
        k_residual_d<<<grd, blk, 0, s>>>(L, f.ah264, f.jh264, f.phi64, f.Df64, f.D64, margin, f.partials);
    } else {
        const float *lo = fam == FAM_F32 ? nullptr : f.phlo;
        k_fresh_D_f<<<grd, blk, 0, s>>>(L, f.sp, f.phi, lo, f.Df, p.lim, (float)p.larsen_n, (float)p.inv2h,
                                        (float)p.floor_);
        k_residual_f<<<grd, blk, 0, s>>>(L, f.ah2, f.jh2, f.phi, lo, f.Df, f.D, margin, f.partials);
    }
    k_finalize<<<1, kRedThreads, 0, s>>>(f.partials, nblocks, f.result);
    return cudaGetLastError();
}

cudaError_t launch_sumsq_source(const Layout &L, const Fields &f, cudaStream_t s) {
    const long long n = (long long)L.nx * L.ny * L.nz;
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb > f.partial_cap) nb = f.partial_cap;
    k_sumsq<<<nb, 256, 0, s>>>(n, f.jsrc, f.partials);
    k_finalize<<<1, kRedThreads, 0, s>>>(f.partials, nb, f.result);
    return cudaGetLastError();
}

cudaError_t launch_validate(long long n, const Fields &f, const float *st, const float *alb, const float *js,
                            cudaStream_t s) {
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb > f.partial_cap) nb = f.partial_cap;
    if (nb < 1) nb = 1;
    k_validate<<<nb, 256, 0, s>>>(n, st, alb, js, f.partials);
    k_finalize<<<1, kRedThreads, 0, s>>>(f.partials, nb, f.result);
    return cudaGetLastError();
}

cudaError_t launch_bake_scan_negz(const Layout &L, const Fields &f, float h, float radiance, int accumulate,
                                  cudaStream_t s) {
    const dim3 blk(32, 4, 1);
    const dim3 grd((L.nx + 31) / 32, (L.ny + 3) / 4, 1);
    k_bake_scan_negz<<<grd, blk, 0, s>>>(L, f.sigma_t, f.albedo, f.jsrc, h, radiance, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_bake_march(const Layout &L, const Fields &f, float h, const double w[3], const double pos[3],
                              int point, float value, float step, int accumulate, cudaStream_t s) {
    k_bake_march<<<vox_grid(L), vox_block(), 0, s>>>(L, f.sigma_t, f.albedo, f.jsrc, h, (float)w[0], (float)w[1],
                                                     (float)w[2], (float)pos[0], (float)pos[1], (float)pos[2], point,
                                                     value, step, accumulate);
    return cudaGetLastError();
}

}  // namespace fld
