// fld_render.cu -- the primary ray march of Koerner et al. 2014 (Sec. 3):
// the radiance reaching the camera along each pixel's ray is the background
// attenuated over the whole chord plus, over march segments, the
// transmittance from the segment to the camera times the source Q times the
// segment length, with 4 pi Q = q_ri + sigma_s phi + j (the source written
// with the diffuse fluence phi; the solver's source field holds q_ri + j).
//
// k_render_pack gathers sigma_t, sigma_s = albedo sigma_t, the source and
// phi into one float4 per voxel (unpadded, x fastest), so that each sample's
// trilinear blend reads eight 16-byte corners; k_render marches one pixel per
// thread in 16x16 tiles (neighbouring rays touch neighbouring voxels, which
// stay in L1/L2) and also writes the gamma-compressed 8-bit code of Sec. 6.2.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fld_device.cuh"
#include "fld_internal.h"

namespace fld {
namespace {

// phi of a grid at a point, blended trilinearly between its voxel centres
// (clamped to the outermost centres); the grid's spacing is hc.
__device__ __forceinline__ float phi_trilinear(const Layout &C, const float *__restrict__ phi,
                                               const float *__restrict__ phlo, const double *__restrict__ phi64,
                                               float hc, float x, float y, float z) {
    const float c[3] = {x / hc - 0.5f, y / hc - 0.5f, z / hc - 0.5f};
    const int n[3] = {C.nx, C.ny, C.nz};
    int i0[3], i1[3];
    float w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float cu = fminf(fmaxf(c[d], 0.0f), (float)(n[d] - 1));
        int b = (int)floorf(cu);
        b = min(max(b, 0), max(n[d] - 2, 0));
        i0[d] = b;
        i1[d] = min(b + 1, n[d] - 1);
        w[d] = n[d] == 1 ? 0.0f : cu - (float)b;
    }
    float acc = 0.0f;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const int q = C.at(cx ? i1[0] : i0[0], cy ? i1[1] : i0[1], cz ? i1[2] : i0[2]);
                float v;
                if (phi64) v = (float)phi64[q];
                else v = phlo ? __fadd_rn(phi[q], phlo[q]) : phi[q];
                const float wt = (cx ? w[0] : 1.0f - w[0]) * (cy ? w[1] : 1.0f - w[1]) * (cz ? w[2] : 1.0f - w[2]);
                acc = fmaf(wt, v, acc);
            }
    return acc;
}

// One float4 {sigma_t, albedo sigma_t, source, phi} per voxel.  phi is the
// grid's own (coarse == false) or a coarser grid's, upsampled trilinearly to
// this grid's voxel centres (the quarter-resolution solve of Sec. 6.2).
__global__ void k_render_pack(Layout L, const float *__restrict__ st, const float *__restrict__ alb,
                              const float *__restrict__ q, const float *__restrict__ phi,
                              const float *__restrict__ phlo, const double *__restrict__ phi64, bool coarse,
                              Layout C, float h, float hc, float4 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const long long v = ((long long)k * L.ny + j) * L.nx + i;
    float ph;
    if (coarse) {
        ph = phi_trilinear(C, phi, phlo, phi64, hc, (i + 0.5f) * h, (j + 0.5f) * h, (k + 0.5f) * h);
    } else {
        const int p = L.at(i, j, k);
        if (phi64) ph = (float)phi64[p];
        else ph = phlo ? __fadd_rn(phi[p], phlo[p]) : phi[p];
    }
    const float s = st[v];
    out[v] = make_float4(s, __fmul_rn(alb[v], s), q[v], ph);
}

__global__ void k_prolong(Layout L, float *__restrict__ phi, float *__restrict__ phlo, const float *__restrict__ cphi,
                          const float *__restrict__ cphlo, const double *__restrict__ cphi64, Layout C, float h,
                          float hc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx || j >= L.ny) return;
    const int q = L.at(i, j, k);
    phi[q] = phi_trilinear(C, cphi, cphlo, cphi64, hc, (i + 0.5f) * h, (j + 0.5f) * h, (k + 0.5f) * h);
    phlo[q] = 0.0f;
}

// Box averages over f^3 blocks (the voxels that exist): sigma_t, albedo =
// mean(albedo sigma_t) / mean(sigma_t) (0 in vacuum) and the source of the
// coarse grid, accumulated in float-float.
__global__ void k_downsample(int nx, int ny, int nz, int f, int cx, int cy, int cz, const float *__restrict__ st,
                             const float *__restrict__ alb, const float *__restrict__ q, float *__restrict__ st_c,
                             float *__restrict__ alb_c, float *__restrict__ q_c) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= cx || J >= cy) return;
    // float-float sums (TwoSum; the albedo products exact by TwoProd), as
    // accurate as double-precision sums, then one division each
    ff s = {0.0f, 0.0f}, ss = {0.0f, 0.0f}, qq = {0.0f, 0.0f};
    int cnt = 0;
    for (int k = K * f; k < K * f + f && k < nz; ++k)
        for (int j = J * f; j < J * f + f && j < ny; ++j)
            for (int i = I * f; i < I * f + f && i < nx; ++i) {
                const long long v = ((long long)k * ny + j) * nx + i;
                const float sv = st[v];
                s = ff_add_f(s, sv);
                ss = ff_add(ss, two_prod(alb[v], sv));
                qq = ff_add_f(qq, q[v]);
                ++cnt;
            }
    const long long c = ((long long)K * cy + J) * cx + I;
    st_c[c] = ff_div_f(s, (float)cnt);
    alb_c[c] = s.hi > 0.0f ? ff_div(ss, s) : 0.0f;
    q_c[c] = ff_div_f(qq, (float)cnt);
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float w) {
    return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                       fmaf(w, b.w - a.w, a.w));
}

struct RenderArgs {
    int nx, ny, nz;
    float h, inv_h;
    float eye[3], f[3], r[3], u[3];
    float tan_half, aspect;
    int width, height;
    float step, background, t_min;
};

// Trilinear blend between voxel centres, clamped to the outermost centres.
__device__ __forceinline__ float4 sample(const RenderArgs &a, const float4 *__restrict__ vol, float x, float y,
                                         float z) {
    const float c[3] = {x * a.inv_h - 0.5f, y * a.inv_h - 0.5f, z * a.inv_h - 0.5f};
    const int n[3] = {a.nx, a.ny, a.nz};
    int i0[3], i1[3];
    float w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float cu = fminf(fmaxf(c[d], 0.0f), (float)(n[d] - 1));
        int b = (int)floorf(cu);
        b = min(max(b, 0), max(n[d] - 2, 0));
        i0[d] = b;
        i1[d] = min(b + 1, n[d] - 1);
        w[d] = n[d] == 1 ? 0.0f : cu - (float)b;
    }
    const long long sy = a.nx, sz = (long long)a.nx * a.ny;
    const long long z0 = i0[2] * sz, z1 = i1[2] * sz, y0 = i0[1] * sy, y1 = i1[1] * sy;
    const float4 c000 = __ldg(vol + z0 + y0 + i0[0]), c100 = __ldg(vol + z0 + y0 + i1[0]);
    const float4 c010 = __ldg(vol + z0 + y1 + i0[0]), c110 = __ldg(vol + z0 + y1 + i1[0]);
    const float4 c001 = __ldg(vol + z1 + y0 + i0[0]), c101 = __ldg(vol + z1 + y0 + i1[0]);
    const float4 c011 = __ldg(vol + z1 + y1 + i0[0]), c111 = __ldg(vol + z1 + y1 + i1[0]);
    const float4 x00 = lerp4(c000, c100, w[0]), x10 = lerp4(c010, c110, w[0]);
    const float4 x01 = lerp4(c001, c101, w[0]), x11 = lerp4(c011, c111, w[0]);
    return lerp4(lerp4(x00, x10, w[1]), lerp4(x01, x11, w[1]), w[2]);
}

__global__ void __launch_bounds__(256) k_render(RenderArgs a, const float4 *__restrict__ vol,
                                                float *__restrict__ radiance, uint8_t *__restrict__ codes,
                                                float exposure, float inv_gamma) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= a.width || py >= a.height) return;
    const float sx = (2.0f * (px + 0.5f) / a.width - 1.0f) * a.tan_half * a.aspect;
    const float sy = (1.0f - 2.0f * (py + 0.5f) / a.height) * a.tan_half;
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = fmaf(sx, a.r[k], fmaf(sy, a.u[k], a.f[k]));
    const float inv_norm = rsqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] *= inv_norm;
    // chord through the box [0, n h]^3 (slab test)
    const float box[3] = {a.nx * a.h, a.ny * a.h, a.nz * a.h};
    float t0 = 0.0f, t1 = INFINITY;
    bool hit = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) {
            if (a.eye[k] < 0.0f || a.eye[k] > box[k]) hit = false;
            continue;
        }
        float ta = (0.0f - a.eye[k]) / d[k], tb = (box[k] - a.eye[k]) / d[k];
        if (ta > tb) {
            const float tt = ta;
            ta = tb;
            tb = tt;
        }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    }
    float L = 0.0f, T = 1.0f;
    if (hit && t1 > t0) {
        // positions from the entry point keep the sample coordinates small
        const float e[3] = {fmaf(t0, d[0], a.eye[0]), fmaf(t0, d[1], a.eye[1]), fmaf(t0, d[2], a.eye[2])};
        const float len_total = t1 - t0;
        const int nseg = (int)ceilf(len_total / a.step);
        const float inv4pi = 0.0795774715459476679f;   // 1 / (4 pi)
        for (int m = 0; m < nseg && T >= a.t_min; ++m) {
            const float s0 = m * a.step;
            const float s1 = fminf(s0 + a.step, len_total);
            const float len = s1 - s0, sm = 0.5f * (s0 + s1);
            const float4 v = sample(a, vol, fmaf(sm, d[0], e[0]), fmaf(sm, d[1], e[1]), fmaf(sm, d[2], e[2]));
            const float Q = fmaf(v.y, v.w, v.z) * inv4pi;      // (q + sigma_s phi) / (4 pi)
            L = fmaf(T * Q, len, L);
            T *= __expf(-v.x * len);
        }
    }
    L = fmaf(a.background, T, L);
    const long long o = (long long)py * a.width + px;
    if (radiance) radiance[o] = L;
    if (codes) {
        const float g = powf(fmaxf(exposure * L, 0.0f), inv_gamma);
        codes[o] = (uint8_t)floorf(255.0f * fminf(g, 1.0f) + 0.5f);
    }
}

}  // namespace

cudaError_t launch_downsample(const Layout &L, const Fields &f, int factor, const Layout &C, Fields &fc,
                              cudaStream_t s) {
    const dim3 b(32, 8, 1), g((C.nx + 31) / 32, (C.ny + 7) / 8, C.nz);
    k_downsample<<<g, b, 0, s>>>(L.nx, L.ny, L.nz, factor, C.nx, C.ny, C.nz, f.sigma_t, f.albedo, f.jsrc,
                                 fc.sigma_t, fc.albedo, fc.jsrc);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const Layout &L, Fields &f, const PhiSource &ps, double h, cudaStream_t s) {
    const dim3 b(32, 8, 1), g((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
    k_prolong<<<g, b, 0, s>>>(L, f.phi, f.phlo, ps.phi, ps.phlo, ps.phi64, ps.C, (float)h, (float)ps.hc);
    return cudaGetLastError();
}

cudaError_t launch_render(const Layout &L, const Fields &f, const PhiSource &ps, const RenderCamera &c,
                          float4 *vol, float *radiance, uint8_t *codes, double exposure, double gamma,
                          cudaStream_t s) {
    const dim3 vb(32, 8, 1), vg((L.nx + 31) / 32, (L.ny + 7) / 8, L.nz);
    k_render_pack<<<vg, vb, 0, s>>>(L, f.sigma_t, f.albedo, f.jsrc, ps.phi, ps.phlo, ps.phi64, ps.coarse, ps.C,
                                    (float)c.h, (float)ps.hc, vol);
    RenderArgs a;
    a.nx = L.nx;
    a.ny = L.ny;
    a.nz = L.nz;
    a.h = (float)c.h;
    a.inv_h = (float)(1.0 / c.h);
    for (int k = 0; k < 3; ++k) {
        a.eye[k] = (float)c.eye[k];
        a.f[k] = (float)c.f[k];
        a.r[k] = (float)c.r[k];
        a.u[k] = (float)c.u[k];
    }
    a.tan_half = (float)c.tan_half;
    a.aspect = (float)c.aspect;
    a.width = c.width;
    a.height = c.height;
    a.step = (float)c.step;
    a.background = (float)c.background;
    a.t_min = (float)c.t_min;
    const dim3 rb(16, 16, 1), rg((c.width + 15) / 16, (c.height + 15) / 16, 1);
    k_render<<<rg, rb, 0, s>>>(a, vol, radiance, codes, (float)exposure, (float)(1.0 / gamma));
    return cudaGetLastError();
}

}  // namespace fld
