// fld_cell.cuh -- arithmetic of one point update of the single-precision
// sweeps (Algorithm 1 of Koerner et al. 2014: Knudsen number Eq. 35, D by
// Eq. 33 with a Table 2 limiter, local update Eq. 32, SOR blend Eq. 36),
// shared by every kernel that runs these sweeps (launched colour passes,
// temporally blocked passes), so all of them produce the same bits for the
// same inputs.
#pragma once

#include <cuda_runtime.h>

#include "fld_device.cuh"

namespace fld {
namespace cell {

// The hardware's approximate reciprocal (PTX rcp.approx.ftz.f32, one
// special-function-unit instruction, within 1 ulp).  Its operands here are
// floored well above the denormal range (sigma' >= sigma_eps, the Knudsen
// denominators >= eps jbar, the update's denominator > 0), so flushing
// denormals changes nothing.
__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Limiter (Table 2) with approximate reciprocals, for the bulk
// single-precision sweeps, whose accuracy is bounded by phi stored in float;
// the correction sweeps and the residual use the correctly rounded forms.
// The sums below are written with explicit round-to-nearest adds: an
// operand here can be a product (the approximate quotients are x * rcp(y)),
// and a plain `+` could then be contracted into an FMA in one kernel and not
// in another, so kernels sharing this code would differ in the last bit.
__device__ __forceinline__ float limiter_fast(int kind, float larsen_n, float R) {
    switch (kind) {
    case LIM_CDA: return 1.0f / 3.0f;
    case LIM_SUM: return fast_rcp(__fadd_rn(3.0f, R));
    case LIM_MAX: return fast_rcp(fmaxf(3.0f, R));
    case LIM_KERSHAW: return 2.0f * fast_rcp(__fadd_rn(3.0f, hypotf(3.0f, 2.0f * R)));
    case LIM_LARSEN: {
        const float m = fmaxf(3.0f, R), s = fminf(3.0f, R);
        return fast_rcp(m * __powf(__fadd_rn(1.0f, __powf(s * fast_rcp(m), larsen_n)), fast_rcp(larsen_n)));
    }
    default: {
        if (R < 1.0f) return lp_series_f(R);
        const float r = fast_rcp(R);
        // 2e/(1-e), e = exp(-2R), is below 3.4e-8 of (1 - 1/R) once R > 9
        const float tail = R < 9.0f ? 2.0f * fast_rcp(__fsub_rn(__expf(2.0f * R), 1.0f)) : 0.0f;
        return r * __fadd_rn(__fsub_rn(1.0f, r), tail);
    }
    }
}

// Arithmetic of one FP32 point update from its gathered values: the
// neighbours' phi and D, its own phi and medium; returns the new phi and D.
template <int LIM, int ROUNDS>
__device__ __forceinline__ void cell_f32(float p0, const float ps[6], const float Ds[6], float s_, float ah, float jj,
                                         int lim_rt, float larsen_n, float omega, float inv2h, float floor_,
                                         int rounds_rt, float &phi_new, float &D_new) {
    const int lim = LIM >= 0 ? LIM : lim_rt;
    const int local_iters = ROUNDS > 0 ? ROUNDS : rounds_rt;
    const float gx = ps[1] - ps[0], gy = ps[3] - ps[2], gz = ps[5] - ps[4];
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    const float g = g2 > 0.0f ? g2 * rsqrtf(g2) * inv2h : 0.0f;     // |grad phi| (Eq. 34)
    const float gmax = fmaxf(g, floor_);
    const float inv_sp = fast_rcp(s_);
    float A = 0.0f, B = 0.0f, C = 0.0f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const float d = ps[s] - p0;
        A += d;
        B = fmaf(Ds[s], d, B);
        C += Ds[s];
    }
    const float base = fmaf(0.5f, B, fmaf(-ah, p0, jj));
    const float den0 = fmaf(0.5f, C, ah);
    float delta = 0.0f, Dp = 0.0f;
#pragma unroll
    for (int r = 0; r < (ROUNDS > 0 ? ROUNDS : 64); ++r) {
        if (ROUNDS == 0 && r >= local_iters) break;
        const float R = gmax * fast_rcp(fmaxf(s_ * __fadd_rn(p0, delta), floor_));     // Eq. 35
        Dp = limiter_fast(lim, larsen_n, R) * inv_sp;                          // Eq. 33
        delta = fmaf(0.5f * Dp, A, base) * fast_rcp(fmaf(3.0f, Dp, den0));   // Eq. 32
    }
    phi_new = fmaf(omega, delta, p0);                                          // Eq. 36
    D_new = Dp;
}

// Middle pass: phi kept as a hi/lo pair (no storage floor) but the update
// summed in plain FP32 with the approximate D of the bulk sweeps -- about the
// cost of the FP32 pass, reaching residuals a few times above the
// float-float pass's.  cell_fh is the arithmetic of one point.
template <int LIM, int ROUNDS>
__device__ __forceinline__ void cell_fh(float p0, float p0lo, const float ps[6], const float ls[6],
                                        const float Ds[6], float s_, float ah, float jj, int lim_rt, float larsen_n,
                                        float omega, float inv2h, float floor_, int rounds_rt, float &hi_new,
                                        float &lo_new, float &D_new) {
    const int lim = LIM >= 0 ? LIM : lim_rt;
    const int local_iters = ROUNDS > 0 ? ROUNDS : rounds_rt;
    float d[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) d[s] = (ps[s] - p0) + (ls[s] - p0lo);   // phi_s - phi_p
    const float gx = d[1] - d[0], gy = d[3] - d[2], gz = d[5] - d[4];
    const float g2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    const float g = g2 > 0.0f ? g2 * rsqrtf(g2) * inv2h : 0.0f;
    const float gmax = fmaxf(g, floor_);
    const float inv_sp = fast_rcp(s_);
    float A = 0.0f, B = 0.0f, C = 0.0f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        A += d[s];
        B = fmaf(Ds[s], d[s], B);
        C += Ds[s];
    }
    const float base = fmaf(0.5f, B, fmaf(-ah, p0, fmaf(-ah, p0lo, jj)));
    const float den0 = fmaf(0.5f, C, ah);
    float delta = 0.0f, Dp = 0.0f;
#pragma unroll
    for (int r = 0; r < (ROUNDS > 0 ? ROUNDS : 64); ++r) {
        if (ROUNDS == 0 && r >= local_iters) break;
        const float R = gmax * fast_rcp(fmaxf(s_ * __fadd_rn(p0, delta), floor_));
        Dp = limiter_fast(lim, larsen_n, R) * inv_sp;
        delta = fmaf(0.5f * Dp, A, base) * fast_rcp(fmaf(3.0f, Dp, den0));
    }
    const ff nw = ff_add_f(ff{p0, p0lo}, __fmul_rn(omega, delta));
    hi_new = nw.hi;
    lo_new = nw.lo;
    D_new = Dp;
}

// Programmatic dependent launch (PTX griddepcontrol): a pass lets the next
// grid in its stream be scheduled as soon as all of its own CTAs are running,
// and waits for the preceding grid to complete (with its writes visible)
// before it reads phi, phi_lo or D.  The medium (sigma', sigma_a' h^2, j h^2)
// is written only by earlier, fully completed kernels and is loaded before
// the wait.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace cell
}  // namespace fld
