// fld_device.cuh -- device helpers of the GB300 FLD solver: grid layout,
// flux limiters (Table 2 of Koerner et al. 2014) in single and double
// precision, the floored Knudsen number (Eq. 35) and float-float arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fld {

// ---------------------------------------------------------------------------
// Layout of padded device fields.
//
// Unknown (i, j, k) lives at element  base + ((k+1)*py + (j+1))*px + (i+1)
// where base = kOx.  The ghost layer sits at i = -1 / nx etc.  kOx = 3 puts
// the first unknown of every row on a 16-byte boundary when px is a multiple
// of 4, so rows can be moved with 128-bit accesses.
// ---------------------------------------------------------------------------
constexpr int kOx = 3;

struct Layout {
    int nx, ny, nz;     // unknowns per axis
    int px, py;         // row pitch (elements) and rows per plane (ny + 2)
    long long plane;    // px * py
    long long total;    // elements per padded field (incl. alignment slack)

    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
        // i, j, k in [-1, n]: -1 and n are the ghost layer
        return kOx + ((long long)(k + 1) * py + (j + 1)) * px + (i + 1);
    }
};

inline Layout make_layout(int nx, int ny, int nz) {
    Layout L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    L.px = ((kOx + nx + 2) + 3) & ~3;
    L.py = ny + 2;
    L.plane = (long long)L.px * L.py;
    L.total = L.plane * (nz + 2) + 4;
    return L;
}

enum Limiter : int { LIM_CDA = 0, LIM_SUM = 1, LIM_MAX = 2, LIM_KERSHAW = 3, LIM_LARSEN = 4, LIM_LP = 5 };

// ---------------------------------------------------------------------------
// Levermore-Pomraning F(R) = (coth R - 1/R) / R.
//
// Small R: the Laurent expansion coth x = 1/x + sum_{n>=1} 2^{2n} B_{2n}
// x^{2n-1} / (2n)! gives F(R) = sum_{n>=1} c_n R^{2n-2}, c_n = 2^{2n} B_{2n} /
// (2n)!, i.e. 1/3, -1/45, 2/945, -1/4725, 2/93555, -1382/638512875,
// 4/18243225, -3617/162820783125.  Eight terms are accurate to < 1e-8 for
// R <= 1 (the first omitted term is ~2.3e-9 R^16).
// Large R: with e = exp(-2R), coth R = 1 + 2e/(1-e), so
// coth R - 1/R = (1 - 1/R) + 2e/(1-e): two non-negative terms for R >= 1,
// free of cancellation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lp_series_f(float R) {
    const float r2 = R * R;
    float a = -3617.0f / 162820783125.0f;
    a = fmaf(a, r2, 4.0f / 18243225.0f);
    a = fmaf(a, r2, -1382.0f / 638512875.0f);
    a = fmaf(a, r2, 2.0f / 93555.0f);
    a = fmaf(a, r2, -1.0f / 4725.0f);
    a = fmaf(a, r2, 2.0f / 945.0f);
    a = fmaf(a, r2, -1.0f / 45.0f);
    a = fmaf(a, r2, 1.0f / 3.0f);
    return a;
}

__device__ __forceinline__ double lp_series_d(double R) {
    const double r2 = R * R;
    double a = -3617.0 / 162820783125.0;
    a = fma(a, r2, 4.0 / 18243225.0);
    a = fma(a, r2, -1382.0 / 638512875.0);
    a = fma(a, r2, 2.0 / 93555.0);
    a = fma(a, r2, -1.0 / 4725.0);
    a = fma(a, r2, 2.0 / 945.0);
    a = fma(a, r2, -1.0 / 45.0);
    a = fma(a, r2, 1.0 / 3.0);
    return a;
}

__device__ __forceinline__ float limiter_f(int kind, float larsen_n, float R) {
    switch (kind) {
    case LIM_CDA: return 1.0f / 3.0f;
    case LIM_SUM: return 1.0f / (3.0f + R);
    case LIM_MAX: return 1.0f / fmaxf(3.0f, R);
    case LIM_KERSHAW: return 2.0f / (3.0f + hypotf(3.0f, 2.0f * R));
    case LIM_LARSEN: {
        // (3^n + R^n)^(-1/n) = 1 / (m (1 + (s/m)^n)^(1/n)), m = max, s = min
        const float m = fmaxf(3.0f, R), s = fminf(3.0f, R);
        return 1.0f / (m * powf(1.0f + powf(s / m, larsen_n), 1.0f / larsen_n));
    }
    default: {  // LIM_LP
        if (R < 1.0f) return lp_series_f(R);
        const float e = expf(-2.0f * R);
        return ((1.0f - 1.0f / R) + 2.0f * e / (1.0f - e)) / R;
    }
    }
}

__device__ __forceinline__ double limiter_d(int kind, double larsen_n, double R) {
    switch (kind) {
    case LIM_CDA: return 1.0 / 3.0;
    case LIM_SUM: return 1.0 / (3.0 + R);
    case LIM_MAX: return 1.0 / fmax(3.0, R);
    case LIM_KERSHAW: return 2.0 / (3.0 + hypot(3.0, 2.0 * R));
    case LIM_LARSEN: {
        const double m = fmax(3.0, R), s = fmin(3.0, R);
        return 1.0 / (m * pow(1.0 + pow(s / m, larsen_n), 1.0 / larsen_n));
    }
    default: {
        // Double precision: the series (8 terms, < 1e-16 relative for
        // R < 0.2) and the cancellation-free large-R form otherwise; the
        // latter loses at most ~60 ulp near R = 0.2.
        if (R < 0.2) return lp_series_d(R);
        const double e = exp(-2.0 * R);
        return ((1.0 - 1.0 / R) + 2.0 * e / (1.0 - e)) / R;
    }
    }
}

// ---------------------------------------------------------------------------
// Float-float (double-single) arithmetic from error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast-TwoSum (Dekker 1971) and TwoProd
// through a fused multiply-add.  A value is hi + lo with |lo| <= ulp(hi)/2.
// Used where the sum of opposing face fluxes cancels (the residual of Eq. 37
// in vacuum): GB300's FP64 rate is a small fraction of its FP32 rate, so the
// accurate sums run on the FP32 pipes instead.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    const float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const ff p = two_prod(a.hi, b);
    const float e = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------------------
// Knudsen number (Eq. 35) and D (Eq. 33) from the central gradient (Eq. 34).
// g_x etc. are the already formed central differences phi(i+1) - phi(i-1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float knudsen_D_f(float gx, float gy, float gz, float inv2h, float sp,
                                             float phi_p, float floor_, int lim, float larsen_n) {
    gx *= inv2h; gy *= inv2h; gz *= inv2h;
    const float g = sqrtf(fmaf(gx, gx, fmaf(gy, gy, gz * gz)));
    const float R = fmaxf(g, floor_) / fmaxf(sp * phi_p, floor_);
    return limiter_f(lim, larsen_n, R) / sp;
}

__device__ __forceinline__ double knudsen_D_d(double gx, double gy, double gz, double inv2h, double sp,
                                              double phi_p, double floor_, int lim, double larsen_n) {
    gx *= inv2h; gy *= inv2h; gz *= inv2h;
    const double g = sqrt(gx * gx + gy * gy + gz * gz);
    const double R = fmax(g, floor_) / fmax(sp * phi_p, floor_);
    return limiter_d(lim, larsen_n, R) / sp;
}

}  // namespace fld
