// fld_device.cuh -- device helpers of the GB300 FLD solver: grid layout,
// flux limiters (Table 2 of Koerner et al. 2014) in single and double
// precision, the floored Knudsen number (Eq. 35) and float-float arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fld {

// ---------------------------------------------------------------------------
// Layout of padded device fields: red-black (colour-split) storage.
//
// Padded coordinates I = i+1, J = j+1, K = k+1 run over [0, n+1] per axis
// (0 and n+1 are the Dirichlet ghost layer).  A cell's colour is
// c = (I + J + K + 1) & 1, so c = 0 ("red") holds the unknowns with i+j+k
// even, which Algorithm 1 updates first.  Each colour has its own array of
// half rows: cell (I, J, K) of colour c lives at
//     c * cs + (K * py + J) * hpx + kXoff + ((I + 1) >> 1).
// In every half row the first unknown (I = 1 or 2) sits at position
// kXoff + 1 = 32, so with hpx a multiple of 32 a warp of 32 consecutive
// unknowns reads one aligned 128-byte line per field.  A colour pass streams
// its own colour for the point's fields and the other colour for the six
// neighbours: the x-neighbours are the adjacent elements (I >> 1) and
// (I >> 1) + 1 of the other colour's row, the y/z-neighbours the same
// position one row/plane away.  All offsets fit in 32 bits (checked at grid
// creation).
// ---------------------------------------------------------------------------
constexpr int kXoff = 31;

struct Layout {
    int nx, ny, nz;     // unknowns per axis
    int hpx;            // half-row pitch (elements), a multiple of 32
    int py;             // rows per plane (ny + 2)
    int cs;             // elements per colour array
    int total;          // elements per padded field (both colours)

    __host__ __device__ __forceinline__ int at(int i, int j, int k) const {
        // i, j, k in [-1, n]: -1 and n are the ghost layer
        const int I = i + 1, J = j + 1, K = k + 1;
        const int c = (I + J + K + 1) & 1;
        return c * cs + (K * py + J) * hpx + kXoff + ((I + 1) >> 1);
    }
    // offset of the half-row (J, K) inside a colour array (incl. kXoff)
    __host__ __device__ __forceinline__ int row(int J, int K) const { return (K * py + J) * hpx + kXoff; }
};

// Largest padded grid whose fields the 32-bit offsets address.
constexpr long long kMaxLayoutElems = 2000000000LL;

inline bool make_layout(int nx, int ny, int nz, Layout *out) {
    Layout L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    L.hpx = (kXoff + (nx + 2) / 2 + 1 + 31) & ~31;
    L.py = ny + 2;
    const long long cs = (long long)L.hpx * L.py * (nz + 2);
    if (2 * cs + 8 > kMaxLayoutElems) return false;
    L.cs = (int)cs;
    L.total = (int)(2 * cs);
    *out = L;
    return true;
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
    case LIM_SUM: return 1.0f / __fadd_rn(3.0f, R);
    case LIM_MAX: return 1.0f / fmaxf(3.0f, R);
    case LIM_KERSHAW: return 2.0f / __fadd_rn(3.0f, hypotf(3.0f, 2.0f * R));
    case LIM_LARSEN: {
        // (3^n + R^n)^(-1/n) = 1 / (m (1 + (s/m)^n)^(1/n)), m = max, s = min
        const float m = fmaxf(3.0f, R), s = fminf(3.0f, R);
        return 1.0f / (m * powf(__fadd_rn(1.0f, powf(s / m, larsen_n)), 1.0f / larsen_n));
    }
    default: {  // LIM_LP
        if (R < 1.0f) return lp_series_f(R);
        // F = r ((1 - r) + 2/(e^{2R} - 1)), r = 1/R; the last term is below
        // 3.4e-8 of the first once R > 9 and is dropped there
        const float r = 1.0f / R;
        const float tail = R < 9.0f ? 2.0f / __fsub_rn(expf(2.0f * R), 1.0f) : 0.0f;
        return r * __fadd_rn(__fsub_rn(1.0f, r), tail);
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

// a * b for float-float a and b (the lo * lo term, ~2^-48 relative, dropped)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const ff p = two_prod(a.hi, b.hi);
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// a / b rounded to single precision (b > 0): the quotient of the high word,
// corrected by the exact remainder (FMA) and the low word.
__device__ __forceinline__ float ff_div_f(ff a, float b) {
    const float q = __fdiv_rn(a.hi, b);
    const float r = __fadd_rn(fmaf(-q, b, a.hi), a.lo);
    return __fadd_rn(q, __fdiv_rn(r, b));
}

// a / b (b.hi > 0) to single precision, likewise.
__device__ __forceinline__ float ff_div(ff a, ff b) {
    const float q = __fdiv_rn(a.hi, b.hi);
    const float r = __fsub_rn(__fadd_rn(fmaf(-q, b.hi, a.hi), a.lo), __fmul_rn(q, b.lo));
    return __fadd_rn(q, __fdiv_rn(r, b.hi));
}

// bfloat16 bit pattern -> float (exact: the pattern is the float's upper half)
__device__ __forceinline__ float bf16_bits_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// ---------------------------------------------------------------------------
// Knudsen number (Eq. 35) and D (Eq. 33) from the central gradient (Eq. 34).
// g_x etc. are the already formed central differences phi(i+1) - phi(i-1).
// The single-precision path is split so a point update can reuse |grad phi|
// across its local rounds; grad_floor_f followed by D_of_f is the one D
// function shared, bit for bit, by the correction sweep and the residual.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float grad_floor_f(float gx, float gy, float gz, float inv2h, float floor_) {
    gx *= inv2h; gy *= inv2h; gz *= inv2h;
    return fmaxf(sqrtf(fmaf(gx, gx, fmaf(gy, gy, gz * gz))), floor_);
}

__device__ __forceinline__ float D_of_f(float gmax, float sp, float phi_p, float floor_, int lim, float larsen_n) {
    const float den = fmaxf(sp * phi_p, floor_);
    if (lim == LIM_LP) {
        // one correctly rounded quotient per branch: R = gmax/den below 1
        // (Laurent series), 1/R = den/gmax above (the exponential term,
        // which needs R itself, only for 1 <= R < 9)
        // (explicit round-to-nearest adds: no contraction into an FMA, so
        // every kernel calling this evaluates it to the same bits)
        float F;
        if (gmax < den) {
            F = lp_series_f(gmax / den);
        } else {
            const float r = den / gmax;
            const float tail = r > (1.0f / 9.0f) ? 2.0f / __fsub_rn(expf(2.0f * (gmax / den)), 1.0f) : 0.0f;
            F = r * __fadd_rn(__fsub_rn(1.0f, r), tail);
        }
        return F / sp;
    }
    return limiter_f(lim, larsen_n, gmax / den) / sp;
}

__device__ __forceinline__ float knudsen_D_f(float gx, float gy, float gz, float inv2h, float sp, float phi_p,
                                             float floor_, int lim, float larsen_n) {
    return D_of_f(grad_floor_f(gx, gy, gz, inv2h, floor_), sp, phi_p, floor_, lim, larsen_n);
}

__device__ __forceinline__ double knudsen_D_d(double gx, double gy, double gz, double inv2h, double sp,
                                              double phi_p, double floor_, int lim, double larsen_n) {
    gx *= inv2h; gy *= inv2h; gz *= inv2h;
    const double g = sqrt(gx * gx + gy * gy + gz * gz);
    const double R = fmax(g, floor_) / fmax(sp * phi_p, floor_);
    return limiter_d(lim, larsen_n, R) / sp;
}

}  // namespace fld
