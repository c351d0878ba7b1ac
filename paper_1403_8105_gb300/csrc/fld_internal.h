// fld_internal.h -- launchers shared by the kernels and the host driver of
// the GB300 FLD solver (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include "fld_device.cuh"

namespace fld {

// Arithmetic of one sweep family: FP32 (phi in float), FH (phi as a hi/lo
// pair, update summed in FP32), FF (phi as a hi/lo pair, update summed in
// float-float with correctly rounded D), FP64.
enum Family : int { FAM_F32 = 0, FAM_FF = 1, FAM_F64 = 2, FAM_FH = 3 };

struct PassParams {
    int lim;
    int local_iters;
    double larsen_n;
    double omega;
    double inv2h;
    double floor_;   // eps * jbar (or the no-emission floor)
    int scheme = 0;  // fld_scheme: red-black SOR or Jacobi
    int bf16 = 0;    // single-precision / hi-lo sweeps read the bfloat16 medium
    double h2 = 0;   // h^2, which scales the bfloat16 sigma_a'
    // temporally blocked configuration (fld_tiled.cu) of the FP32 and hi/lo
    // sweeps; -1: one launch per colour pass
    int tiled_f32 = -1, tiled_fh = -1;
    // launched passes: four unknowns per thread (128-bit loads) instead of two
    int quad_f32 = 0, quad_fh = 0;
};

// Device fields of one grid (padded layout unless noted).
struct Fields {
    // single-precision family
    float *sp = nullptr, *ah2 = nullptr, *jh2 = nullptr;   // sigma', sigma_a' h^2, j h^2
    float *phi = nullptr, *phlo = nullptr, *D = nullptr;   // phi (hi), phi (lo), D
    float *Df = nullptr;                                   // scratch: fresh D for the residual
    // bfloat16 copies of sigma' and sigma_a' (bit patterns; allocated on the
    // first solve with medium_bf16) read by the single-precision and hi/lo
    // sweeps; sp and ah2 then hold the same rounded values
    uint16_t *spb = nullptr, *sab = nullptr;
    // sampling volume of fld_render: sigma_t, sigma_s, source, phi per voxel
    float4 *render_vol = nullptr;
    // second phi buffer of the Jacobi variant (allocated on first use)
    float *phi2 = nullptr;
    double *phi642 = nullptr;
    // double-precision family (allocated on first FP64 use)
    double *sp64 = nullptr, *ah264 = nullptr, *jh264 = nullptr;
    double *phi64 = nullptr, *D64 = nullptr, *Df64 = nullptr;
    // inputs (unpadded, nx*ny*nz floats)
    float *sigma_t = nullptr, *albedo = nullptr, *jsrc = nullptr;
    // reduction scratch
    double *partials = nullptr;   // 2 doubles per block
    double *result = nullptr;     // 2 doubles
    int partial_cap = 0;          // blocks the partials buffer holds
};

// Medium preparation (Algorithm 1: sigma floor; sigma_a', j scaled by h^2).
// bf16: round sigma' and sigma_a' to bfloat16 (formed in single precision)
// and write the bfloat16 copies too (launch_prep_f).
cudaError_t launch_prep_f(const Layout &L, const Fields &f, float sigma_eps, float h2, bool bf16, cudaStream_t s);
cudaError_t launch_prep_d(const Layout &L, const Fields &f, double sigma_eps, double h2, bool bf16,
                          cudaStream_t s);

// One Jacobi iteration: D^k from phi^k at every unknown, then phi^{k+1} from
// phi^k and D^k; to_second = 1 reads phi and writes the second buffer, 0 the
// reverse.  The destination's ghosts must already hold the ghost values.
cudaError_t launch_jacobi(Family fam, const Layout &L, const Fields &f, const PassParams &p, int to_second,
                          cudaStream_t s);

// Primary ray march (fld_render.cu).  The camera basis is formed on the host
// (f forward, r right, u up, unit vectors; tan_half = tan(fov/2)).
struct RenderCamera {
    double eye[3], f[3], r[3], u[3];
    double tan_half, aspect, h;
    int width, height;
    double step, background, t_min;
};
// Where the renderer takes phi from: phi (+ phlo) or phi64 of the rendered
// grid's own layout, or (coarse) of a coarser grid with layout C and spacing
// hc, upsampled trilinearly to the rendered grid's voxel centres.
struct PhiSource {
    const float *phi = nullptr, *phlo = nullptr;
    const double *phi64 = nullptr;
    bool coarse = false;
    Layout C{};
    double hc = 0.0;
};
// Packs sigma_t, albedo sigma_t, the source and phi into vol (one float4 per
// voxel), then renders; radiance (width*height floats) and codes (8-bit
// gamma-compressed) may each be null.
cudaError_t launch_render(const Layout &L, const Fields &f, const PhiSource &ps, const RenderCamera &c,
                          float4 *vol, float *radiance, uint8_t *codes, double exposure, double gamma,
                          cudaStream_t s);
// phi (hi word; low word 0) at the unknowns of L from a coarser grid's phi,
// blended trilinearly between its voxel centres (ps.coarse must be true).
cudaError_t launch_prolong(const Layout &L, Fields &f, const PhiSource &ps, double h, cudaStream_t s);
// D from the current single-precision phi at every unknown (Eq. 33-35), into f.D.
cudaError_t launch_fresh_D_into(const Layout &L, Fields &f, const PassParams &p, cudaStream_t s);

// Box averages of the fine grid's sigma_t, albedo (sigma_s-weighted) and
// source over factor^3 blocks into the coarse grid's input arrays.
cudaError_t launch_downsample(const Layout &L, const Fields &f, int factor, const Layout &C, Fields &fc,
                              cudaStream_t s);

// phi = phi0 / D = D0 on the unknowns, phi_b / D_b on the ghosts, 0 elsewhere.
cudaError_t launch_init_f(const Layout &L, float *phi, float *phlo, float *D, double phi0, double D0,
                          double phi_b, double D_b, cudaStream_t s);
cudaError_t launch_init_d(const Layout &L, double *phi, double *D, double phi0, double D0, double phi_b,
                          double D_b, cudaStream_t s);

// Conversions between the packed (nx+2)(ny+2)(nz+2) double layout and the
// device fields.  dst_lo may be null (single float); src_lo likewise.
cudaError_t launch_unpack_to_f(const Layout &L, const double *src, float *dst_hi, float *dst_lo, cudaStream_t s);
cudaError_t launch_unpack_to_d(const Layout &L, const double *src, double *dst, cudaStream_t s);
cudaError_t launch_pack_from_f(const Layout &L, const float *hi, const float *lo, double *dst, cudaStream_t s);
cudaError_t launch_pack_from_d(const Layout &L, const double *src, double *dst, cudaStream_t s);
// Between families (float-float <-> double) in the device layout.
cudaError_t launch_f_to_d(const Layout &L, const float *hi, const float *lo, double *dst, cudaStream_t s);
cudaError_t launch_d_to_f(const Layout &L, const double *src, float *hi, float *lo, cudaStream_t s);

// One colour pass of Algorithm 1 (colour 0 = red: i+j+k even).
cudaError_t launch_pass(Family fam, const Layout &L, const Fields &f, const PassParams &p, int colour,
                        cudaStream_t s);

// Residual of Eq. 37 with fresh D: writes sum(R h^2)^2 over the margin set
// to result[0] and sum (j h^2)^2 over all unknowns to result[1].
cudaError_t launch_residual(Family fam, const Layout &L, const Fields &f, const PassParams &p, int margin,
                            cudaStream_t s);

// sum j^2 over the unknowns of the unpadded source -> result[0].
cudaError_t launch_sumsq_source(const Layout &L, const Fields &f, cudaStream_t s);

// Blocks the residual / reduction launches use (sizes the partials buffer).
int reduction_blocks(const Layout &L);

// Single-scatter source.
cudaError_t launch_bake_scan_negz(const Layout &L, const Fields &f, float h, float radiance, int accumulate,
                                  cudaStream_t s);
cudaError_t launch_bake_march(const Layout &L, const Fields &f, float h, const double w[3], const double pos[3],
                              int point, float value, float step, int accumulate, cudaStream_t s);

// Validation of n input values (any pointer may be null): result[0] counts
// NaN / negative / infinite sigma_t and j, result[1] albedo outside [0, 1].
cudaError_t launch_validate(long long n, const Fields &f, const float *sigma_t, const float *albedo,
                            const float *j, cudaStream_t s);

// One grid of a batched solve, read by the batched residual kernels at run
// time (so grids can converge or change phase between checks).
struct alignas(16) BatchDesc {
    Layout L;
    float *sp, *ah2, *jh2, *phi, *phlo, *D, *Df;
    float inv2h, floor_, larsen_n;
    int lim;
    int mode;            // 0: single-precision sweeps, 1: float-float correction sweeps
    int active;          // 0: converged / stopped, its CTAs return at once
    int res_first, res_bx, res_by;      // first CTA of this grid in the residual table, grid dims
    int res_slot;                       // first partial-sum slot of this grid
};
static_assert(sizeof(BatchDesc) % 16 == 0, "BatchDesc is read with 16-byte loads");

// One grid of a multi-grid colour pass (launch_pass_multi): its layout,
// fields and pass parameters, and where its work items start.  An item is
// the 32 x 8 pairs of unknowns a CTA of the solo pair pass covers (one
// z-plane); the grid's items are numbered x fastest, then y, then z.
struct alignas(16) SweepDesc {
    Layout L;
    float *sp, *ah2, *jh2, *phi, *phlo, *D;
    const uint16_t *spb, *sab;        // bfloat16 medium, or null
    float h2, omega, inv2h, floor_, larsen_n;
    int lim, local_iters;
    int hl;                           // 0: FP32 sweeps, 1: hi/lo sweeps
    int first;                        // first item of this grid
    int bx, by;                       // items per plane in x and y
    int pad_;
};
static_assert(sizeof(SweepDesc) % 16 == 0, "SweepDesc is read with 16-byte loads");

// Grids one multi-grid table holds.
constexpr int kMultiMaxGrids = 128;
// Item grid of a layout for the multi-grid pass (the solo pair pass's CTAs).
void multi_dims(const Layout &L, int *bx, int *by);
// One colour pass of every grid in descs[0 .. counts[0]) (counts[1] items in
// all), all of family hl (0: FP32, 1: hi/lo) with medium bf16, limiter lim
// and local_iters rounds, each with its own omega and state: a persistent
// grid of nctas CTAs walks the items.  Both counts are read on the device, so
// a captured graph of these launches serves any table contents.
cudaError_t launch_pass_multi(const SweepDesc *descs, const int *counts, int hl, int bf16, int lim, int local_iters,
                              int colour, int nctas, cudaStream_t s);
// CTAs of that persistent pass resident at once on a device of nsm SMs.
int multi_ctas(int nsm, int hl, int bf16, int lim, int local_iters);

// Batched residual: per grid g, result[2g] = sum (R h^2)^2, result[2g+1] = sum (j h^2)^2,
// summed in the same order as launch_residual.
cudaError_t launch_residual_batch(const BatchDesc *descs, const int *cta_grid, int nctas, int ngrids,
                                  const int *res_count, double *partials, double *result, int lim, int margin,
                                  cudaStream_t s);
// Pass / residual grid dimensions of a layout (CTAs = x * y * nz).
void residual_dims(const Layout &L, int *bx, int *by);

// Anderson mixing of blocks of sweeps (fld_anderson.cu): m history slots of
// g (float-float) and f (FP32) per element of the padded field, the current
// start point x (float-float), per-CTA partial dot products and their m sums.
constexpr int kAndersonMax = 16;
struct AndersonBuffers {
    float2 *g = nullptr;      // m * total float-float images
    float *f = nullptr;       // m * total
    float2 *x = nullptr;      // total: the current start point (float-float)
    double *part = nullptr;   // (4 * SMs) * kAndersonMax
    double *dots = nullptr;   // kAndersonMax
};
// x = the current state (hi + lo, hi alone when lo is null, or p64).
cudaError_t launch_anderson_capture(const AndersonBuffers &b, int n, const float *hi, const float *lo,
                                    const double *p64, int nsm, cudaStream_t s);
// g -> slot, f = g - x -> slot, dots[j] = <f, f_j> for the w occupied slots.
cudaError_t launch_anderson_collect(const AndersonBuffers &b, int n, const float *hi, const float *lo,
                                    const double *p64, int slot, int w, int nsm, cudaStream_t s);
// state = x = g_slot + sum_{j != slot} a_j (g_j - g_slot).
cudaError_t launch_anderson_mix(const AndersonBuffers &b, int n, int slot, int w, const double *a, float *hi,
                                float *lo, double *p64, int nsm, cudaStream_t s);

// Temporally blocked red-black sweeps (fld_tiled.cu).  Configuration ids
// 0..kTiledConfigs-1 fix the temporal depth T (iterations per launch) and the
// x-y tile; tiled_config_of(T, TY) finds one (TY <= 0: the first with that T).
constexpr int kTiledConfigs = 3;
struct TiledMaps {
    CUtensorMap phi, D, lo;    // TMA descriptors of the launch's input buffers
};
int tiled_depth(int id);
void tiled_shape(int id, int *T, int *tx, int *ty);
int tiled_config_of(int T, int TY);
// Set up the kernel instance of (fam, id, p) (shared-memory attribute,
// occupancy); call outside stream capture before launching it.
cudaError_t tiled_prepare(Family fam, int id, const PassParams &p);
// Tensor maps of one buffer set (lo may be null) for configuration id.
cudaError_t tiled_maps(const Layout &L, int id, float *phi, float *D, float *lo, TiledMaps *out);
// T iterations (FAM_F32 or FAM_FH) from the buffers described by src into
// dphi / dD / dlo, whose ghosts must already hold the ghost values.  *status
// is set to 1 if a bounded wait gave up.
cudaError_t launch_tiled(Family fam, int id, const Layout &L, const Fields &f, const PassParams &p,
                         const TiledMaps &src, float *dphi, float *dD, float *dlo, int *status, int nsm,
                         cudaStream_t s);

// Relative residual Rbar / jbar of Eq. 37 from the device sums r2 = sum of
// (R_p h^2)^2 over the unknowns at least `margin` voxels from the faces and
// j2 = sum of (j_p h^2)^2 over all unknowns (both RMS, so rel = ||R|| / ||j||
// over their sets); with no emission at all the absolute RMS residual.  Shared
// by every entry point that reports a residual.
inline double rel_residual_from_sums(int nx, int ny, int nz, double h, int margin, double r2, double j2) {
    const long long ex = nx - 2LL * margin, ey = ny - 2LL * margin, ez = nz - 2LL * margin;
    const long long cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    const double rbar_h2 = cnt > 0 ? sqrt(r2 / (double)cnt) : 0.0;
    const double jbar_h2 = sqrt(j2 / ((double)nx * ny * nz));
    return jbar_h2 > 0.0 ? rbar_h2 / jbar_h2 : rbar_h2 / (h * h);
}

// Checks of the limiter (Table 2 or CDA), Larsen's n and the residual margin
// shared by the entry points: null if valid, else the message.
inline const char *check_limiter_margin(int limiter, double larsen_n, int margin) {
    if (limiter < LIM_CDA || limiter > LIM_LP) return "unknown limiter";
    if (limiter == LIM_LARSEN && !(larsen_n > 0.0)) return "larsen_n must be > 0";
    if (margin < 0) return "residual_margin must be >= 0";
    return nullptr;
}

// Sets the thread-local text that fld_last_error() returns.
void set_error_text(const char *msg);

}  // namespace fld
