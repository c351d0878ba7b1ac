// fld_capi.cu -- host side of the GB300 FLD solver: the grid object, the
// solve loop of Algorithm 1 (Koerner et al. 2014) and the C ABI of fld.h.
//
// Each block of `check_every` red-black iterations is captured once into a
// CUDA graph and replayed, so the host issues one launch per block instead
// of two per iteration; the only device-to-host traffic of a solve is the
// 16-byte residual pair read after each block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "../../include/fld.h"
#include "fld_device.cuh"
#include "fld_internal.h"

using namespace fld;

namespace {

thread_local std::string g_last_error;

fld_status fail(fld_status s, const char *what) {
    g_last_error = what ? what : "";
    return s;
}

fld_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return FLD_ERR_CUDA;
}

#define FLD_CK(call)                                      \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr double kFloorNoEmission = 1e-30;   // floor of Eq. 35 when jbar = 0
constexpr int kStallChecks = 48;              // checks without a new minimum before giving up
constexpr int kSwitchChecks = 24;             // ... before single precision hands over (MIXED)
constexpr double kGuardGrowth = 1e3;          // residual growth (vs the best) read as divergence
constexpr int kMaxBackoffs = 8;               // omega reductions before reporting divergence
constexpr double kOmegaMax = 1.93;            // upper clamp of the automatic omega

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int fam = -1;
    int iters = 0;
    PassParams p{};
};

bool same_params(const PassParams &a, const PassParams &b) {
    return a.lim == b.lim && a.local_iters == b.local_iters && a.larsen_n == b.larsen_n && a.omega == b.omega &&
           a.inv2h == b.inv2h && a.floor_ == b.floor_;
}

}  // namespace

void fld::set_error_text(const char *msg) { g_last_error = msg ? msg : ""; }

struct fld_grid_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nx = 0, ny = 0, nz = 0;
    double h = 0.0;
    Layout L{};
    Fields f{};
    bool has_medium = false;
    long long version = 1;          // bumps when medium or source change
    long long prepared_f = 0, prepared_d = 0;
    double prepared_seps_f = -1.0, prepared_seps_d = -1.0;
    double jbar = 0.0;
    long long jbar_version = 0;
    bool valid_float = false, valid_d = false;   // which family holds the state
    bool lo_live = false;                        // phlo may be non-zero
    GraphEntry graphs[3];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evb0 = nullptr, evb1 = nullptr;
    long long kernels = 0;                       // kernel launches issued so far
    // last good state of a solve (float family: phi, lo, D; FP64: phi, D)
    float *snap_phi = nullptr, *snap_lo = nullptr, *snap_D = nullptr;
    double *snap_phi64 = nullptr, *snap_D64 = nullptr;
};

namespace {

long long nvox(const fld_grid_s *g) { return (long long)g->nx * g->ny * g->nz; }

fld_status ensure_f64(fld_grid_s *g) {
    if (g->f.phi64) return FLD_OK;
    const size_t bytes = sizeof(double) * (size_t)g->L.total;
    double **ptrs[6] = {&g->f.sp64, &g->f.ah264, &g->f.jh264, &g->f.phi64, &g->f.D64, &g->f.Df64};
    for (double **p : ptrs) {
        cudaError_t e = cudaMalloc((void **)p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FLD_ERR_OOM, "cudaMalloc of the FP64 fields failed");
        }
        FLD_CK(cudaMemsetAsync(*p, 0, bytes, g->stream));
    }
    return FLD_OK;
}

// sigma_eps = 1e-3 / L with L the largest grid extent (Sec. 5), unless given.
double sigma_eps_of(const fld_grid_s *g, const fld_solve_params *p) {
    if (p->sigma_eps > 0.0) return p->sigma_eps;
    int n = g->nx;
    if (g->ny > n) n = g->ny;
    if (g->nz > n) n = g->nz;
    return 1e-3 / ((double)n * g->h);
}

double omega_of(const fld_grid_s *g, const fld_solve_params *p) {
    if (p->omega > 0.0) return p->omega;
    int n = g->nx;
    if (g->ny > n) n = g->ny;
    if (g->nz > n) n = g->nz;
    double w = 2.0 / (1.0 + sin(M_PI / (n + 1.0)));
    if (w < 1.0) w = 1.0;
    if (w > kOmegaMax) w = kOmegaMax;
    return w;
}

fld_status read_result(fld_grid_s *g, double out[2]) {
    FLD_CK(cudaMemcpyAsync(out, g->f.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    FLD_CK(cudaStreamSynchronize(g->stream));
    return FLD_OK;
}

// jbar = RMS of the source over the unknowns (Algorithm 1).
fld_status update_jbar(fld_grid_s *g) {
    if (g->jbar_version == g->version) return FLD_OK;
    FLD_CK(launch_sumsq_source(g->L, g->f, g->stream));
    g->kernels += 2;
    double r[2];
    fld_status st = read_result(g, r);
    if (st != FLD_OK) return st;
    g->jbar = sqrt(r[0] / (double)nvox(g));
    g->jbar_version = g->version;
    return FLD_OK;
}

fld_status prepare(fld_grid_s *g, const fld_solve_params *p, Family fam) {
    if (!g->has_medium) return fail(FLD_ERR_STATE, "fld_set_medium has not been called");
    fld_status st = update_jbar(g);
    if (st != FLD_OK) return st;
    const double seps = sigma_eps_of(g, p);
    const double h2 = g->h * g->h;
    if (fam == FAM_F64) {
        st = ensure_f64(g);
        if (st != FLD_OK) return st;
        if (g->prepared_d != g->version || g->prepared_seps_d != seps) {
            FLD_CK(launch_prep_d(g->L, g->f, seps, h2, g->stream));
            g->kernels += 1;
            g->prepared_d = g->version;
            g->prepared_seps_d = seps;
        }
    } else {
        if (g->prepared_f != g->version || g->prepared_seps_f != seps) {
            FLD_CK(launch_prep_f(g->L, g->f, (float)seps, (float)h2, g->stream));
            g->kernels += 1;
            g->prepared_f = g->version;
            g->prepared_seps_f = seps;
        }
    }
    return FLD_OK;
}

PassParams pass_params(const fld_grid_s *g, const fld_solve_params *p) {
    PassParams q;
    q.lim = p->limiter;
    q.local_iters = p->local_iters < 1 ? 1 : p->local_iters;
    q.larsen_n = p->larsen_n;
    q.omega = omega_of(g, p);
    q.inv2h = 1.0 / (2.0 * g->h);
    const double eps = p->eps > 0.0 ? p->eps : 1e-20;
    q.floor_ = g->jbar > 0.0 ? eps * g->jbar : kFloorNoEmission;
    return q;
}

// Algorithm 1 initialisation (or the caller's values) of the family's fields.
fld_status init_state(fld_grid_s *g, const fld_solve_params *p, Family fam) {
    const double eps = p->eps > 0.0 ? p->eps : 1e-20;
    const double phi_def = eps * g->jbar * g->h, D_def = eps * g->h;
    const double phi0 = p->phi0 >= 0.0 ? p->phi0 : phi_def;
    const double D0 = p->D0 >= 0.0 ? p->D0 : D_def;
    const double phi_b = p->phi_b >= 0.0 ? p->phi_b : phi_def;
    const double D_b = p->D_b >= 0.0 ? p->D_b : D_def;
    if (fam == FAM_F64) {
        FLD_CK(launch_init_d(g->L, g->f.phi64, g->f.D64, phi0, D0, phi_b, D_b, g->stream));
        g->kernels += 1;
        g->valid_d = true;
        g->valid_float = false;
    } else {
        FLD_CK(launch_init_f(g->L, g->f.phi, g->f.phlo, g->f.D, phi0, D0, phi_b, D_b, g->stream));
        g->kernels += 1;
        g->valid_float = true;
        g->valid_d = false;
        g->lo_live = false;
    }
    return FLD_OK;
}

// Make the family's fields hold the current state.
fld_status sync_family(fld_grid_s *g, Family fam) {
    if (fam == FAM_F64) {
        fld_status st = ensure_f64(g);
        if (st != FLD_OK) return st;
        if (!g->valid_d) {
            if (!g->valid_float) return fail(FLD_ERR_STATE, "no state to continue from");
            FLD_CK(launch_f_to_d(g->L, g->f.phi, g->lo_live ? g->f.phlo : nullptr, g->f.phi64, g->stream));
            FLD_CK(launch_f_to_d(g->L, g->f.D, nullptr, g->f.D64, g->stream));
            g->kernels += 2;
            g->valid_d = true;
        }
        g->valid_float = false;
    } else {
        if (!g->valid_float) {
            if (!g->valid_d) return fail(FLD_ERR_STATE, "no state to continue from");
            FLD_CK(launch_d_to_f(g->L, g->f.phi64, g->f.phi, g->f.phlo, g->stream));
            FLD_CK(launch_d_to_f(g->L, g->f.D64, g->f.D, nullptr, g->stream));
            g->kernels += 2;
            g->valid_float = true;
            g->lo_live = true;
        }
        if (fam == FAM_F32 && g->lo_live) {
            // single-precision sweeps carry no low word: round the state to float
            FLD_CK(cudaMemsetAsync(g->f.phlo, 0, sizeof(float) * (size_t)g->L.total, g->stream));
            g->lo_live = false;
        }
        if (fam == FAM_FF) g->lo_live = true;
        g->valid_d = false;
    }
    return FLD_OK;
}

fld_status enqueue_iterations(fld_grid_s *g, Family fam, const PassParams &pp, int iters) {
    for (int it = 0; it < iters; ++it)
        for (int colour = 0; colour < 2; ++colour) FLD_CK(launch_pass(fam, g->L, g->f, pp, colour, g->stream));
    return FLD_OK;
}

// Replay (capturing on first use) a graph of `iters` iterations.
fld_status run_block(fld_grid_s *g, Family fam, const PassParams &pp, int iters) {
    GraphEntry &e = g->graphs[fam];
    if (!(e.exec && e.iters == iters && same_params(e.p, pp))) {
        if (e.exec) {
            cudaGraphExecDestroy(e.exec);
            e.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        FLD_CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        fld_status st = enqueue_iterations(g, fam, pp, iters);
        cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
        if (st != FLD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            e.exec = nullptr;
            return cuda_fail(ce, "cudaGraphInstantiate");
        }
        e.fam = fam;
        e.iters = iters;
        e.p = pp;
    }
    FLD_CK(cudaGraphLaunch(e.exec, g->stream));
    g->kernels += 2LL * iters;
    return FLD_OK;
}

fld_status residual_now(fld_grid_s *g, Family fam, const PassParams &pp, int margin, double *rel) {
    FLD_CK(launch_residual(fam, g->L, g->f, pp, margin, g->stream));
    g->kernels += 3;
    double r[2];
    fld_status st = read_result(g, r);
    if (st != FLD_OK) return st;
    long long ex = g->nx - 2LL * margin, ey = g->ny - 2LL * margin, ez = g->nz - 2LL * margin;
    const long long cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    // r[0] = sum (R_p h^2)^2 over the margin set, r[1] = sum (j_p h^2)^2
    const double rbar_h2 = cnt > 0 ? sqrt(r[0] / (double)cnt) : 0.0;
    const double jbar_h2 = sqrt(r[1] / (double)nvox(g));
    *rel = jbar_h2 > 0.0 ? rbar_h2 / jbar_h2 : rbar_h2 / (g->h * g->h);
    return FLD_OK;
}

fld_status check_params(const fld_grid_s *g, const fld_solve_params *p) {
    if (!p) return fail(FLD_ERR_INVALID_ARG, "params is NULL");
    if (p->limiter < FLD_LIM_CDA || p->limiter > FLD_LIM_LP) return fail(FLD_ERR_INVALID_ARG, "unknown limiter");
    if (p->limiter == FLD_LIM_LARSEN && !(p->larsen_n > 0.0)) return fail(FLD_ERR_INVALID_ARG, "larsen_n must be > 0");
    if (p->omega > 0.0 && !(p->omega < 2.0)) return fail(FLD_ERR_INVALID_ARG, "omega must lie in (0, 2)");
    if (p->precision < FLD_PREC_FP64 || p->precision > FLD_PREC_MIXED)
        return fail(FLD_ERR_INVALID_ARG, "unknown precision");
    if (p->local_iters > 64) return fail(FLD_ERR_INVALID_ARG, "local_iters must be <= 64");
    if (p->residual_margin < 0) return fail(FLD_ERR_INVALID_ARG, "residual_margin must be >= 0");
    (void)g;
    return FLD_OK;
}

fld_grid_s *as_grid(fld_grid g) { return g; }

fld_status enter(fld_grid g) {
    if (!g) return fail(FLD_ERR_INVALID_ARG, "grid is NULL");
    FLD_CK(cudaSetDevice(g->device));
    return FLD_OK;
}

// Copy n floats from host or device memory into a device buffer.
fld_status copy_in(fld_grid_s *g, float *dst, const float *src, long long n, int where) {
    const cudaMemcpyKind kind = where == FLD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    FLD_CK(cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)n, kind, g->stream));
    return FLD_OK;
}

fld_status validate_inputs(fld_grid_s *g, const float *st, const float *alb, const float *js) {
    FLD_CK(launch_validate(nvox(g), g->f, st, alb, js, g->stream));
    double r[2];
    fld_status s = read_result(g, r);
    if (s != FLD_OK) return s;
    if (r[0] > 0.0) return fail(FLD_ERR_INVALID_ARG, "sigma_t or j has NaN, infinite or negative values");
    if (r[1] > 0.0) return fail(FLD_ERR_INVALID_ARG, "albedo has values outside [0, 1] or NaN");
    return FLD_OK;
}

// Copy the family's state into (save) or out of (restore) the snapshot.
fld_status snapshot(fld_grid_s *g, Family fam, bool save) {
    const size_t nf = sizeof(float) * (size_t)g->L.total, nd = sizeof(double) * (size_t)g->L.total;
    if (fam == FAM_F64) {
        if (!g->snap_phi64) {
            if (cudaMalloc((void **)&g->snap_phi64, nd) != cudaSuccess ||
                cudaMalloc((void **)&g->snap_D64, nd) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(FLD_ERR_OOM, "cudaMalloc of the solve snapshot failed");
            }
        }
        double *a[2] = {g->f.phi64, g->f.D64}, *b[2] = {g->snap_phi64, g->snap_D64};
        for (int i = 0; i < 2; ++i)
            FLD_CK(cudaMemcpyAsync(save ? b[i] : a[i], save ? a[i] : b[i], nd, cudaMemcpyDeviceToDevice, g->stream));
    } else {
        if (!g->snap_phi) {
            if (cudaMalloc((void **)&g->snap_phi, nf) != cudaSuccess ||
                cudaMalloc((void **)&g->snap_lo, nf) != cudaSuccess ||
                cudaMalloc((void **)&g->snap_D, nf) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(FLD_ERR_OOM, "cudaMalloc of the solve snapshot failed");
            }
        }
        float *a[3] = {g->f.phi, g->f.phlo, g->f.D}, *b[3] = {g->snap_phi, g->snap_lo, g->snap_D};
        for (int i = 0; i < 3; ++i)
            FLD_CK(cudaMemcpyAsync(save ? b[i] : a[i], save ? a[i] : b[i], nf, cudaMemcpyDeviceToDevice, g->stream));
    }
    return FLD_OK;
}

// Decisions of one solve after each residual check (shared by fld_solve and
// fld_solve_batch, so a grid takes the same path alone and in a batch).
enum Action { ACT_CONTINUE, ACT_SAVE, ACT_RESTORE, ACT_SWITCH, ACT_CONVERGED, ACT_DIVERGED, ACT_STALLED };

struct Controller {
    int precision = FLD_PREC_MIXED;
    double tol = 1e-6, sw = 2e-5;
    Family fam = FAM_F32;
    double best = INFINITY;   // best residual after at least one block
    int since_best = 0;       // checks without a new minimum
    int backoffs = 0;

    void begin_phase() { since_best = 0; }
    // First check (before any iteration): the state is kept as the fallback of
    // the safeguard, but progress is measured from the first block onwards
    // (SOR's early transient may sit above the initial residual for a while).
    Action first(double rel) const {
        if (rel <= tol) return ACT_CONVERGED;
        if (!isfinite(rel)) return ACT_DIVERGED;
        return ACT_SAVE;
    }
    // After a block of iterations.
    Action next(double rel, double omega) {
        const bool diverging = !isfinite(rel) || rel > kGuardGrowth * best || (since_best >= 16 && rel > 2.0 * best);
        if (diverging) {
            if (backoffs >= kMaxBackoffs || omega <= 1.0) return ACT_DIVERGED;
            ++backoffs;
            since_best = 0;
            return ACT_RESTORE;
        }
        if (rel <= tol) return ACT_CONVERGED;
        Action a = ACT_CONTINUE;
        if (rel < best) {
            best = rel;
            since_best = 0;
            a = ACT_SAVE;
        } else {
            ++since_best;
        }
        // single precision has done what it can (Sec. 6.2: ~1e-4 is its limit)
        if (precision == FLD_PREC_MIXED && fam == FAM_F32 && (rel <= sw || since_best >= kSwitchChecks))
            return ACT_SWITCH;
        // The float-float and FP64 sweeps reach residuals near 1e-7; stalling
        // far above the tolerance there means over-relaxation is cycling, not
        // that the arithmetic is exhausted: back off omega.
        if (fam != FAM_F32 && tol > 0.0 && since_best >= kSwitchChecks && best > 100.0 * tol) {
            if (backoffs >= kMaxBackoffs || omega <= 1.0) return ACT_STALLED;
            ++backoffs;
            since_best = 0;
            return ACT_RESTORE;
        }
        if (since_best >= kStallChecks && !(precision == FLD_PREC_MIXED && fam == FAM_F32)) return ACT_STALLED;
        return a;
    }
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fld_default_params(fld_solve_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->limiter = FLD_LIM_LP;
    p->larsen_n = 2.0;
    p->omega = 0.0;
    p->local_iters = 2;
    p->tol = 1e-6;
    p->max_iters = 1000000;
    p->check_every = 64;
    p->sigma_eps = 0.0;
    p->eps = 0.0;
    p->precision = FLD_PREC_MIXED;
    p->fp32_switch = 0.0;
    p->residual_margin = 0;
    p->warm_start = 0;
    p->phi0 = -1.0;
    p->D0 = -1.0;
    p->phi_b = -1.0;
    p->D_b = -1.0;
}

const char *fld_status_string(fld_status s) {
    switch (s) {
    case FLD_OK: return "FLD_OK";
    case FLD_ERR_INVALID_ARG: return "FLD_ERR_INVALID_ARG";
    case FLD_ERR_OOM: return "FLD_ERR_OOM";
    case FLD_ERR_CUDA: return "FLD_ERR_CUDA";
    case FLD_ERR_STATE: return "FLD_ERR_STATE";
    case FLD_ERR_NOT_CONVERGED: return "FLD_ERR_NOT_CONVERGED";
    case FLD_ERR_DIVERGED: return "FLD_ERR_DIVERGED";
    case FLD_ERR_NO_DEVICE: return "FLD_ERR_NO_DEVICE";
    }
    return "FLD_ERR_UNKNOWN";
}

const char *fld_last_error(void) { return g_last_error.c_str(); }

fld_status fld_create_grid(int nx, int ny, int nz, double h, void *stream, fld_grid *out) {
    if (!out) return fail(FLD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(FLD_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (!(h > 0.0) || !isfinite(h)) return fail(FLD_ERR_INVALID_ARG, "h must be a positive finite number");
    if ((long long)(nx + 2) * (ny + 2) * (nz + 2) > (1LL << 40))
        return fail(FLD_ERR_INVALID_ARG, "grid too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        (void)cudaGetLastError();
        return fail(FLD_ERR_NO_DEVICE, "no CUDA device available");
    }
    fld_grid_s *g = new (std::nothrow) fld_grid_s();
    if (!g) return fail(FLD_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaGetDevice");
    }
    g->nx = nx; g->ny = ny; g->nz = nz; g->h = h;
    if (!make_layout(nx, ny, nz, &g->L)) {
        delete g;
        return fail(FLD_ERR_INVALID_ARG, "grid too large: a padded field must stay below 2e9 elements");
    }
    if (stream) {
        g->stream = (cudaStream_t)stream;
    } else {
        // a blocking stream: ordered with work on the legacy default stream
        e = cudaStreamCreate(&g->stream);
        if (e != cudaSuccess) {
            delete g;
            return cuda_fail(e, "cudaStreamCreate");
        }
        g->own_stream = true;
    }
    const size_t fb = sizeof(float) * (size_t)g->L.total;
    const size_t ub = sizeof(float) * (size_t)nvox(g);
    float **pf[7] = {&g->f.sp, &g->f.ah2, &g->f.jh2, &g->f.phi, &g->f.phlo, &g->f.D, &g->f.Df};
    float **pu[3] = {&g->f.sigma_t, &g->f.albedo, &g->f.jsrc};
    fld_status st = FLD_OK;
    for (float **p : pf)
        if (st == FLD_OK && cudaMalloc((void **)p, fb) != cudaSuccess) st = FLD_ERR_OOM;
    for (float **p : pu)
        if (st == FLD_OK && cudaMalloc((void **)p, ub) != cudaSuccess) st = FLD_ERR_OOM;
    g->f.partial_cap = reduction_blocks(g->L);
    if (st == FLD_OK && cudaMalloc((void **)&g->f.partials, sizeof(double) * 2 * (size_t)g->f.partial_cap) != cudaSuccess)
        st = FLD_ERR_OOM;
    if (st == FLD_OK && cudaMalloc((void **)&g->f.result, sizeof(double) * 2) != cudaSuccess) st = FLD_ERR_OOM;
    if (st == FLD_OK && (cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess ||
                         cudaEventCreate(&g->evb0) != cudaSuccess || cudaEventCreate(&g->evb1) != cudaSuccess))
        st = FLD_ERR_CUDA;
    if (st == FLD_OK) {
        for (float **p : pf)
            if (cudaMemsetAsync(*p, 0, fb, g->stream) != cudaSuccess) st = FLD_ERR_CUDA;
        for (float **p : pu)
            if (cudaMemsetAsync(*p, 0, ub, g->stream) != cudaSuccess) st = FLD_ERR_CUDA;
    }
    if (st != FLD_OK) {
        (void)cudaGetLastError();
        fld_destroy(g);
        return fail(st, st == FLD_ERR_OOM ? "cudaMalloc failed while creating the grid" : "CUDA setup failed");
    }
    *out = g;
    return FLD_OK;
}

void fld_destroy(fld_grid g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (GraphEntry &e : g->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    void *ptrs[] = {g->f.sp, g->f.ah2, g->f.jh2, g->f.phi, g->f.phlo, g->f.D, g->f.Df, g->f.sp64, g->f.ah264,
                    g->f.jh264, g->f.phi64, g->f.D64, g->f.Df64, g->f.sigma_t, g->f.albedo, g->f.jsrc,
                    g->f.partials, g->f.result};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->evb0) cudaEventDestroy(g->evb0);
    if (g->evb1) cudaEventDestroy(g->evb1);
    void *snaps[] = {g->snap_phi, g->snap_lo, g->snap_D, g->snap_phi64, g->snap_D64};
    for (void *p : snaps)
        if (p) cudaFree(p);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

fld_status fld_set_medium(fld_grid g, const float *sigma_t, const float *albedo, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!sigma_t || !albedo) return fail(FLD_ERR_INVALID_ARG, "sigma_t and albedo must not be NULL");
    if (where != FLD_MEM_HOST && where != FLD_MEM_DEVICE) return fail(FLD_ERR_INVALID_ARG, "bad memory kind");
    g->has_medium = false;
    if ((st = copy_in(g, g->f.sigma_t, sigma_t, nvox(g), where)) != FLD_OK) return st;
    if ((st = copy_in(g, g->f.albedo, albedo, nvox(g), where)) != FLD_OK) return st;
    if ((st = validate_inputs(g, g->f.sigma_t, g->f.albedo, nullptr)) != FLD_OK) return st;
    g->has_medium = true;
    ++g->version;
    return FLD_OK;
}

fld_status fld_set_source(fld_grid g, const float *j, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!j) return fail(FLD_ERR_INVALID_ARG, "j must not be NULL");
    if (where != FLD_MEM_HOST && where != FLD_MEM_DEVICE) return fail(FLD_ERR_INVALID_ARG, "bad memory kind");
    if ((st = copy_in(g, g->f.jsrc, j, nvox(g), where)) != FLD_OK) return st;
    ++g->version;
    if ((st = validate_inputs(g, nullptr, nullptr, g->f.jsrc)) != FLD_OK) {
        FLD_CK(cudaMemsetAsync(g->f.jsrc, 0, sizeof(float) * (size_t)nvox(g), g->stream));
        return st;
    }
    return FLD_OK;
}

fld_status fld_get_source(fld_grid g, float *j, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!j) return fail(FLD_ERR_INVALID_ARG, "j must not be NULL");
    const cudaMemcpyKind kind = where == FLD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    FLD_CK(cudaMemcpyAsync(j, g->f.jsrc, sizeof(float) * (size_t)nvox(g), kind, g->stream));
    if (where != FLD_MEM_DEVICE) FLD_CK(cudaStreamSynchronize(g->stream));
    return FLD_OK;
}

fld_status fld_bake_directional(fld_grid g, const double dir[3], double radiance, double step, int accumulate) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!g->has_medium) return fail(FLD_ERR_STATE, "fld_set_medium has not been called");
    if (!dir) return fail(FLD_ERR_INVALID_ARG, "dir is NULL");
    const double n = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(n > 0.0) || !isfinite(n)) return fail(FLD_ERR_INVALID_ARG, "dir must be a nonzero finite vector");
    if (!(radiance >= 0.0) || !isfinite(radiance)) return fail(FLD_ERR_INVALID_ARG, "radiance must be >= 0");
    if (step <= 0.0) step = 0.5 * g->h;
    if (!isfinite(step)) return fail(FLD_ERR_INVALID_ARG, "bad step");
    if (dir[0] == 0.0 && dir[1] == 0.0 && dir[2] < 0.0 && step == 0.5 * g->h) {
        FLD_CK(launch_bake_scan_negz(g->L, g->f, (float)g->h, (float)radiance, accumulate, g->stream));
    } else {
        const double w[3] = {-dir[0] / n, -dir[1] / n, -dir[2] / n};   // towards the light
        const double pos[3] = {0, 0, 0};
        FLD_CK(launch_bake_march(g->L, g->f, (float)g->h, w, pos, 0, (float)radiance, (float)step, accumulate,
                                 g->stream));
    }
    ++g->version;
    return FLD_OK;
}

fld_status fld_bake_point(fld_grid g, const double pos[3], double power, double step, int accumulate) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!g->has_medium) return fail(FLD_ERR_STATE, "fld_set_medium has not been called");
    if (!pos || !isfinite(pos[0]) || !isfinite(pos[1]) || !isfinite(pos[2]))
        return fail(FLD_ERR_INVALID_ARG, "pos must be finite");
    if (!(power >= 0.0) || !isfinite(power)) return fail(FLD_ERR_INVALID_ARG, "power must be >= 0");
    if (step <= 0.0) step = 0.5 * g->h;
    if (!isfinite(step)) return fail(FLD_ERR_INVALID_ARG, "bad step");
    const double w[3] = {0, 0, 0};
    FLD_CK(launch_bake_march(g->L, g->f, (float)g->h, w, pos, 1, (float)power, (float)step, accumulate, g->stream));
    ++g->version;
    return FLD_OK;
}

fld_status fld_set_state(fld_grid g, const double *phi, const double *D, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!phi && !D) return FLD_OK;
    const size_t n = (size_t)(g->nx + 2) * (g->ny + 2) * (g->nz + 2);
    // Both families receive the values, so an FP64 continuation keeps them
    // exactly (the float family rounds D to float).
    if ((st = ensure_f64(g)) != FLD_OK) return st;
    if (!g->valid_float && !g->valid_d) {
        // a partial update of a grid without state: start from zeros
        FLD_CK(launch_init_f(g->L, g->f.phi, g->f.phlo, g->f.D, 0.0, 0.0, 0.0, 0.0, g->stream));
        FLD_CK(launch_init_d(g->L, g->f.phi64, g->f.D64, 0.0, 0.0, 0.0, 0.0, g->stream));
    } else if (g->valid_d && !g->valid_float) {
        FLD_CK(launch_d_to_f(g->L, g->f.phi64, g->f.phi, g->f.phlo, g->stream));
        FLD_CK(launch_d_to_f(g->L, g->f.D64, g->f.D, nullptr, g->stream));
    } else if (g->valid_float && !g->valid_d) {
        FLD_CK(launch_f_to_d(g->L, g->f.phi, g->lo_live ? g->f.phlo : nullptr, g->f.phi64, g->stream));
        FLD_CK(launch_f_to_d(g->L, g->f.D, nullptr, g->f.D64, g->stream));
    }
    double *stage = nullptr;
    if (where != FLD_MEM_DEVICE) FLD_CK(cudaMalloc((void **)&stage, sizeof(double) * n));
    const double *srcs[2] = {phi, D};
    for (int a = 0; a < 2; ++a) {
        if (!srcs[a]) continue;
        const double *src = srcs[a];
        if (stage) {
            cudaError_t e = cudaMemcpyAsync(stage, src, sizeof(double) * n, cudaMemcpyHostToDevice, g->stream);
            if (e != cudaSuccess) {
                cudaFree(stage);
                return cuda_fail(e, "cudaMemcpyAsync(set_state)");
            }
            src = stage;
        }
        cudaError_t e = a == 0 ? launch_unpack_to_f(g->L, src, g->f.phi, g->f.phlo, g->stream)
                               : launch_unpack_to_f(g->L, src, g->f.D, nullptr, g->stream);
        if (e == cudaSuccess) e = launch_unpack_to_d(g->L, src, a == 0 ? g->f.phi64 : g->f.D64, g->stream);
        if (e != cudaSuccess) {
            if (stage) cudaFree(stage);
            return cuda_fail(e, "unpack state");
        }
    }
    if (stage) {
        cudaStreamSynchronize(g->stream);
        cudaFree(stage);
    }
    g->valid_float = true;
    g->lo_live = true;
    g->valid_d = true;
    return FLD_OK;
}

fld_status fld_get_state(fld_grid g, double *phi, double *D, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if (!g->valid_float && !g->valid_d) return fail(FLD_ERR_STATE, "the grid holds no state yet");
    const size_t n = (size_t)(g->nx + 2) * (g->ny + 2) * (g->nz + 2);
    double *outs[2] = {phi, D};
    double *stage = nullptr;
    if (where != FLD_MEM_DEVICE && (phi || D)) FLD_CK(cudaMalloc((void **)&stage, sizeof(double) * n));
    for (int a = 0; a < 2; ++a) {
        if (!outs[a]) continue;
        double *dst = stage ? stage : outs[a];
        cudaError_t e;
        if (g->valid_d)
            e = launch_pack_from_d(g->L, a == 0 ? g->f.phi64 : g->f.D64, dst, g->stream);
        else
            e = a == 0 ? launch_pack_from_f(g->L, g->f.phi, g->lo_live ? g->f.phlo : nullptr, dst, g->stream)
                       : launch_pack_from_f(g->L, g->f.D, nullptr, dst, g->stream);
        if (e == cudaSuccess && stage)
            e = cudaMemcpyAsync(outs[a], stage, sizeof(double) * n, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess && stage) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            if (stage) cudaFree(stage);
            return cuda_fail(e, "get_state");
        }
    }
    if (stage) cudaFree(stage);
    return FLD_OK;
}

fld_status fld_iterate(fld_grid g, const fld_solve_params *p, int iterations) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if ((st = check_params(g, p)) != FLD_OK) return st;
    if (iterations < 0) return fail(FLD_ERR_INVALID_ARG, "iterations must be >= 0");
    const Family fam = p->precision == FLD_PREC_FP64 ? FAM_F64 : (p->precision == FLD_PREC_FP32 ? FAM_F32 : FAM_FF);
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if (!p->warm_start) {
        if ((st = init_state(g, p, fam)) != FLD_OK) return st;
    }
    if ((st = sync_family(g, fam)) != FLD_OK) return st;
    return enqueue_iterations(g, fam, pass_params(g, p), iterations);
}

fld_status fld_residual(fld_grid g, const fld_solve_params *p, double *rel) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if ((st = check_params(g, p)) != FLD_OK) return st;
    if (!rel) return fail(FLD_ERR_INVALID_ARG, "rel is NULL");
    const Family fam = p->precision == FLD_PREC_FP64 ? FAM_F64 : (p->precision == FLD_PREC_FP32 ? FAM_F32 : FAM_FF);
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if (!g->valid_float && !g->valid_d) return fail(FLD_ERR_STATE, "the grid holds no state yet");
    Family use = fam;
    if (fam != FAM_F64) use = g->lo_live ? FAM_FF : FAM_F32;
    if ((st = sync_family(g, use)) != FLD_OK) return st;
    return residual_now(g, use, pass_params(g, p), p->residual_margin, rel);
}

fld_status fld_solve(fld_grid g, const fld_solve_params *p, fld_solve_result *r) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if ((st = check_params(g, p)) != FLD_OK) return st;
    if (!(p->tol >= 0.0)) return fail(FLD_ERR_INVALID_ARG, "tol must be >= 0");
    if (p->max_iters < 0 || p->check_every < 1) return fail(FLD_ERR_INVALID_ARG, "bad max_iters / check_every");
    fld_solve_result res;
    memset(&res, 0, sizeof(res));
    const long long kernels0 = g->kernels;
    Family fam = p->precision == FLD_PREC_FP64 ? FAM_F64 : FAM_F32;
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if (p->precision == FLD_PREC_MIXED && (st = prepare(g, p, FAM_FF)) != FLD_OK) return st;
    if (!p->warm_start) {
        if ((st = init_state(g, p, fam)) != FLD_OK) return st;
    } else if (p->precision == FLD_PREC_MIXED && !g->valid_d && g->lo_live) {
        fam = FAM_FF;   // continue a correction phase
    }
    if ((st = sync_family(g, fam)) != FLD_OK) return st;
    PassParams pp = pass_params(g, p);
    const double sw = p->fp32_switch > 0.0 ? p->fp32_switch : 2e-5;
    res.jbar = g->jbar;
    res.omega = pp.omega;
    FLD_CK(cudaEventRecord(g->ev0, g->stream));
    Controller ctl;
    ctl.precision = p->precision;
    ctl.tol = p->tol;
    ctl.sw = sw;
    ctl.fam = fam;
    double rel = INFINITY;
    int it = 0;
    bool stalled = false;
    fld_status outcome = FLD_ERR_NOT_CONVERGED;
    // Safeguarded over-relaxation: the state with the best residual so far is
    // kept; if the residual turns non-finite, grows kGuardGrowth-fold, or
    // makes no new minimum for 16 checks while above twice the best, the solve
    // returns to it and continues with omega - 1 reduced by 3 %.
    Family snap_fam = fam;
    bool snap_lo_live = g->lo_live;
    auto save = [&]() -> fld_status {
        fld_status s2 = snapshot(g, fam, true);
        snap_fam = fam;
        snap_lo_live = g->lo_live;
        return s2;
    };
    if ((st = residual_now(g, fam, pp, p->residual_margin, &rel)) != FLD_OK) return st;
    ++res.checks;
    Action a = ctl.first(rel);
    if (a == ACT_CONVERGED) outcome = FLD_OK;
    else if (a == ACT_DIVERGED) outcome = FLD_ERR_DIVERGED;
    else if ((st = save()) != FLD_OK) return st;
    while (outcome == FLD_ERR_NOT_CONVERGED && it < p->max_iters) {
        int k = p->check_every;
        if (k > p->max_iters - it) k = p->max_iters - it;
        FLD_CK(cudaEventRecord(g->evb0, g->stream));
        if ((st = run_block(g, fam, pp, k)) != FLD_OK) return st;
        FLD_CK(cudaEventRecord(g->evb1, g->stream));
        it += k;
        if (fam == FAM_F32) res.iterations_fp32 += k;
        else res.iterations_corr += k;
        if ((st = residual_now(g, fam, pp, p->residual_margin, &rel)) != FLD_OK) return st;
        ++res.checks;
        float bms = 0.0f;   // the residual read above synchronised the stream
        FLD_CK(cudaEventElapsedTime(&bms, g->evb0, g->evb1));
        if (fam == FAM_F32) res.ms_sweep_fp32 += bms;
        else res.ms_sweep_corr += bms;
        a = ctl.next(rel, pp.omega);
        switch (a) {
        case ACT_CONVERGED: outcome = FLD_OK; break;
        case ACT_DIVERGED: outcome = FLD_ERR_DIVERGED; break;
        case ACT_STALLED: stalled = true; break;
        case ACT_SAVE:
            if ((st = save()) != FLD_OK) return st;
            break;
        case ACT_RESTORE:
            if ((st = snapshot(g, snap_fam, false)) != FLD_OK) return st;
            fam = snap_fam;
            ctl.fam = fam;
            g->lo_live = snap_lo_live;
            pp.omega = 1.0 + 0.97 * (pp.omega - 1.0);
            rel = ctl.best;
            break;
        case ACT_SWITCH:
            if ((st = sync_family(g, FAM_FF)) != FLD_OK) return st;
            fam = FAM_FF;
            ctl.fam = fam;
            ctl.begin_phase();
            break;
        case ACT_CONTINUE: break;
        }
        if (stalled) break;
    }
    res.omega_backoffs = ctl.backoffs;
    FLD_CK(cudaEventRecord(g->ev1, g->stream));
    FLD_CK(cudaEventSynchronize(g->ev1));
    float ms = 0.0f;
    FLD_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    res.status = outcome;
    res.iterations = it;
    res.rel_residual = rel;
    res.ms = ms;
    res.omega = pp.omega;
    res.kernels = g->kernels - kernels0;
    if (r) *r = res;
    if (outcome == FLD_ERR_DIVERGED) g_last_error = "residual became NaN or infinite";
    if (outcome == FLD_ERR_NOT_CONVERGED)
        g_last_error = stalled ? "residual stalled above tol (floor of the arithmetic)" : "max_iters reached before tol";
    return outcome;
}


// Solve one group of grids in shared launches (see fld_solve_batch).
static fld_status solve_group(fld_grid *grids, int count, const fld_solve_params *p, fld_solve_result *results,
                              double t_offset_ms) {
    fld_status st = FLD_OK;
    // Prepare and initialise every grid on its own stream first.
    std::vector<Family> fam(count, FAM_F32);
    for (int a = 0; a < count; ++a) {
        fld_grid_s *g = grids[a];
        FLD_CK(cudaStreamSynchronize(g->stream));
        if ((st = prepare(g, p, FAM_F32)) != FLD_OK) return st;
        if (!p->warm_start) {
            if ((st = init_state(g, p, FAM_F32)) != FLD_OK) return st;
        } else if (p->precision == FLD_PREC_MIXED && !g->valid_d && g->lo_live) {
            fam[a] = FAM_FF;
        }
        if ((st = sync_family(g, fam[a])) != FLD_OK) return st;
        FLD_CK(cudaStreamSynchronize(g->stream));
    }
    // From here on all work of the batch is ordered on the first grid's stream.
    cudaStream_t bs = grids[0]->stream;
    std::vector<cudaStream_t> own(count);
    for (int a = 0; a < count; ++a) {
        own[a] = grids[a]->stream;
        grids[a]->stream = bs;
    }
    struct Restore {
        fld_grid *g;
        std::vector<cudaStream_t> *s;
        ~Restore() {
            for (size_t a = 0; a < s->size(); ++a) g[a]->stream = (*s)[a];
        }
    } restore{grids, &own};

    const double sw = p->fp32_switch > 0.0 ? p->fp32_switch : 2e-5;
    std::vector<BatchDesc> hd(count);
    std::vector<int> res_count(count);
    int total_res = 0;
    const int rounds = p->local_iters < 1 ? 1 : p->local_iters;
    for (int a = 0; a < count; ++a) {
        fld_grid_s *g = grids[a];
        const PassParams pp = pass_params(g, p);
        BatchDesc &d = hd[a];
        d.L = g->L;
        d.sp = g->f.sp; d.ah2 = g->f.ah2; d.jh2 = g->f.jh2; d.phi = g->f.phi; d.phlo = g->f.phlo;
        d.D = g->f.D; d.Df = g->f.Df;
        d.omega = (float)pp.omega; d.inv2h = (float)pp.inv2h; d.floor_ = (float)pp.floor_;
        d.larsen_n = (float)pp.larsen_n; d.lim = pp.lim; d.rounds = rounds;
        d.mode = fam[a] == FAM_FF ? 1 : 0;
        d.active = 1;
        pass_dims(g->L, &d.pass_bx, &d.pass_by);
        residual_dims(g->L, &d.res_bx, &d.res_by);
        res_count[a] = d.res_bx * d.res_by * g->nz;
        d.res_slot = total_res;
        total_res += res_count[a];
    }
    // CTA table of the batched residual (rebuilt over the active grids as
    // grids finish).
    std::vector<int> res_tab;
    auto build_tables = [&]() {
        res_tab.clear();
        for (int a = 0; a < count; ++a) {
            if (!hd[a].active) continue;
            hd[a].res_first = (int)res_tab.size();
            res_tab.insert(res_tab.end(), (size_t)res_count[a], a);
        }
    };
    build_tables();

    // Device workspace of this call.
    BatchDesc *d_desc = nullptr;
    int *d_res = nullptr, *d_count = nullptr;
    double *d_part = nullptr, *d_out = nullptr;
    struct Free {
        void *p[5];
        ~Free() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } fr{{nullptr, nullptr, nullptr, nullptr, nullptr}};
    if (cudaMalloc((void **)&d_desc, sizeof(BatchDesc) * count) != cudaSuccess ||
        cudaMalloc((void **)&d_res, sizeof(int) * (size_t)total_res) != cudaSuccess ||
        cudaMalloc((void **)&d_count, sizeof(int) * count) != cudaSuccess ||
        cudaMalloc((void **)&d_part, sizeof(double) * 2 * (size_t)total_res) != cudaSuccess ||
        cudaMalloc((void **)&d_out, sizeof(double) * 2 * count) != cudaSuccess) {
        (void)cudaGetLastError();
        fr.p[0] = d_desc; fr.p[1] = d_res; fr.p[2] = d_count; fr.p[3] = d_part; fr.p[4] = d_out;
        return fail(FLD_ERR_OOM, "cudaMalloc of the batch workspace failed");
    }
    fr.p[0] = d_desc; fr.p[1] = d_res; fr.p[2] = d_count; fr.p[3] = d_part; fr.p[4] = d_out;
    FLD_CK(cudaMemcpyAsync(d_count, res_count.data(), sizeof(int) * count, cudaMemcpyHostToDevice, bs));
    auto upload = [&](bool tables) -> fld_status {
        FLD_CK(cudaMemcpyAsync(d_desc, hd.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, bs));
        if (tables) {
            if (!res_tab.empty())
                FLD_CK(cudaMemcpyAsync(d_res, res_tab.data(), sizeof(int) * res_tab.size(), cudaMemcpyHostToDevice, bs));
        }
        return FLD_OK;
    };
    if ((st = upload(true)) != FLD_OK) return st;

    std::vector<fld_solve_result> res(count);
    std::vector<Controller> ctl(count);
    std::vector<PassParams> ppv(count);
    for (int a = 0; a < count; ++a) ppv[a] = pass_params(grids[a], p);
    std::vector<Family> snap_fam(count);
    std::vector<bool> snap_lo(count);
    std::vector<double> host_out(2 * count);
    long long launches = 0;
    for (int a = 0; a < count; ++a) {
        memset(&res[a], 0, sizeof(fld_solve_result));
        res[a].status = FLD_ERR_NOT_CONVERGED;
        res[a].jbar = grids[a]->jbar;
        res[a].omega = hd[a].omega;
        ctl[a].precision = p->precision;
        ctl[a].tol = p->tol;
        ctl[a].sw = sw;
        ctl[a].fam = fam[a];
    }
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return t_offset_ms + std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    auto residuals = [&]() -> fld_status {
        FLD_CK(launch_residual_batch(d_desc, d_res, (int)res_tab.size(), count, d_count, d_part, d_out, p->limiter,
                                     p->residual_margin, bs));
        launches += 3;
        FLD_CK(cudaMemcpyAsync(host_out.data(), d_out, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, bs));
        FLD_CK(cudaStreamSynchronize(bs));
        return FLD_OK;
    };
    auto rel_of = [&](int a) {
        fld_grid_s *g = grids[a];
        const int m = p->residual_margin;
        const long long ex = g->nx - 2LL * m, ey = g->ny - 2LL * m, ez = g->nz - 2LL * m;
        const long long cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
        const double rb = cnt > 0 ? sqrt(host_out[2 * a] / (double)cnt) : 0.0;
        const double jb = sqrt(host_out[2 * a + 1] / (double)nvox(g));
        return jb > 0.0 ? rb / jb : rb / (g->h * g->h);
    };
    auto finish = [&](int a, fld_status s2, double rel) {
        hd[a].active = 0;
        res[a].status = s2;
        res[a].rel_residual = rel;
        res[a].ms = elapsed_ms();
    };
    // first check
    if ((st = residuals()) != FLD_OK) return st;
    int active = 0;
    for (int a = 0; a < count; ++a) {
        const double rel = rel_of(a);
        res[a].rel_residual = rel;
        ++res[a].checks;
        const Action act = ctl[a].first(rel);
        if (act == ACT_CONVERGED) finish(a, FLD_OK, rel);
        else if (act == ACT_DIVERGED) finish(a, FLD_ERR_DIVERGED, rel);
        else {
            if ((st = snapshot(grids[a], fam[a], true)) != FLD_OK) return st;
            snap_fam[a] = fam[a];
            snap_lo[a] = grids[a]->lo_live;
            ++active;
        }
    }
    if ((st = upload(false)) != FLD_OK) return st;

    // The sweeps of the active grids are one CUDA graph: each grid's chain of
    // solo pass kernels is captured on one stream of a small pool, forked from
    // and joined back to the batch stream, so independent grids run
    // concurrently and each runs exactly the kernels of its solo solve.  The
    // graph covers up to kGraphIters iterations and is replayed per check; it
    // is captured again when the active set, a grid's precision or its omega
    // changes.
    constexpr int kGraphIters = 64;
    const int nside = count < 16 ? count : 16;
    std::vector<cudaStream_t> side(nside, nullptr);
    std::vector<cudaEvent_t> join(nside, nullptr);
    cudaEvent_t fork = nullptr;
    struct SideFree {
        std::vector<cudaStream_t> *s;
        std::vector<cudaEvent_t> *j;
        cudaEvent_t *f;
        ~SideFree() {
            for (auto x : *s)
                if (x) cudaStreamDestroy(x);
            for (auto x : *j)
                if (x) cudaEventDestroy(x);
            if (*f) cudaEventDestroy(*f);
        }
    } sf{&side, &join, &fork};
    FLD_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int i = 0; i < nside; ++i) {
        FLD_CK(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
        FLD_CK(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
    }
    cudaGraphExec_t exec = nullptr;
    int graph_k = -1;
    bool dirty = true;
    struct GraphFree {
        cudaGraphExec_t *e;
        ~GraphFree() {
            if (*e) cudaGraphExecDestroy(*e);
        }
    } gf{&exec};
    auto capture = [&](int kg) -> fld_status {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        FLD_CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaEventRecord(fork, bs);
        for (int i = 0; i < nside && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(side[i], fork, 0);
        int slot = 0;
        for (int a = 0; a < count && ce == cudaSuccess; ++a) {
            if (!hd[a].active) continue;
            cudaStream_t ss = side[slot++ % nside];
            for (int i = 0; i < kg && ce == cudaSuccess; ++i)
                for (int c = 0; c < 2 && ce == cudaSuccess; ++c)
                    ce = launch_pass(fam[a], grids[a]->L, grids[a]->f, ppv[a], c, ss);
        }
        for (int i = 0; i < nside && ce == cudaSuccess; ++i) {
            ce = cudaEventRecord(join[i], side[i]);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(bs, join[i], 0);
        }
        cudaError_t ce2 = cudaStreamEndCapture(bs, &graph);
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ce != cudaSuccess ? ce : ce2, "batched graph capture");
        }
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            exec = nullptr;
            return cuda_fail(ce, "cudaGraphInstantiate (batch)");
        }
        graph_k = kg;
        dirty = false;
        return FLD_OK;
    };
    int it = 0;
    while (active > 0 && it < p->max_iters) {
        int k = p->check_every;
        if (k > p->max_iters - it) k = p->max_iters - it;
        // k iterations as reps replays of a kg-iteration graph
        int kg = k < kGraphIters ? k : kGraphIters;
        while (k % kg) --kg;
        if (!exec || dirty || graph_k != kg)
            if ((st = capture(kg)) != FLD_OK) return st;
        for (int rep = 0; rep < k / kg; ++rep) FLD_CK(cudaGraphLaunch(exec, bs));
        launches += 2LL * k * active;
        it += k;
        for (int a = 0; a < count; ++a) {
            if (!hd[a].active) continue;
            res[a].iterations += k;
            if (hd[a].mode == 0) res[a].iterations_fp32 += k;
            else res[a].iterations_corr += k;
        }
        if ((st = residuals()) != FLD_OK) return st;
        bool changed = false;
        for (int a = 0; a < count; ++a) {
            if (!hd[a].active) continue;
            fld_grid_s *g = grids[a];
            const double rel = rel_of(a);
            res[a].rel_residual = rel;
            ++res[a].checks;
            const Action act = ctl[a].next(rel, ppv[a].omega);
            switch (act) {
            case ACT_CONVERGED: finish(a, FLD_OK, rel); --active; changed = dirty = true; break;
            case ACT_DIVERGED: finish(a, FLD_ERR_DIVERGED, rel); --active; changed = dirty = true; break;
            case ACT_STALLED: finish(a, FLD_ERR_NOT_CONVERGED, rel); --active; changed = dirty = true; break;
            case ACT_SAVE:
                if ((st = snapshot(g, fam[a], true)) != FLD_OK) return st;
                snap_fam[a] = fam[a];
                snap_lo[a] = g->lo_live;
                break;
            case ACT_RESTORE:
                if ((st = snapshot(g, snap_fam[a], false)) != FLD_OK) return st;
                fam[a] = snap_fam[a];
                ctl[a].fam = fam[a];
                g->lo_live = snap_lo[a];
                hd[a].mode = fam[a] == FAM_FF ? 1 : 0;
                ppv[a].omega = 1.0 + 0.97 * (ppv[a].omega - 1.0);
                hd[a].omega = (float)ppv[a].omega;
                changed = dirty = true;
                break;
            case ACT_SWITCH:
                if ((st = sync_family(g, FAM_FF)) != FLD_OK) return st;
                fam[a] = FAM_FF;
                ctl[a].fam = FAM_FF;
                ctl[a].begin_phase();
                hd[a].mode = 1;
                changed = dirty = true;
                break;
            case ACT_CONTINUE: break;
            }
        }
        if (changed) {
            long long live = 0;
            for (int a = 0; a < count; ++a)
                if (hd[a].active) live += res_count[a];
            const bool compact = active > 0 && live < (long long)(0.7 * (double)res_tab.size());
            if (compact) build_tables();
            if ((st = upload(compact)) != FLD_OK) return st;
        }
    }
    fld_status worst = FLD_OK;
    for (int a = 0; a < count; ++a) {
        if (hd[a].active) finish(a, FLD_ERR_NOT_CONVERGED, res[a].rel_residual);
        fld_grid_s *g = grids[a];
        g->valid_float = true;
        g->valid_d = false;
        res[a].omega = ppv[a].omega;
        res[a].omega_backoffs = ctl[a].backoffs;
        res[a].kernels = launches;
        if (res[a].status == FLD_ERR_DIVERGED) worst = FLD_ERR_DIVERGED;
        else if (res[a].status != FLD_OK && worst == FLD_OK) worst = FLD_ERR_NOT_CONVERGED;
        if (results) results[a] = res[a];
    }
    FLD_CK(cudaStreamSynchronize(bs));
    if (worst != FLD_OK) g_last_error = "not every solve of the batch converged (see the per-grid results)";
    return worst;
}

fld_status fld_solve_batch(fld_grid *grids, int count, const fld_solve_params *p, fld_solve_result *results) {
    if (!grids || count < 1) return fail(FLD_ERR_INVALID_ARG, "grids must hold count >= 1 handles");
    for (int a = 0; a < count; ++a) {
        if (!grids[a]) return fail(FLD_ERR_INVALID_ARG, "a grid handle is NULL");
        for (int b = 0; b < a; ++b)
            if (grids[a] == grids[b]) return fail(FLD_ERR_INVALID_ARG, "a grid appears twice in the batch");
        if (grids[a]->device != grids[0]->device) return fail(FLD_ERR_INVALID_ARG, "grids live on different devices");
    }
    fld_status st = enter(grids[0]);
    if (st != FLD_OK) return st;
    if ((st = check_params(grids[0], p)) != FLD_OK) return st;
    if (p->precision == FLD_PREC_FP64)
        return fail(FLD_ERR_INVALID_ARG, "batched solves run the FP32 / MIXED sweeps; use fld_solve for FP64");
    if (!(p->tol >= 0.0)) return fail(FLD_ERR_INVALID_ARG, "tol must be >= 0");
    if (p->max_iters < 0 || p->check_every < 1) return fail(FLD_ERR_INVALID_ARG, "bad max_iters / check_every");
    // Grids of one shared launch should keep their per-iteration working set
    // (24 bytes per voxel: sigma', sigma_a', j, phi hi/lo, D) within L2: a
    // group larger than L2 streams from HBM on every pass, while each grid
    // alone would not.  Grids are taken in order of size and packed greedily
    // into groups of at most 3/4 of the L2 capacity; groups run one after
    // another, small grids share launches, large grids run alone.
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, grids[0]->device) != cudaSuccess || l2 <= 0) {
        (void)cudaGetLastError();
        l2 = 64 << 20;
    }
    const double budget = 0.75 * (double)l2;
    std::vector<int> order(count);
    for (int a = 0; a < count; ++a) order[a] = a;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nvox(grids[x]) < nvox(grids[y]); });
    std::vector<fld_solve_result> res(count);
    fld_status worst = FLD_OK;
    const auto t0 = std::chrono::steady_clock::now();
    size_t a = 0;
    while (a < order.size()) {
        std::vector<fld_grid> group;
        std::vector<int> idx;
        double ws = 0.0;
        while (a < order.size()) {
            const double w = 24.0 * (double)nvox(grids[order[a]]);
            if (!group.empty() && ws + w > budget) break;
            group.push_back(grids[order[a]]);
            idx.push_back(order[a]);
            ws += w;
            ++a;
        }
        std::vector<fld_solve_result> gr(group.size());
        const double off = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        st = solve_group(group.data(), (int)group.size(), p, gr.data(), off);
        if (st != FLD_OK && st != FLD_ERR_NOT_CONVERGED && st != FLD_ERR_DIVERGED) return st;
        for (size_t b = 0; b < group.size(); ++b) res[idx[b]] = gr[b];
        if (st == FLD_ERR_DIVERGED) worst = FLD_ERR_DIVERGED;
        else if (st == FLD_ERR_NOT_CONVERGED && worst == FLD_OK) worst = FLD_ERR_NOT_CONVERGED;
    }
    if (results)
        for (int b = 0; b < count; ++b) results[b] = res[b];
    if (worst != FLD_OK) g_last_error = "not every solve of the batch converged (see the per-grid results)";
    return worst;
}

}  // extern "C"
