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

#include <dlfcn.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <mutex>
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
constexpr int kSlowDivergeChecks = 32;        // ... or checks without a new minimum while above 4x the best
constexpr int kFlatWindow = 8;                // single-precision floor: checks compared ...
constexpr int kFlatWindowMax = 64;            // (the window in checks after scaling, at most)
constexpr double kFlatGain = 0.05;            // ... and the smallest relative decrease that is progress
constexpr double kFlatBelow = 0.1;            // ... below this fraction of the starting residual
constexpr int kMaxBackoffs = 8;               // omega reductions before reporting divergence
constexpr double kOmegaMax = 1.98;            // upper clamp of the automatic omega
constexpr int kWarmupPerEdge = 4;             // automatic warm-up: iterations per voxel of the largest extent
constexpr double kNestedTol = 1e-4;           // nested solves: tolerance of the coarser levels
constexpr int kPolishBlock = 16;              // MIXED + fp64_verify: FP64 sweeps between FP64 checks

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int fam = -1;
    int iters = 0;
    long long kernels = 0;   // kernel launches one replay issues
    PassParams p{};
};

bool same_params(const PassParams &a, const PassParams &b) {
    return a.lim == b.lim && a.local_iters == b.local_iters && a.larsen_n == b.larsen_n && a.omega == b.omega &&
           a.inv2h == b.inv2h && a.floor_ == b.floor_ && a.bf16 == b.bf16 && a.h2 == b.h2 && a.scheme == b.scheme &&
           a.tiled_f32 == b.tiled_f32 && a.tiled_fh == b.tiled_fh && a.quad_f32 == b.quad_f32 && a.quad_fh == b.quad_fh;
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
    int prepared_bf16_f = -1, prepared_bf16_d = -1;   // medium rounding of the prepared fields
    double jbar = 0.0;
    long long jbar_version = 0;
    bool valid_float = false, valid_d = false;   // which family holds the state
    bool lo_live = false;                        // phlo may be non-zero
    GraphEntry graphs[4];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evb0 = nullptr, evb1 = nullptr;
    long long kernels = 0;                       // kernel launches issued so far
    fld_grid_s *coarse = nullptr;                // nested solves: the next 2x coarser grid (owned)
    // last good state of a solve (float family: phi, lo, D; FP64: phi, D)
    float *snap_phi = nullptr, *snap_lo = nullptr, *snap_D = nullptr;
    double *snap_phi64 = nullptr, *snap_D64 = nullptr;
    // Anderson mixing (fld_solve_params.anderson): history slots, allocated on first use
    AndersonBuffers anderson{};
    int anderson_slots = 0;
    int nsm = 0;
    // temporally blocked sweeps: the other buffers of the ping-pong pair, the
    // kernels' timeout flag and the TMA descriptors (made on first use)
    float *alt_phi = nullptr, *alt_D = nullptr, *alt_lo = nullptr;
    int *tiled_status = nullptr;
    TiledMaps maps[kTiledConfigs][2];    // [config][0: input in phi/D/phlo, 1: input in alt_*]
    bool maps_ok[kTiledConfigs] = {};
    bool tiled_used = false;             // blocked launches since the status was last read
    // device staging of fld_render's host outputs (kept, grown on demand)
    float *stage_rad = nullptr;
    unsigned char *stage_cod = nullptr;
    size_t stage_px = 0;
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

// bfloat16 copies of sigma' and sigma_a' (medium_bf16).
fld_status ensure_bf16(fld_grid_s *g) {
    if (g->f.spb) return FLD_OK;
    const size_t bytes = sizeof(uint16_t) * (size_t)g->L.total;
    uint16_t **ptrs[2] = {&g->f.spb, &g->f.sab};
    for (uint16_t **p : ptrs) {
        cudaError_t e = cudaMalloc((void **)p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FLD_ERR_OOM, "cudaMalloc of the bfloat16 medium failed");
        }
        FLD_CK(cudaMemsetAsync(*p, 0, bytes, g->stream));
    }
    return FLD_OK;
}

// Second phi buffer of the Jacobi scheme (allocated outside graph capture).
fld_status ensure_jacobi(fld_grid_s *g, Family fam) {
    const size_t n = (size_t)g->L.total;
    cudaError_t e = cudaSuccess;
    if (fam == FAM_F64 && !g->f.phi642) e = cudaMalloc((void **)&g->f.phi642, sizeof(double) * n);
    if (fam != FAM_F64 && !g->f.phi2) e = cudaMalloc((void **)&g->f.phi2, sizeof(float) * n);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(FLD_ERR_OOM, "cudaMalloc of the Jacobi buffer failed");
    }
    return FLD_OK;
}

void free_anderson(fld_grid_s *g) {
    void *ptrs[] = {g->anderson.g, g->anderson.f, g->anderson.x, g->anderson.part, g->anderson.dots};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    g->anderson = AndersonBuffers{};
    g->anderson_slots = 0;
}

// History of m slots for Anderson mixing (allocated outside graph capture).
fld_status ensure_anderson(fld_grid_s *g, int m) {
    if (g->anderson_slots >= m) return FLD_OK;
    FLD_CK(cudaStreamSynchronize(g->stream));
    free_anderson(g);
    if (g->nsm <= 0) {
        FLD_CK(cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device));
        if (g->nsm <= 0) g->nsm = 1;
    }
    const size_t n = (size_t)g->L.total;
    AndersonBuffers &b = g->anderson;
    if (cudaMalloc((void **)&b.g, sizeof(float2) * n * m) != cudaSuccess ||
        cudaMalloc((void **)&b.f, sizeof(float) * n * m) != cudaSuccess ||
        cudaMalloc((void **)&b.x, sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc((void **)&b.part, sizeof(double) * kAndersonMax * 4 * (size_t)g->nsm) != cudaSuccess ||
        cudaMalloc((void **)&b.dots, sizeof(double) * kAndersonMax) != cudaSuccess) {
        (void)cudaGetLastError();
        free_anderson(g);
        return fail(FLD_ERR_OOM, "cudaMalloc of the Anderson history failed");
    }
    g->anderson_slots = m;
    return FLD_OK;
}

// Weights of Anderson mixing over w slots: minimise |sum a_i f_i| subject to
// sum a_i = 1, i.e. a = y / sum(y) with (G + lambda I) y = 1, G the Gram
// matrix <f_i, f_j> and lambda = 1e-12 of its mean diagonal (Tikhonov).
// Gaussian elimination with partial pivoting; false if the system is
// singular or the weights are not finite or exceed kAndersonMaxWeight.
constexpr double kAndersonMaxWeight = 1e3;
bool anderson_weights(const double gram[kAndersonMax][kAndersonMax], int w, double *a) {
    double A[kAndersonMax][kAndersonMax + 1];
    double tr = 0.0;
    for (int i = 0; i < w; ++i) tr += gram[i][i];
    const double lam = 1e-12 * (tr / w);
    if (!(tr > 0.0) || !isfinite(tr)) return false;
    for (int i = 0; i < w; ++i) {
        for (int j = 0; j < w; ++j) A[i][j] = gram[i][j] + (i == j ? lam : 0.0);
        A[i][w] = 1.0;
    }
    for (int c = 0; c < w; ++c) {
        int piv = c;
        for (int r = c + 1; r < w; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 0.0)) return false;
        if (piv != c)
            for (int k = c; k <= w; ++k) std::swap(A[c][k], A[piv][k]);
        for (int r = c + 1; r < w; ++r) {
            const double m = A[r][c] / A[c][c];
            for (int k = c; k <= w; ++k) A[r][k] -= m * A[c][k];
        }
    }
    double y[kAndersonMax];
    for (int r = w - 1; r >= 0; --r) {
        double v = A[r][w];
        for (int k = r + 1; k < w; ++k) v -= A[r][k] * y[k];
        y[r] = v / A[r][r];
    }
    double sum = 0.0;
    for (int i = 0; i < w; ++i) sum += y[i];
    if (!(fabs(sum) > 0.0) || !isfinite(sum)) return false;
    for (int i = 0; i < w; ++i) {
        a[i] = y[i] / sum;
        if (!isfinite(a[i]) || fabs(a[i]) > kAndersonMaxWeight) return false;
    }
    return true;
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
    if (p->scheme == FLD_SCHEME_JACOBI) return 1.0;
    int n = g->nx;
    if (g->ny > n) n = g->ny;
    if (g->nz > n) n = g->nz;
    double w = 2.0 / (1.0 + sin(M_PI / (n + 1.0)));
    if (w < 1.0) w = 1.0;
    if (w > kOmegaMax) w = kOmegaMax;
    return w;
}

// Cold starts relax with omega = 1 for their first iterations.  Over-relaxing
// the paper's near-zero initial state blows up within a few hundred sweeps
// (omega 1.95 at 128^3, 1.93 at 192^3 and 256^3, in single and double
// precision alike), while the same omega, and the Laplacian estimate above
// it, stays stable once the first sweeps have spread the source.
int warmup_of(const fld_grid_s *g, const fld_solve_params *p) {
    if (p->warmup_iters >= 0) return p->warmup_iters;
    if (p->warm_start || p->scheme == FLD_SCHEME_JACOBI) return 0;
    int n = g->nx;
    if (g->ny > n) n = g->ny;
    if (g->nz > n) n = g->nz;
    return kWarmupPerEdge * n;
}

// Length of the next block of iterations: check_every, cut at the end of the
// warm-up and at max_iters.
int block_len(int it, int check_every, int max_iters, int warm) {
    int k = check_every;
    if (it < warm && k > warm - it) k = warm - it;
    if (k > max_iters - it) k = max_iters - it;
    return k;
}

// Iterations between checks in family `fam`: the FP64 sweeps that follow a
// MIXED solve's float-float phase only remove the rounding noise of the
// single-precision D, so they are checked more often.
int check_len(Family fam, int precision, int check_every) {
    if (fam == FAM_F64 && precision == FLD_PREC_MIXED && check_every > kPolishBlock) return kPolishBlock;
    return check_every;
}

// Pass parameters of a block starting at iteration `it`.
PassParams block_params(const PassParams &pp, int it, int warm) {
    PassParams q = pp;
    if (it < warm) q.omega = 1.0;
    return q;
}

fld_status read_result(fld_grid_s *g, double out[2]) {
    FLD_CK(cudaMemcpyAsync(out, g->f.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    int timeout = 0;
    if (g->tiled_used)
        FLD_CK(cudaMemcpyAsync(&timeout, g->tiled_status, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    FLD_CK(cudaStreamSynchronize(g->stream));
    if (g->tiled_used) {
        g->tiled_used = false;
        if (timeout) {
            FLD_CK(cudaMemsetAsync(g->tiled_status, 0, sizeof(int), g->stream));
            return fail(FLD_ERR_TIMEOUT, "a blocked sweep gave up waiting for its tile copies");
        }
    }
    return FLD_OK;
}

// Buffers and TMA descriptors of blocked configuration `id`.
fld_status ensure_tiled(fld_grid_s *g, int id) {
    if (id < 0) return FLD_OK;
    if (!g->alt_phi) {
        const size_t nb = sizeof(float) * (size_t)g->L.total;
        if (cudaMalloc((void **)&g->alt_phi, nb) != cudaSuccess || cudaMalloc((void **)&g->alt_D, nb) != cudaSuccess ||
            cudaMalloc((void **)&g->alt_lo, nb) != cudaSuccess ||
            cudaMalloc((void **)&g->tiled_status, sizeof(int)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FLD_ERR_OOM, "cudaMalloc of the blocked sweeps' buffers failed");
        }
        FLD_CK(cudaMemsetAsync(g->tiled_status, 0, sizeof(int), g->stream));
    }
    if (!g->maps_ok[id]) {
        FLD_CK(tiled_maps(g->L, id, g->f.phi, g->f.D, g->f.phlo, &g->maps[id][0]));
        FLD_CK(tiled_maps(g->L, id, g->alt_phi, g->alt_D, g->alt_lo, &g->maps[id][1]));
        g->maps_ok[id] = true;
    }
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
    const int bf = p->medium_bf16 ? 1 : 0;
    if (fam == FAM_F64) {
        st = ensure_f64(g);
        if (st != FLD_OK) return st;
        if (p->scheme == FLD_SCHEME_JACOBI && (st = ensure_jacobi(g, fam)) != FLD_OK) return st;
        if (g->prepared_d != g->version || g->prepared_seps_d != seps || g->prepared_bf16_d != bf) {
            FLD_CK(launch_prep_d(g->L, g->f, seps, h2, bf != 0, g->stream));
            g->kernels += 1;
            g->prepared_d = g->version;
            g->prepared_seps_d = seps;
            g->prepared_bf16_d = bf;
        }
    } else {
        if (bf && (st = ensure_bf16(g)) != FLD_OK) return st;
        if (p->scheme == FLD_SCHEME_JACOBI && (st = ensure_jacobi(g, fam)) != FLD_OK) return st;
        if (g->prepared_f != g->version || g->prepared_seps_f != seps || g->prepared_bf16_f != bf) {
            FLD_CK(launch_prep_f(g->L, g->f, (float)seps, (float)h2, bf != 0, g->stream));
            g->kernels += 1;
            g->prepared_f = g->version;
            g->prepared_seps_f = seps;
            g->prepared_bf16_f = bf;
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
    q.bf16 = p->medium_bf16 ? 1 : 0;
    q.scheme = p->scheme;
    q.h2 = g->h * g->h;
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

// First sweep family of a precision mode.
Family start_family(int precision) {
    switch (precision) {
    case FLD_PREC_FP64: return FAM_F64;
    case FLD_PREC_PAIR: return FAM_FH;
    default: return FAM_F32;
    }
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
        if (fam == FAM_FF || fam == FAM_FH) g->lo_live = true;
        g->valid_d = false;
    }
    return FLD_OK;
}

fld_status enqueue_iterations(fld_grid_s *g, Family fam, const PassParams &pp, int iters, long long *nk = nullptr) {
    if (nk) *nk = 2LL * iters;
    if (pp.scheme == FLD_SCHEME_JACOBI) {
        // ping-pong between phi and its second buffer; the second buffer first
        // takes phi whole (its ghosts), and an odd count ends with a copy back
        const bool d = fam == FAM_F64;
        const size_t bytes = (d ? sizeof(double) : sizeof(float)) * (size_t)g->L.total;
        void *a = d ? (void *)g->f.phi64 : (void *)g->f.phi;
        void *b = d ? (void *)g->f.phi642 : (void *)g->f.phi2;
        if (!b) return fail(FLD_ERR_STATE, "the Jacobi buffer is not allocated");
        FLD_CK(cudaMemcpyAsync(b, a, bytes, cudaMemcpyDeviceToDevice, g->stream));
        for (int it = 0; it < iters; ++it) FLD_CK(launch_jacobi(fam, g->L, g->f, pp, (it & 1) == 0, g->stream));
        if (iters & 1) FLD_CK(cudaMemcpyAsync(a, b, bytes, cudaMemcpyDeviceToDevice, g->stream));
        return FLD_OK;
    }
    // temporally blocked launches (an even number, ping-ponging between the
    // grid's fields and their second copies, so the state ends where it began),
    // the remaining iterations as launched colour passes
    const int id = fam == FAM_F32 ? pp.tiled_f32 : fam == FAM_FH ? pp.tiled_fh : -1;
    int done = 0;
    if (id >= 0) {
        if (!g->maps_ok[id]) return fail(FLD_ERR_STATE, "blocked sweeps were not prepared");
        const int T = tiled_depth(id);
        const int nl = (iters / T) & ~1;
        if (nl > 0) {
            const size_t nb = sizeof(float) * (size_t)g->L.total;
            FLD_CK(cudaMemcpyAsync(g->alt_phi, g->f.phi, nb, cudaMemcpyDeviceToDevice, g->stream));
            FLD_CK(cudaMemcpyAsync(g->alt_D, g->f.D, nb, cudaMemcpyDeviceToDevice, g->stream));
            if (fam == FAM_FH) FLD_CK(cudaMemcpyAsync(g->alt_lo, g->f.phlo, nb, cudaMemcpyDeviceToDevice, g->stream));
            for (int i = 0; i < nl; ++i) {
                const int from_alt = i & 1;
                float *dphi = from_alt ? g->f.phi : g->alt_phi;
                float *dD = from_alt ? g->f.D : g->alt_D;
                float *dlo = from_alt ? g->f.phlo : g->alt_lo;
                FLD_CK(launch_tiled(fam, id, g->L, g->f, pp, g->maps[id][from_alt], dphi, dD, dlo, g->tiled_status,
                                    g->nsm, g->stream));
            }
            done = nl * T;
            if (nk) *nk = nl + 2LL * (iters - done);
            g->tiled_used = true;
        }
    }
    for (int it = done; it < iters; ++it)
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
        long long nk = 0;
        fld_status st = enqueue_iterations(g, fam, pp, iters, &nk);
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
        e.kernels = nk;
    }
    FLD_CK(cudaGraphLaunch(e.exec, g->stream));
    g->kernels += e.kernels;
    if (e.p.tiled_f32 >= 0 || e.p.tiled_fh >= 0) g->tiled_used = true;
    return FLD_OK;
}

fld_status residual_now(fld_grid_s *g, Family fam, const PassParams &pp, int margin, double *rel) {
    FLD_CK(launch_residual(fam, g->L, g->f, pp, margin, g->stream));
    g->kernels += 3;
    double r[2];
    fld_status st = read_result(g, r);
    if (st != FLD_OK) return st;
    // r[0] = sum (R_p h^2)^2 over the margin set, r[1] = sum (j_p h^2)^2
    *rel = rel_residual_from_sums(g->nx, g->ny, g->nz, g->h, margin, r[0], r[1]);
    return FLD_OK;
}

// The stop test in FP64 (fld_solve_params.fp64_verify): the FP64 medium
// (once per medium version), the current single-precision state converted to
// double (hi + lo) and the residual of Eq. 37 with D recomputed from phi in
// double.  Afterwards the state lives in the FP64 fields.
fld_status fp64_check(fld_grid_s *g, const fld_solve_params *p, const PassParams &pp, double *rel) {
    fld_status st = prepare(g, p, FAM_F64);
    if (st != FLD_OK) return st;
    if ((st = sync_family(g, FAM_F64)) != FLD_OK) return st;
    return residual_now(g, FAM_F64, pp, p->residual_margin, rel);
}

// After a restore: the snapshot's family holds the state.
void set_valid(fld_grid_s *g, Family fam) {
    g->valid_d = fam == FAM_F64;
    g->valid_float = fam != FAM_F64;
}

// ---------------------------------------------------------------------------
// Autotuner (not a paper item): for each grid shape, sweep family, limiter and
// medium it times the launched colour passes against every blocked
// configuration on the grid itself, and the residual check against one
// iteration, and keeps
//   * the fastest sweep launch shape (all of them give the same bits, so the
//     choice changes the time only), and
//   * the check interval: the smallest power of two (32 ... 1024) at which a
//     check costs at most 2 % of the iterations between two checks.
// Choices are kept for the process and appended to a cache file
// (FLD_TUNE_CACHE, else fld_tune_cache.txt beside the library), so later
// processes reuse them.  The candidates read the grid's state and write only
// its second buffers; the state is not changed.
// ---------------------------------------------------------------------------
struct TuneChoice {
    int tiled = -1;           // blocked configuration id; launched passes: -1 two, -2 four unknowns per thread
    int check_every = 64;
    double us_launched = 0.0, us_best = 0.0, us_check = 0.0;   // measured per iteration / per check
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;
constexpr double kCheckShare = 0.02;   // a check may cost this share of the iterations between checks

std::string tune_path() {
    const char *env = getenv("FLD_TUNE_CACHE");
    if (env && *env) return env;
    Dl_info info;
    if (dladdr((void *)&fld_default_params, &info) && info.dli_fname) {
        const std::string p = info.dli_fname;
        const size_t k = p.find_last_of('/');
        if (k != std::string::npos) return p.substr(0, k + 1) + "fld_tune_cache.txt";
    }
    return "";
}

std::string tune_key(const fld_grid_s *g, Family fam, const PassParams &pp) {
    char b[192];
    snprintf(b, sizeof(b), "v2 %dx%dx%d fam%d lim%d r%d bf%d sm%d", g->nx, g->ny, g->nz, (int)fam, pp.lim,
             pp.local_iters, pp.bf16, g->nsm);
    return b;
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_path();
    FILE *fp = path.empty() ? nullptr : fopen(path.c_str(), "r");
    if (!fp) return;
    char line[512];
    while (fgets(line, sizeof(line), fp)) {
        char *bar = strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        std::string key = line;
        while (!key.empty() && key.back() == ' ') key.pop_back();
        TuneChoice c;
        if (sscanf(bar + 1, "%d %d %lf %lf %lf", &c.tiled, &c.check_every, &c.us_launched, &c.us_best, &c.us_check) == 5 &&
            c.tiled >= -2 && c.tiled < kTiledConfigs && c.check_every >= 1)
            g_tune[key] = c;
    }
    fclose(fp);
}

void tune_store_locked(const std::string &key, const TuneChoice &c) {
    g_tune[key] = c;
    const std::string path = tune_path();
    FILE *fp = path.empty() ? nullptr : fopen(path.c_str(), "a");
    if (!fp) return;
    fprintf(fp, "%s | %d %d %.4f %.4f %.4f\n", key.c_str(), c.tiled, c.check_every, c.us_launched, c.us_best,
            c.us_check);
    fclose(fp);
}

// Time the candidates of family fam on g (state in the family's fields).
fld_status tune_family(fld_grid_s *g, const fld_solve_params *p, const PassParams &pp, Family fam, TuneChoice *out) {
    for (int id = 0; id < kTiledConfigs; ++id) {
        fld_status st = ensure_tiled(g, id);
        if (st != FLD_OK) return st;
        FLD_CK(tiled_prepare(fam, id, pp));
    }
    const size_t nb = sizeof(float) * (size_t)g->L.total;
    FLD_CK(cudaMemcpyAsync(g->alt_phi, g->f.phi, nb, cudaMemcpyDeviceToDevice, g->stream));
    FLD_CK(cudaMemcpyAsync(g->alt_D, g->f.D, nb, cudaMemcpyDeviceToDevice, g->stream));
    FLD_CK(cudaMemcpyAsync(g->alt_lo, g->f.phlo, nb, cudaMemcpyDeviceToDevice, g->stream));
    Fields fa = g->f;   // the launched passes run in place on the second buffers
    fa.phi = g->alt_phi;
    fa.D = g->alt_D;
    fa.phlo = g->alt_lo;
    const int n = 16;   // iterations per timing, a multiple of every depth
    TuneChoice c;
    double best = INFINITY;
    for (int cand = -2; cand < kTiledConfigs; ++cand) {
        double t = INFINITY;
        PassParams pc = pp;
        pc.quad_f32 = pc.quad_fh = cand == -2 ? 1 : 0;
        for (int rep = 0; rep < 3; ++rep) {   // the first is a warm-up
            FLD_CK(cudaEventRecord(g->evb0, g->stream));
            if (cand < 0) {
                for (int it = 0; it < n; ++it)
                    for (int colour = 0; colour < 2; ++colour) FLD_CK(launch_pass(fam, g->L, fa, pc, colour, g->stream));
            } else {
                for (int i = 0; i < n / tiled_depth(cand); ++i)
                    FLD_CK(launch_tiled(fam, cand, g->L, g->f, pp, g->maps[cand][0], g->alt_phi, g->alt_D, g->alt_lo,
                                        g->tiled_status, g->nsm, g->stream));
            }
            FLD_CK(cudaEventRecord(g->evb1, g->stream));
            FLD_CK(cudaEventSynchronize(g->evb1));
            float ms = 0.0f;
            FLD_CK(cudaEventElapsedTime(&ms, g->evb0, g->evb1));
            if (rep > 0) t = std::min(t, 1e3 * ms / n);
        }
        if (cand == -1) c.us_launched = t;
        if (t < best) {
            best = t;
            c.tiled = cand;
        }
    }
    g->tiled_used = true;   // surface a timeout of the timed blocked launches at the next check
    c.us_best = best;
    // one residual check, as the solve takes it (kernels + 16-byte readback)
    double tc = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
        double rel = 0.0;
        const auto t0 = std::chrono::steady_clock::now();
        fld_status st = residual_now(g, fam, pp, p->residual_margin, &rel);
        if (st != FLD_OK) return st;
        const double us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
        if (rep > 0) tc = std::min(tc, us);
    }
    c.us_check = tc;
    int ce = 32;
    while (ce < 1024 && tc > kCheckShare * ce * best) ce *= 2;
    c.check_every = ce;
    *out = c;
    return FLD_OK;
}

// The sweep launch shape of each single-precision family (pp.tiled_f32 /
// tiled_fh) and the check interval *ce of a solve, from the parameters or
// the autotuner.  The state must already be initialised.
fld_status choose_sweeps(fld_grid_s *g, const fld_solve_params *p, PassParams *pp, int *ce) {
    pp->tiled_f32 = pp->tiled_fh = -1;
    pp->quad_f32 = pp->quad_fh = p->cells_per_thread == 4 ? 1 : 0;
    *ce = p->check_every > 0 ? p->check_every : 64;
    if (p->scheme != FLD_SCHEME_RED_BLACK || p->precision == FLD_PREC_FP64) return FLD_OK;
    fld_status st = FLD_OK;
    if (p->temporal_depth > 0) {
        const int id = tiled_config_of(p->temporal_depth, p->tile_y);
        if (id < 0) return fail(FLD_ERR_INVALID_ARG, "no blocked configuration with that temporal_depth / tile_y");
        if ((st = ensure_tiled(g, id)) != FLD_OK) return st;
        FLD_CK(tiled_prepare(FAM_F32, id, *pp));
        FLD_CK(tiled_prepare(FAM_FH, id, *pp));
        pp->tiled_f32 = pp->tiled_fh = id;
    }
    if (p->temporal_depth != 0 && p->check_every > 0) return FLD_OK;
    const Family fams[2] = {p->precision == FLD_PREC_PAIR ? FAM_FH : FAM_F32, FAM_FH};
    const int nfam = p->precision == FLD_PREC_MIXED ? 2 : 1;
    for (int k = 0; k < nfam; ++k) {
        const Family fam = fams[k];
        const std::string key = tune_key(g, fam, *pp);
        TuneChoice c;
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_load_locked();
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                c = it->second;
                have = true;
            }
        }
        if (!have) {
            if ((st = tune_family(g, p, *pp, fam, &c)) != FLD_OK) return st;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);   // another thread may have tuned it meanwhile: keep the first
            if (it != g_tune.end()) c = it->second;
            else tune_store_locked(key, c);
        }
        if (p->temporal_depth == 0) {
            if ((st = ensure_tiled(g, c.tiled)) != FLD_OK) return st;
            if (c.tiled >= 0) FLD_CK(tiled_prepare(fam, c.tiled, *pp));
            const int shape = c.tiled >= 0 ? c.tiled : -1;
            const int quad = c.tiled == -2 ? 1 : 0;
            if (fam == FAM_F32) {
                pp->tiled_f32 = shape;
                pp->quad_f32 = quad;
            } else {
                pp->tiled_fh = shape;
                pp->quad_fh = quad;
            }
        }
        if (k == 0 && p->check_every <= 0) *ce = c.check_every;
    }
    return FLD_OK;
}

fld_status check_params(const fld_grid_s *g, const fld_solve_params *p) {
    if (!p) return fail(FLD_ERR_INVALID_ARG, "params is NULL");
    if (const char *bad = check_limiter_margin(p->limiter, p->larsen_n, p->residual_margin))
        return fail(FLD_ERR_INVALID_ARG, bad);
    if (p->omega > 0.0 && !(p->omega < 2.0)) return fail(FLD_ERR_INVALID_ARG, "omega must lie in (0, 2)");
    if (p->precision < FLD_PREC_FP64 || p->precision > FLD_PREC_PAIR)
        return fail(FLD_ERR_INVALID_ARG, "unknown precision");
    if (p->local_iters > 64) return fail(FLD_ERR_INVALID_ARG, "local_iters must be <= 64");
    if (p->medium_bf16 != 0 && p->medium_bf16 != 1) return fail(FLD_ERR_INVALID_ARG, "medium_bf16 must be 0 or 1");
    if (p->warmup_iters < -1) return fail(FLD_ERR_INVALID_ARG, "warmup_iters must be >= -1");
    if (p->scheme != FLD_SCHEME_RED_BLACK && p->scheme != FLD_SCHEME_JACOBI)
        return fail(FLD_ERR_INVALID_ARG, "unknown scheme");
    if (p->anderson < 0 || p->anderson > kAndersonMax)
        return fail(FLD_ERR_INVALID_ARG, "anderson must lie in [0, 16]");
    if (p->anderson > 0 && p->scheme == FLD_SCHEME_JACOBI)
        return fail(FLD_ERR_INVALID_ARG, "Anderson mixing accelerates the red-black scheme only");
    if (p->fp64_verify != 0 && p->fp64_verify != 1) return fail(FLD_ERR_INVALID_ARG, "fp64_verify must be 0 or 1");
    if (p->temporal_depth < -1 || p->temporal_depth == 3 || p->temporal_depth > 4)
        return fail(FLD_ERR_INVALID_ARG, "temporal_depth must be -1, 0, 1, 2 or 4");
    if (p->tile_y < 0) return fail(FLD_ERR_INVALID_ARG, "tile_y must be >= 0");
    if (p->cells_per_thread != 0 && p->cells_per_thread != 2 && p->cells_per_thread != 4)
        return fail(FLD_ERR_INVALID_ARG, "cells_per_thread must be 0, 2 or 4");
    if (p->scheme == FLD_SCHEME_JACOBI) {
        if (p->precision != FLD_PREC_FP32 && p->precision != FLD_PREC_FP64)
            return fail(FLD_ERR_INVALID_ARG, "the Jacobi scheme runs in FP32 or FP64 precision");
        if (p->omega > 1.0) return fail(FLD_ERR_INVALID_ARG, "the Jacobi scheme needs omega <= 1");
    }
    (void)g;
    return FLD_OK;
}

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

// Everything a solve may allocate on the device, allocated before it starts
// (so admission by free memory sees it, and no allocation falls inside the
// solve): the safeguard's snapshot of the single-precision state, and, for a
// MIXED solve with the FP64 stop test, the FP64 fields and their snapshot.
fld_status preallocate(fld_grid_s *g, const fld_solve_params *p) {
    const size_t nf = sizeof(float) * (size_t)g->L.total, nd = sizeof(double) * (size_t)g->L.total;
    const bool f64 = p->precision == FLD_PREC_FP64 || (p->precision == FLD_PREC_MIXED && p->fp64_verify);
    if (f64) {
        fld_status st = ensure_f64(g);
        if (st != FLD_OK) return st;
    }
    bool ok = true;
    if (!g->snap_phi)
        ok = cudaMalloc((void **)&g->snap_phi, nf) == cudaSuccess && cudaMalloc((void **)&g->snap_lo, nf) == cudaSuccess &&
             cudaMalloc((void **)&g->snap_D, nf) == cudaSuccess;
    if (ok && f64 && !g->snap_phi64)
        ok = cudaMalloc((void **)&g->snap_phi64, nd) == cudaSuccess && cudaMalloc((void **)&g->snap_D64, nd) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return fail(FLD_ERR_OOM, "cudaMalloc of the solve's buffers failed");
    }
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

// The precision that follows `f` in a MIXED solve.
Family next_family(Family f) { return f == FAM_F32 ? FAM_FH : FAM_FF; }

struct Controller {
    int precision = FLD_PREC_MIXED;
    double tol = 1e-6, sw = 2e-5;
    Family fam = FAM_F32;
    double best = INFINITY;   // best residual after at least one block
    double initial = INFINITY;
    int since_best = 0;       // checks without a new minimum
    int backoffs = 0;
    double recent[kFlatWindowMax + 1] = {};   // residuals of the last checks of this phase
    int nrecent = 0;
    // Windows of the decisions below, in checks.  The constants above are
    // checks at 256 iterations per check on a 128-voxel edge; a plain SOR
    // solve keeps the same windows in iterations per voxel of its largest
    // edge, i.e. 2 n / check_every checks per constant (never fewer than the
    // constant), so a shorter check interval or a larger grid does not make it
    // give up sooner; so do the FP64 sweeps that end its MIXED solve, at their
    // own check interval.  An Anderson-mixed solve, which progresses many
    // times faster per iteration, keeps the constants until it falls back to
    // plain sweeps.
    int stall_w = kStallChecks, switch_w = kSwitchChecks, slow_w = kSlowDivergeChecks, flat_w = kFlatWindow;

    void scale_windows(int n, int check_every) {
        auto sc = [&](int base, int cap) {
            const long long it = 2LL * base * n;
            long long w = (it + check_every - 1) / check_every;
            if (w < base) w = base;
            if (w > cap) w = cap;
            return (int)w;
        };
        stall_w = sc(kStallChecks, 1 << 20);
        switch_w = sc(kSwitchChecks, 1 << 20);
        slow_w = sc(kSlowDivergeChecks, 1 << 20);
        flat_w = sc(kFlatWindow, kFlatWindowMax);
    }

    void begin_phase() {
        since_best = 0;
        nrecent = 0;
    }
    // End of the warm-up at omega = 1: the over-relaxed iteration starts
    // from here like a new solve (its first blocks may sit above the warm-up's
    // residual while the higher omega settles).
    Action restart(double rel) {
        best = INFINITY;
        begin_phase();
        return first(rel);
    }
    // The residual has reached a floor (of single precision, or of an
    // over-relaxed cycle): it sits at its best, an order of magnitude below
    // where the (over-relaxed) iteration started, and fell by less than
    // kFlatGain over the last kFlatWindow checks.  (Right after omega rises
    // the residual also hovers, but near its start.)
    bool flat(double rel) {
        recent[nrecent % (flat_w + 1)] = rel;
        ++nrecent;
        if (nrecent <= flat_w) return false;
        const double then = recent[(nrecent - 1 - flat_w) % (flat_w + 1)];
        return rel > (1.0 - kFlatGain) * then && rel < 1.1 * best && rel < kFlatBelow * initial;
    }
    // The float-float phase met tol on its single-precision-D residual and the
    // FP64 residual (rel) is above it: FP64 sweeps continue from here, with
    // progress measured against that FP64 value (windows scaled to the FP64
    // check interval on a grid of largest edge n when `scale`).
    void enter_fp64(double rel, int n, bool scale) {
        fam = FAM_F64;
        best = rel;
        stall_w = kStallChecks;
        switch_w = kSwitchChecks;
        slow_w = kSlowDivergeChecks;
        flat_w = kFlatWindow;
        if (scale) scale_windows(n, kPolishBlock);
        begin_phase();
    }
    // First check (before any iteration): the state is kept as the fallback of
    // the safeguard, but progress is measured from the first block onwards
    // (SOR's early transient may sit above the initial residual for a while).
    Action first(double rel) {
        initial = rel;
        if (rel <= tol) return ACT_CONVERGED;
        if (!isfinite(rel)) return ACT_DIVERGED;
        return ACT_SAVE;
    }
    // After a block of iterations.
    Action next(double rel, double omega) {
        // growth is measured against the initial residual too, so a first
        // block that blows up is not taken for the best state
        const double ref = best < initial ? best : initial;
        const bool diverging = !isfinite(rel) || rel > kGuardGrowth * ref ||
                               (since_best >= slow_w && rel > 4.0 * best);
        if (diverging) {
            if (backoffs >= kMaxBackoffs || omega <= 1.0) return ACT_DIVERGED;
            ++backoffs;
            since_best = 0;
            nrecent = 0;
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
        const bool no_progress = since_best >= switch_w;
        // No new minimum for a while and the residual above where the
        // over-relaxed iteration started: that is omega cycling the nonlinear
        // iteration (seen with omega 1.97 at 128^3: 4-6 against a start of
        // 0.43), not a precision floor (which a warm start may begin near) --
        // return to the best state with a smaller omega.
        if (no_progress && omega > 1.0 && rel >= initial && backoffs < kMaxBackoffs) {
            ++backoffs;
            since_best = 0;
            nrecent = 0;
            return ACT_RESTORE;
        }
        // single precision has done what it can (Sec. 6.2: ~1e-4 is its limit):
        // continue with phi as a hi/lo pair, first with FP32-summed updates,
        // then with float-float sums near the tolerance
        const bool at_floor = flat(rel);
        if (precision == FLD_PREC_MIXED && fam == FAM_F32 && (rel <= sw || no_progress || at_floor))
            return ACT_SWITCH;
        if (precision == FLD_PREC_MIXED && fam == FAM_FH && (rel <= 3.0 * tol || no_progress || at_floor))
            return ACT_SWITCH;
        // The float-float and FP64 sweeps reach residuals near 1e-7; a floor
        // above the tolerance there is the over-relaxed nonlinear iteration
        // cycling (seen from omega ~1.95 at 128^3), not the arithmetic: back
        // off omega, which collapses it.
        if ((fam == FAM_FF || fam == FAM_F64) && tol > 0.0 && (no_progress || at_floor) && best > tol) {
            if (backoffs >= kMaxBackoffs || omega <= 1.0) return ACT_STALLED;
            ++backoffs;
            since_best = 0;
            nrecent = 0;
            return ACT_RESTORE;
        }
        if (since_best >= stall_w && !(precision == FLD_PREC_MIXED && fam != FAM_FF)) return ACT_STALLED;
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
    p->warmup_iters = -1;
    p->anderson = 0;
    p->fp64_verify = 1;
    p->temporal_depth = 0;
    p->tile_y = 0;
    p->cells_per_thread = 0;
    p->batch_launch = 0;
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
    case FLD_ERR_TIMEOUT: return "FLD_ERR_TIMEOUT";
    }
    return "FLD_ERR_UNKNOWN";
}

const char *fld_last_error(void) { return g_last_error.c_str(); }

fld_status fld_create_grid(int nx, int ny, int nz, double h, void *stream, fld_grid *out) {
    if (!out) return fail(FLD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(FLD_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (!(h > 0.0) || !isfinite(h)) return fail(FLD_ERR_INVALID_ARG, "h must be a positive finite number");
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) ||
        ((long long)nx + 2) * ((long long)ny + 2) * ((long long)nz + 2) > (1LL << 40))
        return fail(FLD_ERR_INVALID_ARG, "grid too large");
    Layout probe;
    if (!make_layout(nx, ny, nz, &probe))
        return fail(FLD_ERR_INVALID_ARG, "grid too large: a padded field must stay below 2e9 elements");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        (void)cudaGetLastError();
        return fail(FLD_ERR_NO_DEVICE, "no CUDA device available");
    }
    fld_grid_s *g = new (std::nothrow) fld_grid_s();
    if (!g) return fail(FLD_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, g->device);
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
    if (g->coarse) {
        fld_destroy(g->coarse);
        g->coarse = nullptr;
    }
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (GraphEntry &e : g->graphs)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    void *ptrs[] = {g->f.sp, g->f.ah2, g->f.jh2, g->f.phi, g->f.phlo, g->f.D, g->f.Df, g->f.sp64, g->f.ah264,
                    g->f.jh264, g->f.phi64, g->f.D64, g->f.Df64, g->f.sigma_t, g->f.albedo, g->f.jsrc,
                    g->f.partials, g->f.result, g->f.spb, g->f.sab, g->f.phi2, g->f.phi642, g->f.render_vol};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->evb0) cudaEventDestroy(g->evb0);
    if (g->evb1) cudaEventDestroy(g->evb1);
    void *snaps[] = {g->snap_phi, g->snap_lo, g->snap_D, g->snap_phi64, g->snap_D64, g->alt_phi, g->alt_D,
                     g->alt_lo, g->tiled_status, g->stage_rad, g->stage_cod};
    for (void *p : snaps)
        if (p) cudaFree(p);
    free_anderson(g);
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

fld_status fld_downsample(fld_grid fine, fld_grid coarse, int factor) {
    fld_status st = enter(fine);
    if (st != FLD_OK) return st;
    if (!coarse || coarse == fine) return fail(FLD_ERR_INVALID_ARG, "coarse must be another grid");
    if (coarse->device != fine->device) return fail(FLD_ERR_INVALID_ARG, "the grids live on different devices");
    if (factor < 1) return fail(FLD_ERR_INVALID_ARG, "factor must be >= 1");
    if (coarse->nx != (fine->nx + factor - 1) / factor || coarse->ny != (fine->ny + factor - 1) / factor ||
        coarse->nz != (fine->nz + factor - 1) / factor)
        return fail(FLD_ERR_INVALID_ARG, "the coarse grid must have ceil(n / factor) voxels per axis");
    if (fabs(coarse->h - factor * fine->h) > 1e-9 * factor * fine->h)
        return fail(FLD_ERR_INVALID_ARG, "the coarse grid's h must be factor * h");
    if (!fine->has_medium) return fail(FLD_ERR_STATE, "the fine grid has no medium");
    FLD_CK(cudaStreamSynchronize(fine->stream));
    FLD_CK(launch_downsample(fine->L, fine->f, factor, coarse->L, coarse->f, coarse->stream));
    coarse->kernels += 1;
    coarse->has_medium = true;
    ++coarse->version;
    return FLD_OK;
}

fld_status fld_render(fld_grid g, fld_grid phi_grid, const fld_camera *cam, float *radiance, unsigned char *codes,
                      double exposure, double gamma, int where) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    fld_grid_s *pg = phi_grid ? phi_grid : g;
    if (pg->device != g->device) return fail(FLD_ERR_INVALID_ARG, "the phi grid lives on another device");
    if (pg != g && (pg->nx * pg->h < g->nx * g->h * (1 - 1e-9) || pg->ny * pg->h < g->ny * g->h * (1 - 1e-9) ||
                    pg->nz * pg->h < g->nz * g->h * (1 - 1e-9)))
        return fail(FLD_ERR_INVALID_ARG, "the phi grid must cover the rendered grid's box");
    if (!cam) return fail(FLD_ERR_INVALID_ARG, "camera is NULL");
    if (!radiance && !codes) return fail(FLD_ERR_INVALID_ARG, "radiance and codes are both NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return fail(FLD_ERR_INVALID_ARG, "image size must be 1 .. 16384 per side");
    if (!(cam->fov_deg > 0.0 && cam->fov_deg < 180.0)) return fail(FLD_ERR_INVALID_ARG, "fov_deg must be in (0, 180)");
    if (!(exposure > 0.0) || !(gamma > 0.0) || !isfinite(exposure) || !isfinite(gamma))
        return fail(FLD_ERR_INVALID_ARG, "exposure and gamma must be > 0");
    if (!(cam->background >= 0.0) || !isfinite(cam->background)) return fail(FLD_ERR_INVALID_ARG, "bad background");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(cam->eye[k]) || !isfinite(cam->target[k]) || !isfinite(cam->up[k]))
            return fail(FLD_ERR_INVALID_ARG, "camera vectors must be finite");
    if (!g->has_medium) return fail(FLD_ERR_STATE, "fld_set_medium has not been called");
    if (!pg->valid_float && !pg->valid_d) return fail(FLD_ERR_STATE, "the grid holds no state yet");
    RenderCamera c;
    double fn = 0.0;
    for (int k = 0; k < 3; ++k) {
        c.eye[k] = cam->eye[k];
        c.f[k] = cam->target[k] - cam->eye[k];
        fn += c.f[k] * c.f[k];
    }
    fn = sqrt(fn);
    if (!(fn > 0.0)) return fail(FLD_ERR_INVALID_ARG, "eye and target coincide");
    for (int k = 0; k < 3; ++k) c.f[k] /= fn;
    c.r[0] = c.f[1] * cam->up[2] - c.f[2] * cam->up[1];
    c.r[1] = c.f[2] * cam->up[0] - c.f[0] * cam->up[2];
    c.r[2] = c.f[0] * cam->up[1] - c.f[1] * cam->up[0];
    const double rn = sqrt(c.r[0] * c.r[0] + c.r[1] * c.r[1] + c.r[2] * c.r[2]);
    if (!(rn > 1e-12)) return fail(FLD_ERR_INVALID_ARG, "up is parallel to the view direction");
    for (int k = 0; k < 3; ++k) c.r[k] /= rn;
    c.u[0] = c.r[1] * c.f[2] - c.r[2] * c.f[1];
    c.u[1] = c.r[2] * c.f[0] - c.r[0] * c.f[2];
    c.u[2] = c.r[0] * c.f[1] - c.r[1] * c.f[0];
    c.tan_half = tan(0.5 * cam->fov_deg * M_PI / 180.0);
    c.aspect = (double)cam->width / (double)cam->height;
    c.h = g->h;
    c.width = cam->width;
    c.height = cam->height;
    c.step = cam->step > 0.0 ? cam->step : 0.5 * g->h;
    if (!isfinite(c.step)) return fail(FLD_ERR_INVALID_ARG, "bad step");
    c.background = cam->background;
    c.t_min = cam->t_min < 0.0 ? 1e-6 : cam->t_min;
    if (!g->f.render_vol) {
        if (cudaMalloc((void **)&g->f.render_vol, sizeof(float4) * (size_t)nvox(g)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FLD_ERR_OOM, "cudaMalloc of the sampling volume failed");
        }
    }
    const size_t npx = (size_t)cam->width * (size_t)cam->height;
    float *rad = radiance;
    unsigned char *cod = codes;
    if (where != FLD_MEM_DEVICE) {
        // device staging for host outputs: the grid keeps its buffers and
        // grows them only for a larger image, so a render loop allocates
        // nothing after its first frame
        if (npx > g->stage_px) {
            FLD_CK(cudaStreamSynchronize(g->stream));
            if (g->stage_rad) cudaFree(g->stage_rad);
            if (g->stage_cod) cudaFree(g->stage_cod);
            g->stage_rad = nullptr;
            g->stage_cod = nullptr;
            g->stage_px = 0;
            if (cudaMalloc((void **)&g->stage_rad, sizeof(float) * npx) != cudaSuccess ||
                cudaMalloc((void **)&g->stage_cod, npx) != cudaSuccess) {
                (void)cudaGetLastError();
                if (g->stage_rad) cudaFree(g->stage_rad);
                g->stage_rad = nullptr;
                g->stage_cod = nullptr;
                return fail(FLD_ERR_OOM, "cudaMalloc of the image staging buffers failed");
            }
            g->stage_px = npx;
        }
        rad = radiance ? g->stage_rad : nullptr;
        cod = codes ? g->stage_cod : nullptr;
    }
    PhiSource ps;
    const bool use_f = pg->valid_float;
    ps.phi = use_f ? pg->f.phi : nullptr;
    ps.phlo = use_f && pg->lo_live ? pg->f.phlo : nullptr;
    ps.phi64 = use_f ? nullptr : pg->f.phi64;
    ps.coarse = pg != g;
    ps.C = pg->L;
    ps.hc = pg->h;
    cudaError_t e = pg != g ? cudaStreamSynchronize(pg->stream) : cudaSuccess;
    if (e == cudaSuccess)
        e = launch_render(g->L, g->f, ps, c, g->f.render_vol, rad, cod, exposure, gamma, g->stream);
    g->kernels += 2;
    if (e == cudaSuccess && where != FLD_MEM_DEVICE) {
        if (radiance) e = cudaMemcpyAsync(radiance, rad, sizeof(float) * npx, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess && codes) e = cudaMemcpyAsync(codes, cod, npx, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fld_render");
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
    const Family fam = p->precision == FLD_PREC_MIXED ? FAM_FF : start_family(p->precision);
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if (!p->warm_start) {
        if ((st = init_state(g, p, fam)) != FLD_OK) return st;
    }
    if ((st = sync_family(g, fam)) != FLD_OK) return st;
    PassParams pp = pass_params(g, p);
    int ce = 0;
    if ((st = choose_sweeps(g, p, &pp, &ce)) != FLD_OK) return st;
    return enqueue_iterations(g, fam, pp, iterations);
}

fld_status fld_residual(fld_grid g, const fld_solve_params *p, double *rel) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if ((st = check_params(g, p)) != FLD_OK) return st;
    if (!rel) return fail(FLD_ERR_INVALID_ARG, "rel is NULL");
    const Family fam = p->precision == FLD_PREC_FP64 ? FAM_F64 : FAM_FF;
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if (!g->valid_float && !g->valid_d) return fail(FLD_ERR_STATE, "the grid holds no state yet");
    Family use = fam;
    if (fam != FAM_F64) use = g->lo_live ? FAM_FF : FAM_F32;
    if ((st = sync_family(g, use)) != FLD_OK) return st;
    return residual_now(g, use, pass_params(g, p), p->residual_margin, rel);
}

namespace {
fld_status solve_core(fld_grid g, const fld_solve_params *p, fld_solve_result *r);
fld_status solve_nested(fld_grid g, const fld_solve_params *p, fld_solve_result *r);
}  // namespace

fld_status fld_solve(fld_grid g, const fld_solve_params *p, fld_solve_result *r) {
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    if ((st = check_params(g, p)) != FLD_OK) return st;
    if (!(p->tol >= 0.0)) return fail(FLD_ERR_INVALID_ARG, "tol must be >= 0");
    if (p->max_iters < 0 || p->check_every < 0) return fail(FLD_ERR_INVALID_ARG, "bad max_iters / check_every");
    if (p->nested > 0 && !p->warm_start && p->scheme == FLD_SCHEME_RED_BLACK) return solve_nested(g, p, r);
    return solve_core(g, p, r);
}

namespace {

// Start from the solutions of successively coarser problems (fld_solve_params
// .nested): box-averaged medium and source on grids of 2x, 4x, ... the
// spacing, the coarsest solved cold to kNestedTol, each finer one from the
// next coarser phi (blended trilinearly, D recomputed) to kNestedTol, and g
// from its coarser neighbour to the caller's tolerance.
fld_status solve_nested(fld_grid g, const fld_solve_params *p, fld_solve_result *r) {
    int levels = p->nested;
    while (levels > 0) {   // coarse edges stay >= 8
        const int f = 1 << levels;
        if ((g->nx + f - 1) / f >= 8 && (g->ny + f - 1) / f >= 8 && (g->nz + f - 1) / f >= 8) break;
        --levels;
    }
    if (levels == 0) return solve_core(g, p, r);
    // the chain g -> coarse -> ... (kept with the grid, rebuilt if the shape changed)
    std::vector<fld_grid_s *> chain{g};
    for (int l = 1; l <= levels; ++l) {
        fld_grid_s *up = chain.back();
        const int cx = (up->nx + 1) / 2, cy = (up->ny + 1) / 2, cz = (up->nz + 1) / 2;
        if (up->coarse && (up->coarse->nx != cx || up->coarse->ny != cy || up->coarse->nz != cz ||
                           up->coarse->h != 2.0 * up->h)) {
            fld_destroy(up->coarse);
            up->coarse = nullptr;
        }
        if (!up->coarse) {
            fld_grid c = nullptr;
            fld_status st = fld_create_grid(cx, cy, cz, 2.0 * up->h, (void *)up->stream, &c);
            if (st != FLD_OK) return st;
            up->coarse = c;
        }
        chain.push_back(up->coarse);
    }
    fld_status st = FLD_OK;
    for (int l = 1; l <= levels; ++l)
        if ((st = fld_downsample(chain[l - 1], chain[l], 2)) != FLD_OK) return st;
    fld_solve_params q = *p;
    q.nested = 0;
    q.fp64_verify = 0;          // the coarser levels only provide a start
    q.tol = p->tol > kNestedTol ? p->tol : kNestedTol;
    q.check_every = p->check_every < 64 ? p->check_every : 64;
    fld_solve_result acc;
    memset(&acc, 0, sizeof(acc));
    for (int l = levels; l >= 0; --l) {
        fld_grid_s *c = chain[l];
        if (l < levels) {
            // prolong the coarser solution into c's state
            fld_grid_s *from = chain[l + 1];
            const Family fam = FAM_F32;
            if ((st = prepare(c, p, fam)) != FLD_OK) return st;
            if ((st = init_state(c, p, fam)) != FLD_OK) return st;   // ghosts, defaults
            if ((st = sync_family(c, fam)) != FLD_OK) return st;
            if ((st = sync_family(from, from->valid_float ? (from->lo_live ? FAM_FF : FAM_F32) : FAM_F64)) != FLD_OK)
                return st;
            PhiSource ps;
            ps.phi = from->valid_float ? from->f.phi : nullptr;
            ps.phlo = from->valid_float && from->lo_live ? from->f.phlo : nullptr;
            ps.phi64 = from->valid_float ? nullptr : from->f.phi64;
            ps.coarse = true;
            ps.C = from->L;
            ps.hc = from->h;
            FLD_CK(cudaStreamSynchronize(from->stream));
            FLD_CK(launch_prolong(c->L, c->f, ps, c->h, c->stream));
            FLD_CK(launch_fresh_D_into(c->L, c->f, pass_params(c, p), c->stream));
            c->kernels += 2;
            c->lo_live = false;
            c->valid_float = true;
            c->valid_d = false;
            q.warm_start = 1;
        } else {
            q.warm_start = 0;
        }
        if (l == 0) {
            q.tol = p->tol;
            q.check_every = p->check_every;
            q.fp64_verify = p->fp64_verify;
        }
        fld_solve_result rl;
        memset(&rl, 0, sizeof(rl));
        st = solve_core(c, &q, &rl);
        if (st != FLD_OK && st != FLD_ERR_NOT_CONVERGED) return st;
        if (l > 0) {
            acc.iterations_coarse += rl.iterations;
            acc.ms_coarse += rl.ms;
            acc.updates_coarse += (long long)rl.iterations * c->nx * c->ny * c->nz;
            acc.kernels += rl.kernels;
        } else {
            const int ic = acc.iterations_coarse;
            const double mc = acc.ms_coarse;
            const long long uc = acc.updates_coarse;
            const long long kc = acc.kernels;
            acc = rl;
            acc.iterations_coarse = ic;
            acc.ms_coarse = mc;
            acc.updates_coarse = uc;
            acc.ms += mc;
            acc.kernels += kc;
        }
        if (l == 0 && r) *r = acc;
        if (l == 0) return st;
    }
    return st;
}

fld_status solve_core(fld_grid g, const fld_solve_params *p, fld_solve_result *r) {
    fld_status st = FLD_OK;
    fld_solve_result res;
    memset(&res, 0, sizeof(res));
    const long long kernels0 = g->kernels;
    Family fam = start_family(p->precision);
    if ((st = prepare(g, p, fam)) != FLD_OK) return st;
    if ((st = preallocate(g, p)) != FLD_OK) return st;
    if (!p->warm_start) {
        if ((st = init_state(g, p, fam)) != FLD_OK) return st;
    } else if (p->precision == FLD_PREC_MIXED && !g->valid_d && g->lo_live) {
        fam = FAM_FF;   // continue a correction phase
    }
    if ((st = sync_family(g, fam)) != FLD_OK) return st;
    PassParams pp = pass_params(g, p);
    int ce = 0;   // iterations between checks
    if ((st = choose_sweeps(g, p, &pp, &ce)) != FLD_OK) return st;
    const double sw = p->fp32_switch > 0.0 ? p->fp32_switch : 2e-5;
    res.jbar = g->jbar;
    res.omega = pp.omega;
    FLD_CK(cudaEventRecord(g->ev0, g->stream));
    Controller ctl;
    ctl.precision = p->precision;
    if (p->anderson <= 1) ctl.scale_windows(std::max(g->nx, std::max(g->ny, g->nz)), ce);
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
    const bool verify = p->precision == FLD_PREC_MIXED && p->fp64_verify;
    // A MIXED solve whose single-precision-D residual met tol takes the stop
    // test of Algorithm 1 in FP64; above tol it continues with FP64 sweeps.
    auto confirm = [&]() -> fld_status {
        if (!verify || fam == FAM_F64) {
            outcome = FLD_OK;
            return FLD_OK;
        }
        double r64 = 0.0;
        fld_status s2 = fp64_check(g, p, pp, &r64);
        if (s2 != FLD_OK) return s2;
        ++res.checks;
        res.rel_residual_single = rel;
        rel = r64;
        fam = FAM_F64;
        ctl.enter_fp64(r64, std::max(g->nx, std::max(g->ny, g->nz)), p->anderson <= 1);
        if (r64 <= p->tol) outcome = FLD_OK;
        return FLD_OK;
    };
    if ((st = residual_now(g, fam, pp, p->residual_margin, &rel)) != FLD_OK) return st;
    ++res.checks;
    Action a = ctl.first(rel);
    if (a == ACT_CONVERGED) {
        if ((st = confirm()) != FLD_OK) return st;
        if (outcome != FLD_OK && (st = save()) != FLD_OK) return st;
    } else if (a == ACT_DIVERGED) {
        outcome = FLD_ERR_DIVERGED;
    } else if ((st = save()) != FLD_OK) {
        return st;
    }
    const int warm = warmup_of(g, p);
    // Anderson mixing (fld_solve_params.anderson): after the warm-up, each
    // block of sweeps is one application of the fixed-point map G; the next
    // block starts from the mix of the last `am` images.
    const int am = p->anderson;
    if (am > 0 && (st = ensure_anderson(g, am)) != FLD_OK) return st;
    double gram[kAndersonMax][kAndersonMax] = {};
    int acount = 0;          // blocks collected since the history (re)started
    bool have_x = false;     // the Anderson x holds the state the next block starts from
    bool mix_off = false;    // mixing given up after a stall: plain sweeps from the best state
    auto state_ptrs = [&](float **hi, float **lo, double **p64) {
        const bool d = fam == FAM_F64;
        *hi = d ? nullptr : g->f.phi;
        *lo = !d && g->lo_live ? g->f.phlo : nullptr;
        *p64 = d ? g->f.phi64 : nullptr;
    };
    while (outcome == FLD_ERR_NOT_CONVERGED && it < p->max_iters) {
        const int k = block_len(it, check_len(fam, p->precision, ce), p->max_iters, warm);
        const bool mixing = am > 0 && it >= warm && !mix_off;
        if (mixing && !have_x) {
            float *hi, *lo;
            double *p64;
            state_ptrs(&hi, &lo, &p64);
            FLD_CK(launch_anderson_capture(g->anderson, g->L.total, hi, lo, p64, g->nsm, g->stream));
            g->kernels += 1;
            have_x = true;
            acount = 0;
        }
        FLD_CK(cudaEventRecord(g->evb0, g->stream));
        if ((st = run_block(g, fam, block_params(pp, it, warm), k)) != FLD_OK) return st;
        FLD_CK(cudaEventRecord(g->evb1, g->stream));
        it += k;
        const bool polish = fam == FAM_F64 && p->precision == FLD_PREC_MIXED;
        if (fam == FAM_F32) res.iterations_fp32 += k;
        else if (fam == FAM_FH) res.iterations_mid += k;
        else if (polish) res.iterations_fp64 += k;
        else res.iterations_corr += k;
        if ((st = residual_now(g, fam, pp, p->residual_margin, &rel)) != FLD_OK) return st;
        ++res.checks;
        float bms = 0.0f;   // the residual read above synchronised the stream
        FLD_CK(cudaEventElapsedTime(&bms, g->evb0, g->evb1));
        if (fam == FAM_F32) res.ms_sweep_fp32 += bms;
        else if (fam == FAM_FH) res.ms_sweep_mid += bms;
        else if (polish) res.ms_sweep_fp64 += bms;
        else res.ms_sweep_corr += bms;
        a = (warm > 0 && it == warm) ? ctl.restart(rel) : ctl.next(rel, pp.omega);
        switch (a) {
        case ACT_CONVERGED:
            if ((st = confirm()) != FLD_OK) return st;
            have_x = false;
            break;
        case ACT_DIVERGED: outcome = FLD_ERR_DIVERGED; break;
        case ACT_STALLED:
            if (am > 1 && !mix_off && it < p->max_iters) {
                // the mixed iteration stalled above tol: continue with plain
                // sweeps (and the plain solve's windows) from the best state
                if ((st = snapshot(g, snap_fam, false)) != FLD_OK) return st;
                fam = snap_fam;
                ctl.fam = fam;
                set_valid(g, fam);
                g->lo_live = snap_lo_live;
                rel = ctl.best;
                mix_off = true;
                have_x = false;
                ctl.scale_windows(std::max(g->nx, std::max(g->ny, g->nz)), check_len(fam, p->precision, ce));
                ctl.backoffs = 0;   // a fresh omega back-off budget for the plain sweeps
                ctl.begin_phase();
                ++res.anderson_resets;
            } else {
                stalled = true;
            }
            break;
        case ACT_SAVE:
            if ((st = save()) != FLD_OK) return st;
            break;
        case ACT_RESTORE:
            if ((st = snapshot(g, snap_fam, false)) != FLD_OK) return st;
            fam = snap_fam;
            ctl.fam = fam;
            set_valid(g, fam);
            g->lo_live = snap_lo_live;
            pp.omega = 1.0 + 0.97 * (pp.omega - 1.0);
            rel = ctl.best;
            have_x = false;
            break;
        case ACT_SWITCH:
            fam = next_family(fam);
            if ((st = sync_family(g, fam)) != FLD_OK) return st;
            ctl.fam = fam;
            ctl.begin_phase();
            have_x = false;
            break;
        case ACT_CONTINUE: break;
        }
        if (stalled) break;
        // Anderson step after a block that made ordinary progress (never after
        // the last one: the solve ends on a checked state)
        if (mixing && have_x && (a == ACT_CONTINUE || a == ACT_SAVE) && it < p->max_iters) {
            const int slot = acount % am;
            ++acount;
            const int w = acount < am ? acount : am;
            float *hi, *lo;
            double *p64;
            state_ptrs(&hi, &lo, &p64);
            FLD_CK(launch_anderson_collect(g->anderson, g->L.total, hi, lo, p64, slot, w, g->nsm, g->stream));
            double dots[kAndersonMax];
            FLD_CK(cudaMemcpyAsync(dots, g->anderson.dots, sizeof(double) * w, cudaMemcpyDeviceToHost, g->stream));
            FLD_CK(cudaStreamSynchronize(g->stream));
            g->kernels += 2;
            for (int j = 0; j < w; ++j) gram[slot][j] = gram[j][slot] = dots[j];
            double wts[kAndersonMax];
            bool ok = true;
            if (w == 1) wts[0] = 1.0;   // x = g: the next block starts where this one ended
            else ok = anderson_weights(gram, w, wts);
            if (ok) {
                FLD_CK(launch_anderson_mix(g->anderson, g->L.total, slot, w, wts, hi, lo, p64, g->nsm, g->stream));
                g->kernels += 1;
                if (w > 1) ++res.anderson_steps;
            } else {
                // ill-conditioned history: continue from this block's result
                ++res.anderson_resets;
                have_x = false;
            }
        }
    }
    // a MIXED solve that ended in the FP64 sweeps hands its state back to the
    // hi/lo fields (about 48 significant bits), where MIXED warm starts and the
    // batched paths continue from
    if (fam == FAM_F64 && p->precision == FLD_PREC_MIXED && (st = sync_family(g, FAM_FF)) != FLD_OK) return st;
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

}  // namespace


// ===========================================================================
// Server: grids join and leave a running set of solves (continuous batching).
// Each step runs one block of check_every iterations for every active grid --
// each grid replaying its own block graph (the one fld_solve uses) on a
// stream of a small pool, so independent grids run concurrently; with
// batch_launch = 1 the grids in FP32 or hi/lo red-black sweeps whose blocks
// have the same length run instead as graphs of multi-grid launches (one
// launch per colour pass walks the work items of a table of grids) -- then
// reduces the residuals of all active grids in one batched pass and applies
// each grid's own decisions.
// Every grid gets the bits of its own passes, so it takes exactly the path of
// its solo solve.
// ===========================================================================
struct ServerEntry {
    fld_grid_s *g = nullptr;
    long long tag = 0;
    cudaStream_t own_stream = nullptr;
    Controller ctl;
    Family fam = FAM_F32;
    PassParams pp{};
    int ce = 64;                  // iterations between checks
    int warm = 0;                 // warm-up iterations at omega = 1
    Family snap_fam = FAM_F32;
    bool snap_lo = false;
    fld_solve_result res{};
    std::chrono::steady_clock::time_point t_add;
    // Anderson mixing, as in fld_solve
    int am = 0;
    double gram[kAndersonMax][kAndersonMax] = {};
    int acount = 0;
    bool have_x = false;
    bool mix_off = false;         // mixing given up after a stall
};

namespace {
// Multi-grid tables a server step can fill (groups of grids with equal block
// lengths; a further group runs grid by grid).
constexpr int kFuseSlots = 8;

// The state the Anderson kernels read and write for family fam.
void anderson_state(fld_grid_s *g, Family fam, float **hi, float **lo, double **p64) {
    const bool d = fam == FAM_F64;
    *hi = d ? nullptr : g->f.phi;
    *lo = !d && g->lo_live ? g->f.phlo : nullptr;
    *p64 = d ? g->f.phi64 : nullptr;
}
}  // namespace

struct fld_server_s {
    int device = 0;
    cudaStream_t bs = nullptr;
    bool own_bs = false;
    fld_solve_params p{};
    double sw = 2e-5;
    std::vector<ServerEntry> active;
    std::vector<ServerEntry> done;      // finished, not yet reported
    BatchDesc *d_desc = nullptr;
    int *d_res = nullptr, *d_count = nullptr;
    double *d_part = nullptr, *d_out = nullptr;
    int cap_grids = 0, cap_res = 0;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    long long launches = 0;
    long long updates = 0;              // voxel updates of all steps so far
    // multi-grid launches (batch_launch): kFuseSlots device tables of
    // SweepDescs with their counts, and the block graphs captured over them,
    // keyed by (table, iterations)
    SweepDesc *d_sweep[kFuseSlots] = {};
    int *d_sweep_count[kFuseSlots] = {};
    std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> multi_graphs;
    int nsm = 0;
};

namespace {

void server_free_workspace(fld_server_s *s) {
    void *ptrs[] = {s->d_desc, s->d_res, s->d_count, s->d_part, s->d_out};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    s->d_desc = nullptr; s->d_res = nullptr; s->d_count = nullptr; s->d_part = nullptr; s->d_out = nullptr;
    s->cap_grids = s->cap_res = 0;
}

fld_status server_workspace(fld_server_s *s, int grids, int res) {
    if (grids <= s->cap_grids && res <= s->cap_res) return FLD_OK;
    FLD_CK(cudaStreamSynchronize(s->bs));
    server_free_workspace(s);
    const int cg = grids + grids / 2 + 4, cr = res + res / 2 + 64;
    if (cudaMalloc((void **)&s->d_desc, sizeof(BatchDesc) * cg) != cudaSuccess ||
        cudaMalloc((void **)&s->d_res, sizeof(int) * (size_t)cr) != cudaSuccess ||
        cudaMalloc((void **)&s->d_count, sizeof(int) * cg) != cudaSuccess ||
        cudaMalloc((void **)&s->d_part, sizeof(double) * 2 * (size_t)cr) != cudaSuccess ||
        cudaMalloc((void **)&s->d_out, sizeof(double) * 2 * cg) != cudaSuccess) {
        (void)cudaGetLastError();
        server_free_workspace(s);
        return fail(FLD_ERR_OOM, "cudaMalloc of the batch workspace failed");
    }
    s->cap_grids = cg;
    s->cap_res = cr;
    return FLD_OK;
}

double rel_from_sums(const fld_grid_s *g, int margin, double r2, double j2) {
    return rel_residual_from_sums(g->nx, g->ny, g->nz, g->h, margin, r2, j2);
}

void server_retire(fld_server_s *s, size_t i, fld_status st, double rel) {
    ServerEntry &e = s->active[i];
    e.res.status = st;
    e.res.rel_residual = rel;
    e.res.omega = e.pp.omega;
    e.res.omega_backoffs = e.ctl.backoffs;
    e.res.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - e.t_add).count();
    e.g->valid_float = true;
    e.g->valid_d = false;
    e.g->stream = e.own_stream;
    s->done.push_back(e);
    s->active.erase(s->active.begin() + (long)i);
}

// The device tables of the multi-grid launches (allocated on first use).
fld_status server_multi_tables(fld_server_s *s) {
    if (s->d_sweep[0]) return FLD_OK;
    for (int i = 0; i < kFuseSlots; ++i) {
        if (cudaMalloc((void **)&s->d_sweep[i], sizeof(SweepDesc) * kMultiMaxGrids) != cudaSuccess ||
            cudaMalloc((void **)&s->d_sweep_count[i], sizeof(int) * 2) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(FLD_ERR_OOM, "cudaMalloc of the multi-grid tables failed");
        }
    }
    if (cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        (void)cudaGetLastError();
        s->nsm = 1;
    }
    return FLD_OK;
}

// The table row of one grid for a block starting at its current iteration
// (first: its first work item in the table).
SweepDesc sweep_desc(const ServerEntry &e, int first) {
    const fld_grid_s *g = e.g;
    const PassParams q = block_params(e.pp, e.res.iterations, e.warm);
    SweepDesc d;
    memset(&d, 0, sizeof(d));
    d.L = g->L;
    d.sp = g->f.sp; d.ah2 = g->f.ah2; d.jh2 = g->f.jh2;
    d.phi = g->f.phi; d.phlo = g->f.phlo; d.D = g->f.D;
    d.spb = q.bf16 ? g->f.spb : nullptr;
    d.sab = q.bf16 ? g->f.sab : nullptr;
    d.h2 = (float)q.h2;
    d.omega = (float)q.omega;
    d.inv2h = (float)q.inv2h;
    d.floor_ = (float)q.floor_;
    d.larsen_n = (float)q.larsen_n;
    d.lim = q.lim;
    d.local_iters = q.local_iters;
    d.hl = e.fam == FAM_FH ? 1 : 0;
    d.first = first;
    multi_dims(g->L, &d.bx, &d.by);
    return d;
}

// One block of k iterations of the grids in table `tab` (rows from
// sweep_desc, all in FP32 or hi/lo red-black sweeps; items work items in all)
// as multi-grid launches on stream st: the table goes to slot `slot`, then
// the slot's graph of 2k launches runs (captured on first use).
fld_status server_multi_block(fld_server_s *s, int slot, const std::vector<SweepDesc> &tab, int items, int k,
                              int share, cudaStream_t st) {
    const int counts[2] = {(int)tab.size(), items};
    const int hl = tab[0].hl, bf = tab[0].spb != nullptr, lim = tab[0].lim, li = tab[0].local_iters;
    // persistent: the table's share of the CTAs resident at once (one CTA per
    // item in a power-of-two grid measured slower still: 1.86 against 1.77 s
    // for 32 grids of 32^3 to 64^3)
    const int nctas = std::max(1, multi_ctas(s->nsm, hl, bf, lim, li) / std::max(1, share));
    FLD_CK(cudaMemcpyAsync(s->d_sweep[slot], tab.data(), sizeof(SweepDesc) * tab.size(), cudaMemcpyHostToDevice, st));
    FLD_CK(cudaMemcpyAsync(s->d_sweep_count[slot], counts, sizeof(counts), cudaMemcpyHostToDevice, st));
    const std::tuple<int, int, int, int> key(slot, k, nctas, hl);
    auto it = s->multi_graphs.find(key);
    if (it == s->multi_graphs.end()) {
        cudaGraph_t graph = nullptr;
        FLD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        for (int i = 0; i < k && ce == cudaSuccess; ++i)
            for (int colour = 0; colour < 2 && ce == cudaSuccess; ++colour)
                ce = launch_pass_multi(s->d_sweep[slot], s->d_sweep_count[slot], hl, bf, lim, li, colour, nctas, st);
        const cudaError_t ce2 = cudaStreamEndCapture(st, &graph);
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ce != cudaSuccess ? ce : ce2, "capture of the multi-grid block");
        }
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate (multi-grid block)");
        it = s->multi_graphs.emplace(key, exec).first;
    }
    FLD_CK(cudaGraphLaunch(it->second, st));
    s->launches += 2LL * k;
    return FLD_OK;
}

}  // namespace

fld_status fld_server_create(const fld_solve_params *p, void *stream, fld_server *out) {
    if (!out) return fail(FLD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(FLD_ERR_INVALID_ARG, "params is NULL");
    if (p->precision == FLD_PREC_FP64 || p->precision < 0 || p->precision > FLD_PREC_PAIR)
        return fail(FLD_ERR_INVALID_ARG, "the server runs the FP32 / MIXED / PAIR sweeps; use fld_solve for FP64");
    if (p->anderson < 0 || p->anderson > kAndersonMax) return fail(FLD_ERR_INVALID_ARG, "anderson must lie in [0, 16]");
    if (p->anderson > 0 && p->scheme == FLD_SCHEME_JACOBI)
        return fail(FLD_ERR_INVALID_ARG, "Anderson mixing accelerates the red-black scheme only");
    if (const char *bad = check_limiter_margin(p->limiter, p->larsen_n, p->residual_margin))
        return fail(FLD_ERR_INVALID_ARG, bad);
    if (p->temporal_depth < -1 || p->temporal_depth == 3 || p->temporal_depth > 4 || p->tile_y < 0)
        return fail(FLD_ERR_INVALID_ARG, "temporal_depth must be -1, 0, 1, 2 or 4 and tile_y >= 0");
    if (p->fp64_verify != 0 && p->fp64_verify != 1) return fail(FLD_ERR_INVALID_ARG, "fp64_verify must be 0 or 1");
    if (p->batch_launch != 0 && p->batch_launch != 1) return fail(FLD_ERR_INVALID_ARG, "batch_launch must be 0 or 1");
    if (p->omega > 0.0 && !(p->omega < 2.0)) return fail(FLD_ERR_INVALID_ARG, "omega must lie in (0, 2)");
    if (p->local_iters > 64) return fail(FLD_ERR_INVALID_ARG, "local_iters must be <= 64");
    if (!(p->tol >= 0.0) || p->max_iters < 0 || p->check_every < 0)
        return fail(FLD_ERR_INVALID_ARG, "bad tol / max_iters / check_every");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        (void)cudaGetLastError();
        return fail(FLD_ERR_NO_DEVICE, "no CUDA device available");
    }
    fld_server_s *s = new (std::nothrow) fld_server_s();
    if (!s) return fail(FLD_ERR_OOM, "host allocation failed");
    s->p = *p;
    s->sw = p->fp32_switch > 0.0 ? p->fp32_switch : 2e-5;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        if (stream) {
            s->bs = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreate(&s->bs);
            s->own_bs = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    const int nside = 16;
    for (int i = 0; i < nside && e == cudaSuccess; ++i) {
        cudaStream_t ss = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (ss) s->side.push_back(ss);
        if (ev) s->join.push_back(ev);
    }
    if (e != cudaSuccess) {
        fld_server_destroy(s);
        return cuda_fail(e, "server setup");
    }
    *out = s;
    return FLD_OK;
}

void fld_server_destroy(fld_server s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->bs) cudaStreamSynchronize(s->bs);
    for (ServerEntry &e : s->active) e.g->stream = e.own_stream;   // grids go back to their owners
    server_free_workspace(s);
    for (auto &kv : s->multi_graphs) cudaGraphExecDestroy(kv.second);
    for (int i = 0; i < kFuseSlots; ++i) {
        if (s->d_sweep[i]) cudaFree(s->d_sweep[i]);
        if (s->d_sweep_count[i]) cudaFree(s->d_sweep_count[i]);
    }
    for (auto x : s->side) cudaStreamDestroy(x);
    for (auto x : s->join) cudaEventDestroy(x);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->own_bs && s->bs) cudaStreamDestroy(s->bs);
    delete s;
}

fld_status fld_server_add(fld_server s, fld_grid g, long long tag) {
    if (!s || !g) return fail(FLD_ERR_INVALID_ARG, "server or grid is NULL");
    if (g->device != s->device) return fail(FLD_ERR_INVALID_ARG, "the grid lives on another device");
    for (const ServerEntry &e : s->active)
        if (e.g == g) return fail(FLD_ERR_INVALID_ARG, "the grid is already being solved");
    fld_status st = enter(g);
    if (st != FLD_OK) return st;
    const fld_solve_params *p = &s->p;
    ServerEntry e;
    e.g = g;
    e.tag = tag;
    e.t_add = std::chrono::steady_clock::now();
    FLD_CK(cudaStreamSynchronize(g->stream));
    e.fam = start_family(p->precision);
    if ((st = prepare(g, p, e.fam)) != FLD_OK) return st;
    if (!p->warm_start) {
        if ((st = init_state(g, p, e.fam)) != FLD_OK) return st;
    } else if (p->precision == FLD_PREC_MIXED && !g->valid_d && g->lo_live) {
        e.fam = FAM_FF;
    }
    if ((st = sync_family(g, e.fam)) != FLD_OK) return st;
    e.pp = pass_params(g, p);
    if ((st = choose_sweeps(g, p, &e.pp, &e.ce)) != FLD_OK) return st;
    e.warm = warmup_of(g, p);
    e.am = p->anderson;
    if (e.am > 0 && (st = ensure_anderson(g, e.am)) != FLD_OK) return st;
    if ((st = preallocate(g, p)) != FLD_OK) return st;
    e.ctl.precision = p->precision;
    if (p->anderson <= 1) e.ctl.scale_windows(std::max(g->nx, std::max(g->ny, g->nz)), e.ce);
    e.ctl.tol = p->tol;
    e.ctl.sw = s->sw;
    e.ctl.fam = e.fam;
    memset(&e.res, 0, sizeof(e.res));
    e.res.jbar = g->jbar;
    e.res.omega = e.pp.omega;
    // the first check, as in fld_solve
    double rel = 0.0;
    if ((st = residual_now(g, e.fam, e.pp, p->residual_margin, &rel)) != FLD_OK) return st;
    e.res.checks = 1;
    e.res.rel_residual = rel;
    e.own_stream = g->stream;
    Action a = e.ctl.first(rel);
    if (a == ACT_CONVERGED && p->precision == FLD_PREC_MIXED && p->fp64_verify && e.fam != FAM_F64) {
        // the stop test in FP64, as in fld_solve
        double r64 = 0.0;
        if ((st = fp64_check(g, p, e.pp, &r64)) != FLD_OK) return st;
        ++e.res.checks;
        e.res.rel_residual_single = rel;
        e.res.rel_residual = rel = r64;
        e.fam = FAM_F64;
        e.ctl.enter_fp64(r64, std::max(g->nx, std::max(g->ny, g->nz)), p->anderson <= 1);
        if (r64 <= p->tol) {
            if ((st = sync_family(g, FAM_FF)) != FLD_OK) return st;
        } else {
            a = ACT_SAVE;
        }
    }
    if (a == ACT_SAVE) {
        if ((st = snapshot(g, e.fam, true)) != FLD_OK) return st;
        e.snap_fam = e.fam;
        e.snap_lo = g->lo_live;
    }
    FLD_CK(cudaStreamSynchronize(g->stream));
    g->stream = s->bs;   // from here on the grid's work is ordered on the server stream
    s->active.push_back(e);
    if (a == ACT_CONVERGED) server_retire(s, s->active.size() - 1, FLD_OK, rel);
    else if (a == ACT_DIVERGED) server_retire(s, s->active.size() - 1, FLD_ERR_DIVERGED, rel);
    return FLD_OK;
}

fld_status fld_server_updates(fld_server s, long long *updates) {
    if (!s || !updates) return fail(FLD_ERR_INVALID_ARG, "server or updates is NULL");
    *updates = s->updates;
    return FLD_OK;
}

fld_status fld_server_active(fld_server s, int *count) {
    if (!s || !count) return fail(FLD_ERR_INVALID_ARG, "server or count is NULL");
    *count = (int)s->active.size();
    return FLD_OK;
}

fld_status fld_server_step(fld_server s, long long *tags, fld_solve_result *results, int capacity, int *nfinished) {
    if (!s || !nfinished) return fail(FLD_ERR_INVALID_ARG, "server or nfinished is NULL");
    if (capacity > 0 && (!tags || !results)) return fail(FLD_ERR_INVALID_ARG, "tags / results are NULL");
    *nfinished = 0;
    FLD_CK(cudaSetDevice(s->device));
    const fld_solve_params *p = &s->p;
    fld_status st = FLD_OK;
    const size_t n = s->active.size();
    if (n > 0) {
        // -- one block of iterations per active grid, grids spread over the pool
        FLD_CK(cudaEventRecord(s->fork, s->bs));
        const size_t nside = s->side.size() < n ? s->side.size() : n;
        for (size_t i = 0; i < nside; ++i) FLD_CK(cudaStreamWaitEvent(s->side[i], s->fork, 0));
        std::vector<int> k(n);
        std::vector<char> mixing(n, 0);
        for (size_t i = 0; i < n; ++i) {
            const ServerEntry &e = s->active[i];
            k[i] = block_len(e.res.iterations, check_len(e.fam, p->precision, e.ce), p->max_iters, e.warm);
        }
        // multi-grid launches: grids in FP32 / hi-lo red-black sweeps grouped
        // by block length; each group of two grids or more is split into
        // tables (at most kFuseSlots in all, two grids or more each, balanced
        // by voxels) that run on different streams, so the passes of one
        // table overlap the tails of another's; the rest run grid by grid
        std::vector<int> slot_of(n, -1);
        std::vector<std::pair<int, std::vector<size_t>>> groups;   // (block length, grids) per table
        if (p->batch_launch && p->scheme != FLD_SCHEME_JACOBI) {
            // (grids of one table share their family: block length and family as key)
            std::map<std::pair<int, int>, std::vector<size_t>> by_k;
            for (size_t i = 0; i < n; ++i) {
                const Family f = s->active[i].fam;
                if (k[i] > 0 && (f == FAM_F32 || f == FAM_FH)) by_k[{k[i], (int)f}].push_back(i);
            }
            std::vector<std::pair<std::pair<int, int>, std::vector<size_t>>> cand;
            for (auto &kv : by_k)
                if (kv.second.size() >= 2) cand.push_back(kv);
            std::stable_sort(cand.begin(), cand.end(),
                             [](const auto &a, const auto &b) { return a.second.size() > b.second.size(); });
            size_t total = 0;
            for (const auto &c : cand) total += c.second.size();
            for (const auto &c : cand) {
                const size_t left = (size_t)kFuseSlots - groups.size();
                if (left == 0) break;
                size_t parts = std::max<size_t>(1, (size_t)kFuseSlots * c.second.size() / std::max<size_t>(total, 1));
                parts = std::min(parts, std::min(left, c.second.size() / 2));
                if (parts == 0) parts = 1;
                // largest grids first, each to the part with the fewest voxels
                std::vector<size_t> mem = c.second;
                std::stable_sort(mem.begin(), mem.end(),
                                 [&](size_t a, size_t b) { return nvox(s->active[a].g) > nvox(s->active[b].g); });
                std::vector<long long> load(parts, 0);
                std::vector<std::vector<size_t>> part(parts);
                for (size_t i : mem) {
                    const size_t j = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
                    if (part[j].size() >= (size_t)kMultiMaxGrids) continue;
                    part[j].push_back(i);
                    load[j] += nvox(s->active[i].g);
                }
                for (auto &q : part) {
                    std::sort(q.begin(), q.end());
                    if (q.size() >= 2) groups.push_back({c.first.first, q});
                }
            }
            if (!groups.empty() && (st = server_multi_tables(s)) != FLD_OK) return st;
            for (size_t gi = 0; gi < groups.size(); ++gi)
                for (size_t i : groups[gi].second) slot_of[i] = (int)gi;
        }
        // each table's persistent grid gets its share of the resident CTAs (a quarter at least)
        const int share = std::min((int)groups.size(), 4);
        std::vector<std::vector<SweepDesc>> tables(groups.size());
        std::vector<int> table_items(groups.size(), 0);
        size_t solo = 0;
        for (size_t i = 0; i < n; ++i) {
            ServerEntry &e = s->active[i];
            if (k[i] <= 0) continue;
            e.g->stream = slot_of[i] >= 0 ? s->side[(size_t)slot_of[i] % nside]
                                          : s->side[(groups.size() + solo++) % nside];
            // Anderson: after the warm-up each block starts from the mix of
            // the last am images (the history starts from the state here)
            mixing[i] = e.am > 0 && e.res.iterations >= e.warm && !e.mix_off;
            if (mixing[i] && !e.have_x) {
                float *hi, *lo;
                double *p64;
                anderson_state(e.g, e.fam, &hi, &lo, &p64);
                const cudaError_t ce = launch_anderson_capture(e.g->anderson, e.g->L.total, hi, lo, p64, e.g->nsm,
                                                               e.g->stream);
                if (ce != cudaSuccess) {
                    e.g->stream = s->bs;
                    return cuda_fail(ce, "launch_anderson_capture");
                }
                s->launches += 1;
                e.have_x = true;
                e.acount = 0;
            }
            if (slot_of[i] < 0) {
                st = run_block(e.g, e.fam, block_params(e.pp, e.res.iterations, e.warm), k[i]);
                s->launches += 2LL * k[i];
            } else {
                std::vector<SweepDesc> &tab = tables[(size_t)slot_of[i]];
                int &items = table_items[(size_t)slot_of[i]];
                tab.push_back(sweep_desc(e, items));
                items += tab.back().bx * tab.back().by * e.g->nz;
            }
            e.g->stream = s->bs;
            if (st != FLD_OK) return st;
            s->updates += (long long)k[i] * nvox(e.g);
            e.res.iterations += k[i];
            if (e.fam == FAM_F32) e.res.iterations_fp32 += k[i];
            else if (e.fam == FAM_FH) e.res.iterations_mid += k[i];
            else if (e.fam == FAM_F64) e.res.iterations_fp64 += k[i];
            else e.res.iterations_corr += k[i];
        }
        for (size_t gi = 0; gi < groups.size(); ++gi)
            if ((st = server_multi_block(s, (int)gi, tables[gi], table_items[gi], groups[gi].first, share,
                                         s->side[gi % nside])) != FLD_OK)
                return st;
        for (size_t i = 0; i < nside; ++i) {
            FLD_CK(cudaEventRecord(s->join[i], s->side[i]));
            FLD_CK(cudaStreamWaitEvent(s->bs, s->join[i], 0));
        }
        // -- residuals of all active grids in one batched pass
        // (grids in their FP64 sweeps are checked one by one, as fld_solve does)
        std::vector<BatchDesc> hd(n);
        std::vector<int> res_tab, res_count(n);
        int slots = 0;
        for (size_t i = 0; i < n; ++i) {
            const ServerEntry &e = s->active[i];
            BatchDesc &d = hd[i];
            if (e.fam == FAM_F64) {
                memset(&d, 0, sizeof(d));
                res_count[i] = 0;
                continue;
            }
            memset(&d, 0, sizeof(d));
            d.L = e.g->L;
            d.sp = e.g->f.sp; d.ah2 = e.g->f.ah2; d.jh2 = e.g->f.jh2; d.phi = e.g->f.phi; d.phlo = e.g->f.phlo;
            d.D = e.g->f.D; d.Df = e.g->f.Df;
            d.inv2h = (float)e.pp.inv2h; d.floor_ = (float)e.pp.floor_;
            d.larsen_n = (float)e.pp.larsen_n; d.lim = e.pp.lim;
            d.mode = e.fam == FAM_F32 ? 0 : 1;
            d.active = 1;
            residual_dims(e.g->L, &d.res_bx, &d.res_by);
            res_count[i] = d.res_bx * d.res_by * e.g->nz;
            d.res_first = (int)res_tab.size();
            d.res_slot = slots;
            slots += res_count[i];
            res_tab.insert(res_tab.end(), (size_t)res_count[i], (int)i);
        }
        if ((st = server_workspace(s, (int)n, slots)) != FLD_OK) return st;
        FLD_CK(cudaMemcpyAsync(s->d_desc, hd.data(), sizeof(BatchDesc) * n, cudaMemcpyHostToDevice, s->bs));
        FLD_CK(cudaMemcpyAsync(s->d_res, res_tab.data(), sizeof(int) * res_tab.size(), cudaMemcpyHostToDevice, s->bs));
        FLD_CK(cudaMemcpyAsync(s->d_count, res_count.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->bs));
        FLD_CK(launch_residual_batch(s->d_desc, s->d_res, (int)res_tab.size(), (int)n, s->d_count, s->d_part,
                                     s->d_out, p->limiter, p->residual_margin, s->bs));
        s->launches += 3;
        std::vector<double> out(2 * n);
        FLD_CK(cudaMemcpyAsync(out.data(), s->d_out, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s->bs));
        FLD_CK(cudaStreamSynchronize(s->bs));
        std::vector<double> rel64(n, 0.0);
        for (size_t i = 0; i < n; ++i) {
            ServerEntry &e = s->active[i];
            if (e.fam != FAM_F64) continue;
            if ((st = residual_now(e.g, FAM_F64, e.pp, p->residual_margin, &rel64[i])) != FLD_OK) return st;
            s->launches += 3;
        }
        // -- each grid's own decisions (same as fld_solve)
        std::vector<std::pair<size_t, std::pair<fld_status, double>>> retire;
        std::vector<char> mix_now(n, 0);
        for (size_t i = 0; i < n; ++i) {
            ServerEntry &e = s->active[i];
            fld_grid_s *g = e.g;
            double rel = e.fam == FAM_F64 ? rel64[i] : rel_from_sums(g, p->residual_margin, out[2 * i], out[2 * i + 1]);
            e.res.rel_residual = rel;
            ++e.res.checks;
            const Action a = (e.warm > 0 && e.res.iterations == e.warm) ? e.ctl.restart(rel)
                                                                         : e.ctl.next(rel, e.pp.omega);
            switch (a) {
            case ACT_CONVERGED:
                if (p->precision == FLD_PREC_MIXED && p->fp64_verify && e.fam != FAM_F64) {
                    // the stop test in FP64, as in fld_solve
                    double r64 = 0.0;
                    if ((st = fp64_check(g, p, e.pp, &r64)) != FLD_OK) return st;
                    s->launches += 5;
                    ++e.res.checks;
                    e.res.rel_residual_single = rel;
                    e.res.rel_residual = rel = r64;
                    e.fam = FAM_F64;
                    e.ctl.enter_fp64(r64, std::max(g->nx, std::max(g->ny, g->nz)), e.am <= 1 || e.mix_off);
                    if (r64 <= p->tol) retire.push_back({i, {FLD_OK, rel}});
                } else {
                    retire.push_back({i, {FLD_OK, rel}});
                }
                break;
            case ACT_DIVERGED: retire.push_back({i, {FLD_ERR_DIVERGED, rel}}); break;
            case ACT_STALLED:
                if (e.am > 1 && !e.mix_off && e.res.iterations < p->max_iters) {
                    // as fld_solve: plain sweeps from the best state
                    if ((st = snapshot(g, e.snap_fam, false)) != FLD_OK) return st;
                    e.fam = e.snap_fam;
                    e.ctl.fam = e.fam;
                    set_valid(g, e.fam);
                    g->lo_live = e.snap_lo;
                    e.res.rel_residual = rel = e.ctl.best;
                    e.mix_off = true;
                    e.have_x = false;
                    e.ctl.scale_windows(std::max(g->nx, std::max(g->ny, g->nz)),
                                        check_len(e.fam, p->precision, e.ce));
                    e.ctl.backoffs = 0;
                    e.ctl.begin_phase();
                    ++e.res.anderson_resets;
                } else {
                    retire.push_back({i, {FLD_ERR_NOT_CONVERGED, rel}});
                }
                break;
            case ACT_SAVE:
                if ((st = snapshot(g, e.fam, true)) != FLD_OK) return st;
                e.snap_fam = e.fam;
                e.snap_lo = g->lo_live;
                break;
            case ACT_RESTORE:
                if ((st = snapshot(g, e.snap_fam, false)) != FLD_OK) return st;
                e.fam = e.snap_fam;
                e.ctl.fam = e.fam;
                set_valid(g, e.fam);
                g->lo_live = e.snap_lo;
                e.pp.omega = 1.0 + 0.97 * (e.pp.omega - 1.0);
                break;
            case ACT_SWITCH:
                e.fam = next_family(e.fam);
                if ((st = sync_family(g, e.fam)) != FLD_OK) return st;
                e.ctl.fam = e.fam;
                e.ctl.begin_phase();
                break;
            case ACT_CONTINUE: break;
            }
            if (a != ACT_CONVERGED && a != ACT_DIVERGED && a != ACT_STALLED && e.res.iterations >= p->max_iters)
                retire.push_back({i, {FLD_ERR_NOT_CONVERGED, rel}});
            if (a == ACT_RESTORE || a == ACT_SWITCH || a == ACT_CONVERGED) e.have_x = false;
            // Anderson step after a block that made ordinary progress (as in fld_solve)
            mix_now[i] = mixing[i] && e.have_x && (a == ACT_CONTINUE || a == ACT_SAVE) &&
                         e.res.iterations < p->max_iters;
        }
        // -- Anderson: collect every mixing grid's image and dot products, one
        // readback, then each grid's weights and mix (same kernels and order
        // as fld_solve, so a grid's iterates are those of its solo solve)
        std::vector<double> dots(n * kAndersonMax);
        bool any_mix = false;
        for (size_t i = 0; i < n; ++i) {
            if (!mix_now[i]) continue;
            ServerEntry &e = s->active[i];
            const int slot = e.acount % e.am;
            const int w = e.acount + 1 < e.am ? e.acount + 1 : e.am;
            float *hi, *lo;
            double *p64;
            anderson_state(e.g, e.fam, &hi, &lo, &p64);
            FLD_CK(launch_anderson_collect(e.g->anderson, e.g->L.total, hi, lo, p64, slot, w, e.g->nsm, s->bs));
            FLD_CK(cudaMemcpyAsync(&dots[i * kAndersonMax], e.g->anderson.dots, sizeof(double) * w,
                                   cudaMemcpyDeviceToHost, s->bs));
            s->launches += 2;
            any_mix = true;
        }
        if (any_mix) FLD_CK(cudaStreamSynchronize(s->bs));
        for (size_t i = 0; i < n; ++i) {
            if (!mix_now[i]) continue;
            ServerEntry &e = s->active[i];
            const int slot = e.acount % e.am;
            ++e.acount;
            const int w = e.acount < e.am ? e.acount : e.am;
            for (int j = 0; j < w; ++j) e.gram[slot][j] = e.gram[j][slot] = dots[i * kAndersonMax + j];
            double wts[kAndersonMax];
            bool ok = true;
            if (w == 1) wts[0] = 1.0;
            else ok = anderson_weights(e.gram, w, wts);
            if (ok) {
                float *hi, *lo;
                double *p64;
                anderson_state(e.g, e.fam, &hi, &lo, &p64);
                FLD_CK(launch_anderson_mix(e.g->anderson, e.g->L.total, slot, w, wts, hi, lo, p64, e.g->nsm, s->bs));
                s->launches += 1;
                if (w > 1) ++e.res.anderson_steps;
            } else {
                ++e.res.anderson_resets;
                e.have_x = false;
            }
        }
        for (size_t r = retire.size(); r-- > 0;) {
            ServerEntry &e = s->active[retire[r].first];
            if (e.fam == FAM_F64 && (st = sync_family(e.g, FAM_FF)) != FLD_OK) return st;   // as fld_solve
            e.res.kernels = s->launches;
            server_retire(s, retire[r].first, retire[r].second.first, retire[r].second.second);
        }
        FLD_CK(cudaStreamSynchronize(s->bs));
    }
    // -- report finished grids (oldest first)
    int m = 0;
    while (m < capacity && !s->done.empty()) {
        tags[m] = s->done.front().tag;
        results[m] = s->done.front().res;
        s->done.erase(s->done.begin());
        ++m;
    }
    *nfinished = m;
    return FLD_OK;
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
    if (p->max_iters < 0 || p->check_every < 0) return fail(FLD_ERR_INVALID_ARG, "bad max_iters / check_every");
    // Grids of one group should keep their per-iteration working set (24 bytes
    // per voxel: sigma', sigma_a', j, phi hi/lo, D) within L2.  Grids are taken
    // in order of size and packed greedily into groups of at most 3/4 of the
    // L2 capacity; groups run one after another, small grids share steps.
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
    fld_server srv = nullptr;
    if ((st = fld_server_create(p, grids[0]->stream, &srv)) != FLD_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    size_t a = 0;
    std::vector<long long> tags(count);
    std::vector<fld_solve_result> fin(count);
    while (a < order.size() && st == FLD_OK) {
        double ws = 0.0;
        int in_group = 0;
        const double off = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        while (a < order.size()) {
            const double w = 24.0 * (double)nvox(grids[order[a]]);
            if (in_group > 0 && ws + w > budget) break;
            if ((st = fld_server_add(srv, grids[order[a]], order[a])) != FLD_OK) break;
            ws += w;
            ++in_group;
            ++a;
        }
        int left = in_group;
        while (st == FLD_OK && left > 0) {
            int nf = 0;
            if ((st = fld_server_step(srv, tags.data(), fin.data(), count, &nf)) != FLD_OK) break;
            for (int b = 0; b < nf; ++b) {
                res[tags[b]] = fin[b];
                res[tags[b]].ms += off;
            }
            left -= nf;
        }
    }
    fld_server_destroy(srv);
    if (st != FLD_OK) return st;
    fld_status worst = FLD_OK;
    for (int b = 0; b < count; ++b) {
        if (res[b].status == FLD_ERR_DIVERGED) worst = FLD_ERR_DIVERGED;
        else if (res[b].status != FLD_OK && worst == FLD_OK) worst = FLD_ERR_NOT_CONVERGED;
        if (results) results[b] = res[b];
    }
    if (worst != FLD_OK) g_last_error = "not every solve of the batch converged (see the per-grid results)";
    return worst;
}

}  // extern "C"
