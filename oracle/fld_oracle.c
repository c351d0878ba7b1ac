/*
 * fld_oracle.c -- FP64 CPU oracle for flux-limited diffusion (FLD).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes follows Koerner, Portsmouth, Sadlo, Ertl, Eberhardt,
 * "Flux-Limited Diffusion for Multiple Scattering in Participating Media",
 * Computer Graphics Forum 33(2), 2014:
 *
 *   - flux limiters F(R), Table 2 ("sum", "max", Kershaw, Larsen-n,
 *     Levermore-Pomraning) and the CDA constant 1/3 (Sec. 4, after Eq. 15);
 *   - the extinction floor sigma <- max(sigma, sigma_eps) and the RMS emission
 *     jbar (Algorithm 1, first steps; Sec. 5 on sigma_eps = 1e-3/L);
 *   - one red-black Gauss-Seidel iteration with over-relaxation: for every
 *     non-boundary point of one colour, the Knudsen number R (Eq. 35, the
 *     floored form of Eq. 16, with the central gradient of Eq. 34), the
 *     diffusion coefficient D_p (Eq. 33), the face coefficients
 *     D_ps = (D_p + D_s)/2, the local update phi' (Eq. 32) and the SOR
 *     blend (Eq. 36); then the other colour (Algorithm 1);
 *   - the residual R_p = (numerator - phi_p * denominator)/dl^2 (Eq. 37) of
 *     the discrete equation (Eq. 31) and its RMS relative to jbar;
 *   - the single-scatter source q_ri = L sigma_s T for a directional light
 *     (Sec. 3, after Eq. 6) with the transmittance of Eq. 3 evaluated by a
 *     ray march, and its point-light generalisation.
 *
 * Everything is double precision.  No blocking, fusion or reordering beyond
 * what Algorithm 1 states: points of one colour read only the other colour
 * and their own values, so updating them in place in any order (or on
 * several threads) gives the same result as the paper's parallel-for.
 *
 * Storage: phi and D live on a padded grid with one ghost layer,
 *   (nx+2) x (ny+2) x (nz+2), x fastest, index ((K*(ny+2)+J)*(nx+2)+I) with
 *   I = i+1 etc.; the ghost layer is the Dirichlet boundary and is never
 *   updated.  Medium fields (sigma', sigma_a', j) are unpadded nx*ny*nz.
 *
 * Readings of points where the paper is silent are listed in the project's
 * design notes; the ones that matter here:
 *   - s(p) is the six face neighbours (7-point stencil);
 *   - colour "red" is (i+j+k) even in unknown indices, red pass first;
 *   - R uses the old phi_p of the point being updated (Algorithm 1 order);
 *     with local_iters = k > 1 the steps Knudsen -> D_p -> D_ps -> phi' are
 *     repeated k times for the point, each round using the previous round's
 *     phi' in R, before the SOR blend with the old phi_p.  The fixed point
 *     (Eq. 31 with D from Eq. 33-35) is unchanged; only the path differs;
 *   - the convergence test uses a freshly computed D from the current phi
 *     (the in-pass residual of Algorithm 1 goes stale after the next pass);
 *   - when jbar = 0 (no emission anywhere) the floor eps*jbar of Eq. 35 is
 *     replaced by 1e-30 and the relative residual is reported as the
 *     absolute RMS residual.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FLDO_LIM_CDA 0
#define FLDO_LIM_SUM 1
#define FLDO_LIM_MAX 2
#define FLDO_LIM_KERSHAW 3
#define FLDO_LIM_LARSEN 4
#define FLDO_LIM_LP 5

/* Floor of Eq. 35 when there is no emission at all (jbar = 0, so eps*jbar
 * would be 0 and R could be 0/0): a fixed small positive value. */
#define FLDO_FLOOR_NO_EMISSION 1e-30

typedef struct {
    int nx, ny, nz;
    double h;          /* voxel edge length, Delta l */
    int limiter;       /* FLDO_LIM_* */
    double larsen_n;   /* n of Larsen-n */
    double eps;        /* epsilon of Eq. 35 (paper: 1e-20) */
    double jbar;       /* RMS of j over the unknowns */
    double omega;      /* SOR factor, 0 < omega < 2 */
    int nthreads;      /* worker threads for the parallel-for over z planes */
    int local_iters;   /* times the point update (Knudsen -> D_p -> D_ps -> phi')
                          is applied before the SOR blend; 1 = Algorithm 1 */
} fldo_cfg;

/* ------------------------------------------------------------------------ */
/* Flux limiters, Table 2.                                                   */
/* ------------------------------------------------------------------------ */

/* Levermore-Pomraning F(R) = (coth R - 1/R)/R.  For small R the direct form
 * cancels, so below R = 0.2 the Laurent series of coth is used:
 *   coth x = 1/x + sum_{n>=1} 2^{2n} B_{2n} x^{2n-1} / (2n)!
 * hence F(R) = sum_{n>=1} c_n R^{2n-2} with c_n = 2^{2n} B_{2n}/(2n)!,
 * B_2..B_16 = 1/6, -1/30, 1/42, -1/30, 5/66, -691/2730, 7/6, -3617/510. */
static double lp_limiter(double R)
{
    if (R < 0.2) {
        static const double B[8] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0,
                                    5.0 / 66.0, -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0};
        double c[8];
        double pow4 = 1.0, fact = 1.0;
        for (int n = 1; n <= 8; ++n) {
            pow4 *= 4.0;
            fact *= (double)(2 * n - 1) * (double)(2 * n);
            c[n - 1] = pow4 * B[n - 1] / fact;
        }
        double r2 = R * R, acc = 0.0;
        for (int n = 7; n >= 0; --n) acc = acc * r2 + c[n];
        return acc;
    }
    return (1.0 / tanh(R) - 1.0 / R) / R;
}

double fldo_limiter(int kind, double larsen_n, double R)
{
    switch (kind) {
    case FLDO_LIM_CDA: return 1.0 / 3.0;
    case FLDO_LIM_SUM: return 1.0 / (3.0 + R);
    case FLDO_LIM_MAX: return 1.0 / fmax(3.0, R);
    case FLDO_LIM_KERSHAW: return 2.0 / (3.0 + sqrt(9.0 + 4.0 * R * R));
    case FLDO_LIM_LARSEN: {
        /* (3^n + R^n)^(-1/n), written as 1/(m (1 + (s/m)^n)^(1/n)) with
         * m = max(3, R), s = min(3, R) so R^n cannot overflow. */
        double m = fmax(3.0, R), s = fmin(3.0, R);
        return 1.0 / (m * pow(1.0 + pow(s / m, larsen_n), 1.0 / larsen_n));
    }
    case FLDO_LIM_LP: return lp_limiter(R);
    default: return NAN;
    }
}

/* ------------------------------------------------------------------------ */
/* Minimal parallel-for over z planes (deterministic: each worker owns a     */
/* contiguous range of planes; reductions are combined in worker order).     */
/* ------------------------------------------------------------------------ */

typedef void (*plane_fn)(void *ctx, int k0, int k1, int worker);

typedef struct {
    plane_fn fn;
    void *ctx;
    int k0, k1, worker;
} task_t;

static void *task_main(void *arg)
{
    task_t *t = (task_t *)arg;
    t->fn(t->ctx, t->k0, t->k1, t->worker);
    return NULL;
}

static void parallel_planes(int nz, int nthreads, plane_fn fn, void *ctx)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nz) nthreads = nz;
    if (nthreads > 256) nthreads = 256;
    if (nthreads == 1) {
        fn(ctx, 0, nz, 0);
        return;
    }
    pthread_t th[256];
    task_t tk[256];
    int started[256];
    for (int w = 0; w < nthreads; ++w) {
        tk[w].fn = fn;
        tk[w].ctx = ctx;
        tk[w].k0 = (int)((long)nz * w / nthreads);
        tk[w].k1 = (int)((long)nz * (w + 1) / nthreads);
        tk[w].worker = w;
        started[w] = pthread_create(&th[w], NULL, task_main, &tk[w]) == 0;
        if (!started[w]) task_main(&tk[w]);
    }
    for (int w = 0; w < nthreads; ++w)
        if (started[w]) pthread_join(th[w], NULL);
}

/* ------------------------------------------------------------------------ */
/* Medium preparation (Algorithm 1, first three steps).                      */
/* ------------------------------------------------------------------------ */

/* sigma' = max(sigma_t, sigma_eps); sigma_a' = (1 - albedo) sigma'. */
void fldo_prep(long nvox, const float *sigma_t, const float *albedo, double sigma_eps,
               double *sp, double *sa)
{
    for (long v = 0; v < nvox; ++v) {
        double s = fmax((double)sigma_t[v], sigma_eps);
        sp[v] = s;
        sa[v] = (1.0 - (double)albedo[v]) * s;
    }
}

/* The same medium stored in bfloat16 (the reduced-precision medium of the
 * 256^3 runs): sigma' = max(sigma_t, sigma_eps) and sigma_a' = (1 - albedo)
 * sigma' are formed in single precision, one rounding per operation, and
 * each is rounded to bfloat16 (8 significant bits), to nearest with ties to
 * even.  Rounding to 8 bits is a decision taken in floating point, so it is
 * taken on the same single-precision values the device rounds; the solve
 * then uses the rounded values exactly. */
static float bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    /* add half an 8-bit ulp (minus one when the kept part is even) and cut */
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&x, &u, sizeof x);
    return x;
}

void fldo_prep_bf16(long nvox, const float *sigma_t, const float *albedo, double sigma_eps,
                    double *sp, double *sa)
{
    const float seps = (float)sigma_eps;
    for (long v = 0; v < nvox; ++v) {
        const float s = sigma_t[v] > seps ? sigma_t[v] : seps;
        const float one_minus = 1.0f - albedo[v];
        const float a = one_minus * s;
        sp[v] = (double)bf16_round(s);
        sa[v] = (double)bf16_round(a);
    }
}

/* jbar = sqrt(mean(j^2)) over the unknowns. */
double fldo_rms(long nvox, const double *j)
{
    double s = 0.0;
    for (long v = 0; v < nvox; ++v) s += j[v] * j[v];
    return nvox > 0 ? sqrt(s / (double)nvox) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* One colour pass of Algorithm 1.                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    const fldo_cfg *c;
    const double *sp, *sa, *j;
    double *phi, *D;
    int colour;
} pass_ctx;

static inline long pidx(const fldo_cfg *c, int I, int J, int K)
{
    return ((long)K * (c->ny + 2) + J) * (long)(c->nx + 2) + I;
}

/* Knudsen number of Eq. 35 at padded point q, with the central gradient of
 * the neighbours in phi and the value phi_p at q, then D = F(R)/sigma'
 * (Eq. 33). */
static double knudsen_D(const fldo_cfg *c, const double *phi, double sp, long q, double phi_p)
{
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    double gx = (phi[q + sx] - phi[q - sx]) / (2.0 * c->h);   /* Eq. 34 */
    double gy = (phi[q + sy] - phi[q - sy]) / (2.0 * c->h);
    double gz = (phi[q + sz] - phi[q - sz]) / (2.0 * c->h);
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double floor_ = c->jbar > 0.0 ? c->eps * c->jbar : FLDO_FLOOR_NO_EMISSION;
    double R = fmax(g, floor_) / fmax(sp * phi_p, floor_);    /* Eq. 35 */
    return fldo_limiter(c->limiter, c->larsen_n, R) / sp;     /* Eq. 33 */
}

/* D from the current phi at q (Eq. 33-35). */
static double fresh_D(const fldo_cfg *c, const double *phi, double sp, long q)
{
    return knudsen_D(c, phi, sp, q, phi[q]);
}

static void pass_planes(void *vctx, int k0, int k1, int worker)
{
    (void)worker;
    pass_ctx *x = (pass_ctx *)vctx;
    const fldo_cfg *c = x->c;
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    const double h2 = c->h * c->h;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                if (((i + j + k) & 1) != x->colour) continue;
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                const long nb[6] = {q - sx, q + sx, q - sy, q + sy, q - sz, q + sz};
                double phi_old = x->phi[q], phi_new = phi_old, Dp = 0.0;
                int rounds = c->local_iters < 1 ? 1 : c->local_iters;
                for (int r = 0; r < rounds; ++r) {
                    Dp = knudsen_D(c, x->phi, x->sp[v], q, phi_new);   /* Eq. 35, 33 */
                    double num = x->j[v] * h2, den = x->sa[v] * h2;
                    for (int s = 0; s < 6; ++s) {
                        double Dps = 0.5 * (Dp + x->D[nb[s]]);
                        num += Dps * x->phi[nb[s]];
                        den += Dps;
                    }
                    phi_new = num / den;                                /* Eq. 32 */
                }
                x->D[q] = Dp;
                x->phi[q] = c->omega * phi_new + (1.0 - c->omega) * phi_old;  /* Eq. 36 */
            }
}

/* One iteration of Algorithm 1: the red pass, then the black pass.
 * sp, sa, j: unpadded; phi, D: padded (ghosts untouched). */
void fldo_rb_iteration(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
                       double *phi, double *D)
{
    for (int colour = 0; colour < 2; ++colour) {
        pass_ctx x = {c, sp, sa, j, phi, D, colour};
        parallel_planes(c->nz, c->nthreads, pass_planes, &x);
    }
}

/* One colour pass only (colour 0 = red, 1 = black). */
void fldo_pass(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
               double *phi, double *D, int colour)
{
    pass_ctx x = {c, sp, sa, j, phi, D, colour};
    parallel_planes(c->nz, c->nthreads, pass_planes, &x);
}

/* ------------------------------------------------------------------------ */
/* Jacobi iteration: the order-free alternative to Algorithm 1's red-black   */
/* sweep.  Every quantity on the right of Eq. 32 comes from iteration k.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const fldo_cfg *c;
    const double *sp, *sa, *j, *phi;
    double *D, *phi_next;
} jac_ctx;

static void jacobi_D_planes(void *vctx, int k0, int k1, int worker)
{
    (void)worker;
    jac_ctx *x = (jac_ctx *)vctx;
    const fldo_cfg *c = x->c;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                x->D[q] = fresh_D(c, x->phi, x->sp[v], q);         /* D^k, Eq. 33-35 */
            }
}

static void jacobi_phi_planes(void *vctx, int k0, int k1, int worker)
{
    (void)worker;
    jac_ctx *x = (jac_ctx *)vctx;
    const fldo_cfg *c = x->c;
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    const double h2 = c->h * c->h;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                const long nb[6] = {q - sx, q + sx, q - sy, q + sy, q - sz, q + sz};
                double num = x->j[v] * h2, den = x->sa[v] * h2;
                for (int s = 0; s < 6; ++s) {
                    double Dps = 0.5 * (x->D[q] + x->D[nb[s]]);
                    num += Dps * x->phi[nb[s]];
                    den += Dps;
                }
                /* Eq. 32, then the damped blend of Eq. 36 */
                x->phi_next[q] = c->omega * (num / den) + (1.0 - c->omega) * x->phi[q];
            }
}

/* One Jacobi iteration: D^k = F(R(phi^k))/sigma' at every unknown, then
 * phi^{k+1}_p = (1 - omega) phi^k_p + omega num/den with num and den of
 * Eq. 32 from phi^k and D^k only.  D (padded) is overwritten at the unknowns
 * (ghost D untouched); phi_next (padded) receives phi^{k+1} at the unknowns
 * and a copy of phi's ghosts. */
void fldo_jacobi_iteration(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
                           const double *phi, double *D, double *phi_next)
{
    const long np = (long)(c->nx + 2) * (c->ny + 2) * (c->nz + 2);
    memcpy(phi_next, phi, sizeof(double) * (size_t)np);
    jac_ctx x = {c, sp, sa, j, phi, D, phi_next};
    parallel_planes(c->nz, c->nthreads, jacobi_D_planes, &x);
    parallel_planes(c->nz, c->nthreads, jacobi_phi_planes, &x);
}

/* ------------------------------------------------------------------------ */
/* Residual, Eq. 37, with D recomputed from the current phi.                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    const fldo_cfg *c;
    const double *sp, *sa, *j, *phi;
    double *Df;       /* padded scratch: fresh D at unknowns, ghost D at ghosts */
    double *Rout;     /* optional unpadded residual field */
    int margin;
    double partial[256];
} res_ctx;

static void fresh_D_planes(void *vctx, int k0, int k1, int worker)
{
    (void)worker;
    res_ctx *x = (res_ctx *)vctx;
    const fldo_cfg *c = x->c;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                x->Df[q] = fresh_D(c, x->phi, x->sp[v], q);
            }
}

static void residual_planes(void *vctx, int k0, int k1, int worker)
{
    res_ctx *x = (res_ctx *)vctx;
    const fldo_cfg *c = x->c;
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    const double h2 = c->h * c->h;
    const int m = x->margin;
    double acc = 0.0;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                const long nb[6] = {q - sx, q + sx, q - sy, q + sy, q - sz, q + sz};
                double num = x->j[v] * h2, den = x->sa[v] * h2;
                for (int s = 0; s < 6; ++s) {
                    double Dps = 0.5 * (x->Df[q] + x->Df[nb[s]]);
                    num += Dps * x->phi[nb[s]];
                    den += Dps;
                }
                double R = (num - x->phi[q] * den) / h2;   /* Eq. 37 */
                if (x->Rout) x->Rout[v] = R;
                if (i >= m && i < c->nx - m && j >= m && j < c->ny - m && k >= m && k < c->nz - m)
                    acc += R * R;
            }
    x->partial[worker] = acc;
}

/* Returns the relative residual Rbar / jbar.  D holds the ghost values of D
 * (only its ghost layer is read); phi is padded.  *sum_r2 receives the sum of
 * R_p^2 over the residual set (unknowns at least `margin` voxels from the
 * faces), *count the size of that set.  Rout (optional) receives R_p. */
double fldo_residual(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
                     const double *phi, const double *D, int margin, double *sum_r2,
                     long *count, double *Rout)
{
    long npad = (long)(c->nx + 2) * (c->ny + 2) * (c->nz + 2);
    double *Df = (double *)malloc(sizeof(double) * (size_t)npad);
    if (!Df) return NAN;
    memcpy(Df, D, sizeof(double) * (size_t)npad);
    res_ctx x;
    memset(&x, 0, sizeof(x));
    x.c = c; x.sp = sp; x.sa = sa; x.j = j; x.phi = phi; x.Df = Df; x.Rout = Rout; x.margin = margin;
    int nt = c->nthreads < 1 ? 1 : (c->nthreads > 256 ? 256 : c->nthreads);
    parallel_planes(c->nz, nt, fresh_D_planes, &x);
    parallel_planes(c->nz, nt, residual_planes, &x);
    free(Df);
    double s = 0.0;
    for (int w = 0; w < 256; ++w) s += x.partial[w];
    long cnt = 0;
    {
        long ex = c->nx - 2L * margin, ey = c->ny - 2L * margin, ez = c->nz - 2L * margin;
        cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
    }
    if (sum_r2) *sum_r2 = s;
    if (count) *count = cnt;
    double rbar = cnt > 0 ? sqrt(s / (double)cnt) : 0.0;
    return c->jbar > 0.0 ? rbar / c->jbar : rbar;
}

/* Residual R_p at one unknown (i, j, k), D recomputed from phi at p and at its
 * six neighbours (ghost neighbours keep their ghost D). */
double fldo_residual_at(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
                        const double *phi, const double *D, int i, int jj, int k)
{
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    const double h2 = c->h * c->h;
    long v = ((long)k * c->ny + jj) * c->nx + i;
    long q = pidx(c, i + 1, jj + 1, k + 1);
    double Dp = fresh_D(c, phi, sp[v], q);
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
    const long nb[6] = {q - sx, q + sx, q - sy, q + sy, q - sz, q + sz};
    double num = j[v] * h2, den = sa[v] * h2;
    for (int s = 0; s < 6; ++s) {
        int ii = i + di[s], jn = jj + dj[s], kn = k + dk[s];
        double Ds;
        if (ii < 0 || ii >= c->nx || jn < 0 || jn >= c->ny || kn < 0 || kn >= c->nz)
            Ds = D[nb[s]];
        else
            Ds = fresh_D(c, phi, sp[((long)kn * c->ny + jn) * c->nx + ii], nb[s]);
        double Dps = 0.5 * (Dp + Ds);
        num += Dps * phi[nb[s]];
        den += Dps;
    }
    return (num - phi[q] * den) / h2;
}

/* ------------------------------------------------------------------------ */
/* Solve loop of Algorithm 1: iterate until Rbar/jbar <= tol (checked every */
/* check_every iterations) or max_iters.  Returns the iterations done;       */
/* *rel receives the last relative residual; hist (optional, length          */
/* max_iters/check_every + 1) receives every checked value.                  */
/* ------------------------------------------------------------------------ */
int fldo_solve(const fldo_cfg *c, const double *sp, const double *sa, const double *j,
               double *phi, double *D, double tol, int max_iters, int check_every, int margin,
               double *rel, double *hist, int *nhist)
{
    int it = 0, nh = 0;
    double r = fldo_residual(c, sp, sa, j, phi, D, margin, NULL, NULL, NULL);
    if (check_every < 1) check_every = 1;
    while (!(r <= tol) && it < max_iters && isfinite(r)) {
        int k = check_every;
        if (k > max_iters - it) k = max_iters - it;
        for (int s = 0; s < k; ++s) fldo_rb_iteration(c, sp, sa, j, phi, D);
        it += k;
        r = fldo_residual(c, sp, sa, j, phi, D, margin, NULL, NULL, NULL);
        if (hist) hist[nh] = r;
        ++nh;
    }
    if (rel) *rel = r;
    if (nhist) *nhist = nh;
    return it;
}

/* ------------------------------------------------------------------------ */
/* Single-scatter source q_ri (Sec. 3 after Eq. 6; Sec. 6.2 "computed via    */
/* raymarching").  Transmittance T = exp(-sum sigma_t(x_n) dx) (Eq. 3) along */
/* the ray from the voxel centre towards the light; samples at the midpoint  */
/* of each step of length ds, sigma_t blended trilinearly between voxel      */
/* centres (clamped to the outermost centres); the march ends at the domain  */
/* boundary (or at a point light inside the domain), the last step shortened */
/* to fit.  The scattering coefficient is sigma_s = albedo * sigma_t (raw,   */
/* not floored).                                                             */
/* ------------------------------------------------------------------------ */

static double sigma_trilinear(int nx, int ny, int nz, double h, const float *st,
                              double x, double y, double z)
{
    double u[3] = {x / h - 0.5, y / h - 0.5, z / h - 0.5};
    int n[3] = {nx, ny, nz}, i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double w = u[a];
        if (w < 0.0) w = 0.0;
        if (w > (double)(n[a] - 1)) w = (double)(n[a] - 1);
        int b = (int)floor(w);
        if (b > n[a] - 2) b = n[a] - 2;
        if (b < 0) b = 0;
        i0[a] = b;
        f[a] = (n[a] == 1) ? 0.0 : w - (double)b;
    }
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                int ii = i0[0] + cx, jj = i0[1] + cy, kk = i0[2] + cz;
                if (ii >= nx) ii = nx - 1;
                if (jj >= ny) jj = ny - 1;
                if (kk >= nz) kk = nz - 1;
                double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
                acc += w * (double)st[((long)kk * ny + jj) * nx + ii];
            }
    return acc;
}

/* Distance from x (inside the box) along unit w to the box boundary. */
static double exit_distance(int nx, int ny, int nz, double h, const double x[3], const double w[3])
{
    double ext[3] = {nx * h, ny * h, nz * h}, t = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (w[a] > 0.0) t = fmin(t, (ext[a] - x[a]) / w[a]);
        else if (w[a] < 0.0) t = fmin(t, (0.0 - x[a]) / w[a]);
    }
    return t;
}

static double optical_depth(int nx, int ny, int nz, double h, const float *st, const double x[3],
                            const double w[3], double length, double ds)
{
    double tau = 0.0;
    long m_full = (long)floor(length / ds);
    for (long m = 0; m < m_full; ++m) {
        double t = ((double)m + 0.5) * ds;
        tau += sigma_trilinear(nx, ny, nz, h, st, x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]) * ds;
    }
    double rem = length - (double)m_full * ds;
    if (rem > 1e-12 * ds) {
        double t = (double)m_full * ds + 0.5 * rem;
        tau += sigma_trilinear(nx, ny, nz, h, st, x[0] + t * w[0], x[1] + t * w[1], x[2] + t * w[2]) * rem;
    }
    return tau;
}

typedef struct {
    int nx, ny, nz;
    double h;
    const float *st, *alb;
    double w[3];     /* unit vector towards the light (directional) */
    double pos[3];   /* light position (point) */
    double L;        /* radiance (directional) or power (point) */
    double ds;
    int point;
    double *q;
} bake_ctx;

static void bake_planes(void *vctx, int k0, int k1, int worker)
{
    (void)worker;
    bake_ctx *b = (bake_ctx *)vctx;
    for (int k = k0; k < k1; ++k)
        for (int j = 0; j < b->ny; ++j)
            for (int i = 0; i < b->nx; ++i) {
                long v = ((long)k * b->ny + j) * b->nx + i;
                double x[3] = {(i + 0.5) * b->h, (j + 0.5) * b->h, (k + 0.5) * b->h};
                double sigma_s = (double)b->alb[v] * (double)b->st[v];
                if (!b->point) {
                    double len = exit_distance(b->nx, b->ny, b->nz, b->h, x, b->w);
                    double tau = optical_depth(b->nx, b->ny, b->nz, b->h, b->st, x, b->w, len, b->ds);
                    b->q[v] = b->L * sigma_s * exp(-tau);
                } else {
                    double d[3] = {b->pos[0] - x[0], b->pos[1] - x[1], b->pos[2] - x[2]};
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    double tau = 0.0;
                    if (r > 0.0) {
                        double w[3] = {d[0] / r, d[1] / r, d[2] / r};
                        double len = fmin(r, exit_distance(b->nx, b->ny, b->nz, b->h, x, w));
                        tau = optical_depth(b->nx, b->ny, b->nz, b->h, b->st, x, w, len, b->ds);
                    }
                    double rr = fmax(r, 0.5 * b->h);
                    b->q[v] = b->L * sigma_s * exp(-tau) / (4.0 * M_PI * rr * rr);
                }
            }
}

/* Directional light travelling along dir (not necessarily normalised) with
 * radiance L: q = L sigma_s T, T towards the light (along -dir). */
void fldo_bake_directional(int nx, int ny, int nz, double h, const float *sigma_t,
                           const float *albedo, const double dir[3], double L, double ds,
                           int nthreads, double *q)
{
    double n = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    bake_ctx b;
    memset(&b, 0, sizeof(b));
    b.nx = nx; b.ny = ny; b.nz = nz; b.h = h; b.st = sigma_t; b.alb = albedo;
    for (int a = 0; a < 3; ++a) b.w[a] = -dir[a] / n;
    b.L = L; b.ds = ds; b.point = 0; b.q = q;
    parallel_planes(nz, nthreads, bake_planes, &b);
}

/* Isotropic point light of power P at pos: q = P sigma_s T / (4 pi r^2), with
 * r floored at half a voxel. */
void fldo_bake_point(int nx, int ny, int nz, double h, const float *sigma_t, const float *albedo,
                     const double pos[3], double P, double ds, int nthreads, double *q)
{
    bake_ctx b;
    memset(&b, 0, sizeof(b));
    b.nx = nx; b.ny = ny; b.nz = nz; b.h = h; b.st = sigma_t; b.alb = albedo;
    for (int a = 0; a < 3; ++a) b.pos[a] = pos[a];
    b.L = P; b.ds = ds; b.point = 1; b.q = q;
    parallel_planes(nz, nthreads, bake_planes, &b);
}

/* F(R) for an array of R values (Table 2). */
/* ------------------------------------------------------------------------ */
/* Primary ray march (Sec. 3, the equation after Eq. 2): the radiance that   */
/* reaches the camera along a pixel's ray is the background attenuated over  */
/* the whole chord plus, over the march segments, the transmittance from     */
/* each segment to the camera times its source Q times the segment length.  */
/* 4 pi Q = q_ri + sigma_s phi + j (the source in terms of phi, Sec. 3): the  */
/* solver's source field already holds q_ri + j.  Fields are sampled        */
/* trilinearly between voxel centres (clamped to the outermost centres) at   */
/* the midpoint of each segment; segments of length `step` start where the   */
/* ray enters the box [0, nx h] x [0, ny h] x [0, nz h] (or at the eye, if    */
/* inside) and the last one ends at the exit.  The transmittance from a      */
/* segment to the camera covers the segments between them (not its own), so */
/* that over the whole chord it is exp(-sum sigma_t step) as in Sec. 3.  The */
/* march stops once that transmittance is below `t_min` (the rest of the     */
/* ray can add at most t_min times its unattenuated source).                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    double eye[3], target[3], up[3];
    double fov_deg;        /* vertical field of view */
    int width, height;
    double step;           /* segment length (> 0) */
    double background;     /* radiance entering the far end of every ray */
    double t_min;          /* transmittance below which the march stops */
} fldo_camera;

static double field_trilinear(int nx, int ny, int nz, double h, const double *f, const double x[3])
{
    const int n[3] = {nx, ny, nz};
    int i0[3], i1[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        double u = x[a] / h - 0.5;
        if (u < 0.0) u = 0.0;
        if (u > (double)(n[a] - 1)) u = (double)(n[a] - 1);
        int b = (int)floor(u);
        if (b > n[a] - 2) b = n[a] - 2;
        if (b < 0) b = 0;
        i0[a] = b;
        i1[a] = b + 1 < n[a] ? b + 1 : b;
        w[a] = (n[a] == 1) ? 0.0 : u - (double)b;
    }
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                const int i = cx ? i1[0] : i0[0], j = cy ? i1[1] : i0[1], k = cz ? i1[2] : i0[2];
                const double wt = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) * (cz ? w[2] : 1.0 - w[2]);
                acc += wt * f[((long)k * ny + j) * nx + i];
            }
    return acc;
}

typedef struct {
    int nx, ny, nz;
    double h;
    const double *st, *ss, *q, *phi;
    const fldo_camera *cam;
    double *image;
    double f[3], r[3], u[3], tan_half, aspect;
} render_ctx;

static double render_pixel(const render_ctx *x, int px, int py)
{
    const fldo_camera *c = x->cam;
    const double box[3] = {x->nx * x->h, x->ny * x->h, x->nz * x->h};
    const double sx = (2.0 * (px + 0.5) / c->width - 1.0) * x->tan_half * x->aspect;
    const double sy = (1.0 - 2.0 * (py + 0.5) / c->height) * x->tan_half;
    double d[3], norm = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = x->f[a] + sx * x->r[a] + sy * x->u[a];
        norm += d[a] * d[a];
    }
    norm = sqrt(norm);
    for (int a = 0; a < 3; ++a) d[a] /= norm;
    /* chord through the box (slab test) */
    double t0 = 0.0, t1 = INFINITY;
    int hit = 1;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (c->eye[a] < 0.0 || c->eye[a] > box[a]) hit = 0;
            continue;
        }
        double ta = (0.0 - c->eye[a]) / d[a], tb = (box[a] - c->eye[a]) / d[a];
        if (ta > tb) { double tt = ta; ta = tb; tb = tt; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    double L = 0.0, T = 1.0;
    if (hit && t1 > t0) {
        const long nseg = (long)ceil((t1 - t0) / c->step);
        for (long m = 0; m < nseg && T >= c->t_min; ++m) {
            const double a = t0 + m * c->step;
            const double b = fmin(a + c->step, t1);
            const double len = b - a, tm = 0.5 * (a + b);
            double pos[3];
            for (int k = 0; k < 3; ++k) pos[k] = c->eye[k] + tm * d[k];
            const double st = field_trilinear(x->nx, x->ny, x->nz, x->h, x->st, pos);
            const double ss = field_trilinear(x->nx, x->ny, x->nz, x->h, x->ss, pos);
            const double q = field_trilinear(x->nx, x->ny, x->nz, x->h, x->q, pos);
            const double ph = field_trilinear(x->nx, x->ny, x->nz, x->h, x->phi, pos);
            const double Q = (q + ss * ph) / (4.0 * M_PI);   /* Sec. 3, 4 pi Q */
            L += T * Q * len;
            T *= exp(-st * len);
        }
    }
    return L + c->background * T;
}

static void render_rows(void *vctx, int y0, int y1, int worker)
{
    (void)worker;
    render_ctx *x = (render_ctx *)vctx;
    for (int py = y0; py < y1; ++py)
        for (int px = 0; px < x->cam->width; ++px) x->image[(long)py * x->cam->width + px] = render_pixel(x, px, py);
}

static void setup_camera(render_ctx *x, const fldo_camera *cam)
{
    double nf = 0.0;
    for (int a = 0; a < 3; ++a) {
        x->f[a] = cam->target[a] - cam->eye[a];
        nf += x->f[a] * x->f[a];
    }
    nf = sqrt(nf);
    for (int a = 0; a < 3; ++a) x->f[a] /= nf;
    /* r = f x up, u = r x f */
    x->r[0] = x->f[1] * cam->up[2] - x->f[2] * cam->up[1];
    x->r[1] = x->f[2] * cam->up[0] - x->f[0] * cam->up[2];
    x->r[2] = x->f[0] * cam->up[1] - x->f[1] * cam->up[0];
    double nr = sqrt(x->r[0] * x->r[0] + x->r[1] * x->r[1] + x->r[2] * x->r[2]);
    for (int a = 0; a < 3; ++a) x->r[a] /= nr;
    x->u[0] = x->r[1] * x->f[2] - x->r[2] * x->f[1];
    x->u[1] = x->r[2] * x->f[0] - x->r[0] * x->f[2];
    x->u[2] = x->r[0] * x->f[1] - x->r[1] * x->f[0];
    x->tan_half = tan(0.5 * cam->fov_deg * M_PI / 180.0);
    x->aspect = (double)cam->width / (double)cam->height;
}

/* Render the volume: sigma_t, sigma_s, q (= q_ri + j) and phi unpadded
 * (nx*ny*nz, x fastest); image (width*height, row 0 at the top) receives
 * the radiance of each pixel. */
void fldo_render(int nx, int ny, int nz, double h, const double *sigma_t, const double *sigma_s, const double *q,
                 const double *phi, const fldo_camera *cam, double *image, int nthreads)
{
    render_ctx x;
    x.nx = nx; x.ny = ny; x.nz = nz; x.h = h;
    x.st = sigma_t; x.ss = sigma_s; x.q = q; x.phi = phi;
    x.cam = cam;
    x.image = image;
    setup_camera(&x, cam);
    parallel_planes(cam->height, nthreads, render_rows, &x);
}

/* The same for `count` single pixels (px[i], py[i]) of the camera's image. */
void fldo_render_pixels(int nx, int ny, int nz, double h, const double *sigma_t, const double *sigma_s,
                        const double *q, const double *phi, const fldo_camera *cam, const int *px, const int *py,
                        long count, double *out)
{
    render_ctx x;
    x.nx = nx; x.ny = ny; x.nz = nz; x.h = h;
    x.st = sigma_t; x.ss = sigma_s; x.q = q; x.phi = phi;
    x.cam = cam;
    x.image = NULL;
    setup_camera(&x, cam);
    for (long i = 0; i < count; ++i) out[i] = render_pixel(&x, px[i], py[i]);
}

/* ------------------------------------------------------------------------ */
/* Quarter-resolution solve (Sec. 6.2: phi is solved on a grid with a quarter  */
/* of the data's resolution per axis, then used at full resolution in the    */
/* ray march).  Downsampling: the coarse voxel (I,J,K) covers the fine       */
/* voxels f I .. f I + f - 1 per axis (those that exist); sigma_t, sigma_s =  */
/* albedo sigma_t and the source are averaged over them, and the coarse     */
/* albedo is mean sigma_s / mean sigma_t (0 where mean sigma_t is 0).        */
/* Upsampling: phi at each fine voxel centre, blended trilinearly between    */
/* the coarse voxel centres (clamped to the outermost), the coarse grid's    */
/* spacing being f h.                                                        */
/* ------------------------------------------------------------------------ */

void fldo_downsample(int nx, int ny, int nz, int f, const float *sigma_t, const float *albedo, const double *q,
                     double *sigma_t_c, double *albedo_c, double *q_c)
{
    const int cx = (nx + f - 1) / f, cy = (ny + f - 1) / f, cz = (nz + f - 1) / f;
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double st = 0.0, ss = 0.0, qq = 0.0;
                long cnt = 0;
                for (int k = K * f; k < K * f + f && k < nz; ++k)
                    for (int j = J * f; j < J * f + f && j < ny; ++j)
                        for (int i = I * f; i < I * f + f && i < nx; ++i) {
                            const long v = ((long)k * ny + j) * nx + i;
                            st += (double)sigma_t[v];
                            ss += (double)albedo[v] * (double)sigma_t[v];
                            qq += q[v];
                            ++cnt;
                        }
                const long c = ((long)K * cy + J) * cx + I;
                sigma_t_c[c] = st / (double)cnt;
                albedo_c[c] = st > 0.0 ? ss / st : 0.0;
                q_c[c] = qq / (double)cnt;
            }
}

void fldo_upsample(int nx, int ny, int nz, double h, int f, const double *phi_c, double *phi)
{
    const int cx = (nx + f - 1) / f, cy = (ny + f - 1) / f, cz = (nz + f - 1) / f;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double x[3] = {(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h};
                phi[((long)k * ny + j) * nx + i] = field_trilinear(cx, cy, cz, f * h, phi_c, x);
            }
}

void fldo_limiter_array(int kind, double larsen_n, const double *R, double *F, long count)
{
    for (long v = 0; v < count; ++v) F[v] = fldo_limiter(kind, larsen_n, R[v]);
}

/* |E_p| = D_p |grad phi_p| (Eq. 15 with Eq. 33-35, D recomputed from phi) at
 * every unknown, for the flux-limiting constraint |E| <= phi (Eq. 14). */
void fldo_flux(const fldo_cfg *c, const double *sp, const double *phi, double *E)
{
    const long sx = 1, sy = c->nx + 2, sz = (long)(c->nx + 2) * (c->ny + 2);
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                long v = ((long)k * c->ny + j) * c->nx + i;
                long q = pidx(c, i + 1, j + 1, k + 1);
                double gx = (phi[q + sx] - phi[q - sx]) / (2.0 * c->h);
                double gy = (phi[q + sy] - phi[q - sy]) / (2.0 * c->h);
                double gz = (phi[q + sz] - phi[q - sz]) / (2.0 * c->h);
                double g = sqrt(gx * gx + gy * gy + gz * gz);
                E[v] = fresh_D(c, phi, sp[v], q) * g;
            }
}
