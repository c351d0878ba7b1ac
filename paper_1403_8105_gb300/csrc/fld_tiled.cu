// fld_tiled.cu -- temporally blocked red-black sweeps (sm_103a).
//
// One launch performs T iterations of Algorithm 1 (Koerner et al. 2014: the
// red pass, then the black pass, T times) on the single-precision families.
// Each CTA owns an x-y tile of TX x TY unknowns and a chunk of z-planes.  The
// state (phi, D, and the low word of phi for the hi/lo family) of every plane
// the CTA touches is staged in shared memory with cp.async.bulk.tensor (TMA,
// 4-D boxes: half-row x row x plane x colour of the colour-split layout),
// tracked by one mbarrier per ring slot, with a halo of 2T cells in x and y.
// The 2T colour passes then sweep the planes as a wavefront: at step s pass t
// (colour t mod 2) updates plane s - t, so when it runs, pass t - 1 has
// already produced the planes above and below it.  Each pass updates its
// plane over the tile plus 2T - 1 - t halo cells, shrinking by one per pass,
// so the last pass is exact on the tile without any exchange between CTAs.
// The medium (sigma', sigma_a' dl^2, j dl^2; read-only) is read through the
// L1 cache.  Finished planes of the tile are written to the other buffer of a
// ping-pong pair (every CTA reads only the launch's input), so a launch
// reads each field once and writes phi and D once for T iterations.
//
// Every point update is cell::cell_f32 / cell::cell_fh -- the same code as the
// launched colour passes -- with the same inputs, so T blocked iterations
// give the launched passes' state bit for bit (tested).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "fld_cell.cuh"
#include "fld_device.cuh"
#include "fld_internal.h"

namespace fld {

// Device part: compiled in this file for the FP32 family and in
// fld_tiled_hl.cu (which includes this file with FLD_TILED_HL_ONLY) for the
// hi/lo family, so the two halves of the instances build in parallel.
namespace tiled_detail {

using namespace cell;

constexpr int kTiledThreads = 512;
constexpr int kTiledWarps = kTiledThreads / 32;
// bounded waits: polls of an mbarrier (with a short sleep) before the CTA
// records a timeout and continues (about a second)
constexpr int kWaitPolls = 1 << 24;

// Geometry of a tile configuration (shared by host and device).
template <int T, int TX, int TY, bool HL>
struct TileCfg {
    static constexpr int NS = 2 * T + 3;                       // ring slots (planes)
    static constexpr int R4T = (T + 3) & ~3;                   // halo rounded to TMA alignment (4 floats)
    static constexpr int WX = ((TX / 2 + T + R4T) + 3) & ~3;   // half-row elements loaded per row
    static constexpr int WY = TY + 4 * T;                      // rows loaded
    static constexpr int PL = 2 * WY * WX;                     // floats per field-plane (both colours)
    static constexpr int NF = HL ? 3 : 2;                      // phi, D (, phi lo)
    static constexpr size_t SMEM = (size_t)NS * NF * PL * sizeof(float);
    static_assert(TX % 8 == 0 && TX / 2 + 2 * T <= 64, "tile width");
    static_assert(TX / 2 + 2 * T - 1 <= 32, "one warp per half row of a pass region");
};

struct Region {
    int Jr0, Jr1, Ir0, Ir1;
    bool active;
};

struct TiledArgs {
    Layout L;
    const float *sp, *ah2, *jh2;           // medium (single precision)
    const uint16_t *spb, *sab;             // bfloat16 medium (BF)
    float h2;
    float *dphi, *dD, *dlo;                // destination buffers
    int tiles_x, tiles_y, chunk, items;
    int lim, rounds;
    float larsen_n, omega, inv2h, floor_;
    int *status;                            // set to 1 when a wait timed out
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity to complete; false if it
// did not within kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (int i = 0; i < kWaitPolls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

// 4-D tiled TMA load (x = half-row element, y = row, z = plane, w = colour)
// into shared memory, completing on the mbarrier.
__device__ __forceinline__ void tma_load_4d(float *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

template <int T, int TX, int TY, int LIM, int ROUNDS, bool HL, bool BF>
__global__ void __launch_bounds__(kTiledThreads, 1)
    k_rb_tiled(const __grid_constant__ CUtensorMap m_phi, const __grid_constant__ CUtensorMap m_D,
               const __grid_constant__ CUtensorMap m_lo, const TiledArgs a) {
    using C = TileCfg<T, TX, TY, HL>;
    constexpr int NS = C::NS, WX = C::WX, WY = C::WY, PL = C::PL, NF = C::NF;
    constexpr int CW = WY * WX;                              // floats per colour of a field-plane
    constexpr int RMAX = (TY + 2 * (2 * T - 1) + kTiledWarps - 1) / kTiledWarps;   // rows per warp in a pass
    extern __shared__ __align__(128) float sm[];             // [slot][field][colour][WY][WX]
    __shared__ __align__(8) uint64_t bar[NS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Layout &L = a.L;
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t seq = 0;            // planes loaded by this CTA so far (equal in every thread)
    // medium of the current and the next sub-step's cells (RMAX rows per warp)
    float cur_s[RMAX], cur_a[RMAX], cur_j[RMAX], nxt_s[RMAX], nxt_a[RMAX], nxt_j[RMAX];
#pragma unroll
    for (int k = 0; k < RMAX; ++k) nxt_s[k] = nxt_a[k] = nxt_j[k] = 1.0f;
    bool timed_out = false;
    const int lim = LIM >= 0 ? LIM : a.lim;
    for (int item = blockIdx.x; item < a.items; item += gridDim.x) {
        const int tx = item % a.tiles_x;
        const int rest = item / a.tiles_x;
        const int ty = rest % a.tiles_y;
        const int ch = rest / a.tiles_y;
        // padded planes K this item finishes: [Kc0, Kc1)
        const int Kc0 = 1 + ch * a.chunk;
        const int Kc1 = min(L.nz + 1, Kc0 + a.chunk);
        const int x0 = 32 + (TX / 2) * tx - C::R4T;          // first loaded half-row element (16-byte aligned)
        const int J0 = 1 + TY * ty - 2 * T;                  // first loaded row
        const int Lfirst = Kc0 - 2 * T, Llast = Kc1 - 1 + 2 * T;
        // cells pass t updates on plane K: the tile plus 2T - 1 - t halo cells,
        // inside the unknowns (active: K lies in the pass's plane range)
        auto region = [&](int t, int K, Region &r) {
            const int h = 2 * T - 1 - t;
            r.Jr0 = max(1, 1 + TY * ty - h);
            r.Jr1 = min(L.ny, TY * (ty + 1) + h);
            r.Ir0 = max(1, 1 + TX * tx - h);
            r.Ir1 = min(L.nx, TX * (tx + 1) + h);
            r.active = K >= max(1, Kc0 - h) && K <= min(L.nz, Kc1 - 1 + h);
        };
        auto slot_of = [&](int K) { return (int)((seq + (uint32_t)(K - Lfirst)) % NS); };
        auto parity_of = [&](int K) { return ((seq + (uint32_t)(K - Lfirst)) / NS) & 1u; };
        auto plane = [&](int K, int field) { return sm + ((size_t)slot_of(K) * NF + field) * PL; };
        auto issue = [&](int K) {   // thread 0 only
            const int sl = slot_of(K);
            float *base = sm + (size_t)sl * NF * PL;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[sl], (uint32_t)(NF * PL * sizeof(float)));
            tma_load_4d(base, &m_phi, x0, J0, K, 0, &bar[sl]);
            tma_load_4d(base + PL, &m_D, x0, J0, K, 0, &bar[sl]);
            if (HL) tma_load_4d(base + 2 * PL, &m_lo, x0, J0, K, 0, &bar[sl]);
        };
        if (tid == 0) issue(Lfirst);
        for (int s = Lfirst - 1; s <= Kc1 + 2 * T - 2; ++s) {
            if (tid == 0 && s + 2 <= Llast) issue(s + 2);
            // (after one wait has given up, the CTA stops waiting: it finishes
            // without hanging and the host reports the timeout)
            if (s + 1 <= Llast && !timed_out && !mbar_wait(&bar[slot_of(s + 1)], parity_of(s + 1))) timed_out = true;
            // The 2T passes of this step (pass t on plane s - t).  The medium
            // of a pass's cells is fetched into registers one sub-step ahead
            // (during the previous pass, or the previous step's last pass), and
            // each warp gathers the inputs of all its rows before computing
            // them, so their update chains overlap.
#pragma unroll 1
            for (int t = 0; t < 2 * T; ++t) {
                const int K = s - t;
                const int c = t & 1;
                Region rg;
                region(t, K, rg);
#pragma unroll
                for (int k = 0; k < RMAX; ++k) {
                    cur_s[k] = nxt_s[k];
                    cur_a[k] = nxt_a[k];
                    cur_j[k] = nxt_j[k];
                }
                // prefetch for the next sub-step
                {
                    const int tn = t + 1 < 2 * T ? t + 1 : 0;
                    const int Kn = t + 1 < 2 * T ? K - 1 : s + 1;
                    Region rn;
                    region(tn, Kn, rn);
                    if (rn.active) {
                        const int cn = tn & 1;
#pragma unroll
                        for (int k = 0; k < RMAX; ++k) {
                            const int J = rn.Jr0 + warp + kTiledWarps * k;
                            const int pI = (cn + J + Kn + 1) & 1;
                            const int I = rn.Ir0 + ((rn.Ir0 - pI) & 1) + 2 * lane;
                            if (J > rn.Jr1 || I > rn.Ir1) continue;
                            const int q = cn * L.cs + (Kn * L.py + J) * L.hpx + kXoff + ((I + 1) >> 1);
                            if (BF) {
                                nxt_s[k] = bf16_bits_to_f(__ldg(a.spb + q));
                                nxt_a[k] = __fmul_rn(bf16_bits_to_f(__ldg(a.sab + q)), a.h2);
                            } else {
                                nxt_s[k] = __ldg(a.sp + q);
                                nxt_a[k] = __ldg(a.ah2 + q);
                            }
                            nxt_j[k] = __ldg(a.jh2 + q);
                        }
                    }
                }
                if (rg.active) {
                    float *pm = plane(K - 1, 0), *pc = plane(K, 0), *pp = plane(K + 1, 0);
                    const int oc = (1 - c) * CW, ow = c * CW;     // other colour, own colour
                    float ps[RMAX][6], Ds[RMAX][6], ls[RMAX][6], p0[RMAX], l0[RMAX];
                    int own[RMAX];
                    bool ok[RMAX];
                    const int nk = (rg.Jr1 - rg.Jr0 - warp) / kTiledWarps + 1;   // this warp's rows (warp-uniform)
#pragma unroll
                    for (int k = 0; k < RMAX; ++k) {              // gather
                        if (k >= nk) break;
                        const int J = rg.Jr0 + warp + kTiledWarps * k;
                        const int pI = (c + J + K + 1) & 1;        // parity of this row's colour-c cells
                        const int I = rg.Ir0 + ((rg.Ir0 - pI) & 1) + 2 * lane;
                        ok[k] = J <= rg.Jr1 && I <= rg.Ir1;
                        const int ly = ok[k] ? J - J0 : 1;
                        const int lx = ok[k] ? kXoff + ((I + 1) >> 1) - x0 : 1;
                        const int lxm = ok[k] ? kXoff + (I >> 1) - x0 : 0;   // x-neighbours: lxm, lxm + 1
                        const int r0 = ly * WX;
                        own[k] = ow + r0 + lx;
                        const float *phc = pc + oc, *Dc = pc + PL + oc;
                        ps[k][0] = phc[r0 + lxm];
                        ps[k][1] = phc[r0 + lxm + 1];
                        ps[k][2] = phc[r0 - WX + lx];
                        ps[k][3] = phc[r0 + WX + lx];
                        ps[k][4] = pm[oc + r0 + lx];
                        ps[k][5] = pp[oc + r0 + lx];
                        Ds[k][0] = Dc[r0 + lxm];
                        Ds[k][1] = Dc[r0 + lxm + 1];
                        Ds[k][2] = Dc[r0 - WX + lx];
                        Ds[k][3] = Dc[r0 + WX + lx];
                        Ds[k][4] = pm[PL + oc + r0 + lx];
                        Ds[k][5] = pp[PL + oc + r0 + lx];
                        p0[k] = pc[own[k]];
                        if (HL) {
                            const float *lc = pc + 2 * PL + oc;
                            ls[k][0] = lc[r0 + lxm];
                            ls[k][1] = lc[r0 + lxm + 1];
                            ls[k][2] = lc[r0 - WX + lx];
                            ls[k][3] = lc[r0 + WX + lx];
                            ls[k][4] = pm[2 * PL + oc + r0 + lx];
                            ls[k][5] = pp[2 * PL + oc + r0 + lx];
                            l0[k] = pc[2 * PL + own[k]];
                        }
                    }
                    float pn[RMAX], dn[RMAX], ln[RMAX];
#pragma unroll
                    for (int k = 0; k < RMAX; ++k) {              // compute
                        if (k >= nk) break;
                        if (HL)
                            cell_fh<LIM, ROUNDS>(p0[k], l0[k], ps[k], ls[k], Ds[k], cur_s[k], cur_a[k], cur_j[k], lim,
                                                 a.larsen_n, a.omega, a.inv2h, a.floor_, a.rounds, pn[k], ln[k], dn[k]);
                        else
                            cell_f32<LIM, ROUNDS>(p0[k], ps[k], Ds[k], cur_s[k], cur_a[k], cur_j[k], lim, a.larsen_n,
                                                  a.omega, a.inv2h, a.floor_, a.rounds, pn[k], dn[k]);
                    }
#pragma unroll
                    for (int k = 0; k < RMAX; ++k) {              // store
                        if (k >= nk) break;
                        if (!ok[k]) continue;
                        pc[own[k]] = pn[k];
                        pc[PL + own[k]] = dn[k];
                        if (HL) pc[2 * PL + own[k]] = ln[k];
                    }
                }
                __syncthreads();
            }
            // plane s - (2T - 1) has had all 2T passes: write the tile's unknowns out
            const int Kw = s - (2 * T - 1);
            if (Kw >= Kc0 && Kw < Kc1) {
                const float *pw = plane(Kw, 0);
                const int Ja = 1 + TY * ty, Jb = min(L.ny, TY * (ty + 1));
                const int nrow = (Jb - Ja + 1) * 2;
                for (int r = warp; r < nrow; r += kTiledWarps) {
                    const int J = Ja + (r >> 1), c = r & 1;
                    const int pos = (TX / 2) * tx + 1 + lane;
                    if (lane >= TX / 2) continue;
                    const int pI = (c + J + Kw + 1) & 1;
                    const int I = pI ? 2 * pos - 1 : 2 * pos;
                    if (I > L.nx) continue;
                    const int l = c * CW + (J - J0) * WX + kXoff + pos - x0;
                    const int q = c * L.cs + (Kw * L.py + J) * L.hpx + kXoff + pos;
                    a.dphi[q] = pw[l];
                    a.dD[q] = pw[PL + l];
                    if (HL) a.dlo[q] = pw[2 * PL + l];
                }
            }
        }
        seq += (uint32_t)(Llast - Lfirst + 1);
        __syncthreads();
    }
    if (timed_out) atomicExch(a.status, 1);
}

using TiledKernel = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, TiledArgs);

// Kernel instance for a configuration: Levermore-Pomraning with two local
// rounds specialised at compile time, every other limiter / round count
// through the generic instance (the same arithmetic, chosen at run time).
template <int T, int TX, int TY, bool HL, bool BF>
TiledKernel pick_kernel(int lim, int rounds) {
    if (rounds == 2 && lim == LIM_LP) return k_rb_tiled<T, TX, TY, LIM_LP, 2, HL, BF>;
    return k_rb_tiled<T, TX, TY, -1, 0, HL, BF>;
}

// Instances of one family: configuration id (0: T = 1, 56 x 32; 1: T = 2,
// 56 x 24; 2: T = 4, 48 x 8), medium in float or bfloat16.
template <bool HL>
TiledKernel kernel_for(int id, bool bf, int lim, int rounds) {
    switch (id) {
    case 0: return bf ? pick_kernel<1, 56, 32, HL, true>(lim, rounds) : pick_kernel<1, 56, 32, HL, false>(lim, rounds);
    case 1: return bf ? pick_kernel<2, 56, 24, HL, true>(lim, rounds) : pick_kernel<2, 56, 24, HL, false>(lim, rounds);
    default: return bf ? pick_kernel<4, 48, 8, HL, true>(lim, rounds) : pick_kernel<4, 48, 8, HL, false>(lim, rounds);
    }
}

TiledKernel tiled_kernel_hl(int id, bool bf, int lim, int rounds);
TiledKernel tiled_kernel_f32(int id, bool bf, int lim, int rounds);

}  // namespace tiled_detail

#if FLD_TILED_HL_ONLY
namespace tiled_detail {
TiledKernel tiled_kernel_hl(int id, bool bf, int lim, int rounds) { return kernel_for<true>(id, bf, lim, rounds); }
}  // namespace tiled_detail
}  // namespace fld
#else
namespace tiled_detail {
TiledKernel tiled_kernel_f32(int id, bool bf, int lim, int rounds) { return kernel_for<false>(id, bf, lim, rounds); }
}  // namespace tiled_detail

namespace {

using namespace tiled_detail;

// ---------------------------------------------------------------------------
// Host side: tensor maps, configuration table, launch.
// ---------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// One field of the colour-split layout as a 4-D tensor: (half-row element,
// row, plane, colour), boxes of (WX, WY, 1, 2).
cudaError_t encode_field(CUtensorMap *m, const Layout &L, float *base, int wx, int wy) {
    EncodeFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)L.hpx, (cuuint64_t)L.py, (cuuint64_t)(L.nz + 2), 2};
    const cuuint64_t strides[3] = {(cuuint64_t)L.hpx * 4, (cuuint64_t)L.hpx * L.py * 4, (cuuint64_t)L.cs * 4};
    const cuuint32_t box[4] = {(cuuint32_t)wx, (cuuint32_t)wy, 1, 2};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

struct CfgInfo {
    int T, TX, TY, WX, WY;
    size_t smem_f32, smem_hl;
};

template <int T, int TX, int TY>
CfgInfo info() {
    return {T, TX, TY, TileCfg<T, TX, TY, false>::WX, TileCfg<T, TX, TY, false>::WY, TileCfg<T, TX, TY, false>::SMEM,
            TileCfg<T, TX, TY, true>::SMEM};
}

// The configurations (index = TiledConfig id): temporal depth T and tile TX x TY.
const CfgInfo &cfg_info(int id) {
    static const CfgInfo tab[kTiledConfigs] = {info<1, 56, 32>(), info<2, 56, 24>(), info<4, 48, 8>()};
    return tab[id];
}

TiledKernel kernel_of(int id, bool hl, bool bf, int lim, int rounds) {
    return hl ? tiled_kernel_hl(id, bf, lim, rounds) : tiled_kernel_f32(id, bf, lim, rounds);
}

// Resident CTAs per SM of each kernel instance, found once (with its shared
// memory attribute set) outside any stream capture.
std::mutex g_occ_mu;
struct OccEntry {
    const void *k;
    int per_sm;
};
OccEntry g_occ[256];
int g_nocc = 0;

cudaError_t occupancy(TiledKernel k, size_t smem, int *per_sm) {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (int i = 0; i < g_nocc; ++i)
        if (g_occ[i].k == (const void *)k) {
            *per_sm = g_occ[i].per_sm;
            return cudaSuccess;
        }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kTiledThreads, smem);
    if (e != cudaSuccess) return e;
    if (g_nocc < 256) g_occ[g_nocc++] = {(const void *)k, *per_sm};
    return cudaSuccess;
}

}  // namespace

cudaError_t tiled_prepare(Family fam, int id, const PassParams &p) {
    if (id < 0 || id >= kTiledConfigs || (fam != FAM_F32 && fam != FAM_FH)) return cudaErrorInvalidValue;
    const CfgInfo &ci = cfg_info(id);
    const bool hl = fam == FAM_FH;
    int per_sm = 0;
    return occupancy(kernel_of(id, hl, p.bf16 != 0, p.lim, p.local_iters), hl ? ci.smem_hl : ci.smem_f32, &per_sm);
}

int tiled_depth(int id) { return id >= 0 && id < kTiledConfigs ? cfg_info(id).T : 0; }

void tiled_shape(int id, int *T, int *tx, int *ty) {
    const CfgInfo &ci = cfg_info(id);
    *T = ci.T;
    *tx = ci.TX;
    *ty = ci.TY;
}

int tiled_config_of(int T, int TY) {
    for (int id = 0; id < kTiledConfigs; ++id)
        if (cfg_info(id).T == T && (TY <= 0 || cfg_info(id).TY == TY)) return id;
    return -1;
}

cudaError_t tiled_maps(const Layout &L, int id, float *phi, float *D, float *lo, TiledMaps *out) {
    const CfgInfo &ci = cfg_info(id);
    cudaError_t e = encode_field(&out->phi, L, phi, ci.WX, ci.WY);
    if (e == cudaSuccess) e = encode_field(&out->D, L, D, ci.WX, ci.WY);
    if (e == cudaSuccess) e = encode_field(&out->lo, L, lo ? lo : phi, ci.WX, ci.WY);
    return e;
}

cudaError_t launch_tiled(Family fam, int id, const Layout &L, const Fields &f, const PassParams &p,
                         const TiledMaps &src, float *dphi, float *dD, float *dlo, int *status, int nsm,
                         cudaStream_t s) {
    if (fam != FAM_F32 && fam != FAM_FH) return cudaErrorInvalidValue;
    if (id < 0 || id >= kTiledConfigs) return cudaErrorInvalidValue;
    const CfgInfo &ci = cfg_info(id);
    const bool hl = fam == FAM_FH;
    const bool bf = p.bf16 != 0;
    TiledKernel k = kernel_of(id, hl, bf, p.lim, p.local_iters);
    const size_t smem = hl ? ci.smem_hl : ci.smem_f32;
    int per_sm = 0;
    cudaError_t e = occupancy(k, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    TiledArgs a;
    memset(&a, 0, sizeof(a));
    a.L = L;
    a.sp = f.sp; a.ah2 = f.ah2; a.jh2 = f.jh2; a.spb = f.spb; a.sab = f.sab; a.h2 = (float)p.h2;
    a.dphi = dphi; a.dD = dD; a.dlo = dlo;
    a.tiles_x = (L.nx + ci.TX - 1) / ci.TX;
    a.tiles_y = (L.ny + ci.TY - 1) / ci.TY;
    a.lim = p.lim; a.rounds = p.local_iters;
    a.larsen_n = (float)p.larsen_n; a.omega = (float)p.omega; a.inv2h = (float)p.inv2h; a.floor_ = (float)p.floor_;
    a.status = status;
    // z-chunks: balance the work items over the resident CTAs, counting each
    // item's pipeline fill (4T - 1 steps beyond its planes)
    const long long slots = (long long)nsm * per_sm;
    const long long tiles = (long long)a.tiles_x * a.tiles_y;
    double best = 1e300;
    int best_nc = 1;
    for (int nc = 1; nc <= L.nz; ++nc) {
        const int chunk = (L.nz + nc - 1) / nc;
        const int ncc = (L.nz + chunk - 1) / chunk;
        const long long items = tiles * ncc;
        const long long rounds = (items + slots - 1) / slots;
        const double cost = (double)rounds * (chunk + 4 * ci.T - 1);
        if (cost < best - 1e-9) {
            best = cost;
            best_nc = nc;
        }
    }
    a.chunk = (L.nz + best_nc - 1) / best_nc;
    a.items = (int)(tiles * ((L.nz + a.chunk - 1) / a.chunk));
    const long long grid = a.items < slots ? a.items : slots;
    k<<<(unsigned)grid, kTiledThreads, smem, s>>>(src.phi, src.D, src.lo, a);
    return cudaGetLastError();
}

}  // namespace fld
#endif
