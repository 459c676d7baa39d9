/*
 * lb_stream.cu -- the fused time step, streamed form (layout 4).
 *
 * Same arithmetic as the Sec. 3.1 / 3.2 / 2.2 update of lb_step_impl.cuh, in the same
 * order, reorganised so that every population is read from memory exactly once:
 *   - the moments of level n are not summed again at step n: the step that wrote level
 *     n left, per node, sum w d, sum w xi_x d and sum w xi_y d of the values it stored
 *     (aux_in); this step sums them for level n+1 as it stores (aux_out);
 *   - one producer warp streams, for each work unit (128 columns x LB5_TH rows) and each
 *     population plane, the unit's rows plus two halo rows on each side and four ghost
 *     columns on each side into a ring of shared-memory slots with
 *     cp.async.bulk.tensor, each slot guarded by a full / empty mbarrier pair;
 *   - each consumer thread owns 4 columns x LB5_RB rows, reads its radius-2 cross from
 *     the slot (the limited slope of a face between its two rows is formed once) and
 *     writes the new populations to global memory in 16-byte vectors.
 * The kernel does no boundary work: no ghost copies, shadow rebuilds or pressure
 * columns, and on a diffuse wall row it leaves the gas-bound populations to the wall
 * post-pass, to which it hands sum_out |xi.n| w dn (lb_step.cu). Every mbarrier wait is
 * bounded; on expiry the block records the failure in an error word, waits (bounded)
 * for the copies it issued, and returns.
 */
#include <cuda.h>
#include <cuda_runtime.h>

#include "lb_common.cuh"
#include "lb_step_impl.cuh"
#include "lb_tma.cuh"
#include "lb_tma.h"

namespace lbk {

#define LB5_TH 16                  /* rows per work unit */
#define LB5_RB 2                   /* rows per consumer thread */
#define LB5_NC (LB5_TH / LB5_RB)   /* consumer warps */
#define LB5_W 136                  /* columns per slot row: 128 + 4 ghost on each side */
#define LB5_STAGES 16

template <int ST>
__host__ __device__ constexpr size_t slot_bytes5()
{
    return ((size_t)LB5_W * (LB5_TH + 4) * sizeof(typename Store<ST>::T) + 1023) / 1024 * 1024;
}

template <int ST>
struct Stream5Params {
    StepParams<typename Store<ST>::R> p;
    int *err;
    int nunits;
    CUtensorMap map[2];   /* per set: box 136 x (LB5_TH + 4) x 1 */
};

/* sets (bit s) that rows j0 .. j0 + LB5_TH - 1 use */
template <typename R>
__device__ __forceinline__ int unit_sets5(const StepParams<R> &p, int tile, int j0)
{
    int sets = 0;
    for (int r = 0; r < LB5_TH && j0 + r < p.ny; ++r) sets |= 1 << (p.tmap[(size_t)(j0 + r) * p.ntx + tile] & LB_TILE_HIGH);
    return sets;
}

template <int ST, int Q, bool FORCE>
__device__ __forceinline__ void stream_set(const Stream5Params<ST> &P, int s, int tile, int j0, uint8_t *smem_base,
                                           uint64_t *full, uint64_t *empty, uint32_t &it, bool &alive,
                                           const PopC<typename Store<ST>::R> *pcs,
                                           const MomC<typename Store<ST>::R> *mcs)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    constexpr int RB = LB5_RB;
    constexpr size_t SLOTB = slot_bytes5<ST>();
    const StepParams<R> &p = P.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tile * LB_TILE_X + 4 * lane;
    const int jt = j0 + warp * RB;   /* this thread's first row */
    const size_t plane = p.plane;
    const R rho0 = p.rho0;
    const size_t ap = (size_t)p.pitch * p.ny;   /* carried-moment plane */

    bool own[RB], wall_row[RB], any = false;
    int wall[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int j = jt + r;
        own[r] = alive && j < p.ny && x0 < p.nx && ((p.tmap[(size_t)j * p.ntx + tile] & LB_TILE_HIGH) == s);
        wall[r] = -1;
        if (own[r] && j == 0 && p.wall_diffuse[0]) wall[r] = 0;
        if (own[r] && j == p.ny - 1 && p.wall_diffuse[1]) wall[r] = 1;
        wall_row[r] = wall[r] >= 0;
        any = any || own[r];
    }
    bool valid[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) valid[k] = x0 + k < p.nx;
    const bool full_quad = valid[3];

    /* carried moments of level n -> state of the collision */
    R rhod[RB][4], ux[RB][4], uy[RB][4], rho[RB][4], usq[RB][4], om[RB][4], gu[RB][4];
    const R *ain = static_cast<const R *>(p.aux_in);
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = own[r] && valid[k];
            const size_t n = (size_t)(jt + r) * p.pitch + x0 + k;
            rhod[r][k] = ok ? ain[n] : R(0);
            const R jx = ok ? ain[ap + n] : R(0), jy = ok ? ain[2 * ap + n] : R(0);
            rho[r][k] = rho0 + rhod[r][k];
            const R inv = R(1) / rho[r][k];
            ux[r][k] = jx * inv;
            uy[r][k] = jy * inv;
            usq[r][k] = ux[r][k] * ux[r][k] + uy[r][k] * uy[r][k];
            om[r][k] = p.dt / tau_of(p, rho[r][k]);
            if constexpr (FORCE) gu[r][k] = p.gx * ux[r][k] + p.gy * uy[r][k];
        }
    R nr[RB][4], nx_[RB][4], ny_[RB][4], num[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) nr[r][k] = nx_[r][k] = ny_[r][k] = num[r][k] = R(0);

    T *fout = static_cast<T *>(p.fout[s]) + (size_t)jt * p.pitch + (x0 + LB_GHOST);

#pragma unroll 1
    for (int a = 0; a < Q; ++a, ++it) {
        const int slot = it % LB5_STAGES;
        if (alive) alive = mbar_wait(&full[slot], (it / LB5_STAGES) & 1u, P.err, 1);
        if (alive && any) {
            const PopC<R> pc = pcs[a];
            const R winv = pc.winv, crx = pc.crx, cry = pc.cry, cxa = pc.cx, cya = pc.cy;
            /* slot row warp * RB + 2 + r holds row jt + r; column 4 + 4 lane is x0 */
            const T *sb = reinterpret_cast<const T *>(smem_base + (size_t)slot * SLOTB) + (warp * RB + 2) * LB5_W + 4 + 4 * lane;
            R v[RB][4];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                T raw[4];
                ld4(sb + r * LB5_W, raw);
#pragma unroll
                for (int k = 0; k < 4; ++k) v[r][k] = decode<ST>(raw[k], winv, rho0);
            }
            R inc[RB][4];
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const R eu = cxa * ux[r][k] + cya * uy[r][k];
                    inc[r][k] = om[r][k] * (deq(rhod[r][k], rho[r][k], eu, usq[r][k]) - v[r][k]);
                }
            if (crx != R(0)) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    T tl[2], tr[2];
                    ld2(sb + r * LB5_W - 2, tl);
                    ld2(sb + r * LB5_W + 4, tr);
                    const R l[2] = {decode<ST>(tl[0], winv, rho0), decode<ST>(tl[1], winv, rho0)};
                    const R rr[2] = {decode<ST>(tr[0], winv, rho0), decode<ST>(tr[1], winv, rho0)};
                    R Dx[4];
                    x_flux_diff(crx, pc.kx, l, v[r], rr, Dx);
#pragma unroll
                    for (int k = 0; k < 4; ++k) inc[r][k] = fma(-crx, Dx[k], inc[r][k]);
                }
            }
            if (cry != R(0)) {
                const bool up = cry > R(0);
                const R kfs = up ? pc.ky : -pc.ky;
                /* rows beyond the block: up: jt-2, jt-1, jt+RB; down: jt-1, jt+RB, jt+RB+1 */
                T h0[4], h1[4], h2[4];
                ld4(sb + (up ? -2 : -1) * LB5_W, h0);
                ld4(sb + (up ? -1 : RB) * LB5_W, h1);
                ld4(sb + (up ? RB : RB + 1) * LB5_W, h2);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    R W[RB + 3], Dy[RB];
                    const R a0 = decode<ST>(h0[k], winv, rho0), a1 = decode<ST>(h1[k], winv, rho0);
                    const R a2 = decode<ST>(h2[k], winv, rho0);
                    if (up) {
                        W[0] = a0;
                        W[1] = a1;
#pragma unroll
                        for (int r = 0; r < RB; ++r) W[2 + r] = v[r][k];
                        W[RB + 2] = a2;
                    } else {
                        W[0] = a0;
#pragma unroll
                        for (int r = 0; r < RB; ++r) W[1 + r] = v[r][k];
                        W[RB + 1] = a1;
                        W[RB + 2] = a2;
                    }
                    y_flux_window<R, RB>(kfs, W, Dy);
#pragma unroll
                    for (int r = 0; r < RB; ++r) inc[r][k] = fma(-cry, Dy[r], inc[r][k]);
                }
            }
            const R gxi = p.gx * cxa + p.gy * cya;
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (!own[r]) continue;
                R dn[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    R t = inc[r][k];
                    if constexpr (FORCE) {
                        const R eu = cxa * ux[r][k] + cya * uy[r][k];
                        t = fma(p.dt * rho[r][k], gxi + gxi * eu - gu[r][k], t);
                    }
                    dn[k] = v[r][k] + t;
                }
                if (wall_row[r]) {
                    const R xn = cya * (wall[r] == 0 ? R(1) : R(-1));
                    if (xn > R(0)) continue;   /* gas-bound: written by the wall post-pass */
                    if (xn < R(0)) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) num[r][k] = fma(-xn * pc.w, dn[k], num[r][k]);
                    }
                }
                T e[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    e[k] = p.sr ? encode_sr<ST>(dn[k], pc.w, rho0, sr_bits(x0 + k, jt + r, p.nx, a, p.step_key))
                                : encode<ST>(dn[k], pc.w, rho0);
                T *dst = fout + (size_t)a * plane + (size_t)r * p.pitch;
                if (full_quad) {
                    st4(dst, e);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (valid[k]) dst[k] = e[k];
                }
                /* moments of level n+1 from the values as stored, in population order
                 * and with the constants of the one-quad layout's moment pass */
                const MomC<R> mcon = mcs[a];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const R d = decode<ST>(e[k], mcon.winv, rho0);
                    nr[r][k] = fma(mcon.w, d, nr[r][k]);
                    nx_[r][k] = fma(mcon.wcx, d, nx_[r][k]);
                    ny_[r][k] = fma(mcon.wcy, d, ny_[r][k]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    if (!alive) return;
    R *aout = static_cast<R *>(p.aux_out);
    R *wnum = static_cast<R *>(p.wall_num);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (!own[r]) continue;
        const size_t n = (size_t)(jt + r) * p.pitch + x0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!valid[k]) continue;
            aout[n + k] = nr[r][k];
            aout[ap + n + k] = nx_[r][k];
            aout[2 * ap + n + k] = ny_[r][k];
            if (wall_row[r]) wnum[(size_t)wall[r] * p.pitch + x0 + k] = num[r][k];
        }
    }
}

template <int ST, bool FORCE>
__global__ void __launch_bounds__(32 * (LB5_NC + 1), 1) stream_kernel(const __grid_constant__ Stream5Params<ST> P)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr size_t SLOTB = slot_bytes5<ST>();
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)LB5_STAGES * SLOTB);
    uint64_t *empty = full + LB5_STAGES;
    const StepParams<R> &p = P.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        for (int k = 0; k < LB5_STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], LB5_NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == LB5_NC) {
        /* producer */
        if (lane != 0) return;
        uint32_t it = 0;
        bool ok = true;
        const uint32_t bytes = (uint32_t)(LB5_W * (LB5_TH + 4) * sizeof(T));
        for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
            const int tile = u % p.ntx, j0 = (u / p.ntx) * LB5_TH;
            const int sets = unit_sets5(p, tile, j0);
            for (int s = 0; s < 2 && ok; ++s) {
                if (!(sets & (1 << s))) continue;
                const int q = p.set[s].q;
                for (int a = 0; a < q && ok; ++a, ++it) {
                    const int slot = it % LB5_STAGES;
                    if (it >= LB5_STAGES) ok = mbar_wait(&empty[slot], ((it / LB5_STAGES) - 1) & 1u, P.err, 2);
                    if (!ok) break;
                    mbar_arrive_expect_tx(&full[slot], bytes);
                    /* storage row j0 is node row j0 - 2: the unit's rows and two halo rows each side */
                    tma_load_3d(smem + (size_t)slot * SLOTB, &P.map[s], &full[slot], tile * LB_TILE_X, j0, a);
                }
            }
        }
        if (!ok) {
            const uint32_t first = it > LB5_STAGES ? it - LB5_STAGES : 0;
            for (uint32_t k = first; k < it; ++k) {
                const int slot = k % LB5_STAGES;
                for (uint32_t n = 0; n < LB_SPIN_LIMIT && !mbar_try_wait(&full[slot], (k / LB5_STAGES) & 1u); ++n) {
                }
            }
        }
        return;
    }

    /* consumers */
    uint32_t it = 0;
    bool alive = true;
    for (int u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
        const int tile = u % p.ntx, j0 = (u / p.ntx) * LB5_TH;
        const int sets = unit_sets5(p, tile, j0);
#pragma unroll 1
        for (int s = 0; s < 2; ++s) {
            if (!(sets & (1 << s))) continue;
            const int q = p.set[s].q;
            if (q == 9) stream_set<ST, 9, FORCE>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
            else if (q == 16) stream_set<ST, 16, FORCE>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
            else stream_set<ST, 36, FORCE>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
        }
    }
}

template <int ST>
static size_t smem_bytes5()
{
    return (size_t)LB5_STAGES * slot_bytes5<ST>() + 2 * LB5_STAGES * sizeof(uint64_t);
}

template <int ST, bool FORCE>
static int launch5(const StepParams<typename Store<ST>::R> &p, const TmaMaps &maps, int *err, void *stream)
{
    static int configured = 0, nsm = 0;
    const size_t sm = smem_bytes5<ST>();
    if (!configured) {
        if (cudaFuncSetAttribute(stream_kernel<ST, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        configured = 1;
    }
    Stream5Params<ST> P;
    P.p = p;
    P.err = err;
    P.nunits = p.ntx * ((p.ny + LB5_TH - 1) / LB5_TH);
    for (int s = 0; s < 2; ++s) P.map[s] = maps.box5[s];
    int grid = nsm;
    if (grid > P.nunits) grid = P.nunits;
    stream_kernel<ST, FORCE><<<grid, 32 * (LB5_NC + 1), sm, static_cast<cudaStream_t>(stream)>>>(P);
    return 0;
}

int launch_stream(int store, const StepParams<float> &p, const TmaMaps &maps, int *err, void *stream)
{
    const bool f = p.has_force != 0;
    switch (store) {
        case 1: return f ? launch5<1, true>(p, maps, err, stream) : launch5<1, false>(p, maps, err, stream);
        case 2: return f ? launch5<2, true>(p, maps, err, stream) : launch5<2, false>(p, maps, err, stream);
        case 3: return f ? launch5<3, true>(p, maps, err, stream) : launch5<3, false>(p, maps, err, stream);
        case 4: return f ? launch5<4, true>(p, maps, err, stream) : launch5<4, false>(p, maps, err, stream);
        default: return -1;
    }
}

int stream_rows() { return LB5_TH; }
int stream_cols() { return LB5_W; }

}  // namespace lbk
