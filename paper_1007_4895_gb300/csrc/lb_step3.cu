/*
 * lb_step3.cu -- the fused time step, TMA-fed form.
 *
 * Same arithmetic as the Sec. 3.1 / 3.2 / 2.2 update of lb_step.cu. Work unit: a tile
 * of 128 columns x LB3_R rows (one row-block of one map tile). Each block runs
 * persistently over units and has one producer warp and LB3_NC consumer warps:
 *   - the producer streams, per population plane, the unit's rows (pass 1) and then the
 *     unit's rows plus two halo rows above and below and four halo columns on each side
 *     (pass 2) into a ring of shared-memory slots with cp.async.bulk.tensor, each slot
 *     guarded by a full / empty mbarrier pair;
 *   - each consumer thread owns 4 columns of one row; pass 1 sums density and momentum
 *     over the planes, pass 2 reads the radius-2 cross of each population from the slot
 *     and writes the new populations straight to global memory (16-byte stores).
 *   - a slot holds LB3_NP planes, so one barrier round trip serves several populations.
 * Every mbarrier wait is bounded; on expiry the block records the failure in an error
 * word, waits (bounded) for the copies it issued, and returns.
 * Ghost rows and columns live in the storage (see lb_internal.h), so every box the TMA
 * loads lies inside the tensor except, for ragged last tiles / row-blocks, columns and
 * rows past the padded end, which the TMA fills with zeros and nothing reads.
 */
#include <cuda.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_common.cuh"
#include "lb_tma.cuh"
#include "lb_tma.h"

namespace lbk {

#define LB3_NC 15                 /* consumer warps, one row each */
#define LB3_R LB3_NC              /* rows per unit */
#define LB3_W 136                 /* columns per slot row: 128 + 4 halo on each side */
#define LB3_NP 2                  /* population planes per slot */
#define LB3_STAGES 8

/* F_{k+1/2} - F_{k-1/2} along x for four nodes (Sec. 3.1), Courant number c (sign
 * decides the upwind side), limiter factor kf = (1 - |c|) / 2. */
template <typename R>
__device__ __forceinline__ void x_flux_diff(R c, R kf, const R l[2], const R v[4], const R r[2], R D[4])
{
    if (c > R(0)) {
        const R d[6] = {l[1] - l[0], v[0] - l[1], v[1] - v[0], v[2] - v[1], v[3] - v[2], r[0] - v[3]};
        R n[6], m[5];
#pragma unroll
        for (int k = 0; k < 6; ++k) n[k] = neg_part(d[k]);
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = minmod_n(d[k], d[k + 1], n[k], n[k + 1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = fma(kf, m[k + 1] - m[k], d[k + 1]);
    } else if (c < R(0)) {
        const R e[6] = {v[0] - l[1], v[1] - v[0], v[2] - v[1], v[3] - v[2], r[0] - v[3], r[1] - r[0]};
        R n[6], m[5];
#pragma unroll
        for (int k = 0; k < 6; ++k) n[k] = neg_part(e[k]);
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = minmod_n(e[k], e[k + 1], n[k], n[k + 1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = fma(-kf, m[k + 1] - m[k], e[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = R(0);
    }
}

/* Which sets the unit's rows use (bit s), skipping mode-A interface rows. */
template <typename R>
__device__ __forceinline__ int unit_sets(const StepParams<R> &p, int tile, int j0)
{
    int sets = 0;
    for (int r = 0; r < LB3_R && j0 + r < p.ny; ++r) {
        const uint8_t f = p.tmap[(size_t)(j0 + r) * p.ntx + tile];
        if (!(f & LB_TILE_IFACE)) sets |= 1 << (f & LB_TILE_HIGH);
    }
    return sets;
}

/* bytes per ring slot: the larger (pass-2) box, rounded to 1 KB so every slot start is
 * aligned for the bulk tensor copy */
template <int ST>
__host__ __device__ constexpr size_t slot_bytes3()
{
    return ((size_t)LB3_NP * LB3_W * (LB3_R + 4) * sizeof(typename Store<ST>::T) + 1023) / 1024 * 1024;
}

template <int ST>
struct Tma3Params {
    StepParams<typename Store<ST>::R> p;
    int *err;
    int nunits;
    CUtensorMap map1[2];   /* per set: box 136 x LB3_R x LB3_NP (pass 1) */
    CUtensorMap map2[2];   /* per set: box 136 x (LB3_R + 4) x LB3_NP (pass 2) */
};

template <int ST, int Q>
__device__ __forceinline__ void consume_set(const Tma3Params<ST> &P, int s, int tile, int j0, uint8_t *smem_base,
                                            uint64_t *full, uint64_t *empty, uint32_t &it, bool &alive,
                                            const PopC<typename Store<ST>::R> *pcs,
                                            const MomC<typename Store<ST>::R> *mcs)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const StepParams<R> &p = P.p;
    const SetConst<R> &c = p.set[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tile * 128 + 4 * lane;
    const int j = j0 + warp;                  /* this thread's row */
    const size_t plane = p.plane;
    const R rho0 = p.rho0;
    constexpr size_t SLOTB = slot_bytes3<ST>();
    constexpr int NSLOT = (Q + LB3_NP - 1) / LB3_NP;
    constexpr int P1 = LB3_W * LB3_R;         /* elements per plane in a pass-1 slot */
    constexpr int P2 = LB3_W * (LB3_R + 4);   /* elements per plane in a pass-2 slot */

    const uint8_t flags = j < p.ny ? p.tmap[(size_t)j * p.ntx + tile] : LB_TILE_IFACE;
    const bool mine = (j < p.ny) && (x0 < p.nx) && ((flags & LB_TILE_HIGH) == s) && !(flags & LB_TILE_IFACE);
    bool valid[4];
    bool full_row = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        valid[k] = (j < p.ny) && (x0 + k < p.nx) && !is_pressure_node(p, x0 + k, j);
        full_row = full_row && valid[k];
    }

    /* ---- pass 1: moments ---- */
    R rhod[4] = {R(0), R(0), R(0), R(0)}, ux[4] = {R(0), R(0), R(0), R(0)}, uy[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 1
    for (int k = 0; k < NSLOT; ++k, ++it) {
        const int slot = it % LB3_STAGES;
        if (alive) alive = mbar_wait(&full[slot], (it / LB3_STAGES) & 1u, P.err, 1);
        if (alive && mine) {
            const T *sl = reinterpret_cast<const T *>(smem_base + (size_t)slot * SLOTB) + warp * LB3_W + 4 + 4 * lane;
#pragma unroll
            for (int pl = 0; pl < LB3_NP; ++pl) {
                const int a = k * LB3_NP + pl;
                if (a >= Q) break;
                T raw[4];
                ld4(sl + pl * P1, raw);
                const MomC<R> mc = mcs[a];
                const R w = mc.w, wx = mc.wcx, wy = mc.wcy, winv = mc.winv;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const R d = decode<ST>(raw[m], winv, rho0);
                    rhod[m] = fma(w, d, rhod[m]);
                    ux[m] = fma(wx, d, ux[m]);
                    uy[m] = fma(wy, d, uy[m]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    R rho[4], usq[4], om[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        rho[m] = rho0 + rhod[m];
        const R inv = R(1) / rho[m];
        ux[m] *= inv;
        uy[m] *= inv;
        usq[m] = usq_of(ux[m], uy[m]);
        om[m] = p.dt / tau_of(p, inv);
    }

    int wall = -1;
    if (p.wall_diffuse[0] && j == 0 && mine) wall = 0;
    if (p.wall_diffuse[1] && j == p.ny - 1 && mine) wall = 1;
    const R nsgn = wall == 0 ? R(1) : R(-1);
    R num[4] = {R(0), R(0), R(0), R(0)};
    const bool edge = p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST);
    T *fout = static_cast<T *>(p.fout[s]) + (size_t)j * p.pitch + (x0 + LB_GHOST);
    int img[2];
    const int nimg = mine ? row_images(p, j, img) : 0;

    auto store_quad = [&](T *dst, const R dn[4], R w, int a) {
        T e[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
            e[m] = (a >= 0 && p.sr) ? encode_sr<ST>(dn[m], w, rho0, sr_bits(x0 + m, j, p.nx, a, p.step_key))
                                    : encode<ST>(dn[m], w, rho0);
        for (int t = -1; t < nimg; ++t) {
            T *d = t < 0 ? dst : dst + (ptrdiff_t)img[t] * p.pitch;
            if (full_row && !edge) {
                st4(d, e);
            } else {
                T *prow = d - (x0 + LB_GHOST);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (valid[m]) put1(p, prow, x0 + m, e[m]);
            }
        }
    };

    /* ---- pass 2: populations ---- */
#pragma unroll 1
    for (int k = 0; k < NSLOT; ++k, ++it) {
        const int slot = it % LB3_STAGES;
        if (alive) alive = mbar_wait(&full[slot], (it / LB3_STAGES) & 1u, P.err, 1);
        if (alive && mine) {
            /* slot row warp + 2 is this thread's row; rows warp .. warp + 4 its column */
            const T *base = reinterpret_cast<const T *>(smem_base + (size_t)slot * SLOTB) + (warp + 2) * LB3_W + 4 + 4 * lane;
#pragma unroll 1
            for (int pl = 0; pl < LB3_NP; ++pl) {
                const int a = k * LB3_NP + pl;
                if (a >= Q) break;
                const T *pa = base + pl * P2;
                const PopC<R> pc = pcs[a];
                const R winv = pc.winv;
                T raw[4];
                R v[4], l[2], r[2];
                ld4(pa, raw);
#pragma unroll
                for (int m = 0; m < 4; ++m) v[m] = decode<ST>(raw[m], winv, rho0);
                R Dx[4], Dy[4];
                const R crx = pc.crx, cry = pc.cry;
                if (crx != R(0)) {
                    T tl[2], tr[2];
                    ld2(pa - 2, tl);
                    ld2(pa + 4, tr);
                    l[0] = decode<ST>(tl[0], winv, rho0);
                    l[1] = decode<ST>(tl[1], winv, rho0);
                    r[0] = decode<ST>(tr[0], winv, rho0);
                    r[1] = decode<ST>(tr[1], winv, rho0);
                }
                x_flux_diff(crx, pc.kx, l, v, r, Dx);
                if (cry > R(0)) {
                    T t2[4], t1[4], tp[4];
                    ld4(pa - 2 * LB3_W, t2);
                    ld4(pa - LB3_W, t1);
                    ld4(pa + LB3_W, tp);
                    const R kf = pc.ky;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const R ym2 = decode<ST>(t2[m], winv, rho0), ym1 = decode<ST>(t1[m], winv, rho0);
                        const R yp1 = decode<ST>(tp[m], winv, rho0);
                        const R d0 = ym1 - ym2, d1 = v[m] - ym1, d2 = yp1 - v[m];
                        const R n1 = neg_part(d1);
                        Dy[m] = fma(kf, minmod_n(d1, d2, n1, neg_part(d2)) - minmod_n(d0, d1, neg_part(d0), n1), d1);
                    }
                } else if (cry < R(0)) {
                    T t1[4], tp[4], t2[4];
                    ld4(pa - LB3_W, t1);
                    ld4(pa + LB3_W, tp);
                    ld4(pa + 2 * LB3_W, t2);
                    const R kf = pc.ky;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const R ym1 = decode<ST>(t1[m], winv, rho0), yp1 = decode<ST>(tp[m], winv, rho0);
                        const R yp2 = decode<ST>(t2[m], winv, rho0);
                        const R e0 = v[m] - ym1, e1 = yp1 - v[m], e2 = yp2 - yp1;
                        const R n1 = neg_part(e1);
                        Dy[m] = fma(-kf, minmod_n(e1, e2, n1, neg_part(e2)) - minmod_n(e0, e1, neg_part(e0), n1), e1);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) Dy[m] = R(0);
                }
                R dn[4];
                const R cxa = pc.cx, cya = pc.cy;
                const R gxi = xi_dot(cxa, cya, p.gx, p.gy);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const R eu = xi_dot(cxa, cya, ux[m], uy[m]);
                    const R de = deq(rhod[m], rho[m], eu, usq[m]);
                    R inc = om[m] * (de - v[m]);
                    inc = fma(-crx, Dx[m], inc);
                    inc = fma(-cry, Dy[m], inc);
                    if (p.has_force) {
                        const R gu = xi_dot(p.gx, p.gy, ux[m], uy[m]);
                        inc = force_inc(p.dt * rho[m], gxi, eu, gu, inc);
                    }
                    dn[m] = v[m] + inc;
                }
                if (wall >= 0) {
                    const R xn = cya * nsgn;
                    if (xn > R(0)) continue;   /* replaced by the wall pass */
                    if (xn < R(0)) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) num[m] = fma(-xn * pc.w, dn[m], num[m]);
                    }
                }
                store_quad(fout + a * plane, dn, pc.w, a);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    if (!alive || !mine) return;

    /* diffuse wall */
    if (wall >= 0) {
        const R uwx = p.uw_x[wall], uwy = p.uw_y[wall];
        const R usw = uwx * uwx + uwy * uwy;
        const R kd = p.kdiff[s][wall], kout = p.kout[s][wall];
        R rwd[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rwd[m] = fma(rho0, kd, num[m]) / kout;
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if (c.cy[a] * nsgn <= R(0)) continue;
            const R ew = c.cx[a] * uwx + c.cy[a] * uwy;
            const R sm1 = ew + R(0.5) * (ew * ew - usw);
            R dn[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) dn[m] = fma(rwd[m] + rho0, sm1, rwd[m]);
            store_quad(fout + a * plane, dn, c.w[a], -1);
        }
    }

    /* mode B view of a row next to the other set */
    if (flags & LB_TILE_SHADOW) {
        const int t = 1 - s;
        const SetConst<R> &ct = p.set[t];
        R h[4][6];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int qq = 0; qq < 6; ++qq) h[m][qq] = R(0);
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const T *pr = fout + a * plane;
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (valid[m]) hermite_acc(c, a, decode<ST>(pr[m], c.winv[a], rho0), h[m]);
        }
        T *ft = static_cast<T *>(p.fout[t]) + (size_t)j * p.pitch;
#pragma unroll 1
        for (int b = 0; b < ct.q; ++b) {
            T *prow = ft + b * plane;
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (valid[m]) put1r(p, prow, x0 + m, j, encode<ST>(hermite_rebuild(ct, b, h[m]), ct.w[b], rho0));
        }
    }
}

template <int ST>
__global__ void __launch_bounds__(32 * (LB3_NC + 1), 1) step3_kernel(const __grid_constant__ Tma3Params<ST> P)
{
    using T = typename Store<ST>::T;
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr size_t SLOTB = slot_bytes3<ST>();
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)LB3_STAGES * SLOTB);
    uint64_t *empty = full + LB3_STAGES;
    const StepParams<typename Store<ST>::R> &p = P.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {
        for (int k = 0; k < LB3_STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], LB3_NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == LB3_NC) {
        /* producer */
        if (lane != 0) return;
        uint32_t it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < P.nunits && ok; u += gridDim.x) {
            const int tile = u % p.ntx, j0 = (u / p.ntx) * LB3_R;
            const int sets = unit_sets(p, tile, j0);
            for (int s = 0; s < 2 && ok; ++s) {
                if (!(sets & (1 << s))) continue;
                const int q = p.set[s].q;
                const int nslot = (q + LB3_NP - 1) / LB3_NP;
                for (int pass = 0; pass < 2 && ok; ++pass) {
                    const CUtensorMap *map = pass == 0 ? &P.map1[s] : &P.map2[s];
                    const uint32_t bytes = (uint32_t)(LB3_NP * LB3_W * (pass == 0 ? LB3_R : LB3_R + 4) * sizeof(T));
                    /* storage row of the box top: pass 1 starts at row j0, pass 2 two rows above */
                    const int y = pass == 0 ? j0 + LB_GHOST_ROWS : j0;
                    for (int k = 0; k < nslot && ok; ++k, ++it) {
                        const int slot = it % LB3_STAGES;
                        if (it >= LB3_STAGES) ok = mbar_wait(&empty[slot], ((it / LB3_STAGES) - 1) & 1u, P.err, 2);
                        if (!ok) break;
                        mbar_arrive_expect_tx(&full[slot], bytes);
                        /* planes past the last population are filled with zeros and unused */
                        tma_load_3d(smem + (size_t)slot * SLOTB, map, &full[slot], tile * 128, y, k * LB3_NP);
                    }
                }
            }
        }
        if (!ok) {
            /* wait (bounded) for the copies already issued before returning */
            const uint32_t first = it > LB3_STAGES ? it - LB3_STAGES : 0;
            for (uint32_t k = first; k < it; ++k) {
                const int slot = k % LB3_STAGES;
                for (uint32_t n = 0; n < LB_SPIN_LIMIT && !mbar_try_wait(&full[slot], (k / LB3_STAGES) & 1u); ++n) {
                }
            }
        }
        return;
    }

    /* consumers */
    uint32_t it = 0;
    bool alive = true;
    for (int u = blockIdx.x; u < P.nunits && alive; u += gridDim.x) {
        const int tile = u % p.ntx, j0 = (u / p.ntx) * LB3_R;
        const int sets = unit_sets(p, tile, j0);
#pragma unroll 1
        for (int s = 0; s < 2; ++s) {
            if (!(sets & (1 << s))) continue;
            const int q = p.set[s].q;
            if (q == 9) consume_set<ST, 9>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
            else if (q == 16) consume_set<ST, 16>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
            else consume_set<ST, 36>(P, s, tile, j0, smem, full, empty, it, alive, pc[s], mc[s]);
        }
    }
}

template <int ST>
static size_t smem_bytes3()
{
    return (size_t)LB3_STAGES * slot_bytes3<ST>() + 2 * LB3_STAGES * sizeof(uint64_t);
}

template <int ST>
static int launch3(const StepParams<typename Store<ST>::R> &p, const TmaMaps &maps, int *err, void *stream)
{
    static int configured = 0, nsm = 0;
    const size_t sm = smem_bytes3<ST>();
    if (!configured) {
        if (cudaFuncSetAttribute(step3_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return -1;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        configured = 1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step3_kernel<ST>, 32 * (LB3_NC + 1), sm) != cudaSuccess ||
        per_sm < 1)
        return -1;
    Tma3Params<ST> P;
    P.p = p;
    P.err = err;
    P.nunits = p.ntx * ((p.ny + LB3_R - 1) / LB3_R);
    for (int s = 0; s < 2; ++s) {
        P.map1[s] = maps.box1[s];
        P.map2[s] = maps.box2[s];
    }
    int grid = nsm * per_sm;
    if (grid > P.nunits) grid = P.nunits;
    step3_kernel<ST><<<grid, 32 * (LB3_NC + 1), sm, static_cast<cudaStream_t>(stream)>>>(P);
    return 0;
}

int launch_step3(int store, const StepParams<float> &p, const TmaMaps &maps, int *err, void *stream)
{
    switch (store) {
        case 1: return launch3<1>(p, maps, err, stream);
        case 2: return launch3<2>(p, maps, err, stream);
        case 3: return launch3<3>(p, maps, err, stream);
        case 4: return launch3<4>(p, maps, err, stream);
        default: return -1;
    }
}

int step3_rows() { return LB3_R; }
int step3_cols() { return LB3_W; }
int step3_planes() { return LB3_NP; }

}  // namespace lbk
