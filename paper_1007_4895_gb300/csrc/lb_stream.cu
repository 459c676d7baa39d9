/*
 * lb_stream.cu -- the fused time step, streamed form (layout 4).
 *
 * Same arithmetic as the Sec. 3.1 / 3.2 / 2.2 update of lb_step_impl.cuh, in the same
 * order, reorganised so that every population is read from memory exactly once:
 *   - the moments of level n are not summed again at step n: the step that wrote level
 *     n left, per node, sum w d, sum w xi_x d and sum w xi_y d of the values it stored
 *     (aux_in); this step sums them for level n+1 as it stores (aux_out);
 *   - work units are runs of at most LB5_TH rows of one set in one 128-column tile
 *     (built on the host, most work first); one producer warp per block takes units
 *     from a global queue and streams, for each population plane, the unit's rows plus
 *     two halo rows and four ghost columns on each side into a ring of shared-memory
 *     slots with cp.async.bulk.tensor, each slot guarded by a full / empty mbarrier
 *     pair and headed by the unit it belongs to;
 *   - each consumer thread owns 4 columns x LB5_RB rows, reads its radius-2 cross from
 *     the slot (the limited slope of a face between its two rows is formed once) and
 *     writes the new populations to global memory in 16-byte vectors.
 * The boundary work of step_cells is done here too, with the same arithmetic: periodic
 * ghost columns with every store; at the end of a unit the diffuse-wall overwrite (the
 * wall row's moments are then summed again, in population order, from its final values,
 * and its ghost rows written), the ghost rows of periodic-y edge rows, and the mode-B
 * rebuild of shadow nodes from the Hermite sums of their final values (summed as they
 * are stored). Pressure columns are left to the pressure pass, which also writes their
 * carried moments. Every mbarrier wait is bounded; on expiry
 * the block records the failure in an error word, waits (bounded) for the copies it
 * issued, and returns.
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
    const int4 *units;      /* (tile, first row, rows, set), most work first */
    int nunits;
    unsigned int *queue;    /* next unit to take; zero at launch */
    CUtensorMap map[2];     /* per set: box 136 x (LB5_TH + 4) x 1 */
};

/* dynamic shared memory: LB5_STAGES slots, full and empty barriers, slot headers, then
 * three side sums per node of each consumer thread (R [RB * 4 * 3][LB5_NC * 32]) */
template <int ST>
__host__ __device__ constexpr size_t stream_xs_offset5()
{
    return (size_t)LB5_STAGES * slot_bytes5<ST>() + 2 * LB5_STAGES * sizeof(uint64_t) + LB5_STAGES * sizeof(int);
}
template <int ST>
__host__ __device__ constexpr size_t smem_bytes5()
{
    return stream_xs_offset5<ST>() + (size_t)LB5_RB * 4 * 3 * LB5_NC * 32 * sizeof(typename Store<ST>::R);
}

/* second-order Hermite weights of one population: w (xi_x^2-1), w xi_x xi_y, w (xi_y^2-1) */
template <typename R>
struct alignas(4 * sizeof(R)) HerC {
    R wxx, wxy, wyy, pad;
};

/* One unit (tile, rows j0 .. j0 + nrows - 1 of set s) over its Q population slots; the
 * slot of population 0 has already been waited for. */
template <int ST, int Q, bool FORCE>
__device__ __forceinline__ void stream_set(const Stream5Params<ST> &P, int s, int tile, int j0, int nrows,
                                           uint8_t *smem_base, uint64_t *full, uint64_t *empty, uint32_t &it,
                                           bool &alive, const PopC<typename Store<ST>::R> *pcs,
                                           const MomC<typename Store<ST>::R> *mcs,
                                           const HerC<typename Store<ST>::R> *hcs)
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

    bool own[RB], wall_row[RB], shadow[RB], any = false;
    int wall[RB], nimg[RB], img0[RB], img1[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int j = jt + r;
        const uint8_t flags = (j < p.ny) ? p.tmap[(size_t)j * p.ntx + tile] : 0;
        own[r] = alive && j < j0 + nrows && j < p.ny && x0 < p.nx && ((flags & LB_TILE_HIGH) == s);
        wall[r] = -1;
        if (own[r] && j == 0 && p.wall_diffuse[0]) wall[r] = 0;
        if (own[r] && j == p.ny - 1 && p.wall_diffuse[1]) wall[r] = 1;
        wall_row[r] = wall[r] >= 0;
        shadow[r] = own[r] && (flags & LB_TILE_SHADOW);
        int im[2] = {0, 0};
        nimg[r] = own[r] ? row_images(p, j, im) : 0;
        img0[r] = im[0];
        img1[r] = im[1];
        any = any || own[r];
    }
    /* nodes this thread stores: inside the lattice and not a pressure column (set by the
     * pressure pass; the corner nodes of a diffuse wall are wall nodes) */
    bool valid[RB][4], full_quad[RB];
    const bool near_x_edge = p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        full_quad[r] = !near_x_edge;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            valid[r][k] = own[r] && x0 + k < p.nx && !is_pressure_node(p, x0 + k, jt + r);
            full_quad[r] = full_quad[r] && valid[r][k];
        }
    }

    /* carried moments of level n -> state of the collision */
    R rhod[RB][4], ux[RB][4], uy[RB][4], rho[RB][4], usq[RB][4], om[RB][4], gu[RB][4];
    const R *ain = static_cast<const R *>(p.aux_in);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const size_t n = (size_t)(jt + r) * p.pitch + x0;
        R jx[4], jy[4];
        if (full_quad[r]) {
            ld4(ain + n, rhod[r]);
            ld4(ain + ap + n, jx);
            ld4(ain + 2 * ap + n, jy);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = valid[r][k];
                rhod[r][k] = ok ? ain[n + k] : R(0);
                jx[k] = ok ? ain[ap + n + k] : R(0);
                jy[k] = ok ? ain[2 * ap + n + k] : R(0);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rho[r][k] = rho0 + rhod[r][k];
            const R inv = R(1) / rho[r][k];
            ux[r][k] = jx[k] * inv;
            uy[r][k] = jy[k] * inv;
            usq[r][k] = usq_of(ux[r][k], uy[r][k]);
            om[r][k] = p.dt / tau_of(p, inv);
            if constexpr (FORCE) gu[r][k] = xi_dot(p.gx, p.gy, ux[r][k], uy[r][k]);
        }
    }
    /* sums of level n+1 over the values as stored: nr, nx_, ny_ = sum w d, w xi_x d,
     * w xi_y d (the carried moments, and the first three Hermite coefficients of a
     * shadow); ex = sum_out |xi.n| w dn on a wall row, or the three second-order Hermite
     * sums w (xi_x^2-1) d, w xi_x xi_y d, w (xi_y^2-1) d on a shadow row */
    R nr[RB][4], nx_[RB][4], ny_[RB][4];
    bool hsum[RB];
    /* ex lives in shared memory (few rows need it), one column per consumer thread */
    R *xs = reinterpret_cast<R *>(smem_base + stream_xs_offset5<ST>()) + threadIdx.x;
#define LB5_EX(r, k, m) xs[(((r) * 4 + (k)) * 3 + (m)) * (LB5_NC * 32)]
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        hsum[r] = shadow[r] && !wall_row[r];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nr[r][k] = nx_[r][k] = ny_[r][k] = R(0);
            if (wall_row[r] || hsum[r]) LB5_EX(r, k, 0) = LB5_EX(r, k, 1) = LB5_EX(r, k, 2) = R(0);
        }
    }

    T *fout = static_cast<T *>(p.fout[s]) + (size_t)jt * p.pitch + (x0 + LB_GHOST);
    /* a row's four values (with their periodic ghost columns); the ghost-row copies of a
     * wall row or of a periodic-y edge row are written once its values are final, at
     * the end of the unit */
    auto store_one = [&](T *d, int r, const T e[4]) {
        if (full_quad[r]) {
            st4(d, e);
        } else {
            T *prow = d - (x0 + LB_GHOST);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[r][k]) put1(p, prow, x0 + k, e[k]);
        }
    };
    auto store_images = [&](T *dst, int r, const T e[4]) {
        if (nimg[r] > 0) store_one(dst + (ptrdiff_t)img0[r] * p.pitch, r, e);
        if (nimg[r] > 1) store_one(dst + (ptrdiff_t)img1[r] * p.pitch, r, e);
    };
    auto store_row = [&](T *dst, int r, const T e[4]) {
        store_one(dst, r, e);
        store_images(dst, r, e);
    };
    auto load_one = [&](const T *f, int r, T raw[4]) {
        if (full_quad[r]) {
            ld4(f, raw);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) raw[k] = valid[r][k] ? f[k] : T();
        }
    };

#pragma unroll 1
    for (int a = 0; a < Q; ++a, ++it) {
        const int slot = it % LB5_STAGES;
        if (alive && a > 0) alive = mbar_wait(&full[slot], (it / LB5_STAGES) & 1u, P.err, 1);
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
                    const R eu = xi_dot(cxa, cya, ux[r][k], uy[r][k]);
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
            const R gxi = xi_dot(cxa, cya, p.gx, p.gy);
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                if (!own[r]) continue;
                R dn[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    R t = inc[r][k];
                    if constexpr (FORCE) {
                        const R eu = xi_dot(cxa, cya, ux[r][k], uy[r][k]);
                        t = force_inc(p.dt * rho[r][k], gxi, eu, gu[r][k], t);
                    }
                    dn[k] = v[r][k] + t;
                }
                if (wall_row[r]) {
                    const R xn = cya * (wall[r] == 0 ? R(1) : R(-1));
                    if (xn > R(0)) continue;   /* gas-bound: set by the wall overwrite below */
                    if (xn < R(0)) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) LB5_EX(r, k, 0) = fma(-xn * pc.w, dn[k], LB5_EX(r, k, 0));
                    }
                }
                T e[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    e[k] = p.sr ? encode_sr<ST>(dn[k], pc.w, rho0, sr_bits(x0 + k, jt + r, p.nx, a, p.step_key))
                                : encode<ST>(dn[k], pc.w, rho0);
                store_one(fout + (size_t)a * plane + (size_t)r * p.pitch, r, e);
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
                if (hsum[r]) {
                    const HerC<R> hcon = hcs[a];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const R d = decode<ST>(e[k], mcon.winv, rho0);
                        LB5_EX(r, k, 0) = fma(hcon.wxx, d, LB5_EX(r, k, 0));
                        LB5_EX(r, k, 1) = fma(hcon.wxy, d, LB5_EX(r, k, 1));
                        LB5_EX(r, k, 2) = fma(hcon.wyy, d, LB5_EX(r, k, 2));
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }
    if (!alive) return;
    const SetConst<R> &c = p.set[s];
    /* diffuse wall: f_out = rho_W S(u_W) with zero net mass flux, as step_cells part 4;
     * then the wall row's sums again from all its final values in population order */
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (!wall_row[r]) continue;
        const int wl = wall[r];
        const R nsgn = wl == 0 ? R(1) : R(-1);
        const R uwx = p.uw_x[wl], uwy = p.uw_y[wl];
        const R usw = uwx * uwx + uwy * uwy;
        const R kd = p.kdiff[s][wl], kout = p.kout[s][wl];
        R rwd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rwd[k] = fma(rho0, kd, LB5_EX(r, k, 0)) / kout;
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if (c.cy[a] * nsgn <= R(0)) continue;
            const R ew = c.cx[a] * uwx + c.cy[a] * uwy;
            const R sm1 = ew + R(0.5) * (ew * ew - usw);
            T e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = encode<ST>(fma(rwd[k] + rho0, sm1, rwd[k]), c.w[a], rho0);
            store_one(fout + (size_t)a * plane + (size_t)r * p.pitch, r, e);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) nr[r][k] = nx_[r][k] = ny_[r][k] = LB5_EX(r, k, 0) = LB5_EX(r, k, 1) = LB5_EX(r, k, 2) = R(0);
#pragma unroll 4
        for (int a = 0; a < Q; ++a) {
            T *f = fout + (size_t)a * plane + (size_t)r * p.pitch;
            T raw[4];
            load_one(f, r, raw);
            store_images(f, r, raw);
            const MomC<R> mcon = mcs[a];
            const HerC<R> hcon = hcs[a];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const R d = decode<ST>(raw[k], mcon.winv, rho0);
                nr[r][k] = fma(mcon.w, d, nr[r][k]);
                nx_[r][k] = fma(mcon.wcx, d, nx_[r][k]);
                ny_[r][k] = fma(mcon.wcy, d, ny_[r][k]);
                if (shadow[r]) {
                    LB5_EX(r, k, 0) = fma(hcon.wxx, d, LB5_EX(r, k, 0));
                    LB5_EX(r, k, 1) = fma(hcon.wxy, d, LB5_EX(r, k, 1));
                    LB5_EX(r, k, 2) = fma(hcon.wyy, d, LB5_EX(r, k, 2));
                }
            }
        }
    }
    /* ghost-row copies of the other rows that have them (periodic y) */
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (wall_row[r] || nimg[r] == 0) continue;
#pragma unroll 4
        for (int a = 0; a < Q; ++a) {
            T *f = fout + (size_t)a * plane + (size_t)r * p.pitch;
            T raw[4];
            load_one(f, r, raw);
            store_images(f, r, raw);
        }
    }
    /* mode B: the node as the other set's readers will see it, as step_cells part 5,
     * from the Hermite sums of its final values */
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (!shadow[r]) continue;
        const SetConst<R> &ct = p.set[1 - s];
        T *ftd = static_cast<T *>(p.fout[1 - s]) + (size_t)(jt + r) * p.pitch + (x0 + LB_GHOST);
#pragma unroll 1
        for (int b = 0; b < ct.q; ++b) {
            T e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const R h[6] = {nr[r][k], nx_[r][k], ny_[r][k], LB5_EX(r, k, 0), LB5_EX(r, k, 1), LB5_EX(r, k, 2)};
                e[k] = encode<ST>(hermite_rebuild(ct, b, h), ct.w[b], rho0);
            }
            store_row(ftd + (size_t)b * plane, r, e);
        }
    }
#undef LB5_EX
    R *aout = static_cast<R *>(p.aux_out);
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const size_t n = (size_t)(jt + r) * p.pitch + x0;
        if (full_quad[r]) {
            st4(aout + n, nr[r]);
            st4(aout + ap + n, nx_[r]);
            st4(aout + 2 * ap + n, ny_[r]);
            continue;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!valid[r][k]) continue;
            aout[n + k] = nr[r][k];
            aout[ap + n + k] = nx_[r][k];
            aout[2 * ap + n + k] = ny_[r][k];
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
    int *head = reinterpret_cast<int *>(empty + LB5_STAGES);   /* unit of each slot */
    const StepParams<R> &p = P.p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    __shared__ HerC<R> hc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < 2 * LB_QMAX; i += blockDim.x) {
        const int st = i / LB_QMAX, a = i % LB_QMAX;
        const SetConst<R> &c = p.set[st];
        if (a < c.q) hc[st][a] = HerC<R>{c.wxx[a], c.wxy[a], c.wyy[a], R(0)};
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < LB5_STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], LB5_NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == LB5_NC) {
        /* producer: takes units from the queue; slot header = unit index, -1 = no more */
        if (lane != 0) return;
        uint32_t it = 0;
        bool ok = true;
        const uint32_t bytes = (uint32_t)(LB5_W * (LB5_TH + 4) * sizeof(T));
        for (;;) {
            const unsigned k = atomicAdd(P.queue, 1u);
            const int u = k < (unsigned)P.nunits ? (int)k : -1;
            const int4 un = u >= 0 ? P.units[u] : make_int4(0, 0, 0, 0);
            const int q = u >= 0 ? p.set[un.w].q : 1;
            for (int a = 0; a < q && ok; ++a, ++it) {
                const int slot = it % LB5_STAGES;
                if (it >= LB5_STAGES) ok = mbar_wait(&empty[slot], ((it / LB5_STAGES) - 1) & 1u, P.err, 2);
                if (!ok) break;
                head[slot] = u;
                if (u < 0) {
                    mbar_arrive(&full[slot]);   /* end marker: nothing to copy */
                } else {
                    mbar_arrive_expect_tx(&full[slot], bytes);
                    /* storage row j0 is node row j0 - 2: the unit's rows and two halo rows each side */
                    tma_load_3d(smem + (size_t)slot * SLOTB, &P.map[un.w], &full[slot], un.x * LB_TILE_X, un.y, a);
                }
            }
            if (u < 0 || !ok) break;
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

    /* consumers: the unit of the next slot is in its header */
    uint32_t it = 0;
    bool alive = true;
    while (alive) {
        const int slot = it % LB5_STAGES;
        alive = mbar_wait(&full[slot], (it / LB5_STAGES) & 1u, P.err, 1);
        if (!alive) break;
        const int u = *(volatile int *)&head[slot];
        if (u < 0) break;
        const int4 un = P.units[u];
        const int q = p.set[un.w].q;
        if (q == 9) stream_set<ST, 9, FORCE>(P, un.w, un.x, un.y, un.z, smem, full, empty, it, alive, pc[un.w], mc[un.w], hc[un.w]);
        else if (q == 16)
            stream_set<ST, 16, FORCE>(P, un.w, un.x, un.y, un.z, smem, full, empty, it, alive, pc[un.w], mc[un.w], hc[un.w]);
        else stream_set<ST, 36, FORCE>(P, un.w, un.x, un.y, un.z, smem, full, empty, it, alive, pc[un.w], mc[un.w], hc[un.w]);
    }
}


/* Self-test of the bounded wait: one thread waits on an mbarrier that nothing
 * completes, gives up after `polls` polls, records `code` in *err and returns. */
__global__ void wait_selftest_kernel(int *err, uint32_t polls, int code)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0, err, code, polls);
}

int launch_wait_selftest(int *err, uint32_t polls, int code, void *stream)
{
    wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err, polls, code);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int ST, bool FORCE>
static int launch5(const StepParams<typename Store<ST>::R> &p, const TmaMaps &maps, const int4 *units, int nunits,
                   unsigned int *queue, int *err, void *stream)
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
    if (nunits < 1) return 0;
    Stream5Params<ST> P;
    P.p = p;
    P.err = err;
    P.units = units;
    P.nunits = nunits;
    P.queue = queue;
    for (int s = 0; s < 2; ++s) P.map[s] = maps.box5[s];
    int grid = nsm;
    if (grid > nunits) grid = nunits;
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned int), static_cast<cudaStream_t>(stream)) != cudaSuccess) return -1;
    stream_kernel<ST, FORCE><<<grid, 32 * (LB5_NC + 1), sm, static_cast<cudaStream_t>(stream)>>>(P);
    return 0;
}

int launch_stream(int store, const StepParams<float> &p, const TmaMaps &maps, const int4 *units, int nunits,
                  unsigned int *queue, int *err, void *stream)
{
    const bool f = p.has_force != 0;
#define LB5_CASE(ST)                                                                        \
    case ST:                                                                                \
        return f ? launch5<ST, true>(p, maps, units, nunits, queue, err, stream)            \
                 : launch5<ST, false>(p, maps, units, nunits, queue, err, stream)
    switch (store) {
        LB5_CASE(1);
        LB5_CASE(2);
        LB5_CASE(3);
        LB5_CASE(4);
        default: return -1;
    }
#undef LB5_CASE
}

int stream_rows() { return LB5_TH; }
int stream_cols() { return LB5_W; }

}  // namespace lbk
