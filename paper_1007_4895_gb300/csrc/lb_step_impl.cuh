/*
 * lb_step_impl.cuh -- the fused time step kernel (one node quad per thread).
 *
 * One thread owns four consecutive nodes of one row (one 16-byte FP32 vector per
 * plane). For every node it:
 *   1. sums density and momentum over its set's populations (Eq. (demoeq) moments);
 *   2. derives tau from the local density (Eq. (KN): collision rate p / mu);
 *   3. for each population, reads the radius-2 cross of the Sec. 3.1 stencil (x
 *      neighbours from two 2-element vectors beside its own, y neighbours from the rows
 *      above and below; ghost rows are copies of the wall row, Sec. 3.2), forms the two
 *      limited face fluxes in x and in y (minmod, mirrored for negative velocities), and
 *      applies the forward-Euler update with BGK collision towards Eq. (demoeq) and the
 *      Eq. (demoforce) body force;
 *   4. on a diffuse wall row, replaces the gas-bound populations by rho_W S(u_W)
 *      (Sec. 3.2) with rho_W from the streamed wall-bound populations;
 *   5. in mode B, on tiles that neighbour the other set, also writes the node rebuilt
 *      in the other set from its second-order Hermite coefficients (Sec. 2.2), so that
 *      the other set's readers find it at the next step.
 * The stencil reads only level n and writes only level n+1.
 * Each storage format is instantiated in a translation unit of its own (lb_step_st*.cu).
 */
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "lb_common.cuh"

namespace lbk {

#define LB_BX 32
#define LB_BY LB_STEP_BY
/* The one-quad kernel per storage format: the resident blocks per SM its register budget
 * is sized for, and whether it loads population a+1's stencil while computing population
 * a. Chosen by measurement: with FP32 values the prefetch pays at 128 registers (two
 * blocks per SM); with 16-bit values the kernel runs faster at 80 registers (three
 * blocks) without it. */
template <int ST>
__host__ __device__ constexpr int step_min_blocks() { return (ST == 3 || ST == 4) ? 3 : 2; }
template <int ST>
__host__ __device__ constexpr bool step_prefetch() { return ST == 1 || ST == 2; }
/* populations whose moment loads are issued together in the moments pass (measured:
 * 12 rather than 4 takes the 16384 x 128 channel from 152.5 to 146.3 us per step) */
#ifndef LB_MOM_UNROLL
#define LB_MOM_UNROLL 12
#endif
constexpr int kMomUnroll = LB_MOM_UNROLL;

/* Flux difference F_{k+1/2} - F_{k-1/2} along one axis for NQ (2 or 4) nodes in a row
 * (Sec. 3.1), Courant number c, limiter factor kf = (1 - |c|) / 2. l[0..1] are the
 * values at nodes x0-2, x0-1, v[0..NQ-1] the thread's own, r[0..1] those at x0+NQ,
 * x0+NQ+1. A node's result depends only on its own neighbourhood, so it is the same
 * for either NQ. */
template <int NQ = 4, typename R>
__device__ __forceinline__ void x_flux_diff(R c, R kf, const R l[2], const R v[NQ], const R r[2], R D[NQ])
{
    if (c > R(0)) {
        /* upwind node k: F_{k+1/2} = f_k + kf minmod(f_k - f_{k-1}, f_{k+1} - f_k) */
        R d[NQ + 2];
        d[0] = l[1] - l[0];
        d[1] = v[0] - l[1];
#pragma unroll
        for (int k = 1; k < NQ; ++k) d[k + 1] = v[k] - v[k - 1];
        d[NQ + 1] = r[0] - v[NQ - 1];
        R n[NQ + 2], m[NQ + 1];
#pragma unroll
        for (int k = 0; k < NQ + 2; ++k) n[k] = neg_part(d[k]);
#pragma unroll
        for (int k = 0; k < NQ + 1; ++k) m[k] = minmod_n(d[k], d[k + 1], n[k], n[k + 1]);
#pragma unroll
        for (int k = 0; k < NQ; ++k) D[k] = fma(kf, m[k + 1] - m[k], d[k + 1]);
    } else if (c < R(0)) {
        /* mirror image: upwind node k+1 */
        R e[NQ + 2];
        e[0] = v[0] - l[1];
#pragma unroll
        for (int k = 1; k < NQ; ++k) e[k] = v[k] - v[k - 1];
        e[NQ] = r[0] - v[NQ - 1];
        e[NQ + 1] = r[1] - r[0];
        R n[NQ + 2], m[NQ + 1];
#pragma unroll
        for (int k = 0; k < NQ + 2; ++k) n[k] = neg_part(e[k]);
#pragma unroll
        for (int k = 0; k < NQ + 1; ++k) m[k] = minmod_n(e[k], e[k + 1], n[k], n[k + 1]);
#pragma unroll
        for (int k = 0; k < NQ; ++k) D[k] = fma(-kf, m[k + 1] - m[k], e[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < NQ; ++k) D[k] = R(0);
    }
}

/* Stored values one population needs for a quad: its own four, two beside them on each
 * side (x flux, when xi_x != 0) and three rows on the upwind / downwind sides (y flux,
 * when xi_y != 0: rows j-2, j-1, j+1 for xi_y > 0, rows j-1, j+1, j+2 for xi_y < 0). */
template <typename T, int NQ = 4>
struct QuadStencil {
    T v[NQ], l[2], r[2], y0[NQ], y1[NQ], y2[NQ];
};

/* PF: load population a + 1 while population a is computed (one-deep software
 * pipeline), for kernels whose threads are few and latency-bound. */
template <int ST, int Q, bool PF = false, int NQ = 4, bool COL = false>
__device__ __forceinline__ void step_cells(const StepParams<typename Store<ST>::R> &p, int s, uint8_t flags, int x0,
                                           int j, const PopC<typename Store<ST>::R> *pcs,
                                           const MomC<typename Store<ST>::R> *mcs)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const SetConst<R> &c = p.set[s];
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]);
    T *__restrict__ fout = static_cast<T *>(p.fout[s]);
    const size_t plane = p.plane;
    const size_t row0 = (size_t)j * p.pitch + (size_t)(x0 + LB_GHOST);
    const ptrdiff_t om2 = (ptrdiff_t)(row_at(p, j - 2) - j) * p.pitch;
    const ptrdiff_t om1 = (ptrdiff_t)(row_at(p, j - 1) - j) * p.pitch;
    const ptrdiff_t op1 = (ptrdiff_t)(row_at(p, j + 1) - j) * p.pitch;
    const ptrdiff_t op2 = (ptrdiff_t)(row_at(p, j + 2) - j) * p.pitch;
    const R rho0 = p.rho0;
    /* COL: per-column reference density; dl[i] = delta at column x0 - 2 + i (node k at
     * i = k + 2, its x neighbours l at 0, 1 and r at NQ + 2, NQ + 3) */
    R dl[NQ + 4];
    if constexpr (COL) {
#pragma unroll
        for (int i = 0; i < NQ + 4; ++i) dl[i] = p.dcol[x0 + LB_GHOST - 2 + i];
    }
    auto dec = [&](T raw, R winv, int i) -> R {
        if constexpr (COL) return decode_col<ST>(raw, winv, rho0, dl[i]);
        else return decode<ST>(raw, winv, rho0);
    };
    auto enc = [&](R d, R w, int i) -> T {
        if constexpr (COL) return encode_col<ST>(d, w, rho0, dl[i]);
        else return encode<ST>(d, w, rho0);
    };
    auto enc_sr = [&](R d, R w, int i, uint32_t bits) -> T {
        if constexpr (COL) return encode_sr<ST>(d - dl[i], w, rho0, bits);
        else return encode_sr<ST>(d, w, rho0, bits);
    };

    /* 1. moments */
    R rhod[NQ], jx[NQ], jy[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) rhod[k] = jx[k] = jy[k] = R(0);
#pragma unroll kMomUnroll
    for (int a = 0; a < Q; ++a) {
        T raw[NQ];
        ldn<NQ>(fin + a * plane + row0, raw);
        const MomC<R> mc = mcs[a];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            R d = dec(raw[k], mc.winv, k + 2);
            rhod[k] = fma(mc.w, d, rhod[k]);
            jx[k] = fma(mc.wcx, d, jx[k]);
            jy[k] = fma(mc.wcy, d, jy[k]);
        }
    }
    /* 2. macroscopic state and relaxation */
    R rho[NQ], ux[NQ], uy[NQ], usq[NQ], om[NQ], gu[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        rho[k] = rho0 + rhod[k];
        R inv = R(1) / rho[k];
        ux[k] = jx[k] * inv;
        uy[k] = jy[k] * inv;
        usq[k] = usq_of(ux[k], uy[k]);
        om[k] = p.dt / tau_of(p, inv);
        gu[k] = xi_dot(p.gx, p.gy, ux[k], uy[k]);
    }

    int wall = -1;
    if (j == 0 && p.wall_diffuse[0]) wall = 0;
    if (j == p.ny - 1 && p.wall_diffuse[1]) wall = 1;
    const R nsgn = wall == 0 ? R(1) : R(-1);

    bool valid[NQ];
    bool full = true;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        int x = x0 + k;
        valid[k] = x < p.nx && !is_pressure_node(p, x, j);
        full = full && valid[k];
    }
    const bool near_x_edge = p.periodic_x && (x0 < LB_GHOST || x0 + NQ - 1 >= p.nx - LB_GHOST);

    int img[2];
    const int nimg = row_images(p, j, img);
    /* a quad with no ghost copy (no image row, no ghost column, every node stored) */
    const bool plain_store = nimg == 0 && full && !near_x_edge;
    /* a >= 0: an updated population (stochastically rounded when p.sr); a < 0: a value
     * set by the wall (rounded to nearest) */
    auto store_quad = [&](T *dst, const R dn[NQ], R w, int a) {
        T e[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k)
            e[k] = (a >= 0 && p.sr) ? enc_sr(dn[k], w, k + 2, sr_bits(x0 + k, j, p.nx, a, p.step_key))
                                    : enc(dn[k], w, k + 2);
        if (plain_store) {
            stn<NQ>(dst, e);
            return;
        }
        for (int t = -1; t < nimg; ++t) {
            T *d = t < 0 ? dst : dst + (ptrdiff_t)img[t] * p.pitch;
            if (full && !near_x_edge) {
                stn<NQ>(d, e);
            } else {
                T *prow = d - (x0 + LB_GHOST);
#pragma unroll
                for (int k = 0; k < NQ; ++k)
                    if (valid[k]) put1(p, prow, x0 + k, e[k]);
            }
        }
    };

    /* 3. stencil, fluxes, collision, force (PF: loads one population ahead) */
    R num[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) num[k] = R(0);
    if constexpr (!PF) {
    #pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const T *pa = fin + a * plane + row0;
            const PopC<R> pc = pcs[a];
            const R winv = pc.winv;
            T raw[NQ];
            R v[NQ], l[2], r[2];
            ldn<NQ>(pa, raw);
    #pragma unroll
            for (int k = 0; k < NQ; ++k) v[k] = dec(raw[k], winv, k + 2);
            R Dx[NQ], Dy[NQ];
            const R crx = pc.crx, cry = pc.cry;
            if (crx != R(0)) {
                T tl[2], tr[2];
                ld2(pa - 2, tl);
                ld2(pa + NQ, tr);
                l[0] = dec(tl[0], winv, 0);
                l[1] = dec(tl[1], winv, 1);
                r[0] = dec(tr[0], winv, NQ + 2);
                r[1] = dec(tr[1], winv, NQ + 3);
            }
            x_flux_diff<NQ>(crx, pc.kx, l, v, r, Dx);
            if (cry > R(0)) {
                T t2[NQ], t1[NQ], tp[NQ];
                ldn<NQ>(pa + om2, t2);
                ldn<NQ>(pa + om1, t1);
                ldn<NQ>(pa + op1, tp);
                const R kf = pc.ky;
    #pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R ym2 = dec(t2[k], winv, k + 2), ym1 = dec(t1[k], winv, k + 2);
                    R yp1 = dec(tp[k], winv, k + 2);
                    R d0 = ym1 - ym2, d1 = v[k] - ym1, d2 = yp1 - v[k];
                    const R n1 = neg_part(d1);
                    Dy[k] = fma(kf, minmod_n(d1, d2, n1, neg_part(d2)) - minmod_n(d0, d1, neg_part(d0), n1), d1);
                }
            } else if (cry < R(0)) {
                T t1[NQ], tp[NQ], t2[NQ];
                ldn<NQ>(pa + om1, t1);
                ldn<NQ>(pa + op1, tp);
                ldn<NQ>(pa + op2, t2);
                const R kf = pc.ky;
    #pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R ym1 = dec(t1[k], winv, k + 2), yp1 = dec(tp[k], winv, k + 2);
                    R yp2 = dec(t2[k], winv, k + 2);
                    R e0 = v[k] - ym1, e1 = yp1 - v[k], e2 = yp2 - yp1;
                    const R n1 = neg_part(e1);
                    Dy[k] = fma(-kf, minmod_n(e1, e2, n1, neg_part(e2)) - minmod_n(e0, e1, neg_part(e0), n1), e1);
                }
            } else {
    #pragma unroll
                for (int k = 0; k < NQ; ++k) Dy[k] = R(0);
            }
            R dn[NQ];
            const R cxa = pc.cx, cya = pc.cy;
            const R gxi = xi_dot(cxa, cya, p.gx, p.gy);
    #pragma unroll
            for (int k = 0; k < NQ; ++k) {
                R eu = xi_dot(cxa, cya, ux[k], uy[k]);
                R de = deq(rhod[k], rho[k], eu, usq[k]);
                /* sum the small increments first and round onto the stored magnitude once */
                R inc = om[k] * (de - v[k]);
                inc = fma(-crx, Dx[k], inc);
                inc = fma(-cry, Dy[k], inc);
                if (p.has_force) inc = force_inc(p.dt * rho[k], gxi, eu, gu[k], inc);
                dn[k] = v[k] + inc;
            }
            if (wall >= 0) {
                const R xn = cya * nsgn;
                if (xn > R(0)) continue;   /* replaced below */
                if (xn < R(0)) {
    #pragma unroll
                    for (int k = 0; k < NQ; ++k) num[k] = fma(-xn * pc.w, dn[k], num[k]);
                }
            }
            store_quad(fout + a * plane + row0, dn, pc.w, a);
        }

    } else {
        auto load = [&](int a, QuadStencil<T, NQ> &S, PopC<R> &pc) {
            pc = pcs[a];
            const T *pa = fin + a * plane + row0;
            ldn<NQ>(pa, S.v);
            if (pc.crx != R(0)) {
                ld2(pa - 2, S.l);
                ld2(pa + NQ, S.r);
            }
            if (pc.cry > R(0)) {
                ldn<NQ>(pa + om2, S.y0);
                ldn<NQ>(pa + om1, S.y1);
                ldn<NQ>(pa + op1, S.y2);
            } else if (pc.cry < R(0)) {
                ldn<NQ>(pa + om1, S.y0);
                ldn<NQ>(pa + op1, S.y1);
                ldn<NQ>(pa + op2, S.y2);
            }
        };
        QuadStencil<T, NQ> cur, nxt;
        PopC<R> pcur, pnxt;
        if constexpr (PF) load(0, cur, pcur);
    #pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if constexpr (PF) {
                if (a + 1 < Q) load(a + 1, nxt, pnxt);
            } else {
                load(a, cur, pcur);
            }
            const PopC<R> pc = pcur;
            const R winv = pc.winv;
            R v[NQ], l[2], r[2];
    #pragma unroll
            for (int k = 0; k < NQ; ++k) v[k] = dec(cur.v[k], winv, k + 2);
            R Dx[NQ], Dy[NQ];
            const R crx = pc.crx, cry = pc.cry;
            if (crx != R(0)) {
                l[0] = dec(cur.l[0], winv, 0);
                l[1] = dec(cur.l[1], winv, 1);
                r[0] = dec(cur.r[0], winv, NQ + 2);
                r[1] = dec(cur.r[1], winv, NQ + 3);
            }
            x_flux_diff<NQ>(crx, pc.kx, l, v, r, Dx);
            if (cry > R(0)) {
                const R kf = pc.ky;
    #pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R ym2 = dec(cur.y0[k], winv, k + 2), ym1 = dec(cur.y1[k], winv, k + 2);
                    R yp1 = dec(cur.y2[k], winv, k + 2);
                    R d0 = ym1 - ym2, d1 = v[k] - ym1, d2 = yp1 - v[k];
                    const R n1 = neg_part(d1);
                    Dy[k] = fma(kf, minmod_n(d1, d2, n1, neg_part(d2)) - minmod_n(d0, d1, neg_part(d0), n1), d1);
                }
            } else if (cry < R(0)) {
                const R kf = pc.ky;
    #pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    R ym1 = dec(cur.y0[k], winv, k + 2), yp1 = dec(cur.y1[k], winv, k + 2);
                    R yp2 = dec(cur.y2[k], winv, k + 2);
                    R e0 = v[k] - ym1, e1 = yp1 - v[k], e2 = yp2 - yp1;
                    const R n1 = neg_part(e1);
                    Dy[k] = fma(-kf, minmod_n(e1, e2, n1, neg_part(e2)) - minmod_n(e0, e1, neg_part(e0), n1), e1);
                }
            } else {
    #pragma unroll
                for (int k = 0; k < NQ; ++k) Dy[k] = R(0);
            }
            R dn[NQ];
            const R cxa = pc.cx, cya = pc.cy;
            const R gxi = xi_dot(cxa, cya, p.gx, p.gy);
    #pragma unroll
            for (int k = 0; k < NQ; ++k) {
                R eu = xi_dot(cxa, cya, ux[k], uy[k]);
                R de = deq(rhod[k], rho[k], eu, usq[k]);
                /* sum the small increments first and round onto the stored magnitude once */
                R inc = om[k] * (de - v[k]);
                inc = fma(-crx, Dx[k], inc);
                inc = fma(-cry, Dy[k], inc);
                if (p.has_force) inc = force_inc(p.dt * rho[k], gxi, eu, gu[k], inc);
                dn[k] = v[k] + inc;
            }
            bool replaced = false;   /* wall-bound population on a wall row: written below */
            if (wall >= 0) {
                const R xn = cya * nsgn;
                replaced = xn > R(0);
                if (xn < R(0)) {
    #pragma unroll
                    for (int k = 0; k < NQ; ++k) num[k] = fma(-xn * pc.w, dn[k], num[k]);
                }
            }
            if (!replaced) store_quad(fout + a * plane + row0, dn, pc.w, a);
            if constexpr (PF) {
                cur = nxt;
                pcur = pnxt;
            }
        }

    }

    /* 4. diffuse wall: f_out = rho_W S(u_W) with zero net mass flux through the wall */
    if (wall >= 0) {
        const R uwx = p.uw_x[wall], uwy = p.uw_y[wall];
        const R usw = uwx * uwx + uwy * uwy;
        const R kd = p.kdiff[s][wall], kout = p.kout[s][wall];
        R rwd[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) rwd[k] = fma(rho0, kd, num[k]) / kout;   /* rho_W - rho0 */
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if (c.cy[a] * nsgn <= R(0)) continue;
            const R ew = c.cx[a] * uwx + c.cy[a] * uwy;
            const R sm1 = ew + R(0.5) * (ew * ew - usw);    /* S / w - 1 */
            R dn[NQ];
            /* rho_W S / w - rho0 = (rho_W - rho0)(1 + sm1) + rho0 sm1 */
#pragma unroll
            for (int k = 0; k < NQ; ++k) dn[k] = fma(rwd[k] + rho0, sm1, rwd[k]);
            store_quad(fout + a * plane + row0, dn, c.w[a], -1);
        }
    }

    /* 5. mode B: this node as the other set's readers will see it */
    if (flags & LB_TILE_SHADOW) {
        const int t = 1 - s;
        const SetConst<R> &ct = p.set[t];
        R h[NQ][6];
#pragma unroll
        for (int k = 0; k < NQ; ++k)
#pragma unroll
            for (int m = 0; m < 6; ++m) h[k][m] = R(0);
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const T *pa = fout + a * plane + row0;
#pragma unroll
            for (int k = 0; k < NQ; ++k)
                if (valid[k]) hermite_acc(c, a, dec(pa[k], c.winv[a], k + 2), h[k]);
        }
        T *ftd = static_cast<T *>(p.fout[t]);
        const int qt = ct.q;
#pragma unroll 1
        for (int b = 0; b < qt; ++b) {
            T *prow = ftd + b * plane + (size_t)j * p.pitch;
#pragma unroll
            for (int k = 0; k < NQ; ++k)
                if (valid[k]) put1r(p, prow, x0 + k, j, enc(hermite_rebuild(ct, b, h[k]), ct.w[b], k + 2));
        }
    }
}

/* COL: the lattice has a per-column reference density (p.dcol); a separate kernel so
 * that the common one keeps its register budget */
template <int ST, bool COL = false>
__global__ void __launch_bounds__(LB_BX *LB_BY, step_min_blocks<ST>()) step_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.y * LB_BX + threadIdx.x, LB_BX * LB_BY);
    __syncthreads();
    int bx = blockIdx.x, by = blockIdx.y;
    if (p.block_order) {
        const int b = p.block_order[blockIdx.x];
        bx = b % p.ntx;
        by = b / p.ntx;
    }
    const int j = by * LB_BY + threadIdx.y;
    const int x0 = (bx * LB_BX + threadIdx.x) * 4;
    if (j >= p.ny || x0 >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + (x0 / LB_TILE_X)];
    if (flags & LB_TILE_IFACE) return;   /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    constexpr bool PF = step_prefetch<ST>();
    if (q == 9) step_cells<ST, 9, PF, 4, COL>(p, s, flags, x0, j, pc[s], mc[s]);
    else if (q == 16) step_cells<ST, 16, PF, 4, COL>(p, s, flags, x0, j, pc[s], mc[s]);
    else step_cells<ST, 36, PF, 4, COL>(p, s, flags, x0, j, pc[s], mc[s]);
}


/* ------------------------------------------------------------------------------
 * Split form: plain quads (plain_quad(): no wall, ghost-copy, pressure, shadow or
 * interface work) in register blocks of 4 columns x RB rows per thread, with none of
 * the boundary logic of step_cells, so the kernel needs few registers; the remaining
 * quads through step_cells from a list. With RB = 2 a population's y stencil is read
 * once for both rows (RB + 3 rows instead of 3 RB) and the limited face slope between
 * the two rows is formed once. The arithmetic per node is that of step_cells, in the
 * same order, so every layout gives the same bits.
 * ---------------------------------------------------------------------------- */

/* y flux difference of the rows r = 0 .. RB-1 of one column from the RB + 3 rows of
 * its upwind window W: rows j0-2 .. j0+RB for xi_y > 0 (then kfs = kf), rows
 * j0-1 .. j0+RB+1 for xi_y < 0 (kfs = -kf, the mirrored flux). With d_i = W_{i+1} - W_i
 * and the face slope M_i = minmod(d_i, d_{i+1}), D_r = d_{r+1} + kfs (M_{r+1} - M_r):
 * each face slope is formed once for the two rows beside it. */
template <typename R, int RB>
__device__ __forceinline__ void y_flux_window(R kfs, const R (&W)[RB + 3], R (&D)[RB])
{
    R d[RB + 2], n[RB + 2], m[RB + 1];
#pragma unroll
    for (int i = 0; i < RB + 2; ++i) {
        d[i] = W[i + 1] - W[i];
        n[i] = neg_part(d[i]);
    }
#pragma unroll
    for (int i = 0; i < RB + 1; ++i) m[i] = minmod_n(d[i], d[i + 1], n[i], n[i + 1]);
#pragma unroll
    for (int r = 0; r < RB; ++r) D[r] = fma(kfs, m[r + 1] - m[r], d[r + 1]);
}

/* Stored values one population needs for a 4 x RB block: its own rows, the three rows
 * beyond them on the two sides (j0-2, j0-1, j0+RB for xi_y > 0; j0-1, j0+RB,
 * j0+RB+1 for xi_y < 0) and two values beside each own row (when xi_x != 0). */
template <typename T, int RB>
struct BlkStencil {
    T own[RB][4], hy[3][4], l[RB][2], r[RB][2];
};

template <int ST, int Q, int RB, bool FORCE>
__device__ __forceinline__ void blk_cells(const StepParams<typename Store<ST>::R> &p, int s, int x0, int j0,
                                          const PopC<typename Store<ST>::R> *pcs,
                                          const MomC<typename Store<ST>::R> *mcs)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const size_t plane = p.plane;
    const ptrdiff_t pitch = p.pitch;
    const size_t off = (size_t)j0 * pitch + (size_t)(x0 + LB_GHOST);
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]) + off;
    T *__restrict__ fout = static_cast<T *>(p.fout[s]) + off;
    const R rho0 = p.rho0;

    /* 1. moments of the 4 x RB nodes */
    R rhod[RB][4], ux[RB][4], uy[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) rhod[r][k] = ux[r][k] = uy[r][k] = R(0);
#pragma unroll 4
    for (int a = 0; a < Q; ++a) {
        const MomC<R> mc = mcs[a];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            T raw[4];
            ld4(fin + a * plane + r * pitch, raw);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const R d = decode<ST>(raw[k], mc.winv, rho0);
                rhod[r][k] = fma(mc.w, d, rhod[r][k]);
                ux[r][k] = fma(mc.wcx, d, ux[r][k]);
                uy[r][k] = fma(mc.wcy, d, uy[r][k]);
            }
        }
    }
    /* 2. macroscopic state: rho, u, relaxation rate (and force terms) */
    R rho[RB][4], usq[RB][4], om[RB][4], gu[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rho[r][k] = rho0 + rhod[r][k];
            const R inv = R(1) / rho[r][k];
            ux[r][k] *= inv;
            uy[r][k] *= inv;
            usq[r][k] = usq_of(ux[r][k], uy[r][k]);
            om[r][k] = p.dt / tau_of(p, inv);
            if constexpr (FORCE) gu[r][k] = xi_dot(p.gx, p.gy, ux[r][k], uy[r][k]);
        }

    /* 3. per population: stencil (loaded one population ahead), fluxes, collision,
     * force, store */
    auto load = [&](int a, BlkStencil<T, RB> &S, PopC<R> &pc) {
        pc = pcs[a];
        const T *pa = fin + a * plane;
#pragma unroll
        for (int r = 0; r < RB; ++r) ld4(pa + r * pitch, S.own[r]);
        if (pc.cry > R(0)) {
            ld4(pa - 2 * pitch, S.hy[0]);
            ld4(pa - pitch, S.hy[1]);
            ld4(pa + RB * pitch, S.hy[2]);
        } else if (pc.cry < R(0)) {
            ld4(pa - pitch, S.hy[0]);
            ld4(pa + RB * pitch, S.hy[1]);
            ld4(pa + (RB + 1) * pitch, S.hy[2]);
        }
        if (pc.crx != R(0)) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                ld2(pa + r * pitch - 2, S.l[r]);
                ld2(pa + r * pitch + 4, S.r[r]);
            }
        }
    };
    BlkStencil<T, RB> cur, nxt;
    PopC<R> pcur, pnxt;
    load(0, cur, pcur);
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        if (a + 1 < Q) load(a + 1, nxt, pnxt);
        const PopC<R> pc = pcur;
        const R winv = pc.winv, crx = pc.crx, cry = pc.cry;
        const R cxa = pc.cx, cya = pc.cy;
        R v[RB][4];
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) v[r][k] = decode<ST>(cur.own[r][k], winv, rho0);
        /* collision first, then the x and y flux differences, then the force: the
         * increments are summed in the order step_cells uses and rounded onto the
         * stored magnitude once */
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
                const R l[2] = {decode<ST>(cur.l[r][0], winv, rho0), decode<ST>(cur.l[r][1], winv, rho0)};
                const R rr[2] = {decode<ST>(cur.r[r][0], winv, rho0), decode<ST>(cur.r[r][1], winv, rho0)};
                R Dx[4];
                x_flux_diff(crx, pc.kx, l, v[r], rr, Dx);
#pragma unroll
                for (int k = 0; k < 4; ++k) inc[r][k] = fma(-crx, Dx[k], inc[r][k]);
            }
        }
        if (cry != R(0)) {
            const bool up = cry > R(0);
            const R kfs = up ? pc.ky : -pc.ky;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R W[RB + 3], Dy[RB];
                const R h0 = decode<ST>(cur.hy[0][k], winv, rho0), h1 = decode<ST>(cur.hy[1][k], winv, rho0);
                const R h2 = decode<ST>(cur.hy[2][k], winv, rho0);
                if (up) {
                    W[0] = h0;
                    W[1] = h1;
#pragma unroll
                    for (int r = 0; r < RB; ++r) W[2 + r] = v[r][k];
                    W[RB + 2] = h2;
                } else {
                    W[0] = h0;
#pragma unroll
                    for (int r = 0; r < RB; ++r) W[1 + r] = v[r][k];
                    W[RB + 1] = h1;
                    W[RB + 2] = h2;
                }
                y_flux_window<R, RB>(kfs, W, Dy);
#pragma unroll
                for (int r = 0; r < RB; ++r) inc[r][k] = fma(-cry, Dy[r], inc[r][k]);
            }
        }
        const R gxi = xi_dot(cxa, cya, p.gx, p.gy);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            T e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R t = inc[r][k];
                if constexpr (FORCE) {
                    const R eu = xi_dot(cxa, cya, ux[r][k], uy[r][k]);
                    t = force_inc(p.dt * rho[r][k], gxi, eu, gu[r][k], t);
                }
                e[k] = p.sr ? encode_sr<ST>(v[r][k] + t, pc.w, rho0, sr_bits(x0 + k, j0 + r, p.nx, a, p.step_key))
                            : encode<ST>(v[r][k] + t, pc.w, rho0);
            }
            st4(fout + a * plane + r * pitch, e);
        }
        cur = nxt;
        pcur = pnxt;
    }
}

/* Plain kernel of the split step: one thread per 4 x RB block of nodes, which it
 * updates only when every quad of the block is plain (the rest are listed for the
 * edge kernel). */
template <int ST, int RB, bool FORCE>
__global__ void __launch_bounds__(32 * (8 / RB)) step_plain_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.y * 32 + threadIdx.x, 32 * (8 / RB));
    __syncthreads();
    const int x0 = (blockIdx.x * 32 + threadIdx.x) * 4;
    const int j0 = (blockIdx.y * (8 / RB) + threadIdx.y) * RB;
    if (j0 + RB > p.ny || x0 >= p.nx) return;
    const int tile = x0 / LB_TILE_X;
    const uint8_t f0 = p.tmap[(size_t)j0 * p.ntx + tile];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const uint8_t fr = r == 0 ? f0 : p.tmap[(size_t)(j0 + r) * p.ntx + tile];
        if (fr != f0 || !plain_quad(x0, j0 + r, fr, p.nx, p.ny, p.periodic_x, p.periodic_y, p.pressure[0], p.pressure[1]))
            return;
    }
    const int s = f0 & LB_TILE_HIGH;
    const int q = p.set[s].q;
    if (q == 9) blk_cells<ST, 9, RB, FORCE>(p, s, x0, j0, pc[s], mc[s]);
    else if (q == 16) blk_cells<ST, 16, RB, FORCE>(p, s, x0, j0, pc[s], mc[s]);
    else blk_cells<ST, 36, RB, FORCE>(p, s, x0, j0, pc[s], mc[s]);
}

/* Edge kernel of the split step: the one-quad path for each listed quad (x0, j). */
template <int ST>
__global__ void __launch_bounds__(128) step_edge_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p,
                                                        const int2 *__restrict__ list, int n)
{
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.x, 128);
    __syncthreads();
    const int k = blockIdx.x * 128 + threadIdx.x;
    if (k >= n) return;
    const int2 e = list[k];
    const int x0 = e.x, j = e.y;
    if (j < 0 || j >= p.ny || x0 < 0 || x0 >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + x0 / LB_TILE_X];
    if (flags & LB_TILE_IFACE) return;   /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    if (q == 9) step_cells<ST, 9>(p, s, flags, x0, j, pc[s], mc[s]);
    else if (q == 16) step_cells<ST, 16>(p, s, flags, x0, j, pc[s], mc[s]);
    else step_cells<ST, 36>(p, s, flags, x0, j, pc[s], mc[s]);
}

/* The edge kernel goes to edge_stream (the caller orders it after the previous step and
 * before the next one): its few long-running blocks then overlap the plain kernel. */
template <int ST>
void launch_step_split_store(const StepParams<typename Store<ST>::R> &p, int rb, const int2 *edge, int n_edge,
                             void *stream, void *edge_stream)
{
    const dim3 grid((p.nx + 4 * 32 - 1) / (4 * 32), (p.ny + 7) / 8);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_edge > 0)
        step_edge_kernel<ST><<<(n_edge + 127) / 128, 128, 0, static_cast<cudaStream_t>(edge_stream)>>>(p, edge, n_edge);
    if (rb == 2) {
        if (p.has_force) step_plain_kernel<ST, 2, true><<<grid, dim3(32, 4), 0, st>>>(p);
        else step_plain_kernel<ST, 2, false><<<grid, dim3(32, 4), 0, st>>>(p);
    } else {
        if (p.has_force) step_plain_kernel<ST, 1, true><<<grid, dim3(32, 8), 0, st>>>(p);
        else step_plain_kernel<ST, 1, false><<<grid, dim3(32, 8), 0, st>>>(p);
    }
}

/* ------------------------------------------------------------------------------
 * Batched channels: many independent lattices advanced by one persistent launch. Each
 * block takes lattices from a queue (longest first), copies the lattice's two launch
 * parameter sets (level n -> n+1 and back) into shared memory and advances it nsteps
 * steps, a block barrier between steps (the block owns the whole lattice, so no other
 * synchronisation is needed). Every quad goes through step_cells: the same arithmetic,
 * in the same order, as the one-quad layout of a single lattice. The lattices have
 * mode-B interfaces, steady walls and no pressure columns (checked on the host).
 * advance = 0 repeats step 0 (level n -> n+1) nsteps times without moving the state
 * (used to time block shapes).
 * ---------------------------------------------------------------------------- */
template <int ST>
__global__ void __launch_bounds__(512) batch_kernel(const StepParams<typename Store<ST>::R> *__restrict__ params,
                                                   const int *__restrict__ order, int n, int nsteps, int base,
                                                   int advance, unsigned int *queue)
{
    using R = typename Store<ST>::R;
    __shared__ StepParams<R> sp[2];
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    __shared__ int inst_sh;
    static_assert(sizeof(StepParams<R>) % 4 == 0, "parameter copy in 4-byte words");
    constexpr int NW = (int)(sizeof(StepParams<R>) / 4);
    for (;;) {
        __syncthreads();   /* every thread is done with the previous lattice */
        if (threadIdx.x == 0) {
            const unsigned k = atomicAdd(queue, 1u);
            inst_sh = k < (unsigned)n ? order[k] : -1;
        }
        __syncthreads();
        const int inst = inst_sh;
        if (inst < 0) return;
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(params + 2 * (size_t)inst);
            uint32_t *dst = reinterpret_cast<uint32_t *>(sp);
            for (int k = threadIdx.x; k < 2 * NW; k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();
        stage_consts(sp[0], pc, mc, threadIdx.x, blockDim.x);
        __syncthreads();
        const int nqx = (sp[0].nx + 3) / 4, nq = nqx * sp[0].ny;
        for (int st = 0; st < nsteps; ++st) {
            const StepParams<R> &p = sp[advance ? ((base + st) & 1) : base];
            for (int k = threadIdx.x; k < nq; k += blockDim.x) {
                const int j = k / nqx, x0 = (k - j * nqx) * 4;
                const uint8_t flags = p.tmap[(size_t)j * p.ntx + x0 / LB_TILE_X];
                const int s = flags & LB_TILE_HIGH;
                const int q = p.set[s].q;
                if (q == 9) step_cells<ST, 9>(p, s, flags, x0, j, pc[s], mc[s]);
                else if (q == 16) step_cells<ST, 16>(p, s, flags, x0, j, pc[s], mc[s]);
                else step_cells<ST, 36>(p, s, flags, x0, j, pc[s], mc[s]);
            }
            __syncthreads();
        }
    }
}

template <int ST>
int launch_batch_store(const void *params, const int *order, int n, int nsteps, int base, int advance,
                       unsigned int *queue, int threads, int grid, void *stream)
{
    using R = typename Store<ST>::R;
    if (threads < 32 || threads > 512 || grid < 1) return -1;
    batch_kernel<ST><<<grid, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const StepParams<R> *>(params), order, n, nsteps, base, advance, queue);
    return 0;
}

/* Resident blocks per SM of the batch kernel at this block size. */
template <int ST>
int batch_blocks_per_sm(int threads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<ST>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

/* Layout 6: one block per descriptor of p.block_desc, one tile wide. A band that holds
 * high-order rows runs as blocks of 4 rows with two nodes per thread (64 threads per
 * row), so its long population loops are spread over twice the warps; the other bands
 * run as in step_kernel. Each node's arithmetic is the same for either width. */
template <int ST>
__global__ void __launch_bounds__(LB_BX *LB_BY, step_min_blocks<ST>())
    step_desc_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.y * LB_BX + threadIdx.x, LB_BX * LB_BY);
    __syncthreads();
    const int2 d = p.block_desc[blockIdx.x];
    const bool narrow = d.y & 1;
    const int t = threadIdx.y * LB_BX + threadIdx.x;
    const int x0 = d.x * LB_TILE_X + (narrow ? 2 * (t & 63) : 4 * threadIdx.x);
    const int j = (d.y >> 1) + (narrow ? t >> 6 : threadIdx.y);
    if (j >= p.ny || x0 >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + d.x];
    if (flags & LB_TILE_IFACE) return;   /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    constexpr bool PF = step_prefetch<ST>();
    if (narrow) {
        if (q == 9) step_cells<ST, 9, PF, 2>(p, s, flags, x0, j, pc[s], mc[s]);
        else if (q == 16) step_cells<ST, 16, PF, 2>(p, s, flags, x0, j, pc[s], mc[s]);
        else step_cells<ST, 36, PF, 2>(p, s, flags, x0, j, pc[s], mc[s]);
    } else {
        if (q == 9) step_cells<ST, 9, PF, 4>(p, s, flags, x0, j, pc[s], mc[s]);
        else if (q == 16) step_cells<ST, 16, PF, 4>(p, s, flags, x0, j, pc[s], mc[s]);
        else step_cells<ST, 36, PF, 4>(p, s, flags, x0, j, pc[s], mc[s]);
    }
}

template <int ST>
void launch_step_desc_store(const StepParams<typename Store<ST>::R> &p, int n, void *stream)
{
    static_assert(LB_BX * LB_BY == 64 * 4, "a narrow block is 4 rows of 64 threads");
    if (n < 1) return;
    step_desc_kernel<ST><<<n, dim3(LB_BX, LB_BY), 0, static_cast<cudaStream_t>(stream)>>>(p);
}

template <int ST>
void launch_step_store(const StepParams<typename Store<ST>::R> &p, void *stream)
{
    static_assert(4 * LB_BX == LB_TILE_X, "a block of the one-quad kernel is one tile wide");
    dim3 block(LB_BX, LB_BY);
    dim3 grid((p.nx + 4 * LB_BX - 1) / (4 * LB_BX), (p.ny + LB_BY - 1) / LB_BY);
    if (p.block_order) grid = dim3(grid.x * grid.y, 1);
    if constexpr (Store<ST>::dev) {
        if (p.dcol) {
            step_kernel<ST, true><<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(p);
            return;
        }
    }
    step_kernel<ST><<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(p);
}

}  // namespace lbk
