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
#define LB_BY 8
#ifndef LB_MINB
#define LB_MINB 3   /* resident blocks per SM the register budget is sized for */
#endif

/* Flux difference F_{k+1/2} - F_{k-1/2} along one axis for four nodes in a row
 * (Sec. 3.1), Courant number c, limiter factor kf = (1 - |c|) / 2.
 * v[-2..5] are the values at nodes x0-2 .. x0+5 (v[0..3] the thread's own). */
template <typename R>
__device__ __forceinline__ void x_flux_diff(R c, R kf, const R l[2], const R v[4], const R r[2], R D[4])
{
    if (c > R(0)) {
        /* upwind node k: F_{k+1/2} = f_k + kf minmod(f_k - f_{k-1}, f_{k+1} - f_k) */
        R d[6];
        d[0] = l[1] - l[0];
        d[1] = v[0] - l[1];
        d[2] = v[1] - v[0];
        d[3] = v[2] - v[1];
        d[4] = v[3] - v[2];
        d[5] = r[0] - v[3];
        R n[6], m[5];
#pragma unroll
        for (int k = 0; k < 6; ++k) n[k] = neg_part(d[k]);
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = minmod_n(d[k], d[k + 1], n[k], n[k + 1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = fma(kf, m[k + 1] - m[k], d[k + 1]);
    } else if (c < R(0)) {
        /* mirror image: upwind node k+1 */
        R e[6];
        e[0] = v[0] - l[1];
        e[1] = v[1] - v[0];
        e[2] = v[2] - v[1];
        e[3] = v[3] - v[2];
        e[4] = r[0] - v[3];
        e[5] = r[1] - r[0];
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

template <int ST, int Q>
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

    /* 1. moments */
    R rhod[4] = {R(0), R(0), R(0), R(0)}, jx[4] = {R(0), R(0), R(0), R(0)}, jy[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 4
    for (int a = 0; a < Q; ++a) {
        T raw[4];
        ld4(fin + a * plane + row0, raw);
        const MomC<R> mc = mcs[a];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R d = decode<ST>(raw[k], mc.winv, rho0);
            rhod[k] = fma(mc.w, d, rhod[k]);
            jx[k] = fma(mc.wcx, d, jx[k]);
            jy[k] = fma(mc.wcy, d, jy[k]);
        }
    }
    /* 2. macroscopic state and relaxation */
    R rho[4], ux[4], uy[4], usq[4], om[4], gu[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rho[k] = rho0 + rhod[k];
        R inv = R(1) / rho[k];
        ux[k] = jx[k] * inv;
        uy[k] = jy[k] * inv;
        usq[k] = ux[k] * ux[k] + uy[k] * uy[k];
        om[k] = p.dt / tau_of(p, rho[k]);
        gu[k] = p.gx * ux[k] + p.gy * uy[k];
    }

    int wall = -1;
    if (j == 0 && p.wall_diffuse[0]) wall = 0;
    if (j == p.ny - 1 && p.wall_diffuse[1]) wall = 1;
    const R nsgn = wall == 0 ? R(1) : R(-1);

    bool valid[4];
    bool full = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int x = x0 + k;
        valid[k] = x < p.nx && !is_pressure_node(p, x, j);
        full = full && valid[k];
    }
    const bool near_x_edge = p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST);

    int img[2];
    const int nimg = row_images(p, j, img);
    auto store_quad = [&](T *dst, const R dn[4], R w) {
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = encode<ST>(dn[k], w, rho0);
        for (int t = -1; t < nimg; ++t) {
            T *d = t < 0 ? dst : dst + (ptrdiff_t)img[t] * p.pitch;
            if (full && !near_x_edge) {
                st4(d, e);
            } else {
                T *prow = d - (x0 + LB_GHOST);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (valid[k]) put1(p, prow, x0 + k, e[k]);
            }
        }
    };

    /* 3. stencil, fluxes, collision, force */
    R num[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        const T *pa = fin + a * plane + row0;
        const PopC<R> pc = pcs[a];
        const R winv = pc.winv;
        T raw[4];
        R v[4], l[2], r[2];
        ld4(pa, raw);
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = decode<ST>(raw[k], winv, rho0);
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
            ld4(pa + om2, t2);
            ld4(pa + om1, t1);
            ld4(pa + op1, tp);
            const R kf = pc.ky;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R ym2 = decode<ST>(t2[k], winv, rho0), ym1 = decode<ST>(t1[k], winv, rho0);
                R yp1 = decode<ST>(tp[k], winv, rho0);
                R d0 = ym1 - ym2, d1 = v[k] - ym1, d2 = yp1 - v[k];
                const R n1 = neg_part(d1);
                Dy[k] = fma(kf, minmod_n(d1, d2, n1, neg_part(d2)) - minmod_n(d0, d1, neg_part(d0), n1), d1);
            }
        } else if (cry < R(0)) {
            T t1[4], tp[4], t2[4];
            ld4(pa + om1, t1);
            ld4(pa + op1, tp);
            ld4(pa + op2, t2);
            const R kf = pc.ky;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R ym1 = decode<ST>(t1[k], winv, rho0), yp1 = decode<ST>(tp[k], winv, rho0);
                R yp2 = decode<ST>(t2[k], winv, rho0);
                R e0 = v[k] - ym1, e1 = yp1 - v[k], e2 = yp2 - yp1;
                const R n1 = neg_part(e1);
                Dy[k] = fma(-kf, minmod_n(e1, e2, n1, neg_part(e2)) - minmod_n(e0, e1, neg_part(e0), n1), e1);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) Dy[k] = R(0);
        }
        R dn[4];
        const R cxa = pc.cx, cya = pc.cy;
        const R gxi = p.gx * cxa + p.gy * cya;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R eu = cxa * ux[k] + cya * uy[k];
            R de = deq(rhod[k], rho[k], eu, usq[k]);
            /* sum the small increments first and round onto the stored magnitude once */
            R inc = om[k] * (de - v[k]);
            inc = fma(-crx, Dx[k], inc);
            inc = fma(-cry, Dy[k], inc);
            if (p.has_force) inc = fma(p.dt * rho[k], gxi + gxi * eu - gu[k], inc);
            dn[k] = v[k] + inc;
        }
        if (wall >= 0) {
            const R xn = cya * nsgn;
            if (xn > R(0)) continue;   /* replaced below */
            if (xn < R(0)) {
#pragma unroll
                for (int k = 0; k < 4; ++k) num[k] = fma(-xn * pc.w, dn[k], num[k]);
            }
        }
        store_quad(fout + a * plane + row0, dn, pc.w);
    }

    /* 4. diffuse wall: f_out = rho_W S(u_W) with zero net mass flux through the wall */
    if (wall >= 0) {
        const R uwx = p.uw_x[wall], uwy = p.uw_y[wall];
        const R usw = uwx * uwx + uwy * uwy;
        const R kd = p.kdiff[s][wall], kout = p.kout[s][wall];
        R rwd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rwd[k] = fma(rho0, kd, num[k]) / kout;   /* rho_W - rho0 */
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if (c.cy[a] * nsgn <= R(0)) continue;
            const R ew = c.cx[a] * uwx + c.cy[a] * uwy;
            const R sm1 = ew + R(0.5) * (ew * ew - usw);    /* S / w - 1 */
            R dn[4];
            /* rho_W S / w - rho0 = (rho_W - rho0)(1 + sm1) + rho0 sm1 */
#pragma unroll
            for (int k = 0; k < 4; ++k) dn[k] = fma(rwd[k] + rho0, sm1, rwd[k]);
            store_quad(fout + a * plane + row0, dn, c.w[a]);
        }
    }

    /* 5. mode B: this node as the other set's readers will see it */
    if (flags & LB_TILE_SHADOW) {
        const int t = 1 - s;
        const SetConst<R> &ct = p.set[t];
        R h[4][6];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < 6; ++m) h[k][m] = R(0);
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const T *pa = fout + a * plane + row0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[k]) hermite_acc(c, a, decode<ST>(pa[k], c.winv[a], rho0), h[k]);
        }
        T *ftd = static_cast<T *>(p.fout[t]);
        const int qt = ct.q;
#pragma unroll 1
        for (int b = 0; b < qt; ++b) {
            T *prow = ftd + b * plane + (size_t)j * p.pitch;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[k]) put1r(p, prow, x0 + k, j, encode<ST>(hermite_rebuild(ct, b, h[k]), ct.w[b], rho0));
        }
    }
}

template <int ST>
__global__ void __launch_bounds__(LB_BX *LB_BY, ST == 0 ? 2 : LB_MINB) step_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pc[2][LB_QMAX];
    __shared__ MomC<R> mc[2][LB_QMAX];
    stage_consts(p, pc, mc, threadIdx.y * LB_BX + threadIdx.x, LB_BX * LB_BY);
    __syncthreads();
    const int j = blockIdx.y * LB_BY + threadIdx.y;
    const int x0 = (blockIdx.x * LB_BX + threadIdx.x) * 4;
    if (j >= p.ny || x0 >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + (x0 / LB_TILE_X)];
    if (flags & LB_TILE_IFACE) return;   /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    if (q == 9) step_cells<ST, 9>(p, s, flags, x0, j, pc[s], mc[s]);
    else if (q == 16) step_cells<ST, 16>(p, s, flags, x0, j, pc[s], mc[s]);
    else step_cells<ST, 36>(p, s, flags, x0, j, pc[s], mc[s]);
}


template <int ST>
void launch_step_store(const StepParams<typename Store<ST>::R> &p, void *stream)
{
    dim3 block(LB_BX, LB_BY);
    dim3 grid((p.nx + 4 * LB_BX - 1) / (4 * LB_BX), (p.ny + LB_BY - 1) / LB_BY);
    step_kernel<ST><<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(p);
}

}  // namespace lbk
