/*
 * lb_step.cu -- the fused time step of the multiscale lattice Boltzmann method and the
 * small passes that complete a level (interface rows of mode A, pressure columns,
 * rebuilt interface views after the state is replaced).
 *
 * One thread owns four consecutive nodes of one row (one 16-byte FP32 vector per
 * plane). For every node it:
 *   1. sums density and momentum over its set's populations (Eq. (demoeq) moments);
 *   2. derives tau from the local density (Eq. (KN): collision rate p / mu);
 *   3. for each population, reads the radius-2 cross of the Sec. 3.1 stencil (x
 *      neighbours from two 2-element vectors beside its own, y neighbours from the rows
 *      above and below; ghost rows are the wall row, Sec. 3.2), forms the two limited
 *      face fluxes in x and in y (minmod, mirrored for negative velocities), and
 *      applies the forward-Euler update with BGK collision towards Eq. (demoeq) and the
 *      Eq. (demoforce) body force;
 *   4. on a diffuse wall row, replaces the gas-bound populations by rho_W S(u_W)
 *      (Sec. 3.2) with rho_W from the streamed wall-bound populations;
 *   5. in mode B, on tiles that neighbour the other set, also writes the node rebuilt
 *      in the other set from its second-order Hermite coefficients (Sec. 2.2), so that
 *      the other set's readers find it at the next step.
 * The stencil reads only the level n planes and writes only level n + 1.
 */
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_common.cuh"

namespace lbk {

#define LB_BX 32
#define LB_BY 8

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
        R m[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = minmod(d[k], d[k + 1]);
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
        R m[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k] = minmod(e[k], e[k + 1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = fma(-kf, m[k + 1] - m[k], e[k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) D[k] = R(0);
    }
}

template <int ST, int Q>
__device__ __forceinline__ void step_cells(const StepParams<typename Store<ST>::R> &p, int s, uint8_t flags, int x0,
                                           int j)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const SetConst<R> &c = p.set[s];
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]);
    T *__restrict__ fout = static_cast<T *>(p.fout[s]);
    const size_t plane = (size_t)p.ny * p.pitch;
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
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            R d = decode<ST>(raw[k], c.winv[a], rho0);
            rhod[k] = fma(c.w[a], d, rhod[k]);
            jx[k] = fma(c.wcx[a], d, jx[k]);
            jy[k] = fma(c.wcy[a], d, jy[k]);
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

    auto store_quad = [&](T *dst, const R dn[4], R w) {
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = encode<ST>(dn[k], w, rho0);
        if (full && !near_x_edge) {
            st4(dst, e);
        } else {
            T *prow = dst - (x0 + LB_GHOST);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[k]) put1(p, prow, x0 + k, e[k]);
        }
    };

    /* 3. stencil, fluxes, collision, force */
    R num[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        const T *pa = fin + a * plane + row0;
        const R winv = c.winv[a];
        T raw[4];
        R v[4], l[2], r[2];
        ld4(pa, raw);
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = decode<ST>(raw[k], winv, rho0);
        R Dx[4], Dy[4];
        const R crx = c.crx[a], cry = c.cry[a];
        if (crx != R(0)) {
            T tl[2], tr[2];
            ld2(pa - 2, tl);
            ld2(pa + 4, tr);
            l[0] = decode<ST>(tl[0], winv, rho0);
            l[1] = decode<ST>(tl[1], winv, rho0);
            r[0] = decode<ST>(tr[0], winv, rho0);
            r[1] = decode<ST>(tr[1], winv, rho0);
        }
        x_flux_diff(crx, c.kx[a], l, v, r, Dx);
        if (cry > R(0)) {
            T t2[4], t1[4], tp[4];
            ld4(pa + om2, t2);
            ld4(pa + om1, t1);
            ld4(pa + op1, tp);
            const R kf = c.ky[a];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R ym2 = decode<ST>(t2[k], winv, rho0), ym1 = decode<ST>(t1[k], winv, rho0);
                R yp1 = decode<ST>(tp[k], winv, rho0);
                R d0 = ym1 - ym2, d1 = v[k] - ym1, d2 = yp1 - v[k];
                Dy[k] = fma(kf, minmod(d1, d2) - minmod(d0, d1), d1);
            }
        } else if (cry < R(0)) {
            T t1[4], tp[4], t2[4];
            ld4(pa + om1, t1);
            ld4(pa + op1, tp);
            ld4(pa + op2, t2);
            const R kf = c.ky[a];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R ym1 = decode<ST>(t1[k], winv, rho0), yp1 = decode<ST>(tp[k], winv, rho0);
                R yp2 = decode<ST>(t2[k], winv, rho0);
                R e0 = v[k] - ym1, e1 = yp1 - v[k], e2 = yp2 - yp1;
                Dy[k] = fma(-kf, minmod(e1, e2) - minmod(e0, e1), e1);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) Dy[k] = R(0);
        }
        R dn[4];
        const R cxa = c.cx[a], cya = c.cy[a];
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
                for (int k = 0; k < 4; ++k) num[k] = fma(-xn * c.w[a], dn[k], num[k]);
            }
        }
        store_quad(fout + a * plane + row0, dn, c.w[a]);
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
                if (valid[k]) put1(p, prow, x0 + k, encode<ST>(hermite_rebuild(ct, b, h[k]), ct.w[b], rho0));
        }
    }
}

template <int ST>
__global__ void __launch_bounds__(LB_BX *LB_BY) step_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    const int j = blockIdx.y * LB_BY + threadIdx.y;
    const int x0 = (blockIdx.x * LB_BX + threadIdx.x) * 4;
    if (j >= p.ny || x0 >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + (x0 / LB_TILE_X)];
    if (flags & LB_TILE_IFACE) return;   /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    if (q == 9) step_cells<ST, 9>(p, s, flags, x0, j);
    else if (q == 16) step_cells<ST, 16>(p, s, flags, x0, j);
    else step_cells<ST, 36>(p, s, flags, x0, j);
}

/* ---------------------------------------------------------------- mode A -- */

/* Sec. 2.2: interface row I gets, in each set s, f_eq^s(rho_I, u_I) + f_neq^s of the
 * neighbour on s's own side, with rho_I, u_I the means of its two neighbours; the node
 * one beyond I on the other side gets a copy (what a reader reaching past I sees). */
template <int ST>
__global__ void iface_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx || blockIdx.y >= (unsigned)p.n_iface) return;
    const int I = p.iface_row[blockIdx.y];
    const uint8_t flags = p.tmap[(size_t)I * p.ntx + x / LB_TILE_X];
    const int jh = (flags & LB_TILE_NEAR_H) ? I - 1 : I + 1;
    const int jl = (flags & LB_TILE_NEAR_H) ? I + 1 : I - 1;
    const size_t plane = (size_t)p.ny * p.pitch;
    const R rho0 = p.rho0;
    R rhod[2], u[2][2];
    const int rows[2] = {jl, jh};
    for (int s = 0; s < 2; ++s) {
        const SetConst<R> &c = p.set[s];
        const T *f = static_cast<const T *>(p.fout[s]) + (size_t)rows[s] * p.pitch + x + LB_GHOST;
        R r = R(0), mx = R(0), my = R(0);
        for (int a = 0; a < c.q; ++a) {
            R d = decode<ST>(f[a * plane], c.winv[a], rho0);
            r = fma(c.w[a], d, r);
            mx = fma(c.wcx[a], d, mx);
            my = fma(c.wcy[a], d, my);
        }
        rhod[s] = r;
        u[s][0] = mx / (rho0 + r);
        u[s][1] = my / (rho0 + r);
    }
    const R rIdev = R(0.5) * (rhod[0] + rhod[1]);
    const R rI = rho0 + rIdev;
    const R uIx = R(0.5) * (u[0][0] + u[1][0]), uIy = R(0.5) * (u[0][1] + u[1][1]);
    const R usI = uIx * uIx + uIy * uIy;
    for (int s = 0; s < 2; ++s) {
        const SetConst<R> &c = p.set[s];
        const T *fn = static_cast<const T *>(p.fout[s]) + (size_t)rows[s] * p.pitch + x + LB_GHOST;
        T *fo = static_cast<T *>(p.fout[s]);
        const int beyond = rows[1 - s];
        const R rn = rho0 + rhod[s], usn = u[s][0] * u[s][0] + u[s][1] * u[s][1];
        for (int a = 0; a < c.q; ++a) {
            const R dnb = decode<ST>(fn[a * plane], c.winv[a], rho0);
            const R eI = c.cx[a] * uIx + c.cy[a] * uIy;
            const R en = c.cx[a] * u[s][0] + c.cy[a] * u[s][1];
            const R d = deq(rIdev, rI, eI, usI) + (dnb - deq(rhod[s], rn, en, usn));
            const T e = encode<ST>(d, c.w[a], rho0);
            put1(p, fo + a * plane + (size_t)I * p.pitch, x, e);
            put1(p, fo + a * plane + (size_t)beyond * p.pitch, x, e);
        }
    }
}

/* ------------------------------------------------------- pressure columns -- */

/* Column x = 0 (left) or nx-1 (right), interior rows: f = f_eq(rho_b, u_1) +
 * [f - f_eq](node one step inwards), the virtual-boundary construction of Sec. 2.2
 * applied to an open boundary. Then every row's ghost columns beyond the boundary get
 * copies of the boundary node (in its set, and rebuilt in the other set where the tile
 * neighbours it). */
template <int ST>
__global__ void pressure_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int side = blockIdx.y;
    if (j >= p.ny || !p.pressure[side]) return;
    const int xb = side == 0 ? 0 : p.nx - 1;
    const int xi = side == 0 ? 1 : p.nx - 2;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + xb / LB_TILE_X];
    const int s = flags & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const size_t plane = (size_t)p.ny * p.pitch;
    const R rho0 = p.rho0;
    T *f = static_cast<T *>(p.fout[s]) + (size_t)j * p.pitch + LB_GHOST;
    R dv[LB_QMAX];
    if (is_pressure_node(p, xb, j)) {
        R r = R(0), mx = R(0), my = R(0);
        for (int a = 0; a < c.q; ++a) {
            dv[a] = decode<ST>(f[a * plane + xi], c.winv[a], rho0);
            r = fma(c.w[a], dv[a], r);
            mx = fma(c.wcx[a], dv[a], mx);
            my = fma(c.wcy[a], dv[a], my);
        }
        const R rn = rho0 + r, uxn = mx / rn, uyn = my / rn, usn = uxn * uxn + uyn * uyn;
        const R rb = p.rho_side[side];
        for (int a = 0; a < c.q; ++a) {
            const R e = c.cx[a] * uxn + c.cy[a] * uyn;
            dv[a] = deq(rb - rho0, rb, e, usn) + (dv[a] - deq(r, rn, e, usn));
            f[a * plane + xb] = encode<ST>(dv[a], c.w[a], rho0);
        }
    }
    for (int a = 0; a < c.q; ++a) {
        const T e = f[a * plane + xb];
        dv[a] = decode<ST>(e, c.winv[a], rho0);
        for (int g = 1; g <= LB_GHOST; ++g) f[a * plane + (side == 0 ? xb - g : xb + g)] = e;
    }
    if (flags & LB_TILE_SHADOW) {
        R h[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        for (int a = 0; a < c.q; ++a) hermite_acc(c, a, dv[a], h);
        const SetConst<R> &ct = p.set[1 - s];
        T *ft = static_cast<T *>(p.fout[1 - s]) + (size_t)j * p.pitch + LB_GHOST;
        for (int b = 0; b < ct.q; ++b) {
            const T e = encode<ST>(hermite_rebuild(ct, b, h), ct.w[b], rho0);
            for (int g = 0; g <= LB_GHOST; ++g) ft[b * plane + (side == 0 ? xb - g : xb + g)] = e;
        }
    }
}

/* ------------------------------------------------ interface views, ghosts -- */

/* Rebuild every node of a mode-B shadow tile in the other set from its current state
 * (used after the state or the map is replaced, not inside a step). */
template <int ST>
__global__ void shadows_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (x >= p.nx) return;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + x / LB_TILE_X];
    if (!(flags & LB_TILE_SHADOW)) return;
    const int s = flags & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const SetConst<R> &ct = p.set[1 - s];
    const size_t plane = (size_t)p.ny * p.pitch;
    const T *f = static_cast<const T *>(p.fout[s]) + (size_t)j * p.pitch + x + LB_GHOST;
    R h[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int a = 0; a < c.q; ++a) hermite_acc(c, a, decode<ST>(f[a * plane], c.winv[a], p.rho0), h);
    T *ft = static_cast<T *>(p.fout[1 - s]);
    for (int b = 0; b < ct.q; ++b)
        put1(p, ft + b * plane + (size_t)j * p.pitch, x, encode<ST>(hermite_rebuild(ct, b, h), ct.w[b], p.rho0));
}

/* Periodic images of columns 0..3 and nx-4..nx-1 for every plane of both sets. */
template <int ST>
__global__ void ghosts_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using T = typename Store<ST>::T;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int sa = blockIdx.y;   /* set * LB_QMAX + alpha */
    const int s = sa / LB_QMAX, a = sa % LB_QMAX;
    if (j >= p.ny || a >= p.set[s].q || !p.periodic_x) return;
    T *prow = static_cast<T *>(p.fout[s]) + ((size_t)a * p.ny + j) * p.pitch;
    for (int g = 0; g < LB_GHOST; ++g) {
        prow[g + p.nx + LB_GHOST] = prow[g + LB_GHOST];
        prow[g] = prow[p.nx + g];
    }
}

/* ------------------------------------------------------------- launchers -- */

template <typename R>
struct StoreFor;

#define LB_DISPATCH(store, ...)                                   \
    switch (store) {                                               \
        case 0: { constexpr int ST = 0; __VA_ARGS__; } break;             \
        case 1: { constexpr int ST = 1; __VA_ARGS__; } break;             \
        case 2: { constexpr int ST = 2; __VA_ARGS__; } break;             \
        case 3: { constexpr int ST = 3; __VA_ARGS__; } break;             \
        default: { constexpr int ST = 4; __VA_ARGS__; } break;            \
    }

template <typename R, int ST>
constexpr bool store_matches()
{
    return std::is_same<R, typename Store<ST>::R>::value;
}

template <typename R>
void launch_step(int store, const StepParams<R> &p, void *stream)
{
    dim3 block(LB_BX, LB_BY);
    dim3 grid((p.nx + 4 * LB_BX - 1) / (4 * LB_BX), (p.ny + LB_BY - 1) / LB_BY);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) step_kernel<ST><<<grid, block, 0, st>>>(p));
}

template <typename R>
void launch_iface(int store, const StepParams<R> &p, void *stream)
{
    if (p.n_iface <= 0) return;
    dim3 grid((p.nx + 127) / 128, p.n_iface);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) iface_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template <typename R>
void launch_pressure(int store, const StepParams<R> &p, void *stream)
{
    if (!p.pressure[0] && !p.pressure[1]) return;
    dim3 grid((p.ny + 63) / 64, 2);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) pressure_kernel<ST><<<grid, 64, 0, st>>>(p));
}

template <typename R>
void launch_shadows(int store, const StepParams<R> &p, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) shadows_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template <typename R>
void launch_ghosts(int store, const StepParams<R> &p, void *stream)
{
    if (!p.periodic_x) return;
    dim3 grid((p.ny + 127) / 128, 2 * LB_QMAX);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) ghosts_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template void launch_step<float>(int, const StepParams<float> &, void *);
template void launch_step<double>(int, const StepParams<double> &, void *);
template void launch_iface<float>(int, const StepParams<float> &, void *);
template void launch_iface<double>(int, const StepParams<double> &, void *);
template void launch_pressure<float>(int, const StepParams<float> &, void *);
template void launch_pressure<double>(int, const StepParams<double> &, void *);
template void launch_shadows<float>(int, const StepParams<float> &, void *);
template void launch_shadows<double>(int, const StepParams<double> &, void *);
template void launch_ghosts<float>(int, const StepParams<float> &, void *);
template void launch_ghosts<double>(int, const StepParams<double> &, void *);

}  // namespace lbk
