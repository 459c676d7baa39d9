/*
 * lb_common.cuh -- device helpers shared by the step kernels and the auxiliary
 * kernels: stencil row indices, the equilibrium in deviation form, stores with
 * periodic images, and the second-order Hermite rebuild of a node in another set.
 */
#pragma once

#include "lb_internal.h"
#include "lb_store.cuh"

namespace lbk {

/* Per-population constants as read inside the population loops: two 16-byte records
 * (FP32) per population, staged in shared memory once per block, because indexing the
 * kernel-parameter tables with a run-time population index goes through the L1 path on
 * every access. */
template <typename R>
struct alignas(4 * sizeof(R)) PopC {
    R cx, cy, crx, cry;   /* xi and Courant numbers */
    R kx, ky, w, winv;    /* limiter factors (1 - |c|) / 2, weight, 1 / weight */
};
template <typename R>
struct alignas(4 * sizeof(R)) MomC {
    R w, wcx, wcy, winv;
};

template <typename R>
__device__ __forceinline__ void stage_consts(const StepParams<R> &p, PopC<R> (*pc)[LB_QMAX], MomC<R> (*mc)[LB_QMAX],
                                             int tid, int nthreads)
{
    for (int k = tid; k < 2 * LB_QMAX; k += nthreads) {
        const int s = k / LB_QMAX, a = k % LB_QMAX;
        const SetConst<R> &c = p.set[s];
        pc[s][a] = PopC<R>{c.cx[a], c.cy[a], c.crx[a], c.cry[a], c.kx[a], c.ky[a], c.w[a], c.winv[a]};
        mc[s][a] = MomC<R>{c.w[a], c.wcx[a], c.wcy[a], c.winv[a]};
    }
}

/* Stored value at storage column c <-> deviation d, through the lattice's per-column
 * reference density when it has one (p.dcol), else as decode / encode. */
template <int ST>
__device__ __forceinline__ typename Store<ST>::R dec_at(const StepParams<typename Store<ST>::R> &p,
                                                       typename Store<ST>::T v, typename Store<ST>::R winv, int c)
{
    if constexpr (Store<ST>::dev) {
        if (p.dcol) return decode_col<ST>(v, winv, p.rho0, p.dcol[c]);
    }
    return decode<ST>(v, winv, p.rho0);
}
template <int ST>
__device__ __forceinline__ typename Store<ST>::T enc_at(const StepParams<typename Store<ST>::R> &p,
                                                       typename Store<ST>::R d, typename Store<ST>::R w, int c)
{
    if constexpr (Store<ST>::dev) {
        if (p.dcol) return encode_col<ST>(d, w, p.rho0, p.dcol[c]);
    }
    return encode<ST>(d, w, p.rho0);
}

/* sum w d, sum w xi_x d, sum w xi_y d of one node's stored populations (f[a * plane])
 * in population order: the moment pass of the step kernels. dcol (may be NULL): the
 * per-column reference density, the node at storage column c. */
template <int ST, int Q>
__device__ __forceinline__ void node_moments(const typename Store<ST>::T *f, size_t plane,
                                             const MomC<typename Store<ST>::R> *mc, typename Store<ST>::R rho0,
                                             typename Store<ST>::R &rd, typename Store<ST>::R &jx,
                                             typename Store<ST>::R &jy, const typename Store<ST>::R *dcol = nullptr,
                                             int c = 0)
{
    using R = typename Store<ST>::R;
    rd = jx = jy = R(0);
    const R delta = dcol ? dcol[c] : R(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const R d = dcol ? decode_col<ST>(f[a * plane], mc[a].winv, rho0, delta) : decode<ST>(f[a * plane], mc[a].winv, rho0);
        rd = fma(mc[a].w, d, rd);
        jx = fma(mc[a].wcx, d, jx);
        jy = fma(mc[a].wcy, d, jy);
    }
}

/* Row j + offset with ghost = wall node (Sec. 3.2) or a periodic image. |offset| <= 2. */
template <typename R>
__device__ __forceinline__ int row_at(const StepParams<R> &p, int j)
{
    if (j < 0) return p.periodic_y ? j + p.ny : 0;
    if (j >= p.ny) return p.periodic_y ? j - p.ny : p.ny - 1;
    return j;
}

/* Pressure columns are not evolved (corner nodes of diffuse walls are). */
template <typename R>
__device__ __forceinline__ bool is_pressure_node(const StepParams<R> &p, int x, int j)
{
    if ((j == 0 && p.wall_diffuse[0]) || (j == p.ny - 1 && p.wall_diffuse[1])) return false;
    return (x == 0 && p.pressure[0]) || (x == p.nx - 1 && p.pressure[1]);
}

/* f_eq / w - rho0 for Eq. (demoeq) with T = 1: (rho - rho0) + rho [xi.u + ((xi.u)^2 - u^2) / 2]. */
template <typename R>
__device__ __forceinline__ R deq(R rhod, R rho, R eu, R usq)
{
    return fma(rho, fma(R(0.5), fma(eu, eu, -usq), eu), rhod);
}

/* The library is compiled without implicit multiply-add contraction, so that every
 * layout rounds the same expression the same way; the products below are fused where
 * the source says so, in one place for all layouts. */
/* xi . u */
template <typename R>
__device__ __forceinline__ R xi_dot(R cx, R cy, R ux, R uy)
{
    return fma(cy, uy, cx * ux);
}
/* u . u */
template <typename R>
__device__ __forceinline__ R usq_of(R ux, R uy)
{
    return fma(uy, uy, ux * ux);
}
/* Eq. (demoforce) increment of one population: dt rho [g.xi + (g.xi)(xi.u) - g.u],
 * added to t; gxi = g.xi, gu = g.u */
template <typename R>
__device__ __forceinline__ R force_inc(R dt_rho, R gxi, R eu, R gu, R t)
{
    return fma(dt_rho, fma(gxi, eu, gxi) - gu, t);
}

/* tau of Eq. (KN): kn_ref rho_ref / rho (from inv = 1 / rho, already formed by every
 * caller: a multiply instead of a second division), or the constant; minus dt / 2
 * when tau_mode = 1 */
template <typename R>
__device__ __forceinline__ R tau_of(const StepParams<R> &p, R inv)
{
    const R tau = p.tau_const ? p.kn_rho : p.kn_rho * inv;
    return tau - p.tau_shift;
}

/* One element at logical column x of a plane row (prow points at storage column 0),
 * plus its periodic images in the ghost columns. */
template <typename T, typename R>
__device__ __forceinline__ void put1(const StepParams<R> &p, T *prow, int x, T e)
{
    prow[x + LB_GHOST] = e;
    if (p.periodic_x) {
        if (x < LB_GHOST) prow[x + p.nx + LB_GHOST] = e;
        if (x >= p.nx - LB_GHOST) prow[x - p.nx + LB_GHOST] = e;
    }
}

/* Ghost rows that hold a copy of row j: the two rows beyond a wall row (ghost node =
 * wall node) or, for periodic y, the images of rows 0, 1, ny-2, ny-1. Returns the
 * number written to img (0..2) as row offsets relative to j. */
template <typename R>
__device__ __forceinline__ int row_images(const StepParams<R> &p, int j, int img[2])
{
    if (p.periodic_y) {
        if (j == 0 || j == 1) { img[0] = p.ny; return 1; }
        if (j == p.ny - 1 || j == p.ny - 2) { img[0] = -p.ny; return 1; }
        return 0;
    }
    if (j == 0) { img[0] = -1; img[1] = -2; return 2; }
    if (j == p.ny - 1) { img[0] = 1; img[1] = 2; return 2; }
    return 0;
}

/* put1 on row j and on its ghost-row copies. */
template <typename T, typename R>
__device__ __forceinline__ void put1r(const StepParams<R> &p, T *prow, int x, int j, T e)
{
    put1(p, prow, x, e);
    int img[2];
    const int n = row_images(p, j, img);
    for (int k = 0; k < n; ++k) put1(p, prow + (ptrdiff_t)img[k] * p.pitch, x, e);
}

/* Second-order Hermite coefficients of a node from its deviations in its own set:
 * h = {sum w d, sum w xi_x d, sum w xi_y d, sum w (xi_x^2-1) d, sum w xi_x xi_y d,
 *      sum w (xi_y^2-1) d}; the rest-state part w rho0 contributes rho0 to the first
 * and nothing else. */
template <typename R>
__device__ __forceinline__ void hermite_acc(const SetConst<R> &c, int a, R d, R h[6])
{
    h[0] = fma(c.w[a], d, h[0]);
    h[1] = fma(c.wcx[a], d, h[1]);
    h[2] = fma(c.wcy[a], d, h[2]);
    h[3] = fma(c.wxx[a], d, h[3]);
    h[4] = fma(c.wxy[a], d, h[4]);
    h[5] = fma(c.wyy[a], d, h[5]);
}

/* Deviation of population b of set t rebuilt from those coefficients:
 * f_b / w_b - rho0 = h0 + h1 xi_x + h2 xi_y + (1/2) A2 : (xi xi - I). */
template <typename R>
__device__ __forceinline__ R hermite_rebuild(const SetConst<R> &t, int b, const R h[6])
{
    R v = fma(h[1], t.cx[b], h[0]);
    v = fma(h[2], t.cy[b], v);
    v = fma(h[3], t.hxx[b], v);
    v = fma(h[4], t.hxy[b], v);
    v = fma(h[5], t.hyy[b], v);
    return v;
}

}  // namespace lbk
