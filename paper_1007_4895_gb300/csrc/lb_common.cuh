/*
 * lb_common.cuh -- device helpers shared by the step kernels and the auxiliary
 * kernels: stencil row indices, the equilibrium in deviation form, stores with
 * periodic images, and the second-order Hermite rebuild of a node in another set.
 */
#pragma once

#include "lb_internal.h"
#include "lb_store.cuh"

namespace lbk {

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
    return rhod + rho * (eu + R(0.5) * (eu * eu - usq));
}

template <typename R>
__device__ __forceinline__ R tau_of(const StepParams<R> &p, R rho)
{
    R tau = p.tau_const ? p.kn_rho : p.kn_rho / rho;
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
