/*
 * lb_pressure.cuh -- the pressure columns of one row (Sec. 2.2 virtual boundary on an
 * open side), shared by the pressure pass (lb_step.cu) and layout 10 (lb_ring2.cuh),
 * which does this work at the end of the rows of the first and last tiles.
 */
#pragma once

#include "lb_common.cuh"

namespace lbk {

/* Sum over the 32 lanes of a warp (every lane gets the total). */
template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

/* Column x = 0 (left) or nx-1 (right), interior rows: f = f_eq(rho_b, u_1) +
 * [f - f_eq](node one step inwards), the virtual-boundary construction of Sec. 2.2
 * applied to an open boundary. Then every row's ghost columns beyond the boundary get
 * copies of the boundary node (in its set, and rebuilt in the other set where the tile
 * neighbours it). One warp per (row, side); lane l handles populations l and l + 32, and
 * the node sums are warp reductions. */
/* A product and a sum rounded separately: the translation units of the library are built
 * with and without multiply-add contraction, and these are the sums of products below
 * that a contraction could fuse; spelled out, every unit gives the same bits. */
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

/* Column x = 0 (side 0, left) or nx-1 (side 1, right) of row j, done by one whole warp:
 * on an interior row f = f_eq(rho_b, u_1) + [f - f_eq](node one step inwards), the
 * virtual-boundary construction of Sec. 2.2 applied to an open boundary, with its carried
 * moments; then, on every row, the ghost columns beyond the boundary get copies of the
 * boundary node (in its set, and rebuilt in the other set where the tile neighbours it).
 * Lane l handles populations l and l + 32; the node sums are warp reductions. The node
 * one step inwards must be final (this step's value) and visible to the whole warp. */
template <int ST>
__device__ __forceinline__ void pressure_row(const StepParams<typename Store<ST>::R> &p, int j, int side)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int lane = threadIdx.x & 31;
    const int xb = side == 0 ? 0 : p.nx - 1;
    const int xi = side == 0 ? 1 : p.nx - 2;
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + xb / LB_TILE_X];
    const int s = flags & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const int q = c.q;
    const size_t plane = p.plane;
    const R rho0 = p.rho0;
    T *f = static_cast<T *>(p.fout[s]) + (size_t)j * p.pitch + LB_GHOST;
    const int a0 = lane, a1 = lane + 32;
    const bool h0 = a0 < q, h1 = a1 < q;
    int img[2];
    const int nimg = row_images(p, j, img);
    T e0 = T(0), e1 = T(0);   /* the boundary node's final populations a0, a1 */
    if (is_pressure_node(p, xb, j)) {
        R d0 = R(0), d1 = R(0), r = R(0), mx = R(0), my = R(0);
        if (h0) {
            d0 = dec_at<ST>(p, f[a0 * plane + xi], c.winv[a0], xi + LB_GHOST);
            r = c.w[a0] * d0;
            mx = c.wcx[a0] * d0;
            my = c.wcy[a0] * d0;
        }
        if (h1) {
            d1 = dec_at<ST>(p, f[a1 * plane + xi], c.winv[a1], xi + LB_GHOST);
            r = fma(c.w[a1], d1, r);
            mx = fma(c.wcx[a1], d1, mx);
            my = fma(c.wcy[a1], d1, my);
        }
        r = warp_sum(r);
        mx = warp_sum(mx);
        my = warp_sum(my);
        const R rn = rho0 + r, uxn = mx / rn, uyn = my / rn, usn = add_rn(mul_rn(uxn, uxn), mul_rn(uyn, uyn));
        const R rb = p.rho_side[side];
        auto put = [&](int a, R d) -> T {
            const R e = add_rn(mul_rn(c.cx[a], uxn), mul_rn(c.cy[a], uyn));
            const R dv = deq(rb - rho0, rb, e, usn) + (d - deq(r, rn, e, usn));
            const T v = enc_at<ST>(p, dv, c.w[a], xb + LB_GHOST);
            f[a * plane + xb] = v;
            for (int t = 0; t < nimg; ++t) f[a * plane + (ptrdiff_t)img[t] * p.pitch + xb] = v;
            return v;
        };
        if (h0) e0 = put(a0, d0);
        if (h1) e1 = put(a1, d1);
        /* carried moments of the node (layouts 4 and 10): its final populations summed in
         * population order, as the moment pass of the step kernels does */
        R sr = R(0), sx = R(0), sy = R(0);
        for (int a = 0; a < q; ++a) {
            const T e = __shfl_sync(0xffffffffu, a < 32 ? e0 : e1, a & 31);
            const R d = dec_at<ST>(p, e, c.winv[a], xb + LB_GHOST);
            sr = fma(c.w[a], d, sr);
            sx = fma(c.wcx[a], d, sx);
            sy = fma(c.wcy[a], d, sy);
        }
        if (lane == 0 && p.aux_out) {
            R *aout = static_cast<R *>(p.aux_out);
            const size_t ap = (size_t)p.pitch * p.ny, m = (size_t)j * p.pitch + xb;
            aout[m] = sr;
            aout[ap + m] = sx;
            aout[2 * ap + m] = sy;
        }
    } else {
        /* a wall row: the node the step kernel stored */
        if (h0) e0 = f[a0 * plane + xb];
        if (h1) e1 = f[a1 * plane + xb];
    }
    /* ghost columns, and the node's second-order Hermite coefficients for a shadow */
    R hc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    auto ghost = [&](int a, T e) {
        for (int g = 1; g <= LB_GHOST; ++g) f[a * plane + (side == 0 ? xb - g : xb + g)] = e;
        hermite_acc(c, a, dec_at<ST>(p, e, c.winv[a], xb + LB_GHOST), hc);
    };
    if (h0) ghost(a0, e0);
    if (h1) ghost(a1, e1);
    if (flags & LB_TILE_SHADOW) {
#pragma unroll
        for (int m = 0; m < 6; ++m) hc[m] = warp_sum(hc[m]);
        const SetConst<R> &ct = p.set[1 - s];
        T *ft = static_cast<T *>(p.fout[1 - s]) + (size_t)j * p.pitch + LB_GHOST;
        for (int b = lane; b < ct.q; b += 32) {
            const T e = enc_at<ST>(p, hermite_rebuild(ct, b, hc), ct.w[b], xb + LB_GHOST);
            for (int g = 0; g <= LB_GHOST; ++g) ft[b * plane + (side == 0 ? xb - g : xb + g)] = e;
            for (int t = 0; t < nimg; ++t) ft[b * plane + (ptrdiff_t)img[t] * p.pitch + xb] = e;
        }
    }
}

}  // namespace lbk
