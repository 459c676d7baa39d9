/*
 * lb_pair.cuh -- the fused time step with paired FP32 arithmetic (layout 7).
 *
 * The Sec. 3.1 / 3.2 / 2.2 update of lb_step_impl.cuh, with the same threads and blocks
 * (one quad of nodes of one row per thread, blocks of one 128-column tile x 8 rows, the
 * next population's stencil loaded while the current one is computed), rewritten for
 * fewer instructions per population on the rows that need no boundary work:
 *   - the four nodes of a quad are two pairs, and every add, multiply and fused
 *     multiply-add that the two nodes of a pair share runs as one packed two-wide FP32
 *     instruction (sm_100 and later);
 *   - the collision is folded into per-node coefficients formed once per step: with
 *     t = xi.u + (xi.u)^2 / 2 (T = 1, Eq. (demoeq)),
 *        omega (f_eq / w - rho0) = P t + B,   P = omega rho,
 *        B = omega (rho - rho0 - rho u.u / 2) - dt rho g.u,
 *     and the Eq. (demoforce) force is dt rho (g.xi)(1 + xi.u) - dt rho g.u, whose last
 *     term is in B; so each population costs six paired operations of collision;
 *   - the y flux of a node uses the limiter in clamp form, minmod(a, b) =
 *     clamp(a, min(b, 0), max(b, 0)), with the bounds of the middle difference shared
 *     by the node's two faces;
 *   - all addresses are 32-bit element offsets from one base pointer per set.
 * Rows with boundary work (diffuse walls and their ghost rows, periodic-y edge rows,
 * mode-B shadow tiles) run the step_cells path of layout 0 unchanged; a warp is one row
 * of one tile, so the choice never splits a warp. Pressure columns, ragged edges and
 * periodic ghost columns are handled per lane in the store. Mode-A interface rows are
 * left to the interface pass, as in every layout.
 *
 * Results agree with the other layouts to rounding, not bit for bit (different
 * operation order, multiply-add contraction on in this file).
 */
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lb_common.cuh"
#include "lb_step_impl.cuh"

namespace lbk {

/* Per-population constants of the paired path. */
struct alignas(16) PairC {
    float2 cx2, cy2;     /* (xi_x, xi_x), (xi_y, xi_y) */
    float2 ncx2, nacy2;  /* (-c_x, -c_x), (-|c_y|, -|c_y|) */
    float2 ky2;          /* ((1 - |c_y|) / 2, ...) */
    float crx, kx;       /* c_x, (1 - |c_x|) / 2 */
    int ystep;           /* sign(c_y) x pitch: the y window's row step (0: no y flux) */
    int pad[3];
};
struct alignas(16) PairC2 {
    float2 gxi2, w2, winv2, pad; /* (g.xi, g.xi), (w, w), (1 / w, 1 / w) */
};
struct alignas(16) MomC2 {
    float2 w2, wcx2, wcy2, winv2;
};

/* The constant tables of one lattice, one after the other in device memory: the PopC and
 * MomC of layout 0 (for the rows with boundary work), then PairC, PairC2 and MomC2, each
 * [2 sets][LB_QMAX populations]. Built once per lattice; every thread reads the entries it
 * needs straight from there (the same address across a warp). */
struct PairTables {
    PopC<float> pc[2][LB_QMAX];
    MomC<float> mc[2][LB_QMAX];
    PairC pp[2][LB_QMAX];
    PairC2 pp2[2][LB_QMAX];
    MomC2 pm[2][LB_QMAX];
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
/* a - b, exact as a fused b * (-1) + a */
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

static __global__ void pair_table_kernel(const __grid_constant__ StepParams<float> p, PairTables *t)
{
    stage_consts(p, t->pc, t->mc, threadIdx.x, blockDim.x);
    for (int k = threadIdx.x; k < 2 * LB_QMAX; k += blockDim.x) {
        const int s = k / LB_QMAX, a = k % LB_QMAX;
        const SetConst<float> &c = p.set[s];
        PairC q;
        q.cx2 = f2(c.cx[a]);
        q.cy2 = f2(c.cy[a]);
        q.ncx2 = f2(-c.crx[a]);
        q.nacy2 = f2(-fabsf(c.cry[a]));
        q.ky2 = f2(c.ky[a]);
        q.crx = c.crx[a];
        q.kx = c.kx[a];
        q.ystep = c.cry[a] > 0.0f ? p.pitch : (c.cry[a] < 0.0f ? -p.pitch : 0);
        q.pad[0] = q.pad[1] = q.pad[2] = 0;
        t->pp[s][a] = q;
        t->pp2[s][a] = PairC2{f2(xi_dot(c.cx[a], c.cy[a], p.gx, p.gy)), f2(c.w[a]), f2(c.winv[a]), f2(0.0f)};
        t->pm[s][a] = MomC2{f2(c.w[a]), f2(c.wcx[a]), f2(c.wcy[a]), f2(c.winv[a])};
    }
}

/* Four stored values <-> two FP32 pairs (deviations), per storage format. */
template <int ST>
__device__ __forceinline__ void pair_ld(const typename Store<ST>::T *p, float2 &a, float2 &b)
{
    if constexpr (ST == 1 || ST == 2) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        if constexpr (ST == 3) {
            a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
            b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        } else {
            a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
            b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
        }
    }
}
template <int ST>
__device__ __forceinline__ void pair_st(typename Store<ST>::T *p, float2 a, float2 b)
{
    if constexpr (ST == 1 || ST == 2) {
        *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        uint2 q;
        if constexpr (ST == 3) {
            const __half2 ha = __float22half2_rn(a), hb = __float22half2_rn(b);
            q.x = *reinterpret_cast<const uint32_t *>(&ha);
            q.y = *reinterpret_cast<const uint32_t *>(&hb);
        } else {
            const __nv_bfloat162 ha = __float22bfloat162_rn(a), hb = __float22bfloat162_rn(b);
            q.x = *reinterpret_cast<const uint32_t *>(&ha);
            q.y = *reinterpret_cast<const uint32_t *>(&hb);
        }
        *reinterpret_cast<uint2 *>(p) = q;
    }
}

/* The stored values one population needs for a quad: its own four, the y window rows
 * j - 2s, j - s and j + s with s = sign(xi_y) (when xi_y != 0) and two values beside the
 * quad on each side (when xi_x != 0). */
template <typename T>
struct PairStencil {
    T v[4], y[3][4], l[2], r[2];
};

/* The per-node coefficients of the folded collision for a quad (two pairs), from its
 * sums rd = sum w d, jx = sum w xi_x d, jy = sum w xi_y d. */
struct PairNode {
    float2 ux[2], uy[2], P[2], B[2], nom[2], dr[2];
};

template <bool FORCE>
__device__ __forceinline__ PairNode pair_node_state(const StepParams<float> &p, const float2 (&rd)[2],
                                                    const float2 (&jx)[2], const float2 (&jy)[2])
{
    PairNode nd;
    const float rho0 = p.rho0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float uxe[2], uye[2], pe[2], be[2], oe[2], de[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float rdv = e ? rd[h].y : rd[h].x;
            const float rho = rho0 + rdv;
            const float inv = 1.0f / rho;
            const float u = (e ? jx[h].y : jx[h].x) * inv, v = (e ? jy[h].y : jy[h].x) * inv;
            const float o = p.dt / tau_of(p, inv);
            float b = o * fmaf(-0.5f * rho, usq_of(u, v), rdv);
            de[e] = p.dt * rho;
            if constexpr (FORCE) b = fmaf(-de[e], xi_dot(p.gx, p.gy, u, v), b);
            uxe[e] = u;
            uye[e] = v;
            pe[e] = o * rho;
            be[e] = b;
            oe[e] = -o;
        }
        nd.ux[h] = make_float2(uxe[0], uxe[1]);
        nd.uy[h] = make_float2(uye[0], uye[1]);
        nd.P[h] = make_float2(pe[0], pe[1]);
        nd.B[h] = make_float2(be[0], be[1]);
        nd.nom[h] = make_float2(oe[0], oe[1]);
        nd.dr[h] = make_float2(de[0], de[1]);
    }
    return nd;
}

/* The increment of one population at a quad (collision and force, x flux, y flux), from
 * its deviations v (two pairs); xh(i) gives the x halos, i = 0, 1 at columns x0-2, x0-1
 * and i = 2, 3 at x0+4, x0+5 (asked for when c_x != 0), yw(h, i) the pair h of the y
 * window rows i = 0, 1, 2 at rows j-2s, j-s, j+s with s = sign(xi_y) (asked for when
 * c_y != 0), both decoded to deviations. */
template <bool FORCE, typename XH, typename YW>
__device__ __forceinline__ void pair_increment(const PairC &pc, const PairC2 &pc2, const PairNode &nd,
                                               const float2 (&v)[2], const XH &xh, const YW &yw, float2 (&c)[2])
{
    /* collision and force */
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 eu = fma2(pc.cy2, nd.uy[h], mul2(pc.cx2, nd.ux[h]));
        const float2 t = fma2(mul2(f2(0.5f), eu), eu, eu);
        c[h] = fma2(nd.nom[h], v[h], fma2(nd.P[h], t, nd.B[h]));
        if constexpr (FORCE) c[h] = fma2(nd.dr[h], fma2(pc2.gxi2, eu, pc2.gxi2), c[h]);
    }
    /* x flux (Sec. 3.1, mirrored for negative velocities) */
    if (pc.crx != 0.0f) {
        const float vv[4] = {v[0].x, v[0].y, v[1].x, v[1].y};
        const float l0 = xh(0), l1 = xh(1), r0 = xh(2), r1 = xh(3);
        float Dx[4];
        if (pc.crx > 0.0f) {
            float d[6], n[6], m[5];
            d[0] = l1 - l0;
            d[1] = vv[0] - l1;
            d[2] = vv[1] - vv[0];
            d[3] = vv[2] - vv[1];
            d[4] = vv[3] - vv[2];
            d[5] = r0 - vv[3];
#pragma unroll
            for (int i = 0; i < 6; ++i) n[i] = neg_part(d[i]);
#pragma unroll
            for (int i = 0; i < 5; ++i) m[i] = minmod_n(d[i], d[i + 1], n[i], n[i + 1]);
#pragma unroll
            for (int k = 0; k < 4; ++k) Dx[k] = fmaf(pc.kx, m[k + 1] - m[k], d[k + 1]);
        } else {
            float e[6], n[6], m[5];
            e[0] = vv[0] - l1;
            e[1] = vv[1] - vv[0];
            e[2] = vv[2] - vv[1];
            e[3] = vv[3] - vv[2];
            e[4] = r0 - vv[3];
            e[5] = r1 - r0;
#pragma unroll
            for (int i = 0; i < 6; ++i) n[i] = neg_part(e[i]);
#pragma unroll
            for (int i = 0; i < 5; ++i) m[i] = minmod_n(e[i], e[i + 1], n[i], n[i + 1]);
#pragma unroll
            for (int k = 0; k < 4; ++k) Dx[k] = fmaf(-pc.kx, m[k + 1] - m[k], e[k + 1]);
        }
        c[0] = fma2(pc.ncx2, make_float2(Dx[0], Dx[1]), c[0]);
        c[1] = fma2(pc.ncx2, make_float2(Dx[2], Dx[3]), c[1]);
    }
    /* y flux on the window W = (f_{j-2s}, f_{j-s}, f_j, f_{j+s}), s = sign(xi_y): the
     * printed flux for xi_y > 0 and its mirror image for xi_y < 0 are both
     *   c_y (F^{j+1/2} - F^{j-1/2}) = |c_y| (d1 + k (minmod(d1, d2) - minmod(d0, d1)))
     * with d0, d1, d2 the differences along W (the mirror image reverses W and flips the
     * sign of every difference, and minmod is odd) */
    if (pc.ystep != 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 w0 = yw(h, 0), w1 = yw(h, 1), w3 = yw(h, 2);
            const float2 d0 = sub2(w1, w0), d1 = sub2(v[h], w1), d2 = sub2(w3, v[h]);
            float2 ma, mb;
            {
                const float lo = fminf(d1.x, 0.0f), hi = fmaxf(d1.x, 0.0f);
                ma.x = fminf(fmaxf(d0.x, lo), hi);
                mb.x = fminf(fmaxf(d2.x, lo), hi);
            }
            {
                const float lo = fminf(d1.y, 0.0f), hi = fmaxf(d1.y, 0.0f);
                ma.y = fminf(fmaxf(d0.y, lo), hi);
                mb.y = fminf(fmaxf(d2.y, lo), hi);
            }
            const float2 Dy = fma2(pc.ky2, sub2(mb, ma), d1);
            c[h] = fma2(pc.nacy2, Dy, c[h]);
        }
    }
}

/* One quad of a row without boundary work. */
template <int ST, int Q, bool COL, bool FORCE>
__device__ __forceinline__ void pair_cells(const StepParams<float> &p, int s, int x0, int j, const PairC *pcs,
                                           const PairC2 *pcs2, const MomC2 *mcs)
{
    using T = typename Store<ST>::T;
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]);
    T *__restrict__ fout = static_cast<T *>(p.fout[s]);
    const uint32_t plane = (uint32_t)p.plane, pitch = (uint32_t)p.pitch;
    const uint32_t col = (uint32_t)(x0 + LB_GHOST);
    const uint32_t own = (uint32_t)j * pitch + col;
    const float rho0 = p.rho0;
    const float2 nrho02 = f2(-rho0);
    /* per-column reference density: delta at columns x0 - 2 .. x0 + 5 */
    float dl[8];
    if constexpr (COL) {
#pragma unroll
        for (int i = 0; i < 8; ++i) dl[i] = p.dcol[col - 2 + i];
    }
    /* stored pair -> deviation pair at columns k, k + 1 of the quad (k = 0 or 2) */
    auto dec2 = [&](float2 raw, float2 winv2, int k) -> float2 {
        if constexpr (ST == 1) return fma2(raw, winv2, nrho02);
        else if constexpr (COL) return add2(raw, make_float2(dl[k + 2], dl[k + 3]));
        else return raw;
    };
    auto dec1 = [&](T raw, float winv, int i) -> float {
        if constexpr (COL) return decode_col<ST>(raw, winv, rho0, dl[i]);
        else return decode<ST>(raw, winv, rho0);
    };

    /* 1. moments */
    float2 rd[2] = {f2(0.0f), f2(0.0f)}, jx[2] = {f2(0.0f), f2(0.0f)}, jy[2] = {f2(0.0f), f2(0.0f)};
#pragma unroll kMomUnroll
    for (int a = 0; a < Q; ++a) {
        const MomC2 mc = mcs[a];
        float2 v[2];
        pair_ld<ST>(fin + (uint32_t)a * plane + own, v[0], v[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 d = dec2(v[h], mc.winv2, 2 * h);
            rd[h] = fma2(mc.w2, d, rd[h]);
            jx[h] = fma2(mc.wcx2, d, jx[h]);
            jy[h] = fma2(mc.wcy2, d, jy[h]);
        }
    }
    /* 2. per-node collision coefficients (and the force weight) */
    const PairNode nd = pair_node_state<FORCE>(p, rd, jx, jy);

    /* stores: plain 16-byte vectors, or per node for pressure columns, a ragged edge and
     * periodic ghost columns (the row has no ghost-row images here) */
    bool valid[4];
    bool plain = !(p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        valid[k] = x0 + k < p.nx && !is_pressure_node(p, x0 + k, j);
        plain = plain && valid[k];
    }
    const bool fast = plain && !p.sr;

    /* the y window reads rows j - 2s, j - s, j + s (s = +-1): the ghost rows beyond a wall
     * hold copies of the wall row, so the offsets need no clamping on these rows */
    auto load = [&](int a, PairStencil<T> &S, const PairC &pc) {
        const T *pa = fin + (uint32_t)a * plane + own;
        ldn<4>(pa, S.v);
        if (pc.ystep != 0) {
            ldn<4>(pa - 2 * pc.ystep, S.y[0]);
            ldn<4>(pa - pc.ystep, S.y[1]);
            ldn<4>(pa + pc.ystep, S.y[2]);
        }
        if (pc.crx != 0.0f) {
            ld2(pa - 2, S.l);
            ld2(pa + 4, S.r);
        }
    };
    auto pair_of = [&](const T (&q)[4], int h) -> float2 {
        return make_float2(to_r(q[2 * h]), to_r(q[2 * h + 1]));
    };
    auto compute = [&](int a, const PairStencil<T> &S, const PairC &pc, const PairC2 &pc2) {
        float2 v[2], c[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) v[h] = dec2(pair_of(S.v, h), pc2.winv2, 2 * h);
        auto xh = [&](int i) -> float {
            return i < 2 ? dec1(S.l[i], pc2.winv2.x, i) : dec1(S.r[i - 2], pc2.winv2.x, i + 4);
        };
        auto yw = [&](int h, int i) -> float2 { return dec2(pair_of(S.y[i], h), pc2.winv2, 2 * h); };
        pair_increment<FORCE>(pc, pc2, nd, v, xh, yw, c);
        /* store */
        float2 dn[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) dn[h] = add2(v[h], c[h]);
        T *dst = fout + (uint32_t)a * plane + own;
        if (fast) {
            if constexpr (ST == 1) {
                const float2 rr = add2(f2(rho0), dn[0]), ss = add2(f2(rho0), dn[1]);
                pair_st<ST>(dst, mul2(pc2.w2, rr), mul2(pc2.w2, ss));
            } else if constexpr (COL) {
                pair_st<ST>(dst, sub2(dn[0], make_float2(dl[2], dl[3])), sub2(dn[1], make_float2(dl[4], dl[5])));
            } else {
                pair_st<ST>(dst, dn[0], dn[1]);
            }
            return;
        }
        const float dv[4] = {dn[0].x, dn[0].y, dn[1].x, dn[1].y};
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (p.sr) {
                const uint32_t bits = sr_bits(x0 + k, j, p.nx, a, p.step_key);
                if constexpr (COL) e[k] = encode_sr<ST>(dv[k] - dl[k + 2], pc2.w2.x, rho0, bits);
                else e[k] = encode_sr<ST>(dv[k], pc2.w2.x, rho0, bits);
            } else {
                if constexpr (COL) e[k] = encode_col<ST>(dv[k], pc2.w2.x, rho0, dl[k + 2]);
                else e[k] = encode<ST>(dv[k], pc2.w2.x, rho0);
            }
        }
        if (plain) {
            st4(dst, e);
        } else {
            T *prow = dst - col;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[k]) put1(p, prow, x0 + k, e[k]);
        }
    };

    /* 3. population loop, the stencil of population a + 1 loaded while a is computed;
     * two buffers in turn */
    PairStencil<T> A, Bf;
    load(0, A, pcs[0]);
#pragma unroll 1
    for (int a = 0; a < Q; a += 2) {
        const PairC pa = pcs[a];
        const PairC2 pa2 = pcs2[a];
        const bool more = a + 1 < Q;
        PairC pb;
        PairC2 pb2;
        if (more) {
            pb = pcs[a + 1];
            pb2 = pcs2[a + 1];
            load(a + 1, Bf, pb);
        }
        compute(a, A, pa, pa2);
        if (!more) break;
        if (a + 2 < Q) load(a + 2, A, pcs[a + 2]);
        compute(a + 1, Bf, pb, pb2);
    }
}

template <int ST, bool COL, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY, 2) pair_kernel(const __grid_constant__ StepParams<float> p)
{
    const PairTables *tab = static_cast<const PairTables *>(p.ctab);
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
    int img[2];
    const bool edge_row = (flags & LB_TILE_SHADOW) || row_images(p, j, img) > 0 ||
                          (j == 0 && p.wall_diffuse[0]) || (j == p.ny - 1 && p.wall_diffuse[1]);
    if (edge_row) {
        constexpr bool PF = step_prefetch<ST>();
        const PopC<float> *pc = tab->pc[s];
        const MomC<float> *mc = tab->mc[s];
        if (q == 9) step_cells<ST, 9, PF, 4, COL>(p, s, flags, x0, j, pc, mc);
        else if (q == 16) step_cells<ST, 16, PF, 4, COL>(p, s, flags, x0, j, pc, mc);
        else step_cells<ST, 36, PF, 4, COL>(p, s, flags, x0, j, pc, mc);
        return;
    }
    if (q == 9) pair_cells<ST, 9, COL, FORCE>(p, s, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s]);
    else if (q == 16) pair_cells<ST, 16, COL, FORCE>(p, s, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s]);
    else pair_cells<ST, 36, COL, FORCE>(p, s, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s]);
}

template <int ST>
void launch_pair_store(const StepParams<float> &p, void *stream)
{
    static_assert(ST >= 1 && ST <= 4, "paired FP32 arithmetic: FP32 and 16-bit storage");
    dim3 block(LB_BX, LB_BY);
    dim3 grid((p.nx + 4 * LB_BX - 1) / (4 * LB_BX), (p.ny + LB_BY - 1) / LB_BY);
    if (p.block_order) grid = dim3(grid.x * grid.y, 1);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool col = Store<ST>::dev && p.dcol;
    if (col) {
        if constexpr (Store<ST>::dev) {
            if (p.has_force) pair_kernel<ST, true, true><<<grid, block, 0, st>>>(p);
            else pair_kernel<ST, true, false><<<grid, block, 0, st>>>(p);
        }
        return;
    }
    if (p.has_force) pair_kernel<ST, false, true><<<grid, block, 0, st>>>(p);
    else pair_kernel<ST, false, false><<<grid, block, 0, st>>>(p);
}

}  // namespace lbk
