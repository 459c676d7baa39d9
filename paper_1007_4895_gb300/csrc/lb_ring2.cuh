/*
 * lb_ring2.cuh -- the ring-fed step of lb_ring.cuh as a persistent kernel over row work
 * queues (layout 10).
 *
 * Work item: one row of one 128-column tile, done by one warp (a quad of nodes per
 * lane). The host groups the rows in block units of LB_STEP_BY rows of a tile (what a
 * block of layout 9 does), sorts the units most work first, and deals them round-robin
 * to one queue per SM, keeping the last (cheapest) tenth in a shared queue. A warp takes
 * rows from the queue of the SM it runs on, then from the shared queue, then whatever
 * is left anywhere (so an SM that got fewer blocks loses no work). The warps of an SM
 * thus work on neighbouring rows of the same tiles and share their stencil rows in L1,
 * no warp waits for another, and the long high-order rows start first.
 *
 * The rows are of four kinds, decided on the host (stochastic rounding makes every row
 * general):
 *   - lean: no boundary work (pressure columns count as none: the pressure pass
 *     overwrites what the step stores there);
 *   - row: a diffuse wall, ghost-row copies, a mode-B shadow or periodic ghost columns:
 *     the lean population loop (plus the wall sums of a wall row), then that work;
 *   - edge: a tile that ends inside the grid's last 128 columns, stored node by node;
 *   - general: stochastic rounding, or boundary work in such a tile.
 * Lean, row and edge rows run a body specialised on the velocity set: the loop is
 * unrolled over the abscissae of the product rule (alpha = iy n + ix), so the sign of
 * xi_x, whether xi_y is zero and the ring slot of every population are compile-time
 * constants, and the per-population constants are read from kernel-parameter space
 * with a warp-uniform index. General rows run the body of layout 9, not inlined.
 *
 * Without a body force, the rows of the first and last tiles also do the pressure
 * columns' update (lb_pressure.cuh, the same code as the pressure pass), so such a step
 * needs no pressure pass.
 *
 * The arithmetic is that of layout 9 (lb_pair.cuh) and of the pressure pass, operation for
 * operation, so the two layouts give the same bits.
 */
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "lb_pressure.cuh"
#include "lb_ring.cuh"

namespace lbk {

/* sign of abscissa i of the ascending n-point Gauss-Hermite rule (0 at the middle of an
 * odd rule); the host checks each lattice's sets against it before offering layout 10 */
__host__ __device__ constexpr int gh_sign(int n, int i) { return (n & 1) && i == n / 2 ? 0 : (i < n / 2 ? -1 : 1); }

/* a pair of deviations rounded as the storage format stores them */
template <int ST>
__device__ __forceinline__ float2 pair_round(float2 v)
{
    if constexpr (ST == 3) return __half22float2(__float22half2_rn(v));
    else if constexpr (ST == 4) return __bfloat1622float2(__float22bfloat162_rn(v));
    else return v;
}

/* Row kinds of the queues */
enum : uint32_t { RING_LEAN = 0u, RING_EDGE = 1u, RING_ROW = 2u, RING_GENERAL = 3u, RING_BATCH = 4u };

/* Ring stages of layout 10 (each laid out as a stage of layout 9's ring, so that the
 * general rows' body uses the first three) and resident blocks per SM, by measurement
 * on the 16384 x 128 channel and the 1024 x 512 Poiseuille channel: FP32 storage four
 * stages, two blocks of 128 registers (three stages at three blocks of 80 registers
 * were as fast on the channel and 12 % slower on the Poiseuille lattice); 16-bit
 * storage three stages, three blocks (a fourth stage was 4 % slower). */
#ifndef RING10_STAGES_F32
#define RING10_STAGES_F32 4
#endif
#ifndef RING10_STAGES_16
#define RING10_STAGES_16 3
#endif
#ifndef RING10_BLOCKS_F32
#define RING10_BLOCKS_F32 2
#endif
template <int ST>
__host__ __device__ constexpr int ring10_stages()
{
    return sizeof(typename Store<ST>::T) == 4 ? RING10_STAGES_F32 : RING10_STAGES_16;
}
template <int ST>
__host__ __device__ constexpr int ring10_blocks()
{
    return sizeof(typename Store<ST>::T) == 4 ? RING10_BLOCKS_F32 : 3;
}
static_assert(RING10_STAGES_F32 >= RING_STAGES && RING10_STAGES_16 >= RING_STAGES, "layout 9's body needs its stages");
/* Dynamic shared memory of a layout-10 block: the ring, then 16 bytes per thread for the
 * wall sums of a wall row. */
template <int ST>
__host__ __device__ constexpr size_t ring_unit_smem_bytes()
{
    return ring10_stages<ST>() * ring_stage_bytes<ST>() + (size_t)LB_BX * LB_BY * sizeof(float4);
}

/* The boundary work of a row of kind RING_ROW (set S of Q populations, the other set of
 * QT), after the population loop has stored every node of the lane's quad as an inner
 * node: the diffuse-wall fill (Sec. 3.2; num = sum over the wall-bound populations of
 * |xi.n| w d, wsgn = +1 bottom wall, -1 top wall) with the wall row's carried moments
 * summed again from its final values, the copies of the row into its ghost rows and of
 * the lane's nodes into periodic ghost columns, and the mode-B rebuild of a shadow row
 * in the other set (Sec. 2.2). Few rows take this path, so its loops stay rolled (the
 * code stays small and in the instruction cache), with the constants read from the
 * parameter-space table by a warp-uniform index. */
template <int ST, int Q, int S, int QT, bool COL, int G>
__device__ __forceinline__ void ring_row_finish(const StepParams<float> &p, const RingTab &tab, int x0, int j,
                                                uint8_t flags, float wsgn, const float4 &num, const float (&dl)[8],
                                                bool noimg)
{
    using T = typename Store<ST>::T;
    const RingPop *tp = tab.pop[S];
    const float rho0 = p.rho0;
    const uint32_t plane = (uint32_t)p.plane, pitch = (uint32_t)p.pitch;
    const uint32_t col = (uint32_t)(x0 + LB_GHOST);
    T *const frow = static_cast<T *>(p.fout[S]) + (size_t)j * pitch;   /* row j of plane 0, column 0 - LB_GHOST */
    int img[2] = {0, 0};
    const int nimg = row_images(p, j, img);
    const bool gx = !noimg && p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST);
    /* a quad whose one periodic image is a whole quad: its offset (one vector store) */
    int img_dx = 0;
    if (gx && (p.nx & 3) == 0) {
        if (x0 + 3 < LB_GHOST && x0 + 3 < p.nx - LB_GHOST) img_dx = p.nx;
        else if (x0 >= p.nx - LB_GHOST && x0 >= LB_GHOST) img_dx = -p.nx;
    }
    const bool shadow = flags & LB_TILE_SHADOW;
    const int wall = wsgn > 0.0f ? 0 : (wsgn < 0.0f ? 1 : -1);
    auto enc = [&](float d, float w, int k) -> T {
        if constexpr (COL) return encode_col<ST>(d, w, rho0, dl[k + 2]);
        else return encode<ST>(d, w, rho0);
    };
    /* quad e of row prow (column 0 - LB_GHOST) into the row itself (self), its ghost rows
     * and, for this lane's nodes, the periodic ghost columns of each */
    auto copies = [&](T *prow, const T (&e)[4], bool self) {
        for (int t = -1; t < nimg; ++t) {
            T *r = t < 0 ? prow : prow + (ptrdiff_t)img[t] * (ptrdiff_t)pitch;
            if (t >= 0 || self) st4(r + col, e);
            if (img_dx != 0) {
                st4(r + col + img_dx, e);
            } else if (gx) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int x = x0 + k;
                    if (x < LB_GHOST) r[x + p.nx + LB_GHOST] = e[k];
                    if (x >= p.nx - LB_GHOST) r[x - p.nx + LB_GHOST] = e[k];
                }
            }
        }
    };
    /* diffuse wall: f = rho_W S(u_W) for the gas-bound populations, zero net mass flux */
    if (wall >= 0) {
        const float uwx = p.uw_x[wall], uwy = p.uw_y[wall];
        const float usw = uwx * uwx + uwy * uwy;
        const float kd = p.kdiff[S][wall], kout = p.kout[S][wall];
        const float nm[4] = {num.x, num.y, num.z, num.w};
        float rwd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rwd[k] = fmaf(rho0, kd, nm[k]) / kout;   /* rho_W - rho0 */
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const RingPop &rp = tp[a];
            if (rp.cy2.x * wsgn <= 0.0f) continue;
            const float ew = rp.cx2.x * uwx + rp.cy2.x * uwy;
            const float sm1 = ew + 0.5f * (ew * ew - usw);    /* S / w - 1 */
            T e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] = enc(fmaf(rwd[k] + rho0, sm1, rwd[k]), rp.w2.x, k);
            copies(frow + (size_t)a * plane, e, true);
        }
    }
    if (nimg == 0 && !gx && !shadow) return;
    /* copies of the populations the loop stored, the shadow's Hermite coefficients and,
     * for a wall row, its carried moments summed again from its final values */
    float h[4][6], mo[3][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        mo[0][k] = mo[1][k] = mo[2][k] = 0.0f;
#pragma unroll
        for (int m = 0; m < 6; ++m) h[k][m] = 0.0f;
    }
    /* G populations' quads loaded together (the stores of copies() go to other rows and
     * columns, never to a quad still to be read), then taken in population order; G > 1
     * only where the registers allow it */
#pragma unroll 1
    for (int a0 = 0; a0 < Q; a0 += G) {
        T raw4[G][4];
#pragma unroll
        for (int i = 0; i < G; ++i)
            if (a0 + i < Q) ldn<4>(frow + (size_t)(a0 + i) * plane + col, raw4[i]);
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int a = a0 + i;
            if (a >= Q) break;
            const RingPop &rp = tp[a];
            const T(&raw)[4] = raw4[i];
            if (!(wall >= 0 && rp.cy2.x * wsgn > 0.0f)) copies(frow + (size_t)a * plane, raw, false);
            if (shadow || wall >= 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float d;
                    if constexpr (COL) d = decode_col<ST>(raw[k], rp.winv2.x, rho0, dl[k + 2]);
                    else d = decode<ST>(raw[k], rp.winv2.x, rho0);
                    if (shadow) {   /* the terms of hermite_acc, in its order */
                        h[k][0] = fmaf(rp.w2.x, d, h[k][0]);
                        h[k][1] = fmaf(rp.wcx2.x, d, h[k][1]);
                        h[k][2] = fmaf(rp.wcy2.x, d, h[k][2]);
                        h[k][3] = fmaf(rp.wxx, d, h[k][3]);
                        h[k][4] = fmaf(rp.wxy, d, h[k][4]);
                        h[k][5] = fmaf(rp.wyy, d, h[k][5]);
                    }
                    mo[0][k] = fmaf(rp.w2.x, d, mo[0][k]);
                    mo[1][k] = fmaf(rp.wcx2.x, d, mo[1][k]);
                    mo[2][k] = fmaf(rp.wcy2.x, d, mo[2][k]);
                }
            }
        }
    }
    if (wall >= 0) {
        float *aout = static_cast<float *>(p.aux_out) + (size_t)j * pitch + x0;
        const size_t ap = (size_t)pitch * p.ny;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            __stcg(reinterpret_cast<float4 *>(aout + i * ap), make_float4(mo[i][0], mo[i][1], mo[i][2], mo[i][3]));
    }
    if (!shadow) return;
    const RingPop *tq = tab.pop[1 - S];
    T *const trow = static_cast<T *>(p.fout[1 - S]) + (size_t)j * pitch;
#pragma unroll 1
    for (int b = 0; b < QT; ++b) {
        const RingPop &rb = tq[b];
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {   /* hermite_rebuild, term by term */
            float v = fmaf(h[k][1], rb.cx2.x, h[k][0]);
            v = fmaf(h[k][2], rb.cy2.x, v);
            v = fmaf(h[k][3], rb.hxx, v);
            v = fmaf(h[k][4], rb.hxy, v);
            v = fmaf(h[k][5], rb.hyy, v);
            e[k] = enc(v, rb.w2.x, k);
        }
        copies(trow + (size_t)b * plane, e, true);
    }
}

/* One row of set S of Q = n^2 populations (n = 3, 4 or 6; the other set has QT) of kind
 * KIND, the quad of nodes x0 .. x0 + 3 of this lane (x0 < nx). Lean and row kinds store
 * every node as an inner node (a pressure node is then overwritten by the pressure pass,
 * with its ghost columns, images and shadow); the row kind then does its boundary work
 * (ring_row_finish); the edge kind stores node by node (ragged end, periodic ghost
 * columns). */
template <int ST, int Q, int S, int QT, bool COL, bool FORCE, uint32_t KIND>
__device__ __forceinline__ void ring_lean(const StepParams<float> &p, const RingTab &tab, int x0, int j,
                                          uint8_t flags, unsigned char *ring, int xmode = 0, bool rowk = true)
{
    /* RING_BATCH: the edge and row kinds of an x-periodic lattice of whole quads in one
     * body, with its halos read inside the row and no ghost-column images (xmode 3), the
     * row work run where `rowk` says so: a batch's steps then run two bodies, not four */
    constexpr bool MIX = KIND == RING_BATCH;
    constexpr bool ROW = KIND == RING_ROW || MIX;
    constexpr bool EDGE = KIND == RING_EDGE;   /* lanes store node by node */
    using T = typename Store<ST>::T;
    constexpr int N = Q == 9 ? 3 : (Q == 16 ? 4 : 6);
    constexpr int NT = LB_BX * LB_BY;
    constexpr int C4 = 4 * (int)sizeof(T), C2 = 2 * (int)sizeof(T);
    constexpr size_t STAGE = ring_stage_bytes<ST>();
    constexpr int RS = ring10_stages<ST>();
    const RingPop *tp = tab.pop[S];
    const int tid = threadIdx.x;
    /* edge kind: nodes this lane stores one by one (pressure column, beyond nx, periodic
     * ghost-column images) */
    bool valid[4] = {true, true, true, true};
    bool plain = true, allv = true;
    int img_dx = 0;   /* a whole quad whose one periodic image is a whole quad: its offset */
    /* xmode (edge and row kinds of an x-periodic lattice whose width is a whole number of
     * quads): bit 0, the x halos of the row's end quads are read from its other end, not
     * from the ghost columns; bit 1, no periodic ghost-column images are written. Within
     * a launch of several steps only the last writes them: the others' are never read. */
    const bool wrapx = (EDGE || ROW) && (xmode & 1) != 0, noimg = (EDGE || ROW) && (xmode & 2) != 0;
    const int hlo = (wrapx && x0 == 0) ? p.nx - 2 : -2;
    const int hro = (wrapx && x0 + 4 == p.nx) ? 4 - p.nx : 4;
    if constexpr (EDGE) {
        plain = !(p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST));
        bool all = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            valid[k] = x0 + k < p.nx && !is_pressure_node(p, x0 + k, j);
            plain = plain && valid[k];
            all = all && valid[k];
        }
        allv = all;
        if (!plain && all && p.periodic_x && (p.nx & 3) == 0) {
            if (x0 + 3 < LB_GHOST && x0 + 3 < p.nx - LB_GHOST) img_dx = p.nx;
            else if (x0 >= p.nx - LB_GHOST && x0 >= LB_GHOST) img_dx = -p.nx;
        }
    }
    /* row kind: the wall of a diffuse-wall row (+1 bottom, -1 top, 0 none) and the lane's
     * wall sums in shared memory after the ring */
    float wsgn = 0.0f;
    if constexpr (ROW) {
        if (j == 0 && p.wall_diffuse[0]) wsgn = 1.0f;
        if (j == p.ny - 1 && p.wall_diffuse[1]) wsgn = -1.0f;
    }
    float4 *const numslot = reinterpret_cast<float4 *>(ring + RS * STAGE) + tid;
    if constexpr (ROW) *numslot = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const T *__restrict__ fin = static_cast<const T *>(p.fin[S]);
    T *__restrict__ fout = static_cast<T *>(p.fout[S]);
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
    unsigned char *const mine4 = ring + (size_t)tid * C4;
    unsigned char *const mine2 = ring + (size_t)4 * NT * C4 + (size_t)tid * C2;
    /* copies of population b into ring stage b % RS (HX: xi_x != 0, HY: xi_y != 0) */
    auto issue = [&](int b, auto hx, auto hy, auto stage) {
        constexpr int st = decltype(stage)::value;
        const T *pa = fin + (uint32_t)b * plane + own;
        unsigned char *s4 = mine4 + st * STAGE;
        unsigned char *s2 = mine2 + st * STAGE;
        ring_cp<C4>(s4, pa);
        if constexpr (decltype(hy)::value) {
            const int ys = tp[b].ystep;
            ring_cp<C4>(s4 + (size_t)NT * C4, pa - 2 * ys);
            ring_cp<C4>(s4 + (size_t)2 * NT * C4, pa - ys);
            ring_cp<C4>(s4 + (size_t)3 * NT * C4, pa + ys);
        }
        if constexpr (decltype(hx)::value) {
            ring_cp<C2>(s2, pa + hlo);
            ring_cp<C2>(s2 + (size_t)NT * C2, pa + hro);
        }
    };
    using BT = std::true_type;
    /* population b, b < Q: whether xi_x and xi_y are nonzero, and its stage */
    auto hxc = [](auto bc) { return std::bool_constant<gh_sign(N, decltype(bc)::value % N) != 0>{}; };
    auto hyc = [](auto bc) { return std::bool_constant<gh_sign(N, decltype(bc)::value / N) != 0>{}; };
    auto stc = [](auto bc) { return std::integral_constant<int, decltype(bc)::value % RS>{}; };
    /* populations 0 .. RS - 2 */
    [&]<int... B>(std::integer_sequence<int, B...>) {
        ((issue(B, hxc(std::integral_constant<int, B>{}), hyc(std::integral_constant<int, B>{}),
                stc(std::integral_constant<int, B>{})),
          ring_commit()),
         ...);
    }(std::make_integer_sequence<int, RS - 1>{});

    auto dec2 = [&](float2 raw, float2 winv2, int k) -> float2 {
        if constexpr (ST == 1) return fma2(raw, winv2, nrho02);
        else if constexpr (COL) return add2(raw, make_float2(dl[k + 2], dl[k + 3]));
        else return raw;
    };
    auto dec1 = [&](T raw, float winv, int i) -> float {
        if constexpr (COL) return decode_col<ST>(raw, winv, rho0, dl[i]);
        else return decode<ST>(raw, winv, rho0);
    };

    /* 1. moments of the level read, carried from the step that wrote it: per node the
     * sums sum w d, sum w xi_x d, sum w xi_y d of the stored deviations, in population
     * order (aux_in, [3][ny][pitch]; loaded before the ring's first copies are waited
     * for) */
    const size_t ap = (size_t)pitch * p.ny;
    const uint32_t m = (uint32_t)j * pitch + (uint32_t)x0;
    float2 rd[2], jx[2], jy[2];
    {
        const float *ain = static_cast<const float *>(p.aux_in);
        const float4 r4 = __ldcg(reinterpret_cast<const float4 *>(ain + m));
        const float4 x4 = __ldcg(reinterpret_cast<const float4 *>(ain + ap + m));
        const float4 y4 = __ldcg(reinterpret_cast<const float4 *>(ain + 2 * ap + m));
        rd[0] = make_float2(r4.x, r4.y);
        rd[1] = make_float2(r4.z, r4.w);
        jx[0] = make_float2(x4.x, x4.y);
        jx[1] = make_float2(x4.z, x4.w);
        jy[0] = make_float2(y4.x, y4.y);
        jy[1] = make_float2(y4.z, y4.w);
    }
    const PairNode nd = pair_node_state<FORCE>(p, rd, jx, jy);
    /* the same sums of the values this step stores */
#pragma unroll
    for (int h = 0; h < 2; ++h) rd[h] = jx[h] = jy[h] = f2(0.0f);

    /* 2. populations: a = iy N + ix in stage a % RS; population a + RS - 1 is copied */
    auto body = [&](int a, auto sxc, auto hyc, auto stc, int b, auto bhx, auto bhy, auto bst, bool more) {
        constexpr int SX = decltype(sxc)::value;
        constexpr bool HY = decltype(hyc)::value;
        constexpr int st = decltype(stc)::value;
        ring_wait<RS - 2>();
        const RingPop &rp = tp[a];
        T own_v[4], yv[3][4], hl[2], hr[2];
        const unsigned char *s4 = mine4 + st * STAGE;
        const unsigned char *s2 = mine2 + st * STAGE;
        ldn<4>(reinterpret_cast<const T *>(s4), own_v);
        if constexpr (HY) {
#pragma unroll
            for (int i = 0; i < 3; ++i) ldn<4>(reinterpret_cast<const T *>(s4 + (size_t)(1 + i) * NT * C4), yv[i]);
        }
        if constexpr (SX != 0) {
            ld2(reinterpret_cast<const T *>(s2), hl);
            ld2(reinterpret_cast<const T *>(s2 + (size_t)NT * C2), hr);
        }
        if (more) issue(b, bhx, bhy, bst);
        ring_commit();
        float2 v[2], c[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) v[h] = dec2(make_float2(to_r(own_v[2 * h]), to_r(own_v[2 * h + 1])), rp.winv2, 2 * h);
        /* collision and force */
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 eu;
            if constexpr (SX == 0 && !HY) eu = f2(0.0f);
            else if constexpr (SX == 0) eu = mul2(rp.cy2, nd.uy[h]);
            else if constexpr (!HY) eu = mul2(rp.cx2, nd.ux[h]);
            else eu = fma2(rp.cy2, nd.uy[h], mul2(rp.cx2, nd.ux[h]));
            const float2 t = fma2(mul2(f2(0.5f), eu), eu, eu);
            c[h] = fma2(nd.nom[h], v[h], fma2(nd.P[h], t, nd.B[h]));
            if constexpr (FORCE) c[h] = fma2(nd.dr[h], fma2(rp.gxi2, eu, rp.gxi2), c[h]);
        }
        /* x flux, upwind side by the sign of xi_x */
        if constexpr (SX != 0) {
            const float vv[4] = {v[0].x, v[0].y, v[1].x, v[1].y};
            const float winv = rp.winv2.x;
            const float l0 = dec1(hl[0], winv, 0), l1 = dec1(hl[1], winv, 1);
            const float r0 = dec1(hr[0], winv, 6), r1 = dec1(hr[1], winv, 7);
            const float kx = rp.kx;
            float Dx[4];
            if constexpr (SX > 0) {
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
                for (int k = 0; k < 4; ++k) Dx[k] = fmaf(kx, m[k + 1] - m[k], d[k + 1]);
                (void)r1;
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
                for (int k = 0; k < 4; ++k) Dx[k] = fmaf(-kx, m[k + 1] - m[k], e[k + 1]);
                (void)l0;
            }
            c[0] = fma2(rp.ncx2, make_float2(Dx[0], Dx[1]), c[0]);
            c[1] = fma2(rp.ncx2, make_float2(Dx[2], Dx[3]), c[1]);
        }
        /* y flux on the sign-reflected window (rows j - 2s, j - s, j, j + s) */
        if constexpr (HY) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 w0 = dec2(make_float2(to_r(yv[0][2 * h]), to_r(yv[0][2 * h + 1])), rp.winv2, 2 * h);
                const float2 w1 = dec2(make_float2(to_r(yv[1][2 * h]), to_r(yv[1][2 * h + 1])), rp.winv2, 2 * h);
                const float2 w3 = dec2(make_float2(to_r(yv[2][2 * h]), to_r(yv[2][2 * h + 1])), rp.winv2, 2 * h);
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
                const float2 Dy = fma2(rp.ky2, sub2(mb, ma), d1);
                c[h] = fma2(rp.nacy2, Dy, c[h]);
            }
        }
        float2 dn[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) dn[h] = add2(v[h], c[h]);
        /* carried moments: the deviations as stored (what the next step would read) */
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 ds;
            if constexpr (ST == 1) ds = fma2(mul2(rp.w2, add2(f2(rho0), dn[h])), rp.winv2, nrho02);
            else if constexpr (COL) {
                const float2 dc = make_float2(dl[2 * h + 2], dl[2 * h + 3]);
                ds = add2(pair_round<ST>(sub2(dn[h], dc)), dc);
            } else ds = pair_round<ST>(dn[h]);
            rd[h] = fma2(rp.w2, ds, rd[h]);
            jx[h] = fma2(rp.wcx2, ds, jx[h]);
            jy[h] = fma2(rp.wcy2, ds, jy[h]);
        }
        T *dst = fout + (uint32_t)a * plane + own;
        if constexpr (ROW) {
            /* wall row: the wall-bound populations' |xi.n| w d, summed in population order */
            const float xn = rp.cy2.x * wsgn;
            if (xn < 0.0f) {
                const float cw = -xn * rp.w2.x;
                float4 n = *numslot;
                n.x = fmaf(cw, dn[0].x, n.x);
                n.y = fmaf(cw, dn[0].y, n.y);
                n.z = fmaf(cw, dn[1].x, n.z);
                n.w = fmaf(cw, dn[1].y, n.w);
                *numslot = n;
            }
        }
        if (!EDGE || plain || img_dx != 0 || (noimg && allv)) {
            float2 e0, e1;
            if constexpr (ST == 1) {
                e0 = mul2(rp.w2, add2(f2(rho0), dn[0]));
                e1 = mul2(rp.w2, add2(f2(rho0), dn[1]));
            } else if constexpr (COL) {
                e0 = sub2(dn[0], make_float2(dl[2], dl[3]));
                e1 = sub2(dn[1], make_float2(dl[4], dl[5]));
            } else {
                e0 = dn[0];
                e1 = dn[1];
            }
            pair_st<ST>(dst, e0, e1);
            if (EDGE && img_dx != 0 && !noimg) pair_st<ST>(dst + img_dx, e0, e1);
        } else {
            const float dv[4] = {dn[0].x, dn[0].y, dn[1].x, dn[1].y};
            T *prow = dst - col;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!valid[k]) continue;
                T e;
                if constexpr (COL) e = encode_col<ST>(dv[k], rp.w2.x, rho0, dl[k + 2]);
                else e = encode<ST>(dv[k], rp.w2.x, rho0);
                put1(p, prow, x0 + k, e);
            }
        }
    };

    /* population A (compile-time): its sign pattern and stage, and the copy of A + RS - 1 */
    auto one = [&](int a, auto ac) {
        constexpr int A = decltype(ac)::value, B = A + RS - 1;
        using IB = std::integral_constant<int, (B < Q ? B : 0)>;
        body(a, std::integral_constant<int, gh_sign(N, A % N)>{}, hyc(ac), stc(ac), a + RS - 1, hxc(IB{}), hyc(IB{}),
             stc(std::integral_constant<int, B>{}), a + RS - 1 < Q);
    };
    if constexpr (N == 6) {
        /* D2Q36: a loop over blocks of P abscissa rows, P N populations each, so that every
         * population's stage is the same in each pass (P N a multiple of RS) */
        constexpr int P = (RS == 3) ? 1 : 2;
        static_assert((P * N) % RS == 0, "D2Q36 passes");
#pragma unroll 1
        for (int a0 = 0; a0 < Q; a0 += P * N) {
            [&]<int... I>(std::integer_sequence<int, I...>) {
                (one(a0 + I, std::integral_constant<int, I>{}), ...);
            }(std::make_integer_sequence<int, P * N>{});
        }
    } else {
        /* D2Q9 and D2Q16: fully unrolled */
        [&]<int... A>(std::integer_sequence<int, A...>) {
            (one(A, std::integral_constant<int, A>{}), ...);
        }(std::make_integer_sequence<int, Q>{});
    }
    ring_wait<0>();
    {
        float *aout = static_cast<float *>(p.aux_out);
        __stcg(reinterpret_cast<float4 *>(aout + m), make_float4(rd[0].x, rd[0].y, rd[1].x, rd[1].y));
        __stcg(reinterpret_cast<float4 *>(aout + ap + m), make_float4(jx[0].x, jx[0].y, jx[1].x, jx[1].y));
        __stcg(reinterpret_cast<float4 *>(aout + 2 * ap + m), make_float4(jy[0].x, jy[0].y, jy[1].x, jy[1].y));
    }
    if constexpr (ROW) {
        if (!MIX || rowk) ring_row_finish<ST, Q, S, QT, COL, MIX ? 4 : 1>(p, tab, x0, j, flags, wsgn, *numslot, dl, noimg);
    }
}

/* general units (boundary work, stochastic rounding): the body of layout 9, not inlined,
 * so that its register demand does not weigh on the lean bodies */
template <int ST, bool COL, bool FORCE>
__device__ __noinline__ void ring_general(const StepParams<float> &p, int s, uint8_t flags, int x0, int j, unsigned char *ring)
{
    const PairTables *tab = static_cast<const PairTables *>(p.ctab);
    const int q = p.set[s].q;
    if (q == 9) ring_cells<ST, 9, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring);
    else if (q == 16) ring_cells<ST, 16, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring);
    else ring_cells<ST, 36, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring);
}

__device__ __forceinline__ uint32_t ring_smid()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

/* Sets of D2Q9 (set 0) and Q1 = 16 or 36 populations (set 1). */
template <int ST, bool COL, bool FORCE, int Q1>
__global__ void __launch_bounds__(LB_BX *LB_BY, ring10_blocks<ST>())
    ring_unit_kernel(const __grid_constant__ StepParams<float> p, const __grid_constant__ RingTab tab,
                     const RowQueues rq)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    constexpr uint32_t EMPTY = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31u;
    const int nq = rq.nq;
    /* phase 0: this SM's queue; 1: the shared queue; 2: leftovers of every SM queue */
    int phase = 0;
    const int own = (int)(ring_smid() % (uint32_t)nq);
    for (;;) {
        uint32_t item = EMPTY;
        while (phase < 3) {
            int q = -1;
            if (phase == 0) {
                q = own;
            } else if (phase == 1) {
                q = nq;
            } else {
                /* lanes look at 32 queues at a time; the first with items left is tried */
                for (int base = 0; base < nq && q < 0; base += 32) {
                    const int qq = base + (int)lane;
                    const bool left = qq < nq && __ldcg(rq.ctr + qq) < (uint32_t)rq.desc[qq].y;
                    const uint32_t m = __ballot_sync(0xffffffffu, left);
                    if (m) q = base + __ffs(m) - 1;
                }
                if (q < 0) {
                    phase = 3;
                    break;
                }
            }
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(rq.ctr + q, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            const int2 d = rq.desc[q];
            if (t < (uint32_t)d.y) {
                item = rq.rows[d.x + t];
                break;
            }
            if (phase < 2) ++phase;   /* this queue is used up (phase 2 looks again) */
        }
        if (item == EMPTY) break;
        const int tx = (int)(item & 0x3fffu), j = (int)(item >> 16);
        const uint32_t kind = (item >> 14) & 3u;
        const uint8_t flags = p.tmap[(size_t)j * p.ntx + tx];
        const int s = flags & LB_TILE_HIGH;
        const int x0 = tx * LB_TILE_X + (int)lane * 4;
        if (kind == RING_LEAN) {
            if (s == 0) ring_lean<ST, 9, 0, Q1, COL, FORCE, RING_LEAN>(p, tab, x0, j, flags, ring_smem);
            else ring_lean<ST, Q1, 1, 9, COL, FORCE, RING_LEAN>(p, tab, x0, j, flags, ring_smem);
        } else if (kind == RING_ROW) {
            if (s == 0) ring_lean<ST, 9, 0, Q1, COL, FORCE, RING_ROW>(p, tab, x0, j, flags, ring_smem);
            else ring_lean<ST, Q1, 1, 9, COL, FORCE, RING_ROW>(p, tab, x0, j, flags, ring_smem);
        } else if (x0 < p.nx) {
            if (kind == RING_GENERAL) ring_general<ST, COL, FORCE>(p, s, flags, x0, j, ring_smem);
            else if (s == 0) ring_lean<ST, 9, 0, Q1, COL, FORCE, RING_EDGE>(p, tab, x0, j, flags, ring_smem);
            else ring_lean<ST, Q1, 1, 9, COL, FORCE, RING_EDGE>(p, tab, x0, j, flags, ring_smem);
        }
        __syncwarp();
        /* the pressure columns of this row: the pressure pass's work, done here once the
         * row's nodes are stored (the warp barrier above makes them visible to all lanes);
         * lattices with a body force keep the pressure pass (its registers would weigh on
         * the force kernels) */
        if constexpr (!FORCE) {
            if (tx == 0 && p.pressure[0]) pressure_row<ST>(p, j, 0);
            if (tx == p.ntx - 1 && p.pressure[1]) pressure_row<ST>(p, j, 1);
        }
    }
    /* the last warp out zeroes the counters for the next launch */
    uint32_t done = 0;
    if (lane == 0) {
        __threadfence();
        done = atomicAdd(rq.ctr + nq + 1, 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done == gridDim.x * (blockDim.x >> 5) - 1u) {
        for (int k = (int)lane; k <= nq + 1; k += 32) rq.ctr[k] = 0u;
        __threadfence();
    }
}

template <int ST, bool COL, bool FORCE, int Q1>
void ring_unit_launch(const StepParams<float> &p, const RingTab &tab, const RowQueues &rq, int nblocks,
                      cudaStream_t st)
{
    constexpr size_t smem = ring_unit_smem_bytes<ST>();
    /* per device: the raised shared-memory limit and the resident blocks of the GPU */
    static std::atomic<int> resident[64];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    int nb = resident[dev].load();
    if (nb == 0) {
        auto kern = ring_unit_kernel<ST, COL, FORCE, Q1>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LB_BX * LB_BY, smem);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        nb = std::max(1, per_sm) * std::max(1, nsm);
        resident[dev].store(nb);
    }
    const int grid = std::min(nb, nblocks);
    if (grid <= 0) return;
    ring_unit_kernel<ST, COL, FORCE, Q1><<<grid, LB_BX * LB_BY, smem, st>>>(p, tab, rq);
}

/* ------------------------------------------------------------------------------
 * Batched lattices on layout 10's bodies. A block takes a lattice from the queue (most
 * work first), copies its two launch parameter sets (level n -> n+1 and back) and its
 * constants table into shared memory after its ring, and advances it nsteps steps with a
 * block barrier between steps. Within a step the block's warps take the lattice's items
 * (host-built, longest first): up to 32 quads of rows of one set and kind, lane l on quad
 * l % qpr of the item's row l / qpr (qpr quads per row). Rows without walls, ghost-row
 * copies or shadows run the edge body (its stores do the periodic ghost columns), the
 * others the row body (its epilogue does them), or layout 9's body where a row ends inside
 * a quad: the same bits as layout 9 stepping each lattice alone. The rows of a row-body
 * item need not be adjacent (a lattice's wall rows of one set share one item, its shadow
 * rows another: a lane's time is its population chain, whatever the number of rows).
 * Item: two words, the index in `items` of its row list (one word per row) and
 * (rows - 1) | set << 5 | kind << 6 (0 edge, 1 row, 2 general).
 * ---------------------------------------------------------------------------- */
constexpr size_t ring_batch_params_bytes() { return (2 * sizeof(StepParams<float>) + 15) / 16 * 16; }
template <int ST>
__host__ __device__ constexpr size_t ring_batch_smem_bytes()
{
    return ring_unit_smem_bytes<ST>() + ring_batch_params_bytes() + sizeof(RingTab);
}

/* Two blocks of 128 registers per SM for every storage: the batch's mixed body spills
 * heavily under the 80 registers of three 16-bit blocks (BF16, 512 channels: 6970 MLUPS
 * with two blocks against 5320 with three) */
template <int ST, bool FORCE, int Q1>
__global__ void __launch_bounds__(LB_BX *LB_BY, 2)
    ring_batch_kernel(const StepParams<float> *__restrict__ params, const RingTab *__restrict__ tabs,
                      const uint32_t *__restrict__ items, const int2 *__restrict__ ranges,
                      const int *__restrict__ order, int n, int nsteps, int base, int advance, unsigned int *queue)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    static_assert(ring_unit_smem_bytes<ST>() % 16 == 0 && sizeof(RingTab) % 16 == 0 && sizeof(StepParams<float>) % 4 == 0,
                  "aligned copies");
    StepParams<float> *sp = reinterpret_cast<StepParams<float> *>(ring_smem + ring_unit_smem_bytes<ST>());
    RingTab *tab = reinterpret_cast<RingTab *>(ring_smem + ring_unit_smem_bytes<ST>() + ring_batch_params_bytes());
    __shared__ int inst_sh;
    __shared__ unsigned int icount;
    const uint32_t lane = threadIdx.x & 31u;
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
            for (int k = threadIdx.x; k < (int)(2 * sizeof(StepParams<float>) / 4); k += blockDim.x) dst[k] = src[k];
            const uint4 *ts = reinterpret_cast<const uint4 *>(tabs + inst);
            uint4 *td = reinterpret_cast<uint4 *>(tab);
            for (int k = threadIdx.x; k < (int)(sizeof(RingTab) / 16); k += blockDim.x) td[k] = ts[k];
        }
        const int2 rg = ranges[inst];
        for (int st = 0; st < nsteps; ++st) {
            if (threadIdx.x == 0) icount = 0u;
            __syncthreads();   /* parameters in place; the previous step done by every warp */
            const StepParams<float> &p = sp[advance ? ((base + st) & 1) : base];
            const int qpr = (p.nx + 3) / 4;
            /* x-periodic lattices of whole quads: halos read inside the row, ghost-column
             * images written by the launch's last step only */
            const int xm = (p.periodic_x && (p.nx & 3) == 0) ? (st + 1 < nsteps ? 3 : 1) : 0;
            for (;;) {
                unsigned it = 0;
                if (lane == 0) it = atomicAdd(&icount, 1u);
                it = __shfl_sync(0xffffffffu, it, 0);
                if (it >= (unsigned)rg.y) break;
                const uint2 w = reinterpret_cast<const uint2 *>(items)[rg.x + it];
                const int nr = (int)(w.y & 31u) + 1, s = (int)((w.y >> 5) & 1u);
                const int r = (int)lane / qpr, x0 = ((int)lane - r * qpr) * 4;
                if (r < nr && x0 < p.nx) {
                    const int j = (int)items[w.x + (uint32_t)r];
                    const uint8_t flags = p.tmap[(size_t)j * p.ntx + x0 / LB_TILE_X];
                    const uint32_t kind = (w.y >> 6) & 3u;
                    if (xm == 3) {
                        if (s == 0) ring_lean<ST, 9, 0, Q1, false, FORCE, RING_BATCH>(p, *tab, x0, j, flags, ring_smem, xm, kind == 1u);
                        else ring_lean<ST, Q1, 1, 9, false, FORCE, RING_BATCH>(p, *tab, x0, j, flags, ring_smem, xm, kind == 1u);
                    } else if (kind == 2u) ring_general<ST, false, FORCE>(p, s, flags, x0, j, ring_smem);
                    else if (kind == 1u && s == 0) ring_lean<ST, 9, 0, Q1, false, FORCE, RING_ROW>(p, *tab, x0, j, flags, ring_smem, xm);
                    else if (kind == 1u) ring_lean<ST, Q1, 1, 9, false, FORCE, RING_ROW>(p, *tab, x0, j, flags, ring_smem, xm);
                    else if (s == 0) ring_lean<ST, 9, 0, Q1, false, FORCE, RING_EDGE>(p, *tab, x0, j, flags, ring_smem, xm);
                    else ring_lean<ST, Q1, 1, 9, false, FORCE, RING_EDGE>(p, *tab, x0, j, flags, ring_smem, xm);
                }
                __syncwarp();
            }
            __syncthreads();   /* the step is complete for the whole lattice */
        }
    }
}

/* force: some lattice of the batch has a body force (the force terms then run for every
 * lattice; with g = 0 they add exact zeros). grid 0: the resident blocks of the device
 * are returned in *grid_out and nothing is launched. */
template <int ST, int Q1>
int launch_ring_batch_store(const StepParams<float> *params, const RingTab *tabs, const uint32_t *items,
                            const int2 *ranges, const int *order, int n, int nsteps, int base, int advance,
                            unsigned int *queue, bool force, int grid, int *grid_out, void *stream)
{
    constexpr size_t smem = ring_batch_smem_bytes<ST>();
    auto kern = force ? ring_batch_kernel<ST, true, Q1> : ring_batch_kernel<ST, false, Q1>;
    if (grid < 1) {
        cudaFuncSetAttribute(ring_batch_kernel<ST, true, Q1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(ring_batch_kernel<ST, false, Q1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0, dev = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LB_BX * LB_BY, smem) != cudaSuccess ||
            cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        *grid_out = per_sm * nsm;
        return per_sm > 0 ? 0 : -1;
    }
    kern<<<grid, LB_BX * LB_BY, smem, static_cast<cudaStream_t>(stream)>>>(params, tabs, items, ranges, order, n,
                                                                        nsteps, base, advance, queue);
    return 0;
}

/* layout 10 for one storage format and high-order set size */
template <int ST, int Q1>
void launch_ring_units_store(const StepParams<float> &p, const RingTab &tab, const RowQueues &rq, int nblocks,
                             void *stream)
{
    static_assert(ST >= 1 && ST <= 4, "paired FP32 arithmetic: FP32 and 16-bit storage");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if constexpr (Store<ST>::dev) {
        if (p.dcol) {
            if (p.has_force) ring_unit_launch<ST, true, true, Q1>(p, tab, rq, nblocks, st);
            else ring_unit_launch<ST, true, false, Q1>(p, tab, rq, nblocks, st);
            return;
        }
    }
    if (p.has_force) ring_unit_launch<ST, false, true, Q1>(p, tab, rq, nblocks, st);
    else ring_unit_launch<ST, false, false, Q1>(p, tab, rq, nblocks, st);
}

}  // namespace lbk
