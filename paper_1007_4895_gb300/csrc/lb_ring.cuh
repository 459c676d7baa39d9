/*
 * lb_ring.cuh -- the fused time step with paired FP32 arithmetic fed by a per-thread ring
 * of asynchronous copies (layout 9).
 *
 * The arithmetic of layout 7 (lb_pair.cuh: node pairs in packed two-wide FP32, the
 * folded collision, the clamp-form y limiter on the sign-reflected window), with the
 * same threads and blocks (one quad of nodes of one row per thread, blocks of one
 * 128-column tile x 8 rows), but the stencil of each population reaches the thread
 * through shared memory:
 *   - every thread owns RING_STAGES slots of shared memory, each holding one
 *     population's stencil of its quad (its own four values, the three y window rows,
 *     the two x halos); it copies the stencil of population a + RING_STAGES - 1 into a
 *     slot with cp.async while it computes population a from another. The copies hold
 *     no registers while in flight, so the thread keeps two populations ahead without
 *     the register cost of a prefetch buffer, and no thread waits on another (no block
 *     barrier): each reads only the slots it filled.
 *   - the boundary work of a row is done by the row's own threads, in the same kernel:
 *     ghost-row copies with every store of a wall row or a periodic-y edge row, the
 *     diffuse-wall overwrite of Sec. 3.2 after the population loop (rho_W from the
 *     streamed wall-bound populations, summed as they are stored), and the mode-B
 *     rebuild of Sec. 2.2 (second-order Hermite coefficients of the final populations,
 *     read back) for shadow tiles. Pressure columns, ragged edges and periodic ghost
 *     columns are handled per lane in the store; pressure columns are then set by the
 *     pressure pass and mode-A interface rows by the interface pass, as in every layout.
 * FP32 and 16-bit storage. Results agree with layout 0 to rounding, not bit for bit.
 */
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "lb_pair.cuh"

namespace lbk {

#define RING_STAGES 3
#ifndef RING_MIN_BLOCKS
#define RING_MIN_BLOCKS 3
#endif
#ifndef RING_MOM_UNROLL
#define RING_MOM_UNROLL 6
#endif
constexpr int kRingMomUnroll = RING_MOM_UNROLL;

/* bytes of one stage of the ring of a block: per thread, four 4-element chunks (its own
 * values and the three window rows) and two 2-element chunks (the x halos), stored as
 * structure of arrays so that a warp's reads of one chunk are contiguous */
template <int ST>
__host__ __device__ constexpr size_t ring_stage_bytes()
{
    return (size_t)LB_BX * LB_BY * (4 * 4 + 2 * 2) * sizeof(typename Store<ST>::T);
}
template <int ST>
__host__ __device__ constexpr size_t ring_smem_bytes()
{
    return RING_STAGES * ring_stage_bytes<ST>();
}

template <int N>
__device__ __forceinline__ void ring_cp(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem), "n"(N)
                 : "memory");
}
__device__ __forceinline__ void ring_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ring_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

/* Sec. 3.2, diffuse wall: f = rho_W S(u_W) for the gas-bound populations of a wall-row
 * quad (set s, wall 0 bottom / 1 top, nsgn = +1 / -1), with zero net mass flux through
 * the wall node; num[k] = sum over the wall-bound populations of |xi.n| w d. store(dst,
 * -1, dv, w) writes four deviations rounded to nearest, with the row's ghost copies. */
template <int Q, typename T, typename STORE>
__device__ __forceinline__ void ring_wall_fill(const StepParams<float> &p, int s, int wall, float nsgn,
                                               const float (&num)[4], T *fout, uint32_t own, const STORE &store)
{
    const SetConst<float> &c = p.set[s];
    const float rho0 = p.rho0;
    const uint32_t plane = (uint32_t)p.plane;
    const float uwx = p.uw_x[wall], uwy = p.uw_y[wall];
    const float usw = uwx * uwx + uwy * uwy;
    const float kd = p.kdiff[s][wall], kout = p.kout[s][wall];
    float rwd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rwd[k] = fmaf(rho0, kd, num[k]) / kout;   /* rho_W - rho0 */
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        if (c.cy[a] * nsgn <= 0.0f) continue;
        const float ew = c.cx[a] * uwx + c.cy[a] * uwy;
        const float sm1 = ew + 0.5f * (ew * ew - usw);    /* S / w - 1 */
        float dv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dv[k] = fmaf(rwd[k] + rho0, sm1, rwd[k]);
        store(fout + (uint32_t)a * plane + own, -1, dv, c.w[a]);
    }
}

/* Sec. 2.2, mode B: the quad x0 .. x0 + 3 of row j (set s, final populations already
 * stored) rebuilt in the other set from its second-order Hermite coefficients, with the
 * row's ghost copies (nimg rows at offsets img) and per-node stores where not plain. */
template <int ST, int Q, bool COL>
__device__ __forceinline__ void ring_shadow(const StepParams<float> &p, int s, int x0, int j, const bool (&valid)[4],
                                            bool plain, int nimg, const int (&img)[2], const float (&dl)[8])
{
    using T = typename Store<ST>::T;
    const SetConst<float> &c = p.set[s];
    const int t = 1 - s;
    const SetConst<float> &ct = p.set[t];
    const float rho0 = p.rho0;
    const uint32_t plane = (uint32_t)p.plane, pitch = (uint32_t)p.pitch;
    const uint32_t col = (uint32_t)(x0 + LB_GHOST);
    const uint32_t own = (uint32_t)j * pitch + col;
    const T *fown = static_cast<const T *>(p.fout[s]);
    float h[4][6];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int m = 0; m < 6; ++m) h[k][m] = 0.0f;
#pragma unroll 9
    for (int a = 0; a < Q; ++a) {
        T raw[4];
        ldn<4>(fown + (uint32_t)a * plane + own, raw);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!valid[k]) continue;
            float d;
            if constexpr (COL) d = decode_col<ST>(raw[k], c.winv[a], rho0, dl[k + 2]);
            else d = decode<ST>(raw[k], c.winv[a], rho0);
            hermite_acc(c, a, d, h[k]);
        }
    }
    T *ftd = static_cast<T *>(p.fout[t]);
#pragma unroll 4
    for (int b = 0; b < ct.q; ++b) {
        T *prow = ftd + (size_t)b * p.plane + (size_t)j * pitch;
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float v = hermite_rebuild(ct, b, h[k]);
            if constexpr (COL) e[k] = encode_col<ST>(v, ct.w[b], rho0, dl[k + 2]);
            else e[k] = encode<ST>(v, ct.w[b], rho0);
        }
        if (plain) {
            st4(prow + col, e);
            for (int m = 0; m < nimg; ++m) st4(prow + (ptrdiff_t)img[m] * (ptrdiff_t)pitch + col, e);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[k]) put1r(p, prow, x0 + k, j, e[k]);
        }
    }
}

template <int ST, int Q, bool COL, bool FORCE>
__device__ __forceinline__ void ring_cells(const StepParams<float> &p, int s, uint8_t flags, int x0, int j,
                                           const PairC *pcs, const PairC2 *pcs2, const MomC2 *mcs,
                                           unsigned char *ring)
{
    using T = typename Store<ST>::T;
    constexpr int NT = LB_BX * LB_BY;
    constexpr int C4 = 4 * (int)sizeof(T), C2 = 2 * (int)sizeof(T);
    constexpr size_t STAGE = ring_stage_bytes<ST>();
    const int tid = threadIdx.y * LB_BX + threadIdx.x;
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]);
    T *__restrict__ fout = static_cast<T *>(p.fout[s]);
    const uint32_t plane = (uint32_t)p.plane, pitch = (uint32_t)p.pitch;
    const uint32_t col = (uint32_t)(x0 + LB_GHOST);
    const uint32_t own = (uint32_t)j * pitch + col;
    const float rho0 = p.rho0;
    const float2 nrho02 = f2(-rho0);
    /* slot addresses of this thread: own values, window rows 0..2, left / right halo */
    auto sl = [&](int st, int chunk) -> unsigned char * {
        unsigned char *base = ring + (size_t)st * STAGE;
        return chunk < 4 ? base + ((size_t)chunk * NT + tid) * C4 : base + (size_t)4 * NT * C4 + ((size_t)(chunk - 4) * NT + tid) * C2;
    };
    /* the window rows j - 2s, j - s, j + s (s = +-1 by the sign of xi_y) lie within the two
     * ghost rows beyond every edge row, which hold the wall row (or the periodic image) */
    auto issue = [&](int a) {
        if (a < Q) {
            const PairC &pc = pcs[a];
            const int st = a % RING_STAGES;
            const T *pa = fin + (uint32_t)a * plane + own;
            ring_cp<C4>(sl(st, 0), pa);
            if (pc.ystep != 0) {
                ring_cp<C4>(sl(st, 1), pa - 2 * pc.ystep);
                ring_cp<C4>(sl(st, 2), pa - pc.ystep);
                ring_cp<C4>(sl(st, 3), pa + pc.ystep);
            }
            if (pc.crx != 0.0f) {
                ring_cp<C2>(sl(st, 4), pa - 2);
                ring_cp<C2>(sl(st, 5), pa + 4);
            }
        }
        ring_commit();
    };
#pragma unroll
    for (int a = 0; a < RING_STAGES - 1; ++a) issue(a);

    /* per-column reference density: delta at columns x0 - 2 .. x0 + 5 */
    float dl[8];
    if constexpr (COL) {
#pragma unroll
        for (int i = 0; i < 8; ++i) dl[i] = p.dcol[col - 2 + i];
    }
    auto dec2 = [&](float2 raw, float2 winv2, int k) -> float2 {
        if constexpr (ST == 1) return fma2(raw, winv2, nrho02);
        else if constexpr (COL) return add2(raw, make_float2(dl[k + 2], dl[k + 3]));
        else return raw;
    };
    auto dec1 = [&](T raw, float winv, int i) -> float {
        if constexpr (COL) return decode_col<ST>(raw, winv, rho0, dl[i]);
        else return decode<ST>(raw, winv, rho0);
    };

    /* 1. moments (loads of several populations in flight) */
    float2 rd[2] = {f2(0.0f), f2(0.0f)}, jx[2] = {f2(0.0f), f2(0.0f)}, jy[2] = {f2(0.0f), f2(0.0f)};
#pragma unroll kRingMomUnroll
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
    const PairNode nd = pair_node_state<FORCE>(p, rd, jx, jy);

    /* 2. the row's boundary work and the lane's stores */
    int wall = -1;
    if (j == 0 && p.wall_diffuse[0]) wall = 0;
    if (j == p.ny - 1 && p.wall_diffuse[1]) wall = 1;
    const float nsgn = wall == 0 ? 1.0f : -1.0f;
    int img[2] = {0, 0};
    const int nimg = row_images(p, j, img);
    bool valid[4];
    bool plain = !(p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        valid[k] = x0 + k < p.nx && !is_pressure_node(p, x0 + k, j);
        plain = plain && valid[k];
    }
    const bool fast = plain && nimg == 0 && !p.sr;
    /* four deviations of population a (a < 0: a value set by the wall, rounded to
     * nearest) to storage, with the ghost-row images of the row */
    auto store = [&](T *dst, int a, const float (&dv)[4], float w) {
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (a >= 0 && p.sr) {
                const uint32_t bits = sr_bits(x0 + k, j, p.nx, a, p.step_key);
                if constexpr (COL) e[k] = encode_sr<ST>(dv[k] - dl[k + 2], w, rho0, bits);
                else e[k] = encode_sr<ST>(dv[k], w, rho0, bits);
            } else {
                if constexpr (COL) e[k] = encode_col<ST>(dv[k], w, rho0, dl[k + 2]);
                else e[k] = encode<ST>(dv[k], w, rho0);
            }
        }
        for (int t = -1; t < nimg; ++t) {
            T *d = t < 0 ? dst : dst + (ptrdiff_t)(t == 0 ? img[0] : img[1]) * (ptrdiff_t)pitch;
            if (plain) {
                st4(d, e);
            } else {
                T *prow = d - col;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (valid[k]) put1(p, prow, x0 + k, e[k]);
            }
        }
    };

    /* 3. population loop: population a from its slot, a + RING_STAGES - 1 copied */
    float num[4] = {0.0f, 0.0f, 0.0f, 0.0f};   /* wall row: sum over wall-bound |xi.n| w f */
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        ring_wait<RING_STAGES - 2>();   /* this thread's copies of population a have landed */
        const int st = a % RING_STAGES;
        const PairC pc = pcs[a];
        const PairC2 pc2 = pcs2[a];
        T own_v[4];
        ldn<4>(reinterpret_cast<const T *>(sl(st, 0)), own_v);
        T yv[3][4], hl[2], hr[2];
        if (pc.ystep != 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) ldn<4>(reinterpret_cast<const T *>(sl(st, 1 + i)), yv[i]);
        }
        if (pc.crx != 0.0f) {
            ld2(reinterpret_cast<const T *>(sl(st, 4)), hl);
            ld2(reinterpret_cast<const T *>(sl(st, 5)), hr);
        }
        issue(a + RING_STAGES - 1);
        float2 v[2], c[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) v[h] = dec2(make_float2(to_r(own_v[2 * h]), to_r(own_v[2 * h + 1])), pc2.winv2, 2 * h);
        auto xh = [&](int i) -> float { return i < 2 ? dec1(hl[i], pc2.winv2.x, i) : dec1(hr[i - 2], pc2.winv2.x, i + 4); };
        auto yw = [&](int h, int i) -> float2 {
            return dec2(make_float2(to_r(yv[i][2 * h]), to_r(yv[i][2 * h + 1])), pc2.winv2, 2 * h);
        };
        pair_increment<FORCE>(pc, pc2, nd, v, xh, yw, c);
        float2 dn[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) dn[h] = add2(v[h], c[h]);
        T *dst = fout + (uint32_t)a * plane + own;
        if (fast) {
            if constexpr (ST == 1) {
                pair_st<ST>(dst, mul2(pc2.w2, add2(f2(rho0), dn[0])), mul2(pc2.w2, add2(f2(rho0), dn[1])));
            } else if constexpr (COL) {
                pair_st<ST>(dst, sub2(dn[0], make_float2(dl[2], dl[3])), sub2(dn[1], make_float2(dl[4], dl[5])));
            } else {
                pair_st<ST>(dst, dn[0], dn[1]);
            }
            continue;
        }
        const float dv[4] = {dn[0].x, dn[0].y, dn[1].x, dn[1].y};
        if (wall >= 0) {
            const float xn = pc.cy2.x * nsgn;
            if (xn > 0.0f) continue;   /* gas-bound: replaced below */
            if (xn < 0.0f) {
#pragma unroll
                for (int k = 0; k < 4; ++k) num[k] = fmaf(-xn * pc2.w2.x, dv[k], num[k]);
            }
        }
        store(dst, a, dv, pc2.w2.x);
    }
    ring_wait<0>();

    /* 4. diffuse wall, 5. mode-B rebuild */
    if (wall >= 0) ring_wall_fill<Q>(p, s, wall, nsgn, num, fout, own, store);
    if (flags & LB_TILE_SHADOW) ring_shadow<ST, Q, COL>(p, s, x0, j, valid, plain, nimg, img, dl);
}

template <int ST, bool COL, bool FORCE>
__global__ void __launch_bounds__(LB_BX *LB_BY, RING_MIN_BLOCKS) ring_kernel(const __grid_constant__ StepParams<float> p)
{
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const PairTables *tab = static_cast<const PairTables *>(p.ctab);
    int bx = blockIdx.x, by = blockIdx.y;
    if (p.block_order) {
        const int b = p.block_order[blockIdx.x];
        bx = b % p.ntx;
        by = b / p.ntx;
    }
    const int j = by * LB_BY + threadIdx.y;
    const int x0 = (bx * LB_BX + threadIdx.x) * 4;
    if (j >= p.ny || x0 >= p.nx) return;   /* no block barrier follows */
    const uint8_t flags = p.tmap[(size_t)j * p.ntx + (x0 / LB_TILE_X)];
    if (flags & LB_TILE_IFACE) return;    /* mode A interface rows: set by iface_kernel */
    const int s = flags & LB_TILE_HIGH;
    const int q = p.set[s].q;
    if (q == 9) ring_cells<ST, 9, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring_smem);
    else if (q == 16) ring_cells<ST, 16, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring_smem);
    else ring_cells<ST, 36, COL, FORCE>(p, s, flags, x0, j, tab->pp[s], tab->pp2[s], tab->pm[s], ring_smem);
}

template <int ST, bool COL, bool FORCE>
void ring_launch(const StepParams<float> &p, dim3 grid, cudaStream_t st)
{
    constexpr size_t smem = ring_smem_bytes<ST>();
    /* the dynamic shared-memory limit is raised once per instantiation and device */
    static std::atomic<uint64_t> raised{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(raised.load() & bit)) {
        cudaFuncSetAttribute(ring_kernel<ST, COL, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        raised.fetch_or(bit);
    }
    ring_kernel<ST, COL, FORCE><<<grid, dim3(LB_BX, LB_BY), smem, st>>>(p);
}

template <int ST>
void launch_ring_store(const StepParams<float> &p, void *stream)
{
    static_assert(ST >= 1 && ST <= 4, "paired FP32 arithmetic: FP32 and 16-bit storage");
    dim3 grid((p.nx + 4 * LB_BX - 1) / (4 * LB_BX), (p.ny + LB_BY - 1) / LB_BY);
    if (p.block_order) grid = dim3(grid.x * grid.y, 1);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if constexpr (Store<ST>::dev) {
        if (p.dcol) {
            if (p.has_force) ring_launch<ST, true, true>(p, grid, st);
            else ring_launch<ST, true, false>(p, grid, st);
            return;
        }
    }
    if (p.has_force) ring_launch<ST, false, true>(p, grid, st);
    else ring_launch<ST, false, false>(p, grid, st);
}

}  // namespace lbk
