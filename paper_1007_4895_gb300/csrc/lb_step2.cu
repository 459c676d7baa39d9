/*
 * lb_step2.cu -- the fused time step, register-window form.
 *
 * Same arithmetic as the Sec. 3.1 / 3.2 / 2.2 update described in lb_step.cu; what
 * changes is how the work is laid out on the GPU:
 *   - a warp covers one 128-column tile (4 nodes per lane, one 16-byte vector per
 *     plane row in FP32) and RB consecutive rows; warps of a block are stacked in y,
 *     so the rows a warp reads above and below its own are mostly rows its neighbours
 *     just read (L1 hits);
 *   - pass 1 sums density and momentum of the 4 x RB nodes over all populations of
 *     their set and keeps (rho, u, omega) in registers;
 *   - pass 2 loops over the populations; for each it loads the RB + 4 rows of the
 *     column strip the stencil needs into registers, walks down the rows reusing the
 *     limited y-slope of the shared face, takes the x neighbours from two 2-element
 *     vectors beside the thread's own, and writes the new value;
 *   - diffuse-wall rows, mode-B interface views and masked columns are handled as in
 *     the one-row form.
 * Rows of the two sets inside one RB block are processed set by set; the neighbours of
 * a row are always read from the planes of its own set (which hold the other set's
 * nodes rebuilt next to an interface).
 */
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_common.cuh"

namespace lbk {

#define LB2_WY 4   /* warps per block, stacked in y */

template <int ST, int Q, int RB>
__device__ __forceinline__ void pass_set(const StepParams<typename Store<ST>::R> &p, int s, int x0, int j0,
                                         const uint8_t (&flags)[RB], const bool (&valid)[RB][4],
                                         const bool (&full)[RB])
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const SetConst<R> &c = p.set[s];
    const size_t plane = (size_t)p.ny * p.pitch;
    const T *__restrict__ fin = static_cast<const T *>(p.fin[s]) + (size_t)j0 * p.pitch + (x0 + LB_GHOST);
    T *__restrict__ fout = static_cast<T *>(p.fout[s]) + (size_t)j0 * p.pitch + (x0 + LB_GHOST);
    const R rho0 = p.rho0;

    /* rows of this set that this pass updates */
    bool mine[RB];
    bool any = false;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        mine[r] = (j0 + r < p.ny) && ((flags[r] & LB_TILE_HIGH) == s) && !(flags[r] & LB_TILE_IFACE);
        any = any || mine[r];
    }
    if (!any) return;

    /* offsets of window rows j0-2 .. j0+RB+1 relative to row j0 (ghost / periodic rows) */
    ptrdiff_t roff[RB + 4];
#pragma unroll
    for (int k = 0; k < RB + 4; ++k) {
        /* ghost rows = wall row (Sec. 3.2) or periodic images; rows past the end of a
         * partial block are clamped too (they feed no stored value) */
        int j = j0 - 2 + k;
        if (p.periodic_y) j = ((j % p.ny) + p.ny) % p.ny;
        else j = j < 0 ? 0 : (j > p.ny - 1 ? p.ny - 1 : j);
        roff[k] = (ptrdiff_t)(j - j0) * p.pitch;
    }

    /* pass 1: moments */
    R rhod[RB][4], ux[RB][4], uy[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) rhod[r][k] = ux[r][k] = uy[r][k] = R(0);
#pragma unroll 2
    for (int a = 0; a < Q; ++a) {
        const T *pa = fin + a * plane;
        const R w = c.w[a], wx = c.wcx[a], wy = c.wcy[a], winv = c.winv[a];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            if (!mine[r]) continue;
            T raw[4];
            ld4(pa + roff[r + 2], raw);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const R d = decode<ST>(raw[k], winv, rho0);
                rhod[r][k] = fma(w, d, rhod[r][k]);
                ux[r][k] = fma(wx, d, ux[r][k]);
                uy[r][k] = fma(wy, d, uy[r][k]);
            }
        }
    }
    /* per node: A = (rho - rho0) - rho u^2 / 2, rho, u, omega (so f_eq / w - rho0 =
     * A + rho eu (1 + eu / 2) with eu = xi.u) */
    R A[RB][4], rho[RB][4], om[RB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            rho[r][k] = rho0 + rhod[r][k];
            const R inv = R(1) / rho[r][k];
            ux[r][k] *= inv;
            uy[r][k] *= inv;
            const R usq = ux[r][k] * ux[r][k] + uy[r][k] * uy[r][k];
            A[r][k] = fma(R(-0.5) * rho[r][k], usq, rhod[r][k]);
            om[r][k] = p.dt / tau_of(p, rho[r][k]);
        }

    /* wall rows inside this block */
    int wall_r = -1, wall = -1;
    if (p.wall_diffuse[0] && j0 == 0 && mine[0]) { wall_r = 0; wall = 0; }
#pragma unroll
    for (int r = 0; r < RB; ++r)
        if (p.wall_diffuse[1] && j0 + r == p.ny - 1 && mine[r]) { wall_r = r; wall = 1; }
    const R nsgn = wall == 0 ? R(1) : R(-1);
    R num[4] = {R(0), R(0), R(0), R(0)};
    const bool edge = p.periodic_x && (x0 < LB_GHOST || x0 + 3 >= p.nx - LB_GHOST);

    auto store_row = [&](T *dst, const R dn[4], R w, int r) {
        T e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] = encode<ST>(dn[k], w, rho0);
        if (full[r] && !edge) {
            st4(dst, e);
        } else {
            T *prow = dst - (x0 + LB_GHOST);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (valid[r][k]) put1(p, prow, x0 + k, e[k]);
        }
    };

    /* pass 2: populations */
#pragma unroll 1
    for (int a = 0; a < Q; ++a) {
        const T *pa = fin + a * plane;
        T *po = fout + a * plane;
        const R winv = c.winv[a], crx = c.crx[a], cry = c.cry[a], kx = c.kx[a], ky = c.ky[a];
        const R cxa = c.cx[a], cya = c.cy[a];
        const R gxi = p.gx * cxa + p.gy * cya;
        /* the column strip: window rows 0 .. RB+3 = rows j0-2 .. j0+RB+1 */
        R y[RB + 4][4];
#pragma unroll
        for (int k = 0; k < RB + 4; ++k) {
            T raw[4];
            ld4(pa + roff[k], raw);
#pragma unroll
            for (int m = 0; m < 4; ++m) y[k][m] = decode<ST>(raw[m], winv, rho0);
        }
        /* carried limited y-slope at the face below the current row */
        R mprev[4];
        if (cry > R(0)) {
#pragma unroll
            for (int m = 0; m < 4; ++m) mprev[m] = minmod(y[1][m] - y[0][m], y[2][m] - y[1][m]);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) mprev[m] = minmod(y[2][m] - y[1][m], y[3][m] - y[2][m]);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int k = r + 2;   /* window index of this row */
            R Dy[4], mnext[4];
            if (cry > R(0)) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const R d1 = y[k][m] - y[k - 1][m], d2 = y[k + 1][m] - y[k][m];
                    mnext[m] = minmod(d1, d2);
                    Dy[m] = fma(ky, mnext[m] - mprev[m], d1);
                }
            } else if (cry < R(0)) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const R e1 = y[k + 1][m] - y[k][m], e2 = y[k + 2][m] - y[k + 1][m];
                    mnext[m] = minmod(e1, e2);
                    Dy[m] = fma(-ky, mnext[m] - mprev[m], e1);
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) { Dy[m] = R(0); mnext[m] = R(0); }
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) mprev[m] = mnext[m];
            if (!mine[r]) continue;
            const R *v = y[k];
            R Dx[4];
            if (crx != R(0)) {
                T tl[2], tr[2];
                ld2(pa + roff[k] - 2, tl);
                ld2(pa + roff[k] + 4, tr);
                R l[2] = {decode<ST>(tl[0], winv, rho0), decode<ST>(tl[1], winv, rho0)};
                R rr[2] = {decode<ST>(tr[0], winv, rho0), decode<ST>(tr[1], winv, rho0)};
                if (crx > R(0)) {
                    R d[6] = {l[1] - l[0], v[0] - l[1], v[1] - v[0], v[2] - v[1], v[3] - v[2], rr[0] - v[3]};
                    R mx[5];
#pragma unroll
                    for (int m = 0; m < 5; ++m) mx[m] = minmod(d[m], d[m + 1]);
#pragma unroll
                    for (int m = 0; m < 4; ++m) Dx[m] = fma(kx, mx[m + 1] - mx[m], d[m + 1]);
                } else {
                    R e[6] = {v[0] - l[1], v[1] - v[0], v[2] - v[1], v[3] - v[2], rr[0] - v[3], rr[1] - rr[0]};
                    R mx[5];
#pragma unroll
                    for (int m = 0; m < 5; ++m) mx[m] = minmod(e[m], e[m + 1]);
#pragma unroll
                    for (int m = 0; m < 4; ++m) Dx[m] = fma(-kx, mx[m + 1] - mx[m], e[m + 1]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) Dx[m] = R(0);
            }
            R dn[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const R eu = fma(cya, uy[r][m], cxa * ux[r][m]);
                const R de = fma(rho[r][m], eu * fma(R(0.5), eu, R(1)), A[r][m]);
                R inc = om[r][m] * (de - v[m]);
                inc = fma(-crx, Dx[m], inc);
                inc = fma(-cry, Dy[m], inc);
                if (p.has_force) {
                    const R gu = fma(p.gy, uy[r][m], p.gx * ux[r][m]);
                    inc = fma(p.dt * rho[r][m], gxi + gxi * eu - gu, inc);
                }
                dn[m] = v[m] + inc;
            }
            if (r == wall_r) {
                const R xn = cya * nsgn;
                if (xn > R(0)) continue;   /* replaced by the wall pass */
                if (xn < R(0)) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) num[m] = fma(-xn * c.w[a], dn[m], num[m]);
                }
            }
            store_row(po + roff[k], dn, c.w[a], r);
        }
    }

    /* diffuse wall: gas-bound populations = rho_W S(u_W) (zero net mass flux) */
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (r != wall_r) continue;
        const R uwx = p.uw_x[wall], uwy = p.uw_y[wall];
        const R usw = uwx * uwx + uwy * uwy;
        const R kd = p.kdiff[s][wall], kout = p.kout[s][wall];
        R rwd[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rwd[m] = fma(rho0, kd, num[m]) / kout;
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            if (c.cy[a] * nsgn <= R(0)) continue;
            const R ew = c.cx[a] * uwx + c.cy[a] * uwy;
            const R sm1 = ew + R(0.5) * (ew * ew - usw);
            R dn[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) dn[m] = fma(rwd[m] + rho0, sm1, rwd[m]);
            store_row(fout + a * plane + roff[r + 2], dn, c.w[a], r);
        }
    }

    /* mode B: rows next to the other set, rebuilt in it from what was just written */
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (!mine[r] || !(flags[r] & LB_TILE_SHADOW)) continue;
        const int t = 1 - s;
        const SetConst<R> &ct = p.set[t];
        R h[4][6];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int q = 0; q < 6; ++q) h[m][q] = R(0);
#pragma unroll 1
        for (int a = 0; a < Q; ++a) {
            const T *pr = fout + a * plane + roff[r + 2];
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (valid[r][m]) hermite_acc(c, a, decode<ST>(pr[m], c.winv[a], rho0), h[m]);
        }
        T *ft = static_cast<T *>(p.fout[t]) + (size_t)(j0 + r) * p.pitch;
#pragma unroll 1
        for (int b = 0; b < ct.q; ++b) {
            T *prow = ft + b * plane;
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (valid[r][m]) put1(p, prow, x0 + m, encode<ST>(hermite_rebuild(ct, b, h[m]), ct.w[b], rho0));
        }
    }
}

/* RB rows per thread; MINB resident blocks per SM the register budget is sized for. */
template <int ST, int RB, int MINB>
__global__ void __launch_bounds__(32 * LB2_WY, MINB) step2_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    const int x0 = (blockIdx.x * 32 + threadIdx.x) * 4;
    const int j0 = (blockIdx.y * LB2_WY + threadIdx.y) * RB;
    if (x0 >= p.nx || j0 >= p.ny) return;
    const int tile = x0 / LB_TILE_X;
    uint8_t flags[RB];
    bool valid[RB][4], full[RB];
    int sets = 0;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const int j = j0 + r;
        flags[r] = j < p.ny ? p.tmap[(size_t)j * p.ntx + tile] : LB_TILE_IFACE;
        if (!(flags[r] & LB_TILE_IFACE)) sets |= 1 << (flags[r] & LB_TILE_HIGH);
        full[r] = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            valid[r][k] = (j < p.ny) && (x0 + k < p.nx) && !is_pressure_node(p, x0 + k, j);
            full[r] = full[r] && valid[r][k];
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (!(sets & (1 << s))) continue;
        const int q = p.set[s].q;
        if (q == 9) pass_set<ST, 9, RB>(p, s, x0, j0, flags, valid, full);
        else if (q == 16) pass_set<ST, 16, RB>(p, s, x0, j0, flags, valid, full);
        else pass_set<ST, 36, RB>(p, s, x0, j0, flags, valid, full);
    }
}

#define LB_DISPATCH(store, ...)                                    \
    switch (store) {                                               \
        case 0: { constexpr int ST = 0; __VA_ARGS__; } break;      \
        case 1: { constexpr int ST = 1; __VA_ARGS__; } break;      \
        case 2: { constexpr int ST = 2; __VA_ARGS__; } break;      \
        case 3: { constexpr int ST = 3; __VA_ARGS__; } break;      \
        default: { constexpr int ST = 4; __VA_ARGS__; } break;     \
    }

template <typename R, int ST>
constexpr bool store_matches2()
{
    return std::is_same<R, typename Store<ST>::R>::value;
}

template <int ST, int RB, int MINB>
void launch_rb(const StepParams<typename Store<ST>::R> &p, cudaStream_t st)
{
    dim3 block(32, LB2_WY);
    dim3 grid((p.nx + 127) / 128, (p.ny + RB * LB2_WY - 1) / (RB * LB2_WY));
    step2_kernel<ST, RB, MINB><<<grid, block, 0, st>>>(p);
}

/* variant 1: 2 rows per thread (<= 128 registers), 2: 3 rows (<= 168), 3: 4 rows
 * (<= 255). FP64 storage has one variant (2 rows, 2 blocks per SM). */
template <typename R>
void launch_step2(int store, int variant, const StepParams<R> &p, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches2<R, ST>()) {
        if constexpr (ST == 0) {
            launch_rb<ST, 2, 2>(p, st);
        } else {
            if (variant == 1) launch_rb<ST, 2, 4>(p, st);
            else if (variant == 2) launch_rb<ST, 3, 3>(p, st);
            else launch_rb<ST, 4, 2>(p, st);
        }
    });
}

template void launch_step2<float>(int, int, const StepParams<float> &, void *);
template void launch_step2<double>(int, int, const StepParams<double> &, void *);

}  // namespace lbk
