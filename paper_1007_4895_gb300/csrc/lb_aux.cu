/*
 * lb_aux.cu -- kernels around the step: initial equilibrium, population import /
 * export in the canonical layout, moment fields, and the FP64 mass / residual
 * reduction.
 */
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_common.cuh"

namespace lbk {

/* f = f_eq(rho, u) (Eq. (demoeq)) in every node's own set. One thread per node. */
template <int ST>
__global__ void init_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p, const double *rho,
                            const double *ux, const double *uy)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    const size_t n = (size_t)j * p.nx + x;
    const int s = p.tmap[(size_t)j * p.ntx + x / LB_TILE_X] & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const R r = R(rho[n]), u = R(ux[n]), v = R(uy[n]);
    const R rd = R(rho[n] - double(p.rho0)), usq = u * u + v * v;
    const size_t plane = p.plane;
    T *f = static_cast<T *>(p.fout[s]);
    for (int a = 0; a < c.q; ++a)
        put1r(p, f + a * plane + (size_t)j * p.pitch, x, j,
              enc_at<ST>(p, deq(rd, r, c.cx[a] * u + c.cy[a] * v, usq), c.w[a], x + LB_GHOST));
}

/* Compact state: each node's populations in its own set and nothing else (shadows,
 * ghosts, interface and pressure nodes and carried moments are rebuilt from them).
 * seg[k] = (tile, row, set, index of the segment within its set): one tile row of a
 * set, sets in order, rows and tiles ascending. Population a of segment k of set s
 * sits at base_s + (a * nseg_s + k) * LB_TILE_X + column in the tile, with base_0 = 0,
 * base_1 = q_0 nseg_0 LB_TILE_X; columns beyond nx hold zero.
 * One warp per (set, population, segment) in the order of the compact buffer, four
 * columns per lane: 16-byte vectors on both sides where the quad lies inside the
 * lattice (and, unpacking, needs no ghost copy). Returns false for a warp past the end. */
struct PackPos {
    int s, a, tile, row;
    size_t off;   /* element offset of this lane's four values in the compact buffer */
};
__device__ __forceinline__ bool pack_pos(const int4 *seg, int q0, int q1, int nseg0, int nseg1, PackPos &pp)
{
    const size_t w = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const size_t n0 = (size_t)q0 * nseg0;
    size_t k;
    if (w < n0) {
        pp.s = 0;
        pp.a = (int)(w / nseg0);
        k = w % nseg0;
    } else {
        const size_t w1 = w - n0;
        if (nseg1 == 0 || w1 >= (size_t)q1 * nseg1) return false;
        pp.s = 1;
        pp.a = (int)(w1 / nseg1);
        k = nseg0 + w1 % nseg1;
    }
    const int4 g = seg[k];
    pp.tile = g.x;
    pp.row = g.y;
    pp.off = w * LB_TILE_X + 4 * (threadIdx.x & 31);
    return true;
}

template <int ST>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p,
                                                   const int4 *seg, int nseg0, int nseg1, typename Store<ST>::T *dst)
{
    using T = typename Store<ST>::T;
    PackPos pp;
    if (!pack_pos(seg, p.set[0].q, p.set[1].q, nseg0, nseg1, pp)) return;
    const int x = pp.tile * LB_TILE_X + 4 * (threadIdx.x & 31);
    const T *f = static_cast<const T *>(p.fin[pp.s]) + pp.a * p.plane + (size_t)pp.row * p.pitch + LB_GHOST + x;
    T v[4];
    if (x + 3 < p.nx) {
        ld4(f, v);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = x + k < p.nx ? f[k] : T();
    }
    st4(dst + pp.off, v);
}

template <int ST>
__global__ void __launch_bounds__(256) unpack_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p,
                                                     const int4 *seg, int nseg0, int nseg1,
                                                     const typename Store<ST>::T *src)
{
    using T = typename Store<ST>::T;
    PackPos pp;
    if (!pack_pos(seg, p.set[0].q, p.set[1].q, nseg0, nseg1, pp)) return;
    const int x = pp.tile * LB_TILE_X + 4 * (threadIdx.x & 31);
    if (x >= p.nx) return;
    T v[4];
    ld4(src + pp.off, v);
    T *row = static_cast<T *>(p.fout[pp.s]) + pp.a * p.plane + (size_t)pp.row * p.pitch;
    int img[2];
    const bool plain = x + 3 < p.nx && row_images(p, pp.row, img) == 0 &&
                       !(p.periodic_x && (x < LB_GHOST || x + 3 >= p.nx - LB_GHOST));
    if (plain) {
        st4(row + LB_GHOST + x, v);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x + k < p.nx) put1r(p, row, x + k, pp.row, v[k]);
    }
}

/* Canonical double [q][ny][nx] -> planes of set `set`, at nodes that use that set. */
template <int ST>
__global__ void set_pops_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p, int set,
                                const double *src)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    if ((p.tmap[(size_t)j * p.ntx + x / LB_TILE_X] & LB_TILE_HIGH) != set) return;
    const SetConst<R> &c = p.set[set];
    const size_t plane = p.plane;
    T *f = static_cast<T *>(p.fout[set]);
    for (int a = 0; a < c.q; ++a) {
        const double fv = src[((size_t)a * p.ny + j) * p.nx + x];
        const R d = R(fv * double(c.winv[a]) - double(p.rho0));
        put1r(p, f + a * plane + (size_t)j * p.pitch, x, j, enc_at<ST>(p, d, c.w[a], x + LB_GHOST));
    }
}

/* Planes of set `set` -> canonical double f [q][ny][nx] (every node). */
template <int ST>
__global__ void get_pops_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p, int set, double *dst)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    const SetConst<R> &c = p.set[set];
    const size_t plane = p.plane;
    const T *f = static_cast<const T *>(p.fin[set]) + (size_t)j * p.pitch + x + LB_GHOST;
    for (int a = 0; a < c.q; ++a) {
        const R d = dec_at<ST>(p, f[a * plane], c.winv[a], x + LB_GHOST);
        dst[((size_t)a * p.ny + j) * p.nx + x] = double(c.w[a]) * (double(p.rho0) + double(d));
    }
}

/* Moment fields of every node from its own set: rho, u, P_xy = sum f (xi-u)_x (xi-u)_y,
 * Pi^neq = sum (f - f_eq) xi xi, q = (1/2) sum f |xi - u|^2 (xi - u). The rest-state
 * part w rho0 is summed in closed form (Gaussian moments up to third order, exact for
 * every set), so only deviations enter the sums. */
template <int ST, typename OUT>
__global__ void moments_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p, uint32_t mask,
                               OUT *dst)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    const int s = p.tmap[(size_t)j * p.ntx + x / LB_TILE_X] & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const size_t plane = p.plane;
    const T *f = static_cast<const T *>(p.fin[s]) + (size_t)j * p.pitch + x + LB_GHOST;
    const R rho0 = p.rho0;
    R d[LB_QMAX];
    R rd = R(0), jx = R(0), jy = R(0);
    for (int a = 0; a < c.q; ++a) {
        d[a] = dec_at<ST>(p, f[a * plane], c.winv[a], x + LB_GHOST);
        rd = fma(c.w[a], d[a], rd);
        jx = fma(c.wcx[a], d[a], jx);
        jy = fma(c.wcy[a], d[a], jy);
    }
    const R rho = rho0 + rd, ux = jx / rho, uy = jy / rho, usq = ux * ux + uy * uy;
    /* rest-state parts: sum w (xi-u)_x (xi-u)_y = ux uy; sum w |xi-u|^2 (xi-u)_x = -ux (4 + u^2) */
    R pxy = rho0 * ux * uy, nxx = R(0), nxy = R(0), nyy = R(0);
    R qx = R(-0.5) * rho0 * ux * (R(4) + usq), qy = R(-0.5) * rho0 * uy * (R(4) + usq);
    for (int a = 0; a < c.q; ++a) {
        const R cx = c.cx[a], cy = c.cy[a];
        const R wd = c.w[a] * d[a];
        const R dx = cx - ux, dy = cy - uy, dd = dx * dx + dy * dy;
        const R eu = cx * ux + cy * uy;
        const R wne = c.w[a] * (d[a] - deq(rd, rho, eu, usq));
        pxy = fma(wd, dx * dy, pxy);
        nxx = fma(wne, cx * cx, nxx);
        nxy = fma(wne, cx * cy, nxy);
        nyy = fma(wne, cy * cy, nyy);
        qx = fma(R(0.5) * wd, dd * dx, qx);
        qy = fma(R(0.5) * wd, dd * dy, qy);
    }
    const R vals[9] = {rho, ux, uy, pxy, nxx, nxy, nyy, qx, qy};
    const size_t N = (size_t)p.nx * p.ny, n = (size_t)j * p.nx + x;
    int k = 0;
    for (int m = 0; m < 9; ++m)
        if (mask & (1u << m)) dst[(size_t)(k++) * N + n] = OUT(vals[m]);
}

/* FP64 sums over every node: mass, |u - u_prev|^2, |u|^2, count of non-finite nodes.
 * Warp shuffles, then shared memory, then one partial per block; the last block to
 * finish adds the partials in block order (deterministic) and resets the counter. */
template <int ST>
__global__ void __launch_bounds__(256) reduce_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p,
                                                     typename Store<ST>::R *uprev, double *part, unsigned int *counter,
                                                     double *out)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pcs[2][LB_QMAX];
    __shared__ MomC<R> mcs[2][LB_QMAX];
    stage_consts(p, pcs, mcs, threadIdx.x, blockDim.x);
    __syncthreads();
    const size_t N = (size_t)p.nx * p.ny;
    const size_t plane = p.plane;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(n / p.nx), x = (int)(n - (size_t)j * p.nx);
        const int s = p.tmap[(size_t)j * p.ntx + x / LB_TILE_X] & LB_TILE_HIGH;
        const T *f = static_cast<const T *>(p.fin[s]) + (size_t)j * p.pitch + x + LB_GHOST;
        R rd, jx, jy;
        const int q = p.set[s].q;
        if (q == 9) node_moments<ST, 9>(f, plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, x + LB_GHOST);
        else if (q == 16) node_moments<ST, 16>(f, plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, x + LB_GHOST);
        else node_moments<ST, 36>(f, plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, x + LB_GHOST);
        /* u as the step forms it (one reciprocal in the arithmetic type); FP64 only for
         * the sums: the FP64 rate is a small fraction of the FP32 rate here */
        const R rr = p.rho0 + rd, inv = R(1) / rr;
        const R uxr = jx * inv, uyr = jy * inv;
        const double rho = double(p.rho0) + double(rd);
        const double ux = double(uxr), uy = double(uyr);
        if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy)) {
            acc[3] += 1.0;
        } else {
            const double px = double(uprev[2 * n]), py = double(uprev[2 * n + 1]);
            acc[0] += rho;
            acc[1] += (ux - px) * (ux - px) + (uy - py) * (uy - py);
            acc[2] += ux * ux + uy * uy;
        }
        /* every node keeps this reduction's velocity, a non-finite one included */
        uprev[2 * n] = uxr;
        uprev[2 * n + 1] = uyr;
    }
    for (int m = 0; m < 4; ++m)
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_down_sync(0xffffffffu, acc[m], o);
    __shared__ double sh[32][4];
    __shared__ bool last;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nw = (int)(blockDim.x / 32);
    if (lane == 0)
        for (int m = 0; m < 4; ++m) sh[warp][m] = acc[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        double b[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < nw; ++w)
            for (int m = 0; m < 4; ++m) b[m] += sh[w][m];
        for (int m = 0; m < 4; ++m) part[4 * blockIdx.x + m] = b[m];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    /* last block: each thread adds the partials b = t, t + blockDim, ... in order, then
     * a fixed warp and block tree (same order every call) */
    __threadfence();
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
        for (int m = 0; m < 4; ++m) t[m] += __ldcg(&part[4 * b + m]);
    for (int m = 0; m < 4; ++m)
        for (int o = 16; o > 0; o >>= 1) t[m] += __shfl_down_sync(0xffffffffu, t[m], o);
    __syncthreads();
    if (lane == 0)
        for (int m = 0; m < 4; ++m) sh[warp][m] = t[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        double u[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < nw; ++w)
            for (int m = 0; m < 4; ++m) u[m] += sh[w][m];
        out[0] = u[0];
        out[1] = u[2] > 0.0 ? sqrt(u[1] / u[2]) : 0.0;
        out[2] = u[3];
        *counter = 0u;
    }
}

/* Features of the learned placement, from moment fields m [9][ny][nx] (rho, u,
 * P_xy, Pi^neq xx / xy / yy, q): Pi^neq / rho (3), q / rho (2), wall distance / H,
 * local Kn = tau (Eq. (KN), without the dt / 2 shift) and Kn |grad rho| / rho with
 * central differences (one-sided at non-periodic edges). out [8][ny][nx]. */
template <typename R>
__global__ void features_kernel(const StepParams<R> p, const float *m, float *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    const size_t N = (size_t)p.nx * p.ny, n = (size_t)j * p.nx + x;
    const float rho = m[n];
    auto rho_at = [&](int xx, int jj) -> float {
        if (p.periodic_x) xx = (xx + p.nx) % p.nx;
        if (p.periodic_y) jj = (jj + p.ny) % p.ny;
        return m[(size_t)jj * p.nx + xx];
    };
    const float h = (float)p.h_grid;
    float gx, gy;
    {
        const bool lo = !p.periodic_x && x == 0, hi = !p.periodic_x && x == p.nx - 1;
        const int xa = lo ? x : x - 1, xb = hi ? x : x + 1;
        gx = (rho_at(xb, j) - rho_at(xa, j)) / (h * (float)(xb - xa));
    }
    {
        const bool lo = !p.periodic_y && j == 0, hi = !p.periodic_y && j == p.ny - 1;
        const int ja = lo ? j : j - 1, jb = hi ? j : j + 1;
        gy = (rho_at(x, jb) - rho_at(x, ja)) / (h * (float)(jb - ja));
    }
    const float kn = p.tau_const ? (float)p.kn_rho : (float)p.kn_rho / rho;
    float dw = 1.0f;
    if (p.wall_diffuse[0] || p.wall_diffuse[1]) {
        const int d0 = p.wall_diffuse[0] ? j : 1 << 30, d1 = p.wall_diffuse[1] ? p.ny - 1 - j : 1 << 30;
        dw = (float)min(d0, d1) * h;
    }
    const float inv = 1.0f / rho;
    out[0 * N + n] = m[4 * N + n] * inv;
    out[1 * N + n] = m[5 * N + n] * inv;
    out[2 * N + n] = m[6 * N + n] * inv;
    out[3 * N + n] = m[7 * N + n] * inv;
    out[4 * N + n] = m[8 * N + n] * inv;
    out[5 * N + n] = dw;
    out[6 * N + n] = kn;
    out[7 * N + n] = kn * sqrtf(gx * gx + gy * gy) * inv;
}

/* Part of a node's populations beyond a second-order Hermite expansion (what a
 * low-order node cannot hold, Sec. 2.2), per unit mass: ||f - P2 f|| / rho in the norm
 * sum_a g_a^2 / w_a, from the node's own set. With f = w (rho0 + d) the norm is
 * sum_a w_a (d_a - d2_a)^2. out [ny][nx]. */
template <int ST>
__global__ void hermite_residual_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p, float *out)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    const int s = p.tmap[(size_t)j * p.ntx + x / LB_TILE_X] & LB_TILE_HIGH;
    const SetConst<R> &c = p.set[s];
    const T *f = static_cast<const T *>(p.fin[s]) + (size_t)j * p.pitch + x + LB_GHOST;
    R d[LB_QMAX], h[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int a = 0; a < c.q; ++a) {
        d[a] = dec_at<ST>(p, f[a * p.plane], c.winv[a], x + LB_GHOST);
        hermite_acc(c, a, d[a], h);
    }
    R num = R(0);
    for (int a = 0; a < c.q; ++a) {
        const R e2 = d[a] - hermite_rebuild(c, a, h);
        num = fma(c.w[a] * e2, e2, num);
    }
    out[(size_t)j * p.nx + x] = (float)(sqrt(num) / (p.rho0 + h[0]));
}

/* Largest p over each map tile (NaN if any node's p is NaN). */
__global__ void tile_max_kernel(const float *p, int nx, int ny, int ntx, float *out)
{
    const int tx = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (tx >= ntx) return;
    float mx = -1.0f;
    bool bad = false;
    for (int x = tx * LB_TILE_X; x < min(nx, (tx + 1) * LB_TILE_X); ++x) {
        const float v = p[(size_t)j * nx + x];
        if (!(v == v)) bad = true;
        mx = fmaxf(mx, v);
    }
    out[(size_t)j * ntx + tx] = bad ? nanf("") : mx;
}

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
void launch_init(int store, const StepParams<R> &p, const double *rho, const double *ux, const double *uy,
                 void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) init_kernel<ST><<<grid, 128, 0, st>>>(p, rho, ux, uy));
}

template <typename R>
void launch_pack(int store, const StepParams<R> &p, const int4 *seg, int nseg0, int nseg1, int qmax, void *dst,
                 int unpack, void *stream)
{
    (void)qmax;
    const size_t warps = (size_t)p.set[0].q * nseg0 + (size_t)p.set[1].q * nseg1;
    if (warps == 0) return;
    const unsigned grid = (unsigned)((warps + 7) / 8);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) {
        using T = typename Store<ST>::T;
        if (unpack) unpack_kernel<ST><<<grid, 256, 0, st>>>(p, seg, nseg0, nseg1, static_cast<const T *>(dst));
        else pack_kernel<ST><<<grid, 256, 0, st>>>(p, seg, nseg0, nseg1, static_cast<T *>(dst));
    });
}

template <typename R>
void launch_set_pops(int store, const StepParams<R> &p, int set, const double *src, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) set_pops_kernel<ST><<<grid, 128, 0, st>>>(p, set, src));
}

template <typename R>
void launch_get_pops(int store, const StepParams<R> &p, int set, double *dst, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) get_pops_kernel<ST><<<grid, 128, 0, st>>>(p, set, dst));
}

template <typename R>
void launch_moments(int store, const StepParams<R> &p, uint32_t mask, void *dst, int dst_f64, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dst_f64) {
        LB_DISPATCH(store, if constexpr (store_matches<R, ST>())
                               moments_kernel<ST, double><<<grid, 128, 0, st>>>(p, mask, static_cast<double *>(dst)));
    } else {
        LB_DISPATCH(store, if constexpr (store_matches<R, ST>())
                               moments_kernel<ST, float><<<grid, 128, 0, st>>>(p, mask, static_cast<float *>(dst)));
    }
}

template <typename R>
void launch_features(const StepParams<R> &p, const float *moments, float *out, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    features_kernel<R><<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(p, moments, out);
}

template <typename R>
void launch_hermite_residual(int store, const StepParams<R> &p, float *out, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) hermite_residual_kernel<ST><<<grid, 128, 0, st>>>(p, out));
}

void launch_tile_max(const float *pr, int nx, int ny, int ntx, float *out, void *stream)
{
    dim3 grid((ntx + 63) / 64, ny);
    tile_max_kernel<<<grid, 64, 0, static_cast<cudaStream_t>(stream)>>>(pr, nx, ny, ntx, out);
}

template void launch_features<float>(const StepParams<float> &, const float *, float *, void *);
template void launch_features<double>(const StepParams<double> &, const float *, float *, void *);
template void launch_hermite_residual<float>(int, const StepParams<float> &, float *, void *);
template void launch_hermite_residual<double>(int, const StepParams<double> &, float *, void *);

/* One node per thread (at most 16384 blocks; larger lattices loop). */
int reduce_blocks(int nx, int ny, int nsm)
{
    /* four 256-thread blocks per SM: each thread sums several nodes before the FP64
     * warp and block trees, whose cost per thread is fixed (the FP64 rate is a small
     * fraction of the FP32 rate here) */
    long long n = (long long)nx * ny;
    long long b = (n + 255) / 256;
    const long long cap = nsm > 0 ? 4LL * nsm : 16384;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename R>
void launch_reduce(int store, const StepParams<R> &p, R *uprev, double *part, unsigned int *counter, double *out,
                   int nblocks, void *stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>())
                           reduce_kernel<ST><<<nblocks, 256, 0, st>>>(p, uprev, part, counter, out));
}

template void launch_init<float>(int, const StepParams<float> &, const double *, const double *, const double *, void *);
template void launch_init<double>(int, const StepParams<double> &, const double *, const double *, const double *, void *);
template void launch_pack<float>(int, const StepParams<float> &, const int4 *, int, int, int, void *, int, void *);
template void launch_pack<double>(int, const StepParams<double> &, const int4 *, int, int, int, void *, int, void *);
template void launch_set_pops<float>(int, const StepParams<float> &, int, const double *, void *);
template void launch_set_pops<double>(int, const StepParams<double> &, int, const double *, void *);
template void launch_get_pops<float>(int, const StepParams<float> &, int, double *, void *);
template void launch_get_pops<double>(int, const StepParams<double> &, int, double *, void *);
template void launch_moments<float>(int, const StepParams<float> &, uint32_t, void *, int, void *);
template void launch_moments<double>(int, const StepParams<double> &, uint32_t, void *, int, void *);
template void launch_reduce<float>(int, const StepParams<float> &, float *, double *, unsigned int *, double *, int, void *);
template void launch_reduce<double>(int, const StepParams<double> &, double *, double *, unsigned int *, double *, int, void *);

}  // namespace lbk
