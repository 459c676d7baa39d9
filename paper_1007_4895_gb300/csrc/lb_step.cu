/*
 * lb_step.cu -- the small passes that complete a time level (interface rows of mode A,
 * pressure columns, rebuilt interface views after the state is replaced) and the
 * dispatch of the step kernel (lb_step_impl.cuh) to its per-storage instantiations.
 */
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_common.cuh"
#include "lb_pressure.cuh"

namespace lbk {

template <int ST>
void launch_step_store(const StepParams<typename Store<ST>::R> &p, void *stream);
template <int ST>
void launch_step_desc_store(const StepParams<typename Store<ST>::R> &p, int n, void *stream);
template <int ST>
void launch_step_split_store(const StepParams<typename Store<ST>::R> &p, int rb, const int2 *edge, int n_edge,
                             void *stream, void *edge_stream);
template <int ST>
void launch_pair_store(const StepParams<float> &p, void *stream);
template <int ST>
void launch_ring_store(const StepParams<float> &p, void *stream);
template <int ST, int Q1>
void launch_ring_units_store(const StepParams<float> &p, const RingTab &tab, const RowQueues &rq, int nblocks,
                             void *stream);
template <int ST, int Q1>
int launch_ring_batch_store(const StepParams<float> *params, const RingTab *tabs, const uint32_t *items,
                            const int2 *ranges, const int *order, int n, int nsteps, int base, int advance,
                            unsigned int *queue, bool force, int grid, int *grid_out, void *stream);

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
    const size_t plane = p.plane;
    const R rho0 = p.rho0;
    R rhod[2], u[2][2];
    const int rows[2] = {jl, jh};
    for (int s = 0; s < 2; ++s) {
        const SetConst<R> &c = p.set[s];
        const T *f = static_cast<const T *>(p.fout[s]) + (size_t)rows[s] * p.pitch + x + LB_GHOST;
        R r = R(0), mx = R(0), my = R(0);
        for (int a = 0; a < c.q; ++a) {
            R d = dec_at<ST>(p, f[a * plane], c.winv[a], x + LB_GHOST);
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
            const R dnb = dec_at<ST>(p, fn[a * plane], c.winv[a], x + LB_GHOST);
            const R eI = c.cx[a] * uIx + c.cy[a] * uIy;
            const R en = c.cx[a] * u[s][0] + c.cy[a] * u[s][1];
            const R d = deq(rIdev, rI, eI, usI) + (dnb - deq(rhod[s], rn, en, usn));
            const T e = enc_at<ST>(p, d, c.w[a], x + LB_GHOST);
            put1r(p, fo + a * plane + (size_t)I * p.pitch, x, I, e);
            put1r(p, fo + a * plane + (size_t)beyond * p.pitch, x, beyond, e);
        }
    }
}

/* ------------------------------------------------------- pressure columns -- */

/* One warp per (row, side) of the pressure columns (lb_pressure.cuh). */
template <int ST>
__global__ void pressure_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int side = blockIdx.y;
    if (j >= p.ny || !p.pressure[side]) return;   /* uniform over the warp */
    pressure_row<ST>(p, j, side);
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
    const size_t plane = p.plane;
    const T *f = static_cast<const T *>(p.fout[s]) + (size_t)j * p.pitch + x + LB_GHOST;
    R h[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int a = 0; a < c.q; ++a) hermite_acc(c, a, dec_at<ST>(p, f[a * plane], c.winv[a], x + LB_GHOST), h);
    T *ft = static_cast<T *>(p.fout[1 - s]);
    for (int b = 0; b < ct.q; ++b)
        put1r(p, ft + b * plane + (size_t)j * p.pitch, x, j, enc_at<ST>(p, hermite_rebuild(ct, b, h), ct.w[b], x + LB_GHOST));
}

/* ----------------------------------------------- D2Q9 stream and collide -- */

/* The D2Q9 reduction of the Sec. 3.1 update at Courant number one (dt = h / sqrt(3),
 * abscissae +-sqrt(3)): every population moves exactly one node along sign(xi) per step
 * (stream), then relaxes towards Eq. (demoeq) with the Eq. (demoforce) force at the
 * streamed state (collide). Periodic lattice of one set; one thread per node. The
 * ghost rows and columns hold the periodic images, so the pull needs no index logic. */
template <int ST>
__global__ void __launch_bounds__(128) exact_stream_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (x >= p.nx) return;
    /* the population loops are unrolled, so the set's constants are read from the
     * parameter block at fixed offsets; population a = 3 iy + ix over ascending
     * abscissae moves by (ix - 1, iy - 1) */
    const SetConst<R> &c = p.set[0];
    const T *fin = static_cast<const T *>(p.fin[0]);
    T *fout = static_cast<T *>(p.fout[0]);
    const size_t plane = p.plane;
    const R rho0 = p.rho0;
    R d[9], rd = R(0), jx = R(0), jy = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int sx = a % 3 - 1, sy = a / 3 - 1;
        const int col = x - sx + LB_GHOST;
        d[a] = dec_at<ST>(p, fin[a * plane + (ptrdiff_t)(j - sy) * p.pitch + col], c.winv[a], col);
        rd = fma(c.w[a], d[a], rd);
        jx = fma(c.wcx[a], d[a], jx);
        jy = fma(c.wcy[a], d[a], jy);
    }
    const R rho = rho0 + rd, inv = R(1) / rho;
    const R ux = jx * inv, uy = jy * inv;
    const R usq = usq_of(ux, uy), om = p.dt / tau_of(p, inv), gu = xi_dot(p.gx, p.gy, ux, uy);
    int img[2];
    /* a node whose value has no ghost copy: stored once */
    const bool plain = row_images(p, j, img) == 0 && x >= LB_GHOST && x < p.nx - LB_GHOST;
    T *row = fout + (size_t)j * p.pitch;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const R eu = xi_dot(c.cx[a], c.cy[a], ux, uy);
        R inc = om * (deq(rd, rho, eu, usq) - d[a]);
        if (p.has_force) inc = force_inc(p.dt * rho, xi_dot(c.cx[a], c.cy[a], p.gx, p.gy), eu, gu, inc);
        const T e = enc_at<ST>(p, d[a] + inc, c.w[a], x + LB_GHOST);
        if (plain) row[a * plane + x + LB_GHOST] = e;
        else put1r(p, row + a * plane, x, j, e);
    }
}

/* ------------------------------------------------------ carried moments -- */

/* Carried moments of the written level, sum w d, sum w xi_x d, sum w xi_y d per node
 * from its stored populations in population order: of every node (list == NULL) or of
 * the listed quads (x0, j). */
template <int ST>
__global__ void __launch_bounds__(128) aux_kernel(const __grid_constant__ StepParams<typename Store<ST>::R> p,
                                                  const int2 *__restrict__ list, int n)
{
    using T = typename Store<ST>::T;
    using R = typename Store<ST>::R;
    __shared__ PopC<R> pcs[2][LB_QMAX];
    __shared__ MomC<R> mcs[2][LB_QMAX];
    stage_consts(p, pcs, mcs, threadIdx.x, blockDim.x);
    __syncthreads();
    int x, j, cnt;
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        if (k >= (size_t)n) return;
        x = list[k].x;
        j = list[k].y;
        cnt = 4;
    } else {
        if (k >= (size_t)p.nx * p.ny) return;
        j = (int)(k / p.nx);
        x = (int)(k - (size_t)j * p.nx);
        cnt = 1;
    }
    if (j < 0 || j >= p.ny) return;
    R *aout = static_cast<R *>(p.aux_out);
    const size_t ap = (size_t)p.pitch * p.ny;
    for (int i = 0; i < cnt && x + i < p.nx; ++i) {
        const int xi = x + i;
        const int s = p.tmap[(size_t)j * p.ntx + xi / LB_TILE_X] & LB_TILE_HIGH;
        const T *f = static_cast<const T *>(p.fout[s]) + (size_t)j * p.pitch + xi + LB_GHOST;
        R rd, jx, jy;
        const int q = p.set[s].q;
        if (q == 9) node_moments<ST, 9>(f, p.plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, xi + LB_GHOST);
        else if (q == 16) node_moments<ST, 16>(f, p.plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, xi + LB_GHOST);
        else node_moments<ST, 36>(f, p.plane, mcs[s], p.rho0, rd, jx, jy, p.dcol, xi + LB_GHOST);
        const size_t m = (size_t)j * p.pitch + xi;
        aout[m] = rd;
        aout[ap + m] = jx;
        aout[2 * ap + m] = jy;
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
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) launch_step_store<ST>(p, stream));
}

void launch_ring(int store, const StepParams<float> &p, void *stream)
{
    switch (store) {
        case 1: launch_ring_store<1>(p, stream); break;
        case 2: launch_ring_store<2>(p, stream); break;
        case 3: launch_ring_store<3>(p, stream); break;
        case 4: launch_ring_store<4>(p, stream); break;
        default: break;
    }
}

void launch_ring_units(int store, const StepParams<float> &p, const RingTab &tab, const RowQueues &rq, int nblocks,
                       void *stream)
{
    const bool q36 = p.set[1].q == 36;
    switch (store) {
        case 1: (q36 ? launch_ring_units_store<1, 36> : launch_ring_units_store<1, 16>)(p, tab, rq, nblocks, stream); break;
        case 2: (q36 ? launch_ring_units_store<2, 36> : launch_ring_units_store<2, 16>)(p, tab, rq, nblocks, stream); break;
        case 3: (q36 ? launch_ring_units_store<3, 36> : launch_ring_units_store<3, 16>)(p, tab, rq, nblocks, stream); break;
        case 4: (q36 ? launch_ring_units_store<4, 36> : launch_ring_units_store<4, 16>)(p, tab, rq, nblocks, stream); break;
        default: break;
    }
}

int launch_ring_batch(int store, int q1, const StepParams<float> *params, const RingTab *tabs, const uint32_t *items,
                      const int2 *ranges, const int *order, int n, int nsteps, int base, int advance,
                      unsigned int *queue, bool force, int grid, int *grid_out, void *stream)
{
    const bool q36 = q1 == 36;
    if (!q36 && q1 != 16) return -1;
#define LB_RB(ST) (q36 ? launch_ring_batch_store<ST, 36> : launch_ring_batch_store<ST, 16>)( \
        params, tabs, items, ranges, order, n, nsteps, base, advance, queue, force, grid, grid_out, stream)
    switch (store) {
        case 1: return LB_RB(1);
        case 2: return LB_RB(2);
        case 3: return LB_RB(3);
        case 4: return LB_RB(4);
        default: return -1;
    }
#undef LB_RB
}

void launch_pair(int store, const StepParams<float> &p, void *stream)
{
    switch (store) {
        case 1: launch_pair_store<1>(p, stream); break;
        case 2: launch_pair_store<2>(p, stream); break;
        case 3: launch_pair_store<3>(p, stream); break;
        case 4: launch_pair_store<4>(p, stream); break;
        default: break;
    }
}

template <typename R>
void launch_exact_stream(int store, const StepParams<R> &p, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) exact_stream_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template <typename R>
void launch_step_desc(int store, const StepParams<R> &p, int n, void *stream)
{
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) launch_step_desc_store<ST>(p, n, stream));
}

template <int ST>
int launch_batch_store(const void *params, const int *order, int n, int nsteps, int base, int advance,
                       unsigned int *queue, int threads, int grid, void *stream);
template <int ST>
int batch_blocks_per_sm(int threads);

int launch_batch(int store, const void *params, const int *order, int n, int nsteps, int base, int advance,
                 unsigned int *queue, int threads, int grid, void *stream)
{
    int r = -1;
    LB_DISPATCH(store, r = launch_batch_store<ST>(params, order, n, nsteps, base, advance, queue, threads, grid, stream));
    return r;
}

int batch_blocks(int store, int threads)
{
    int r = 0;
    LB_DISPATCH(store, r = batch_blocks_per_sm<ST>(threads));
    return r;
}

template <typename R>
void launch_step_split(int store, const StepParams<R> &p, int rb, const int2 *edge, int n_edge, void *stream,
                       void *edge_stream)
{
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>())
                           launch_step_split_store<ST>(p, rb, edge, n_edge, stream, edge_stream));
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
    dim3 grid((p.ny + 3) / 4, 2);   /* four warps (rows) per block */
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) pressure_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template <typename R>
void launch_shadows(int store, const StepParams<R> &p, void *stream)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>()) shadows_kernel<ST><<<grid, 128, 0, st>>>(p));
}

template void launch_step<float>(int, const StepParams<float> &, void *);
template void launch_step<double>(int, const StepParams<double> &, void *);
template void launch_exact_stream<float>(int, const StepParams<float> &, void *);
template void launch_exact_stream<double>(int, const StepParams<double> &, void *);
template void launch_step_desc<float>(int, const StepParams<float> &, int, void *);
template void launch_step_desc<double>(int, const StepParams<double> &, int, void *);
template void launch_step_split<float>(int, const StepParams<float> &, int, const int2 *, int, void *, void *);
template void launch_step_split<double>(int, const StepParams<double> &, int, const int2 *, int, void *, void *);
template void launch_iface<float>(int, const StepParams<float> &, void *);
template void launch_iface<double>(int, const StepParams<double> &, void *);



template <typename R>
void launch_aux(int store, const StepParams<R> &p, const int2 *list, int n, void *stream)
{
    const long long items = list ? n : (long long)p.nx * p.ny;
    if (items <= 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LB_DISPATCH(store, if constexpr (store_matches<R, ST>())
                           aux_kernel<ST><<<(unsigned)((items + 127) / 128), 128, 0, st>>>(p, list, n));
}

template void launch_aux<float>(int, const StepParams<float> &, const int2 *, int, void *);
template void launch_aux<double>(int, const StepParams<double> &, const int2 *, int, void *);
template void launch_pressure<float>(int, const StepParams<float> &, void *);
template void launch_pressure<double>(int, const StepParams<double> &, void *);
template void launch_shadows<float>(int, const StepParams<float> &, void *);
template void launch_shadows<double>(int, const StepParams<double> &, void *);

}  // namespace lbk
