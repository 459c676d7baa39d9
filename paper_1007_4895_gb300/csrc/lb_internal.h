/*
 * lb_internal.h -- data layout and launch parameters shared by the host side of the
 * library (lb_api.cu) and its kernels (lb_step.cu, lb_aux.cu).
 *
 * Device layout of one time level of one velocity set: Q planes, each
 * [ny + 2 LB_GHOST_ROWS][pitch] elements, x contiguous. Logical column x lives at
 * storage column x + LB_GHOST, logical row j at storage row j + LB_GHOST_ROWS. The ghost
 * columns hold periodic images (periodic x) or copies of the boundary column (pressure
 * sides); the ghost rows hold copies of the wall row (Sec. 3.2: ghost node = wall node)
 * or periodic images. So the radius-2 stencil never wraps or clamps an index, and a
 * tile plus its halo is one dense box (what the TMA loads). Pointers handed to kernels
 * point at logical row 0, column 0 - LB_GHOST.
 * Both sets have planes over the whole grid: a node's own set holds its state; the
 * other set's planes hold, at nodes next to an interface, that node rebuilt in the
 * other set (written by the step that produced the node), which is exactly what the
 * readers of the other set need at the next step.
 *
 * The region map is kept per tile of LB_TILE_X columns x 1 row, one byte of flags.
 */
#pragma once

#include <cstddef>
#include <cstdint>

#include <vector_types.h>

#define LB_GHOST 4
#define LB_GHOST_ROWS 2
#define LB_TILE_X 128
#define LB_QMAX 36
#define LB_MAX_IFACE 64
#define LB_STEP_BY 8    /* rows per block of the one-quad kernel (its blocks are one tile wide) */

enum : uint8_t {
    LB_TILE_HIGH = 1u,     /* tile uses set 1 */
    LB_TILE_SHADOW = 2u,   /* mode B: also write this tile rebuilt in the other set */
    LB_TILE_IFACE = 4u,    /* mode A: interface row, set by the interface pass */
    LB_TILE_NEAR_H = 8u,   /* mode A: interface row whose high-order neighbour is j - 1 */
};

template <typename R>
struct SetConst {
    int q;
    int n1d;
    R cx[LB_QMAX], cy[LB_QMAX];     /* abscissae xi_x, xi_y */
    R w[LB_QMAX], winv[LB_QMAX];    /* weights and 1 / w */
    R wcx[LB_QMAX], wcy[LB_QMAX];   /* w xi_x, w xi_y */
    R crx[LB_QMAX], cry[LB_QMAX];   /* Courant numbers xi dt / h */
    R kx[LB_QMAX], ky[LB_QMAX];     /* (1 - |Courant|) / 2 */
    R wxx[LB_QMAX], wxy[LB_QMAX], wyy[LB_QMAX];   /* w (xi_x^2 - 1), w xi_x xi_y, w (xi_y^2 - 1) */
    R hxx[LB_QMAX], hxy[LB_QMAX], hyy[LB_QMAX];   /* (xi_x^2 - 1) / 2, xi_x xi_y, (xi_y^2 - 1) / 2 */
};

template <typename R>
struct StepParams {
    int nx, ny, pitch, ntx;
    double h_grid;                  /* grid spacing h */
    size_t plane;                   /* elements per plane, (ny + 2 LB_GHOST_ROWS) * pitch */
    const uint8_t *tmap;            /* [ny][ntx] tile flags */
    const void *fin[2];             /* planes of the level read, per set */
    void *fout[2];                  /* planes of the level written, per set */
    /* carried moments (streamed layout): per node, in its own set, the sums
     * sum w d, sum w xi_x d, sum w xi_y d of the stored deviations, R [3][ny][nx],
     * of the level read (aux_in) and of the level written (aux_out) */
    const void *aux_in;
    void *aux_out;
    /* one-quad kernel: launch order of its blocks (tile + ntx * band of LB_STEP_BY rows),
     * blocks with a high-order row first, so that the long blocks start in the first
     * wave; NULL: the natural two-dimensional grid */
    const int *block_order;
    /* layout 6: block descriptors (tile, 2 * first row + h); h = 1: 4 rows, two nodes
     * per thread (bands holding high-order rows), h = 0: LB_STEP_BY rows, one quad per
     * thread */
    const int2 *block_desc;
    /* per-column reference density (deviation formats): delta = rho0(x) - rho0 per
     * storage column [pitch] (ghost columns hold the delta of the column they copy);
     * NULL: one reference density */
    const R *dcol;
    /* layouts 7 / 8: the per-population constant tables in device memory, built once per
     * lattice by launch_pair_table (NULL for the other layouts) */
    const void *ctab;
    int sr;                         /* stochastic rounding of the updated populations */
    uint32_t step_key;              /* the step being computed (random-bit key) */
    R rho0, dt;
    R kn_rho;                       /* kn_ref * rho_ref (tau = kn_rho / rho), or tau if const */
    int tau_const;                  /* 1: tau = kn_rho */
    R tau_shift;                    /* subtracted from tau (dt / 2 or 0) */
    R gx, gy;
    int has_force;
    int periodic_x, periodic_y;
    int wall_diffuse[2];            /* bottom, top */
    int pressure[2];                /* left, right */
    R rho_side[2];                  /* pressure densities, left / right */
    R uw_x[2], uw_y[2];             /* wall velocities at the new time level */
    R kin[2][2];                    /* [set][wall] sum_{in} |xi.n| w */
    R kout[2][2];                   /* [set][wall] sum_{out} |xi.n| w S(u_W) / w */
    R kdiff[2][2];                  /* kin - kout, formed in FP64 (zero for a tangential wall) */
    int n_iface;                    /* mode A: interface rows (x-uniform bands) */
    int iface_row[LB_MAX_IFACE];
    SetConst<R> set[2];
};

/* storage codes match LB_STORE_* */
namespace lbk {

/* step kernel layouts: 0 = one node quad per thread (lb_step_impl.cuh),
 * 1 = TMA-fed producer / consumer blocks (lb_step3.cu, FP32 / FP16 / BF16 storage) */
template <typename R>
void launch_step(int store, const StepParams<R> &p, void *stream);
/* layout 6: the one-quad kernel over n block descriptors (p.block_desc) */
template <typename R>
void launch_step_desc(int store, const StepParams<R> &p, int n, void *stream);
/* Split form of the step: a plain kernel over the quads for which plain_quad() holds,
 * in register blocks of 4 x rb nodes (rb = 1 or 2; a block is plain when all its rb
 * quads are), and the one-quad kernel over the listed remaining quads (x0, j) on
 * edge_stream, which the caller forks from and joins back into stream. */
template <typename R>
void launch_step_split(int store, const StepParams<R> &p, int rb, const int2 *edge, int n_edge, void *stream,
                       void *edge_stream);
/* Batched lattices, one persistent launch: params [n][2] launch parameter sets
 * (StepParams of the storage's arithmetic type; [i][0] reads level cur, [i][1] the
 * other level), order [n] the queue order, base the parity of level cur relative to
 * [i][0]; advance = 0 repeats the first step without moving the state. Returns 0 or -1
 * for a bad shape. */
int launch_batch(int store, const void *params, const int *order, int n, int nsteps, int base, int advance,
                 unsigned int *queue, int threads, int grid, void *stream);
/* resident blocks per SM of the batch kernel for a block size (0 on error) */
int batch_blocks(int store, int threads);
/* carried moments (streamed layout) of every node of the written level (list == NULL)
 * or of the listed quads (x0, j), from their stored populations */
template <typename R>
void launch_aux(int store, const StepParams<R> &p, const int2 *list, int n, void *stream);
/* step-kernel layouts: 0 one node quad per thread, 1 TMA-fed producer / consumer,
 * 2 and 3 split plain / edge kernels with register blocks of 4 x 1 and 4 x 2 nodes,
 * 4 streamed (TMA, carried moments, boundary work at the end of each unit), 5 layout 0
 * with its blocks launched in block_order, 6 the same kernel on block_desc (two nodes
 * per thread in high-order bands), 7 layout 0's threads with paired FP32 arithmetic on
 * the rows without boundary work (lb_pair.cuh; FP32 and 16-bit storage), 8 layout 7
 * with its blocks launched in block_order, 9 layout 7's arithmetic fed by a per-thread
 * ring of asynchronous copies, boundary work in the same kernel (lb_ring.cuh), 10 layout
 * 9's arithmetic in a persistent kernel over row units, most expensive first, with the
 * rows without boundary work specialised on the velocity set (lb_ring2.cuh) */
#define LB_NUM_VARIANTS 11
/* layout 7 / 8: p.block_order selects between them (FP32 and 16-bit storage); p.ctab
 * must hold the tables that launch_pair_table wrote for this lattice */
void launch_pair(int store, const StepParams<float> &p, void *stream);
/* layout 9 (FP32 and 16-bit storage; p.ctab as for launch_pair) */
void launch_ring(int store, const StepParams<float> &p, void *stream);
size_t pair_table_bytes();
void launch_pair_table(const StepParams<float> &p, void *dst, void *stream);

/* Layout 10: the per-population constants of one lattice, passed by value in kernel
 * parameter space (read with a warp-uniform index) */
struct alignas(16) RingPop {
    float2 cx2, cy2;      /* (xi_x, xi_x), (xi_y, xi_y) */
    float2 ncx2, nacy2;   /* (-c_x, -c_x), (-|c_y|, -|c_y|): Courant numbers */
    float2 ky2, gxi2;     /* ((1 - |c_y|) / 2, ...), (g.xi, g.xi) */
    float2 w2, winv2;     /* (w, w), (1 / w, 1 / w) */
    float2 wcx2, wcy2;    /* (w xi_x, ...), (w xi_y, ...) */
    float kx;             /* (1 - |c_x|) / 2 */
    int ystep;            /* sign(c_y) x pitch */
    float wxx, wxy, wyy;  /* w (xi_x^2 - 1), w xi_x xi_y, w (xi_y^2 - 1) */
    float hxx, hxy, hyy;  /* (xi_x^2 - 1) / 2, xi_x xi_y, (xi_y^2 - 1) / 2 */
};
struct RingTab {
    RingPop pop[2][LB_QMAX];
};
/* Fills tab from the tables at d_ctab (launch_pair_table) and the set constants of p;
 * synchronises stream. Returns 0, or -1 when a set's populations are not in the order
 * the layout-10 kernel is specialised on (the product rule, ascending abscissae) or a
 * copy failed. */
int ring_tab_build(const void *d_ctab, const StepParams<float> &p, RingTab *tab, void *stream);
/* Layout 10: the row queues of one lattice. rows[] holds work items (row << 16 | kind
 * << 14 | tile; kind 0 lean, 1 edge, 2 general); queue q owns rows[desc[q].x ..
 * desc[q].x + desc[q].y); queues 0 .. nq - 1 belong to SMs (by %smid modulo nq), queue
 * nq is shared. ctr[0 .. nq] count the items taken from each queue, ctr[nq + 1] the
 * warps that have finished; all are zero between launches, and every launch leaves
 * them so. */
struct RowQueues {
    const uint32_t *rows;
    const int2 *desc;
    uint32_t *ctr;
    int nq;
};
/* Batched lattices on layout 10's bodies (FP32 and 16-bit storage, sets of 9 and q1 = 16
 * or 36 populations, lattices at most one tile wide): params [n][2] as for launch_batch,
 * tabs [n], items of lattice i at items[ranges[i].x ..][ranges[i].y] (first row | (rows -
 * 1) << 16 | set << 21 | kind << 22, kind 0 edge, 1 row, 2 general), force when some
 * lattice has a body force. grid
 * 0: the number of resident blocks goes to *grid_out and nothing is launched. Returns 0
 * or -1. */
int launch_ring_batch(int store, int q1, const StepParams<float> *params, const RingTab *tabs, const uint32_t *items,
                      const int2 *ranges, const int *order, int n, int nsteps, int base, int advance,
                      unsigned int *queue, bool force, int grid, int *grid_out, void *stream);
/* Layout 10 (sets of 9 and of 16 or 36 populations), at most nblocks blocks */
void launch_ring_units(int store, const StepParams<float> &p, const RingTab &tab, const RowQueues &rq, int nblocks,
                       void *stream);

/* The quad of nodes x0 .. x0+3 of row j needs none of the boundary work of the step
 * (wall overwrite, ghost-row or ghost-column copies, pressure column, mode-B shadow or
 * mode-A interface row): the plain kernels update it, the one-quad kernel the rest.
 * Host and device share this one definition. */
__host__ __device__ inline bool plain_quad(int x0, int j, uint8_t flags, int nx, int ny, bool periodic_x,
                                           bool periodic_y, bool pressure_lo, bool pressure_hi)
{
    if (flags & (LB_TILE_SHADOW | LB_TILE_IFACE)) return false;
    if (periodic_y ? (j < 2 || j >= ny - 2) : (j == 0 || j == ny - 1)) return false;
    if (x0 + 3 >= nx) return false;
    if (pressure_lo && x0 == 0) return false;
    if (pressure_hi && x0 + 3 >= nx - 1) return false;
    if (periodic_x && (x0 < LB_GHOST || x0 + 3 >= nx - LB_GHOST)) return false;
    return true;
}
template <typename R>
void launch_iface(int store, const StepParams<R> &p, void *stream);
/* D2Q9 stream-and-collide step (Courant number one, periodic, one set) */
template <typename R>
void launch_exact_stream(int store, const StepParams<R> &p, void *stream);
template <typename R>
void launch_pressure(int store, const StepParams<R> &p, void *stream);
template <typename R>
void launch_shadows(int store, const StepParams<R> &p, void *stream);
template <typename R>
void launch_init(int store, const StepParams<R> &p, const double *rho, const double *ux, const double *uy,
                 void *stream);
template <typename R>
void launch_set_pops(int store, const StepParams<R> &p, int set, const double *src, void *stream);
/* compact state (own-set populations only, segment list seg of nseg0 + nseg1 tile rows):
 * pack p.fin into dst, or (unpack != 0) write dst into p.fout with ghost copies */
template <typename R>
void launch_pack(int store, const StepParams<R> &p, const int4 *seg, int nseg0, int nseg1, int qmax, void *dst,
                 int unpack, void *stream);
template <typename R>
void launch_get_pops(int store, const StepParams<R> &p, int set, double *dst, void *stream);
template <typename R>
void launch_moments(int store, const StepParams<R> &p, uint32_t mask, void *dst, int dst_f64, void *stream);
/* partial sums per block into part[nblocks][4]; the last block folds them into out[4]
 * in block order. uprev [ny][nx][2] (R) is read and replaced. */
template <typename R>
void launch_reduce(int store, const StepParams<R> &p, R *uprev, double *part, unsigned int *counter,
                   double *out, int nblocks, void *stream);
int reduce_blocks(int nx, int ny, int nsm);
/* learned placement: features [8][ny][nx] from moment fields [9][ny][nx] (float) */
template <typename R>
void launch_features(const StepParams<R> &p, const float *moments, float *out, void *stream);
/* ||f - P2 f|| / rho per node (beyond-second-order Hermite content), [ny][nx] */
template <typename R>
void launch_hermite_residual(int store, const StepParams<R> &p, float *out, void *stream);
/* per-tile maximum of p [ny][nx] -> out [ny][ntx] */
void launch_tile_max(const float *p, int nx, int ny, int ntx, float *out, void *stream);

}  // namespace lbk
