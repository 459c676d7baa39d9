/*
 * lb.h -- C ABI of the GB300 multiscale lattice Boltzmann library (liblbgb.so).
 *
 * The library advances a 2-D lattice split into regions that use different discrete
 * velocity sets: a low-order Gauss-Hermite set (D2Q9) in the less rarefied part and a
 * high-order one (D2Q36, or D2Q16) near the walls, as in Meng, Zhang & Shan,
 * "Multiscale lattice Boltzmann approach to modeling gas flows":
 *   - velocity sets: roots of Hermite polynomials, weights by Eq. (weight), 2-D sets by
 *     the product rule (Sec. 2.1);
 *   - collision: BGK towards the second-order Hermite equilibrium Eq. (demoeq), with the
 *     body force Eq. (demoforce), relaxation time from the local Knudsen number
 *     (Eq. (KN): collision rate p / mu);
 *   - space-time scheme: forward Euler plus second-order TVD minmod fluxes (Sec. 3.1);
 *   - walls: Maxwell diffuse reflection, ghost node = wall node (Sec. 3.2);
 *   - interface coupling (Sec. 2.2): mode LB_IFACE_PAPER is the paper's virtual
 *     boundary (interpolated rho, u; non-equilibrium part extrapolated from each set's
 *     own side); mode LB_IFACE_HERMITE rebuilds a foreign neighbour in the reader's set
 *     from its Hermite coefficients up to second order (density, momentum and the full
 *     second moment, so the non-equilibrium stress crosses the interface).
 *
 * Units are the paper's nondimensional ones (Eq. (nondime)): lengths in l0, velocities
 * in sqrt(R T0), time in l0 / sqrt(R T0).
 *
 * Conventions shared by every entry point:
 *   - Node (i, j) has x = i h, y = j h; arrays "[ny][nx]" are row-major with x fastest.
 *   - Population order inside a set: alpha = iy * n + ix for the n-point 1-D rule,
 *     abscissae ascending, xi_alpha = (r_ix, r_iy).
 *   - Pointers marked "host" are ordinary host memory; "device" pointers are CUDA
 *     device memory of the current device. The caller keeps ownership of everything
 *     it passes in; inputs are copied before the call returns unless stated.
 *   - Every call returns an lb_status. Errors are sticky per context: after a CUDA or
 *     divergence error, further calls on that context return the same status.
 *     lb_last_error() gives a message for the calling thread's most recent failure.
 *   - Work is enqueued on the context's stream (lb_opts.stream, NULL = legacy default
 *     stream) and is asynchronous unless stated. One context is used by one host
 *     thread at a time.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID = 1,   /* bad argument, map, set, CFL > 1 or dt / tau > 1 */
    LB_ERR_NOMEM = 2,     /* the allocator returned NULL */
    LB_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    LB_ERR_DIVERGED = 4,  /* a reduction found a NaN / Inf density or velocity */
    LB_ERR_TIMEOUT = 5    /* a bounded device wait ran out */
} lb_status;

/* Velocity sets: the number of populations of the product Gauss-Hermite set. */
enum { LB_D2Q9 = 9, LB_D2Q16 = 16, LB_D2Q36 = 36 };

/* Population storage in device memory. The *_DEV forms store the deviation
 * d = f / w_alpha - rho0 from the rest state w_alpha rho0; all forms except
 * LB_STORE_F64 collide in FP32; LB_STORE_F64 computes in FP64. */
enum {
    LB_STORE_F64 = 0,
    LB_STORE_F32 = 1,
    LB_STORE_F32_DEV = 2,
    LB_STORE_F16_DEV = 3,
    LB_STORE_BF16_DEV = 4
};

enum { LB_IFACE_PAPER = 0, LB_IFACE_HERMITE = 1 };

enum { LB_WALL_PERIODIC = 0, LB_WALL_DIFFUSE = 1, LB_WALL_PRESSURE = 2 };

/* Moment fields for lb_moments (bit mask; fields are written in bit order). */
enum {
    LB_M_RHO = 1u << 0,
    LB_M_UX = 1u << 1,
    LB_M_UY = 1u << 2,
    LB_M_PXY = 1u << 3,      /* sum f (xi_x - u_x)(xi_y - u_y) */
    LB_M_NEQ_XX = 1u << 4,   /* sum (f - f_eq) xi_x xi_x */
    LB_M_NEQ_XY = 1u << 5,
    LB_M_NEQ_YY = 1u << 6,
    LB_M_QX = 1u << 7,       /* (1/2) sum f |xi - u|^2 (xi_x - u_x) */
    LB_M_QY = 1u << 8,
    LB_M_ALL = (1u << 9) - 1u
};

/* Grid: nx x ny nodes, spacing h in both directions (h <= 0: 1/(ny-1) when the
 * bottom and top are walls, 1/ny when y is periodic). Time step dt > 0 is taken as
 * given; dt <= 0 means dt = cfl * h / xi_max over the two sets (Sec. 3.1 leaves dt
 * open). nx >= 4, ny >= 4. */
typedef struct {
    int32_t nx, ny;
    double h;
    double cfl;
    double dt;
} lb_grid;

/* One side of the domain, in the order bottom (y = 0), top (y = (ny-1) h), left
 * (x = 0), right (x = (nx-1) h).
 *   LB_WALL_DIFFUSE (bottom / top only): wall node moving at (ux, uy), multiplied by
 *     sin(omega t) when omega > 0 (oscillating plate, Sec. 3.5).
 *   LB_WALL_PRESSURE (left / right only): the column is not evolved; it holds
 *     f_eq(rho, u_inner) + f_neq of the next node inwards.
 *   LB_WALL_PERIODIC: bottom and top together, left and right together. */
typedef struct {
    int32_t kind;
    double ux, uy;
    double rho;
    double omega;
} lb_wall;

/* Relaxation time tau = kn_ref * rho_ref / rho (rho_ref <= 0: tau = kn_ref), minus
 * dt / 2 when tau_mode = 1. */
typedef struct {
    double kn_ref, rho_ref;
    int32_t tau_mode;
} lb_kn;

/* Device memory comes from alloc(bytes, alloc_user) and goes back through
 * free(ptr, alloc_user) when both are set, else from cudaMalloc / cudaFree.
 * stream is a cudaStream_t. reduce_every > 0 runs the mass / residual reduction
 * every that many steps inside lb_step and flags divergence. variant < 0 lets
 * lb_create time the step-kernel layouts on this lattice and keep the fastest
 * (cached per process); 0 .. 10 forces one:
 *   0: one quad of nodes per thread, loads through L1;
 *   1: tiles streamed through shared memory by the tensor memory accelerator, two
 *      passes (FP32 / FP16 / BF16 storage only);
 *   2, 3: boundary-free quads in register blocks of 4 x 1 / 4 x 2 nodes, the rest from
 *      a list on a second stream;
 *   4: single pass on moments carried from the previous step, plane tiles streamed by
 *      the tensor memory accelerator, boundary work at the end of each work unit
 *      (FP32 / FP16 / BF16 storage, LB_IFACE_HERMITE only);
 *   5: layout 0 with the blocks that hold high-order rows launched first (only when
 *      the map has both sets);
 *   6: as 5, with two nodes per thread in the bands that hold rows of a set of 16 or
 *      36 populations (twice the threads on the long population loops);
 *   7: layout 0's threads, with the rows that need no boundary work computed in packed
 *      two-wide FP32 arithmetic on a folded form of the collision (FP32 and 16-bit
 *      storage);
 *   8: as 7, with the block order of 5 (only when the map has both sets);
 *   9: 7's arithmetic on every row, the neighbour rows brought into a per-thread ring
 *      of shared-memory slots by asynchronous copies issued two nodes ahead, wall and
 *      shadow-row updates done by the same kernel (FP32 and 16-bit storage);
 *  10: 9's arithmetic in one persistent launch: warps take rows of 128 columns from
 *      per-SM queues (longest rows first), with the population loop unrolled over the
 *      velocity set (D2Q9 with D2Q16 or D2Q36; FP32 and 16-bit storage).
 * A layout this lattice cannot use falls back to 0. All layouts give the same result
 * (0, 2, 3 and 4 the same bits; 1, 5, 6 the same bits as 0 or differing in rounding;
 * 7, 8 and 9 differ from 0 in rounding; 10 the same bits as 9). */
typedef struct {
    int32_t store;
    int32_t iface;
    double rho0;
    double gx, gy;
    int32_t reduce_every;
    int32_t variant;
    void *stream;
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *alloc_user;
    int32_t rounding;   /* LB_ROUND_NEAREST (0) or LB_ROUND_STOCHASTIC (1), see below */
    const double *rho0_col;   /* NULL, or host [nx]: per-column reference density, see below */
    int32_t scheme;     /* LB_SCHEME_TVD (0) or LB_SCHEME_STREAM (1), see below */
} lb_opts;

/* Update rule. LB_SCHEME_TVD: the Sec. 3.1 forward-Euler + TVD-minmod update, any sets,
 * maps and walls. LB_SCHEME_STREAM: its D2Q9 reduction at Courant number one, where
 * every population moves exactly one node per step and the update is the lattice BGK
 * stream-and-collide (effective viscosity c_s^2 (tau - dt / 2)); needs sets[0] = 9, an
 * all-zero region map, periodic walls on all four sides and dt = h / sqrt(3) (taken
 * when grid.dt is 0; cfl is ignored), else LB_ERR_INVALID. */
enum { LB_SCHEME_TVD = 0, LB_SCHEME_STREAM = 1 };

/* Rounding of the updated populations into FP16 / BF16 deviation storage (other
 * formats ignore it). Nearest (ties to even) loses every per-step increment smaller
 * than half a unit in the last place of the stored deviation, so slow flows stagnate
 * away from the solution; stochastic rounding (to the neighbour above or below with
 * the probabilities that keep the expected stored value exact, random bits from a
 * counter-based hash of node, population and step) keeps them on average. Values set
 * by boundary rules are rounded to nearest. */
enum { LB_ROUND_NEAREST = 0, LB_ROUND_STOCHASTIC = 1 };

/* Per-column reference density (deviation formats F32_DEV / F16_DEV / BF16_DEV only,
 * else LB_ERR_INVALID): column x stores f / w - rho0_col[x] instead of f / w - rho0, so a
 * lattice whose density varies along x (a pressure-driven channel) keeps small stored
 * magnitudes and loses less to 16-bit rounding. The arithmetic and its results in FP32
 * are those of one reference density; only the rounding of the stored values changes.
 * Values must be finite and positive; the array is copied at create. Layouts 0 and 5
 * support it (a forced other layout falls back to 0); batched lattices do not. The
 * compact state (lb_state_*, checkpoints) holds the shifted values, so it belongs to a
 * lattice with the same reference densities. */

typedef struct lb_ctx lb_ctx;

/* Creates a lattice.
 *   region_map: host [ny][nx], 0 = low-order set sets[0], 1 = high-order set sets[1].
 *     The library quantises it to tiles of 128 columns x 1 row: a tile uses the
 *     high-order set if any of its nodes asks for it (lb_effective_map returns the
 *     result). Mode LB_IFACE_PAPER needs every row to use one set across x.
 *   sets: {low, high} population counts, each 9, 16 or 36.
 * The state starts at rest: f = w_alpha rho0. */
int lb_create(const lb_grid *grid, const uint8_t *region_map, const int32_t sets[2], const lb_kn *kn,
              const lb_wall walls[4], const lb_opts *opts, lb_ctx **out);

/* f = f_eq(rho, u) at every node (Eq. (demoeq)), host arrays [ny][nx]; a NULL array
 * means rho0 (rho) or 0 (ux, uy). Synchronous. */
int lb_init_equilibrium(lb_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* Advances n time steps (Sec. 3.1 scheme, Sec. 3.2 walls, Sec. 2.2 coupling),
 * asynchronously on the context's stream. */
int lb_step(lb_ctx *ctx, int64_t n);

/* Moment fields of the current level into dst, laid out [k][ny][nx] for the k-th set
 * bit of mask, as float (dst_f64 = 0) or double. dst is device memory when
 * dst_is_device != 0 (asynchronous), else host memory (synchronous). */
int lb_moments(lb_ctx *ctx, uint32_t mask, void *dst, int32_t dst_is_device, int32_t dst_f64);

/* Runs the reduction on the current level now and returns, synchronously,
 * out[0] = total mass sum rho (FP64), out[1] = residual ||u - u_prev|| / ||u|| against
 * the previous reduction (1 on the first call, which compares with u = 0),
 * out[2] = number of non-finite nodes, out[3] = step count. One wait on the context's
 * stream brings back the results and the device error word together. Errors (sticky):
 * LB_ERR_DIVERGED when a density or velocity is not finite, LB_ERR_TIMEOUT when a
 * bounded device wait of an earlier step ran out, LB_ERR_CUDA when the launch or the
 * copy failed. */
int lb_reductions(lb_ctx *ctx, double out[4]);

/* The tile-quantised map actually run, host [ny][nx] (0 / 1). */
int lb_effective_map(lb_ctx *ctx, uint8_t *dst);

/* Replaces the region map; nodes that change set are rebuilt in the new set from
 * their second-order Hermite coefficients. Synchronous. */
int lb_set_region_map(lb_ctx *ctx, const uint8_t *region_map);

/* Populations of set s (0 low, 1 high) as stored, decoded to f, host
 * double [q_s][ny][nx]. Nodes of the other set hold the set-s view that readers of
 * set s use next to an interface, or unspecified values elsewhere. Synchronous. */
int lb_get_populations(lb_ctx *ctx, int32_t set, double *dst);

/* Sets the populations of the nodes that use set s from host double [q_s][ny][nx]
 * (values at other nodes are ignored), then refreshes interface views. Synchronous. */
int lb_set_populations(lb_ctx *ctx, int32_t set, const double *src);

/* State of the current level for checkpoints and host-resident pipelines, in the
 * storage format and compact: every node's populations in its own set only, tile row
 * by tile row (the size follows from the map: sum over sets of Q_s x tile rows of s x
 * 128 elements). Loading rebuilds what derives from it: ghost copies, mode-B shadow
 * values, mode-A interface rows, pressure columns and carried moments, so a load
 * followed by a step gives the same bits as the step that was never interrupted.
 * lb_state_bytes gives the size; load / store copy from / to host memory through a
 * device staging buffer of that size, on the context's stream. lb_state_store returns
 * once dst holds the state. lb_state_load is asynchronous: it returns once the copy and
 * the rebuild are queued, and src must stay valid and unchanged until the stream has
 * passed them (lb_sync, or any later synchronous call on this context); from pinned
 * memory the copy overlaps other streams' work. LB_ERR_INVALID for a size that does
 * not match. */
int lb_state_bytes(lb_ctx *ctx, size_t *bytes);
int lb_state_load(lb_ctx *ctx, const void *src, size_t bytes);
int lb_state_store(lb_ctx *ctx, void *dst, size_t bytes);

/* Self-test of the bounded waits of the TMA-fed kernels: one thread waits on an
 * mbarrier that nothing completes, gives up after `polls` polls (a poll takes tens of
 * nanoseconds), records a code in a device word and returns; the host reads it back.
 * *expired = 1 when the wait gave up as designed. Nothing faults or hangs: the kernel
 * always returns. LB_ERR_CUDA if the launch or the copy failed. */
int lb_selftest_bounded_wait(void *stream, uint32_t polls, int32_t *expired);

/* Checkpoint file: header (grid, sets, storage, step, time, a hash of the per-column
 * reference densities) + the tile map + the compact state. lb_load returns
 * LB_ERR_INVALID for a file of another lattice (grid, sets, storage, interface mode, dt,
 * h, rho0 or reference densities differ). */
int lb_save(lb_ctx *ctx, const char *path);
int lb_load(lb_ctx *ctx, const char *path);

/* dt, h, step count, time of the current level and the step-kernel layout in use
 * (any pointer may be NULL). */
int lb_info(lb_ctx *ctx, double *dt, double *h, int64_t *step, double *time, int32_t *variant);

/* Waits for the context's stream; returns the sticky status. */
int lb_sync(lb_ctx *ctx);

void lb_destroy(lb_ctx *ctx);

/* Message of the calling thread's most recent error ("" if none). */
const char *lb_last_error(void);

/* ---------------------------------------------------------------------------------
 * Learned interface placement. Sec. 2.2 leaves the switching criterion open (it cites
 * local Knudsen numbers and stress / heat-flux based breakdown parameters). This part
 * lets a small network choose, between steps, which tiles use the high-order set:
 * 8 features per node -> 64 -> 64 -> 1 with GELU (erf form) hidden layers and a sigmoid
 * output p(high-order set needed); trained in FP32, run with BF16 weights and FP32
 * accumulation. Parameters: 4801 floats laid out W1 [64][8], b1 [64], W2 [64][64],
 * b2 [64], W3 [64], b3 [1]; inputs are normalised as (x - mean) / scale.
 * ------------------------------------------------------------------------------- */

/* Features of every node of the current level into device float dst [8][ny][nx]:
 * Pi^neq_xx / rho, Pi^neq_xy / rho, Pi^neq_yy / rho, q_x / rho, q_y / rho, distance to
 * the nearest diffuse wall (in l0), local Kn (kn_ref rho_ref / rho, Eq. (KN)) and
 * Kn |grad rho| / rho (central differences). Asynchronous. */
int lb_features(lb_ctx *ctx, float *dst);

/* Training label source, device float dst [ny][nx]: the part of each node's
 * populations that a second-order Hermite expansion (Eq. (approxf), N = 2) cannot hold,
 * per unit mass: ||f - P2 f|| / rho in the norm ||g||^2 = sum_a g_a^2 / w_a, from the
 * node's own set (0 at equilibrium and for any second-order disturbance). Asynchronous. */
int lb_hermite_residual(lb_ctx *ctx, float *dst);

typedef struct lb_mlp lb_mlp;

/* params: host float [4801]; norm: host float {mean[8], scale[8]} (scale > 0); device
 * memory and stream come from opts (alloc / free / alloc_user / stream; other fields
 * are ignored). */
int lb_mlp_create(const float *params, const float norm[16], const lb_opts *opts, lb_mlp **out);
/* Mean binary cross-entropy gradient over n samples (x: device float [8][n] raw
 * features, column k = sample k; y: device float [n] in {0, 1}) into host grad [4801];
 * the loss into *loss. n <= 2^20. Synchronous. */
int lb_mlp_grad(lb_mlp *m, const float *x, const float *y, int64_t n, float *grad, double *loss);
/* One full-batch Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
int lb_mlp_adam_step(lb_mlp *m, const float *x, const float *y, int64_t n, float lr);
/* Mini-batch Adam training: epochs passes over the n samples in an order shuffled from
 * seed, batches of `batch`; *last_epoch_loss = mean loss over the last epoch. */
int lb_mlp_train(lb_mlp *m, const float *x, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, double *last_epoch_loss);
int lb_mlp_get_params(lb_mlp *m, float *params);
/* p [n] (device) from x [8][n] (device) with the BF16 copy of the weights. Synchronous. */
int lb_mlp_infer(lb_mlp *m, const float *x, int64_t n, float *p);
void lb_mlp_destroy(lb_mlp *m);

/* Attach a network to a lattice (NULL detaches: the map stays as it is). Every `every`
 * steps lb_step evaluates p at every node, takes its maximum per tile, turns a tile
 * high-order when it reaches p_on and back to low-order when it drops below p_off
 * (0 <= p_off < p_on <= 1), keeps the two rows next to each diffuse wall high-order,
 * and rebuilds moved tiles in their new set (as lb_set_region_map). A non-finite p
 * keeps the current map (counted as a fallback). Needs LB_IFACE_HERMITE. The network
 * must outlive its use by the lattice. */
int lb_set_mlp(lb_ctx *ctx, lb_mlp *m, int32_t every, float p_on, float p_off);
/* Run that update now (synchronous). */
int lb_learned_map_now(lb_ctx *ctx);
/* Map updates run, fallbacks taken, and the share of nodes on high-order tiles. */
int lb_map_stats(lb_ctx *ctx, int64_t *updates, int64_t *fallbacks, double *high_fraction);

/* ---------------------------------------------------------------------------------
 * Batched channels. Many small independent lattices (e.g. a sweep of channel heights,
 * Knudsen numbers and wall speeds) advanced together by ONE persistent kernel launch
 * per call instead of one launch per lattice and step. Each lattice is an ordinary
 * context (lb_batch_instance gives it back for lb_moments, lb_get_populations, ...) and
 * takes exactly the steps of lb_step: the batched kernel does the one-quad layout's
 * arithmetic in the same order, so the results are the same bits.
 * ------------------------------------------------------------------------------- */
typedef struct lb_batch lb_batch;

/* n lattices, lattice i described by grids[i], maps[i] (host [ny_i][nx_i]), kn[i],
 * walls[4 i .. 4 i + 3] and opts[i] as for lb_create. All share `sets`, opts.store and
 * opts.rho0; every lattice needs opts.iface = LB_IFACE_HERMITE, reduce_every = 0, walls
 * without oscillation (omega = 0) and no pressure sides (else LB_ERR_INVALID, checked
 * before any device work). The kernel runs on opts[0].stream; device memory comes from
 * opts[0]'s allocator. Lattices start from rest (rho0, u = 0). lb_batch_create times
 * block sizes 128 / 256 / 512 on the batch and keeps the fastest. */
int lb_batch_create(int32_t n, const lb_grid *grids, const uint8_t *const *maps, const int32_t sets[2],
                    const lb_kn *kn, const lb_wall *walls, const lb_opts *opts, lb_batch **out);
/* Every lattice nsteps steps: one persistent launch. Asynchronous. */
int lb_batch_step(lb_batch *b, int64_t nsteps);
/* The same through lb_step on each lattice in turn, one step at a time (the
 * one-launch-per-lattice path, for comparison). */
int lb_batch_step_each(lb_batch *b, int64_t nsteps);
/* Capture lb_batch_step(nsteps) (nsteps even) in a CUDA graph and replay it `replays`
 * times; synchronous. */
int lb_batch_graph(lb_batch *b, int64_t nsteps, int32_t replays);
/* Lattice i (owned by the batch: do not destroy, do not step it alone). */
lb_ctx *lb_batch_instance(lb_batch *b, int32_t i);
/* Block size and persistent grid chosen by the timing at creation. */
int lb_batch_info(lb_batch *b, int32_t *block_threads, int32_t *grid_blocks);
/* Waits for the batch's stream; returns the first sticky lattice status. */
int lb_batch_sync(lb_batch *b);
void lb_batch_destroy(lb_batch *b);

/* Mass / residual reduction that allocates no device memory (the paper has no
 * counterpart: this is for callers that cannot allocate, e.g. code running under a
 * memory budget fixed by its host application, or code whose allocator belongs to
 * another framework and cannot be reached from C). It computes what lb_reductions
 * computes, but on moment fields
 * the caller owns (e.g. filled by lb_moments with dst_is_device = 1, dst_f64 = 1):
 *   rho, ux, uy: device double arrays of n nodes (1 <= n <= LB_NOALLOC_MAX_NODES);
 *   restart != 0: compare with u = 0 instead of the previous call's velocity;
 *   stream: cudaStream_t to run on (NULL = legacy default stream);
 *   out (host): [0] = sum rho (FP64), [1] = ||u - u_prev|| / ||u||, [2] = number of
 *     non-finite nodes, [3] = n.
 * Synchronous: it copies the result to the host and waits for the stream, so it must
 * not be called while that stream is being captured into a CUDA graph. Every node's
 * velocity is kept for the next call, a non-finite one included: after a call that
 * found non-finite nodes, the next call's residual is non-finite unless restart != 0.
 * Returns LB_OK, LB_ERR_INVALID (null pointer, n out of range: nothing is launched),
 * LB_ERR_CUDA, or LB_ERR_DIVERGED (non-finite node; out is still filled); the message is
 * in lb_last_error().
 * Everything it needs beyond its arguments lives in one fixed array inside the library
 * (about 8.1 MB: per-block partial sums and the previous velocity of up to
 * LB_NOALLOC_MAX_NODES nodes), which every GPU that loads the library holds until the
 * process exits. The first call on a device looks up the array's device address on
 * that device. All calls share the
 * array and it keeps the last call's velocity: calls that can overlap on the GPU (other
 * streams, other host threads) race with each other and must be serialised by the
 * caller. */
#define LB_NOALLOC_MAX_NODES 524288
int lb_reduce_fields_noalloc(const double *rho, const double *ux, const double *uy, int64_t n, int32_t restart,
                             void *stream, double out[4]);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
