/*
 * lb_api.cu -- host side of liblbgb.so: the C ABI declared in include/lb.h.
 *
 * Holds the lattice description, builds the velocity-set constants and the tile map,
 * owns the device planes (two time levels per set), and sequences the kernels of one
 * time step: the fused update, then the mode-A interface rows and the pressure
 * columns of the new level, then (every reduce_every steps) the FP64 reduction.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"
#include "lb_mlp.h"
#include "lb_tma.h"

namespace lbq {
int velocity_set(int q, double *cx, double *cy, double *w);
}

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

size_t elem_size(int store)
{
    switch (store) {
        case LB_STORE_F64: return 8;
        case LB_STORE_F32:
        case LB_STORE_F32_DEV: return 4;
        default: return 2;
    }
}

}  // namespace

namespace lbk {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace lbk

struct lb_ctx {
    int nx = 0, ny = 0, pitch = 0, ntx = 0;
    double h = 0.0, dt = 0.0;
    int q[2] = {0, 0};
    double cx[2][LB_QMAX], cy[2][LB_QMAX], w[2][LB_QMAX];
    lb_kn kn{};
    lb_wall walls[4]{};
    lb_opts opts{};
    int store = 0;
    size_t esize = 0;
    void *planes[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   /* [level][set] */
    size_t set_bytes[2] = {0, 0};
    int cur = 0;
    uint8_t *d_tmap = nullptr;
    std::vector<uint8_t> tmap;
    std::vector<int> iface_rows;
    double *d_part = nullptr, *d_out = nullptr;
    unsigned int *d_counter = nullptr;
    void *d_uprev = nullptr;
    double *h_out = nullptr;        /* pinned */
    cudaEvent_t red_event = nullptr;
    bool red_pending = false;
    int red_blocks = 1;
    cudaStream_t stream = nullptr;
    double t = 0.0;
    int64_t step = 0;
    int status = LB_OK;
    int variant = -1;               /* step kernel layout in use (see launch_variant) */
    bool tma_ok = false;            /* tensor maps built (FP32 / FP16 / BF16 storage) */
    TmaMaps maps[2];                /* per time level */
    int *d_err = nullptr;           /* bounded device waits that ran out */
    /* split step: quads left to the one-quad kernel, for register blocks of 1 and 2 rows */
    std::vector<int2> edge_h[2];
    int2 *d_edge[2] = {nullptr, nullptr};
    size_t edge_cap[2] = {0, 0};
    cudaStream_t edge_stream = nullptr;   /* the edge kernel runs here, overlapping */
    /* streamed layout: carried moments per level and work units */
    void *aux[2] = {nullptr, nullptr};
    std::vector<int4> units_h;      /* (tile, first row, rows, set) runs, most work first */
    int4 *d_units = nullptr;
    size_t units_cap = 0;
    unsigned int *d_squeue = nullptr;
    /* one-quad kernel: block launch order, most work first */
    std::vector<int> border_h;
    int *d_border = nullptr;
    size_t border_cap = 0;
    bool border_used = false;       /* false: the order is the raster order */
    /* compact state (lb_state_*, lb_save / lb_load): one segment per tile row of a set */
    std::vector<int4> seg_h;
    int4 *d_seg = nullptr;
    size_t seg_cap = 0;
    int nseg[2] = {0, 0};
    void *d_stage = nullptr;        /* device staging buffer of the compact state */
    size_t stage_cap = 0;
    std::vector<int2> bdesc_h;      /* layout 6 block descriptors */
    int2 *d_bdesc = nullptr;
    size_t bdesc_cap = 0;
    bool bdesc_narrow = false;      /* some band runs two nodes per thread */
    void *d_dcol = nullptr;         /* per-column reference density: delta per storage column (R) */
    void *d_ctab = nullptr;         /* layouts 7 / 8: per-population constant tables */
    int nsm = 0;                    /* SMs of the device */
    bool ring_batch = false;        /* a member of a batch stepped on layout 10's bodies */
    /* layout 10: row queues (per SM and shared), their counters, and the constants
     * passed in kernel-parameter space */
    std::vector<uint32_t> rrows_h;
    std::vector<int2> rdesc_h;
    uint32_t *d_rrows = nullptr;
    size_t rrows_cap = 0;
    int2 *d_rdesc = nullptr;
    uint32_t *d_rctr = nullptr;
    std::unique_ptr<lbk::RingTab> rtab;
    uint32_t dcol_hash = 0;         /* FNV-1a of those deltas (0: one reference density) */
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    /* learned placement */
    lb_mlp *mlp = nullptr;
    int mlp_every = 0;
    float p_on = 0.5f, p_off = 0.3f;
    float *d_mom = nullptr, *d_feat = nullptr, *d_p = nullptr, *d_tp = nullptr;
    int64_t map_updates = 0, map_fallbacks = 0;
    std::vector<void *> owned;
};

namespace {

bool use_f64(const lb_ctx *c) { return c->store == LB_STORE_F64; }

void *dev_alloc(lb_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (c->opts.alloc && c->opts.free) {
        p = c->opts.alloc(bytes, c->opts.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(lb_ctx *c, void *p)
{
    if (!p) return;
    if (c->opts.alloc && c->opts.free) c->opts.free(p, c->opts.alloc_user);
    else cudaFree(p);
}

int cuda_check(lb_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return LB_OK;
    c->status = LB_ERR_CUDA;
    return fail(LB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int launch_check(lb_ctx *c, const char *what) { return cuda_check(c, cudaGetLastError(), what); }

double wall_speed(const lb_wall &wl, double t, int comp)
{
    double u = comp == 0 ? wl.ux : wl.uy;
    if (wl.omega > 0.0) u *= std::sin(wl.omega * t);
    return u;
}

template <typename R>
void fill_set(const lb_ctx *c, int s, SetConst<R> &k)
{
    k.q = c->q[s];
    k.n1d = c->q[s] == 9 ? 3 : c->q[s] == 16 ? 4 : 6;
    for (int a = 0; a < LB_QMAX; ++a) {
        const bool on = a < c->q[s];
        const double x = on ? c->cx[s][a] : 0.0, y = on ? c->cy[s][a] : 0.0, w = on ? c->w[s][a] : 1.0;
        const double crx = x * c->dt / c->h, cry = y * c->dt / c->h;
        k.cx[a] = R(x);
        k.cy[a] = R(y);
        k.w[a] = R(w);
        k.winv[a] = R(1.0 / w);
        k.wcx[a] = R(w * x);
        k.wcy[a] = R(w * y);
        k.crx[a] = R(crx);
        k.cry[a] = R(cry);
        k.kx[a] = R(0.5 * (1.0 - std::fabs(crx)));
        k.ky[a] = R(0.5 * (1.0 - std::fabs(cry)));
        k.wxx[a] = R(w * (x * x - 1.0));
        k.wxy[a] = R(w * x * y);
        k.wyy[a] = R(w * (y * y - 1.0));
        k.hxx[a] = R(0.5 * (x * x - 1.0));
        k.hxy[a] = R(x * y);
        k.hyy[a] = R(0.5 * (y * y - 1.0));
    }
}

/* Launch parameters; level `in` is read, level `out` written; walls at time t_new. */
template <typename R>
StepParams<R> make_params(const lb_ctx *c, int in, int out, double t_new)
{
    StepParams<R> p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.h_grid = c->h;
    p.pitch = c->pitch;
    p.ntx = c->ntx;
    p.tmap = c->d_tmap;
    const size_t row0 = (size_t)LB_GHOST_ROWS * c->pitch * c->esize;   /* logical row 0 */
    for (int s = 0; s < 2; ++s) {
        p.fin[s] = static_cast<const char *>(c->planes[in][s]) + row0;
        p.fout[s] = static_cast<char *>(c->planes[out][s]) + row0;
    }
    p.plane = (size_t)(c->ny + 2 * LB_GHOST_ROWS) * c->pitch;
    p.sr = (c->opts.rounding == LB_ROUND_STOCHASTIC &&
            (c->store == LB_STORE_F16_DEV || c->store == LB_STORE_BF16_DEV)) ? 1 : 0;
    p.step_key = (uint32_t)(c->step + (in != out ? 1 : 0));
    p.block_order = nullptr;   /* layout 5 sets it */
    p.block_desc = nullptr;    /* layout 6 sets it */
    p.dcol = static_cast<const R *>(c->d_dcol);
    p.ctab = c->d_ctab;
    p.aux_in = c->aux[in];
    p.aux_out = c->aux[out];
    p.rho0 = R(c->opts.rho0);
    p.dt = R(c->dt);
    p.tau_const = c->kn.rho_ref > 0.0 ? 0 : 1;
    p.kn_rho = R(c->kn.rho_ref > 0.0 ? c->kn.kn_ref * c->kn.rho_ref : c->kn.kn_ref);
    p.tau_shift = R(c->kn.tau_mode == 1 ? 0.5 * c->dt : 0.0);
    p.gx = R(c->opts.gx);
    p.gy = R(c->opts.gy);
    p.has_force = (c->opts.gx != 0.0 || c->opts.gy != 0.0) ? 1 : 0;
    p.periodic_x = c->walls[2].kind == LB_WALL_PERIODIC;
    p.periodic_y = c->walls[0].kind == LB_WALL_PERIODIC;
    for (int side = 0; side < 2; ++side) {
        p.wall_diffuse[side] = c->walls[side].kind == LB_WALL_DIFFUSE;
        p.pressure[side] = c->walls[2 + side].kind == LB_WALL_PRESSURE;
        p.rho_side[side] = R(c->walls[2 + side].rho);
        const double ux = wall_speed(c->walls[side], t_new, 0), uy = wall_speed(c->walls[side], t_new, 1);
        p.uw_x[side] = R(ux);
        p.uw_y[side] = R(uy);
        const double nsg = side == 0 ? 1.0 : -1.0;
        for (int s = 0; s < 2; ++s) {
            /* kin - kout = -sum_out |xi.n| w (S / w - 1), summed as such (no cancellation) */
            double kin = 0.0, kout = 0.0, kdiff = 0.0;
            for (int a = 0; a < c->q[s]; ++a) {
                const double xn = c->cy[s][a] * nsg;
                const double ew = c->cx[s][a] * ux + c->cy[s][a] * uy;
                const double sm1 = ew + 0.5 * (ew * ew - (ux * ux + uy * uy));
                if (xn < 0.0) kin += -xn * c->w[s][a];
                if (xn > 0.0) {
                    kout += xn * c->w[s][a] * (1.0 + sm1);
                    kdiff -= xn * c->w[s][a] * sm1;
                }
            }
            p.kin[s][side] = R(kin);
            p.kout[s][side] = R(kout);
            p.kdiff[s][side] = R(kdiff);
        }
    }
    p.n_iface = (int)c->iface_rows.size();
    for (int k = 0; k < p.n_iface && k < LB_MAX_IFACE; ++k) p.iface_row[k] = c->iface_rows[k];
    fill_set(c, 0, p.set[0]);
    fill_set(c, 1, p.set[1]);
    return p;
}

/* Tile flags from a per-node map; mode A rows and validation. */
int build_tiles(lb_ctx *c, const uint8_t *map, std::vector<uint8_t> &tm, std::vector<int> &rows)
{
    const int nx = c->nx, ny = c->ny, ntx = c->ntx;
    tm.assign((size_t)ny * ntx, 0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const uint8_t v = map[(size_t)j * nx + i];
            if (v > 1) return fail(LB_ERR_INVALID, "region map values must be 0 or 1");
            if (v) tm[(size_t)j * ntx + i / LB_TILE_X] |= LB_TILE_HIGH;
        }
    const bool px = c->walls[2].kind == LB_WALL_PERIODIC, py = c->walls[0].kind == LB_WALL_PERIODIC;
    auto hi = [&](int tx, int j) -> int {
        if (py) j = (j % ny + ny) % ny;
        else if (j < 0 || j >= ny) return -1;
        if (px) tx = (tx % ntx + ntx) % ntx;
        else if (tx < 0 || tx >= ntx) return -1;
        return tm[(size_t)j * ntx + tx] & LB_TILE_HIGH;
    };
    rows.clear();
    if (c->opts.iface == LB_IFACE_HERMITE) {
        for (int j = 0; j < ny; ++j)
            for (int tx = 0; tx < ntx; ++tx) {
                const int s = hi(tx, j);
                bool sh = false;
                for (int d = -2; d <= 2; ++d) {
                    if (d == 0) continue;
                    const int o = hi(tx, j + d);
                    if (o >= 0 && o != s) sh = true;
                }
                for (int d = -1; d <= 1; d += 2) {
                    const int o = hi(tx + d, j);
                    if (o >= 0 && o != s) sh = true;
                }
                if (sh) tm[(size_t)j * ntx + tx] |= LB_TILE_SHADOW;
            }
        return LB_OK;
    }
    /* mode A: x-uniform rows; interface row = low-order row next to a high-order row */
    if (c->walls[2].kind == LB_WALL_PRESSURE || c->walls[3].kind == LB_WALL_PRESSURE)
        return fail(LB_ERR_INVALID, "LB_IFACE_PAPER does not combine with pressure columns");
    std::vector<int> rs(ny);
    for (int j = 0; j < ny; ++j) {
        rs[j] = hi(0, j);
        for (int tx = 1; tx < ntx; ++tx)
            if (hi(tx, j) != rs[j]) return fail(LB_ERR_INVALID, "LB_IFACE_PAPER needs every row in one set");
    }
    for (int j = 0; j < ny; ++j) {
        if (rs[j] != 0) continue;
        const int below = (j > 0 || py) ? rs[(j - 1 + ny) % ny] : -1;
        const int above = (j < ny - 1 || py) ? rs[(j + 1) % ny] : -1;
        if (below == 1 && above == 1) return fail(LB_ERR_INVALID, "low-order band one row thick");
        if (below == 1 || above == 1) {
            const int jl = below == 1 ? j + 1 : j - 1;
            if (jl < 0 || jl >= ny || rs[jl] != 0) return fail(LB_ERR_INVALID, "interface row without a low-order side");
            if (j == 0 || j == ny - 1) return fail(LB_ERR_INVALID, "interface row on a wall");
            rows.push_back(j);
            for (int tx = 0; tx < ntx; ++tx)
                tm[(size_t)j * ntx + tx] |= LB_TILE_IFACE | (below == 1 ? LB_TILE_NEAR_H : 0);
        }
    }
    for (size_t a = 0; a < rows.size(); ++a)
        for (size_t b = a + 1; b < rows.size(); ++b)
            if (std::abs(rows[a] - rows[b]) < 4) return fail(LB_ERR_INVALID, "interface rows closer than 4 rows");
    for (int r : rows) {
        const int jl = (tm[(size_t)r * ntx] & LB_TILE_NEAR_H) ? r + 1 : r - 1;
        for (int r2 : rows)
            if (jl == r2) return fail(LB_ERR_INVALID, "interface rows share a neighbour");
    }
    if ((int)rows.size() > LB_MAX_IFACE) return fail(LB_ERR_INVALID, "too many interface rows");
    return LB_OK;
}

template <typename R>
int finalize_level_t(lb_ctx *c, int level)
{
    StepParams<R> p = make_params<R>(c, level, level, c->t);
    void *st = c->stream;
    if (c->opts.iface == LB_IFACE_HERMITE) lbk::launch_shadows<R>(c->store, p, st);
    lbk::launch_iface<R>(c->store, p, st);
    lbk::launch_pressure<R>(c->store, p, st);
    /* carried moments of this level: read only by layouts 4 and 10 (and by the
     * autotuner, which runs while no layout is chosen yet) */
    if (c->variant < 0 || c->variant == 4 || c->variant == 10 || c->ring_batch)
        lbk::launch_aux<R>(c->store, p, nullptr, 0, st);
    return launch_check(c, "finalize");
}

int finalize_level(lb_ctx *c, int level)
{
    return use_f64(c) ? finalize_level_t<double>(c, level) : finalize_level_t<float>(c, level);
}

void *own(lb_ctx *c, size_t bytes);

/* Compact state: every node's populations in its own set, one segment per tile row of
 * a set (sets in order, rows and tiles ascending; mode-A interface rows are rebuilt, not
 * stored). See pack_kernel for the byte layout. */
void compact_segments(const lb_ctx *c, const std::vector<uint8_t> &tm, std::vector<int4> &seg, int nseg[2])
{
    seg.clear();
    nseg[0] = nseg[1] = 0;
    for (int s = 0; s < 2; ++s)
        for (int j = 0; j < c->ny; ++j)
            for (int tx = 0; tx < c->ntx; ++tx) {
                const uint8_t f = tm[(size_t)j * c->ntx + tx];
                if ((f & LB_TILE_IFACE) || (f & LB_TILE_HIGH) != s) continue;
                seg.push_back(make_int4(tx, j, s, nseg[s]++));
            }
}

size_t compact_bytes(const lb_ctx *c, const int nseg[2])
{
    return ((size_t)c->q[0] * nseg[0] + (size_t)c->q[1] * nseg[1]) * LB_TILE_X * c->esize;
}

/* the staging buffer of the compact state, grown as needed */
int ensure_stage(lb_ctx *c, size_t bytes)
{
    if (bytes <= c->stage_cap) return LB_OK;
    void *d = own(c, bytes);
    if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
    c->d_stage = d;
    c->stage_cap = bytes;
    return LB_OK;
}

template <typename R>
void launch_pack_t(lb_ctx *c, int unpack)
{
    lbk::launch_pack<R>(c->store, make_params<R>(c, c->cur, c->cur, c->t), c->d_seg, c->nseg[0], c->nseg[1],
                        std::max(c->q[0], c->q[1]), c->d_stage, unpack, c->stream);
}

/* Lists of the quads the plain kernels of the split step leave to the one-quad kernel:
 * every quad of a 4 x rb block that is not plain as a whole (plain_quad(), shared with
 * the device), except mode-A interface rows, which no step kernel updates. */
int build_edge_lists(lb_ctx *c)
{
    const bool px = c->walls[2].kind == LB_WALL_PERIODIC, py = c->walls[0].kind == LB_WALL_PERIODIC;
    const bool pl = c->walls[2].kind == LB_WALL_PRESSURE, ph = c->walls[3].kind == LB_WALL_PRESSURE;
    for (int v = 0; v < 2; ++v) {
        const int rb = v + 1;
        std::vector<int2> &L = c->edge_h[v];
        L.clear();
        for (int j0 = 0; j0 < c->ny; j0 += rb)
            for (int x0 = 0; x0 < c->nx; x0 += 4) {
                const int tile = x0 / LB_TILE_X;
                const uint8_t f0 = c->tmap[(size_t)j0 * c->ntx + tile];
                bool plain = j0 + rb <= c->ny;
                for (int r = 0; r < rb && plain; ++r) {
                    const uint8_t fr = c->tmap[(size_t)(j0 + r) * c->ntx + tile];
                    plain = fr == f0 && lbk::plain_quad(x0, j0 + r, fr, c->nx, c->ny, px, py, pl, ph);
                }
                if (plain) continue;
                for (int r = 0; r < rb && j0 + r < c->ny; ++r)
                    if (!(c->tmap[(size_t)(j0 + r) * c->ntx + tile] & LB_TILE_IFACE)) L.push_back(make_int2(x0, j0 + r));
            }
        if (L.empty()) continue;
        if (L.size() > c->edge_cap[v]) {
            const size_t cap = std::max(L.size(), 2 * c->edge_cap[v]);
            int2 *d = static_cast<int2 *>(own(c, cap * sizeof(int2)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_edge[v] = d;
            c->edge_cap[v] = cap;
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_edge[v], L.data(), L.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                                  c->stream), "edge list upload"))
            return e;
    }
    /* launch order of the one-quad kernel's blocks for layout 5 (one tile x LB_STEP_BY
     * rows): blocks with a high-order row first, so that the long blocks are all in the
     * first wave, raster order within each group. Few waves: the tail shrinks; many
     * waves over a lattice larger than L2: the raster order, which mixes long and short
     * blocks, can be faster. The autotuner decides; layout 5 is not offered when the
     * order is the raster order. */
    {
        const int nby = (c->ny + LB_STEP_BY - 1) / LB_STEP_BY;
        std::vector<int> &B = c->border_h;
        std::vector<int> key((size_t)nby * c->ntx);
        B.resize(key.size());
        for (int by = 0; by < nby; ++by)
            for (int tx = 0; tx < c->ntx; ++tx) {
                int qmax = 0;
                for (int j = by * LB_STEP_BY; j < std::min(c->ny, (by + 1) * LB_STEP_BY); ++j) {
                    const uint8_t f = c->tmap[(size_t)j * c->ntx + tx];
                    if (!(f & LB_TILE_IFACE)) qmax = std::max(qmax, c->q[f & LB_TILE_HIGH]);
                }
                const int b = by * c->ntx + tx;
                B[b] = b;
                key[b] = qmax;
            }
        std::stable_sort(B.begin(), B.end(), [&](int a, int b) { return key[a] > key[b]; });
        c->border_used = false;
        for (size_t k = 0; k < B.size() && !c->border_used; ++k) c->border_used = B[k] != (int)k;
        if (B.size() > c->border_cap) {
            int *d = static_cast<int *>(own(c, B.size() * sizeof(int)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_border = d;
            c->border_cap = B.size();
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_border, B.data(), B.size() * sizeof(int), cudaMemcpyHostToDevice,
                                                  c->stream), "block order upload"))
            return e;
    }
    /* layout 10 row queues. Rows are grouped in block units of LB_STEP_BY rows of a tile,
     * the units sorted most work first (raster order among equals) and dealt round-robin
     * to one queue per SM, the last tenth to the shared queue; within a queue the rows
     * are then sorted by their own work, longest first (stable: the rows of a unit stay
     * together among equals). Row kinds (the kernel's RING_*): lean (no boundary work;
     * pressure columns count as none), row (diffuse wall, ghost-row copies, shadow or
     * periodic ghost columns), edge (a tile ending inside the last 128 columns, no
     * boundary work), general (stochastic rounding, or boundary work in such a tile);
     * mode-A interface rows are left out. Work of a row, in units of a population of
     * a lean row: its set size, times 1.25 with a wall, ghost rows or ghost columns, plus
     * twice the other set's size for a shadow; edge rows count 1.5, general rows 2. */
    c->rrows_h.clear();
    c->rdesc_h.clear();
    if (c->nsm > 0 && c->ny <= 0xffff && c->ntx <= 0x3fff) {
        const bool sr = c->opts.rounding == LB_ROUND_STOCHASTIC &&
                        (c->store == LB_STORE_F16_DEV || c->store == LB_STORE_BF16_DEV);
        const int nby = (c->ny + LB_STEP_BY - 1) / LB_STEP_BY;
        struct Row {
            int cost;
            uint32_t item;
        };
        struct Unit {
            int cost;
            Row rows[LB_STEP_BY];
            int n;
        };
        std::vector<Unit> K;
        for (int by = 0; by < nby; ++by)
            for (int tx = 0; tx < c->ntx; ++tx) {
                Unit u{0, {}, 0};
                const bool ragged = (tx + 1) * LB_TILE_X > c->nx;
                const bool gcols = px && (tx == 0 || (tx + 1) * LB_TILE_X > c->nx - LB_GHOST);
                for (int j = by * LB_STEP_BY; j < std::min(c->ny, (by + 1) * LB_STEP_BY); ++j) {
                    const uint8_t f = c->tmap[(size_t)j * c->ntx + tx];
                    if (f & LB_TILE_IFACE) continue;
                    const int q = c->q[f & LB_TILE_HIGH], qt = c->q[(f & LB_TILE_HIGH) ^ 1];
                    const bool images = py ? (j < 2 || j >= c->ny - 2) : (j == 0 || j == c->ny - 1);
                    const bool shadow = f & LB_TILE_SHADOW;
                    const bool boundary = images || shadow || gcols;
                    const uint32_t kind = sr ? 3u : ragged ? (boundary ? 3u : 1u) : boundary ? 2u : 0u;
                    int cost = 4 * q;
                    if (kind == 2u) cost = 5 * q + (shadow ? 8 * qt : 0);
                    if (kind == 1u) cost = 6 * q;
                    if (kind == 3u) cost = 8 * q;
                    u.cost += cost;
                    u.rows[u.n++] = Row{cost, ((uint32_t)j << 16) | (kind << 14) | (uint32_t)tx};
                }
                if (u.n > 0) K.push_back(u);
            }
        std::stable_sort(K.begin(), K.end(), [](const Unit &a, const Unit &b) { return a.cost > b.cost; });
        const int nq = c->nsm;
        const size_t shared_from = K.size() - K.size() / 10;
        std::vector<std::vector<Row>> Qs(nq + 1);
        for (size_t i = 0; i < K.size(); ++i) {
            std::vector<Row> &dst = i < shared_from ? Qs[i % nq] : Qs[nq];
            dst.insert(dst.end(), K[i].rows, K[i].rows + K[i].n);
        }
        for (auto &q : Qs) {
            std::stable_sort(q.begin(), q.end(), [](const Row &a, const Row &b) { return a.cost > b.cost; });
            c->rdesc_h.push_back(make_int2((int)c->rrows_h.size(), (int)q.size()));
            for (const Row &r : q) c->rrows_h.push_back(r.item);
        }
    }
    if (!c->rrows_h.empty()) {
        if (!c->d_rctr) {   /* counters: zero between launches */
            c->d_rctr = static_cast<uint32_t *>(own(c, sizeof(uint32_t) * (c->nsm + 2)));
            c->d_rdesc = static_cast<int2 *>(own(c, sizeof(int2) * (c->nsm + 1)));
            if (!c->d_rctr || !c->d_rdesc) return fail(LB_ERR_NOMEM, "device allocation failed");
            if (int e = cuda_check(c, cudaMemsetAsync(c->d_rctr, 0, sizeof(uint32_t) * (c->nsm + 2), c->stream),
                                   "row queue counters"))
                return e;
        }
        if (c->rrows_h.size() > c->rrows_cap) {
            const size_t cap = std::max(c->rrows_h.size(), 2 * c->rrows_cap);
            uint32_t *d = static_cast<uint32_t *>(own(c, cap * sizeof(uint32_t)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_rrows = d;
            c->rrows_cap = cap;
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_rrows, c->rrows_h.data(), c->rrows_h.size() * sizeof(uint32_t),
                                                  cudaMemcpyHostToDevice, c->stream), "row queue upload"))
            return e;
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_rdesc, c->rdesc_h.data(), c->rdesc_h.size() * sizeof(int2),
                                                  cudaMemcpyHostToDevice, c->stream), "row queue upload"))
            return e;
    }
    /* compact-state segments */
    compact_segments(c, c->tmap, c->seg_h, c->nseg);
    if (!c->seg_h.empty()) {
        if (c->seg_h.size() > c->seg_cap) {
            int4 *d = static_cast<int4 *>(own(c, c->seg_h.size() * sizeof(int4)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_seg = d;
            c->seg_cap = c->seg_h.size();
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_seg, c->seg_h.data(), c->seg_h.size() * sizeof(int4),
                                                  cudaMemcpyHostToDevice, c->stream), "segment list upload"))
            return e;
    }
    /* layout 6: a band of LB_STEP_BY rows holding a row of a set with 16 or more
     * populations runs as two blocks of 4 rows with two nodes per thread; these come
     * first, then the other bands, raster order within each group */
    {
        const int nby = (c->ny + LB_STEP_BY - 1) / LB_STEP_BY;
        std::vector<int2> &D = c->bdesc_h;
        std::vector<int2> wide;
        D.clear();
        for (int by = 0; by < nby; ++by)
            for (int tx = 0; tx < c->ntx; ++tx) {
                bool high = false;
                for (int j = by * LB_STEP_BY; j < std::min(c->ny, (by + 1) * LB_STEP_BY); ++j) {
                    const uint8_t f = c->tmap[(size_t)j * c->ntx + tx];
                    if (!(f & LB_TILE_IFACE) && c->q[f & LB_TILE_HIGH] >= 16) high = true;
                }
                const int j0 = by * LB_STEP_BY;
                if (high) {
                    for (int h = 0; h < LB_STEP_BY && j0 + h < c->ny; h += 4) D.push_back(make_int2(tx, 2 * (j0 + h) + 1));
                } else {
                    wide.push_back(make_int2(tx, 2 * j0));
                }
            }
        c->bdesc_narrow = !D.empty();
        D.insert(D.end(), wide.begin(), wide.end());
        if (D.size() > c->bdesc_cap) {
            int2 *d = static_cast<int2 *>(own(c, D.size() * sizeof(int2)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_bdesc = d;
            c->bdesc_cap = D.size();
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_bdesc, D.data(), D.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                                  c->stream), "block descriptor upload"))
            return e;
    }
    /* work units of the streamed layout: runs of one set in a tile column, at most
     * stream_rows() rows each, most work (populations x rows) first */
    std::vector<int4> &U = c->units_h;
    U.clear();
    const int th = lbk::stream_rows();
    for (int tx = 0; tx < c->ntx; ++tx) {
        int j = 0;
        while (j < c->ny) {
            const int s = c->tmap[(size_t)j * c->ntx + tx] & LB_TILE_HIGH;
            int k = j;
            while (k < c->ny && k - j < th && (c->tmap[(size_t)k * c->ntx + tx] & LB_TILE_HIGH) == s) ++k;
            U.push_back(make_int4(tx, j, k - j, s));
            j = k;
        }
    }
    std::stable_sort(U.begin(), U.end(), [&](const int4 &a, const int4 &b) {
        return (long long)c->q[a.w] * a.z > (long long)c->q[b.w] * b.z;
    });
    if (!U.empty()) {
        if (U.size() > c->units_cap) {
            const size_t cap = std::max(U.size(), 2 * c->units_cap);
            int4 *d = static_cast<int4 *>(own(c, cap * sizeof(int4)));
            if (!d) return fail(LB_ERR_NOMEM, "device allocation failed");
            c->d_units = d;
            c->units_cap = cap;
        }
        if (int e = cuda_check(c, cudaMemcpyAsync(c->d_units, U.data(), U.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                                  c->stream), "unit list upload"))
            return e;
    }
    return LB_OK;
}

int upload_tiles(lb_ctx *c)
{
    if (int e = cuda_check(c, cudaMemcpyAsync(c->d_tmap, c->tmap.data(), c->tmap.size(), cudaMemcpyHostToDevice,
                                              c->stream), "tile map upload"))
        return e;
    return build_edge_lists(c);
}

/* variant 0: one node quad per thread (lb_step_impl.cuh); 1: TMA-fed producer /
 * consumer blocks (lb_step3.cu, not for FP64 storage); 2, 3: split step, plain kernel
 * on 4 x 1 or 4 x 2 register blocks plus the one-quad kernel on the edge list
 * (lb_step_impl.cuh); 4: streamed (lb_stream.cu); 5: variant 0 with the blocks that
 * hold high-order rows launched first; 6: as 5, with two nodes per thread in the bands
 * that hold high-order rows; 7: layout 0's threads with paired FP32 arithmetic on the
 * rows without boundary work (lb_pair.cuh); 8: 7 with the block order of 5; 9: 7's
 * arithmetic fed by a per-thread ring of asynchronous copies (lb_ring.cuh). */
template <typename R>
void launch_variant(lb_ctx *c, int variant, const StepParams<R> &p)
{
    if constexpr (std::is_same<R, float>::value) {
        if (variant == 1 && c->tma_ok && lbk::launch_step3(c->store, p, c->maps[c->cur], c->d_err, c->stream) == 0)
            return;
    }
    if constexpr (std::is_same<R, float>::value) {
        if (variant == 4 && c->tma_ok &&
            lbk::launch_stream(c->store, p, c->maps[c->cur], c->d_units, (int)c->units_h.size(), c->d_squeue, c->d_err,
                               c->stream) == 0) {
            return;
        }
    }
    if (variant == 2 || variant == 3) {
        const int v = variant - 2;
        const int n = (int)c->edge_h[v].size();
        if (n > 0) {
            cudaEventRecord(c->ev_fork, c->stream);
            cudaStreamWaitEvent(c->edge_stream, c->ev_fork, 0);
        }
        lbk::launch_step_split<R>(c->store, p, v + 1, c->d_edge[v], n, c->stream, c->edge_stream);
        if (n > 0) {
            cudaEventRecord(c->ev_join, c->edge_stream);
            cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        }
        return;
    }
    if constexpr (std::is_same<R, float>::value) {
        if (variant == 7 || variant == 8) {
            StepParams<R> q = p;
            if (variant == 8 && c->border_used) q.block_order = c->d_border;
            lbk::launch_pair(c->store, q, c->stream);
            return;
        }
        if (variant == 9) {
            lbk::launch_ring(c->store, p, c->stream);
            return;
        }
        if (variant == 10) {
            const lbk::RowQueues rq{c->d_rrows, c->d_rdesc, c->d_rctr, c->nsm};
            lbk::launch_ring_units(c->store, p, *c->rtab, rq, (int)((c->rrows_h.size() + 7) / 8), c->stream);
            return;
        }
    }
    if (variant == 6 && c->bdesc_narrow) {
        StepParams<R> q = p;
        q.block_desc = c->d_bdesc;
        lbk::launch_step_desc<R>(c->store, q, (int)c->bdesc_h.size(), c->stream);
        return;
    }
    if (variant == 5 && c->border_used) {
        StepParams<R> q = p;
        q.block_order = c->d_border;
        lbk::launch_step<R>(c->store, q, c->stream);
        return;
    }
    lbk::launch_step<R>(c->store, p, c->stream);
}

/* layouts this context can run */
bool variant_available(const lb_ctx *c, int v)
{
    if (c->d_dcol && v != 0 && v != 5 && v != 7 && v != 8 && v != 9 && v != 10) return false;   /* per-column reference density */
    if (v == 7 || v == 8 || v == 9 || v == 10) {
        /* paired FP32 arithmetic: FP32 and 16-bit storage, 32-bit element offsets */
        const size_t span = std::max(c->q[0], c->q[1]) * (size_t)(c->ny + 2 * LB_GHOST_ROWS) * c->pitch;
        if (use_f64(c) || !c->d_ctab || span >= (1ull << 32)) return false;
        if (v == 10)   /* D2Q9 with D2Q16 or D2Q36, constants checked, rows listed */
            return c->rtab && c->d_rctr && c->q[0] == 9 && (c->q[1] == 16 || c->q[1] == 36) && !c->rrows_h.empty();
        return v != 8 || c->border_used;
    }
    if (v == 1) return c->tma_ok;
    if (v == 2 || v == 3) return c->edge_stream != nullptr;
    if (v == 4) return c->tma_ok && c->opts.iface == LB_IFACE_HERMITE;
    if (v == 5) return c->border_used;
    if (v == 6) return c->bdesc_narrow;
    return v >= 0 && v < LB_NUM_VARIANTS;
}

/* Autotuner: times every step-kernel layout on this lattice (reading the current level,
 * writing the other one, which the next step overwrites) and keeps the fastest. Results
 * are cached per (storage, grid, sets, interface mode, map) for the process. */
using TuneKey = std::tuple<int, int, int, int, int, int, uint64_t>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

template <typename R>
int autotune_t(lb_ctx *c)
{
    uint64_t hsh = 1469598103934665603ull;
    for (uint8_t b : c->tmap) hsh = (hsh ^ b) * 1099511628211ull;
    if (c->d_dcol) hsh = (hsh ^ 0x9e3779b97f4a7c15ull) * 1099511628211ull;   /* fewer layouts available */
    /* the rounding and the body force change which layout is fastest */
    hsh = (hsh ^ (uint64_t)(c->opts.rounding + 2 * (c->opts.gx != 0.0 || c->opts.gy != 0.0))) * 1099511628211ull;
    TuneKey key{c->store, c->nx, c->ny, c->q[0], c->q[1], c->opts.iface, hsh};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    StepParams<R> p = make_params<R>(c, c->cur, c->cur ^ 1, c->t + c->dt);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int best = 0;
    float best_ms = 1e30f;
    /* under stochastic rounding every row of layout 10 takes layout 9's body: not offered */
    const bool sr = c->opts.rounding == LB_ROUND_STOCHASTIC &&
                    (c->store == LB_STORE_F16_DEV || c->store == LB_STORE_BF16_DEV);
    for (int v = 0; v < LB_NUM_VARIANTS; ++v) {
        if (!variant_available(c, v) || (v == 10 && sr)) continue;
        /* with the pressure pass, which layout 10 does inside its kernel when the lattice
         * has no body force */
        auto one = [&] {
            launch_variant<R>(c, v, p);
            if (v != 10 || p.has_force) lbk::launch_pressure<R>(c->store, p, c->stream);
        };
        for (int k = 0; k < 2; ++k) one();
        cudaEventRecord(e0, c->stream);
        for (int k = 0; k < 5; ++k) one();
        cudaEventRecord(e1, c->stream);
        float ms = 0.0f;
        /* A later layout must win by more than 3 %: closer timings are within the noise of
         * five launches, and a layout that wins alone by that little can lose when several
         * lattices step concurrently. */
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < 0.97f * best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return 0;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = best;
    return best;
}

int choose_variant(lb_ctx *c)
{
    if (c->opts.scheme == LB_SCHEME_STREAM) return 0;   /* one kernel */
    if (c->opts.variant >= 0) return variant_available(c, c->opts.variant) ? c->opts.variant : 0;
    return use_f64(c) ? autotune_t<double>(c) : autotune_t<float>(c);
}


int ensure_learned_buffers(lb_ctx *c)
{
    const size_t N = (size_t)c->nx * c->ny;
    /* each buffer on its own, so a failed allocation is retried by the next call (what
     * did succeed stays owned by the context) */
    if (!c->d_mom) c->d_mom = static_cast<float *>(own(c, 9 * N * sizeof(float)));
    if (!c->d_feat) c->d_feat = static_cast<float *>(own(c, 8 * N * sizeof(float)));
    if (!c->d_p) c->d_p = static_cast<float *>(own(c, N * sizeof(float)));
    if (!c->d_tp) c->d_tp = static_cast<float *>(own(c, (size_t)c->ny * c->ntx * sizeof(float)));
    if (!c->d_mom || !c->d_feat || !c->d_p || !c->d_tp) return fail(LB_ERR_NOMEM, "device allocation failed");
    return LB_OK;
}

template <typename R>
int features_t(lb_ctx *c, float *dst)
{
    StepParams<R> p = make_params<R>(c, c->cur, c->cur, c->t);
    lbk::launch_moments<R>(c->store, p, LB_M_ALL, c->d_mom, 0, c->stream);
    lbk::launch_features<R>(p, c->d_mom, dst, c->stream);
    return launch_check(c, "features");
}

int features(lb_ctx *c, float *dst)
{
    if (int e = ensure_learned_buffers(c)) return e;
    return use_f64(c) ? features_t<double>(c, dst) : features_t<float>(c, dst);
}

int set_region_map_impl(lb_ctx *c, const uint8_t *map);

/* Learned placement: p for every node, its maximum per tile, then a tile turns
 * high-order at p >= p_on and back to low-order at p < p_off (hysteresis); the two rows
 * next to each diffuse wall stay high-order. Any non-finite p keeps the current map. */
int learned_update(lb_ctx *c)
{
    /* allocate first: the feature buffer is the destination passed below */
    if (int e = ensure_learned_buffers(c)) return e;
    if (int e = features(c, c->d_feat)) return e;
    const int64_t N = (int64_t)c->nx * c->ny;
    if (int e = lbk::mlp_infer_dev(c->mlp, c->d_feat, N, c->d_p, c->stream)) return e;
    lbk::launch_tile_max(c->d_p, c->nx, c->ny, c->ntx, c->d_tp, c->stream);
    if (int e = launch_check(c, "learned map")) return e;
    std::vector<float> tp((size_t)c->ny * c->ntx);
    if (int e = cuda_check(c, cudaMemcpyAsync(tp.data(), c->d_tp, tp.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                              c->stream), "learned map copy"))
        return e;
    if (int e = cuda_check(c, cudaStreamSynchronize(c->stream), "learned map sync")) return e;
    for (float v : tp)
        if (!std::isfinite(v)) {
            c->map_fallbacks += 1;
            return LB_OK;
        }
    std::vector<uint8_t> cell((size_t)N);
    bool changed = false;
    for (int j = 0; j < c->ny; ++j) {
        const bool wall_band = (c->walls[0].kind == LB_WALL_DIFFUSE && j < 2) ||
                               (c->walls[1].kind == LB_WALL_DIFFUSE && j > c->ny - 3);
        for (int tx = 0; tx < c->ntx; ++tx) {
            const size_t k = (size_t)j * c->ntx + tx;
            const int cur = c->tmap[k] & LB_TILE_HIGH;
            int nw = cur ? (tp[k] >= c->p_off) : (tp[k] >= c->p_on);
            if (wall_band) nw = 1;
            changed = changed || (nw != cur);
            for (int x = tx * LB_TILE_X; x < std::min(c->nx, (tx + 1) * LB_TILE_X); ++x)
                cell[(size_t)j * c->nx + x] = (uint8_t)nw;
        }
    }
    c->map_updates += 1;
    if (!changed) return LB_OK;
    return set_region_map_impl(c, cell.data());
}

template <typename R>
int step_t(lb_ctx *c, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) {
        const double t_new = c->t + c->dt;
        StepParams<R> p = make_params<R>(c, c->cur, c->cur ^ 1, t_new);
        if (c->opts.scheme == LB_SCHEME_STREAM) {
            lbk::launch_exact_stream<R>(c->store, p, c->stream);
        } else {
            launch_variant<R>(c, c->variant, p);
            lbk::launch_iface<R>(c->store, p, c->stream);
            if (c->variant != 10 || p.has_force) lbk::launch_pressure<R>(c->store, p, c->stream);   /* else 10 does it */
        }
        if (int e = launch_check(c, "step")) return e;
        c->cur ^= 1;
        c->t = t_new;
        c->step += 1;
        if (c->opts.reduce_every > 0 && c->step % c->opts.reduce_every == 0) {
            StepParams<R> q = make_params<R>(c, c->cur, c->cur, c->t);
            lbk::launch_reduce<R>(c->store, q, static_cast<R *>(c->d_uprev), c->d_part, c->d_counter, c->d_out,
                                  c->red_blocks, c->stream);
            if (int e = launch_check(c, "reduce")) return e;
            if (int e = cuda_check(c, cudaMemcpyAsync(c->h_out, c->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                                      c->stream), "reduce copy"))
                return e;
            cudaEventRecord(c->red_event, c->stream);
            c->red_pending = true;
        }
        if (c->mlp && c->mlp_every > 0 && c->step % c->mlp_every == 0)
            if (int e = learned_update(c)) return e;
    }
    return LB_OK;
}

void check_reduction(lb_ctx *c)
{
    if (!c->red_pending) return;
    if (cudaEventQuery(c->red_event) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    c->red_pending = false;
    if (c->h_out[2] > 0.0 || !std::isfinite(c->h_out[0])) {
        c->status = LB_ERR_DIVERGED;
        g_err = "non-finite density or velocity found by the reduction";
    }
}

int sticky(lb_ctx *c)
{
    if (!c) return fail(LB_ERR_INVALID, "null context");
    if (c->status != LB_OK) {
        if (g_err.empty()) g_err = "context is in an error state";
        return c->status;
    }
    return LB_OK;
}

void free_all(lb_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->edge_stream) cudaStreamSynchronize(c->edge_stream);
    for (void *p : c->owned) dev_free(c, p);
    c->owned.clear();
    if (c->h_out) cudaFreeHost(c->h_out);
    if (c->red_event) cudaEventDestroy(c->red_event);
    if (c->edge_stream) cudaStreamDestroy(c->edge_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
}

void *own(lb_ctx *c, size_t bytes)
{
    void *p = dev_alloc(c, bytes);
    if (p) c->owned.push_back(p);
    return p;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

/* Tensor maps over (storage column, storage row, plane) of every level and set. */
bool make_maps(lb_ctx *c)
{
    if (c->store == LB_STORE_F64) return false;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = c->store == LB_STORE_F16_DEV    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : c->store == LB_STORE_BF16_DEV ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t rows = (cuuint64_t)c->ny + 2 * LB_GHOST_ROWS;
    for (int lv = 0; lv < 2; ++lv)
        for (int s = 0; s < 2; ++s) {
            const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, rows, (cuuint64_t)c->q[s]};
            const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * c->esize, (cuuint64_t)c->pitch * rows * c->esize};
            const cuuint32_t estr[3] = {1, 1, 1};
            const cuuint32_t np = (cuuint32_t)lbk::step3_planes();
            const cuuint32_t b1[3] = {(cuuint32_t)lbk::step3_cols(), (cuuint32_t)lbk::step3_rows(), np};
            const cuuint32_t b2[3] = {(cuuint32_t)lbk::step3_cols(), (cuuint32_t)lbk::step3_rows() + 4, np};
            if (enc(&c->maps[lv].box1[s], dt, 3, c->planes[lv][s], dims, strides, b1, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
            if (enc(&c->maps[lv].box2[s], dt, 3, c->planes[lv][s], dims, strides, b2, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
            const cuuint32_t b5[3] = {(cuuint32_t)lbk::stream_cols(), (cuuint32_t)lbk::stream_rows() + 4, 1};
            if (enc(&c->maps[lv].box5[s], dt, 3, c->planes[lv][s], dims, strides, b5, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return false;
        }
    return true;
}

/* A bounded wait inside a kernel ran out: the context is left in LB_ERR_TIMEOUT. */
int check_device_error(lb_ctx *c)
{
    if (!c->d_err || c->status != LB_OK) return c->status;
    int h = 0;
    if (cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        c->status = LB_ERR_CUDA;
        g_err = "reading the device error word failed";
        return c->status;
    }
    if (h != 0) {
        c->status = LB_ERR_TIMEOUT;
        g_err = "a bounded device wait ran out in the step kernel";
    }
    return c->status;
}

struct TmpBuf {
    lb_ctx *c;
    void *p;
    TmpBuf(lb_ctx *cc, size_t bytes) : c(cc), p(dev_alloc(cc, bytes)) {}
    ~TmpBuf()
    {
        if (p) {
            cudaStreamSynchronize(c->stream);
            dev_free(c, p);
        }
    }
};

}  // namespace

extern "C" {

const char *lb_last_error(void) { return g_err.c_str(); }

int lb_create(const lb_grid *grid, const uint8_t *region_map, const int32_t sets[2], const lb_kn *kn,
              const lb_wall walls[4], const lb_opts *opts, lb_ctx **out)
{
    g_err.clear();
    if (!grid || !region_map || !sets || !kn || !walls || !opts || !out) return fail(LB_ERR_INVALID, "null argument");
    *out = nullptr;
    if (grid->nx < 4 || grid->ny < 4) return fail(LB_ERR_INVALID, "nx and ny must be >= 4");
    if ((long long)grid->nx * grid->ny > (1LL << 31)) return fail(LB_ERR_INVALID, "grid too large");
    if (opts->store < LB_STORE_F64 || opts->store > LB_STORE_BF16_DEV) return fail(LB_ERR_INVALID, "unknown storage");
    if (opts->iface != LB_IFACE_PAPER && opts->iface != LB_IFACE_HERMITE) return fail(LB_ERR_INVALID, "unknown interface mode");
    if (opts->variant >= LB_NUM_VARIANTS) return fail(LB_ERR_INVALID, "unknown kernel variant");
    if (opts->rounding != LB_ROUND_NEAREST && opts->rounding != LB_ROUND_STOCHASTIC)
        return fail(LB_ERR_INVALID, "unknown rounding mode");
    if (!(opts->rho0 > 0.0)) return fail(LB_ERR_INVALID, "rho0 must be positive");
    if (opts->scheme != LB_SCHEME_TVD && opts->scheme != LB_SCHEME_STREAM) return fail(LB_ERR_INVALID, "unknown scheme");
    if (opts->scheme == LB_SCHEME_STREAM) {
        if (sets[0] != 9) return fail(LB_ERR_INVALID, "the stream-and-collide scheme needs sets[0] = 9");
        for (int k = 0; k < 4; ++k)
            if (walls[k].kind != LB_WALL_PERIODIC)
                return fail(LB_ERR_INVALID, "the stream-and-collide scheme needs periodic walls on every side");
        for (size_t n = 0; n < (size_t)grid->nx * grid->ny; ++n)
            if (region_map[n] != 0) return fail(LB_ERR_INVALID, "the stream-and-collide scheme takes one set (map all 0)");
    }
    if (opts->rho0_col) {
        if (opts->store != LB_STORE_F32_DEV && opts->store != LB_STORE_F16_DEV && opts->store != LB_STORE_BF16_DEV)
            return fail(LB_ERR_INVALID, "a per-column reference density needs a deviation storage format");
        for (int x = 0; x < grid->nx; ++x)
            if (!(opts->rho0_col[x] > 0.0) || !std::isfinite(opts->rho0_col[x]))
                return fail(LB_ERR_INVALID, "per-column reference densities must be finite and positive");
    }
    for (int k = 0; k < 4; ++k)
        if (walls[k].kind < LB_WALL_PERIODIC || walls[k].kind > LB_WALL_PRESSURE)
            return fail(LB_ERR_INVALID, "unknown wall kind");
    if ((walls[0].kind == LB_WALL_PERIODIC) != (walls[1].kind == LB_WALL_PERIODIC))
        return fail(LB_ERR_INVALID, "bottom and top must both be periodic or both not");
    if ((walls[2].kind == LB_WALL_PERIODIC) != (walls[3].kind == LB_WALL_PERIODIC))
        return fail(LB_ERR_INVALID, "left and right must both be periodic or both not");
    if (walls[0].kind == LB_WALL_PRESSURE || walls[1].kind == LB_WALL_PRESSURE)
        return fail(LB_ERR_INVALID, "pressure sides are left / right only");
    if (walls[2].kind == LB_WALL_DIFFUSE || walls[3].kind == LB_WALL_DIFFUSE)
        return fail(LB_ERR_INVALID, "diffuse walls are bottom / top only");
    for (int k = 2; k < 4; ++k)
        if (walls[k].kind == LB_WALL_PRESSURE && !(walls[k].rho > 0.0))
            return fail(LB_ERR_INVALID, "pressure side density must be positive");
    if (!(kn->kn_ref > 0.0)) return fail(LB_ERR_INVALID, "kn_ref must be positive");

    lb_ctx *c = new lb_ctx();
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->kn = *kn;
    for (int k = 0; k < 4; ++k) c->walls[k] = walls[k];
    c->opts = *opts;
    c->store = opts->store;
    c->esize = elem_size(opts->store);
    c->stream = static_cast<cudaStream_t>(opts->stream);
    const bool stream_scheme = opts->scheme == LB_SCHEME_STREAM;
    double xmax = 0.0;
    for (int s = 0; s < 2; ++s) {
        c->q[s] = sets[s];
        if (lbq::velocity_set(sets[s], c->cx[s], c->cy[s], c->w[s]) != sets[s]) {
            delete c;
            return fail(LB_ERR_INVALID, "velocity sets must be 9, 16 or 36");
        }
        if (stream_scheme && s == 1) continue;   /* one set in use */
        for (int a = 0; a < c->q[s]; ++a) xmax = std::fmax(xmax, std::fabs(c->cx[s][a]));
    }
    c->h = grid->h > 0.0 ? grid->h : (walls[0].kind == LB_WALL_PERIODIC ? 1.0 / grid->ny : 1.0 / (grid->ny - 1));
    c->dt = grid->dt > 0.0 ? grid->dt : (stream_scheme ? c->h / xmax : grid->cfl * c->h / xmax);
    if (stream_scheme && std::fabs(xmax * c->dt / c->h - 1.0) > 1e-12) {
        delete c;
        return fail(LB_ERR_INVALID, "the stream-and-collide scheme needs dt = h / sqrt(3)");
    }
    if (!(c->dt > 0.0)) {
        delete c;
        return fail(LB_ERR_INVALID, "dt must be positive (cfl > 0 or dt > 0)");
    }
    if (xmax * c->dt / c->h > 1.0 + 1e-12) {
        delete c;
        return fail(LB_ERR_INVALID, "CFL number xi_max dt / h exceeds 1");
    }
    double tau0 = (kn->rho_ref > 0.0 ? kn->kn_ref * kn->rho_ref / opts->rho0 : kn->kn_ref) -
                  (kn->tau_mode == 1 ? 0.5 * c->dt : 0.0);
    if (!(tau0 > 0.0) || c->dt / tau0 > 1.0) {
        delete c;
        return fail(LB_ERR_INVALID, "dt / tau exceeds 1 at rho0");
    }
    c->ntx = (c->nx + LB_TILE_X - 1) / LB_TILE_X;
    c->pitch = (int)round_up((size_t)c->nx + 16, 32);
    int e = build_tiles(c, region_map, c->tmap, c->iface_rows);
    if (e) {
        delete c;
        return e;
    }
    for (int s = 0; s < 2; ++s)
        c->set_bytes[s] = (size_t)c->q[s] * (c->ny + 2 * LB_GHOST_ROWS) * c->pitch * c->esize;
    for (int lv = 0; lv < 2; ++lv)
        for (int s = 0; s < 2; ++s) c->planes[lv][s] = own(c, c->set_bytes[s]);
    c->d_tmap = static_cast<uint8_t *>(own(c, c->tmap.size()));
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 0;
        }
        c->red_blocks = lbk::reduce_blocks(c->nx, c->ny, nsm);
        c->nsm = nsm;
    }
    c->d_part = static_cast<double *>(own(c, sizeof(double) * 4 * c->red_blocks));
    c->d_out = static_cast<double *>(own(c, sizeof(double) * 4));
    c->d_counter = static_cast<unsigned int *>(own(c, 256));
    c->d_uprev = own(c, (size_t)c->nx * c->ny * 2 * (use_f64(c) ? 8 : 4));
    c->d_err = static_cast<int *>(own(c, 256));
    const size_t rsize = use_f64(c) ? 8 : 4;
    for (int lv = 0; lv < 2; ++lv) c->aux[lv] = own(c, 3 * (size_t)c->pitch * c->ny * rsize);
    c->d_squeue = static_cast<unsigned int *>(own(c, 256));
    bool col_ok = true;
    if (opts->rho0_col) {
        /* delta = rho0(x) - rho0 per storage column; a ghost column takes the delta of the
         * column it copies (periodic image, or the boundary column of a pressure side);
         * the padding beyond holds 0 */
        std::vector<float> dc(c->pitch, 0.0f);
        const bool px = walls[2].kind == LB_WALL_PERIODIC;
        for (int col = 0; col < c->nx + 2 * LB_GHOST; ++col) {
            int x = col - LB_GHOST;
            if (x < 0) x = px ? x + c->nx : 0;
            if (x >= c->nx) x = px ? x - c->nx : c->nx - 1;
            dc[col] = (float)(opts->rho0_col[x] - opts->rho0);
        }
        uint32_t hsh = 2166136261u;
        for (float v : dc) {
            uint32_t b;
            std::memcpy(&b, &v, 4);
            for (int k = 0; k < 4; ++k) hsh = (hsh ^ ((b >> (8 * k)) & 0xffu)) * 16777619u;
        }
        c->dcol_hash = hsh ? hsh : 1u;
        c->d_dcol = own(c, dc.size() * sizeof(float));
        col_ok = c->d_dcol && cudaMemcpy(c->d_dcol, dc.data(), dc.size() * sizeof(float), cudaMemcpyHostToDevice) ==
                                  cudaSuccess;
        c->opts.rho0_col = nullptr;   /* the caller's array is not kept */
    }
    bool ok = col_ok && c->d_tmap && c->d_part && c->d_out && c->d_counter && c->d_uprev && c->d_err && c->aux[0] &&
              c->aux[1] && c->d_squeue;
    for (int lv = 0; lv < 2; ++lv)
        for (int s = 0; s < 2; ++s) ok = ok && c->planes[lv][s];
    if (!ok) {
        free_all(c);
        delete c;
        return fail(LB_ERR_NOMEM, "device allocation failed");
    }
    /* four doubles of results, then the device error word */
    if (cudaMallocHost(reinterpret_cast<void **>(&c->h_out), 4 * sizeof(double) + 16) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->red_event, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return fail(LB_ERR_CUDA, "pinned buffer / event creation failed");
    }
    std::memset(c->h_out, 0, 4 * sizeof(double) + 16);
    /* second stream and fork / join events of the split step; without them that layout
     * is simply not offered */
    if (cudaStreamCreateWithFlags(&c->edge_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->edge_stream) cudaStreamDestroy(c->edge_stream);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        c->edge_stream = nullptr;
        c->ev_fork = c->ev_join = nullptr;
    }
    cudaError_t ce = cudaSuccess;
    for (int lv = 0; lv < 2 && ce == cudaSuccess; ++lv)
        for (int s = 0; s < 2 && ce == cudaSuccess; ++s) ce = cudaMemsetAsync(c->planes[lv][s], 0, c->set_bytes[s], c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_counter, 0, 256, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_err, 0, 256, c->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->d_uprev, 0, (size_t)c->nx * c->ny * 2 * (use_f64(c) ? 8 : 4), c->stream);
    if (ce != cudaSuccess || upload_tiles(c) != LB_OK) {
        free_all(c);
        delete c;
        return fail(LB_ERR_CUDA, std::string("initial fill failed: ") + cudaGetErrorString(ce));
    }
    c->tma_ok = make_maps(c);
    if (!use_f64(c)) {
        /* constant tables of layouts 7 / 8 (without them those layouts are not offered) */
        c->d_ctab = own(c, lbk::pair_table_bytes());
        if (c->d_ctab) lbk::launch_pair_table(make_params<float>(c, 0, 1, 0.0), c->d_ctab, c->stream);
        /* layout 10: the same constants for kernel-parameter space */
        if (c->d_ctab) {
            c->rtab.reset(new lbk::RingTab());
            if (lbk::ring_tab_build(c->d_ctab, make_params<float>(c, 0, 1, 0.0), c->rtab.get(), c->stream) != 0)
                c->rtab.reset();
        }
    }
    *out = c;
    e = lb_init_equilibrium(c, nullptr, nullptr, nullptr);
    if (e) {
        lb_destroy(c);
        *out = nullptr;
        return e;
    }
    c->variant = choose_variant(c);
    if (int e2 = launch_check(c, "autotune")) {
        lb_destroy(c);
        *out = nullptr;
        return e2;
    }
    return LB_OK;
}

int lb_init_equilibrium(lb_ctx *c, const double *rho, const double *ux, const double *uy)
{
    if (int e = sticky(c)) return e;
    const size_t N = (size_t)c->nx * c->ny;
    std::vector<double> h(3 * N);
    for (size_t n = 0; n < N; ++n) {
        h[n] = rho ? rho[n] : c->opts.rho0;
        h[N + n] = ux ? ux[n] : 0.0;
        h[2 * N + n] = uy ? uy[n] : 0.0;
        if (!(h[n] > 0.0) || !std::isfinite(h[N + n]) || !std::isfinite(h[2 * N + n]))
            return fail(LB_ERR_INVALID, "initial density must be positive and velocities finite");
    }
    TmpBuf tmp(c, 3 * N * sizeof(double));
    if (!tmp.p) return fail(LB_ERR_NOMEM, "device allocation failed");
    double *d = static_cast<double *>(tmp.p);
    if (int e = cuda_check(c, cudaMemcpyAsync(d, h.data(), 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                           "upload"))
        return e;
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_init<double>(c->store, p, d, d + N, d + 2 * N, c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_init<float>(c->store, p, d, d + N, d + 2 * N, c->stream);
    }
    if (int e = launch_check(c, "init")) return e;
    if (int e = finalize_level(c, c->cur)) return e;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "init sync");
}

int lb_step(lb_ctx *c, int64_t n)
{
    if (!c) return fail(LB_ERR_INVALID, "null context");
    check_reduction(c);
    if (int e = sticky(c)) return e;
    if (n < 0) return fail(LB_ERR_INVALID, "negative step count");
    return use_f64(c) ? step_t<double>(c, n) : step_t<float>(c, n);
}

int lb_moments(lb_ctx *c, uint32_t mask, void *dst, int32_t dst_is_device, int32_t dst_f64)
{
    if (int e = sticky(c)) return e;
    if (!dst || (mask & ~(uint32_t)LB_M_ALL) || mask == 0) return fail(LB_ERR_INVALID, "bad moments request");
    int nf = 0;
    for (int m = 0; m < 9; ++m) nf += (mask >> m) & 1u;
    const size_t bytes = (size_t)nf * c->nx * c->ny * (dst_f64 ? 8 : 4);
    void *target = dst;
    TmpBuf tmp(c, dst_is_device ? 0 : bytes);
    if (!dst_is_device) {
        if (!tmp.p) return fail(LB_ERR_NOMEM, "device allocation failed");
        target = tmp.p;
    }
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_moments<double>(c->store, p, mask, target, dst_f64, c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_moments<float>(c->store, p, mask, target, dst_f64, c->stream);
    }
    if (int e = launch_check(c, "moments")) return e;
    if (!dst_is_device) {
        if (int e = cuda_check(c, cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, c->stream), "moments copy"))
            return e;
        return cuda_check(c, cudaStreamSynchronize(c->stream), "moments sync");
    }
    return LB_OK;
}

int lb_reductions(lb_ctx *c, double out[4])
{
    if (int e = sticky(c)) return e;
    if (!out) return fail(LB_ERR_INVALID, "null output");
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_reduce<double>(c->store, p, static_cast<double *>(c->d_uprev), c->d_part, c->d_counter, c->d_out,
                                   c->red_blocks, c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_reduce<float>(c->store, p, static_cast<float *>(c->d_uprev), c->d_part, c->d_counter, c->d_out,
                                  c->red_blocks, c->stream);
    }
    if (int e = launch_check(c, "reduce")) return e;
    if (int e = cuda_check(c, cudaMemcpyAsync(c->h_out, c->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                           "reduce copy"))
        return e;
    /* the device error word comes back with the results: one wait for both */
    int *h_err = reinterpret_cast<int *>(c->h_out + 4);
    if (int e = cuda_check(c, cudaMemcpyAsync(h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                           "error word copy"))
        return e;
    if (int e = cuda_check(c, cudaStreamSynchronize(c->stream), "reduce sync")) return e;
    if (*h_err != 0) {
        c->status = LB_ERR_TIMEOUT;
        return fail(c->status, "a bounded device wait ran out in the step kernel");
    }
    c->red_pending = false;
    out[0] = c->h_out[0];
    out[1] = c->h_out[1];
    out[2] = c->h_out[2];
    out[3] = (double)c->step;
    if (c->h_out[2] > 0.0 || !std::isfinite(c->h_out[0])) {
        c->status = LB_ERR_DIVERGED;
        return fail(LB_ERR_DIVERGED, "non-finite density or velocity found by the reduction");
    }
    return LB_OK;
}

int lb_effective_map(lb_ctx *c, uint8_t *dst)
{
    if (!c || !dst) return fail(LB_ERR_INVALID, "null argument");
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
            dst[(size_t)j * c->nx + i] = c->tmap[(size_t)j * c->ntx + i / LB_TILE_X] & LB_TILE_HIGH;
    return LB_OK;
}

int lb_set_region_map(lb_ctx *c, const uint8_t *map)
{
    if (int e = sticky(c)) return e;
    if (!map) return fail(LB_ERR_INVALID, "null map");
    return set_region_map_impl(c, map);
}

int lb_features(lb_ctx *c, float *dst)
{
    if (int e = sticky(c)) return e;
    if (!dst) return fail(LB_ERR_INVALID, "null destination");
    return features(c, dst);
}

int lb_hermite_residual(lb_ctx *c, float *dst)
{
    if (int e = sticky(c)) return e;
    if (!dst) return fail(LB_ERR_INVALID, "null destination");
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_hermite_residual<double>(c->store, p, dst, c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_hermite_residual<float>(c->store, p, dst, c->stream);
    }
    return launch_check(c, "hermite residual");
}

int lb_set_mlp(lb_ctx *c, lb_mlp *m, int32_t every, float p_on, float p_off)
{
    if (int e = sticky(c)) return e;
    if (m && (every < 1 || !(p_on > p_off) || !(p_off >= 0.0f) || !(p_on <= 1.0f)))
        return fail(LB_ERR_INVALID, "lb_set_mlp: need every >= 1 and 0 <= p_off < p_on <= 1");
    if (m && c->opts.iface != LB_IFACE_HERMITE)
        return fail(LB_ERR_INVALID, "lb_set_mlp: learned maps need LB_IFACE_HERMITE (any tile layout)");
    c->mlp = m;
    c->mlp_every = m ? every : 0;
    c->p_on = p_on;
    c->p_off = p_off;
    return LB_OK;
}

int lb_learned_map_now(lb_ctx *c)
{
    if (int e = sticky(c)) return e;
    if (!c->mlp) return fail(LB_ERR_INVALID, "no network set (lb_set_mlp)");
    return learned_update(c);
}

}  // extern "C"

namespace {
int set_region_map_impl(lb_ctx *c, const uint8_t *map)
{
    std::vector<uint8_t> tm;
    std::vector<int> rows;
    if (int e = build_tiles(c, map, tm, rows)) return e;
    /* first rebuild every tile that changes set in its new set (shadow pass with the old
     * sets and only the changing tiles flagged), then install the new map */
    std::vector<uint8_t> moving(c->tmap.size());
    for (size_t k = 0; k < tm.size(); ++k)
        moving[k] = (uint8_t)((c->tmap[k] & LB_TILE_HIGH) |
                              (((c->tmap[k] ^ tm[k]) & LB_TILE_HIGH) ? LB_TILE_SHADOW : 0));
    c->tmap = moving;
    if (int e = upload_tiles(c)) return e;
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_shadows<double>(c->store, p, c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_shadows<float>(c->store, p, c->stream);
    }
    if (int e = launch_check(c, "remap")) return e;
    c->tmap = tm;
    c->iface_rows = rows;
    if (int e = upload_tiles(c)) return e;
    if (int e = finalize_level(c, c->cur)) return e;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "remap sync");
}
}  // namespace

extern "C" {

int lb_get_populations(lb_ctx *c, int32_t set, double *dst)
{
    if (int e = sticky(c)) return e;
    if (!dst || set < 0 || set > 1) return fail(LB_ERR_INVALID, "bad argument");
    const size_t bytes = (size_t)c->q[set] * c->nx * c->ny * sizeof(double);
    TmpBuf tmp(c, bytes);
    if (!tmp.p) return fail(LB_ERR_NOMEM, "device allocation failed");
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_get_pops<double>(c->store, p, set, static_cast<double *>(tmp.p), c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_get_pops<float>(c->store, p, set, static_cast<double *>(tmp.p), c->stream);
    }
    if (int e = launch_check(c, "get populations")) return e;
    if (int e = cuda_check(c, cudaMemcpyAsync(dst, tmp.p, bytes, cudaMemcpyDeviceToHost, c->stream), "copy")) return e;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
}

int lb_set_populations(lb_ctx *c, int32_t set, const double *src)
{
    if (int e = sticky(c)) return e;
    if (!src || set < 0 || set > 1) return fail(LB_ERR_INVALID, "bad argument");
    const size_t bytes = (size_t)c->q[set] * c->nx * c->ny * sizeof(double);
    TmpBuf tmp(c, bytes);
    if (!tmp.p) return fail(LB_ERR_NOMEM, "device allocation failed");
    if (int e = cuda_check(c, cudaMemcpyAsync(tmp.p, src, bytes, cudaMemcpyHostToDevice, c->stream), "copy")) return e;
    if (use_f64(c)) {
        StepParams<double> p = make_params<double>(c, c->cur, c->cur, c->t);
        lbk::launch_set_pops<double>(c->store, p, set, static_cast<const double *>(tmp.p), c->stream);
    } else {
        StepParams<float> p = make_params<float>(c, c->cur, c->cur, c->t);
        lbk::launch_set_pops<float>(c->store, p, set, static_cast<const double *>(tmp.p), c->stream);
    }
    if (int e = launch_check(c, "set populations")) return e;
    if (int e = finalize_level(c, c->cur)) return e;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
}

int lb_state_bytes(lb_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return fail(LB_ERR_INVALID, "null argument");
    *bytes = compact_bytes(c, c->nseg);
    return LB_OK;
}

int lb_state_load(lb_ctx *c, const void *src, size_t bytes)
{
    if (int e = sticky(c)) return e;
    if (!src || bytes != compact_bytes(c, c->nseg)) return fail(LB_ERR_INVALID, "state size mismatch");
    if (int e = ensure_stage(c, bytes)) return e;
    if (int e = cuda_check(c, cudaMemcpyAsync(c->d_stage, src, bytes, cudaMemcpyHostToDevice, c->stream), "state load"))
        return e;
    /* own-set populations with their ghost copies, then everything derived from them:
     * shadows, interface rows, pressure columns, carried moments */
    if (use_f64(c)) launch_pack_t<double>(c, 1);
    else launch_pack_t<float>(c, 1);
    if (int e = launch_check(c, "state load")) return e;
    return finalize_level(c, c->cur);   /* asynchronous: the caller keeps src until the stream passes */
}

int lb_state_store(lb_ctx *c, void *dst, size_t bytes)
{
    if (int e = sticky(c)) return e;
    if (!dst || bytes != compact_bytes(c, c->nseg)) return fail(LB_ERR_INVALID, "state size mismatch");
    if (int e = ensure_stage(c, bytes)) return e;
    if (use_f64(c)) launch_pack_t<double>(c, 0);
    else launch_pack_t<float>(c, 0);
    if (int e = launch_check(c, "state store")) return e;
    if (int e = cuda_check(c, cudaMemcpyAsync(dst, c->d_stage, bytes, cudaMemcpyDeviceToHost, c->stream), "state store"))
        return e;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "state store sync");
}

struct lb_file_header {
    char magic[8];
    int32_t version, nx, ny, q0, q1, store, iface, pad;
    int64_t step;
    double t, dt, h, rho0;
    uint64_t bytes;
};

int lb_save(lb_ctx *c, const char *path)
{
    if (int e = sticky(c)) return e;
    if (!path) return fail(LB_ERR_INVALID, "null path");
    size_t bytes = compact_bytes(c, c->nseg);
    std::vector<char> buf(bytes);
    if (int e = lb_state_store(c, buf.data(), bytes)) return e;
    lb_file_header hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBGBCKP", 8);
    hd.version = 2;   /* 2: compact state */
    hd.nx = c->nx; hd.ny = c->ny; hd.q0 = c->q[0]; hd.q1 = c->q[1]; hd.store = c->store; hd.iface = c->opts.iface;
    hd.step = c->step; hd.t = c->t; hd.dt = c->dt; hd.h = c->h; hd.rho0 = c->opts.rho0; hd.bytes = bytes;
    hd.pad = (int32_t)c->dcol_hash;   /* the state's values are relative to these reference densities */
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(LB_ERR_INVALID, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 && std::fwrite(c->tmap.data(), 1, c->tmap.size(), f) == c->tmap.size() &&
              std::fwrite(buf.data(), 1, bytes, f) == bytes;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LB_OK : fail(LB_ERR_INVALID, "write failed");
}

int lb_load(lb_ctx *c, const char *path)
{
    if (int e = sticky(c)) return e;
    if (!path) return fail(LB_ERR_INVALID, "null path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(LB_ERR_INVALID, std::string("cannot open ") + path);
    lb_file_header hd;
    std::vector<uint8_t> tm(c->tmap.size());
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && std::memcmp(hd.magic, "LBGBCKP", 8) == 0 && hd.version == 2 && hd.nx == c->nx && hd.ny == c->ny &&
         hd.q0 == c->q[0] && hd.q1 == c->q[1] && hd.store == c->store && hd.iface == c->opts.iface &&
         hd.dt == c->dt && hd.h == c->h && hd.rho0 == c->opts.rho0 && (uint32_t)hd.pad == c->dcol_hash;
    ok = ok && std::fread(tm.data(), 1, tm.size(), f) == tm.size();
    /* the state's size follows from the stored map */
    size_t bytes = 0;
    if (ok) {
        std::vector<int4> seg;
        int nseg[2];
        compact_segments(c, tm, seg, nseg);
        bytes = compact_bytes(c, nseg);
        ok = hd.bytes == bytes;
    }
    std::vector<char> buf(ok ? bytes : 0);
    ok = ok && std::fread(buf.data(), 1, bytes, f) == bytes;
    std::fclose(f);
    if (!ok) return fail(LB_ERR_INVALID, "checkpoint does not match this lattice");
    c->tmap = tm;
    c->iface_rows.clear();
    for (int j = 0; j < c->ny; ++j)
        if (c->tmap[(size_t)j * c->ntx] & LB_TILE_IFACE) c->iface_rows.push_back(j);
    if (int e = upload_tiles(c)) return e;
    if (int e = lb_state_load(c, buf.data(), bytes)) return e;
    if (int e = cuda_check(c, cudaStreamSynchronize(c->stream), "load sync")) return e;   /* buf goes away */
    c->step = hd.step;
    c->t = hd.t;
    return LB_OK;
}

int lb_selftest_bounded_wait(void *stream, uint32_t polls, int32_t *expired)
{
    if (!expired) return fail(LB_ERR_INVALID, "null argument");
    *expired = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LB_ERR_NOMEM, "device allocation failed");
    }
    const int code = 7;
    int h = 0;
    cudaError_t ce = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (ce == cudaSuccess && lbk::launch_wait_selftest(d, polls, code, st) != 0) ce = cudaErrorLaunchFailure;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(d);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(LB_ERR_CUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(ce));
    }
    *expired = h == code ? 1 : 0;
    return LB_OK;
}

int lb_map_stats(lb_ctx *c, int64_t *updates, int64_t *fallbacks, double *high_fraction)
{
    if (!c) return fail(LB_ERR_INVALID, "null context");
    if (updates) *updates = c->map_updates;
    if (fallbacks) *fallbacks = c->map_fallbacks;
    if (high_fraction) {
        int64_t hi = 0;
        for (int j = 0; j < c->ny; ++j)
            for (int tx = 0; tx < c->ntx; ++tx)
                if (c->tmap[(size_t)j * c->ntx + tx] & LB_TILE_HIGH)
                    hi += std::min(c->nx, (tx + 1) * LB_TILE_X) - tx * LB_TILE_X;
        *high_fraction = (double)hi / ((double)c->nx * c->ny);
    }
    return LB_OK;
}

}  // extern "C"

/* ---------------------------------------------------------------- batches -- */

struct lb_batch {
    std::vector<lb_ctx *> inst;
    int n = 0, store = 0;
    lb_opts opts{};
    cudaStream_t stream = nullptr, cstream = nullptr;
    void *d_params = nullptr;       /* StepParams [n][2] of the storage's arithmetic type */
    int *d_order = nullptr;         /* queue order: most work first */
    unsigned int *d_queue = nullptr;
    int threads = 256, grid = 1;
    int phase = 0;                  /* lattices' current level, relative to params [i][0] */
    /* on layout 10's bodies: constants tables [n], work items and their range per lattice */
    bool ring = false, force = false;
    int q1 = 0;
    lbk::RingTab *d_tabs = nullptr;
    uint32_t *d_items = nullptr;
    int2 *d_ranges = nullptr;
    int status = LB_OK;
    std::vector<void *> owned;
};

namespace {

void *batch_alloc(lb_batch *b, size_t bytes)
{
    void *p = nullptr;
    if (b->opts.alloc && b->opts.free) {
        p = b->opts.alloc(bytes, b->opts.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) b->owned.push_back(p);
    return p;
}

void batch_release(lb_batch *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (lb_ctx *c : b->inst) lb_destroy(c);
    b->inst.clear();
    for (void *p : b->owned) {
        if (b->opts.alloc && b->opts.free) b->opts.free(p, b->opts.alloc_user);
        else cudaFree(p);
    }
    b->owned.clear();
    if (b->cstream) cudaStreamDestroy(b->cstream);
    b->cstream = nullptr;
}

template <typename R>
int batch_upload_params(lb_batch *b)
{
    std::vector<StepParams<R>> h(2 * (size_t)b->n);
    for (int i = 0; i < b->n; ++i) {
        const lb_ctx *c = b->inst[i];
        h[2 * (size_t)i] = make_params<R>(c, c->cur, c->cur ^ 1, c->t + c->dt);
        h[2 * (size_t)i + 1] = make_params<R>(c, c->cur ^ 1, c->cur, c->t + 2.0 * c->dt);
        /* the parameters serve every step of a launch: no per-step random key */
        h[2 * (size_t)i].sr = h[2 * (size_t)i + 1].sr = 0;
    }
    b->d_params = batch_alloc(b, h.size() * sizeof(StepParams<R>));
    if (!b->d_params) return fail(LB_ERR_NOMEM, "device allocation failed");
    if (cudaMemcpyAsync(b->d_params, h.data(), h.size() * sizeof(StepParams<R>), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fail(LB_ERR_CUDA, "batch parameter upload failed");
    return LB_OK;
}

/* Work items of the ring batch (see launch_ring_batch): per lattice, runs of consecutive
 * rows of one set and kind, at most 32 quads each, most work first; and every lattice's
 * constants table. */
int batch_ring_setup(lb_batch *b)
{
    /* items (two words each, longest first per lattice), then the row lists they index */
    struct Item {
        int cost;
        uint32_t meta;
        std::vector<uint32_t> rows;
    };
    std::vector<std::vector<Item>> all(b->n);
    std::vector<int2> ranges(b->n);
    std::vector<lbk::RingTab> tabs(b->n);
    size_t nitems = 0, nrows = 0;
    for (int i = 0; i < b->n; ++i) {
        const lb_ctx *c = b->inst[i];
        if (!c->rtab) return fail(LB_ERR_INVALID, "a batched lattice has no layout-10 constants");
        tabs[i] = *c->rtab;
        const bool py = c->walls[0].kind == LB_WALL_PERIODIC;
        const int qpr = (c->nx + 3) / 4, per = 32 / qpr;
        /* set | kind << 1: 0 edge (stores node by node where not plain), 1 row (ghost-row
         * copies, wall or shadow: the row body), 2 general (such a row ending inside a
         * quad: layout 9's body) */
        auto key = [&](int r) {
            const uint8_t f = c->tmap[(size_t)r * c->ntx];
            const bool bound = (f & LB_TILE_SHADOW) || (py ? (r < 2 || r >= c->ny - 2) : (r == 0 || r == c->ny - 1));
            const int kind = !bound ? 0 : (c->nx % 4 == 0 ? 1 : 2);
            return (int)(f & LB_TILE_HIGH) | (kind << 1);
        };
        /* a lane's time is its chain of populations (the row body's epilogue adds to it),
         * nearly whatever the item's number of rows: that is the cost */
        auto add = [&](int k, std::vector<uint32_t> &rows) {
            const int kind = k >> 1;
            const int cost = c->q[k & 1] * (kind == 0 ? 5 : (kind == 1 ? 7 : 9)) * 64 + (int)rows.size();
            all[i].push_back({cost, (uint32_t)(rows.size() - 1) | ((uint32_t)(k & 1) << 5) | ((uint32_t)kind << 6), rows});
            rows.clear();
        };
        /* row-body rows of each set, merged across the lattice: wall (and periodic image)
         * rows apart from shadow rows, so that no lane's epilogue waits on the other's */
        std::vector<uint32_t> pend[2][2];
        std::vector<uint32_t> run;
        int j = 0;
        while (j < c->ny) {
            const int k0 = key(j);
            int r = j;
            while (r < c->ny && r - j < per && key(r) == k0) ++r;
            if ((k0 >> 1) == 1) {
                for (int t = j; t < r; ++t) {
                    const bool edge_row = py ? (t < 2 || t >= c->ny - 2) : (t == 0 || t == c->ny - 1);
                    std::vector<uint32_t> &pl = pend[k0 & 1][edge_row ? 0 : 1];
                    pl.push_back((uint32_t)t);
                    if ((int)pl.size() == per) add(k0, pl);
                }
            } else {
                for (int t = j; t < r; ++t) run.push_back((uint32_t)t);
                add(k0, run);
            }
            j = r;
        }
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t)
                if (!pend[s][t].empty()) add(s | 2, pend[s][t]);
        std::stable_sort(all[i].begin(), all[i].end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
        ranges[i] = make_int2((int)nitems, (int)all[i].size());
        nitems += all[i].size();
        for (const Item &it : all[i]) nrows += it.rows.size();
    }
    if (2 * nitems + nrows > 0xffffffffull) return fail(LB_ERR_INVALID, "batch item list too large");
    std::vector<uint32_t> items(2 * nitems);
    items.reserve(2 * nitems + nrows);
    size_t k = 0;
    for (int i = 0; i < b->n; ++i)
        for (const Item &it : all[i]) {
            items[2 * k] = (uint32_t)items.size();
            items[2 * k + 1] = it.meta;
            items.insert(items.end(), it.rows.begin(), it.rows.end());
            ++k;
        }
    b->d_tabs = static_cast<lbk::RingTab *>(batch_alloc(b, sizeof(lbk::RingTab) * b->n));
    b->d_items = static_cast<uint32_t *>(batch_alloc(b, sizeof(uint32_t) * items.size()));
    b->d_ranges = static_cast<int2 *>(batch_alloc(b, sizeof(int2) * b->n));
    if (!b->d_tabs || !b->d_items || !b->d_ranges) return fail(LB_ERR_NOMEM, "device allocation failed");
    if (cudaMemcpyAsync(b->d_tabs, tabs.data(), sizeof(lbk::RingTab) * b->n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_items, items.data(), sizeof(uint32_t) * items.size(), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_ranges, ranges.data(), sizeof(int2) * b->n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fail(LB_ERR_CUDA, "batch item upload failed");
    int resident = 0;
    if (lbk::launch_ring_batch(b->store, b->q1, nullptr, nullptr, nullptr, nullptr, nullptr, b->n, 0, 0, 0, nullptr,
                               b->force, 0, &resident, b->stream) != 0 || resident < 1)
        return fail(LB_ERR_CUDA, "the batch kernel cannot be resident");
    b->threads = 256;   /* the block the kernel is built for */
    b->grid = std::min(b->n, resident);
    return LB_OK;
}

int batch_launch(lb_batch *b, int64_t nsteps, int advance, cudaStream_t st)
{
    if (cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), st) != cudaSuccess)
        return fail(LB_ERR_CUDA, "batch queue reset failed");
    const int r = b->ring ? lbk::launch_ring_batch(b->store, b->q1, static_cast<const StepParams<float> *>(b->d_params),
                                                   b->d_tabs, b->d_items, b->d_ranges, b->d_order, b->n, (int)nsteps,
                                                   b->phase, advance, b->d_queue, b->force, b->grid, nullptr, st)
                          : lbk::launch_batch(b->store, b->d_params, b->d_order, b->n, (int)nsteps, b->phase, advance,
                                              b->d_queue, b->threads, b->grid, st);
    if (r != 0)
        return fail(LB_ERR_INVALID, "bad batch block shape");
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        b->status = LB_ERR_CUDA;
        return fail(LB_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

/* after nsteps steps of every lattice */
void batch_advance(lb_batch *b, int64_t nsteps)
{
    for (lb_ctx *c : b->inst) {
        c->cur ^= (int)(nsteps & 1);
        c->t += (double)nsteps * c->dt;
        c->step += nsteps;
    }
    b->phase ^= (int)(nsteps & 1);
}

int batch_ready(lb_batch *b)
{
    if (!b) return fail(LB_ERR_INVALID, "null batch");
    if (b->status != LB_OK) return b->status;
    for (lb_ctx *c : b->inst) {
        if (c->status != LB_OK) return c->status;
        if (c->cur != b->phase) return fail(LB_ERR_INVALID, "a lattice of the batch was stepped on its own");
    }
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_batch_create(int32_t n, const lb_grid *grids, const uint8_t *const *maps, const int32_t sets[2], const lb_kn *kn,
                    const lb_wall *walls, const lb_opts *opts, lb_batch **out)
{
    g_err.clear();
    if (!out) return fail(LB_ERR_INVALID, "null output");
    *out = nullptr;
    if (n < 1 || !grids || !maps || !sets || !kn || !walls || !opts) return fail(LB_ERR_INVALID, "null argument or n < 1");
    for (int i = 0; i < n; ++i) {
        const lb_opts &o = opts[i];
        if (!maps[i]) return fail(LB_ERR_INVALID, "null region map");
        if (o.iface != LB_IFACE_HERMITE) return fail(LB_ERR_INVALID, "batched lattices need LB_IFACE_HERMITE");
        if (o.reduce_every != 0) return fail(LB_ERR_INVALID, "batched lattices take no in-step reductions");
        if (o.store != opts[0].store || o.rho0 != opts[0].rho0)
            return fail(LB_ERR_INVALID, "batched lattices share the storage format and rho0");
        if (o.rho0_col) return fail(LB_ERR_INVALID, "batched lattices take one reference density");
        if (o.scheme != LB_SCHEME_TVD) return fail(LB_ERR_INVALID, "batched lattices use the TVD scheme");
        for (int k = 0; k < 4; ++k) {
            const lb_wall &wl = walls[4 * (size_t)i + k];
            if (wl.kind == LB_WALL_PRESSURE) return fail(LB_ERR_INVALID, "batched lattices have no pressure sides");
            if (wl.omega != 0.0) return fail(LB_ERR_INVALID, "batched lattices have steady walls");
        }
    }
    lb_batch *b = new lb_batch();
    b->n = n;
    b->opts = opts[0];
    b->store = opts[0].store;
    b->stream = static_cast<cudaStream_t>(opts[0].stream);
    /* layout 10's bodies for FP32 and 16-bit storage, D2Q9 with D2Q16 or D2Q36, lattices at
     * most one tile wide; else the one-quad batch kernel */
    b->ring = b->store != LB_STORE_F64 && sets[0] == 9 && (sets[1] == 16 || sets[1] == 36);
    for (int i = 0; i < n; ++i) {
        b->ring = b->ring && grids[i].nx <= LB_TILE_X;
        b->force = b->force || opts[i].gx != 0.0 || opts[i].gy != 0.0;
    }
    b->q1 = sets[1];
    for (int i = 0; i < n; ++i) {
        lb_opts o = opts[i];
        /* no per-lattice timing: the batch kernel does the stepping, with the bits of
         * layout 9 (ring batch) or layout 0, which a lattice then takes on its own too */
        o.variant = b->ring ? 9 : 0;
        o.stream = opts[0].stream;
        lb_ctx *c = nullptr;
        if (int e = lb_create(&grids[i], maps[i], sets, &kn[i], walls + 4 * (size_t)i, &o, &c)) {
            const std::string msg = "lattice " + std::to_string(i) + ": " + g_err;
            batch_release(b);
            delete b;
            return fail(e, msg);
        }
        c->ring_batch = b->ring;
        b->inst.push_back(c);
    }
    /* most work first */
    std::vector<std::pair<double, int>> work(n);
    for (int i = 0; i < n; ++i) {
        const lb_ctx *c = b->inst[i];
        double w = 0.0;
        for (int j = 0; j < c->ny; ++j)
            for (int tx = 0; tx < c->ntx; ++tx) {
                const int cols = std::min(c->nx, (tx + 1) * LB_TILE_X) - tx * LB_TILE_X;
                w += (double)cols * c->q[c->tmap[(size_t)j * c->ntx + tx] & LB_TILE_HIGH];
            }
        work[i] = {-w, i};
    }
    std::sort(work.begin(), work.end());
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = work[i].second;
    b->d_order = static_cast<int *>(batch_alloc(b, sizeof(int) * n));
    b->d_queue = static_cast<unsigned int *>(batch_alloc(b, 256));
    int e = (b->d_order && b->d_queue) ? LB_OK : fail(LB_ERR_NOMEM, "device allocation failed");
    if (!e && cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        e = fail(LB_ERR_CUDA, "batch order upload failed");
    if (!e) e = b->store == LB_STORE_F64 ? batch_upload_params<double>(b) : batch_upload_params<float>(b);
    if (!e && b->ring) e = batch_ring_setup(b);
    /* block size of the one-quad kernel: time each candidate without moving the state */
    int dev = 0, nsm = 0;
    if (!e && !b->ring &&
        (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
        e = fail(LB_ERR_CUDA, "device query failed");
    if (!e && !b->ring) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_threads = 0, best_grid = 0;
        for (int threads : {128, 256, 512}) {
            const int per_sm = lbk::batch_blocks(b->store, threads);
            if (per_sm < 1) continue;
            b->threads = threads;
            b->grid = std::min(n, nsm * per_sm);
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && !e; ++rep) {
                cudaEventRecord(e0, b->stream);
                e = batch_launch(b, 4, 0, b->stream);
                cudaEventRecord(e1, b->stream);
                float t = 0.0f;
                if (!e && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
                    ms = std::min(ms, t);
            }
            if (!e && ms < best) {
                best = ms;
                best_threads = b->threads;
                best_grid = b->grid;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (!e && best_threads > 0) {
            b->threads = best_threads;
            b->grid = best_grid;
        } else if (!e) {
            e = fail(LB_ERR_CUDA, "no batch block size could be launched");
        }
    }
    if (e) {
        batch_release(b);
        delete b;
        return e;
    }
    *out = b;
    return LB_OK;
}

int lb_batch_step(lb_batch *b, int64_t nsteps)
{
    if (int e = batch_ready(b)) return e;
    if (nsteps < 0 || nsteps > (1LL << 30)) return fail(LB_ERR_INVALID, "step count out of range");
    if (nsteps == 0) return LB_OK;
    if (int e = batch_launch(b, nsteps, 1, b->stream)) return e;
    batch_advance(b, nsteps);
    return LB_OK;
}

int lb_batch_step_each(lb_batch *b, int64_t nsteps)
{
    if (int e = batch_ready(b)) return e;
    if (nsteps < 0) return fail(LB_ERR_INVALID, "negative step count");
    for (int64_t k = 0; k < nsteps; ++k)
        for (lb_ctx *c : b->inst)
            if (int e = lb_step(c, 1)) return e;
    b->phase ^= (int)(nsteps & 1);
    /* layout 9 carries no moments: the ring batch's are summed again */
    if (b->ring && nsteps > 0)
        for (lb_ctx *c : b->inst) {
            lbk::launch_aux<float>(c->store, make_params<float>(c, c->cur, c->cur, c->t), nullptr, 0, c->stream);
            if (int e = launch_check(c, "carried moments")) return e;
        }
    return LB_OK;
}

int lb_batch_graph(lb_batch *b, int64_t nsteps, int32_t replays)
{
    if (int e = batch_ready(b)) return e;
    if (nsteps < 2 || (nsteps & 1) || nsteps > (1LL << 30) || replays < 1)
        return fail(LB_ERR_INVALID, "graph replays need an even step count >= 2 and replays >= 1");
    if (!b->cstream && cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->cstream = nullptr;
        return fail(LB_ERR_CUDA, "capture stream creation failed");
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(LB_ERR_CUDA, "batch stream sync failed");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    if (cudaStreamBeginCapture(b->cstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return fail(LB_ERR_CUDA, "stream capture failed to start");
    }
    const int el = batch_launch(b, nsteps, 1, b->cstream);
    const cudaError_t ec = cudaStreamEndCapture(b->cstream, &g);
    if (el || ec != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return el ? el : fail(LB_ERR_CUDA, "stream capture failed");
    }
    cudaError_t ce = cudaGraphInstantiate(&x, g, 0);
    for (int r = 0; r < replays && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(x, b->cstream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->cstream);
    if (x) cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        b->status = LB_ERR_CUDA;
        return fail(LB_ERR_CUDA, std::string("graph replay: ") + cudaGetErrorString(ce));
    }
    batch_advance(b, nsteps * (int64_t)replays);
    return LB_OK;
}

lb_ctx *lb_batch_instance(lb_batch *b, int32_t i)
{
    if (!b || i < 0 || i >= b->n) {
        fail(LB_ERR_INVALID, "no such lattice in the batch");
        return nullptr;
    }
    return b->inst[i];
}

int lb_batch_info(lb_batch *b, int32_t *block_threads, int32_t *grid_blocks)
{
    if (!b) return fail(LB_ERR_INVALID, "null batch");
    if (block_threads) *block_threads = b->threads;
    if (grid_blocks) *grid_blocks = b->grid;
    return LB_OK;
}

int lb_batch_sync(lb_batch *b)
{
    if (!b) return fail(LB_ERR_INVALID, "null batch");
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        b->status = LB_ERR_CUDA;
        return fail(LB_ERR_CUDA, "batch stream sync failed");
    }
    if (b->status != LB_OK) return b->status;
    for (lb_ctx *c : b->inst)
        if (c->status != LB_OK) return c->status;
    return LB_OK;
}

void lb_batch_destroy(lb_batch *b)
{
    if (!b) return;
    batch_release(b);
    delete b;
}

int lb_info(lb_ctx *c, double *dt, double *h, int64_t *step, double *time, int32_t *variant)
{
    if (!c) return fail(LB_ERR_INVALID, "null context");
    if (variant) *variant = c->variant;
    if (dt) *dt = c->dt;
    if (h) *h = c->h;
    if (step) *step = c->step;
    if (time) *time = c->t;
    return LB_OK;
}

int lb_sync(lb_ctx *c)
{
    if (!c) return fail(LB_ERR_INVALID, "null context");
    if (c->status == LB_OK) cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
    check_reduction(c);
    check_device_error(c);
    return c->status;
}

void lb_destroy(lb_ctx *c)
{
    if (!c) return;
    free_all(c);
    delete c;
}

}  // extern "C"
