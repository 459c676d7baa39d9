/*
 * lb_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the multiscale
 * lattice Boltzmann method of Meng, Zhang & Shan, "Multiscale lattice Boltzmann
 * approach to modeling gas flows".
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library; the product (CUDA) path never does, and
 * the two share no code, header, table or constant generator.
 *
 * Everything is double precision and written in the order and notation of the
 * paper, node by node, population by population:
 *
 *   Eq. (weight) + product rule (Sec. 2.1)  velocity sets from Hermite roots
 *   Eq. (demoeq), Eq. (demoforce)          second-order equilibrium and force
 *   Eq. (lbgk) discretised as in Sec. 3.1  forward Euler + TVD minmod fluxes
 *   Sec. 3.2                               diffuse-reflection wall, ghost = wall node
 *   Sec. 2.2                               interface coupling ("virtual boundary"),
 *                                          mode A = the paper's interpolation /
 *                                          extrapolation rule, mode B = Hermite
 *                                          projection of the foreign node (rho, rho u,
 *                                          full second moment) into the reader's set
 *
 * Values that are not state -- wall ghosts, periodic images, interface nodes, the
 * pressure-boundary columns and foreign-set neighbours -- are produced lazily, at
 * the moment a reader asks for them, straight from the definitions. Nothing is
 * cached, fused or reordered.
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - TVD flux for negative velocities: the mirror image of the printed positive
 *     form (the upwind node becomes i+1).
 *   - Theta with a zero denominator: the limited slope is zero.
 *   - tau = kn_ref * rho_ref / rho (collision rate p / mu with mu fixed, Eq. (KN)),
 *     optionally minus dt/2 (tau_mode 1).
 *   - Wall: both superscripts of the wall formula refer to the wall node at the
 *     new time level; the streamed values with xi.n < 0 set rho_W, the values with
 *     xi.n > 0 are then replaced by rho_W S.
 *   - Mode A: the interface node I is the first low-order row next to the
 *     high-order band; it is not evolved; it holds both sets; a reader that
 *     reaches one node beyond I sees a copy of I (as for wall ghosts).
 *   - Pressure columns (x = 0, x = nx-1, interior rows): f = f_eq(rho_b, u_1)
 *     + [f - f_eq](node 1 step inwards), the same virtual-boundary construction
 *     as Sec. 2.2; ghosts beyond them are copies.
 *
 * A storage model (or_set_storage, off by default) rounds the stored populations of
 * every evolved node after each update the way a finite-precision storage format does,
 * so that the error a format adds can be computed here, in FP64 otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_QMAX 36

/* ------------------------------------------------------------------ sets -- */

typedef struct {
    int n1d;                 /* points of the 1-D rule */
    int q;                   /* n1d * n1d */
    double cx[OR_QMAX], cy[OR_QMAX], w[OR_QMAX];
} or_vset;

/* Probabilists' Hermite polynomial He_n(x) = chi^(n) in 1-D (Eq. (hermipol) with
 * omega = exp(-x^2/2)/sqrt(2 pi)), by the recurrence He_{k+1} = x He_k - k He_{k-1}. */
static double he(int n, double x)
{
    if (n == 0) return 1.0;
    double a = 1.0, b = x;
    for (int k = 1; k < n; ++k) {
        double c = x * b - (double)k * a;
        a = b;
        b = c;
    }
    return b;
}

static double factorial(int n)
{
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= (double)k;
    return r;
}

/* 1-D Gauss-Hermite rule (Sec. 2.1): abscissae are the n roots of He_n, located by
 * a sign-change scan and refined by bisection; weights by Eq. (weight),
 * w = n! / [n He_{n-1}(xi)]^2.  Roots ascending.  Returns the number found. */
int or_gauss_hermite(int n, double *xi, double *w)
{
    int found = 0;
    double lo = -sqrt(4.0 * n + 2.0) - 1.0, step = 1e-3;
    double x0 = lo, p0 = he(n, x0);
    while (found < n && x0 < -lo) {
        double x1 = x0 + step, p1 = he(n, x1);
        if (p1 == 0.0) {
            xi[found++] = x1;
            x0 = x1 + step * 0.5;
            p0 = he(n, x0);
            continue;
        }
        if ((p0 < 0.0) != (p1 < 0.0)) {
            double a = x0, b = x1, pa = p0;
            for (int it = 0; it < 200; ++it) {
                double m = 0.5 * (a + b), pm = he(n, m);
                if (pm == 0.0) { a = b = m; break; }
                if ((pa < 0.0) == (pm < 0.0)) { a = m; pa = pm; } else { b = m; }
            }
            xi[found++] = 0.5 * (a + b);
        }
        x0 = x1;
        p0 = p1;
    }
    /* He_n has the parity of n, so its roots come in +/- pairs (and 0 for odd n):
     * impose that symmetry exactly on the bisected values. */
    if (found == n)
        for (int k = 0; k < n / 2 + n % 2; ++k) {
            double m = 0.5 * (xi[n - 1 - k] - xi[k]);
            xi[k] = -m;
            xi[n - 1 - k] = m;
        }
    for (int k = 0; k < found; ++k) {
        double d = (double)n * he(n - 1, xi[k]);
        w[k] = factorial(n) / (d * d);
    }
    return found;
}

/* 2-D set by the product rule: alpha = iy * n1d + ix, xi = (r_ix, r_iy), w = w_ix w_iy. */
static int make_set(int n1d, or_vset *s)
{
    double r[8], w[8];
    if (n1d < 2 || n1d > 6) return -1;
    if (or_gauss_hermite(n1d, r, w) != n1d) return -1;
    s->n1d = n1d;
    s->q = n1d * n1d;
    for (int iy = 0; iy < n1d; ++iy)
        for (int ix = 0; ix < n1d; ++ix) {
            int a = iy * n1d + ix;
            s->cx[a] = r[ix];
            s->cy[a] = r[iy];
            s->w[a] = w[ix] * w[iy];
        }
    return 0;
}

int or_velocity_set(int n1d, double *cx, double *cy, double *w)
{
    or_vset s;
    if (make_set(n1d, &s)) return -1;
    for (int a = 0; a < s.q; ++a) { cx[a] = s.cx[a]; cy[a] = s.cy[a]; w[a] = s.w[a]; }
    return s.q;
}

/* Eq. (demoeq) with T = 1, D = 2:
 * f_eq = w rho {1 + xi.u + [(xi.u)^2 - u^2]/2}. */
static double feq(const or_vset *s, int a, double rho, double ux, double uy)
{
    double xu = s->cx[a] * ux + s->cy[a] * uy;
    double uu = ux * ux + uy * uy;
    return s->w[a] * rho * (1.0 + xu + 0.5 * (xu * xu - uu));
}

/* Eq. (demoforce): g_a = w rho {g.xi + (g.xi)(u.xi) - g.u}. */
static double force(const or_vset *s, int a, double rho, double ux, double uy,
                    double gx, double gy)
{
    double gxi = gx * s->cx[a] + gy * s->cy[a];
    double uxi = ux * s->cx[a] + uy * s->cy[a];
    return s->w[a] * rho * (gxi + gxi * uxi - (gx * ux + gy * uy));
}

int or_feq(int n1d, double rho, double ux, double uy, double *out)
{
    or_vset s;
    if (make_set(n1d, &s)) return -1;
    for (int a = 0; a < s.q; ++a) out[a] = feq(&s, a, rho, ux, uy);
    return s.q;
}

int or_force(int n1d, double rho, double ux, double uy, double gx, double gy, double *out)
{
    or_vset s;
    if (make_set(n1d, &s)) return -1;
    for (int a = 0; a < s.q; ++a) out[a] = force(&s, a, rho, ux, uy, gx, gy);
    return s.q;
}

/* Hermite coefficients up to second order (Eq. (an) with the quadrature of the
 * node's own set): a0 = sum f, a1 = sum f xi, a2 = sum f (xi xi - I). */
static void hermite_coeffs(const or_vset *s, const double *f, double a0[1], double a1[2],
                           double a2[3])
{
    a0[0] = 0.0; a1[0] = a1[1] = 0.0; a2[0] = a2[1] = a2[2] = 0.0;
    for (int a = 0; a < s->q; ++a) {
        a0[0] += f[a];
        a1[0] += f[a] * s->cx[a];
        a1[1] += f[a] * s->cy[a];
        a2[0] += f[a] * (s->cx[a] * s->cx[a] - 1.0);
        a2[1] += f[a] * (s->cx[a] * s->cy[a]);
        a2[2] += f[a] * (s->cy[a] * s->cy[a] - 1.0);
    }
}

/* Mode B: value of population a of set `to` rebuilt from the second-order Hermite
 * expansion (Eq. (approxf), N = 2) whose coefficients are those of the foreign node:
 * f_a = w_a [a0 + a1.xi + (1/2) a2 : (xi xi - I)]. */
static double project_one(const or_vset *to, int a, const double a0[1], const double a1[2],
                          const double a2[3])
{
    double x = to->cx[a], y = to->cy[a];
    double h2 = a2[0] * (x * x - 1.0) + 2.0 * a2[1] * x * y + a2[2] * (y * y - 1.0);
    return to->w[a] * (a0[0] + a1[0] * x + a1[1] * y + 0.5 * h2);
}

int or_project(int n1d_from, const double *f_from, int n1d_to, double *out)
{
    or_vset s, t;
    double a0[1], a1[2], a2[3];
    if (make_set(n1d_from, &s) || make_set(n1d_to, &t)) return -1;
    hermite_coeffs(&s, f_from, a0, a1, a2);
    for (int a = 0; a < t.q; ++a) out[a] = project_one(&t, a, a0, a1, a2);
    return t.q;
}

/* ---------------------------------------------------------------- lattice -- */

enum { W_PERIODIC = 0, W_DIFFUSE = 1, W_PRESSURE = 2 };
enum { SIDE_BOTTOM = 0, SIDE_TOP = 1, SIDE_LEFT = 2, SIDE_RIGHT = 3 };

typedef struct {
    int32_t nx, ny;
    int32_t n1d_lo, n1d_hi;      /* 1-D orders of the low- and high-order sets */
    double h, dt;                /* grid spacing (dx = dy) and time step */
    double kn_ref, rho_ref;      /* tau = kn_ref rho_ref / rho (rho_ref <= 0: tau = kn_ref) */
    int32_t tau_mode;            /* 1: subtract dt/2 from tau */
    double gx, gy;               /* body force */
    int32_t iface;               /* 0: mode A (paper), 1: mode B (projection) */
    int32_t limiter;             /* 0: minmod (paper); 1: Psi = 0; 2: Psi = 1 (test switch) */
    int32_t wall_kind[4];        /* bottom, top, left, right */
    double wall_ux[4], wall_uy[4], wall_rho[4], wall_omega[4];
} or_cfg;

/* Storage model (a test switch, off by default): after each update the populations of
 * an evolved node are stored the way a finite-precision format holds them, so that the
 * error a storage format adds to the method can be computed in FP64 and compared with
 * what a finite-precision implementation shows. */
enum {
    ST_EXACT = 0,        /* no rounding (the oracle proper) */
    ST_F32 = 1,          /* f itself rounded to FP32 */
    ST_F32_DEV = 2,      /* the deviation f / w - rho_r rounded to FP32 */
    ST_F16_DEV = 3,      /* ... to FP16, to nearest */
    ST_BF16_DEV = 4,     /* ... to BF16, to nearest */
    ST_F16_DEV_SR = 5,   /* ... to FP16, stochastically */
    ST_BF16_DEV_SR = 6   /* ... to BF16, stochastically */
};

typedef struct {
    or_cfg c;
    or_vset set[2];
    uint8_t *map;                /* [ny][nx]: 0 low-order, 1 high-order */
    double *f[2];                /* per set, [q][ny][nx], valid where map == set */
    double *fn[2];
    double t;
    int64_t step;
    int32_t store;               /* storage model, ST_* */
    double *rho_r;               /* [nx]: reference density of each column's deviation */
} or_lattice;

#define F(L, s, a, i, j) ((L)->f[s][((size_t)(a) * (L)->c.ny + (size_t)(j)) * (L)->c.nx + (size_t)(i)])
#define FN(L, s, a, i, j) ((L)->fn[s][((size_t)(a) * (L)->c.ny + (size_t)(j)) * (L)->c.nx + (size_t)(i)])
#define MAP(L, i, j) ((L)->map[(size_t)(j) * (L)->c.nx + (size_t)(i)])

static int is_pressure_node(const or_lattice *L, int i, int j)
{
    if (j <= 0 || j >= L->c.ny - 1) {
        /* corner rows belong to the walls when the walls are walls */
        if (L->c.wall_kind[SIDE_BOTTOM] != W_PERIODIC && j == 0) return 0;
        if (L->c.wall_kind[SIDE_TOP] != W_PERIODIC && j == L->c.ny - 1) return 0;
    }
    if (i == 0 && L->c.wall_kind[SIDE_LEFT] == W_PRESSURE) return 1;
    if (i == L->c.nx - 1 && L->c.wall_kind[SIDE_RIGHT] == W_PRESSURE) return 1;
    return 0;
}

/* Mode A: a low-order node with a high-order node directly above or below it. */
static int is_iface_node(const or_lattice *L, int i, int j)
{
    if (L->c.iface != 0 || MAP(L, i, j) != 0) return 0;
    if (j > 0 && MAP(L, i, j - 1) == 1) return 1;
    if (j < L->c.ny - 1 && MAP(L, i, j + 1) == 1) return 1;
    return 0;
}

static double native_value(const or_lattice *L, int a, int i, int j);

static void native_moments(const or_lattice *L, int i, int j, double *rho, double *ux, double *uy)
{
    const or_vset *s = &L->set[MAP(L, i, j)];
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < s->q; ++a) {
        double v = native_value(L, a, i, j);
        r += v;
        jx += v * s->cx[a];
        jy += v * s->cy[a];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* Mode A, Sec. 2.2: value of population a of set s at interface node (i, j).
 * rho_I, u_I are the means of the neighbours l (low-order side) and h (high-order
 * side); the non-equilibrium part is extrapolated from the neighbour on s's own side. */
static double iface_value(const or_lattice *L, int s, int a, int i, int j)
{
    int jh, jl;
    if (j > 0 && MAP(L, i, j - 1) == 1) { jh = j - 1; jl = j + 1; }
    else { jh = j + 1; jl = j - 1; }
    double rl, ulx, uly, rh, uhx, uhy;
    native_moments(L, i, jl, &rl, &ulx, &uly);
    native_moments(L, i, jh, &rh, &uhx, &uhy);
    double rI = 0.5 * (rl + rh), uIx = 0.5 * (ulx + uhx), uIy = 0.5 * (uly + uhy);
    const or_vset *vs = &L->set[s];
    int jn = (s == 0) ? jl : jh;
    double rn = (s == 0) ? rl : rh, unx = (s == 0) ? ulx : uhx, uny = (s == 0) ? uly : uhy;
    double fneq = native_value(L, a, i, jn) - feq(vs, a, rn, unx, uny);
    return feq(vs, a, rI, uIx, uIy) + fneq;
}

/* Pressure column (reading of the paper's virtual-boundary construction): node
 * (i, j) with i = 0 or nx-1, in its own set s, gets f_eq(rho_b, u_in) + f_neq of the
 * node one step inwards (seen in set s). */
static double in_set_value(const or_lattice *L, int s, int a, int i, int j);

static double pressure_value(const or_lattice *L, int a, int i, int j)
{
    int s = MAP(L, i, j);
    int ii = (i == 0) ? 1 : L->c.nx - 2;
    int side = (i == 0) ? SIDE_LEFT : SIDE_RIGHT;
    const or_vset *vs = &L->set[s];
    /* moments of the inner node, computed from its values seen in set s */
    double r = 0.0, jx = 0.0, jy = 0.0, vals[OR_QMAX];
    for (int b = 0; b < vs->q; ++b) {
        vals[b] = in_set_value(L, s, b, ii, j);
        r += vals[b];
        jx += vals[b] * vs->cx[b];
        jy += vals[b] * vs->cy[b];
    }
    double ux = jx / r, uy = jy / r;
    return feq(vs, a, L->c.wall_rho[side], ux, uy) + (vals[a] - feq(vs, a, r, ux, uy));
}

/* Population a of the node's own set at a real node (0 <= i < nx, 0 <= j < ny). */
static double native_value(const or_lattice *L, int a, int i, int j)
{
    if (is_pressure_node(L, i, j)) return pressure_value(L, a, i, j);
    if (is_iface_node(L, i, j)) return iface_value(L, 0, a, i, j);
    return F(L, MAP(L, i, j), a, i, j);
}

/* Population a of set s at a real node, as a reader of set s sees it. */
static double in_set_value(const or_lattice *L, int s, int a, int i, int j)
{
    int m = MAP(L, i, j);
    if (m == s) return native_value(L, a, i, j);
    if (L->c.iface == 0) {
        /* mode A */
        if (is_iface_node(L, i, j)) return iface_value(L, s, a, i, j);
        /* one node beyond I: a copy of I */
        if (j > 0 && is_iface_node(L, i, j - 1)) return iface_value(L, s, a, i, j - 1);
        if (j < L->c.ny - 1 && is_iface_node(L, i, j + 1)) return iface_value(L, s, a, i, j + 1);
        return NAN;  /* not reachable for a valid mode-A map */
    }
    /* mode B: Hermite projection of the foreign node into set s */
    const or_vset *vm = &L->set[m];
    double fv[OR_QMAX], a0[1], a1[2], a2[3];
    for (int b = 0; b < vm->q; ++b) fv[b] = native_value(L, b, i, j);
    hermite_coeffs(vm, fv, a0, a1, a2);
    return project_one(&L->set[s], a, a0, a1, a2);
}

/* Stencil read with ghosts (Sec. 3.2: ghost = wall node) and periodic images. */
static double read_value(const or_lattice *L, int s, int a, int i, int j)
{
    int nx = L->c.nx, ny = L->c.ny;
    if (j < 0) j = (L->c.wall_kind[SIDE_BOTTOM] == W_PERIODIC) ? ((j % ny) + ny) % ny : 0;
    if (j > ny - 1) j = (L->c.wall_kind[SIDE_TOP] == W_PERIODIC) ? j % ny : ny - 1;
    if (i < 0) i = (L->c.wall_kind[SIDE_LEFT] == W_PERIODIC) ? ((i % nx) + nx) % nx : 0;
    if (i > nx - 1) i = (L->c.wall_kind[SIDE_RIGHT] == W_PERIODIC) ? i % nx : nx - 1;
    return in_set_value(L, s, a, i, j);
}

/* Psi(Theta) = max[0, min(1, Theta)] (Sec. 3.1) times the difference it limits;
 * a zero difference gives zero. */
static double limited(int limiter, double d_up, double d_down)
{
    if (limiter == 1) return 0.0;
    if (limiter == 2) return d_down;
    if (d_down == 0.0) return 0.0;
    double theta = d_up / d_down;
    double psi = theta < 1.0 ? theta : 1.0;
    if (psi < 0.0) psi = 0.0;
    return d_down * psi;
}

/* Sec. 3.1: face value F_{k+1/2} between nodes k and k+1 for Courant number c,
 * given f at k-1, k, k+1, k+2.  c >= 0: the printed form (upwind node k);
 * c < 0: its mirror image (upwind node k+1). */
static double face_flux(int limiter, double c, double fkm1, double fk, double fkp1, double fkp2)
{
    if (c >= 0.0)
        return fk + 0.5 * (1.0 - c) * limited(limiter, fk - fkm1, fkp1 - fk);
    return fkp1 + 0.5 * (1.0 - fabs(c)) * limited(limiter, fkp1 - fkp2, fk - fkp1);
}

static double tau_of(const or_lattice *L, double rho)
{
    double tau = (L->c.rho_ref > 0.0) ? L->c.kn_ref * L->c.rho_ref / rho : L->c.kn_ref;
    if (L->c.tau_mode == 1) tau -= 0.5 * L->c.dt;
    return tau;
}

static double wall_speed(const or_lattice *L, int side, double t, int comp)
{
    double u = comp == 0 ? L->c.wall_ux[side] : L->c.wall_uy[side];
    if (L->c.wall_omega[side] > 0.0) u *= sin(L->c.wall_omega[side] * t);
    return u;
}

static int is_evolved(const or_lattice *L, int i, int j)
{
    return !is_pressure_node(L, i, j) && !is_iface_node(L, i, j);
}

/* ------------------------------------------------------- storage model -- */

/* C. Wellons' "lowbias32" integer hash (xorshift-multiply finaliser, published 2018):
 * the counter-based source of the stochastic-rounding bits. The key of one stored value
 * names the node, the population and the step that produces it. */
static uint32_t lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

static uint32_t round_key(int i, int j, int nx, int a, uint32_t step)
{
    return lowbias32(lowbias32((uint32_t)j * (uint32_t)nx + (uint32_t)i) ^ lowbias32(((uint32_t)a << 24) ^ step));
}

static float f32_of_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t bits_of_f32(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* BF16 = the upper 16 bits of FP32. Nearest (ties to even) by adding half an ulp of the
 * kept part, or stochastically by adding 16 random bits: the kept part then rounds up
 * with probability equal to the dropped fraction of its magnitude. */
static double bf16_round(float v, int stochastic, uint32_t r)
{
    uint32_t b = bits_of_f32(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return v;
    if (stochastic) b += r & 0xffffu;
    else b += 0x7fffu + ((b >> 16) & 1u);
    return f32_of_bits(b & 0xffff0000u);
}

/* FP16: nearest (ties to even), or stochastically between the two codes that bracket
 * v: the one further from zero with probability (v - lo) / (hi - lo), lo the code
 * towards zero; a 24-bit uniform from the key's upper bits. */
static double f16_round(float v, int stochastic, uint32_t r)
{
    _Float16 h = (_Float16)v;
    if (!stochastic || !(fabsf(v) < 65504.0f) || (float)h == v) return (double)(float)h;
    /* lo: the code next to v towards zero */
    _Float16 lo = h;
    if (fabsf((float)h) > fabsf(v)) {
        uint16_t hb;
        memcpy(&hb, &h, 2);
        hb = (uint16_t)(hb - 1u);
        memcpy(&lo, &hb, 2);
    }
    uint16_t lb;
    memcpy(&lb, &lo, 2);
    uint16_t ub = (uint16_t)(lb + 1u);
    _Float16 hi;
    memcpy(&hi, &ub, 2);
    float lof = (float)lo, hif = (float)hi;
    float frac = (v - lof) / (hif - lof);
    float u = (float)(r >> 8) * (1.0f / 16777216.0f);
    return (double)(u < frac ? hif : lof);
}

/* One stored value of population a at node (i, j): f -> the format -> f. `set_value`:
 * a value the wall sets (rounded to nearest, as every value that is not an update of
 * the population's own previous value). */
double or_store_round(int mode, double d, uint32_t bits, int set_value)
{
    switch (mode) {
        case ST_F32_DEV: return (double)(float)d;
        case ST_F16_DEV: return f16_round((float)d, 0, 0);
        case ST_BF16_DEV: return bf16_round((float)d, 0, 0);
        case ST_F16_DEV_SR: return f16_round((float)d, !set_value, bits);
        case ST_BF16_DEV_SR: return bf16_round((float)d, !set_value, bits);
        default: return d;
    }
}

static double stored(const or_lattice *L, int s, int a, int i, int j, double f, int set_value)
{
    if (L->store == ST_EXACT) return f;
    if (L->store == ST_F32) return (double)(float)f;
    const double w = L->set[s].w[a], r = L->rho_r[i];
    const uint32_t key = round_key(i, j, L->c.nx, a, (uint32_t)(L->step + 1));
    return w * (r + or_store_round(L->store, f / w - r, key, set_value));
}

/* One node: Sec. 3.1 update of every population of its set, then the Sec. 3.2 wall
 * overwrite when the node lies on a diffuse wall. */
static void update_node(or_lattice *L, int i, int j)
{
    int s = MAP(L, i, j);
    const or_vset *vs = &L->set[s];
    double rho, ux, uy;
    native_moments(L, i, j, &rho, &ux, &uy);
    double tau = tau_of(L, rho);
    double dt = L->c.dt, h = L->c.h;
    double fnew[OR_QMAX];
    for (int a = 0; a < vs->q; ++a) {
        double cxa = vs->cx[a] * dt / h, cya = vs->cy[a] * dt / h;
        double x[5], y[5];
        for (int k = -2; k <= 2; ++k) {
            x[k + 2] = read_value(L, s, a, i + k, j);
            y[k + 2] = read_value(L, s, a, i, j + k);
        }
        double fpx = face_flux(L->c.limiter, cxa, x[1], x[2], x[3], x[4]);  /* F_{i+1/2} */
        double fmx = face_flux(L->c.limiter, cxa, x[0], x[1], x[2], x[3]);  /* F_{i-1/2} */
        double fpy = face_flux(L->c.limiter, cya, y[1], y[2], y[3], y[4]);
        double fmy = face_flux(L->c.limiter, cya, y[0], y[1], y[2], y[3]);
        double f0 = x[2];
        fnew[a] = f0 - cxa * (fpx - fmx) - cya * (fpy - fmy)
                + (dt / tau) * (feq(vs, a, rho, ux, uy) - f0)
                + force(vs, a, rho, ux, uy, L->c.gx, L->c.gy) * dt;
    }
    int side = -1, set_by_wall[OR_QMAX] = {0};
    if (j == 0 && L->c.wall_kind[SIDE_BOTTOM] == W_DIFFUSE) side = SIDE_BOTTOM;
    if (j == L->c.ny - 1 && L->c.wall_kind[SIDE_TOP] == W_DIFFUSE) side = SIDE_TOP;
    if (side >= 0) {
        double ny_ = (side == SIDE_BOTTOM) ? 1.0 : -1.0;   /* wall normal into the gas */
        double tnew = L->t + dt;
        double uwx = wall_speed(L, side, tnew, 0), uwy = wall_speed(L, side, tnew, 1);
        double num = 0.0, den = 0.0;
        for (int a = 0; a < vs->q; ++a) {
            double xn = vs->cy[a] * ny_;
            if (xn < 0.0) num += fabs(xn) * fnew[a];
            if (xn > 0.0) den += fabs(xn) * feq(vs, a, 1.0, uwx, uwy);
        }
        double rho_w = num / den;
        for (int a = 0; a < vs->q; ++a)
            if (vs->cy[a] * ny_ > 0.0) {
                fnew[a] = rho_w * feq(vs, a, 1.0, uwx, uwy);
                set_by_wall[a] = 1;
            }
    }
    for (int a = 0; a < vs->q; ++a) FN(L, s, a, i, j) = stored(L, s, a, i, j, fnew[a], set_by_wall[a]);
}

/* ------------------------------------------------------------- public API -- */

or_lattice *or_create(const or_cfg *cfg, const uint8_t *map)
{
    or_lattice *L = (or_lattice *)calloc(1, sizeof(or_lattice));
    if (!L) return NULL;
    L->c = *cfg;
    if (make_set(cfg->n1d_lo, &L->set[0]) || make_set(cfg->n1d_hi, &L->set[1])) {
        free(L);
        return NULL;
    }
    size_t cells = (size_t)cfg->nx * (size_t)cfg->ny;
    L->store = ST_EXACT;
    L->rho_r = (double *)calloc((size_t)cfg->nx, sizeof(double));
    L->map = (uint8_t *)malloc(cells);
    memcpy(L->map, map, cells);
    for (int s = 0; s < 2; ++s) {
        L->f[s] = (double *)calloc(cells * (size_t)L->set[s].q, sizeof(double));
        L->fn[s] = (double *)calloc(cells * (size_t)L->set[s].q, sizeof(double));
    }
    return L;
}

void or_destroy(or_lattice *L)
{
    if (!L) return;
    for (int s = 0; s < 2; ++s) { free(L->f[s]); free(L->fn[s]); }
    free(L->rho_r);
    free(L->map);
    free(L);
}

/* f = f_eq(rho, u) in every node's own set (rho, ux, uy are [ny][nx]). */
void or_init_equilibrium(or_lattice *L, const double *rho, const double *ux, const double *uy)
{
    for (int j = 0; j < L->c.ny; ++j)
        for (int i = 0; i < L->c.nx; ++i) {
            size_t c = (size_t)j * L->c.nx + i;
            int s = MAP(L, i, j);
            for (int a = 0; a < L->set[s].q; ++a)
                F(L, s, a, i, j) = feq(&L->set[s], a, rho[c], ux[c], uy[c]);
        }
    L->t = 0.0;
    L->step = 0;
}

/* Stored populations of set s ([q][ny][nx]); only nodes whose map is s are read. */
void or_set_populations(or_lattice *L, int s, const double *src)
{
    memcpy(L->f[s], src, sizeof(double) * (size_t)L->set[s].q * L->c.nx * L->c.ny);
}

/* Populations of set s as a reader of set s sees every node: own-set nodes give
 * their state (or the boundary / interface rule), foreign nodes their mode-A/B view. */
void or_get_populations(const or_lattice *L, int s, double *dst)
{
    int nx = L->c.nx, ny = L->c.ny;
    for (int a = 0; a < L->set[s].q; ++a)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                dst[((size_t)a * ny + j) * nx + i] = in_set_value(L, s, a, i, j);
}

/* Storage model for the following steps (ST_*), with the reference density of each
 * column's deviation (rho_r[nx]; NULL: rho0 everywhere). */
int or_set_storage(or_lattice *L, int mode, double rho0, const double *rho_r)
{
    if (mode < ST_EXACT || mode > ST_BF16_DEV_SR) return -1;
    L->store = mode;
    for (int i = 0; i < L->c.nx; ++i) L->rho_r[i] = rho_r ? rho_r[i] : rho0;
    return 0;
}

void or_step(or_lattice *L, int64_t n)
{
    int nx = L->c.nx, ny = L->c.ny;
    for (int64_t k = 0; k < n; ++k) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (is_evolved(L, i, j)) update_node(L, i, j);
        for (int s = 0; s < 2; ++s) {
            double *tmp = L->f[s];
            L->f[s] = L->fn[s];
            L->fn[s] = tmp;
        }
        /* nodes that are not evolved keep no state of their own; carry the old
         * buffer's contents so that the state arrays stay defined */
        L->t += L->c.dt;
        L->step += 1;
    }
}

/* Moments of every node from its own-set populations, out = [10][ny][nx]:
 * rho, ux, uy, P_xy = sum f (xi_x - u_x)(xi_y - u_y),
 * Pi^neq_xx, Pi^neq_xy, Pi^neq_yy = sum (f - f_eq) xi xi,
 * q_x, q_y = (1/2) sum f |xi - u|^2 (xi - u). */
void or_moments(const or_lattice *L, double *out)
{
    int nx = L->c.nx, ny = L->c.ny;
    size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const or_vset *vs = &L->set[MAP(L, i, j)];
            double fv[OR_QMAX], rho = 0.0, jx = 0.0, jy = 0.0;
            for (int a = 0; a < vs->q; ++a) {
                fv[a] = native_value(L, a, i, j);
                rho += fv[a];
                jx += fv[a] * vs->cx[a];
                jy += fv[a] * vs->cy[a];
            }
            double ux = jx / rho, uy = jy / rho;
            double pxy = 0, nxx = 0, nxy = 0, nyy = 0, qx = 0, qy = 0;
            for (int a = 0; a < vs->q; ++a) {
                double cx = vs->cx[a] - ux, cy = vs->cy[a] - uy;
                double fne = fv[a] - feq(vs, a, rho, ux, uy);
                pxy += fv[a] * cx * cy;
                nxx += fne * vs->cx[a] * vs->cx[a];
                nxy += fne * vs->cx[a] * vs->cy[a];
                nyy += fne * vs->cy[a] * vs->cy[a];
                qx += 0.5 * fv[a] * (cx * cx + cy * cy) * cx;
                qy += 0.5 * fv[a] * (cx * cx + cy * cy) * cy;
            }
            size_t c = (size_t)j * nx + i;
            double vals[10] = {rho, ux, uy, pxy, nxx, nxy, nyy, qx, qy, 0.0};
            for (int m = 0; m < 9; ++m) out[m * N + c] = vals[m];
            out[9 * N + c] = (double)MAP(L, i, j);
        }
}

double or_time(const or_lattice *L) { return L->t; }
int64_t or_steps(const or_lattice *L) { return L->step; }
