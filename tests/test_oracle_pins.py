"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms of the
Gauss-Hermite rules (Eq. (weight)), library routines (numpy's Gauss-Hermite rule),
moment identities of Eq. (demoeq) / Eq. (demoforce), textbook reductions of the
Sec. 3.1 TVD scheme (exact shift, first-order upwind, Lax-Wendroff), conservation
and fixed-point invariants, the modified-equation viscosity of the forward-Euler
scheme, and exact solutions of the discrete-velocity model between diffuse walls
(Sec. 3.2) computed by eigen-modes in ``dvm_exact``.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

import oracle
from lbinputs import band_map

import dvm_exact

PERIODIC_Y = {"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}}


def dfact(k):
    """(k-1)!! for even k: the k-th moment of the unit Gaussian; 0 for odd k."""
    if k % 2:
        return 0.0
    return float(np.prod(np.arange(k - 1, 0, -2))) if k > 0 else 1.0


# ------------------------------------------------------------------ Eq. (weight)

@pytest.mark.parametrize("n", [3, 4, 6])
def test_gauss_hermite_matches_library(n):
    x, w = oracle.gauss_hermite(n)
    xr, wr = hermegauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(w, wr / math.sqrt(2 * math.pi), rtol=1e-13, atol=0)


def test_gauss_hermite_closed_forms():
    # n = 3: He_3 = x^3 - 3x; weights n!/[n He_2]^2 with He_2 = x^2 - 1
    x, w = oracle.gauss_hermite(3)
    np.testing.assert_allclose(x, [-math.sqrt(3), 0.0, math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 2 / 3, 1 / 6], rtol=1e-14)
    # n = 4: He_4 = x^4 - 6x^2 + 3, x^2 = 3 -/+ sqrt(6), w = (3 +/- sqrt(6)) / 12
    x, w = oracle.gauss_hermite(4)
    s6 = math.sqrt(6)
    np.testing.assert_allclose(x, [-math.sqrt(3 + s6), -math.sqrt(3 - s6), math.sqrt(3 - s6), math.sqrt(3 + s6)],
                               rtol=1e-14)
    np.testing.assert_allclose(w, [(3 - s6) / 12, (3 + s6) / 12, (3 + s6) / 12, (3 - s6) / 12], rtol=1e-13)
    # n = 6: He_6 = x^6 - 15x^4 + 45x^2 - 15: x^2 solves z^3 - 15 z^2 + 45 z - 15 = 0
    x, _ = oracle.gauss_hermite(6)
    z = np.sort(np.roots([1, -15, 45, -15]).real)
    np.testing.assert_allclose(np.sort(x[3:] ** 2), z, rtol=1e-13)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_gauss_hermite_degree(n):
    x, w = oracle.gauss_hermite(n)
    for k in range(0, 2 * n):
        np.testing.assert_allclose(np.sum(w * x ** k), dfact(k), atol=1e-12 * max(1, dfact(k)))
    # and not beyond: degree 2n fails
    assert abs(np.sum(w * x ** (2 * n)) - dfact(2 * n)) > 1e-3


@pytest.mark.parametrize("n", [3, 4, 6])
def test_product_set(n):
    cx, cy, w = oracle.velocity_set(n)
    x, w1 = oracle.gauss_hermite(n)
    assert len(w) == n * n
    a = np.arange(n * n)
    np.testing.assert_allclose(cx, x[a % n])
    np.testing.assert_allclose(cy, x[a // n])
    np.testing.assert_allclose(w, w1[a % n] * w1[a // n], rtol=1e-15)


# ---------------------------------------------------- Eq. (demoeq), (demoforce)

def gauss_moment(a, b):
    return dfact(a) * dfact(b)


def truncated_feq_moment(a, b, rho, ux, uy):
    """Integral of omega rho {1 + xi.u + [(xi.u)^2 - u^2]/2} xi_x^a xi_y^b."""
    M = gauss_moment
    return rho * (M(a, b) + ux * M(a + 1, b) + uy * M(a, b + 1)
                  + 0.5 * (ux * ux * M(a + 2, b) + 2 * ux * uy * M(a + 1, b + 1) + uy * uy * M(a, b + 2))
                  - 0.5 * (ux * ux + uy * uy) * M(a, b))


@pytest.mark.parametrize("n", [3, 4, 6])
def test_feq_moments_equal_continuous(n):
    cx, cy, _ = oracle.velocity_set(n)
    rng = np.random.default_rng(11 + n)
    for _ in range(5):
        rho, ux, uy = rng.uniform(0.5, 2.0), rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)
        f = oracle.feq(n, rho, ux, uy)
        top = 2 * n - 3       # the quadrature integrates degree 2n-1 per axis exactly
        for a in range(top + 1):
            for b in range(top + 1):
                ref = truncated_feq_moment(a, b, rho, ux, uy)
                np.testing.assert_allclose(np.sum(f * cx ** a * cy ** b), ref, rtol=1e-12, atol=1e-13)
        # order <= 2 are the Maxwellian's: rho, rho u, rho (I + u u)
        np.testing.assert_allclose(np.sum(f), rho, rtol=1e-14)
        np.testing.assert_allclose(np.sum(f * cx * cx), rho * (1 + ux * ux), rtol=1e-13)
        np.testing.assert_allclose(np.sum(f * cx * cy), rho * ux * uy, rtol=1e-12, atol=1e-15)
        # third order: the truncated form has no u u u term (N = 2, Eq. (demoeq))
        np.testing.assert_allclose(np.sum(f * cx ** 3), 3 * rho * ux, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_collision_conserves_mass_and_momentum(n):
    cx, cy, w = oracle.velocity_set(n)
    rng = np.random.default_rng(5 + n)
    for _ in range(5):
        f = w * (1 + 0.2 * rng.standard_normal(len(w)))
        rho = f.sum()
        ux, uy = (f * cx).sum() / rho, (f * cy).sum() / rho
        fe = oracle.feq(n, rho, ux, uy)
        np.testing.assert_allclose(np.sum(fe - f), 0.0, atol=1e-14)
        np.testing.assert_allclose(np.sum((fe - f) * cx), 0.0, atol=1e-14)
        np.testing.assert_allclose(np.sum((fe - f) * cy), 0.0, atol=1e-14)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_force_moments(n):
    cx, cy, _ = oracle.velocity_set(n)
    rho, ux, uy, gx, gy = 1.3, 0.07, -0.04, 0.011, -0.023
    g = oracle.force(n, rho, ux, uy, gx, gy)
    np.testing.assert_allclose(g.sum(), 0.0, atol=1e-15)
    np.testing.assert_allclose([np.sum(g * cx), np.sum(g * cy)], [rho * gx, rho * gy], rtol=1e-13)
    np.testing.assert_allclose(np.sum(g * cx * cx), rho * 2 * gx * ux, rtol=1e-12)
    np.testing.assert_allclose(np.sum(g * cx * cy), rho * (gx * uy + gy * ux), rtol=1e-12)
    np.testing.assert_allclose(np.sum(g * cy * cy), rho * 2 * gy * uy, rtol=1e-12)


# ------------------------------------------------------- Hermite projection (B)

def hermite2(n, f):
    cx, cy, _ = oracle.velocity_set(n)
    return np.array([f.sum(), (f * cx).sum(), (f * cy).sum(), (f * (cx * cx - 1)).sum(),
                     (f * cx * cy).sum(), (f * (cy * cy - 1)).sum()])


@pytest.mark.parametrize("src,dst", [(3, 6), (6, 3), (3, 4), (4, 6), (6, 4)])
def test_projection_keeps_second_order_coefficients(src, dst):
    _, _, w = oracle.velocity_set(src)
    rng = np.random.default_rng(src * 10 + dst)
    f = w * (1 + 0.3 * rng.standard_normal(len(w)))
    g = oracle.project(src, f, dst)
    np.testing.assert_allclose(hermite2(dst, g), hermite2(src, f), rtol=1e-12, atol=1e-14)
    # and back again
    np.testing.assert_allclose(hermite2(src, oracle.project(dst, g, src)), hermite2(src, f), rtol=1e-12,
                               atol=1e-14)


def test_projection_of_equilibrium_is_equilibrium():
    for src, dst in [(3, 6), (6, 3), (4, 6)]:
        f = oracle.feq(src, 1.2, 0.05, -0.08)
        np.testing.assert_allclose(oracle.project(src, f, dst), oracle.feq(dst, 1.2, 0.05, -0.08), rtol=1e-12,
                                   atol=1e-15)


# ----------------------------------------------------------- Sec. 3.1 (TVD)

def x_profile_state(o, n1d, rng):
    cx, cy, w = oracle.velocity_set(n1d)
    prof = 1 + 0.3 * rng.standard_normal((len(w), 1, o.nx))
    return (w[:, None, None] * np.broadcast_to(prof, (len(w), o.ny, o.nx))).copy()


def test_tvd_unit_courant_is_exact_shift():
    # D2Q9, |c_x| = 1 for xi_x = +/- sqrt(3): the scheme must move each population one node
    nx = 16
    o = oracle.Oracle(nx, 4, np.zeros((4, nx)), n1d_lo=3, n1d_hi=6, h=1.0 / nx, dt=(1.0 / nx) / math.sqrt(3),
                      kn_ref=1e300, rho_ref=0.0, walls=PERIODIC_Y)
    rng = np.random.default_rng(1)
    f0 = x_profile_state(o, 3, rng)
    o.set_populations(0, f0)
    o.step(1)
    f1 = o.populations(0)
    cx, _, _ = oracle.velocity_set(3)
    for a in range(9):
        shift = int(round(cx[a] / math.sqrt(3)))
        np.testing.assert_allclose(f1[a], np.roll(f0[a], shift, axis=1), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("limiter,scheme", [(1, "upwind"), (2, "lax-wendroff")])
def test_tvd_limiter_extremes_are_textbook_schemes(limiter, scheme):
    nx = 24
    o = oracle.Oracle(nx, 4, np.zeros((4, nx)), n1d_lo=3, n1d_hi=6, h=1.0 / nx, cfl=0.45, kn_ref=1e300,
                      rho_ref=0.0, limiter=limiter, walls=PERIODIC_Y)
    rng = np.random.default_rng(2)
    f0 = x_profile_state(o, 3, rng)
    o.set_populations(0, f0)
    o.step(1)
    f1 = o.populations(0)
    cx, _, _ = oracle.velocity_set(3)
    for a in range(9):
        c = cx[a] * o.dt / o.h
        u = f0[a]
        um, up = np.roll(u, 1, axis=1), np.roll(u, -1, axis=1)
        if scheme == "upwind":
            ref = u - c * (u - um) if c >= 0 else u - c * (up - u)
        else:
            ref = u - 0.5 * c * (up - um) + 0.5 * c * c * (up - 2 * u + um)
        np.testing.assert_allclose(f1[a], ref, rtol=1e-13, atol=1e-15)


def test_tvd_minmod_total_variation_does_not_grow():
    nx = 64
    o = oracle.Oracle(nx, 4, np.zeros((4, nx)), n1d_lo=3, n1d_hi=6, h=1.0 / nx, cfl=0.9, kn_ref=1e300,
                      rho_ref=0.0, walls=PERIODIC_Y)
    rng = np.random.default_rng(3)
    f = x_profile_state(o, 3, rng)
    f[:, :, nx // 3: nx // 2] *= 3.0   # a discontinuity too
    o.set_populations(0, f)
    tv = lambda g: np.abs(np.diff(np.concatenate([g[:, 0, :], g[:, 0, :1]], axis=1), axis=1)).sum(axis=1)
    prev = tv(f)
    for _ in range(20):
        o.step(1)
        cur = tv(o.populations(0))
        assert np.all(cur <= prev * (1 + 1e-13) + 1e-15)
        prev = cur


# ----------------------------------------------------- invariants of a step

@pytest.mark.parametrize("n1d_set", [(3, 0), (6, 1), (4, 1)])
def test_periodic_box_conserves_mass_and_momentum(n1d_set):
    n1d, s = n1d_set
    nx, ny = 12, 10
    m = np.full((ny, nx), s, dtype=np.uint8)
    o = oracle.Oracle(nx, ny, m, n1d_lo=3 if s else n1d, n1d_hi=n1d if s else 6, h=1.0 / ny, cfl=0.5,
                      kn_ref=0.05, walls=PERIODIC_Y)
    rng = np.random.default_rng(4)
    cx, cy, w = oracle.velocity_set(n1d)
    f = w[:, None, None] * (1 + 0.1 * rng.standard_normal((len(w), ny, nx)))
    o.set_populations(s, f)
    tot = lambda g: np.array([g.sum(), (g * cx[:, None, None]).sum(), (g * cy[:, None, None]).sum()])
    t0 = tot(o.populations(s))
    o.step(15)
    np.testing.assert_allclose(tot(o.populations(s)), t0, rtol=0, atol=1e-12 * abs(t0[0]))


def test_body_force_momentum_gain():
    nx, ny = 8, 8
    m = np.zeros((ny, nx), dtype=np.uint8)
    gx, gy = 2e-3, -1e-3
    o = oracle.Oracle(nx, ny, m, h=1.0 / ny, kn_ref=0.05, gx=gx, gy=gy, walls=PERIODIC_Y)
    rng = np.random.default_rng(7)
    cx, cy, w = oracle.velocity_set(3)
    f = w[:, None, None] * (1 + 0.05 * rng.standard_normal((9, ny, nx)))
    o.set_populations(0, f)
    mass = f.sum()
    p0 = np.array([(f * cx[:, None, None]).sum(), (f * cy[:, None, None]).sum()])
    o.step(10)
    g1 = o.populations(0)
    p1 = np.array([(g1 * cx[:, None, None]).sum(), (g1 * cy[:, None, None]).sum()])
    np.testing.assert_allclose(p1 - p0, 10 * o.dt * mass * np.array([gx, gy]), rtol=1e-10)


@pytest.mark.parametrize("iface", ["hermite", "paper"])
def test_rest_state_with_resting_walls_is_fixed_point(iface):
    nx, ny = 8, 24
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 5), kn_ref=0.1, iface=iface,
                      walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"}})
    o.init_equilibrium(1.0, 0.0, 0.0)
    f0 = [o.populations(0), o.populations(1)]
    o.step(10)
    for s in (0, 1):
        np.testing.assert_allclose(o.populations(s), f0[s], rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("iface", ["hermite", "paper"])
def test_uniform_flow_is_fixed_point_across_interfaces(iface):
    nx, ny = 8, 24
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 6), h=1.0 / ny, kn_ref=0.1, iface=iface, walls=PERIODIC_Y)
    o.init_equilibrium(1.1, 0.13, -0.07)
    f0 = [o.populations(0), o.populations(1)]
    o.step(8)
    for s in (0, 1):
        np.testing.assert_allclose(o.populations(s), f0[s], rtol=1e-13, atol=1e-16)


def test_diffuse_wall_zero_normal_mass_flux():
    nx, ny = 4, 20
    uw = 0.1
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 4), kn_ref=0.2,
                      walls={"bottom": {"kind": "diffuse", "ux": -uw}, "top": {"kind": "diffuse", "ux": uw}})
    o.init_equilibrium(1.0, 0.0, 0.0)
    o.step(25)
    cx, cy, w = oracle.velocity_set(6)
    f = o.populations(1)
    for j in (0, ny - 1):
        flux = np.sum(f[:, j, :] * cy[:, None], axis=0)
        np.testing.assert_allclose(flux, 0.0, atol=1e-15)
        # the gas-bound half is a wall Maxwellian: ratio to S(u_W) is one constant
        sgn = 1 if j == 0 else -1
        out = sgn * cy > 0
        S = oracle.feq(6, 1.0, -uw if j == 0 else uw, 0.0)
        ratio = f[out, j, 0] / S[out]
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-13)


# --------------------------------------------------- viscosity of the scheme

def shear_wave_viscosity(ny, kn, n1d, tau_mode=0):
    s = 0 if n1d == 3 else 1
    o = oracle.Oracle(4, ny, np.full((ny, 4), s), n1d_lo=3, n1d_hi=n1d if s else 6, kn_ref=kn, rho_ref=0.0,
                      tau_mode=tau_mode, walls=PERIODIC_Y, cfl=0.5)
    y = np.arange(ny) / ny
    o.init_equilibrium(1.0, np.broadcast_to((1e-3 * np.sin(2 * np.pi * y))[:, None], (ny, 4)), 0.0)
    amp = lambda: 2 * np.mean(o.moments()["ux"][:, 0] * np.sin(2 * np.pi * y))
    o.step(int(20 * kn / o.dt) + 1)             # let the stress build up first
    a0, t0 = amp(), o.time
    o.step(int(0.3 / ((kn + o.dt / 2) * (2 * np.pi) ** 2) / o.dt) + 1)
    return -math.log(amp() / a0) / ((2 * np.pi) ** 2 * (o.time - t0)), o.dt


@pytest.mark.parametrize("n1d,ny", [(3, 128), (6, 256)])
def test_shear_wave_viscosity_is_tau_plus_half_dt(n1d, ny):
    """Forward Euler + a second-order flux: the modified equation gives
    nu = c_s^2 (tau + dt/2) with c_s^2 = T = 1 (collide-then-stream would give tau - dt/2)."""
    kn = 0.005
    nu, dt = shear_wave_viscosity(ny, kn, n1d)
    assert abs(nu - (kn + 0.5 * dt)) < 0.12 * (0.5 * dt), (nu, kn, dt)
    nu1, dt1 = shear_wave_viscosity(ny, kn, n1d, tau_mode=1)
    assert abs(nu1 - kn) < 0.12 * (0.5 * dt1), (nu1, kn, dt1)


# ------------------------------- exact discrete-velocity solutions, Sec. 3.2

def run_channel(ny, n1d, kn, u_bottom=0.0, u_top=0.0, G=0.0, t_visc=1.0):
    s = 0 if n1d == 3 else 1
    o = oracle.Oracle(4, ny, np.full((ny, 4), s), n1d_lo=3, n1d_hi=n1d if s else 6, kn_ref=kn, gx=G,
                      walls={"bottom": {"kind": "diffuse", "ux": u_bottom}, "top": {"kind": "diffuse", "ux": u_top}})
    exact = dvm_exact.channel(n1d, kn, u_bottom=u_bottom, u_top=u_top, G=G)
    y = np.arange(ny) / (ny - 1)
    o.init_equilibrium(1.0, np.broadcast_to(exact(y)[:, None], (ny, 4)), 0.0)
    o.step(int(t_visc / kn / o.dt))
    return y, o.moments()["ux"][:, 0], exact


@pytest.mark.parametrize("n1d", [3, 6])
def test_couette_converges_to_exact_discrete_velocity_solution(n1d):
    kn, U = 0.1, 0.01
    res = []
    for ny in (48, 96):
        y, u, exact = run_channel(ny, n1d, kn, -U, U)
        err = np.max(np.abs(u - exact(y))) / U
        res.append(err)
    # first-order convergence in h (ghost = wall node) towards the exact profile
    assert res[1] < 0.6 * res[0], res
    assert res[1] < 0.02, res
    # and the slip length of the bulk, extrapolated in h
    zs = []
    for ny in (48, 96):
        y, u, exact = run_channel(ny, n1d, kn, -U, U)
        c = (y > 0.3) & (y < 0.7)
        zs.append((2 * U / np.polyfit(y[c], u[c], 1)[0] - 1) / 2)
    ye = np.linspace(0.3, 0.7, 41)
    z_exact = (2 * U / np.polyfit(ye, exact(ye), 1)[0] - 1) / 2
    z_extrap = 2 * zs[1] - zs[0]
    assert abs(z_extrap - z_exact) < 0.01 * z_exact, (zs, z_extrap, z_exact)


@pytest.mark.parametrize("n1d", [3, 6])
def test_poiseuille_converges_to_exact_discrete_velocity_solution(n1d):
    kn, G = 0.1, 2e-3
    uc = []
    for ny in (48, 96):
        y, u, exact = run_channel(ny, n1d, kn, G=G)
        uc.append(u[ny // 2] if ny % 2 else 0.5 * (u[ny // 2 - 1] + u[ny // 2]))
    ref = float(exact(0.5))
    extrap = 2 * uc[1] - uc[0]
    assert abs(extrap - ref) < 0.006 * ref, (uc, extrap, ref)


# -------------------------------------------------- Sec. 2.2 (mode A) and the
# pressure columns, on states where the rule has a plain answer

def test_mode_a_interface_values_on_a_linear_equilibrium():
    nx, ny, rows = 4, 20, 4
    o = oracle.Oracle(nx, ny, band_map(nx, ny, rows), kn_ref=0.1, iface="paper",
                      walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"}})
    y = np.arange(ny) / (ny - 1)
    u = 0.05 * (2 * y - 1)
    o.init_equilibrium(1.0, np.broadcast_to(u[:, None], (ny, nx)), 0.0)
    fl, fh = o.populations(0), o.populations(1)
    for I, beyond_l, beyond_h in ((rows, rows - 1, rows + 1), (ny - 1 - rows, ny - rows, ny - 2 - rows)):
        # linear u: the mean of the two neighbours is u at I; no non-equilibrium part
        np.testing.assert_allclose(fl[:, I, 0], oracle.feq(3, 1.0, u[I], 0.0), rtol=1e-13)
        np.testing.assert_allclose(fh[:, I, 0], oracle.feq(6, 1.0, u[I], 0.0), rtol=1e-13)
        # one node beyond I, each set sees a copy of I
        np.testing.assert_allclose(fl[:, beyond_l, 0], fl[:, I, 0], rtol=1e-15)
        np.testing.assert_allclose(fh[:, beyond_h, 0], fh[:, I, 0], rtol=1e-15)


def test_pressure_column_rule_on_equilibrium():
    nx, ny = 12, 10
    rho = np.broadcast_to(np.linspace(1.4, 1.0, nx)[None, :], (ny, nx))
    o = oracle.Oracle(nx, ny, np.zeros((ny, nx)), kn_ref=0.2,
                      walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"},
                             "left": {"kind": "pressure", "rho": 1.7}, "right": {"kind": "pressure", "rho": 0.9}})
    o.init_equilibrium(rho, 0.02, 0.0)
    f = o.populations(0)
    for j in range(1, ny - 1):
        np.testing.assert_allclose(f[:, j, 0], oracle.feq(3, 1.7, 0.02, 0.0), rtol=1e-13)
        np.testing.assert_allclose(f[:, j, nx - 1], oracle.feq(3, 0.9, 0.02, 0.0), rtol=1e-13)
    # corners stay wall nodes
    np.testing.assert_allclose(f[:, 0, 0], oracle.feq(3, rho[0, 0], 0.02, 0.0), rtol=1e-13)


# ------------------------------------------------------------- moments output

def test_moment_definitions():
    nx, ny = 4, 12
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 3), kn_ref=0.2,
                      walls={"bottom": {"kind": "diffuse", "ux": -0.1}, "top": {"kind": "diffuse", "ux": 0.1}})
    o.init_equilibrium(1.0, 0.03, -0.01)
    m = o.moments()
    for k in ("pxy", "neq_xx", "neq_xy", "neq_yy"):
        np.testing.assert_allclose(m[k], 0.0, atol=1e-15)
    o.step(30)
    m = o.moments()
    # P_xy = sum f (xi_x - u_x)(xi_y - u_y) = sum f xi_x xi_y - rho u_x u_y = Pi^neq_xy
    np.testing.assert_allclose(m["pxy"], m["neq_xy"], rtol=1e-10, atol=1e-15)
    assert np.abs(m["pxy"]).max() > 1e-4


def test_relaxation_time_follows_local_density():
    """tau = Kn_ref rho_ref / rho (collision rate p / mu, Eq. (KN) with mu fixed): at
    rho = 2 the shear wave decays with nu = kn_ref rho_ref / 2 + dt / 2."""
    ny, kn_ref = 128, 0.01
    o = oracle.Oracle(4, ny, np.zeros((ny, 4)), kn_ref=kn_ref, rho_ref=1.0, walls=PERIODIC_Y, cfl=0.5)
    y = np.arange(ny) / ny
    o.init_equilibrium(2.0, np.broadcast_to((1e-3 * np.sin(2 * np.pi * y))[:, None], (ny, 4)), 0.0)
    amp = lambda: 2 * np.mean(o.moments()["ux"][:, 0] * np.sin(2 * np.pi * y))
    o.step(int(20 * 0.005 / o.dt) + 1)
    a0, t0 = amp(), o.time
    o.step(600)
    nu = -math.log(amp() / a0) / ((2 * np.pi) ** 2 * (o.time - t0))
    assert abs(nu - (0.005 + 0.5 * o.dt)) < 0.12 * (0.5 * o.dt), (nu, o.dt)
