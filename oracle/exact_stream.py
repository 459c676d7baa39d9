"""FP64 CPU oracle of the D2Q9 stream-and-collide reduction of the method.

TEST INFRASTRUCTURE. Only ``tests/`` import this module; the product path never does.

With the D2Q9 abscissae +-sqrt(3) (Sec. 2.1: roots of the third Hermite polynomial,
weights 1/6, 2/3, 1/6) and the time step dt = h / sqrt(3), every Courant number
xi dt / h of the Sec. 3.1 update is 0 or +-1: a population moves exactly one node per
step. This is the textbook lattice BGK form, the one in which the effective viscosity
is c_s^2 (tau - dt / 2) (here c_s^2 = T = 1). One step, in this order:

    stream:  f'_a(x, y) = f_a(x - s_x(a), y - s_y(a)),  s = sign(xi_a)
    collide: f_a <- f'_a + (dt / tau) [f_eq_a(rho', u') - f'_a] + dt g_a(rho', u')

with f_eq of Eq. (demoeq) (second-order Hermite equilibrium, T = 1), g of
Eq. (demoforce) and tau = kn_ref rho_ref / rho' (Eq. (KN) as the library reads it;
constant kn_ref when rho_ref <= 0), minus dt / 2 when tau_mode = 1. Periodic in x and y.
Populations are [9][ny][nx], population a = iy * 3 + ix over ascending abscissae.
"""
from __future__ import annotations

import numpy as np


def d2q9():
    """Abscissae and weights: product of the three-point Gauss-Hermite rule."""
    r = np.sqrt(3.0)
    c1 = np.array([-r, 0.0, r])
    w1 = np.array([1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0])
    cx = np.tile(c1, 3)
    cy = np.repeat(c1, 3)
    w = np.outer(w1, w1).ravel()
    return cx, cy, w


def equilibrium(rho, ux, uy):
    """f_eq_a = w_a rho [1 + xi.u + ((xi.u)^2 - u^2) / 2], Eq. (demoeq) with T = 1."""
    cx, cy, w = d2q9()
    eu = cx[:, None, None] * ux[None] + cy[:, None, None] * uy[None]
    usq = ux * ux + uy * uy
    return w[:, None, None] * rho[None] * (1.0 + eu + 0.5 * (eu * eu - usq[None]))


def force(rho, ux, uy, gx, gy):
    """g_a = w_a rho [g.xi + (g.xi)(xi.u) - g.u], Eq. (demoforce) with T = 1."""
    cx, cy, w = d2q9()
    gxi = gx * cx + gy * cy
    eu = cx[:, None, None] * ux[None] + cy[:, None, None] * uy[None]
    gu = gx * ux + gy * uy
    return w[:, None, None] * rho[None] * (gxi[:, None, None] + gxi[:, None, None] * eu - gu[None])


def moments(f):
    cx, cy, _ = d2q9()
    rho = f.sum(axis=0)
    ux = (cx[:, None, None] * f).sum(axis=0) / rho
    uy = (cy[:, None, None] * f).sum(axis=0) / rho
    return rho, ux, uy


def stream(f):
    """f'_a(x) = f_a(x - sign(xi_a)) on the periodic lattice."""
    cx, cy, _ = d2q9()
    out = np.empty_like(f)
    for a in range(9):
        out[a] = np.roll(f[a], shift=(int(np.sign(cy[a])), int(np.sign(cx[a]))), axis=(0, 1))
    return out


def step(f, dt, kn_ref, rho_ref=0.0, tau_mode=0, gx=0.0, gy=0.0):
    """One stream-and-collide step."""
    fs = stream(f)
    rho, ux, uy = moments(fs)
    tau = kn_ref * rho_ref / rho if rho_ref > 0.0 else np.full_like(rho, kn_ref)
    if tau_mode == 1:
        tau = tau - 0.5 * dt
    om = dt / tau
    return fs + om[None] * (equilibrium(rho, ux, uy) - fs) + dt * force(rho, ux, uy, gx, gy)


def run(f, nsteps, **kw):
    for _ in range(nsteps):
        f = step(f, **kw)
    return f
