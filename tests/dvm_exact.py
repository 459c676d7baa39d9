"""Exact steady solutions of the linearised discrete-velocity BGK model (continuous in
space) for plane Couette and force-driven Poiseuille flow between diffuse walls.

Used as independent pins of the oracle: for a shear flow the perturbation of a
Gauss-Hermite product set is xi_x g(xi_y, y), and g obeys, for each 1-D abscissa r_j,
    r_j g_j' = -(g_j - <g>) / tau + G,      <g> = sum_j w_j g_j,
with g_j = u_wall on the gas-bound abscissae at each wall (linearised diffuse
reflection). Its solution is a polynomial bulk part plus the half-range modes
exp(-lambda y / tau) with sum_j w_j / (1 - lambda r_j) = 1. Everything here is
numpy / scipy linear algebra, written from that derivation, not from the oracle.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.hermite_e import hermegauss
from scipy.optimize import brentq


def rule(n):
    r, w = hermegauss(n)
    return r, w / np.sqrt(2.0 * np.pi)


def decay_rates(n):
    """Positive roots lambda of sum_j w_j / (1 - lambda r_j) = 1."""
    r, w = rule(n)
    f = lambda lam: float(np.sum(w / (1.0 - lam * r)) - 1.0)
    poles = sorted(1.0 / x for x in r if x > 1e-12)
    edges = [1e-9] + poles + [1e9]
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        xs = np.linspace(a * (1 + 1e-9), b * (1 - 1e-9), 100001)
        v = np.sum(w[None, :] / (1.0 - xs[:, None] * r[None, :]), axis=1) - 1.0
        # a sign change between finite samples (not across a pole)
        ks = np.nonzero((np.sign(v[:-1]) != np.sign(v[1:])) & (np.abs(v[:-1]) < 1e6) & (np.abs(v[1:]) < 1e6))[0]
        out.extend(brentq(f, xs[k], xs[k + 1]) for k in ks)
    return [x for x in out if x > 1e-6]


def channel(n, tau, H=1.0, u_bottom=0.0, u_top=0.0, G=0.0):
    """Velocity profile u(y) between diffuse walls at y = 0 and y = H (callable)."""
    r, w = rule(n)
    lams = decay_rates(n)
    M = len(lams)
    # bulk: g_j = a0 + a1 y + a2 y^2 + r_j (b0 + b1 y) + c r_j^2, with
    # a2 = -G/(2 tau), b1 = G, c = -G tau, b0 = -tau a1
    a2, b1, c = -G / (2 * tau), G, -G * tau
    rows, rhs = [], []
    for rj in r:
        if rj > 1e-12:      # leaving the bottom wall
            y = 0.0
            rows.append([1.0, y - tau * rj] + [1 / (1 - l * rj) for l in lams]
                        + [np.exp(-l * H / tau) / (1 + l * rj) for l in lams])
            rhs.append(u_bottom - (a2 * y * y + rj * b1 * y + c * rj * rj))
        if rj < -1e-12:     # leaving the top wall
            y = H
            rows.append([1.0, y - tau * rj] + [np.exp(-l * H / tau) / (1 - l * rj) for l in lams]
                        + [1 / (1 + l * rj) for l in lams])
            rhs.append(u_top - (a2 * y * y + rj * b1 * y + c * rj * rj))
    sol = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    a0, a1 = sol[0], sol[1]
    cm, dm = sol[2:2 + M], sol[2 + M:]

    def u(y):
        y = np.asarray(y, dtype=float)
        out = a0 + a1 * y + a2 * y * y + c
        for k, l in enumerate(lams):
            out = out + cm[k] * np.exp(-l * y / tau) + dm[k] * np.exp(-l * (H - y) / tau)
        return out

    return u


def half_space(n):
    """Kramers' half-space problem (Sec. 3.3) for the linearised discrete-velocity model:
    a diffuse plate at rest at y = 0 and a unit shear rate far from it. With lengths in
    units of tau the solution is
        g_j(y) = y + zeta - r_j + sum_m c_m exp(-lambda_m y) / (1 - lambda_m r_j),
        u(y) = y + zeta + sum_m c_m exp(-lambda_m y),
    the Chapman-Enskog bulk plus the decaying half-range modes; zeta (the slip
    coefficient) and c_m follow from g_j(0) = 0 on every gas-bound abscissa r_j > 0
    (as many equations as unknowns). Returns (zeta, lambdas, c, u) with u callable."""
    r, w = rule(n)
    lams = decay_rates(n)
    pos = r[r > 1e-12]
    A = np.zeros((len(pos), 1 + len(lams)))
    A[:, 0] = 1.0
    for m, l in enumerate(lams):
        A[:, 1 + m] = 1.0 / (1.0 - l * pos)
    sol = np.linalg.solve(A, pos)
    zeta, c = float(sol[0]), sol[1:]

    def u(y):
        y = np.asarray(y, dtype=float)
        out = y + zeta
        for m, l in enumerate(lams):
            out = out + c[m] * np.exp(-l * y)
        return out

    return zeta, np.array(lams), c, u
