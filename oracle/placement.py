"""FP64 oracle of the learned-placement inputs: per-node features and training labels.

TEST INFRASTRUCTURE (see oracle/__init__.py): used only by tests/, the smoke check and
the benchmark's CPU-baseline leg.

Sec. 2.2 chooses where the high-order set runs with a switching criterion that it leaves
open (local Knudsen numbers, stress / heat-flux based breakdown parameters from the
literature). The learned map reads these quantities per node, computed here from the
oracle's moments and populations in plain numpy:

  features (8 per node, Sec. 2.2 candidates):
    0..2  Pi^neq_xx / rho, Pi^neq_xy / rho, Pi^neq_yy / rho
          (Pi^neq = sum_a (f_a - f_a^eq) xi_a xi_a, the non-equilibrium stress)
    3..4  q_x / rho, q_y / rho   (q = 1/2 sum_a f_a |xi_a - u|^2 (xi_a - u))
    5     distance to the nearest diffuse wall, j h or (ny - 1 - j) h (1 without walls)
    6     local Kn = kn_ref rho_ref / rho (the Eq. (KN) density scaling; kn_ref when
          rho_ref = 0)
    7     Kn |grad rho| / rho, grad by central differences (one-sided at a non-periodic
          edge, wrapped at a periodic one)

  label source: the part of a node's populations that a second-order Hermite expansion
    cannot hold, per unit mass, e3 = ||f - P2 f|| / rho with ||g||^2 = sum_a g_a^2 / w_a
    and P2 the second-order Hermite expansion (Eq. (approxf), N = 2, coefficients by
    Eq. (an)) rebuilt on the node's own set. P2 is the orthogonal projection in that
    norm and f^eq lies in its range, so ||f - f^eq||^2 = ||f - P2 f||^2 + ||P2 f - f^eq||^2.
"""
from __future__ import annotations

import numpy as np

from . import project as _project
from . import velocity_set

FEATURE_NAMES = ("neq_xx/rho", "neq_xy/rho", "neq_yy/rho", "qx/rho", "qy/rho", "d_wall", "kn", "kn_grad_rho")


def local_kn(rho, kn_ref, rho_ref):
    return kn_ref * rho_ref / rho if rho_ref > 0.0 else np.full_like(rho, kn_ref)


def _gradient(a, h, periodic, axis):
    """Central differences along `axis`; one-sided at the ends unless periodic."""
    if periodic:
        return (np.roll(a, -1, axis) - np.roll(a, 1, axis)) / (2.0 * h)
    g = np.empty_like(a)
    n = a.shape[axis]
    sl = lambda i: tuple(slice(None) if k != axis else i for k in range(a.ndim))   # noqa: E731
    g[sl(slice(1, n - 1))] = (a[sl(slice(2, n))] - a[sl(slice(0, n - 2))]) / (2.0 * h)
    g[sl(0)] = (a[sl(1)] - a[sl(0)]) / h
    g[sl(n - 1)] = (a[sl(n - 1)] - a[sl(n - 2)]) / h
    return g


def features(mom, h, kn_ref, rho_ref, periodic_x, periodic_y, wall_bottom, wall_top):
    """mom: the oracle's moment dict (fields [ny][nx]) -> features [8][ny][nx]."""
    rho = mom["rho"]
    ny, nx = rho.shape
    kn = local_kn(rho, kn_ref, rho_ref)
    gx = _gradient(rho, h, periodic_x, 1)
    gy = _gradient(rho, h, periodic_y, 0)
    j = np.arange(ny, dtype=np.float64)[:, None]
    if wall_bottom or wall_top:
        d0 = j if wall_bottom else np.full_like(j, np.inf)
        d1 = (ny - 1 - j) if wall_top else np.full_like(j, np.inf)
        dw = np.broadcast_to(np.minimum(d0, d1) * h, (ny, nx))
    else:
        dw = np.ones((ny, nx))
    out = np.empty((8, ny, nx))
    for k, name in enumerate(("neq_xx", "neq_xy", "neq_yy", "qx", "qy")):
        out[k] = mom[name] / rho
    out[5] = dw
    out[6] = kn
    out[7] = kn * np.sqrt(gx * gx + gy * gy) / rho
    return out


def hermite_residual_node(f, n1d):
    """e3 for one node's populations f [Q] of the n1d-point product set."""
    w = velocity_set(n1d)[2]
    p2 = _project(n1d, f, n1d)
    return float(np.sqrt(((f - p2) ** 2 / w).sum()) / f.sum())


def hermite_residual(pops, region_map, n1d):
    """pops: (f_low [Q0][ny][nx], f_high [Q1][ny][nx]); region_map [ny][nx] picks the
    node's own set -> e3 [ny][nx]. Pure-Python loop over nodes: small lattices only."""
    ny, nx = region_map.shape
    out = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            s = int(region_map[j, i])
            out[j, i] = hermite_residual_node(pops[s][:, j, i], n1d[s])
    return out
