"""Seeded synthetic workloads shaped like the paper's channel flows.

This module is shared by the tests, the benchmark and the smoke check. It holds only
geometry and parameters (grid sizes, region maps, wall speeds, Kn, forces, initial
macroscopic fields, seeded instance lists); it contains none of the method's
arithmetic, so both the CUDA path and the CPU oracle can be driven from it without
sharing any of their code.

Units are the paper's nondimensional ones (Eq. (nondime)): lengths in l0 = H, the
channel height between the two wall nodes, velocities in sqrt(R T0). Speeds given
"in lattice units" follow the D2Q9 convention c_s^2 = 1/3 (lattice), so
u = sqrt(3) u_lat and g = 3 g_lat (ny - 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT3 = math.sqrt(3.0)


@dataclass
class Workload:
    """One lattice: everything lb_create needs, plus the initial macroscopic state."""

    name: str
    nx: int
    ny: int
    region_map: np.ndarray                  # [ny][nx] uint8, 1 = high-order set
    sets: tuple = (9, 36)                   # (low, high) populations per node
    kn_ref: float = 0.1
    rho_ref: float = 1.0
    tau_mode: int = 0
    gx: float = 0.0
    gy: float = 0.0
    rho0: float = 1.0
    walls: dict = field(default_factory=dict)
    cfl: float = 0.5
    steps: int = 1
    init: tuple | None = None               # (rho, ux, uy) arrays [ny][nx], None = rest
    iface: str = "hermite"

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def lattice_speed(u_lat: float) -> float:
    return SQRT3 * u_lat


def lattice_force(g_lat: float, ny: int) -> float:
    return 3.0 * g_lat * (ny - 1)


def band_map(nx: int, ny: int, rows_bottom: int, rows_top: int | None = None) -> np.ndarray:
    """High-order rows next to each wall, low-order core (Sec. 3.4 partitions)."""
    rows_top = rows_bottom if rows_top is None else rows_top
    m = np.zeros((ny, nx), dtype=np.uint8)
    m[:rows_bottom, :] = 1
    if rows_top > 0:
        m[ny - rows_top:, :] = 1
    return m


def couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=5000, sets=(9, 36),
            iface="hermite") -> Workload:
    """Plane Couette flow: plates at y = 0 and y = H moving at -/+ u_wall (Sec. 3.4)."""
    uw = lattice_speed(u_wall_lat)
    return Workload(
        name=f"couette_{nx}x{ny}_kn{kn:g}", nx=nx, ny=ny, region_map=band_map(nx, ny, rows),
        sets=sets, kn_ref=kn, walls={"bottom": {"kind": "diffuse", "ux": -uw},
                                     "top": {"kind": "diffuse", "ux": uw}},
        steps=steps, iface=iface)


def poiseuille(nx=1024, ny=512, rows=32, kn=0.1, g_lat=1e-6, steps=20000, sets=(9, 36),
               iface="hermite") -> Workload:
    """Force-driven channel with resting diffuse walls."""
    return Workload(
        name=f"poiseuille_{nx}x{ny}_kn{kn:g}", nx=nx, ny=ny, region_map=band_map(nx, ny, rows),
        sets=sets, kn_ref=kn, gx=lattice_force(g_lat, ny),
        walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"}}, steps=steps, iface=iface)


def oscillatory_couette(nx=4, ny=64, rows=None, kn=0.1, u_wall_lat=0.05, stokes_omega=1.0,
                        steps=2000, sets=(9, 36)) -> Workload:
    """Bottom plate oscillating as u_w sin(omega t), top plate at rest (Sec. 3.5)."""
    rows = int(round(0.15 * ny)) if rows is None else rows
    uw = lattice_speed(u_wall_lat)
    return Workload(
        name=f"osc_couette_{nx}x{ny}_kn{kn:g}", nx=nx, ny=ny, region_map=band_map(nx, ny, rows),
        sets=sets, kn_ref=kn,
        walls={"bottom": {"kind": "diffuse", "ux": uw, "omega": stokes_omega},
               "top": {"kind": "diffuse"}}, steps=steps)


def kramers(ny=201, span=40.0, layer=10.0, u_lat=0.01, nx=4, sets=(9, 36), iface="hermite",
            steps=2000) -> Workload:
    """Kramers' problem (Sec. 3.3): a diffuse plate at rest at y = 0 and the shear imposed
    by a diffuse plate moving at u_w at y = H, `span` mean free paths away (the paper's
    200), far enough that the Knudsen layer of the resting plate does not reach it. The
    high-order set covers y <= `layer` mean free paths (the paper's 10), the low-order
    set the rest. The mean free path is lambda = tau = Kn (Eq. (KN) at rho = rho_ref) in
    units of H, so Kn = 1 / span. Starts from the uniform shear u = u_w y / H."""
    kn = 1.0 / span
    rows = int(math.floor((ny - 1) * layer / span + 1e-9)) + 1
    uw = lattice_speed(u_lat)
    y = np.arange(ny) / (ny - 1)
    ux = np.broadcast_to((uw * y)[:, None], (ny, nx)).copy()
    return Workload(
        name=f"kramers_{nx}x{ny}_span{span:g}", nx=nx, ny=ny, region_map=band_map(nx, ny, rows, 0),
        sets=sets, kn_ref=kn, walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse", "ux": uw}},
        steps=steps, init=(np.ones((ny, nx)), ux, np.zeros((ny, nx))), iface=iface)


def long_channel_density(nx: int, rho_in: float, rho_out: float) -> np.ndarray:
    """Isothermal lubrication estimate: rho^2 falls linearly from inlet to outlet."""
    x = np.arange(nx) / max(nx - 1, 1)
    return np.sqrt(rho_in ** 2 - (rho_in ** 2 - rho_out ** 2) * x)


def long_channel(nx=16384, ny=128, rho_in=2.0, rho_out=1.0, kn_out=0.2, kn_threshold=0.2 / 0.15,
                 min_rows=2, steps=2000, sets=(9, 36), cfl=0.5) -> Workload:
    """Pressure-driven microchannel with Kn growing along x.

    Region map: a node is high-order when the wall Knudsen number Kn(x) H / d_wall
    exceeds kn_threshold, with Kn(x) = kn_out rho_out / rho_est(x); at the outlet this
    gives the paper's 15 % band per wall; at least min_rows rows per wall are
    high-order everywhere. The initial state is the lubrication density estimate
    with a parabolic velocity of the local pressure gradient (mean free path scaled).
    An all-high-order map of this geometry needs cfl <= (3 - sqrt 5) / 2 (about 0.38):
    at 0.5 the unsplit update of the diagonal D2Q36 populations is not positive and
    two-dimensional disturbances grow.
    """
    h = 1.0 / (ny - 1)
    rho_est = long_channel_density(nx, rho_in, rho_out)
    kn_x = kn_out * rho_out / rho_est
    j = np.arange(ny)
    d_wall = np.minimum(j, ny - 1 - j) * h
    m = (kn_x[None, :] / np.maximum(d_wall[:, None], 1e-300) > kn_threshold).astype(np.uint8)
    m[:min_rows, :] = 1
    m[ny - min_rows:, :] = 1
    # parabola of the local pressure gradient with a slip of about 1.4 mean free paths
    dpdx = np.gradient(rho_est, h)
    mu = kn_out * rho_out
    y = (j * h)[:, None]
    prof = y * (1.0 - y) + 2.0 * 1.4 * kn_x[None, :]
    ux = (-dpdx[None, :] / (2.0 * mu)) * prof
    rho = np.broadcast_to(rho_est[None, :], (ny, nx)).copy()
    uy = np.zeros((ny, nx))
    return Workload(
        name=f"long_channel_{nx}x{ny}", nx=nx, ny=ny, region_map=m, sets=sets,
        kn_ref=kn_out, rho_ref=rho_out, rho0=0.5 * (rho_in + rho_out),
        walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"},
               "left": {"kind": "pressure", "rho": rho_in},
               "right": {"kind": "pressure", "rho": rho_out}},
        steps=steps, init=(rho, ux, uy), cfl=cfl)


def batched_instances(n=512, seed=1007, nx=8, ny_range=(16, 256), kn_log_range=(-2.0, 0.0),
                      uw_range=(0.01, 0.1)) -> list[Workload]:
    """Independent Couette / Poiseuille channels of uneven height and Kn, seeded."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        kn = float(10.0 ** rng.uniform(*kn_log_range))
        kind = "couette" if rng.random() < 0.5 else "poiseuille"
        u_lat = float(rng.uniform(*uw_range))
        rows = max(2, int(round(0.15 * ny)))
        if kind == "couette":
            w = couette(nx=nx, ny=ny, rows=rows, kn=kn, u_wall_lat=u_lat, steps=5000)
        else:
            # body force that gives the same peak speed for a no-slip parabola:
            # u_max = g H^2 / (8 nu), nu = kn, H = 1
            g = 8.0 * kn * lattice_speed(u_lat)
            w = poiseuille(nx=nx, ny=ny, rows=rows, kn=kn, g_lat=g / (3.0 * (ny - 1)), steps=5000)
        w.name = f"inst{k}_{kind}_{ny}_kn{kn:.4g}"
        out.append(w)
    return out


def placement_channel(kn: float, region_map=None, nx=8, ny=64, u_lat=0.05, cfl=0.38) -> Workload:
    """Steady force-driven channel of the learned-placement study: periodic x, resting
    diffuse walls, the body force of a no-slip parabola with peak lattice speed u_lat,
    CFL 0.38 so that an all-high-order map is stable; region_map defaults to all
    high-order (the reference run)."""
    g = 8.0 * kn * lattice_speed(u_lat)
    w = poiseuille(nx=nx, ny=ny, rows=1, kn=kn, g_lat=g / (3.0 * (ny - 1)))
    w.region_map = np.ones((ny, nx), np.uint8) if region_map is None else np.asarray(region_map, np.uint8)
    w.cfl = cfl
    w.name = f"placement_{nx}x{ny}_kn{kn:g}"
    return w


def mlp_init(seed: int = 1007, nf: int = 8, nh: int = 64) -> np.ndarray:
    """Seeded starting weights of the learned-placement network (8 -> 64 -> 64 -> 1),
    packed W1 [nh][nf], b1, W2 [nh][nh], b2, W3 [nh], b3: normal with standard deviation
    sqrt(2 / fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((nh, nf)) * math.sqrt(2.0 / nf)
    w2 = rng.standard_normal((nh, nh)) * math.sqrt(2.0 / nh)
    w3 = rng.standard_normal(nh) * math.sqrt(2.0 / nh)
    return np.concatenate([w1.ravel(), np.zeros(nh), w2.ravel(), np.zeros(nh), w3, np.zeros(1)]).astype(np.float32)


def wall_stratified_sample(ny: int, nx: int, n: int, seed: int = 1007) -> np.ndarray:
    """n node indices (j * nx + i) of an ny x nx channel, the same number from every
    distance to the nearer wall (each distance holds two rows), uniformly within it,
    without replacement."""
    rng = np.random.default_rng(seed)
    dist = np.minimum(np.arange(ny), ny - 1 - np.arange(ny))
    levels = np.unique(dist)
    per = -(-n // len(levels))
    out = []
    for d in levels:
        rows = np.nonzero(dist == d)[0]
        pool = (rows[:, None] * nx + np.arange(nx)[None, :]).ravel()
        out.append(rng.choice(pool, size=min(per, pool.size), replace=False))
    idx = np.concatenate(out)
    return np.sort(rng.choice(idx, size=min(n, idx.size), replace=False))


def steady_steps(kn: float, dt: float) -> int:
    """Steps to two viscous times H^2 / nu (nu ~ Kn) of the placement channel."""
    return int(min(60000, max(4000, 2.0 / (kn * dt))))


def config1() -> Workload:
    return couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=5000)


def config2(kn=0.1, nx=1024, ny=512) -> Workload:
    return poiseuille(nx=nx, ny=ny, rows=32, kn=kn, g_lat=1e-6, steps=20000)


def config3(nx=16384, ny=128) -> Workload:
    return long_channel(nx=nx, ny=ny)
