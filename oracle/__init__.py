"""FP64 CPU oracle of the multiscale lattice Boltzmann step (Meng, Zhang & Shan).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` import this package. The product path (the CUDA library and its
Python binding) never imports, links or runs anything here, and shares no code with it.

The arithmetic lives in ``lb_oracle.c`` (plain loops, double precision, in the order the
paper states the method); this module only compiles it with gcc and marshals arguments.
``mlp.py`` holds the numpy FP64 oracle of the learned interface-placement network;
``exact_stream.py`` the D2Q9 stream-and-collide reduction (Courant number one).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_SO = os.path.join(_HERE, "liblboracle.so")
_lock = threading.Lock()
_lib = None

SIDES = ("bottom", "top", "left", "right")
# storage models of the oracle (set_storage): the formats of the GPU path's lb_opts.store
# and lb_opts.rounding
STORAGE_MODES = {"exact": 0, "f32": 1, "f32_dev": 2, "f16_dev": 3, "bf16_dev": 4, "f16_dev_sr": 5, "bf16_dev_sr": 6}


def store_round(mode: str, d: float, bits: int = 0, set_value: bool = False) -> float:
    """One deviation through a storage model's rounding (bits: the 32 random bits of a
    stochastic mode)."""
    return lib().or_store_round(STORAGE_MODES[mode], float(d), int(bits) & 0xffffffff, 1 if set_value else 0)
WALL_KIND = {"periodic": 0, "diffuse": 1, "pressure": 2}


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into liblboracle.so (gcc, OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _SO + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class OrCfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("n1d_lo", ctypes.c_int32), ("n1d_hi", ctypes.c_int32),
        ("h", ctypes.c_double), ("dt", ctypes.c_double),
        ("kn_ref", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("tau_mode", ctypes.c_int32),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("iface", ctypes.c_int32), ("limiter", ctypes.c_int32),
        ("wall_kind", ctypes.c_int32 * 4),
        ("wall_ux", ctypes.c_double * 4), ("wall_uy", ctypes.c_double * 4),
        ("wall_rho", ctypes.c_double * 4), ("wall_omega", ctypes.c_double * 4),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_gauss_hermite.argtypes = [ctypes.c_int, dp, dp]
            L.or_velocity_set.argtypes = [ctypes.c_int, dp, dp, dp]
            L.or_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.or_force.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5 + [dp]
            L.or_project.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
            L.or_create.argtypes = [ctypes.POINTER(OrCfg), ctypes.POINTER(ctypes.c_uint8)]
            L.or_create.restype = ctypes.c_void_p
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_init_equilibrium.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.or_set_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.or_get_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.or_moments.argtypes = [ctypes.c_void_p, dp]
            L.or_set_storage.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, dp]
            L.or_store_round.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_int]
            L.or_store_round.restype = ctypes.c_double
            L.or_time.argtypes = [ctypes.c_void_p]
            L.or_time.restype = ctypes.c_double
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gauss_hermite(n: int):
    """1-D rule by Eq. (weight): (abscissae ascending, weights)."""
    x = np.zeros(8)
    w = np.zeros(8)
    k = lib().or_gauss_hermite(n, _dp(x), _dp(w))
    return x[:k].copy(), w[:k].copy()


def velocity_set(n1d: int):
    """Product set of the n1d-point rule: (cx, cy, w), alpha = iy * n1d + ix."""
    cx, cy, w = np.zeros(36), np.zeros(36), np.zeros(36)
    q = lib().or_velocity_set(n1d, _dp(cx), _dp(cy), _dp(w))
    if q < 0:
        raise ValueError(f"unsupported 1-D order {n1d}")
    return cx[:q].copy(), cy[:q].copy(), w[:q].copy()


def feq(n1d: int, rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(36)
    q = lib().or_feq(n1d, rho, ux, uy, _dp(out))
    return out[:q].copy()


def force(n1d: int, rho: float, ux: float, uy: float, gx: float, gy: float) -> np.ndarray:
    out = np.zeros(36)
    q = lib().or_force(n1d, rho, ux, uy, gx, gy, _dp(out))
    return out[:q].copy()


def project(n1d_from: int, f_from: np.ndarray, n1d_to: int) -> np.ndarray:
    f_from = np.ascontiguousarray(f_from, dtype=np.float64)
    out = np.zeros(36)
    q = lib().or_project(n1d_from, _dp(f_from), n1d_to, _dp(out))
    return out[:q].copy()


class Oracle:
    """One lattice: nx x ny nodes, per-node set map (0 low-order, 1 high-order)."""

    def __init__(self, nx, ny, region_map, n1d_lo=3, n1d_hi=6, h=None, dt=None, cfl=0.5,
                 kn_ref=0.1, rho_ref=1.0, tau_mode=0, gx=0.0, gy=0.0, iface="hermite",
                 limiter=0, walls=None):
        walls = walls or {}
        kinds = [WALL_KIND[walls.get(s, {}).get("kind", "periodic" if s in ("left", "right") else "diffuse")]
                 for s in SIDES]
        if h is None:
            h = 1.0 / (ny - 1) if kinds[0] != 0 else 1.0 / ny
        if dt is None:
            xmax = max(abs(velocity_set(n1d_lo)[0]).max(), abs(velocity_set(n1d_hi)[0]).max())
            dt = cfl * h / xmax
        self.nx, self.ny, self.h, self.dt = nx, ny, h, dt
        self.n1d = (n1d_lo, n1d_hi)
        c = OrCfg()
        c.nx, c.ny, c.n1d_lo, c.n1d_hi = nx, ny, n1d_lo, n1d_hi
        c.h, c.dt, c.kn_ref, c.rho_ref, c.tau_mode = h, dt, kn_ref, rho_ref, tau_mode
        c.gx, c.gy = gx, gy
        c.iface = {"paper": 0, "hermite": 1}[iface]
        c.limiter = limiter
        for k, s in enumerate(SIDES):
            wd = walls.get(s, {})
            c.wall_kind[k] = kinds[k]
            c.wall_ux[k] = wd.get("ux", 0.0)
            c.wall_uy[k] = wd.get("uy", 0.0)
            c.wall_rho[k] = wd.get("rho", 1.0)
            c.wall_omega[k] = wd.get("omega", 0.0)
        self.cfg = c
        self.map = np.ascontiguousarray(np.asarray(region_map, dtype=np.uint8).reshape(ny, nx))
        self._p = lib().or_create(ctypes.byref(c), self.map.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        if not self._p:
            raise ValueError("oracle: bad configuration")
        self.q = (len(velocity_set(n1d_lo)[0]), len(velocity_set(n1d_hi)[0]))

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().or_destroy(p)
            self._p = None

    def init_equilibrium(self, rho, ux, uy):
        shape = (self.ny, self.nx)
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), shape))
        u = np.ascontiguousarray(np.broadcast_to(np.asarray(ux, dtype=np.float64), shape))
        v = np.ascontiguousarray(np.broadcast_to(np.asarray(uy, dtype=np.float64), shape))
        lib().or_init_equilibrium(self._p, _dp(r), _dp(u), _dp(v))

    def set_populations(self, s: int, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.q[s], self.ny, self.nx)
        lib().or_set_populations(self._p, s, _dp(f))

    def populations(self, s: int) -> np.ndarray:
        out = np.zeros((self.q[s], self.ny, self.nx))
        lib().or_get_populations(self._p, s, _dp(out))
        return out

    def set_storage(self, mode: str, rho0: float = 1.0, rho0_col=None):
        """Round the stored populations of every evolved node after each update the way
        a storage format holds them (STORAGE_MODES); "exact" turns it off."""
        col = None
        if rho0_col is not None:
            self._rho_r = np.ascontiguousarray(np.asarray(rho0_col, dtype=np.float64).reshape(self.nx))
            col = _dp(self._rho_r)
        if lib().or_set_storage(self._p, STORAGE_MODES[mode], float(rho0), col) != 0:
            raise ValueError(mode)

    def step(self, n: int = 1):
        lib().or_step(self._p, int(n))

    def moments(self) -> dict:
        out = np.zeros((10, self.ny, self.nx))
        lib().or_moments(self._p, _dp(out))
        names = ("rho", "ux", "uy", "pxy", "neq_xx", "neq_xy", "neq_yy", "qx", "qy", "set")
        return {k: out[m] for m, k in enumerate(names)}

    @property
    def time(self) -> float:
        return lib().or_time(self._p)
