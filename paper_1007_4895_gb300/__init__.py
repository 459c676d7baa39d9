"""Python binding of liblbgb.so, the GB300 multiscale lattice Boltzmann library.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. The functions below carry the C names of ``include/lb.h``; ``Lattice`` wraps
one context. Device memory can come from PyTorch's caching allocator
(``torch_allocator=True``) and work runs on PyTorch's current CUDA stream.

There is no CPU fallback: importing this package raises if the CUDA library has not
been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbgb.so")

LB_OK, LB_ERR_INVALID, LB_ERR_NOMEM, LB_ERR_CUDA, LB_ERR_DIVERGED, LB_ERR_TIMEOUT = range(6)
LB_ROUND_NEAREST, LB_ROUND_STOCHASTIC = 0, 1
ROUNDING = {"nearest": LB_ROUND_NEAREST, "stochastic": LB_ROUND_STOCHASTIC}
LB_SCHEME_TVD, LB_SCHEME_STREAM = 0, 1
SCHEMES = {"tvd": LB_SCHEME_TVD, "stream": LB_SCHEME_STREAM}
LB_STORE_F64, LB_STORE_F32, LB_STORE_F32_DEV, LB_STORE_F16_DEV, LB_STORE_BF16_DEV = range(5)
LB_IFACE_PAPER, LB_IFACE_HERMITE = 0, 1
LB_WALL_PERIODIC, LB_WALL_DIFFUSE, LB_WALL_PRESSURE = 0, 1, 2
MOMENT_NAMES = ("rho", "ux", "uy", "pxy", "neq_xx", "neq_xy", "neq_yy", "qx", "qy")
LB_M_ALL = (1 << 9) - 1
STORES = {"f64": LB_STORE_F64, "f32": LB_STORE_F32, "f32_dev": LB_STORE_F32_DEV,
          "f16_dev": LB_STORE_F16_DEV, "bf16_dev": LB_STORE_BF16_DEV}
STORE_DTYPE = {LB_STORE_F64: "f64", LB_STORE_F32: "f32", LB_STORE_F32_DEV: "f32",
               LB_STORE_F16_DEV: "f16", LB_STORE_BF16_DEV: "bf16"}
EXPORTS = ("lb_create", "lb_init_equilibrium", "lb_step", "lb_moments", "lb_reductions", "lb_effective_map",
           "lb_set_region_map", "lb_get_populations", "lb_set_populations", "lb_state_bytes", "lb_state_load",
           "lb_state_store", "lb_save", "lb_load", "lb_info", "lb_sync", "lb_destroy", "lb_last_error",
           "lb_reduce_fields_noalloc", "lb_features", "lb_hermite_residual", "lb_mlp_create", "lb_mlp_grad",
           "lb_mlp_adam_step", "lb_mlp_train", "lb_mlp_get_params", "lb_mlp_infer", "lb_mlp_destroy", "lb_set_mlp",
           "lb_learned_map_now", "lb_map_stats", "lb_batch_create", "lb_batch_step", "lb_batch_step_each",
           "lb_batch_graph", "lb_batch_instance", "lb_batch_info", "lb_batch_sync", "lb_batch_destroy",
           "lb_selftest_bounded_wait")
LB_NOALLOC_MAX_NODES = 524288


class LBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lb status {code}: {msg}")
        self.code = code


class lb_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("h", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double)]


class lb_wall(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("ux", ctypes.c_double), ("uy", ctypes.c_double),
                ("rho", ctypes.c_double), ("omega", ctypes.c_double)]


class lb_kn(ctypes.Structure):
    _fields_ = [("kn_ref", ctypes.c_double), ("rho_ref", ctypes.c_double), ("tau_mode", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lb_opts(ctypes.Structure):
    _fields_ = [("store", ctypes.c_int32), ("iface", ctypes.c_int32), ("rho0", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("reduce_every", ctypes.c_int32),
                ("variant", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("rounding", ctypes.c_int32),
                ("rho0_col", ctypes.POINTER(ctypes.c_double)), ("scheme", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.lb_create.argtypes = [ctypes.POINTER(lb_grid), u8p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(lb_kn),
                            ctypes.POINTER(lb_wall), ctypes.POINTER(lb_opts), ctypes.POINTER(P)]
    L.lb_init_equilibrium.argtypes = [P, dp, dp, dp]
    L.lb_step.argtypes = [P, ctypes.c_int64]
    L.lb_moments.argtypes = [P, ctypes.c_uint32, P, ctypes.c_int32, ctypes.c_int32]
    L.lb_reductions.argtypes = [P, dp]
    L.lb_effective_map.argtypes = [P, u8p]
    L.lb_set_region_map.argtypes = [P, u8p]
    L.lb_get_populations.argtypes = [P, ctypes.c_int32, dp]
    L.lb_set_populations.argtypes = [P, ctypes.c_int32, dp]
    L.lb_state_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.lb_state_load.argtypes = [P, P, ctypes.c_size_t]
    L.lb_state_store.argtypes = [P, P, ctypes.c_size_t]
    L.lb_save.argtypes = [P, ctypes.c_char_p]
    L.lb_load.argtypes = [P, ctypes.c_char_p]
    L.lb_info.argtypes = [P, dp, dp, ctypes.POINTER(ctypes.c_int64), dp, ctypes.POINTER(ctypes.c_int32)]
    L.lb_sync.argtypes = [P]
    L.lb_destroy.argtypes = [P]
    L.lb_destroy.restype = None
    L.lb_last_error.restype = ctypes.c_char_p
    L.lb_reduce_fields_noalloc.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, P, dp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.lb_features.argtypes = [P, P]
    L.lb_hermite_residual.argtypes = [P, P]
    L.lb_mlp_create.argtypes = [fp, fp, ctypes.POINTER(lb_opts), ctypes.POINTER(P)]
    L.lb_mlp_grad.argtypes = [P, P, P, ctypes.c_int64, fp, dp]
    L.lb_mlp_adam_step.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_float]
    L.lb_mlp_train.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                               ctypes.c_uint64, dp]
    L.lb_mlp_get_params.argtypes = [P, fp]
    L.lb_mlp_infer.argtypes = [P, P, ctypes.c_int64, P]
    L.lb_mlp_destroy.argtypes = [P]
    L.lb_mlp_destroy.restype = None
    L.lb_set_mlp.argtypes = [P, P, ctypes.c_int32, ctypes.c_float, ctypes.c_float]
    L.lb_learned_map_now.argtypes = [P]
    L.lb_map_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), dp]
    L.lb_batch_create.argtypes = [ctypes.c_int32, ctypes.POINTER(lb_grid), ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(lb_kn), ctypes.POINTER(lb_wall), ctypes.POINTER(lb_opts), ctypes.POINTER(P)]
    L.lb_batch_step.argtypes = [P, ctypes.c_int64]
    L.lb_batch_step_each.argtypes = [P, ctypes.c_int64]
    L.lb_batch_graph.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    L.lb_batch_instance.argtypes = [P, ctypes.c_int32]
    L.lb_batch_instance.restype = P
    L.lb_batch_info.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.lb_batch_sync.argtypes = [P]
    L.lb_batch_destroy.argtypes = [P]
    L.lb_batch_destroy.restype = None
    L.lb_selftest_bounded_wait.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]
    return L


_lib = _load()


def lib():
    return _lib


def _check(code):
    if code != LB_OK:
        raise LBError(code, _lib.lb_last_error().decode())
    return code


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ C-named calls

def lb_create(grid, region_map, sets, kn, walls, opts):
    ctx = ctypes.c_void_p()
    m = np.ascontiguousarray(region_map, dtype=np.uint8)
    s = (ctypes.c_int32 * 2)(*sets)
    w = (lb_wall * 4)(*walls)
    _check(_lib.lb_create(ctypes.byref(grid), m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), s,
                          ctypes.byref(kn), w, ctypes.byref(opts), ctypes.byref(ctx)))
    return ctx


def lb_init_equilibrium(ctx, rho=None, ux=None, uy=None):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy)]
    ptrs = [None if a is None else _dp(a) for a in arrs]
    _check(_lib.lb_init_equilibrium(ctx, *ptrs))


def lb_step(ctx, n):
    _check(_lib.lb_step(ctx, int(n)))


def lb_moments(ctx, mask, dst_ptr, dst_is_device, dst_f64):
    _check(_lib.lb_moments(ctx, mask, ctypes.c_void_p(dst_ptr), int(dst_is_device), int(dst_f64)))


def lb_reductions(ctx):
    out = np.zeros(4)
    _check(_lib.lb_reductions(ctx, _dp(out)))
    return out


def lb_effective_map(ctx, nx, ny):
    out = np.zeros((ny, nx), dtype=np.uint8)
    _check(_lib.lb_effective_map(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
    return out


def lb_set_region_map(ctx, region_map):
    m = np.ascontiguousarray(region_map, dtype=np.uint8)
    _check(_lib.lb_set_region_map(ctx, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))


def lb_get_populations(ctx, s, q, nx, ny):
    out = np.zeros((q, ny, nx))
    _check(_lib.lb_get_populations(ctx, int(s), _dp(out)))
    return out


def lb_set_populations(ctx, s, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(_lib.lb_set_populations(ctx, int(s), _dp(f)))


def lb_state_bytes(ctx):
    n = ctypes.c_size_t()
    _check(_lib.lb_state_bytes(ctx, ctypes.byref(n)))
    return n.value


def lb_selftest_bounded_wait(stream=None, polls=100000):
    """True when a wait on a barrier that nothing completes gave up and reported it."""
    out = ctypes.c_int32()
    _check(_lib.lb_selftest_bounded_wait(ctypes.c_void_p(stream or 0), ctypes.c_uint32(polls), ctypes.byref(out)))
    return bool(out.value)


def lb_state_load(ctx, ptr, nbytes):
    _check(_lib.lb_state_load(ctx, ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes)))


def lb_state_store(ctx, ptr, nbytes):
    _check(_lib.lb_state_store(ctx, ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes)))


def lb_save(ctx, path):
    _check(_lib.lb_save(ctx, os.fsencode(path)))


def lb_load(ctx, path):
    _check(_lib.lb_load(ctx, os.fsencode(path)))


def lb_info(ctx):
    dt, h, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = ctypes.c_int64()
    var = ctypes.c_int32()
    _check(_lib.lb_info(ctx, ctypes.byref(dt), ctypes.byref(h), ctypes.byref(st), ctypes.byref(t), ctypes.byref(var)))
    return {"dt": dt.value, "h": h.value, "step": st.value, "time": t.value, "variant": var.value}


def lb_sync(ctx):
    return _check(_lib.lb_sync(ctx))


def lb_destroy(ctx):
    _lib.lb_destroy(ctx)


def lb_last_error():
    return _lib.lb_last_error().decode()


def lb_reduce_fields_noalloc(rho_ptr, ux_ptr, uy_ptr, n, restart=False, stream=None):
    """Reduction over caller-owned device double fields without any device allocation
    (see include/lb.h). Returns [mass, residual, non-finite count, n]."""
    out = np.zeros(4)
    _check(_lib.lb_reduce_fields_noalloc(ctypes.c_void_p(rho_ptr), ctypes.c_void_p(ux_ptr), ctypes.c_void_p(uy_ptr),
                                         int(n), 1 if restart else 0, ctypes.c_void_p(stream or 0), _dp(out)))
    return out


# ------------------------------------------------------------ learned map

NPARAM = 4801


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class MLP:
    """The learned-placement network (include/lb.h). Arrays passed to the methods are
    CUDA torch tensors (float32); x is [8][n], y is [n]."""

    def __init__(self, params, norm, stream=None, torch_allocator=True):
        import torch
        stream = stream or torch.cuda.current_stream()
        self._alloc = _TorchAllocator(stream) if torch_allocator else None
        opts = lb_opts()
        opts.stream = getattr(stream, "cuda_stream", stream)
        if self._alloc:
            opts.alloc, opts.free = self._alloc.alloc, self._alloc.free
        self._opts = opts
        p = np.ascontiguousarray(params, dtype=np.float32)
        nm = np.ascontiguousarray(norm, dtype=np.float32)
        assert p.size == NPARAM and nm.size == 16
        self.ptr = ctypes.c_void_p()
        _check(_lib.lb_mlp_create(_fp(p), _fp(nm), ctypes.byref(opts), ctypes.byref(self.ptr)))

    def close(self):
        if getattr(self, "ptr", None):
            _lib.lb_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def grad(self, x, y):
        g = np.zeros(NPARAM, dtype=np.float32)
        loss = ctypes.c_double()
        _check(_lib.lb_mlp_grad(self.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), y.numel(),
                                _fp(g), ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, x, y, lr=1e-3):
        _check(_lib.lb_mlp_adam_step(self.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     y.numel(), lr))

    def train(self, x, y, epochs=20, batch=256, lr=1e-3, seed=1007):
        loss = ctypes.c_double()
        _check(_lib.lb_mlp_train(self.ptr, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), y.numel(),
                                 epochs, batch, lr, seed, ctypes.byref(loss)))
        return loss.value

    def params(self):
        p = np.zeros(NPARAM, dtype=np.float32)
        _check(_lib.lb_mlp_get_params(self.ptr, _fp(p)))
        return p

    def infer(self, x, out):
        _check(_lib.lb_mlp_infer(self.ptr, ctypes.c_void_p(x.data_ptr()), out.numel(), ctypes.c_void_p(out.data_ptr())))


# ----------------------------------------------------------------- Lattice

_SIDES = ("bottom", "top", "left", "right")
_KINDS = {"periodic": LB_WALL_PERIODIC, "diffuse": LB_WALL_DIFFUSE, "pressure": LB_WALL_PRESSURE}


def _walls(spec):
    spec = spec or {}
    out = []
    for s in _SIDES:
        d = spec.get(s, {})
        kind = d.get("kind", "periodic" if s in ("left", "right") else "diffuse")
        out.append(lb_wall(_KINDS[kind], d.get("ux", 0.0), d.get("uy", 0.0), d.get("rho", 1.0), d.get("omega", 0.0)))
    return out


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, stream):
        import torch
        self._torch = torch
        self._stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=self._stream)
        except Exception:   # out of memory: the library reports LB_ERR_NOMEM
            return None

    def _free(self, ptr, user):
        self._torch.cuda.caching_allocator_delete(ptr)


class Lattice:
    """One lattice context (see include/lb.h for the meaning of every field)."""

    def __init__(self, nx, ny, region_map, sets=(9, 36), kn_ref=0.1, rho_ref=1.0, tau_mode=0, walls=None,
                 store="f32", iface="hermite", rho0=1.0, gx=0.0, gy=0.0, cfl=0.5, dt=0.0, h=0.0,
                 reduce_every=0, stream=None, torch_allocator=True, variant=-1, rounding="nearest",
                 rho0_col=None, scheme="tvd"):
        self.nx, self.ny = int(nx), int(ny)
        self.sets = tuple(int(s) for s in sets)
        self.store = STORES[store] if isinstance(store, str) else int(store)
        self._alloc = None
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        self._stream_obj = stream
        sp = getattr(stream, "cuda_stream", stream)
        opts = lb_opts()
        opts.store = self.store
        opts.iface = LB_IFACE_HERMITE if iface == "hermite" else LB_IFACE_PAPER
        opts.rho0, opts.gx, opts.gy = rho0, gx, gy
        opts.reduce_every = int(reduce_every)
        opts.variant = int(variant)
        opts.rounding = ROUNDING[rounding] if isinstance(rounding, str) else int(rounding)
        opts.stream = sp
        opts.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        if rho0_col is not None:   # per-column reference density (deviation formats)
            self._rho0_col = np.ascontiguousarray(np.asarray(rho0_col, dtype=np.float64).reshape(self.nx))
            opts.rho0_col = self._rho0_col.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if torch_allocator:
            self._alloc = _TorchAllocator(stream)
            opts.alloc, opts.free = self._alloc.alloc, self._alloc.free
        self._opts = opts
        grid = lb_grid(self.nx, self.ny, h, cfl, dt)
        kn = lb_kn(kn_ref, rho_ref, tau_mode)
        self.ctx = lb_create(grid, np.asarray(region_map, dtype=np.uint8).reshape(self.ny, self.nx), self.sets, kn,
                             _walls(walls), opts)
        info = lb_info(self.ctx)
        self.dt, self.h = info["dt"], info["h"]

    @classmethod
    def from_workload(cls, w, store="f32", **kw):
        args = dict(sets=w.sets, kn_ref=w.kn_ref, rho_ref=w.rho_ref, tau_mode=w.tau_mode, walls=w.walls,
                    store=store, iface=w.iface, rho0=w.rho0, gx=w.gx, gy=w.gy, cfl=w.cfl)
        args.update(kw)
        lat = cls(w.nx, w.ny, w.region_map, **args)
        if w.init is not None:
            lat.init_equilibrium(*w.init)
        return lat

    def close(self):
        if getattr(self, "ctx", None):
            if getattr(self, "_owned", True):
                lb_destroy(self.ctx)
            self.ctx = None

    @classmethod
    def _view(cls, ctx, nx, ny, sets, store, owner):
        """A lattice owned by something else (a batch): used like any lattice, never
        destroyed through this object."""
        lat = cls.__new__(cls)
        lat.nx, lat.ny, lat.sets, lat.store = int(nx), int(ny), tuple(sets), store
        lat.ctx, lat._owned, lat._owner, lat._alloc = ctx, False, owner, None
        info = lb_info(ctx)
        lat.dt, lat.h = info["dt"], info["h"]
        return lat

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self, rho=None, ux=None, uy=None):
        shape = (self.ny, self.nx)
        bc = lambda a: None if a is None else np.broadcast_to(np.asarray(a, dtype=np.float64), shape)
        lb_init_equilibrium(self.ctx, bc(rho), bc(ux), bc(uy))

    def step(self, n=1):
        lb_step(self.ctx, n)

    def moments(self, mask=LB_M_ALL, f64=True):
        nf = bin(mask).count("1")
        out = np.zeros((nf, self.ny, self.nx), dtype=np.float64 if f64 else np.float32)
        lb_moments(self.ctx, mask, out.ctypes.data, 0, 1 if f64 else 0)
        names = [n for k, n in enumerate(MOMENT_NAMES) if mask & (1 << k)]
        return dict(zip(names, out))

    def moments_into(self, tensor, mask=LB_M_ALL):
        """Asynchronous write of the moment fields into a CUDA tensor [k][ny][nx]."""
        import torch
        assert tensor.is_cuda and tensor.is_contiguous() and tensor.dtype in (torch.float32, torch.float64)
        lb_moments(self.ctx, mask, tensor.data_ptr(), 1, 1 if tensor.dtype == torch.float64 else 0)

    def reductions(self):
        r = lb_reductions(self.ctx)
        return {"mass": r[0], "residual": r[1], "nonfinite": r[2], "step": r[3]}

    def effective_map(self):
        return lb_effective_map(self.ctx, self.nx, self.ny)

    def set_region_map(self, m):
        lb_set_region_map(self.ctx, np.asarray(m, dtype=np.uint8).reshape(self.ny, self.nx))

    def populations(self, s):
        return lb_get_populations(self.ctx, s, self.sets[s], self.nx, self.ny)

    def set_populations(self, s, f):
        lb_set_populations(self.ctx, s, f)

    def state_bytes(self):
        return lb_state_bytes(self.ctx)

    def save(self, path):
        lb_save(self.ctx, path)

    def load(self, path):
        lb_load(self.ctx, path)

    def info(self):
        return lb_info(self.ctx)

    def features_into(self, tensor):
        """Asynchronous: learned-placement features into a CUDA float32 tensor [8][ny][nx]."""
        _check(_lib.lb_features(self.ctx, ctypes.c_void_p(tensor.data_ptr())))

    def hermite_residual_into(self, tensor):
        """Asynchronous: ||f - P2 f|| / rho per node into a CUDA float32 tensor [ny][nx]."""
        _check(_lib.lb_hermite_residual(self.ctx, ctypes.c_void_p(tensor.data_ptr())))

    def set_mlp(self, mlp, every=100, p_on=0.5, p_off=0.3):
        self._mlp = mlp
        _check(_lib.lb_set_mlp(self.ctx, mlp.ptr if mlp else None, every, p_on, p_off))

    def learned_map_now(self):
        _check(_lib.lb_learned_map_now(self.ctx))

    def map_stats(self):
        u, f, h = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(_lib.lb_map_stats(self.ctx, ctypes.byref(u), ctypes.byref(f), ctypes.byref(h)))
        return {"updates": u.value, "fallbacks": f.value, "high_fraction": h.value}

    def sync(self):
        return lb_sync(self.ctx)


# ----------------------------------------------------------------- Batch

class Batch:
    """Many small lattices advanced together by one persistent kernel launch per call
    (include/lb.h, lb_batch_*). `workloads` are lbinputs.Workload objects sharing the
    velocity sets; a workload's `init` (rho, ux, uy) is applied to its lattice."""

    def __init__(self, workloads, store="f32", stream=None, torch_allocator=True):
        import torch
        stream = stream or torch.cuda.current_stream()
        self._alloc = _TorchAllocator(stream) if torch_allocator else None
        sp = getattr(stream, "cuda_stream", stream)
        ws = list(workloads)
        n = len(ws)
        self.store = STORES[store] if isinstance(store, str) else int(store)
        self.sets = tuple(int(x) for x in ws[0].sets)
        grids, kns = (lb_grid * n)(), (lb_kn * n)()
        walls, opts = (lb_wall * (4 * n))(), (lb_opts * n)()
        maps = [np.ascontiguousarray(np.asarray(w.region_map, dtype=np.uint8).reshape(w.ny, w.nx)) for w in ws]
        mp = (ctypes.c_void_p * n)(*[m.ctypes.data for m in maps])
        for i, w in enumerate(ws):
            if tuple(int(x) for x in w.sets) != self.sets:
                raise ValueError("batched lattices share the velocity sets")
            grids[i] = lb_grid(w.nx, w.ny, 0.0, w.cfl, 0.0)
            kns[i] = lb_kn(w.kn_ref, w.rho_ref, w.tau_mode)
            for k, wl in enumerate(_walls(w.walls)):
                walls[4 * i + k] = wl
            o = opts[i]
            o.store = self.store
            o.iface = LB_IFACE_HERMITE if w.iface == "hermite" else LB_IFACE_PAPER
            o.rho0, o.gx, o.gy = w.rho0, w.gx, w.gy
            o.reduce_every, o.variant, o.stream = 0, 0, sp
            if self._alloc:
                o.alloc, o.free = self._alloc.alloc, self._alloc.free
        self._keep = (grids, kns, walls, opts, maps, mp)
        self.ptr = ctypes.c_void_p()
        _check(_lib.lb_batch_create(n, grids, mp, (ctypes.c_int32 * 2)(*self.sets), kns, walls, opts,
                                    ctypes.byref(self.ptr)))
        self.n, self.workloads = n, ws
        self._views = [None] * n
        for i, w in enumerate(ws):
            if w.init is not None:
                self.lattice(i).init_equilibrium(*w.init)

    def step(self, n=1):
        _check(_lib.lb_batch_step(self.ptr, int(n)))

    def step_each(self, n=1):
        _check(_lib.lb_batch_step_each(self.ptr, int(n)))

    def graph(self, nsteps, replays=1):
        _check(_lib.lb_batch_graph(self.ptr, int(nsteps), int(replays)))

    def sync(self):
        _check(_lib.lb_batch_sync(self.ptr))

    def info(self):
        t, g = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.lb_batch_info(self.ptr, ctypes.byref(t), ctypes.byref(g)))
        return {"block_threads": t.value, "grid_blocks": g.value}

    def lattice(self, i):
        if self._views[i] is None:
            ctx = _lib.lb_batch_instance(self.ptr, int(i))
            if not ctx:
                raise LBError(LB_ERR_INVALID, _lib.lb_last_error().decode())
            w = self.workloads[i]
            self._views[i] = Lattice._view(ctypes.c_void_p(ctx), w.nx, w.ny, self.sets, self.store, self)
        return self._views[i]

    @property
    def cells(self):
        return sum(w.nx * w.ny for w in self.workloads)

    def close(self):
        if getattr(self, "ptr", None):
            for v in self._views:
                if v is not None:
                    v.ctx = None
            _lib.lb_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
