"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a,
loads, exports every entry point include/lb.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1007_4895_gb300 as lb
    return lb


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("lb_create", "lb_step", "lb_moments", "lb_reductions", "lb_destroy", "lb_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lb):
    so = ctypes.CDLL(lb.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(so, n)]
    assert not missing, missing
    assert set(lb.EXPORTS) == declared_symbols()


def _args(lb, nx=8, ny=8, **over):
    grid = lb.lb_grid(nx, ny, 0.0, 0.5, 0.0)
    kn = lb.lb_kn(over.get("kn", 0.1), 1.0, 0)
    walls = [lb.lb_wall(1, 0, 0, 1, 0), lb.lb_wall(1, 0, 0, 1, 0), lb.lb_wall(0, 0, 0, 1, 0), lb.lb_wall(0, 0, 0, 1, 0)]
    for k, v in over.get("walls", {}).items():
        walls[k] = v
    opts = lb.lb_opts()
    opts.store, opts.iface, opts.rho0 = over.get("store", 1), over.get("iface", 1), over.get("rho0", 1.0)
    opts.rounding = over.get("rounding", 0)
    opts.scheme = over.get("scheme", 0)
    if "rho0_col" in over:
        col = np.full(nx, 1.0) if over["rho0_col"] == "ones" else np.where(np.arange(nx) == 3, -1.0, 1.0)
        opts.rho0_col = np.ascontiguousarray(col).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return grid, np.zeros((ny, nx), np.uint8), over.get("sets", (9, 36)), kn, walls, opts


@pytest.mark.parametrize("case", [
    dict(nx=2), dict(ny=3), dict(sets=(9, 25)), dict(store=9), dict(iface=5), dict(rho0=0.0), dict(kn=-1.0),
    dict(kn=1e-6),                                  # dt / tau > 1
    dict(rounding=2),                               # unknown rounding mode
    dict(store=1, rho0_col="ones"),                 # per-column reference density: deviation formats only
    dict(store=2, rho0_col="negative"),             # per-column reference densities must be positive
    dict(scheme=2),                                 # unknown scheme
    dict(scheme=1),                                 # stream-and-collide: walls must be periodic
    dict(scheme=1, sets=(16, 36), walls="periodic"),    # stream-and-collide: D2Q9 only
    dict(walls={0: None}),                          # bottom periodic, top diffuse (filled below)
])
def test_invalid_arguments_are_rejected_on_the_host(lb, case):
    over = dict(case)
    if over.get("walls") == "periodic":
        over["walls"] = {0: lb.lb_wall(0, 0, 0, 1, 0), 1: lb.lb_wall(0, 0, 0, 1, 0)}
    elif "walls" in over:
        over["walls"] = {0: lb.lb_wall(0, 0, 0, 1, 0)}
    nx, ny = over.pop("nx", 8), over.pop("ny", 8)
    args = _args(lb, nx, ny, **over)
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(*args)
    assert e.value.code == lb.LB_ERR_INVALID
    assert lb.lb_last_error()


def test_region_map_values_checked(lb):
    grid, m, sets, kn, walls, opts = _args(lb)
    m[3, 3] = 2
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(grid, m, sets, kn, walls, opts)
    assert e.value.code == lb.LB_ERR_INVALID


def test_paper_interface_mode_needs_x_uniform_rows(lb):
    grid, m, sets, kn, walls, opts = _args(lb, nx=256, ny=16, iface=0)
    m[:3, :128] = 1         # one 128-column tile high-order, its neighbour not
    with pytest.raises(lb.LBError) as e:
        lb.lb_create(grid, m, sets, kn, walls, opts)
    assert e.value.code == lb.LB_ERR_INVALID


def _batch_call(lb, n=2, **over):
    """lb_batch_create with n small lattices; `over` changes lattice 1."""
    grids = (lb.lb_grid * n)(*[lb.lb_grid(8, 16, 0.0, 0.5, 0.0) for _ in range(n)])
    kns = (lb.lb_kn * n)(*[lb.lb_kn(0.1, 1.0, 0) for _ in range(n)])
    walls = (lb.lb_wall * (4 * n))()
    for i in range(n):
        walls[4 * i + 0] = lb.lb_wall(1, 0.0, 0.0, 1.0, 0.0)
        walls[4 * i + 1] = lb.lb_wall(1, 0.05, 0.0, 1.0, 0.0)
        walls[4 * i + 2] = lb.lb_wall(0, 0.0, 0.0, 1.0, 0.0)
        walls[4 * i + 3] = lb.lb_wall(0, 0.0, 0.0, 1.0, 0.0)
    opts = (lb.lb_opts * n)()
    for i in range(n):
        opts[i].store, opts[i].iface, opts[i].rho0 = 1, 1, 1.0
    for k, v in over.get("walls", {}).items():
        walls[4 + k] = v
    keep = []
    for k, v in over.get("opts", {}).items():
        if k == "rho0_col":
            keep.append(np.ones(8))
            v = keep[-1].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        setattr(opts[1], k, v)
    maps = [np.zeros((16, 8), np.uint8) for _ in range(n)]
    mp = (ctypes.c_void_p * n)(*[m.ctypes.data for m in maps])
    out = ctypes.c_void_p()
    code = lb._lib.lb_batch_create(n, grids, mp, (ctypes.c_int32 * 2)(9, 36), kns, walls, opts, ctypes.byref(out))
    return code, out


@pytest.mark.parametrize("case", [
    dict(opts={"iface": 0}),                        # mode A interface rows need their own pass
    dict(opts={"reduce_every": 10}),                # no in-step reductions inside the batch
    dict(opts={"store": 2}),                        # one storage format for the batch
    dict(opts={"rho0": 2.0}),                       # one rest density for the batch
    dict(opts={"rho0_col": "ones"}),                # one reference density per lattice
    dict(walls={1: "osc"}),                         # oscillating wall
    dict(walls={2: "pressure"}),                    # pressure side
])
def test_batch_restrictions_rejected_before_device_work(lb, case):
    over = dict(case)
    if "walls" in over:
        k, kind = next(iter(over["walls"].items()))
        if kind == "osc":
            w = lb.lb_wall(1, 0.05, 0.0, 1.0, 2.0)
            over["walls"] = {k: w}
        else:
            over["walls"] = {2: lb.lb_wall(2, 0.0, 0.0, 1.5, 0.0), 3: lb.lb_wall(2, 0.0, 0.0, 1.0, 0.0)}
    code, out = _batch_call(lb, **over)
    assert code == lb.LB_ERR_INVALID
    assert not out.value
    assert lb.lb_last_error()


def test_batch_argument_checks(lb):
    out = ctypes.c_void_p()
    assert lb._lib.lb_batch_create(0, None, None, None, None, None, None, ctypes.byref(out)) == lb.LB_ERR_INVALID
    assert lb._lib.lb_batch_step(None, 1) == lb.LB_ERR_INVALID
    assert lb._lib.lb_batch_instance(None, 0) is None
