"""The D2Q9 stream-and-collide reduction (lb_opts.scheme = LB_SCHEME_STREAM) through the
C ABI against its FP64 oracle (oracle/exact_stream.py): populations on a periodic box
with a ragged tile, a non-uniform start and a body force; FP32 deviations within the
FP32 bound; the shear-wave viscosity c_s^2 (tau - dt / 2) measured on the GPU."""
import numpy as np
import pytest

from oracle import exact_stream as es

pytestmark = pytest.mark.gpu

PERIODIC = {s: {"kind": "periodic"} for s in ("bottom", "top", "left", "right")}


def _box(nx, ny, store, kn_ref, rho_ref=0.0, gx=0.0, gy=0.0, init=None):
    import paper_1007_4895_gb300 as lb
    lat = lb.Lattice(nx, ny, np.zeros((ny, nx), np.uint8), sets=(9, 36), kn_ref=kn_ref, rho_ref=rho_ref, walls=PERIODIC,
                     store=store, gx=gx, gy=gy, scheme="stream")
    if init is not None:
        lat.init_equilibrium(*init)
    return lat


def _start(nx, ny, seed=2):
    rng = np.random.default_rng(seed)
    y = (np.arange(ny)[:, None] + 0.5) / ny
    x = (np.arange(nx)[None, :] + 0.5) / nx
    rho = 1.0 + 0.01 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 1e-3 * rng.standard_normal((ny, nx))
    ux = 0.02 * np.sin(2 * np.pi * y) + 1e-3 * rng.standard_normal((ny, nx))
    uy = 0.01 * np.sin(2 * np.pi * x) + 1e-3 * rng.standard_normal((ny, nx))
    return rho, ux * np.ones((ny, nx)), uy * np.ones((ny, nx))


@pytest.mark.parametrize("nx,ny", [(200, 48), (203, 19), (37, 9), (1029, 6)])
def test_stream_scheme_fp64_populations_match_oracle(nx, ny):
    """Four nodes per thread with neighbours by warp shuffles: widths that end inside a
    quad, inside a warp, and one warp past a block."""
    steps = 120
    kn = 0.02 * 48 / ny   # dt scales with 1 / ny: dt / tau about 0.6 at every size
    rho, ux, uy = _start(nx, ny)
    lat = _box(nx, ny, "f64", kn_ref=kn, rho_ref=1.0, gx=2e-3, gy=-1e-3, init=(rho, ux, uy))
    assert np.isclose(lat.dt, lat.h / np.sqrt(3.0), rtol=1e-15)
    lat.step(steps)
    f = es.run(es.equilibrium(rho, ux, uy), steps, dt=lat.dt, kn_ref=kn, rho_ref=1.0, gx=2e-3, gy=-1e-3)
    got = lat.populations(0)
    assert np.max(np.abs(got - f)) / np.max(np.abs(f)) < 1e-12


@pytest.mark.parametrize("nx,ny", [(200, 48), (203, 19)])
def test_stream_scheme_fp32_deviations_match_oracle(nx, ny):
    steps = 120
    kn = 0.02 * 48 / ny
    rho, ux, uy = _start(nx, ny)
    lat = _box(nx, ny, "f32_dev", kn_ref=kn, rho_ref=1.0, gx=2e-3, init=(rho, ux, uy))
    lat.step(steps)
    f = es.run(es.equilibrium(rho, ux, uy), steps, dt=lat.dt, kn_ref=kn, rho_ref=1.0, gx=2e-3)
    r, u, v = es.moments(f)
    m = lat.moments()
    uref = np.max(np.hypot(u, v))
    assert np.max(np.hypot(m["ux"] - u, m["uy"] - v)) / uref < 1e-6
    assert np.max(np.abs(m["rho"] - r)) < 1e-6


def test_stream_scheme_viscosity_is_tau_minus_half_dt():
    """Shear wave on the GPU: decay rate nu = tau - dt / 2 within 1 %."""
    ny, nx = 128, 8
    y = (np.arange(ny) + 0.5) / ny
    ux = np.broadcast_to(1e-3 * np.sin(2 * np.pi * y)[:, None], (ny, nx))
    dt = (1.0 / ny) / np.sqrt(3.0)
    tau = 1.5 * dt
    lat = _box(nx, ny, "f64", kn_ref=tau, init=(np.ones((ny, nx)), ux, np.zeros((ny, nx))))
    lat.step(200)
    a1 = lat.moments()["ux"][:, 0] @ np.sin(2 * np.pi * y)
    lat.step(2000)
    a2 = lat.moments()["ux"][:, 0] @ np.sin(2 * np.pi * y)
    nu = -np.log(a2 / a1) / ((2 * np.pi) ** 2 * 2000 * lat.dt)
    assert abs(nu / (tau - 0.5 * lat.dt) - 1.0) < 0.01, (nu, tau - 0.5 * lat.dt)
