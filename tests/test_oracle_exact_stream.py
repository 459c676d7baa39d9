"""Pins of the D2Q9 stream-and-collide oracle (oracle/exact_stream.py) against what the
mathematics fixes: the quadrature, exact streaming by one node along xi, conservation
of mass and momentum by the collision, the uniform equilibrium as a fixed point, and
the shear-wave decay rate of lattice BGK, nu = c_s^2 (tau - dt / 2) with c_s^2 = 1."""
import numpy as np
import pytest

from oracle import exact_stream as es


def test_d2q9_weights_and_moments():
    """Sum w = 1, sum w xi = 0, sum w xi xi = I (T = 1), fourth moment 3 (Gauss-Hermite)."""
    cx, cy, w = es.d2q9()
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert abs((w * cx).sum()) < 1e-15 and abs((w * cy).sum()) < 1e-15
    assert np.isclose((w * cx * cx).sum(), 1.0) and np.isclose((w * cy * cy).sum(), 1.0)
    assert abs((w * cx * cy).sum()) < 1e-15
    assert np.isclose((w * cx ** 4).sum(), 3.0)


def test_streaming_moves_each_population_one_node_along_its_velocity():
    cx, cy, _ = es.d2q9()
    ny, nx, x0, y0 = 7, 9, 4, 3
    for a in range(9):
        f = np.zeros((9, ny, nx))
        f[a, y0, x0] = 1.0
        g = es.stream(f)
        ys, xs = np.nonzero(g[a])
        assert (ys[0] - y0, xs[0] - x0) == (int(np.sign(cy[a])), int(np.sign(cx[a]))), a
        assert g.sum() == 1.0


def test_collision_conserves_mass_and_momentum():
    rng = np.random.default_rng(5)
    ny, nx = 12, 10
    rho = 1.0 + 0.05 * rng.standard_normal((ny, nx))
    ux, uy = 0.05 * rng.standard_normal((2, ny, nx))
    f = es.equilibrium(rho, ux, uy) * (1.0 + 0.01 * rng.standard_normal((9, ny, nx)))
    cx, cy, _ = es.d2q9()
    m0 = f.sum()
    px0, py0 = (cx[:, None, None] * f).sum(), (cy[:, None, None] * f).sum()
    g = es.run(f, 20, dt=0.01, kn_ref=0.02, rho_ref=1.0)
    assert abs(g.sum() - m0) < 1e-12 * m0
    assert abs((cx[:, None, None] * g).sum() - px0) < 1e-12 * m0
    assert abs((cy[:, None, None] * g).sum() - py0) < 1e-12 * m0


def test_uniform_equilibrium_is_a_fixed_point():
    ny, nx = 5, 6
    f = es.equilibrium(np.full((ny, nx), 1.3), np.full((ny, nx), 0.04), np.full((ny, nx), -0.02))
    g = es.step(f, dt=0.01, kn_ref=0.02)
    assert np.max(np.abs(g - f)) < 1e-15


@pytest.mark.parametrize("tau_over_dt", [0.8, 1.0, 2.0])
def test_shear_wave_decays_with_viscosity_tau_minus_half_dt(tau_over_dt):
    """u_x = U sin(2 pi y / L) decays as exp(-nu k^2 t); the rate measured after the
    initial transient gives nu = tau - dt / 2 within 1 % (k h = 2 pi / 128), and not
    tau or tau + dt / 2."""
    ny, nx = 128, 4
    h = 1.0 / ny
    dt = h / np.sqrt(3.0)
    tau = tau_over_dt * dt
    y = (np.arange(ny) + 0.5) * h
    ux = np.broadcast_to(1e-3 * np.sin(2 * np.pi * y)[:, None], (ny, nx)).copy()
    f = es.equilibrium(np.ones((ny, nx)), ux, np.zeros((ny, nx)))
    f = es.run(f, 200, dt=dt, kn_ref=tau)
    a1 = es.moments(f)[1][:, 0] @ np.sin(2 * np.pi * y)
    n = 2000
    f = es.run(f, n, dt=dt, kn_ref=tau)
    a2 = es.moments(f)[1][:, 0] @ np.sin(2 * np.pi * y)
    nu = -np.log(a2 / a1) / ((2 * np.pi) ** 2 * n * dt)
    assert abs(nu / (tau - 0.5 * dt) - 1.0) < 0.01, (nu, tau - 0.5 * dt)
