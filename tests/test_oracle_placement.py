"""Pins of the learned-placement oracle (oracle/placement.py) against facts fixed by the
Hermite expansion (Sec. 2.1) and by the definitions of its features: equilibrium and
second-order perturbations leave no beyond-second-order residual, third- and
fourth-order Hermite modes leave all of theirs (with closed-form norms), the norm splits
orthogonally (Pythagoras), and the features of known fields take their closed-form
values."""
import numpy as np
import pytest

import oracle
from oracle import placement

N1DS = (3, 4, 6)


def _modes(n1d):
    cx, cy, w = oracle.velocity_set(n1d)
    return cx, cy, w


@pytest.mark.parametrize("n1d", N1DS)
def test_equilibrium_in_second_order_span(n1d):
    """f^eq (Eq. (demoeq)) is a second-order Hermite polynomial times w, so the
    projection returns it unchanged (r is 0 / 0 there: both norms are rounding)."""
    rng = np.random.default_rng(5)
    w = _modes(n1d)[2]
    for _ in range(5):
        rho, ux, uy = 0.5 + rng.random(), 0.2 * rng.standard_normal(), 0.2 * rng.standard_normal()
        f = oracle.feq(n1d, rho, ux, uy)
        p2 = oracle.project(n1d, f, n1d)
        assert ((f - p2) ** 2 / w).sum() < 1e-28 * (f ** 2 / w).sum()


@pytest.mark.parametrize("n1d", N1DS)
def test_residual_zero_for_second_order_disturbance(n1d):
    """A non-equilibrium part inside the second-order Hermite span (xi_x xi_y and
    xi_x^2 - 1 modes, no mass or momentum) is fully held: e3 = 0."""
    cx, cy, w = _modes(n1d)
    f0 = oracle.feq(n1d, 1.2, 0.05, -0.03)
    g = w * (0.01 * cx * cy + 0.004 * (cx * cx - 1.0))
    assert placement.hermite_residual_node(f0 + g, n1d) < 1e-15


@pytest.mark.parametrize("n1d", N1DS)
def test_residual_of_third_and_fourth_order_modes(n1d):
    """Pure Hermite modes above second order have no mass, momentum or second-order
    moment on any of the product sets (each 1-D rule integrates degree <= 5 exactly), so
    none of them is held: e3 = eps sqrt(sum_a w_a H_a^2) / rho, with
    sum w ((xi_x^2 - 1) xi_y)^2 = 2 * 1 and sum w ((xi_x^2 - 1)(xi_y^2 - 1))^2 = 2 * 2."""
    cx, cy, w = _modes(n1d)
    rho, eps = 1.3, 1e-3
    f0 = oracle.feq(n1d, rho, 0.0, 0.0)
    h3 = (cx * cx - 1.0) * cy
    assert abs(placement.hermite_residual_node(f0 + eps * w * h3, n1d) - eps * np.sqrt(2.0) / rho) < 1e-15
    h4 = (cx * cx - 1.0) * (cy * cy - 1.0)
    assert abs(placement.hermite_residual_node(f0 + eps * w * h4, n1d) - eps * 2.0 / rho) < 1e-15


@pytest.mark.parametrize("n1d", N1DS)
def test_residual_pythagoras(n1d):
    """||f - feq||^2 = ||f - P2 f||^2 + ||P2 f - feq||^2 in sum g^2 / w for arbitrary
    positive populations (pins the norm and the projection together), and e3 is the
    first of those norms over rho."""
    cx, cy, w = _modes(n1d)
    rng = np.random.default_rng(11)
    for _ in range(10):
        f = w * (1.0 + 0.3 * rng.random(w.size))
        rho = f.sum()
        ux, uy = (f * cx).sum() / rho, (f * cy).sum() / rho
        fe = oracle.feq(n1d, rho, ux, uy)
        p2 = oracle.project(n1d, f, n1d)
        a = ((f - fe) ** 2 / w).sum()
        b = ((f - p2) ** 2 / w).sum()
        c = ((p2 - fe) ** 2 / w).sum()
        assert abs(a - (b + c)) <= 1e-12 * a
        assert abs(placement.hermite_residual_node(f, n1d) - np.sqrt(b) / rho) < 1e-14


def test_features_closed_forms():
    """Rest state with a linear density along x between diffuse walls: no stress or
    heat flux, the exact slope in the gradient feature (central differences are exact
    on a line, one-sided ones too), wall distance j h, Kn from the density scaling."""
    nx, ny = 12, 9
    o = oracle.Oracle(nx, ny, np.zeros((ny, nx)), kn_ref=0.2, rho_ref=1.0,
                      walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"}})
    h = o.h
    slope = 0.3
    x = np.arange(nx) * h
    rho = np.broadcast_to(1.0 + slope * x, (ny, nx)).copy()
    o.init_equilibrium(rho, 0.0, 0.0)
    m = o.moments()
    F = placement.features(m, h, 0.2, 1.0, periodic_x=False, periodic_y=False, wall_bottom=True, wall_top=True)
    assert np.abs(F[:5]).max() < 1e-13
    j = np.arange(ny)[:, None]
    np.testing.assert_allclose(F[5], np.broadcast_to(np.minimum(j, ny - 1 - j) * h, (ny, nx)), rtol=0, atol=1e-15)
    kn = 0.2 / rho
    np.testing.assert_allclose(F[6], kn, rtol=1e-14)
    np.testing.assert_allclose(F[7], kn * slope / rho, rtol=1e-10)


def test_features_periodic_gradient_and_no_walls():
    """Periodic sine density: the wrapped central difference equals sin(kh)/h times the
    exact derivative; with no diffuse wall the distance feature is 1."""
    nx, ny = 16, 6
    o = oracle.Oracle(nx, ny, np.zeros((ny, nx)), h=1.0 / nx, kn_ref=0.1, rho_ref=0.0,
                      walls={"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}})
    h = o.h
    k = 2.0 * np.pi
    x = np.arange(nx) * h
    rho = np.broadcast_to(1.0 + 0.05 * np.sin(k * x), (ny, nx)).copy()
    o.init_equilibrium(rho, 0.0, 0.0)
    F = placement.features(o.moments(), h, 0.1, 0.0, periodic_x=True, periodic_y=True, wall_bottom=False,
                           wall_top=False)
    grad = 0.05 * k * np.cos(k * x) * np.sin(k * h) / (k * h)
    np.testing.assert_allclose(F[7], 0.1 * np.abs(grad) / rho, rtol=1e-10, atol=1e-15)
    assert np.all(F[5] == 1.0)
    assert np.all(F[6] == 0.1)


def test_shear_stress_feature_sign():
    """Couette flow with the top wall moving +x: du/dy > 0, so the non-equilibrium
    shear stress Pi^neq_xy = -tau rho du/dy is negative in the bulk (Chapman-Enskog,
    tau = Kn at rho = rho_ref), within the forward-Euler and Knudsen-layer corrections."""
    from lbinputs import couette
    w = couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=0)
    o = oracle.Oracle(w.nx, w.ny, w.region_map, kn_ref=w.kn_ref, rho_ref=w.rho_ref, walls=w.walls)
    o.init_equilibrium(1.0, 0.0, 0.0)
    o.step(4000)
    m = o.moments()
    F = placement.features(m, o.h, w.kn_ref, w.rho_ref, True, False, True, True)
    mid = slice(12, 20)
    dudy = np.gradient(m["ux"][:, 0], o.h)[mid]
    pred = -w.kn_ref * dudy
    got = F[1][mid, 0]
    assert np.all(got < 0)
    np.testing.assert_allclose(got, pred, rtol=0.1)
