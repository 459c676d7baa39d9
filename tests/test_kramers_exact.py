"""Pins of the exact half-space solution used for Kramers' problem (Sec. 3.3),
``dvm_exact.half_space``: the discrete BGK equations and the wall condition hold at
every point, the D2Q9 slip coefficient has its closed form, and the same profile comes
out of the two-wall solution of a wide channel (an independent linear system)."""
import math

import numpy as np
import pytest

import dvm_exact


def test_d2q9_half_space_slip_is_sqrt3_with_no_knudsen_layer():
    """One gas-bound abscissa (sqrt 3) and no decaying mode: g(0) = zeta - sqrt 3 = 0."""
    zeta, lams, c, _ = dvm_exact.half_space(3)
    assert len(lams) == 0
    assert abs(zeta - math.sqrt(3.0)) < 1e-14


@pytest.mark.parametrize("n", [4, 6, 8])
def test_half_space_solution_satisfies_the_discrete_bgk_equations(n):
    """r_j g_j' = -(g_j - u) for every abscissa (lengths in tau), u = sum_j w_j g_j,
    g_j(0) = 0 on the gas-bound abscissae, and each mode solves the dispersion relation."""
    r, w = dvm_exact.rule(n)
    zeta, lams, c, u = dvm_exact.half_space(n)
    assert len(lams) == n // 2 - 1
    for l in lams:
        assert abs(np.sum(w / (1.0 - l * r)) - 1.0) < 1e-10
    y = np.linspace(0.0, 12.0, 97)
    g = np.array([y + zeta - rj + sum(cm * np.exp(-l * y) / (1.0 - l * rj) for cm, l in zip(c, lams)) for rj in r])
    dg = np.array([1.0 + sum(-l * cm * np.exp(-l * y) / (1.0 - l * rj) for cm, l in zip(c, lams)) for rj in r])
    assert np.max(np.abs(w @ g - u(y))) < 1e-12
    assert np.max(np.abs(r[:, None] * dg + g - u(y)[None])) < 1e-12
    assert np.max(np.abs(g[r > 0, 0])) < 1e-12


@pytest.mark.parametrize("n", [4, 6])
def test_half_space_profile_matches_a_wide_channel(n):
    """Between diffuse plates 400 tau apart (bottom at rest, top moving) the layer at the
    bottom plate is the half-space one, scaled by the bulk shear rate."""
    H, U = 400.0, 1.0
    ch = dvm_exact.channel(n, 1.0, H=H, u_bottom=0.0, u_top=U)
    gamma = (ch(220.0) - ch(180.0)) / 40.0
    zeta, _, _, u = dvm_exact.half_space(n)
    y = np.linspace(0.0, 30.0, 61)
    assert np.max(np.abs(ch(y) / gamma - u(y))) < 1e-8 * H
    # the bulk line extrapolates to zero at y = -zeta (in units of tau)
    assert abs(ch(200.0) / gamma - (200.0 + zeta)) < 1e-8 * H


def test_slip_coefficient_grows_with_the_set_below_the_bgk_value():
    """More abscissae resolve the Knudsen layer better: zeta increases with n (D2Q16,
    D2Q36, D2Q64, D2Q144 1-D rules) and stays below the continuous BGK value
    1.1466 in units of (mu / p) sqrt(pi R T / 2), i.e. 1.437 tau."""
    z = [dvm_exact.half_space(n)[0] for n in (4, 6, 8, 12)]
    assert all(a < b for a, b in zip(z, z[1:])), z
    assert z[-1] < 1.1466 * math.sqrt(math.pi / 2.0), z
