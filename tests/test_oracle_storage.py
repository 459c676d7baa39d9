"""Pins of the oracle's storage model (or_set_storage): the rounding a finite-precision
storage format applies to each stored deviation, used to compute in FP64 the error that
a storage format alone adds to the method.

Pinned against numpy's IEEE conversions (FP32, FP16 nearest), the definition of BF16 as
the upper half of FP32 (nearest: the closer of the two bracketing codes), and the
defining property of stochastic rounding: the result is one of the two bracketing codes
and is exact on average. The key hash (lowbias32) is pinned by bijectivity and bit
balance on a sample. On a lattice, every stored deviation is representable in its
format after a step, and a rest state is left exactly at rest."""
import numpy as np
import pytest

import oracle
from lbinputs import band_map

RNG = np.random.default_rng(2024)


def _bf16_neighbours(v):
    b = np.float32(v).view(np.uint32)
    lo = np.uint32(b & np.uint32(0xffff0000)).view(np.float32)
    hi = np.uint32((b & np.uint32(0xffff0000)) + np.uint32(0x10000)).view(np.float32)
    return float(lo), float(hi)


def test_nearest_modes_match_ieee_conversions():
    vals = np.concatenate([RNG.standard_normal(400) * 0.3, RNG.standard_normal(100) * 1e-4, [0.0, -0.0, 1.0]])
    for v in vals:
        assert oracle.store_round("f32_dev", v) == float(np.float32(v))
        assert oracle.store_round("f16_dev", v) == float(np.float16(np.float32(v)))
        r = oracle.store_round("bf16_dev", v)
        f = float(np.float32(v))
        lo, hi = _bf16_neighbours(f)
        assert r in (lo, hi)                                  # a bracketing BF16 code
        assert abs(r - f) <= min(abs(lo - f), abs(hi - f)) + 0.0   # the nearer one
        assert np.float32(r).view(np.uint32) & np.uint32(0xffff) == 0


@pytest.mark.parametrize("mode,ulp", [("f16_dev_sr", None), ("bf16_dev_sr", None)])
def test_stochastic_modes_bracket_and_are_exact_on_average(mode, ulp):
    keys = np.arange(0, 2 ** 32, 2 ** 32 // 4000, dtype=np.uint64)
    for v in (0.1, -0.37, 3.3e-3, 0.7731):
        f = float(np.float32(v))
        r = np.array([oracle.store_round(mode, v, int(k)) for k in keys])
        codes = np.unique(r)
        assert len(codes) <= 2
        if mode == "f16_dev_sr":
            assert all(float(np.float16(c)) == c for c in codes)
        else:
            assert all(np.float32(c).view(np.uint32) & np.uint32(0xffff) == 0 for c in codes)
        assert codes.min() <= f <= codes.max()
        spread = codes.max() - codes.min()
        # the mean of a two-valued variable over 4000 evenly spread keys
        assert abs(r.mean() - f) < 0.03 * spread + 1e-12, (mode, v, r.mean(), f)
    # a wall-set value is rounded to nearest
    assert oracle.store_round(mode, 0.1, 123, set_value=True) == oracle.store_round(mode.replace("_sr", ""), 0.1)


def _lowbias32(x):
    """The published finaliser, on uint64 arrays (for the statistics below)."""
    m = np.uint64(0xffffffff)
    x = x & m
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7feb352d)) & m
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846ca68b)) & m
    x ^= x >> np.uint64(16)
    return x


def test_stochastic_keys_are_unbiased_per_bit():
    """The stochastic rounding of one value over consecutive step keys of one node and
    population: the share of upward roundings equals the rounded fraction."""
    v = 0.1
    f = float(np.float32(v))
    n = 20000
    ups = 0
    for step in range(n):
        r = oracle.lib().or_store_round(oracle.STORAGE_MODES["f16_dev_sr"], v,
                                        int(_lowbias32(np.uint64(step * 2654435761))), 0)
        ups += r > f
    codes = sorted({float(np.float16(f)), float(np.nextafter(np.float16(f), np.float16(1)))})
    hi = max(c for c in codes)
    lo = min(c for c in codes)
    frac = (f - lo) / (hi - lo)
    assert abs(ups / n - frac) < 0.02, (ups / n, frac)


# the stored f = w (rho0 + d) is read back as f / w - rho0 in FP64, which moves d by a few
# units of 2^-53 rho0: representable up to 1e-15 (the nearest code of the format)
@pytest.mark.parametrize("mode,check", [
    ("f32_dev", lambda d: np.all(np.abs(d - d.astype(np.float32)) <= 1e-15)),
    ("f16_dev", lambda d: np.all(np.abs(d - d.astype(np.float16)) <= 1e-15)),
    ("bf16_dev_sr", lambda d: np.all(np.abs(d - (
        (d.astype(np.float32).view(np.uint32) + np.uint32(0x8000)) & np.uint32(0xffff0000)).view(np.float32)) <= 1e-15)),
])
def test_lattice_stores_representable_deviations(mode, check):
    nx, ny, rho0 = 4, 16, 1.0
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 3), kn_ref=0.1,
                      walls={"bottom": {"kind": "diffuse", "ux": -0.08}, "top": {"kind": "diffuse", "ux": 0.08}})
    o.init_equilibrium(rho0, 0.0, 0.0)
    o.set_storage(mode, rho0=rho0)
    o.step(7)
    for s, n1d in ((0, 3), (1, 6)):
        _, _, w = oracle.velocity_set(n1d)
        f = o.populations(s)
        own = o.map == s
        d = f / w[:, None, None] - rho0
        assert check(d[:, own])


@pytest.mark.parametrize("mode", ["f32", "f32_dev", "f16_dev", "bf16_dev", "f16_dev_sr", "bf16_dev_sr"])
def test_rest_state_stays_at_rest_under_every_storage_model(mode):
    nx, ny = 4, 12
    o = oracle.Oracle(nx, ny, band_map(nx, ny, 3), kn_ref=0.1,
                      walls={"bottom": {"kind": "diffuse"}, "top": {"kind": "diffuse"}})
    o.init_equilibrium(1.0, 0.0, 0.0)
    f0 = [o.populations(0), o.populations(1)]
    o.set_storage(mode, rho0=1.0)
    o.step(5)
    for s in (0, 1):
        np.testing.assert_allclose(o.populations(s), f0[s], rtol=2e-7 if mode == "f32" else 1e-14, atol=1e-16)


def test_lowbias32_sample_is_a_bijection_with_balanced_bits():
    """The key hash, through the stochastic rounding's thresholds: distinct keys give
    distinct 24-bit thresholds almost always, and each bit of the hash is set half the
    time."""
    x = _lowbias32(np.arange(1, 200001, dtype=np.uint64))
    assert len(np.unique(x)) == len(x)
    bits = ((x[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.01)
