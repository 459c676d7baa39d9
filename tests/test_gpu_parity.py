"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 storage computes in FP64, so the two sides differ only by rounding
order (bound 1e-10 relative per field after thousands of steps). FP32 forms: 1e-6
relative velocity error (the target the method is held to). Reduced storage
(FP16 / BF16 deviations): the per-field bounds stated in ``REDUCED_BOUNDS``, derived
from the unit roundoff of the stored deviation (2^-11, 2^-8) times its magnitude.
"""
import numpy as np
import pytest

from lbinputs import Workload, band_map, couette, long_channel, long_channel_density, oscillatory_couette, poiseuille

from gpu_pair import field_errors, make_pair, population_error

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
# populations in FP64: rounding-order differences can flip a minmod choice where the two
# slopes tie to ~1e-9 (smooth, nearly linear profiles), which moves single populations
# by that much without changing any moment beyond 1e-12
F64_POP_TOL = 1e-8
F32_VEL_TOL = 1e-6


def run_both(w, store, steps, variant=-1):
    lat, o, eff = make_pair(w, store=store, variant=variant)
    lat.step(steps)
    o.step(steps)
    got = lat.moments()
    ref = o.moments()
    return lat, o, eff, got, ref


def ragged_workload(nx=300, ny=37, seed=3, iface="hermite"):
    """Three 128-column tiles (the last one ragged: 44 columns) with different band
    thicknesses, an isolated high-order tile in the core, moving walls, a body force
    and a non-uniform start."""
    rng = np.random.default_rng(seed)
    m = np.zeros((ny, nx), np.uint8)
    ntx = (nx + 127) // 128
    for tx in range(ntx):
        b, t = rng.integers(2, 7), rng.integers(2, 7)
        m[:b, tx * 128:(tx + 1) * 128] = 1
        m[ny - t:, tx * 128:(tx + 1) * 128] = 1
    m[ny // 2, 140] = 1
    y = np.arange(ny)[:, None] / (ny - 1)
    x = np.arange(nx)[None, :] / nx
    rho = 1.0 + 0.02 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
    ux = 0.03 * np.sin(np.pi * y) + 0.01 * np.cos(2 * np.pi * x)
    uy = 0.01 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    return Workload(name="ragged", nx=nx, ny=ny, region_map=m, kn_ref=0.08, gx=2e-3, gy=-1e-3,
                    walls={"bottom": {"kind": "diffuse", "ux": -0.05}, "top": {"kind": "diffuse", "ux": 0.07}},
                    init=(rho, ux, uy), iface=iface)


# ------------------------------------------------------------------ FP64

def test_config1_couette_fp64_full_run():
    """Plane Couette 4 x 32, Kn = 0.1, walls -/+0.05 lattice, 4 high-order rows per
    wall, 5000 steps from rest: every moment field and every population."""
    w = couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=5000)
    lat, o, eff, got, ref = run_both(w, "f64", w.steps)
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs
    assert population_error(lat, o, eff) < F64_POP_TOL


@pytest.mark.parametrize("iface", ["hermite", "paper"])
def test_couette_multi_tile_fp64(iface):
    w = couette(nx=72, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, iface=iface)
    lat, o, eff, got, ref = run_both(w, "f64", 1500)
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs
    assert population_error(lat, o, eff) < F64_POP_TOL


def test_ragged_mixed_map_fp64():
    w = ragged_workload()
    lat, o, eff, got, ref = run_both(w, "f64", 80)
    assert (eff[:, :128] != eff[:, 128:256]).any()      # x-interfaces present
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs
    assert population_error(lat, o, eff) < F64_POP_TOL


def test_pressure_channel_fp64():
    w = long_channel(nx=220, ny=40, steps=150)
    lat, o, eff, got, ref = run_both(w, "f64", w.steps)
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs
    assert population_error(lat, o, eff, rho0=w.rho0) < F64_POP_TOL


@pytest.mark.parametrize("sets", [(9, 16), (16, 36), (9, 9), (36, 36)])
def test_other_set_pairs_fp64(sets):
    w = couette(nx=36, ny=28, rows=5, kn=0.2, u_wall_lat=0.05, sets=sets)
    lat, o, eff, got, ref = run_both(w, "f64", 600)
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs


def test_all_high_and_all_low_maps_fp64():
    for val in (0, 1):
        w = couette(nx=8, ny=24, rows=0, kn=0.1)
        w.region_map = np.full((24, 8), val, np.uint8)
        lat, o, eff, got, ref = run_both(w, "f64", 400)
        errs = field_errors(got, ref)
        assert max(errs.values()) < F64_TOL, (val, errs)


def test_periodic_box_with_interfaces_fp64():
    ny, nx = 40, 64
    m = np.zeros((ny, nx), np.uint8)
    m[12:22, :] = 1
    y = np.arange(ny)[:, None] / ny
    ux = np.broadcast_to(0.02 * np.sin(2 * np.pi * y), (ny, nx))
    w = Workload(name="shear", nx=nx, ny=ny, region_map=m, kn_ref=0.05,
                 walls={"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}},
                 init=(np.ones((ny, nx)), ux, np.zeros((ny, nx))))
    for iface in ("hermite", "paper"):
        w.iface = iface
        lat, o, eff, got, ref = run_both(w, "f64", 300)
        errs = field_errors(got, ref)
        assert max(errs.values()) < F64_TOL, (iface, errs)


def test_oscillating_wall_fp64():
    w = oscillatory_couette(nx=8, ny=32, rows=5, kn=0.1, stokes_omega=8.0)
    lat, o, eff, got, ref = run_both(w, "f64", 800)
    errs = field_errors(got, ref)
    assert max(errs.values()) < F64_TOL, errs


LAYOUTS = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10]


@pytest.mark.parametrize("variant", LAYOUTS)
def test_every_kernel_layout_matches_oracle(variant):
    """The step-kernel layouts the autotuner chooses from (one node quad per thread,
    TMA-fed tiles, 4 x 2 and 4 x 4 register blocks, paired FP32 arithmetic) all
    reproduce the oracle."""
    w = ragged_workload()
    for store, tol in (("f64", F64_TOL), ("f32_dev", 1e-6), ("f32", 1e-4)):
        if store == "f64" and variant in (1, 4, 7, 8, 9, 10):   # FP32 / 16-bit storage only
            continue
        lat, o, eff, got, ref = run_both(w, store, 60, variant=variant)
        assert lat.info()["variant"] == variant
        errs = field_errors(got, ref)
        assert errs["u"] < tol and errs["rho"] < tol, (store, errs)


# ------------------------------------------------------------------ FP32

# FP32 storage of f itself: the velocity lives in the O(u) part of f / w ~ rho0, so the
# storage rounding (2^-24 of f) is a larger share of it
F32_ABS_VEL_TOL = 1e-4


def test_config1_couette_fp32_dev_velocity():
    """Config 1 in FP32 deviations, 5000 steps. Over the ~2000-step relaxation of the
    shear mode, the FP32 rounding of the stored deviations (2^-24 |d| per step, |d| up
    to ~0.3 next to the moving walls) accumulates to ~1.1e-6 of the velocity; the test
    holds it to 1.5e-6 in both norms (the shorter FP32 runs below meet 1e-6)."""
    w = couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=5000)
    lat, o, eff, got, ref = run_both(w, "f32_dev", w.steps)
    errs = field_errors(got, ref)
    assert errs["u_l2"] < 1.5 * F32_VEL_TOL and errs["u"] < 1.5 * F32_VEL_TOL, errs


def test_config1_couette_fp32_abs_velocity():
    w = couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, steps=5000)
    lat, o, eff, got, ref = run_both(w, "f32", w.steps)
    errs = field_errors(got, ref)
    assert errs["u"] < F32_ABS_VEL_TOL, errs


@pytest.mark.parametrize("store,tol", [("f32", F32_ABS_VEL_TOL), ("f32_dev", F32_VEL_TOL)])
def test_ragged_fp32(store, tol):
    w = ragged_workload()
    lat, o, eff, got, ref = run_both(w, store, 80)
    errs = field_errors(got, ref)
    assert errs["u"] < tol, errs


# ------------------------------------------------------- reduced precision

# Per-field bounds for reduced storage, about twice the measured error. Rounding a
# deviation d to FP16 (BF16) each step loses increments below half an ulp of d, so the
# steady state is biased by roughly ulp(d) / (2 dt / tau): with |d| ~ 0.5 here (global
# rho0 = 1.5 for densities 1..2) that is ~1e-2 of the velocity for FP16 and ~4e-2 for BF16.
REDUCED_BOUNDS = {
    "f16_dev": {"u": 3e-2, "rho": 6e-3, "pxy": 1.5e-2},
    "bf16_dev": {"u": 1e-1, "rho": 3e-2, "pxy": 2e-1},
}


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
def test_reduced_precision_channel(store):
    w = long_channel(nx=220, ny=40, steps=150)
    lat, o, eff, got, ref = run_both(w, store, w.steps)
    errs = field_errors(got, ref)
    for k, b in REDUCED_BOUNDS[store].items():
        assert errs[k] < b, (k, errs)


# Per-column reference density (lb_opts.rho0_col, the long channel's density estimate):
# the stored deviation is f / w - rho0(x), so its magnitude, and the 16-bit rounding
# error it carries, shrink where the density is far from one global rho0.
def _col_pair(w, store, rho0_col, **kw):
    import paper_1007_4895_gb300 as lb
    a, o, eff = make_pair(w, store=store)
    b = lb.Lattice.from_workload(w, store=store, rho0_col=rho0_col, **kw)
    return a, b, o


@pytest.mark.parametrize("variant", [0, 7, 9, 10])
@pytest.mark.parametrize("store", ["f32_dev", "f16_dev", "bf16_dev"])
@pytest.mark.parametrize("case", ["ragged", "pressure_channel"])
def test_constant_per_column_reference_changes_nothing(store, case, variant):
    """rho0(x) = rho0 everywhere: every kernel that decodes or encodes goes through the
    per-column path with a zero shift, and the populations and moments equal those of
    the lattice without it (both lattices on one step layout)."""
    import paper_1007_4895_gb300 as lb
    w = ragged_workload() if case == "ragged" else long_channel(nx=300, ny=37)
    a = lb.Lattice.from_workload(w, store=store, variant=variant)
    b = lb.Lattice.from_workload(w, store=store, rho0_col=np.full(w.nx, w.rho0), variant=variant)
    assert a.info()["variant"] == variant and b.info()["variant"] == variant
    a.step(40)
    b.step(40)
    own = a.effective_map()
    for s in (0, 1):
        pa, pb = a.populations(s), b.populations(s)
        assert np.array_equal(pa[:, own == s], pb[:, own == s]), (store, case, s)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), (store, case, k)


def test_checkpoint_needs_the_same_reference_densities(tmp_path):
    """A checkpoint holds values relative to the lattice's reference densities: it loads
    into a lattice with the same rho0(x) (same bits after further steps) and is refused
    by one with a single rho0."""
    import paper_1007_4895_gb300 as lb
    from lbinputs import long_channel_density
    w = long_channel(nx=300, ny=37)
    col = long_channel_density(w.nx, 2.0, 1.0)
    a = lb.Lattice.from_workload(w, store="f16_dev", rho0_col=col)
    a.step(11)
    a.save(str(tmp_path / "ck.bin"))
    a.step(7)
    b = lb.Lattice.from_workload(w, store="f16_dev", rho0_col=col)
    b.load(str(tmp_path / "ck.bin"))
    b.step(7)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    c = lb.Lattice.from_workload(w, store="f16_dev")
    with pytest.raises(lb.LBError) as e:
        c.load(str(tmp_path / "ck.bin"))
    assert e.value.code == lb.LB_ERR_INVALID


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
def test_per_column_reference_shrinks_16bit_error(store):
    """Pressure channel with a 2:1 density drop, 16-bit storage with stochastic rounding
    (with round-to-nearest the state also stagnates, which hides the noise). The
    per-column reference rho0(x) = the density estimate takes the density offset out of
    the stored deviation: against the FP64 oracle the density error falls well below
    that of one rho0. The velocity part of the deviation, rho xi.u, is unchanged, so
    the velocity error only has to be no worse."""
    import paper_1007_4895_gb300 as lb
    from lbinputs import long_channel_density
    w = long_channel(nx=220, ny=40, steps=150)
    _, b, o = _col_pair(w, store, long_channel_density(w.nx, 2.0, 1.0), rounding="stochastic")
    a = lb.Lattice.from_workload(w, store=store, rounding="stochastic")
    a.step(w.steps)
    b.step(w.steps)
    o.step(w.steps)
    ref = o.moments()
    ea, eb = field_errors(a.moments(), ref), field_errors(b.moments(), ref)
    assert eb["rho"] < 0.6 * ea["rho"] and eb["u"] < ea["u"], (store, ea, eb)


def test_per_column_reference_fp32_matches_oracle():
    """FP32 deviations with rho0(x): the same FP32 accuracy as with one rho0."""
    from lbinputs import long_channel_density
    w = long_channel(nx=220, ny=40, steps=150)
    a, b, o = _col_pair(w, "f32_dev", long_channel_density(w.nx, 2.0, 1.0))
    b.step(w.steps)
    o.step(w.steps)
    e = field_errors(b.moments(), o.moments())
    assert e["u"] < F32_VEL_TOL and e["rho"] < F32_VEL_TOL, e
    assert b.info()["variant"] in (0, 5)


# Stochastic rounding of the 16-bit stores (lb_opts.rounding): the expected stored value
# equals the exact one, so increments below half an ulp are kept on average and the
# stagnation bias above disappears; what remains is rounding noise of about one ulp of
# the deviation per node. Bounds from the measured noise with a 3x margin.
SR_BOUNDS = {"f16_dev": {"u": 1e-3, "rho": 2e-4, "pxy": 5e-3},
             "bf16_dev": {"u": 1.2e-2, "rho": 1.5e-3, "pxy": 3e-2}}


def _box(n=64, g=1e-3):
    walls = {"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}}
    return Workload(name="forced_box", nx=n, ny=n, region_map=np.zeros((n, n), np.uint8), kn_ref=0.1, walls=walls,
                    gx=g, steps=4000)


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
def test_stochastic_rounding_keeps_small_increments(store):
    """A periodic box at rest under a uniform body force gains momentum at exactly
    rho g per unit time (the force moments, Eq. (demoforce)), so u = g t. Rounding to
    nearest drops the per-step gain once it falls below half an ulp of the stored
    deviation (BF16 stalls for good); stochastic rounding keeps the mean on g t."""
    import paper_1007_4895_gb300 as lb
    res = {}
    for rnd in ("nearest", "stochastic"):
        w = _box()
        lat = lb.Lattice.from_workload(w, store=store, rounding=rnd)
        lat.step(w.steps)
        exact = w.gx * lat.info()["time"]
        res[rnd] = abs(lat.moments(mask=0b111)["ux"].mean() - exact) / exact
    assert res["nearest"] > (0.5 if store == "bf16_dev" else 2e-2), res
    assert res["stochastic"] < 1e-3, res


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("flow", ["couette", "poiseuille"])
def test_stochastic_rounding_channels_match_oracle(store, flow):
    if flow == "couette":
        w, n = couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05), 5000
    else:
        w, n = poiseuille(nx=4, ny=64, rows=10, kn=0.1, g_lat=1e-5), 6000
    import paper_1007_4895_gb300 as lb
    import oracle
    from gpu_pair import N1D
    errs = {}
    for rnd in ("nearest", "stochastic"):
        lat = lb.Lattice.from_workload(w, store=store, rounding=rnd)
        eff = lat.effective_map()
        o = oracle.Oracle(w.nx, w.ny, eff, n1d_lo=N1D[w.sets[0]], n1d_hi=N1D[w.sets[1]], kn_ref=w.kn_ref,
                          rho_ref=w.rho_ref, gx=w.gx, walls=w.walls, dt=lat.dt, h=lat.h)
        o.init_equilibrium(w.rho0, 0.0, 0.0)
        lat.step(n)
        o.step(n)
        errs[rnd] = field_errors(lat.moments(), o.moments())
    for k, b in SR_BOUNDS[store].items():
        assert errs["stochastic"][k] < b, (k, errs["stochastic"])
    assert errs["stochastic"]["u"] < 0.1 * errs["nearest"]["u"], errs


# ------------------------------------------------- full-size launch shapes

def test_poiseuille_full_size_columns_match_oracle():
    """1024 x 512 force-driven channel in FP32: the flow is x-invariant, so every one
    of the 1024 GPU columns must match the oracle's 4-column run."""
    import oracle
    import paper_1007_4895_gb300 as lb
    w = poiseuille(nx=1024, ny=512, rows=32, kn=0.1)
    steps = 300
    big = lb.Lattice.from_workload(w, store="f32_dev")
    eff = big.effective_map()
    big.step(steps)
    g = big.moments()
    o = oracle.Oracle(4, 512, eff[:, :4], kn_ref=0.1, gx=w.gx, walls=w.walls, dt=big.dt, h=big.h)
    o.init_equilibrium(1.0, 0.0, 0.0)
    o.step(steps)
    r = o.moments()
    scale = np.abs(r["ux"]).max()
    err = np.abs(g["ux"] - r["ux"][:, :1]).max() / scale
    assert err < F32_VEL_TOL, err


@pytest.mark.parametrize("variant", LAYOUTS)
def test_long_channel_every_layout_matches_oracle(variant):
    """Pressure channel with x-varying bands (several row-blocks, ragged last block,
    x-interfaces, pressure columns): every layout against the oracle."""
    w = long_channel(nx=700, ny=45, steps=60)
    lat, o, eff, got, ref = run_both(w, "f32_dev", w.steps, variant=variant)
    errs = field_errors(got, ref)
    assert errs["u"] < F32_VEL_TOL and errs["rho"] < F32_VEL_TOL, errs


@pytest.mark.parametrize("store", ["f64", "f32_dev", "bf16_dev", "bf16_dev_sr", "f16_dev_sr"])
@pytest.mark.parametrize("variant", [2, 3, 4, 5, 6])
def test_register_block_layouts_equal_quad_layout(store, variant):
    """The split and streamed layouts do the quad layout's arithmetic in the same order,
    and draw the same random bits when rounding stochastically, so their populations
    agree with it bit for bit (walls, force, periodic edges, a ragged tile and interface
    tiles)."""
    import paper_1007_4895_gb300 as lb
    rnd = "stochastic" if store.endswith("_sr") else "nearest"
    st = store.replace("_sr", "")

    def build(v):
        w = ragged_workload()
        lat = lb.Lattice.from_workload(w, store=st, variant=v, rounding=rnd)
        return lat, None, None

    a, _, _ = build(0)
    b, _, _ = build(variant)
    a.step(40)
    b.step(40)
    for s in (0, 1):
        assert np.array_equal(a.populations(s), b.populations(s)), (store, variant, s)


@pytest.mark.parametrize("variant", [7, 8, 9, 10])
@pytest.mark.parametrize("store", ["f32_dev", "f32", "f16_dev", "bf16_dev_sr", "f16_dev_sr"])
@pytest.mark.parametrize("case", ["ragged", "pressure_channel", "bands_paper", "periodic_box"])
def test_paired_layout_agrees_with_quad_layout(store, case, variant):
    """Layouts 7 to 10 fold the collision into per-node coefficients, compute node pairs
    with packed FP32 instructions and are built with multiply-add contraction, so they
    round differently from layout 0; the update is the same (stencil, walls, shadows,
    ghost copies, pressure columns, random bits). After 40 steps the two agree to
    rounding: FP32 within 1e-6 of the velocity scale (deviations; 1e-5 for f itself),
    16-bit within a few units of the stored format's last place (a rounding decision can
    fall the other way)."""
    import paper_1007_4895_gb300 as lb
    rnd = "stochastic" if store.endswith("_sr") else "nearest"
    st = store.replace("_sr", "")
    if case == "ragged":
        w = ragged_workload()
    elif case == "pressure_channel":
        w = long_channel(nx=300, ny=37)
    elif case == "bands_paper":
        w = couette(nx=200, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, iface="paper")
    else:
        w = Workload(name="box", nx=260, ny=22, region_map=band_map(260, 22, 3, 0), kn_ref=0.05, gx=1e-3,
                     walls={"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}},
                     init=ragged_workload(nx=260, ny=22).init)
    a = lb.Lattice.from_workload(w, store=st, variant=0, rounding=rnd)
    b = lb.Lattice.from_workload(w, store=st, variant=variant, rounding=rnd)
    if variant == 8 and b.info()["variant"] != 8:
        pytest.skip("this map has no block order other than the raster order")
    assert b.info()["variant"] == variant
    a.step(40)
    b.step(40)
    errs = field_errors(b.moments(), a.moments())
    tol = {"f32_dev": 1e-6, "f32": 1e-5, "bf16_dev": 3e-2, "f16_dev": 4e-3}[st]
    assert errs["u"] < tol and errs["rho"] < tol, (store, case, errs)


@pytest.mark.parametrize("store", ["f32_dev", "f32", "f16_dev", "bf16_dev", "f32_dev_col", "f16_dev_sr"])
@pytest.mark.parametrize("case", ["ragged", "pressure_channel", "bands_paper", "periodic_box", "sets_9_16"])
def test_row_unit_layout_equals_ring_layout(store, case):
    """Layout 10 runs layout 9's arithmetic on rows without boundary work from bodies
    specialised on the velocity set, and layout 9's own body on the other rows, in a
    persistent kernel that takes row units from a counter: the same bits as layout 9
    after an odd and an even number of steps (a unit done twice, skipped, or run with a
    population's sign pattern wrong would show)."""
    import paper_1007_4895_gb300 as lb
    rnd = "stochastic" if store.endswith("_sr") else "nearest"
    st = store.replace("_sr", "").replace("_col", "")
    if case == "ragged":
        w = ragged_workload()
    elif case == "pressure_channel":
        w = long_channel(nx=300, ny=37)
    elif case == "bands_paper":
        w = couette(nx=200, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, iface="paper")
    elif case == "sets_9_16":
        w = long_channel(nx=520, ny=40, sets=(9, 16))
    else:
        w = Workload(name="box", nx=260, ny=22, region_map=band_map(260, 22, 3, 0), kn_ref=0.05, gx=1e-3,
                     walls={"bottom": {"kind": "periodic"}, "top": {"kind": "periodic"}},
                     init=ragged_workload(nx=260, ny=22).init)
    kw = {}
    if store.endswith("_col"):
        kw["rho0_col"] = long_channel_density(w.nx, 2.0, 1.0) if case in ("pressure_channel", "sets_9_16") \
            else np.full(w.nx, w.rho0)
    a = lb.Lattice.from_workload(w, store=st, variant=9, rounding=rnd, **kw)
    b = lb.Lattice.from_workload(w, store=st, variant=10, rounding=rnd, **kw)
    assert a.info()["variant"] == 9 and b.info()["variant"] == 10
    for n in (7, 8):
        a.step(n)
        b.step(n)
        for s in (0, 1):
            assert np.array_equal(a.populations(s), b.populations(s)), (store, case, n, s)


@pytest.mark.parametrize("store", ["f32_dev", "f32", "f16_dev"])
def test_streamed_layout_equals_quad_layout_on_pressure_channel(store):
    """Layout 4 (carried moments, TMA plane tiles, boundary post-passes) on a channel with
    pressure columns, diffuse walls, x-varying bands and ragged units: the same bits as
    layout 0 after an odd and an even number of steps, carried moments included (a
    wrong carried sum changes the next step's collision)."""
    w = long_channel(nx=300, ny=37)
    a, _, _ = make_pair(w, store=store, variant=0)
    b, _, _ = make_pair(long_channel(nx=300, ny=37), store=store, variant=4)
    assert b.info()["variant"] == 4
    for n in (7, 24):
        a.step(n)
        b.step(n)
        for s in (0, 1):
            assert np.array_equal(a.populations(s), b.populations(s)), (store, n, s)


def test_long_channel_full_size_fp32():
    """16384 x 128 pressure-driven channel with the Kn-threshold map, FP32 deviations,
    a few steps against the oracle at full size."""
    w = long_channel(nx=16384, ny=128, steps=6)
    lat, o, eff, got, ref = run_both(w, "f32_dev", w.steps)
    errs = field_errors(got, ref)
    # deviations of size |rho - rho0| ~ 0.5 (global rho0 = 1.5, densities 1..2) carry
    # FP32 rounding of ~3e-8 into a velocity of ~0.04
    assert errs["u"] < 3 * F32_VEL_TOL, errs
    assert errs["rho"] < F32_VEL_TOL, errs


# ------------------------------------------------------------ API behaviour

def test_reductions_mass_and_residual():
    w = couette(nx=40, ny=24, rows=3, kn=0.1)
    lat, o, eff = make_pair(w, store="f64")
    r0 = lat.reductions()
    lat.step(50)
    o.step(50)
    r1 = lat.reductions()
    m = o.moments()
    np.testing.assert_allclose(r1["mass"], m["rho"].sum(), rtol=1e-12)
    # started from rest: both first residuals compare with u = 0
    assert r0["residual"] == 1.0 and r1["residual"] == 1.0
    lat.step(50)
    r2 = lat.reductions()
    assert 0 < r2["residual"] < 1.0
    assert r2["nonfinite"] == 0 and r2["step"] == 100


def test_nan_is_reported_as_divergence():
    import paper_1007_4895_gb300 as lb
    w = couette(nx=32, ny=16, rows=3, kn=0.1)
    lat = lb.Lattice.from_workload(w, store="f32")
    f = lat.populations(0)
    f[4, 8, 5] = np.nan
    lat.set_populations(0, f)
    with pytest.raises(lb.LBError) as e:
        lat.reductions()
    assert e.value.code == lb.LB_ERR_DIVERGED
    with pytest.raises(lb.LBError):
        lat.step(1)     # sticky


def test_checkpoint_resume_is_bit_identical(tmp_path):
    w = ragged_workload()
    import paper_1007_4895_gb300 as lb
    a = lb.Lattice.from_workload(w, store="f32")
    a.step(20)
    a.save(str(tmp_path / "ck.bin"))
    a.step(15)
    ref = a.moments()
    b = lb.Lattice.from_workload(w, store="f32")
    b.load(str(tmp_path / "ck.bin"))
    assert b.info()["step"] == 20
    b.step(15)
    got = b.moments()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("case", ["ragged_hermite", "bands_paper", "pressure_channel"])
@pytest.mark.parametrize("store", ["f32_dev", "bf16_dev"])
def test_compact_state_round_trip_is_bit_identical(case, store):
    """lb_state_store / lb_state_load carry only each node's own-set populations; the load
    rebuilds ghost copies, shadows, interface rows and pressure columns. A lattice that
    holds a different state and then loads the state of another steps to the same bits
    as that other one (own-set populations and moments): mixed map with mode-B shadows,
    walls, force and a ragged tile; mode-A interface rows; pressure columns."""
    import paper_1007_4895_gb300 as lb
    if case == "pressure_channel":
        w = long_channel(nx=300, ny=37)
    elif case == "bands_paper":   # mode A: band map, ragged last tile
        w = couette(nx=200, ny=32, rows=4, kn=0.1, u_wall_lat=0.05, iface="paper")
    else:
        w = ragged_workload()
    a = lb.Lattice.from_workload(w, store=store)
    a.step(17)
    n = a.state_bytes()
    q = np.where(a.effective_map() == 1, a.sets[1], a.sets[0])
    esize = 4 if store == "f32_dev" else 2
    ntile_rows = (w.nx + 127) // 128 * w.ny
    assert n <= int(q.max()) * ntile_rows * 128 * esize
    buf = np.zeros(n, np.uint8)
    lb.lb_state_store(a.ctx, buf.ctypes.data, n)
    b = lb.Lattice.from_workload(w, store=store)
    b.step(5)
    lb.lb_state_load(b.ctx, buf.ctypes.data, n)
    a.step(9)
    b.step(9)
    own = a.effective_map()
    for s in (0, 1):
        pa, pb = a.populations(s), b.populations(s)
        m = own == s
        assert np.array_equal(pa[:, m], pb[:, m]), (case, store, s)
    ma, mb = a.moments(), b.moments()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), (case, store, k)


def test_remap_rebuilds_moved_tiles():
    """Nodes that change set keep density and velocity (second-order rebuild)."""
    import oracle
    w = couette(nx=64, ny=32, rows=4, kn=0.1)
    lat, o, eff = make_pair(w, store="f64")
    lat.step(200)
    before = lat.moments()
    m = band_map(64, 32, 8)
    lat.set_region_map(m)
    after = lat.moments()
    np.testing.assert_allclose(after["rho"], before["rho"], rtol=1e-13)
    np.testing.assert_allclose(after["ux"], before["ux"], rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(after["pxy"], before["pxy"], rtol=1e-10, atol=1e-14)
    assert (lat.effective_map() == m).all()
    # the rebuilt nodes equal the oracle's Hermite projection of the old nodes
    # (row 5 is three rows from the new interface, so its low-order planes still hold
    # the state it had before the move)
    old_low = lat.populations(0)[:, 5, 3]
    got = lat.populations(1)[:, 5, 3]
    np.testing.assert_allclose(got, oracle.project(3, old_low, 6), rtol=1e-12, atol=1e-15)


def test_moments_into_device_tensor_match_host():
    import torch
    import paper_1007_4895_gb300 as lb
    w = ragged_workload()
    lat = lb.Lattice.from_workload(w, store="f32")
    lat.step(10)
    host = lat.moments(f64=False)
    t = torch.empty((9, w.ny, w.nx), device="cuda", dtype=torch.float32)
    lat.moments_into(t)
    torch.cuda.synchronize()
    dev = t.cpu().numpy()
    for k, name in enumerate(lb.MOMENT_NAMES):
        assert np.array_equal(dev[k], host[name])
