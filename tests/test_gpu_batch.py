"""Batched channels (lb_batch_*): many independent lattices advanced by one persistent
launch. In FP64 the batch does the one-quad layout's arithmetic, in FP32 and 16-bit
storage layout 10's bodies (the bits of layout 9), so every lattice must equal the same
lattice stepped on its own with that layout, bit for bit; a few lattices are also
checked against the FP64 oracle, and the full 512-channel sweep against the oracle on
sampled channels."""
import numpy as np
import pytest

from lbinputs import batched_instances

pytestmark = pytest.mark.gpu


def _pops(lat):
    return [lat.populations(s) for s in (0, 1)]


@pytest.mark.parametrize("store", ["f64", "f32_dev", "bf16_dev"])
def test_batch_equals_lattices_stepped_alone(store):
    import paper_1007_4895_gb300 as lb
    ws = batched_instances(n=24, seed=7)
    b = lb.Batch(ws, store=store)
    b.step(31)
    for i in (0, 5, 11, 23):
        alone = lb.Lattice.from_workload(batched_instances(n=24, seed=7)[i], store=store,
                                         variant=0 if store == "f64" else 9)
        alone.step(31)
        got, ref = _pops(b.lattice(i)), _pops(alone)
        for s in (0, 1):
            assert np.array_equal(got[s], ref[s]), (store, i, s)
        assert b.lattice(i).info()["step"] == 31


def test_per_lattice_launches_and_graph_replays_equal_batch_steps():
    import paper_1007_4895_gb300 as lb
    a = lb.Batch(batched_instances(n=40, seed=3), store="f32_dev")
    c = lb.Batch(batched_instances(n=40, seed=3), store="f32_dev")
    d = lb.Batch(batched_instances(n=40, seed=3), store="f32_dev")
    a.step(7)
    a.step(13)       # odd counts: the current level alternates
    c.step_each(20)
    d.graph(10, replays=2)
    for i in range(0, 40, 7):
        ra = _pops(a.lattice(i))
        for other in (c, d):
            ro = _pops(other.lattice(i))
            for s in (0, 1):
                assert np.array_equal(ra[s], ro[s]), i


@pytest.mark.parametrize("store", ["f32_dev", "bf16_dev"])
def test_per_lattice_steps_after_a_batch_launch_read_its_ghost_columns(store):
    """Inside a launch of several steps the batch reads the halos of an x-periodic
    lattice's end quads from the other end of the row and writes the periodic
    ghost-column images only at the launch's last step. Per-lattice launches read the
    ghost columns, so batch launches followed by per-lattice steps must give the bits of
    per-lattice steps throughout."""
    import paper_1007_4895_gb300 as lb
    a = lb.Batch(batched_instances(n=16, seed=5), store=store)
    c = lb.Batch(batched_instances(n=16, seed=5), store=store)
    a.step(9)
    a.step_each(3)
    a.step(5)
    c.step_each(17)
    for i in range(16):
        ra, rc = _pops(a.lattice(i)), _pops(c.lattice(i))
        for s in (0, 1):
            assert np.array_equal(ra[s], rc[s]), (store, i, s)


def test_stepping_one_lattice_alone_is_refused():
    import paper_1007_4895_gb300 as lb
    b = lb.Batch(batched_instances(n=4, seed=1), store="f32_dev")
    b.lattice(2).step(1)
    with pytest.raises(lb.LBError) as e:
        b.step(1)
    assert e.value.code == lb.LB_ERR_INVALID


def test_batch_matches_oracle():
    import paper_1007_4895_gb300 as lb
    import oracle
    from gpu_pair import N1D, field_errors
    ws = [w for w in batched_instances(n=40, seed=11) if w.ny <= 64][:3]
    assert len(ws) == 3
    b = lb.Batch(ws, store="f64")
    b.step(200)
    for i, w in enumerate(ws):
        lat = b.lattice(i)
        o = oracle.Oracle(w.nx, w.ny, lat.effective_map(), n1d_lo=N1D[w.sets[0]], n1d_hi=N1D[w.sets[1]],
                          kn_ref=w.kn_ref, rho_ref=w.rho_ref, tau_mode=w.tau_mode, gx=w.gx, gy=w.gy,
                          iface=w.iface, walls=w.walls, dt=lat.dt, h=lat.h)
        o.init_equilibrium(w.rho0, 0.0, 0.0)
        o.step(200)
        e = field_errors(lat.moments(), o.moments())
        assert e["u"] < 1e-10 and e["rho"] < 1e-12, (i, e)


def test_full_sweep_of_512_channels():
    """All 512 seeded channels, 5000 steps each in graph-captured persistent launches:
    every field finite, and three sampled channels (smallest, largest, a middle one)
    against the FP64 oracle. (Total mass is not an invariant here: the diffuse wall
    zeroes the normal mass flux at the wall node, not the ghost-node exchange.)
    Tolerance: FP32 storage rounds each stored deviation by up to 2^-24 relative per
    step; over N = 5000 steps these errors add like a random walk, sqrt(N) 2^-24 = 4.2e-6
    of the velocity scale, so e_u < 5e-6."""
    import paper_1007_4895_gb300 as lb
    import oracle
    from gpu_pair import N1D, field_errors
    ws = batched_instances()
    assert len(ws) == 512
    b = lb.Batch(ws, store="f32_dev")
    b.graph(1000, replays=5)
    b.sync()
    for i in range(512):
        m = b.lattice(i).moments(mask=0b111)
        assert np.isfinite(m["rho"]).all() and np.isfinite(m["ux"]).all(), i
    ny = np.array([w.ny for w in ws])
    for i in (int(ny.argmin()), int(ny.argmax()), int(np.argsort(ny)[256])):
        w, lat = ws[i], b.lattice(i)
        o = oracle.Oracle(w.nx, w.ny, lat.effective_map(), n1d_lo=N1D[w.sets[0]], n1d_hi=N1D[w.sets[1]],
                          kn_ref=w.kn_ref, rho_ref=w.rho_ref, tau_mode=w.tau_mode, gx=w.gx, gy=w.gy,
                          iface=w.iface, walls=w.walls, dt=lat.dt, h=lat.h)
        o.init_equilibrium(w.rho0, 0.0, 0.0)
        o.step(5000)
        e = field_errors(lat.moments(), o.moments())
        assert e["u"] < 5e-6 and e["rho"] < 1e-6, (i, w.ny, e)
