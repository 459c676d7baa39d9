"""What the learned interface placement gains over the method without it.

Steady force-driven channels (8 x 64, resting diffuse walls) across Knudsen numbers.
The reference is the all-high-order (D2Q36) run; the method without the network is the
fixed partition of the Sec. 3.4 tests (low-order set in the middle 70 %), i.e. 15 % of
the rows next to each wall high-order.
The network is trained on GPU with the library's kernels, on nodes of the reference runs
and of two fixed-map runs per Kn (features as those maps show them), labelled by the
reference run's beyond-second-order residual e3 = ||f - P2 f|| / rho > 3e-4 at that node. It
then steers the map of runs that start from the fixed partition, including at Knudsen
numbers it never saw. Velocity errors are e_u = max |u - u_ref| / max |u_ref|. A gain is
counted only at a high-order fraction no larger than the fixed partition's, and the
learned map is also compared with the whole cost-accuracy curve of fixed band maps of
every thickness."""
import numpy as np
import pytest

from lbinputs import band_map, placement_channel, steady_steps

pytestmark = pytest.mark.gpu

NX, NY = 8, 64
TRAIN_KN = (0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0)
EVAL_KN = (0.01, 0.015, 0.03, 0.3)       # 0.015, 0.03 and 0.3 are not in the training set
FIXED_ROWS = round(0.15 * NY)
BAND_ROWS = (2, 4, 6, FIXED_ROWS, 16, 24)   # fixed band maps: high-order rows per wall
THRESHOLD = 3e-4


def _run(kn, region_map, steps=None, mlp=None, every=500):
    import paper_1007_4895_gb300 as lb
    lat = lb.Lattice.from_workload(placement_channel(kn, region_map, NX, NY), store="f32_dev")
    n = steps or steady_steps(kn, lat.dt)
    if mlp is not None:
        lat.set_mlp(mlp, every=every)
    lat.step(n)
    return lat, n


def _features(lat):
    import torch
    F = torch.empty((8, NY, NX), device="cuda")
    lat.features_into(F)
    torch.cuda.synchronize()
    return F.cpu().numpy().reshape(8, -1)


def _residual(lat):
    import torch
    R = torch.empty((NY, NX), device="cuda")
    lat.hermite_residual_into(R)
    torch.cuda.synchronize()
    return R.cpu().numpy().reshape(-1)


def _e_u(m, ref):
    du = np.sqrt((m["ux"] - ref["ux"]) ** 2 + (m["uy"] - ref["uy"]) ** 2)
    return float(du.max() / np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max())


@pytest.fixture(scope="module")
def study():
    import torch
    import paper_1007_4895_gb300 as lb
    from oracle import mlp as omlp
    allh = np.ones((NY, NX), np.uint8)
    full, X, E = {}, [], []
    for kn in TRAIN_KN:
        lat, n = _run(kn, allh)
        full[kn] = (lat.moments(mask=0b111), n)
        e3 = _residual(lat)
        X.append(_features(lat))
        E.append(e3)
        for rows in (2, FIXED_ROWS):
            other, _ = _run(kn, band_map(NX, NY, rows), steps=n)
            X.append(_features(other))
            E.append(e3)
    X, E = np.concatenate(X, 1), np.concatenate(E)
    Y = (E > THRESHOLD).astype(np.float32)
    norm = np.concatenate([X.mean(1), X.std(1) + 1e-12])
    net = lb.MLP(omlp.init_params(1007), norm)
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, device="cuda")
    loss0 = net.grad(xd, yd)[1]
    loss = net.train(xd, yd, epochs=100, batch=128, lr=1e-3, seed=1007)
    p = torch.empty(X.shape[1], device="cuda")
    net.infer(xd, p)
    acc = float(((p.cpu().numpy() > 0.5) == (Y > 0.5)).mean())
    for kn in EVAL_KN:
        if kn not in full:
            lat, n = _run(kn, allh)
            full[kn] = (lat.moments(mask=0b111), n)
    rows, bands = [], {}
    for kn in EVAL_KN:
        ref, n = full[kn]
        fixed, _ = _run(kn, band_map(NX, NY, FIXED_ROWS), steps=n)
        learned, _ = _run(kn, band_map(NX, NY, FIXED_ROWS), steps=n, mlp=net)
        st = learned.map_stats()
        rows.append((kn, _e_u(fixed.moments(mask=0b111), ref), 2.0 * FIXED_ROWS / NY,
                     _e_u(learned.moments(mask=0b111), ref), st["high_fraction"], st["fallbacks"]))
        # the cost-accuracy curve of the fixed band maps (high-order rows next to each wall)
        curve = []
        for t in BAND_ROWS:
            b, _ = _run(kn, band_map(NX, NY, t), steps=n)
            curve.append((2.0 * t / NY, _e_u(b.moments(mask=0b111), ref)))
        bands[kn] = curve
    for r in rows:
        print("Kn %-6g fixed e_u %.2e phi_H %.2f | learned e_u %.2e phi_H %.2f (fallbacks %d)" % r)
        print("   bands (phi_H, e_u):", " ".join("(%.2f, %.2e)" % c for c in bands[r[0]]))
    return {"loss0": loss0, "loss": loss, "acc": acc, "rows": rows, "bands": bands}


def test_network_learns_the_labels(study):
    assert study["loss"] < 0.1 * study["loss0"]
    assert study["acc"] > 0.98


def test_learned_map_is_cheaper_and_more_accurate_near_continuum(study):
    kn, e_fixed, phi_fixed, e_learned, phi_learned, _ = study["rows"][0]
    assert kn == 0.01
    assert phi_learned < 0.5 * phi_fixed
    assert e_learned < e_fixed


def test_learned_map_against_the_fixed_partition_at_no_greater_cost(study):
    """A win is a lower velocity error at a high-order fraction no larger than the fixed
    partition's. Report every case; near continuum the learned map must win."""
    rows = study["rows"]
    wins = [r for r in rows if r[3] < r[1] and r[4] <= r[2]]
    print("wins at no greater cost:", [r[0] for r in wins])
    assert any(r[0] == 0.01 for r in wins), rows
    assert all(r[5] == 0 for r in rows)


def test_learned_map_is_on_the_band_maps_cost_accuracy_front(study):
    """Pareto comparison with the fixed band maps of every thickness. On this grid the
    coupled error grows with the band thickness at small Kn (the two sets' numerical
    viscous fluxes differ, and the mismatch acts over more rows), so thin bands are the
    cheap and accurate maps there, and only the all-high-order map reaches the reference
    at large Kn. The learned map counts as on the front at a Kn when no band map of no
    greater high-order fraction is more accurate than it by more than a factor 1.5.
    Measured: on the front at Kn 0.01 (thin bands), 0.03 and 0.3 (all high-order);
    dominated at Kn 0.015, where it keeps 59 % of the rows high-order for e_u 2.4e-2 and
    a 4-row band gives 6.6e-3 at 12 %."""
    on_front = []
    for r in study["rows"]:
        kn, phi_l, e_l = r[0], r[4], r[3]
        cheaper = [e for phi, e in study["bands"][kn] if phi <= phi_l + 1e-9]
        if not cheaper or e_l <= 1.5 * min(cheaper) + 1e-5:
            on_front.append(kn)
    print("on the cost-accuracy front at Kn:", on_front)
    assert len(on_front) >= 3 and 0.01 in on_front, (on_front, study["rows"], study["bands"])
