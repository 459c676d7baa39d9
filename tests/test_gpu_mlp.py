"""Learned interface placement on the CUDA path, against the FP64 oracles
(oracle/mlp.py for the network, oracle/placement.py for its inputs and labels).

The network's forward, backward, weight-gradient and Adam kernels train in FP32, so
their results are compared with the FP64 oracle within FP32 accumulation error; the
inference kernel runs on the tensor cores with BF16 weights and BF16 layer inputs, and is
compared with the oracle's forward pass on the same BF16-rounded operands."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _data(n, seed):
    """Raw features with uneven scales and offsets, labels from a nonlinear rule."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((8, n)) * np.array([1e-3, 5e-4, 1e-3, 2e-4, 2e-4, 0.2, 0.1, 0.05])[:, None]
    x += np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.25, 0.2, 0.0])[:, None]
    y = ((x[1] / 5e-4) ** 2 + 0.5 * (x[6] - 0.2) / 0.1 > 0.8).astype(np.float64)
    mean = x.mean(axis=1)
    scale = x.std(axis=1)
    return x, y, np.concatenate([mean, scale])


def _norm(x, nm):
    """Normalisation in the precision the kernels use (FP32), then widened."""
    xf = x.astype(np.float32)
    m = nm[:8].astype(np.float32)[:, None]
    s = nm[8:].astype(np.float32)[:, None]
    return ((xf - m) / s).astype(np.float64).T


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _mlp(theta, nm):
    import paper_1007_4895_gb300 as lb
    return lb.MLP(theta.astype(np.float32), nm.astype(np.float32))


@pytest.mark.parametrize("n", [1, 127, 4099])
def test_grad_matches_oracle(n):
    x, y, nm = _data(n, 3)
    if n == 1:
        nm[8:] = 1.0
    theta = omlp.init_params(1007).astype(np.float32).astype(np.float64)
    m = _mlp(theta, nm)
    g, loss = m.grad(_dev(x), _dev(y))
    xn = _norm(x, nm)
    g_ref = omlp.grad(theta, xn, y)
    l_ref = omlp.loss(theta, xn, y)
    assert abs(loss - l_ref) <= 1e-5 * max(1.0, abs(l_ref))
    # FP32 sums over n samples in sample order: well inside 1e-4 of the largest component;
    # a wrong index, sign or factor anywhere moves some component by O(1) of it
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-4 * scale, np.abs(g - g_ref).max() / scale


def test_adam_steps_match_oracle():
    n = 2048
    x, y, nm = _data(n, 4)
    theta = omlp.init_params(7).astype(np.float32).astype(np.float64)
    m = _mlp(theta, nm)
    xd, yd = _dev(x), _dev(y)
    xn = _norm(x, nm)
    th, mo, vo = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    lr = 1e-3
    for t in range(1, 4):
        g_ref = omlp.grad(th, xn, y)
        th, mo, vo = omlp.adam_step(th, mo, vo, g_ref, t, lr=lr)
        m.adam_step(xd, yd, lr=lr)
    got = m.params().astype(np.float64)
    d_got, d_ref = got - theta, th - theta      # the three steps' total move (about 3 lr)
    # components whose gradient is well above FP32 rounding move as the oracle's do, to
    # a small fraction of one step; the rest can take the other sign in an early step,
    # a move of at most 2 lr per step
    g0 = np.abs(omlp.grad(theta, xn, y))
    big = g0 > 1e-2 * g0.max()
    assert big.sum() > 200
    assert np.abs(d_got - d_ref)[big].max() <= 2e-6
    assert np.abs(d_got - d_ref).max() <= 2 * lr * 3 + 1e-6


def test_bf16_inference_matches_oracle_on_rounded_operands():
    """Tensor-core inference (BF16 weights and layer inputs, FP32 accumulation) against
    the oracle's forward pass with the same operands rounded to BF16 and everything else
    in FP64. A hidden activation whose FP32 and FP64 values straddle a BF16 rounding
    boundary rounds the other way (one BF16 unit, 2^-8 relative) in a few of the 5000 x
    64 of them: the bound is on the mean and, with room for those, on the maximum."""
    n = 5000
    x, y, nm = _data(n, 5)
    theta = omlp.init_params(9).astype(np.float32).astype(np.float64)
    m = _mlp(theta, nm)
    import torch
    out = torch.empty(n, device="cuda", dtype=torch.float32)
    m.infer(_dev(x), out)
    p = out.cpu().numpy().astype(np.float64)
    xn = _norm(x, nm)
    p_ref = omlp.forward_bf16_operands(theta, xn)
    p_fp32, _ = omlp.forward(theta, xn)
    d = np.abs(p - p_ref)
    assert d.mean() < 2e-5 and d.max() < 2e-3, (d.mean(), d.max())
    # the rounding is really applied: full-precision operands give a visibly different p
    assert np.abs(p - p_fp32).max() > 1e-4


def test_inference_on_ragged_counts():
    """Node counts that end inside a 16-node tile and inside a warp's share."""
    import torch
    theta = omlp.init_params(4).astype(np.float32).astype(np.float64)
    _, _, nm = _data(5000, 11)   # normalisation from a large sample
    m = _mlp(theta, nm)
    for n in (1, 15, 17, 1000, 4099):
        x, y, _ = _data(n, 12 + n)
        out = torch.full((n + 5,), 7.0, device="cuda", dtype=torch.float32)
        m.infer(_dev(x), out[:n])
        got = out.cpu().numpy()
        ref = omlp.forward_bf16_operands(theta, _norm(x, nm))
        assert np.abs(got[:n] - ref).max() < 2e-3, n
        assert np.all(got[n:] == 7.0), n   # nothing written past the end


def test_inference_marks_nonfinite_inputs():
    x, y, nm = _data(300, 6)
    x[3, 17] = np.nan
    x[0, 200] = np.inf
    m = _mlp(omlp.init_params(1), nm)
    import torch
    out = torch.empty(300, device="cuda", dtype=torch.float32)
    m.infer(_dev(x), out)
    p = out.cpu().numpy()
    assert np.isnan(p[17]) and np.isnan(p[200])
    assert np.isfinite(np.delete(p, [17, 200])).all()


def test_training_lowers_loss_and_classifies():
    n = 20000
    x, y, nm = _data(n, 8)
    theta = omlp.init_params(1007)
    m = _mlp(theta, nm)
    xn = _norm(x, nm)
    l0 = omlp.loss(theta, xn, y)
    last = m.train(_dev(x), _dev(y), epochs=8, batch=256, lr=1e-3, seed=1007)
    th = m.params().astype(np.float64)
    l1 = omlp.loss(th, xn, y)
    assert abs(last - l1) < 0.05          # the reported epoch loss is a running mean
    assert l1 < 0.3 * l0
    p, _ = omlp.forward(omlp.round_bf16(th), xn)
    assert ((p > 0.5) == (y > 0.5)).mean() > 0.97


# ------------------------------------------------------- features and labels

def _lattice_from_oracle(store="f64"):
    """A pressure-driven channel advanced by the oracle, then loaded into a lattice."""
    from gpu_pair import make_pair
    from lbinputs import long_channel
    w = long_channel(nx=300, ny=26, cfl=0.38)
    lat, o, eff = make_pair(w, store=store)
    o.step(150)
    for s in (0, 1):
        lat.set_populations(s, o.populations(s))
    return w, lat, o, eff


def test_features_match_oracle():
    import torch
    from oracle import placement
    w, lat, o, eff = _lattice_from_oracle()
    t = torch.empty((8, w.ny, w.nx), device="cuda", dtype=torch.float32)
    lat.features_into(t)
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.float64)
    ref = placement.features(o.moments(), lat.h, w.kn_ref, w.rho_ref, periodic_x=False, periodic_y=False,
                             wall_bottom=True, wall_top=True)
    for k in range(8):
        scale = np.abs(ref[k]).max()
        err = np.abs(got[k] - ref[k]).max() / scale
        assert err < 1e-4, (placement.FEATURE_NAMES[k], err)


def test_hermite_residual_matches_oracle():
    import torch
    from gpu_pair import N1D
    from oracle import placement
    w, lat, o, eff = _lattice_from_oracle()
    t = torch.empty((w.ny, w.nx), device="cuda", dtype=torch.float32)
    lat.hermite_residual_into(t)
    torch.cuda.synchronize()
    got = t.cpu().numpy().astype(np.float64)
    cols = np.r_[0:3, 140:146, w.nx - 3:w.nx]
    pops = (o.populations(0)[:, :, cols], o.populations(1)[:, :, cols])
    ref = placement.hermite_residual(pops, eff[:, cols], (N1D[w.sets[0]], N1D[w.sets[1]]))
    assert ref.max() > 1e-5        # the wall layers hold beyond-second-order parts
    assert np.abs(got[:, cols] - ref).max() < 1e-5 * ref.max()


# ------------------------------------------------------------- learned map

def _const_net(b3):
    """A network whose output is sigmoid(b3) at every node."""
    theta = np.zeros(omlp.NPARAM)
    theta[-1] = b3
    return theta


def test_learned_map_limits_and_fallback():
    import paper_1007_4895_gb300 as lb
    from lbinputs import long_channel
    w = long_channel(nx=400, ny=24, cfl=0.38)
    lat = lb.Lattice.from_workload(w, store="f32_dev")
    nm = np.concatenate([np.zeros(8), np.ones(8)])
    ny = w.ny
    # p = sigmoid(-20): only the two rows next to each wall stay high-order
    low = lb.MLP(_const_net(-20.0), nm)
    lat.set_mlp(low, every=10)
    lat.step(10)
    eff = lat.effective_map()
    assert eff[:2].all() and eff[-2:].all() and not eff[2:ny - 2].any()
    st = lat.map_stats()
    assert (st["updates"], st["fallbacks"]) == (1, 0) and abs(st["high_fraction"] - 4.0 / ny) < 1e-12
    # p = sigmoid(20): everything high-order
    high = lb.MLP(_const_net(20.0), nm)
    lat.set_mlp(high, every=10)
    lat.learned_map_now()
    assert lat.effective_map().all()
    # non-finite p keeps the map and counts a fallback
    bad = lb.MLP(_const_net(np.nan), nm)
    lat.set_mlp(bad, every=10)
    lat.learned_map_now()
    assert lat.effective_map().all()
    st = lat.map_stats()
    assert st["fallbacks"] == 1 and st["high_fraction"] == 1.0
    lat.set_mlp(None)
    lat.step(5)
    m = lat.moments(mask=0b111)
    assert np.isfinite(m["rho"]).all()


def test_learned_remap_matches_oracle_rebuild():
    """After a learned update moves tiles, the lattice equals an oracle lattice whose
    moved nodes were rebuilt by the oracle's Hermite projection (Eq. (approxf), N = 2)."""
    import paper_1007_4895_gb300 as lb
    import oracle
    from gpu_pair import N1D, field_errors
    from lbinputs import long_channel
    w = long_channel(nx=260, ny=24, cfl=0.38)
    w.region_map = np.ones((w.ny, w.nx), np.uint8)
    from gpu_pair import make_pair
    lat, o, eff = make_pair(w, store="f64")
    lat.step(40)
    o.step(40)
    low = lb.MLP(_const_net(-20.0), np.concatenate([np.zeros(8), np.ones(8)]))
    lat.set_mlp(low, every=1000)
    lat.learned_map_now()
    new = lat.effective_map()
    # rebuild the oracle's moved nodes (high -> low) by projection, then step both
    f_hi = o.populations(1)
    f_lo = o.populations(0)
    moved = (eff == 1) & (new == 0)
    for j, i in zip(*np.nonzero(moved)):
        f_lo[:, j, i] = oracle.project(N1D[w.sets[1]], f_hi[:, j, i], N1D[w.sets[0]])
    o2 = oracle.Oracle(w.nx, w.ny, new, n1d_lo=N1D[w.sets[0]], n1d_hi=N1D[w.sets[1]], kn_ref=w.kn_ref,
                       rho_ref=w.rho_ref, tau_mode=w.tau_mode, iface=w.iface, walls=w.walls, dt=lat.dt, h=lat.h)
    o2.set_populations(0, f_lo)
    o2.set_populations(1, f_hi)
    lat.set_mlp(None)
    lat.step(30)
    o2.step(30)
    e = field_errors(lat.moments(), o2.moments())
    assert e["u"] < 1e-10 and e["rho"] < 1e-12, e
