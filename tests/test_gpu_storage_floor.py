"""The error a storage format adds, computed by the FP64 oracle, bounds what the CUDA path
may show.

The oracle's storage model (tests/test_oracle_storage.py) rounds every stored population
after each update the way the GPU format does: FP32 deviations, FP16 / BF16 deviations
to nearest or stochastically, with the same keys for the random bits. Everything else
stays FP64. Its distance from the exact oracle, e_model, is the error of the format
itself: the accumulated rounding of the stored values over the flow's relaxation. The
CUDA path, which also computes in FP32, must stay within that floor: e_gpu <=
1.25 e_model + 2e-7 (the second term: FP32 arithmetic on the increments). For the
deterministic formats it must also follow the model itself closely (e_gpu_vs_model well
below e_model); stochastic rounding makes the two runs draw their bits at slightly
different values, so there only the sizes compare.

The tolerances are derived from the oracle, not from a GPU measurement; the FP32 target
of 1e-6 holds where the format's own floor is below it (the forced box, short runs) and
is replaced by that floor where it is not (the measured e_model is recorded beside each
case)."""
import numpy as np
import pytest

from lbinputs import couette, poiseuille

from gpu_pair import field_errors, make_pair

pytestmark = pytest.mark.gpu


def _floor(w, store, rounding, steps):
    import paper_1007_4895_gb300 as lb
    lat, exact, eff = make_pair(w, store=store)
    if rounding != "nearest":
        lat = lb.Lattice.from_workload(w, store=store, rounding=rounding)
    model, _, _ = None, None, None
    _, model, _ = make_pair(w, store="f64")
    mode = store + ("_sr" if rounding == "stochastic" else "")
    model.set_storage(mode, rho0=w.rho0)
    lat.step(steps)
    exact.step(steps)
    model.step(steps)
    ex = exact.moments()
    e_gpu = field_errors(lat.moments(), ex)["u"]
    e_model = field_errors(model.moments(), ex)["u"]
    e_gm = field_errors(lat.moments(), model.moments())["u"]
    return e_gpu, e_model, e_gm


CASES = {
    # Couette 4 x 32, Kn 0.1, walls -/+0.05 lattice (config 1), from rest
    "couette": (lambda: couette(nx=4, ny=32, rows=4, kn=0.1, u_wall_lat=0.05), 5000),
    # steady force-driven channel 4 x 64, Kn 0.1, 10 high-order rows per wall
    "poiseuille": (lambda: poiseuille(nx=4, ny=64, rows=10, kn=0.1, g_lat=1e-5), 6000),
}


@pytest.mark.parametrize("case", ["couette", "poiseuille"])
@pytest.mark.parametrize("store,rounding", [("f32_dev", "nearest"), ("f16_dev", "nearest"),
                                            ("f16_dev", "stochastic"), ("bf16_dev", "stochastic")])
def test_gpu_error_is_the_storage_floor(case, store, rounding):
    make, steps = CASES[case]
    e_gpu, e_model, e_gm = _floor(make(), store, rounding, steps)
    print(f"{case} {store} {rounding}: e_gpu {e_gpu:.3g}  e_model {e_model:.3g}  gpu-model {e_gm:.3g}")
    # stochastic rounding: the two runs draw different bits; their errors agree in size only
    factor = 1.25 if rounding == "nearest" else 2.0
    assert e_gpu <= factor * e_model + 2e-7, (e_gpu, e_model)
    if rounding == "nearest":
        assert e_gm < 0.5 * e_model + 2e-7, (e_gm, e_model)
