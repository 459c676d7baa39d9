"""The learned-placement pipeline of the benchmark (features and labels from an
all-high-order run, wall-stratified samples, training on the GPU, a run whose map the
network updates), on a shorter channel: the network learns its labels, inference and
map updates run without fallback, and every map's figures are well defined."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_config5_pipeline_on_a_shorter_channel():
    import torch

    import paper_1007_4895_gb300 as lb
    sys.path.insert(0, ROOT)
    import bench
    r = bench.config5_study(lb, torch, nx=1024, ny=128, steps=600, every=100, samples=20000, epochs=10)
    print(r)
    assert r["train"]["loss"] < r["train"]["loss0"]
    assert r["train"]["accuracy"] > 0.9
    maps = r["maps"]
    assert maps["all_high"]["phi_H"] == 1.0 and maps["all_high"]["e_u_vs_all_high"] == 0.0
    assert 0.0 < maps["fixed"]["phi_H"] < 1.0
    assert maps["learned"]["fallbacks"] == 0 and maps["learned"]["map_updates"] >= 6
    for m in maps.values():
        assert np.isfinite(m["e_u_vs_all_high"]) and m["MLUPS"] > 0
    assert r["infer_ms_whole_lattice"] > 0 and maps["learned"]["map_update_ms"] > 0
