"""Small driver for profiling the step kernel (e.g. under ncu).

    python -m paper_1007_4895_gb300.profile_step --workload long_channel --store f32_dev --variant 0 --steps 6
    python -m paper_1007_4895_gb300.profile_step --workload stream_box --store f32_dev --steps 6

Creates one lattice of the named synthetic workload, advances it ``--steps`` steps and
exits. ``--variant`` forces a step-kernel layout (see lb_opts.variant); by default the
library's autotuner chooses.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_1007_4895_gb300 as lb
    from lbinputs import config2, config3

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="long_channel", choices=["long_channel", "poiseuille", "stream_box"])
    ap.add_argument("--store", default="f32_dev")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--steps", type=int, default=6)
    a = ap.parse_args()
    if a.workload == "stream_box":
        # D2Q9 stream-and-collide scheme on a periodic 2048 x 1024 box
        import numpy as np
        periodic = {s: {"kind": "periodic"} for s in ("bottom", "top", "left", "right")}
        lat = lb.Lattice(2048, 1024, np.zeros((1024, 2048), np.uint8), kn_ref=0.002, rho_ref=1.0, walls=periodic,
                         store=a.store, scheme="stream")
        lat.step(a.steps)
        torch.cuda.synchronize()
        print("stream_box", a.store, lat.info())
        return
    w = config3() if a.workload == "long_channel" else config2(0.1)
    lat = lb.Lattice.from_workload(w, store=a.store, variant=a.variant)
    lat.step(a.steps)
    torch.cuda.synchronize()
    print(w.name, a.store, lat.info())


if __name__ == "__main__":
    main()
