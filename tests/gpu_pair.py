"""Runs one workload on the CUDA path (through the C ABI) and on the FP64 oracle with
the same effective map, grid spacing and time step, and measures their differences.
The two sides share only the workload description from ``lbinputs``."""
from __future__ import annotations

import numpy as np

import oracle

N1D = {9: 3, 16: 4, 36: 6}
FIELDS = ("rho", "ux", "uy", "pxy", "neq_xx", "neq_xy", "neq_yy", "qx", "qy")


def make_pair(w, store="f64", reduce_every=0, map_override=None, variant=-1):
    import paper_1007_4895_gb300 as lb
    if map_override is not None:
        w.region_map = map_override
    lat = lb.Lattice.from_workload(w, store=store, reduce_every=reduce_every, variant=variant)
    eff = lat.effective_map()
    o = oracle.Oracle(w.nx, w.ny, eff, n1d_lo=N1D[w.sets[0]], n1d_hi=N1D[w.sets[1]], kn_ref=w.kn_ref,
                      rho_ref=w.rho_ref, tau_mode=w.tau_mode, gx=w.gx, gy=w.gy, iface=w.iface, walls=w.walls,
                      dt=lat.dt, h=lat.h)
    if w.init is not None:
        o.init_equilibrium(*w.init)
    else:
        o.init_equilibrium(w.rho0, 0.0, 0.0)
    return lat, o, eff


def field_errors(got, ref):
    """Relative errors per field, each scaled by a magnitude of its own physical
    quantity: velocity components by max |u_ref| (vector norm), P_xy by max |P_xy|,
    the non-equilibrium components by the largest of them, heat-flux components by
    max |q_ref|, density by max rho."""
    umax = np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max()
    nmax = max(np.abs(ref[k]).max() for k in ("neq_xx", "neq_xy", "neq_yy"))
    qmax = np.sqrt(ref["qx"] ** 2 + ref["qy"] ** 2).max()
    rscale = np.abs(ref["rho"]).max()
    scale = {"rho": rscale, "ux": umax, "uy": umax, "pxy": np.abs(ref["pxy"]).max(), "neq_xx": nmax,
             "neq_xy": nmax, "neq_yy": nmax, "qx": qmax, "qy": qmax}
    out = {}
    for k in FIELDS:
        d = np.abs(got[k] - ref[k]).max()
        out[k] = float(d / scale[k]) if scale[k] > 0 else float(d)
    du2 = (got["ux"] - ref["ux"]) ** 2 + (got["uy"] - ref["uy"]) ** 2
    out["u"] = float(np.sqrt(du2).max() / umax)
    out["u_l2"] = float(np.sqrt(du2.sum() / (ref["ux"] ** 2 + ref["uy"] ** 2).sum()))
    return out


def population_error(lat, o, eff, rho0=1.0):
    """Max over both sets of max |d_gpu - d_oracle| / max |d_oracle| at the nodes of the
    set, with d = f / w_alpha - rho0 (the deviation from the rest state)."""
    errs = []
    for s in (0, 1):
        if not (eff == s).any():
            continue
        w = oracle.velocity_set(N1D[lat.sets[s]])[2][:, None, None]
        g = lat.populations(s) / w - rho0
        r = o.populations(s) / w - rho0
        mask = np.broadcast_to(eff == s, g.shape)
        scale = np.abs(r[mask]).max()
        errs.append(float(np.abs(g[mask] - r[mask]).max() / max(scale, 1e-300)))
    return max(errs)
