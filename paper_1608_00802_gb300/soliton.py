"""Static soliton test (Sec. II.B, Fig. 1 of the paper): particles drawn from
the Schroedinger-Poisson ground state, at rest, evolve under gravity and the
quantum pressure in a static box (a = 1).  The scheme should keep the total
energy K_v + W_g + K_rho to better than 1e-2 while the profile oscillates
about the ground state, energy passing back and forth between the gradient
energy K_rho and the gravitational energy W_g.

    python -m paper_1608_00802_gb300.soliton --n-part 1000000 --n-mesh 128 --r95 18.6 --h 4
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(n_part=1_000_000, n_mesh=128, r95_cells=18.6, h_cells=4.0, t_end_units=10.0, samples=40, cfl=0.25,
        precision=None, force_mode=None, m22=2.5, box=1.0, seed=0, max_steps_per_sample=100000,
        steps_per_sample=None):
    """Returns a dict of time series: t (also in units of the soliton's
    dynamical time alpha^2 m/hbar), the energies, the central density, and
    the steps taken.  Steps are adaptive (cfl), or, with steps_per_sample,
    equal (a fixed step keeps the leapfrog time-symmetric)."""
    from paper_1608_00802_gb300 import ics, pm
    precision = pm.FP32 if precision is None else precision
    force_mode = pm.FORCE_LAGRANGIAN if force_mode is None else force_mode
    probe = pm.make_config(8, 8, 1.0, m22=m22)
    hbm = float(pm.lib().pm_hbar_over_m(pm.C.byref(probe)))
    x, p, omega_m, info = ics.soliton_particles(n_part, box, n_mesh, r95_cells, hbm, seed=seed)
    cfg = pm.make_config(n_part, n_mesh, box, precision=precision, omega_m=omega_m, omega_l=0.0, m22=m22,
                         force_mode=force_mode, cosmological=False, kernel=pm.KERNEL_SPLINE, smooth_h=h_cells)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    t_unit = info["t_unit"]
    ts = np.linspace(0.0, t_end_units * t_unit, samples + 1)
    out = {"t": [], "K_v": [], "W_g": [], "K_rho": [], "rho_c": [], "steps": [], "info": info, "omega_m": omega_m}

    def record(t, steps):
        e = sim.energy(1.0)
        rho = sim.get_field(pm.FIELD_RHO)
        out["t"].append(t)
        out["K_v"].append(float(e[0]))
        out["W_g"].append(float(e[1]))
        out["K_rho"].append(float(e[2]))
        out["rho_c"].append(float(rho.max()))
        out["steps"].append(int(steps))

    record(0.0, 0)
    total = 0
    for k in range(samples):
        if steps_per_sample:
            sim.run(int(steps_per_sample), ts[k], ts[k + 1])
            total += int(steps_per_sample)
        else:
            b = sim.run_adaptive(ts[k], ts[k + 1], cfl=cfl, max_steps=max_steps_per_sample)
            total += len(b) - 1
        record(ts[k + 1], total)
    sim.close()
    for key in ("t", "K_v", "W_g", "K_rho", "rho_c"):
        out[key] = np.asarray(out[key])
    out["E"] = out["K_v"] + out["W_g"] + out["K_rho"]
    out["t_units"] = out["t"] / t_unit
    return out


def summary(out):
    e = out["E"]
    dk, dw = out["K_rho"] - out["K_rho"][0], out["W_g"] - out["W_g"][0]
    return {"max_rel_energy_error": float(np.max(np.abs(e - e[0])) / abs(e[0])),
            "K_rho_range_rel": float(np.ptp(out["K_rho"]) / abs(e[0])),
            "W_g_range_rel": float(np.ptp(out["W_g"]) / abs(e[0])),
            "corr_dK_rho_dW_g": float(np.corrcoef(dk[1:], dw[1:])[0, 1]) if len(dk) > 2 else None,
            "rho_c_range": [float(out["rho_c"].min() / out["rho_c"][0]), float(out["rho_c"].max() / out["rho_c"][0])],
            "steps": int(out["steps"][-1]), "t_end_units": float(out["t_units"][-1])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-part", type=int, default=1_000_000)
    ap.add_argument("--n-mesh", type=int, default=128)
    ap.add_argument("--r95", type=float, default=18.6, help="radius enclosing 95%% of the mass, in mesh cells")
    ap.add_argument("--h", type=float, default=4.0, help="spline smoothing length in mesh cells")
    ap.add_argument("--t-end", type=float, default=10.0, help="in units of alpha^2 m/hbar")
    ap.add_argument("--samples", type=int, default=40)
    ap.add_argument("--cfl", type=float, default=0.25)
    ap.add_argument("--steps-per-sample", type=int, default=None, help="equal steps instead of adaptive ones")
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    from paper_1608_00802_gb300 import build
    build.build()
    out = run(args.n_part, args.n_mesh, args.r95, args.h, args.t_end, args.samples, args.cfl,
              steps_per_sample=args.steps_per_sample)
    print(json.dumps(summary(out)))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in out.items()}, fh)


if __name__ == "__main__":
    main()
