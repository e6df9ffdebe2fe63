"""Runs a few particle-mesh steps of one synthetic simulation, for profilers.

    python -m paper_1608_00802_gb300.profile_step --n-side 128 --n-mesh 256 --box 2 --steps 3

Prints per-stage device times from the library's CUDA-event profiler.  Meant
to be wrapped by ncu (e.g. ``ncu --set full -k regex:k_stencil -c 1``).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-side", type=int, default=128)
    ap.add_argument("--n-mesh", type=int, default=256)
    ap.add_argument("--box", type=float, default=2.0)
    ap.add_argument("--m22", type=float, default=2.5)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--start", type=int, default=0, help="steps run before the profiled ones")
    ap.add_argument("--nsteps", type=int, default=500, help="steps of the whole run (z = 100 -> 3)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--mode", choices=["meshgrad", "hybrid", "lagrangian"], default="hybrid")
    ap.add_argument("--rho-fp64", type=float, default=1e-2,
                    help="density below which Q is recomputed in extended precision (0: never)")
    ap.add_argument("--tuning", default=None, help="launch shapes as JSON (pm_tuning fields), e.g. "
                    "'{\"stencil_rows\": 8, \"stencil_planes\": 8, \"stencil_stages\": 4}'")
    ap.add_argument("--autotune", action="store_true", help="measure the launch shapes first")
    ap.add_argument("--kernel", choices=["cic", "spline"], default="cic", help="density kernel (spline: h = 3.5)")
    args = ap.parse_args()
    import numpy as np
    import torch

    from paper_1608_00802_gb300 import build, ics, pm
    build.build()
    modes = {"meshgrad": pm.FORCE_MESHGRAD, "hybrid": pm.FORCE_HYBRID, "lagrangian": pm.FORCE_LAGRANGIAN}
    a0, a1 = 1 / 101.0, 1 / 4.0
    x, p = ics.zeldovich(args.n_side, args.n_mesh, args.box, a0, 42, m22=args.m22)
    cfg = pm.make_config(len(x), args.n_mesh, args.box, m22=args.m22, force_mode=modes[args.mode],
                         precision=pm.FP64 if args.precision == "fp64" else pm.FP32, rho_fp64=args.rho_fp64,
                         kernel=pm.KERNEL_SPLINE if args.kernel == "spline" else pm.KERNEL_CIC, smooth_h=3.5)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    if args.tuning:
        sim.set_tuning(dict(sim.get_tuning(), **json.loads(args.tuning)))
    if args.autotune:
        sim.autotune()
    print(json.dumps({"tuning": sim.get_tuning()}))
    a = a0 * (a1 / a0) ** (np.arange(args.nsteps + 1) / args.nsteps)
    if args.start:
        sim.run(args.start, a[0], a[args.start])
    sim.profile_begin(64 * (args.steps + 1))
    sim.run(args.steps, a[args.start], a[args.start + args.steps])
    stages = sim.profile_end()
    torch.cuda.synchronize()
    print(json.dumps({k: {"ms": v[0], "launches": v[1]} for k, v in stages.items() if v[1]}))


if __name__ == "__main__":
    main()
