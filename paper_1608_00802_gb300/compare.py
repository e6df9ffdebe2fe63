"""Dynamical effect of the quantum pressure: the same initial conditions run
with and without the Q force, compared through their power spectra and their
densities cell by cell (the FDM-versus-pressureless comparison of Sec. III,
Figs. 6-8 of the paper).

Both runs start from identical Zel'dovich particles drawn with the FDM
transfer function (Eq. transferhu), so every difference is the nonlinear
effect of the quantum pressure; ``cdm_ics=True`` draws the pressureless run's
initial conditions without that cut-off instead (same seed and white noise).
At each output redshift the result holds, per k shell, the mean |k|, both
P(k) and (P_FDM - P_CDM) / P_CDM, and the root-mean-square of
(rho_FDM - rho_CDM) / rho_CDM over the mesh cells where rho_CDM > 0 and over
those at or above the mean density (the ratio is dominated by near-empty cells
otherwise), next to
the quantum Jeans wavenumber k_J(a) = (6 Omega_m a)^(1/4) (m/hbar)^(1/2).

    python -m paper_1608_00802_gb300.compare --n-side 256 --n-mesh 512 --box 10 --m22 1 --nsteps 1000

The paper's runs smooth the density with its cubic spline (h = 3.5 dx); with
cloud-in-cell on a mesh of eight cells per particle the quantum pressure acts
on the particle shot noise instead (the CIC option is kept for comparison).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def jeans_k(a, m22, h=0.7, omega_m=0.3):
    """k_J in h/Mpc (code units: H0 = 1, lengths in Mpc/h)."""
    from paper_1608_00802_gb300 import pm
    cfg = pm.make_config(8, 8, 1.0, m22=m22, h=h, omega_m=omega_m)
    hbm = float(pm.lib().pm_hbar_over_m(pm.C.byref(cfg)))
    return (6.0 * omega_m * a) ** 0.25 / math.sqrt(hbm)


def run_pair(n_side, n_mesh, box, m22, z_start=100.0, z_end=3.0, nsteps=1000, z_out=(10.0, 5.0, 3.0), seed=42,
             cdm_ics=False, force_mode=None, precision=None, keep_density=False, stream=None, kernel=None,
             smooth_h=3.5):
    """Runs the FDM (quantum pressure on) and pressureless simulations side by
    side on the ln a-uniform schedule and returns a list of outputs, one per
    redshift in z_out (the schedule point nearest to it)."""
    from paper_1608_00802_gb300 import ics, pm
    force_mode = pm.FORCE_HYBRID if force_mode is None else force_mode
    precision = pm.FP32 if precision is None else precision
    kernel = pm.KERNEL_CIC if kernel is None else kernel
    a0, a1 = 1.0 / (1.0 + z_start), 1.0 / (1.0 + z_end)
    a = a0 * (a1 / a0) ** (np.arange(nsteps + 1) / nsteps)
    a[-1] = a1
    x, p = ics.zeldovich(n_side, n_mesh, box, a0, seed, m22=m22, fdm_ics=True)
    if cdm_ics:
        xc, pc = ics.zeldovich(n_side, n_mesh, box, a0, seed, m22=m22, fdm_ics=False)
    else:
        xc, pc = x, p
    n = n_side ** 3
    sims = {}
    for name, quantum, (xi, pi) in (("fdm", True, (x, p)), ("cdm", False, (xc, pc))):
        cfg = pm.make_config(n, n_mesh, box, m22=m22, precision=precision, force_mode=force_mode, quantum=quantum,
                             kernel=kernel, smooth_h=smooth_h)
        sims[name] = pm.Sim(cfg, stream=stream)
        sims[name].set_particles(xi, pi)
    steps = sorted({int(np.argmin(np.abs(1.0 / a - 1.0 - z))) for z in z_out})
    out = []
    done = 0
    for k in steps:
        if k > done:
            for s in sims.values():
                s.run(k - done, a[done], a[k])
            done = k
        kf, pf, cnt = sims["fdm"].power_spectrum()
        _, pcdm, _ = sims["cdm"].power_spectrum()
        rf = sims["fdm"].get_field(pm.FIELD_RHO)
        rc = sims["cdm"].get_field(pm.FIELD_RHO)
        pos = rc > 0
        rel = (rf[pos] - rc[pos]) / rc[pos]
        over = rc >= 1.0  # cells at or above the mean density
        rel_over = (rf[over] - rc[over]) / rc[over]
        rec = {"step": k, "a": float(a[k]), "z": float(1.0 / a[k] - 1.0), "k": kf, "P_fdm": pf, "P_cdm": pcdm,
               "modes": cnt, "rel_dP": (pf - pcdm) / pcdm, "rms_rel_density": float(np.sqrt(np.mean(rel ** 2))),
               "rms_rel_density_overdense": float(np.sqrt(np.mean(rel_over ** 2))) if rel_over.size else float("nan"),
               "cells_used": float(np.mean(pos)), "k_jeans": jeans_k(float(a[k]), m22)}
        if keep_density:
            rec["rho_fdm"], rec["rho_cdm"] = rf, rc
        out.append(rec)
    for s in sims.values():
        s.close()
    return out


def summary(out, box, n_mesh):
    """Per output: the largest |rel_dP| among the shells below half the Nyquist
    wavenumber where the pressureless spectrum holds at least 1e-3 of its peak
    (above the initial cut-off the ratio divides by almost nothing), with its
    k; rel_dP in the shell nearest k_J; and the RMS density differences."""
    k_nyq = math.pi * n_mesh / box
    rows = []
    for r in out:
        sel = (r["k"] <= 0.5 * k_nyq) & (r["P_cdm"] >= 1e-3 * np.max(r["P_cdm"]))
        i = int(np.argmax(np.abs(r["rel_dP"][sel])))
        j = int(np.argmin(np.abs(r["k"] - r["k_jeans"])))
        rows.append({"z": r["z"], "max_rel_dP": float(r["rel_dP"][sel][i]), "at_k": float(r["k"][sel][i]),
                     "k_jeans": r["k_jeans"], "rel_dP_at_kJ": float(r["rel_dP"][j]),
                     "rel_dP_at_kf": float(r["rel_dP"][0]), "rms_rel_density": r["rms_rel_density"],
                     "rms_rel_density_overdense": r["rms_rel_density_overdense"]})
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-side", type=int, default=256)
    ap.add_argument("--n-mesh", type=int, default=512)
    ap.add_argument("--box", type=float, default=10.0)
    ap.add_argument("--m22", type=float, default=1.0)
    ap.add_argument("--z-start", type=float, default=100.0)
    ap.add_argument("--z-end", type=float, default=3.0)
    ap.add_argument("--nsteps", type=int, default=1000)
    ap.add_argument("--z-out", default="10,5,3")
    ap.add_argument("--cdm-ics", action="store_true", help="pressureless run from CDM initial conditions")
    ap.add_argument("--kernel", choices=["cic", "spline"], default="spline",
                    help="density kernel (the paper's runs: the cubic spline)")
    ap.add_argument("--smooth-h", type=float, default=3.5, help="spline smoothing length in mesh cells")
    ap.add_argument("--json", default=None, help="write the full spectra here")
    args = ap.parse_args()
    from paper_1608_00802_gb300 import build, pm
    build.build()
    out = run_pair(args.n_side, args.n_mesh, args.box, args.m22, args.z_start, args.z_end, args.nsteps,
                   tuple(float(z) for z in args.z_out.split(",")), cdm_ics=args.cdm_ics,
                   kernel=pm.KERNEL_SPLINE if args.kernel == "spline" else pm.KERNEL_CIC, smooth_h=args.smooth_h)
    for row in summary(out, args.box, args.n_mesh):
        print(json.dumps(row))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump([{k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in r.items()} for r in out], fh)


if __name__ == "__main__":
    main()
