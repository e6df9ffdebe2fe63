"""The bench workload run in full (128^3 particles on 256^3, L = 2 Mpc/h,
z = 100 -> 3 in 500 steps): the fp32 path against the plain fp64 path (which
matches the oracle to 1e-10 in the parity tests; the oracle itself would need
about half an hour of host time here), for P(k) and for the energy budget."""
import math

import numpy as np
import pytest

from oracle import pm_oracle as O
from paper_1608_00802_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00802_gb300 import build
    build.build()
    from paper_1608_00802_gb300 import pm as _pm
    return _pm


def _full_run(pm, precision, mode, kernel=0, quantum=True, chunks=20, nsteps=500):
    x, p = ics.zeldovich(128, 256, 2.0, 1 / 101.0, 42, m22=2.5)
    cfg = pm.make_config(len(x), 256, 2.0, m22=2.5, precision=precision, force_mode=mode, kernel=kernel,
                         quantum=quantum)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    a0, a1 = 1 / 101.0, 1 / 4.0
    a = a0 * (a1 / a0) ** (np.arange(nsteps + 1) / nsteps)
    a[-1] = a1
    per = nsteps // chunks
    hist = [(a[0],) + tuple(sim.energy(a[0])[:3])]
    for c in range(chunks):
        sim.run(per, a[c * per], a[(c + 1) * per])
        hist.append((a[(c + 1) * per],) + tuple(sim.energy(a[(c + 1) * per])[:3]))
    k, pk, _ = sim.power_spectrum()
    sim.close()
    return k, pk, np.array(hist)


def _compare(pm, **kw):
    k, p32, h32 = _full_run(pm, pm.FP32, **kw)
    _, p64, h64 = _full_run(pm, pm.FP64, **kw)
    sel = k <= 0.5 * math.pi * 256 / 2.0
    ocfg = O.Config(n_mesh=256, box=2.0, m22=2.5)
    return (np.abs(p32[sel] / p64[sel] - 1).max(), O.layzer_irvine_residual(h32, ocfg),
            O.layzer_irvine_residual(h64, ocfg))


def test_pressureless_bench_workload_fp32_matches_fp64(pm):
    """Without the quantum force: P(k) within 1e-4, energy budget closed to 1e-2."""
    dp, li32, li64 = _compare(pm, mode=pm.FORCE_HYBRID, quantum=False)
    assert dp < 1e-4
    assert np.abs(li32).max() < 1e-2 and np.abs(li64).max() < 1e-2


@pytest.mark.parametrize("mode", ["hybrid", "lagrangian"])
def test_spline_bench_workload_fp32_matches_fp64(pm, mode):
    """With the quantum force and the paper's spline kernel (h = 3.5 dx): P(k)
    within 3e-3 (the sensitivity of the nonlinear evolution to rounding; the
    pressureless run stays within 1e-5), energy budget closed to 1e-2 by both
    paths, alike to 1e-3.  (With cloud-in-cell at this resolution the quantum
    pressure acts on the particle shot noise and the budget does not close;
    the design notes give the numbers.)"""
    fm = pm.FORCE_HYBRID if mode == "hybrid" else pm.FORCE_LAGRANGIAN
    dp, li32, li64 = _compare(pm, mode=fm, kernel=pm.KERNEL_SPLINE)
    assert dp < 3e-3
    assert np.abs(li32).max() < 1e-2 and np.abs(li64).max() < 1e-2
    assert np.abs(li32 - li64).max() < 1e-3
