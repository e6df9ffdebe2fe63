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


def _full_run(pm, precision, mode, kernel=0, quantum=True, chunks=20, nsteps=500, ulp_shift=False):
    x, p = ics.zeldovich(128, 256, 2.0, 1 / 101.0, 42, m22=2.5)
    if ulp_shift:
        # every input position moved by one fp32 ulp (alternating sign): the
        # run's sensitivity to rounding, measured in fp64
        ulp = np.spacing(x.astype(np.float32)).astype(np.float64)
        x = np.mod(x + np.where(np.arange(x.size).reshape(x.shape) % 2 == 0, ulp, -ulp), 2.0)
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


OCFG = O.Config(n_mesh=256, box=2.0, m22=2.5)


def _dp(k, pa, pb):
    sel = k <= 0.5 * math.pi * 256 / 2.0  # k <= k_Nyq / 2
    return np.abs(pa[sel] / pb[sel] - 1).max()


def _compare(pm, **kw):
    k, p32, h32 = _full_run(pm, pm.FP32, **kw)
    _, p64, h64 = _full_run(pm, pm.FP64, **kw)
    return (_dp(k, p32, p64), O.layzer_irvine_residual(h32, OCFG), O.layzer_irvine_residual(h64, OCFG))


def test_pressureless_bench_workload_fp32_matches_fp64(pm):
    """Without the quantum force: P(k) within 1e-4, energy budget closed to 1e-2."""
    dp, li32, li64 = _compare(pm, mode=pm.FORCE_HYBRID, quantum=False)
    assert dp < 1e-4
    assert np.abs(li32).max() < 1e-2 and np.abs(li64).max() < 1e-2


@pytest.mark.parametrize("mode", ["hybrid", "lagrangian"])
def test_spline_bench_workload_fp32_matches_fp64(pm, mode):
    """With the quantum force and the paper's spline kernel (h = 3.5 dx): P(k)
    within 1e-3 after the full run (the accuracy bar for full runs; the fp64
    run moved by one fp32 ulp per position stays within ~1e-4 of itself, so
    the bar is not below the problem's own rounding sensitivity), the energy
    budget closed to 1e-2 by both paths and alike to 1e-3."""
    fm = pm.FORCE_HYBRID if mode == "hybrid" else pm.FORCE_LAGRANGIAN
    dp, li32, li64 = _compare(pm, mode=fm, kernel=pm.KERNEL_SPLINE)
    assert dp < 1e-3
    assert np.abs(li32).max() < 1e-2 and np.abs(li64).max() < 1e-2
    assert np.abs(li32 - li64).max() < 1e-3


def test_cloud_in_cell_quantum_bench_workload_fp32_within_the_rounding_floor(pm):
    """The benchmarked cloud-in-cell run with the quantum force (HYBRID).  On a
    mesh of eight cells per particle the quantum pressure acts on the particles'
    shot noise and the run is chaotic: the fp64 run against itself with every
    input position moved by one fp32 ulp already differs by several per cent in
    P(k) (measured here, not assumed), so a 1e-3 bar cannot hold for any
    precision.  The fp32 path must stay within twice that floor, and its
    Layzer-Irvine residual (which does not close for this scheme at this
    resolution, in fp64 either) within twice the floor's change of it."""
    k, p64, h64 = _full_run(pm, pm.FP64, mode=pm.FORCE_HYBRID)
    _, p64b, h64b = _full_run(pm, pm.FP64, mode=pm.FORCE_HYBRID, ulp_shift=True)
    _, p32, h32 = _full_run(pm, pm.FP32, mode=pm.FORCE_HYBRID)
    floor = _dp(k, p64b, p64)
    assert floor > 1e-3  # the bar of 1e-3 is below this run's own rounding sensitivity
    assert _dp(k, p32, p64) < 2 * floor
    li64 = np.abs(O.layzer_irvine_residual(h64, OCFG)).max()
    li64b = np.abs(O.layzer_irvine_residual(h64b, OCFG)).max()
    li32 = np.abs(O.layzer_irvine_residual(h32, OCFG)).max()
    assert abs(li32 - li64) < 2 * abs(li64b - li64) + 1e-3 * li64
