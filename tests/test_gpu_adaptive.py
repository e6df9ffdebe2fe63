"""Adaptive leapfrog steps (the one-cell-per-step condition of Sec. II.A with
the quantum acceleration) on the GPU against the oracle's controller."""
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


def make(pm, precision, kernel=0, amplitude=6.0, n_side=16, n_mesh=32, box=1.0, m22=2.5):
    x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, 7, m22=m22, amplitude=amplitude)
    cfg = pm.make_config(len(x), n_mesh, box, m22=m22, force_mode=pm.FORCE_HYBRID, kernel=kernel,
                         precision=pm.FP64 if precision == "fp64" else pm.FP32)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    ocfg = O.Config(n_mesh=n_mesh, box=box, m22=m22, force_mode=O.HYBRID, kernel=kernel)
    return sim, ocfg


def test_adaptive_controller_matches_oracle_stepwise(pm):
    """From the GPU's own state before every step, the oracle's rule picks the
    same step end (fp64).  (Over many steps the two sequences may part: the
    maxima are taken over the kernel-gradient forces, which jump where a
    particle crosses a cell face, so a 1e-12 difference in a position can move
    a maximum.)"""
    sim, ocfg = make(pm, "fp64")
    a, a_end, cfl = 1 / 101.0, 1 / 30.0, 0.5
    steps = 0
    while a < a_end:
        x, p = sim.get_particles()
        ref = O.next_scale_factor(p, O.force_parts(x, ocfg), a, a_end, ocfg, cfl)
        b = sim.run_adaptive(a, a_end, cfl=cfl, max_steps=1)
        assert b[1] == pytest.approx(ref, rel=1e-9)
        a = b[1]
        steps += 1
    assert steps > 4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-3)])
def test_adaptive_run_power_spectrum_matches_oracle(pm, precision, tol):
    """The whole adaptive run: the oracle integrates over the GPU's step
    boundaries (the controller itself is compared step by step above), and
    P(k) agrees within the bar for k <= k_Nyq/2; the oracle's own adaptive
    run takes as many steps."""
    sim, ocfg = make(pm, precision, amplitude=1.0, n_side=32, n_mesh=64)
    x0, p0 = sim.get_particles()
    a0, a1, cfl = 1 / 101.0, 1 / 4.0, 0.25
    bounds = sim.run_adaptive(a0, a1, cfl=cfl)
    _, _, bo = O.run_adaptive(x0, p0, a0, a1, ocfg, cfl=cfl)
    assert abs(len(bounds) - len(bo)) <= 1 and len(bo) > 10
    xo, po, parts = x0, p0, None
    for k in range(len(bounds) - 1):
        xo, po, parts = O.kdk_step(xo, po, bounds[k], bounds[k + 1], ocfg, parts)
    k, pk, _ = sim.power_spectrum()
    ko, pko, _ = O.power_spectrum(xo, ocfg)
    # shells below k_Nyq/2 with power above the fp32 floor of this small, cut-off
    # spectrum (offsets carry 24 bits: shells 10^7 below the peak are rounding)
    sel = np.arange(16)
    if precision == "fp32":
        sel = sel[pko[:16] >= 1e-7 * pko.max()]
    assert len(sel) >= 6
    np.testing.assert_allclose(pk[sel], pko[sel], rtol=tol)


def test_adaptive_steps_keep_every_particle_within_cfl_cells(pm):
    """One step per call: every displacement stays within cfl*dx, and the calls
    reproduce a single multi-step call bit for bit."""
    sim, ocfg = make(pm, "fp32", kernel=1)
    ref, _ = make(pm, "fp32", kernel=1)
    a, a_end, cfl = 1 / 101.0, 1 / 40.0, 0.7
    dx = ocfg.dx
    x, _ = sim.get_particles()
    bounds = [a]
    while a < a_end:
        b = sim.run_adaptive(a, a_end, cfl=cfl, max_steps=1)
        assert len(b) == 2 and b[0] == a
        xn, _ = sim.get_particles()
        d = xn - x
        d -= np.round(d / ocfg.box) * ocfg.box
        assert np.linalg.norm(d, axis=1).max() <= cfl * dx * (1 + 1e-5)
        x, a = xn, b[1]
        bounds.append(a)
    assert len(bounds) > 3
    b2 = ref.run_adaptive(1 / 101.0, a_end, cfl=cfl)
    np.testing.assert_array_equal(np.array(bounds), b2)
    np.testing.assert_array_equal(sim.get_particles()[0], ref.get_particles()[0])


def test_adaptive_invalid_arguments(pm):
    sim, _ = make(pm, "fp32", n_side=8, n_mesh=16)
    for args in [(1 / 50.0, 1 / 60.0, 0.5), (1 / 50.0, 1 / 40.0, 0.0), (1 / 50.0, 1 / 40.0, 1.5)]:
        with pytest.raises(pm.PMError) as e:
            sim.run_adaptive(*args)
        assert e.value.status == 1
