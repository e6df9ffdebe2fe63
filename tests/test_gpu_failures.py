"""Failure paths of the library on the GPU, made without any GPU fault: a
bounded device wait that gives up (the decoupled look-back of a radix pass
waiting on a tile that never publishes) and a non-finite particle state (a
momentum that overflows in the drift).  Both must come back as status codes
through the C ABI, and the simulation must stay usable."""
import numpy as np
import pytest

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


def _sim(pm, x, p, precision):
    sim = pm.Sim(pm.make_config(len(x), 64, 1.0, precision=precision, force_mode=pm.FORCE_HYBRID))
    sim.set_particles(x, p)
    return sim


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_lookback_timeout_is_reported_and_the_simulation_recovers(pm, precision):
    prec = pm.FP64 if precision == "fp64" else pm.FP32
    x, p = ics.zeldovich(32, 64, 1.0, 1 / 101.0, 5, amplitude=2.0)
    a0, a1 = 1 / 101.0, 1 / 90.0
    sim = _sim(pm, x, p, prec)
    assert sim.debug_sort_timeout(spin_limit=64) == 7  # PM_ERR_TIMEOUT
    # the error word was read and cleared; the state is intact: a step gives the same bits as a fresh run
    sim.step(a0, a1)
    e = sim.energy(a1)
    xa, pa = sim.get_particles()
    ref = _sim(pm, x, p, prec)
    ref.step(a0, a1)
    er = ref.energy(a1)
    xr, pr = ref.get_particles()
    np.testing.assert_array_equal(xa, xr)
    np.testing.assert_array_equal(pa, pr)
    np.testing.assert_array_equal(e, er)
    sim.close()
    ref.close()


def test_overflowing_momentum_reports_nonfinite(pm):
    """A momentum that fits in fp32 but whose drift overflows: the kick keeps
    the particle's old offset, flags the error word, and the next synchronous
    call returns PM_ERR_NONFINITE."""
    x, p = ics.zeldovich(16, 64, 1.0, 1 / 101.0, 6, amplitude=2.0)
    p = p.copy()
    p[5] = [3e38, 0.0, 0.0]
    sim = pm.Sim(pm.make_config(len(x), 64, 1.0, precision=pm.FP32, force_mode=pm.FORCE_HYBRID))
    sim.set_particles(x, p)
    x0, _ = sim.get_particles()
    sim.step(1 / 101.0, 1 / 50.0)
    with pytest.raises(pm.PMError) as exc:
        sim.get_particles()
    assert exc.value.status == 5  # PM_ERR_NONFINITE
    # the error word was cleared with the report; the particle kept its position
    x1, _ = sim.get_particles()
    assert np.all(np.isfinite(x1))
    assert np.abs(x1[5] - x0[5]).max() < 1e-6
    sim.close()
