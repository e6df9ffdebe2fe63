"""Checkpoint and resume (pm_save / pm_load): a run of N steps equals k steps,
a checkpoint, and N - k steps continued from it (in a new simulation or in the
same one after other work), bit for bit; a checkpoint of another configuration
is refused and leaves the simulation unchanged."""
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


CASES = [  # (n_side, n_mesh, box, precision, kernel, mode)
    (32, 64, 1.0, "fp32", "cic", "hybrid"),
    (64, 128, 2.0, "fp32", "cic", "hybrid"),       # the 2D transforms with the z kernel
    (16, 32, 1.0, "fp64", "cic", "lagrangian"),
    (16, 32, 1.0, "fp32", "spline", "hybrid"),
]
MODES = {"meshgrad": 0, "hybrid": 1, "lagrangian": 2}


def _cfg(pm, c):
    n_side, n_mesh, box, prec, kernel, mode = c
    return pm.make_config(n_side ** 3, n_mesh, box, force_mode=MODES[mode],
                          precision=pm.FP64 if prec == "fp64" else pm.FP32,
                          kernel=pm.KERNEL_SPLINE if kernel == "spline" else pm.KERNEL_CIC)


@pytest.mark.parametrize("case", CASES)
def test_resume_equals_uninterrupted_run(pm, case):
    n_side, n_mesh, box = case[:3]
    a = np.geomspace(1 / 101.0, 1 / 60.0, 9)
    x, p = ics.zeldovich(n_side, n_mesh, box, a[0], 5, amplitude=3.0)
    ref = pm.Sim(_cfg(pm, case))
    ref.set_particles(x, p)
    ref.run(3, a[0], a[3])
    ref.run(5, a[3], a[8])
    x_ref, p_ref = ref.get_particles()
    e_ref = ref.energy(a[8])
    first = pm.Sim(_cfg(pm, case))
    first.set_particles(x, p)
    first.run(3, a[0], a[3])
    ck = first.save()
    assert ck.nbytes == 256 + len(x) * (2 * (32 if case[3] == "fp64" else 16) + 4)
    first.close()
    resumed = pm.Sim(_cfg(pm, case))       # a new simulation, no particles of its own
    resumed.load(ck)
    resumed.run(5, a[3], a[8])
    xr, pr = resumed.get_particles()
    np.testing.assert_array_equal(xr, x_ref)
    np.testing.assert_array_equal(pr, p_ref)
    np.testing.assert_array_equal(resumed.energy(a[8]), e_ref)
    # the same simulation taken elsewhere and brought back
    resumed.run(2, a[8], a[8] * 1.05)
    resumed.load(ck)
    resumed.run(5, a[3], a[8])
    np.testing.assert_array_equal(resumed.get_particles()[0], x_ref)
    resumed.close()
    ref.close()


def test_checkpoint_of_another_configuration_is_refused(pm):
    x, p = ics.zeldovich(16, 32, 1.0, 1 / 101.0, 1)
    a = pm.Sim(pm.make_config(len(x), 32, 1.0))
    a.set_particles(x, p)
    ck = a.save()
    b = pm.Sim(pm.make_config(len(x), 64, 1.0))
    x2, p2 = ics.zeldovich(16, 64, 1.0, 1 / 101.0, 2)
    b.set_particles(x2, p2)
    before = b.get_particles()
    with pytest.raises(pm.PMError, match="another configuration"):
        b.load(ck)
    with pytest.raises(pm.PMError, match="version"):
        b.load(np.zeros(ck.nbytes, dtype=np.uint8))
    with pytest.raises(pm.PMError, match="short"):
        a.load(ck[:100])
    np.testing.assert_array_equal(b.get_particles()[0], before[0])
    a.close()
    b.close()
