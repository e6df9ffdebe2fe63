"""Batches of independent simulations (pm_batch_*): each member of a batch,
stepped inside the captured graph together with members of other sizes,
gives the same result as the same simulation run alone with pm_run."""
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


MEMBERS = [  # (n_side, n_mesh, box, m22, seed, precision, mode)
    (16, 32, 1.0, 2.5, 0, "fp32", "hybrid"),
    (32, 64, 1.7, 10.0, 1, "fp32", "hybrid"),
    (16, 32, 3.1, 1.0, 2, "fp32", "lagrangian"),
    (20, 40, 2.2, 5.0, 3, "fp32", "meshgrad"),
    (16, 32, 1.3, 2.5, 4, "fp64", "hybrid"),
]
MODES = {"meshgrad": 0, "hybrid": 1, "lagrangian": 2}


def _cfg(pm, m):
    n_side, n_mesh, box, m22, seed, prec, mode = m
    return pm.make_config(n_side ** 3, n_mesh, box, m22=m22, force_mode=MODES[mode],
                          precision=pm.FP64 if prec == "fp64" else pm.FP32)


def _ics(m, a0):
    n_side, n_mesh, box, m22, seed, _, _ = m
    return ics.zeldovich(n_side, n_mesh, box, a0, seed, m22=m22, amplitude=2.0)


@pytest.mark.parametrize("nsteps", [6, 7])
def test_batch_members_equal_single_runs(pm, nsteps):
    a0 = 1 / 101.0
    a1 = np.array([1 / 60.0, 1 / 50.0, 1 / 70.0, 1 / 55.0, 1 / 40.0])
    batch = pm.Batch([_cfg(pm, m) for m in MEMBERS])
    for mem, m in zip(batch.members, MEMBERS):
        mem.set_particles(*_ics(m, a0))
    batch.run(nsteps, a0, a1)
    for i, m in enumerate(MEMBERS):
        xb, pb = batch.members[i].get_particles()
        eb = batch.members[i].energy(a1[i])
        single = pm.Sim(_cfg(pm, m))
        single.set_particles(*_ics(m, a0))
        single.run(nsteps, a0, a1[i])
        xs, ps = single.get_particles()
        es = single.energy(a1[i])
        np.testing.assert_array_equal(xb, xs)
        np.testing.assert_array_equal(pb, ps)
        np.testing.assert_array_equal(eb, es)
    batch.close()


def test_batch_member_matches_oracle(pm):
    """One member of a mixed batch against the FP64 oracle over a few steps."""
    a0, a1, nsteps = 1 / 101.0, 1 / 80.0, 4
    m = (32, 64, 1.0, 2.5, 9, "fp64", "hybrid")
    batch = pm.Batch([_cfg(pm, MEMBERS[0]), _cfg(pm, m)])
    batch.members[0].set_particles(*_ics(MEMBERS[0], a0))
    x, p = _ics(m, a0)
    batch.members[1].set_particles(x, p)
    xg, pg = batch.members[1].get_particles()
    batch.run(nsteps, a0, [a1, a1])
    xb, pb = batch.members[1].get_particles()
    ocfg = O.Config(n_mesh=64, box=1.0, force_mode=O.HYBRID)
    xo, po, _ = O.run(xg, pg, a0, a1, nsteps, ocfg)
    d = xb - xo
    d -= np.round(d)
    assert np.abs(d).max() < 1e-9
    assert np.sqrt(np.mean((pb - po) ** 2) / np.mean(po ** 2)) < 1e-9
    batch.close()
