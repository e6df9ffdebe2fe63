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


# a batch whose members share configurations (size, precision, kernel, force
# mode) but not box, mass or seed: the members of each class are stepped by
# one launch per kernel and one batched transform per class
PACKED = [  # (n_side, n_mesh, box, m22, seed, precision, mode)
    (16, 32, 1.0, 2.5, 10, "fp32", "hybrid"),
    (32, 64, 1.7, 10.0, 11, "fp32", "hybrid"),
    (16, 32, 3.1, 1.0, 12, "fp32", "hybrid"),
    (32, 64, 2.9, 5.0, 13, "fp32", "hybrid"),
    (16, 32, 1.3, 2.5, 14, "fp32", "hybrid"),
    (16, 32, 2.2, 5.0, 15, "fp32", "lagrangian"),
    (16, 32, 1.5, 1.0, 16, "fp32", "lagrangian"),
]


def _packed_vs_single(pm, nsteps, a1):
    a0 = 1 / 101.0
    batch = pm.Batch([_cfg(pm, m) for m in PACKED])
    for mem, m in zip(batch.members, PACKED):
        mem.set_particles(*_ics(m, a0))
    batch.run(nsteps, a0, a1)
    assert batch.info() == (3, len(PACKED))  # three classes, every member stepped packed
    out = []
    for i, m in enumerate(PACKED):
        xb, pb = batch.members[i].get_particles()
        eb = batch.members[i].energy(a1[i])
        cb, ib = batch.members[i].get_order()
        kb, pkb, _ = batch.members[i].power_spectrum()
        single = pm.Sim(_cfg(pm, m))
        single.set_particles(*_ics(m, a0))
        single.run(nsteps, a0, a1[i])
        xs, ps = single.get_particles()
        es = single.energy(a1[i])
        _, pks, _ = single.power_spectrum()
        single.close()
        # the storage order is the stable order of the cells (ties by previous order)
        assert np.all(np.diff(cb.astype(np.int64)) >= 0)
        assert sorted(ib.tolist()) == list(range(len(ib)))
        d = xb - xs
        d -= m[2] * np.round(d / m[2])
        out.append((m, np.abs(d).max() / (m[2] / m[1]), np.abs(pb - ps).max() / np.abs(ps).max(),
                    np.abs(eb[:3] - es[:3]).max() / np.abs(es[:3]).max(), np.abs(pkb / pks - 1).max()))
    batch.close()
    return out


A1 = np.array([1 / 60.0, 1 / 50.0, 1 / 70.0, 1 / 55.0, 1 / 40.0, 1 / 65.0, 1 / 45.0])


def test_packed_batch_members_match_single_runs_over_two_steps(pm):
    """Members stepped in packed launches against the same simulations run
    alone, over one captured pair of steps: the re-sort, deposit, stencil and
    kick are the same kernels, the batched transforms may round differently
    from the single ones, so the states agree to fp32 rounding (1e-5 of a
    cell, 1e-5 relative in momenta and energies)."""
    a1 = (1 / 101.0) * (A1 * 101.0) ** 0.05  # two short steps
    for m, dx, dp, de, dpk in _packed_vs_single(pm, 2, a1):
        assert dx < 1e-5, (m, dx)
        assert dp < 1e-5, (m, dp)
        assert de < 1e-5, (m, de)


def test_packed_batch_members_match_single_runs_over_nine_steps(pm):
    """Nine steps: with the quantum force on meshes of eight cells per particle
    a rounding difference can flip a discrete choice (a cell, the extended-
    precision branch of a near-empty node), so single particles may part by a
    fraction of a cell; P(k) and the energies stay within 1e-3."""
    for m, dx, dp, de, dpk in _packed_vs_single(pm, 9, A1):
        assert dx < 1e-2, (m, dx)
        assert de < 1e-3, (m, de)
        assert dpk < 1e-3, (m, dpk)
