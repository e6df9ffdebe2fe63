"""The cubic spline kernel of Sec. II.A (h = 3.5 dx by default) on the GPU
against the oracle: density, mesh potentials, accelerations, a full run's
P(k), and the properties the smoothing must keep (mass, symmetric weights)."""
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


MODES = {"hybrid": O.HYBRID, "lagrangian": O.LAGRANGIAN, "meshgrad": O.MESHGRAD}


def make(pm, n_side, n_mesh, box, precision="fp32", mode="hybrid", h=3.5, m22=2.5, amplitude=4.0, seed=42,
         real=False):
    x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, seed, m22=m22, amplitude=amplitude)
    prec = pm.FP64 if precision == "fp64" else pm.FP32
    cfg = pm.make_config(len(x), n_mesh, box, precision=prec, m22=m22, force_mode=MODES[mode],
                         kernel=pm.KERNEL_SPLINE, smooth_h=h, smooth_real=real)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    ocfg = O.Config(n_mesh=n_mesh, box=box, m22=m22, force_mode=MODES[mode], kernel=O.KERNEL_SPLINE, smooth_h=h)
    return sim, ocfg


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
@pytest.mark.parametrize("n_side,n_mesh,box,h", [(16, 32, 1.0, 3.5), (24, 48, 1.5, 2.0), (32, 64, 1.0, 3.5)])
def test_spline_density_matches_oracle(pm, precision, tol, n_side, n_mesh, box, h):
    sim, ocfg = make(pm, n_side, n_mesh, box, precision, h=h)
    rho = sim.deposit()
    xg, _ = sim.get_particles()
    ref = O.density(xg, ocfg)
    assert np.abs(rho - ref).max() < tol * np.abs(ref).max()
    assert rho.sum() == pytest.approx(n_mesh ** 3, rel=1e-5 if precision == "fp32" else 1e-12)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("mode", ["hybrid", "lagrangian"])
def test_spline_fields_and_accelerations_match_oracle(pm, precision, tol, mode):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, mode=mode)
    a = 1 / 101.0
    acc = sim.forces(a)
    xg, _ = sim.get_particles()
    rho, phi, q = O.mesh_fields(xg, ocfg)
    assert rel_rms(sim.get_field(pm.FIELD_RHO), rho) < tol
    assert rel_rms(sim.get_field(pm.FIELD_PHI), phi) < tol
    assert rel_rms(sim.get_field(pm.FIELD_Q), q) < tol
    ref = O.accelerations(xg, a, ocfg)
    assert rel_rms(acc, ref) < tol


def test_spline_energies_match_oracle(pm):
    sim, ocfg = make(pm, 32, 64, 1.0, "fp64", mode="lagrangian")
    a = 1 / 101.0
    e = sim.energy(a)
    xg, pg = sim.get_particles()
    ref = O.energies(xg, pg, a, ocfg)
    np.testing.assert_allclose(e[:3], ref[:3], rtol=1e-10)


@pytest.mark.parametrize("precision,mode", [("fp64", "hybrid"), ("fp64", "lagrangian"), ("fp32", "hybrid")])
def test_spline_full_run_power_spectrum(pm, precision, mode):
    """32^3 particles on 64^3, z = 100 -> 3 in 200 steps with the spline kernel
    (h = 3.5 dx) vs the oracle: P(k) within 0.1% for k <= k_Nyq/2."""
    sim, ocfg = make(pm, 32, 64, 1.0, precision, mode=mode, amplitude=1.0)
    x0, p0 = sim.get_particles()
    sim.run(200, 1 / 101.0, 1 / 4.0)
    k, pk, _ = sim.power_spectrum()
    xo, _, _ = O.run(x0, p0, 1 / 101.0, 1 / 4.0, 200, ocfg)
    ko, pko, _ = O.power_spectrum(xo, ocfg)
    np.testing.assert_allclose(k, ko, rtol=1e-12)
    sel = slice(0, 16)
    np.testing.assert_allclose(pk[sel], pko[sel], rtol=1e-3)


def test_spline_lowers_the_quantum_noise(pm):
    """The point of the smoothing (Sec. II.A): on a mesh of 8 cells per particle
    the spline density carries far less cell-scale noise than cloud-in-cell,
    and so does Q."""
    x, p = ics.zeldovich(32, 64, 1.0, 1 / 101.0, 42, amplitude=4.0)
    out = {}
    for kern in (pm.KERNEL_CIC, pm.KERNEL_SPLINE):
        cfg = pm.make_config(len(x), 64, 1.0, force_mode=pm.FORCE_HYBRID, kernel=kern)
        sim = pm.Sim(cfg)
        sim.set_particles(x, p)
        sim.forces(1 / 101.0)
        out[kern] = (sim.get_field(pm.FIELD_RHO), sim.get_field(pm.FIELD_Q))
    rc, qc = out[pm.KERNEL_CIC]
    rs, qs = out[pm.KERNEL_SPLINE]
    assert np.std(rs) < 0.5 * np.std(rc)
    assert np.std(qs) < 0.1 * np.std(qc)


def test_spline_config_validation(pm):
    base = dict(n_part=8 ** 3, n_mesh=16, box=1.0)
    for h in (0.5, 4.5):   # outside [1, N/4]
        cfg = pm.make_config(base["n_part"], base["n_mesh"], base["box"], kernel=pm.KERNEL_SPLINE, smooth_h=h)
        assert pm.arena_bytes(cfg) == 0
    cfg = pm.make_config(base["n_part"], base["n_mesh"], base["box"], kernel=7)
    assert pm.arena_bytes(cfg) == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_energy_calls_leave_the_trajectory_unchanged(pm, precision):
    """pm_energy recomputes Q~ with the K_rho sums; with the spline kernel the
    field the particles feel is the smoothed one, so the recomputation must
    smooth it again: a run with energy calls between its parts ends on the
    same bits as the same run without them."""
    a0, a1 = 1 / 101.0, 1 / 20.0
    am = math.sqrt(a0 * a1)
    finals = []
    for with_energy in (False, True):
        sim, _ = make(pm, 16, 32, 1.0, precision, mode="hybrid")
        sim.run(8, a0, am)
        if with_energy:
            sim.energy(am)
        sim.run(8, am, a1)
        finals.append(sim.get_particles())
        sim.close()
    np.testing.assert_array_equal(finals[0][0], finals[1][0])
    np.testing.assert_array_equal(finals[0][1], finals[1][1])


@pytest.mark.parametrize("n_side,n_mesh,box,h", [(16, 32, 1.0, 3.5), (24, 48, 1.5, 2.0), (32, 64, 1.0, 4.0),
                                                 (20, 40, 1.0, 3.0)])
def test_real_space_smoothing_matches_oracle(pm, n_side, n_mesh, box, h):
    """smooth_real = 1: the density and Q smoothed by the direct sum over the
    node weights in real space (the same operator as the spectral one): the
    smoothed density within 2e-6 of the oracle's, the mesh fields and the
    accelerations within 1e-5, for supports of 2, 3 and 4 cells and mesh
    sizes that are not powers of two."""
    sim, ocfg = make(pm, n_side, n_mesh, box, "fp32", h=h, real=True)
    rho = sim.deposit()
    xg, _ = sim.get_particles()
    ref = O.density(xg, ocfg)
    assert np.abs(rho - ref).max() < 2e-6 * np.abs(ref).max()
    a = 1 / 101.0
    acc = sim.forces(a)
    r, phi, q = O.mesh_fields(xg, ocfg)
    assert rel_rms(sim.get_field(pm.FIELD_RHO), r) < 1e-5
    assert rel_rms(sim.get_field(pm.FIELD_Q), q) < 1e-5
    assert rel_rms(acc, O.accelerations(xg, a, ocfg)) < 1e-5


def test_real_space_smoothing_steps_match_the_spectral_run(pm):
    """20 steps with each smoothing: the same state to fp32 rounding."""
    a0, a1 = 1 / 101.0, 1 / 40.0
    out = []
    for real in (False, True):
        sim, _ = make(pm, 32, 64, 1.0, "fp32", mode="hybrid", real=real)
        sim.run(20, a0, a1)
        out.append(sim.get_particles())
        sim.close()
    d = out[0][0] - out[1][0]
    d -= np.round(d)
    assert np.abs(d).max() < 1e-5 / 64
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-4 * np.abs(out[0][1]).max()


def test_real_space_smoothing_config_validation(pm):
    n = 16 ** 3
    for kw in (dict(kernel=pm.KERNEL_CIC), dict(kernel=pm.KERNEL_SPLINE, smooth_h=4.5),
               dict(kernel=pm.KERNEL_SPLINE, precision=pm.FP64)):
        cfg = pm.make_config(n, 32, 1.0, smooth_real=True, **kw)
        assert pm.arena_bytes(cfg) == 0
