"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: bit-exact cell keys and storage order; fp32 one-step accelerations
within 1e-5 relative RMS; fp64 path within 1e-10; P(k) within 0.1% after
full runs (k <= k_Nyq/2).  Inputs are the seeded synthetic Zel'dovich
initial conditions; the oracle always receives the GPU's own (quantised)
positions so that both evaluate the same particles.
"""
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


MODES = {"meshgrad": O.MESHGRAD, "hybrid": O.HYBRID, "lagrangian": O.LAGRANGIAN}


def make(pm, n_side, n_mesh, box, precision="fp32", seed=42, a=1 / 101.0, m22=2.5, mode="meshgrad",
         lap=0, quantum=True, cosmological=True, x=None, p=None, amplitude=1.0):
    prec = pm.FP64 if precision == "fp64" else pm.FP32
    if x is None:
        x, p = ics.zeldovich(n_side, n_mesh, box, a, seed, m22=m22, amplitude=amplitude)
    cfg = pm.make_config(len(x), n_mesh, box, precision=prec, m22=m22, force_mode=MODES[mode], lap=lap,
                         quantum=quantum, cosmological=cosmological)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    ocfg = O.Config(n_mesh=n_mesh, box=box, m22=m22, force_mode=MODES[mode], lap=lap, quantum=quantum,
                    cosmological=cosmological)
    return sim, ocfg


def rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


def oracle_order(xg, ocfg, prev_ids):
    """stable order of the oracle keys, ties by the previous storage order"""
    keys = O.cell_key(xg, ocfg)
    prev_pos = np.empty(len(prev_ids), dtype=np.int64)
    prev_pos[prev_ids] = np.arange(len(prev_ids))
    order = np.lexsort((prev_pos, keys))
    return keys, order


# ------------------------------------------------------------------ sort
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n_side,n_mesh,box", [(32, 64, 1.0), (20, 40, 1.0), (64, 128, 2.0)])
def test_initial_sort_is_bit_exact(pm, precision, n_side, n_mesh, box):
    sim, ocfg = make(pm, n_side, n_mesh, box, precision)
    xg, _ = sim.get_particles()
    cell, ids = sim.get_order()
    keys, order = oracle_order(xg, ocfg, np.arange(len(xg)))
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(cell, keys[order])


def test_sort_after_step_is_stable_wrt_previous_order(pm):
    sim, ocfg = make(pm, 32, 64, 1.0, "fp32", amplitude=8.0)
    _, ids0 = sim.get_order()
    sim.step(1 / 101.0, 1 / 90.0)
    xg, _ = sim.get_particles()
    cell, ids = sim.get_order()
    keys, order = oracle_order(xg, ocfg, ids0)
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(cell, keys[order])
    assert np.any(ids != ids0)       # particles did change cells


def _check_steps_resort(sim, ocfg, a_sched):
    """steps one by one; after each, the storage order must be the stable order
    of the new keys with ties in the previous storage order; returns the
    fraction of particles that changed cell in each step"""
    cell_prev, ids_prev = sim.get_order()
    moved = []
    for k in range(len(a_sched) - 1):
        sim.step(a_sched[k], a_sched[k + 1])
        xg, _ = sim.get_particles()
        cell, ids = sim.get_order()
        keys, order = oracle_order(xg, ocfg, ids_prev)
        np.testing.assert_array_equal(ids, order)
        np.testing.assert_array_equal(cell, keys[order])
        before = np.empty_like(cell_prev)
        before[ids_prev] = cell_prev
        moved.append(float(np.mean(keys != before)))
        cell_prev, ids_prev = cell, ids
    return moved


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resort_of_movers_over_several_steps(pm, precision):
    # 24^3 = 13,824 particles: six full sort tiles and a ragged seventh
    sim, ocfg = make(pm, 24, 48, 1.0, precision, amplitude=8.0, mode="hybrid")
    moved = _check_steps_resort(sim, ocfg, np.geomspace(1 / 101.0, 1 / 40.0, 6))
    assert 0.0 < min(moved) and max(moved) < 1.0


def test_resort_when_every_particle_moves(pm):
    # static box, no quantum pressure, uniform velocity of 1.5 cells per step:
    # every particle changes cell, so all of them take the movers' radix sort
    rng = np.random.default_rng(3)
    n, n_mesh, box = 7000, 32, 1.0
    x = rng.uniform(0, box, size=(n, 3))
    dt = 0.01
    p = np.zeros((n, 3))
    p[:, 0] = 1.5 * (box / n_mesh) / dt
    p[:, 1] = -1.25 * (box / n_mesh) / dt
    sim, ocfg = make(pm, 0, n_mesh, box, "fp32", x=x, p=p, quantum=False, cosmological=False)
    moved = _check_steps_resort(sim, ocfg, [1.0, 1.0 + dt, 1.0 + 2 * dt, 1.0 + 3 * dt])
    assert min(moved) == 1.0


def test_resort_when_no_particle_moves(pm):
    # particles at rest at cell centres, a static box without forces: no movers
    n_mesh, box = 16, 1.0
    g = (np.arange(n_mesh) + 0.5) * box / n_mesh
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([x, x])                # two particles per cell: ties kept in order
    p = np.zeros_like(x)
    sim, ocfg = make(pm, 0, n_mesh, box, "fp32", x=x, p=p, quantum=False, cosmological=False)
    moved = _check_steps_resort(sim, ocfg, [1.0, 1.1, 1.2])
    assert max(moved) == 0.0


def test_resort_with_fewer_particles_than_a_warp(pm):
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1.0, size=(19, 3))
    p = rng.normal(scale=3.0, size=(19, 3))
    sim, ocfg = make(pm, 0, 8, 1.0, "fp32", x=x, p=p, quantum=False, cosmological=False)
    moved = _check_steps_resort(sim, ocfg, [1.0, 1.02, 1.04, 1.06])
    assert max(moved) > 0.0


def test_resort_at_bench_size(pm):
    # 128^3 particles on 256^3, L = 2 Mpc/h, hybrid force, three steps
    sim, ocfg = make(pm, 128, 256, 2.0, "fp32", mode="hybrid")
    moved = _check_steps_resort(sim, ocfg, np.geomspace(1 / 101.0, 1 / 90.0, 4))
    assert max(moved) > 0.0


# ------------------------------------------------------------------ deposit
@pytest.mark.parametrize("precision,tol", [("fp32", 2e-6), ("fp64", 1e-13)])
@pytest.mark.parametrize("n_side,n_mesh,box", [(32, 64, 1.0), (24, 48, 1.5), (128, 256, 2.0)])
def test_deposit_matches_oracle(pm, precision, tol, n_side, n_mesh, box):
    sim, ocfg = make(pm, n_side, n_mesh, box, precision, amplitude=4.0)
    rho = sim.deposit()
    xg, _ = sim.get_particles()
    ref = O.cic_deposit(xg, ocfg)
    assert np.abs(rho - ref).max() < tol * max(1.0, np.abs(ref).max())
    assert rho.sum() == pytest.approx(n_mesh ** 3, rel=1e-6 if precision == "fp32" else 1e-12)


# ------------------------------------------------------------------ mesh stages
@pytest.mark.parametrize("precision,tol", [("fp32", 2e-6), ("fp64", 1e-12)])
@pytest.mark.parametrize("lap", [0, 1])
def test_potential_and_quantum_pressure_match_oracle(pm, precision, tol, lap):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, lap=lap, amplitude=4.0)
    sim.forces(0.01)
    rho = sim.get_field(pm.FIELD_RHO)
    phi = sim.get_field(pm.FIELD_PHI)
    q = sim.get_field(pm.FIELD_Q)
    phi_ref = O.poisson_phi(rho, ocfg)
    q_ref = O.quantum_potential(rho, ocfg)
    assert np.abs(phi - phi_ref).max() < tol * np.abs(phi_ref).max()
    assert rel_rms(q, q_ref) < tol * 10


def test_gaussian_quantum_pressure_closed_form_on_gpu(pm):
    """Prescribed Gaussian density through pm_set_density: Q~ equals the exact
    discrete closed form of the compact stencil (see the oracle pins)."""
    n, box, sigma = 64, 1.0, 0.09
    x, p = ics.lattice(32, n, box)
    cfg = pm.make_config(len(x), n, box, precision=pm.FP64, rho_floor=1e-300)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    dx = box / n
    c = (np.arange(n) - n // 2) * dx
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    rho = np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * sigma ** 2))
    sim.set_density(rho)
    q = sim.get_field(pm.FIELD_Q)
    s2 = sigma ** 2
    term = sum(np.exp(-(2 * v * dx + dx * dx) / (4 * s2)) + np.exp((2 * v * dx - dx * dx) / (4 * s2)) - 2.0
               for v in (xx, yy, zz)) / dx ** 2
    hbm = O.hbar_over_m(2.5, 0.7)
    expect = -0.5 * hbm ** 2 * term
    inner = (slice(2, -2),) * 3
    np.testing.assert_allclose(q[inner], expect[inner], rtol=1e-9, atol=1e-12 * np.abs(expect).max())


# ------------------------------------------------------------------ forces
@pytest.mark.parametrize("mode", ["meshgrad", "hybrid", "lagrangian"])
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_one_step_accelerations_match_oracle(pm, mode, precision, tol):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, mode=mode, amplitude=4.0)
    a = 0.05
    acc = sim.forces(a)
    xg, _ = sim.get_particles()
    ref = O.accelerations(xg, a, ocfg)
    assert rel_rms(acc, ref) < tol


@pytest.mark.parametrize("lap", [0, 1])
def test_accelerations_wide_and_compact_laplacian(pm, lap):
    sim, ocfg = make(pm, 24, 48, 1.0, "fp32", mode="lagrangian", lap=lap, amplitude=4.0)
    acc = sim.forces(0.1)
    xg, _ = sim.get_particles()
    assert rel_rms(acc, O.accelerations(xg, 0.1, ocfg)) < 1e-5


def test_full_size_accelerations_128_on_256(pm):
    """The bench workload (128^3 particles on a 256^3 mesh, L = 2 Mpc/h, fp32)."""
    sim, ocfg = make(pm, 128, 256, 2.0, "fp32")
    acc = sim.forces(1 / 101.0)
    xg, _ = sim.get_particles()
    ref = O.accelerations(xg, 1 / 101.0, ocfg)
    assert rel_rms(acc, ref) < 1e-5


def test_gravity_conserves_momentum_on_gpu(pm):
    sim, ocfg = make(pm, 16, 32, 1.0, "fp64", quantum=False, amplitude=8.0)
    acc = sim.forces(1.0)
    assert np.abs(acc.sum(axis=0)).max() < 1e-10 * np.abs(acc).sum()


# ------------------------------------------------------------------ leapfrog
@pytest.mark.parametrize("mode", ["meshgrad", "lagrangian"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_one_kdk_step_matches_oracle(pm, mode, precision):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, mode=mode, amplitude=4.0)
    x0, p0 = sim.get_particles()
    a0, a1 = 1 / 101.0, 1 / 95.0
    sim.step(a0, a1)
    xg, pg = sim.get_particles()
    xo, po, _ = O.kdk_step(x0, p0, a0, a1, ocfg)
    d = xg - xo
    d -= np.round(d / ocfg.box) * ocfg.box
    tol = 2e-6 if precision == "fp32" else 1e-11
    assert np.abs(d).max() < tol * ocfg.dx * 10
    assert rel_rms(pg, po) < (1e-5 if precision == "fp32" else 1e-10)
    # cell indices agree except within roundoff of a face
    cg = O.cell_index(xg, ocfg)
    co = O.cell_index(xo, ocfg)
    bad = np.any(cg != co, axis=1)
    if bad.any():
        frac = xo[bad] / ocfg.dx
        assert np.all(np.min(np.abs(frac - np.round(frac)), axis=1) < 1e-5)


def test_run_equals_repeated_steps(pm):
    """pm_run merges the closing and opening half kicks; the result equals n
    pm_step calls to rounding."""
    s1, _ = make(pm, 32, 64, 1.0, "fp64")
    s2, _ = make(pm, 32, 64, 1.0, "fp64")
    a = O.scale_factors(1 / 101.0, 1 / 50.0, 5, O.Config(8, 1.0))
    for i in range(5):
        s1.step(a[i], a[i + 1])
    s2.run(5, a[0], a[-1])
    x1, p1 = s1.get_particles()
    x2, p2 = s2.get_particles()
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    assert rel_rms(p2, p1) < 1e-12


def test_runs_are_bitwise_reproducible(pm):
    outs = []
    for _ in range(2):
        sim, _ = make(pm, 32, 64, 1.0, "fp32")
        sim.run(10, 1 / 101.0, 1 / 50.0)
        outs.append(sim.get_particles())
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


# ------------------------------------------------------------------ energies
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-11)])
@pytest.mark.parametrize("lap", [0, 1])
def test_energies_match_oracle(pm, precision, tol, lap):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, lap=lap, amplitude=4.0)
    sim.step(1 / 101.0, 1 / 99.0)
    a = 1 / 99.0
    e = sim.energy(a)
    xg, pg = sim.get_particles()
    ref = np.array(O.energies(xg, pg, a, ocfg))
    for k in range(3):
        assert e[k] == pytest.approx(ref[k], rel=tol)
    scale = np.abs(pg).sum() * ocfg.box ** 3 / len(pg)
    assert np.abs(e[3:] - ref[3:]).max() < tol * scale


# ------------------------------------------------------------------ power spectrum
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_power_spectrum_matches_oracle(pm, precision):
    sim, ocfg = make(pm, 32, 64, 1.0, precision, amplitude=4.0)
    k, pk, cnt = sim.power_spectrum()
    xg, _ = sim.get_particles()
    ko, po, co = O.power_spectrum(xg, ocfg)
    np.testing.assert_array_equal(cnt, co)
    np.testing.assert_allclose(k, ko, rtol=1e-12)
    np.testing.assert_allclose(pk, po, rtol=1e-4 if precision == "fp32" else 1e-10)


@pytest.mark.parametrize("precision,mode", [("fp64", "hybrid"), ("fp64", "lagrangian"), ("fp32", "hybrid")])
def test_power_spectrum_after_full_run(pm, precision, mode):
    """32^3 particles on 64^3, z = 100 -> 3 in 200 steps (the 32^3/64^3
    workload) vs the oracle: P(k) within 0.1% for k <= k_Nyq/2.  (The central-
    difference Q force is chaotic on this 2x CIC mesh, see the design notes,
    so the full-run comparison uses the kernel-gradient Q force.)"""
    sim, ocfg = make(pm, 32, 64, 1.0, precision, mode=mode)
    x0, p0 = sim.get_particles()
    sim.run(200, 1 / 101.0, 1 / 4.0)
    k, pk, _ = sim.power_spectrum()
    xo, po, _ = O.run(x0, p0, 1 / 101.0, 1 / 4.0, 200, ocfg)
    ko, pko, _ = O.power_spectrum(xo, ocfg)
    sel = slice(0, 16)
    np.testing.assert_allclose(pk[sel], pko[sel], rtol=1e-3)


# ------------------------------------------------------------------ edge cases
def test_single_particle(pm):
    x = np.array([[0.3, 0.7, 0.1]])
    p = np.zeros((1, 3))
    sim, ocfg = make(pm, 0, 16, 1.0, "fp64", x=x, p=p, quantum=False)
    rho = sim.deposit()
    assert rho.sum() == pytest.approx(16 ** 3)
    acc = sim.forces(1.0)
    assert np.abs(acc).max() < 1e-12       # no self-force


def test_all_particles_in_one_cell_and_ragged_tile(pm):
    rng = np.random.default_rng(0)
    n = 5000                               # one full sort tile plus a ragged tail
    x = 0.25 + 0.01 * rng.uniform(size=(n, 3))   # all inside one cell of a 16^3 mesh of L = 1
    p = np.zeros((n, 3))
    sim, ocfg = make(pm, 0, 16, 1.0, "fp32", x=x, p=p)
    cell, ids = sim.get_order()
    assert np.all(cell == cell[0])
    np.testing.assert_array_equal(ids, np.arange(n))      # stable
    xg, _ = sim.get_particles()
    rho = sim.deposit()
    ref = O.cic_deposit(xg, ocfg)
    assert np.abs(rho - ref).max() < 2e-6 * ref.max()


def test_positions_on_faces_and_box_edge(pm):
    n_mesh, box = 16, 1.0
    dx = box / n_mesh
    x = np.array([[0.0, 0.0, 0.0], [dx, 2 * dx, 3 * dx], [box - 1e-12, 0.5, 0.5],
                  [box, 0.25, 0.75], [-1e-9, 0.5, 0.5], [1.5 * box, -0.25, 2.0]])
    p = np.zeros_like(x)
    sim, ocfg = make(pm, 0, n_mesh, box, "fp32", x=x, p=p)
    xg, _ = sim.get_particles()
    assert np.all((xg >= 0) & (xg < box))
    cell, ids = sim.get_order()
    keys = O.cell_key(xg, ocfg)
    np.testing.assert_array_equal(cell, keys[ids])
    u = np.mod(x, box) / dx
    expect = np.mod(np.floor(u + 1e-6), n_mesh)         # fp32 offsets round up to the next face
    np.testing.assert_array_equal(O.cell_index(xg, ocfg), expect.astype(np.int64))


@pytest.mark.parametrize("n_mesh", [24, 40])
def test_non_power_of_two_mesh(pm, n_mesh):
    sim, ocfg = make(pm, n_mesh // 2, n_mesh, 1.0, "fp32", amplitude=4.0)
    acc = sim.forces(0.02)
    xg, _ = sim.get_particles()
    assert rel_rms(acc, O.accelerations(xg, 0.02, ocfg)) < 1e-5


def test_static_mode_lagrangian_energy_conservation(pm):
    """Static run, quantum only: K_v + K_rho conserved to O(dt^2) (fp64 path)."""
    x0, _ = ics.lattice(16, 16, 1.0)
    rng = np.random.default_rng(11)
    x0 = np.mod(x0 + 0.01 * rng.standard_normal(x0.shape), 1.0)
    sim, ocfg = make(pm, 0, 16, 1.0, "fp64", x=x0, p=np.zeros_like(x0), mode="lagrangian", m22=0.05,
                     cosmological=False)
    e0 = sim.energy(0.0)
    es = []
    for i in range(80):
        sim.step(i * 0.05, (i + 1) * 0.05)
        if (i + 1) % 10 == 0:
            es.append(sim.energy((i + 1) * 0.05))
    tot0 = e0[0] + e0[1] + e0[2]
    tots = np.array([e[0] + e[1] + e[2] for e in es])
    assert es[-1][0] > 0.1 * e0[2]
    assert np.abs(tots - tot0).max() < 2e-3 * abs(e0[1] + e0[2])


def test_invalid_arguments_are_reported(pm):
    cfg = pm.make_config(10, 16, 1.0)
    sim = pm.Sim(cfg)
    with pytest.raises(pm.PMError):
        sim.step(0.1, 0.2)                 # no particles yet
    with pytest.raises(pm.PMError):
        sim.power_spectrum(100)            # more bins than N/2
    x = np.full((10, 3), np.nan)
    with pytest.raises(pm.PMError):
        sim.set_particles(x, np.zeros((10, 3)))


# ------------------------------------------------------------------ largest configuration
def test_largest_configuration_256_on_512(pm):
    """256^3 particles on a 512^3 mesh, L = 10 Mpc/h, m22 = 1 (the largest
    single-simulation workload), fp32, hybrid force, in the launch shapes of
    the bench: bit-exact keys and order, full-mesh density, and the
    accelerations of 20,000 sampled particles (the oracle computes the mesh
    fields in full and interpolates at the sample only)."""
    n_side, n_mesh, box, m22 = 256, 512, 10.0, 1.0
    sim, ocfg = make(pm, n_side, n_mesh, box, "fp32", m22=m22, mode="hybrid")
    xg, _ = sim.get_particles()
    cell, ids = sim.get_order()
    keys, order = oracle_order(xg, ocfg, np.arange(len(xg)))
    np.testing.assert_array_equal(ids, order)
    np.testing.assert_array_equal(cell, keys[order])
    del cell, ids, keys, order
    a = 1 / 101.0
    acc = sim.forces(a)
    rho = sim.get_field(pm.FIELD_RHO)
    ref = O.cic_deposit(xg, ocfg)
    assert np.abs(rho - ref).max() < 2e-6 * np.abs(ref).max()
    fields = (ref, O.poisson_phi(ref, ocfg), O.quantum_potential(ref, ocfg))
    del rho
    sample = np.random.default_rng(7).choice(len(xg), 20000, replace=False)
    gphi, gq = O.force_parts(xg[sample], ocfg, fields=fields)
    ref_acc = gphi / a + gq / (a * a)
    assert rel_rms(acc[sample], ref_acc) < 1e-5


def test_energies_after_replayed_graph_steps(pm):
    """pm_run replays its captured steps on later calls; the energies after such
    a call must describe the new state (the replayed stencils skip the K_rho
    sums, so pm_energy has to redo them), as for a fresh simulation there."""
    sim, ocfg = make(pm, 24, 48, 1.0, "fp64", mode="lagrangian", amplitude=4.0)
    a = np.geomspace(1 / 101.0, 1 / 60.0, 9)
    sim.run(4, a[0], a[4])
    sim.energy(a[4])
    sim.run(4, a[4], a[8])                      # the graphs of the first call are reused
    e = sim.energy(a[8])
    x, p = sim.get_particles()
    ref = O.energies(x, p, a[8], ocfg)
    np.testing.assert_allclose(e[:3], ref[:3], rtol=1e-9)


def test_patient_jit_plans_keep_parity(pm):
    """Simulations planned in cuFFT's patient JIT mode (fft_jit) compute the same
    accelerations within the fp32 bar."""
    x, p = ics.zeldovich(32, 64, 1.0, 1 / 101.0, 42, amplitude=4.0)
    cfg = pm.make_config(len(x), 64, 1.0, force_mode=pm.FORCE_HYBRID, fft_jit=True)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    acc = sim.forces(1 / 101.0)
    xg, _ = sim.get_particles()
    ref = O.accelerations(xg, 1 / 101.0, O.Config(n_mesh=64, box=1.0, force_mode=O.HYBRID))
    assert rel_rms(acc, ref) < 1e-5
