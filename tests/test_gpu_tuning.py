"""Launch shapes and the autotuner: every stencil tile gives the same Q~ bits
as the register-column kernel, the kick and deposit shapes the same states,
and pm_autotune leaves the simulation as it found it."""
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


def _sim(pm, n_side, n_mesh, box, amplitude=8.0, mode=None):
    x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, 42, m22=2.5, amplitude=amplitude)
    cfg = pm.make_config(len(x), n_mesh, box, m22=2.5, force_mode=pm.FORCE_HYBRID if mode is None else mode)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    return sim


def _void_density(n, seed=1):
    """clustered density with empty regions, near-empty nodes and isolated peaks"""
    rng = np.random.default_rng(seed)
    rho = rng.lognormal(0.0, 2.0, size=(n, n, n))
    rho[rng.uniform(size=rho.shape) < 0.35] = 0.0               # empty nodes (floored)
    rho[rng.uniform(size=rho.shape) < 0.05] *= 1e-5              # near-empty, not floored
    rho[: n // 4] = 0.0                                          # a void slab
    return rho * (n ** 3 / rho.sum())


# sweeps (stages 4..8) and one-shot tiles (stages 0), ragged last tiles included
SHAPES = [dict(stencil_rows=r, stencil_planes=z, stencil_stages=s)
          for r, z, s in [(1, 4, 4), (1, 16, 8), (2, 8, 5), (4, 16, 6), (4, 64, 4), (8, 32, 8), (8, 7, 6),
                          (1, 2, 0), (2, 5, 0), (4, 4, 0), (4, 16, 0), (8, 3, 0), (8, 8, 0)]]


@pytest.mark.parametrize("n_mesh", [32, 64, 48])
def test_every_stencil_tile_gives_the_register_column_bits(pm, n_mesh):
    sim = _sim(pm, n_mesh // 2, n_mesh, 1.0)
    rho = _void_density(n_mesh)
    base = sim.get_tuning()
    sim.set_tuning(dict(base, stencil_rows=0))
    sim.set_density(rho)
    q_ref = sim.get_field(pm.FIELD_Q)
    e_ref = sim.energy(1 / 101.0)
    assert np.isfinite(q_ref).all()
    for shape in SHAPES:
        if n_mesh % shape["stencil_rows"] or shape["stencil_planes"] > n_mesh:
            continue
        sim.set_tuning(dict(base, **shape))
        sim.set_density(rho)
        q = sim.get_field(pm.FIELD_Q)
        np.testing.assert_array_equal(q, q_ref, err_msg=str(shape))
        # K_rho is summed in another grouping (float-float per thread, fp64 across)
        assert sim.energy(1 / 101.0)[2] == pytest.approx(e_ref[2], rel=1e-11)


def test_bulk_stencil_matches_oracle_near_empty(pm):
    n = 32
    sim = _sim(pm, 16, n, 1.0)
    rho = _void_density(n, seed=7)
    sim.set_density(rho)
    assert sim.get_tuning()["stencil_rows"] > 0          # the bulk-copy kernel is the default here
    q = sim.get_field(pm.FIELD_Q)
    rho32 = rho.astype(np.float32).astype(np.float64)    # the mesh holds fp32 densities
    ocfg = O.Config(n_mesh=n, box=1.0, m22=2.5)
    ref = O.quantum_potential(rho32, ocfg)
    # fp32 arithmetic (float-float below rho_fp64): a few fp32 ulps of the
    # magnitude of the terms, (hbar/m)^2/2 sum_d (s+ + s- + 2 s) / (dx^2 s)
    s = np.sqrt(np.maximum(rho32, ocfg.rho_floor))
    terms = sum(np.roll(s, 1, a) + np.roll(s, -1, a) + 2 * s for a in range(3)) / s
    scale = 0.5 * O.hbar_over_m(2.5, 0.7) ** 2 / (1.0 / n) ** 2 * terms
    assert np.all(np.abs(q - ref) <= 1e-6 * scale)


def _q_rel_rms(pm, rho, rho_fp64, shape=None):
    n = rho.shape[0]
    cfg = pm.make_config((n // 2) ** 3, n, 1.0, m22=2.5, force_mode=pm.FORCE_HYBRID, rho_fp64=rho_fp64)
    sim = pm.Sim(cfg)
    if shape is not None:
        sim.set_tuning(dict(sim.get_tuning(), **shape))
    sim.set_density(rho)
    q = sim.get_field(pm.FIELD_Q)
    sim.close()
    ref = O.quantum_potential(rho.astype(np.float32).astype(np.float64), O.Config(n_mesh=n, box=1.0, m22=2.5))
    return float(np.sqrt(np.mean((q - ref) ** 2) / np.mean(ref ** 2)))


@pytest.mark.parametrize("shape", [None, dict(stencil_rows=0), dict(stencil_rows=4, stencil_planes=8, stencil_stages=4)],
                         ids=["tiles", "register-columns", "sweep"])
def test_near_empty_branch_keeps_the_digits_fp32_loses(pm, shape):
    """A smooth low-density field (all nodes below rho_fp64): the seven-point
    Laplacian of s cancels to ~1e-5 of s (condition number ~1e5), so the fp32
    formula keeps only a few digits of Q~; the extended-precision branch keeps
    it to about fp32 rounding of Q~ itself.  The one-shot tile kernel
    (default), the register-column kernel and the sweeping tile kernel."""
    n = 32
    z, y, x = np.indices((n, n, n)) * (2 * np.pi / n)
    rho = 1e-3 * (1.0 + 1e-3 * (np.sin(x) + np.cos(2 * y + 0.4) + np.sin(z + 0.3)))
    extended = _q_rel_rms(pm, rho, 1e-2, shape)
    plain = _q_rel_rms(pm, rho, 0.0, shape)
    assert extended < 1e-6
    assert plain > 100 * extended    # the control: the same field without the branch


def test_kick_and_deposit_shapes_give_identical_states(pm):
    ref = None
    for kt, dw in [(256, 8), (128, 2), (128, 8), (256, 1)]:
        sim = _sim(pm, 24, 48, 1.0, amplitude=4.0)
        sim.set_tuning(dict(sim.get_tuning(), kick_threads=kt, deposit_warps=dw))
        sim.run(4, 1 / 101.0, 1 / 80.0)
        x, p = sim.get_particles()
        rho = sim.get_field(pm.FIELD_RHO)
        if ref is None:
            ref = (x, p, rho)
        else:
            np.testing.assert_array_equal(x, ref[0])
            np.testing.assert_array_equal(p, ref[1])
            np.testing.assert_array_equal(rho, ref[2])


def test_autotune_keeps_state_and_fields(pm):
    sim = _sim(pm, 32, 64, 1.0)
    sim.run(3, 1 / 101.0, 1 / 90.0)
    x0, p0 = sim.get_particles()
    q0 = sim.get_field(pm.FIELD_Q)
    cache = pm.TuningCache()
    t = sim.autotune(reps=2, cache=cache)
    assert t == sim.get_tuning() and pm.tuning_key(sim.cfg) in cache
    x1, p1 = sim.get_particles()
    np.testing.assert_array_equal(x0, x1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(sim.get_field(pm.FIELD_Q), q0)
    # a second simulation of the same configuration takes the cached shapes
    other = _sim(pm, 32, 64, 1.0)
    assert other.autotune(cache=cache) == t and other.get_tuning() == t
    # and steps on with them exactly like the first one would with its defaults
    sim.run(2, 1 / 90.0, 1 / 85.0)
    ref = _sim(pm, 32, 64, 1.0)
    ref.run(3, 1 / 101.0, 1 / 90.0)
    ref.run(2, 1 / 90.0, 1 / 85.0)
    np.testing.assert_array_equal(sim.get_particles()[0], ref.get_particles()[0])


def test_invalid_shapes_are_refused(pm):
    sim = _sim(pm, 8, 16, 1.0)
    base = sim.get_tuning()
    for bad in [dict(stencil_rows=3), dict(stencil_rows=32), dict(stencil_rows=4, stencil_planes=2, stencil_stages=6),
                dict(stencil_rows=4, stencil_planes=1, stencil_stages=0),
                dict(stencil_rows=4, stencil_planes=17, stencil_stages=0),
                dict(stencil_rows=4, stencil_planes=8, stencil_stages=9),
                dict(stencil_rows=4, stencil_planes=8, stencil_stages=2), dict(kick_threads=64),
                dict(deposit_warps=0), dict(deposit_warps=9)]:
        with pytest.raises(pm.PMError) as e:
            sim.set_tuning(dict(base, **bad))
        assert e.value.status == 1
    assert sim.get_tuning() == base


def test_mesh_not_a_multiple_of_four_uses_the_register_column_kernel(pm):
    sim = _sim(pm, 7, 14, 1.0)
    assert sim.get_tuning()["stencil_rows"] == 0
    with pytest.raises(pm.PMError):
        sim.set_tuning(dict(sim.get_tuning(), stencil_rows=2, stencil_planes=7, stencil_stages=4))
