"""The Green multiplication inside the z transform (pm_tuning's green_fused):
batched 2D transforms of the z planes, and between them one kernel that
transforms each column of the half spectrum along z, multiplies by the Green's
function phi^ = G rho^ (Sec. II, the exact inverse of the seven-point
Laplacian, k = 0 removed) and transforms back.  The potential must match the
oracle's Poisson solve and the 3D-transform path; W_g, summed by the same
kernel over the spectrum, must match the oracle's energy.  Every factorisation
of the z transform is covered: N = 16 (4 x 4), 32 (8 x 4), 64 (8 x 8), 128
(16 x 8), 256 (16 x 16), 512 (32 x 16)."""
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


def _sim(pm, n_side, n_mesh, box=1.0, seed=42, fused=None, **kw):
    x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, seed, amplitude=4.0)
    cfg = pm.make_config(len(x), n_mesh, box, force_mode=pm.FORCE_HYBRID, **kw)
    sim = pm.Sim(cfg)
    sim.set_particles(x, p)
    if fused is not None:
        sim.set_tuning({"green_fused": int(fused)})
    return sim, x, p


def test_fused_by_default_where_it_applies(pm):
    """On by default for fp32 cloud-in-cell power-of-two meshes from 128^3 up;
    smaller ones keep the 3D transforms (and take it through pm_set_tuning)."""
    cases = [((32, 128), {}, 1), ((8, 16), {}, 0), ((32, 64), {}, 0), ((24, 48), {}, 0), ((8, 8), {}, 0),
             ((16, 128), {"precision": pm.FP64}, 0), ((16, 128), {"kernel": pm.KERNEL_SPLINE}, 0)]
    for (n_side, n_mesh), kw, want in cases:
        sim, _, _ = _sim(pm, n_side, n_mesh, **kw)
        assert sim.get_tuning()["green_fused"] == want, (n_side, n_mesh, kw)
        sim.close()


def test_fused_refused_where_it_does_not_apply(pm):
    for n_mesh, kw in ((32, {"precision": pm.FP64}), (32, {"kernel": pm.KERNEL_SPLINE}), (48, {})):
        sim, _, _ = _sim(pm, 16, n_mesh, **kw)
        with pytest.raises(pm.PMError, match="green_fused"):
            sim.set_tuning({"green_fused": 1})
        sim.close()


@pytest.mark.parametrize("n_side,n_mesh,box", [(8, 16, 0.7), (16, 32, 1.3), (32, 64, 1.0), (64, 128, 2.0),
                                               (64, 256, 2.0)])
def test_fused_potential_matches_oracle_and_3d_path(pm, n_side, n_mesh, box):
    """The potential of the fused path against the oracle's Poisson solve of
    the same density (fp32 bar 2e-6 of the largest |phi|), and against the 3D
    transforms with the separate Green pass within fp32 rounding."""
    sim, _, _ = _sim(pm, n_side, n_mesh, box, fused=1)
    sim.forces(1 / 101.0)
    rho = sim.get_field(pm.FIELD_RHO)
    phi = sim.get_field(pm.FIELD_PHI)
    ref = O.poisson_phi(rho, O.Config(n_mesh=n_mesh, box=box))
    assert np.abs(phi - ref).max() < 2e-6 * np.abs(ref).max()
    sim.set_tuning({"green_fused": 0})
    sim.forces(1 / 101.0)
    phi0 = sim.get_field(pm.FIELD_PHI)
    np.testing.assert_array_equal(sim.get_field(pm.FIELD_RHO), rho)
    assert np.abs(phi - phi0).max() <= 1e-6 * np.abs(phi0).max()
    sim.close()


def test_fused_potential_512_follows_3d_path(pm):
    """N = 512 (32 x 16 columns), where the oracle's solve is too slow for a
    test: against the 3D-transform path (pinned to the oracle by the parity
    tests) within fp32 rounding."""
    sim, _, _ = _sim(pm, 64, 512, 4.0, fused=1)
    sim.forces(1 / 101.0)
    phi = sim.get_field(pm.FIELD_PHI)
    sim.set_tuning({"green_fused": 0})
    sim.forces(1 / 101.0)
    phi0 = sim.get_field(pm.FIELD_PHI)
    assert np.abs(phi - phi0).max() <= 1e-6 * np.abs(phi0).max()
    sim.close()


@pytest.mark.parametrize("n_mesh", [64, 512])
def test_fused_potential_of_plane_waves_in_closed_form(pm, n_mesh):
    """rho = 1 + sum_w A_w cos(2 pi k_w . n / N) on the nodes n: the seven-point
    Poisson equation of Sec. II has the exact solution
    phi = -(3/2) Omega_m dx^2 / 4 * sum_w A_w cos(2 pi k_w . n / N) / sum_d sin^2(pi k_wd / N)
    (a fixed point of the discrete Laplacian).  Waves with a large k_z, the x
    Nyquist index and mixed components reach every twiddle of both factors."""
    N, box = n_mesh, 2.0
    waves = [((3, 5, N // 2 - 9), 0.3), ((N // 2, 0, 7), 0.2), ((1, N - 2, N - 3), 0.1)]
    n = np.arange(N, dtype=np.float64)
    z, y, x = np.meshgrid(n, n, n, indexing="ij")
    rho = np.ones((N, N, N))
    ref = np.zeros((N, N, N))
    dx = box / N
    for (kx, ky, kz), amp in waves:
        c = np.cos(2 * np.pi * (kx * x + ky * y + kz * z) / N)
        s = sum(np.sin(np.pi * k / N) ** 2 for k in (kx, ky, kz))
        rho += amp * c
        ref += -1.5 * 0.3 * dx * dx / 4.0 * amp * c / s
    cfg = pm.make_config(8, N, box, force_mode=pm.FORCE_HYBRID)
    sim = pm.Sim(cfg)
    sim.set_tuning({"green_fused": 1})
    x0 = np.random.default_rng(1).random((8, 3)) * box
    sim.set_particles(x0, np.zeros((8, 3)))
    sim.set_density(rho)
    phi = sim.get_field(pm.FIELD_PHI)
    assert np.abs(phi - ref).max() < 2e-6 * np.abs(ref).max()
    sim.close()


def test_fused_energies_match_oracle(pm):
    """W_g, summed over the half spectrum by the z kernel (one partial per
    tile of columns), against the oracle's energies after a step, at the fp32
    bar."""
    sim, _, _ = _sim(pm, 32, 64, fused=1)
    a = 1 / 99.0
    sim.step(1 / 101.0, a)
    e = sim.energy(a)
    xg, pg = sim.get_particles()
    ref = np.array(O.energies(xg, pg, a, O.Config(n_mesh=64, box=1.0, force_mode=O.HYBRID)))
    for k in range(3):
        assert e[k] == pytest.approx(ref[k], rel=1e-5)
    sim.close()


@pytest.mark.parametrize("quantum,nsteps", [(False, 8), (True, 2)])
def test_fused_runs_follow_the_separate_pass(pm, quantum, nsteps):
    """Captured steps, 64^3 particles on 128^3, with and without the fusion:
    the transforms round differently, so the states agree to fp32 rounding
    (1e-4 of a cell, momenta and energies 1e-5).  With the quantum force on
    this mesh of eight cells per particle the run is chaotic (a rounding
    difference in the first step sends single particles apart within a few
    steps, as moving every position by one fp32 ulp does in fp64), so that
    case is compared over two steps."""
    a0 = 1 / 101.0
    a1 = a0 * (1.25 if nsteps > 2 else 1.03)
    out = []
    for fused in (1, 0):
        sim, _, _ = _sim(pm, 64, 128, fused=fused, quantum=quantum)
        sim.run(nsteps, a0, a1)
        x, p = sim.get_particles()
        out.append((x, p, sim.energy(a1)))
        sim.close()
    d = out[0][0] - out[1][0]
    d -= np.round(d)
    assert np.abs(d).max() < 1e-4 / 128
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-5 * np.abs(out[1][1]).max()
    np.testing.assert_allclose(out[0][2][:3], out[1][2][:3], rtol=1e-5, atol=1e-12)


def test_packed_batch_class_with_the_fusion_equals_single_runs(pm):
    """Three members of one configuration class on 128^3 (different boxes,
    masses and seeds) stepped by packed launches: each member's own 2D
    transforms and one z kernel over the class, so every member ends on the
    bits of the same simulation run alone."""
    members = [(32, 128, 1.0, 2.5, 20), (32, 128, 2.0, 10.0, 21), (32, 128, 3.0, 1.0, 22)]
    a0 = 1 / 101.0
    a1 = np.array([1 / 90.0, 1 / 85.0, 1 / 95.0])
    cfgs = [pm.make_config(n ** 3, N, box, m22=m22, force_mode=pm.FORCE_HYBRID) for n, N, box, m22, _ in members]
    batch = pm.Batch(cfgs)
    ics_ = [ics.zeldovich(n, N, box, a0, seed, m22=m22, amplitude=2.0) for n, N, box, m22, seed in members]
    for mem, (x, p) in zip(batch.members, ics_):
        mem.set_particles(x, p)
    batch.run(4, a0, a1)
    assert batch.info() == (1, 3)
    for i, cfg in enumerate(cfgs):
        assert batch.members[i].get_tuning()["green_fused"] == 1
        xb, pb = batch.members[i].get_particles()
        eb = batch.members[i].energy(a1[i])
        single = pm.Sim(cfg)
        single.set_particles(*ics_[i])
        single.run(4, a0, a1[i])
        xs, ps = single.get_particles()
        es = single.energy(a1[i])
        single.close()
        np.testing.assert_array_equal(xb, xs)
        np.testing.assert_array_equal(pb, ps)
        np.testing.assert_allclose(eb, es, rtol=1e-12)
    batch.close()
