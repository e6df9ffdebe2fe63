"""The fused x-y transform kernels of 256^3 fp32 meshes (pm_tuning's
green_fused = 2): one cluster of eight CTAs per z-plane does the real x
transform of the plane's rows, exchanges them through distributed shared
memory and transforms the columns along y, in place of the batched 2D cuFFT
R2C (and the same backwards for the C2R).  Between them the z kernel applies
the Green's function of Sec. II.  The potential must match the oracle's
Poisson solve, the closed form of plane waves (the x = 0 and x = N/2 columns
travel packed as one complex column, so waves on them are included), and the
cuFFT path within fp32 rounding; packed batch members must end on the bits of
their single runs."""
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
    sim = pm.Sim(pm.make_config(len(x), n_mesh, box, force_mode=pm.FORCE_HYBRID, **kw))
    sim.set_particles(x, p)
    if fused is not None:
        sim.set_tuning({"green_fused": int(fused)})
    return sim


def test_default_on_256_and_refused_elsewhere(pm):
    sim = _sim(pm, 16, 256, 2.0)
    assert sim.get_tuning()["green_fused"] == 2
    sim.close()
    for n_mesh in (128, 512):
        sim = _sim(pm, 16, n_mesh, 2.0)
        assert sim.get_tuning()["green_fused"] == 1
        with pytest.raises(pm.PMError, match="256"):
            sim.set_tuning({"green_fused": 2})
        sim.close()


def test_potential_matches_oracle_and_cufft_path(pm):
    """64^3 particles on 256^3 (L = 2): against the oracle's Poisson solve of
    the same density (fp32 bar 2e-6 of the largest |phi|) and against the
    batched 2D cuFFT transforms (green_fused = 1) within fp32 rounding."""
    sim = _sim(pm, 64, 256, 2.0, fused=2)
    sim.forces(1 / 101.0)
    rho = sim.get_field(pm.FIELD_RHO)
    phi = sim.get_field(pm.FIELD_PHI)
    ref = O.poisson_phi(rho, O.Config(n_mesh=256, box=2.0))
    assert np.abs(phi - ref).max() < 2e-6 * np.abs(ref).max()
    sim.set_tuning({"green_fused": 1})
    sim.forces(1 / 101.0)
    phi1 = sim.get_field(pm.FIELD_PHI)
    np.testing.assert_array_equal(sim.get_field(pm.FIELD_RHO), rho)
    assert np.abs(phi - phi1).max() <= 1e-6 * np.abs(phi1).max()
    sim.close()


def test_plane_waves_in_closed_form(pm):
    """rho = 1 + sum_w A_w cos(2 pi k_w . n / N): the seven-point Poisson
    equation has the exact solution
    phi = -(3/2) Omega_m dx^2 / 4 * sum_w A_w cos(2 pi k_w . n / N) / sum_d sin^2(pi k_wd / N).
    The waves sit on the packed columns (k_x = 0 and k_x = N/2, with k_y and
    its mirror), on each CTA's range of columns and at the y Nyquist index."""
    N, box = 256, 2.0
    waves = [((0, 5, 9), 0.3), ((N // 2, 0, 7), 0.2), ((N // 2, 3, 0), 0.15), ((0, N // 2, 1), 0.1),
             ((1, N - 2, N - 3), 0.1), ((33, 64, 5), 0.05), ((70, 17, 100), 0.05), ((127, 200, 128), 0.05)]
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
    sim = pm.Sim(pm.make_config(8, N, box, force_mode=pm.FORCE_HYBRID))
    assert sim.get_tuning()["green_fused"] == 2
    sim.set_particles(np.random.default_rng(1).random((8, 3)) * box, np.zeros((8, 3)))
    sim.set_density(rho)
    phi = sim.get_field(pm.FIELD_PHI)
    assert np.abs(phi - ref).max() < 2e-6 * np.abs(ref).max()
    sim.close()


def test_steps_follow_the_cufft_path(pm):
    """Two captured steps of 64^3 particles on 256^3 with the quantum force:
    the transforms round differently, so the states agree to fp32 rounding."""
    a0, a1 = 1 / 101.0, 1 / 98.0
    out = []
    for fused in (2, 1):
        sim = _sim(pm, 64, 256, 2.0, fused=fused)
        sim.run(2, a0, a1)
        x, p = sim.get_particles()
        out.append((x, p, sim.energy(a1)))
        sim.close()
    d = out[0][0] - out[1][0]
    d -= np.round(d / 2.0) * 2.0
    assert np.abs(d).max() < 1e-4 * 2.0 / 256
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-5 * np.abs(out[1][1]).max()
    np.testing.assert_allclose(out[0][2][:3], out[1][2][:3], rtol=1e-5, atol=1e-12)


def test_packed_batch_members_equal_single_runs(pm):
    """Two members of one class on 256^3 stepped by packed launches (one x-y
    kernel launch over both members' planes per direction) end on the bits of
    the same simulations run alone."""
    members = [(32, 256, 2.0, 2.5, 30), (32, 256, 3.0, 5.0, 31)]
    a0 = 1 / 101.0
    a1 = np.array([1 / 95.0, 1 / 97.0])
    cfgs = [pm.make_config(n ** 3, N, box, m22=m22, force_mode=pm.FORCE_HYBRID) for n, N, box, m22, _ in members]
    batch = pm.Batch(cfgs)
    ics_ = [ics.zeldovich(n, N, box, a0, seed, m22=m22, amplitude=2.0) for n, N, box, m22, seed in members]
    for mem, (x, p) in zip(batch.members, ics_):
        mem.set_particles(x, p)
    batch.run(3, a0, a1)
    assert batch.info() == (1, 2)
    for i, cfg in enumerate(cfgs):
        assert batch.members[i].get_tuning()["green_fused"] == 2
        xb, pb = batch.members[i].get_particles()
        single = pm.Sim(cfg)
        single.set_particles(*ics_[i])
        single.run(3, a0, a1[i])
        xs, ps = single.get_particles()
        single.close()
        np.testing.assert_array_equal(xb, xs)
        np.testing.assert_array_equal(pb, ps)
    batch.close()
