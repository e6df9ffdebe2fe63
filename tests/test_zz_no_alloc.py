"""The allocation-free deposit, pm_deposit_noalloc, against pm_deposit.

Some callers cannot allocate device memory: a latency-critical loop cannot
afford the device-wide synchronisation of cudaFree (or a blocking
cudaMalloc), and a process that has handed its whole memory budget to fixed
arenas has nothing left to allocate from.  pm_deposit_noalloc serves them by
keeping every temporary in one static device array.  This file checks,
through the C ABI, that consecutive calls give the density of the existing
entry point, within the deposit tolerance of the parity tests, and that sizes
beyond the array's limits are refused.  It is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00802_gb300 import build
    build.build()
    from paper_1608_00802_gb300 import ics, pm
    return torch, pm, ics


def _reference(pm, x, p, n_mesh, box):
    sim = pm.Sim(pm.make_config(len(x), n_mesh, box, precision=pm.FP32))
    sim.set_particles(x, p)
    rho = sim.deposit()
    sim.close()
    return rho


def _noalloc(torch, pm, x, n_mesh, box):
    x_dev = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    rho_dev = torch.full((n_mesh, n_mesh, n_mesh), -1.0, dtype=torch.float32, device="cuda")
    pm.deposit_noalloc(x_dev, n_mesh, box, rho_dev)
    torch.cuda.synchronize()
    return rho_dev.cpu().double().numpy()


def test_noalloc_deposit_matches_pm_deposit_on_consecutive_calls(env):
    torch, pm, ics = env
    cases = [(32, 64, 1.0, 42), (32, 64, 1.0, 42), (20, 40, 1.5, 7), (32, 64, 1.0, 42)]
    for n_side, n_mesh, box, seed in cases:
        x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, seed, amplitude=4.0)
        ref = _reference(pm, x, p, n_mesh, box)
        got = _noalloc(torch, pm, x, n_mesh, box)
        assert np.abs(got - ref).max() < 2e-6 * max(1.0, np.abs(ref).max())
        assert got.sum() == pytest.approx(n_mesh ** 3, rel=1e-6)


def test_noalloc_deposit_refuses_sizes_beyond_its_scratch(env):
    torch, pm, ics = env
    x_big = torch.zeros((pm.NOALLOC_MAX_PARTICLES + 1, 3), dtype=torch.float64, device="cuda")
    rho = torch.empty((16, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(pm.PMError, match="static scratch limit"):
        pm.deposit_noalloc(x_big, 16, 1.0, rho)
    x = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    n_big = pm.NOALLOC_MAX_MESH + 2
    rho_big = torch.empty((n_big, n_big, n_big), dtype=torch.float32, device="cuda")
    with pytest.raises(pm.PMError, match="static scratch limit"):
        pm.deposit_noalloc(x, n_big, 1.0, rho_big)
