"""The allocation-free deposit, pm_deposit_noalloc.

Some callers cannot allocate device memory: a latency-critical loop cannot
afford the device-wide synchronisation of cudaFree (or a blocking
cudaMalloc), and a process that has handed its whole memory budget to fixed
arenas has nothing left to allocate from.  pm_deposit_noalloc serves them by
keeping every temporary in one static device array.  This file checks,
through the C ABI, that consecutive calls give the same bits as the existing
entry point pm_deposit (both run the same conversion, sort and gather on the
same positions), that a call at the stated limits (65536 particles on a 128^3
mesh) matches the oracle's direct scatter, that the device error word reaches
the caller, and that sizes beyond the limits are refused.  It is collected
last on purpose.
"""
import numpy as np
import pytest

from oracle import pm_oracle as O

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
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    pm.deposit_noalloc(x_dev, n_mesh, box, rho_dev, err_dev=err)
    torch.cuda.synchronize()
    return rho_dev.cpu().numpy(), int(err.item())


def test_noalloc_deposit_equals_pm_deposit_on_consecutive_calls(env):
    torch, pm, ics = env
    cases = [(32, 64, 1.0, 42), (32, 64, 1.0, 42), (20, 40, 1.5, 7), (32, 64, 1.0, 42)]
    for n_side, n_mesh, box, seed in cases:
        x, p = ics.zeldovich(n_side, n_mesh, box, 1 / 101.0, seed, amplitude=4.0)
        ref = _reference(pm, x, p, n_mesh, box)
        got, err = _noalloc(torch, pm, x, n_mesh, box)
        assert err == 0
        np.testing.assert_array_equal(got, ref.astype(np.float32))
        assert got.astype(np.float64).sum() == pytest.approx(n_mesh ** 3, rel=1e-6)


def test_noalloc_deposit_at_its_limits_matches_the_oracle(env):
    """65536 particles on a 128^3 mesh (both limits), after a smaller call has
    left its contents in the array: the direct scatter of Eq. (rhodis) in fp64
    on the same positions (cells and fp32 offsets exact in double, dx = 2^-7),
    within the fp32 deposit tolerance of the parity tests."""
    torch, pm, ics = env
    n, N, box = pm.NOALLOC_MAX_PARTICLES, pm.NOALLOC_MAX_MESH, 1.0
    rng = np.random.default_rng(11)
    # clustered: half the particles in a small clump, so that rows hold long runs of one cell
    cells = rng.integers(0, N, size=(n, 3))
    cells[: n // 2] = rng.integers(56, 64, size=(n // 2, 3))
    off = rng.random((n, 3)).astype(np.float32).astype(np.float64)
    x = (cells + off) * (box / N)
    for warm in (8, 96):  # a call on another size first: the array keeps its contents
        xs = x[: 1000] * 0.5
        _noalloc(torch, pm, xs, warm, 0.5)
    got, err = _noalloc(torch, pm, x, N, box)
    assert err == 0
    ref = O.cic_deposit(x, O.Config(n_mesh=N, box=box))
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()
    assert got.astype(np.float64).sum() == pytest.approx(N ** 3, rel=1e-6)


def test_noalloc_deposit_reports_nonfinite_positions(env):
    """A NaN position is placed at 0 and bit 0 of the error word reaches the
    caller's device word; the next clean call reports 0 again."""
    torch, pm, ics = env
    x, p = ics.zeldovich(16, 32, 1.0, 1 / 101.0, 3, amplitude=4.0)
    bad = x.copy()
    bad[5, 1] = np.nan
    _, err = _noalloc(torch, pm, bad, 32, 1.0)
    assert err == 1
    got, err = _noalloc(torch, pm, x, 32, 1.0)
    assert err == 0
    np.testing.assert_array_equal(got, _reference(pm, x, p, 32, 1.0).astype(np.float32))


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
