"""Continuous batching: requests that arrive while others run are admitted
as memory frees up, run concurrently on their own streams, and each result is
the same as the request run alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00802_gb300 import build
    build.build()
    from paper_1608_00802_gb300 import pm, serve
    return pm, serve


def test_served_results_equal_results_alone(mods):
    pm, serve = mods
    reqs = serve.request_stream(10, rate=200.0, seed=3, sizes=(16, 24, 32), weights=(0.4, 0.3, 0.3),
                                nsteps=24, z_start=50.0, z_end=20.0)
    # a budget of about three of the largest arenas forces queueing and admission as memory frees
    budget = 3 * max(pm.arena_bytes(r.config()) for r in reqs)
    srv = serve.Server(budget, max_slots=8, chunk_steps=5, keep_particles=True)
    res = srv.run(reqs, realtime=True)
    assert srv.stats["admitted"] == len(reqs)
    assert srv.stats["max_active"] >= 2                    # work overlapped on the device
    assert srv.stats["peak_bytes"] <= budget
    for r, out in zip(reqs, res):
        e, k, pk, x, p = serve.run_alone(r, chunk_steps=5)
        np.testing.assert_array_equal(out.x, x)
        np.testing.assert_array_equal(out.p, p)
        np.testing.assert_array_equal(out.energy, e)
        # P(k) bins are summed with fp64 shared-memory atomics (order-dependent at 1 ulp)
        np.testing.assert_allclose(out.pk, pk, rtol=1e-12)
        assert out.finished >= out.admitted >= 0.0


def test_admission_respects_budget_and_fifo(mods):
    pm, serve = mods
    reqs = serve.request_stream(6, rate=1000.0, seed=5, sizes=(16,), weights=(1.0,), nsteps=4,
                                z_start=50.0, z_end=40.0)
    one = pm.arena_bytes(reqs[0].config())
    srv = serve.Server(one, max_slots=4, chunk_steps=2)
    res = srv.run(reqs, realtime=False)
    assert srv.stats["max_active"] == 1                    # only one arena fits
    fin = [r.finished for r in res]
    assert fin == sorted(fin)                              # served in arrival order
    lat = serve.latency_percentiles(res)
    assert lat["p99"] >= lat["p50"] > 0
