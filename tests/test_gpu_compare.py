"""The FDM-versus-pressureless comparison (same initial conditions, quantum
pressure on and off): the GPU pair against the oracle pair, and the limits
the comparison must reach."""
import math

import numpy as np
import pytest

from oracle import pm_oracle as O
from paper_1608_00802_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_00802_gb300 import build
    build.build()
    from paper_1608_00802_gb300 import compare, pm
    return pm, compare


def test_pair_matches_oracle_pair(mods):
    pm, compare = mods
    n_side, n_mesh, box, m22, nsteps = 16, 32, 1.0, 2.5, 24
    z0, z1 = 100.0, 20.0
    out = compare.run_pair(n_side, n_mesh, box, m22, z0, z1, nsteps, z_out=(z1,))
    r = out[0]
    # the oracle from the same (quantised) initial particles
    x, p = ics.zeldovich(n_side, n_mesh, box, 1 / (1 + z0), 42, m22=m22)
    q = pm.Sim(pm.make_config(len(x), n_mesh, box, m22=m22, force_mode=pm.FORCE_HYBRID))
    q.set_particles(x, p)
    xq, pq = q.get_particles()
    q.close()
    res = {}
    for name, quantum in (("fdm", True), ("cdm", False)):
        cfg = O.Config(n_mesh=n_mesh, box=box, m22=m22, force_mode=O.HYBRID, quantum=quantum)
        xo, _ = O.run(xq.copy(), pq.copy(), 1 / (1 + z0), 1 / (1 + z1), nsteps, cfg)[:2]
        res[name] = (O.power_spectrum(xo, cfg), O.cic_deposit(xo, cfg))
    (k_o, pf_o, _), rf_o = res["fdm"]
    (_, pc_o, _), rc_o = res["cdm"]
    sel = k_o <= 0.5 * math.pi * n_mesh / box
    rel_o = (pf_o - pc_o) / pc_o
    np.testing.assert_allclose(r["k"], k_o, rtol=1e-12)
    assert np.all(np.abs(r["rel_dP"][sel] - rel_o[sel]) <= 2e-4 + 0.02 * np.abs(rel_o[sel]))
    pos = rc_o > 0
    rms_o = float(np.sqrt(np.mean(((rf_o[pos] - rc_o[pos]) / rc_o[pos]) ** 2)))
    assert r["rms_rel_density"] == pytest.approx(rms_o, rel=0.02, abs=1e-5)
    # the quantum pressure did act: a measurable difference, largest at small scales
    assert np.abs(rel_o[sel]).max() > 1e-4
    assert abs(rel_o[0]) < np.abs(rel_o[sel]).max()


def test_heavy_axion_limit_has_no_difference(mods):
    # hbar/m -> 0: Q ~ (hbar/m)^2 vanishes, the two runs agree to rounding
    pm, compare = mods
    out = compare.run_pair(16, 32, 1.0, 1e8, 100.0, 20.0, 16, z_out=(20.0,))
    assert np.abs(out[0]["rel_dP"]).max() < 1e-5
    assert out[0]["rms_rel_density"] < 1e-5


def test_jeans_wavenumber(mods):
    pm, compare = mods
    # k_J(a = 1) for m22 = 2.5, h = 0.7: (1.8)^(1/4) / sqrt(1.91715e-4 h / m22)
    hbm = 1.91715e-4 * 0.7 / 2.5
    assert compare.jeans_k(1.0, 2.5) == pytest.approx(1.8 ** 0.25 / math.sqrt(hbm), rel=1e-5)
    assert compare.jeans_k(1.0, 2.5) == pytest.approx(O.jeans_k(1.0, 0.3, O.hbar_over_m(2.5, 0.7)), rel=1e-12)
