"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, brute force on tiny meshes, invariants, special cases, or physical
constants from an independent source.  No GPU needed.
"""
import math
import os

import numpy as np
import pytest

from oracle import pm_oracle as O
from paper_1608_00802_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "constants.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _rand_particles(rng, npart, box):
    return rng.uniform(0.0, box, size=(npart, 3))


# ---------------------------------------------------------------- units
def test_hbar_over_m_from_independent_constants():
    """hbar/m in (Mpc/h)^2 H0 recomputed from hbar [J s], the eV and c, and the
    parsec from the au (IAU 2015), against the oracle's hbar*c route."""
    g = _golden_constants()
    h = g["H0_paper_km_s_Mpc"] / 100.0
    m_kg = g["m22_paper"] * 1e-22 * g["eV_J"] / g["c_m_s"] ** 2
    hbar_m = g["hbar_J_s"] / m_kg                       # m^2/s
    mpc = 1e6 * 648000.0 / math.pi * g["au_m"]
    unit = (mpc / h) ** 2 * (100.0 * h * 1e3 / mpc)      # (Mpc/h)^2 * H0 in m^2/s
    expect = hbar_m / unit
    assert O.hbar_over_m(g["m22_paper"], h) == pytest.approx(expect, rel=1e-8)


def test_jeans_scale_from_si_units():
    """Eq. (jeansscale) evaluated in SI units (G, rho_crit from H0) equals the
    oracle's code-unit form."""
    g = _golden_constants()
    h, om, m22 = 0.7, 0.3, 2.5
    h0 = 100.0 * h * 1e3 / (1e6 * 648000.0 / math.pi * g["au_m"])  # 1/s
    rho_m0 = om * 3.0 * h0 ** 2 / (8.0 * math.pi * g["G_m3_kg_s2"])   # comoving mean, kg/m^3
    m_kg = m22 * 1e-22 * g["eV_J"] / g["c_m_s"] ** 2
    mpc = 1e6 * 648000.0 / math.pi * g["au_m"]
    for a in (0.01, 0.3, 1.0):
        kj = (2.0 * math.pi ** 0.25 * a ** 0.25 * (g["G_m3_kg_s2"] * rho_m0) ** 0.25
              * (m_kg / g["hbar_J_s"]) ** 0.5)          # 1/m comoving
        kj_hmpc = kj * mpc / h
        assert O.jeans_k(a, om, O.hbar_over_m(m22, h)) == pytest.approx(kj_hmpc, rel=1e-8)


# ---------------------------------------------------------------- time weights
def test_time_weights_einstein_de_sitter_closed_form():
    cfg = O.Config(n_mesh=8, box=1.0, omega_m=1.0, omega_l=0.0)
    for a0, a1 in [(0.01, 0.0123), (0.2, 0.9), (0.5, 1.0)]:
        assert O.kick_factor(a0, a1, cfg) == pytest.approx(2 * (math.sqrt(a1) - math.sqrt(a0)), rel=1e-13)
        assert O.drift_factor(a0, a1, cfg) == pytest.approx(2 * (1 / math.sqrt(a0) - 1 / math.sqrt(a1)), rel=1e-13)


def test_time_weights_lcdm_against_adaptive_quadrature():
    from scipy.integrate import quad
    cfg = O.Config(n_mesh=8, box=1.0)
    hz = lambda a: math.sqrt(0.3 / a ** 3 + 0.7)
    for a0, a1 in [(1 / 101, 1 / 100), (0.05, 0.25)]:
        kg = quad(lambda a: 1 / (a * a * hz(a)), a0, a1, epsabs=0, epsrel=1e-13)[0]
        kd = quad(lambda a: 1 / (a ** 3 * hz(a)), a0, a1, epsabs=0, epsrel=1e-13)[0]
        assert O.kick_factor(a0, a1, cfg) == pytest.approx(kg, rel=1e-12)
        assert O.drift_factor(a0, a1, cfg) == pytest.approx(kd, rel=1e-12)


def test_static_mode_weights_are_elapsed_time():
    cfg = O.Config(n_mesh=8, box=1.0, cosmological=False)
    assert O.kick_factor(1.0, 1.5, cfg) == 0.5
    assert O.drift_factor(2.0, 2.25, cfg) == 0.25
    assert O.half_point(1.0, 2.0, cfg) == 1.5


# ---------------------------------------------------------------- keys and order
def test_keys_and_stable_order_brute_force():
    rng = np.random.default_rng(1)
    cfg = O.Config(n_mesh=8, box=2.0)
    x = _rand_particles(rng, 300, cfg.box)
    x[:40] = x[40:80]                      # duplicates -> equal keys
    keys = O.cell_key(x, cfg)
    for i in range(len(x)):
        c = [int(math.floor(x[i, d] / cfg.dx)) for d in range(3)]
        assert keys[i] == (c[2] * 8 + c[1]) * 8 + c[0]
    order = O.stable_cell_order(keys)
    brute = sorted(range(len(x)), key=lambda i: (keys[i], i))
    assert list(order) == brute


# ---------------------------------------------------------------- deposit
def test_cic_deposit_equals_direct_sum_8cubed():
    """Every particle x every node, tent weights with the minimum image."""
    rng = np.random.default_rng(2)
    cfg = O.Config(n_mesh=8, box=1.0)
    x = _rand_particles(rng, 57, cfg.box)
    rho = O.cic_deposit(x, cfg)
    n, dx, box = cfg.n_mesh, cfg.dx, cfg.box
    mp = box ** 3 / len(x)
    brute = np.zeros((n, n, n))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                node = np.array([ix, iy, iz]) * dx
                d = x - node
                d -= box * np.round(d / box)
                w = np.prod(np.maximum(0.0, 1.0 - np.abs(d) / dx), axis=1)
                brute[iz, iy, ix] = mp * w.sum() / dx ** 3
    np.testing.assert_allclose(rho, brute, rtol=0, atol=1e-12)
    assert rho.sum() * dx ** 3 == pytest.approx(box ** 3, rel=1e-13)


def test_unperturbed_lattice_gives_uniform_density():
    for npart, nmesh in [(4, 8), (8, 8), (8, 16)]:
        cfg = O.Config(n_mesh=nmesh, box=3.0)
        x, _ = ics.lattice(npart, nmesh, cfg.box)
        np.testing.assert_allclose(O.cic_deposit(x, cfg), 1.0, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- gravity
def _dft3_bruteforce(f):
    n = f.shape[0]
    idx = np.arange(n)
    out = np.zeros(f.shape, dtype=complex)
    grid = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), axis=-1).reshape(-1, 3)
    vals = f.reshape(-1)
    for kz in range(n):
        for ky in range(n):
            for kx in range(n):
                ph = np.exp(-2j * np.pi * (grid @ np.array([kz, ky, kx])) / n)
                out[kz, ky, kx] = np.sum(vals * ph)
    return out


def test_poisson_matches_bruteforce_dft_8cubed():
    rng = np.random.default_rng(3)
    cfg = O.Config(n_mesh=8, box=1.5, omega_m=0.3)
    rho = 1.0 + 0.3 * rng.standard_normal((8, 8, 8))
    phi = O.poisson_phi(rho, cfg)
    rk = _dft3_bruteforce(rho - 1.0)
    n, dx = 8, cfg.dx
    phik = np.zeros_like(rk)
    for kz in range(n):
        for ky in range(n):
            for kx in range(n):
                if kx == ky == kz == 0:
                    continue
                kap2 = sum((2 / dx * math.sin(math.pi * m / n)) ** 2 for m in (kx, ky, kz))
                phik[kz, ky, kx] = -1.5 * cfg.omega_m * rk[kz, ky, kx] / kap2
    # inverse by brute force: conj trick
    phi_b = np.real(np.conj(_dft3_bruteforce(np.conj(phik)))) / n ** 3
    np.testing.assert_allclose(phi, phi_b, rtol=0, atol=1e-12)


def test_poisson_residual_of_seven_point_operator():
    """Applying the seven-point stencil to phi~ returns (3/2) Om (rho - mean)."""
    rng = np.random.default_rng(4)
    cfg = O.Config(n_mesh=16, box=2.0, omega_m=0.3)
    rho = np.exp(0.5 * rng.standard_normal((16, 16, 16)))
    phi = O.poisson_phi(rho, cfg)
    dx = cfg.dx
    lap = sum(np.roll(phi, 1, a) + np.roll(phi, -1, a) for a in range(3)) - 6 * phi
    lap /= dx * dx
    np.testing.assert_allclose(lap, 1.5 * cfg.omega_m * (rho - rho.mean()), rtol=0, atol=1e-10)
    assert abs(phi.mean()) < 1e-14


def test_gravity_momentum_conservation_and_no_self_force():
    rng = np.random.default_rng(5)
    cfg = O.Config(n_mesh=16, box=1.0, quantum=False)
    x = _rand_particles(rng, 200, cfg.box)
    gphi, gq = O.force_parts(x, cfg)
    assert np.abs(gq).max() == 0.0
    scale = np.abs(gphi).max()
    assert np.abs(gphi.sum(axis=0)).max() < 1e-11 * scale * len(x)
    one = rng.uniform(0, 1, size=(1, 3))
    g1, _ = O.force_parts(one, cfg)
    assert np.abs(g1).max() < 1e-12


def test_two_particles_attract():
    cfg = O.Config(n_mesh=32, box=1.0, quantum=False)
    x = np.array([[0.40, 0.5, 0.5], [0.60, 0.5, 0.5]])
    g, _ = O.force_parts(x, cfg)
    assert g[0, 0] > 0 and g[1, 0] < 0
    assert g[0, 0] == pytest.approx(-g[1, 0], rel=1e-12)


# ---------------------------------------------------------------- quantum pressure
def _gaussian_rho(n, box, sigma):
    dx = box / n
    c = (np.arange(n) - n // 2) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = x * x + y * y + z * z
    return np.exp(-r2 / (2 * sigma ** 2)), (x, y, z), dx


def test_gaussian_q_discrete_closed_form():
    """rho = exp(-r^2/2 sigma^2): s = prod_d g(x_d), g = exp(-x^2/4 sigma^2), so
    the compact stencil gives lap7(s)/s = sum_d [g(x+dx)+g(x-dx)-2g(x)]/(dx^2 g(x))
    = sum_d [exp(-(2x dx + dx^2)/4s2) + exp((2x dx - dx^2)/4s2) - 2]/dx^2 exactly."""
    n, box, sigma = 32, 1.0, 0.09
    cfg = O.Config(n_mesh=n, box=box, m22=2.5, h=0.7, rho_floor=1e-300)
    rho, (x, y, z), dx = _gaussian_rho(n, box, sigma)
    q = O.quantum_potential(rho, cfg)
    s2 = sigma ** 2
    term = sum(np.exp(-(2 * c * dx + dx * dx) / (4 * s2)) + np.exp((2 * c * dx - dx * dx) / (4 * s2)) - 2.0
               for c in (x, y, z)) / dx ** 2
    expect = -0.5 * cfg.hbm ** 2 * term
    inner = (slice(2, -2),) * 3          # away from the periodic seam
    np.testing.assert_allclose(q[inner], expect[inner], rtol=1e-9,
                               atol=1e-12 * np.abs(expect[inner]).max())


def test_gaussian_q_continuum_limit():
    """Continuum Q = -(hbar^2/2m^2)(r^2/(4 sigma^4) - 3/(2 sigma^2)); the discrete
    Q agrees to O((dx/sigma)^2) near the centre, and the error falls ~4x when dx
    halves."""
    errs = []
    for n in (32, 64):
        box, sigma = 1.0, 0.08
        cfg = O.Config(n_mesh=n, box=box, rho_floor=1e-300)
        rho, (x, y, z), dx = _gaussian_rho(n, box, sigma)
        q = O.quantum_potential(rho, cfg)
        r2 = x * x + y * y + z * z
        qc = -0.5 * cfg.hbm ** 2 * (r2 / (4 * sigma ** 4) - 1.5 / sigma ** 2)
        sel = r2 < (1.5 * sigma) ** 2
        errs.append(np.abs(q[sel] - qc[sel]).max() / np.abs(qc).max())
    assert errs[0] < 0.05
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_gaussian_quantum_force_points_outward():
    """-grad Q for a Gaussian is (hbar^2/4m^2 sigma^4) r: linear and outward."""
    n, box, sigma = 64, 1.0, 0.1
    cfg = O.Config(n_mesh=n, box=box, rho_floor=1e-300)
    rho, (x, y, z), dx = _gaussian_rho(n, box, sigma)
    q = O.quantum_potential(rho, cfg)
    g = -O.central_gradient(q, dx)
    sel = (np.abs(x) < 0.1) & (np.abs(y) < 1e-12) & (np.abs(z) < 1e-12) & (np.abs(x) > 0)
    slope = cfg.hbm ** 2 / (4 * sigma ** 4)
    ratio = g[0][sel] / (slope * x[sel])
    assert np.all(ratio > 0.9) and np.all(ratio < 1.1)


def test_q_invariant_under_density_scaling_and_zero_for_uniform():
    rng = np.random.default_rng(6)
    cfg = O.Config(n_mesh=16, box=1.0, rho_floor=1e-300)
    rho = np.exp(0.3 * rng.standard_normal((16, 16, 16)))
    q1 = O.quantum_potential(rho, cfg)
    q2 = O.quantum_potential(7.5 * rho, cfg)
    np.testing.assert_allclose(q1, q2, rtol=1e-12, atol=1e-12 * np.abs(q1).max())
    assert np.abs(O.quantum_potential(np.full((16, 16, 16), 2.0), cfg)).max() == 0.0


def test_wide_laplacian_is_the_central_difference_adjoint():
    """Sum_n s_n lap_wide(s)_n = -(1/4 dx^2) sum_n sum_d (s_{n+d}-s_{n-d})^2, the
    summation-by-parts identity pairing the printed K_rho of Eq. (diskpoten)
    with the wide stencil; the compact stencil pairs with forward differences."""
    rng = np.random.default_rng(7)
    s = rng.uniform(0.5, 1.5, (12, 12, 12))
    dx = 0.3
    lw = O.laplacian7(s, dx, O.LAP_WIDE)
    lc = O.laplacian7(s, dx, O.LAP_COMPACT)
    cen = sum(np.sum((np.roll(s, -1, a) - np.roll(s, 1, a)) ** 2) for a in range(3))
    fwd = sum(np.sum((np.roll(s, -1, a) - s) ** 2) for a in range(3))
    assert np.sum(s * lw) == pytest.approx(-cen / (4 * dx * dx), rel=1e-12)
    assert np.sum(s * lc) == pytest.approx(-fwd / (dx * dx), rel=1e-12)


def test_lagrangian_quantum_force_is_minus_energy_gradient():
    """Eq. (equationofmotion): m_i dp_i/dt = -dK_rho/dq_i.  Finite-difference the
    discrete K_rho (Eq. diskpoten, static, a = 1) with respect to one particle's
    position and compare with the oracle's quantum force times the particle mass."""
    rng = np.random.default_rng(8)
    for lap in (O.LAP_COMPACT, O.LAP_WIDE):
        cfg = O.Config(n_mesh=8, box=1.0, omega_m=0.0, cosmological=False,
                       force_mode=O.LAGRANGIAN, lap=lap, m22=0.01)
        x, _ = ics.lattice(8, 8, 1.0)
        x = np.mod(x + 0.02 * rng.standard_normal(x.shape), 1.0)
        p = np.zeros_like(x)
        _, gq = O.force_parts(x, cfg)
        mp = 1.0 / len(x)
        for i in (0, 100, 333):
            for d in range(3):
                eps = 1e-6
                xp, xm = x.copy(), x.copy()
                xp[i, d] += eps
                xm[i, d] -= eps
                kp = O.energies(xp, p, 1.0, cfg)[2]
                km = O.energies(xm, p, 1.0, cfg)[2]
                fd = -(kp - km) / (2 * eps)
                assert mp * gq[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(fd) + 1e-18)


# ---------------------------------------------------------------- interpolation
def test_interpolation_reproduces_linear_fields_and_constants():
    rng = np.random.default_rng(9)
    cfg = O.Config(n_mesh=16, box=2.0)
    x = _rand_particles(rng, 100, cfg.box)
    const = np.full((16, 16, 16), 3.25)
    np.testing.assert_allclose(O.cic_interpolate(const, x, cfg), 3.25, rtol=1e-14)
    g = O.cic_interpolate_gradient(const, x, cfg)
    assert np.abs(g).max() < 1e-12
    # a field linear in x on nodes (away from the seam) has exact gradient
    n = 16
    xs = np.arange(n) * cfg.dx
    lin = np.broadcast_to(2.5 * xs[None, None, :], (n, n, n)).copy()
    inner = (x[:, 0] < cfg.box - cfg.dx) & (x[:, 0] > 0)
    np.testing.assert_allclose(O.cic_interpolate(lin, x, cfg)[inner], 2.5 * x[inner, 0], rtol=1e-12)
    np.testing.assert_allclose(O.cic_interpolate_gradient(lin, x, cfg)[inner, 0], 2.5, rtol=1e-12)


# ---------------------------------------------------------------- power spectrum
def test_power_spectrum_zero_for_uniform_and_counts_modes():
    cfg = O.Config(n_mesh=8, box=1.0)
    x, _ = ics.lattice(4, 8, 1.0)
    k, pk, cnt = O.power_spectrum(x, cfg)
    assert np.all(pk == 0.0)
    # brute-force count of integer vectors with |m| rounded to each shell
    n = 8
    m = np.fft.fftfreq(n, 1.0 / n)
    cnt_b = np.zeros(n // 2, dtype=int)
    for a in m:
        for b in m:
            for c in m:
                s = int(math.floor(math.sqrt(a * a + b * b + c * c) + 0.5))
                if 1 <= s <= n // 2:
                    cnt_b[s - 1] += 1
    np.testing.assert_array_equal(cnt, cnt_b)


def test_power_spectrum_single_mode_amplitude():
    """A 1-per-cell lattice sitting on the nodes with a sinusoidal mass-weight
    gives rho = 1 + eps cos(k x) exactly; the estimator then returns
    L^3 eps^2/4 / sinc^4(k dx/2) for the two modes +-k."""
    n, box, eps, m = 16, 2.0, 0.05, 3
    cfg = O.Config(n_mesh=n, box=box)
    dx = box / n
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([ix * dx, iy * dx, iz * dx], axis=-1).reshape(-1, 3)
    k = 2 * np.pi * m / box
    mass = box ** 3 / n ** 3 * (1 + eps * np.cos(k * x[:, 0]))
    rho = O.cic_deposit(x, cfg, mass=mass)
    np.testing.assert_allclose(rho.mean(axis=(0, 1)), 1 + eps * np.cos(k * np.arange(n) * dx), atol=1e-13)
    # P(k) estimator applied to this density (reuse the mesh route)
    dk = np.fft.fftn(rho - 1.0)
    p_mode = box ** 3 / n ** 6 * abs(dk[0, 0, m]) ** 2 / np.sinc(k * dx / (2 * np.pi)) ** 4
    assert p_mode == pytest.approx(box ** 3 * eps ** 2 / 4 / np.sinc(k * dx / (2 * np.pi)) ** 4, rel=1e-12)


# ---------------------------------------------------------------- leapfrog
def test_static_kdk_is_time_reversible():
    """Kick-drift-kick is symmetric in time: n steps, reversed momenta, n steps
    return every particle to its start (both force modes)."""
    rng = np.random.default_rng(10)
    for fm in (O.MESHGRAD, O.LAGRANGIAN):
        cfg = O.Config(n_mesh=16, box=1.0, cosmological=False, omega_m=0.3, m22=0.05, force_mode=fm)
        x0, _ = ics.lattice(16, 16, 1.0)
        x0 = np.mod(x0 + 0.005 * rng.standard_normal(x0.shape), 1.0)
        p0 = 0.005 * rng.standard_normal(x0.shape)
        x, p, _ = O.run(x0, p0, 0.0, 2.0, 10, cfg)
        assert np.abs(p - p0).max() > 1e-4          # the forces did act
        x, p, _ = O.run(x, -p, 0.0, 2.0, 10, cfg)
        d = x - x0
        d -= np.round(d)
        assert np.abs(d).max() < 1e-12
        np.testing.assert_allclose(-p, p0, atol=1e-12)


# ---------------------------------------------------------------- linear growth
def _single_mode_ics(n, box, a_i, delta0, cfg):
    """1-per-cell lattice, one x-mode: psi_x = -(delta0/k) sin(k q_x), growing-mode
    velocity p = a^2 H psi (dln delta/dln a = 1 at a_i)."""
    dx = box / n
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    q = np.stack([(ix + 0.5) * dx, (iy + 0.5) * dx, (iz + 0.5) * dx], axis=-1).reshape(-1, 3)
    k = 2 * np.pi / box
    psi = np.zeros_like(q)
    psi[:, 0] = -(delta0 / k) * np.sin(k * q[:, 0])
    hub = math.sqrt(cfg.omega_m / a_i ** 3 + cfg.omega_l)
    return np.mod(q + psi, box), a_i ** 2 * hub * psi


def _mode_amplitude(x, cfg):
    dk = np.fft.fftn(O.cic_deposit(x, cfg) - 1.0)
    return 2 * dk[0, 0, 1].real / cfg.n_mesh ** 3


def _growth_ode(cfg, kk, cg, cq, a_i):
    """delta'' + (2 + dlnH/dlna) delta' = [cg (3/2) Om a^-3 - cq (hbar/m)^2 kk^4/(4 a^4)] delta / H^2
    (' = d/dln a): linear FDM growth (Jeans scale of Eq. jeansscale), RK by scipy."""
    from scipy.integrate import solve_ivp
    om, ol, hbm = cfg.omega_m, cfg.omega_l, cfg.hbm

    def rhs(lna, y):
        a = math.exp(lna)
        h2 = om / a ** 3 + ol
        src = (cg * 1.5 * om / a ** 3 - cq * hbm ** 2 * kk ** 4 / (4 * a ** 4)) / h2
        return [y[1], -(2 - 1.5 * om / a ** 3 / h2) * y[1] + src * y[0]]
    return solve_ivp(rhs, (math.log(a_i), 0.0), [1.0, 1.0], dense_output=True,
                     rtol=1e-11, atol=1e-14, method="DOP853")


@pytest.mark.parametrize("fm", [O.MESHGRAD, O.LAGRANGIAN])
@pytest.mark.parametrize("box,n,a_i,nsteps", [(1.0, 16, 0.01, 100), (0.05, 16, 0.1, 300)])
def test_linear_mode_follows_fdm_growth_equation(fm, box, n, a_i, nsteps):
    """One Fourier mode of amplitude 1e-4.  box = 1: k << k_J, CDM-like growth.
    box = 0.05: k > k_J(a_i), so the mode is suppressed and oscillates (it
    changes sign) until k_J(a) ~ a^(1/4) overtakes k near a ~ 0.4.  The run
    follows the linear ODE with the discrete symbols of the scheme: deposit
    and compact Laplacian kappa = 2 sin(k dx/2)/dx, central gradient plus
    interpolation cos^2(k dx/2) (the kernel-gradient form gives kappa exactly),
    and agrees with the continuum ODE within the discretisation error."""
    cfg = O.Config(n_mesh=n, box=box, force_mode=fm)
    x, p = _single_mode_ics(n, box, a_i, 1e-4, cfg)
    a0 = _mode_amplitude(x, cfg)
    avals = O.scale_factors(a_i, 1.0, nsteps, cfg)
    parts, meas = None, []
    for i in range(nsteps):
        x, p, parts = O.kdk_step(x, p, avals[i], avals[i + 1], cfg, parts)
        if (i + 1) % (nsteps // 5) == 0:
            meas.append((avals[i + 1], _mode_amplitude(x, cfg) / a0))
    k = 2 * np.pi / box
    dx = box / n
    kap = 2 * math.sin(k * dx / 2) / dx
    c2 = math.cos(k * dx / 2) ** 2
    lagr = fm == O.LAGRANGIAN
    disc = _growth_ode(cfg, kap, 1.0 if lagr else c2, 1.0 if lagr else c2, a_i)
    cont = _growth_ode(cfg, k, 1.0, 1.0, a_i)
    scale = max(abs(m) for _, m in meas)
    for a, m in meas:
        assert m == pytest.approx(disc.sol(math.log(a))[0], abs=1e-3 * scale)
        assert m == pytest.approx(cont.sol(math.log(a))[0], abs=0.25 * scale)
    kj = O.jeans_k(a_i, cfg.omega_m, cfg.hbm)
    vals = [m for _, m in meas]
    if k > kj:
        assert min(vals) < 0 < max(vals)                # oscillation
    else:
        assert all(b > a_ for a_, b in zip(vals, vals[1:]))   # monotonic growth


# ---------------------------------------------------------------- energy conservation
@pytest.mark.parametrize("om,lap", [(0.0, O.LAP_COMPACT), (0.0, O.LAP_WIDE), (0.3, O.LAP_COMPACT)])
def test_lagrangian_scheme_conserves_discrete_energy_to_second_order(om, lap):
    """Sec. II.A: the equation of motion derived from the Lagrangian conserves
    the discrete K_v (Eq. diskkinen) + K_rho (Eq. diskpoten) (+ W_g) by
    construction, so in a static run the only error is the leapfrog's O(dt^2):
    halving dt divides it by 4, while K_rho and K_v exchange energy."""
    errs = []
    for ns in (40, 80):
        cfg = O.Config(n_mesh=16, box=1.0, omega_m=om, cosmological=False,
                       force_mode=O.LAGRANGIAN, lap=lap, m22=0.05)
        x0, _ = ics.lattice(16, 16, 1.0)
        rng = np.random.default_rng(11)
        x0 = np.mod(x0 + 0.01 * rng.standard_normal(x0.shape), 1.0)
        _, _, hist = O.run(x0, np.zeros_like(x0), 0.0, 4.0, ns, cfg, energy_every=ns // 8)
        h = np.array(hist)
        e = h[:, 1] + h[:, 2] + h[:, 3]
        assert h[-1, 1] > 0.1 * h[0, 3]                 # kinetic energy was generated
        errs.append(np.abs(e - e[0]).max() / abs(h[0, 2] + h[0, 3]))
    assert errs[0] < 5e-3
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_layzer_irvine_holds_for_lagrangian_cosmology():
    """Cosmic energy equation d(K_v+W_g+K_rho)/da = -(2K_v+W_g+2K_rho)/a
    (Layzer-Irvine with the quantum term, K_rho ~ a^-2) holds to < 1e-2 from
    z = 100 to z = 3 for the energy-conserving force form."""
    cfg = O.Config(n_mesh=16, box=1.0, force_mode=O.LAGRANGIAN)
    x, p = ics.zeldovich(16, 16, 1.0, 1 / 101.0, 42)
    _, _, hist = O.run(x, p, 1 / 101.0, 1 / 4.0, 100, cfg, energy_every=1)
    eps = O.layzer_irvine_residual(hist, cfg)
    h = np.array(hist)
    assert abs(h[-1, 2]) > 20 * abs(h[1, 2])           # structure did grow
    assert np.abs(eps).max() < 1e-2


# ---------------------------------------------------------------- cubic spline kernel (Sec. II.A)
def test_spline_kernel_closed_form_properties():
    """W of Sec. II.A: unit integral over space, continuous value and slope at
    r = h/2, zero at and beyond r = h, W(0) = 8/(pi h^3)."""
    from scipy.integrate import quad
    h = 0.37
    total = quad(lambda r: 4 * math.pi * r * r * float(O.spline_w(r, h)), 0, h, points=[h / 2],
                 epsabs=0, epsrel=1e-13)[0]
    assert total == pytest.approx(1.0, rel=1e-12)
    c = 8 / (math.pi * h ** 3)
    assert float(O.spline_w(0.0, h)) == pytest.approx(c, rel=1e-15)
    eps = 1e-7 * h
    lo, mid, hi = (float(O.spline_w(h / 2 + d, h)) for d in (-eps, 0.0, eps))
    assert mid == pytest.approx(c / 4, rel=1e-14)                 # both branches give 1/4 there
    assert (mid - lo) / eps == pytest.approx((hi - mid) / eps, rel=1e-5)   # same slope on both sides:
    assert (mid - lo) / eps == pytest.approx(-1.5 * c / h, rel=1e-5)       # -12u + 18u^2 = -6(1-u)^2 = -3/2
    assert float(O.spline_w(h, h)) == 0.0 and float(O.spline_w(1.5 * h, h)) == 0.0


def test_spline_node_weights_sum_and_symbol():
    cfg = O.Config(n_mesh=16, box=1.0, kernel=O.KERNEL_SPLINE, smooth_h=3.5)
    w = O.spline_node_weights(cfg)
    assert w.sum() == pytest.approx(1.0, rel=1e-14)
    # the raw node sum of W dx^3 is a Riemann sum of a unit integral
    d = np.fft.fftfreq(16, d=1 / 16)
    dz, dy, dx_ = np.meshgrid(d, d, d, indexing="ij")
    raw = O.spline_w(np.sqrt(dx_ ** 2 + dy ** 2 + dz ** 2) * cfg.dx, 3.5 * cfg.dx).sum() * cfg.dx ** 3
    assert raw == pytest.approx(1.0, abs=2e-3)
    sym = O.smoothing_symbol(cfg)
    assert sym[0, 0, 0] == pytest.approx(1.0, rel=1e-14)
    assert np.abs(np.fft.fftn(w).imag).max() < 1e-14                   # even weights: real symbol
    assert np.all(np.abs(sym) <= 1.0 + 1e-14)


def test_spline_density_on_nodes_is_the_direct_kernel_sum():
    """Eq. (rhodis) by brute force for particles sitting on nodes: sum over
    particles of m W(|x_n - q_i|, h) at every node (minimum image), divided by
    the weights' normalisation."""
    rng = np.random.default_rng(21)
    n, box, h = 12, 1.5, 3.5
    cfg = O.Config(n_mesh=n, box=box, kernel=O.KERNEL_SPLINE, smooth_h=h)
    dx = box / n
    cells = rng.integers(0, n, size=(7, 3))
    x = cells * dx
    rho = O.density(x, cfg)
    mp = box ** 3 / len(x)
    d = np.fft.fftfreq(n, d=1 / n)
    dz, dy, dx_ = np.meshgrid(d, d, d, indexing="ij")
    raw = O.spline_w(np.sqrt(dx_ ** 2 + dy ** 2 + dz ** 2) * dx, h * dx).sum() * dx ** 3
    direct = np.zeros((n, n, n))
    grid = np.arange(n)
    for c in cells:
        ox = (grid - c[0] + n // 2) % n - n // 2
        oy = (grid - c[1] + n // 2) % n - n // 2
        oz = (grid - c[2] + n // 2) % n - n // 2
        r = np.sqrt(oz[:, None, None] ** 2 + oy[None, :, None] ** 2 + ox[None, None, :] ** 2) * dx
        direct += mp * O.spline_w(r, h * dx)
    np.testing.assert_allclose(rho, direct / raw, rtol=1e-11, atol=1e-12 * direct.max())


def test_spline_density_is_the_weights_convolved_with_cic():
    """Off-node particles: rho_n = sum_m w_{n-m} rho_cic_m, brute-force double sum."""
    rng = np.random.default_rng(22)
    n = 8
    cfg = O.Config(n_mesh=n, box=1.0, kernel=O.KERNEL_SPLINE, smooth_h=2.5)
    x = rng.uniform(0, 1, size=(5, 3))
    rc = O.cic_deposit(x, O.Config(n_mesh=n, box=1.0))
    w = O.spline_node_weights(cfg)
    ref = np.zeros((n, n, n))
    for mz in range(n):
        for my in range(n):
            for mx in range(n):
                if rc[mz, my, mx] != 0.0:
                    ref += rc[mz, my, mx] * np.roll(w, (mz, my, mx), axis=(0, 1, 2))
    np.testing.assert_allclose(O.density(x, cfg), ref, rtol=1e-12, atol=1e-13)
    assert O.density(x, cfg).sum() * cfg.dx ** 3 == pytest.approx(1.0, rel=1e-13)   # mass kept


def test_spline_lagrangian_forces_are_minus_energy_gradients():
    """With the spline kernel the LAGRANGIAN forces stay the derivatives of the
    discrete energies: Q force vs -dK_rho/dq and gravity vs -dW_g/dq (static,
    a = 1), by central finite differences in one particle's position."""
    rng = np.random.default_rng(23)
    cfg = O.Config(n_mesh=8, box=1.0, omega_m=0.3, cosmological=False, force_mode=O.LAGRANGIAN,
                   m22=0.01, kernel=O.KERNEL_SPLINE, smooth_h=2.0)
    x, _ = ics.lattice(4, 8, 1.0)
    x = np.mod(x + 0.03 * rng.standard_normal(x.shape), 1.0)
    p = np.zeros_like(x)
    gphi, gq = O.force_parts(x, cfg)
    mp = 1.0 / len(x)
    for i in (0, 17, 41):
        for d in range(3):
            eps = 1e-6
            xp, xm = x.copy(), x.copy()
            xp[i, d] += eps
            xm[i, d] -= eps
            ep, em = O.energies(xp, p, 1.0, cfg), O.energies(xm, p, 1.0, cfg)
            fq = -(ep[2] - em[2]) / (2 * eps)
            fg = -(ep[1] - em[1]) / (2 * eps)
            assert mp * gq[i, d] == pytest.approx(fq, rel=1e-5, abs=1e-8 * abs(fq) + 1e-16)
            assert mp * gphi[i, d] == pytest.approx(fg, rel=1e-5, abs=1e-8 * abs(fg) + 1e-16)


def test_spline_gravity_conserves_momentum():
    """The spline-smoothed mesh-gradient gravity (MESHGRAD, HYBRID) keeps the
    PM pair symmetry: the forces sum to zero.  (The kernel-gradient forms are
    derivatives of mesh energies, not pair forces, and conserve momentum only
    approximately, with cloud-in-cell as with the spline.)"""
    rng = np.random.default_rng(24)
    for fm in (O.MESHGRAD, O.HYBRID):
        cfg = O.Config(n_mesh=16, box=1.0, force_mode=fm, kernel=O.KERNEL_SPLINE)
        x = rng.uniform(0, 1, size=(300, 3))
        gphi, _ = O.force_parts(x, cfg)
        assert np.abs(gphi.sum(axis=0)).max() < 1e-12 * np.abs(gphi).sum()


# ---------------------------------------------------------------- adaptive step (Sec. II.A)
def _min_image(d, box):
    return d - box * np.round(d / box)


def test_adaptive_step_bounds_every_displacement():
    """Every particle moves at most cfl*dx per step, and a step that stops
    before a_end sits on the bound (the bisection finds its edge)."""
    rng = np.random.default_rng(31)
    cfg = O.Config(n_mesh=16, box=1.0, force_mode=O.HYBRID, m22=2.5)
    x, p = ics.zeldovich(8, 16, 1.0, 1 / 101.0, 5, amplitude=6.0)
    p = p * 3.0 + 0.02 * rng.standard_normal(p.shape)
    cfl = 0.4
    parts = O.force_parts(x, cfg)
    a0, a_end = 1 / 101.0, 1 / 20.0
    a1 = O.next_scale_factor(p, parts, a0, a_end, cfg, cfl)
    assert a0 < a1 < a_end
    gphi, gq = parts
    ah = O.half_point(a0, a1, cfg)
    b = (np.linalg.norm(p, axis=1).max() + O.kick_factor(a0, ah, cfg) * np.linalg.norm(gphi, axis=1).max()
         + O.drift_factor(a0, ah, cfg) * np.linalg.norm(gq, axis=1).max()) * O.drift_factor(a0, a1, cfg)
    assert b == pytest.approx(cfl * cfg.dx, rel=1e-9)
    xs, ps, bounds = O.run_adaptive(x, p, a0, 1 / 60.0, cfg, cfl=cfl)
    assert bounds[-1] == 1 / 60.0 and len(bounds) > 3
    # replay the steps and check each one's displacement
    xi, pi, parts = x, p, O.force_parts(x, cfg)
    for k in range(len(bounds) - 1):
        xn, pi, parts = O.kdk_step(xi, pi, bounds[k], bounds[k + 1], cfg, parts)
        assert np.linalg.norm(_min_image(xn - xi, cfg.box), axis=1).max() <= cfl * cfg.dx * (1 + 1e-12)
        xi = xn
    np.testing.assert_allclose(xi, xs, rtol=0, atol=1e-14)


def test_adaptive_step_free_streaming_count():
    """No forces, static box, speed v: steps of exactly cfl*dx/v, so a span T
    takes ceil(T v / (cfl dx)) steps."""
    cfg = O.Config(n_mesh=16, box=1.0, omega_m=0.0, quantum=False, cosmological=False)
    x, _ = ics.lattice(4, 16, 1.0)
    v = 0.37
    p = np.zeros_like(x)
    p[:, 0] = v
    p[:, 1] = -v * 0.5
    speed = v * math.sqrt(1.25)
    cfl, T = 0.5, 0.9
    _, _, bounds = O.run_adaptive(x, p, 0.0, T, cfg, cfl=cfl)
    assert len(bounds) - 1 == math.ceil(T * speed / (cfl * cfg.dx))
    np.testing.assert_allclose(np.diff(bounds)[:-1], cfl * cfg.dx / speed, rtol=1e-12)


def test_adaptive_step_at_rest_takes_one_step():
    cfg = O.Config(n_mesh=8, box=1.0, omega_m=0.3, quantum=True, cosmological=False)
    x, _ = ics.lattice(4, 8, 1.0)      # uniform density: no force
    _, _, bounds = O.run_adaptive(x, np.zeros_like(x), 0.0, 2.0, cfg)
    assert len(bounds) == 2
