"""Seeded synthetic initial conditions (Zel'dovich approximation).

This module is the input generator shared by the CUDA path, its tests and the
CPU oracle's tests.  It holds none of the particle-mesh step's arithmetic
(no deposit, Poisson solve, quantum pressure, interpolation or leapfrog): it
only turns a seed into particle positions and momenta.

Recipe (stands in for the MUSIC initial conditions of Sec. III, which are not
available here):

  * white noise w ~ N(0, 1) on the n_p^3 particle lattice from numpy's Philox
    generator keyed by the seed;
  * linear spectrum P(k) = A k^n_s T_BBKS(k)^2 T_FDM(k)^2, n_s = 0.96, with A
    fixed by sigma_8 = 0.8 at z = 0 for the CDM part (T_FDM = 1) and scaled by
    the linear growth D(a_i)/D(1);
  * T_BBKS: the Bardeen-Bond-Kaiser-Szalay (1986) fit with shape Gamma =
    Omega_m h, k in h/Mpc;
  * T_FDM(k) = cos(x^3)/(1 + x^8), x = 1.61 m22^(1/18) k / k_Jeq, Eq.
    (transferhu); k_Jeq = 9 m22^(1/2) Mpc^-1 (Hu, Barkana & Gruzinov 2000)
    = 9 m22^(1/2) / h  h/Mpc;
  * delta^_k = w^_k sqrt(P(k) / dV) with dV = (L/n_p)^3, Nyquist planes
    zeroed; displacement psi^ = i k delta^ / k^2;
  * lattice q = (i r + 1/2) dx with r = N/n_p, so the cloud-in-cell density of
    the unperturbed lattice on the N^3 mesh is exactly uniform;
  * x = q + D psi, p = a^2 H f D psi (p = a^2 dx/dt, f = dln D/dln a).

Length Mpc/h, time 1/H0, H0 = 1.
"""
from __future__ import annotations

import math

import numpy as np


def _hubble(a, om, ol):
    return np.sqrt(om / a ** 3 + ol)


def growth(a, om, ol, n=4096):
    """Linear growth D(a) (normalised to a at early times) and f = dlnD/dlna
    for flat matter + Lambda: D = (5 Om / 2) H(a) int_0^a da'/(a' H(a'))^3."""
    # substitution a' = a t^2 removes the endpoint behaviour; Gauss-Legendre on t
    tg, wg = np.polynomial.legendre.leggauss(n // 16)
    t = 0.5 * (tg + 1.0)
    w = 0.5 * wg
    ap = a * t * t
    integrand = 1.0 / (ap * _hubble(ap, om, ol)) ** 3 * (2.0 * a * t)
    integral = float(np.sum(w * integrand))
    h = float(_hubble(a, om, ol))
    d = 2.5 * om * h * integral
    dlnh = -1.5 * om / a ** 3 / h ** 2
    f = dlnh + 2.5 * om / (a * a * h * h * d)
    return d, f


def t_bbks(k, om, h):
    q = k / (om * h)
    q = np.where(q <= 0, 1e-30, q)
    return (np.log1p(2.34 * q) / (2.34 * q)
            * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)


def t_fdm(k, m22, h):
    k_jeq = 9.0 * math.sqrt(m22) / h
    x = 1.61 * m22 ** (1.0 / 18.0) * k / k_jeq
    return np.cos(x ** 3) / (1.0 + x ** 8)


def _sigma8_norm(om, h, ns):
    k = np.logspace(-4, 3, 20000)
    x = k * 8.0
    wth = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    pk = k ** ns * t_bbks(k, om, h) ** 2
    integ = k ** 2 * pk * wth ** 2 / (2 * np.pi ** 2)
    s2 = float(np.sum(0.5 * (integ[1:] + integ[:-1]) * np.diff(k)))
    return 0.8 ** 2 / s2


def linear_power(k, a, om, ol, h, m22, fdm_ics=True, ns=0.96):
    amp = _sigma8_norm(om, h, ns)
    d1, _ = growth(1.0, om, ol)
    da, _ = growth(a, om, ol)
    pk = amp * np.where(k > 0, k, 1.0) ** ns * t_bbks(k, om, h) ** 2 * (da / d1) ** 2
    if fdm_ics:
        pk = pk * t_fdm(k, m22, h) ** 2
    return np.where(k > 0, pk, 0.0)


def zeldovich(n_part_side, n_mesh, box, a_init, seed, om=0.3, ol=0.7, h=0.7, m22=2.5,
              fdm_ics=True, amplitude=1.0):
    """Particles (x, p) of shape (n^3, 3), float64, lattice order (x fastest).

    `amplitude` scales the displacement field (1 = the recipe above)."""
    n = n_part_side
    if n_mesh % n:
        raise ValueError("mesh size must be a multiple of the particle lattice size")
    dq = box / n
    r = n_mesh // n
    dxm = box / n_mesh
    rng = np.random.Generator(np.random.Philox(seed))
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    k1 = 2 * np.pi * np.fft.fftfreq(n, d=dq)
    k1z = 2 * np.pi * np.fft.rfftfreq(n, d=dq)
    kz, ky, kx = np.meshgrid(k1, k1, k1z, indexing="ij")   # array axes [z, y, x]
    # rfftn over axes (0,1,2) halves the last axis -> it is the x axis here
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    pk = linear_power(kmag, a_init, om, ol, h, m22, fdm_ics)
    dk = wk * np.sqrt(pk / dq ** 3) * amplitude
    nyq = n // 2
    dk[nyq, :, :] = 0
    dk[:, nyq, :] = 0
    dk[:, :, nyq] = 0
    k2 = np.where(kmag > 0, kmag ** 2, 1.0)
    psi = []
    for kc in (kx, ky, kz):
        psik = 1j * kc * dk / k2
        psik[0, 0, 0] = 0
        psi.append(np.fft.irfftn(psik, s=(n, n, n), axes=(0, 1, 2)))
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    q = np.stack([(ix * r + 0.5) * dxm, (iy * r + 0.5) * dxm, (iz * r + 0.5) * dxm], axis=-1).reshape(-1, 3)
    psi = np.stack([c.reshape(-1) for c in psi], axis=1)
    _, f = growth(a_init, om, ol)
    hub = float(_hubble(a_init, om, ol))
    x = np.mod(q + psi, box)
    p = a_init ** 2 * hub * f * psi
    return x, p


def lattice(n_part_side, n_mesh, box):
    """Unperturbed lattice positions (x fastest), zero momenta."""
    n = n_part_side
    r = n_mesh // n
    dxm = box / n_mesh
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([(ix * r + 0.5) * dxm, (iy * r + 0.5) * dxm, (iz * r + 0.5) * dxm], axis=-1).reshape(-1, 3)
    return x, np.zeros_like(x)


# --------------------------------------------------------------------------
# solitonic core: the spherically symmetric ground state of the
# Schroedinger-Poisson equations (the initial profile of the paper's static
# soliton test, Sec. II.B, after Guzman & Urena-Lopez 2004)
# --------------------------------------------------------------------------
def _sp_rhs(r, y):
    # units hbar/m = 1, 4 pi G = 1, psi(0) = 1; u = V - eps
    psi, dpsi, u, du = y
    if r == 0.0:
        return [dpsi, 2.0 * u * psi / 3.0, du, psi * psi / 3.0]
    return [dpsi, 2.0 * u * psi - 2.0 * dpsi / r, du, psi * psi - 2.0 * du / r]


def _sp_shoot(u0, rmax=20.0):
    from scipy.integrate import solve_ivp

    def crosses(r, y):
        return y[0]
    crosses.terminal, crosses.direction = True, -1

    def turns_up(r, y):
        return y[1]
    turns_up.terminal, turns_up.direction = True, 1
    return solve_ivp(_sp_rhs, [0.0, rmax], [1.0, 0.0, u0, 0.0], rtol=1e-12, atol=1e-15,
                     events=[crosses, turns_up], dense_output=True)


def soliton_ground_state(npts=4000):
    """(r, psi, u0) of the nodeless stationary state in units hbar/m = 1,
    4 pi G = 1, psi(0) = 1 (rho = psi^2): psi'' + 2psi'/r = 2(V - eps) psi,
    V'' + 2V'/r = psi^2.  The central value u0 = V(0) - eps is found by
    bisection between solutions that cross zero and ones that turn up; psi is
    cut where the bracketing solutions part (psi ~ 1e-6 of its centre)."""
    lo, hi = -1.0, -0.25   # lo: crosses zero, hi: turns up
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        s = _sp_shoot(mid)
        if len(s.t_events[0]):
            lo = mid
        else:
            hi = mid
    s_lo, s_hi = _sp_shoot(lo), _sp_shoot(hi)
    r_end = min(s_lo.t[-1], s_hi.t[-1])
    r = np.linspace(0.0, r_end, npts)
    a, b = s_lo.sol(r)[0], s_hi.sol(r)[0]
    psi = 0.5 * (a + b)
    cut = np.argmax(np.abs(a - b) > 1e-6) if np.any(np.abs(a - b) > 1e-6) else npts
    psi[cut:] = 0.0
    return r, np.clip(psi, 0.0, None), 0.5 * (lo + hi)


def soliton_particles(n_part, box, n_mesh, r95_cells, hbm, seed=0, center=None):
    """n_part particles (mass box^3 / n_part each, so the mean density is 1)
    drawn from the ground-state profile scaled to enclose 95 % of the mass
    within r95_cells mesh cells, at rest.  The scaling symmetry of the SP
    equations fixes the coupling: with hbar/m = hbm the profile of total mass
    box^3 and that radius needs 4 pi G = gamma, returned as omega_m =
    gamma / 1.5 for a static run (4 pi G rho_bar = 1.5 omega_m, rho_bar = 1).
    Returns (x, p, omega_m, info)."""
    r_d, psi, u0 = soliton_ground_state()
    rho_d = psi * psi
    dr = r_d[1] - r_d[0]
    shell = 4.0 * np.pi * r_d * r_d * rho_d
    m_cum = np.concatenate([[0.0], np.cumsum(0.5 * (shell[1:] + shell[:-1]) * dr)])
    m_d = m_cum[-1]
    r95_d = float(np.interp(0.95 * m_d, m_cum, r_d))
    alpha = r95_cells * (box / n_mesh) / r95_d      # length scale
    mass = box ** 3
    gamma = hbm * hbm * m_d / (alpha * mass)        # 4 pi G
    rng = np.random.Generator(np.random.Philox(seed))
    u = rng.uniform(size=(n_part, 3))
    rr = alpha * np.interp(u[:, 0] * m_d, m_cum, r_d)
    cz = 2.0 * u[:, 1] - 1.0
    ph = 2.0 * np.pi * u[:, 2]
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    c = np.full(3, 0.5 * box) if center is None else np.asarray(center, dtype=np.float64)
    x = np.stack([rr * sz * np.cos(ph), rr * sz * np.sin(ph), rr * cz], axis=1) + c
    x = np.mod(x, box)
    info = {"alpha": alpha, "gamma": gamma, "rho_c": hbm * hbm / (alpha ** 4 * gamma), "t_unit": alpha * alpha / hbm,
            "r95": r95_cells * box / n_mesh, "u0": u0, "mass_dimless": m_d, "r95_dimless": r95_d}
    return x, np.zeros_like(x), gamma / 1.5, info
