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
