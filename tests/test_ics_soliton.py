"""The Schroedinger-Poisson ground state used as the soliton test's input
(no GPU): pinned by the virial theorem, the published core fit and mass, and
the sampler's mass and radius."""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid, trapezoid

from paper_1608_00802_gb300 import ics


def test_ground_state_is_nodeless_and_virialised():
    r, psi, u0 = ics.soliton_ground_state(npts=20000)
    assert psi[0] == 1.0 and np.all(psi >= 0) and np.all(np.diff(psi[psi > 1e-8]) <= 1e-12)   # monotone, no node
    rho = psi * psi
    m = cumulative_trapezoid(4 * np.pi * r * r * rho, r, initial=0.0)
    dpsi = ics._sp_shoot(u0).sol(r)[1]
    dpsi[psi == 0.0] = 0.0
    kin = 0.5 * trapezoid(4 * np.pi * r * r * dpsi ** 2, r)        # (hbar/m)^2/2 int |grad psi|^2
    pot = -trapezoid(m * rho * r, r)                               # -G int M dM / r with 4 pi G = 1
    assert (2 * kin + pot) / abs(pot) == pytest.approx(0.0, abs=1e-6)   # stationary: 2K + W = 0


def test_ground_state_mass_and_core_fit():
    """Mass int psi^2 r^2 dr = 2.062 for psi(0) = 1 (Guzman & Urena-Lopez 2004);
    within three core radii the density follows the fit (1 + 0.091 (r/r_c)^2)^-8
    of Schive et al. 2014 to a few per cent."""
    r, psi, _ = ics.soliton_ground_state(npts=20000)
    rho = psi * psi
    assert trapezoid(rho * r * r, r) == pytest.approx(2.062, abs=1e-3)
    rc = np.interp(0.5, rho[::-1], r[::-1])
    sel = r <= 3 * rc
    fit = (1 + 0.091 * (r[sel] / rc) ** 2) ** -8
    assert np.max(np.abs(rho[sel] - fit) / fit) < 0.08


def test_soliton_particles_mass_radius_and_centre():
    n, box, nm, r95 = 200000, 2.0, 64, 9.3
    x, p, om, info = ics.soliton_particles(n, box, nm, r95, 5e-5, seed=3)
    assert x.shape == (n, 3) and np.all(p == 0) and om > 0
    d = x - box / 2
    rr = np.linalg.norm(d, axis=1)
    frac = np.mean(rr <= r95 * box / nm)
    assert frac == pytest.approx(0.95, abs=4 * np.sqrt(0.95 * 0.05 / n))
    assert np.abs(d.mean(axis=0)).max() < 4 * rr.std() / np.sqrt(n)
    # the coupling reproduces the profile's central density with the scaling of the SP equations
    assert info["rho_c"] == pytest.approx((5e-5) ** 2 / (info["alpha"] ** 4 * info["gamma"]), rel=1e-12)
