"""Plain FP64 CPU oracle for the particle-mesh step with quantum pressure.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path and imports nothing from the package.

It follows Veltmaat & Niemeyer, "Cosmological particle-in-cell simulations with
ultralight axion dark matter" (arXiv:1608.00802), Sec. II.A:

  * density by a kernel estimate, Eq. (rhodis): the cloud-in-cell kernel (a
    tensor tent of width dx), or the paper's cubic spline W(r, h) of
    Sec. II.A (h = 3.5 dx in its cosmological runs) applied as a mesh
    convolution of the cloud-in-cell density with the spline sampled at the
    nodes; the force side then uses the same convolution (its transpose);
  * quantum pressure Q = -(hbar^2/2m^2) lap(sqrt rho)/sqrt rho,
    Eq. (quantumpressure), in comoving form Eq. (comquantumpressure), with the
    seven-point Laplacian named after Eq. (equationofmotion);
  * the three principal steps (i) density, (ii) Q on the grid, (iii) force on
    each particle, inside a kick-drift-kick leapfrog;
  * energies K_v, Eq. (diskkinen), and K_rho, Eq. (diskpoten);
  * the gravity solve of the PM scheme (Sec. II.A names the Nyx PM solver, a
    solver of the discrete seven-point Poisson equation; here its exact
    periodic solution, obtained with the discrete Green's function in Fourier
    space, numpy.fft serving as the FFT primitive).

Everything is float64, vectorised numpy, in the order the paper states the
steps; no blocking, fusion or reordering beyond that.

Code units: length Mpc/h (box L), time 1/H0 (H0 = 1), mean comoving density
1, so 4 pi G rho_bar = (3/2) Omega_m and a particle of an N_p-particle box has
mass L^3/N_p.  Positions x in [0, L)^3 (comoving), momentum p = a^2 dx/dt.
Mesh arrays are indexed [z, y, x] (x fastest); position columns are (x, y, z).
Mesh node n sits at n * dx.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# constants and units
# --------------------------------------------------------------------------
HBARC_EV_M = 1.973269804e-7      # hbar*c, CODATA 2018, eV m
C_M_S = 299792458.0              # speed of light, m/s (exact)
MPC_M = 3.0856775814913673e22    # 1 Mpc in m (IAU 2015 parsec)

# force modes (how each mesh potential becomes a particle force)
MESHGRAD = 0     # gravity and Q: central-difference mesh gradient, CIC-interpolated
HYBRID = 1       # gravity as MESHGRAD; Q by Eq. (equationofmotion) (the paper's Nyx scheme)
LAGRANGIAN = 2   # gravity and Q both by the kernel-gradient form (fully energy-conserving)
LAP_COMPACT = 0
LAP_WIDE = 1
KERNEL_CIC = 0     # cloud-in-cell assignment only
KERNEL_SPLINE = 1  # cloud-in-cell assignment convolved with the node-sampled cubic spline


def hbar_over_m(m22: float, h: float) -> float:
    """hbar/m in code units (Mpc/h)^2 H0 for an axion of m = m22 * 1e-22 eV.

    hbar/m = (hbar c) c / (m c^2); one code unit of (length^2/time) is
    (Mpc/h)^2 * 100 h km/s/Mpc = (100/h) Mpc km/s.
    """
    hbar_m_si = HBARC_EV_M * C_M_S / (m22 * 1e-22)          # m^2/s
    hbar_m_mpc_kms = hbar_m_si / (MPC_M * 1e3)               # Mpc km/s
    return hbar_m_mpc_kms / (100.0 / h)


def jeans_k(a: float, omega_m: float, hbm: float) -> float:
    """Quantum Jeans wavenumber, Eq. (jeansscale), in comoving h/Mpc.

    k_J = 2 pi^(1/4) a^(1/4) (G rho)^(1/4) (m/hbar)^(1/2) with the comoving
    mean density: 4 pi G rho_bar = (3/2) Omega_m gives k_J = (6 Omega_m a)^(1/4)
    (hbar/m)^(-1/2).
    """
    g_rho = 1.5 * omega_m / (4.0 * math.pi)
    return 2.0 * math.pi ** 0.25 * a ** 0.25 * g_rho ** 0.25 / math.sqrt(hbm)


@dataclass
class Config:
    """Run parameters (mirrors the C-ABI configuration)."""
    n_mesh: int
    box: float
    omega_m: float = 0.3
    omega_l: float = 0.7
    h: float = 0.7
    m22: float = 2.5
    quantum: bool = True
    force_mode: int = MESHGRAD
    lap: int = LAP_COMPACT
    cosmological: bool = True
    rho_floor: float = 1e-6
    kernel: int = KERNEL_CIC
    smooth_h: float = 3.5          # spline smoothing length in mesh cells

    @property
    def dx(self) -> float:
        return self.box / self.n_mesh

    @property
    def hbm(self) -> float:
        return hbar_over_m(self.m22, self.h)


# --------------------------------------------------------------------------
# background cosmology and leapfrog weights
# --------------------------------------------------------------------------
def hubble(a, omega_m, omega_l):
    """H(a)/H0 for a flat matter + Lambda background (no radiation)."""
    return np.sqrt(omega_m / a ** 3 + omega_l)


def _gauss_legendre(f, lo, hi, n=48):
    xg, wg = np.polynomial.legendre.leggauss(n)
    mid, half = 0.5 * (hi + lo), 0.5 * (hi - lo)
    return half * float(np.sum(wg * f(mid + half * xg)))


def kick_factor(a0, a1, cfg: Config) -> float:
    """Momentum weight of a kick, int dt / a = int da / (a^2 H).

    With p = a^2 dx/dt the comoving equation of motion reads
    dp/dt = -grad(phi)/a - grad(Q~)/a^2; the 1/a of the gravity term and
    dt = da/(a H) give this integral.  Static (non-cosmological) runs use
    a = 1, so the weight is the elapsed time a1 - a0.
    """
    if not cfg.cosmological:
        return a1 - a0
    return _gauss_legendre(lambda a: 1.0 / (a * a * hubble(a, cfg.omega_m, cfg.omega_l)), a0, a1)


def drift_factor(a0, a1, cfg: Config) -> float:
    """Position weight int dt / a^2 = int da / (a^3 H); also the weight of the
    quantum kick, whose comoving force carries 1/a^2 (Eq. comquantumpressure).
    Static runs: the elapsed time."""
    if not cfg.cosmological:
        return a1 - a0
    return _gauss_legendre(lambda a: 1.0 / (a ** 3 * hubble(a, cfg.omega_m, cfg.omega_l)), a0, a1)


def half_point(a0, a1, cfg: Config) -> float:
    """Leapfrog half point: midpoint in ln a (cosmological) or in t (static)."""
    return math.sqrt(a0 * a1) if cfg.cosmological else 0.5 * (a0 + a1)


# --------------------------------------------------------------------------
# cell keys and order
# --------------------------------------------------------------------------
def cell_index(x, cfg: Config):
    """Integer cell (ix, iy, iz) = floor(x/dx) per dimension, periodic."""
    n = cfg.n_mesh
    return np.mod(np.floor(x / cfg.dx).astype(np.int64), n)


def cell_key(x, cfg: Config):
    """Linear cell key (iz*N + iy)*N + ix."""
    n = cfg.n_mesh
    c = cell_index(x, cfg)
    return (c[:, 2] * n + c[:, 1]) * n + c[:, 0]


def stable_cell_order(keys):
    """Permutation sorting by key; equal keys keep their present order."""
    return np.argsort(keys, kind="stable")


# --------------------------------------------------------------------------
# (i) density, Eq. (rhodis), cloud-in-cell kernel
# --------------------------------------------------------------------------
def cic_weights(x, cfg: Config):
    """For each particle: base node (the lower corner of its cell) and the
    fractional offset f in [0,1) per dimension.  The cloud-in-cell weight of
    node base + d (d in {0,1}^3) is prod_k (1 - f_k if d_k == 0 else f_k),
    i.e. the tent W(x_n - q) = prod_k (1 - |x_n,k - q_k|/dx)_+ ."""
    u = x / cfg.dx
    base = np.floor(u)
    f = u - base
    return np.mod(base.astype(np.int64), cfg.n_mesh), f


def cic_deposit(x, cfg: Config, mass=None):
    """rho_n = sum_i m_i W(x_n - q_i) / dx^3 on the periodic mesh.

    Scatter over particles (each adds to its eight nodes).  With the default
    mass L^3/N_p the mean density is exactly 1.
    """
    n = cfg.n_mesh
    npart = x.shape[0]
    if mass is None:
        mass = np.full(npart, cfg.box ** 3 / max(npart, 1))
    base, f = cic_weights(x, cfg)
    rho = np.zeros(n * n * n)
    for dz in (0, 1):
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        iz = (base[:, 2] + dz) % n
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            iy = (base[:, 1] + dy) % n
            for dxo in (0, 1):
                wx = f[:, 0] if dxo else 1.0 - f[:, 0]
                ix = (base[:, 0] + dxo) % n
                idx = (iz * n + iy) * n + ix
                rho += np.bincount(idx, weights=mass * wx * wy * wz, minlength=n ** 3)
    return rho.reshape(n, n, n) / cfg.dx ** 3


# --------------------------------------------------------------------------
# the cubic spline of Sec. II.A and the smoothed density
# --------------------------------------------------------------------------
def spline_w(r, h):
    """W(r, h) = 8/(pi h^3) * {1 - 6u^2 + 6u^3 for u <= 1/2; 2(1-u)^3 for
    1/2 < u <= 1; 0 beyond}, u = r/h (the kernel chosen in Sec. II.A)."""
    u = np.asarray(r, dtype=np.float64) / h
    inner = 1.0 - 6.0 * u ** 2 + 6.0 * u ** 3
    outer = 2.0 * (1.0 - u) ** 3
    return 8.0 / (math.pi * h ** 3) * np.where(u <= 0.5, inner, np.where(u <= 1.0, outer, 0.0))


def spline_node_weights(cfg: Config):
    """w_n = W(|x_n|, h) dx^3 at every node offset of the periodic mesh
    (minimum image), divided by their sum so that mass is kept exactly."""
    n = cfg.n_mesh
    d = np.fft.fftfreq(n, d=1.0 / n)  # 0, 1, .., n/2-1, -n/2, .., -1 (in cells)
    dz, dy, dx_ = np.meshgrid(d, d, d, indexing="ij")
    r = np.sqrt(dx_ ** 2 + dy ** 2 + dz ** 2) * cfg.dx
    w = spline_w(r, cfg.smooth_h * cfg.dx) * cfg.dx ** 3
    return w / w.sum()


def smoothing_symbol(cfg: Config):
    """DFT of the node weights (real: the weights are even in every axis)."""
    return _symbol(cfg.n_mesh, cfg.box, cfg.smooth_h).copy()


@functools.lru_cache(maxsize=8)
def _symbol(n, box, smooth_h):
    # memo of the symbol per mesh (the weights depend only on n, box and h)
    return np.real(np.fft.fftn(spline_node_weights(Config(n_mesh=n, box=box, smooth_h=smooth_h))))


def smooth(field, cfg: Config):
    """Periodic convolution of a mesh field with the node weights (a symmetric
    operator, its own transpose)."""
    return np.real(np.fft.ifftn(np.fft.fftn(field) * smoothing_symbol(cfg)))


def density(x, cfg: Config):
    """The density of Eq. (rhodis) on the mesh: cloud-in-cell, then (spline
    kernel) the convolution with the node weights.  For a particle on a node
    this is exactly sum_i m_i W(|x_n - q_i|, h) up to the weights' normalisation."""
    rho = cic_deposit(x, cfg)
    if cfg.kernel == KERNEL_SPLINE:
        rho = smooth(rho, cfg)
    return rho


# --------------------------------------------------------------------------
# gravity: discrete seven-point Poisson equation, periodic, exact solution
# --------------------------------------------------------------------------
def laplacian_symbol(n, box):
    """Fourier symbol of the compact seven-point Laplacian,
    -kappa^2 = -(4/dx^2) sum_d sin^2(k_d dx / 2), on the full FFT grid
    (numpy fftn axis order [z, y, x])."""
    dx = box / n
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=dx)
    s2 = (2.0 / dx * np.sin(0.5 * k * dx)) ** 2
    return s2[:, None, None] + s2[None, :, None] + s2[None, None, :]


def poisson_phi(rho, cfg: Config):
    """phi~ solving lap7(phi~) = (3/2) Omega_m (rho - 1), zero mean.

    Physical peculiar potential Phi = phi~/a.  Solved exactly for the periodic
    discrete operator: phi^_k = -(3/2) Omega_m rho^_k / kappa^2, phi^_0 = 0.
    """
    n = cfg.n_mesh
    kap2 = laplacian_symbol(n, cfg.box)
    rhok = np.fft.fftn(rho - 1.0)
    kap2[0, 0, 0] = 1.0
    phik = -1.5 * cfg.omega_m * rhok / kap2
    phik[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(phik))


def laplacian7(f, dx, lap=LAP_COMPACT):
    """Seven-point Laplacian on the periodic mesh: compact (spacing dx) or the
    wide form (spacing 2 dx, the adjoint partner of central differences)."""
    step = 1 if lap == LAP_COMPACT else 2
    h2 = (step * dx) ** 2
    out = np.zeros_like(f)
    for ax in range(3):
        out += (np.roll(f, -step, axis=ax) + np.roll(f, step, axis=ax) - 2.0 * f)
    return out / h2


# --------------------------------------------------------------------------
# (ii) quantum pressure on the grid, Eq. (quantumpressure)/(comquantumpressure)
# --------------------------------------------------------------------------
def sqrt_rho(rho, cfg: Config):
    """s = sqrt(max(rho, rho_floor)): Q is undefined where rho vanishes, so the
    density is floored at rho_floor (in units of the mean)."""
    return np.sqrt(np.maximum(rho, cfg.rho_floor))


def quantum_potential(rho, cfg: Config):
    """Q~ = -(hbar/m)^2/2 * lap7(s)/s with s = sqrt(rho) (floored).

    The comoving Q of Eq. (comquantumpressure) is Q~/a^2; the 1/a^2 is applied
    with the time weights.  The neighbour differences are formed before the
    division by s.
    """
    s = sqrt_rho(rho, cfg)
    return -0.5 * cfg.hbm ** 2 * laplacian7(s, cfg.dx, cfg.lap) / s


def central_gradient(u, dx):
    """(d/dx, d/dy, d/dz) of a mesh field by central differences, periodic.
    Returns shape (3, N, N, N) in position-column order."""
    gx = (np.roll(u, -1, axis=2) - np.roll(u, 1, axis=2)) / (2 * dx)
    gy = (np.roll(u, -1, axis=1) - np.roll(u, 1, axis=1)) / (2 * dx)
    gz = (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0)) / (2 * dx)
    return np.stack([gx, gy, gz])


# --------------------------------------------------------------------------
# (iii) mesh -> particles
# --------------------------------------------------------------------------
def cic_interpolate(field, x, cfg: Config):
    """sum_n field_n w(x_n - q) for each particle (same tent as the deposit)."""
    n = cfg.n_mesh
    base, f = cic_weights(x, cfg)
    flat = field.reshape(-1)
    out = np.zeros(x.shape[0])
    for dz in (0, 1):
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        iz = (base[:, 2] + dz) % n
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            iy = (base[:, 1] + dy) % n
            for dxo in (0, 1):
                wx = f[:, 0] if dxo else 1.0 - f[:, 0]
                ix = (base[:, 0] + dxo) % n
                out += flat[(iz * n + iy) * n + ix] * wx * wy * wz
    return out


def cic_interpolate_gradient(field, x, cfg: Config):
    """grad_q sum_n field_n w(x_n - q): the gradient, with respect to the
    particle position, of the cloud-in-cell interpolant.  This is the
    convolution of the mesh field with grad W of Eq. (equationofmotion)
    (grad_q W(x_n - q) = -grad W |_{x_n - q}).  Shape (N_p, 3)."""
    n = cfg.n_mesh
    base, f = cic_weights(x, cfg)
    flat = field.reshape(-1)
    g = np.zeros((x.shape[0], 3))
    for dz in (0, 1):
        wz, dwz = (f[:, 2], 1.0) if dz else (1.0 - f[:, 2], -1.0)
        iz = (base[:, 2] + dz) % n
        for dy in (0, 1):
            wy, dwy = (f[:, 1], 1.0) if dy else (1.0 - f[:, 1], -1.0)
            iy = (base[:, 1] + dy) % n
            for dxo in (0, 1):
                wx, dwx = (f[:, 0], 1.0) if dxo else (1.0 - f[:, 0], -1.0)
                ix = (base[:, 0] + dxo) % n
                v = flat[(iz * n + iy) * n + ix]
                g[:, 0] += v * dwx * wy * wz
                g[:, 1] += v * wx * dwy * wz
                g[:, 2] += v * wx * wy * dwz
    return g / cfg.dx


# --------------------------------------------------------------------------
# forces: steps (i)-(iii)
# --------------------------------------------------------------------------
def mesh_fields(x, cfg: Config):
    """Steps (i) and (ii) plus the gravity solve: rho, and the potentials the
    particles feel, phi~ and Q~ (Q~ = 0 for CDM).  With the spline kernel both
    potentials are convolved with the node weights once more: the density is
    S rho_cic, so the force, the derivative of the energy with respect to a
    particle position, goes through the transpose S (= S) back to the
    cloud-in-cell interpolant."""
    rho = density(x, cfg)
    phi = poisson_phi(rho, cfg)
    q = quantum_potential(rho, cfg) if cfg.quantum else np.zeros_like(rho)
    if cfg.kernel == KERNEL_SPLINE:
        phi = smooth(phi, cfg)
        if cfg.quantum:
            q = smooth(q, cfg)
    return rho, phi, q


def force_parts(x, cfg: Config, fields=None):
    """Per-particle gravity part g_phi and quantum part g_Q (shape (N_p, 3)) such
    that dp/dt = g_phi / a + g_Q / a^2.

    Two ways turn a mesh potential U into a particle force:
      central : -sum_n w(x_n - q) (grad_c U)_n, the central-difference mesh
                gradient interpolated with the deposit kernel (standard PM);
      kernel  : -grad_q sum_n U_n w(x_n - q), Eq. (equationofmotion): the
                potential convolved with the gradient of the kernel, which is
                minus the derivative of the discrete energy with respect to the
                particle position (sign from the Lagrange equation with
                L = K_v - K_rho - W_g).
    MESHGRAD uses central for both, HYBRID central for gravity and kernel for
    Q (the paper's scheme inside an unchanged PM gravity solver), LAGRANGIAN
    kernel for both.
    """
    rho, phi, q = fields if fields is not None else mesh_fields(x, cfg)

    def central(u):
        return -np.stack([cic_interpolate(c, x, cfg) for c in central_gradient(u, cfg.dx)], axis=1)

    def kernel(u):
        return -cic_interpolate_gradient(u, x, cfg)

    gphi = kernel(phi) if cfg.force_mode == LAGRANGIAN else central(phi)
    if not cfg.quantum:
        gq = np.zeros_like(gphi)
    elif cfg.force_mode == MESHGRAD:
        gq = central(q)
    else:
        gq = kernel(q)
    return gphi, gq


def accelerations(x, a, cfg: Config):
    """dp/dt = -grad(phi~)/a - grad(Q~)/a^2 at the particle positions (static
    runs: a = 1)."""
    gphi, gq = force_parts(x, cfg)
    aa = a if cfg.cosmological else 1.0
    return gphi / aa + gq / (aa * aa)


# --------------------------------------------------------------------------
# leapfrog (kick-drift-kick)
# --------------------------------------------------------------------------
def kick(p, parts, a0, a1, cfg: Config):
    gphi, gq = parts
    return p + kick_factor(a0, a1, cfg) * gphi + drift_factor(a0, a1, cfg) * gq


def drift(x, p, a0, a1, cfg: Config):
    return np.mod(x + drift_factor(a0, a1, cfg) * p, cfg.box)


def kdk_step(x, p, a0, a1, cfg: Config, parts0=None):
    """One kick-drift-kick step from a0 to a1.  Returns (x, p, parts at a1).

    The same density feeds gravity and the quantum pressure (Sec. II.A)."""
    ah = half_point(a0, a1, cfg)
    if parts0 is None:
        parts0 = force_parts(x, cfg)
    p = kick(p, parts0, a0, ah, cfg)
    x = drift(x, p, a0, a1, cfg)
    parts1 = force_parts(x, cfg)
    p = kick(p, parts1, ah, a1, cfg)
    return x, p, parts1


def scale_factors(a_start, a_end, nsteps, cfg: Config):
    """Step boundaries: uniform in ln a (cosmological) or in t (static)."""
    i = np.arange(nsteps + 1)
    if cfg.cosmological:
        return a_start * (a_end / a_start) ** (i / nsteps)
    return a_start + (a_end - a_start) * i / nsteps


def run(x, p, a_start, a_end, nsteps, cfg: Config, energy_every=0):
    """nsteps KDK steps; optionally energies every `energy_every` steps."""
    avals = scale_factors(a_start, a_end, nsteps, cfg)
    parts = None
    hist = []
    if energy_every:
        hist.append((avals[0],) + tuple(energies(x, p, avals[0], cfg)))
    for i in range(nsteps):
        x, p, parts = kdk_step(x, p, avals[i], avals[i + 1], cfg, parts)
        if energy_every and (i + 1) % energy_every == 0:
            hist.append((avals[i + 1],) + tuple(energies(x, p, avals[i + 1], cfg)))
    return x, p, hist


def next_scale_factor(p_sync, parts, a0, a_end, cfg: Config, cfl):
    """Adaptive step (Sec. II.A: the quantum acceleration enters the condition
    that no particle moves farther than dx in one step).  The step's drift is
    bounded by
        (max|p_sync| + K_g(a0, a_h) max|g_phi| + K_q(a0, a_h) max|g_Q|) D(a0, a1)
    (the opening half kick, then the drift with the kicked momentum); the
    step ends at the largest a1 <= a_end that keeps the bound within cfl*dx,
    found by bisection in ln a (static runs: in t)."""
    gphi, gq = parts
    pmax = float(np.max(np.sqrt(np.sum(p_sync * p_sync, axis=1)))) if len(p_sync) else 0.0
    gmax = float(np.max(np.sqrt(np.sum(gphi * gphi, axis=1)))) if len(gphi) else 0.0
    qmax = float(np.max(np.sqrt(np.sum(gq * gq, axis=1)))) if len(gq) else 0.0
    limit = cfl * cfg.dx

    def bound(a1):
        ah = half_point(a0, a1, cfg)
        return (pmax + kick_factor(a0, ah, cfg) * gmax + drift_factor(a0, ah, cfg) * qmax) * drift_factor(a0, a1, cfg)

    if bound(a_end) <= limit:
        return a_end
    lo, hi = 0.0, 1.0  # fraction of the interval in ln a (or t)

    def at(f):
        if cfg.cosmological:
            return a0 * (a_end / a0) ** f
        return a0 + (a_end - a0) * f

    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if bound(at(mid)) <= limit:
            lo = mid
        else:
            hi = mid
    return at(lo)


def run_adaptive(x, p, a_start, a_end, cfg: Config, cfl=0.5, max_steps=100000):
    """KDK steps from a_start to a_end with the adaptive step above; returns
    (x, p, the step boundaries)."""
    a = a_start
    parts = force_parts(x, cfg)
    bounds = [a]
    while a < a_end and len(bounds) <= max_steps:
        a1 = next_scale_factor(p, parts, a, a_end, cfg, cfl)
        x, p, parts = kdk_step(x, p, a, a1, cfg, parts)
        a = a1
        bounds.append(a)
    return x, p, np.array(bounds)


# --------------------------------------------------------------------------
# energies, Eq. (diskkinen) and Eq. (diskpoten)
# --------------------------------------------------------------------------
def energies(x, p, a, cfg: Config):
    """(K_v, W_g, K_rho, P_x, P_y, P_z) at scale factor a.

    K_v  = sum_i m_i (p_i/a)^2 / 2                 Eq. (diskkinen), peculiar u = p/a
    W_g  = (1/2a) sum_n (rho_n - 1) phi~_n dx^3     gravitational energy, Phi = phi~/a
    K_rho: compact Laplacian -> (hbar/m)^2/(2 a^2) dx sum_n sum_d (s_{n+d} - s_n)^2
           wide Laplacian    -> (hbar/m)^2/(2 a^2) (dx/4) sum_n sum_d (s_{n+d} - s_{n-d})^2,
           the printed form of Eq. (diskpoten); each is the energy whose
           derivative gives the matching Laplacian in Q.
    P    = sum_i m_i p_i.
    """
    aa = a if cfg.cosmological else 1.0
    npart = x.shape[0]
    mp = cfg.box ** 3 / npart
    kv = 0.5 * mp * float(np.sum(p * p)) / (aa * aa)
    rho = density(x, cfg)
    phi = poisson_phi(rho, cfg)
    wg = 0.5 / aa * float(np.sum((rho - 1.0) * phi)) * cfg.dx ** 3
    krho = 0.0
    if cfg.quantum:
        s = sqrt_rho(rho, cfg)
        acc = 0.0
        for ax in range(3):
            if cfg.lap == LAP_COMPACT:
                acc += float(np.sum((np.roll(s, -1, axis=ax) - s) ** 2))
            else:
                acc += 0.25 * float(np.sum((np.roll(s, -1, axis=ax) - np.roll(s, 1, axis=ax)) ** 2))
        krho = 0.5 * cfg.hbm ** 2 / (aa * aa) * cfg.dx * acc
    mom = mp * p.sum(axis=0)
    return kv, wg, krho, float(mom[0]), float(mom[1]), float(mom[2])


def layzer_irvine_residual(hist, cfg: Config):
    """eps(a) = [E(a) - E(a0) + int_{a0}^{a} (2K_v + W_g + 2K_rho)/a' da'] / |W_g(a)|
    with E = K_v + W_g + K_rho and the integral by the trapezoid rule over the
    recorded points.  W_g ~ 1/a and K_rho ~ 1/a^2 at fixed comoving positions
    give dE/da = -(2K_v + W_g + 2K_rho)/a for a conservative scheme."""
    h = np.asarray(hist)
    a, kv, wg, kr = h[:, 0], h[:, 1], h[:, 2], h[:, 3]
    e = kv + wg + kr
    integrand = (2 * kv + wg + 2 * kr) / a
    integral = np.concatenate([[0.0], np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(a))])
    return (e - e[0] + integral) / np.abs(wg)


# --------------------------------------------------------------------------
# power spectrum of the CIC density
# --------------------------------------------------------------------------
def power_spectrum(x, cfg: Config, nbins=None):
    """P(k) of delta = rho - 1 on the CIC mesh, deconvolved by the CIC window.

    P = (L^3/N^6) |delta^_k|^2 / prod_d sinc^4(k_d dx/2); shell i = 1..N/2
    collects (i - 1/2) k_f <= |k| < (i + 1/2) k_f over the full grid (both
    k and -k), k_f = 2 pi / L.  Returns (mean |k|, mean P, mode count) per
    shell; no shot-noise subtraction.
    """
    n = cfg.n_mesh
    if nbins is None:
        nbins = n // 2
    rho = cic_deposit(x, cfg)
    dk = np.fft.fftn(rho - 1.0)
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=cfg.dx)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    win = (np.sinc(kx * cfg.dx / (2 * np.pi)) * np.sinc(ky * cfg.dx / (2 * np.pi))
           * np.sinc(kz * cfg.dx / (2 * np.pi))) ** 2
    pk = cfg.box ** 3 / float(n) ** 6 * np.abs(dk) ** 2 / win ** 2
    kf = 2.0 * np.pi / cfg.box
    shell = np.floor(kmag / kf + 0.5).astype(np.int64)
    sel = (shell >= 1) & (shell <= nbins)
    cnt = np.bincount(shell[sel], minlength=nbins + 1)[1:]
    ksum = np.bincount(shell[sel], weights=kmag[sel], minlength=nbins + 1)[1:]
    psum = np.bincount(shell[sel], weights=pk[sel], minlength=nbins + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt
