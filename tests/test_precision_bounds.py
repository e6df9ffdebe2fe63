"""The error bound behind the fp32 stencil's choice of which near-empty
nodes to redo in float-float: with every s = sqrt(rho) within 2^-22 of its
value and the sums of the seven-point Laplacian rounded in fp32, the fp32
Laplacian lies within 2^-21 * mag of the exact one (mag = the six
neighbours' s + 6 s_0, the absolute terms of the Laplacian), so where mag <= 4 |lap| the fp32 Q~ keeps ~1.9e-6 relative
accuracy.  Checked here by emulating the fp32 arithmetic (numpy float32, each
s perturbed by up to 2^-22 as an approximate reciprocal square root may be)
against float64."""
import numpy as np


def _fp32_laplacian(s):
    """The kernels' association: (dxp + (sxm - s0)) + (dyp + (sym - s0)) + (dzp + (szm - s0))."""
    s0, sxp, sxm, syp, sym, szp, szm = (v.astype(np.float32) for v in s)
    dxp, dyp, dzp = sxp - s0, syp - s0, szp - s0
    return ((dxp + (sxm - s0)) + (dyp + (sym - s0))) + (dzp + (szm - s0))


def _samples(rng, m):
    """Near-empty centres next to neighbours of every kind: denser, equally
    sparse, floored, and nearly equal (cancelling) ones."""
    rho = np.exp(rng.uniform(np.log(1e-6), np.log(1e-2), size=(7, m)))
    kind = rng.integers(0, 4, size=(6, m))
    dense = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), size=(6, m)))
    close = rho[0] * (1.0 + rng.normal(0.0, 1e-5, size=(6, m)))
    rho[1:] = np.where(kind == 0, dense, np.where(kind == 1, close, np.where(kind == 2, 1e-6, rho[1:])))
    return np.maximum(rho.astype(np.float32).astype(np.float64), 1e-6)


def test_fp32_laplacian_error_is_within_2_pow_minus_21_of_mag():
    rng = np.random.default_rng(11)
    rho = _samples(rng, 200_000)
    s_exact = np.sqrt(rho)
    s_fp32 = (s_exact * (1.0 + rng.uniform(-1.0, 1.0, size=rho.shape) * 2.0 ** -22)).astype(np.float32)
    lap32 = _fp32_laplacian(s_fp32).astype(np.float64)
    lap = s_exact[1:].sum(axis=0) - 6.0 * s_exact[0]
    mag = s_exact.sum(axis=0) + 5.0 * s_exact[0]
    err = np.abs(lap32 - lap)
    assert np.all(err <= 2.0 ** -21 * mag)
    # the kept nodes (mag <= 4 |lap|) are within 1.9e-6 relative, the others can be far off
    kept = mag <= 4.0 * np.abs(lap)
    assert kept.any() and (~kept).any()
    assert np.max(err[kept] / np.abs(lap[kept])) <= 4.0 * 2.0 ** -21
    assert np.max(err[~kept] / np.maximum(np.abs(lap[~kept]), 1e-300)) > 1e-4
