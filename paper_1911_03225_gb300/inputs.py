"""Seeded synthetic initial fields for the FDM layer problem.

This module is shared by the GPU path's callers (tests, benchmark) and by the oracle's
tests; it holds none of the method's arithmetic (no static solve, no transport step),
only closed-form or filtered initial data:

* ``lines_alpha`` / ``lines_up``: two straight edge-dislocation walls of opposite sign
  (alpha12 = +-Gaussian bands, alpha11 = 0), the annihilation problem of Sec. 4.3 with
  Gaussian cross-sections in place of the half-square waves;
* ``ring_alpha`` / ``ring_up``: a smooth circular loop (Sec. 4.4.1), tangent-oriented
  Nye vector with a Gaussian cross-section, U13 = integral of the profile;
* ``modulus_factor``: a smooth random shear-modulus factor for the heterogeneous static
  problem;
* ``random_up``: a zero-mean Gaussian random U13 field (Sec. 5.4 microstructure B) from a
  counter-based generator (SplitMix64, Steele-Lea-Flood 2014, and the Box-Muller
  transform), smoothed by a Gaussian filter exp(-|xi|^2 l^2 / 4) and scaled to a target
  RMS of |alpha|.

All fields are row-major [n2][n1] float64 (x1 fastest).
"""
import math

import numpy as np
from scipy.special import erf, erfc

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (stateless form)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def normal_field(n1: int, n2: int, seed: int) -> np.ndarray:
    """Per-cell N(0,1) draws keyed by (seed, cell index), Box-Muller on two uniforms."""
    idx = np.arange(n1 * n2, dtype=np.uint64)
    base = np.uint64(seed) << np.uint64(40)
    u1 = (splitmix64(base + np.uint64(2) * idx) >> np.uint64(11)).astype(np.float64)
    u2 = (splitmix64(base + np.uint64(2) * idx + np.uint64(1)) >> np.uint64(11)).astype(np.float64)
    u1 = (u1 + 0.5) * 2.0 ** -53          # in (0, 1)
    u2 = u2 * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return z.reshape(n2, n1)


def _centred_coords(n1, n2, cx, cy):
    """Minimum-image offsets of every node from (cx, cy) on the periodic grid."""
    x = np.arange(n1, dtype=np.float64) - cx
    y = np.arange(n2, dtype=np.float64) - cy
    x = (x + n1 / 2.0) % n1 - n1 / 2.0
    y = (y + n2 / 2.0) % n2 - n2 / 2.0
    return np.meshgrid(x, y)


def lines_alpha(n: int, sep: float = 32.0, sigma: float = 3.0, amp: float = 1.0):
    """Two straight edge walls at x1 = n/2 -+ sep/2, alpha12 = +-amp G, alpha11 = 0.

    Returns (alpha11, alpha12)."""
    x = np.arange(n, dtype=np.float64)
    c1, c2 = n / 2.0 - sep / 2.0, n / 2.0 + sep / 2.0
    g = amp * (np.exp(-((x - c1) ** 2) / (2 * sigma ** 2)) - np.exp(-((x - c2) ** 2) / (2 * sigma ** 2)))
    a12 = np.tile(g, (n, 1))
    return np.zeros_like(a12), a12


def lines_up(n: int, sep: float = 32.0, sigma: float = 3.0, amp: float = 1.0):
    """U13 whose x1-derivative is ``lines_alpha``'s alpha12 (closed form with erf)."""
    x = np.arange(n, dtype=np.float64)
    c1, c2 = n / 2.0 - sep / 2.0, n / 2.0 + sep / 2.0
    s = sigma * math.sqrt(2.0)
    f = amp * sigma * math.sqrt(math.pi / 2.0) * (erf((x - c1) / s) - erf((x - c2) / s))
    return np.tile(f, (n, 1))


def ring_profile(r, r0: float, sigma: float, amp: float = 1.0):
    """U13 of the smooth loop as a function of radius: amp * int_r^inf exp(-(s-r0)^2/(2 sigma^2)) ds."""
    return amp * sigma * math.sqrt(math.pi / 2.0) * erfc((np.asarray(r) - r0) / (sigma * math.sqrt(2.0)))


def ring_up(n: int, r0: float = 100.0, sigma: float = 2.0, amp: float = 1.0):
    x, y = _centred_coords(n, n, n / 2.0, n / 2.0)
    return ring_profile(np.hypot(x, y), r0, sigma, amp)


def ring_alpha(n: int, r0: float = 100.0, sigma: float = 2.0, amp: float = 1.0):
    """Tangent-oriented Nye field of the loop: alpha11 = -dU/dx2, alpha12 = dU/dx1 with
    U = ring_profile(r).  Returns (alpha11, alpha12)."""
    x, y = _centred_coords(n, n, n / 2.0, n / 2.0)
    r = np.hypot(x, y)
    g = amp * np.exp(-((r - r0) ** 2) / (2 * sigma ** 2))
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(r > 0, x / r, 0.0)
        uy = np.where(r > 0, y / r, 0.0)
    # dU/dr = -g  ->  dU/dx1 = -g x/r, dU/dx2 = -g y/r
    return g * uy, -g * ux


def square_signed_distance(x, y, half_side: float):
    """Signed Euclidean distance to the square |x|, |y| <= half_side (negative inside)."""
    qx, qy = np.abs(x) - half_side, np.abs(y) - half_side
    outside = np.hypot(np.maximum(qx, 0.0), np.maximum(qy, 0.0))
    return outside + np.minimum(np.maximum(qx, qy), 0.0)


def loop_profile(d, sigma: float, amp: float = 1.0):
    """U13 across a loop with a Gaussian cross-section centred on the loop line, as a
    function of the signed distance d to that line: amp * int_d^inf exp(-s^2/(2 sigma^2)) ds."""
    return amp * sigma * math.sqrt(math.pi / 2.0) * erfc(np.asarray(d) / (sigma * math.sqrt(2.0)))


def square_up(n: int, half_side: float = 60.0, sigma: float = 2.0, amp: float = 1.0, centre=None):
    """Polygonal (square) loop: U13 = loop_profile(signed distance to the square's edges)
    (Sec. 4.4.2's loop with corners), centred at `centre` (default: the cell centre)."""
    cx, cy = centre if centre is not None else (n / 2.0, n / 2.0)
    x, y = _centred_coords(n, n, cx, cy)
    return loop_profile(square_signed_distance(x, y, half_side), sigma, amp)


def random_up(n: int, seed: int = 0, ell: float = 16.0, rms_alpha: float = 0.1, dx: float = 1.0):
    """Zero-mean smoothed Gaussian random U13 with RMS |grad U13| = rms_alpha."""
    z = normal_field(n, n, seed)
    k = np.fft.fftfreq(n, d=dx) * 2.0 * math.pi
    kx, ky = np.meshgrid(k, k)
    q = kx ** 2 + ky ** 2
    zh = np.fft.fft2(z) * np.exp(-q * ell ** 2 / 4.0)
    zh[0, 0] = 0.0
    u = np.real(np.fft.ifft2(zh))
    # RMS of the gradient by Parseval on the filtered spectrum (scale factor only)
    g2 = np.sum(q * np.abs(zh) ** 2) / float(n * n) ** 2
    u *= rms_alpha / math.sqrt(g2)
    return u - u.mean()


def modulus_factor(n1: int, n2: int, seed: int = 0, lo: float = 0.25, hi: float = 1.0, ell: float = 16.0):
    """Smooth random factor of the shear modulus with values spread over [lo, hi] (contrast
    hi / lo), for the heterogeneous static problem: the counter-based normals of
    ``normal_field`` smoothed by exp(-|xi|^2 l^2 / 4) and mapped affinely onto [lo, hi]."""
    z = normal_field(n1, n2, seed)
    k1 = np.fft.fftfreq(n1) * 2.0 * math.pi
    k2 = np.fft.fftfreq(n2) * 2.0 * math.pi
    q = k1[None, :] ** 2 + k2[:, None] ** 2
    f = np.real(np.fft.ifft2(np.fft.fft2(z) * np.exp(-q * ell ** 2 / 4.0)))
    f = (f - f.min()) / (f.max() - f.min())
    return lo + (hi - lo) * f
