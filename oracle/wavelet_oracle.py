"""FP64 CPU oracle of the Daubechies wavelet sparsity basis Psi (Section 2.3, Eq. 7;
Daubechies 8 wavelets are the paper's second dictionary, Section 4).

TEST INFRASTRUCTURE ONLY: imported by tests/ (never by the product package).
It shares no code with the CUDA path; the filter taps are generated here from
their mathematical definition with numpy.roots as the only library primitive.

Readings of the paper (it names the basis and nothing else):
  * "Daubechies 8" is the extremal-phase (minimum-phase) orthonormal Daubechies
    wavelet with p = 8 vanishing moments, 2p = 16 taps (the usual db8).
  * The image boundary is periodic, so Psi is an orthonormal N^2 x N^2 matrix
    and the synthesis problem of Eq. 7 (min ||alpha||_1 s.t.
    ||y - Phi Psi alpha|| <= eps) equals the analysis problem in x = Psi alpha.
  * Decomposition depth: `levels` (default 4) dyadic levels of the separable
    2-D transform; N must be divisible by 2^levels.

Construction of the taps (Daubechies' spectral factorisation): with
y = sin^2(omega/2), the squared modulus of the low-pass response is
cos^{2p}(omega/2) P_p(y), P_p(y) = sum_{k<p} C(p-1+k, k) y^k.  Each root y_k of
P_p gives the pair of z-roots of z^2 - (2 - 4 y_k) z + 1 = 0; the one inside the
unit circle is kept (minimum phase).  H(z) = (1 + z)^p prod_k (z - z_k), scaled
to sum sqrt(2), listed so that the taps' energy is front-loaded.

Transform conventions (one level on an even length n, periodic):
  a_i = sum_k h_k x_{(2i + k) mod n},   d_i = sum_k g_k x_{(2i + k) mod n},
  g_k = (-1)^k h_{2p-1-k};  i in [0, n/2).
Its inverse is its transpose.  In 2-D one level filters the fast axis (columns
index) and then the slow axis; the n x n block becomes four n/2 x n/2 blocks of
the Mallat layout: [0:h, 0:h] low-low, [0:h, h:n] low (slow) / high (fast),
[h:n, 0:h] high (slow) / low (fast), [h:n, h:n] high-high.  The next level
transforms the low-low block in place of the array.
"""
from __future__ import annotations

import math

import numpy as np


def daubechies_taps(p: int) -> np.ndarray:
    """Low-pass analysis taps h_0 .. h_{2p-1} of the extremal-phase Daubechies
    wavelet with p vanishing moments (sum h = sqrt 2, sum h^2 = 1)."""
    if p < 1:
        raise ValueError("p >= 1")
    # P_p(y) = sum_{k<p} C(p-1+k, k) y^k; numpy.roots wants the highest power first
    coef = [math.comb(p - 1 + k, k) for k in range(p)]
    yk = np.roots(coef[::-1]) if p > 1 else np.zeros(0)
    zk = []
    for y in yk:
        b = 2.0 - 4.0 * y                  # z^2 - b z + 1 = 0
        disc = np.sqrt(complex(b * b - 4.0))
        r1, r2 = (b + disc) / 2.0, (b - disc) / 2.0
        zk.append(r1 if abs(r1) < 1.0 else r2)
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])    # (z + 1)
    for z in zk:
        poly = np.convolve(poly, [1.0, -z])     # (z - z_k)
    h = np.real(poly)                            # conjugate roots pair up: real coefficients
    h = h * (math.sqrt(2.0) / h.sum())
    # front-load the energy: the order whose early partial energies are larger
    e_fwd = np.cumsum(h ** 2)
    e_rev = np.cumsum(h[::-1] ** 2)
    if e_rev.sum() > e_fwd.sum():
        h = h[::-1]
    return h.copy()


def highpass_taps(h: np.ndarray) -> np.ndarray:
    """g_k = (-1)^k h_{L-1-k} (quadrature mirror)."""
    L = h.size
    return np.array([(-1.0) ** k * h[L - 1 - k] for k in range(L)])


def dwt1(x: np.ndarray, h: np.ndarray, axis: int = -1) -> tuple[np.ndarray, np.ndarray]:
    """One periodic analysis level along `axis` (even length n):
    a_i = sum_k h_k x_{(2i + k) mod n}, d_i = sum_k g_k x_{(2i + k) mod n}."""
    x = np.moveaxis(np.asarray(x), axis, -1)
    n = x.shape[-1]
    g = highpass_taps(h)
    i = np.arange(n // 2)
    a = np.zeros(x.shape[:-1] + (n // 2,), dtype=np.result_type(x, h))
    d = np.zeros_like(a)
    for k in range(h.size):
        xs = x[..., (2 * i + k) % n]
        a += h[k] * xs
        d += g[k] * xs
    return np.moveaxis(a, -1, axis), np.moveaxis(d, -1, axis)


def idwt1(a: np.ndarray, d: np.ndarray, h: np.ndarray, axis: int = -1) -> np.ndarray:
    """Transpose of dwt1: x_j = sum_{i,k : (2i + k) mod n = j} (h_k a_i + g_k d_i)."""
    a = np.moveaxis(np.asarray(a), axis, -1)
    d = np.moveaxis(np.asarray(d), axis, -1)
    n = 2 * a.shape[-1]
    g = highpass_taps(h)
    i = np.arange(n // 2)
    x = np.zeros(a.shape[:-1] + (n,), dtype=np.result_type(a, h))
    for k in range(h.size):
        # the positions (2i + k) mod n are distinct over i for a fixed k
        x[..., (2 * i + k) % n] += h[k] * a + g[k] * d
    return np.moveaxis(x, -1, axis)


def _level_2d(block: np.ndarray, h: np.ndarray) -> np.ndarray:
    n = block.shape[0]
    hh = n // 2
    lo, hi = dwt1(block, h, axis=1)          # fast axis
    out = np.empty_like(block)
    out[:hh, :hh], out[hh:, :hh] = dwt1(lo, h, axis=0)     # slow axis
    out[:hh, hh:], out[hh:, hh:] = dwt1(hi, h, axis=0)
    return out


def _ilevel_2d(block: np.ndarray, h: np.ndarray) -> np.ndarray:
    hh = block.shape[0] // 2
    lo = idwt1(block[:hh, :hh], block[hh:, :hh], h, axis=0)   # slow axis first (reverse order)
    hi = idwt1(block[:hh, hh:], block[hh:, hh:], h, axis=0)
    return idwt1(lo, hi, h, axis=1)


def check_levels(N: int, levels: int) -> None:
    if levels < 0 or N % (1 << levels) != 0:
        raise ValueError("N must be divisible by 2^levels")


def dwt2(x: np.ndarray, levels: int = 4, p: int = 8) -> np.ndarray:
    """alpha = Psi^T x: the periodic 2-D Daubechies-p analysis in Mallat layout."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    check_levels(N, levels)
    h = daubechies_taps(p)
    c = x.copy()
    n = N
    for _ in range(levels):
        c[:n, :n] = _level_2d(c[:n, :n], h)
        n //= 2
    return c


def idwt2(c: np.ndarray, levels: int = 4, p: int = 8) -> np.ndarray:
    """x = Psi alpha: the synthesis (inverse and transpose of dwt2)."""
    c = np.asarray(c, dtype=np.float64)
    N = c.shape[0]
    check_levels(N, levels)
    h = daubechies_taps(p)
    x = c.copy()
    n = N >> levels
    for _ in range(levels):
        n *= 2
        x[:n, :n] = _ilevel_2d(x[:n, :n], h)
    return x
