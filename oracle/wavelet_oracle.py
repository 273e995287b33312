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


def dwt1(x: np.ndarray, h: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """One periodic analysis level of a 1-D signal of even length n."""
    n = x.size
    g = highpass_taps(h)
    a = np.zeros(n // 2, dtype=np.result_type(x, h))
    d = np.zeros(n // 2, dtype=np.result_type(x, h))
    for i in range(n // 2):
        for k in range(h.size):
            a[i] += h[k] * x[(2 * i + k) % n]
            d[i] += g[k] * x[(2 * i + k) % n]
    return a, d


def idwt1(a: np.ndarray, d: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Transpose of dwt1: x_j = sum_{i,k : (2i + k) mod n = j} (h_k a_i + g_k d_i)."""
    n = 2 * a.size
    g = highpass_taps(h)
    x = np.zeros(n, dtype=np.result_type(a, h))
    for i in range(n // 2):
        for k in range(h.size):
            x[(2 * i + k) % n] += h[k] * a[i] + g[k] * d[i]
    return x


def _level_2d(block: np.ndarray, h: np.ndarray) -> np.ndarray:
    n = block.shape[0]
    hh = n // 2
    tmp = np.empty_like(block)
    for r in range(n):                       # fast axis
        a, d = dwt1(block[r], h)
        tmp[r, :hh], tmp[r, hh:] = a, d
    out = np.empty_like(block)
    for c in range(n):                       # slow axis
        a, d = dwt1(tmp[:, c], h)
        out[:hh, c], out[hh:, c] = a, d
    return out


def _ilevel_2d(block: np.ndarray, h: np.ndarray) -> np.ndarray:
    n = block.shape[0]
    hh = n // 2
    tmp = np.empty_like(block)
    for c in range(n):                       # slow axis first (reverse order)
        tmp[:, c] = idwt1(block[:hh, c], block[hh:, c], h)
    out = np.empty_like(block)
    for r in range(n):
        out[r] = idwt1(tmp[r, :hh], tmp[r, hh:], h)
    return out


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
