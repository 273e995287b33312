"""Pins of the Daubechies wavelet oracle (the Psi of Eq. 7) against facts that do
not come from the oracle: closed forms of the short filters, the defining
conditions of the Daubechies family, a convolution computed by FFT, the Haar
averages and differences, orthonormality of the whole matrix, and BPDN's closed
form for an isometry."""
import math

import numpy as np
import pytest

from oracle import wavelet_oracle as W
from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

L = synth.fov_L()


def test_short_filters_closed_forms():
    # p = 1 is Haar; p = 2 is Daubechies' (1 + sqrt3, 3 + sqrt3, 3 - sqrt3, 1 - sqrt3) / (4 sqrt2)
    assert np.allclose(W.daubechies_taps(1), [1 / math.sqrt(2)] * 2, atol=1e-15)
    s3 = math.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.allclose(W.daubechies_taps(2), ref, atol=1e-14)


@pytest.mark.parametrize("p", [3, 4, 6, 8])
def test_daubechies_defining_conditions(p):
    h = W.daubechies_taps(p)
    assert h.size == 2 * p
    # orthonormal to its even shifts
    for m in range(p):
        acc = math.fsum(h[k] * h[k + 2 * m] for k in range(2 * p - 2 * m))
        assert abs(acc - (1.0 if m == 0 else 0.0)) <= 1e-13, (m, acc)
    assert abs(math.fsum(h) - math.sqrt(2.0)) <= 1e-13
    # p vanishing moments of the wavelet: sum_k (-1)^k k^j h_k = 0 for j < p
    for j in range(p):
        terms = [(-1) ** k * float(k) ** j * h[k] for k in range(2 * p)]
        assert abs(math.fsum(terms)) <= 1e-11 * math.fsum(abs(t) for t in terms), j
    terms = [(-1) ** k * float(k) ** p * h[k] for k in range(2 * p)]
    assert abs(math.fsum(terms)) > 1e-3 * math.fsum(abs(t) for t in terms)     # exactly p, not more
    # extremal phase: H(zeta) = sum h_k zeta^k has its p-fold zero at -1 and all
    # other zeros outside the unit circle
    q = np.array(h[::-1], dtype=np.float64)            # highest power first
    for _ in range(p):
        q, rem = np.polydiv(q, [1.0, 1.0])
        assert abs(rem[-1]) <= 1e-9
    assert np.all(np.abs(np.roots(q)) > 1.0 + 1e-6)


@pytest.mark.parametrize("p", [1, 2, 8])
def test_one_level_is_periodic_correlation_by_fft(p):
    # a_i = (x correlated with h)[2i], computed here with an FFT
    rng = np.random.default_rng(p)
    n = 32
    x = rng.standard_normal(n)
    h = W.daubechies_taps(p)
    g = W.highpass_taps(h)
    a, d = W.dwt1(x, h)
    for f, got in ((h, a), (g, d)):
        fp = np.zeros(n)
        for k in range(f.size):
            fp[k % n] += f[k]
        corr = np.real(np.fft.ifft(np.fft.fft(x) * np.conj(np.fft.fft(fp))))
        assert np.allclose(got, corr[::2], atol=1e-13)
    assert np.allclose(W.idwt1(a, d, h), x, atol=1e-13)


def test_haar_level_is_averages_and_differences():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((8, 8))
    c = W.dwt2(x, levels=1, p=1)
    x00, x01, x10, x11 = x[0::2, 0::2], x[0::2, 1::2], x[1::2, 0::2], x[1::2, 1::2]
    assert np.allclose(c[:4, :4], (x00 + x01 + x10 + x11) / 2, atol=1e-14)
    assert np.allclose(c[:4, 4:], (x00 - x01 + x10 - x11) / 2, atol=1e-14)    # high along the fast axis
    assert np.allclose(c[4:, :4], (x00 + x01 - x10 - x11) / 2, atol=1e-14)    # high along the slow axis
    assert np.allclose(c[4:, 4:], (x00 - x01 - x10 + x11) / 2, atol=1e-14)


@pytest.mark.parametrize("N,levels,p", [(16, 2, 8), (16, 4, 8), (8, 3, 2)])
def test_psi_is_an_orthonormal_matrix(N, levels, p):
    # columns Psi e_j for every pixel: Psi^T Psi = I, and dwt2 is its transpose
    cols = np.empty((N * N, N * N))
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        cols[:, j] = W.idwt2(e.reshape(N, N), levels, p).ravel()
    assert np.allclose(cols.T @ cols, np.eye(N * N), atol=1e-12)
    rng = np.random.default_rng(N + levels)
    x = rng.standard_normal((N, N))
    assert np.allclose(W.dwt2(x, levels, p).ravel(), cols.T @ x.ravel(), atol=1e-12)


def test_smooth_image_is_sparse_in_db8():
    # 8 vanishing moments: a smooth periodic image leaves only tiny detail
    # coefficients at the finest level
    N = 64
    t = np.arange(N) / N
    x = np.outer(np.cos(2 * np.pi * t), np.sin(2 * np.pi * t) + 0.5)
    c = W.dwt2(x, levels=1, p=8)
    assert np.max(np.abs(c[32:, :])) <= 1e-6 * np.max(np.abs(c))
    assert np.max(np.abs(c[:32, 32:])) <= 1e-6 * np.max(np.abs(c))


def test_levels_must_divide_the_side():
    with pytest.raises(ValueError):
        W.dwt2(np.zeros((24, 24)), levels=4)


def test_bpdn_with_db8_reaches_closed_form_for_an_isometry():
    # Eq. 7 with Psi = Db8: Phi Psi is an isometry when Phi is, so the solution
    # in alpha is soft(Psi^T Re Phi^H y, l*) and x = Psi alpha.
    N, levels = 8, 2
    geo = O.Geometry(N, L, W=1)
    G = geo.G
    qu, qv = np.meshgrid(np.arange(G) - G // 2, np.arange(G) - G // 2, indexing="ij")
    uvw = np.stack([qu.ravel() * geo.du, qv.ravel() * geo.du, np.zeros(G * G)], 1)
    Gm = O.build_G(geo, uvw, 1.0)

    def ap(a):
        return O.phi(geo, Gm, W.idwt2(a, levels))

    def aa(r):
        return W.dwt2(np.real(O.phi_adj(geo, Gm, r)), levels)

    rng = np.random.default_rng(1)
    x = np.maximum(rng.standard_normal((N, N)), 0)
    y = O.phi(geo, Gm, x) + 0.05 * (rng.standard_normal(G * G) + 1j * rng.standard_normal(G * G))
    b = aa(y)
    c0 = np.sum(np.abs(y) ** 2) - np.sum(b ** 2)
    eps = math.sqrt(c0 + 0.3 * np.sum(b ** 2))
    a_star = O.bpdn_closed_form_isometry(b, eps, c0)
    ar, _ = O.solve_bpdn(ap, aa, y, eps, N, 200, inner_iters=10, phi_norm2=1.0)
    assert np.linalg.norm(ar - a_star) <= 1e-6 * np.linalg.norm(a_star)
    assert np.linalg.norm(y - ap(ar)) <= eps * (1 + 1e-6)
