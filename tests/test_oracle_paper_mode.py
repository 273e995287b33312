"""Pins of the oracle's paper mode (Section 2.2, Eq. 8: Phi' = C-hat F U with
Fourier-space upsampling, on-grid visibilities, linear chirp of Eq. 5)."""
import math
import os

import numpy as np

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

L = synth.fov_L()
HERE = os.path.dirname(os.path.abspath(__file__))


def test_sparse_rows_reproduce_the_definition_at_E1():
    # C-hat rows (FFT of the chirp on the upsampled image) applied to F U x equal
    # F(c_k . U x) sampled at the visibility's cell, evaluated directly
    N = 8
    prob = synth.paper_problem(N, 0.3, seed=1)
    x = np.random.default_rng(2).standard_normal((N, N))
    Gm = O.build_G(O.paper_geometry(N, L), prob.uvw, 1.0)
    y = O.paper_phi(N, Gm, x)
    yd = O.paper_visibilities_direct(N, L, x, prob.uvw)
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)


def test_upsampling_is_an_isometry_and_band_limited():
    N, G = 16, 32
    x = np.random.default_rng(3).standard_normal((N, N))
    ux = O.paper_upsample(x, G)
    assert abs(np.linalg.norm(ux) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)
    X = np.fft.fft2(ux)
    k = np.abs(np.where(np.arange(G) < G // 2, np.arange(G), np.arange(G) - G))
    outside = (k[:, None] > N // 2) | (k[None, :] > N // 2)
    assert np.max(np.abs(X[outside])) <= 1e-10 * np.max(np.abs(X))
    # even-indexed samples of U x are x scaled by N/G (interpolation through the pixels)
    xn = np.roll(x, (-(N // 2), -(N // 2)), axis=(0, 1))
    assert np.allclose(ux[::2, ::2].real * G / N, xn, atol=1e-12)


def test_adjoint_identity_and_zero_w():
    N = 8
    rng = np.random.default_rng(4)
    prob = synth.paper_problem(N, 0.5, seed=5)
    Gm = O.build_G(O.paper_geometry(N, L), prob.uvw, 1.0)
    x = rng.standard_normal((N, N))
    y = rng.standard_normal(Gm.shape[0]) + 1j * rng.standard_normal(Gm.shape[0])
    lhs = np.vdot(y, O.paper_phi(N, Gm, x))
    rhs = np.vdot(O.paper_phi_adj(N, Gm, y), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # w = 0: every row is the single entry 1 at the visibility's cell, so Phi' x
    # samples the upsampled spectrum
    p0 = synth.paper_problem(N, 0.5, seed=6, wd=0.0)
    G0 = O.build_G(O.paper_geometry(N, L), p0.uvw, 0.75).tocsr()
    assert np.all(np.diff(G0.indptr) == 1) and np.allclose(G0.data, 1.0)
    X = O.paper_spectrum(x, 2 * N)
    j = np.floor(p0.uvw[:, :2] * L).astype(int) % (2 * N)
    assert np.allclose(O.paper_phi(N, G0, x), X[j[:, 0], j[:, 1]])


def test_row_energy_is_one():
    # unitary transforms: the chirp has unit modulus, so every C-hat row has
    # energy sum |C-hat|^2 = 1 (Parseval)
    N = 16
    prob = synth.paper_problem(N, 0.05, seed=7)
    geo = O.paper_geometry(N, L)
    for k in range(5):
        K, _, _ = O.kernel_box(geo, *prob.uvw[k], 2 * N)
        assert abs(np.sum(np.abs(K) ** 2) - 1.0) <= 1e-12


def test_nonzero_proportion_follows_the_paper():
    # the proportion of non-zero entries of C-hat against E (Section 3.2):
    # within a factor 2 of the printed values, increasing in E
    ref = np.loadtxt(os.path.join(HERE, "golden", "paper_nnz_fraction.txt"))
    N = 64
    prob = synth.paper_problem(N, 0.01, seed=0)
    rows = prob.uvw[:60]
    geo = O.paper_geometry(N, L)
    frac = []
    for E, printed in ref:
        nnz = sum(O.kernel_row(geo, *r, 2 * N, E)[0].size for r in rows)
        f = nnz / (rows.shape[0] * (2 * N) ** 2)
        frac.append(f)
        assert printed / 2 <= f <= printed * 2, (E, f, printed)
    assert frac[0] > frac[1] > frac[2]


def test_linear_chirp_box_is_separable():
    # exp(pi i w (l^2 + m^2)) = exp(pi i w l^2) exp(pi i w m^2): the kernel box of
    # a paper-mode row (one tap at offset 0) is, up to one constant, the outer
    # product g g^T with g[a] = f[-a mod G] and f the 1-D centred DFT of the axis
    # chirp (what a separable build computes instead of a 2-D FFT)
    N = 16
    geo = O.paper_geometry(N, L)
    G = geo.G
    prob = synth.paper_problem(N, 0.1, seed=6)
    lp = O.box_coords(G, geo.L, geo.extension)
    for k in range(5):
        u, v, w = prob.uvw[k]
        K, _, _ = O.kernel_box(geo, u, v, w, G)
        f = np.fft.fft(np.fft.ifftshift(O.chirp(lp, 0.0, w, "linear")))
        g = f[(-np.arange(G)) % G]
        P = np.outer(g, g)
        c = K[0, 0] / P[0, 0]
        assert abs(abs(c) - 1.0 / G ** 2) <= 1e-12 / G ** 2   # 1/G of the unitary 2-D DFT, 1/G of the box
        assert np.allclose(K, c * P, rtol=0, atol=1e-12 * np.abs(K).max())
