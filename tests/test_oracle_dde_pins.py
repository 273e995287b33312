"""Pins of the oracle's direction-dependent screens (Section 3.2: the per-row
threshold makes no assumption on a row's structure, so any image-space
modulation goes through the same FFT and threshold).  Each fact below holds
without the oracle: a unit screen changes nothing, a phase ramp is the Fourier
shift theorem, a constant modulus scales the energy, and the rows reproduce a
brute-force pixel sum of the measurement equation with the screen."""
import math

import numpy as np
import pytest

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

L = synth.fov_L()


def test_unit_screen_changes_nothing():
    geo = O.Geometry(16, L)
    uvw = synth.random_uvw(np.random.default_rng(0), 12, 16, L)
    ones = np.ones((1, geo.G, geo.G), dtype=np.complex128)
    a = O.build_G(geo, uvw, 0.99)
    b = O.build_G(geo, uvw, 0.99, screens=ones, screen_id=np.zeros(12, int))
    assert (a != b).nnz == 0


@pytest.mark.parametrize("su,sv", [(3, 0), (0, -5), (2, 7)])
def test_phase_ramp_screen_shifts_the_visibility(su, sv):
    # A(l, m) = exp(-2 pi i (su du l + sv du m)) at l = (P - G/2) L / N moves the
    # visibility by (su, sv) grid cells: the rows agree as functions of the column
    N = 16
    geo = O.Geometry(N, L)
    G = geo.G
    off = np.arange(G) - G // 2
    ramp = np.exp(-2j * np.pi * (su * off[:, None] + sv * off[None, :]) / G)
    rng = np.random.default_rng(abs(su) + 10 * abs(sv))
    for _ in range(4):
        u, v = rng.uniform(-0.3, 0.3, 2) * synth.band_limit(N, L)
        w = rng.uniform(0, 1) * N / (L * L)
        K1, a0, b0 = O.kernel_box(geo, u, v, w, G, ramp)
        K2, a1, b1 = O.kernel_box(geo, u + su * geo.du, v + sv * geo.du, w, G)
        c1 = O.box_columns(geo, a0, b0, G).ravel()
        c2 = O.box_columns(geo, a1, b1, G).ravel()
        r1 = np.zeros(G * G, complex)
        r2 = np.zeros(G * G, complex)
        r1[c1] = K1.ravel()
        r2[c2] = K2.ravel()
        assert np.allclose(r1, r2, atol=1e-12 * np.abs(r2).max())


def test_constant_modulus_screen_scales_the_energy():
    # Parseval: |A| = 2 everywhere -> E = 4 (sum kb^2)(sum kb^2)
    geo = O.Geometry(16, L)
    rng = np.random.default_rng(3)
    scr = 2.0 * np.exp(2j * np.pi * rng.uniform(size=(geo.G, geo.G)))
    for _ in range(3):
        u, v = rng.uniform(-100, 100, 2)
        w = rng.uniform(0, 50)
        K, _, _ = O.kernel_box(geo, u, v, w, geo.G, scr)
        assert abs(math.fsum(np.abs(K.ravel()) ** 2) - 4 * O.energy_closed_form(geo, u, v)) <= \
            1e-12 * 4 * O.energy_closed_form(geo, u, v)


@pytest.mark.parametrize("N", [8, 16])
def test_dde_phi_matches_brute_force_measurement_equation(N):
    # e = 1, S = G: Phi with screens against the pixel sum, to the KB error
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(N)
    M = 60
    uvw = synth.random_uvw(rng, M, N, L)
    screens = synth.dde_screens(3, N, L, seed=N).astype(np.complex128)
    sid = rng.integers(0, 3, M)
    x = rng.uniform(size=(N, N))
    Gm = O.build_G(geo, uvw, 1.0, screens=screens, screen_id=sid)
    y = O.phi(geo, Gm, x)
    yd = O.visibilities_direct_dde(geo, x, uvw, screens, sid)
    err = np.linalg.norm(y - yd) / np.linalg.norm(yd)
    # the same bound as without screens: the KB interpolation error of W = 4
    y0 = O.phi(geo, O.build_G(geo, uvw, 1.0), x)
    err0 = np.linalg.norm(y0 - O.visibilities_direct(geo, x, uvw)) / np.linalg.norm(y0)
    assert err <= 3e-3 and err <= 3 * err0 + 1e-4, (err, err0)
    # a wrong screen (transposed) is far off
    Gt = O.build_G(geo, uvw, 1.0, screens=np.transpose(screens, (0, 2, 1)).copy(), screen_id=sid)
    assert np.linalg.norm(O.phi(geo, Gt, x) - yd) / np.linalg.norm(yd) > 10 * err


def test_dde_adjoint_identity():
    geo = O.Geometry(16, L)
    rng = np.random.default_rng(5)
    uvw = synth.random_uvw(rng, 40, 16, L)
    screens = synth.dde_screens(2, 16, L, seed=1)
    Gm = O.build_G(geo, uvw, 0.9, screens=screens, screen_id=rng.integers(0, 2, 40))
    x = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    y = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    Xt = O.F(geo, O.AZ(geo, x))
    lhs = np.vdot(y, Gm @ Xt.ravel())
    rhs = np.vdot(O.phi_adj(geo, Gm, y), x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_screen_needs_the_full_box():
    geo = O.Geometry(16, L)
    with pytest.raises(ValueError):
        O.kernel_box(geo, 1.0, 2.0, 3.0, 16, np.ones((16, 16)))
