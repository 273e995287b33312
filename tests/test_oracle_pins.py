"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, brute force on tiny inputs, special cases that reduce to a
textbook routine, and invariants.  Each test names the passage it checks."""
import itertools
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

L = synth.fov_L()


def test_fov_and_beta_values():
    # Section 4.1: theta = 2 deg, L = 2 sin(theta/2); Beatty et al. 2005 beta for W=4, sigma=2
    assert abs(L - 2 * math.sin(math.pi / 180.0)) < 1e-15
    assert abs(L - 0.0349048128745) < 1e-12
    assert abs(O.kb_beta(4, 2.0) - 8.9962) < 5e-5   # pi sqrt(8.2), Beatty et al. 2005


@pytest.mark.parametrize("S", [8, 16])
def test_centred_dft_is_the_direct_sum(S):
    # The library FFT route equals the DFT written as an explicit sum.
    rng = np.random.default_rng(S)
    a = rng.standard_normal((S, S)) + 1j * rng.standard_normal((S, S))
    ref = O.direct_centred_dft2(a)
    assert np.max(np.abs(O.centred_dft2(a) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("W", [4, 6, 8])
def test_kb_fourier_transform_matches_quadrature(W):
    # a(l): closed form of the KB transform vs numerical quadrature of its definition
    beta = O.kb_beta(W, 2.0)
    nus = np.array([0.0, 0.05, 0.1, 0.2, 0.25, 0.4, 0.7, 1.3])   # includes sin branch
    got = O.kb_ft(nus, W, beta)
    for nu, g in zip(nus, got):
        val, _ = scipy.integrate.quad(lambda t: float(O.kb(t, W, beta)) * math.cos(2 * math.pi * nu * t),
                                      -W / 2, W / 2, epsabs=0, epsrel=1e-13, limit=400)
        assert abs(g - val) <= 1e-12 * max(abs(val), 1e-3 * W * math.sinh(beta) / beta)


@pytest.mark.parametrize("S,ext,kind", [(16, "full", "exact"), (32, "clamp", "exact"),
                                        (64, "full", "linear"), (32, "full", "exact")])
def test_energy_closed_form_parseval(S, ext, kind):
    # Section 3.2 energy = sum |K|^2; with |c| = 1 Parseval gives the product of
    # the per-axis tap energies, for every w and every box size.
    geo = O.Geometry(16, L, extension=ext, chirp_kind=kind)
    rng = np.random.default_rng(S)
    for _ in range(4):
        u, v = rng.uniform(-200, 200, 2)
        w = rng.uniform(0, 20000)
        K, _, _ = O.kernel_box(geo, u, v, w, S)
        E = O.energy_closed_form(geo, u, v)
        assert abs(np.sum(np.abs(K) ** 2) - E) <= 1e-12 * E


def test_w0_kernel_is_the_kb_taps():
    # w = 0: C = 1, C-hat is a delta, the row holds only the KB taps
    geo = O.Geometry(16, L)
    for S in (16, 32):
        u, v = 123.4, -55.5
        K, j0u, j0v = O.kernel_box(geo, u, v, 0.0, S)
        tu = O.tap_weights(u / geo.du - j0u, 4, geo.beta)
        tv = O.tap_weights(v / geo.du - j0v, 4, geo.beta)
        ref = np.zeros((S, S))
        for a_, ta in enumerate(O.taps(4)):
            for b_, tb in enumerate(O.taps(4)):
                ref[ta % S, tb % S] = tu[a_] * tv[b_]
        assert np.max(np.abs(K - ref)) <= 1e-14 * np.max(ref)


def test_w0_phi_is_plain_type2_nufft():
    # Eq. 2 (small-field limit): at w = 0 Phi reduces to the KB type-2 NUFFT
    N = 16
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(3)
    uvw = synth.random_uvw(rng, 60, N, L, 0.0)
    x = rng.standard_normal((N, N))
    y_ref = O.nufft_type2_direct(geo, x, uvw[:, :2])
    for S in (geo.G, 32):
        Gm = O.build_G(geo, uvw, 1.0, S=S)
        y = O.phi(geo, Gm, x)
        assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("kind", ["exact", "linear"])
def test_eq6_constant_w_on_grid_is_fft_of_modulated_image(kind):
    # Eq. 6 / Eq. 8: with constant w, on-grid visibilities and delta-gridding,
    # w-projection equals the FFT of the chirp-modulated zero-padded image.
    N = 16
    geo = O.Geometry(N, L, W=1, chirp_kind=kind)
    G = geo.G
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, N))
    w = 0.7 * N / L ** 2
    q = rng.integers(-N, N, (40, 2))
    uvw = np.stack([q[:, 0] * geo.du, q[:, 1] * geo.du, np.full(40, w)], axis=1)
    Gm = O.build_G(geo, uvw, 1.0)
    y = O.phi(geo, Gm, x)
    off = np.arange(G) - G // 2            # offset held at padded index off mod G
    lg = off * geo.dl
    c = np.zeros((G, G), complex)
    c[np.ix_(off % G, off % G)] = O.chirp(lg[:, None], lg[None, :], w, kind)
    xp = np.zeros((G, G), complex)
    idx = (np.arange(N) - N // 2) % G
    xp[np.ix_(idx, idx)] = x
    Y = np.fft.fft2(xp * c) / G
    y_ref = Y[q[:, 0] % G, q[:, 1] % G]
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)


@pytest.mark.parametrize("N", [8, 16, 32])
def test_phi_matches_brute_force_measurement_equation(N):
    # Eq. 1 / Eq. 3 with the chirp of Eq. 4, evaluated directly: Phi at e = 1 and
    # S = G reproduces it to KB accuracy, and the error falls with W.
    M = 100
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N))
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    errs = []
    for W in (4, 6, 8):
        geo = O.Geometry(N, L, W=W)
        y_dir = O.visibilities_direct(geo, x, uvw)
        y = O.phi(geo, O.build_G(geo, uvw, 1.0), x)
        errs.append(np.linalg.norm(y - y_dir) / np.linalg.norm(y_dir))
    assert errs[0] < 2e-3
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("e", [0.9, 1.0])
def test_adjoint_identity(e):
    N = 16
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(7)
    uvw = synth.random_uvw(rng, 80, N, L, 1.0)
    Gm = O.build_G(geo, uvw, e)
    x = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    y = rng.standard_normal(80) + 1j * rng.standard_normal(80)
    lhs = np.vdot(y, O.phi(geo, Gm, x))
    rhs = np.vdot(O.phi_adj(geo, Gm, y), x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(O.phi(geo, Gm, x)) * np.linalg.norm(y)


def test_discarded_energy_and_retained_fraction():
    # Section 3.2: entries below the threshold are set to zero; the kept energy
    # reaches e*E and dropping the last kept entry would not.
    geo = O.Geometry(32, L)
    rng = np.random.default_rng(11)
    for _ in range(5):
        u, v = rng.uniform(-300, 300, 2)
        w = rng.uniform(0, 1) * 32 / L ** 2
        K, j0u, j0v = O.kernel_box(geo, u, v, w, geo.G)
        cols = O.box_columns(geo, j0u, j0v, geo.G)
        E = math.fsum(np.abs(K.ravel()) ** 2)
        for e in (0.5, 0.9, 0.99):
            kept = O.select_sort(K, cols, e)
            Ke = np.zeros(K.size, complex)
            Ke[kept] = K.ravel()[kept]
            retained = math.fsum(np.abs(Ke) ** 2)
            assert abs(np.sum(np.abs(K.ravel() - Ke) ** 2) - (E - retained)) <= 1e-12 * E
            assert retained >= e * E
            p = np.abs(K.ravel()[kept]) ** 2
            assert math.fsum(p[:-1]) < e * E


def test_sparsification_converges_as_e_to_1():
    # Section 3.2 / Fig. 3: nnz is non-decreasing in e, the discarded energy
    # ||G_e - G_1||_F^2 is non-increasing and vanishes at e = 1.
    N = 16
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(13)
    uvw = synth.random_uvw(rng, 30, N, L, 1.0)
    x = rng.standard_normal((N, N))
    G1 = O.build_G(geo, uvw, 1.0)
    y1 = O.phi(geo, G1, x)
    prev_nnz, prev_d = -1, np.inf
    for e in (0.3, 0.6, 0.9, 0.99, 0.999, 1.0):
        Ge = O.build_G(geo, uvw, e)
        d = scipy_fro2(Ge - G1)
        assert Ge.nnz >= prev_nnz
        assert d <= prev_d
        prev_nnz, prev_d = Ge.nnz, d
    assert prev_d == 0.0
    assert np.linalg.norm(O.phi(geo, Ge, x) - y1) == 0.0


def scipy_fro2(A):
    return float(np.sum(np.abs(A.data) ** 2)) if A.nnz else 0.0


def test_support_grows_with_w_trend():
    # Fig. 1: the support of the kernel rows grows with w_d (as a trend)
    N = 32
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(17)
    offs = rng.uniform(-100, 100, (6, 2))
    means = []
    for wd in (0.1, 0.25, 0.5, 0.75, 1.0):
        w = wd * N / L ** 2
        n = [O.kernel_row(geo, u, v, w, geo.G, 0.99)[0].size for u, v in offs]
        means.append(np.mean(n))
    assert all(b > a for a, b in zip(means, means[1:]))


def test_select_is_minimal_against_all_subsets():
    # Brute force over every subset of a 3x3 kernel: the sort-based selection
    # has the minimal cardinality, maximal energy at that cardinality, and the
    # paper's bisection route gives the same set (no ties here).
    rng = np.random.default_rng(19)
    for trial in range(40):
        vals = rng.standard_normal(9) + 1j * rng.standard_normal(9)
        cols = np.arange(9)
        p = np.abs(vals) ** 2
        E = math.fsum(p)
        for e in (0.2, 0.5, 0.8, 0.95, 0.999):
            best_n, best_E = None, -1.0
            for n in range(1, 10):
                for sub in itertools.combinations(range(9), n):
                    s = math.fsum(p[list(sub)])
                    if s >= e * E and s > best_E:
                        best_E = s
                if best_E >= 0:
                    best_n = n
                    break
            kept = O.select_sort(vals, cols, e)
            assert kept.size == best_n
            assert abs(math.fsum(p[kept]) - best_E) <= 1e-15 * E
            mask = O.select_bisect(vals, e)
            assert set(np.nonzero(mask)[0]) == set(kept.tolist())


def test_select_tie_break_lower_column_first():
    vals = np.array([1.0, 1.0, 1.0, 1.0])
    cols = np.array([7, 3, 9, 1])
    kept = O.select_sort(vals, cols, 0.5)
    assert sorted(cols[kept].tolist()) == [1, 3]


def test_mirror_symmetry_at_half_cell_offset():
    # delta = (1/2, 1/2): the taps are symmetric about 1/2 and the sampled chirp is
    # even, so K[s] = K[1 - s]; the conjugate chirp sign (Eq. 5 vs Eq. 4 reading)
    # gives the same moduli and therefore the same support.
    geo = O.Geometry(16, L)
    S = 32
    u = (10 + 0.5) * geo.du
    v = (-7 + 0.5) * geo.du
    w = 0.8 * 16 / L ** 2
    K, _, _ = O.kernel_box(geo, u, v, w, S)
    s = np.arange(S)
    mirror = (1 - np.fft.fftfreq(S, 1.0 / S).astype(int)) % S
    Km = K[np.ix_(mirror, mirror)]
    assert np.max(np.abs(K - Km)) <= 1e-12 * np.max(np.abs(K))
    Kc, _, _ = O.kernel_box(geo, u, v, -w, S)     # conj chirp == chirp with -w
    assert np.max(np.abs(np.abs(Kc) - np.abs(K))) <= 1e-12 * np.max(np.abs(K))
    cols = O.box_columns(geo, 10, -7, S)
    a = O.select_sort(K, cols, 0.9)
    b = O.select_sort(Kc, cols, 0.9)
    assert len(a) == len(b)
    del s


def test_full_and_clamp_extension_agree_at_e1():
    # The image is zero outside the field of view, so any extension of the chirp
    # there gives the same Phi before thresholding (convolution theorem).
    N = 16
    rng = np.random.default_rng(23)
    uvw = synth.random_uvw(rng, 40, N, L, 1.0)
    x = rng.standard_normal((N, N))
    ys = []
    for ext in ("full", "clamp"):
        geo = O.Geometry(N, L, extension=ext)
        ys.append(O.phi(geo, O.build_G(geo, uvw, 1.0), x))
    assert np.linalg.norm(ys[0] - ys[1]) <= 1e-12 * np.linalg.norm(ys[0])


def test_bpdn_dr_reaches_closed_form_for_an_isometry():
    # Eq. 7 with Psi = Dirac: with full on-grid coverage, w = 0 and
    # delta-gridding Phi = F Z is an isometry and BPDN is a soft threshold of
    # Re Phi^H y; Douglas-Rachford must converge to it.
    N = 8
    geo = O.Geometry(N, L, W=1)
    G = geo.G
    qu, qv = np.meshgrid(np.arange(G) - G // 2, np.arange(G) - G // 2, indexing="ij")
    uvw = np.stack([qu.ravel() * geo.du, qv.ravel() * geo.du, np.zeros(G * G)], 1)
    Gm = O.build_G(geo, uvw, 1.0)

    def ap(v):
        return O.phi(geo, Gm, v)

    def aa(v):
        return O.phi_adj(geo, Gm, v)

    rng = np.random.default_rng(0)
    x = np.maximum(rng.standard_normal((N, N)), 0)
    y = ap(x) + 0.05 * (rng.standard_normal(G * G) + 1j * rng.standard_normal(G * G))
    b = np.real(aa(y))
    c0 = np.sum(np.abs(y) ** 2) - np.sum(b ** 2)
    eps = math.sqrt(c0 + 0.3 * np.sum(b ** 2))
    xs = O.bpdn_closed_form_isometry(b, eps, c0)
    assert abs(O.power_norm2(ap, aa, N, 20) - 1.0) < 1e-12
    xr, _ = O.solve_bpdn(ap, aa, y, eps, N, 200, inner_iters=10, phi_norm2=1.0)
    assert np.linalg.norm(xr - xs) <= 1e-6 * np.linalg.norm(xs)
    assert np.linalg.norm(y - ap(xr)) <= eps * (1 + 1e-6)


def test_snr_definition():
    # Section 4.1: SNR_out = 20 log10(std(x)/std(x - x_rec)); a constant offset is not penalised
    x = np.arange(16.0).reshape(4, 4)
    assert O.snr_db(x, x + 0.5 + 0.1 * np.cos(x)) == pytest.approx(
        20 * math.log10(np.std(x) / np.std(0.1 * np.cos(x))))


def test_box_rule():
    geo = O.Geometry(1024, L)
    assert O.box_size_rule(geo, 0.0) == 32
    assert O.box_size_rule(geo, 3.0) == 32
    assert O.box_size_rule(geo, 8.0) == 64
    assert O.box_size_rule(geo, 1e6) == geo.G


def test_noise_level_definition():
    # Section 4.1: sigma(n) = 10^(-SNR_in/20) sigma(x), SNR_in = 30 dB
    prob = synth.make_problem(synth.SMALL, seed=0)
    n, s = synth.draw_noise(prob)
    assert s == pytest.approx(10 ** (-1.5) * np.std(prob.x))
    assert np.std(n) == pytest.approx(s, rel=0.1)


def test_point_source_phase_depends_only_on_delay():
    # Eq. 1: a point source at direction s = (l0, m0, n0) gives a plane wave whose
    # phase is set by the geometric delay b.(s - s0), s0 = (0, 0, 1) the phase
    # centre.  So its visibility does not change when the baseline b = (u, v, w)
    # moves orthogonally to s - s0.  This fixes the sign and scale of the chirp
    # (Eq. 4) relative to the Fourier kernel; a wrong sign breaks it.
    N = 16
    geo = O.Geometry(N, L)
    p0, q0 = 13, 2
    x = np.zeros((N, N))
    x[p0, q0] = 1.0
    l0 = (p0 - N // 2) * geo.dl
    m0 = (q0 - N // 2) * geo.dl
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    b1 = np.array([300.0, -200.0, 40000.0])
    for d in (np.array([n0 - 1.0, 0.0, -l0]), np.array([0.0, n0 - 1.0, -m0])):
        d = d / np.linalg.norm(d)
        b2 = b1 + 5e4 * d
        y = O.visibilities_direct(geo, x, np.stack([b1, b2]))
        assert abs(y[0] - y[1]) <= 1e-9 * abs(y[0])
    # a move along s - s0 itself does change it
    d = np.array([l0, m0, n0 - 1.0])
    y = O.visibilities_direct(geo, x, np.stack([b1, b1 + 0.5 / np.dot(d, d) * d]))
    assert abs(y[0] + y[1]) <= 1e-9 * abs(y[0])       # half a turn of phase


def test_linear_chirp_is_first_order_of_exact():
    # Eq. 5 is the first-order approximation of Eq. 4: their phase difference is
    # O(w r^4) (the next term of 1 - n = r^2/2 + r^4/8 + ...).
    w = 2.0e5
    for r in (1e-3, 2e-3, 4e-3):
        ce = O.chirp(r, 0.0, w, "exact")
        cl = O.chirp(r, 0.0, w, "linear")
        dphi = np.angle(ce / cl)
        assert abs(dphi - 2 * math.pi * w * r ** 4 / 8) <= 2 * math.pi * w * r ** 6


def test_power_iteration_matches_dense_svd():
    N = 8
    geo = O.Geometry(N, L)
    rng = np.random.default_rng(29)
    uvw = synth.random_uvw(rng, 40, N, L, 1.0)
    Gm = O.build_G(geo, uvw, 0.95)
    cols = []
    for i in range(N * N):
        e_i = np.zeros(N * N)
        e_i[i] = 1.0
        yv = O.phi(geo, Gm, e_i.reshape(N, N))
        cols.append(np.concatenate([yv.real, yv.imag]))
    A = np.array(cols).T                       # real 2M x N^2 matrix of the operator
    s_max = np.linalg.svd(A, compute_uv=False)[0]
    n2 = O.power_norm2(lambda v: O.phi(geo, Gm, v), lambda v: O.phi_adj(geo, Gm, v), N, 300)
    assert abs(n2 - s_max ** 2) <= 1e-8 * s_max ** 2
