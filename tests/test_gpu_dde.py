"""Direction-dependent screens on the GPU (Section 3.2: the per-row threshold
applies to any image-space modulation): rows built from chirp x screen against
the FP64 oracle, the Fourier-shift property of a phase-ramp screen, and the
argument checks."""
import math

import numpy as np
import pytest
import torch

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

pytestmark = pytest.mark.gpu

L = synth.fov_L()


@pytest.fixture(scope="module")
def wp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import wproj
    return wproj


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(N, M, n_scr, seed):
    rng = np.random.default_rng(seed)
    uvw = synth.random_uvw(rng, M, N, L)
    screens = synth.dde_screens(n_scr, N, L, seed=seed)
    sid = rng.integers(0, n_scr, M).astype(np.int32)
    return uvw, screens, sid


def gpu_plan(wp, N, uvw, screens, sid, e, fmt="columns", vdt="f32"):
    plan = wp.Plan(N, L, index_format=fmt, value_dtype=vdt)
    plan.set_screens(torch.from_numpy(screens).to(dev()))
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), e, screen_id=torch.from_numpy(sid).to(dev()))
    return plan


@pytest.mark.parametrize("N,fmt", [(16, "columns"), (32, "columns"), (32, "mask"), (16, "runs"), (32, "runs")])
def test_operators_with_screens_match_oracle_at_e1(wp, N, fmt):
    uvw, screens, sid = problem(N, 150, 4, N)
    geo = O.Geometry(N, L)
    Gm = O.build_G(geo, uvw, 1.0, screens=screens.astype(np.complex128), screen_id=sid)
    plan = gpu_plan(wp, N, uvw, screens, sid, 1.0, fmt)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((N, N))
    y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
    assert rel(y, O.phi(geo, Gm, x)) <= 1e-5
    yv = rng.standard_normal(uvw.shape[0]) + 1j * rng.standard_normal(uvw.shape[0])
    xa = plan.phi_adj(torch.from_numpy(yv.astype(np.complex64)).to(dev()), complex_out=True).cpu().numpy()
    assert rel(xa, O.phi_adj(geo, Gm, yv)) <= 1e-5
    plan.close()


@pytest.mark.parametrize("e", [0.9, 0.99])
def test_rows_with_screens_follow_the_energy_rule(wp, e):
    # Section 3.2 with screens: kept oracle energy >= e E_k, no more entries than
    # the oracle needs for e + 2e-5, and the values on the kept support
    N = 32
    uvw, screens, sid = problem(N, 120, 3, 7)
    geo = O.Geometry(N, L)
    plan = gpu_plan(wp, N, uvw, screens, sid, e)
    c = plan.csr()
    num = den = 0.0
    for k in range(0, uvw.shape[0], 3):
        col, val = c.rows(k, k + 1)
        col, val = col.cpu().numpy(), val.cpu().numpy().astype(np.complex128)
        scr = screens[sid[k]].astype(np.complex128)
        K, j0u, j0v = O.kernel_box(geo, *uvw[k], geo.G, scr)
        cols = O.box_columns(geo, j0u, j0v, geo.G).ravel()
        lut = np.full(geo.G * geo.G, -1)
        lut[cols] = np.arange(cols.size)
        vo = K.ravel()[lut[col]]
        E = math.fsum(np.abs(K.ravel()) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= e * E
        assert col.size <= O.select_sort(K, cols, e + 2e-5).size
        num += np.sum(np.abs(val - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
    assert math.sqrt(num / den) <= 1e-5
    plan.close()


def test_phase_ramp_screen_is_a_shift_on_the_gpu(wp):
    # a ramp of (su, sv) cycles per padded box moves every visibility by (su, sv)
    # cells (Fourier shift): the rows agree as functions of the column
    N, su, sv = 32, 3, -2
    G = 2 * N
    rng = np.random.default_rng(4)
    uvw = synth.random_uvw(rng, 64, N, L)
    uvw[:, :2] *= 0.8
    off = np.arange(G) - G // 2
    ramp = np.exp(-2j * np.pi * (su * off[:, None] + sv * off[None, :]) / G)[None].astype(np.complex64)
    sid = np.zeros(64, np.int32)
    pa = gpu_plan(wp, N, uvw, ramp, sid, 1.0)
    shifted = uvw.copy()
    shifted[:, 0] += su / (2 * L)
    shifted[:, 1] += sv / (2 * L)
    pb = wp.Plan(N, L, index_format="columns")
    pb.build_kernels(torch.from_numpy(shifted).to(dev()), 1.0)
    ca, cb = pa.csr(), pb.csr()
    for k in range(0, 64, 5):
        c1, v1 = (t.cpu().numpy() for t in ca.rows(k, k + 1))
        c2, v2 = (t.cpu().numpy() for t in cb.rows(k, k + 1))
        r1 = np.zeros(G * G, complex)
        r2 = np.zeros(G * G, complex)
        r1[c1] = v1
        r2[c2] = v2
        assert rel(r1, r2) <= 2e-5
    pa.close()
    pb.close()


def test_screen_arguments_are_checked(wp):
    N = 16
    uvw, screens, sid = problem(N, 20, 2, 3)
    plan = wp.Plan(N, L)
    ug = torch.from_numpy(uvw).to(dev())
    with pytest.raises(wp.WprojError):       # no screens set
        plan.build_kernels(ug, 0.9, screen_id=torch.from_numpy(sid).to(dev()))
    plan.set_screens(torch.from_numpy(screens).to(dev()))
    bad = sid.copy()
    bad[5] = 2
    with pytest.raises(wp.WprojError):       # id out of range
        plan.build_kernels(ug, 0.9, screen_id=torch.from_numpy(bad).to(dev()))
    nan = screens.copy()
    nan[1, 3, 4] = np.nan
    with pytest.raises(wp.WprojError):
        plan.set_screens(torch.from_numpy(nan).to(dev()))
    plan.close()
    rule = wp.Plan(N, L, box="rule")
    rule.set_screens(torch.from_numpy(screens).to(dev()))
    with pytest.raises(wp.WprojError):       # a screen needs the full box
        rule.build_kernels(ug, 0.9, screen_id=torch.from_numpy(sid).to(dev()))
    rule.close()


def test_reconstruction_with_screens(wp):
    # BPDN with the screened operator: the SNR of the oracle's solver, data
    # simulated with each side's own operator
    N = 32
    geo = O.Geometry(N, L)
    x = synth.blob_sky(np.random.default_rng(2), N, 10)
    rng = np.random.default_rng(11)
    screens = synth.dde_screens(4, N, L, seed=5)
    uvw = synth.random_uvw(rng, 600, N, L)
    sid = rng.integers(0, 4, 600).astype(np.int32)
    sigma_n = synth.noise_sigma(x, 30.0)
    noise = synth.complex_noise(np.random.default_rng(12), 600, sigma_n)
    eps = sigma_n * math.sqrt(600 + 2 * math.sqrt(600))
    Gm = O.build_G(geo, uvw, 0.99, screens=screens.astype(np.complex128), screen_id=sid)
    y = O.phi(geo, Gm, x) + noise
    xo, _ = O.solve_bpdn(lambda v: O.phi(geo, Gm, v), lambda r: O.phi_adj(geo, Gm, r), y, eps, N, 30)
    plan = gpu_plan(wp, N, uvw, screens, sid, 0.99)
    yg = torch.from_numpy(y.astype(np.complex64)).to(dev())
    xg, _ = plan.solve_bpdn(yg, eps, iters=30)
    s_o, s_g = O.snr_db(x, xo), O.snr_db(x, xg.cpu().numpy().astype(np.float64))
    print(f"screens: SNR oracle {s_o:.3f} dB, GPU {s_g:.3f} dB")
    assert abs(s_o - s_g) <= 0.1
    plan.close()


@pytest.mark.parametrize("fmt", ["columns", "mask"])
def test_screened_rows_at_size_sampled(wp, fmt):
    # N = 128 (64 grid tiles), M = 4096, 8 screens: sampled rows against the oracle
    # (values, kept energy, cardinality) and the adjoint identity of the whole operator
    N, M, e = 128, 4096, 0.99
    uvw, screens, sid = problem(N, M, 8, 31)
    geo = O.Geometry(N, L)
    plan = gpu_plan(wp, N, uvw, screens, sid, e, fmt)
    c = plan.csr()
    G = geo.G
    num = den = 0.0
    for k in np.random.default_rng(5).choice(M, 12, replace=False):
        col, val = (t.cpu().numpy() for t in c.rows(int(k), int(k) + 1))
        val = val.astype(np.complex128)
        K, j0u, j0v = O.kernel_box(geo, *uvw[k], G, screens[sid[k]].astype(np.complex128))
        su = ((col // G - j0u + G // 2) % G) - G // 2
        sv = ((col % G - j0v + G // 2) % G) - G // 2
        vo = K[su % G, sv % G]
        num += np.sum(np.abs(val - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= e * math.fsum(np.abs(K.ravel()) ** 2)
        assert col.size <= O.select_sort(K, O.box_columns(geo, j0u, j0v, G), e + 2e-5).size
    assert math.sqrt(num / den) <= 1e-5
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).to(dev())
    yv = torch.from_numpy((rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)).to(dev())
    lhs = torch.vdot(yv.to(torch.complex128), plan.phi(x).to(torch.complex128)).real.item()
    rhs = float((x.double() * plan.phi_adj(yv).double()).sum().item())
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    plan.close()
