"""The Daubechies sparsity basis on the GPU (Psi of Eq. 7; Db8 in Section 4):
filter taps, the 2-D analysis and synthesis, and Douglas-Rachford with Psi,
against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import wavelet_oracle as W
from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("p", list(range(1, 11)))
def test_taps_match_oracle(wp, p):
    h = np.array(wp.daubechies_taps(p))
    assert np.allclose(h, W.daubechies_taps(p), rtol=0, atol=1e-12)


def test_taps_reject_bad_order(wp):
    for p in (0, 11):
        with pytest.raises(wp.WprojError):
            wp.daubechies_taps(p)


# sides and depths: several tiles, a ragged tile, bands smaller than a tile, an odd last band
@pytest.mark.parametrize("N,levels,p", [(64, 4, 8), (256, 4, 8), (48, 4, 8), (96, 5, 2), (32, 5, 8),
                                        (128, 1, 1), (512, 6, 8)])
def test_analysis_and_synthesis_match_oracle(wp, N, levels, p):
    rng = np.random.default_rng(N + levels + p)
    x = rng.standard_normal((N, N))
    a_o = W.dwt2(x, levels, p) if N <= 128 else None
    xg = torch.from_numpy(x.astype(np.float32)).to(dev())
    a_g = wp.dwt2(xg, levels, p)
    if a_o is not None:
        assert rel(a_g.cpu().numpy(), a_o) <= 2e-6
        x_o = W.idwt2(a_o, levels, p)
        x_g = wp.idwt2(torch.from_numpy(a_o.astype(np.float32)).to(dev()), levels, p)
        assert rel(x_g.cpu().numpy(), x_o) <= 2e-6
    # orthonormal at every size: Parseval and perfect reconstruction
    assert abs(float(a_g.double().norm()) - float(np.linalg.norm(x))) <= 2e-6 * np.linalg.norm(x)
    back = wp.idwt2(a_g, levels, p).cpu().numpy()
    assert rel(back, x) <= 2e-6


def test_large_side_sampled_against_oracle_rows(wp):
    # N = 1024, one level: the oracle's 1-D transform of sampled rows and columns
    N = 1024
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, N)).astype(np.float32)
    a = wp.dwt2(torch.from_numpy(x).to(dev()), 1, 8).cpu().numpy().astype(np.float64)
    h = W.daubechies_taps(8)
    # one level = fast axis then slow axis; check a few full columns of the result
    tmp_lo = np.empty((N, N // 2))
    tmp_hi = np.empty((N, N // 2))
    for r in range(N):
        tmp_lo[r], tmp_hi[r] = W.dwt1(x[r].astype(np.float64), h)
    for c in (0, 1, 77, 511):
        lo, hi = W.dwt1(tmp_lo[:, c], h)
        assert np.allclose(a[:N // 2, c], lo, atol=2e-5) and np.allclose(a[N // 2:, c], hi, atol=2e-5)
        lo, hi = W.dwt1(tmp_hi[:, c], h)
        assert np.allclose(a[:N // 2, N // 2 + c], lo, atol=2e-5) and np.allclose(a[N // 2:, N // 2 + c], hi,
                                                                                  atol=2e-5)


def test_bad_geometry_is_rejected(wp):
    x = torch.zeros((48, 48), dtype=torch.float32, device=dev())
    with pytest.raises(wp.WprojError):
        wp.dwt2(x, 5, 8)           # 48 is not divisible by 32
    with pytest.raises(wp.WprojError):
        wp.dwt2(x, 0, 8)


def test_dr_with_db8_matches_oracle(wp):
    # Eq. 7 with Psi = Db8 on the 64 x 64 blob sky (e = 0.99, Kaiser-Bessel gridding)
    wl = synth.SMALL
    prob = synth.make_problem(wl, seed=0)
    noise, sigma_n = synth.draw_noise(prob)
    geo = O.Geometry(wl.N, prob.L)
    Gm = O.build_G(geo, prob.uvw, wl.e)
    y = O.phi(geo, Gm, prob.x) + noise
    eps = O.epsilon_chi2(sigma_n, wl.M)
    levels, iters = 4, 30

    def ap(a):
        return O.phi(geo, Gm, W.idwt2(a, levels, 8))

    def aa(r):
        return W.dwt2(np.real(O.phi_adj(geo, Gm, r)), levels, 8)

    # Psi is orthonormal, so ||Phi Psi|| = ||Phi||: both sides take the power
    # iteration of Phi alone (from the centre impulse)
    n2 = O.power_norm2(lambda v: O.phi(geo, Gm, v), lambda r: np.real(O.phi_adj(geo, Gm, r)), wl.N, 100)
    a_or, info_or = O.solve_bpdn(ap, aa, y, eps, wl.N, iters, inner_iters=wl.inner_iters, phi_norm2=n2)
    x_or = W.idwt2(a_or, levels, 8)
    plan = wp.Plan(wl.N, prob.L)
    plan.build_kernels(torch.from_numpy(prob.uvw).to(dev()), wl.e)
    yg = torch.from_numpy(y.astype(np.complex64)).to(dev())
    x_gpu, info = plan.solve_bpdn(yg, eps, iters=iters, inner_iters=wl.inner_iters, psi=8, psi_levels=levels)
    x_gpu = x_gpu.cpu().numpy().astype(np.float64)
    s_or, s_gpu = O.snr_db(prob.x, x_or), O.snr_db(prob.x, x_gpu)
    print(f"Db8: SNR oracle {s_or:.3f} dB, GPU {s_gpu:.3f} dB")
    assert abs(info.phi_norm2 - info_or["phi_norm2"]) <= 1e-3 * info_or["phi_norm2"]
    assert abs(info.gamma - info_or["gamma"]) <= 5e-3 * info_or["gamma"]
    assert abs(s_gpu - s_or) <= 0.1
    assert np.linalg.norm(x_gpu - x_or) <= 1e-2 * np.linalg.norm(x_or)
    # final_l1 is ||alpha||_1 = ||Psi^T x||_1 of the returned image
    l1 = np.sum(np.abs(W.dwt2(x_gpu, levels, 8)))
    assert abs(info.final_l1 - l1) <= 1e-4 * l1
    # zero iterations return Psi z0 = Re Phi^H y (Psi orthonormal); the GPU keeps
    # e + 1e-5 of each row's energy, so its Phi^H differs from the oracle's
    # e-operator by up to ~sqrt(1e-5) relative
    x0, _ = plan.solve_bpdn(yg, eps, iters=0, psi=8, psi_levels=levels)
    x0d, _ = plan.solve_bpdn(yg, eps, iters=0)
    ref = np.real(O.phi_adj(geo, Gm, y))
    assert rel(x0.cpu().numpy(), ref) <= 5e-3
    assert rel(x0.cpu().numpy(), x0d.cpu().numpy()) <= 2e-6
    with pytest.raises(wp.WprojError):
        plan.solve_bpdn(yg, eps, iters=1, psi=11)
    with pytest.raises(wp.WprojError):
        plan.solve_bpdn(yg, eps, iters=1, psi=8, psi_levels=7)     # 64 is not divisible by 128
    plan.close()
