"""Batched form: many problems of uneven size run through shared launches.

Every batch result is compared with the same problems run one by one through
single plans (whose G and operators are checked against the FP64 oracle in the
other test files), and the smallest problems also directly with the oracle.
Schedules (row-piece and chunk sizes) change only the summation order.
"""
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


def make_case(ns, ms, seed=0, wc_max=2.0):
    rng = np.random.default_rng(seed)
    uvws, xs = [], []
    for n, m in zip(ns, ms):
        B = synth.band_limit(n, L)
        uv = synth.uv_points(rng, m, B, n, "uniform")
        w = 2.0 * rng.uniform(0.0, wc_max, m) / (L * L)
        uvws.append(np.concatenate([uv, w[:, None]], axis=1))
        xs.append(rng.standard_normal((n, n)))
    return uvws, xs


def build_batch(wp, ns, uvws, e, box="rule"):
    b = wp.Batch(ns, L, box=box)
    b.build_kernels(torch.from_numpy(np.concatenate(uvws)).to(dev()), [u.shape[0] for u in uvws], e)
    return b


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


NS = [16, 64, 32, 64, 16, 128, 32]
MS = [40, 700, 300, 1, 90, 2000, 150]


def test_batch_operators_match_single_plans(wp):
    uvws, xs = make_case(NS, MS, seed=1)
    b = build_batch(wp, NS, uvws, 0.99)
    x_cat = torch.from_numpy(np.concatenate([x.ravel() for x in xs]).astype(np.float32)).to(dev())
    y_cat = b.phi(x_cat)
    rng = np.random.default_rng(2)
    yv = [(rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64) for m in MS]
    xa_cat = b.phi_adj(torch.from_numpy(np.concatenate(yv)).to(dev()))
    ys, xas = b.split_vis(y_cat), b.split_images(xa_cat)
    for i, (n, uvw, x) in enumerate(zip(NS, uvws, xs)):
        p = wp.Plan(n, L, box="rule", index_format="columns")
        p.build_kernels(torch.from_numpy(uvw).to(dev()), 0.99)
        y1 = p.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
        xa1 = p.phi_adj(torch.from_numpy(yv[i]).to(dev())).cpu().numpy()
        assert rel(ys[i].cpu().numpy(), y1) <= 1e-6, i
        assert rel(xas[i].cpu().numpy(), xa1) <= 1e-6, i
        p.close()
    info = b.info()
    assert info["n_problems"] == len(NS) and info["m"] == sum(MS) and info["pixels"] == sum(n * n for n in NS)
    b.close()


def test_batch_matches_oracle_at_e1(wp):
    # at e = 1 every problem's operator equals the oracle's (no selection freedom)
    ns, ms = [16, 32, 16], [30, 80, 5]
    uvws, xs = make_case(ns, ms, seed=3, wc_max=1.0)
    b = build_batch(wp, ns, uvws, 1.0, box="G")
    x_cat = torch.from_numpy(np.concatenate([x.ravel() for x in xs]).astype(np.float32)).to(dev())
    ys = b.split_vis(b.phi(x_cat))
    rng = np.random.default_rng(4)
    yv = [rng.standard_normal(m) + 1j * rng.standard_normal(m) for m in ms]
    xas = b.split_images(b.phi_adj(torch.from_numpy(np.concatenate(yv).astype(np.complex64)).to(dev())))
    for i, (n, uvw, x) in enumerate(zip(ns, uvws, xs)):
        geo = O.Geometry(n, L)
        Gm = O.build_G(geo, uvw, 1.0)
        assert rel(ys[i].cpu().numpy(), O.phi(geo, Gm, x)) <= 1e-5
        assert rel(xas[i].cpu().numpy(), O.phi_adj(geo, Gm, yv[i]).real) <= 1e-5
    b.close()


def test_batch_adjoint_identity_and_schedules(wp):
    uvws, xs = make_case(NS, MS, seed=5)
    b = build_batch(wp, NS, uvws, 0.99)
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.standard_normal(b.pixels).astype(np.float32)).to(dev())
    y = torch.from_numpy((rng.standard_normal(b.m) + 1j * rng.standard_normal(b.m)).astype(np.complex64)).to(dev())
    ref_y, ref_x = b.phi(x).cpu().numpy(), b.phi_adj(y).cpu().numpy()
    # <Phi x, y> = <x, Re Phi^H y> per problem (x real)
    for a, bb, c, d in zip(b.split_vis(torch.from_numpy(ref_y)), b.split_vis(y.cpu()),
                           b.split_images(x.cpu()), b.split_images(torch.from_numpy(ref_x))):
        lhs = np.real(np.vdot(bb.numpy().astype(np.complex128), a.numpy().astype(np.complex128)))
        rhs = float(np.dot(c.numpy().ravel().astype(np.float64), d.numpy().ravel().astype(np.float64)))
        assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(lhs))
    for piece, chunk, lanes in ((32, 32, 8), (300, 5000, 32), (64, 2048, 4), (16384, 65536, 16),
                                (16384, 65536, 4)):
        b.set_schedule(piece, chunk, lanes)
        assert b.info()["lanes_per_piece"] == lanes
        assert rel(b.phi(x).cpu().numpy(), ref_y) <= 1e-6
        assert rel(b.phi_adj(y).cpu().numpy(), ref_x) <= 1e-6
    with pytest.raises(wp.WprojError):
        b.set_schedule(256, 256, 12)
    sch = b.tune()
    assert sch["piece"] >= 32 and sch["chunk"] >= 32 and sch["degrid_ms"] > 0 and sch["grid_ms"] > 0
    assert sch["lanes_per_piece"] in (4, 8, 16, 32) and b.info()["lanes_per_piece"] == sch["lanes_per_piece"]
    assert rel(b.phi(x).cpu().numpy(), ref_y) <= 1e-6
    b.close()


def test_batch_solver_matches_single_plans_and_resumes(wp):
    ns, ms = [32, 64, 16, 64], [400, 1500, 100, 900]
    uvws, _ = make_case(ns, ms, seed=7)
    rng = np.random.default_rng(8)
    skies = [synth.blob_sky(rng, n, 5) for n in ns]
    b = build_batch(wp, ns, uvws, 0.99)
    x_cat = torch.from_numpy(np.concatenate([x.ravel() for x in skies]).astype(np.float32)).to(dev())
    y_clean = b.phi(x_cat)
    sig = [synth.noise_sigma(x, 30.0) for x in skies]
    noise = np.concatenate([synth.complex_noise(rng, m, s) for m, s in zip(ms, sig)]).astype(np.complex64)
    y = y_clean + torch.from_numpy(noise).to(dev())
    eps = [O.epsilon_chi2(s, m) for s, m in zip(sig, ms)]
    xb = b.solve_bpdn(y, eps, iters=12, power_iters=50)
    info = b.info()
    assert info["iter_launches"] > 0
    # resume: 6 + 6 iterations replay the same graph as 12
    b.solve_bpdn(y, eps, iters=6, power_iters=50)
    x2 = b.solve_bpdn(y, eps, iters=6, resume=True)
    assert torch.equal(x2, xb)
    ys = b.split_vis(y)
    for i, (n, uvw) in enumerate(zip(ns, uvws)):
        p = wp.Plan(n, L, box="rule", index_format="columns")
        p.build_kernels(torch.from_numpy(uvw).to(dev()), 0.99)
        x1, _ = p.solve_bpdn(ys[i].contiguous(), eps[i], iters=12, power_iters=50)
        xbi = b.split_images(xb)[i].cpu().numpy()
        s_b = O.snr_db(skies[i], xbi.astype(np.float64))
        s_1 = O.snr_db(skies[i], x1.cpu().numpy().astype(np.float64))
        assert abs(s_b - s_1) <= 0.1, (i, s_b, s_1)
        assert rel(xbi, x1.cpu().numpy()) <= 1e-3
        p.close()
    b.close()


def test_batch_bad_input(wp):
    with pytest.raises(wp.WprojError):
        wp.Batch([], L)
    b = wp.Batch([16, 32], L)
    with pytest.raises(wp.WprojError):
        b.phi(torch.zeros(16 * 16 + 32 * 32, device=dev()))          # not built
    uvw = torch.zeros((3, 3), dtype=torch.float64, device=dev())
    with pytest.raises(wp.WprojError):
        b.build_kernels(uvw, [3, 0], 0.99)                            # a problem without rows
    with pytest.raises(wp.WprojError):
        b.build_kernels(uvw, [2, 1], 1.5)                             # e outside (0, 1]
    b.close()


def test_batch_db8_solver_matches_single_plans(wp):
    # Eq. 7 with the Daubechies-8 basis in the batched solver: problems of
    # different sides, levels 3 (every side divisible by 8), against single plans
    ns, ms = [32, 64, 16, 64, 128], [400, 1500, 100, 900, 3000]
    uvws, _ = make_case(ns, ms, seed=17)
    rng = np.random.default_rng(18)
    skies = [synth.blob_sky(rng, n, 5) for n in ns]
    b = build_batch(wp, ns, uvws, 0.99)
    x_cat = torch.from_numpy(np.concatenate([x.ravel() for x in skies]).astype(np.float32)).to(dev())
    sig = [synth.noise_sigma(x, 30.0) for x in skies]
    noise = np.concatenate([synth.complex_noise(rng, m, s) for m, s in zip(ms, sig)]).astype(np.complex64)
    y = b.phi(x_cat) + torch.from_numpy(noise).to(dev())
    eps = [O.epsilon_chi2(s, m) for s, m in zip(sig, ms)]
    xb = b.solve_bpdn(y, eps, iters=12, power_iters=50, psi=8, psi_levels=3)
    xd = b.solve_bpdn(y, eps, iters=12, power_iters=50)            # the Dirac graph is recaptured
    assert not torch.equal(xb, xd)
    x0 = b.solve_bpdn(y, eps, iters=0, psi=8, psi_levels=3)        # Psi z0 = Re Phi^H y
    assert rel(x0.cpu().numpy(), b.phi_adj(y).cpu().numpy()) <= 2e-6
    ys = b.split_vis(y)
    for i, (n, uvw) in enumerate(zip(ns, uvws)):
        p = wp.Plan(n, L, box="rule", index_format="columns")
        p.build_kernels(torch.from_numpy(uvw).to(dev()), 0.99)
        x1, _ = p.solve_bpdn(ys[i].contiguous(), eps[i], iters=12, power_iters=50, psi=8, psi_levels=3)
        xbi = b.split_images(xb)[i].cpu().numpy()
        s_b = O.snr_db(skies[i], xbi.astype(np.float64))
        s_1 = O.snr_db(skies[i], x1.cpu().numpy().astype(np.float64))
        assert abs(s_b - s_1) <= 0.1, (i, s_b, s_1)
        assert rel(xbi, x1.cpu().numpy()) <= 1e-3
        p.close()
    with pytest.raises(wp.WprojError):
        b.solve_bpdn(y, eps, iters=1, psi=8, psi_levels=5)            # 16 is not divisible by 32
    b.close()
