"""Paper mode on the GPU (upsampling=1): the paper's operator C-hat F U with
visibilities on the grid and the linear chirp, against the FP64 oracle."""
import math

import numpy as np
import pytest
import scipy.sparse
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


def paper_plan(wp, N, fmt="auto", vdt="f32"):
    return wp.Plan(N, L, kb_support=1, chirp="linear", box="G", upsampling=True, index_format=fmt, value_dtype=vdt)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,cov", [(16, 0.2), (32, 0.1)])
def test_operators_match_the_definition_at_E1(wp, N, cov):
    prob = synth.paper_problem(N, cov, seed=N)
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N))
    M = prob.uvw.shape[0]
    yv = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    for fmt in ("columns", "mask", "runs"):     # G = 2N <= 64: run lengths apply
        plan = paper_plan(wp, N, fmt)
        plan.build_kernels(torch.from_numpy(prob.uvw).to(dev()), 1.0)
        y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
        assert rel(y, O.paper_visibilities_direct(N, L, x, prob.uvw)) <= 1e-5
        Gm = O.build_G(O.paper_geometry(N, L), prob.uvw, 1.0)
        xa = plan.phi_adj(torch.from_numpy(yv.astype(np.complex64)).to(dev()), complex_out=True).cpu().numpy()
        assert rel(xa, O.paper_phi_adj(N, Gm, yv)) <= 1e-5
        plan.close()


def test_build_at_E075_matches_oracle(wp):
    # the paper's working point E = 0.75 (Section 3.2)
    N, E = 32, 0.75
    prob = synth.paper_problem(N, 0.2, seed=3)
    geo = O.paper_geometry(N, L)
    plan = paper_plan(wp, N, "columns")
    plan.build_kernels(torch.from_numpy(prob.uvw).to(dev()), E)
    c = plan.csr()
    G = 2 * N
    num = den = 0.0
    for k in range(0, prob.uvw.shape[0], 7):
        col, val = c.rows(k, k + 1)
        col, val = col.cpu().numpy(), val.cpu().numpy().astype(np.complex128)
        K, j0u, j0v = O.kernel_box(geo, *prob.uvw[k], G)
        su = ((col // G - j0u + G // 2) % G) - G // 2
        sv = ((col % G - j0v + G // 2) % G) - G // 2
        vo = K[su % G, sv % G]
        num += np.sum(np.abs(val - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= E                     # unit row energy
        n_hi = O.select_sort(K, O.box_columns(geo, j0u, j0v, G), E + 2e-5).size
        assert col.size <= n_hi
    assert math.sqrt(num / den) <= 1e-5
    plan.close()


def test_nonzero_proportion_matches_oracle(wp):
    N = 64
    prob = synth.paper_problem(N, 0.05, seed=0)
    rows = prob.uvw[:256]
    geo = O.paper_geometry(N, L)
    plan = paper_plan(wp, N, "columns")
    for E in (0.1, 0.75, 0.9, 0.999):
        plan.build_kernels(torch.from_numpy(rows).to(dev()), E)
        gpu = plan.csr().nnz
        ora = sum(O.kernel_row(geo, *r, 2 * N, E)[0].size for r in rows[:64])
        ora_hi = sum(O.kernel_row(geo, *r, 2 * N, E + 2e-5)[0].size for r in rows[:64])
        gpu64 = int(plan.csr().row_ptr[64].item())
        assert ora <= gpu64 <= ora_hi + 64, (E, gpu64, ora, ora_hi)
        frac = gpu / (rows.shape[0] * (2 * N) ** 2)
        print(f"E={E}: proportion of non-zero entries {frac:.4f}")
    plan.close()


def test_paper_mode_rejects_bad_geometry(wp):
    with pytest.raises(wp.WprojError):
        wp.Plan(16, L, kb_support=4, upsampling=True)      # paper mode grids on cells: one tap
    with pytest.raises(wp.WprojError):
        wp.Plan(8, L, kb_support=1, upsampling=True)


def oracle_G_tie_choice(geo, uvw, e, rng):
    """The oracle's E-threshold rows (Section 3.2) with the members of each group
    of equal magnitudes (to 1e-9 of the row's peak) taken in a random order
    instead of by column: another valid support of the same rule."""
    G = geo.G
    cols_, vals, ptr = [], [], [0]
    for k in range(uvw.shape[0]):
        K, j0u, j0v = O.kernel_box(geo, *uvw[k], G)
        cols = O.box_columns(geo, j0u, j0v, G).ravel()
        Kf = K.ravel()
        p = np.abs(Kf) ** 2
        order = np.lexsort((rng.permutation(p.size), -np.round(p / p.max(), 9)))
        ps = p[order]
        target = e * math.fsum(p)
        n = int(np.searchsorted(np.cumsum(ps), target)) + 1
        while n < ps.size and math.fsum(ps[:n]) < target:
            n += 1
        while n > 1 and math.fsum(ps[:n - 1]) >= target:
            n -= 1
        c = cols[order[:n]]
        o = np.argsort(c)
        cols_.append(c[o])
        vals.append(Kf[order[:n]][o])
        ptr.append(ptr[-1] + n)
    return scipy.sparse.csr_matrix((np.concatenate(vals), np.concatenate(cols_), np.array(ptr)),
                                   shape=(uvw.shape[0], G * G))


def test_reconstruction_in_paper_mode(wp):
    # Douglas-Rachford with the paper's operator at E = 0.75, data simulated with
    # the same operator as the reconstruction (Section 4).  The linear chirp's
    # mirror symmetries put the E-cut inside a group of equal magnitudes in most
    # rows, so several supports are valid and FP32 picks its own; the oracle's
    # SNR over a few valid tie choices bounds what the GPU may reach.
    N, E = 32, 0.75
    prob = synth.paper_problem(N, 0.3, seed=9, n_blobs=8)
    noise, sigma_n = synth.draw_noise(prob)
    geo = O.paper_geometry(N, L)
    eps = O.epsilon_chi2(sigma_n, prob.uvw.shape[0])
    snr_o = []
    for Gm in [O.build_G(geo, prob.uvw, E)] + [oracle_G_tie_choice(geo, prob.uvw, E, np.random.default_rng(s))
                                               for s in range(3)]:
        y = O.paper_phi(N, Gm, prob.x) + noise
        xo, _ = O.solve_bpdn(lambda v: O.paper_phi(N, Gm, v), lambda r: O.paper_phi_adj(N, Gm, r).real, y, eps,
                             N, iters=30)
        snr_o.append(O.snr_db(prob.x, xo))
    plan = paper_plan(wp, N, "columns")
    plan.build_kernels(torch.from_numpy(prob.uvw).to(dev()), E)
    xg = torch.from_numpy(prob.x.astype(np.float32)).to(dev())
    yg = plan.phi(xg) + torch.from_numpy(noise.astype(np.complex64)).to(dev())
    xr, info = plan.solve_bpdn(yg, eps, iters=30)
    s_g = O.snr_db(prob.x, xr.cpu().numpy().astype(np.float64))
    print(f"SNR GPU {s_g:.3f} dB, oracle over tie choices {min(snr_o):.3f} .. {max(snr_o):.3f} dB")
    assert min(snr_o) - 0.1 <= s_g <= max(snr_o) + 0.1, (s_g, snr_o)
    assert info.final_resid <= eps * 1.05
    plan.close()


def test_paper_mode_at_256_sampled(wp):
    # N = 256 (G = 512, 256 tiles), 20 % coverage, E = 0.75: sampled rows against
    # the oracle's support rule and values; Phi' against the literal definition
    # on sampled visibilities at E = 1
    N, E = 256, 0.75
    prob = synth.paper_problem(N, 0.2, seed=4)
    geo = O.paper_geometry(N, L)
    M = prob.uvw.shape[0]
    ug = torch.from_numpy(prob.uvw).to(dev())
    plan = paper_plan(wp, N)
    plan.build_kernels(ug, E)
    c = plan.csr()
    G = 2 * N
    num = den = 0.0
    for k in np.random.default_rng(8).choice(M, 10, replace=False):
        col, val = (t.cpu().numpy() for t in c.rows(int(k), int(k) + 1))
        val = val.astype(np.complex128)
        K, j0u, j0v = O.kernel_box(geo, *prob.uvw[k], G)
        su = ((col // G - j0u + G // 2) % G) - G // 2
        sv = ((col % G - j0v + G // 2) % G) - G // 2
        vo = K[su % G, sv % G]
        num += np.sum(np.abs(val - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= E
        assert col.size <= O.select_sort(K, O.box_columns(geo, j0u, j0v, G), E + 2e-5).size
    assert math.sqrt(num / den) <= 1e-5
    # E = 1 keeps whole G x G rows: build the sampled visibilities alone
    pick = np.random.default_rng(10).choice(M, 16, replace=False)
    plan.build_kernels(torch.from_numpy(np.ascontiguousarray(prob.uvw[pick])).to(dev()), 1.0)
    x = np.random.default_rng(9).standard_normal((N, N))
    y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
    yd = O.paper_visibilities_direct(N, L, x, prob.uvw[pick])
    assert rel(y, yd) <= 1e-5
    plan.close()
