"""The largest image side a plan takes (N = 2048, G = 4096, 128 x 128 grid
tiles) with the box rule S(w): sampled rows of G and sampled visibilities of
Phi x against the FP64 oracle, and the adjoint identity of the whole operator."""
import math

import numpy as np
import pytest
import torch

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

pytestmark = pytest.mark.gpu

L = synth.fov_L()


def test_largest_side_sampled_against_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import wproj
    dev = torch.device("cuda", torch.cuda.current_device())
    N, M, e = 2048, 4096, 0.99
    rng = np.random.default_rng(2048)
    B = synth.band_limit(N, L)
    uv = synth.uv_points(rng, M, B, N, "uniform")
    w = 2.0 * rng.uniform(0.0, 4.0, M) / (L * L)          # w_c ~ U[0, 4] cells
    uvw = np.ascontiguousarray(np.concatenate([uv, w[:, None]], axis=1))
    geo = O.Geometry(N, L)
    for fmt in ("columns", "mask"):
        plan = wproj.Plan(N, L, box="rule", index_format=fmt)
        plan.build_kernels(torch.from_numpy(uvw).to(dev), e)
        c = plan.csr()
        G = geo.G
        rows = np.sort(rng.choice(M, 8, replace=False))
        for k in rows:
            col, val = (t.cpu().numpy() for t in c.rows(int(k), int(k) + 1))
            val = val.astype(np.complex128)
            S = O.row_box(geo, uvw[k, 2], "rule")
            K, j0u, j0v = O.kernel_box(geo, *uvw[k], S)
            su = ((col // G - j0u + G // 2) % G) - G // 2
            sv = ((col % G - j0v + G // 2) % G) - G // 2
            assert np.all(np.abs(su) <= S // 2) and np.all(np.abs(sv) <= S // 2)
            vo = K[su % S, sv % S]
            assert np.linalg.norm(val - vo) <= 1e-5 * np.linalg.norm(vo)
            assert math.fsum(np.abs(vo) ** 2) >= e * math.fsum(np.abs(K.ravel()) ** 2)
            assert col.size <= O.select_sort(K, O.box_columns(geo, j0u, j0v, S), e + 2e-5).size
        # Phi x on the sampled visibilities: the oracle's rows times its F Z A x
        x = rng.standard_normal((N, N))
        y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev)).cpu().numpy()
        Gs = O.build_G(geo, uvw[rows], e, S="rule")
        ys = Gs @ O.F(geo, O.AZ(geo, x)).ravel()
        # the GPU keeps e + 1e-5 of each row's energy: its rows differ from the
        # oracle's e-rows in their tails by up to ~sqrt(1e-5) of the row norm
        assert np.linalg.norm(y[rows] - ys) <= 5e-3 * np.linalg.norm(ys)
        xg = torch.from_numpy(x.astype(np.float32)).to(dev)
        yv = torch.from_numpy((rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)).to(dev)
        lhs = torch.vdot(yv.to(torch.complex128), plan.phi(xg).to(torch.complex128)).real.item()
        rhs = float((xg.double() * plan.phi_adj(yv).double()).sum().item())
        assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
        plan.close()
