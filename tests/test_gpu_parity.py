"""Parity of the CUDA path (called through the C-ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic on the device):
  * G values on the GPU's support vs the oracle's unthresholded kernel: rel-L2 <= 1e-5
  * Phi x and Phi^H y at e = 1 (no selection freedom): rel-L2 <= 1e-5
  * retained energy of every GPU row >= e E_k, judged with the oracle's values in
    FP64, and |support| <= n_oracle(e + 2e-5) (the GPU keeps e + 1e-5 to cover FP32)
  * at e < 1 the two supports may differ in near-tie entries at the threshold, so
    Phi is compared with a tolerance set by the energy those entries can carry.
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
    wproj.lib()
    return wproj


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def gpu_rows(plan):
    c = plan.csr()
    rp = c.row_ptr.cpu().numpy()
    col = c.col.cpu().numpy()
    if c.value_dtype == "f32":
        val = c.val.cpu().numpy().astype(np.complex128)
    else:
        v = c.val.float().cpu().numpy()
        val = (v[:, 0] + 1j * v[:, 1]).astype(np.complex128)
        rs = c.row_scale.cpu().numpy().astype(np.float64)
        val = val * np.repeat(rs, np.diff(rp))
    return rp, col, val


def oracle_values_at(geo, u, v, w, S, cols):
    K, j0u, j0v = O.kernel_box(geo, u, v, w, S)
    G = geo.G
    su = ((cols // G - j0u + G // 2) % G) - G // 2
    sv = ((cols % G - j0v + G // 2) % G) - G // 2
    inside = (su >= -S // 2) & (su < S // 2) & (sv >= -S // 2) & (sv < S // 2)
    return K[su % S, sv % S], inside, K, j0u, j0v


def check_build(plan, geo, uvw, e, box, tol=1e-5, rows=None):
    """box: None (S = G), "rule" (S(w) per row) or a fixed side."""
    rp, col, val = gpu_rows(plan)
    M = uvw.shape[0]
    rows = range(M) if rows is None else rows
    num = den = 0.0
    for k in rows:
        c = col[rp[k]:rp[k + 1]]
        vg = val[rp[k]:rp[k + 1]]
        assert np.unique(c).size == c.size, f"duplicate columns in row {k}"
        S = O.row_box(geo, uvw[k, 2], box)
        vo, inside, K, j0u, j0v = oracle_values_at(geo, *uvw[k], S, c)
        assert inside.all(), f"row {k}: entries outside the box"
        num += np.sum(np.abs(vg - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        # retained energy judged by the oracle, and the cardinality bound
        p_all = np.abs(K.ravel()) ** 2
        E = math.fsum(p_all)
        kept = math.fsum(np.abs(vo) ** 2)
        assert kept >= e * E, f"row {k}: kept {kept / E} < e = {e}"
        if e + 2e-5 < 1.0:
            # (at e + 1e-5 >= 1 the GPU keeps the whole box by definition)
            cols_box = O.box_columns(geo, j0u, j0v, S)
            n_hi = O.select_sort(K, cols_box, e + 2e-5).size
            assert c.size <= n_hi, f"row {k}: {c.size} > n_oracle(e + 2 delta) = {n_hi}"
        else:
            assert c.size == S * S
    rel = math.sqrt(num / den)
    assert rel <= tol, rel
    return rel


# ---- FFT ---------------------------------------------------------------------------


@pytest.mark.parametrize("n,batch", [(16, 3), (32, 2), (128, 2), (512, 1), (2048, 1), (4096, 1)])
@pytest.mark.parametrize("inverse", [0, 1])
def test_fft2d_matches_library_fft(wp, n, batch, inverse):
    rng = np.random.default_rng(n)
    a = (rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n)))
    ref = np.fft.ifft2(a) * n * n if inverse else np.fft.fft2(a)
    x = torch.from_numpy(a.astype(np.complex64)).to(dev())
    y = wp.fft2d(x, inverse=bool(inverse)).cpu().numpy()
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel < 2e-6, rel


# ---- build -------------------------------------------------------------------------


@pytest.mark.parametrize("N,M,e,box,ext,kind", [
    (16, 40, 1.0, None, "full", "exact"),
    (16, 40, 0.99, None, "full", "exact"),
    (32, 50, 0.9, None, "full", "exact"),
    (32, 50, 0.99, 32, "full", "exact"),
    (32, 37, 0.99, None, "clamp", "exact"),
    (16, 30, 0.999, None, "full", "linear"),
    (64, 25, 0.99, None, "full", "exact"),
    (64, 60, 0.99, "rule", "full", "exact"),
    (128, 40, 0.9, "rule", "clamp", "exact"),
])
def test_build_matches_oracle(wp, N, M, e, box, ext, kind):
    rng = np.random.default_rng(N + M)
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    plan = wp.Plan(N, L, box=box or "G", extension=ext, chirp=kind)
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), e)
    geo = O.Geometry(N, L, extension=ext, chirp_kind=kind)
    check_build(plan, geo, uvw, e, box)


def test_build_edge_cases(wp):
    # single visibility; visibilities on the band edges (wrap of the taps and
    # boxes around the grid), exactly on a cell (delta = 0), and w = 0
    N = 16
    geo = O.Geometry(N, L)
    B = N / (2 * L)
    du = geo.du
    uvw = np.array([[-B, -B, 0.0],
                    [B * (1 - 1e-12), -B + 0.5 * du, 3e4],
                    [3 * du, -5 * du, 1e4],
                    [0.0, 0.0, 0.0],
                    [-0.25 * du, 7.75 * du, 2e4]])
    for M in (1, uvw.shape[0]):
        plan = wp.Plan(N, L)
        plan.build_kernels(torch.from_numpy(np.ascontiguousarray(uvw[:M])).to(dev()), 0.99)
        check_build(plan, geo, uvw[:M], 0.99, None)
    plan = wp.Plan(N, L, box=16)
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), 0.9)
    check_build(plan, geo, uvw, 0.9, 16)


def test_build_rejects_bad_input(wp):
    N = 16
    plan = wp.Plan(N, L)
    B = N / (2 * L)
    bad = [np.array([[np.nan, 0.0, 0.0]]), np.array([[B, 0.0, 0.0]]), np.array([[0.0, -B * 1.01, 0.0]])]
    for uvw in bad:
        with pytest.raises(wp.WprojError) as ei:
            plan.build_kernels(torch.from_numpy(uvw).to(dev()), 0.99)
        assert ei.value.status == wp.ERR_INVALID_ARG
    good = torch.zeros((2, 3), dtype=torch.float64, device=dev())
    for e in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(wp.WprojError) as ei:
            plan.build_kernels(good, e)
        assert ei.value.status == wp.ERR_INVALID_ARG
    with pytest.raises(wp.WprojError) as ei:
        plan.phi(torch.zeros((N, N), device=dev()))
    assert ei.value.status == wp.ERR_NOT_BUILT
    # run lengths need boxes of at most 64 x 64 cells (here S = G = 128)
    big = wp.Plan(64, L, index_format="runs")
    with pytest.raises(wp.WprojError) as ei:
        big.build_kernels(torch.zeros((2, 3), dtype=torch.float64, device=dev()), 0.99)
    assert ei.value.status == wp.ERR_UNSUPPORTED


# ---- operators ------------------------------------------------------------------------


# N = 8 (a 16 x 16 grid, one 16 x 16 tile) takes the chunked shared-memory
# gridding; the others the cell-major or tile-stream gridding
@pytest.mark.parametrize("N,M,box,vdt", [(8, 20, None, "f32"), (16, 60, None, "f32"), (32, 200, None, "f32"),
                                         (64, 300, 32, "f32"), (128, 150, None, "f32"), (64, 200, "rule", "f32")])
def test_phi_and_adjoint_match_oracle_at_e1(wp, N, M, box, vdt):
    rng = np.random.default_rng(N)
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    x = rng.standard_normal((N, N))
    yv = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    plan = wp.Plan(N, L, box=box or "G", value_dtype=vdt)
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), 1.0)
    geo = O.Geometry(N, L)
    Gm = O.build_G(geo, uvw, 1.0, S=box)
    y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
    y_ref = O.phi(geo, Gm, x)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) <= 1e-5
    xa = plan.phi_adj(torch.from_numpy(yv.astype(np.complex64)).to(dev()), complex_out=True).cpu().numpy()
    xa_ref = O.phi_adj(geo, Gm, yv)
    assert np.linalg.norm(xa - xa_ref) / np.linalg.norm(xa_ref) <= 1e-5
    xr = plan.phi_adj(torch.from_numpy(yv.astype(np.complex64)).to(dev())).cpu().numpy()
    assert np.linalg.norm(xr - xa_ref.real) / np.linalg.norm(xa_ref.real) <= 1e-5
    if plan.csr().index_format == "mask":
        # the tile-stream gridding split every tile's records over several chunks
        # (>= 4096 entries each) whose partial tiles were summed: that path is the
        # one compared element by element above
        G = 2 * N
        n_tiles = (G // min(32, G)) ** 2
        assert plan.stats()["grid_chunks"] >= 2 * n_tiles


def test_adjoint_identity_on_gpu(wp):
    N, M = 32, 300
    rng = np.random.default_rng(5)
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    plan = wp.Plan(N, L)
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), 0.95)
    x = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    yv = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
    px = plan.phi_cplx(torch.from_numpy(x).to(dev())).cpu().numpy().astype(np.complex128)
    ay = plan.phi_adj(torch.from_numpy(yv).to(dev()), complex_out=True).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(yv.astype(np.complex128), px)
    rhs = np.vdot(ay, x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(px) * np.linalg.norm(yv)


def test_phi_at_e_below_1_within_selection_tolerance(wp):
    N, M, e = 32, 200, 0.99
    rng = np.random.default_rng(9)
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    x = rng.standard_normal((N, N))
    plan = wp.Plan(N, L)
    plan.build_kernels(torch.from_numpy(uvw).to(dev()), e)
    geo = O.Geometry(N, L)
    y = plan.phi(torch.from_numpy(x.astype(np.float32)).to(dev())).cpu().numpy()
    y_e = O.phi(geo, O.build_G(geo, uvw, e), x)
    y_hi = O.phi(geo, O.build_G(geo, uvw, min(1.0, e + 2e-5)), x)
    # the GPU operator lies between the oracle's e and e + 2 delta operators up to
    # FP32 error: its distance to either is bounded by their mutual distance
    gap = np.linalg.norm(y_hi - y_e)
    assert np.linalg.norm(y - y_e) <= 1.5 * gap + 1e-5 * np.linalg.norm(y_e)


def test_bf16_and_f16_values(wp):
    N, M, e = 32, 120, 0.99
    rng = np.random.default_rng(17)
    uvw = synth.random_uvw(rng, M, N, L, 1.0)
    geo = O.Geometry(N, L)
    for vdt, tol in (("bf16", 8e-3), ("f16", 1e-3)):
        plan = wp.Plan(N, L, value_dtype=vdt)
        plan.build_kernels(torch.from_numpy(uvw).to(dev()), e)
        check_build(plan, geo, uvw, e, None, tol=tol)


@pytest.mark.parametrize("N,M,e,box,vdt,wd", [(32, 200, 1.0, None, "f32", 1.0), (64, 150, 0.99, None, "f32", 1.0),
                                              (64, 120, 0.99, None, "bf16", 1.0), (128, 60, 0.9, "rule", "f32", 1.0),
                                              (64, 300, 0.99, 32, "f32", 0.05), (64, 250, 1.0, 64, "f32", 1.0),
                                              (64, 200, 0.95, 64, "bf16", 0.1), (32, 150, 0.9, None, "f16", 0.3),
                                              (128, 400, 0.99, 32, "bf16", 0.02)])
def test_index_formats_build_and_operators(wp, N, M, e, box, vdt, wd):
    # the column storages hold the same G (each checked against the oracle) and
    # give the same operators; at e = 1 all match the oracle's operators.  Run
    # lengths apply when every box is at most 64 x 64 cells and no row or
    # segment holds more than 64 runs (w small enough for the box).
    rng = np.random.default_rng(N + M + 1)
    uvw = synth.random_uvw(rng, M, N, L, wd)
    geo = O.Geometry(N, L)
    x = rng.standard_normal((N, N))
    yv = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    xg = torch.from_numpy(x.astype(np.float32)).to(dev())
    yg = torch.from_numpy(yv.astype(np.complex64)).to(dev())
    out, exported = {}, {}
    S = 2 * N if box is None else (box if box != "rule" else 2 * N)
    fmts = ("columns", "mask", "runs") if S <= 64 else ("columns", "mask")
    for fmt in fmts:
        plan = wp.Plan(N, L, box=box or "G", value_dtype=vdt, index_format=fmt)
        plan.build_kernels(torch.from_numpy(uvw).to(dev()), e)
        c = plan.csr()
        assert c.index_format == fmt
        check_build(plan, geo, uvw, e, box, tol=1e-5 if vdt == "f32" else 8e-3)
        out[fmt] = (plan.phi(xg).cpu().numpy(), plan.phi_adj(yg, complex_out=True).cpu().numpy())
        # row-range export agrees with the whole-matrix view, ragged ranges included
        col, val = c.col.cpu(), torch.view_as_real(c.val).cpu() if vdt == "f32" else c.val.cpu()
        rp = c.row_ptr.cpu().numpy()
        for k0, k1 in ((0, 1), (3, 17), (M - 5, M), (7, 7)):
            ck, vk = c.rows(k0, k1)
            vk = torch.view_as_real(vk) if vdt == "f32" else vk
            assert torch.equal(ck.cpu(), col[rp[k0]:rp[k1]])
            assert torch.equal(vk.cpu(), val[rp[k0]:rp[k1]])
        exported[fmt] = (col, val)
        plan.close()
    # the same G: identical columns and stored values in CSR order
    for fmt in fmts[1:]:
        assert torch.equal(exported["columns"][0], exported[fmt][0])
        assert torch.equal(exported["columns"][1], exported[fmt][1])
        for a, b in zip(out["columns"], out[fmt]):
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    if e == 1.0 and vdt == "f32":
        Gm = O.build_G(geo, uvw, 1.0, S=box)
        y_ref, xa_ref = O.phi(geo, Gm, x), O.phi_adj(geo, Gm, yv)
        for y, xa in out.values():
            assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) <= 1e-5
            assert np.linalg.norm(xa - xa_ref) / np.linalg.norm(xa_ref) <= 1e-5
