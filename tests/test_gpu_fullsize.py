"""Parity at the paper-scale workload (N = 256, G = 512, M = 32768, radially
Gaussian uv, w_d ~ U[0, 1], complex64 G) for e in {0.9, 0.99, 0.999}, built in
the launch configuration the benchmark times (tile stream, 262,144-entry
gridding chunks, so every grid tile's records span dozens of chunks whose
partial tiles the reduction sums).

The oracle cannot hold the whole G (up to 5.5e9 entries), so it computes
sampled rows one by one (Section 3.2: the chirp's FFT convolved with the taps,
then the energy threshold) and the tests compare element by element:
  * G's values on the sampled rows (rel-L2 <= 1e-5), retained energy >= e E_k
    judged by the oracle in FP64, cardinality <= n_oracle(e + 2e-5);
  * the support: the GPU keeps the smallest set reaching (e + 1e-5) E_k by its
    FP32 values, which must be the oracle's own (e + 1e-5) set up to entries
    tied with the cut within FP32 rounding;
  * Phi x on the sampled visibilities and Phi^H y for y supported on the sampled
    rows (and on a contiguous range of rows), both against the oracle's values
    on the GPU's support at rel-L2 <= 1e-5, and against the oracle's own
    (e + 1e-5) operator within the energy the near-tie entries carry.
"""
import math

import numpy as np
import pytest
import torch

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

pytestmark = pytest.mark.gpu

N_SAMPLE = 10
N_RANGE = 24          # contiguous rows of the Phi^H range case
E_VALUES = [0.9, 0.99, 0.999]
MARGIN = 1e-5         # the GPU's selection margin (kept energy >= (e + 1e-5) E_k)
AMP_TIE = 1e-6        # near-tie: |K| within 1e-6 sqrt(E_k) of the cut's modulus


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.PAPER_SCALE
    prob = synth.make_problem(wl, seed=0)
    geo = O.Geometry(wl.N, prob.L)
    rng = np.random.default_rng(123)
    rows = np.sort(rng.choice(wl.M, N_SAMPLE, replace=False))
    k0 = int(rng.integers(0, wl.M - N_RANGE))
    boxes = {}   # unthresholded oracle kernels (independent of e), computed once per row

    def box(k):
        if k not in boxes:
            K, j0u, j0v = O.kernel_box(geo, *prob.uvw[k], geo.G)
            boxes[k] = (K, O.box_columns(geo, j0u, j0v, geo.G))
        return boxes[k]

    X = O.F(geo, O.AZ(geo, prob.x)).ravel()
    return dict(wl=wl, prob=prob, geo=geo, rows=rows, range=np.arange(k0, k0 + N_RANGE), box=box, X=X,
                dev=torch.device("cuda", torch.cuda.current_device()))


@pytest.fixture(scope="module", params=E_VALUES, ids=[f"e{e}" for e in E_VALUES])
def built(request, problem):
    from paper_1307_3424_gb300 import wproj
    e = request.param
    plan = wproj.Plan(problem["wl"].N, problem["prob"].L)
    plan.build_kernels(torch.from_numpy(problem["prob"].uvw).to(problem["dev"]), e)
    yield dict(problem, plan=plan, e=e, wproj=wproj)
    plan.close()


def gpu_row(plan, k):
    col_k, val_k = plan.csr().rows(k, k + 1)
    return col_k.cpu().numpy().astype(np.int64), val_k.cpu().numpy().astype(np.complex128)


def oracle_on(box, col):
    """Oracle values at the given absolute columns (all must be in the box)."""
    K, cols = box
    pos = {c: i for i, c in enumerate(cols.ravel())}
    idx = np.array([pos[c] for c in col], dtype=np.int64)
    return K.ravel()[idx]


def oracle_sparse_rows(built, ks, e_sel):
    """(columns, values) of the oracle's own rows at energy fraction e_sel."""
    out = []
    for k in ks:
        K, cols = built["box"](k)
        kept = O.select_sort(K, cols, min(1.0, e_sel))
        out.append((cols.ravel()[kept], K.ravel()[kept]))
    return out


def test_sampled_rows_match_oracle(built):
    plan, e = built["plan"], built["e"]
    num = den = 0.0
    for k in built["rows"]:
        col, vg = gpu_row(plan, k)
        assert np.unique(col).size == col.size
        K, cols = built["box"](k)
        vo = oracle_on((K, cols), col)
        num += np.sum(np.abs(vg - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        E = math.fsum(np.abs(K.ravel()) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= e * E
        n_hi = O.select_sort(K, cols, min(1.0, e + 2 * MARGIN)).size
        assert col.size <= n_hi
    assert math.sqrt(num / den) <= 1e-5


def test_sampled_supports_are_the_oracles_up_to_near_ties(built):
    """The GPU's support of each sampled row is the oracle's (e + 1e-5) support,
    except for entries whose modulus equals the cut's within FP32 rounding."""
    plan, e = built["plan"], built["e"]
    identical = 0
    for k in built["rows"]:
        col, _ = gpu_row(plan, k)
        K, cols = built["box"](k)
        E = math.fsum(np.abs(K.ravel()) ** 2)
        own = set(cols.ravel()[O.select_sort(K, cols, min(1.0, e + MARGIN))].tolist())
        mine = set(col.tolist())
        if own == mine:
            identical += 1
            continue
        amp = dict(zip(cols.ravel().tolist(), np.abs(K.ravel()).tolist()))
        # the cut's modulus: the smallest modulus either support keeps
        cut = min(min(amp[c] for c in own), min(amp[c] for c in mine))
        diff = own ^ mine
        worst = max(abs(amp[c] - cut) for c in diff)
        assert worst <= AMP_TIE * math.sqrt(E), (k, len(diff), worst / math.sqrt(E))
    print(f"e={e}: {identical}/{len(built['rows'])} sampled supports identical to the oracle's")


def test_sampled_visibilities_match_oracle(built):
    plan, dev, e, X = built["plan"], built["dev"], built["e"], built["X"]
    y = plan.phi(torch.from_numpy(built["prob"].x.astype(np.float32)).to(dev)).cpu().numpy()
    rows = built["rows"]
    # (1) the oracle's values on the GPU's support: FP32 rounding only
    y_on = []
    for k in rows:
        col, _ = gpu_row(plan, k)
        y_on.append(np.sum(oracle_on(built["box"](k), col) * X[col]))
    y_on = np.array(y_on)
    assert np.linalg.norm(y[rows] - y_on) <= 1e-5 * np.linalg.norm(y_on)
    # (2) the oracle's own (e + 1e-5) operator, up to the near-tie entries
    own = np.array([np.sum(v * X[c]) for c, v in oracle_sparse_rows(built, rows, e + MARGIN)])
    lo = np.array([np.sum(v * X[c]) for c, v in oracle_sparse_rows(built, rows, e)])
    hi = np.array([np.sum(v * X[c]) for c, v in oracle_sparse_rows(built, rows, e + 2 * MARGIN)])
    gap = np.linalg.norm(hi - lo)
    assert np.linalg.norm(y[rows] - own) <= gap + 1e-5 * np.linalg.norm(own)


def _adjoint_case(built, ks, seed):
    """GPU Phi^H y for y supported on rows ks, and the oracle's
    A^H Z^H F^H (sum_k conj(G_k) y_k) with the oracle's values on the GPU's support."""
    plan, dev, geo, M = built["plan"], built["dev"], built["geo"], built["wl"].M
    rng = np.random.default_rng(seed)
    ys = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    yfull = np.zeros(M, np.complex64)
    yfull[ks] = ys
    xa = plan.phi_adj(torch.from_numpy(yfull).to(dev), complex_out=True).cpu().numpy().astype(np.complex128)
    G = geo.G
    grid_on = np.zeros(G * G, np.complex128)
    grid_own = np.zeros(G * G, np.complex128)
    for yk, k, (c_own, v_own) in zip(ys.astype(np.complex64).astype(np.complex128), ks,
                                     oracle_sparse_rows(built, ks, built["e"] + MARGIN)):
        col, _ = gpu_row(plan, k)
        np.add.at(grid_on, col, np.conj(oracle_on(built["box"](k), col)) * yk)
        np.add.at(grid_own, c_own, np.conj(v_own) * yk)
    ref_on = O.AZ_adj(geo, O.F_adj(geo, grid_on.reshape(G, G)))
    ref_own = O.AZ_adj(geo, O.F_adj(geo, grid_own.reshape(G, G)))
    return xa, ref_on, ref_own


def test_phi_adj_of_sampled_rows_matches_oracle(built):
    xa, ref_on, ref_own = _adjoint_case(built, built["rows"], 5)
    rel = np.linalg.norm(xa - ref_on) / np.linalg.norm(ref_on)
    print(f"e={built['e']}: Phi^H of sampled rows, rel-L2 {rel:.2e} (oracle values on the GPU support), "
          f"{np.linalg.norm(xa - ref_own) / np.linalg.norm(ref_own):.2e} (oracle's own support)")
    assert rel <= 1e-5
    # the near-tie entries carry at most MARGIN of each row's energy
    assert np.linalg.norm(xa - ref_own) <= (math.sqrt(2 * MARGIN) + 1e-5) * np.linalg.norm(ref_own)


def test_phi_adj_of_a_row_range_matches_oracle(built):
    # N_RANGE consecutive rows: their records sit side by side in every tile and
    # in the same gridding chunks, so partial tiles carry several rows at once
    if built["e"] != 0.99:
        pytest.skip("one energy fraction is enough for the range case")
    xa, ref_on, _ = _adjoint_case(built, built["range"], 6)
    rel = np.linalg.norm(xa - ref_on) / np.linalg.norm(ref_on)
    assert rel <= 1e-5, rel


def test_gridding_spans_many_chunks_per_tile(built):
    st = built["plan"].stats()
    n_tiles = (built["geo"].G // 32) ** 2
    assert built["plan"].csr().index_format == "mask"
    assert st["grid_chunks"] >= 8 * n_tiles, (st["grid_chunks"], n_tiles)


def test_adjoint_identity_full_size(built):
    plan, dev, wl = built["plan"], built["dev"], built["wl"]
    rng = np.random.default_rng(7)
    x = (rng.standard_normal((wl.N, wl.N)) + 1j * rng.standard_normal((wl.N, wl.N))).astype(np.complex64)
    yv = (rng.standard_normal(wl.M) + 1j * rng.standard_normal(wl.M)).astype(np.complex64)
    px = plan.phi_cplx(torch.from_numpy(x).to(dev)).cpu().numpy().astype(np.complex128)
    ay = plan.phi_adj(torch.from_numpy(yv).to(dev), complex_out=True).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(yv.astype(np.complex128), px)
    rhs = np.vdot(ay, x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(px) * np.linalg.norm(yv)


def test_gridding_is_deterministic(built):
    plan, dev, wl = built["plan"], built["dev"], built["wl"]
    yv = torch.randn(wl.M, dtype=torch.complex64, device=dev)
    a = plan.phi_adj(yv).clone()
    b = plan.phi_adj(yv).clone()
    assert torch.equal(a, b)


def test_phi_noalloc_refuses_this_workload(built):
    # the tile-stream degridding keeps 4 partial sums per (row, tile) segment:
    # 8.4 million segments need far more than the no-allocation variant's fixed array
    import ctypes
    if built["e"] != 0.99:
        pytest.skip("one energy fraction is enough")
    plan, dev, wp = built["plan"], built["dev"], built["wproj"]
    lib = wp.lib()
    x = torch.zeros((built["wl"].N, built["wl"].N), dtype=torch.float32, device=dev)
    y = torch.empty(built["wl"].M, dtype=torch.complex64, device=dev)
    st = lib.wproj_phi_noalloc(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == wp.ERR_INVALID_ARG
    assert b"limit" in lib.wproj_last_error()
