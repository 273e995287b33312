"""Precision form at full size: N = 1024 (G = 2048), M = 2^21, 2000 blobs plus a
power-law diffuse part, w_c ~ U[0, 4] cells, box rule S(w) in {32, 64}, G values
stored in FP32, BF16 or FP16 with a per-row scale, FP32 accumulation.

Errors against the FP64 oracle are reported (and bounded) per result:
  * G values on sampled rows;
  * Phi on the sampled visibilities (the oracle computes those rows one by one);
  * Phi^H of visibilities supported on the sampled rows (full-size oracle FFT);
  * final image: SNR of a Douglas-Rachford solve; the oracle cannot hold this G,
    so the FP32 GPU form is the comparator for the 16-bit forms (within 0.1 dB).
"""
import math

import numpy as np
import pytest
import torch

from oracle import wproj_oracle as O
from paper_1307_3424_gb300 import synth

pytestmark = pytest.mark.gpu

N_SAMPLE = 12
TOL = {"f32": (1e-5, 5e-3), "bf16": (8e-3, 1.5e-2), "f16": (1e-3, 5e-3)}   # (G values, Phi / Phi^H)


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import wproj
    wl = synth.PRECISION
    prob = synth.make_problem(wl, seed=0)
    noise, sigma_n = synth.draw_noise(prob)
    geo = O.Geometry(wl.N, prob.L)
    rng = np.random.default_rng(99)
    rows = np.sort(rng.choice(wl.M, N_SAMPLE, replace=False))
    oracle_rows = {}
    for k in rows:
        S = O.row_box(geo, prob.uvw[k, 2], "rule")
        oracle_rows[k] = (S, O.kernel_row(geo, *prob.uvw[k], S, wl.e),
                          O.kernel_row(geo, *prob.uvw[k], S, wl.e + 2e-5), O.kernel_box(geo, *prob.uvw[k], S))
    X = O.F(geo, O.AZ(geo, prob.x)).ravel()
    return dict(wproj=wproj, wl=wl, prob=prob, geo=geo, rows=rows, orows=oracle_rows, X=X,
                noise=noise, sigma_n=sigma_n, dev=torch.device("cuda", torch.cuda.current_device()))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fmt", ["auto", "runs", "columns"])
@pytest.mark.parametrize("vdt", ["f32", "bf16", "f16"])
def test_precision_form_against_oracle(case, vdt, fmt):
    wp, wl, prob, geo, dev = case["wproj"], case["wl"], case["prob"], case["geo"], case["dev"]
    tol_val, tol_op = TOL[vdt]
    plan = wp.Plan(wl.N, prob.L, box="rule", value_dtype=vdt, index_format=fmt)
    plan.build_kernels(torch.from_numpy(prob.uvw).to(dev), wl.e)
    c = plan.csr()
    if fmt == "auto":   # boxes of 32 and 64 cells: run lengths for f32, columns for 16-bit values
        assert c.index_format == ("runs" if vdt == "f32" else "columns")
    else:
        assert c.index_format == fmt
    G = geo.G
    num = den = 0.0
    for k in case["rows"]:
        S, _, _, (K, j0u, j0v) = case["orows"][k]
        col_k, val_k = c.rows(k, k + 1)
        col = col_k.cpu().numpy()
        if vdt == "f32":
            vg = val_k.cpu().numpy().astype(np.complex128)
        else:
            v = val_k.float().cpu().numpy()
            vg = (v[:, 0] + 1j * v[:, 1]) * float(c.row_scale[k])
        su = ((col // G - j0u + G // 2) % G) - G // 2
        sv = ((col % G - j0v + G // 2) % G) - G // 2
        assert np.all(np.abs(su) <= S // 2) and np.all(np.abs(sv) <= S // 2)
        vo = K[su % S, sv % S]
        num += np.sum(np.abs(vg - vo) ** 2)
        den += np.sum(np.abs(vo) ** 2)
        E = math.fsum(np.abs(K.ravel()) ** 2)
        assert math.fsum(np.abs(vo) ** 2) >= wl.e * E
    err_val = math.sqrt(num / den)
    # Phi on the sampled visibilities
    y = plan.phi(torch.from_numpy(prob.x.astype(np.float32)).to(dev)).cpu().numpy()
    X = case["X"]
    ye = np.array([np.sum(case["orows"][k][1][1] * X[case["orows"][k][1][0]]) for k in case["rows"]])
    err_phi = _rel(y[case["rows"]], ye)
    # Phi^H of visibilities on the sampled rows only
    rng = np.random.default_rng(5)
    ys = rng.standard_normal(N_SAMPLE) + 1j * rng.standard_normal(N_SAMPLE)
    yfull = np.zeros(wl.M, np.complex64)
    yfull[case["rows"]] = ys
    xa = plan.phi_adj(torch.from_numpy(yfull).to(dev), complex_out=True).cpu().numpy()
    Gs = np.zeros(G * G, np.complex128)
    for yk, k in zip(ys, case["rows"]):
        cols, vals = case["orows"][k][1]
        np.add.at(Gs, cols, np.conj(vals) * yk)
    xa_ref = O.AZ_adj(geo, O.F_adj(geo, Gs.reshape(G, G)))
    err_adj = _rel(xa, xa_ref)
    print(f"{vdt}/{fmt}: nnz={c.nnz} format={c.index_format} err(G)={err_val:.2e} err(Phi)={err_phi:.2e} "
          f"err(Phi^H)={err_adj:.2e}")
    assert err_val <= tol_val
    assert err_phi <= tol_op
    assert err_adj <= tol_op
    plan.close()


def test_precision_form_reconstruction_snr(case):
    wp, wl, prob, dev = case["wproj"], case["wl"], case["prob"], case["dev"]
    iters = 30
    snr = {}
    y = None
    for vdt in ("f32", "bf16", "f16"):
        plan = wp.Plan(wl.N, prob.L, box="rule", value_dtype=vdt)
        plan.build_kernels(torch.from_numpy(prob.uvw).to(dev), wl.e)
        if y is None:   # the data: FP32 operator plus noise
            y = plan.phi(torch.from_numpy(prob.x.astype(np.float32)).to(dev)) + \
                torch.from_numpy(case["noise"].astype(np.complex64)).to(dev)
            eps = O.epsilon_chi2(case["sigma_n"], wl.M)
        x, info = plan.solve_bpdn(y, eps, iters=iters, power_iters=50)
        snr[vdt] = O.snr_db(prob.x, x.cpu().numpy().astype(np.float64))
        plan.close()
    print("SNR_out after", iters, "DR iterations:", {k: round(v, 3) for k, v in snr.items()})
    assert abs(snr["bf16"] - snr["f32"]) <= 0.1
    assert abs(snr["f16"] - snr["f32"]) <= 0.1
