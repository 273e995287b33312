"""The learned-kernel network on the GPU: forward and gradients against the FP64
oracle (with the same BF16-rounded weights the tensor cores use), training data
taken from the plain build, and training that reduces the loss."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as MO
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


def oracle_params_as_gpu(p32):
    """The parameters the GPU computes with: W2..W4 in BF16, the rest FP32."""
    parts = MO.unpack(p32.astype(np.float64))
    for k in ("W2", "W3", "W4"):
        parts[k] = MO.round_bf16(parts[k])
    return MO.pack(parts)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_and_gradients_match_oracle(wp):
    rng = np.random.default_rng(0)
    p = synth.mlp_init_params(0)
    p[MO.N_PARAMS - MO.N_OUT:] = (rng.standard_normal(MO.N_OUT) * 0.05).astype(np.float32)
    B = 256
    x0 = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
    tv = (rng.standard_normal((B, MO.N_VAL)) * 0.05).astype(np.float32)
    tm = (rng.uniform(size=(B, MO.N_MASK)) < 0.3).astype(np.float32)
    net = wp.MLP(torch.from_numpy(p))
    xg, tvg, tmg = (torch.from_numpy(a).to(dev()) for a in (x0, tv, tm))
    y = net.forward(xg).cpu().numpy().astype(np.float64)
    po = oracle_params_as_gpu(p)
    f = MO.forward(po, x0.astype(np.float64))
    assert rel(y, f["y"]) <= 2e-2
    mw = 0.2
    loss, g = net.gradients(xg, tvg, tmg, mask_weight=mw)
    lo, go = MO.gradients(po, x0.astype(np.float64), tv.astype(np.float64), tm.astype(np.float64), mw)
    assert abs(loss - lo) <= 1e-2 * abs(lo)
    g = g.cpu().numpy().astype(np.float64)
    o = 0
    for name, shp in MO.SHAPES:
        n = int(np.prod(shp))
        a, b = g[o:o + n], go[o:o + n]
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel(a, b) <= 5e-2 and cos >= 0.998, (name, rel(a, b), cos)
        o += n
    # the parameters round-trip
    assert torch.equal(net.params(), torch.from_numpy(p))
    net.close()


def make_dataset(wp, m, seed, N=256):
    offs, wc = synth.mlp_samples(m, seed)
    uvw = synth.mlp_uvw(offs, wc, N, L, seed + 1)
    plan = wp.Plan(N, L, box="rule", index_format="columns")
    ug = torch.from_numpy(uvw).to(dev())
    plan.build_kernels(ug, 0.99)
    x0, tv, tm = wp.MLP.targets(plan, ug)
    return plan, uvw, offs, wc, x0, tv, tm


def test_targets_hold_the_plain_kernels(wp):
    plan, uvw, offs, wc, x0, tv, tm = make_dataset(wp, 256, 5)
    c = plan.csr()
    beta = O.kb_beta()
    kb = lambda t: float(O.kb(t, 4, beta))
    x0, tv, tm = x0.cpu().numpy(), tv.cpu().numpy(), tm.cpu().numpy()
    G = plan.G
    du_cell = 1.0 / (2.0 * L)
    for k in range(0, 256, 17):
        col, val = c.rows(k, k + 1)
        col, val = col.cpu().numpy(), val.cpu().numpy().astype(np.complex128)
        e_row = float(np.sum(np.abs(val) ** 2))
        # window cells (j0 - 16 + a, j0 - 16 + b) mod G
        j0 = np.floor(uvw[k, :2] / du_cell).astype(int)
        a = (col // G - (j0[0] - 16)) % G
        b = (col % G - (j0[1] - 16)) % G
        inside = (a < 32) & (b < 32)
        e_in = float(np.sum(np.abs(val[inside]) ** 2))
        du, dv = offs[k]
        ekb = sum(kb(du - t) ** 2 for t in (-1, 0, 1, 2)) * sum(kb(dv - t) ** 2 for t in (-1, 0, 1, 2))
        assert abs(np.sum(tv[k].astype(np.float64) ** 2) * ekb - e_in) <= 1e-5 * e_in
        assert int(tm[k].sum()) == int(inside.sum())
        assert e_in >= 0.99 * e_row            # the window holds the kernel up to its far tails
        t = tv[k].reshape(32, 32, 2)
        assert np.allclose(t[a[inside], b[inside], 0] + 1j * t[a[inside], b[inside], 1],
                           val[inside] / math.sqrt(ekb), rtol=1e-5, atol=1e-7)
        assert np.allclose(x0[k], [wc[k] / 2 - 1, 2 * du - 1, 2 * dv - 1], atol=1e-6)
    plan.close()


def test_training_reduces_the_loss(wp):
    plan, uvw, offs, wc, x0, tv, tm = make_dataset(wp, 8192, 11)
    plan.close()
    net = wp.MLP(torch.from_numpy(synth.mlp_init_params(1)))
    y0 = net.forward(x0[:1024]).cpu().numpy()
    losses = net.train(x0, tv, tm, batch=1024, steps=300, lr=1e-3, mask_weight=0.1)
    assert all(math.isfinite(v) for v in losses)
    assert np.mean(losses[-10:]) < 0.2 * np.mean(losses[:3]), (losses[:3], losses[-10:])
    y1 = net.forward(x0[:1024]).cpu().numpy()
    t = tv[:1024].cpu().numpy()
    assert rel(y1[:, :2048], t) < 0.5 * rel(y0[:, :2048], t)
    net.close()


def test_learned_build_judges_every_row(wp):
    # a briefly trained network; rows take its kernel only when they pass
    plan, uvw, offs, wc, x0, tv, tm = make_dataset(wp, 8192, 21)
    plan.close()
    net = wp.MLP(torch.from_numpy(synth.mlp_init_params(2)))
    net.train(x0, tv, tm, batch=1024, steps=200, lr=1e-3, mask_weight=0.1)
    m, N = 1024, 256
    offs2, wc2 = synth.mlp_samples(m, 31)
    uvw2 = torch.from_numpy(synth.mlp_uvw(offs2, wc2, N, L, 32)).to(dev())
    ref = wp.Plan(N, L, box="rule", index_format="columns")
    ref.build_kernels(uvw2, 0.99)
    c_ref = ref.csr()
    # threshold 0: every row falls back, G is the plain one bit for bit
    p0 = wp.Plan(N, L, box="rule", index_format="columns")
    info0, err0 = p0.build_kernels_learned(net, uvw2, 0.99, rel_l2_max=0.0)
    assert info0["learned"] == 0 and info0["rows"] == m
    assert torch.equal(p0.csr().val, c_ref.val) and torch.equal(p0.csr().col, c_ref.col)
    # no error threshold: rows whose predicted support holds >= e take the prediction
    p1 = wp.Plan(N, L, box="rule", index_format="columns")
    info1, err1 = p1.build_kernels_learned(net, uvw2, 0.99, rel_l2_max=1e9)
    assert torch.equal(err0, err1) and 0 <= info1["learned"] <= m
    c1 = p1.csr()
    assert torch.equal(c1.col, c_ref.col)                      # the support is the plain one
    changed = (c1.val != c_ref.val).any().item()
    assert changed == (info1["learned"] > 0)
    # predicted values on a passing row's support, from the network's own forward
    xf, _, _ = wp.MLP.targets(ref, uvw2)
    y = net.forward(xf).cpu().numpy()
    rp = c_ref.row_ptr.cpu().numpy()
    beta = O.kb_beta()
    du_cell = 1.0 / (2.0 * L)
    checked = 0
    for k in range(m):
        col, v1 = c1.rows(k, k + 1)
        _, v0 = c_ref.rows(k, k + 1)
        if torch.equal(v1, v0):
            continue
        col, v1 = col.cpu().numpy(), v1.cpu().numpy()
        j0 = np.floor(uvw2[k, :2].cpu().numpy() / du_cell).astype(int)
        a = (col // (2 * N) - (j0[0] - 16)) % (2 * N)
        b = (col % (2 * N) - (j0[1] - 16)) % (2 * N)
        du, dv = offs2[k]
        ekb = (sum(float(O.kb(du - t, 4, beta)) ** 2 for t in (-1, 0, 1, 2)) *
               sum(float(O.kb(dv - t, 4, beta)) ** 2 for t in (-1, 0, 1, 2)))
        cidx = a * 32 + b
        pred = (y[k, 2 * cidx] + 1j * y[k, 2 * cidx + 1]) * math.sqrt(ekb)
        assert np.allclose(v1, pred, rtol=1e-5, atol=1e-6 * np.abs(pred).max())
        checked += 1
        if checked == 5:
            break
    # the operator of the learned G is still self-adjoint-consistent (cells rebuilt)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).to(dev())
    yv = torch.from_numpy((rng.standard_normal(m) + 1j * rng.standard_normal(m)).astype(np.complex64)).to(dev())
    lhs = torch.vdot(yv.to(torch.complex128), p1.phi(x).to(torch.complex128)).real.item()
    rhs = float((x.double() * p1.phi_adj(yv).double()).sum().item())
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    for p in (ref, p0, p1):
        p.close()
    net.close()
